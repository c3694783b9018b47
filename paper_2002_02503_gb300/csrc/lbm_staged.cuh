// lbm_staged.cuh -- step variant 1: persistent CTAs that stage the source rows of
// each tile into shared memory with bulk asynchronous copies (cp.async.bulk, the
// non-tensor TMA path) completing on mbarriers, in a ring of S stages.
//
// A tile is R consecutive x-rows (row index y + ny z) of nx cells.  For each tile
// and velocity i the source row (y - c_iy, z - c_iz) of plane i is copied whole
// (nx values, contiguous and 16-byte aligned), so the x shift and its periodic
// wrap become shared-memory indexing.  A producer warp issues the Q*R copies of a
// tile as soon as its stage is free; consumer warps wait on the stage's "full"
// mbarrier, compute their cells from shared memory, store coalesced rows to the
// other buffer and release the stage on its "empty" mbarrier.
//
// Every wait is bounded by a clock budget: on expiry the CTA records
// kStagedTimeout in the status word, drains (again bounded) the copies it has in
// flight, and returns.  The host reports it as LBM_ERR_TIMEOUT.
#pragma once

#include <cuda_runtime.h>
#include <stdlib.h>

#include <atomic>

#include "lbm_core.cuh"
#include "lbm_internal.h"

namespace lbm {

constexpr unsigned int kStagedTimeout = kStatusTimeout;
constexpr long long kWaitBudgetCycles = 2000000000LL;  // ~1 s at the maximum SM clock
constexpr int kStagedThreads = 32 + 512;  // one producer warp + sixteen consumer warps

__device__ __forceinline__ unsigned int smem_addr(const void *p) {
    return static_cast<unsigned int>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned int count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long *bar, unsigned int bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, unsigned int parity) {
    unsigned int ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait on a stage's phase; false when the clock budget ran out.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long *bar, unsigned int parity) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > kWaitBudgetCycles) return false;
    }
    return true;
}

__device__ __forceinline__ void bulk_copy_g2s(void *dst_smem, const void *src_gmem, unsigned int bytes,
                                              unsigned long long *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst_smem)),
        "l"(src_gmem), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// Stage layout in dynamic shared memory: S mbarriers, then S stages of Q*R rows of nx values.
template <class LT, class ST>
__device__ __forceinline__ void issue_tile(const typename ST::S *__restrict__ src, typename ST::S *stage,
                                           unsigned long long *bar, int tile, int R, int rows, int nx, int ny,
                                           int nz, long long P, unsigned int extra_tx) {
    using S = typename ST::S;
    const int r0 = tile * R;
    const int nr = min(R, rows - r0);
    const unsigned int row_bytes = unsigned(nx) * sizeof(S);
    mbar_arrive_expect_tx(bar, unsigned(LT::Q * nr) * row_bytes + extra_tx);
    for (int r = 0; r < nr; ++r) {
        const int row = r0 + r;
        const int y = row % ny, z = row / ny;
#pragma unroll
        for (int i = 0; i < LT::Q; ++i) {
            int ys = y - vel<LT>(i, 1), zs = z - vel<LT>(i, 2);
            ys = ys < 0 ? ys + ny : (ys >= ny ? ys - ny : ys);  // dims >= max|c| (host-checked)
            zs = zs < 0 ? zs + nz : (zs >= nz ? zs - nz : zs);
            bulk_copy_g2s(stage + (size_t(i) * R + r) * nx, src + i * P + (long long)(zs * ny + ys) * nx, row_bytes,
                          bar);
        }
    }
}

// Warp roles: warp 0 is the producer (its lanes issue the bulk copies), the other
// warps (up to kConsumerWarps) compute.  Stage s has a "full" barrier (the producer's
// arrive.expect_tx plus the copies' bytes) and an "empty" barrier (one arrival per
// consumer warp once it has read the stage).
constexpr int kConsumerWarps = 16;
constexpr int kConsumers = 32 * kConsumerWarps;
constexpr int kStagedMaxCpt = 4;  // cells per consumer thread per tile

// The producer warp's lanes share a tile's Q*R copies (lane 0 posts the expected bytes first).
template <class LT, class ST>
__device__ __forceinline__ void issue_tile_warp(const typename ST::S *__restrict__ src, typename ST::S *stage,
                                                unsigned long long *bar, int tile, int R, int rows, int nx, int ny,
                                                int nz, long long P, unsigned int extra_tx, int lane,
                                                unsigned int *status) {
    using S = typename ST::S;
    const int r0 = tile * R;
    const int nr = min(R, rows - r0);
    const unsigned int row_bytes = unsigned(nx) * sizeof(S);
    if (lane == 0) mbar_arrive_expect_tx(bar, unsigned(LT::Q * nr) * row_bytes + extra_tx);
    __syncwarp();
    for (int q = lane; q < LT::Q * nr; q += 32) {
        const int i = q % LT::Q, r = q / LT::Q;
        const int row = r0 + r;
        const int y = row % ny, z = row / ny;
        int ys = y - vel_rt<LT>(i, 1), zs = z - vel_rt<LT>(i, 2);
        ys = ys < 0 ? ys + ny : (ys >= ny ? ys - ny : ys);  // dims >= max|c| (host-checked)
        zs = zs < 0 ? zs + nz : (zs >= nz ? zs - nz : zs);
        long long roff = (long long)(zs * ny + ys) * nx;
        if constexpr (kBoundsCheck) {
            // a row outside the plane is recorded and replaced by the plane's first row, so the
            // stage still receives the bytes its barrier expects
            if (!span_in(roff, nx, P)) {
                if (status) atomicOr(status, kStatusBounds);
                roff = 0;
            }
        }
        bulk_copy_g2s(stage + (size_t(i) * R + r) * nx, src + i * P + roff, row_bytes, bar);
    }
}

template <class LT, int K, class ST>
__global__ void __launch_bounds__(kStagedThreads) step_staged_kernel(const typename ST::S *__restrict__ src,
                                                                     typename ST::S *__restrict__ dst, int nx, int ny,
                                                                     int nz, long long P, int R, int S_stages,
                                                                     typename ST::T relax, typename ST::T rho0,
                                                                     unsigned int *__restrict__ status,
                                                                     unsigned int extra_tx) {
    using S = typename ST::S;
    using T = typename ST::T;
    constexpr int Q = LT::Q, M = LT::MAXC;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned long long *full = reinterpret_cast<unsigned long long *>(smem_raw);
    unsigned long long *empty = full + 8;
    S *stages = reinterpret_cast<S *>(smem_raw + 128);
    const size_t stage_elems = size_t(Q) * R * nx;
    const int rows = ny * nz;
    const int tiles = (rows + R - 1) / R;
    const int cells = R * nx;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int my_tiles = blockIdx.x < tiles ? (tiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x : 0;

    if (threadIdx.x == 0) {
        for (int s = 0; s < S_stages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], (blockDim.x - 32) / 32);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    if (warp == 0) {
        // ---------------- producer warp
        int issued = 0;
        bool ok = true;
        for (int k = 0; k < my_tiles; ++k) {
            const int s = k % S_stages;
            // first round: parity 1 of a fresh barrier counts as complete
            const bool free_stage = mbar_wait_bounded(&empty[s], ((k / S_stages) & 1) ^ 1);
            if (__any_sync(0xffffffffu, !free_stage)) {
                ok = false;
                break;
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            issue_tile_warp<LT, ST>(src, stages + s * stage_elems, &full[s], blockIdx.x + k * gridDim.x, R, rows, nx,
                                    ny, nz, P, k == 0 ? extra_tx : 0u, lane, status);
            ++issued;
        }
        if (!ok && lane == 0) {
            if (status) atomicOr(status, kStagedTimeout);
            // copies must land before the CTA exits: wait (bounded) for every issued phase
            for (int k = 0; k < issued; ++k) mbar_wait_bounded(&full[k % S_stages], (k / S_stages) & 1);
        }
        // (normal path: the consumers wait on every issued phase before the CTA can exit)
        return;
    }

    // ---------------- consumers: fixed cell positions within a tile
    const int ct = threadIdx.x - 32;
    const int consumers = blockDim.x - 32;
    int cr[kStagedMaxCpt], cx[kStagedMaxCpt];
    int ncell = 0;
#pragma unroll
    for (int j = 0; j < kStagedMaxCpt; ++j) {
        const int c = ct + j * consumers;
        cr[j] = c / nx;
        cx[j] = c - cr[j] * nx;
        if (c < cells) ncell = j + 1;
    }
    for (int k = 0; k < my_tiles; ++k) {
        const int s = k % S_stages;
        const bool ok = mbar_wait_bounded(&full[s], (k / S_stages) & 1);
        if (__any_sync(0xffffffffu, !ok)) {  // a warp-wide decision: the warp leaves together
            if (lane == 0 && status) atomicOr(status, kStagedTimeout);
            return;  // the producer drains the copies it issued
        }
        const S *st = stages + s * stage_elems;
        const int r0 = (blockIdx.x + k * gridDim.x) * R;
#pragma unroll 1
        for (int j = 0; j < kStagedMaxCpt; ++j) {
            if (j >= ncell) break;
            const int row = r0 + cr[j];
            if (row >= rows) break;
            const int x = cx[j];
            int xs[2 * M + 1];
#pragma unroll
            for (int q = -M; q <= M; ++q) {
                const int v = x - q;
                xs[q + M] = v < 0 ? v + nx : (v >= nx ? v - nx : v);
            }
            const S *base = st + size_t(cr[j]) * nx;
            T g[Q];
#pragma unroll
            for (int i = 0; i < Q; ++i) g[i] = decode<ST>(base[size_t(i) * R * nx + xs[vel<LT>(i, 0) + M]], QScale{}, i);
            collide<LT, K, T>(g, relax, rho0);
            S *out = dst + (long long)row * nx + x;
            unsigned int acc = 0u;  // floating storage only: no range to leave
            if (!guard((long long)row * nx + x, 1, P, status)) continue;
#pragma unroll
            for (int i = 0; i < Q; ++i) out[(long long)i * P] = encode<ST>(g[i], QScale{}, i, acc);
        }
        __syncwarp();
        if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(&empty[s])) : "memory");
    }
}

// Rows per tile and stages for a lattice / storage / nx; 0 when the variant does not apply.
// Tile geometry: R rows of about kConsumers cells, a ring of S >= 2 stages that lets two
// CTAs share an SM when it can (else one CTA with a deeper ring), and one consumer thread
// per cell of a tile (rounded to warps).  R = 0 when the variant does not apply.
template <class LT, class ST>
inline void staged_geometry(int nx, int *R, int *S, size_t *smem, int *threads) {
    *R = 0;
    *S = 0;
    *smem = 0;
    *threads = 0;
    const size_t row_bytes = size_t(nx) * sizeof(typename ST::S);
    if (row_bytes % 16 != 0 || nx > kStagedMaxCpt * kConsumers) return;
    constexpr size_t kTwoCtaRing = 110u * 1024u, kOneCtaRing = 220u * 1024u;
    int r = kConsumers / nx;
    if (r < 1) r = 1;
    while (r > 1 && 2 * size_t(LT::Q) * r * row_bytes > kTwoCtaRing) --r;
    const size_t stage = size_t(LT::Q) * r * row_bytes;
    int s = int((2 * stage <= kTwoCtaRing ? kTwoCtaRing : kOneCtaRing) / stage);
    if (s > 4) s = 4;
    if (s < 2) return;
    const int cells = r * nx;
    int consumers = ((cells < kConsumers ? cells : kConsumers) + 31) / 32 * 32;
    *R = r;
    *S = s;
    *smem = 128 + size_t(s) * stage;
    *threads = 32 + consumers;
}

template <class LT, class ST>
bool staged_applies(int nx) {
    int R, S, threads;
    size_t smem;
    staged_geometry<LT, ST>(nx, &R, &S, &smem, &threads);
    return R > 0;
}

template <class LT, int K, class ST>
cudaError_t launch_step_staged(const StepArgs &a, int block, cudaStream_t stream) {
    using T = typename ST::T;
    (void)block;
    int R, S, threads;
    size_t smem;
    staged_geometry<LT, ST>(a.nx, &R, &S, &smem, &threads);
    if (R == 0) return cudaErrorInvalidValue;
    // opt in to large dynamic shared memory once per device (the attribute is per device)
    static std::atomic<unsigned long long> configured{0};  // solvers on other threads share it
    {
        int cur = 0;
        cudaError_t e = cudaGetDevice(&cur);
        if (e != cudaSuccess) return e;
        const unsigned long long bit = cur < 64 ? (1ull << cur) : 0ull;
        if (!bit || !(configured.load() & bit)) {
            e = cudaFuncSetAttribute(step_staged_kernel<LT, K, ST>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     227 * 1024);
            if (e != cudaSuccess) return e;
            configured.fetch_or(bit);
        }
    }
    // LBM_TEST_STAGED_EXTRA_TX=<bytes>: test hook that makes every CTA's first wait expire (read once)
    static const unsigned int extra_tx = [] {
        const char *v = getenv("LBM_TEST_STAGED_EXTRA_TX");
        return v ? unsigned(strtoul(v, nullptr, 10)) : 0u;
    }();
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, step_staged_kernel<LT, K, ST>,
                                                                  threads, smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const int rows = a.ny * a.nz;
    const int tiles = (rows + R - 1) / R;
    int grid = per_sm * sms;
    if (grid > tiles) grid = tiles;
    step_staged_kernel<LT, K, ST><<<grid, threads, smem, stream>>>(
        static_cast<const typename ST::S *>(a.src), static_cast<typename ST::S *>(a.dst), a.nx, a.ny, a.nz, a.P, R,
        S, T(a.relax), T(a.rho0), a.status, extra_tx);
    return cudaGetLastError();
}

}  // namespace lbm
