// lbm_batch_kernels.cuh -- flat cell pairs (two consecutive cells of the flat index per
// thread, any nx), the single-lattice step built on them (variant 2), and the batched
// multi-lattice step of the pools: persistent kernels over a device slot table.  Included
// by lbm_kernels.cuh after the register-pull step (pull_collide_store), which it reuses.
#pragma once

namespace lbm {

// ------------------------------------------------------------------ flat cell pairs
// Pre-collision values of one cell pulled with direct shifted loads (any nx).
template <class LT, class ST>
__device__ __forceinline__ void pull_cell_scaled(const typename ST::S *__restrict__ src, int nx, int ny, int nz,
                                                 long long P, int x, int y, int z, const QScale &qs,
                                                 typename ST::T (&f)[LT::Q], unsigned int *status) {
    constexpr int M = LT::MAXC;
    int xs[2 * M + 1], ys[2 * M + 1], zs[2 * M + 1];
#pragma unroll
    for (int k = -M; k <= M; ++k) {
        xs[k + M] = wrap1(x - k, nx);  // dims >= max|c| is checked on the host
        ys[k + M] = wrap1(y - k, ny);
        zs[k + M] = wrap1(z - k, nz);
    }
#pragma unroll
    for (int i = 0; i < LT::Q; ++i) {
        const long long in_plane =
            (long long)(zs[vel<LT>(i, 2) + M] * ny + ys[vel<LT>(i, 1) + M]) * nx + xs[vel<LT>(i, 0) + M];
        f[i] = guard(in_plane, 1, P, status) ? decode<ST>(src[(long long)i * P + in_plane], qs, i) : typename ST::T(0);
    }
}

// Two consecutive cells of the flat index, c0 = x0 + nx (y0 + ny z0) and c0 + 1 (when
// `second`), for any nx: each is pulled with direct loads, and the pair runs one pass of
// the collision on the paired FP32 instructions (two scalar passes in FP64).  No warp
// collectives: a thread with nothing to do may skip the call.
template <class LT, int K, class ST>
__device__ __forceinline__ void pull_collide_store_pair(const typename ST::S *__restrict__ src,
                                                        typename ST::S *__restrict__ dst, int nx, int ny, int nz,
                                                        long long P, int x0, int y0, int z0, bool second,
                                                        typename ST::T relax, typename ST::T rho0,
                                                        const QScale &qs, unsigned int *__restrict__ status) {
    using T = typename ST::T;
    constexpr int Q = LT::Q;
    int x1 = x0 + 1, y1 = y0, z1 = z0;  // the next cell in flat order (the same cell when !second)
    if (!second) {
        x1 = x0;
    } else if (x1 == nx) {
        x1 = 0;
        if (++y1 == ny) {
            y1 = 0;
            ++z1;
        }
    }
    T f0[Q], f1[Q];
    pull_cell_scaled<LT, ST>(src, nx, ny, nz, P, x0, y0, z0, qs, f0, status);
    pull_cell_scaled<LT, ST>(src, nx, ny, nz, P, x1, y1, z1, qs, f1, status);
    if constexpr (sizeof(T) == 4) {
        F2 g[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) g[i] = F2(make_float2(f0[i], f1[i]));
        collide<LT, K, F2>(g, F2(relax), F2(rho0), F2(0.0));
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            f0[i] = g[i].v.x;
            f1[i] = g[i].v.y;
        }
    } else {
        collide<LT, K, T>(f0, relax, rho0);
        collide<LT, K, T>(f1, relax, rho0);
    }
    const long long c0 = x0 + (long long)nx * (y0 + (long long)ny * z0);
    unsigned int acc = 0u;
    if (!guard(c0, second ? 2 : 1, P, status)) return;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        dst[(long long)i * P + c0] = encode<ST>(f0[i], qs, i, acc);
        if (second) dst[(long long)i * P + c0 + 1] = encode<ST>(f1[i], qs, i, acc);
    }
    if constexpr (ST::id == LBM_STORE_Q16) {
        if (range_exceeded(acc) && status) atomicOr(status, kStatusRange);
    }
}

// Single-lattice step on flat cell pairs (step variant 2): thread t updates cells 2t and
// 2t + 1 of the flat index, for any nx -- the variant that gives odd-sized lattices the
// paired collision.  Grid-stride over ceil(C / 2) pairs.
template <class LT, int K, class ST>
__global__ void __launch_bounds__(256) step_pair_kernel(const typename ST::S *__restrict__ src,
                                                        typename ST::S *__restrict__ dst, int nx, int ny, int nz,
                                                        long long P, typename ST::T relax, typename ST::T rho0,
                                                        QScale qs, unsigned int *__restrict__ status) {
    const long long pairs = (P + 1) / 2;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < pairs;
         t += (long long)gridDim.x * blockDim.x) {
        const long long c0 = 2 * t;
        const long long row = c0 / nx;
        const int z = int(row / ny);
        pull_collide_store_pair<LT, K, ST>(src, dst, nx, ny, nz, P, int(c0 - row * nx), int(row - (long long)z * ny),
                                           z, c0 + 1 < P, relax, rho0, qs, status);
    }
}

template <class LT, int K, class ST>
cudaError_t launch_step_pair(const StepArgs &a, int block, cudaStream_t stream) {
    using T = typename ST::T;
    if (block <= 0 || block > 256) block = 256;  // __launch_bounds__(256)
    int per_sm = 0, dev = 0, sms = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, step_pair_kernel<LT, K, ST>, block, 0);
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const long long pairs = (a.P + 1) / 2;
    long long grid = (pairs + block - 1) / block;
    const long long cap = (long long)(per_sm > 0 ? per_sm : 1) * sms * 8;  // a few waves, then stride
    if (grid > cap) grid = cap;
    step_pair_kernel<LT, K, ST><<<(unsigned)grid, block, 0, stream>>>(
        static_cast<const typename ST::S *>(a.src), static_cast<typename ST::S *>(a.dst), a.nx, a.ny, a.nz, a.P,
        T(a.relax), T(a.rho0), a.qs, a.status);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ batched step
// Persistent kernels over the work units of a slot table (one unit = blockDim.x consecutive
// threads of one lattice).  A pool stores every lattice with its rows padded to a pitch of a
// multiple of 4 whose pad cells hold periodic images (pull_collide_store, PADDED), so each
// lattice, whatever its nx, runs the register pull with V = 1, 2 or 4 cells per thread (MODE 0,
// 1, 2) on aligned row vectors: the pool's slot mode is one V for every resident lattice, and
// one launch of that mode's kernel advances every slot with step_index < steps_left by one
// step; the slot's buffers alternate with its parity.  A request's results do not depend on
// the other residents.  Header: [total units, slots, first unit of modes 0..2, end unit of
// modes 0..2] (kBatchHeaderInts).  The table lives in device memory, so a captured graph of
// launches stays valid while the host rewrites the table between chunks.

__device__ __forceinline__ int fastdiv(int n, unsigned int m, unsigned int s) {
    return int((__umulhi((unsigned int)n, m) + (unsigned int)n) >> s);
}

template <int MODE>
constexpr int batch_cells() {
    return MODE == 0 ? 1 : (MODE == 1 ? 2 : 4);
}

template <class LT, int K, class ST, int MODE>
__device__ __forceinline__ void batch_step_body(const BatchSlot *__restrict__ slots, const int *__restrict__ header,
                                                int step_index) {
    const int nslots = header[1];
    const int u_begin = header[2 + MODE], u_end = header[5 + MODE];
    // grid-stride over units (neighbouring CTAs work on neighbouring rows at the same time);
    // units only increase, so each thread walks the slot index forward without a barrier
    int slot = 0;
    for (int unit = u_begin + int(blockIdx.x); unit < u_end; unit += gridDim.x) {
        if (slot + 1 < nslots && slots[slot + 1].unit0 <= unit) {
            int lo = slot + 1, hi = nslots - 1;  // last slot with unit0 <= unit
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (slots[mid].unit0 <= unit) lo = mid;
                else hi = mid - 1;
            }
            slot = lo;
        }
        const BatchSlot &sl = slots[slot];
        if (step_index >= sl.steps_left) continue;  // uniform across the CTA
        const int cur = (sl.parity + step_index) & 1;
        const int total = sl.threads;
        int t = (unit - sl.unit0) * blockDim.x + threadIdx.x;
        const auto *src = static_cast<const typename ST::S *>(sl.buf[cur]);
        auto *dst = static_cast<typename ST::S *>(sl.buf[cur ^ 1]);
        const typename ST::T relax(sl.relax), rho0(sl.rho0), kq(0);
        const QScale qs = qscale_plain(sl.qmul, sl.qinv);
        const bool active = t < total;
        if (!active) t = total - 1;  // inactive lanes still take part in the shuffles
        const int row = fastdiv(t, sl.mx, sl.sx);  // t / ncx
        const int chunk = t - row * sl.ncx;
        const int z = fastdiv(row, sl.my, sl.sy);
        const int y = row - z * sl.ny;
        pull_collide_store<LT, K, ST, batch_cells<MODE>(), false, false, true>(
            src, dst, sl.nx, sl.ny, sl.nz, sl.ncx, sl.P, y, z, chunk, active, relax, rho0, kq, qs, sl.status, sl.px);
    }
}

template <class LT, int K, class ST, int MODE>
__global__ void __launch_bounds__(256) batch_step_kernel(const BatchSlot *__restrict__ slots,
                                                         const int *__restrict__ header, int step_index) {
    batch_step_body<LT, K, ST, MODE>(slots, header, step_index);
}

// Register cap of a mode's kernel (0 = none; a no-op cap would still change the allocation).
// Measured on 40 resident D3Q19 lattices, K = 3, four cells per thread: FP16 and BF16 at 96
// registers instead of 126 (five 128-thread CTAs per SM instead of four) gain 1.3% and 2.2%;
// the fixed-point form loses 2.3% there, and 80 registers lose for all three.  Otherwise the
// four-cell mode takes the single-lattice four-cell step's cap.
template <class LT, int K, class ST, int MODE>
constexpr int batch_cap() {
    if constexpr (MODE == 2 && LT::Q == 19 && (ST::id == LBM_STORE_F16 || ST::id == LBM_STORE_BF16)) return 96;
    else if constexpr (MODE == 2) return step_direct_cap<LT, K, ST, 4, false, false>();
    else return 0;
}

// The same kernel under a register cap (the qualifier excludes __launch_bounds__; blocks
// stay at <= 256 threads).
template <int REGS, class LT, int K, class ST, int MODE>
__global__ void __maxnreg__(REGS) batch_step_kernel_capped(const BatchSlot *__restrict__ slots,
                                                           const int *__restrict__ header, int step_index) {
    batch_step_body<LT, K, ST, MODE>(slots, header, step_index);
}

using BatchKernel = void (*)(const BatchSlot *, const int *, int);

template <class LT, int K, class ST, int MODE>
BatchKernel batch_kernel() {
    constexpr int cap = batch_cap<LT, K, ST, MODE>();
    if constexpr (cap > 0) return batch_step_kernel_capped<cap, LT, K, ST, MODE>;
    else return batch_step_kernel<LT, K, ST, MODE>;
}

template <class LT, int K, class ST>
BatchKernel batch_kernel_of_mode(int mode) {
    return mode == 2 ? batch_kernel<LT, K, ST, 2>() : (mode == 1 ? batch_kernel<LT, K, ST, 1>()
                                                                  : batch_kernel<LT, K, ST, 0>());
}

// One step of every slot: the kernel of the pool's mode (cells per thread 1, 2 or 4);
// grids[m] is mode m's persistent grid.
template <class LT, int K, class ST>
cudaError_t launch_batch(const BatchSlot *slots, const int *header, int step_index, const int *grids, int block,
                         int cpt, cudaStream_t stream) {
    const int mode = cpt == 4 ? 2 : (cpt == 2 ? 1 : 0);
    batch_kernel_of_mode<LT, K, ST>(mode)<<<grids[mode], block, 0, stream>>>(slots, header, step_index);
    return cudaGetLastError();
}

template <class LT, int K, class ST>
int batch_occupancy(int block, int mode) {
    int n = 0;
    const cudaError_t e =
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_kernel_of_mode<LT, K, ST>(mode), block, 0);
    return e == cudaSuccess ? n : 0;
}

}  // namespace lbm
