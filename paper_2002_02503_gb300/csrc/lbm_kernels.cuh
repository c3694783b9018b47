// lbm_kernels.cuh -- kernel templates of the fused lattice Boltzmann step and
// its helpers.  Included once per lattice by an instantiation unit.
//
// Storage: SoA planes g[i][z][y][x] (x fastest), one plane of P = nx*ny*nz
// values per velocity, in the lattice's pair order.  The stored field at step t
// is the post-collision distribution of step t-1 before streaming, so step t
// pulls f_i(x, t) = g_i(x - c_i) (Eq. lbe read backwards along each link),
// collides (Eq. lbe-reg) and writes g_i(x) of step t+1 to the other buffer.
#pragma once

#include <cuda_runtime.h>

#include <type_traits>

#include "lbm_core.cuh"
#include "lbm_internal.h"
#include "lbm_staged.cuh"

namespace lbm {

constexpr unsigned kFull = 0xffffffffu;

// ------------------------------------------------------------------ vector IO
template <int BYTES>
struct RawOf;
template <>
struct RawOf<2> { using type = unsigned short; };
template <>
struct RawOf<4> { using type = unsigned int; };
template <>
struct RawOf<8> { using type = uint2; };
template <>
struct RawOf<16> { using type = uint4; };

template <typename S, int V>
__device__ __forceinline__ void load_vec(const S *__restrict__ p, S (&out)[V]) {
    constexpr int B = int(sizeof(S)) * V;
    if constexpr (B <= 16) {
        using R = typename RawOf<B>::type;
        R r = *reinterpret_cast<const R *>(p);
        memcpy(out, &r, B);
    } else {
        static_assert(B % 16 == 0, "vector width");
#pragma unroll
        for (int k = 0; k < B / 16; ++k) {
            uint4 r = reinterpret_cast<const uint4 *>(p)[k];
            memcpy(reinterpret_cast<char *>(out) + 16 * k, &r, 16);
        }
    }
}

template <typename S, int V>
__device__ __forceinline__ void store_vec(S *__restrict__ p, const S (&in)[V]) {
    constexpr int B = int(sizeof(S)) * V;
    if constexpr (B <= 16) {
        using R = typename RawOf<B>::type;
        R r;
        memcpy(&r, in, B);
        *reinterpret_cast<R *>(p) = r;
    } else {
#pragma unroll
        for (int k = 0; k < B / 16; ++k) {
            uint4 r;
            memcpy(&r, reinterpret_cast<const char *>(in) + 16 * k, 16);
            reinterpret_cast<uint4 *>(p)[k] = r;
        }
    }
}

__device__ __forceinline__ int wrap1(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }
__device__ __forceinline__ int wrapn(int v, int n) {
    v %= n;
    return v < 0 ? v + n : v;
}
__host__ __device__ constexpr int floordiv(int e, int V) { return e >= 0 ? e / V : -((-e + V - 1) / V); }

// ------------------------------------------------------------------ fused step, variant 0
// One thread owns V consecutive cells (a chunk) of one x-row.  For velocity c it needs the
// source row's values at x0 - c_x ... x0 + V - 1 - c_x.  Two ways to get them:
//  - whole-chunk loads (unpadded rows of D3Q39 and of the reference-velocity forms): every
//    chunk holding one of them is loaded as an aligned vector -- its own and up to
//    ceil(max|c_x| / V) neighbours, which the neighbouring lanes load as well, so they come
//    from L1 -- with no shuffles and no per-lane fix-ups;
//  - shuffles (the other sets, and the pools' padded rows): the thread loads its own chunk and
//    realigns the shift with warp shuffles; lanes whose neighbour does not hold the adjacent
//    chunk of the same row (warp or row edge, periodic wrap) read the missing values directly.
// Every lane of the warp must call this (the shuffles use the full mask); lanes with
// active == false compute on a valid clamped position and store nothing.
//
// PADDED (the pools' layout): rows are stored with a pitch px >= nx (a multiple of 4), and
// the pad cells x = nx + k hold periodic images of cells k.  A pad cell pulls exactly the
// values its original pulls (its sources are images or, past the row, wrap onto the same
// cells), so it computes and stores the same bits and the images stay exact; chunks run over
// the whole pitch (ncx = px / V), and a source x outside the stored row moves by one period
// nx into it.  Without it px = nx.
template <class LT, int K, class ST, int V, bool BGK = false, bool THETA = false, bool PADDED = false>
__device__ __forceinline__ void pull_collide_store(const typename ST::S *__restrict__ src,
                                                   typename ST::S *__restrict__ dst, int nx, int ny, int nz, int ncx,
                                                   long long P, int y, int z, int chunk, bool active,
                                                   typename ST::T relax, typename ST::T rho0, typename ST::T kq,
                                                   const QScale &qs, unsigned int *__restrict__ status,
                                                   int pitch = 0) {
    using S = typename ST::S;
    using T = typename ST::T;
    constexpr int Q = LT::Q, M = LT::MAXC;
    const int lane = threadIdx.x & 31;
    const int x0 = chunk * V;
    const int px = PADDED ? pitch : nx;  // row pitch in stored elements
    // x of a source cell brought into the stored row [0, px) by one period nx: every stored
    // position congruent to it modulo nx holds its value (pads are images), and x lies in
    // [-M, px - 1 + M] with nx >= M, so one step either way is enough
    auto wrapx = [&](int v) { return v < 0 ? v + nx : (v >= px ? v - nx : v); };

    int ys[2 * M + 1], zs[2 * M + 1];
#pragma unroll
    for (int k = -M; k <= M; ++k) {
        ys[k + M] = wrap1(y - k, ny);  // dims >= max|c| is checked on the host
        zs[k + M] = wrap1(z - k, nz);
    }
    // lane offsets dl of the x shift: |dl| <= ceil(M / V); ok[dl] = neighbour lane holds chunk + dl
    constexpr int kMaxDl = (M + V - 1) / V;
    bool ok[2 * kMaxDl + 1];
#pragma unroll
    for (int dl = -kMaxDl; dl <= kMaxDl; ++dl)
        ok[dl + kMaxDl] = V > 1 && lane + dl >= 0 && lane + dl <= 31 && chunk + dl >= 0 && chunk + dl < ncx;

    int xs[2 * M + 1];  // wrapped source x of one cell per thread (V = 1)
#pragma unroll
    for (int k = -M; k <= M; ++k) xs[k + M] = wrapx(x0 - k);
    // Whole-chunk loads on unpadded rows (which hold a whole number of chunks, so the periodic
    // wrap moves whole chunks): xc[dl] is the first x of chunk + dl of the same row (nx >= max|c|
    // keeps |dl| <= ncx).  Measured against the shuffles: D3Q39 K = 4 FP16 +27%, the reference-
    // velocity forms +8%; on the max|c| = 1 sets with the held values the extra addresses cost
    // registers (fixed point -10% from a spill, D3Q27 FP16 -3.5%), so those keep the shuffles.
    constexpr bool kChunkLoads = !PADDED && V > 1 && (M >= 2 || RefOf<ST>::value);
    int xc[2 * kMaxDl + 1];
#pragma unroll
    for (int dl = -kMaxDl; dl <= kMaxDl; ++dl) xc[dl + kMaxDl] = kChunkLoads ? wrap1(chunk + dl, ncx) * V : 0;

    // Offsets within a plane (< P <= 2^31 - 1, checked on the host) as 32-bit ints on unpadded
    // D3Q19 rows with the plain storage forms, 64-bit elsewhere -- the addressing form that
    // measured faster per case (ints: D3Q19 K = 3 FP16 four cells +9%, fixed point +1%; D3Q27
    // K = 3 FP16 -15%, D3Q39 K = 4 FP16 -6%, FP16 with a reference velocity -3%, the FP32 pool
    // -10%, the FP16 pool +0.7%), as ptxas schedules and allocates the address arithmetic
    // differently.
    constexpr bool kIntOffsets = !PADDED && LT::Q == 19 && !RefOf<ST>::value;
    using Off = typename std::conditional<kIntOffsets, int, long long>::type;

    // The V values of one stored plane pulled along velocity (cx, cy, cz): out[j] holds the
    // plane's value at x0 + j - cx of row (y - cy, z - cz).  ci: the codec's velocity index.
    auto pull = [&](const S *__restrict__ plane, int cx, int cy, int cz, int ci, T(&out)[V]) {
        const Off roff = Off(zs[cz + M] * ny + ys[cy + M]) * Off(px);  // row offset in its plane
        const S *row = plane + roff;  // (the 64-bit form addresses element x as row + x)
        if constexpr (V == 1) {
            // one cell per thread: load the x-shifted element directly (the warp's load is still
            // one contiguous span; the neighbour warps' loads keep the extra sector in cache)
            out[0] = guard(roff + xs[cx + M], 1, P, status) ? decode<ST>(kIntOffsets ? plane[roff + xs[cx + M]] : row[xs[cx + M]], qs, ci) : T(0);
        } else if constexpr (kChunkLoads) {
            // load each chunk that holds a shifted value whole (an aligned vector load; the
            // neighbour lanes' chunks come from L1) and take the values from it
#pragma unroll
            for (int dl = -kMaxDl; dl <= kMaxDl; ++dl) {
                bool need = false;
#pragma unroll
                for (int j = 0; j < V; ++j) need |= floordiv(j - cx, V) == dl;
                if (!need) continue;
                const int xo = xc[dl + kMaxDl];
                S raw[V] = {};
                if (guard(roff + xo, V, P, status)) load_vec<S, V>(kIntOffsets ? plane + (roff + xo) : row + xo, raw);
                T v[V];
                decode_vec<ST, V>(raw, v, qs, ci);
#pragma unroll
                for (int j = 0; j < V; ++j) {
                    const int e = j - cx;  // source element relative to x0
                    if (floordiv(e, V) == dl) out[j] = v[e - dl * V];
                }
            }
        } else {
            S raw[V] = {};
            if (guard(roff + x0, V, P, status)) load_vec<S, V>(kIntOffsets ? plane + (roff + x0) : row + x0, raw);
            T v[V];
            decode_vec<ST, V>(raw, v, qs, ci);
            if (cx == 0) {
#pragma unroll
                for (int j = 0; j < V; ++j) out[j] = v[j];
            } else {
#pragma unroll
                for (int j = 0; j < V; ++j) {
                    const int e = j - cx;  // source element relative to x0
                    const int dl = floordiv(e, V);
                    const int ei = e - dl * V;
                    if (dl == 0) {
                        out[j] = v[ei];
                    } else {
                        // source lane lane+dl holds chunk+dl of the same row unless at a warp or row edge
                        const int sl = lane + dl;
                        T sh = __shfl_sync(kFull, v[ei], sl < 0 ? 0 : (sl > 31 ? 31 : sl));
                        if (!ok[dl + kMaxDl]) {
                            const int xw = wrapx(x0 + e);
                            sh = guard(roff + xw, 1, P, status) ? decode<ST>(kIntOffsets ? plane[roff + xw] : row[xw], qs, ci) : T(0);
                        }
                        out[j] = sh;
                    }
                }
            }
        }
    };

    // reference-velocity forms: add back r_i of the cell each value of velocity i came from (its
    // reference planes, pulled along the same velocity); two cells per instruction where V allows
    auto add_reference = [&](int i, T(&v)[V]) {
        if constexpr (RefOf<ST>::value) {
            T a[3][V];
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                if (d < LT::D && vel<LT>(i, d) != 0) {
                    pull(src + (long long)(Q + d) * P, vel<LT>(i, 0), vel<LT>(i, 1), vel<LT>(i, 2), 0, a[d]);
                } else {
#pragma unroll
                    for (int j = 0; j < V; ++j) a[d][j] = T(0);
                }
            }
            if constexpr (V % 2 == 0) {
#pragma unroll
                for (int j = 0; j < V; j += 2) {
                    F2 a2[3];
#pragma unroll
                    for (int d = 0; d < 3; ++d) a2[d] = F2(make_float2(a[d][j], a[d][j + 1]));
                    const F2 h = F2(make_float2(v[j], v[j + 1])) + ref_value<LT>(i, a2);
                    v[j] = h.v.x;
                    v[j + 1] = h.v.y;
                }
            } else {
#pragma unroll
                for (int j = 0; j < V; ++j) {
                    const T a1[3] = {a[0][j], a[1][j], a[2][j]};
                    v[j] += ref_value<LT>(i, a1);
                }
            }
        }
    };

    constexpr bool kRef = RefOf<ST>::value;
    constexpr bool kPaired = V % 2 == 0 && sizeof(T) == 4;
    unsigned int acc = 0u;

    // The filtered collision needs the pulled values only through their moments: on the large
    // velocity sets (Q >= 27) each value is folded into MomentSums as it arrives and dropped, and
    // each post-collision value is formed from the moments just before it is stored -- no Q x V
    // array of values is held, which frees the registers four cells per thread need there
    // (D3Q39 K = 4, FP16, two cells per thread: 126 -> 74 registers).  On the smaller sets the
    // held values cost fewer registers than the per-cell output constants, and holding them
    // measured faster (D3Q19 K = 3 FP16 -9%, fixed point -11% when streamed).
    constexpr bool kStream = !BGK && !THETA && LT::Q >= 27;
    if constexpr (kStream) {
        // FP32 arithmetic with V >= 2 runs two cells per pass on the paired FP32 instructions.
        const Off ooff = Off(z * ny + y) * Off(px) + x0;  // offset of the thread's cells in a plane
        S *out = dst + ooff;
        const bool store_ok = active && guard(ooff, V, P, status);
        using A = typename std::conditional<kPaired, F2, T>::type;
        constexpr int NA = kPaired ? V / 2 : V;
        auto pack = [&](const T(&v)[V], int n) -> A {
            if constexpr (kPaired) return F2(make_float2(v[2 * n], v[2 * n + 1]));
            else return v[n];
        };
        auto unpack = [&](A x, T(&v)[V], int n) {
            if constexpr (kPaired) {
                v[2 * n] = x.v.x;
                v[2 * n + 1] = x.v.y;
            } else {
                v[n] = x;
            }
        };
        auto store_plane = [&](int i, const T(&v)[V]) {
            S raw[V];
            encode_vec<ST, V>(v, raw, qs, i, acc);
            if (store_ok) store_vec<S, V>(out + (long long)i * P, raw);
        };
        MomentSums<LT, A> ms[NA];
        {
            T v0[V];
            pull(src, 0, 0, 0, 0, v0);
#pragma unroll
            for (int n = 0; n < NA; ++n) ms[n].start(pack(v0, n));
        }
#pragma unroll
        for (int p = 0; p < LT::NP; ++p) {
            const int ip = 2 * p + 1, im = 2 * p + 2;
            T vp[V], vm[V];
            pull(src + (long long)ip * P, vel<LT>(ip, 0), vel<LT>(ip, 1), vel<LT>(ip, 2), ip, vp);
            pull(src + (long long)im * P, vel<LT>(im, 0), vel<LT>(im, 1), vel<LT>(im, 2), im, vm);
            add_reference(ip, vp);
            add_reference(im, vm);
#pragma unroll
            for (int n = 0; n < NA; ++n) ms[n].add_pair(p, pack(vp, n), pack(vm, n));
        }
        FilteredOutput<LT, K, A> fo[NA];
        A us_n[NA][3];
#pragma unroll
        for (int n = 0; n < NA; ++n) fo[n].init(ms[n], A(relax), A(rho0), kRef ? us_n[n] : nullptr);
        A ar[NA][3];  // the rounded reference a = u / T0 (reference forms)
        if constexpr (kRef) {
            S refraw[3][V];
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                if (d < LT::D) {
                    T v[V], back[V];
#pragma unroll
                    for (int n = 0; n < NA; ++n) unpack(us_n[n][d], v, n);
                    encode_vec<ST, V>(v, refraw[d], qs, 0, acc);
                    decode_vec<ST, V>(refraw[d], back, qs, 0);
#pragma unroll
                    for (int n = 0; n < NA; ++n) ar[n][d] = pack(back, n);
                    if (store_ok) store_vec<S, V>(out + (long long)(Q + d) * P, refraw[d]);
                } else {
#pragma unroll
                    for (int n = 0; n < NA; ++n) ar[n][d] = A(0.0);
                }
            }
        }
        {
            T v[V];
#pragma unroll
            for (int n = 0; n < NA; ++n) unpack(fo[n].rest(), v, n);
            store_plane(0, v);
        }
#pragma unroll
        for (int p = 0; p < LT::NP; ++p) {
            T vp[V], vm[V];
#pragma unroll
            for (int n = 0; n < NA; ++n) {
                A gp, gm;
                fo[n].pair(p, gp, gm);
                if constexpr (kRef) {
                    A rp, rm;
                    ref_pair<LT>(p, ar[n], rp, rm);
                    gp -= rp;
                    gm -= rm;
                }
                unpack(gp, vp, n);
                unpack(gm, vm, n);
            }
            store_plane(2 * p + 1, vp);
            store_plane(2 * p + 2, vm);
        }
        if constexpr (ST::id == LBM_STORE_Q16) {
            // one flag per warp that met a value outside the fixed-point range
            if (__any_sync(kFull, range_exceeded(acc)) && lane == 0 && status) atomicOr(status, kStatusRange);
        }
    } else {
    // held values (smaller velocity sets, BGK and the energy-flux term, which need the values
    // themselves): pull all of them, collide, store
    T f[Q][V];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        pull(src + (long long)i * P, vel<LT>(i, 0), vel<LT>(i, 1), vel<LT>(i, 2), i, f[i]);
        if (i > 0) add_reference(i, f[i]);
    }

    S refraw[3][V];  // the rounded reference a = u / T0 of each cell (reference forms only)
    if constexpr (kPaired) {
#pragma unroll
        for (int j = 0; j < V; j += 2) {
            F2 g[Q];
#pragma unroll
            for (int i = 0; i < Q; ++i) g[i] = F2(make_float2(f[i][j], f[i][j + 1]));
            F2 u2[3];
            if constexpr (BGK) collide_bgk<LT, K, F2>(g, F2(relax), F2(rho0), kRef ? u2 : nullptr);
            else collide<LT, K, F2, THETA>(g, F2(relax), F2(rho0), F2(kq), kRef ? u2 : nullptr);
            if constexpr (kRef) {
                // the reference a = u / T0 of both cells rounded to the storage type; the values
                // keep only their residual h_i - r_i
                F2 a2[3];
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    if (d < LT::D) {
                        T v[2] = {u2[d].v.x, u2[d].v.y}, back[2];
                        S raw2[2];
                        encode_vec<ST, 2>(v, raw2, qs, 0, acc);
                        decode_vec<ST, 2>(raw2, back, qs, 0);
                        a2[d] = F2(make_float2(back[0], back[1]));
                        refraw[d][j] = raw2[0];
                        refraw[d][j + 1] = raw2[1];
                    } else {
                        a2[d] = F2(0.0);
                    }
                }
#pragma unroll
                for (int p = 0; p < LT::NP; ++p) {
                    F2 rp, rm;
                    ref_pair<LT>(p, a2, rp, rm);
                    g[2 * p + 1] -= rp;
                    g[2 * p + 2] -= rm;
                }
            }
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                f[i][j] = g[i].v.x;
                f[i][j + 1] = g[i].v.y;
            }
        }
    } else {
#pragma unroll
        for (int j = 0; j < V; ++j) {
            T g[Q];
#pragma unroll
            for (int i = 0; i < Q; ++i) g[i] = f[i][j];
            T u1[3];
            if constexpr (BGK) collide_bgk<LT, K, T>(g, relax, rho0, kRef ? u1 : nullptr);
            else collide<LT, K, T, THETA>(g, relax, rho0, kq, kRef ? u1 : nullptr);
            if constexpr (kRef) {
                T a1[3];
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    if (d < LT::D) {
                        refraw[d][j] = encode<ST>(u1[d], qs, 0, acc);
                        a1[d] = decode<ST>(refraw[d][j], qs, 0);
                    } else {
                        a1[d] = T(0);
                    }
                }
#pragma unroll
                for (int p = 0; p < LT::NP; ++p) {
                    T rp, rm;
                    ref_pair<LT>(p, a1, rp, rm);
                    g[2 * p + 1] -= rp;
                    g[2 * p + 2] -= rm;
                }
            }
#pragma unroll
            for (int i = 0; i < Q; ++i) f[i][j] = g[i];
        }
    }

    const Off ooff = Off(z * ny + y) * Off(px) + x0;  // offset of the thread's cells in a plane
    S *out = dst + ooff;
    const bool store_ok = active && guard(ooff, V, P, status);
    if constexpr (kRef) {
        if (store_ok) {
#pragma unroll
            for (int d = 0; d < LT::D; ++d) store_vec<S, V>(out + (long long)(Q + d) * P, refraw[d]);
        }
    }
    if (store_ok) {
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            S raw[V];
            encode_vec<ST, V>(f[i], raw, qs, i, acc);
            store_vec<S, V>(out + (long long)i * P, raw);
        }
    }
    if constexpr (ST::id == LBM_STORE_Q16) {
        // one flag per warp that met a value outside the fixed-point range
        if (__any_sync(kFull, range_exceeded(acc)) && lane == 0 && status) atomicOr(status, kStatusRange);
    }
    }
}

template <class LT, int K, class ST, int V, bool BGK, bool THETA>
__device__ __forceinline__ void step_direct_body(const typename ST::S *__restrict__ src, typename ST::S *__restrict__ dst,
                                                 int nx, int ny, int ncx, long long P, typename ST::T relax,
                                                 typename ST::T rho0, typename ST::T kq, const QScale &qs,
                                                 unsigned int *__restrict__ status) {
    const int z = blockIdx.y;
    const int total = ncx * ny;
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = t < total;
    if (!active) t = total - 1;  // inactive lanes still take part in the shuffles
    const int y = t / ncx;
    const int chunk = t - y * ncx;
    pull_collide_store<LT, K, ST, V, BGK, THETA>(src, dst, nx, ny, gridDim.y, ncx, P, y, z, chunk, active, relax,
                                                 rho0, kq, qs, status);
}

template <class LT, int K, class ST, int V, bool BGK = false, bool THETA = false>
__global__ void __launch_bounds__(256) step_direct_kernel(const typename ST::S *__restrict__ src,
                                                          typename ST::S *__restrict__ dst, int nx, int ny,
                                                          int ncx, long long P, typename ST::T relax,
                                                          typename ST::T rho0, typename ST::T kq, QScale qs,
                                                          unsigned int *__restrict__ status) {
    step_direct_body<LT, K, ST, V, BGK, THETA>(src, dst, nx, ny, ncx, P, relax, rho0, kq, qs, status);
}

// The same step with a register cap, for the configurations where a cap pays (the cap that
// takes one more CTA per SM without spills, chosen by measurement):
//  - fixed point, four cells per thread, D3Q19, K = 2: ~108 registers, four 128-thread CTAs
//    per SM; at 96 five fit and the step runs 8% faster;
//  - FP32 energy-flux step, D3Q39, K = 4: 128 registers, four CTAs; at 96 five, 1.6% faster
//    even with the 56-byte spill it had then (at 104, with four CTAs still, 2% slower); since the
//    energy-flux contractions run over the distinct tensor components it fits 96 without one;
//  - reference-velocity storage, four cells per thread, D3Q19: 130 registers, three CTAs; at
//    128 four.
// A cap is not applied elsewhere: even a no-op cap changes the register allocation.  The
// qualifier excludes __launch_bounds__; the launcher keeps blocks at <= 256 threads.
template <class LT, int K, class ST, int V, bool BGK, bool THETA>
constexpr int step_direct_cap() {
    if constexpr (THETA && LT::Q == 39 && K == 4 && V == 1 && ST::id == LBM_STORE_F32) return 96;
    else if constexpr (RefOf<ST>::value && LT::Q == 19 && V == 4 && !BGK && !THETA) return 128;
    else if constexpr (ST::id != LBM_STORE_Q16 || BGK || THETA) return 0;
    else if constexpr (LT::Q == 19 && K == 2 && V == 4) return 96;
    else return 0;
}

template <int REGS, class LT, int K, class ST, int V, bool BGK = false, bool THETA = false>
__global__ void __maxnreg__(REGS) step_direct_kernel_capped(const typename ST::S *__restrict__ src,
                                                            typename ST::S *__restrict__ dst, int nx, int ny,
                                                            int ncx, long long P, typename ST::T relax,
                                                            typename ST::T rho0, typename ST::T kq, QScale qs,
                                                            unsigned int *__restrict__ status) {
    step_direct_body<LT, K, ST, V, BGK, THETA>(src, dst, nx, ny, ncx, P, relax, rho0, kq, qs, status);
}

template <class LT, int K, class ST, int V, bool BGK = false, bool THETA = false>
cudaError_t launch_step_direct(const StepArgs &a, int block, cudaStream_t stream) {
    using T = typename ST::T;
    if (a.nx % V) return cudaErrorInvalidValue;
    const int ncx = a.nx / V;
    const long long total = (long long)ncx * a.ny;
    if (block <= 0) block = 256;
    if (block > 256) block = 256;  // __launch_bounds__(256)
    const long long gx = (total + block - 1) / block;
    if (gx > 0x7fffffffLL || a.nz > 65535) return cudaErrorInvalidConfiguration;
    dim3 grid((unsigned)gx, (unsigned)a.nz);
    // (1 - 1/tau) theta / (6 T0^3): weight of the energy-flux part (Eq. pq)
    const double kq = a.relax * a.theta / (6.0 * LT::T0 * LT::T0 * LT::T0);
    constexpr int kCap = step_direct_cap<LT, K, ST, V, BGK, THETA>();
    if constexpr (kCap > 0)
        step_direct_kernel_capped<kCap, LT, K, ST, V, BGK, THETA><<<grid, block, 0, stream>>>(
            static_cast<const typename ST::S *>(a.src), static_cast<typename ST::S *>(a.dst), a.nx, a.ny, ncx, a.P,
            T(a.relax), T(a.rho0), T(kq), a.qs, a.status);
    else
        step_direct_kernel<LT, K, ST, V, BGK, THETA><<<grid, block, 0, stream>>>(
            static_cast<const typename ST::S *>(a.src), static_cast<typename ST::S *>(a.dst), a.nx, a.ny, ncx, a.P,
            T(a.relax), T(a.rho0), T(kq), a.qs, a.status);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ set_fields
// f_i(x, 0) = f^eq_i(rho(x), u(x)) is computed in the collision's arithmetic type
// and written to the stored field at x - c_i, so that the first pull of step 0
// reads it back at x.
// The forms with a reference velocity take two passes over the cells: phase 0 stores each
// cell's reference a = u / T0 (rounded) at its own position; phase 1 stores f^eq relative to
// the reference of the position it is written to.
// px: the row pitch of the stored field (nx, or the pools' padded pitch, whose pad cells
// x = nx + k receive the images of cells k).
template <class LT, int K, class ST>
__global__ void init_kernel(typename ST::S *__restrict__ dst, const double *__restrict__ rho,
                            const double *__restrict__ u, long long ustride, long long c0, long long count, int nx,
                            int ny, int nz, long long P, double rho0, QScale qs,
                            unsigned int *__restrict__ status, unsigned int *__restrict__ hmax, int phase, int px) {
    using S = typename ST::S;
    using T = typename ST::T;
    unsigned int acc = 0u;
    unsigned int hbits = 0u;  // largest |h| seen, as float bits (ordered like the values; NaN above all)
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < count;
         k += (long long)gridDim.x * blockDim.x) {
        const long long cell = c0 + k;
        const int x = int(cell % nx);
        const int y = int((cell / nx) % ny);
        const int z = int(cell / ((long long)nx * ny));
        const double r = rho[k];
        T uu[3] = {T(0), T(0), T(0)};
#pragma unroll
        for (int a = 0; a < LT::D; ++a) uu[a] = T(u[a * ustride + k]);
        if constexpr (RefOf<ST>::value) {
            if (phase == 0) {
                if (guard(cell, 1, P, status)) {  // (reference forms run on single lattices: px = nx)
#pragma unroll
                    for (int a = 0; a < LT::D; ++a)
                        dst[(long long)(LT::Q + a) * P + cell] = encode<ST>(uu[a] * T(1.0 / LT::T0), qs, 0, acc);
                }
                continue;
            }
        }
        T g[LT::Q];
        equilibrium_shifted<LT, K, T>(T(r), T(r - rho0), uu, g);
        if (hmax) {  // measuring pass (automatic fixed-point range): nothing is stored
#pragma unroll
            for (int i = 0; i < LT::Q; ++i) hbits = max(hbits, __float_as_uint(fabsf(float(g[i]) - qs.ref[i])));
            continue;
        }
#pragma unroll
        for (int i = 0; i < LT::Q; ++i) {
            const int xs = wrapn(x - vel<LT>(i, 0), nx);
            const int ysrc = wrapn(y - vel<LT>(i, 1), ny);
            const int zsrc = wrapn(z - vel<LT>(i, 2), nz);
            const long long at = (long long)(zsrc * ny + ysrc) * px + xs;
            if (!guard(at, 1, P, status)) continue;
            T v = g[i];
            if constexpr (RefOf<ST>::value) {
                if (i > 0) {
                    T a[3];
#pragma unroll
                    for (int d = 0; d < 3; ++d)
                        a[d] = (d < LT::D && vel<LT>(i, d) != 0) ? decode<ST>(dst[(long long)(LT::Q + d) * P + at], qs, 0)
                                                                  : T(0);
                    v -= ref_value<LT>(i, a);
                }
            }
            const typename ST::S code = encode<ST>(v, qs, i, acc);
            dst[(long long)i * P + at] = code;
            for (int q = xs + nx; q < px; q += nx)  // the pad images of this position (padded rows)
                if (guard(at - xs + q, 1, P, status)) dst[(long long)i * P + at - xs + q] = code;
        }
    }
    if constexpr (ST::id == LBM_STORE_Q16) {
        if (range_exceeded(acc) && status) atomicOr(status, kStatusRange);
    }
    if (hmax) {  // every thread of the (full) warps gets here: one atomic per warp
        hbits = __reduce_max_sync(kFull, hbits);
        if ((threadIdx.x & 31) == 0) atomicMax(hmax, hbits);
    }
}

template <class LT, int K, class ST>
cudaError_t launch_init(const InitArgs &a, cudaStream_t stream) {
    if (a.count <= 0) return cudaSuccess;
    long long blocks = (a.count + 255) / 256;
    if (blocks > 65535) blocks = 65535;
    init_kernel<LT, K, ST><<<(unsigned)blocks, 256, 0, stream>>>(static_cast<typename ST::S *>(a.dst), a.rho, a.u,
                                                                  a.ustride, a.c0, a.count, a.nx, a.ny, a.nz, a.P,
                                                                  a.rho0, a.qs, a.status, a.hmax, a.phase,
                                                                  a.px > 0 ? a.px : a.nx);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ pulled observables
// Pre-collision f_i(x, t) = g_i(x - c_i) decoded to FP64; rho and u per Eq. mme.
template <class LT, class ST>
__device__ __forceinline__ void pull_cell(const typename ST::S *__restrict__ src, long long cell, int nx, int ny,
                                          int nz, long long P, const QScale &qs, double (&gt)[LT::Q],
                                          unsigned int *status, int px) {
    const int x = int(cell % nx);
    const int y = int((cell / nx) % ny);
    const int z = int(cell / ((long long)nx * ny));
#pragma unroll
    for (int i = 0; i < LT::Q; ++i) {
        const int xs = wrapn(x - vel<LT>(i, 0), nx);
        const int ysrc = wrapn(y - vel<LT>(i, 1), ny);
        const int zsrc = wrapn(z - vel<LT>(i, 2), nz);
        const long long at = (long long)(zsrc * ny + ysrc) * px + xs;
        if (!guard(at, 1, P, status)) {
            gt[i] = 0.0;
            continue;
        }
        typename ST::T h = decode<ST>(src[(long long)i * P + at], qs, i);
        if constexpr (RefOf<ST>::value) {  // the value's reference, as the step adds it back
            using T = typename ST::T;
            T a[3];
#pragma unroll
            for (int d = 0; d < 3; ++d)
                a[d] = (d < LT::D && vel<LT>(i, d) != 0) ? decode<ST>(src[(long long)(LT::Q + d) * P + at], qs, 0)
                                                          : T(0);
            if (i > 0) h += ref_value<LT>(i, a);
        }
        gt[i] = weight<LT>(i) * double(h);
    }
}

template <class LT, class ST>
__global__ void moments_kernel(const typename ST::S *__restrict__ src, double *__restrict__ rho,
                               double *__restrict__ u, double *__restrict__ f, long long ustride, long long fstride,
                               long long c0, long long count, int nx, int ny, int nz, long long P, double rho0,
                               QScale qs, unsigned int *__restrict__ status, int px) {
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < count;
         k += (long long)gridDim.x * blockDim.x) {
        double gt[LT::Q];
        pull_cell<LT, ST>(src, c0 + k, nx, ny, nz, P, qs, gt, status, px);
        if (f) {
#pragma unroll
            for (int i = 0; i < LT::Q; ++i) f[i * fstride + k] = gt[i] + weight<LT>(i) * rho0;
        }
        if (rho || u) {
            double dr = 0.0, j[3] = {0.0, 0.0, 0.0};
#pragma unroll
            for (int i = 0; i < LT::Q; ++i) {
                dr += gt[i];
#pragma unroll
                for (int a = 0; a < LT::D; ++a) j[a] += double(vel<LT>(i, a)) * gt[i];
            }
            const double r = rho0 + dr;
            if (rho) rho[k] = r;
            if (u) {
#pragma unroll
                for (int a = 0; a < LT::D; ++a) u[a * ustride + k] = j[a] / r;
            }
        }
    }
}

template <class LT, class ST>
cudaError_t launch_moments(const PullArgs &a, cudaStream_t stream) {
    if (a.count <= 0) return cudaSuccess;
    long long blocks = (a.count + 255) / 256;
    if (blocks > 65535) blocks = 65535;
    moments_kernel<LT, ST><<<(unsigned)blocks, 256, 0, stream>>>(static_cast<const typename ST::S *>(a.src), a.rho,
                                                                  a.u, nullptr, a.ustride, a.fstride, a.c0, a.count,
                                                                  a.nx, a.ny, a.nz, a.P, a.rho0, a.qs, a.status,
                                                                  a.px > 0 ? a.px : a.nx);
    return cudaGetLastError();
}

template <class LT, class ST>
cudaError_t launch_pull_f(const PullArgs &a, cudaStream_t stream) {
    if (a.count <= 0) return cudaSuccess;
    long long blocks = (a.count + 255) / 256;
    if (blocks > 65535) blocks = 65535;
    moments_kernel<LT, ST><<<(unsigned)blocks, 256, 0, stream>>>(static_cast<const typename ST::S *>(a.src), nullptr,
                                                                  nullptr, a.f, a.ustride, a.fstride, a.c0, a.count,
                                                                  a.nx, a.ny, a.nz, a.P, a.rho0, a.qs, a.status,
                                                                  a.px > 0 ? a.px : a.nx);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ FP64 reductions
// Deterministic two-pass sums: each block reduces a fixed cell range with warp
// shuffles and shared memory, writes its partials, and one block adds the
// partials in block order.
template <int NV>
__device__ __forceinline__ void block_reduce_store(double (&v)[NV], double *__restrict__ partials) {
    __shared__ double sh[kReduceThreads / 32][NV];
#pragma unroll
    for (int q = 0; q < NV; ++q)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_down_sync(kFull, v[q], o);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < NV; ++q) sh[warp][q] = v[q];
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            double s = 0.0;
            for (int w = 0; w < kReduceThreads / 32; ++w) s += sh[w][q];
            partials[blockIdx.x * NV + q] = s;
        }
    }
}

template <int NV>
__global__ void final_reduce_kernel(const double *__restrict__ partials, int blocks, double *__restrict__ out) {
    // one warp per value, lanes stride over blocks in a fixed order
    const int q = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (q >= NV) return;
    double s = 0.0;
    for (int b = lane; b < blocks; b += 32) s += partials[b * NV + q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(kFull, s, o);
    if (lane == 0) out[q] = s;
}

// Total mass and momentum: shift-invariant sums, so the stored field is summed
// plane by plane without pulling: sum_x rho = C rho0 + sum_i sum_y g~_i(y).
template <class LT, class ST>
__global__ void __launch_bounds__(kReduceThreads) conservation_kernel(const typename ST::S *__restrict__ src,
                                                                      long long P, double rho0, QScale qs,
                                                                      double *__restrict__ partials,
                                                                      unsigned int *__restrict__ status) {
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    const long long per = (P + gridDim.x - 1) / gridDim.x;
    const long long b0 = blockIdx.x * per;
    const long long b1 = b0 + per < P ? b0 + per : P;
    // one FP64 accumulator per velocity plane (FP64 adds are scarce on this GPU);
    // the lattice velocities weight the plane sums once at the end
    double acc[LT::Q];
#pragma unroll
    for (int i = 0; i < LT::Q; ++i) acc[i] = 0.0;
    long long n = 0;
    for (long long k = b0 + threadIdx.x; k < b1; k += blockDim.x) {
        if (!guard(k, 1, P, status)) continue;
        if constexpr (RefOf<ST>::value) {
            using T = typename ST::T;
            T a[3];
#pragma unroll
            for (int d = 0; d < 3; ++d) a[d] = d < LT::D ? decode<ST>(src[(long long)(LT::Q + d) * P + k], qs, 0) : T(0);
#pragma unroll
            for (int i = 0; i < LT::Q; ++i) {
                T h = decode<ST>(src[(long long)i * P + k], qs, i);
                if (i > 0) h += ref_value<LT>(i, a);
                acc[i] += double(h);
            }
        } else {
#pragma unroll
            for (int i = 0; i < LT::Q; ++i) acc[i] += double(decode<ST>(src[(long long)i * P + k], qs, i));
        }
        ++n;
    }
    v[0] = double(n) * rho0;
#pragma unroll
    for (int i = 0; i < LT::Q; ++i) {
        const double gsum = weight<LT>(i) * acc[i];  // stored values are scaled by 1/w_i
        v[0] += gsum;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const int c = vel<LT>(i, a);
            if (c == 1) v[1 + a] += gsum;
            else if (c == -1) v[1 + a] -= gsum;
            else if (c != 0) v[1 + a] += double(c) * gsum;
        }
    }
    block_reduce_store<4>(v, partials);
}

template <class LT, class ST>
cudaError_t launch_conservation(const ReduceArgs &a, cudaStream_t stream) {
    conservation_kernel<LT, ST><<<a.blocks, kReduceThreads, 0, stream>>>(static_cast<const typename ST::S *>(a.src),
                                                                         a.P, a.rho0, a.qs, a.partials, a.status);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    final_reduce_kernel<4><<<1, 4 * 32, 0, stream>>>(a.partials, a.blocks, a.out);
    return cudaGetLastError();
}

// Fourier amplitude of u_comp at wave vector k (FP64, pulled moments per cell).
template <class LT, class ST>
__global__ void __launch_bounds__(kReduceThreads) mode_kernel(const typename ST::S *__restrict__ src, int nx, int ny,
                                                              int nz, long long P, double rho0, int kx, int ky,
                                                              int kz, int comp, QScale qs,
                                                              double *__restrict__ partials,
                                                              unsigned int *__restrict__ status) {
    double v[2] = {0.0, 0.0};
    const long long per = (P + gridDim.x - 1) / gridDim.x;
    const long long b0 = blockIdx.x * per;
    const long long b1 = b0 + per < P ? b0 + per : P;
    for (long long cell = b0 + threadIdx.x; cell < b1; cell += blockDim.x) {
        double gt[LT::Q];
        pull_cell<LT, ST>(src, cell, nx, ny, nz, P, qs, gt, status, nx);
        double dr = 0.0, j[3] = {0.0, 0.0, 0.0};
#pragma unroll
        for (int i = 0; i < LT::Q; ++i) {
            dr += gt[i];
#pragma unroll
            for (int a = 0; a < 3; ++a) j[a] += double(vel<LT>(i, a)) * gt[i];
        }
        const double uc = (comp == 0 ? j[0] : (comp == 1 ? j[1] : j[2])) / (rho0 + dr);
        const int x = int(cell % nx);
        const int y = int((cell / nx) % ny);
        const int z = int(cell / ((long long)nx * ny));
        // phase / pi = 2 (kx x/nx + ky y/ny + kz z/nz), reduced modulo 2 before sincospi
        double ph = 2.0 * ((double)((long long)kx * x % nx) / nx + (double)((long long)ky * y % ny) / ny +
                           (double)((long long)kz * z % nz) / nz);
        double sn, cs;
        sincospi(ph, &sn, &cs);
        v[0] += uc * cs;
        v[1] -= uc * sn;
    }
    block_reduce_store<2>(v, partials);
}

template <class LT, class ST>
cudaError_t launch_mode(const ReduceArgs &a, cudaStream_t stream) {
    mode_kernel<LT, ST><<<a.blocks, kReduceThreads, 0, stream>>>(static_cast<const typename ST::S *>(a.src), a.nx,
                                                                 a.ny, a.nz, a.P, a.rho0, a.k[0], a.k[1], a.k[2],
                                                                 a.component, a.qs, a.partials, a.status);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    final_reduce_kernel<2><<<1, 2 * 32, 0, stream>>>(a.partials, a.blocks, a.out);
    return cudaGetLastError();
}

}  // namespace lbm

#include "lbm_batch_kernels.cuh"

namespace lbm {

// ------------------------------------------------------------------ kernel sets
template <class LT, int K, class ST, int V>
constexpr step_fn direct_if_built() {
    // Register budget: at most 160 stored values per thread (80 for FP64, whose
    // values take two registers); vectors of up to 32 bytes.
    if constexpr (int(sizeof(typename ST::S)) * V > 32) return nullptr;
    else if constexpr (LT::Q * V * (sizeof(typename ST::T) == 8 ? 2 : 1) > 160) return nullptr;
    else return &launch_step_direct<LT, K, ST, V>;
}

// FP64, fixed-point and reference-velocity storage run on the register pull only (no staged
// variant).
template <class ST>
constexpr bool register_pull_only() {
    return sizeof(typename ST::S) == 8 || ST::id == LBM_STORE_Q16 || RefOf<ST>::value;
}

template <class LT, int K, class ST>
constexpr step_fn staged_if_built() {
    if constexpr (register_pull_only<ST>()) return nullptr;
    else return &launch_step_staged<LT, K, ST>;
}

template <class LT, class ST>
constexpr bool (*staged_check_if_built())(int) {
    if constexpr (register_pull_only<ST>()) return nullptr;
    else return &staged_applies<LT, ST>;
}


template <class LT, int K, class ST>
constexpr step_fn theta_if_built() {
    if constexpr (K >= 3) return &launch_step_direct<LT, K, ST, 1, false, true>;
    else return nullptr;
}

template <class LT, int K, class ST>
const KernelSet *make_kernel_set();

// The fixed-point form's companion set with the reference shift (no batched step: pools run
// without one); null for the other forms.
template <class LT, int K, class ST>
const KernelSet *shifted_set_if_built() {
    if constexpr (ST::id == LBM_STORE_Q16 && !ShiftedOf<ST>::value) return make_kernel_set<LT, K, StoreQ16S>();
    else return nullptr;
}

// Pools run neither the shifted fixed-point codec nor the reference-velocity forms.
template <class LT, int K, class ST>
constexpr batch_fn batch_if_built() {
    if constexpr (ShiftedOf<ST>::value || RefOf<ST>::value) return nullptr;
    else return &launch_batch<LT, K, ST>;
}

template <class LT, int K, class ST>
constexpr int (*batch_occupancy_if_built())(int, int) {
    if constexpr (ShiftedOf<ST>::value || RefOf<ST>::value) return nullptr;
    else return &batch_occupancy<LT, K, ST>;
}

// The flat-pair variant pulls with per-cell direct loads and has no reference planes.
template <class LT, int K, class ST>
constexpr step_fn pair_if_built() {
    if constexpr (RefOf<ST>::value) return nullptr;
    else return &launch_step_pair<LT, K, ST>;
}

template <class LT, int K, class ST>
const KernelSet *make_kernel_set() {
    static const KernelSet ks = {
        {direct_if_built<LT, K, ST, 1>(), direct_if_built<LT, K, ST, 2>(), direct_if_built<LT, K, ST, 4>(),
         direct_if_built<LT, K, ST, 8>()},
        staged_if_built<LT, K, ST>(),
        kStagedThreads,
        &launch_init<LT, K, ST>,
        &launch_moments<LT, ST>,
        &launch_pull_f<LT, ST>,
        &launch_conservation<LT, ST>,
        &launch_mode<LT, ST>,
        batch_if_built<LT, K, ST>(),
        batch_occupancy_if_built<LT, K, ST>(),
        &launch_step_direct<LT, K, ST, 1, true>,
        theta_if_built<LT, K, ST>(),
        staged_check_if_built<LT, ST>(),
        pair_if_built<LT, K, ST>(),
        shifted_set_if_built<LT, K, ST>(),
    };
    return &ks;
}

template <class LT, int K>
const KernelSet *kernel_set_for_storage(lbm_storage st) {
    switch (st) {
    case LBM_STORE_F32: return make_kernel_set<LT, K, StoreF32>();
    case LBM_STORE_F16: return make_kernel_set<LT, K, StoreF16>();
    case LBM_STORE_BF16: return make_kernel_set<LT, K, StoreBF16>();
    case LBM_STORE_F64: return make_kernel_set<LT, K, StoreF64>();
    case LBM_STORE_Q16: return make_kernel_set<LT, K, StoreQ16>();
    case LBM_STORE_F16_REF: return make_kernel_set<LT, K, StoreF16Ref>();
    case LBM_STORE_BF16_REF: return make_kernel_set<LT, K, StoreBF16Ref>();
    }
    return nullptr;
}

}  // namespace lbm
