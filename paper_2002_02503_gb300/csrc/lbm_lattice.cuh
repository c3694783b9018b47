// lbm_lattice.cuh -- compile-time velocity sets for the CUDA kernels.
//
// Velocities are kept in pair order: index 0 is the rest velocity, pair p
// occupies indices 2p+1 (+c_p) and 2p+2 (-c_p).  Opposite velocities share the
// even and odd parts of the collision (c -> -c flips s = c.u/T0 and c.Pi.u, and
// keeps c.Pi.c), so a kernel evaluates the collision once per pair.
//
// The paper fixes T0 = 1/3 for D3Q15 and D3Q19 and the isotropy classes 2N (D2Q9,
// D3Q15 and D3Q19: 4, D3Q39: 6) in Sec. 2 after Eq. iso; the weights are the standard ones of each
// set (D3Q27 is not in the paper; its class is 4).  kmax = 2N - 1 is the highest
// Hermite order a truncation may keep (Sec. 2 and Sec. 3 truncation rule).
#pragma once

#include "../../include/lbm.h"

namespace lbm {

struct D2Q9 {
    static constexpr lbm_lattice id = LBM_D2Q9;
    static constexpr int D = 2, Q = 9, NP = 4, MAXC = 1, KMAX = 3;
    static constexpr double T0 = 1.0 / 3.0;
    static constexpr double w0 = 4.0 / 9.0;
    __host__ __device__ static constexpr int c(int p, int a) {
        constexpr int t[NP][3] = {{1, 0, 0}, {0, 1, 0}, {1, 1, 0}, {1, -1, 0}};
        return t[p][a];
    }
    __host__ __device__ static constexpr double w(int p) { return p < 2 ? 1.0 / 9.0 : 1.0 / 36.0; }
};

struct D3Q15 {
    static constexpr lbm_lattice id = LBM_D3Q15;
    static constexpr int D = 3, Q = 15, NP = 7, MAXC = 1, KMAX = 3;
    static constexpr double T0 = 1.0 / 3.0;
    static constexpr double w0 = 2.0 / 9.0;
    __host__ __device__ static constexpr int c(int p, int a) {
        constexpr int t[NP][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}, {1, 1, 1}, {1, 1, -1}, {1, -1, 1}, {1, -1, -1}};
        return t[p][a];
    }
    __host__ __device__ static constexpr double w(int p) { return p < 3 ? 1.0 / 9.0 : 1.0 / 72.0; }
};

struct D3Q19 {
    static constexpr lbm_lattice id = LBM_D3Q19;
    static constexpr int D = 3, Q = 19, NP = 9, MAXC = 1, KMAX = 3;
    static constexpr double T0 = 1.0 / 3.0;
    static constexpr double w0 = 1.0 / 3.0;
    __host__ __device__ static constexpr int c(int p, int a) {
        constexpr int t[NP][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}, {1, 1, 0}, {1, -1, 0},
                                  {1, 0, 1}, {1, 0, -1}, {0, 1, 1}, {0, 1, -1}};
        return t[p][a];
    }
    __host__ __device__ static constexpr double w(int p) { return p < 3 ? 1.0 / 18.0 : 1.0 / 36.0; }
};

struct D3Q27 {
    static constexpr lbm_lattice id = LBM_D3Q27;
    static constexpr int D = 3, Q = 27, NP = 13, MAXC = 1, KMAX = 3;
    static constexpr double T0 = 1.0 / 3.0;
    static constexpr double w0 = 8.0 / 27.0;
    __host__ __device__ static constexpr int c(int p, int a) {
        constexpr int t[NP][3] = {{1, 0, 0},  {0, 1, 0}, {0, 0, 1},  {1, 1, 0},  {1, -1, 0},
                                  {1, 0, 1},  {1, 0, -1}, {0, 1, 1}, {0, 1, -1}, {1, 1, 1},
                                  {1, 1, -1}, {1, -1, 1}, {1, -1, -1}};
        return t[p][a];
    }
    __host__ __device__ static constexpr double w(int p) {
        return p < 3 ? 2.0 / 27.0 : (p < 9 ? 1.0 / 54.0 : 1.0 / 216.0);
    }
};

struct D3Q39 {
    static constexpr lbm_lattice id = LBM_D3Q39;
    static constexpr int D = 3, Q = 39, NP = 19, MAXC = 3, KMAX = 5;
    static constexpr double T0 = 2.0 / 3.0;
    static constexpr double w0 = 1.0 / 12.0;
    __host__ __device__ static constexpr int c(int p, int a) {
        constexpr int t[NP][3] = {{1, 0, 0},  {0, 1, 0},  {0, 0, 1},                              // |c|^2 = 1
                                  {1, 1, 1},  {1, 1, -1}, {1, -1, 1}, {1, -1, -1},                // |c|^2 = 3
                                  {2, 0, 0},  {0, 2, 0},  {0, 0, 2},                              // |c|^2 = 4
                                  {2, 2, 0},  {2, -2, 0}, {2, 0, 2},  {2, 0, -2}, {0, 2, 2}, {0, 2, -2},  // 8
                                  {3, 0, 0},  {0, 3, 0},  {0, 0, 3}};                             // |c|^2 = 9
        return t[p][a];
    }
    __host__ __device__ static constexpr double w(int p) {
        return p < 3 ? 1.0 / 12.0
                     : (p < 7 ? 1.0 / 27.0 : (p < 10 ? 2.0 / 135.0 : (p < 16 ? 1.0 / 432.0 : 1.0 / 1620.0)));
    }
};

// Component a of velocity i in pair order.
template <class LT>
__host__ __device__ constexpr int vel(int i, int a) {
    return i == 0 ? 0 : ((i & 1) ? LT::c((i - 1) >> 1, a) : -LT::c((i - 1) >> 1, a));
}
// Runtime-index form (a small table in constant-folded code is not possible when i is not a
// compile-time constant): component a of velocity i.
template <class LT>
__device__ __forceinline__ int vel_rt(int i, int a) {
    if (i == 0) return 0;
    const int p = (i - 1) >> 1;
    int v = 0;
#pragma unroll
    for (int q = 0; q < LT::NP; ++q)
        if (q == p) v = LT::c(q, a);
    return (i & 1) ? v : -v;
}

template <class LT>
__host__ __device__ constexpr double weight(int i) {
    return i == 0 ? LT::w0 : LT::w((i - 1) >> 1);
}

}  // namespace lbm
