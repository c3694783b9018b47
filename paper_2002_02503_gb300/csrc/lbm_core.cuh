// lbm_core.cuh -- per-cell arithmetic of the Galilean-invariant filtered
// collision (arXiv 2002.02503) and the storage codecs.
//
// Notation (lattice units): T0 lattice constant, xi = c/sqrt(T0), V = u/sqrt(T0).
//   s  = xi.V = c.u/T0          v2 = V.V = u.u/T0
//   A  = (c c/T0 - I) : Pi      B  = c.Pi.u/T0          R = u.Pi.u/T0
// The Hermite tensors enter only through full contractions, which reduce to
// scalars: H^(n)(xi):V^[n] = h_n with h_0 = 1, h_1 = s, h_{n+1} = s h_n - n v2 h_{n-1}
// (the scalar form of Eq. recurG).  With E_n = sum_{m<=n} h_m/m! (E_n = 0 for n < 0):
//   truncated Eq. hermite        f^eq_i  = w_i rho E_K
//   truncated Eq. hermite-coll   fhat_i  = w_i/(2 T0) [E_{K-2} A - 2 E_{K-3} B + E_{K-4} R]
// which for K = 2, 3, 4 are Eq. filter-Pi, Eq. filter-1st and Eq. filter-2nd.
// The post-collision value is Eq. lbe-reg: f'_i = f^eq_i + (1 - 1/tau) fhat_i.
//
// Shifted storage: every kernel works with g~_i = g_i - w_i rho0, so that
//   rho - rho0 = sum g~_i,   rho u = sum c_i g~_i   (sum_i w_i c_i = 0),
//   Pi = sum c c g~ - T0 (rho - rho0) I - rho u u   (sum_i w_i c_i c_i = T0 I),
// and the output is f^eq - w rho0 = w (rho - rho0) + w rho (E_K - 1) plus the
// filtered part: no large constant is ever added and then subtracted.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include "lbm_lattice.cuh"

namespace lbm {

// ------------------------------------------------------------------ codecs
struct StoreF32 {
    using S = float;
    using T = float;
    static constexpr lbm_storage id = LBM_STORE_F32;
    __device__ __forceinline__ static T dec(S v, T) { return v; }
    __device__ __forceinline__ static S enc(T x, T) { return x; }
};
struct StoreF64 {
    using S = double;
    using T = double;
    static constexpr lbm_storage id = LBM_STORE_F64;
    __device__ __forceinline__ static T dec(S v, T) { return v; }
    __device__ __forceinline__ static S enc(T x, T) { return x; }
};
// 16-bit forms store g~_i / w_i (all velocities then share one magnitude range).
struct StoreF16 {
    using S = __half;
    using T = float;
    static constexpr lbm_storage id = LBM_STORE_F16;
    __device__ __forceinline__ static T dec(S v, T w) { return w * __half2float(v); }
    __device__ __forceinline__ static S enc(T x, T inv_w) { return __float2half_rn(x * inv_w); }
};
struct StoreBF16 {
    using S = __nv_bfloat16;
    using T = float;
    static constexpr lbm_storage id = LBM_STORE_BF16;
    __device__ __forceinline__ static T dec(S v, T w) { return w * __bfloat162float(v); }
    __device__ __forceinline__ static S enc(T x, T inv_w) { return __float2bfloat16_rn(x * inv_w); }
};

template <class ST, class LT>
__device__ __forceinline__ typename ST::T decode(typename ST::S v, int i) {
    return ST::dec(v, typename ST::T(weight<LT>(i)));
}
template <class ST, class LT>
__device__ __forceinline__ typename ST::S encode(typename ST::T x, int i) {
    return ST::enc(x, typename ST::T(1.0 / weight<LT>(i)));
}

// ------------------------------------------------------------------ Hermite sums
__host__ __device__ constexpr double inv_fact(int m) {
    double r = 1.0;
    for (int k = 2; k <= m; ++k) r /= k;
    return r;
}

// Even and odd parts (under c -> -c) of E_n = sum_{m<=n} h_m/m! for n = -1..K.
// ev[n+1], od[n+1] hold E_n's even / odd parts (index 0 is n = -1, all zero).
template <int K, typename T>
struct HermiteSums {
    T ev[K + 2], od[K + 2];
    __device__ __forceinline__ HermiteSums(T s, T v2) {
        T h[K + 1];
        h[0] = T(1);
        if (K >= 1) h[1] = s;
#pragma unroll
        for (int m = 1; m < K; ++m) h[m + 1] = s * h[m] - T(m) * v2 * h[m - 1];
        ev[0] = T(0);
        od[0] = T(0);
#pragma unroll
        for (int n = 0; n <= K; ++n) {
            T add = (n == 0) ? T(1) : h[n] * T(inv_fact(n));
            ev[n + 1] = ev[n] + ((n & 1) ? T(0) : add);
            od[n + 1] = od[n] + ((n & 1) ? add : T(0));
        }
    }
    __device__ __forceinline__ T E_even(int n) const { return n < 0 ? T(0) : ev[n + 1]; }
    __device__ __forceinline__ T E_odd(int n) const { return n < 0 ? T(0) : od[n + 1]; }
};

// Rest velocity (s = 0): h_m = He_m(0) |V|^m, only even m survive.
template <int K, typename T>
struct HermiteSumsRest {
    T ev[K + 2];
    __device__ __forceinline__ explicit HermiteSumsRest(T v2) {
        T h[K + 1];
        h[0] = T(1);
        if (K >= 1) h[1] = T(0);
#pragma unroll
        for (int m = 1; m < K; ++m) h[m + 1] = (m & 1) ? -T(m) * v2 * h[m - 1] : T(0);
        ev[0] = T(0);
#pragma unroll
        for (int n = 0; n <= K; ++n) ev[n + 1] = ev[n] + ((n & 1) ? T(0) : ((n == 0) ? T(1) : h[n] * T(inv_fact(n))));
    }
    __device__ __forceinline__ T E(int n) const { return n < 0 ? T(0) : ev[n + 1]; }
};

// ------------------------------------------------------------------ moments
template <class LT, typename T>
struct Moments {
    T drho, rho;
    T j[3], u[3];
    T m2[3][3];  // sum c c g~ (upper triangle used)
};

// Accumulate drho, j, sum c c g~ from shifted values in pair order.
template <class LT, typename T>
__device__ __forceinline__ void accumulate_moments(const T (&g)[LT::Q], T &drho, T (&j)[3], T (&m2)[3][3]) {
    drho = g[0];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        j[a] = T(0);
#pragma unroll
        for (int b = 0; b < 3; ++b) m2[a][b] = T(0);
    }
#pragma unroll
    for (int p = 0; p < LT::NP; ++p) {
        const T sp = g[2 * p + 1] + g[2 * p + 2];
        const T dp = g[2 * p + 1] - g[2 * p + 2];
        drho += sp;
#pragma unroll
        for (int a = 0; a < LT::D; ++a) {
            const int ca = LT::c(p, a);
            if (ca == 1) j[a] += dp;
            else if (ca == -1) j[a] -= dp;
            else if (ca != 0) j[a] += T(ca) * dp;
#pragma unroll
            for (int b = a; b < LT::D; ++b) {
                const int cab = ca * LT::c(p, b);
                if (cab == 1) m2[a][b] += sp;
                else if (cab == -1) m2[a][b] -= sp;
                else if (cab != 0) m2[a][b] += T(cab) * sp;
            }
        }
    }
}

// ------------------------------------------------------------------ collision
// g: shifted pre-collision values in pair order; overwritten with the shifted
// post-collision values of Eq. lbe-reg.  relax = 1 - 1/tau.
template <class LT, int K, typename T>
__device__ __forceinline__ void collide(T (&g)[LT::Q], T relax, T rho0) {
    constexpr int D = LT::D;
    const T iT0 = T(1.0 / LT::T0);
    const T T0 = T(LT::T0);
    T drho, j[3], m2[3][3];
    accumulate_moments<LT, T>(g, drho, j, m2);
    const T rho = rho0 + drho;
    const T irho = T(1) / rho;
    T u[3] = {T(0), T(0), T(0)};
#pragma unroll
    for (int a = 0; a < D; ++a) u[a] = j[a] * irho;
    // Pi^neq = sum c c g~ - T0 drho I - j u  (Eq. coeff-2; equal to Eq. Pi_def)
    T P[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) P[a][b] = T(0);
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
        for (int b = a; b < D; ++b) {
            T v = m2[a][b] - j[a] * u[b];
            if (a == b) v -= T0 * drho;
            P[a][b] = v;
            P[b][a] = v;
        }
    T v2 = T(0), trP = T(0);
#pragma unroll
    for (int a = 0; a < D; ++a) {
        v2 += u[a] * u[a];
        trP += P[a][a];
    }
    v2 *= iT0;
    T Pu[3] = {T(0), T(0), T(0)};
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
        for (int b = 0; b < D; ++b) Pu[a] += P[a][b] * u[b];
    T R = T(0);
#pragma unroll
    for (int a = 0; a < D; ++a) R += u[a] * Pu[a];
    R *= iT0;

    // rest velocity: A = -tr Pi, B = 0
    {
        HermiteSumsRest<K, T> H(v2);
        const T w = T(LT::w0);
        const T feq = w * drho + w * rho * (H.E(K) - T(1));
        const T fh = T(LT::w0 / (2.0 * LT::T0)) * (-trP * H.E(K - 2) + R * H.E(K - 4));
        g[0] = feq + relax * fh;
    }
#pragma unroll
    for (int p = 0; p < LT::NP; ++p) {
        T s = T(0), cPc = T(0), cPu = T(0);
#pragma unroll
        for (int a = 0; a < D; ++a) {
            const int ca = LT::c(p, a);
            if (ca == 0) continue;
            s += T(ca) * u[a];
            cPu += T(ca) * Pu[a];
#pragma unroll
            for (int b = 0; b < D; ++b) {
                const int cb = LT::c(p, b);
                if (cb == 0) continue;
                cPc += T(ca * cb) * P[a][b];
            }
        }
        s *= iT0;
        const T A = cPc * iT0 - trP;
        const T B = cPu * iT0;
        HermiteSums<K, T> H(s, v2);
        const T w = T(LT::w(p));
        const T wr = w * rho;
        const T feq_e = w * drho + wr * (H.E_even(K) - T(1));
        const T feq_o = wr * H.E_odd(K);
        const T cw = T(LT::w(p) / (2.0 * LT::T0));
        const T fh_e = cw * (A * H.E_even(K - 2) - T(2) * B * H.E_odd(K - 3) + R * H.E_even(K - 4));
        const T fh_o = cw * (A * H.E_odd(K - 2) - T(2) * B * H.E_even(K - 3) + R * H.E_odd(K - 4));
        g[2 * p + 1] = feq_e + feq_o + relax * (fh_e + fh_o);
        g[2 * p + 2] = feq_e - feq_o + relax * (fh_e - fh_o);
    }
}

// Shifted equilibrium f^eq_K(rho, u) - w rho0 for every velocity (set_fields).
template <class LT, int K, typename T>
__device__ __forceinline__ void equilibrium_shifted(T rho, T drho, const T (&u)[3], T (&g)[LT::Q]) {
    constexpr int D = LT::D;
    const T iT0 = T(1.0 / LT::T0);
    T v2 = T(0);
#pragma unroll
    for (int a = 0; a < D; ++a) v2 += u[a] * u[a];
    v2 *= iT0;
    {
        HermiteSumsRest<K, T> H(v2);
        const T w = T(LT::w0);
        g[0] = w * drho + w * rho * (H.E(K) - T(1));
    }
#pragma unroll
    for (int p = 0; p < LT::NP; ++p) {
        T s = T(0);
#pragma unroll
        for (int a = 0; a < D; ++a) s += T(LT::c(p, a)) * u[a];
        s *= iT0;
        HermiteSums<K, T> H(s, v2);
        const T w = T(LT::w(p));
        const T feq_e = w * drho + w * rho * (H.E_even(K) - T(1));
        const T feq_o = w * rho * H.E_odd(K);
        g[2 * p + 1] = feq_e + feq_o;
        g[2 * p + 2] = feq_e - feq_o;
    }
}

}  // namespace lbm
