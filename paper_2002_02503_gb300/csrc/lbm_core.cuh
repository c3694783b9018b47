// lbm_core.cuh -- per-cell arithmetic of the Galilean-invariant filtered
// collision (arXiv 2002.02503) and the storage codecs.
//
// Notation (lattice units): T0 lattice constant, xi = c/sqrt(T0), V = u/sqrt(T0).
//   s  = xi.V = c.u/T0          v2 = V.V = u.u/T0
//   A  = (c c/T0 - I) : Pi      B  = c.Pi.u/T0          R = u.Pi.u/T0
// The Hermite tensors enter only through full contractions, which reduce to
// scalars (the Appendix identity): H^(n)(xi):V^[n] = h_n with h_0 = 1, h_1 = s,
// h_{n+1} = s h_n - n v2 h_{n-1} (the scalar form of Eq. recurG).  With
// E_n = sum_{m<=n} h_m/m! (E_n = 0 for n < 0):
//   truncated Eq. hermite        f^eq_i  = w_i rho E_K
//   truncated Eq. hermite-coll   fhat_i  = w_i/(2 T0) [E_{K-2} A - 2 E_{K-3} B + E_{K-4} R]
// which for K = 2, 3, 4 are Eq. filter-Pi, Eq. filter-1st and Eq. filter-2nd.
// The post-collision value is Eq. lbe-reg: f'_i = f^eq_i + (1 - 1/tau) fhat_i.
//
// Shifted, scaled storage: every kernel works with h_i = (g_i - w_i rho0) / w_i, so that
//   rho - rho0 = sum w h,   rho u = sum w c h   (sum_i w_i c_i = 0),
//   Pi = sum w c c h - T0 (rho - rho0) I - rho u u   (sum_i w_i c_i c_i = T0 I),
// and the output is (f^eq - w rho0)/w = (rho - rho0) + rho (E_K - 1) plus the
// filtered part over w: no large constant is ever added and then subtracted, and
// every weight multiplies only inside the moment sums.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include "lbm_internal.h"
#include "lbm_lattice.cuh"

namespace lbm {

// ------------------------------------------------------------------ codecs
// Every storage form holds the scaled shifted value h_i = (g_i - w_i rho0) / w_i:
// all velocities then share one magnitude range (the D3Q39 weights span 1/12 to
// 1/1620), and the collision below works on h directly, so neither decoding nor
// encoding multiplies by a weight.
//
// QScale (lbm_internal.h) carries the step 2^e of the fixed-point form
// (LBM_STORE_Q16); the floating forms ignore it.  A power-of-two step keeps both
// directions below exact apart from the one rounding of h to the grid.

struct StoreF32 {
    using S = float;
    using T = float;
    static constexpr lbm_storage id = LBM_STORE_F32;
    __device__ __forceinline__ static T dec(S v, const QScale &, int) { return v; }
    __device__ __forceinline__ static S enc(T x, const QScale &, int, unsigned int &) { return x; }
};
struct StoreF64 {
    using S = double;
    using T = double;
    static constexpr lbm_storage id = LBM_STORE_F64;
    __device__ __forceinline__ static T dec(S v, const QScale &, int) { return v; }
    __device__ __forceinline__ static S enc(T x, const QScale &, int, unsigned int &) { return x; }
};
struct StoreF16 {
    using S = __half;
    using T = float;
    static constexpr lbm_storage id = LBM_STORE_F16;
    __device__ __forceinline__ static T dec(S v, const QScale &, int) { return __half2float(v); }
    __device__ __forceinline__ static S enc(T x, const QScale &, int, unsigned int &) { return __float2half_rn(x); }
};
struct StoreBF16 {
    using S = __nv_bfloat16;
    using T = float;
    static constexpr lbm_storage id = LBM_STORE_BF16;
    __device__ __forceinline__ static T dec(S v, const QScale &, int) { return __bfloat162float(v); }
    __device__ __forceinline__ static S enc(T x, const QScale &, int, unsigned int &) {
        return __float2bfloat16_rn(x);
    }
};
// 16-bit fixed point: h = q 2^e with the integer q in [-32768, 32767], held in offset
// binary (q + 2^15).  Both directions use the FP32 adder's rounding at magnitude 2^23,
// where the spacing of floats is exactly 1:
//   encode  v = fma(h, 2^-e, 2^23 + 2^15) rounds h 2^-e to the nearest integer (ties to
//           even); for q in range v lies in [2^23, 2^23 + 65535], whose encodings are
//           exactly 0x4B00xxxx with q + 2^15 in the low 16 bits.  Any other v (out of
//           range, negative, not finite) has different upper 16 bits, so OR-ing
//           (bits ^ 0x4B000000) into an accumulator and testing its upper half once per
//           cell (range_exceeded) detects it at one logic operation per value;
//   decode  the bits 0x4B000000 | (q + 2^15) are the float 2^23 + 2^15 + q, and
//           fma(that, 2^e, -(2^23 + 2^15) 2^e) = q 2^e exactly.
// With a reference shift of k_i grid steps for velocity i (QScale), the stored code is
// q - k_i + 2^15: both constants carry -k_i, so the codec costs the same instructions.
template <bool SHIFT>
struct StoreQ16Codec {
    using S = unsigned short;
    using T = float;
    static constexpr lbm_storage id = LBM_STORE_Q16;
    static constexpr bool shifted = SHIFT;
    static constexpr float kBias = 8421376.0f;  // 2^23 + 2^15
    static constexpr unsigned int kExp = 0x4B000000u;
    // the FMA constants of velocity i: uniform without a reference shift (hoisted out of the
    // velocity loops), per velocity with one
    __device__ __forceinline__ static float dec_off(const QScale &q, int i) { return SHIFT ? q.dec[i] : q.off; }
    __device__ __forceinline__ static float enc_off(const QScale &q, int i) { return SHIFT ? q.enc[i] : kBias; }
    __device__ __forceinline__ static T dec(S v, const QScale &q, int i) {
        return fmaf(__uint_as_float(kExp | unsigned(v)), q.mul, dec_off(q, i));
    }
    __device__ __forceinline__ static S enc(T x, const QScale &q, int i, unsigned int &acc) {
        const unsigned int b = __float_as_uint(fmaf(x, q.inv, enc_off(q, i)));
        acc |= b ^ kExp;
        return static_cast<S>(b);
    }
};
using StoreQ16 = StoreQ16Codec<false>;
using StoreQ16S = StoreQ16Codec<true>;  // with the per-velocity reference shift

// True for the fixed-point codec with the reference shift.
template <class ST>
struct ShiftedOf {
    static constexpr bool value = false;
};
template <bool S>
struct ShiftedOf<StoreQ16Codec<S>> {
    static constexpr bool value = S;
};
// Per-cell reference velocity (LBM_STORE_F16_REF, LBM_STORE_BF16_REF): the base 16-bit codec,
// applied to the residual h_i - r_i with r_i = s + s^2 / 2, s = c_i . a, where a = u / T0 of the
// cell that wrote the value, rounded to the same 16-bit type and stored in D extra planes after
// the Q distribution planes.  A reader adds r_i of that cell back in FP32 (ref_value, the same
// operations on both sides), so only the residual is rounded.  For a flow of speed |u| the
// momentum part c_i . u / T0 of h_i is the largest term (about 0.15 at |u| = 0.05 on T0 = 1/3
// lattices) and its square the next; what is left (rho - rho0, rho |u|^2 / (2 T0), higher
// orders and the non-equilibrium part) is more than an order of magnitude smaller, and so is
// the rounding step of a 16-bit float.
template <class Base>
struct StoreRef : Base {
    static constexpr lbm_storage id = Base::id == LBM_STORE_F16 ? LBM_STORE_F16_REF : LBM_STORE_BF16_REF;
    static constexpr lbm_storage codec = Base::id;  // the element codec (vector conversions key on it)
};
using StoreF16Ref = StoreRef<StoreF16>;
using StoreBF16Ref = StoreRef<StoreBF16>;

// Element codec of a storage form (the form itself, or the base of a reference form).
template <class ST>
struct CodecOf {
    static constexpr lbm_storage value = ST::id;
};
template <class B>
struct CodecOf<StoreRef<B>> {
    static constexpr lbm_storage value = B::id;
};
// True for the forms with reference-velocity planes.
template <class ST>
struct RefOf {
    static constexpr bool value = false;
};
template <class B>
struct RefOf<StoreRef<B>> {
    static constexpr bool value = true;
};

// True when an encode since acc = 0 met a value outside the fixed-point range.
__device__ __forceinline__ bool range_exceeded(unsigned int acc) { return (acc >> 16) != 0u; }

// Vector decode / encode of V consecutive values of one velocity plane; the 16-bit
// floating forms convert two values per instruction (half2 / bfloat162).  encode_vec
// accumulates the fixed-point form's range check into acc (range_exceeded).
template <class ST, int V>
__device__ __forceinline__ void decode_vec(const typename ST::S (&raw)[V], typename ST::T (&out)[V],
                                           const QScale &q, int i) {
    if constexpr (CodecOf<ST>::value == LBM_STORE_F16 && V % 2 == 0) {
#pragma unroll
        for (int j = 0; j < V; j += 2) {
            const float2 f = __half22float2(__halves2half2(raw[j], raw[j + 1]));
            out[j] = f.x;
            out[j + 1] = f.y;
        }
    } else if constexpr (CodecOf<ST>::value == LBM_STORE_BF16 && V % 2 == 0) {
#pragma unroll
        for (int j = 0; j < V; j += 2) {
            const float2 f = __bfloat1622float2(__halves2bfloat162(raw[j], raw[j + 1]));
            out[j] = f.x;
            out[j + 1] = f.y;
        }
    } else if constexpr (ST::id == LBM_STORE_Q16 && V % 2 == 0) {
        // two codes per 32-bit word: one byte permute builds each float's bits, one paired
        // FMA scales both
        const float2 mul = make_float2(q.mul, q.mul), off = make_float2(ST::dec_off(q, i), ST::dec_off(q, i));
#pragma unroll
        for (int j = 0; j < V; j += 2) {
            const unsigned int w = unsigned(raw[j]) | (unsigned(raw[j + 1]) << 16);
            const float2 v = make_float2(__uint_as_float(__byte_perm(w, StoreQ16::kExp, 0x7610)),
                                         __uint_as_float(__byte_perm(w, StoreQ16::kExp, 0x7632)));
            const float2 h = __ffma2_rn(v, mul, off);
            out[j] = h.x;
            out[j + 1] = h.y;
        }
    } else {
#pragma unroll
        for (int j = 0; j < V; ++j) out[j] = ST::dec(raw[j], q, i);
    }
}

template <class ST, int V>
__device__ __forceinline__ void encode_vec(const typename ST::T (&in)[V], typename ST::S (&raw)[V],
                                           const QScale &q, int i, unsigned int &acc) {
    if constexpr (CodecOf<ST>::value == LBM_STORE_F16 && V % 2 == 0) {
#pragma unroll
        for (int j = 0; j < V; j += 2) {
            const __half2 h = __floats2half2_rn(in[j], in[j + 1]);
            raw[j] = __low2half(h);
            raw[j + 1] = __high2half(h);
        }
    } else if constexpr (CodecOf<ST>::value == LBM_STORE_BF16 && V % 2 == 0) {
#pragma unroll
        for (int j = 0; j < V; j += 2) {
            const __nv_bfloat162 h = __floats2bfloat162_rn(in[j], in[j + 1]);
            raw[j] = __low2bfloat16(h);
            raw[j + 1] = __high2bfloat16(h);
        }
    } else if constexpr (ST::id == LBM_STORE_Q16 && V % 2 == 0) {
        // one paired FMA encodes two values; the low halves of both encodings pack into one word
        const float2 inv = make_float2(q.inv, q.inv), bias = make_float2(ST::enc_off(q, i), ST::enc_off(q, i));
#pragma unroll
        for (int j = 0; j < V; j += 2) {
            const float2 v = __ffma2_rn(make_float2(in[j], in[j + 1]), inv, bias);
            const unsigned int b0 = __float_as_uint(v.x), b1 = __float_as_uint(v.y);
            acc |= (b0 ^ StoreQ16::kExp) | (b1 ^ StoreQ16::kExp);
            const unsigned int w = __byte_perm(b0, b1, 0x5410);
            raw[j] = static_cast<unsigned short>(w);
            raw[j + 1] = static_cast<unsigned short>(w >> 16);
        }
    } else {
#pragma unroll
        for (int j = 0; j < V; ++j) raw[j] = ST::enc(in[j], q, i, acc);
    }
}

// Scaled value h of one stored value of velocity i, and back.
template <class ST>
__device__ __forceinline__ typename ST::T decode(typename ST::S v, const QScale &q, int i) {
    return ST::dec(v, q, i);
}
template <class ST>
__device__ __forceinline__ typename ST::S encode(typename ST::T x, const QScale &q, int i, unsigned int &acc) {
    return ST::enc(x, q, i, acc);
}

// The codec constants of a grid step 2^e = mul with no reference shift (built in registers;
// with i known at compile time the arrays fold to constants).
__device__ __forceinline__ QScale qscale_plain(float mul, float inv) {
    QScale q;
    q.mul = mul;
    q.inv = inv;
    q.off = -StoreQ16::kBias * mul;
#pragma unroll
    for (int i = 0; i < kQMax; ++i) {
        q.enc[i] = StoreQ16::kBias;
        q.dec[i] = -StoreQ16::kBias * mul;
        q.ref[i] = 0.0f;
    }
    return q;
}

// ------------------------------------------------------------------ paired FP32
// F2 holds one FP32 value of each of two cells, and its arithmetic maps to the paired
// FP32 instructions of sm_100+ (two lanes per instruction, each rounded as the scalar
// operation).  The collision below is a template over its arithmetic type, so with
// T = F2 one pass of its code updates two cells.  A product stays unevaluated (F2P)
// until it meets an addition, so a*b + c issues one paired fused multiply-add, as the
// compiler's contraction does for scalars; a product used otherwise is rounded once.
struct F2P;
struct F2 {
    float2 v;
    F2() = default;
    __device__ __forceinline__ F2(float2 x) : v(x) {}
    __device__ __forceinline__ explicit F2(double c) : v(make_float2(float(c), float(c))) {}
    __device__ __forceinline__ F2(const F2P &p);
};
struct F2P {
    float2 a, b;
};
__device__ __forceinline__ float2 neg2(float2 x) { return make_float2(-x.x, -x.y); }
__device__ __forceinline__ F2::F2(const F2P &p) : v(__fmul2_rn(p.a, p.b)) {}
__device__ __forceinline__ F2P operator*(F2 x, F2 y) { return {x.v, y.v}; }
__device__ __forceinline__ F2P operator*(const F2P &p, F2 y) { return {F2(p).v, y.v}; }
__device__ __forceinline__ F2P operator*(F2 x, const F2P &p) { return {x.v, F2(p).v}; }
__device__ __forceinline__ F2P operator*(const F2P &p, const F2P &q) { return {F2(p).v, F2(q).v}; }
__device__ __forceinline__ F2 operator-(F2 x) { return F2(neg2(x.v)); }
__device__ __forceinline__ F2P operator-(const F2P &p) { return {neg2(p.a), p.b}; }
__device__ __forceinline__ F2 operator+(F2 x, F2 y) { return F2(__fadd2_rn(x.v, y.v)); }
__device__ __forceinline__ F2 operator-(F2 x, F2 y) { return F2(__fadd2_rn(x.v, neg2(y.v))); }
__device__ __forceinline__ F2 operator+(const F2P &p, F2 c) { return F2(__ffma2_rn(p.a, p.b, c.v)); }
__device__ __forceinline__ F2 operator+(F2 c, const F2P &p) { return F2(__ffma2_rn(p.a, p.b, c.v)); }
__device__ __forceinline__ F2 operator-(const F2P &p, F2 c) { return F2(__ffma2_rn(p.a, p.b, neg2(c.v))); }
__device__ __forceinline__ F2 operator-(F2 c, const F2P &p) { return F2(__ffma2_rn(neg2(p.a), p.b, c.v)); }
__device__ __forceinline__ F2 operator+(const F2P &p, const F2P &q) { return F2(__ffma2_rn(p.a, p.b, F2(q).v)); }
__device__ __forceinline__ F2 operator-(const F2P &p, const F2P &q) {
    return F2(__ffma2_rn(p.a, p.b, neg2(F2(q).v)));
}
__device__ __forceinline__ F2 operator/(F2 x, F2 y) { return F2(make_float2(x.v.x / y.v.x, x.v.y / y.v.y)); }
__device__ __forceinline__ F2 &operator+=(F2 &x, F2 y) { return x = x + y; }
__device__ __forceinline__ F2 &operator-=(F2 &x, F2 y) { return x = x - y; }
__device__ __forceinline__ F2 &operator+=(F2 &x, const F2P &p) { return x = x + p; }
__device__ __forceinline__ F2 &operator-=(F2 &x, const F2P &p) { return x = x - p; }

// ------------------------------------------------------------------ reference velocity
// r_i = s + s^2 / 2 with s = c_i . a, for velocity i of lattice LT and a the reference
// velocity over T0 of the cell that wrote the value (reference-velocity storage forms).  The
// writer subtracts it and the reader adds it back, each with this same sequence of
// correctly rounded operations (explicit intrinsics, so no contraction choice can differ
// between the two sides); on F2 each lane is rounded as the scalar operation, so one cell's
// r_i is the same bits on the scalar and the paired path.
__device__ __forceinline__ float ref_add(float s, int c, float a) {
    return c == 1 ? __fadd_rn(s, a) : (c == -1 ? __fsub_rn(s, a) : (c != 0 ? __fmaf_rn(float(c), a, s) : s));
}
__device__ __forceinline__ F2 ref_add(F2 s, int c, F2 a) {
    return c == 1 ? s + a : (c == -1 ? s - a : (c != 0 ? F2(double(c)) * a + s : s));
}
template <class LT, typename T>
__device__ __forceinline__ T ref_dot(int i, const T (&a)[3]) {
    T s = T(-0.0);
#pragma unroll
    for (int d = 0; d < LT::D; ++d) s = ref_add(s, vel<LT>(i, d), a[d]);
    return s;
}
__device__ __forceinline__ float ref_of_dot(float s) { return __fmaf_rn(s * 0.5f, s, s); }
__device__ __forceinline__ F2 ref_of_dot(F2 s) { return F2(s * F2(0.5)) * s + s; }
template <class LT, typename T>
__device__ __forceinline__ T ref_value(int i, const T (&a)[3]) {
    return ref_of_dot(ref_dot<LT>(i, a));
}
// r of the pair (+c_p, -c_p) at once: s_- = -s_+ exactly, so r_- = fma(s/2, s, -s) is the
// value ref_value gives for the -c_p velocity.
template <class LT, typename T>
__device__ __forceinline__ void ref_pair(int p, const T (&a)[3], T &r_plus, T &r_minus) {
    const T s = ref_dot<LT>(2 * p + 1, a);
    if constexpr (sizeof(T) == 4) {
        const float h = s * 0.5f;
        r_plus = __fmaf_rn(h, s, s);
        r_minus = __fmaf_rn(h, s, -s);
    } else {
        const F2 h = F2(s * F2(0.5));
        r_plus = h * s + s;
        r_minus = h * s - s;
    }
}

// ------------------------------------------------------------------ moments
// Accumulators start at -0.0: x + (-0.0) == x for every x, so the compiler drops
// the first addition (it cannot drop x + 0.0, which differs for x = -0.0).
template <typename T>
__device__ __forceinline__ constexpr T neg_zero() {
    return T(-0.0);
}

// c * v for a small integer constant c (no multiply for c = +-1).
template <typename T>
__device__ __forceinline__ void accumulate_scaled(T &acc, int c, T v) {
    if (c == 1) acc += v;
    else if (c == -1) acc -= v;
    else if (c != 0) acc += T(c) * v;
}

// ------------------------------------------------------------------ collision
// Scalar Hermite values h_2..h_K at (s, v2): h_{n+1} = s h_n - n v2 h_{n-1}.
// Only the orders that exist for this K are formed.
template <int K, typename T>
struct ScalarHermite {
    T h2, h3, h4, h5;
    __device__ __forceinline__ ScalarHermite(T s, T v2) {
        h2 = s * s - v2;
        if constexpr (K >= 3) h3 = s * (h2 - T(2) * v2);
        if constexpr (K >= 4) h4 = s * h3 - T(3) * v2 * h2;
        if constexpr (K >= 5) h5 = s * h4 - T(4) * v2 * h3;
    }
    // E_K - 1 split into even and odd parts (truncated Eq. hermite without its constant term)
    __device__ __forceinline__ T feq_even() const {
        if constexpr (K >= 4) return h2 * T(0.5) + h4 * T(1.0 / 24.0);
        else return h2 * T(0.5);
    }
    __device__ __forceinline__ T feq_odd(T s) const {
        if constexpr (K >= 5) return s + h3 * T(1.0 / 6.0) + h5 * T(1.0 / 120.0);
        else if constexpr (K >= 3) return s + h3 * T(1.0 / 6.0);
        else return s;
    }
};

// c * v as the first term of a sum (no addition; no multiply for c = +-1), else added to acc.
// `has` is known at compile time once the velocity loops are unrolled.
template <typename T>
__device__ __forceinline__ void add_term(T &acc, bool &has, int c, T v) {
    if (c == 0) return;
    if (has) {
        accumulate_scaled(acc, c, v);
    } else {
        acc = c == 1 ? v : (c == -1 ? -v : T(T(double(c)) * v));
        has = true;
    }
}

// The post-collision values of a velocity pair (+c_p, -c_p), Eq. lbe-reg in scaled shifted
// form, written as polynomials in s = c_p.u / T0 and q = s^2 whose coefficients depend on the
// cell only, so they are formed once per cell and each pair costs a few multiply-adds.  With
//   kappa = (1 - 1/tau) / (2 T0),  kt = kappa tr Pi,  a1 = 1 - v2/2  (v2 = u.u / T0),
//   Z  = c.(kappa Pi / T0).c = kappa A + kt,   B' = c.(-2 kappa Pi u / T0) = -2 kappa B,
// and the Hermite values of collide() in s and q,
//   h2 = q - v2,  h3 = s (q - 3 v2),  h4 = q^2 - 6 v2 q + 3 v2^2,  h5 = s (q^2 - 10 v2 q + 15 v2^2),
// the even part e and odd part o of drho + rho (E_K - 1) + kappa [bracket] collect to
//   K = 2:  e = E0 + Z + (rho/2) q,                                    o = rho s
//   K = 3:  e as K = 2,                                                o = s (O0 + Z + (rho/6) q) + B'
//   K = 4:  e = E0 + a1 Z + q (E1 + Z/2 + (rho/24) q) + B' s,          o as K = 3
//   K = 5:  e as K = 4,  o = s (O0 + a1 Z + q (O1 + Z/6 + (rho/120) q)) + B' (a1 + q/2)
// with the per-cell constants
//   K = 2, 3:  E0 = drho - (rho/2) v2 - kt,                    O0 = rho a1 - kt
//   K = 4, 5:  E0 = drho + rho (v2^2/8 - v2/2) + kappa R - kt a1,   E1 = rho (1/2 - v2/4) - kt/2
//   K = 4:     O0 = rho a1 - kt
//   K = 5:     O0 = rho (1 - v2/2 + v2^2/8) - kt a1 + kappa R,      O1 = rho (1/6 - v2/12) - kt/6.
// At s = 0 (the rest velocity, where A = -tr Pi and B = 0) the value is E0 for every K.
template <class LT, int K, typename T>
struct PairPoly {
    T us[3], Pk[3][3], Bk[3];
    T E0, E1, O0, O1, a1, rE, rO;
    __device__ __forceinline__ void init(T drho, T rho, const T (&us_)[3], const T (&P)[3][3], T v2, T trP,
                                         const T (&Pu)[3], T R, T kappa) {
        constexpr int D = LT::D;
        const T kP = kappa * T(1.0 / LT::T0);
#pragma unroll
        for (int a = 0; a < 3; ++a) us[a] = us_[a];
#pragma unroll
        for (int a = 0; a < D; ++a)
#pragma unroll
            for (int b = a; b < D; ++b) Pk[a][b] = kP * P[a][b];
        if constexpr (K >= 3) {
            const T m2k = kappa * T(-2.0);
#pragma unroll
            for (int a = 0; a < D; ++a) Bk[a] = m2k * Pu[a];
        }
        const T kt = kappa * trP;
        a1 = T(1) - v2 * T(0.5);
        if constexpr (K <= 3) {
            const T rh = rho * T(0.5);
            E0 = drho - rh * v2;
            E0 = E0 - kt;
            rE = rh;
            if constexpr (K == 2) {
                rO = rho;
            } else {
                O0 = rho * a1 - kt;
                rO = rho * T(1.0 / 6.0);
            }
        } else {
            const T c2 = v2 * T(0.125) - T(0.5);  // v2/8 - 1/2
            const T t = c2 * v2;
            E0 = drho + rho * t;
            E0 = E0 + kappa * R;
            E0 = E0 - kt * a1;
            const T c1 = T(0.5) - v2 * T(0.25);
            E1 = rho * c1 - kt * T(0.5);
            rE = rho * T(1.0 / 24.0);
            if constexpr (K == 4) {
                O0 = rho * a1 - kt;
                rO = rho * T(1.0 / 6.0);
            } else {
                const T c0 = c2 * v2 + T(1);  // 1 - v2/2 + v2^2/8
                O0 = rho * c0;
                O0 = O0 - kt * a1;
                O0 = O0 + kappa * R;
                const T c3 = T(1.0 / 6.0) - v2 * T(1.0 / 12.0);
                O1 = rho * c3 - kt * T(1.0 / 6.0);
                rO = rho * T(1.0 / 120.0);
            }
        }
    }
    __device__ __forceinline__ T rest() const { return E0; }
    // s = c_p.u / T0
    __device__ __forceinline__ T dot(int p) const {
        T s = neg_zero<T>();
        bool has = false;
#pragma unroll
        for (int a = 0; a < LT::D; ++a) add_term(s, has, LT::c(p, a), us[a]);
        return s;
    }
    // even and odd parts of the pair's values: g(+c_p) = e + o, g(-c_p) = e - o
    __device__ __forceinline__ void eo(int p, T s, T &e, T &o) const {
        constexpr int D = LT::D;
        T Z = neg_zero<T>(), B = neg_zero<T>();
        bool hz = false, hb = false;
#pragma unroll
        for (int a = 0; a < D; ++a) {
            const int ca = LT::c(p, a);
            if (ca == 0) continue;
            if constexpr (K >= 3) add_term(B, hb, ca, Bk[a]);
            add_term(Z, hz, ca * ca, Pk[a][a]);
#pragma unroll
            for (int b = a + 1; b < D; ++b) add_term(Z, hz, 2 * ca * LT::c(p, b), Pk[a][b]);
        }
        const T q = s * s;
        if constexpr (K <= 3) {
            const T ez = E0 + Z;
            e = ez + rE * q;
            if constexpr (K == 2) {
                o = rO * s;
            } else {
                const T oz = O0 + Z;
                const T y = oz + rO * q;
                o = s * y + B;
            }
        } else {
            const T t1 = E0 + a1 * Z;
            const T t2 = E1 + Z * T(0.5);
            const T t3 = t2 + rE * q;
            const T t4 = t1 + q * t3;
            e = t4 + B * s;
            if constexpr (K == 4) {
                const T oz = O0 + Z;
                const T y = oz + rO * q;
                o = s * y + B;
            } else {
                const T t5 = O0 + a1 * Z;
                const T t6 = O1 + Z * T(1.0 / 6.0);
                const T t7 = t6 + rO * q;
                const T t8 = t5 + q * t7;
                const T w = a1 + q * T(0.5);
                const T bw = B * w;
                o = s * t8 + bw;
            }
        }
    }
    __device__ __forceinline__ void pair(int p, T &gp, T &gm) const {
        T e, o;
        eo(p, dot(p), e, o);
        gp = e + o;
        gm = e - o;
    }
};

// The filtered collision in two parts.  Its output depends on the distributions only through
// drho = sum w h, j = sum w c h and sum w c c h (the moments), so a step may fold each value
// into MomentSums as it is pulled and drop it, and FilteredOutput forms each post-collision
// value from the moments just before it is stored.  The operations are those of collide()
// below (without the energy-flux term), in the same order.
template <class LT, typename T>
struct MomentSums {
    T drho, j[3], m2[3][3];
    __device__ __forceinline__ void start(T g0) {
        drho = T(LT::w0) * g0;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            j[a] = neg_zero<T>();
#pragma unroll
            for (int b = 0; b < 3; ++b) m2[a][b] = neg_zero<T>();
        }
    }
    // the values of velocity pair p: gp of +c_p, gm of -c_p
    __device__ __forceinline__ void add_pair(int p, T gp, T gm) {
        const T w = T(LT::w(p));
        const T sp = gp + gm;
        const T dp = gp - gm;
        drho += w * sp;
#pragma unroll
        for (int a = 0; a < LT::D; ++a) {
            const int ca = LT::c(p, a);
            if (ca != 0) j[a] += T(ca * LT::w(p)) * dp;
#pragma unroll
            for (int b = a; b < LT::D; ++b) {
                const int cab = ca * LT::c(p, b);
                if (cab != 0) m2[a][b] += T(cab * LT::w(p)) * sp;
            }
        }
    }
};

// Accumulate drho = sum w h, j = sum w c h, sum w c c h from scaled values h in
// pair order (each term is one fused multiply-add with a compile-time constant).
template <class LT, typename T>
__device__ __forceinline__ void accumulate_moments(const T (&g)[LT::Q], T &drho, T (&j)[3], T (&m2)[3][3]) {
    MomentSums<LT, T> ms;
    ms.start(g[0]);
#pragma unroll
    for (int p = 0; p < LT::NP; ++p) ms.add_pair(p, g[2 * p + 1], g[2 * p + 2]);
    drho = ms.drho;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        j[a] = ms.j[a];
#pragma unroll
        for (int b = 0; b < 3; ++b) m2[a][b] = ms.m2[a][b];
    }
}

// Post-collision values (Eq. lbe-reg, scaled and shifted) from the moments: rest() for the rest
// velocity, pair(p) for the pair (+c_p, -c_p).  See collide() for the notation.
template <class LT, int K, typename T>
struct FilteredOutput {
    PairPoly<LT, K, T> poly;
    FilteredOutput() = default;
    __device__ __forceinline__ FilteredOutput(const MomentSums<LT, T> &m, T relax, T rho0, T *us_out = nullptr) {
        init(m, relax, rho0, us_out);
    }
    // us_out, when given, receives u / T0
    __device__ __forceinline__ void init(const MomentSums<LT, T> &m, T relax, T rho0, T *us_out = nullptr) {
        constexpr int D = LT::D;
        const T iT0 = T(1.0 / LT::T0);
        const T T0 = T(LT::T0);
        const T drho = m.drho;
        const T rho = rho0 + drho;
        const T irho = T(1) / rho;
        T u[3], us[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) us[a] = T(0);
#pragma unroll
        for (int a = 0; a < D; ++a) {
            u[a] = m.j[a] * irho;
            us[a] = u[a] * iT0;
            if (us_out) us_out[a] = us[a];
        }
        // Pi^neq = sum c c g~ - T0 drho I - j u  (Eq. coeff-2; equal to Eq. Pi_def)
        T P[3][3];
#pragma unroll
        for (int a = 0; a < D; ++a)
#pragma unroll
            for (int b = a; b < D; ++b) {
                T v = m.m2[a][b] - m.j[a] * u[b];
                if (a == b) v -= T0 * drho;
                P[a][b] = v;
                P[b][a] = v;
            }
        T v2 = neg_zero<T>(), trP = neg_zero<T>();
#pragma unroll
        for (int a = 0; a < D; ++a) {
            v2 += u[a] * us[a];  // u.u / T0
            trP += P[a][a];
        }
        T Pu[3] = {neg_zero<T>(), neg_zero<T>(), neg_zero<T>()};  // Pi u / T0
        T R = neg_zero<T>();                                      // u.Pi.u / T0
        if constexpr (K >= 3) {
#pragma unroll
            for (int a = 0; a < D; ++a)
#pragma unroll
                for (int b = 0; b < D; ++b) Pu[a] += P[a][b] * us[b];
        }
        if constexpr (K >= 4) {
#pragma unroll
            for (int a = 0; a < D; ++a) R += u[a] * Pu[a];
        }
        const T kappa = relax * T(1.0 / (2.0 * LT::T0));  // (1 - 1/tau) / (2 T0)
        poly.init(drho, rho, us, P, v2, trP, Pu, R, kappa);
    }
    __device__ __forceinline__ T rest() const { return poly.rest(); }
    __device__ __forceinline__ void pair(int p, T &gp, T &gm) const { poly.pair(p, gp, gm); }
};

// g: scaled shifted pre-collision values h = (f - w rho0)/w in pair order;
// overwritten with the scaled post-collision values of Eq. lbe-reg.
// relax = 1 - 1/tau.  Divided by w_i, the two parts read
//   (f^eq - w rho0)/w = drho + rho (E_K - 1)
//   fhat / w          = 1/(2 T0) [E_{K-2} A - 2 E_{K-3} B + E_{K-4} R]
// with the even/odd parts of E_n written out for K = 2..5 (E_n = 0 for n < 0); PairPoly
// forms them for each velocity pair as polynomials in s = c.u / T0 with per-cell coefficients.
// Energy-flux part (Eq. pq, theta != 0): the series of Eq. filter-Q truncated at the same
// K reduces, with Qt the relative-frame flux of Eq. Q_def and q_a = Qt_abb, to
//   fhat^q / w = 1/(6 T0^3) sum_{m=0}^{K-3} sum_k a_k h_{m-k}/(m-k)!
//   a_0 = Qt(c,c,c) - 3 T0 c.q,  a_1 = -3 (c.(Qt u).c - T0 u.q),  a_2 = 3 c.(Qt u u),
// a_0, a_2 odd and a_1 even under c -> -c.  Qt = sum w c c c (h - h^eq) - 3 sym(u Pi).
// kq = (1 - 1/tau) theta / (6 T0^3).
// us_out, when given, receives u / T0 (the collision conserves rho and u).
template <class LT, int K, typename T, bool THETA = false>
__device__ __forceinline__ void collide(T (&g)[LT::Q], T relax, T rho0, T kq = T(0), T *us_out = nullptr) {
    static_assert(K >= 2 && K <= 5, "truncation order");
    static_assert(!THETA || K >= 3, "the energy-flux series starts at Hermite order 3");
    constexpr int D = LT::D;
    const T iT0 = T(1.0 / LT::T0);
    const T T0 = T(LT::T0);
    T drho, j[3], m2[3][3];
    accumulate_moments<LT, T>(g, drho, j, m2);
    const T rho = rho0 + drho;
    const T irho = T(1) / rho;
    T u[3], us[3];  // u and u / T0
#pragma unroll
    for (int a = 0; a < D; ++a) {
        u[a] = j[a] * irho;
        us[a] = u[a] * iT0;
        if (us_out) us_out[a] = us[a];
    }
    // Pi^neq = sum c c g~ - T0 drho I - j u  (Eq. coeff-2; equal to Eq. Pi_def)
    T P[3][3];
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
        for (int b = a; b < D; ++b) {
            T v = m2[a][b] - j[a] * u[b];
            if (a == b) v -= T0 * drho;
            P[a][b] = v;
            P[b][a] = v;
        }
    T v2 = neg_zero<T>(), trP = neg_zero<T>();
#pragma unroll
    for (int a = 0; a < D; ++a) {
        v2 += u[a] * us[a];  // u.u / T0
        trP += P[a][a];
    }
    T Pu[3] = {neg_zero<T>(), neg_zero<T>(), neg_zero<T>()};  // Pi u / T0
    T R = neg_zero<T>();                                      // u.Pi.u / T0
    if constexpr (K >= 3) {
#pragma unroll
        for (int a = 0; a < D; ++a)
#pragma unroll
            for (int b = 0; b < D; ++b) Pu[a] += P[a][b] * us[b];
    }
    if constexpr (K >= 4) {
#pragma unroll
        for (int a = 0; a < D; ++a) R += u[a] * Pu[a];
    }
    const T kappa = relax * T(1.0 / (2.0 * LT::T0));  // (1 - 1/tau) / (2 T0)
    PairPoly<LT, K, T> poly;
    poly.init(drho, rho, us, P, v2, trP, Pu, R, kappa);

    // energy flux: Qt (symmetric, stored for a <= b <= c), q, Qt u (symmetric), Qt u u
    T Qt[3][3][3], q[3], Qu[3][3], Quu[3];
    T uq = T(0);
    if constexpr (THETA) {
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b)
#pragma unroll
                for (int c = 0; c < 3; ++c) Qt[a][b][c] = neg_zero<T>();
        // 2 rho feq_odd(s) = s y(q): y = 2 rho (1 - v2/2 + q/6) for K = 3, 4 and
        // 2 rho (1 - v2/2 + v2^2/8 + q (1/6 - v2/12) + q^2/120) for K = 5 (q = s^2)
        const T r2 = rho * T(2);
        T f0, f1, f2;
        if constexpr (K <= 4) {
            f0 = r2 * poly.a1;
            f1 = rho * T(1.0 / 3.0);
        } else {
            const T c0 = v2 * (v2 * T(0.125) - T(0.5)) + T(1);
            f0 = r2 * c0;
            const T c1 = T(1.0 / 6.0) - v2 * T(1.0 / 12.0);
            f1 = r2 * c1;
            f2 = rho * T(1.0 / 60.0);
        }
#pragma unroll
        for (int p = 0; p < LT::NP; ++p) {
            const T s = poly.dot(p);
            const T qq = s * s;
            T y;
            if constexpr (K <= 4) {
                y = f0 + f1 * qq;
            } else {
                const T y1 = f1 + f2 * qq;
                y = f0 + qq * y1;
            }
            const T d = (g[2 * p + 1] - g[2 * p + 2]) - s * y;  // odd part of h - h^eq
#pragma unroll
            for (int a = 0; a < D; ++a)
#pragma unroll
                for (int b = a; b < D; ++b)
#pragma unroll
                    for (int c = b; c < D; ++c) {
                        const int cabc = LT::c(p, a) * LT::c(p, b) * LT::c(p, c);
                        if (cabc != 0) Qt[a][b][c] += T(cabc * LT::w(p)) * d;
                    }
        }
#pragma unroll
        for (int a = 0; a < D; ++a)
#pragma unroll
            for (int b = a; b < D; ++b)
#pragma unroll
                for (int c = b; c < D; ++c) {
                    const T v = Qt[a][b][c] - (u[a] * P[b][c] + u[b] * P[a][c] + u[c] * P[a][b]);
                    Qt[a][b][c] = v;  // fill every permutation of (a, b, c)
                    Qt[a][c][b] = v;
                    Qt[b][a][c] = v;
                    Qt[b][c][a] = v;
                    Qt[c][a][b] = v;
                    Qt[c][b][a] = v;
                }
#pragma unroll
        for (int a = 0; a < D; ++a) {
            q[a] = neg_zero<T>();
            Quu[a] = neg_zero<T>();
#pragma unroll
            for (int b = 0; b < D; ++b) q[a] += Qt[a][b][b];
#pragma unroll
            for (int b = a; b < D; ++b) {
                T v = neg_zero<T>();
#pragma unroll
                for (int c = 0; c < D; ++c) v += Qt[a][b][c] * u[c];
                Qu[a][b] = v;
                Qu[b][a] = v;
            }
        }
#pragma unroll
        for (int a = 0; a < D; ++a) {
#pragma unroll
            for (int b = 0; b < D; ++b) Quu[a] += Qu[a][b] * u[b];
            uq += u[a] * q[a];
        }
    }

    g[0] = poly.rest();
    // energy flux at c = 0: a_0 = a_2 = 0, a_1 = 3 T0 u.q enters from K = 4 on
    if constexpr (THETA && K >= 4) g[0] += kq * T(3.0 * LT::T0) * uq;
#pragma unroll
    for (int p = 0; p < LT::NP; ++p) {
        const T s = poly.dot(p);
        T e, o;
        poly.eo(p, s, e, o);
        if constexpr (THETA) {
            // c.Qt.c.c and c.(Qt u).c over the distinct components of the symmetric tensors
            // (a <= b <= c), each with its number of index orders
            T Qccc = neg_zero<T>(), cq = neg_zero<T>(), cQuc = neg_zero<T>(), cQuu = neg_zero<T>();
            bool h0 = false, h1 = false, h2 = false, h3 = false;
#pragma unroll
            for (int a = 0; a < D; ++a) {
                const int ca = LT::c(p, a);
                if (ca == 0) continue;
                add_term(cq, h1, ca, q[a]);
                add_term(cQuu, h3, ca, Quu[a]);
#pragma unroll
                for (int b = a; b < D; ++b) {
                    const int cb = LT::c(p, b);
                    if (cb == 0) continue;
                    add_term(cQuc, h2, (a == b ? 1 : 2) * ca * cb, Qu[a][b]);
#pragma unroll
                    for (int c = b; c < D; ++c) {
                        const int cc = LT::c(p, c);
                        const int orders = (a == b && b == c) ? 1 : ((a == b || b == c) ? 3 : 6);
                        if (cc != 0) add_term(Qccc, h0, orders * ca * cb * cc, Qt[a][b][c]);
                    }
                }
            }
            const T a0 = Qccc - T(3.0 * LT::T0) * cq;
            const T a1 = T(-3) * (cQuc - T(LT::T0) * uq);
            T q_odd = a0, q_even = T(0);
            if constexpr (K >= 4) q_even = a0 * s + a1;
            if constexpr (K >= 5) {
                const T e2 = poly.a1 + T(s * s) * T(0.5);  // 1 + h2/2
                q_odd = a0 * e2 + a1 * s + T(3) * cQuu;
            }
            if constexpr (K >= 4) e += kq * q_even;
            o += kq * q_odd;
        }
        g[2 * p + 1] = e + o;
        g[2 * p + 2] = e - o;
    }
}

// Scaled shifted equilibrium (f^eq_K(rho, u) - w rho0) / w for every velocity (set_fields).
template <class LT, int K, typename T>
__device__ __forceinline__ void equilibrium_shifted(T rho, T drho, const T (&u)[3], T (&g)[LT::Q]) {
    constexpr int D = LT::D;
    const T iT0 = T(1.0 / LT::T0);
    T us[3] = {T(0), T(0), T(0)};
    T v2 = neg_zero<T>();
#pragma unroll
    for (int a = 0; a < D; ++a) {
        us[a] = u[a] * iT0;
        v2 += u[a] * us[a];
    }
    {
        T e = -v2 * T(0.5);
        if constexpr (K >= 4) e += v2 * v2 * T(3.0 / 24.0);
        g[0] = drho + rho * e;
    }
#pragma unroll
    for (int p = 0; p < LT::NP; ++p) {
        T s = neg_zero<T>();
#pragma unroll
        for (int a = 0; a < D; ++a) accumulate_scaled(s, LT::c(p, a), us[a]);
        const ScalarHermite<K, T> H(s, v2);
        const T feq_e = drho + rho * H.feq_even();
        const T feq_o = rho * H.feq_odd(s);
        g[2 * p + 1] = feq_e + feq_o;
        g[2 * p + 2] = feq_e - feq_o;
    }
}

// The BGK operator of Eq. BGK with the same truncated equilibrium, in scaled
// variables: h' = h^eq + (1 - 1/tau)(h - h^eq).  A comparison baseline: it relaxes
// every non-equilibrium moment, including those the lattice does not support.
template <class LT, int K, typename T>
__device__ __forceinline__ void collide_bgk(T (&g)[LT::Q], T relax, T rho0, T *us_out = nullptr) {
    constexpr int D = LT::D;
    T drho, j[3], m2[3][3];
    accumulate_moments<LT, T>(g, drho, j, m2);
    const T rho = rho0 + drho;
    const T irho = T(1) / rho;
    T u[3] = {T(0), T(0), T(0)};
#pragma unroll
    for (int a = 0; a < D; ++a) {
        u[a] = j[a] * irho;
        if (us_out) us_out[a] = u[a] * T(1.0 / LT::T0);
    }
    T feq[LT::Q];
    equilibrium_shifted<LT, K, T>(rho, drho, u, feq);
#pragma unroll
    for (int i = 0; i < LT::Q; ++i) g[i] = feq[i] + relax * (g[i] - feq[i]);
}

}  // namespace lbm
