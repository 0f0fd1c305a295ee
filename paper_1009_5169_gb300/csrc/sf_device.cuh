// sf_device.cuh -- device-side types shared by the sm_103a kernels of the
// SF Wilson fermion library: complex arithmetic, the per-lattice descriptor,
// even/odd site decoding, spin projectors and the field layouts.
//
// Field layouts in HBM (structure of arrays, one plane per component):
//   FP64 spinor   double2 [rhs][12][Vpad]   component c = 3*spin + colour
//   FP32 spinor   float4  [rhs][6][Vpad]    float4 k holds components 2k, 2k+1
//   FP16 spinor   uint4   [rhs][3][Vpad]    8 halves = components 4k..4k+3,
//                 float   [rhs][Vpad]       times a per-(site, rhs) scale
//   FP64 links    double2 [mu][parity][9][Vpad]   complex 0..8 of the 3x3
//   FP32 links    float4  [mu][parity][3][Vpad]   rows 0, 1 (row 2 rebuilt)
//   FP16 links    uint2   [mu][parity][3][Vpad]   rows 0, 1 (row 2 rebuilt)
//   spatial links times the twist phase e^{i theta/L} (see LinkLoad)
// Sites of one parity are numbered in lexicographic order of the fermion
// lattice x0 = 1..T-1, x1..x3 = 0..L-1 (x3 fastest): cb = lex / 2 for even L.
// Batched vectors put lattice l's block at element offset soff_l * (planes
// per site) so one launch can walk several lattices of different sizes.
#pragma once
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace sf {

// ------------------------------------------------- programmatic launches
// The solver's kernels are launched with programmatic stream serialization:
// the next kernel of the stream may be scheduled while this one drains.
// Every such kernel first waits for its predecessor to complete and flush
// (griddepcontrol.wait; a no-op for a plain launch), then lets its own
// successor start launching.  The wait is the hardware's, no spin of ours.
__device__ __forceinline__ void pdl_enter() {
    asm volatile("griddepcontrol.wait;\n" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
}

// ------------------------------------------------------------- complex
template <typename R>
struct cpx {
    R re, im;
};

template <typename R>
__device__ __forceinline__ cpx<R> mk(R a, R b) { return cpx<R>{a, b}; }
template <typename R>
__device__ __forceinline__ cpx<R> operator+(cpx<R> a, cpx<R> b) { return {a.re + b.re, a.im + b.im}; }
template <typename R>
__device__ __forceinline__ cpx<R> operator-(cpx<R> a, cpx<R> b) { return {a.re - b.re, a.im - b.im}; }
template <typename R>
__device__ __forceinline__ cpx<R> operator-(cpx<R> a) { return {-a.re, -a.im}; }
template <typename R>
__device__ __forceinline__ cpx<R> operator*(cpx<R> a, cpx<R> b) {
    return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <typename R>
__device__ __forceinline__ cpx<R> operator*(R s, cpx<R> a) { return {s * a.re, s * a.im}; }
template <typename R>
__device__ __forceinline__ cpx<R> conj(cpx<R> a) { return {a.re, -a.im}; }
// conj(a) * b
template <typename R>
__device__ __forceinline__ cpx<R> cmulc(cpx<R> a, cpx<R> b) {
    return {a.re * b.re + a.im * b.im, a.re * b.im - a.im * b.re};
}
// i * a, -i * a
template <typename R>
__device__ __forceinline__ cpx<R> ti(cpx<R> a) { return {-a.im, a.re}; }
template <typename R>
__device__ __forceinline__ cpx<R> tmi(cpx<R> a) { return {a.im, -a.re}; }
// acc += a * b
template <typename R>
__device__ __forceinline__ void cfma(cpx<R>& acc, cpx<R> a, cpx<R> b) {
    acc.re = fma(a.re, b.re, acc.re);
    acc.re = fma(-a.im, b.im, acc.re);
    acc.im = fma(a.re, b.im, acc.im);
    acc.im = fma(a.im, b.re, acc.im);
}
// acc += conj(a) * b
template <typename R>
__device__ __forceinline__ void cfmac(cpx<R>& acc, cpx<R> a, cpx<R> b) {
    acc.re = fma(a.re, b.re, acc.re);
    acc.re = fma(a.im, b.im, acc.re);
    acc.im = fma(a.re, b.im, acc.im);
    acc.im = fma(-a.im, b.re, acc.im);
}

// ------------------------------------------------------ integer division
// q = (n * m) >> 40 with m = ceil(2^40 / d) is exact for n < 2^24 and
// d < 2^16 (the rounding error n (m - 2^40/d) / 2^40 < 2^-16 < 1/d).
struct FastDiv {
    uint32_t d;
    uint64_t m;
};
inline FastDiv make_fastdiv(uint32_t d) { return FastDiv{d, ((1ull << 40) + d - 1) / d}; }
__device__ __forceinline__ uint32_t fdiv(uint32_t n, const FastDiv& f) {
    return (uint32_t)(((uint64_t)n * f.m) >> 40);
}

// ------------------------------------------------------ lattice descriptor
struct LatDev {
    int L, T, Lh, Vh, Vpad;
    int L2, L3;
    FastDiv divLh, divL;
    double kappa;
    double ph_re, ph_im;          // lambda = e^{i theta / L}, folded into the stored spatial links
    double ph3_re, ph3_im;        // lambda^3 (third-row rebuild of the 12-real links)
    const double2* u64;           // [4][2][9][Vpad]  complex 0..8
    const float4* u32;            // [4][2][3][Vpad]  rows 0, 1
    const uint2* u16;             // [4][2][3][Vpad]  rows 0, 1 (halves)
    long long soff;               // batched-vector offset, in (site, rhs) units
    int blk0, nblk;               // blocks of this lattice in a launch
    int ntiles;                   // (T-1) x ceil(L3h / TS) tiles
    int L3h;                      // sites of one parity in a time slice, L^3 / 2
    FastDiv divTm1;               // division by T - 1
};

struct SiteX {
    int x0, x1, x2, x3;
    int lex;
};

// decode the checkerboard index cb of parity par
__device__ __forceinline__ SiteX decode_site(const LatDev& g, int cb, int par) {
    SiteX s;
    const uint32_t r = fdiv((uint32_t)cb, g.divLh);  // (x0-1) L^2 + x1 L + x2
    const int x3b = 2 * (cb - (int)r * g.Lh);
    const uint32_t q = fdiv(r, g.divL);
    s.x2 = (int)r - (int)q * g.L;
    const uint32_t t = fdiv(q, g.divL);
    s.x1 = (int)q - (int)t * g.L;
    s.x0 = (int)t + 1;
    const int b = (par + s.x0 + s.x1 + s.x2) & 1;
    s.x3 = x3b + b;
    s.lex = 2 * cb + b;
    return s;
}

// checkerboard index of the neighbour x +- mu (spatial wrap; the caller
// drops time hops that leave x0 = 1..T-1)
template <int MU, int DIR>
__device__ __forceinline__ int neighbour_cb(const LatDev& g, const SiteX& s) {
    int lex = s.lex;
    if (MU == 0) {
        lex += DIR * g.L3;
    } else {
        const int xc = (MU == 1) ? s.x1 : (MU == 2) ? s.x2 : s.x3;
        const int st = (MU == 1) ? g.L2 : (MU == 2) ? g.L : 1;
        if (DIR > 0) lex += (xc == g.L - 1) ? -(g.L - 1) * st : st;
        else lex += (xc == 0) ? (g.L - 1) * st : -st;
    }
    return lex >> 1;
}

// ------------------------------------------------------ spin projection
// Chiral basis: gamma_0 = [[0,1],[1,0]] (2x2 blocks), gamma_k off-diagonal
// with the signs of the documented basis; gamma_5 = diag(1,1,-1,-1).
// For P = 1 + S gamma_mu (S = +-1) the projected spinor is determined by two
// spin components h0 = psi0 + c0 psi_j0, h1 = psi1 + c1 psi_j1 and rows 2, 3
// are multiples of h0 / h1.
template <int MU, int S, typename R>
__device__ __forceinline__ void project(const cpx<R> (&p)[4][3], cpx<R> (&h)[2][3]) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (MU == 0) {
            if (S < 0) { h[0][a] = p[0][a] - p[2][a]; h[1][a] = p[1][a] - p[3][a]; }
            else       { h[0][a] = p[0][a] + p[2][a]; h[1][a] = p[1][a] + p[3][a]; }
        } else if (MU == 1) {
            if (S < 0) { h[0][a] = p[0][a] - ti(p[3][a]); h[1][a] = p[1][a] - ti(p[2][a]); }
            else       { h[0][a] = p[0][a] + ti(p[3][a]); h[1][a] = p[1][a] + ti(p[2][a]); }
        } else if (MU == 2) {
            if (S < 0) { h[0][a] = p[0][a] + p[3][a]; h[1][a] = p[1][a] - p[2][a]; }
            else       { h[0][a] = p[0][a] - p[3][a]; h[1][a] = p[1][a] + p[2][a]; }
        } else {
            if (S < 0) { h[0][a] = p[0][a] - ti(p[2][a]); h[1][a] = p[1][a] + ti(p[3][a]); }
            else       { h[0][a] = p[0][a] + ti(p[2][a]); h[1][a] = p[1][a] - ti(p[3][a]); }
        }
    }
}

// acc += P h, the four spin rows of the projected (and multiplied) spinor
template <int MU, int S, typename R>
__device__ __forceinline__ void expand_add(cpx<R> (&acc)[4][3], const cpx<R> (&u)[2][3]) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        acc[0][a] = acc[0][a] + u[0][a];
        acc[1][a] = acc[1][a] + u[1][a];
        if (MU == 0) {
            if (S < 0) { acc[2][a] = acc[2][a] - u[0][a]; acc[3][a] = acc[3][a] - u[1][a]; }
            else       { acc[2][a] = acc[2][a] + u[0][a]; acc[3][a] = acc[3][a] + u[1][a]; }
        } else if (MU == 1) {
            if (S < 0) { acc[2][a] = acc[2][a] + ti(u[1][a]); acc[3][a] = acc[3][a] + ti(u[0][a]); }
            else       { acc[2][a] = acc[2][a] + tmi(u[1][a]); acc[3][a] = acc[3][a] + tmi(u[0][a]); }
        } else if (MU == 2) {
            if (S < 0) { acc[2][a] = acc[2][a] - u[1][a]; acc[3][a] = acc[3][a] + u[0][a]; }
            else       { acc[2][a] = acc[2][a] + u[1][a]; acc[3][a] = acc[3][a] - u[0][a]; }
        } else {
            if (S < 0) { acc[2][a] = acc[2][a] + ti(u[0][a]); acc[3][a] = acc[3][a] + tmi(u[1][a]); }
            else       { acc[2][a] = acc[2][a] + tmi(u[0][a]); acc[3][a] = acc[3][a] + ti(u[1][a]); }
        }
    }
}

// acc += sc (the spin expansion of u): expand_add with the FP16 spinor scale
// applied in the sum, one FFMA per real component in place of the add (the
// loaded components are then used unscaled)
__device__ __forceinline__ void acc_fma(cpx<float>& a, const cpx<float>& u, float s) {
    a.re = fmaf(s, u.re, a.re);
    a.im = fmaf(s, u.im, a.im);
}
template <int MU, int S>
__device__ __forceinline__ void expand_fma(cpx<float> (&acc)[4][3], const cpx<float> (&u)[2][3], float sc) {
    const float nsc = -sc;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        acc_fma(acc[0][a], u[0][a], sc);
        acc_fma(acc[1][a], u[1][a], sc);
        if (MU == 0) {
            acc_fma(acc[2][a], u[0][a], S < 0 ? nsc : sc);
            acc_fma(acc[3][a], u[1][a], S < 0 ? nsc : sc);
        } else if (MU == 1) {
            acc_fma(acc[2][a], S < 0 ? ti(u[1][a]) : tmi(u[1][a]), sc);
            acc_fma(acc[3][a], S < 0 ? ti(u[0][a]) : tmi(u[0][a]), sc);
        } else if (MU == 2) {
            acc_fma(acc[2][a], u[1][a], S < 0 ? nsc : sc);
            acc_fma(acc[3][a], u[0][a], S < 0 ? sc : nsc);
        } else {
            acc_fma(acc[2][a], S < 0 ? ti(u[0][a]) : tmi(u[0][a]), sc);
            acc_fma(acc[3][a], S < 0 ? tmi(u[1][a]) : ti(u[1][a]), sc);
        }
    }
}

// ------------------------------------------------------ field access
// Precision tags: storage type of a spinor field and its arithmetic type.
struct P64 { using real = double; static constexpr int NC = 12; using vec = double2; };
struct P32 { using real = float;  static constexpr int NC = 6;  using vec = float4; };
struct P16 { using real = float;  static constexpr int NC = 3;  using vec = uint4; };

template <typename P>
struct Field {
    typename P::vec* v;   // planes
    float* scale;         // FP16 only
};

template <typename P>
struct CField {
    const typename P::vec* v;
    const float* scale;
};

__device__ __forceinline__ float2 h2f(uint32_t u) {
    __half2 h = *reinterpret_cast<__half2*>(&u);
    return __half22float2(h);
}
__device__ __forceinline__ uint32_t f2h(float a, float b) {
    __half2 h = __floats2half2_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&h);
}

// load the spinor of (site, rhs) of a lattice block starting at plane base
template <typename P, typename R>
__device__ __forceinline__ void load_spinor(const CField<P>& f, long long base, int Vpad, int site,
                                            long long sbase, cpx<R> (&p)[4][3]);

template <>
__device__ __forceinline__ void load_spinor<P64, double>(const CField<P64>& f, long long base, int Vpad,
                                                         int site, long long, cpx<double> (&p)[4][3]) {
#pragma unroll
    for (int c = 0; c < 12; ++c) {
        double2 v = __ldg(f.v + base + (long long)c * Vpad + site);
        p[c / 3][c % 3] = cpx<double>{v.x, v.y};
    }
}

template <>
__device__ __forceinline__ void load_spinor<P32, float>(const CField<P32>& f, long long base, int Vpad,
                                                        int site, long long, cpx<float> (&p)[4][3]) {
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        float4 v = __ldg(f.v + base + (long long)k * Vpad + site);
        p[(2 * k) / 3][(2 * k) % 3] = cpx<float>{v.x, v.y};
        p[(2 * k + 1) / 3][(2 * k + 1) % 3] = cpx<float>{v.z, v.w};
    }
}

template <>
__device__ __forceinline__ void load_spinor<P16, float>(const CField<P16>& f, long long base, int Vpad,
                                                        int site, long long sbase, cpx<float> (&p)[4][3]) {
    const float sc = __ldg(f.scale + sbase + site);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        uint4 v = __ldg(f.v + base + (long long)k * Vpad + site);
        float2 a = h2f(v.x), b = h2f(v.y), c = h2f(v.z), d = h2f(v.w);
        p[(4 * k) / 3][(4 * k) % 3] = cpx<float>{a.x * sc, a.y * sc};
        p[(4 * k + 1) / 3][(4 * k + 1) % 3] = cpx<float>{b.x * sc, b.y * sc};
        p[(4 * k + 2) / 3][(4 * k + 2) % 3] = cpx<float>{c.x * sc, c.y * sc};
        p[(4 * k + 3) / 3][(4 * k + 3) % 3] = cpx<float>{d.x * sc, d.y * sc};
    }
}

// ------------------------------------------------------ FP16 projection
// The spin projection h = p_a + c p_b (c = +1, -1, +i, -i; see project) of
// an FP16 spinor in FP32 arithmetic: the half q is converted (exactly) to
// FP32 and added to or subtracted from the half p by the mixed-precision
// add / sub of PTX (one f16 and one f32 source, f32 result), which rounds
// once.  h is bit for bit what converting both halves and adding in FP32
// gives, with one conversion fewer per component (measured: the FP16
// staged-link hop 4-5% faster at 32^4, 12% at 12^4).  p, q: (re, im) half
// pairs.
#define SF_PROJ_H16(OPRE, TRE, OPIM, TIM)                                                              \
    asm("{\n .reg .f16 pa, pb, qa, qb;\n .reg .f32 ta, tb;\n"                                          \
        " mov.b32 {pa, pb}, %2;\n mov.b32 {qa, qb}, %3;\n"                                             \
        " cvt.f32.f16 ta, qa;\n cvt.f32.f16 tb, qb;\n"                                                 \
        " " OPRE ".rn.f32.f16 %0, pa, " TRE ";\n " OPIM ".rn.f32.f16 %1, pb, " TIM ";\n}"             \
        : "=f"(r.re), "=f"(r.im) : "r"(p), "r"(q))
// C: 0 (+1), 1 (-1), 2 (+i), 3 (-i)
template <int C>
__device__ __forceinline__ cpx<float> proj_h16(uint32_t p, uint32_t q) {
    cpx<float> r;
    if (C == 0) SF_PROJ_H16("add", "ta", "add", "tb");
    else if (C == 1) SF_PROJ_H16("sub", "ta", "sub", "tb");
    else if (C == 2) SF_PROJ_H16("sub", "tb", "add", "ta");   // p + i q = (p.re - q.im, p.im + q.re)
    else SF_PROJ_H16("add", "tb", "sub", "ta");               // p - i q = (p.re + q.im, p.im - q.re)
    return r;
}
#undef SF_PROJ_H16

// The two spin components (b, coefficient) that project<MU, S> combines with
// spins 0 and 1: h0 = p0 + c0 p_j0, h1 = p1 + c1 p_j1.
template <int MU, int S> struct ProjPair;
template <int S> struct ProjPair<0, S> { static constexpr int j0 = 2, j1 = 3, c0 = S < 0 ? 1 : 0, c1 = S < 0 ? 1 : 0; };
template <int S> struct ProjPair<1, S> { static constexpr int j0 = 3, j1 = 2, c0 = S < 0 ? 3 : 2, c1 = S < 0 ? 3 : 2; };
template <int S> struct ProjPair<2, S> { static constexpr int j0 = 3, j1 = 2, c0 = S < 0 ? 0 : 1, c1 = S < 0 ? 1 : 0; };
template <int S> struct ProjPair<3, S> { static constexpr int j0 = 2, j1 = 3, c0 = S < 0 ? 3 : 2, c1 = S < 0 ? 2 : 3; };

// project<MU, S> of an FP16 spinor given as its 12 stored (re, im) half
// pairs w[3 spin + colour] (unscaled)
template <int MU, int S>
__device__ __forceinline__ void project_h16(const uint32_t (&w)[12], cpx<float> (&h)[2][3]) {
    using PP = ProjPair<MU, S>;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        h[0][a] = proj_h16<PP::c0>(w[a], w[3 * PP::j0 + a]);
        h[1][a] = proj_h16<PP::c1>(w[3 + a], w[3 * PP::j1 + a]);
    }
}

// the stored half pairs of the FP16 spinor of (site, rhs), without its scale
__device__ __forceinline__ void load_spinor_h16(const CField<P16>& f, long long base, int Vpad, int site,
                                                uint32_t (&w)[12]) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const uint4 v = __ldg(f.v + base + (long long)k * Vpad + site);
        w[4 * k] = v.x;
        w[4 * k + 1] = v.y;
        w[4 * k + 2] = v.z;
        w[4 * k + 3] = v.w;
    }
}

template <typename P, typename R>
__device__ __forceinline__ void store_spinor(const Field<P>& f, long long base, int Vpad, int site,
                                             long long sbase, const cpx<R> (&p)[4][3]);

template <>
__device__ __forceinline__ void store_spinor<P64, double>(const Field<P64>& f, long long base, int Vpad,
                                                          int site, long long, const cpx<double> (&p)[4][3]) {
#pragma unroll
    for (int c = 0; c < 12; ++c)
        f.v[base + (long long)c * Vpad + site] = make_double2(p[c / 3][c % 3].re, p[c / 3][c % 3].im);
}

template <>
__device__ __forceinline__ void store_spinor<P32, float>(const Field<P32>& f, long long base, int Vpad,
                                                         int site, long long, const cpx<float> (&p)[4][3]) {
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        const cpx<float> a = p[(2 * k) / 3][(2 * k) % 3], b = p[(2 * k + 1) / 3][(2 * k + 1) % 3];
        f.v[base + (long long)k * Vpad + site] = make_float4(a.re, a.im, b.re, b.im);
    }
}

template <>
__device__ __forceinline__ void store_spinor<P16, float>(const Field<P16>& f, long long base, int Vpad,
                                                         int site, long long sbase, const cpx<float> (&p)[4][3]) {
    float m = 0.f;
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int a = 0; a < 3; ++a) m = fmaxf(m, fmaxf(fabsf(p[s][a].re), fabsf(p[s][a].im)));
    const float inv = (m > 0.f) ? 1.0f / m : 0.f;
    f.scale[sbase + site] = m;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        cpx<float> c0 = p[(4 * k) / 3][(4 * k) % 3], c1 = p[(4 * k + 1) / 3][(4 * k + 1) % 3];
        cpx<float> c2 = p[(4 * k + 2) / 3][(4 * k + 2) % 3], c3 = p[(4 * k + 3) / 3][(4 * k + 3) % 3];
        uint4 v;
        v.x = f2h(c0.re * inv, c0.im * inv);
        v.y = f2h(c1.re * inv, c1.im * inv);
        v.z = f2h(c2.re * inv, c2.im * inv);
        v.w = f2h(c3.re * inv, c3.im * inv);
        f.v[base + (long long)k * Vpad + site] = v;
    }
}

// ------------------------------------------------------ links
// Links of a hop: U_mu(x) at the output site (forward) or U_mu(x - mu) at the
// neighbour (backward), both addressed by (mu, parity, cb).  The stored
// spatial links carry the twist phase: V_k(x) = e^{i theta/L} U_k(x), so the
// forward hop needs V_k(x) and the backward hop V_k(x-k)^dag with no further
// phase factor.  V_k is in U(3): FP64 stores all 18 reals, FP32/FP16 two
// rows and rebuild the third with the phase (rebuild_row2).
template <typename R>
struct Link {
    cpx<R> m[3][3];
};

template <typename P> struct LinkLoad;

template <>
struct LinkLoad<P64> {
    template <int MU>
    static __device__ __forceinline__ void load(const LatDev& g, int par, int cb, Link<double>& U) {
        const double2* b = g.u64 + ((long long)(MU * 2 + par) * 9) * g.Vpad + cb;
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            double2 v = __ldg(b + (long long)k * g.Vpad);
            U.m[k / 3][k % 3] = cpx<double>{v.x, v.y};
        }
    }
};

// FP32 and FP16 keep the first two rows only.  For V = lambda U with U in
// SU(3) the third row is lambda^3 conj(row0 x row1) (lambda = 1 in time).
template <int MU, typename R>
__device__ __forceinline__ void rebuild_row2(const LatDev& g, Link<R>& U) {
    cpx<R> c0 = conj(U.m[0][1] * U.m[1][2] - U.m[0][2] * U.m[1][1]);
    cpx<R> c1 = conj(U.m[0][2] * U.m[1][0] - U.m[0][0] * U.m[1][2]);
    cpx<R> c2 = conj(U.m[0][0] * U.m[1][1] - U.m[0][1] * U.m[1][0]);
    if (MU != 0) {
        const cpx<R> l3 = cpx<R>{(R)g.ph3_re, (R)g.ph3_im};
        c0 = l3 * c0;
        c1 = l3 * c1;
        c2 = l3 * c2;
    }
    U.m[2][0] = c0;
    U.m[2][1] = c1;
    U.m[2][2] = c2;
}

template <>
struct LinkLoad<P32> {
    template <int MU>
    static __device__ __forceinline__ void load(const LatDev& g, int par, int cb, Link<float>& U) {
        const float4* b = g.u32 + ((long long)(MU * 2 + par) * 3) * g.Vpad + cb;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            float4 v = __ldg(b + (long long)k * g.Vpad);
            U.m[(2 * k) / 3][(2 * k) % 3] = cpx<float>{v.x, v.y};
            U.m[(2 * k + 1) / 3][(2 * k + 1) % 3] = cpx<float>{v.z, v.w};
        }
        rebuild_row2<MU>(g, U);
    }
};

template <>
struct LinkLoad<P16> {
    template <int MU>
    static __device__ __forceinline__ void load(const LatDev& g, int par, int cb, Link<float>& U) {
        const uint2* b = g.u16 + ((long long)(MU * 2 + par) * 3) * g.Vpad + cb;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            uint2 v = __ldg(b + (long long)k * g.Vpad);
            const float2 a = h2f(v.x), c = h2f(v.y);
            U.m[(2 * k) / 3][(2 * k) % 3] = cpx<float>{a.x, a.y};
            U.m[(2 * k + 1) / 3][(2 * k + 1) % 3] = cpx<float>{c.x, c.y};
        }
        rebuild_row2<MU>(g, U);
    }
};

// u = U h (two colour vectors)
template <typename R>
__device__ __forceinline__ void mul_link(const Link<R>& U, const cpx<R> (&h)[2][3], cpx<R> (&u)[2][3]) {
#pragma unroll
    for (int k = 0; k < 2; ++k)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            cpx<R> t = U.m[a][0] * h[k][0];
            cfma(t, U.m[a][1], h[k][1]);
            cfma(t, U.m[a][2], h[k][2]);
            u[k][a] = t;
        }
}

// u = U^dag h
template <typename R>
__device__ __forceinline__ void mul_link_dag(const Link<R>& U, const cpx<R> (&h)[2][3], cpx<R> (&u)[2][3]) {
#pragma unroll
    for (int k = 0; k < 2; ++k)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            cpx<R> t = cmulc(U.m[0][a], h[k][0]);
            cfmac(t, U.m[1][a], h[k][1]);
            cfmac(t, U.m[2][a], h[k][2]);
            u[k][a] = t;
        }
}

// ------------------------------------------------------ block lookup
// The launch walks the lattices' blocks back to back; find this block's lattice.
__device__ __forceinline__ int find_lattice(const LatDev* __restrict__ lats, int nlat, int blk) {
    int l = 0;
    while (l + 1 < nlat && blk >= lats[l + 1].blk0) ++l;
    return l;
}

// Tiles are ordered time-slice fastest: tile t covers TS consecutive sites
// of one parity inside the time slice x0 = 1 + t % (T-1), spatial stretch
// t / (T-1).  A block owns a contiguous range of tiles, so it walks x0 over
// the same spatial stretch (the x0 +- 1 neighbour slices are reused from one
// step to the next) and all resident blocks sweep the same few time slices
// at once (the x1, x2, x3 neighbours are read by blocks running alongside).
__device__ __forceinline__ int tile_begin(const LatDev& g) {
    return (int)((long long)(blockIdx.x - g.blk0) * g.ntiles / g.nblk);
}
__device__ __forceinline__ int tile_end(const LatDev& g) {
    return (int)((long long)(blockIdx.x - g.blk0 + 1) * g.ntiles / g.nblk);
}
// checkerboard index of lane tx of tile t, or -1 past the end of its slice
__device__ __forceinline__ int tile_cb(const LatDev& g, int t, int tx) {
    const uint32_t sp = fdiv((uint32_t)t, g.divTm1);
    const int x0i = t - (int)sp * (g.T - 1);
    const int off = (int)sp * (int)blockDim.x + tx;
    if (off >= g.L3h) return -1;
    return x0i * g.L3h + off;
}

}  // namespace sf
