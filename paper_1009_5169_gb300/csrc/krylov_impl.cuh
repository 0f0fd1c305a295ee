// krylov_impl.cuh -- the fused Dhat tail, the lattice reductions and the
// Krylov step kernels (BiCGStab, Alg. 1; CG on the normal equations; the
// defect-correction updates of Sec. 3.2), templated over field storage, and
// the KrylovOps table that sequences them.  Included by one translation unit
// per precision configuration (krylov_f64.cu, krylov_f32.cu, krylov_f16.cu).
//
// Even/odd preconditioning (Sec. 3.1) with the hop H of hop.cuh:
//   Dhat = 1 - kappa^2 H_eo H_oe,  Dhat^dag = gamma_5 Dhat gamma_5, where
//   gamma_5 H gamma_5 swaps the projectors (1 -+ gamma_mu).
// Each block owns a lattice's tiles of TS sites x (nrhs / NR) groups of NR
// right-hand sides.  Reductions are deterministic: a fixed shuffle tree per
// warp, a fixed sum over warps into per-block partials, and a fixed-order sum
// of the partials (k_finish).
#pragma once
#include <type_traits>

#include "hop.cuh"
#include "sf_kernels.h"

namespace sf {

// ------------------------------------------------------------ reductions
constexpr int MAX_WARPS = 32;
constexpr int MAX_RHS = 16;

// Reduction accumulators.  FP64 fields reduce in double.  The FP32 / FP16
// solver reduces in float-float (an unevaluated sum hi + lo of two floats,
// combined with Knuth's error-free TwoSum), about 44 significant bits: the
// FP64 pipe of this GPU retires a small fraction of the FP32 rate, and a
// double shuffle tree per warp would cost more than the kernel's memory
// traffic.  Results leave the reduction as double.
struct ff {
    float hi, lo;
};
__device__ __forceinline__ ff acc_add(ff a, ff b) {
    const float s = __fadd_rn(a.hi, b.hi);  // TwoSum: s + e = a.hi + b.hi exactly
    const float bv = __fsub_rn(s, a.hi);
    const float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bv)), __fsub_rn(b.hi, bv));
    const float lo = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
    const float h = __fadd_rn(s, lo);  // renormalise (FastTwoSum, |s| >= |lo|)
    return ff{h, __fsub_rn(lo, __fsub_rn(h, s))};
}
__device__ __forceinline__ double acc_add(double a, double b) { return a + b; }
__device__ __forceinline__ ff acc_shfl_down(ff v, int off) {
    return ff{__shfl_down_sync(0xffffffffu, v.hi, off), __shfl_down_sync(0xffffffffu, v.lo, off)};
}
__device__ __forceinline__ double acc_shfl_down(double v, int off) { return __shfl_down_sync(0xffffffffu, v, off); }
__device__ __forceinline__ double acc_to_double(ff v) { return (double)v.hi + (double)v.lo; }
__device__ __forceinline__ double acc_to_double(double v) { return v; }
__device__ __forceinline__ ff acc_ldcg(const ff* p) {
    const float2 v = __ldcg(reinterpret_cast<const float2*>(p));
    return ff{v.x, v.y};
}
__device__ __forceinline__ double acc_ldcg(const double* p) { return __ldcg(p); }
template <typename A> __device__ __forceinline__ A acc_zero() { return A{}; }
__device__ __forceinline__ void store_acc(ff* p, ff v) { *p = v; }
__device__ __forceinline__ void store_acc(double* p, double v) { *p = v; }
__device__ __forceinline__ void store_acc(double* p, ff v) { *p = acc_to_double(v); }
template <typename R> struct AccOf { using T = double; };
template <> struct AccOf<float> { using T = ff; };

// Per-block partial sums: vals[j][q] of every thread (rhs = threadIdx.y * NR
// + j) -> partials[(rhs * NQ + q) * gridDim.x + blockIdx.x], a fixed shuffle
// tree per warp and a fixed sum over the warps of a rhs group (the block's
// threads write the rhs x NQ sums in turn, so NQ may exceed a warp).  Every
// thread of the block calls it.  The lattice sums are formed by k_finish, launched
// next on the same stream: the kernel boundary orders the partials, where a
// last-block-done scheme inside the kernel pays device-scope fences on every
// block's critical path.
template <int NR, int NQ, typename A>
__device__ __forceinline__ void block_partials(const A (&vals)[NR][NQ], int nrhs, double* __restrict__ partials_) {
    static_assert(sizeof(A) == sizeof(double), "partials hold 8-byte accumulators");
    A* __restrict__ partials = reinterpret_cast<A*>(partials_);
    __shared__ A sw[MAX_WARPS][NR][NQ];
    const int lane = threadIdx.x & 31;
    const int wpr = blockDim.x >> 5;
    const int w = threadIdx.y * wpr + (threadIdx.x >> 5);
#pragma unroll
    for (int j = 0; j < NR; ++j)
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            A v = vals[j][q];
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) v = acc_add(v, acc_shfl_down(v, off));
            if (lane == 0) sw[w][j][q] = v;
        }
    __syncthreads();
    const int nt = blockDim.x * blockDim.y;
    for (int e = threadIdx.y * blockDim.x + threadIdx.x; e < (int)blockDim.y * NR * NQ; e += nt) {
        const int y = e / (NR * NQ), jq = e % (NR * NQ), j = jq / NQ, q = jq % NQ;
        const int rhs = y * NR + j;
        if (rhs < nrhs) {
            A s = acc_zero<A>();
            for (int k = 0; k < wpr; ++k) s = acc_add(s, sw[y * wpr + k][j][q]);
            partials[(long long)(rhs * NQ + q) * gridDim.x + blockIdx.x] = s;
        }
    }
}

// ------------------------------------------------------------ coefficients
// BiCGStab scalars alpha = rho / <r0, v>, omega = <t, s> / |t|^2,
// beta = (rho' / rho)(alpha / omega).  The FP64 solver forms them in double.
// The FP32 inner solver forms them in float from the double sums: they only
// scale FP32 vectors, and one thread's double complex divisions on this GPU's
// narrow FP64 pipe take microseconds per iteration.  KState keeps both forms.
__device__ __forceinline__ float2 f2of(double2 a) { return make_float2((float)a.x, (float)a.y); }
// a / b by Smith's scaled algorithm (no overflow of |b|^2)
__device__ __forceinline__ float2 cdivf(float2 a, float2 b) {
    if (fabsf(b.x) >= fabsf(b.y)) {
        const float r = b.y / b.x, d = b.x + r * b.y;
        return make_float2((a.x + r * a.y) / d, (a.y - r * a.x) / d);
    }
    const float r = b.x / b.y, d = b.y + r * b.x;
    return make_float2((a.x * r + a.y) / d, (a.y * r - a.x) / d);
}
__device__ __forceinline__ float2 cmulf(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 d2of(float2 a) { return make_double2((double)a.x, (double)a.y); }

template <typename RV> struct Coef;
template <>
struct Coef<double> {
    static __device__ __forceinline__ cpx<double> alpha(const KState& k) { return cpx<double>{k.alpha.x, k.alpha.y}; }
    static __device__ __forceinline__ cpx<double> omega(const KState& k) { return cpx<double>{k.omega.x, k.omega.y}; }
    static __device__ __forceinline__ cpx<double> beta(const KState& k) { return cpx<double>{k.beta.x, k.beta.y}; }
    static __device__ __forceinline__ void set_alpha(KState& k, double2 r0v) { k.alpha = cdiv(k.rho, r0v); }
    static __device__ __forceinline__ void set_omega(KState& k, double2 ts, double tt) {
        k.omega = make_double2(ts.x / tt, ts.y / tt);
    }
    static __device__ __forceinline__ void set_beta(KState& k, double2 rho_new) {
        k.beta = cmul(cdiv(rho_new, k.rho), cdiv(k.alpha, k.omega));
    }
};
template <>
struct Coef<float> {
    static __device__ __forceinline__ cpx<float> alpha(const KState& k) { return cpx<float>{k.alpha_f.x, k.alpha_f.y}; }
    static __device__ __forceinline__ cpx<float> omega(const KState& k) { return cpx<float>{k.omega_f.x, k.omega_f.y}; }
    static __device__ __forceinline__ cpx<float> beta(const KState& k) { return cpx<float>{k.beta_f.x, k.beta_f.y}; }
    static __device__ __forceinline__ void set_alpha(KState& k, double2 r0v) {
        k.alpha_f = cdivf(f2of(k.rho), f2of(r0v));
        k.alpha = d2of(k.alpha_f);
    }
    static __device__ __forceinline__ void set_omega(KState& k, double2 ts, double tt) {
        const float t = (float)tt;
        k.omega_f = make_float2((float)ts.x / t, (float)ts.y / t);
        k.omega = d2of(k.omega_f);
    }
    static __device__ __forceinline__ void set_beta(KState& k, double2 rho_new) {
        k.beta_f = cmulf(cdivf(f2of(rho_new), f2of(k.rho)), cdivf(k.alpha_f, k.omega_f));
        k.beta = d2of(k.beta_f);
    }
};

// What k_finish does with the lattice sums of a reduction.
enum FinMode {
    FIN_R0V = 0,   // alpha = rho / <r0, v>
    FIN_TS = 1,    // omega = <t, s> / |t|^2
    FIN_XR = 2,    // rho', |r|^2, beta, iteration count and convergence
    FIN_INIT = 3,  // inner-solve start from |b|^2
    FIN_NORM = 4,  // out[i] = sum
    FIN_DOT = 5,   // ((double2*) out)[i] = (re, im)
    FIN_INIT_CG = 7,   // CG start: gamma = |b|^2, iters = 0 (k_cg_tail's first step), active, target2
};
constexpr int FIN_THREADS = 512;

// The WHILE node of the iteration graph: continue while any rhs of any
// lattice is active and the device-side cap is not reached (one thread).
__device__ __forceinline__ void set_loop_cond(const SolverCtx& ctx, int nlat, int nrhs) {
    int any = 0;
    for (int i = 0; i < nlat * nrhs; ++i) any |= ctx.st[i].active;
    const int n = atomicAdd(ctx.loop_count, 1) + 1;
    ctx.loop_count[3] += 1;  // iterations of the whole solve (launch accounting)
    const int go = (any && n < ctx.loop_count[1]) ? 1 : 0;
    ctx.loop_count[2] = go;  // read by the host when the loop runs without a graph
    if (ctx.use_cond) cudaGraphSetConditional(ctx.cond, (unsigned)go);
}

// the per-rhs effect of a reduction's lattice sums sres
template <int MODE, typename RV>
__device__ __forceinline__ void fin_apply(const SolverCtx& ctx, int i, int tid, const double* sres,
                                          double* __restrict__ out, int maxiter) {
    if (MODE == FIN_NORM) {
        out[i] = sres[tid];
        return;
    }
    if (MODE == FIN_DOT) {
        reinterpret_cast<double2*>(out)[i] = make_double2(sres[2 * tid], sres[2 * tid + 1]);
        return;
    }
    if (ctx.st == nullptr) return;
    KState& st = ctx.st[i];
    if (MODE == FIN_INIT || MODE == FIN_INIT_CG) {
        const OState& o = ctx.ost[i];
        const float om = (MODE == FIN_INIT_CG) ? 0.f : 1.f;
        st.rho = make_double2(sres[tid], 0.0);
        st.rr = sres[tid];
        st.alpha = make_double2(1.0, 0.0);
        st.omega = make_double2((double)om, 0.0);
        st.beta = make_double2(0.0, 0.0);
        st.alpha_f = make_float2(1.f, 0.f);
        st.omega_f = make_float2(om, 0.f);
        st.beta_f = make_float2(0.f, 0.f);
        st.iters = 0;
        st.maxiter = maxiter;
        st.flags = 0;
        st.target2 = o.delta2;
        st.active = (o.active && sres[tid] > o.delta2) ? 1 : 0;
        return;
    }
    if (!st.active) return;
    if (MODE == FIN_R0V) {
        const double2 r0v = make_double2(sres[2 * tid], sres[2 * tid + 1]);
        if (r0v.x == 0.0 && r0v.y == 0.0) {
            st.active = 0;
            st.flags |= 1;
        } else {
            Coef<RV>::set_alpha(st, r0v);
        }
    } else if (MODE == FIN_TS) {
        const double2 ts = make_double2(sres[3 * tid], sres[3 * tid + 1]);
        const double tt = sres[3 * tid + 2];
        if (tt > 0.0) {
            Coef<RV>::set_omega(st, ts, tt);
        } else {
            st.omega = make_double2(0.0, 0.0);
            st.omega_f = make_float2(0.f, 0.f);
        }
    } else if (MODE == FIN_XR) {
        const double2 rho_new = make_double2(sres[3 * tid], sres[3 * tid + 1]);
        const double rr = sres[3 * tid + 2];
        st.rr = rr;
        st.iters += 1;
        const bool om0 = (st.omega.x == 0.0 && st.omega.y == 0.0);
        const bool rho0 = (rho_new.x == 0.0 && rho_new.y == 0.0);
        if (!om0 && !rho0) Coef<RV>::set_beta(st, rho_new);
        st.rho = rho_new;
        if (om0) st.flags |= 2;
        if (rho0) st.flags |= 1;
        const bool go = (rr > st.target2) && (st.iters < st.maxiter) && !om0 && !rho0;
        st.active = go ? 1 : 0;
    }
}

// The lattice sums of NQ quantities per rhs from the per-block partials: row
// rhs * NQ + q over the lattice's blocks blk0 .. blk0 + nblk - 1.  Warp w of
// nw takes rows w, w + nw, ...; lane k adds blocks k, k + 32, ... in batches
// of 16 independent loads, then a shuffle tree.  The order depends on nw and
// nblk only, so every block of a launch that calls it forms bitwise the same
// sums.  Writes sres[rhs * NQ + q]; the caller synchronises before reading.
template <int NQ, typename A>
__device__ __forceinline__ void lattice_sums(const double* __restrict__ partials_, int nrhs, int nblocks, int blk0,
                                             int nblk, int tid, int nthreads, double* sres) {
    const A* __restrict__ partials = reinterpret_cast<const A*>(partials_);
    const int lane = tid & 31, w = tid >> 5, nw = nthreads >> 5;
    for (int r = w; r < nrhs * NQ; r += nw) {
        const A* src = partials + (long long)r * nblocks + blk0;
        A a = acc_zero<A>();
        for (int c0 = 0; c0 < nblk; c0 += 32 * 16) {
            A v[16];
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                const int c = c0 + 32 * k + lane;
                v[k] = (c < nblk) ? acc_ldcg(src + c) : acc_zero<A>();
            }
#pragma unroll
            for (int k = 0; k < 16; ++k) a = acc_add(a, v[k]);
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) a = acc_add(a, acc_shfl_down(a, off));
        if (lane == 0) sres[r] = acc_to_double(a);
    }
}

// Sum the block partials of each lattice (block l of this launch) and apply
// MODE for each rhs.
template <int NQ, typename A, int MODE, typename RV>
__global__ void __launch_bounds__(FIN_THREADS) k_finish(const LatDev* __restrict__ lats, int nrhs, int nblocks,
                                                         SolverCtx ctx, double* __restrict__ out, int maxiter) {
    pdl_enter();
    __shared__ double sres[MAX_RHS * 3];
    const int l = blockIdx.x;
    const int tid = threadIdx.x;
    lattice_sums<NQ, A>(ctx.partials, nrhs, nblocks, lats[l].blk0, lats[l].nblk, tid, (int)blockDim.x, sres);
    __syncthreads();
    if ((MODE == FIN_INIT || MODE == FIN_INIT_CG) && l == 0 && tid == 0) {
        *ctx.loop_count = 0;
        // inside the graph-resident solve: start the iteration loop of this sweep
        if (ctx.use_cond) cudaGraphSetConditional(ctx.cond, 1u);
    }
    if (tid < nrhs) fin_apply<MODE, RV>(ctx, l * nrhs + tid, tid, sres, out, maxiter);
}

template <int NQ, typename A, int MODE, typename RV>
inline void launch_finish(const LaunchCfg& c, const SolverCtx& ctx, double* out, int maxiter, cudaStream_t st) {
    launch_pdl(k_finish<NQ, A, MODE, RV>, dim3(c.nlat), dim3(FIN_THREADS), st, c.lats, c.nrhs, c.nblocks, ctx, out,
               maxiter);
}

template <typename R, typename A>
__device__ __forceinline__ void dotc_acc(const cpx<R> (&a)[4][3], const cpx<R> (&b)[4][3], A& re, A& im) {
    R sr = 0, si = 0;
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            sr = fma(a[s][c].re, b[s][c].re, sr);
            sr = fma(a[s][c].im, b[s][c].im, sr);
            si = fma(a[s][c].re, b[s][c].im, si);
            si = fma(-a[s][c].im, b[s][c].re, si);
        }
    re = acc_add(re, A{sr});
    im = acc_add(im, A{si});
}
template <typename R, typename A>
__device__ __forceinline__ void norm_acc(const cpx<R> (&a)[4][3], A& n) {
    R s = 0;
#pragma unroll
    for (int sp = 0; sp < 4; ++sp)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            s = fma(a[sp][c].re, a[sp][c].re, s);
            s = fma(a[sp][c].im, a[sp][c].im, s);
        }
    n = acc_add(n, A{s});
}

// ------------------------------------------------------------ kernels
// out(out_par) = a * xv + coef * H hin (+ zv) with a fused reduction.
// RED_CG also opens a CG step: block 0 copies each rhs's state into the
// *_prev fields and sets the loop condition from the active flags the
// previous step left (the loop runs one pass with every rhs idle after the
// last one stops).
template <typename PH, typename PV, int NR, bool DAG, int RED, bool HASZ, int HM>
__global__ void __launch_bounds__(KBT<PH, NR, HM>::MAXT, KBT<PH, NR, HM>::MINB) k_tail(const LatDev* __restrict__ lats, int nlat, int nrhs, int out_par,
                                               CField<PH> hin, CField<PV> xv, CField<PV> zv, Field<PV> out,
                                               CField<PV> ra, double a, double coef, int kpow,
                                               SolverCtx ctx) {
    pdl_enter();
    using RH = typename PH::real;
    using RV = typename PV::real;
    constexpr int NQ = (RED == RED_TS) ? 3 : (RED == RED_R0V || RED == RED_CG) ? 2 : 1;
    const int l = find_lattice(lats, nlat, blockIdx.x);
    const LatDev g = lats[l];
    const int r0 = threadIdx.y * NR;
    const int nval = min(NR, nrhs - r0);
    bool act[NR];
    bool any = false;
#pragma unroll
    for (int j = 0; j < NR; ++j) {
        act[j] = (j < nval) && rhs_active(ctx.st, l * nrhs + r0 + j);
        any = any || act[j];
    }
    using A = typename AccOf<RV>::T;
    A red[NR][NQ];
#pragma unroll
    for (int j = 0; j < NR; ++j)
#pragma unroll
        for (int q = 0; q < NQ; ++q) red[j][q] = acc_zero<A>();
    const RV av = (RV)a;
    const RV cv = (RV)(coef * (kpow == 0 ? 1.0 : kpow == 1 ? g.kappa : g.kappa * g.kappa));
    extern __shared__ float2 hop_sm[];   // hop mode 2: the tile's links
    bool block_any = any;
    if constexpr (HM == 2) block_any = __syncthreads_or(any);   // block-uniform: the staging needs every thread
    if (block_any) {
        for (int tile = tile_begin(g), tile_end_ = tile_end(g); tile < tile_end_; ++tile) {
            stage_if_needed<PH, HM>(g, tile, out_par, hop_sm);
            const int cb = tile_cb(g, tile, threadIdx.x);
            if (cb < 0 || !any) continue;
            const SiteX s = decode_site(g, cb, out_par);
            cpx<RH> acc[NR][4][3];
            hop_any<PH, NR, DAG, HM>(g, s, cb, out_par, hin, r0, nval, acc, hop_sm);
#pragma unroll
            for (int j = 0; j < NR; ++j) {
                if (!act[j]) continue;
                cpx<RV> x[4][3], o[4][3];
                load_spinor<PV, RV>(xv, vbase<PV>(g, r0 + j), g.Vpad, cb, sbase(g, r0 + j), x);
#pragma unroll
                for (int sp = 0; sp < 4; ++sp)
#pragma unroll
                    for (int c = 0; c < 3; ++c)
                        o[sp][c] = cpx<RV>{av * x[sp][c].re + cv * (RV)acc[j][sp][c].re,
                                           av * x[sp][c].im + cv * (RV)acc[j][sp][c].im};
                if (HASZ) {
                    cpx<RV> z[4][3];
                    load_spinor<PV, RV>(zv, vbase<PV>(g, r0 + j), g.Vpad, cb, sbase(g, r0 + j), z);
#pragma unroll
                    for (int sp = 0; sp < 4; ++sp)
#pragma unroll
                        for (int c = 0; c < 3; ++c) o[sp][c] = o[sp][c] + z[sp][c];
                }
                store_spinor<PV, RV>(out, vbase<PV>(g, r0 + j), g.Vpad, cb, sbase(g, r0 + j), o);
                if (RED == RED_R0V) {
                    cpx<RV> q0[4][3];
                    load_spinor<PV, RV>(ra, vbase<PV>(g, r0 + j), g.Vpad, cb, sbase(g, r0 + j), q0);
                    dotc_acc(q0, o, red[j][0], red[j][NQ > 1 ? 1 : 0]);
                } else if (RED == RED_TS) {
                    dotc_acc(o, x, red[j][0], red[j][NQ > 1 ? 1 : 0]);
                    norm_acc(o, red[j][NQ > 2 ? 2 : 0]);
                } else if (RED == RED_NORM) {
                    norm_acc(o, red[j][0]);
                } else if (RED == RED_CG) {
                    norm_acc(x, red[j][0]);
                    norm_acc(o, red[j][NQ > 1 ? 1 : 0]);
                }
            }
        }
    }
    if (RED == RED_NONE) return;
    if (RED == RED_CG && blockIdx.x == 0) {
        // start of a CG step (k_cg_tail reads these copies while it writes the state)
        const int tid = threadIdx.y * blockDim.x + threadIdx.x, nt = blockDim.x * blockDim.y;
        for (int i = tid; i < nlat * nrhs; i += nt) {
            KState& k = ctx.st[i];
            k.gamma_prev = k.rho.x;
            k.alpha_prev = k.alpha.x;
            k.active_prev = k.active;
            k.iters_prev = k.iters;
        }
        if (tid == 0) set_loop_cond(ctx, nlat, nrhs);
    }
    block_partials<NR, NQ>(red, nrhs, ctx.partials);
}

// s = r - alpha v (and its hop-precision copy)
template <typename PV, typename PH, int NR>
__global__ void __launch_bounds__(KB<PV, NR>::MAXT, KB<PV, NR>::MINB) k_s_update(const LatDev* __restrict__ lats, int nlat, int nrhs,
                                                   CField<PV> r, CField<PV> v, Field<PV> s, Field<PH> sh,
                                                   const KState* __restrict__ st) {
    pdl_enter();
    using RV = typename PV::real;
    const int l = find_lattice(lats, nlat, blockIdx.x);
    const LatDev g = lats[l];
    const int r0 = threadIdx.y * NR;
    const int nval = min(NR, nrhs - r0);
    constexpr bool COPY = !std::is_same<PV, PH>::value;
    for (int tile = tile_begin(g), tile_end_ = tile_end(g); tile < tile_end_; ++tile) {
        const int cb = tile_cb(g, tile, threadIdx.x);
        if (cb < 0) continue;
#pragma unroll
        for (int j = 0; j < NR; ++j) {
            if (j >= nval) continue;
            const KState& k = st[l * nrhs + r0 + j];
            if (!k.active) continue;
            const cpx<RV> al = Coef<RV>::alpha(k);
            cpx<RV> a[4][3], b[4][3];
            load_spinor<PV, RV>(r, vbase<PV>(g, r0 + j), g.Vpad, cb, sbase(g, r0 + j), a);
            load_spinor<PV, RV>(v, vbase<PV>(g, r0 + j), g.Vpad, cb, sbase(g, r0 + j), b);
#pragma unroll
            for (int sp = 0; sp < 4; ++sp)
#pragma unroll
                for (int c = 0; c < 3; ++c) a[sp][c] = a[sp][c] - al * b[sp][c];
            store_spinor<PV, RV>(s, vbase<PV>(g, r0 + j), g.Vpad, cb, sbase(g, r0 + j), a);
            if (COPY) store_spinor<PH, RV>(sh, vbase<PH>(g, r0 + j), g.Vpad, cb, sbase(g, r0 + j), a);
        }
    }
}

// One CG step on A = Dhat Dhat^dag in the single-reduction form of
// Chronopoulos and Gear (1989), fused into the second D-hat tail of the
// step: both inner products of a step come from one pass.  From the lattice
// sums gamma = |r|^2 and delta = <r, A r> = |Dhat^dag r|^2 of the partials
// the RED_CG tail wrote for this r,
//   beta = gamma / gamma_prev,  alpha = gamma / (delta - beta gamma / alpha_prev)
//   (beta = 0 and alpha = gamma / delta at the first step);
// then at every site w = A r = t - kappa^2 H_eo (H_oe t) (t = Dhat^dag r from
// that tail, hin = H_oe t), and
//   p = r + beta p,  s = w + beta s  (s = A p),  x += alpha p,  r -= alpha s,
// so w is never stored.  A rhs stops, before its update, when gamma <=
// target2, on breakdown (gamma or the denominator not positive), and after
// maxiter steps.  Every block sums its lattice's partials itself in a fixed
// order, so all blocks take the same decisions; the lattice's first block
// records the step in KState.  What the step reads of KState (*_prev,
// target2, maxiter) no block of this launch writes.  alpha and beta are
// formed in double (the denominator is a difference) and applied in the
// vector precision.
template <typename PV, int NR, int HM>
__global__ void __launch_bounds__(KBT<PV, NR, HM>::MAXT, KBT<PV, NR, HM>::MINB) k_cg_tail(
    const LatDev* __restrict__ lats, int nlat, int nrhs, CField<PV> hin, CField<PV> t, Field<PV> x, Field<PV> r,
    Field<PV> p, Field<PV> s, SolverCtx ctx) {
    pdl_enter();
    using RV = typename PV::real;
    using A = typename AccOf<RV>::T;
    __shared__ double sres[MAX_RHS * 2];
    __shared__ RV scoef[MAX_RHS][2];
    __shared__ int smode[MAX_RHS];
    const int l = find_lattice(lats, nlat, blockIdx.x);
    const LatDev g = lats[l];
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    lattice_sums<2, A>(ctx.partials, nrhs, (int)gridDim.x, g.blk0, g.nblk, tid, (int)(blockDim.x * blockDim.y), sres);
    __syncthreads();
    if (tid < nrhs) {
        KState& k = ctx.st[l * nrhs + tid];
        const double gam = sres[2 * tid], del = sres[2 * tid + 1];
        int mode = 0;  // 0: no update, 1: first step, 2: later step
        int fl = 0;
        double al = 0.0, be = 0.0;
        const bool act = k.active_prev != 0;
        if (act && gam > k.target2) {
            const bool first = (k.iters_prev == 0);
            be = first ? 0.0 : gam / k.gamma_prev;
            const double den = first ? del : del - be * gam / k.alpha_prev;
            if (gam > 0.0 && den > 0.0 && isfinite(gam / den)) {
                al = gam / den;
                mode = first ? 1 : 2;
            } else {
                fl = 1;
            }
        }
        const RV alr = (RV)al, ber = (RV)be;
        scoef[tid][0] = alr;
        scoef[tid][1] = ber;
        smode[tid] = mode;
        if (act && blockIdx.x == g.blk0) {
            k.rr = gam;
            if (mode) {
                k.rho = make_double2(gam, 0.0);
                k.alpha = make_double2((double)alr, 0.0);
                k.beta = make_double2((double)ber, 0.0);
                k.iters = k.iters_prev + 1;
                k.active = (k.iters < k.maxiter) ? 1 : 0;
            } else {
                k.active = 0;
                k.flags |= fl;
            }
        }
    }
    __syncthreads();
    const int r0 = threadIdx.y * NR;
    const int nval = min(NR, nrhs - r0);
    int md[NR];
    RV al[NR], be[NR];
    bool any = false;
#pragma unroll
    for (int j = 0; j < NR; ++j) {
        md[j] = (j < nval) ? smode[r0 + j] : 0;
        al[j] = (j < nval) ? scoef[r0 + j][0] : (RV)0;
        be[j] = (j < nval) ? scoef[r0 + j][1] : (RV)0;
        any = any || md[j] != 0;
    }
    extern __shared__ float2 hop_sm[];   // hop mode 2: the tile's links
    if constexpr (HM == 2) {
        if (!__syncthreads_or(any)) return;   // block-uniform: the staging needs every thread
    } else if (!any) {
        return;
    }
    const RV cv = (RV)(-g.kappa * g.kappa);
    for (int tile = tile_begin(g), tile_end_ = tile_end(g); tile < tile_end_; ++tile) {
        stage_if_needed<PV, HM>(g, tile, 0, hop_sm);
        const int cb = tile_cb(g, tile, threadIdx.x);
        if (cb < 0 || !any) continue;
        const SiteX site = decode_site(g, cb, 0);
        cpx<RV> acc[NR][4][3];
        hop_any<PV, NR, false, HM>(g, site, cb, 0, hin, r0, nval, acc, hop_sm);
#pragma unroll
        for (int j = 0; j < NR; ++j) {
            if (!md[j]) continue;
            const long long vb = vbase<PV>(g, r0 + j), sb = sbase(g, r0 + j);
            const bool later = (md[j] == 2);
            // in stages (s; p; x; r) to bound the live registers
            cpx<RV> sa[4][3], ra[4][3], ua[4][3];
            load_spinor<PV, RV>(t, vb, g.Vpad, cb, sb, sa);
#pragma unroll
            for (int sp = 0; sp < 4; ++sp)
#pragma unroll
                for (int c = 0; c < 3; ++c)
                    sa[sp][c] = cpx<RV>{sa[sp][c].re + cv * acc[j][sp][c].re, sa[sp][c].im + cv * acc[j][sp][c].im};
            if (later) {  // s = w + beta s
                load_spinor<PV, RV>(CField<PV>{s.v, s.scale}, vb, g.Vpad, cb, sb, ua);
#pragma unroll
                for (int sp = 0; sp < 4; ++sp)
#pragma unroll
                    for (int c = 0; c < 3; ++c) sa[sp][c] = sa[sp][c] + be[j] * ua[sp][c];
            }
            store_spinor<PV, RV>(s, vb, g.Vpad, cb, sb, sa);
            load_spinor<PV, RV>(CField<PV>{r.v, r.scale}, vb, g.Vpad, cb, sb, ra);
            if (later) {  // p = r + beta p
                load_spinor<PV, RV>(CField<PV>{p.v, p.scale}, vb, g.Vpad, cb, sb, ua);
#pragma unroll
                for (int sp = 0; sp < 4; ++sp)
#pragma unroll
                    for (int c = 0; c < 3; ++c) ua[sp][c] = ra[sp][c] + be[j] * ua[sp][c];
            } else {
#pragma unroll
                for (int sp = 0; sp < 4; ++sp)
#pragma unroll
                    for (int c = 0; c < 3; ++c) ua[sp][c] = ra[sp][c];
            }
            store_spinor<PV, RV>(p, vb, g.Vpad, cb, sb, ua);
            cpx<RV> xa[4][3];
            load_spinor<PV, RV>(CField<PV>{x.v, x.scale}, vb, g.Vpad, cb, sb, xa);
#pragma unroll
            for (int sp = 0; sp < 4; ++sp)
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    xa[sp][c] = xa[sp][c] + al[j] * ua[sp][c];
                    ra[sp][c] = ra[sp][c] - al[j] * sa[sp][c];
                }
            store_spinor<PV, RV>(x, vb, g.Vpad, cb, sb, xa);
            store_spinor<PV, RV>(r, vb, g.Vpad, cb, sb, ra);
        }
    }
}

// x += alpha p + omega s ; r = s - omega t ; rho' = <r0, r>, rr = |r|^2
template <typename PV, int NR>
__global__ void __launch_bounds__(KB<PV, NR>::MAXT, KB<PV, NR>::MINB) k_xr_update(const LatDev* __restrict__ lats, int nlat, int nrhs,
                                                    Field<PV> x, Field<PV> r, CField<PV> p, CField<PV> s,
                                                    CField<PV> t, CField<PV> r0f, SolverCtx ctx) {
    pdl_enter();
    using RV = typename PV::real;
    const int l = find_lattice(lats, nlat, blockIdx.x);
    const LatDev g = lats[l];
    const int r0 = threadIdx.y * NR;
    const int nval = min(NR, nrhs - r0);
    using A = typename AccOf<RV>::T;
    A red[NR][3];
    bool act[NR];
    cpx<RV> al[NR], om[NR];
#pragma unroll
    for (int j = 0; j < NR; ++j) {
        red[j][0] = red[j][1] = red[j][2] = acc_zero<A>();
        act[j] = (j < nval) && ctx.st[l * nrhs + r0 + j].active;
        if (act[j]) {
            const KState& k = ctx.st[l * nrhs + r0 + j];
            al[j] = Coef<RV>::alpha(k);
            om[j] = Coef<RV>::omega(k);
        }
    }
    for (int tile = tile_begin(g), tile_end_ = tile_end(g); tile < tile_end_; ++tile) {
        const int cb = tile_cb(g, tile, threadIdx.x);
        if (cb < 0) continue;
#pragma unroll
        for (int j = 0; j < NR; ++j) {
            if (!act[j]) continue;
            const long long vb = vbase<PV>(g, r0 + j), sb = sbase(g, r0 + j);
            cpx<RV> xa[4][3], pa[4][3], sa[4][3], ta[4][3];
            load_spinor<PV, RV>(CField<PV>{x.v, x.scale}, vb, g.Vpad, cb, sb, xa);
            load_spinor<PV, RV>(p, vb, g.Vpad, cb, sb, pa);
            load_spinor<PV, RV>(s, vb, g.Vpad, cb, sb, sa);
            load_spinor<PV, RV>(t, vb, g.Vpad, cb, sb, ta);
#pragma unroll
            for (int sp = 0; sp < 4; ++sp)
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    xa[sp][c] = xa[sp][c] + al[j] * pa[sp][c] + om[j] * sa[sp][c];
                    sa[sp][c] = sa[sp][c] - om[j] * ta[sp][c];
                }
            store_spinor<PV, RV>(x, vb, g.Vpad, cb, sb, xa);
            store_spinor<PV, RV>(r, vb, g.Vpad, cb, sb, sa);
            cpx<RV> q0[4][3];
            load_spinor<PV, RV>(r0f, vb, g.Vpad, cb, sb, q0);
            dotc_acc(q0, sa, red[j][0], red[j][1]);
            norm_acc(sa, red[j][2]);
        }
    }
    block_partials<NR, 3>(red, nrhs, ctx.partials);
}

// p = r + beta (p - omega v); the first block also drives the WHILE node
template <typename PV, typename PH, int NR>
__global__ void __launch_bounds__(KB<PV, NR>::MAXT, KB<PV, NR>::MINB) k_p_update(const LatDev* __restrict__ lats, int nlat, int nrhs,
                                                   Field<PV> p, Field<PH> ph, CField<PV> r, CField<PV> v,
                                                   SolverCtx ctx) {
    pdl_enter();
    using RV = typename PV::real;
    constexpr bool COPY = !std::is_same<PV, PH>::value;
    const int l = find_lattice(lats, nlat, blockIdx.x);
    const LatDev g = lats[l];
    const int r0 = threadIdx.y * NR;
    const int nval = min(NR, nrhs - r0);
    for (int tile = tile_begin(g), tile_end_ = tile_end(g); tile < tile_end_; ++tile) {
        const int cb = tile_cb(g, tile, threadIdx.x);
        if (cb < 0) continue;
#pragma unroll
        for (int j = 0; j < NR; ++j) {
            if (j >= nval) continue;
            const KState& k = ctx.st[l * nrhs + r0 + j];
            if (!k.active) continue;
            const cpx<RV> be = Coef<RV>::beta(k);
            const cpx<RV> om = Coef<RV>::omega(k);
            const long long vb = vbase<PV>(g, r0 + j), sb = sbase(g, r0 + j);
            cpx<RV> pa[4][3], ra[4][3];
            load_spinor<PV, RV>(CField<PV>{p.v, p.scale}, vb, g.Vpad, cb, sb, pa);
            load_spinor<PV, RV>(r, vb, g.Vpad, cb, sb, ra);
            if (om.re != (RV)0 || om.im != (RV)0) {  // BiCGStab; CG runs with omega = 0 and skips v
                cpx<RV> va[4][3];
                load_spinor<PV, RV>(v, vb, g.Vpad, cb, sb, va);
#pragma unroll
                for (int sp = 0; sp < 4; ++sp)
#pragma unroll
                    for (int c = 0; c < 3; ++c) pa[sp][c] = pa[sp][c] - om * va[sp][c];
            }
#pragma unroll
            for (int sp = 0; sp < 4; ++sp)
#pragma unroll
                for (int c = 0; c < 3; ++c) pa[sp][c] = ra[sp][c] + be * pa[sp][c];
            store_spinor<PV, RV>(p, vb, g.Vpad, cb, sb, pa);
            if (COPY) store_spinor<PH, RV>(ph, vbase<PH>(g, r0 + j), g.Vpad, cb, sb, pa);
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0 && threadIdx.y == 0) set_loop_cond(ctx, nlat, nrhs);
}

// inner start: b = r64 / |r64|; x = 0, r = r0 = p = b
template <typename PV, typename PH, int NR>
__global__ void __launch_bounds__(KB<PV, NR>::MAXT, KB<PV, NR>::MINB) k_inner_init(const LatDev* __restrict__ lats, int nlat, int nrhs,
                                                     CField<P64> r64, Field<PV> x, Field<PV> r, Field<PV> r0f,
                                                     Field<PV> p, Field<PH> ph, SolverCtx ctx) {
    pdl_enter();
    using RV = typename PV::real;
    constexpr bool COPY = !std::is_same<PV, PH>::value;
    const int l = find_lattice(lats, nlat, blockIdx.x);
    const LatDev g = lats[l];
    const int r0 = threadIdx.y * NR;
    const int nval = min(NR, nrhs - r0);
    using A = typename AccOf<RV>::T;
    A red[NR][1];
    bool act[NR];
    double inv[NR];
#pragma unroll
    for (int j = 0; j < NR; ++j) {
        red[j][0] = acc_zero<A>();
        act[j] = (j < nval) && ctx.ost[l * nrhs + r0 + j].active;
        inv[j] = act[j] ? ctx.ost[l * nrhs + r0 + j].inv_norm : 0.0;
    }
    for (int tile = tile_begin(g), tile_end_ = tile_end(g); tile < tile_end_; ++tile) {
        const int cb = tile_cb(g, tile, threadIdx.x);
        if (cb < 0) continue;
#pragma unroll
        for (int j = 0; j < NR; ++j) {
            if (!act[j]) continue;
            const long long sb = sbase(g, r0 + j);
            cpx<double> b64[4][3];
            load_spinor<P64, double>(r64, vbase<P64>(g, r0 + j), g.Vpad, cb, sb, b64);
            cpx<RV> b[4][3], z[4][3];
#pragma unroll
            for (int sp = 0; sp < 4; ++sp)
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    b[sp][c] = cpx<RV>{(RV)(b64[sp][c].re * inv[j]), (RV)(b64[sp][c].im * inv[j])};
                    z[sp][c] = cpx<RV>{(RV)0, (RV)0};
                }
            const long long vb = vbase<PV>(g, r0 + j);
            store_spinor<PV, RV>(x, vb, g.Vpad, cb, sb, z);
            store_spinor<PV, RV>(r, vb, g.Vpad, cb, sb, b);
            store_spinor<PV, RV>(r0f, vb, g.Vpad, cb, sb, b);
            store_spinor<PV, RV>(p, vb, g.Vpad, cb, sb, b);
            if (COPY) store_spinor<PH, RV>(ph, vbase<PH>(g, r0 + j), g.Vpad, cb, sb, b);
            norm_acc(b, red[j][0]);
        }
    }
    block_partials<NR, 1>(red, nrhs, ctx.partials);
}

// x64 += x / inv_norm for the rhs that iterated in this sweep
template <typename PV, int NR>
__global__ void __launch_bounds__(KB<PV, NR>::MAXT, KB<PV, NR>::MINB) k_dc_update(const LatDev* __restrict__ lats, int nlat, int nrhs,
                                                    Field<P64> x64, CField<PV> x, SolverCtx ctx) {
    pdl_enter();
    using RV = typename PV::real;
    const int l = find_lattice(lats, nlat, blockIdx.x);
    const LatDev g = lats[l];
    const int r0 = threadIdx.y * NR;
    const int nval = min(NR, nrhs - r0);
    for (int tile = tile_begin(g), tile_end_ = tile_end(g); tile < tile_end_; ++tile) {
        const int cb = tile_cb(g, tile, threadIdx.x);
        if (cb < 0) continue;
#pragma unroll
        for (int j = 0; j < NR; ++j) {
            if (j >= nval) continue;
            const OState& o = ctx.ost[l * nrhs + r0 + j];
            if (!o.active) continue;
            const double sc = 1.0 / o.inv_norm;
            const long long sb = sbase(g, r0 + j);
            cpx<RV> e[4][3];
            cpx<double> xa[4][3];
            load_spinor<PV, RV>(x, vbase<PV>(g, r0 + j), g.Vpad, cb, sb, e);
            load_spinor<P64, double>(CField<P64>{x64.v, nullptr}, vbase<P64>(g, r0 + j), g.Vpad, cb, sb, xa);
#pragma unroll
            for (int sp = 0; sp < 4; ++sp)
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    xa[sp][c].re += sc * (double)e[sp][c].re;
                    xa[sp][c].im += sc * (double)e[sp][c].im;
                }
            store_spinor<P64, double>(x64, vbase<P64>(g, r0 + j), g.Vpad, cb, sb, xa);
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0 && threadIdx.y == 0) {
        for (int i = 0; i < nlat * nrhs; ++i)
            if (ctx.ost[i].active) {
                ctx.ost[i].sweeps += 1;
                ctx.ost[i].inner_iters += ctx.st[i].iters;
            }
    }
}

// canonical AoS FP64 [rhs][Vh][12 complex] of one lattice <-> field
template <typename P>
__global__ void k_pack(const LatDev* __restrict__ lat, int nrhs, const double* __restrict__ aos, Field<P> out) {
    pdl_enter();
    using R = typename P::real;
    const LatDev g = *lat;
    const int rhs = blockIdx.y;
    for (int cb = blockIdx.x * blockDim.x + threadIdx.x; cb < g.Vh; cb += gridDim.x * blockDim.x) {
        const double2* src = reinterpret_cast<const double2*>(aos) + ((long long)rhs * g.Vh + cb) * 12;
        cpx<R> p[4][3];
#pragma unroll
        for (int c = 0; c < 12; ++c) {
            const double2 v = src[c];
            p[c / 3][c % 3] = cpx<R>{(R)v.x, (R)v.y};
        }
        store_spinor<P, R>(out, vbase<P>(g, rhs), g.Vpad, cb, sbase(g, rhs), p);
    }
}

template <typename P>
__global__ void k_unpack(const LatDev* __restrict__ lat, int nrhs, CField<P> in, double* __restrict__ aos) {
    pdl_enter();
    using R = typename P::real;
    const LatDev g = *lat;
    const int rhs = blockIdx.y;
    for (int cb = blockIdx.x * blockDim.x + threadIdx.x; cb < g.Vh; cb += gridDim.x * blockDim.x) {
        cpx<R> p[4][3];
        load_spinor<P, R>(in, vbase<P>(g, rhs), g.Vpad, cb, sbase(g, rhs), p);
        double2* dst = reinterpret_cast<double2*>(aos) + ((long long)rhs * g.Vh + cb) * 12;
#pragma unroll
        for (int c = 0; c < 12; ++c) dst[c] = make_double2((double)p[c / 3][c % 3].re, (double)p[c / 3][c % 3].im);
    }
}

// ------------------------------------------------------------ launchers
inline dim3 block_of(const LaunchCfg& c) { return dim3(c.TS, (c.nrhs + c.NR - 1) / c.NR); }

// RHS block widths compiled per precision: FP64 keeps to 1 and 2 (wider
// blocks spill; the FP64 hop is bound by the FP64 pipe, not by link reuse).
#define SF_NR_SWITCH(NRV, ...)                                                    \
    switch (NRV) {                                                                \
        case 1: { constexpr int NR_ = 1; __VA_ARGS__; break; }                    \
        case 2: { constexpr int NR_ = 2; __VA_ARGS__; break; }                    \
        case 3: { if constexpr (!std::is_same<PV, P64>::value) { constexpr int NR_ = 3; __VA_ARGS__; } else return cudaErrorInvalidValue; break; } \
        case 5: { if constexpr (!std::is_same<PV, P64>::value) { constexpr int NR_ = 5; __VA_ARGS__; } else return cudaErrorInvalidValue; break; } \
        default: return cudaErrorInvalidValue;                                    \
    }

template <typename PV, typename PH>
struct OpsImpl {
    // hop modes (c.pipe): 1 the pipelined hop (FP32 / FP16 operands, NR <= 2,
    // blocks of <= 256 threads); 2 links staged per tile (FP32 / FP16
    // operands, NR = 1, TS = 32, blocks of <= 320 threads)
    static bool pipe_ok(const LaunchCfg& c) {
        if (std::is_same<PH, P64>::value) return false;
        const int threads = c.TS * ((c.nrhs + c.NR - 1) / c.NR);
        if (c.pipe == 2) return c.NR == 1 && c.TS == HOP_SM_TS && threads <= 320;
        return c.pipe == 1 && c.NR <= 2 && threads <= 256;
    }
    static size_t smem_of(const LaunchCfg& c) { return c.pipe == 2 ? (size_t)HOP_SM_BYTES : 0; }

    template <int NR, int HM>
    static void hop_nr(const LaunchCfg& c, int out_par, bool dag, FieldPtr in, FieldPtr out, double coef, int kpow,
                       const KState* ks, cudaStream_t st) {
        if (dag)
            launch_pdl_smem(k_hop<PH, PH, NR, true, HM>, dim3(c.nblocks), dim3(block_of(c)), smem_of(c), st, c.lats,
                            c.nlat, c.nrhs, out_par, cf<PH>(in), wf<PH>(out), coef, kpow, ks);
        else
            launch_pdl_smem(k_hop<PH, PH, NR, false, HM>, dim3(c.nblocks), dim3(block_of(c)), smem_of(c), st, c.lats,
                            c.nlat, c.nrhs, out_par, cf<PH>(in), wf<PH>(out), coef, kpow, ks);
    }

    static cudaError_t hop(const LaunchCfg& c, int out_par, bool dag, FieldPtr in, FieldPtr out, double coef,
                           int kpow, const SolverCtx* ctx, cudaStream_t st) {
        const KState* ks = ctx ? ctx->st : nullptr;
        if (c.pipe && !pipe_ok(c)) return cudaErrorInvalidValue;
        SF_NR_SWITCH(c.NR, {
            if constexpr (!std::is_same<PH, P64>::value) {
                if constexpr (NR_ == 1) {
                    if (c.pipe == 2) {
                        hop_nr<1, 2>(c, out_par, dag, in, out, coef, kpow, ks, st);
                        break;
                    }
                }
                if constexpr (NR_ <= 2) {
                    if (c.pipe == 1) {
                        hop_nr<NR_, 1>(c, out_par, dag, in, out, coef, kpow, ks, st);
                        break;
                    }
                }
            }
            hop_nr<NR_, 0>(c, out_par, dag, in, out, coef, kpow, ks, st);
        });
        return cudaGetLastError();
    }

    template <int NR, bool DAG, int HM>
    static void tail_red(const LaunchCfg& c, int out_par, int red, FieldPtr hin, FieldPtr xv, FieldPtr zv,
                         FieldPtr out, FieldPtr ra, double a, double coef, int kpow, SolverCtx k,
                         double* norm_out, cudaStream_t st) {
        const dim3 b = block_of(c);
        const bool hz = zv.v != nullptr;
#define SF_TAIL(RED, HZ)                                                                                        \
    launch_pdl_smem(k_tail<PH, PV, NR, DAG, RED, HZ, HM>, dim3(c.nblocks), dim3(b), smem_of(c), st, c.lats,    \
                    c.nlat, c.nrhs, out_par, cf<PH>(hin), cf<PV>(xv), cf<PV>(zv), wf<PV>(out), cf<PV>(ra), a, coef, \
                    kpow, k)
        using A = typename AccOf<typename PV::real>::T;
        using RV = typename PV::real;
        switch (red) {
            case RED_NONE: if (hz) SF_TAIL(RED_NONE, true); else SF_TAIL(RED_NONE, false); break;
            // without solver states (the block solvers' own finishing kernels
            // read the partials) only the tail runs
            case RED_R0V:
                SF_TAIL(RED_R0V, false);
                if (k.st) launch_finish<2, A, FIN_R0V, RV>(c, k, nullptr, 0, st);
                break;
            case RED_TS:
                SF_TAIL(RED_TS, false);
                if (k.st) launch_finish<3, A, FIN_TS, RV>(c, k, nullptr, 0, st);
                break;
            case RED_NORM:
                if (hz) SF_TAIL(RED_NORM, true); else SF_TAIL(RED_NORM, false);
                launch_finish<1, A, FIN_NORM, RV>(c, k, norm_out, 0, st);
                break;
            case RED_CG:  // only Dhat^dag on the vector precision (tail() checks)
                if constexpr (DAG && std::is_same<PV, PH>::value) SF_TAIL(RED_CG, false);
                break;
        }
#undef SF_TAIL
    }

    static cudaError_t tail(const LaunchCfg& c, int out_par, bool dag, int red, FieldPtr hin, FieldPtr xv,
                            FieldPtr zv, FieldPtr out, FieldPtr ra, double a, double coef, int kpow,
                            const SolverCtx* ctx, double* norm_out, cudaStream_t st) {
        SolverCtx k{};
        if (ctx) k = *ctx;
        if (c.pipe && !pipe_ok(c)) return cudaErrorInvalidValue;
        if (red == RED_CG && (!dag || !std::is_same<PV, PH>::value || !ctx || zv.v)) return cudaErrorInvalidValue;
        SF_NR_SWITCH(c.NR, {
            if constexpr (!std::is_same<PH, P64>::value) {
                if constexpr (NR_ == 1) {
                    if (c.pipe == 2) {
                        if (dag) tail_red<1, true, 2>(c, out_par, red, hin, xv, zv, out, ra, a, coef, kpow, k, norm_out, st);
                        else tail_red<1, false, 2>(c, out_par, red, hin, xv, zv, out, ra, a, coef, kpow, k, norm_out, st);
                        break;
                    }
                }
                if constexpr (NR_ <= 2) {
                    if (c.pipe == 1) {
                        if (dag) tail_red<NR_, true, 1>(c, out_par, red, hin, xv, zv, out, ra, a, coef, kpow, k, norm_out, st);
                        else tail_red<NR_, false, 1>(c, out_par, red, hin, xv, zv, out, ra, a, coef, kpow, k, norm_out, st);
                        break;
                    }
                }
            }
            if (dag) tail_red<NR_, true, 0>(c, out_par, red, hin, xv, zv, out, ra, a, coef, kpow, k, norm_out, st);
            else tail_red<NR_, false, 0>(c, out_par, red, hin, xv, zv, out, ra, a, coef, kpow, k, norm_out, st);
        });
        return cudaGetLastError();
    }

    // ---- one BiCGStab iteration on every rhs of every lattice: hop, tail (v,
    // <r0,v> -> alpha), s_update, hop, tail (t, <t,s>, |t|^2 -> omega),
    // xr_update (<r0,r>, |r|^2 -> beta, convergence), p_update (sets the loop
    // condition): 7 kernels and the lattice sums of 3 reductions.
    static cudaError_t iterate(const LaunchCfg& c, bool dag, const IterFields& f, const SolverCtx* ctx,
                               cudaStream_t st) {
        const FieldPtr none{nullptr, nullptr};
        const bool copy = !std::is_same<PV, PH>::value;
        cudaError_t e;
        if ((e = hop(c, 1, dag, copy ? f.ph : f.p, f.tmp, 1.0, 0, ctx, st)) != cudaSuccess) return e;
        if ((e = tail(c, 0, dag, RED_R0V, f.tmp, f.p, none, f.v, f.r0, 1.0, -1.0, 2, ctx, nullptr, st)) != cudaSuccess)
            return e;
        if ((e = s_update(c, f.r, f.v, f.s, f.sh, ctx, st)) != cudaSuccess) return e;
        if ((e = hop(c, 1, dag, copy ? f.sh : f.s, f.tmp, 1.0, 0, ctx, st)) != cudaSuccess) return e;
        if ((e = tail(c, 0, dag, RED_TS, f.tmp, f.s, none, f.t, none, 1.0, -1.0, 2, ctx, nullptr, st)) != cudaSuccess)
            return e;
        if ((e = xr_update(c, f.x, f.r, f.p, f.s, f.t, f.r0, ctx, st)) != cudaSuccess) return e;
        return p_update(c, f.p, f.ph, f.r, f.v, ctx, st);
    }
    static int iteration_kernels(const LaunchCfg&) { return 10; }

    // ---- one CG step on A = Dhat Dhat^dag (Hermitian, positive) for every
    // active rhs, in the single-reduction form (k_cg_tail):
    //   tmp = H^dag r; t = Dhat^dag r with |r|^2, |t|^2 = <r, A r> (opens the
    //   step, sets the loop condition); tmp = H t; k_cg_tail (alpha, beta,
    //   w = Dhat t at each site, then p, s, x, r).  4 kernels.
    static cudaError_t iterate_cg(const LaunchCfg& c, bool, const IterFields& f, const SolverCtx* ctx,
                                  cudaStream_t st) {
        const FieldPtr none{nullptr, nullptr};
        const bool copy = !std::is_same<PV, PH>::value;
        if (copy) return cudaErrorInvalidValue;  // CG runs with FP32 (or FP64) hop operands
        if (c.pipe && !pipe_ok(c)) return cudaErrorInvalidValue;
        cudaError_t e;
        if ((e = hop(c, 1, true, f.r, f.tmp, 1.0, 0, ctx, st)) != cudaSuccess) return e;
        if ((e = tail(c, 0, true, RED_CG, f.tmp, f.r, none, f.t, none, 1.0, -1.0, 2, ctx, nullptr, st)) !=
            cudaSuccess)
            return e;
        if ((e = hop(c, 1, false, f.t, f.tmp, 1.0, 0, ctx, st)) != cudaSuccess) return e;
#define SF_CG_TAIL(HM_)                                                                                          \
    launch_pdl_smem(k_cg_tail<PV, NR_, HM_>, dim3(c.nblocks), dim3(block_of(c)), smem_of(c), st, c.lats, c.nlat,  \
                    c.nrhs, cf<PV>(f.tmp), cf<PV>(f.t), wf<PV>(f.x), wf<PV>(f.r), wf<PV>(f.p), wf<PV>(f.s), *ctx)
        SF_NR_SWITCH(c.NR, {
            if constexpr (!std::is_same<PH, P64>::value) {
                if constexpr (NR_ == 1) {
                    if (c.pipe == 2) {
                        SF_CG_TAIL(2);
                        break;
                    }
                }
                if constexpr (NR_ <= 2) {
                    if (c.pipe == 1) {
                        SF_CG_TAIL(1);
                        break;
                    }
                }
            }
            SF_CG_TAIL(0);
        });
#undef SF_CG_TAIL
        return cudaGetLastError();
    }
    static int iteration_kernels_cg(const LaunchCfg&) { return 4; }

    static cudaError_t init(const LaunchCfg& c, FieldPtr r64, FieldPtr x, FieldPtr r, FieldPtr r0, FieldPtr p,
                            FieldPtr ph, const SolverCtx* ctx, int maxiter, cudaStream_t st) {
        SF_NR_SWITCH(c.NR, {
            launch_pdl(k_inner_init<PV, PH, NR_>, dim3(c.nblocks), dim3(block_of(c)), st, 
                c.lats, c.nlat, c.nrhs, cf<P64>(r64), wf<PV>(x), wf<PV>(r), wf<PV>(r0), wf<PV>(p), wf<PH>(ph),
                *ctx);
        });
        launch_finish<1, typename AccOf<typename PV::real>::T, FIN_INIT, typename PV::real>(c, *ctx, nullptr, maxiter,
                                                                                           st);
        return cudaGetLastError();
    }

    static cudaError_t init_cg(const LaunchCfg& c, FieldPtr r64, FieldPtr x, FieldPtr r, FieldPtr r0, FieldPtr p,
                               FieldPtr ph, const SolverCtx* ctx, int maxiter, cudaStream_t st) {
        SF_NR_SWITCH(c.NR, {
            launch_pdl(k_inner_init<PV, PH, NR_>, dim3(c.nblocks), dim3(block_of(c)), st, c.lats, c.nlat, c.nrhs,
                       cf<P64>(r64), wf<PV>(x), wf<PV>(r), wf<PV>(r0), wf<PV>(p), wf<PH>(ph), *ctx);
        });
        launch_finish<1, typename AccOf<typename PV::real>::T, FIN_INIT_CG, typename PV::real>(c, *ctx, nullptr,
                                                                                              maxiter, st);
        return cudaGetLastError();
    }

    static cudaError_t s_update(const LaunchCfg& c, FieldPtr r, FieldPtr v, FieldPtr s, FieldPtr sh,
                                const SolverCtx* ctx, cudaStream_t st) {
        SF_NR_SWITCH(c.NR, {
            launch_pdl(k_s_update<PV, PH, NR_>, dim3(c.nblocks), dim3(block_of(c)), st, c.lats, c.nlat, c.nrhs, cf<PV>(r),
                                                                        cf<PV>(v), wf<PV>(s), wf<PH>(sh), ctx->st);
        });
        return cudaGetLastError();
    }

    static cudaError_t xr_update(const LaunchCfg& c, FieldPtr x, FieldPtr r, FieldPtr p, FieldPtr s, FieldPtr t,
                                 FieldPtr r0, const SolverCtx* ctx, cudaStream_t st) {
        SF_NR_SWITCH(c.NR, {
            launch_pdl(k_xr_update<PV, NR_>, dim3(c.nblocks), dim3(block_of(c)), st, c.lats, c.nlat, c.nrhs,
                       wf<PV>(x), wf<PV>(r), cf<PV>(p), cf<PV>(s), cf<PV>(t), cf<PV>(r0), *ctx);
        });
        launch_finish<3, typename AccOf<typename PV::real>::T, FIN_XR, typename PV::real>(c, *ctx, nullptr, 0, st);
        return cudaGetLastError();
    }

    static cudaError_t p_update(const LaunchCfg& c, FieldPtr p, FieldPtr ph, FieldPtr r, FieldPtr v,
                                const SolverCtx* ctx, cudaStream_t st) {
        SF_NR_SWITCH(c.NR, {
            launch_pdl(k_p_update<PV, PH, NR_>, dim3(c.nblocks), dim3(block_of(c)), st, c.lats, c.nlat, c.nrhs, wf<PV>(p),
                                                                        wf<PH>(ph), cf<PV>(r), cf<PV>(v), *ctx);
        });
        return cudaGetLastError();
    }

    static cudaError_t dc_update(const LaunchCfg& c, FieldPtr x64, FieldPtr x, const SolverCtx* ctx,
                                 cudaStream_t st) {
        SF_NR_SWITCH(c.NR, {
            launch_pdl(k_dc_update<PV, NR_>, dim3(c.nblocks), dim3(block_of(c)), st, c.lats, c.nlat, c.nrhs, wf<P64>(x64),
                                                                     cf<PV>(x), *ctx);
        });
        return cudaGetLastError();
    }

    static cudaError_t pack(const LaunchCfg& c, const double* aos, FieldPtr out, cudaStream_t st) {
        k_pack<PV><<<dim3(64, c.nrhs), 256, 0, st>>>(c.lats, c.nrhs, aos, wf<PV>(out));
        return cudaGetLastError();
    }
    static cudaError_t unpack(const LaunchCfg& c, FieldPtr in, double* aos, cudaStream_t st) {
        k_unpack<PV><<<dim3(64, c.nrhs), 256, 0, st>>>(c.lats, c.nrhs, cf<PV>(in), aos);
        return cudaGetLastError();
    }
    static cudaError_t pack_h(const LaunchCfg& c, const double* aos, FieldPtr out, cudaStream_t st) {
        k_pack<PH><<<dim3(64, c.nrhs), 256, 0, st>>>(c.lats, c.nrhs, aos, wf<PH>(out));
        return cudaGetLastError();
    }
    static cudaError_t unpack_h(const LaunchCfg& c, FieldPtr in, double* aos, cudaStream_t st) {
        k_unpack<PH><<<dim3(64, c.nrhs), 256, 0, st>>>(c.lats, c.nrhs, cf<PH>(in), aos);
        return cudaGetLastError();
    }

    static KrylovOps table(Prec pv, Prec ph) {
        KrylovOps o;
        o.pv = pv;
        o.ph = ph;
        o.hop = &hop;
        o.tail = &tail;
        o.init = &init;
        o.s_update = &s_update;
        o.xr_update = &xr_update;
        o.p_update = &p_update;
        o.dc_update = &dc_update;
        o.pack = &pack;
        o.unpack = &unpack;
        o.pack_h = &pack_h;
        o.unpack_h = &unpack_h;
        o.iterate = &iterate;
        o.iteration_kernels = &iteration_kernels;
        o.init_cg = &init_cg;
        o.iterate_cg = &iterate_cg;
        o.iteration_kernels_cg = &iteration_kernels_cg;
        return o;
    }
};

}  // namespace sf
