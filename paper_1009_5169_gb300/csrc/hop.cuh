// hop.cuh -- the Wilson hop H_oe / H_eo of the even/odd operator (Sec. 3.1,
// Eq. 2 with the SF boundaries of Sec. 4) on the SoA field storage, for NR
// right-hand sides per thread, plain, with the next directions' operands
// fetched ahead, or with each tile's links staged once in shared memory, and
// the k_hop kernel that applies it to a whole block of lattices.  The fused Dhat tail and the solver kernels build on it
// (krylov_impl.cuh).
//   (H psi)(x) = sum_mu (1 - gamma_mu) U_mu(x) lambda_mu psi(x+mu)
//              + (1 + gamma_mu) U_mu(x-mu)^dag lambda_mu^* psi(x-mu),
//   lambda_0 = 1, lambda_k = e^{i theta/L} (stored inside the spatial links);
//   time hops leaving x0 = 1..T-1 are dropped (Dirichlet).
#pragma once
#include <type_traits>

#include "sf_kernels.h"

namespace sf {

template <typename P> __host__ __device__ __forceinline__ CField<P> cf(FieldPtr f) {
    return CField<P>{reinterpret_cast<const typename P::vec*>(f.v), f.s};
}
template <typename P> __host__ __device__ __forceinline__ Field<P> wf(FieldPtr f) {
    return Field<P>{reinterpret_cast<typename P::vec*>(f.v), f.s};
}

__device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
    const double d = b.x * b.x + b.y * b.y;
    return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// element offsets of (lattice block, rhs)
template <typename P>
__device__ __forceinline__ long long vbase(const LatDev& g, int rhs) {
    return (g.soff + (long long)rhs * g.Vpad) * P::NC;
}
__device__ __forceinline__ long long sbase(const LatDev& g, int rhs) { return g.soff + (long long)rhs * g.Vpad; }

// Threads per block a kernel of a (precision, NR) configuration may be
// launched with; it sets the register budget 65536 / MAXT per thread.
// FP32/FP16 with NR = 1 is held to 96 registers (two 320-thread blocks per
// SM): the hop is latency-bound and gains more from resident warps than from
// the extra load hoisting a larger budget buys.
template <typename P, int NR>
struct KB {
    static constexpr bool F64 = std::is_same<P, P64>::value;
    static constexpr int MAXT = F64 ? 256 : (NR == 1 ? 320 : NR == 2 ? 384 : 256);
    static constexpr int MINB = F64 ? 1 : (NR == 1 ? 2 : 1);
};
// Hop modes (the HM template argument of the hop and tail kernels):
//   0  plain: every thread loads and rebuilds the links of its site itself;
//   1  pipelined: the operands of later directions are loaded ahead (FP32 /
//      FP16, NR <= 2, blocks of at most 256 threads, up to 255 registers);
//   2  links staged per tile: FP32 / FP16 operands, one right-hand side per
//      thread, tiles of 32 sites; the block reads and rebuilds each site's
//      eight links once into shared memory and all its right-hand-side rows
//      apply them from there, at 64 registers (six 160-thread blocks per SM).
template <typename P, int NR, int HM>
struct KBH {
    static constexpr int MAXT = HM == 2 ? 320 : HM == 1 ? 256 : KB<P, NR>::MAXT;
    static constexpr int MINB = HM == 2 ? 3 : HM == 1 ? 1 : KB<P, NR>::MINB;
};
// the fused tails (more live state than the bare hop): in hop mode 2 held to
// about 100 registers instead of 64
template <typename P, int NR, int HM>
struct KBT {
    static constexpr int MAXT = KBH<P, NR, HM>::MAXT;
    static constexpr int MINB = HM == 2 ? 2 : KBH<P, NR, HM>::MINB;
};

// ------------------------------------------------------------ hop
template <int MU, typename P, int NR, bool DAG>
__device__ __forceinline__ void hop_dir(const LatDev& g, const SiteX& s, int cb, int out_par,
                                        const CField<P>& in, int r0, int nval,
                                        cpx<typename P::real> (&acc)[NR][4][3]) {
    using R = typename P::real;
    constexpr int SF = DAG ? +1 : -1;  // forward projector 1 + SF gamma_mu
    constexpr int SB = -SF;
    if (MU != 0 || s.x0 < g.T - 1) {
        const int ncb = neighbour_cb<MU, +1>(g, s);
        Link<R> U;
        LinkLoad<P>::template load<MU>(g, out_par, cb, U);
#pragma unroll
        for (int j = 0; j < NR; ++j) {
            if (j < nval) {
                cpx<R> p[4][3];
                cpx<R> h[2][3], w[2][3];
                if constexpr (std::is_same<P, P16>::value) {
                    uint32_t q[12];
                    load_spinor_h16(in, vbase<P>(g, r0 + j), g.Vpad, ncb, q);
                    project_h16<MU, SF>(q, h);
                    const float sc = __ldg(in.scale + sbase(g, r0 + j) + ncb);
                    mul_link(U, h, w);
                    expand_fma<MU, SF>(acc[j], w, sc);
                } else {
                    load_spinor<P, R>(in, vbase<P>(g, r0 + j), g.Vpad, ncb, sbase(g, r0 + j), p);
                    project<MU, SF>(p, h);
                    mul_link(U, h, w);
                    expand_add<MU, SF>(acc[j], w);
                }
            }
        }
    }
    if (MU != 0 || s.x0 > 1) {
        const int ncb = neighbour_cb<MU, -1>(g, s);
        Link<R> U;
        LinkLoad<P>::template load<MU>(g, out_par ^ 1, ncb, U);
#pragma unroll
        for (int j = 0; j < NR; ++j) {
            if (j < nval) {
                cpx<R> p[4][3];
                cpx<R> h[2][3], w[2][3];
                if constexpr (std::is_same<P, P16>::value) {
                    uint32_t q[12];
                    load_spinor_h16(in, vbase<P>(g, r0 + j), g.Vpad, ncb, q);
                    project_h16<MU, SB>(q, h);
                    const float sc = __ldg(in.scale + sbase(g, r0 + j) + ncb);
                    mul_link_dag(U, h, w);
                    expand_fma<MU, SB>(acc[j], w, sc);
                } else {
                    load_spinor<P, R>(in, vbase<P>(g, r0 + j), g.Vpad, ncb, sbase(g, r0 + j), p);
                    project<MU, SB>(p, h);
                    mul_link_dag(U, h, w);
                    expand_add<MU, SB>(acc[j], w);
                }
            }
        }
    }
}

template <typename P, int NR, bool DAG>
__device__ __forceinline__ void hop_site(const LatDev& g, const SiteX& s, int cb, int out_par,
                                         const CField<P>& in, int r0, int nval,
                                         cpx<typename P::real> (&acc)[NR][4][3]) {
#pragma unroll
    for (int j = 0; j < NR; ++j)
#pragma unroll
        for (int sp = 0; sp < 4; ++sp)
#pragma unroll
            for (int a = 0; a < 3; ++a) acc[j][sp][a] = cpx<typename P::real>{0, 0};
    hop_dir<0, P, NR, DAG>(g, s, cb, out_par, in, r0, nval, acc);
    hop_dir<1, P, NR, DAG>(g, s, cb, out_par, in, r0, nval, acc);
    hop_dir<2, P, NR, DAG>(g, s, cb, out_par, in, r0, nval, acc);
    hop_dir<3, P, NR, DAG>(g, s, cb, out_par, in, r0, nval, acc);
}

// ------------------------------------------------------------ pipelined hop
// FP32 / FP16 operands with NR <= 2: the raw operands of hop H (H = 2 mu,
// + 1 for the backward hop) are loaded PF hops ahead of their use, so a
// site's eight dependent load round trips overlap about PF at a time.  This
// pays in registers (PF buffers) what it saves in latency: for small
// lattices, whose launches hold a few warps per SM; the autotuner chooses.
template <typename P, int NR> struct HopBuf;
template <int NR> struct HopBuf<P32, NR> {
    float4 u[3];       // link rows 0, 1
    float4 s[NR][6];   // neighbour spinors
};
template <int NR> struct HopBuf<P16, NR> {
    uint2 u[3];
    uint4 s[NR][3];
    float sc[NR];
};
template <int NR> struct PipeDepth { static constexpr int PF = (NR == 1) ? 4 : 2; };

template <int H, typename P, int NR>
__device__ __forceinline__ void hop_fetch(const LatDev& g, const SiteX& s, int cb, int out_par, const CField<P>& in,
                                          int r0, int nval, HopBuf<P, NR>& b, bool& valid) {
    constexpr int MU = H >> 1;
    constexpr bool FWD = (H & 1) == 0;
    valid = (MU != 0) || (FWD ? (s.x0 < g.T - 1) : (s.x0 > 1));
    if (!valid) return;
    const int ncb = neighbour_cb<MU, FWD ? +1 : -1>(g, s);
    const int lpar = FWD ? out_par : (out_par ^ 1);
    const int lcb = FWD ? cb : ncb;
    if constexpr (std::is_same<P, P32>::value) {
        const float4* ub = g.u32 + ((long long)(MU * 2 + lpar) * 3) * g.Vpad + lcb;
#pragma unroll
        for (int k = 0; k < 3; ++k) b.u[k] = __ldg(ub + (long long)k * g.Vpad);
#pragma unroll
        for (int j = 0; j < NR; ++j)
            if (j < nval) {
                const float4* sp = in.v + vbase<P32>(g, r0 + j) + ncb;
#pragma unroll
                for (int k = 0; k < 6; ++k) b.s[j][k] = __ldg(sp + (long long)k * g.Vpad);
            }
    } else {
        const uint2* ub = g.u16 + ((long long)(MU * 2 + lpar) * 3) * g.Vpad + lcb;
#pragma unroll
        for (int k = 0; k < 3; ++k) b.u[k] = __ldg(ub + (long long)k * g.Vpad);
#pragma unroll
        for (int j = 0; j < NR; ++j)
            if (j < nval) {
                const uint4* sp = in.v + vbase<P16>(g, r0 + j) + ncb;
#pragma unroll
                for (int k = 0; k < 3; ++k) b.s[j][k] = __ldg(sp + (long long)k * g.Vpad);
                b.sc[j] = __ldg(in.scale + sbase(g, r0 + j) + ncb);
            }
    }
}

template <int H, typename P, int NR, bool DAG>
__device__ __forceinline__ void hop_apply(const LatDev& g, const HopBuf<P, NR>& b, bool valid, int nval,
                                          cpx<float> (&acc)[NR][4][3]) {
    constexpr int MU = H >> 1;
    constexpr bool FWD = (H & 1) == 0;
    constexpr int S = (FWD == DAG) ? +1 : -1;  // projector 1 + S gamma_mu
    if (!valid) return;
    Link<float> U;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        float2 a, c;
        if constexpr (std::is_same<P, P32>::value) {
            a = make_float2(b.u[k].x, b.u[k].y);
            c = make_float2(b.u[k].z, b.u[k].w);
        } else {
            a = h2f(b.u[k].x);
            c = h2f(b.u[k].y);
        }
        U.m[(2 * k) / 3][(2 * k) % 3] = cpx<float>{a.x, a.y};
        U.m[(2 * k + 1) / 3][(2 * k + 1) % 3] = cpx<float>{c.x, c.y};
    }
    rebuild_row2<MU>(g, U);
#pragma unroll
    for (int j = 0; j < NR; ++j) {
        if (j < nval) {
            cpx<float> h[2][3], w[2][3];
            if constexpr (std::is_same<P, P32>::value) {
                cpx<float> p[4][3];
#pragma unroll
                for (int k = 0; k < 6; ++k) {
                    p[(2 * k) / 3][(2 * k) % 3] = cpx<float>{b.s[j][k].x, b.s[j][k].y};
                    p[(2 * k + 1) / 3][(2 * k + 1) % 3] = cpx<float>{b.s[j][k].z, b.s[j][k].w};
                }
                project<MU, S>(p, h);
            } else {
                uint32_t q[12];
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    q[4 * k] = b.s[j][k].x;
                    q[4 * k + 1] = b.s[j][k].y;
                    q[4 * k + 2] = b.s[j][k].z;
                    q[4 * k + 3] = b.s[j][k].w;
                }
                project_h16<MU, S>(q, h);
            }
            if (FWD) mul_link(U, h, w);
            else mul_link_dag(U, h, w);
            if constexpr (std::is_same<P, P32>::value) expand_add<MU, S>(acc[j], w);
            else expand_fma<MU, S>(acc[j], w, b.sc[j]);   // the FP16 scale, applied in the sum
        }
    }
}

// apply hop H from its buffer, then reuse the buffer for hop H + PF
template <int H, typename P, int NR, bool DAG, int PF>
__device__ __forceinline__ void hop_step(const LatDev& g, const SiteX& s, int cb, int out_par, const CField<P>& in,
                                         int r0, int nval, HopBuf<P, NR> (&b)[PF], bool (&v)[8],
                                         cpx<float> (&acc)[NR][4][3]) {
    hop_apply<H, P, NR, DAG>(g, b[H % PF], v[H], nval, acc);
    if constexpr (H + PF < 8) hop_fetch<H + PF, P, NR>(g, s, cb, out_par, in, r0, nval, b[H % PF], v[H + PF]);
}

template <typename P, int NR, bool DAG>
__device__ __forceinline__ void hop_site_pipe(const LatDev& g, const SiteX& s, int cb, int out_par,
                                              const CField<P>& in, int r0, int nval, cpx<float> (&acc)[NR][4][3]) {
    constexpr int PF = PipeDepth<NR>::PF;
#pragma unroll
    for (int j = 0; j < NR; ++j)
#pragma unroll
        for (int sp = 0; sp < 4; ++sp)
#pragma unroll
            for (int a = 0; a < 3; ++a) acc[j][sp][a] = cpx<float>{0.f, 0.f};
    HopBuf<P, NR> b[PF];
    bool v[8];
    hop_fetch<0, P, NR>(g, s, cb, out_par, in, r0, nval, b[0], v[0]);
    hop_fetch<1, P, NR>(g, s, cb, out_par, in, r0, nval, b[1 % PF], v[1]);
    if constexpr (PF > 2) hop_fetch<2, P, NR>(g, s, cb, out_par, in, r0, nval, b[2 % PF], v[2]);
    if constexpr (PF > 3) hop_fetch<3, P, NR>(g, s, cb, out_par, in, r0, nval, b[3 % PF], v[3]);
    hop_step<0, P, NR, DAG, PF>(g, s, cb, out_par, in, r0, nval, b, v, acc);
    hop_step<1, P, NR, DAG, PF>(g, s, cb, out_par, in, r0, nval, b, v, acc);
    hop_step<2, P, NR, DAG, PF>(g, s, cb, out_par, in, r0, nval, b, v, acc);
    hop_step<3, P, NR, DAG, PF>(g, s, cb, out_par, in, r0, nval, b, v, acc);
    hop_step<4, P, NR, DAG, PF>(g, s, cb, out_par, in, r0, nval, b, v, acc);
    hop_step<5, P, NR, DAG, PF>(g, s, cb, out_par, in, r0, nval, b, v, acc);
    hop_step<6, P, NR, DAG, PF>(g, s, cb, out_par, in, r0, nval, b, v, acc);
    hop_step<7, P, NR, DAG, PF>(g, s, cb, out_par, in, r0, nval, b, v, acc);
}

// ------------------------------------------------------------ links staged per tile (hop mode 2)
// Tiles of HOP_SM_TS = 32 sites (blockDim.x); shared memory per block:
// float2 [8 directions][9 elements][32 sites], the FP32 complex elements of
// U_mu(x) (direction 2 mu) and U_mu(x - mu) (direction 2 mu + 1), 18 KiB.
constexpr int HOP_SM_TS = 32;
constexpr int HOP_SM_BYTES = 8 * 9 * HOP_SM_TS * (int)sizeof(float2);

// All threads of the block: read the links of the tile's sites and rebuild
// their third rows, once per (site, direction).
template <typename P>
__device__ __forceinline__ void stage_tile_links(const LatDev& g, int tile, int out_par, float2* __restrict__ sm) {
    constexpr int TS = HOP_SM_TS;
    const int nthr = TS * blockDim.y;
    for (int li = threadIdx.y * TS + threadIdx.x; li < 8 * TS; li += nthr) {
        const int dir = li / TS, sl = li % TS;
        const int cb = tile_cb(g, tile, sl);
        if (cb < 0) continue;
        const SiteX s = decode_site(g, cb, out_par);
        Link<float> U;
        switch (dir) {
            case 0: if (s.x0 >= g.T - 1) continue; LinkLoad<P>::template load<0>(g, out_par, cb, U); break;
            case 1: if (s.x0 <= 1) continue; LinkLoad<P>::template load<0>(g, out_par ^ 1, neighbour_cb<0, -1>(g, s), U); break;
            case 2: LinkLoad<P>::template load<1>(g, out_par, cb, U); break;
            case 3: LinkLoad<P>::template load<1>(g, out_par ^ 1, neighbour_cb<1, -1>(g, s), U); break;
            case 4: LinkLoad<P>::template load<2>(g, out_par, cb, U); break;
            case 5: LinkLoad<P>::template load<2>(g, out_par ^ 1, neighbour_cb<2, -1>(g, s), U); break;
            case 6: LinkLoad<P>::template load<3>(g, out_par, cb, U); break;
            default: LinkLoad<P>::template load<3>(g, out_par ^ 1, neighbour_cb<3, -1>(g, s), U); break;
        }
        float2* d = sm + dir * 9 * TS + sl;
#pragma unroll
        for (int k = 0; k < 9; ++k) d[k * TS] = make_float2(U.m[k / 3][k % 3].re, U.m[k / 3][k % 3].im);
    }
}

template <int MU, bool FWD, typename P, bool DAG>
__device__ __forceinline__ void hop_dir_staged(const LatDev& g, const SiteX& s, const CField<P>& in, int rhs,
                                               const float2* __restrict__ sm, cpx<float> (&acc)[4][3]) {
    if (MU == 0 && (FWD ? s.x0 >= g.T - 1 : s.x0 <= 1)) return;
    constexpr int SF = DAG ? +1 : -1;   // forward projector 1 + SF gamma_mu, backward 1 - SF gamma_mu
    constexpr int S = FWD ? SF : -SF;
    const int ncb = neighbour_cb<MU, FWD ? +1 : -1>(g, s);
    float sc = 1.f;
    cpx<float> h[2][3], w[2][3];
    if constexpr (std::is_same<P, P16>::value) {
        uint32_t q[12];
        load_spinor_h16(in, vbase<P>(g, rhs), g.Vpad, ncb, q);
        project_h16<MU, S>(q, h);
        sc = __ldg(in.scale + sbase(g, rhs) + ncb);
    } else {
        cpx<float> p[4][3];
        load_spinor<P, float>(in, vbase<P>(g, rhs), g.Vpad, ncb, sbase(g, rhs), p);
        project<MU, S>(p, h);
    }
    constexpr int TS = HOP_SM_TS;
    const float2* u = sm + (2 * MU + (FWD ? 0 : 1)) * 9 * TS + threadIdx.x;
    Link<float> U;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        const float2 v = u[k * TS];
        U.m[k / 3][k % 3] = cpx<float>{v.x, v.y};
    }
    if (FWD) mul_link(U, h, w);
    else mul_link_dag(U, h, w);
    if constexpr (std::is_same<P, P16>::value) expand_fma<MU, S>(acc, w, sc);   // the FP16 scale, in the sum
    else expand_add<MU, S>(acc, w);
}

template <typename P, bool DAG>
__device__ __forceinline__ void hop_site_staged(const LatDev& g, const SiteX& s, const CField<P>& in, int rhs,
                                                const float2* __restrict__ sm, cpx<float> (&acc)[1][4][3]) {
#pragma unroll
    for (int sp = 0; sp < 4; ++sp)
#pragma unroll
        for (int a = 0; a < 3; ++a) acc[0][sp][a] = cpx<float>{0.f, 0.f};
    hop_dir_staged<0, true, P, DAG>(g, s, in, rhs, sm, acc[0]);
    hop_dir_staged<0, false, P, DAG>(g, s, in, rhs, sm, acc[0]);
    hop_dir_staged<1, true, P, DAG>(g, s, in, rhs, sm, acc[0]);
    hop_dir_staged<1, false, P, DAG>(g, s, in, rhs, sm, acc[0]);
    hop_dir_staged<2, true, P, DAG>(g, s, in, rhs, sm, acc[0]);
    hop_dir_staged<2, false, P, DAG>(g, s, in, rhs, sm, acc[0]);
    hop_dir_staged<3, true, P, DAG>(g, s, in, rhs, sm, acc[0]);
    hop_dir_staged<3, false, P, DAG>(g, s, in, rhs, sm, acc[0]);
}

// At the top of each tile of a hop-mode-2 kernel: every thread of the block
// takes part, whether or not its right-hand side is active.
template <typename P, int HM>
__device__ __forceinline__ void stage_if_needed(const LatDev& g, int tile, int out_par, float2* sm) {
    if constexpr (HM == 2) {
        __syncthreads();   // the previous tile's links are no longer read
        stage_tile_links<P>(g, tile, out_par, sm);
        __syncthreads();
    }
}

// the hop of one site for NR right-hand sides in hop mode HM (sm: the
// tile's staged links, mode 2 only)
template <typename P, int NR, bool DAG, int HM>
__device__ __forceinline__ void hop_any(const LatDev& g, const SiteX& s, int cb, int out_par, const CField<P>& in,
                                        int r0, int nval, cpx<typename P::real> (&acc)[NR][4][3],
                                        const float2* sm = nullptr) {
    if constexpr (HM == 2) {
        static_assert(NR == 1 && !std::is_same<P, P64>::value, "staged links: FP32 / FP16 operands, NR = 1");
        hop_site_staged<P, DAG>(g, s, in, r0, sm, acc);
    } else if constexpr (HM == 1) {
        hop_site_pipe<P, NR, DAG>(g, s, cb, out_par, in, r0, nval, acc);
    } else {
        hop_site<P, NR, DAG>(g, s, cb, out_par, in, r0, nval, acc);
    }
}

__device__ __forceinline__ bool rhs_active(const KState* st, int idx) { return st == nullptr || st[idx].active != 0; }


// ------------------------------------------------------------ kernels
// coef * kappa^kpow for the FP16-operand hop.  Kept out of line: inlined,
// the kpow selects change how the compiler schedules the tile loop, and the
// FP16 staged-link hop then spills more at its 64-register budget.
__device__ __noinline__ inline float hop_scale(double coef, int kpow, double kappa) {
    return (float)(coef * (kpow == 0 ? 1.0 : kpow == 1 ? kappa : kappa * kappa));
}

// out(out_par) = coef * H in
template <typename PI, typename PO, int NR, bool DAG, int HM>
__global__ void __launch_bounds__(KBH<PI, NR, HM>::MAXT, KBH<PI, NR, HM>::MINB) k_hop(const LatDev* __restrict__ lats, int nlat, int nrhs, int out_par,
                                              CField<PI> in, Field<PO> out, double coef, int kpow,
                                              const KState* __restrict__ st) {
    pdl_enter();
    extern __shared__ float2 hop_sm[];   // hop mode 2: the tile's links
    using R = typename PI::real;
    const int l = find_lattice(lats, nlat, blockIdx.x);
    const LatDev g = lats[l];
    const int r0 = threadIdx.y * NR;
    const int nval = min(NR, nrhs - r0);
    bool any = false;
#pragma unroll
    for (int j = 0; j < NR; ++j)
        if (j < nval && rhs_active(st, l * nrhs + r0 + j)) any = true;
    if constexpr (HM == 2) {
        if (!__syncthreads_or(any)) return;   // block-uniform: the staging needs every thread
    } else if (!any) {
        return;
    }
    R c;
    if constexpr (std::is_same<PI, P16>::value) c = hop_scale(coef, kpow, g.kappa);
    else c = (R)(coef * (kpow == 0 ? 1.0 : kpow == 1 ? g.kappa : g.kappa * g.kappa));
    for (int tile = tile_begin(g), tile_end_ = tile_end(g); tile < tile_end_; ++tile) {
        stage_if_needed<PI, HM>(g, tile, out_par, hop_sm);
        const int cb = tile_cb(g, tile, threadIdx.x);
        if (cb < 0 || !any) continue;
        const SiteX s = decode_site(g, cb, out_par);
        cpx<R> acc[NR][4][3];
        hop_any<PI, NR, DAG, HM>(g, s, cb, out_par, in, r0, nval, acc, hop_sm);
#pragma unroll
        for (int j = 0; j < NR; ++j) {
            if (j < nval) {
#pragma unroll
                for (int sp = 0; sp < 4; ++sp)
#pragma unroll
                    for (int a = 0; a < 3; ++a) acc[j][sp][a] = c * acc[j][sp][a];
                store_spinor<PO, R>(out, vbase<PO>(g, r0 + j), g.Vpad, cb, sbase(g, r0 + j), acc[j]);
            }
        }
    }
}

}  // namespace sf
