// gauge.cu -- gauge-field kernels: link preparation into the hop layouts,
// the SU(3) check of an input field, the SF plaquette action (Sec. 4) and the
// MD force of Eq. (3) summed over the pseudo-fermion fields (the force steps of Alg. 2).
#include <algorithm>
#include <type_traits>

#include "krylov_impl.cuh"

namespace sf {

// ------------------------------------------------------------ link prep
// canon: [(T+1) L^3][mu][3][3] complex FP64; fermion site (par, cb) has gauge
// index lex + L^3.  Writes every (mu, parity, cb) of the fermion lattice in
// the three hop layouts (FP64 all 18 reals, FP32 and FP16 rows 0 and 1),
// spatial links multiplied by the twist phase e^{i theta/L} in FP64 before
// rounding.
__global__ void k_link_prep(LatDev g, const double2* __restrict__ canon, double2* __restrict__ u64,
                            float4* __restrict__ u32, uint2* __restrict__ u16) {
    pdl_enter();
    const int par = blockIdx.y;
    for (int cb = blockIdx.x * blockDim.x + threadIdx.x; cb < g.Vh; cb += gridDim.x * blockDim.x) {
        const SiteX s = decode_site(g, cb, par);
        const long long gi = (long long)s.lex + g.L3;
#pragma unroll
        for (int mu = 0; mu < 4; ++mu) {
            const double2* src = canon + (gi * 4 + mu) * 9;
            double2 m[9];
#pragma unroll
            for (int k = 0; k < 9; ++k) {
                const double2 v = src[k];
                m[k] = (mu == 0) ? v : make_double2(g.ph_re * v.x - g.ph_im * v.y, g.ph_re * v.y + g.ph_im * v.x);
            }
            const long long pl = (long long)(mu * 2 + par);
            const long long b9 = pl * 9 * g.Vpad + cb;
#pragma unroll
            for (int k = 0; k < 9; ++k) u64[b9 + (long long)k * g.Vpad] = m[k];
            const long long b3 = pl * 3 * g.Vpad + cb;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const double2 a = m[2 * k], b = m[2 * k + 1];
                u32[b3 + (long long)k * g.Vpad] = make_float4((float)a.x, (float)a.y, (float)b.x, (float)b.y);
                uint2 h;
                h.x = f2h((float)a.x, (float)a.y);
                h.y = f2h((float)b.x, (float)b.y);
                u16[b3 + (long long)k * g.Vpad] = h;
            }
        }
    }
}

cudaError_t launch_link_prep(const LatDev& g, const double* canon, cudaStream_t st) {
    const int blocks = (g.Vh + 255) / 256;
    launch_pdl(k_link_prep, dim3(dim3(blocks < 1 ? 1 : blocks, 2)), dim3(256), st, 
        g, reinterpret_cast<const double2*>(canon), const_cast<double2*>(g.u64), const_cast<float4*>(g.u32),
        const_cast<uint2*>(g.u16));
    return cudaGetLastError();
}

// ------------------------------------------------------------ SU(3) check
// max over links of max_ij |(U^dag U - 1)_ij| and |det U - 1|, as the bit
// patterns of non-negative doubles (atomicMax on them is order-preserving).
__global__ void k_su3_check(int L, int T, const double2* __restrict__ canon, unsigned long long* out) {
    pdl_enter();
    const long long L3 = (long long)L * L * L;
    const long long n = (long long)(T + 1) * L3 * 4;
    double e1 = 0.0, e2 = 0.0;
    bool bad = false;  // NaN or Inf anywhere (fmax would drop a NaN)
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int mu = (int)(i & 3);
        const long long gi = i >> 2;
        if (mu == 0 && gi >= (long long)T * L3) continue;  // no time link leaves x0 = T
        cpx<double> U[3][3];
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            const double2 v = canon[i * 9 + k];
            U[k / 3][k % 3] = cpx<double>{v.x, v.y};
            if (!(fabs(v.x) <= 1e300) || !(fabs(v.y) <= 1e300)) bad = true;
        }
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                cpx<double> t{0, 0};
                for (int k = 0; k < 3; ++k) cfmac(t, U[k][a], U[k][b]);
                if (a == b) t.re -= 1.0;
                e1 = fmax(e1, fabs(t.re) + fabs(t.im));
            }
        const cpx<double> det = U[0][0] * (U[1][1] * U[2][2] - U[1][2] * U[2][1]) -
                                U[0][1] * (U[1][0] * U[2][2] - U[1][2] * U[2][0]) +
                                U[0][2] * (U[1][0] * U[2][1] - U[1][1] * U[2][0]);
        e2 = fmax(e2, fabs(det.re - 1.0) + fabs(det.im));
    }
    if (bad || !(e1 == e1)) e1 = 1e300;
    if (bad || !(e2 == e2)) e2 = 1e300;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        e1 = fmax(e1, __shfl_down_sync(0xffffffffu, e1, off));
        e2 = fmax(e2, __shfl_down_sync(0xffffffffu, e2, off));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(out, (unsigned long long)__double_as_longlong(e1));
        atomicMax(out + 1, (unsigned long long)__double_as_longlong(e2));
    }
}

cudaError_t launch_su3_check(int L, int T, const double* canon, unsigned long long* out2, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(out2, 0, 2 * sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    launch_pdl(k_su3_check, dim3(4 * 152), dim3(256), st, L, T, reinterpret_cast<const double2*>(canon), out2);
    return cudaGetLastError();
}

// ------------------------------------------------------------ plaquette
// S_g = beta sum_p w(p) (1 - Re tr U_p / 3) over the SF gauge lattice
// x0 = 0..T; w = 1/2 for spatial plaquettes on x0 = 0 and x0 = T, 1 otherwise
// (c_t = 1).  Deterministic: fixed per-block tree, last block sums partials
// in block order.
__device__ __forceinline__ void ld_link(const double2* canon, long long gi, int mu, cpx<double> (&U)[3][3]) {
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        const double2 v = __ldg(canon + (gi * 4 + mu) * 9 + k);
        U[k / 3][k % 3] = cpx<double>{v.x, v.y};
    }
}

__global__ void __launch_bounds__(256) k_plaquette(int L, int T, double beta, const double2* __restrict__ canon,
                                                   double* __restrict__ partials, unsigned* counter,
                                                   double* out) {
    __shared__ double sw[8];
    __shared__ int is_last;
    const long long L3 = (long long)L * L * L;
    const long long n = (long long)(T + 1) * L3;
    double acc = 0.0;
    for (long long gi = blockIdx.x * (long long)blockDim.x + threadIdx.x; gi < n;
         gi += (long long)gridDim.x * blockDim.x) {
        long long r = gi;
        int x[4];
        x[3] = (int)(r % L); r /= L;
        x[2] = (int)(r % L); r /= L;
        x[1] = (int)(r % L); r /= L;
        x[0] = (int)r;
        for (int mu = 0; mu < 4; ++mu)
            for (int nu = mu + 1; nu < 4; ++nu) {
                double w = 1.0;
                if (mu == 0) {
                    if (x[0] > T - 1) continue;
                } else if (x[0] == 0 || x[0] == T) {
                    w = 0.5;
                }
                int xm[4] = {x[0], x[1], x[2], x[3]}, xn[4] = {x[0], x[1], x[2], x[3]};
                if (mu == 0) xm[0] += 1; else xm[mu] = (xm[mu] + 1) % L;
                xn[nu] = (xn[nu] + 1) % L;
                const long long gm = (((long long)xm[0] * L + xm[1]) * L + xm[2]) * L + xm[3];
                const long long gn = (((long long)xn[0] * L + xn[1]) * L + xn[2]) * L + xn[3];
                cpx<double> A[3][3], B[3][3], C[3][3], D[3][3];
                ld_link(canon, gi, mu, A);
                ld_link(canon, gm, nu, B);
                ld_link(canon, gn, mu, C);
                ld_link(canon, gi, nu, D);
                // tr[A B C^dag D^dag] = sum_{abcd} A_ab B_bc conj(C_dc) conj(D_ad)
                cpx<double> AB[3][3];
                for (int a = 0; a < 3; ++a)
                    for (int c = 0; c < 3; ++c) {
                        cpx<double> t{0, 0};
                        for (int b = 0; b < 3; ++b) cfma(t, A[a][b], B[b][c]);
                        AB[a][c] = t;
                    }
                double tr = 0.0;
                for (int a = 0; a < 3; ++a)
                    for (int c = 0; c < 3; ++c) {
                        // (C^dag D^dag)_{ca} = sum_d conj(C_dc) conj(D_ad)
                        cpx<double> t{0, 0};
                        for (int d = 0; d < 3; ++d) t = t + conj(C[d][c]) * conj(D[a][d]);
                        tr += (AB[a][c] * t).re;
                    }
                acc += w * (1.0 - tr / 3.0);
            }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
    if ((threadIdx.x & 31) == 0) sw[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += sw[k];
        partials[blockIdx.x] = s;
        __threadfence();
        is_last = (atomicAdd(counter, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (is_last && threadIdx.x < 32) {
        __threadfence();
        double s = 0.0;
        for (int b = threadIdx.x; b < (int)gridDim.x; b += 32) s += __ldcg(partials + b);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
        if (threadIdx.x == 0) {
            *out = beta * s;
            *counter = 0u;
        }
    }
}

cudaError_t launch_plaquette(int L, int T, double beta, const double* canon, double* partials, unsigned* counter,
                             double* out, cudaStream_t st) {
    const long long n = (long long)(T + 1) * L * L * L;
    int blocks = (int)((n + 255) / 256);
    if (blocks > 2 * 152) blocks = 2 * 152;
    k_plaquette<<<blocks, 256, 0, st>>>(L, T, beta, reinterpret_cast<const double2*>(canon), partials, counter, out);
    return cudaGetLastError();
}

// ------------------------------------------------------------ force
// For the link U_mu(x) with both ends on the fermion lattice:
//   M1 = sum_i sum_s Xh_i(x+mu)_s [(1-gamma_mu) Yh_i(x)]_s^dag
//   M2 = sum_i sum_s Xh_i(x)_s    [(1+gamma_mu) Yh_i(x+mu)]_s^dag
//   W  = lambda U M1 - lambda^* M2 U^dag,
//   F^a = -2 kappa Im tr[T^a W] = -kappa Im tr[lambda^a W]  (lambda^a Gell-Mann).
// Because (1 -+ gamma_mu) = sum_k v_k v_k^dag with the two spin vectors that
// define the half spinors of the hop, each spin sum is two colour outer
// products of half spinors: M = sum_k h_k(X) h_k(Y)^dag.
template <int MU>
__device__ __forceinline__ void force_dir(const LatDev& g, const SiteX& s, int cb, int par, int nrhs,
                                          const CField<P64>& xs, const CField<P64>& ys,  // at x (parity par)
                                          const CField<P64>& xn, const CField<P64>& yn,  // at x+mu
                                          double* __restrict__ F, double* __restrict__ mom, double eps) {
    if (MU == 0 && s.x0 >= g.T - 1) return;  // the time link into x0 = T has no fermion force
    const int ncb = neighbour_cb<MU, +1>(g, s);
    cpx<double> M1[3][3], M2[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) M1[a][b] = M2[a][b] = cpx<double>{0, 0};
    for (int i = 0; i < nrhs; ++i) {
        const long long vb = vbase<P64>(g, i);
        cpx<double> p[4][3], hX[2][3], hY[2][3];
        load_spinor<P64, double>(xn, vb, g.Vpad, ncb, 0, p);
        project<MU, -1>(p, hX);
        load_spinor<P64, double>(ys, vb, g.Vpad, cb, 0, p);
        project<MU, -1>(p, hY);
#pragma unroll
        for (int k = 0; k < 2; ++k)
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int b = 0; b < 3; ++b) M1[a][b] = M1[a][b] + hX[k][a] * conj(hY[k][b]);
        load_spinor<P64, double>(xs, vb, g.Vpad, cb, 0, p);
        project<MU, +1>(p, hX);
        load_spinor<P64, double>(yn, vb, g.Vpad, ncb, 0, p);
        project<MU, +1>(p, hY);
#pragma unroll
        for (int k = 0; k < 2; ++k)
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int b = 0; b < 3; ++b) M2[a][b] = M2[a][b] + hX[k][a] * conj(hY[k][b]);
    }
    // the stored link is V = lambda U, so lambda U M1 = V M1 and
    // lambda^* M2 U^dag = M2 V^dag: W = V M1 - M2 V^dag
    Link<double> V;
    LinkLoad<P64>::load<MU>(g, par, cb, V);
    cpx<double> W[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            cpx<double> t1{0, 0}, t2{0, 0};
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                cfma(t1, V.m[a][k], M1[k][b]);
                t2 = t2 + M2[a][k] * conj(V.m[b][k]);
            }
            W[a][b] = t1 - t2;
        }
    const double r3 = 0.57735026918962576451;  // 1/sqrt(3)
    double f[8];
    // Im tr[lambda^a W] for the Gell-Mann matrices
    f[0] = W[1][0].im + W[0][1].im;
    f[1] = -W[1][0].re + W[0][1].re;
    f[2] = W[0][0].im - W[1][1].im;
    f[3] = W[2][0].im + W[0][2].im;
    f[4] = -W[2][0].re + W[0][2].re;
    f[5] = W[2][1].im + W[1][2].im;
    f[6] = -W[2][1].re + W[1][2].re;
    f[7] = r3 * (W[0][0].im + W[1][1].im - 2.0 * W[2][2].im);
    const long long gi = (long long)s.lex + g.L3;
    double* Fp = F + (gi * 4 + MU) * 8;
#pragma unroll
    for (int a = 0; a < 8; ++a) {
        const double fa = -g.kappa * f[a];
        if (F) Fp[a] = fa;
        if (mom) mom[(gi * 4 + MU) * 8 + a] -= eps * fa;
    }
}

__global__ void __launch_bounds__(128) k_force(const LatDev* __restrict__ lat, int nrhs, CField<P64> xe,
                                               CField<P64> xo, CField<P64> ye, CField<P64> yo, double* F,
                                               double* mom, double eps) {
    pdl_enter();
    const LatDev g = *lat;
    const int par = blockIdx.y;
    const CField<P64> xs = par ? xo : xe, ys = par ? yo : ye;
    const CField<P64> xn = par ? xe : xo, yn = par ? ye : yo;
    const int mu = blockIdx.z;  // one direction per grid layer: four times the threads of one per site
    for (int cb = blockIdx.x * blockDim.x + threadIdx.x; cb < g.Vh; cb += gridDim.x * blockDim.x) {
        const SiteX s = decode_site(g, cb, par);
        switch (mu) {
            case 0: force_dir<0>(g, s, cb, par, nrhs, xs, ys, xn, yn, F, mom, eps); break;
            case 1: force_dir<1>(g, s, cb, par, nrhs, xs, ys, xn, yn, F, mom, eps); break;
            case 2: force_dir<2>(g, s, cb, par, nrhs, xs, ys, xn, yn, F, mom, eps); break;
            default: force_dir<3>(g, s, cb, par, nrhs, xs, ys, xn, yn, F, mom, eps); break;
        }
    }
}

cudaError_t launch_force(const LaunchCfg& c, FieldPtr xe, FieldPtr xo, FieldPtr ye, FieldPtr yo, double* F,
                         double* mom, double eps, cudaStream_t st) {
    // c.lats points at this lattice's descriptor; Vh is read on the device, the
    // grid is sized from the host copy passed through nblocks.
    int blocks = c.nblocks;
    if (blocks < 1) blocks = 1;
    launch_pdl(k_force, dim3(dim3(blocks, 2, 4)), dim3(128), st, c.lats, c.nrhs, cf<P64>(xe), cf<P64>(xo), cf<P64>(ye), cf<P64>(yo),
                                             F, mom, eps);
    return cudaGetLastError();
}

// ------------------------------------------------------------ misc
__global__ void k_outer_check(int n, OState* __restrict__ ost, const double* __restrict__ rr,
                              const double* __restrict__ bb, int max_sweeps, int* n_active,
                              cudaGraphConditionalHandle cond, int use_cond, int* sweeps_run) {
    pdl_enter();
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int cnt = 0;
    for (int i = 0; i < n; ++i) {
        OState& o = ost[i];
        if (bb) o.bb = bb[i];
        const double r = rr[i];
        o.rr = r;
        const bool finite = (r == r) && (r < 1e300);
        const bool go = finite && (r > o.tol2 * o.bb) && (o.sweeps < max_sweeps) && (o.bb > 0.0);
        o.active = go ? 1 : 0;
        if (go) {
            o.inv_norm = 1.0 / sqrt(r);
            // solve the normalised inner system to max(delta, what the outer tolerance still needs)
            const double need2 = 0.01 * o.tol2 * o.bb / r;
            o.delta2 = fmax(o.delta2_floor, need2);
            ++cnt;
        }
    }
    *n_active = cnt;
    if (use_cond) {
        // the graph-resident solve: another sweep while any rhs is active
        if (cnt > 0 && sweeps_run) *sweeps_run += 1;
        cudaGraphSetConditional(cond, cnt > 0 ? 1u : 0u);
    }
}

cudaError_t launch_outer_check(int n, OState* ost, const double* rr, const double* bb, int max_sweeps,
                               int* n_active, cudaStream_t st, cudaGraphConditionalHandle cond, int use_cond,
                               int* sweeps_run) {
    launch_pdl(k_outer_check, dim3(1), dim3(32), st, n, ost, rr, bb, max_sweeps, n_active, cond, use_cond,
               sweeps_run);
    return cudaGetLastError();
}

// dst = src (or 0 when src is NULL), n doubles, as a kernel: the copies
// inside the graph-resident solve stay kernel nodes
__global__ void k_copy_f64(double* __restrict__ dst, const double* __restrict__ src, long long n) {
    pdl_enter();
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        dst[i] = src ? src[i] : 0.0;
}

cudaError_t launch_copy_f64(double* dst, const double* src, long long n, int sm_count, cudaStream_t st) {
    const long long want = (n + 255) / 256;
    const int blocks = (int)std::max(1LL, std::min<long long>(want, 4LL * sm_count));
    launch_pdl(k_copy_f64, dim3(blocks), dim3(256), st, dst, src, n);
    return cudaGetLastError();
}

// |f_i|^2 per (lattice, rhs): block partials here, the sums by k_finish
template <int NR>
__global__ void __launch_bounds__(KB<P64, NR>::MAXT, KB<P64, NR>::MINB) k_norm2(const LatDev* __restrict__ lats, int nlat, int nrhs,
                                                CField<P64> f, SolverCtx ctx) {
    pdl_enter();
    const int l = find_lattice(lats, nlat, blockIdx.x);
    const LatDev g = lats[l];
    const int r0 = threadIdx.y * NR;
    const int nval = min(NR, nrhs - r0);
    double red[NR][1];
#pragma unroll
    for (int j = 0; j < NR; ++j) red[j][0] = 0.0;
    for (int tile = tile_begin(g), tile_end_ = tile_end(g); tile < tile_end_; ++tile) {
        const int cb = tile_cb(g, tile, threadIdx.x);
        if (cb < 0) continue;
#pragma unroll
        for (int j = 0; j < NR; ++j) {
            if (j >= nval) continue;
            cpx<double> a[4][3];
            load_spinor<P64, double>(f, vbase<P64>(g, r0 + j), g.Vpad, cb, 0, a);
            norm_acc(a, red[j][0]);
        }
    }
    block_partials<NR, 1>(red, nrhs, ctx.partials);
}

cudaError_t launch_norm2(const LaunchCfg& c, FieldPtr f, const SolverCtx* ctx, double* out, cudaStream_t st) {
    if (c.NR == 1)
        launch_pdl(k_norm2<1>, dim3(c.nblocks), dim3(block_of(c)), st, c.lats, c.nlat, c.nrhs, cf<P64>(f), *ctx);
    else if (c.NR == 2)
        launch_pdl(k_norm2<2>, dim3(c.nblocks), dim3(block_of(c)), st, c.lats, c.nlat, c.nrhs, cf<P64>(f), *ctx);
    else
        return cudaErrorInvalidValue;
    launch_finish<1, double, FIN_NORM, double>(c, *ctx, out, 0, st);
    return cudaGetLastError();
}

// ------------------------------------------------------------ FP64 BLAS for FGCR
// out[l*nrhs + i] = <a_i, b_i> (complex, sum conj(a) b) for every (lattice, rhs)
__global__ void __launch_bounds__(KB<P64, 1>::MAXT) k_dot64(const LatDev* __restrict__ lats, int nlat, int nrhs,
                                                          CField<P64> a, CField<P64> b, SolverCtx ctx) {
    pdl_enter();
    const int l = find_lattice(lats, nlat, blockIdx.x);
    const LatDev g = lats[l];
    const int r0 = threadIdx.y;
    double red[1][2] = {{0.0, 0.0}};
    if (r0 < nrhs) {
        for (int tile = tile_begin(g), te = tile_end(g); tile < te; ++tile) {
            const int cb = tile_cb(g, tile, threadIdx.x);
            if (cb < 0) continue;
            cpx<double> x[4][3], y[4][3];
            load_spinor<P64, double>(a, vbase<P64>(g, r0), g.Vpad, cb, 0, x);
            load_spinor<P64, double>(b, vbase<P64>(g, r0), g.Vpad, cb, 0, y);
            dotc_acc(x, y, red[0][0], red[0][1]);
        }
    }
    block_partials<1, 2>(red, nrhs, ctx.partials);
}

// y_i += sum_j c[j][i] x_j for nvec vectors x_j (coefficients per rhs, device)
__global__ void __launch_bounds__(KB<P64, 1>::MAXT) k_multi_axpy64(const LatDev* __restrict__ lats, int nlat, int nrhs,
                                                                 int nvec, const double2* const* __restrict__ xs,
                                                                 const double2* __restrict__ c, double2* __restrict__ y) {
    pdl_enter();
    const int l = find_lattice(lats, nlat, blockIdx.x);
    const LatDev g = lats[l];
    const int r0 = threadIdx.y;
    if (r0 >= nrhs) return;
    for (int tile = tile_begin(g), te = tile_end(g); tile < te; ++tile) {
        const int cb = tile_cb(g, tile, threadIdx.x);
        if (cb < 0) continue;
        const long long base = vbase<P64>(g, r0) + cb;
#pragma unroll
        for (int comp = 0; comp < 12; ++comp) {
            const long long idx = base + (long long)comp * g.Vpad;
            double2 acc = y[idx];
            for (int j = 0; j < nvec; ++j) {
                const double2 cj = c[j * nlat * nrhs + l * nrhs + r0];
                const double2 xv = xs[j][idx];
                acc.x += cj.x * xv.x - cj.y * xv.y;
                acc.y += cj.x * xv.y + cj.y * xv.x;
            }
            y[idx] = acc;
        }
    }
}

// ------------------------------------------------------------ FP64 block BLAS for Bl-BiCGStab
// Gram block G[i][j] = <a_i, b_j> (sum over the lattice of a_i^dag b_j) for
// all pairs of rhs of one lattice: thread (site, j) loads b_j once and runs
// over the a_i; per-block partials in the layout of block_partials with
// "rhs" j and quantity q = 2 i + (re, im).
template <int S>
__global__ void __launch_bounds__(KB<P64, 1>::MAXT) k_gram64(const LatDev* __restrict__ lats, int nlat, int nrhs,
                                                           CField<P64> a, CField<P64> b, double* __restrict__ partials) {
    pdl_enter();
    const int l = find_lattice(lats, nlat, blockIdx.x);
    const LatDev g = lats[l];
    const int j = threadIdx.y;
    double red[1][2 * S];
#pragma unroll
    for (int q = 0; q < 2 * S; ++q) red[0][q] = 0.0;
    if (j < nrhs) {
        for (int tile = tile_begin(g), te = tile_end(g); tile < te; ++tile) {
            const int cb = tile_cb(g, tile, threadIdx.x);
            if (cb < 0) continue;
            cpx<double> y[4][3];
            load_spinor<P64, double>(b, vbase<P64>(g, j), g.Vpad, cb, 0, y);
#pragma unroll
            for (int i = 0; i < S; ++i) {
                if (i >= nrhs) break;
                cpx<double> x[4][3];
                load_spinor<P64, double>(a, vbase<P64>(g, i), g.Vpad, cb, 0, x);
                dotc_acc(x, y, red[0][2 * i], red[0][2 * i + 1]);
            }
        }
    }
    block_partials<1, 2 * S>(red, nrhs, partials);
}

// the lattice sums of the Gram partials: out[(j * 2S + 2i) + (0, 1)] = G[i][j]
// (one block, lattice 0)
template <int S>
__global__ void __launch_bounds__(FIN_THREADS) k_gram64_finish(const LatDev* __restrict__ lats, int nrhs,
                                                               int nblocks, const double* __restrict__ partials,
                                                               double* __restrict__ out) {
    pdl_enter();
    __shared__ double sres[MAX_RHS * 2 * S];
    lattice_sums<2 * S, double>(partials, nrhs, nblocks, lats[0].blk0, lats[0].nblk, threadIdx.x, (int)blockDim.x,
                                sres);
    __syncthreads();
    for (int r = threadIdx.x; r < nrhs * 2 * S; r += blockDim.x) out[r] = sres[r];
}

// Y_j += sum_i X_i C[i * nrhs + j] for every column j (C an nrhs x nrhs
// complex matrix, device; X and Y distinct fields)
__global__ void __launch_bounds__(KB<P64, 1>::MAXT) k_block_axpy64(const LatDev* __restrict__ lats, int nlat,
                                                                 int nrhs, const double2* __restrict__ x,
                                                                 const double2* __restrict__ c,
                                                                 double2* __restrict__ y) {
    pdl_enter();
    const int l = find_lattice(lats, nlat, blockIdx.x);
    const LatDev g = lats[l];
    const int j = threadIdx.y;
    if (j >= nrhs) return;
    for (int tile = tile_begin(g), te = tile_end(g); tile < te; ++tile) {
        const int cb = tile_cb(g, tile, threadIdx.x);
        if (cb < 0) continue;
        const long long yb = vbase<P64>(g, j) + cb;
        double2 acc[12];
#pragma unroll
        for (int comp = 0; comp < 12; ++comp) acc[comp] = y[yb + (long long)comp * g.Vpad];
        for (int i = 0; i < nrhs; ++i) {
            const double2 ci = c[i * nrhs + j];
            const long long xb = vbase<P64>(g, i) + cb;
#pragma unroll
            for (int comp = 0; comp < 12; ++comp) {
                const double2 xv = __ldg(x + xb + (long long)comp * g.Vpad);
                acc[comp].x += ci.x * xv.x - ci.y * xv.y;
                acc[comp].y += ci.x * xv.y + ci.y * xv.x;
            }
        }
#pragma unroll
        for (int comp = 0; comp < 12; ++comp) y[yb + (long long)comp * g.Vpad] = acc[comp];
    }
}

cudaError_t launch_gram64(const LaunchCfg& c, FieldPtr a, FieldPtr b, double* partials, double* out,
                          cudaStream_t st) {
    if (c.nlat != 1 || c.nrhs > MAX_RHS) return cudaErrorInvalidValue;
    if (c.nrhs <= 8) {
        launch_pdl(k_gram64<8>, dim3(c.nblocks), dim3(dim3(c.TS, c.nrhs)), st, c.lats, c.nlat, c.nrhs, cf<P64>(a),
                   cf<P64>(b), partials);
        if (out)
            launch_pdl(k_gram64_finish<8>, dim3(1), dim3(FIN_THREADS), st, c.lats, c.nrhs, c.nblocks,
                       (const double*)partials, out);
    } else {
        launch_pdl(k_gram64<16>, dim3(c.nblocks), dim3(dim3(c.TS, c.nrhs)), st, c.lats, c.nlat, c.nrhs, cf<P64>(a),
                   cf<P64>(b), partials);
        if (out)
            launch_pdl(k_gram64_finish<16>, dim3(1), dim3(FIN_THREADS), st, c.lats, c.nrhs, c.nblocks,
                       (const double*)partials, out);
    }
    return cudaGetLastError();
}

cudaError_t launch_block_axpy64(const LaunchCfg& c, FieldPtr x, const double2* coef, FieldPtr y, cudaStream_t st) {
    launch_pdl(k_block_axpy64, dim3(c.nblocks), dim3(dim3(c.TS, c.nrhs)), st, c.lats, c.nlat, c.nrhs,
               reinterpret_cast<const double2*>(x.v), coef, reinterpret_cast<double2*>(y.v));
    return cudaGetLastError();
}

// out = gamma_5 in (spin components 2, 3 negated)
__global__ void k_gamma5_64(long long n_per_rhs_planes, int Vpad, const double2* __restrict__ in, double2* __restrict__ out,
                            long long total) {
    pdl_enter();
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        const int comp = (int)((i / Vpad) % 12);
        const double2 v = in[i];
        out[i] = (comp >= 6) ? make_double2(-v.x, -v.y) : v;
    }
    (void)n_per_rhs_planes;
}

cudaError_t launch_dot64(const LaunchCfg& c, FieldPtr a, FieldPtr b, const SolverCtx* ctx, double2* out,
                         cudaStream_t st) {
    launch_pdl(k_dot64, dim3(c.nblocks), dim3(dim3(c.TS, c.nrhs)), st, c.lats, c.nlat, c.nrhs, cf<P64>(a), cf<P64>(b), *ctx);
    launch_finish<2, double, FIN_DOT, double>(c, *ctx, reinterpret_cast<double*>(out), 0, st);
    return cudaGetLastError();
}

cudaError_t launch_multi_axpy64(const LaunchCfg& c, int nvec, const double2* const* xs, const double2* coef,
                                FieldPtr y, cudaStream_t st) {
    launch_pdl(k_multi_axpy64, dim3(c.nblocks), dim3(dim3(c.TS, c.nrhs)), st, c.lats, c.nlat, c.nrhs, nvec, xs, coef,
                                                            reinterpret_cast<double2*>(y.v));
    return cudaGetLastError();
}

cudaError_t launch_gamma5_64(long long total_elems, int Vpad, FieldPtr in, FieldPtr out, cudaStream_t st) {
    launch_pdl(k_gamma5_64, dim3(4 * 152), dim3(256), st, 0, Vpad, reinterpret_cast<const double2*>(in.v),
                                          reinterpret_cast<double2*>(out.v), total_elems);
    return cudaGetLastError();
}

}  // namespace sf
