// Device-resident Bl-BiCGStab and Gl-BiCGStab (Sec. 3.2, Table 1 cases C and
// D1): the fused field updates and the one-block finishing kernels that take
// every decision of the outer iteration on the device.  The host captures
// them, with the FP64 Dhat applications and (Gl) the FP32 preconditioner
// solves, into one CUDA graph per solve (api.cu).
#include "blocksolve.h"
#include "krylov_impl.cuh"

namespace sf {
namespace {

__device__ __forceinline__ double2 c_add(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 c_sub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 c_mul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// conj(a) b
__device__ __forceinline__ double2 c_cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ double2 c_scale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
// a / b by Smith's scaled division
__device__ __forceinline__ double2 c_div(double2 a, double2 b) {
    if (fabs(b.x) >= fabs(b.y)) {
        const double r = b.y / b.x, d = b.x + r * b.y;
        return make_double2((a.x + r * a.y) / d, (a.y - r * a.x) / d);
    }
    const double r = b.x / b.y, d = b.y + r * b.x;
    return make_double2((a.x * r + a.y) / d, (a.y * r - a.x) / d);
}
__device__ __forceinline__ double c_abs(double2 a) { return hypot(a.x, a.y); }

// Lattice sums of NQ quantities per rhs (one lattice, blocks 0 .. nblocks-1)
// into sres[rhs * NQ + q]; every thread of the block calls it.
template <int NQ>
__device__ __forceinline__ void fin_sums(const double* partials, int n, int nblocks, double* sres) {
    lattice_sums<NQ, double>(partials, n, nblocks, 0, nblocks, (int)threadIdx.x, (int)blockDim.x, sres);
    __syncthreads();
}

constexpr int QW = 2 * BLK_MAX;   // row stride of the [M | I] working matrix

// Householder QR of the n x n matrix in the left half of sA ([n][QW], left
// half M, right half the identity), one warp: lane c keeps column c of
// [M | I]; reflection k (built by lane 0 from column k, H = I - v v^H /
// (sigma (sigma + |x0|)), v = x + e^{i arg x0} sigma e_0) is applied by every
// lane to its own column.  Afterwards the left half holds R and the right
// half Q^H (M = Q R).  False if a column norm sigma_k falls to 1e-14 |M|_F
// or below (the block has lost rank: breakdown).
__device__ bool warp_qr(double2* sA, int n) {
    const int lane = threadIdx.x & 31;
    __shared__ double2 sv[BLK_MAX];
    __shared__ double sc;
    __shared__ int sbad;
    __shared__ double sfro;
    if (lane == 0) {
        double f = 0.0;
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) f += sA[i * QW + j].x * sA[i * QW + j].x + sA[i * QW + j].y * sA[i * QW + j].y;
        sfro = sqrt(f);
        sbad = 0;
    }
    __syncwarp();
    for (int k = 0; k < n; ++k) {
        if (lane == 0) {
            double s2 = 0.0;
            for (int i = k; i < n; ++i) s2 += sA[i * QW + k].x * sA[i * QW + k].x + sA[i * QW + k].y * sA[i * QW + k].y;
            const double sigma = sqrt(s2);
            const double2 x0 = sA[k * QW + k];
            const double ax0 = c_abs(x0);
            if (!(sigma > 1e-14 * sfro)) {
                sbad = 1;
            } else {
                const double2 ph = ax0 > 0.0 ? c_scale(x0, 1.0 / ax0) : make_double2(1.0, 0.0);
                sv[k] = c_add(x0, c_scale(ph, sigma));
                for (int i = k + 1; i < n; ++i) sv[i] = sA[i * QW + k];
                sc = 1.0 / (sigma * (sigma + ax0));
            }
        }
        __syncwarp();
        if (sbad) return false;
        if (lane >= k && lane < 2 * n) {
            double2 w = make_double2(0.0, 0.0);
            for (int i = k; i < n; ++i) w = c_add(w, c_cmul(sv[i], sA[i * QW + lane]));
            w = c_scale(w, sc);
            for (int i = k; i < n; ++i) sA[i * QW + lane] = c_sub(sA[i * QW + lane], c_mul(sv[i], w));
        }
        __syncwarp();
    }
    return true;
}

// X = M^-1 B = R^-1 (Q^H B) for the n x n matrix B (sB, stride BLK_MAX),
// from the factors in sA; lane c < n solves column c; the result replaces sB.
__device__ void warp_qr_solve(const double2* sA, double2* sB, int n) {
    const int c = threadIdx.x & 31;
    if (c < n) {
        double2 y[BLK_MAX];
#pragma unroll
        for (int i = 0; i < BLK_MAX; ++i) {
            y[i] = make_double2(0.0, 0.0);
            if (i < n)
                for (int l = 0; l < n; ++l) y[i] = c_add(y[i], c_mul(sA[i * QW + n + l], sB[l * BLK_MAX + c]));
        }
#pragma unroll
        for (int i = BLK_MAX - 1; i >= 0; --i) {
            if (i >= n) continue;
            double2 v = y[i];
#pragma unroll
            for (int l = i + 1; l < BLK_MAX; ++l)
                if (l < n) v = c_sub(v, c_mul(sA[i * QW + l], y[l]));
            y[i] = c_div(v, sA[i * QW + i]);
        }
#pragma unroll
        for (int i = 0; i < BLK_MAX; ++i)
            if (i < n) sB[i * BLK_MAX + c] = y[i];
    }
    __syncwarp();
}

__device__ __forceinline__ void set_cond(cudaGraphConditionalHandle h, bool v) {
    cudaGraphSetConditional(h, v ? 1u : 0u);
}

}  // namespace

// ====================================================================== Bl-BiCGStab
__global__ void k_bl_init(BlState* st, int n, const double* __restrict__ bb, double tol, int maxiter, int max_cycles,
                          cudaGraphConditionalHandle h_cycle) {
    pdl_enter();
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    st->n = n;
    for (int j = 0; j < n; ++j) {
        st->bb[j] = bb[j];
        st->rr[j] = bb[j];
    }
    st->stop2 = 0.25 * tol * tol;
    st->tol2 = tol * tol;
    st->iters = 0;
    st->maxiter = maxiter;
    st->cycles = 0;
    st->max_cycles = max_cycles;
    st->stop = 0;
    st->fail = 0;
    st->body_runs = 0;
    st->if_runs = 0;
    set_cond(h_cycle, true);
}

// every rhs's recursive residual below tol / 2 (a zero rhs counts as converged)
__device__ __forceinline__ bool all_below(const double* rr, const double* bb, int n, double stop2, int stride) {
    bool ok = true;
    for (int j = 0; j < n; ++j) ok = ok && (rr[j * stride] <= stop2 * bb[j]);
    return ok;
}

__global__ void __launch_bounds__(FIN_THREADS) k_bl_fin_q(BlState* st, const double* __restrict__ partials, int nblocks,
                                                          cudaGraphConditionalHandle h_iter) {
    pdl_enter();
    __shared__ double sres[BLK_MAX * 2 * BLK_MAX];
    const int n = st->n;
    fin_sums<2 * BLK_MAX>(partials, n, nblocks, sres);
    if (threadIdx.x == 0) {
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j)
                st->Q[i * BLK_MAX + j] = make_double2(sres[j * 2 * BLK_MAX + 2 * i], sres[j * 2 * BLK_MAX + 2 * i + 1]);
        for (int j = 0; j < n; ++j) st->rr[j] = sres[j * 2 * BLK_MAX + 2 * j];
        const bool stop = all_below(st->rr, st->bb, n, st->stop2, 1);
        st->stop = stop ? 1 : 0;
        st->cycles += 1;
        set_cond(h_iter, !stop && st->iters < st->maxiter);
    }
}

__global__ void __launch_bounds__(FIN_THREADS) k_bl_fin_alpha(BlState* st, const double* __restrict__ partials,
                                                              int nblocks) {
    pdl_enter();
    if (st->stop) return;
    __shared__ double sres[BLK_MAX * 2 * BLK_MAX];
    __shared__ double2 sA[BLK_MAX * QW];
    __shared__ double2 sB[BLK_MAX * BLK_MAX];
    const int n = st->n;
    fin_sums<2 * BLK_MAX>(partials, n, nblocks, sres);
    if (threadIdx.x >= 32) return;
    const int lane = threadIdx.x;
    for (int e = lane; e < n * n; e += 32) {
        const int i = e / n, j = e % n;
        const double2 m = make_double2(sres[j * 2 * BLK_MAX + 2 * i], sres[j * 2 * BLK_MAX + 2 * i + 1]);
        st->M[i * BLK_MAX + j] = m;
        sA[i * QW + j] = m;
        sA[i * QW + n + j] = make_double2(i == j ? 1.0 : 0.0, 0.0);
        sB[i * BLK_MAX + j] = st->Q[i * BLK_MAX + j];
    }
    __syncwarp();
    if (!warp_qr(sA, n)) {
        if (lane == 0) {
            st->stop = 1;
            st->fail += 1;
        }
        return;
    }
    warp_qr_solve(sA, sB, n);
    for (int e = lane; e < n * n; e += 32) {
        const int i = e / n, j = e % n;
        st->alpha[i * BLK_MAX + j] = sB[i * BLK_MAX + j];
        st->Rf[i * BLK_MAX + j] = sA[i * QW + j];
        st->Qh[i * BLK_MAX + j] = sA[i * QW + n + j];
    }
    if (lane == 0) st->iters += 1;
}

__global__ void __launch_bounds__(FIN_THREADS) k_bl_fin_s(BlState* st, const double* __restrict__ partials, int nblocks,
                                                          cudaGraphConditionalHandle h_if) {
    pdl_enter();
    if (st->stop) {
        if (threadIdx.x == 0) set_cond(h_if, false);
        return;
    }
    __shared__ double sres[BLK_MAX];
    const int n = st->n;
    fin_sums<1>(partials, n, nblocks, sres);
    if (threadIdx.x == 0) {
        for (int j = 0; j < n; ++j) st->rr[j] = sres[j];
        const bool below = all_below(sres, st->bb, n, st->stop2, 1);
        if (below) st->stop = 1;
        set_cond(h_if, !below);
    }
}

__global__ void __launch_bounds__(FIN_THREADS) k_bl_fin_omega(BlState* st, const double* __restrict__ partials,
                                                              int nblocks) {
    pdl_enter();
    __shared__ double sres[BLK_MAX * 3];
    const int n = st->n;
    fin_sums<3>(partials, n, nblocks, sres);
    if (threadIdx.x == 0) {
        st->if_runs += 1;
        double2 ts = make_double2(0.0, 0.0);
        double tt = 0.0;
        for (int j = 0; j < n; ++j) {
            ts = c_add(ts, make_double2(sres[3 * j], sres[3 * j + 1]));
            tt += sres[3 * j + 2];
        }
        if (tt > 0.0) {
            st->omega = c_scale(ts, 1.0 / tt);
        } else {   // T = 0: keep X + P alpha, R = S; the cycle's true residual decides
            st->omega = make_double2(0.0, 0.0);
            st->stop = 1;
            st->fail += 1;
        }
    }
}

__global__ void __launch_bounds__(FIN_THREADS) k_bl_fin_r(BlState* st, const double* __restrict__ partials, int nblocks) {
    pdl_enter();
    if (st->stop) return;
    __shared__ double sres[BLK_MAX * BLK_NQ_R];
    __shared__ double2 sA[BLK_MAX * QW];
    __shared__ double2 sB[BLK_MAX * BLK_MAX];
    __shared__ int sgo;
    const int n = st->n;
    fin_sums<BLK_NQ_R>(partials, n, nblocks, sres);
    if (threadIdx.x >= 32) return;
    const int lane = threadIdx.x;
    if (lane == 0) {
        for (int j = 0; j < n; ++j) st->rr[j] = sres[j * BLK_NQ_R];
        int go = 1;
        if (all_below(sres, st->bb, n, st->stop2, BLK_NQ_R)) {
            go = 0;
        } else if (st->omega.x == 0.0 && st->omega.y == 0.0) {
            go = 0;
            st->fail += 1;
        }
        if (!go) st->stop = 1;
        sgo = go;
    }
    __syncwarp();
    if (!sgo) return;
    for (int e = lane; e < n * n; e += 32) {
        const int i = e / n, j = e % n;
        st->Q[i * BLK_MAX + j] = make_double2(sres[j * BLK_NQ_R + 1 + 2 * i], sres[j * BLK_NQ_R + 2 + 2 * i]);
        sB[i * BLK_MAX + j] = make_double2(-sres[j * BLK_NQ_R + 1 + 2 * BLK_MAX + 2 * i],
                                           -sres[j * BLK_NQ_R + 2 + 2 * BLK_MAX + 2 * i]);
        sA[i * QW + j] = st->Rf[i * BLK_MAX + j];
        sA[i * QW + n + j] = st->Qh[i * BLK_MAX + j];
    }
    __syncwarp();
    warp_qr_solve(sA, sB, n);
    for (int e = lane; e < n * n; e += 32) {
        const int i = e / n, j = e % n;
        st->beta[i * BLK_MAX + j] = sB[i * BLK_MAX + j];
    }
}

__global__ void k_bl_cycle(BlState* st, const double* __restrict__ rr, cudaGraphConditionalHandle h_cycle) {
    pdl_enter();
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int n = st->n;
    bool ok = true;
    for (int j = 0; j < n; ++j) {
        st->rr[j] = rr[j];
        ok = ok && (rr[j] <= st->tol2 * st->bb[j] || st->bb[j] == 0.0);
    }
    st->stop = 0;
    set_cond(h_cycle, !ok && st->cycles < st->max_cycles && st->iters < st->maxiter);
}

// S_j = R_j - sum_i V_i alpha[i][j], X_j += sum_i P_i alpha[i][j], |S_j|^2:
// thread (site, j) reads R_j, X_j and every V_i, P_i of its site (the other
// rhs' rows come from L1 / L2: the block holds all rhs of its tile)
__global__ void __launch_bounds__(KB<P64, 1>::MAXT) k_bl_s(const LatDev* __restrict__ lats, const BlState* st,
                                                         const double2* __restrict__ R, const double2* __restrict__ V,
                                                         const double2* __restrict__ P, double2* __restrict__ S,
                                                         double2* __restrict__ X, double* __restrict__ partials) {
    pdl_enter();
    if (st->stop) return;
    __shared__ double2 sal[BLK_MAX * BLK_MAX];
    const int n = st->n, j = threadIdx.y;
    for (int e = threadIdx.y * blockDim.x + threadIdx.x; e < BLK_MAX * BLK_MAX; e += blockDim.x * blockDim.y)
        sal[e] = st->alpha[e];
    __syncthreads();
    const LatDev g = lats[0];
    double red[1][1] = {{0.0}};
    for (int tile = tile_begin(g), te = tile_end(g); tile < te; ++tile) {
        const int cb = tile_cb(g, tile, threadIdx.x);
        if (cb < 0) continue;
        const long long bj = vbase<P64>(g, j) + cb;
        for (int comp = 0; comp < 12; ++comp) {
            const long long o = (long long)comp * g.Vpad;
            double2 s = R[bj + o], x = X[bj + o];
            for (int i = 0; i < n; ++i) {
                const long long bi = vbase<P64>(g, i) + cb + o;
                const double2 a = sal[i * BLK_MAX + j];
                s = c_sub(s, c_mul(V[bi], a));
                x = c_add(x, c_mul(P[bi], a));
            }
            S[bj + o] = s;
            X[bj + o] = x;
            red[0][0] += s.x * s.x + s.y * s.y;
        }
    }
    block_partials<1, 1>(red, n, partials);
}

// X_j += omega S_j, R_j = S_j - omega T_j; |R_j|^2, <R0_i, R_j>, <R0_i, T_j>
__global__ void __launch_bounds__(KB<P64, 1>::MAXT) k_bl_r(const LatDev* __restrict__ lats, const BlState* st,
                                                         const double2* __restrict__ S, const double2* __restrict__ T,
                                                         const double2* __restrict__ R0, double2* __restrict__ X,
                                                         double2* __restrict__ R, double* __restrict__ partials) {
    pdl_enter();
    const int n = st->n, j = threadIdx.y;
    const double2 om = st->omega;
    const LatDev g = lats[0];
    double red[1][BLK_NQ_R];
#pragma unroll
    for (int q = 0; q < BLK_NQ_R; ++q) red[0][q] = 0.0;
    for (int tile = tile_begin(g), te = tile_end(g); tile < te; ++tile) {
        const int cb = tile_cb(g, tile, threadIdx.x);
        if (cb < 0) continue;
        const long long bj = vbase<P64>(g, j) + cb;
        for (int comp = 0; comp < 12; ++comp) {
            const long long o = (long long)comp * g.Vpad;
            const double2 s = S[bj + o], t = T[bj + o];
            X[bj + o] = c_add(X[bj + o], c_mul(om, s));
            const double2 r = c_sub(s, c_mul(om, t));
            R[bj + o] = r;
            red[0][0] += r.x * r.x + r.y * r.y;
#pragma unroll
            for (int i = 0; i < BLK_MAX; ++i) {
                if (i >= n) break;
                const double2 z = R0[vbase<P64>(g, i) + cb + o];
                const double2 zr = c_cmul(z, r), zt = c_cmul(z, t);
                red[0][1 + 2 * i] += zr.x;
                red[0][2 + 2 * i] += zr.y;
                red[0][1 + 2 * BLK_MAX + 2 * i] += zt.x;
                red[0][2 + 2 * BLK_MAX + 2 * i] += zt.y;
            }
        }
    }
    block_partials<1, BLK_NQ_R>(red, n, partials);
}

// P_j = R_j + sum_i (P_i - omega V_i) beta[i][j] in place: the block stages
// W_i = P_i - omega V_i of its tile (all rhs, half the components at a time)
// in shared memory before any thread overwrites P; block 0 sets the
// iteration loop's condition
constexpr int BLP_HALF = 6;
__global__ void __launch_bounds__(KB<P64, 1>::MAXT) k_bl_p(const LatDev* __restrict__ lats, BlState* st,
                                                         double2* __restrict__ P, const double2* __restrict__ V,
                                                         const double2* __restrict__ R,
                                                         cudaGraphConditionalHandle h_iter) {
    pdl_enter();
    const int stop = st->stop;
    if (blockIdx.x == 0 && threadIdx.x == 0 && threadIdx.y == 0) {
        st->body_runs += 1;
        set_cond(h_iter, !stop && st->iters < st->maxiter);
    }
    if (stop) return;
    __shared__ double2 sbeta[BLK_MAX * BLK_MAX];
    __shared__ double2 sw[BLK_MAX][BLP_HALF][32];
    const int n = st->n, j = threadIdx.y, tx = threadIdx.x;
    for (int e = threadIdx.y * blockDim.x + threadIdx.x; e < BLK_MAX * BLK_MAX; e += blockDim.x * blockDim.y)
        sbeta[e] = st->beta[e];
    const double2 om = st->omega;
    __syncthreads();
    const LatDev g = lats[0];
    for (int tile = tile_begin(g), te = tile_end(g); tile < te; ++tile) {
        const int cb = tile_cb(g, tile, tx);
        const long long bj = vbase<P64>(g, j) + cb;
        for (int h = 0; h < 12; h += BLP_HALF) {
            if (cb >= 0)
                for (int c = 0; c < BLP_HALF; ++c) {
                    const long long o = (long long)(h + c) * g.Vpad;
                    sw[j][c][tx] = c_sub(P[bj + o], c_mul(om, V[bj + o]));
                }
            __syncthreads();
            if (cb >= 0)
                for (int c = 0; c < BLP_HALF; ++c) {
                    const long long o = (long long)(h + c) * g.Vpad;
                    double2 p = R[bj + o];
                    for (int i = 0; i < n; ++i) p = c_add(p, c_mul(sw[i][c][tx], sbeta[i * BLK_MAX + j]));
                    P[bj + o] = p;
                }
            __syncthreads();
        }
    }
}

cudaError_t launch_bl_init(BlState* st, int n, const double* bb, double tol, int maxiter, int max_cycles,
                           cudaGraphConditionalHandle h_cycle, cudaStream_t s) {
    if (n < 1 || n > BLK_MAX) return cudaErrorInvalidValue;
    launch_pdl(k_bl_init, dim3(1), dim3(32), s, st, n, bb, tol, maxiter, max_cycles, h_cycle);
    return cudaGetLastError();
}
cudaError_t launch_bl_fin_q(BlState* st, const double* partials, int nblocks, cudaGraphConditionalHandle h_iter,
                            cudaStream_t s) {
    launch_pdl(k_bl_fin_q, dim3(1), dim3(FIN_THREADS), s, st, partials, nblocks, h_iter);
    return cudaGetLastError();
}
cudaError_t launch_bl_fin_alpha(BlState* st, const double* partials, int nblocks, cudaStream_t s) {
    launch_pdl(k_bl_fin_alpha, dim3(1), dim3(FIN_THREADS), s, st, partials, nblocks);
    return cudaGetLastError();
}
cudaError_t launch_bl_s(const LaunchCfg& c, BlState* st, FieldPtr R, FieldPtr V, FieldPtr P, FieldPtr S, FieldPtr X,
                        double* partials, cudaStream_t s) {
    if (c.nlat != 1 || c.NR != 1 || c.nrhs > BLK_MAX) return cudaErrorInvalidValue;
    launch_pdl(k_bl_s, dim3(c.nblocks), dim3(c.TS, c.nrhs), s, c.lats, (const BlState*)st,
               (const double2*)R.v, (const double2*)V.v, (const double2*)P.v, (double2*)S.v, (double2*)X.v, partials);
    return cudaGetLastError();
}
cudaError_t launch_bl_fin_s(BlState* st, const double* partials, int nblocks, cudaGraphConditionalHandle h_if,
                            cudaStream_t s) {
    launch_pdl(k_bl_fin_s, dim3(1), dim3(FIN_THREADS), s, st, partials, nblocks, h_if);
    return cudaGetLastError();
}
cudaError_t launch_bl_fin_omega(BlState* st, const double* partials, int nblocks, cudaStream_t s) {
    launch_pdl(k_bl_fin_omega, dim3(1), dim3(FIN_THREADS), s, st, partials, nblocks);
    return cudaGetLastError();
}
cudaError_t launch_bl_r(const LaunchCfg& c, BlState* st, FieldPtr S, FieldPtr T, FieldPtr R0, FieldPtr X, FieldPtr R,
                        double* partials, cudaStream_t s) {
    if (c.nlat != 1 || c.NR != 1 || c.nrhs > BLK_MAX) return cudaErrorInvalidValue;
    launch_pdl(k_bl_r, dim3(c.nblocks), dim3(c.TS, c.nrhs), s, c.lats, (const BlState*)st, (const double2*)S.v,
               (const double2*)T.v, (const double2*)R0.v, (double2*)X.v, (double2*)R.v, partials);
    return cudaGetLastError();
}
cudaError_t launch_bl_fin_r(BlState* st, const double* partials, int nblocks, cudaStream_t s) {
    launch_pdl(k_bl_fin_r, dim3(1), dim3(FIN_THREADS), s, st, partials, nblocks);
    return cudaGetLastError();
}
cudaError_t launch_bl_p(const LaunchCfg& c, BlState* st, FieldPtr P, FieldPtr V, FieldPtr R,
                        cudaGraphConditionalHandle h_iter, cudaStream_t s) {
    if (c.nlat != 1 || c.NR != 1 || c.TS != 32 || c.nrhs > BLK_MAX) return cudaErrorInvalidValue;
    launch_pdl(k_bl_p, dim3(c.nblocks), dim3(c.TS, c.nrhs), s, c.lats, st, (double2*)P.v, (const double2*)V.v,
               (const double2*)R.v, h_iter);
    return cudaGetLastError();
}
cudaError_t launch_bl_cycle(BlState* st, const double* rr, cudaGraphConditionalHandle h_cycle, cudaStream_t s) {
    launch_pdl(k_bl_cycle, dim3(1), dim3(32), s, st, rr, h_cycle);
    return cudaGetLastError();
}

// ====================================================================== Gl-BiCGStab
__global__ void k_gl_init(GlState* st, int n, const double* __restrict__ bb, double tol, double delta, int max_outer,
                          int max_cycles, OState* ost, cudaGraphConditionalHandle h_cycle) {
    pdl_enter();
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    st->n = n;
    for (int j = 0; j < n; ++j) {
        st->bb[j] = bb[j];
        st->rr[j] = bb[j];
        ost[j].inner_iters = 0;
        ost[j].sweeps = 0;
        ost[j].active = 0;
    }
    st->stop2 = 0.25 * tol * tol;
    st->tol2 = tol * tol;
    st->delta2 = delta * delta;
    st->iters = 0;
    st->max_outer = max_outer;
    st->cycles = 0;
    st->max_cycles = max_cycles;
    st->calls = 0;
    st->stop = 0;
    st->fail = 0;
    st->body_runs = 0;
    st->if_runs = 0;
    set_cond(h_cycle, true);
}

__global__ void __launch_bounds__(FIN_THREADS) k_gl_fin_start(GlState* st, const double* __restrict__ partials,
                                                              int nblocks, cudaGraphConditionalHandle h_iter) {
    pdl_enter();
    __shared__ double sres[BLK_MAX * 3];
    const int n = st->n;
    fin_sums<3>(partials, n, nblocks, sres);
    if (threadIdx.x == 0) {
        double2 rho = make_double2(0.0, 0.0);
        for (int j = 0; j < n; ++j) {
            rho = c_add(rho, make_double2(sres[3 * j], sres[3 * j + 1]));
            st->rr[j] = sres[3 * j + 2];
        }
        st->rho = rho;
        const bool stop = all_below(st->rr, st->bb, n, st->stop2, 1) || rho.x == 0.0;
        st->stop = stop ? 1 : 0;
        st->iters = 0;
        st->cycles += 1;
        set_cond(h_iter, !stop && st->max_outer > 0);
    }
}

// the outer states of the FP32 inner solves of one preconditioner call on a
// vector with |in_j|^2 = nin[j]: active while |in_j| > tol |phi_j|, 1 / |in_j|
// normalises the inner rhs, and each inner solve stops at the relative
// residual max(delta, 0.1 tol |phi_j| / |in_j|) (a finer inner solve would
// only resolve what lies below the outer tolerance)
__global__ void k_gl_prep(GlState* st, OState* ost, const double* __restrict__ nin) {
    pdl_enter();
    if (blockIdx.x != 0) return;
    const int n = st->n, j = threadIdx.x;
    if (j == 0) st->calls += 1;
    if (j >= n) return;
    OState& o = ost[j];
    const double r = nin[j], bb = st->bb[j];
    o.bb = bb;
    o.rr = r;
    o.tol2 = st->tol2;
    o.delta2_floor = st->delta2;
    o.sweeps = 0;
    const bool finite = (r == r) && (r < 1e300);
    const bool go = finite && bb > 0.0 && r > st->tol2 * bb;
    o.active = go ? 1 : 0;
    o.inv_norm = go ? 1.0 / sqrt(r) : 0.0;
    o.delta2 = go ? fmax(st->delta2, 0.01 * st->tol2 * bb / r) : 1.0;
}

__global__ void __launch_bounds__(FIN_THREADS) k_gl_fin_alpha(GlState* st, const double* __restrict__ partials,
                                                              int nblocks) {
    pdl_enter();
    __shared__ double sres[BLK_MAX * 2];
    const int n = st->n;
    fin_sums<2>(partials, n, nblocks, sres);
    if (threadIdx.x == 0) {
        double2 r0v = make_double2(0.0, 0.0);
        for (int j = 0; j < n; ++j) r0v = c_add(r0v, make_double2(sres[2 * j], sres[2 * j + 1]));
        if (r0v.x == 0.0 && r0v.y == 0.0) {
            st->stop = 1;
            st->fail += 1;
            st->alpha = make_double2(0.0, 0.0);
        } else {
            st->alpha = c_div(st->rho, r0v);
            st->iters += 1;
        }
    }
}

// S = R - alpha V, X += alpha PH, |S_j|^2 (skipped once stopped)
__global__ void __launch_bounds__(KB<P64, 1>::MAXT) k_gl_s(const LatDev* __restrict__ lats, const GlState* st,
                                                         const double2* __restrict__ R, const double2* __restrict__ V,
                                                         const double2* __restrict__ PH, double2* __restrict__ S,
                                                         double2* __restrict__ X, double* __restrict__ partials) {
    pdl_enter();
    if (st->stop) return;
    const int n = st->n, j = threadIdx.y;
    const double2 al = st->alpha;
    const LatDev g = lats[0];
    double red[1][1] = {{0.0}};
    for (int tile = tile_begin(g), te = tile_end(g); tile < te; ++tile) {
        const int cb = tile_cb(g, tile, threadIdx.x);
        if (cb < 0) continue;
        const long long bj = vbase<P64>(g, j) + cb;
#pragma unroll 4
        for (int comp = 0; comp < 12; ++comp) {
            const long long i = bj + (long long)comp * g.Vpad;
            const double2 s = c_sub(R[i], c_mul(al, V[i]));
            S[i] = s;
            X[i] = c_add(X[i], c_mul(al, PH[i]));
            red[0][0] += s.x * s.x + s.y * s.y;
        }
    }
    block_partials<1, 1>(red, n, partials);
}

__global__ void __launch_bounds__(FIN_THREADS) k_gl_fin_s(GlState* st, const double* __restrict__ partials, int nblocks,
                                                          cudaGraphConditionalHandle h_if) {
    pdl_enter();
    if (st->stop) {
        if (threadIdx.x == 0) set_cond(h_if, false);
        return;
    }
    __shared__ double sres[BLK_MAX];
    const int n = st->n;
    fin_sums<1>(partials, n, nblocks, sres);
    if (threadIdx.x == 0) {
        for (int j = 0; j < n; ++j) st->rr[j] = sres[j];
        const bool below = all_below(sres, st->bb, n, st->stop2, 1);
        if (below) st->stop = 1;
        set_cond(h_if, !below);
    }
}

// <T_j, S_j> and |T_j|^2
__global__ void __launch_bounds__(KB<P64, 1>::MAXT) k_gl_ts(const LatDev* __restrict__ lats, const GlState* st,
                                                          const double2* __restrict__ T, const double2* __restrict__ S,
                                                          double* __restrict__ partials) {
    pdl_enter();
    const int n = st->n, j = threadIdx.y;
    const LatDev g = lats[0];
    double red[1][3] = {{0.0, 0.0, 0.0}};
    for (int tile = tile_begin(g), te = tile_end(g); tile < te; ++tile) {
        const int cb = tile_cb(g, tile, threadIdx.x);
        if (cb < 0) continue;
        const long long bj = vbase<P64>(g, j) + cb;
#pragma unroll 4
        for (int comp = 0; comp < 12; ++comp) {
            const long long i = bj + (long long)comp * g.Vpad;
            const double2 t = T[i], s = S[i];
            const double2 ts = c_cmul(t, s);
            red[0][0] += ts.x;
            red[0][1] += ts.y;
            red[0][2] += t.x * t.x + t.y * t.y;
        }
    }
    block_partials<1, 3>(red, n, partials);
}

__global__ void __launch_bounds__(FIN_THREADS) k_gl_fin_omega(GlState* st, const double* __restrict__ partials,
                                                              int nblocks) {
    pdl_enter();
    __shared__ double sres[BLK_MAX * 3];
    const int n = st->n;
    fin_sums<3>(partials, n, nblocks, sres);
    if (threadIdx.x == 0) {
        st->if_runs += 1;
        double2 ts = make_double2(0.0, 0.0);
        double tt = 0.0;
        for (int j = 0; j < n; ++j) {
            ts = c_add(ts, make_double2(sres[3 * j], sres[3 * j + 1]));
            tt += sres[3 * j + 2];
        }
        if (tt > 0.0) {
            st->omega = c_scale(ts, 1.0 / tt);
        } else {
            st->omega = make_double2(0.0, 0.0);
            st->stop = 1;
            st->fail += 1;
        }
    }
}

// X += omega SH, R = S - omega T; |R_j|^2, <R0_j, R_j>
__global__ void __launch_bounds__(KB<P64, 1>::MAXT) k_gl_r(const LatDev* __restrict__ lats, const GlState* st,
                                                         const double2* __restrict__ S, const double2* __restrict__ T,
                                                         const double2* __restrict__ SH, const double2* __restrict__ R0,
                                                         double2* __restrict__ X, double2* __restrict__ R,
                                                         double* __restrict__ partials) {
    pdl_enter();
    const int n = st->n, j = threadIdx.y;
    const double2 om = st->omega;
    const LatDev g = lats[0];
    double red[1][3] = {{0.0, 0.0, 0.0}};
    for (int tile = tile_begin(g), te = tile_end(g); tile < te; ++tile) {
        const int cb = tile_cb(g, tile, threadIdx.x);
        if (cb < 0) continue;
        const long long bj = vbase<P64>(g, j) + cb;
#pragma unroll 4
        for (int comp = 0; comp < 12; ++comp) {
            const long long i = bj + (long long)comp * g.Vpad;
            X[i] = c_add(X[i], c_mul(om, SH[i]));
            const double2 r = c_sub(S[i], c_mul(om, T[i]));
            R[i] = r;
            red[0][0] += r.x * r.x + r.y * r.y;
            const double2 zr = c_cmul(R0[i], r);
            red[0][1] += zr.x;
            red[0][2] += zr.y;
        }
    }
    block_partials<1, 3>(red, n, partials);
}

__global__ void __launch_bounds__(FIN_THREADS) k_gl_fin_r(GlState* st, const double* __restrict__ partials, int nblocks) {
    pdl_enter();
    if (st->stop) return;
    __shared__ double sres[BLK_MAX * 3];
    const int n = st->n;
    fin_sums<3>(partials, n, nblocks, sres);
    if (threadIdx.x == 0) {
        double2 rho1 = make_double2(0.0, 0.0);
        for (int j = 0; j < n; ++j) {
            st->rr[j] = sres[3 * j];
            rho1 = c_add(rho1, make_double2(sres[3 * j + 1], sres[3 * j + 2]));
        }
        if (all_below(sres, st->bb, n, st->stop2, 3)) {
            st->stop = 1;
        } else if (st->omega.x == 0.0 && st->omega.y == 0.0) {
            st->stop = 1;
            st->fail += 1;
        } else {
            st->beta = c_mul(c_div(rho1, st->rho), c_div(st->alpha, st->omega));
            st->rho = rho1;
        }
    }
}

// P = R + beta (P - omega V); block 0 sets the iteration loop's condition
__global__ void __launch_bounds__(KB<P64, 1>::MAXT) k_gl_p(const LatDev* __restrict__ lats, GlState* st,
                                                         double2* __restrict__ P, const double2* __restrict__ V,
                                                         const double2* __restrict__ R,
                                                         cudaGraphConditionalHandle h_iter) {
    pdl_enter();
    const int stop = st->stop;
    if (blockIdx.x == 0 && threadIdx.x == 0 && threadIdx.y == 0) {
        st->body_runs += 1;
        set_cond(h_iter, !stop && st->iters < st->max_outer);
    }
    if (stop) return;
    const int j = threadIdx.y;
    const double2 be = st->beta, om = st->omega;
    const LatDev g = lats[0];
    for (int tile = tile_begin(g), te = tile_end(g); tile < te; ++tile) {
        const int cb = tile_cb(g, tile, threadIdx.x);
        if (cb < 0) continue;
        const long long bj = vbase<P64>(g, j) + cb;
#pragma unroll 4
        for (int comp = 0; comp < 12; ++comp) {
            const long long i = bj + (long long)comp * g.Vpad;
            P[i] = c_add(R[i], c_mul(be, c_sub(P[i], c_mul(om, V[i]))));
        }
    }
}

__global__ void k_gl_cycle(GlState* st, const double* __restrict__ rr, cudaGraphConditionalHandle h_cycle) {
    pdl_enter();
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int n = st->n;
    bool ok = true;
    for (int j = 0; j < n; ++j) {
        st->rr[j] = rr[j];
        ok = ok && (rr[j] <= st->tol2 * st->bb[j] || st->bb[j] == 0.0);
    }
    st->stop = 0;
    set_cond(h_cycle, !ok && st->cycles < st->max_cycles);
}

cudaError_t launch_gl_init(GlState* st, int n, const double* bb, double tol, double delta, int max_outer,
                           int max_cycles, OState* ost, cudaGraphConditionalHandle h_cycle, cudaStream_t s) {
    if (n < 1 || n > BLK_MAX) return cudaErrorInvalidValue;
    launch_pdl(k_gl_init, dim3(1), dim3(32), s, st, n, bb, tol, delta, max_outer, max_cycles, ost, h_cycle);
    return cudaGetLastError();
}
cudaError_t launch_gl_fin_start(GlState* st, const double* partials, int nblocks, cudaGraphConditionalHandle h_iter,
                                cudaStream_t s) {
    launch_pdl(k_gl_fin_start, dim3(1), dim3(FIN_THREADS), s, st, partials, nblocks, h_iter);
    return cudaGetLastError();
}
cudaError_t launch_gl_prep(GlState* st, OState* ost, const double* nin, cudaStream_t s) {
    launch_pdl(k_gl_prep, dim3(1), dim3(32), s, st, ost, nin);
    return cudaGetLastError();
}
cudaError_t launch_gl_fin_alpha(GlState* st, const double* partials, int nblocks, cudaStream_t s) {
    launch_pdl(k_gl_fin_alpha, dim3(1), dim3(FIN_THREADS), s, st, partials, nblocks);
    return cudaGetLastError();
}
cudaError_t launch_gl_s(const LaunchCfg& c, GlState* st, FieldPtr R, FieldPtr V, FieldPtr PH, FieldPtr S, FieldPtr X,
                        double* partials, cudaStream_t s) {
    if (c.nlat != 1 || c.NR != 1 || c.nrhs > BLK_MAX) return cudaErrorInvalidValue;
    launch_pdl(k_gl_s, dim3(c.nblocks), dim3(c.TS, c.nrhs), s, c.lats, (const GlState*)st, (const double2*)R.v,
               (const double2*)V.v, (const double2*)PH.v, (double2*)S.v, (double2*)X.v, partials);
    return cudaGetLastError();
}
cudaError_t launch_gl_fin_s(GlState* st, const double* partials, int nblocks, cudaGraphConditionalHandle h_if,
                            cudaStream_t s) {
    launch_pdl(k_gl_fin_s, dim3(1), dim3(FIN_THREADS), s, st, partials, nblocks, h_if);
    return cudaGetLastError();
}
cudaError_t launch_gl_ts(const LaunchCfg& c, GlState* st, FieldPtr T, FieldPtr S, double* partials, cudaStream_t s) {
    if (c.nlat != 1 || c.NR != 1 || c.nrhs > BLK_MAX) return cudaErrorInvalidValue;
    launch_pdl(k_gl_ts, dim3(c.nblocks), dim3(c.TS, c.nrhs), s, c.lats, (const GlState*)st, (const double2*)T.v,
               (const double2*)S.v, partials);
    return cudaGetLastError();
}
cudaError_t launch_gl_fin_omega(GlState* st, const double* partials, int nblocks, cudaStream_t s) {
    launch_pdl(k_gl_fin_omega, dim3(1), dim3(FIN_THREADS), s, st, partials, nblocks);
    return cudaGetLastError();
}
cudaError_t launch_gl_r(const LaunchCfg& c, GlState* st, FieldPtr S, FieldPtr T, FieldPtr SH, FieldPtr R0,
                        FieldPtr X, FieldPtr R, double* partials, cudaStream_t s) {
    if (c.nlat != 1 || c.NR != 1 || c.nrhs > BLK_MAX) return cudaErrorInvalidValue;
    launch_pdl(k_gl_r, dim3(c.nblocks), dim3(c.TS, c.nrhs), s, c.lats, (const GlState*)st, (const double2*)S.v,
               (const double2*)T.v, (const double2*)SH.v, (const double2*)R0.v, (double2*)X.v, (double2*)R.v,
               partials);
    return cudaGetLastError();
}
cudaError_t launch_gl_fin_r(GlState* st, const double* partials, int nblocks, cudaStream_t s) {
    launch_pdl(k_gl_fin_r, dim3(1), dim3(FIN_THREADS), s, st, partials, nblocks);
    return cudaGetLastError();
}
cudaError_t launch_gl_p(const LaunchCfg& c, GlState* st, FieldPtr P, FieldPtr V, FieldPtr R,
                        cudaGraphConditionalHandle h_iter, cudaStream_t s) {
    if (c.nlat != 1 || c.NR != 1 || c.nrhs > BLK_MAX) return cudaErrorInvalidValue;
    launch_pdl(k_gl_p, dim3(c.nblocks), dim3(c.TS, c.nrhs), s, c.lats, st, (double2*)P.v, (const double2*)V.v,
               (const double2*)R.v, h_iter);
    return cudaGetLastError();
}
cudaError_t launch_gl_cycle(GlState* st, const double* rr, cudaGraphConditionalHandle h_cycle, cudaStream_t s) {
    launch_pdl(k_gl_cycle, dim3(1), dim3(32), s, st, rr, h_cycle);
    return cudaGetLastError();
}

}  // namespace sf
