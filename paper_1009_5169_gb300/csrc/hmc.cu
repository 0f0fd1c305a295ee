// hmc.cu -- the gauge side of the HMC trajectory the MD step of Alg. 2
// belongs to: the force of the SF plaquette action, the link update
// U -> exp(i dt P) U, the momenta on the fixed boundary links, and the sums
// of squares that give the kinetic energy and the fermion action.  All FP64,
// on the canonical link layout [(T+1) L^3][4][3][3] and the momentum / force
// layout [(T+1) L^3][4][8] (components along T^a = lambda^a / 2).
//
// Dynamic links on the SF lattice: U_0(x) for x0 = 0..T-1 and U_k(x) for
// x0 = 1..T-1; the spatial links at x0 = 0 and x0 = T are the fixed boundary
// fields and keep zero momentum.
#include "krylov_impl.cuh"

namespace sf {

namespace {

__device__ __forceinline__ void hmc_ld(const double2* __restrict__ canon, long long gi, int mu,
                                       cpx<double> (&U)[3][3]) {
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        const double2 v = canon[(gi * 4 + mu) * 9 + k];
        U[k / 3][k % 3] = cpx<double>{v.x, v.y};
    }
}

// C = A B, C = A B^dag, C = A^dag B
__device__ __forceinline__ void mm(const cpx<double> (&A)[3][3], const cpx<double> (&B)[3][3], cpx<double> (&C)[3][3]) {
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            cpx<double> t{0, 0};
#pragma unroll
            for (int k = 0; k < 3; ++k) cfma(t, A[a][k], B[k][b]);
            C[a][b] = t;
        }
}
__device__ __forceinline__ void mmd(const cpx<double> (&A)[3][3], const cpx<double> (&B)[3][3],
                                    cpx<double> (&C)[3][3]) {
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            cpx<double> t{0, 0};
#pragma unroll
            for (int k = 0; k < 3; ++k) t = t + A[a][k] * conj(B[b][k]);
            C[a][b] = t;
        }
}
__device__ __forceinline__ void mdm(const cpx<double> (&A)[3][3], const cpx<double> (&B)[3][3],
                                    cpx<double> (&C)[3][3]) {
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            cpx<double> t{0, 0};
#pragma unroll
            for (int k = 0; k < 3; ++k) t = t + conj(A[k][a]) * B[k][b];
            C[a][b] = t;
        }
}

struct GSite {
    int x0, x1, x2, x3;
};
__device__ __forceinline__ GSite gdecode(long long gi, int L) {
    GSite s;
    s.x3 = (int)(gi % L);
    gi /= L;
    s.x2 = (int)(gi % L);
    gi /= L;
    s.x1 = (int)(gi % L);
    s.x0 = (int)(gi / L);
    return s;
}
__device__ __forceinline__ long long gindex(const GSite& s, int L) {
    return (((long long)s.x0 * L + s.x1) * L + s.x2) * L + s.x3;
}
__device__ __forceinline__ GSite gshift(GSite s, int nu, int d, int L) {
    if (nu == 0) s.x0 += d;
    else if (nu == 1) s.x1 = (s.x1 + d + L) % L;
    else if (nu == 2) s.x2 = (s.x2 + d + L) % L;
    else s.x3 = (s.x3 + d + L) % L;
    return s;
}
__device__ __forceinline__ bool dynamic_link(int x0, int mu, int T) {
    return mu == 0 ? (x0 <= T - 1) : (x0 >= 1 && x0 <= T - 1);
}
// weight of the plaquette with base time slice y0 in the plane {mu, nu} of
// the SF action (0: not part of it): 1 for time-like ones inside, 1/2 for
// spatial ones on the boundary slices
__device__ __forceinline__ double plaq_w(int y0, int mu, int nu, int T) {
    if (y0 < 0 || y0 > T) return 0.0;
    if (mu == 0 || nu == 0) return (y0 <= T - 1) ? 1.0 : 0.0;
    return (y0 == 0 || y0 == T) ? 0.5 : 1.0;
}

// F^a = (beta / 6) Im tr(lambda^a W), W = U sum_staples w A
__device__ __forceinline__ void gell_im_tr(const cpx<double> (&W)[3][3], double (&f)[8]) {
    const double r3 = 0.57735026918962576451;  // 1/sqrt(3)
    f[0] = W[1][0].im + W[0][1].im;
    f[1] = -W[1][0].re + W[0][1].re;
    f[2] = W[0][0].im - W[1][1].im;
    f[3] = W[2][0].im + W[0][2].im;
    f[4] = -W[2][0].re + W[0][2].re;
    f[5] = W[2][1].im + W[1][2].im;
    f[6] = -W[2][1].re + W[1][2].re;
    f[7] = r3 * (W[0][0].im + W[1][1].im - 2.0 * W[2][2].im);
}

}  // namespace

// Force of the SF plaquette action S_g = beta sum_p w(p) (1 - Re tr U_p / 3)
// on every dynamic link: every plaquette through U_mu(x), traced from that
// link, is Re tr(U_mu(x) A) with the staple
//   up   A = U_nu(x+mu) U_mu(x+nu)^dag U_nu(x)^dag          (base x),
//   down A = U_nu(x+mu-nu)^dag U_mu(x-nu)^dag U_nu(x-nu)     (base x-nu),
// and d/d omega^a Re tr(e^{i omega T^a} U A) = -Im tr(T^a U A), so
//   F^a = (beta / 3) sum w Im tr(T^a U A).
// One thread per (site, mu); F (if set) = F_g, mom (if set) -= eps F_g.
__global__ void __launch_bounds__(128) k_gauge_force(int L, int T, double beta, const double2* __restrict__ canon,
                                                     double* __restrict__ F, double* __restrict__ mom, double eps) {
    pdl_enter();
    const long long n = (long long)(T + 1) * L * L * L * 4;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int mu = (int)(i & 3);
        const long long gi = i >> 2;
        const GSite x = gdecode(gi, L);
        if (!dynamic_link(x.x0, mu, T)) {
            if (F) {
#pragma unroll
                for (int a = 0; a < 8; ++a) F[i * 8 + a] = 0.0;
            }
            continue;
        }
        cpx<double> S[3][3];
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) S[a][b] = cpx<double>{0, 0};
        const GSite xm = gshift(x, mu, +1, L);
        for (int nu = 0; nu < 4; ++nu) {
            if (nu == mu) continue;
            cpx<double> P[3][3], Q[3][3], R[3][3];
            const double wu = plaq_w(x.x0, mu, nu, T);
            if (wu != 0.0) {
                const GSite xn = gshift(x, nu, +1, L);
                hmc_ld(canon, gindex(xm, L), nu, P);
                hmc_ld(canon, gindex(xn, L), mu, Q);
                mmd(P, Q, R);                            // U_nu(x+mu) U_mu(x+nu)^dag
                hmc_ld(canon, gi, nu, P);
                mmd(R, P, Q);                            // ... U_nu(x)^dag
#pragma unroll
                for (int a = 0; a < 3; ++a)
#pragma unroll
                    for (int b = 0; b < 3; ++b) S[a][b] = S[a][b] + wu * Q[a][b];
            }
            const GSite xd = gshift(x, nu, -1, L);
            const double wd = plaq_w(xd.x0, mu, nu, T);
            if (wd != 0.0) {
                const GSite xmd = gshift(xm, nu, -1, L);
                hmc_ld(canon, gindex(xmd, L), nu, P);
                hmc_ld(canon, gindex(xd, L), mu, Q);
                cpx<double> PQ[3][3];
#pragma unroll
                for (int a = 0; a < 3; ++a)
#pragma unroll
                    for (int b = 0; b < 3; ++b) {
                        // (U_nu(x+mu-nu)^dag U_mu(x-nu)^dag)_{ab} = sum_k conj(P_ka) conj(Q_bk)
                        cpx<double> t{0, 0};
#pragma unroll
                        for (int k = 0; k < 3; ++k) t = t + conj(P[k][a]) * conj(Q[b][k]);
                        PQ[a][b] = t;
                    }
                hmc_ld(canon, gindex(xd, L), nu, P);
                mm(PQ, P, R);                            // ... U_nu(x-nu)
#pragma unroll
                for (int a = 0; a < 3; ++a)
#pragma unroll
                    for (int b = 0; b < 3; ++b) S[a][b] = S[a][b] + wd * R[a][b];
            }
        }
        cpx<double> U[3][3], W[3][3];
        hmc_ld(canon, gi, mu, U);
        mm(U, S, W);
        double f[8];
        gell_im_tr(W, f);
#pragma unroll
        for (int a = 0; a < 8; ++a) {
            const double fa = beta / 6.0 * f[a];
            if (F) F[i * 8 + a] = fa;
            if (mom) mom[i * 8 + a] -= eps * fa;
        }
    }
}

// U_mu(x) <- exp(i dt P_mu(x)) U_mu(x) on every dynamic link, P = sum_a P^a
// lambda^a / 2.  exp of the traceless anti-Hermitian X = i dt P by scaling
// and squaring: X / 2^s with |X / 2^s|_F = n <= 1/4, the Taylor sum to the
// first order K with n^K / K! <= 1e-20 (so the remainder, below n^(K+1) /
// (K+1)!, is under 1e-20 relative; K <= 14 at n = 1/4, about 10 for the
// n ~ 0.04 of an MD step dt = 0.02), then s squarings.
__global__ void __launch_bounds__(128) k_link_update(int L, int T, double2* __restrict__ canon,
                                                     const double* __restrict__ mom, double dt) {
    pdl_enter();
    const long long n = (long long)(T + 1) * L * L * L * 4;
    const double r3 = 0.57735026918962576451;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int mu = (int)(i & 3);
        const GSite x = gdecode(i >> 2, L);
        if (!dynamic_link(x.x0, mu, T)) continue;
        const double* p = mom + i * 8;
        // H = sum_a p_a lambda^a / 2 (Hermitian), X = i dt H
        cpx<double> H[3][3];
        H[0][0] = cpx<double>{0.5 * (p[2] + r3 * p[7]), 0};
        H[1][1] = cpx<double>{0.5 * (-p[2] + r3 * p[7]), 0};
        H[2][2] = cpx<double>{0.5 * (-2.0 * r3 * p[7]), 0};
        H[0][1] = cpx<double>{0.5 * p[0], -0.5 * p[1]};
        H[1][0] = conj(H[0][1]);
        H[0][2] = cpx<double>{0.5 * p[3], -0.5 * p[4]};
        H[2][0] = conj(H[0][2]);
        H[1][2] = cpx<double>{0.5 * p[5], -0.5 * p[6]};
        H[2][1] = conj(H[1][2]);
        cpx<double> X[3][3];
        double nrm2 = 0.0;
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                X[a][b] = cpx<double>{-dt * H[a][b].im, dt * H[a][b].re};
                nrm2 += X[a][b].re * X[a][b].re + X[a][b].im * X[a][b].im;
            }
        int s = 0;
        double sc = 1.0;
        while (nrm2 * sc * sc > 0.0625 && s < 60) {
            sc *= 0.5;
            ++s;
        }
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) X[a][b] = sc * X[a][b];
        // the order: the first K with n^K / K! <= 1e-20, n = |X|_F after scaling
        const double n = sqrt(nrm2) * sc;
        int K = 0;
        for (double t = 1.0; K < 14 && t > 1e-20;) {
            ++K;
            t *= n / K;
        }
        // E = sum_{k=0}^{K} X^k / k!  (Horner: E = 1 + X (1 + X/2 (1 + X/3 (...))))
        cpx<double> E[3][3], Tm[3][3];
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) E[a][b] = cpx<double>{a == b ? 1.0 : 0.0, 0.0};
        for (int k = K; k >= 1; --k) {
            mm(X, E, Tm);
            const double c = 1.0 / (double)k;
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int b = 0; b < 3; ++b)
                    E[a][b] = cpx<double>{(a == b ? 1.0 : 0.0) + c * Tm[a][b].re, c * Tm[a][b].im};
        }
        for (int q = 0; q < s; ++q) {
            mm(E, E, Tm);
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int b = 0; b < 3; ++b) E[a][b] = Tm[a][b];
        }
        cpx<double> U[3][3], V[3][3];
        hmc_ld(canon, i >> 2, mu, U);
        mm(E, U, V);
#pragma unroll
        for (int k = 0; k < 9; ++k) canon[i * 9 + k] = make_double2(V[k / 3][k % 3].re, V[k / 3][k % 3].im);
    }
}

// zero the momenta of the fixed boundary links
__global__ void k_mom_fix(int L, int T, double* __restrict__ mom) {
    pdl_enter();
    const long long n = (long long)(T + 1) * L * L * L * 4;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int mu = (int)(i & 3);
        const GSite x = gdecode(i >> 2, L);
        if (!dynamic_link(x.x0, mu, T)) {
#pragma unroll
            for (int a = 0; a < 8; ++a) mom[i * 8 + a] = 0.0;
        }
    }
}

// sum of squares of n doubles: SUMSQ_BLOCKS block partials (grid stride,
// fixed tree), then one block adds them in order
constexpr int SUMSQ_BLOCKS = 304;
__global__ void __launch_bounds__(256) k_sumsq(long long n, const double* __restrict__ x, double* __restrict__ part) {
    pdl_enter();
    __shared__ double sw[8];
    double acc = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        acc = fma(x[i], x[i], acc);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
    if ((threadIdx.x & 31) == 0) sw[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += sw[k];
        part[blockIdx.x] = s;
    }
}
__global__ void __launch_bounds__(32) k_sumsq_finish(const double* __restrict__ part, double scale,
                                                     double* __restrict__ out) {
    pdl_enter();
    double s = 0.0;
    for (int b = threadIdx.x; b < SUMSQ_BLOCKS; b += 32) s += part[b];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    if (threadIdx.x == 0) *out = scale * s;
}

static int hmc_blocks(long long n, int per) {
    long long b = (n + per - 1) / per;
    if (b > 4 * 152) b = 4 * 152;
    return (int)(b < 1 ? 1 : b);
}

cudaError_t launch_gauge_force(int L, int T, double beta, const double* canon, double* F, double* mom, double eps,
                               cudaStream_t st) {
    const long long n = (long long)(T + 1) * L * L * L * 4;
    launch_pdl(k_gauge_force, dim3(hmc_blocks(n, 128)), dim3(128), st, L, T, beta,
               reinterpret_cast<const double2*>(canon), F, mom, eps);
    return cudaGetLastError();
}

cudaError_t launch_link_update(int L, int T, double* canon, const double* mom, double dt, cudaStream_t st) {
    const long long n = (long long)(T + 1) * L * L * L * 4;
    launch_pdl(k_link_update, dim3(hmc_blocks(n, 128)), dim3(128), st, L, T, reinterpret_cast<double2*>(canon), mom,
               dt);
    return cudaGetLastError();
}

cudaError_t launch_mom_fix(int L, int T, double* mom, cudaStream_t st) {
    const long long n = (long long)(T + 1) * L * L * L * 4;
    launch_pdl(k_mom_fix, dim3(hmc_blocks(n, 256)), dim3(256), st, L, T, mom);
    return cudaGetLastError();
}

cudaError_t launch_sumsq(long long n, const double* x, double scale, double* part, double* out, cudaStream_t st) {
    launch_pdl(k_sumsq, dim3(SUMSQ_BLOCKS), dim3(256), st, n, x, part);
    launch_pdl(k_sumsq_finish, dim3(1), dim3(32), st, (const double*)part, scale, out);
    return cudaGetLastError();
}

}  // namespace sf
