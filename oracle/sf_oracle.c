/*
 * sf_oracle.c -- plain, slow FP64 CPU oracle for the fermion part of the
 * many-flavour HMC molecular-dynamics step of arXiv:1009.5169
 * ("Improving many flavor QCD simulations using multiple GPUs").
 *
 * TEST INFRASTRUCTURE. Only tests/, __graft_entry__.smoke() and bench.py's
 * cpu_baseline / reference legs load this library.  It shares no code,
 * header, table or helper with the CUDA library: every index map, gamma
 * matrix and formula below is written out here on its own.
 *
 * What it computes (each function cites the passage it follows):
 *   - the Wilson hopping term H and D = 1 - kappa H on the Schroedinger-
 *     functional lattice (Sec. 3.1, "N_f = 10 QCD with Wilson fermions",
 *     Sec. 4, SF setup; explicit form: the readings listed below);
 *   - the site even/odd preconditioned operator Dhat = 1 - kappa^2 H_eo H_oe
 *     and its adjoint (Sec. 3.1, "site even/odd preconditioning");
 *   - textbook BiCGStab on Dhat or Dhat^dag, one right-hand side at a time,
 *     i.e. the sequential solver of Alg. 1 / case A of Table 1;
 *   - the MD force F_mu(n) = sum_i f[x_i, y_i] of Eq. (3) with x = Dhat^-1 phi,
 *     y = Dhat^-dag x (Alg. 2), written as the exact gradient of
 *     S = sum_i |Dhat^-1 phi_i|^2 (Eq. 2);
 *   - the SU(3) plaquette action with SF boundary weights (Sec. 4) and its
 *     force (the gauge part of the HMC trajectory the MD step belongs to).
 *
 * Readings of the paper (it fixes none of these):
 *   - gamma matrices: Euclidean, Hermitian, chiral basis; gamma_5 =
 *     gamma_1 gamma_2 gamma_3 gamma_0 = diag(1,1,-1,-1);
 *   - (H psi)(x) = sum_mu [ (1-gamma_mu) U_mu(x) lambda_mu psi(x+mu)
 *                         + (1+gamma_mu) U_mu(x-mu)^dag lambda_mu^* psi(x-mu) ],
 *     Wilson r = 1, no clover term;
 *   - SF: the fermion lives on x0 = 1..T-1, psi(0) = psi(T) = 0 (hops that
 *     reach x0 = 0 or x0 = T are dropped), fermion boundary coefficient 1;
 *   - spatial directions periodic with psi(x + L k) = e^{i theta} psi(x),
 *     implemented as the uniform phase lambda_k = e^{i theta / L} on every
 *     forward spatial hop (lambda_0 = 1).  Mode 1 of the hop instead puts the
 *     whole phase e^{+-i theta} on the hops that wrap around the box;
 *   - force: U_mu(x) -> exp(i omega^a T^a) U_mu(x), T^a = lambda^a / 2 (Gell-Mann),
 *     F^a_mu(x) = dS/d omega^a at omega = 0;
 *   - plaquette action S_g = beta sum_p w(p) (1 - Re tr U_p / 3), w = 1/2 for
 *     spatial plaquettes on the boundary slices x0 = 0, T and 1 otherwise
 *     (c_t = 1).
 *
 * Layouts (identical to the library's canonical host layout):
 *   links  U[gsite][mu][a][b] complex, gsite lexicographic over x0 = 0..T,
 *          x1..x3 = 0..L-1, x3 fastest;
 *   full fermion field psi[site][spin][colour], site lexicographic over
 *          x0 = 1..T-1 (x0 slowest), x3 fastest;
 *   even (odd) field: the sites of that parity in the same lexicographic
 *          order; for even L the rank of lexicographic site i is i / 2.
 *   force  F[gsite][mu][a], a = 0..7 for the generators T^1..T^8.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double _Complex cplx;

/* ------------------------------------------------------------------ tables */

static cplx GAM[5][4][4];   /* gamma_0..gamma_3, then gamma_5 */
static cplx GELL[8][3][3];  /* Gell-Mann lambda^1..lambda^8 */
static int tables_ready = 0;

static void init_tables(void)
{
    if (tables_ready) return;
    memset(GAM, 0, sizeof GAM);
    memset(GELL, 0, sizeof GELL);
    const cplx i = I;
    /* gamma_0 (time) */
    GAM[0][0][2] = 1; GAM[0][1][3] = 1; GAM[0][2][0] = 1; GAM[0][3][1] = 1;
    /* gamma_1 */
    GAM[1][0][3] = i; GAM[1][1][2] = i; GAM[1][2][1] = -i; GAM[1][3][0] = -i;
    /* gamma_2 */
    GAM[2][0][3] = -1; GAM[2][1][2] = 1; GAM[2][2][1] = 1; GAM[2][3][0] = -1;
    /* gamma_3 */
    GAM[3][0][2] = i; GAM[3][1][3] = -i; GAM[3][2][0] = -i; GAM[3][3][1] = i;
    /* gamma_5 = gamma_1 gamma_2 gamma_3 gamma_0, formed by matrix products */
    cplx a[4][4], b[4][4];
    for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 4; ++c) {
            cplx s = 0;
            for (int k = 0; k < 4; ++k) s += GAM[1][r][k] * GAM[2][k][c];
            a[r][c] = s;
        }
    for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 4; ++c) {
            cplx s = 0;
            for (int k = 0; k < 4; ++k) s += a[r][k] * GAM[3][k][c];
            b[r][c] = s;
        }
    for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 4; ++c) {
            cplx s = 0;
            for (int k = 0; k < 4; ++k) s += b[r][k] * GAM[0][k][c];
            GAM[4][r][c] = s;
        }
    /* Gell-Mann matrices */
    GELL[0][0][1] = 1; GELL[0][1][0] = 1;
    GELL[1][0][1] = -i; GELL[1][1][0] = i;
    GELL[2][0][0] = 1; GELL[2][1][1] = -1;
    GELL[3][0][2] = 1; GELL[3][2][0] = 1;
    GELL[4][0][2] = -i; GELL[4][2][0] = i;
    GELL[5][1][2] = 1; GELL[5][2][1] = 1;
    GELL[6][1][2] = -i; GELL[6][2][1] = i;
    GELL[7][0][0] = 1.0 / sqrt(3.0); GELL[7][1][1] = 1.0 / sqrt(3.0);
    GELL[7][2][2] = -2.0 / sqrt(3.0);
    tables_ready = 1;
}

/* exported so tests can check the basis the oracle actually uses */
void sfo_gamma(int which, double* out /* 4x4 complex */)
{
    init_tables();
    memcpy(out, GAM[which], sizeof(cplx) * 16);
}

/* --------------------------------------------------------------- geometry */

typedef struct {
    int L, T;
    double theta;
    int theta_mode;  /* 0: uniform phase e^{i theta/L}; 1: phase on wrapping hops */
    long Vf;         /* fermion sites (T-1) L^3 */
    long Vg;         /* gauge sites (T+1) L^3 */
} geom;

static geom make_geom(int L, int T, double theta, int theta_mode)
{
    geom g;
    g.L = L; g.T = T; g.theta = theta; g.theta_mode = theta_mode;
    g.Vf = (long)(T - 1) * L * L * L;
    g.Vg = (long)(T + 1) * L * L * L;
    return g;
}

/* fermion site index of x = (x0, x1, x2, x3), x0 in 1..T-1 */
static long fidx(const geom* g, const int x[4])
{
    return (((long)(x[0] - 1) * g->L + x[1]) * g->L + x[2]) * g->L + x[3];
}

/* gauge site index, x0 in 0..T */
static long gidx(const geom* g, const int x[4])
{
    return (((long)x[0] * g->L + x[1]) * g->L + x[2]) * g->L + x[3];
}

static void fcoords(const geom* g, long i, int x[4])
{
    x[3] = (int)(i % g->L); i /= g->L;
    x[2] = (int)(i % g->L); i /= g->L;
    x[1] = (int)(i % g->L); i /= g->L;
    x[0] = (int)i + 1;
}

static void gcoords(const geom* g, long i, int x[4])
{
    x[3] = (int)(i % g->L); i /= g->L;
    x[2] = (int)(i % g->L); i /= g->L;
    x[1] = (int)(i % g->L); i /= g->L;
    x[0] = (int)i;
}

static int parity(const int x[4]) { return (x[0] + x[1] + x[2] + x[3]) & 1; }

static const cplx* link(const geom* g, const cplx* U, const int x[4], int mu)
{
    return U + (gidx(g, x) * 4 + mu) * 9;
}

/* ------------------------------------------------------ the hopping term H */

/* out = H in on the full fermion lattice (one field). */
static void hop_full(const geom* g, const cplx* U, const cplx* in, cplx* out)
{
    init_tables();
    const int L = g->L, T = g->T;
    const cplx lam_sp = cexp(I * g->theta / L);
    const cplx wrap = cexp(I * g->theta);
#pragma omp parallel for schedule(static)
    for (long i = 0; i < g->Vf; ++i) {
        int x[4];
        fcoords(g, i, x);
        cplx acc[4][3];
        memset(acc, 0, sizeof acc);
        for (int mu = 0; mu < 4; ++mu) {
            /* forward: (1 - gamma_mu) U_mu(x) lambda psi(x + mu) */
            int y[4] = {x[0], x[1], x[2], x[3]};
            int ok = 1;
            cplx lam = 1.0;
            if (mu == 0) {
                y[0] += 1;
                if (y[0] > T - 1) ok = 0;
            } else {
                y[mu] += 1;
                if (g->theta_mode == 0) lam = lam_sp;
                if (y[mu] == L) {
                    y[mu] = 0;
                    if (g->theta_mode == 1) lam = wrap;
                }
            }
            if (ok) {
                const cplx* Ux = link(g, U, x, mu);
                const cplx* p = in + fidx(g, y) * 12;
                cplx w[4][3];
                for (int s = 0; s < 4; ++s)
                    for (int a = 0; a < 3; ++a) {
                        cplx t = 0;
                        for (int b = 0; b < 3; ++b) t += Ux[a * 3 + b] * p[s * 3 + b];
                        w[s][a] = t;
                    }
                for (int s = 0; s < 4; ++s)
                    for (int a = 0; a < 3; ++a) {
                        cplx t = 0;
                        for (int r = 0; r < 4; ++r)
                            t += ((s == r ? 1.0 : 0.0) - GAM[mu][s][r]) * w[r][a];
                        acc[s][a] += lam * t;
                    }
            }
            /* backward: (1 + gamma_mu) U_mu(x - mu)^dag lambda^* psi(x - mu) */
            int z[4] = {x[0], x[1], x[2], x[3]};
            ok = 1;
            lam = 1.0;
            if (mu == 0) {
                z[0] -= 1;
                if (z[0] < 1) ok = 0;
            } else {
                z[mu] -= 1;
                if (g->theta_mode == 0) lam = conj(lam_sp);
                if (z[mu] < 0) {
                    z[mu] = L - 1;
                    if (g->theta_mode == 1) lam = conj(wrap);
                }
            }
            if (ok) {
                const cplx* Uz = link(g, U, z, mu);
                const cplx* p = in + fidx(g, z) * 12;
                cplx w[4][3];
                for (int s = 0; s < 4; ++s)
                    for (int a = 0; a < 3; ++a) {
                        cplx t = 0;
                        for (int b = 0; b < 3; ++b) t += conj(Uz[b * 3 + a]) * p[s * 3 + b];
                        w[s][a] = t;
                    }
                for (int s = 0; s < 4; ++s)
                    for (int a = 0; a < 3; ++a) {
                        cplx t = 0;
                        for (int r = 0; r < 4; ++r)
                            t += ((s == r ? 1.0 : 0.0) + GAM[mu][s][r]) * w[r][a];
                        acc[s][a] += lam * t;
                    }
            }
        }
        memcpy(out + i * 12, acc, sizeof acc);
    }
}

static void gamma5_full(long nsites, const cplx* in, cplx* out)
{
    init_tables();
    for (long i = 0; i < nsites; ++i) {
        cplx t[12];
        for (int s = 0; s < 4; ++s)
            for (int a = 0; a < 3; ++a) {
                cplx u = 0;
                for (int r = 0; r < 4; ++r) u += GAM[4][s][r] * in[i * 12 + r * 3 + a];
                t[s * 3 + a] = u;
            }
        memcpy(out + i * 12, t, sizeof t);  /* in == out is allowed */
    }
}

/* embed a parity-p field into the full lattice (zeros on the other parity) */
static void embed(const geom* g, int p, const cplx* half, cplx* full)
{
    for (long i = 0; i < g->Vf; ++i) {
        int x[4];
        fcoords(g, i, x);
        if (parity(x) == p) memcpy(full + i * 12, half + (i / 2) * 12, sizeof(cplx) * 12);
        else memset(full + i * 12, 0, sizeof(cplx) * 12);
    }
}

/* extract the parity-p sites of a full field */
static void extract(const geom* g, int p, const cplx* full, cplx* half)
{
    for (long i = 0; i < g->Vf; ++i) {
        int x[4];
        fcoords(g, i, x);
        if (parity(x) == p) memcpy(half + (i / 2) * 12, full + i * 12, sizeof(cplx) * 12);
    }
}

/* out_e = Dhat in_e, Dhat = 1 - kappa^2 H_eo H_oe (even/odd preconditioning) */
static void dhat(const geom* g, const cplx* U, double kappa, const cplx* in_e, cplx* out_e,
                 cplx* w1, cplx* w2)
{
    const long Vh = g->Vf / 2;
    embed(g, 0, in_e, w1);          /* w1 = in on even sites */
    hop_full(g, U, w1, w2);         /* w2 = H in; its odd part is H_oe in */
    cplx* tmp_o = (cplx*)malloc(sizeof(cplx) * 12 * Vh);
    extract(g, 1, w2, tmp_o);
    embed(g, 1, tmp_o, w1);         /* w1 = H_oe in on odd sites */
    free(tmp_o);
    hop_full(g, U, w1, w2);         /* even part of w2 = H_eo H_oe in */
    cplx* hh = (cplx*)malloc(sizeof(cplx) * 12 * Vh);
    extract(g, 0, w2, hh);
    for (long k = 0; k < 12 * Vh; ++k) out_e[k] = in_e[k] - kappa * kappa * hh[k];
    free(hh);
}

/* Dhat^dag = gamma_5 Dhat gamma_5 (checked by the tests, not assumed) */
static void dhat_dag(const geom* g, const cplx* U, double kappa, const cplx* in_e, cplx* out_e,
                     cplx* w1, cplx* w2)
{
    const long Vh = g->Vf / 2;
    cplx* t = (cplx*)malloc(sizeof(cplx) * 12 * Vh);
    cplx* u = (cplx*)malloc(sizeof(cplx) * 12 * Vh);
    gamma5_full(Vh, in_e, t);
    dhat(g, U, kappa, t, u, w1, w2);
    gamma5_full(Vh, u, out_e);
    free(t);
    free(u);
}

static int check_args(int L, int T)
{
    if (L < 2 || (L & 1) || T < 2) return -1;
    return 0;
}

/* ------------------------------------------------------------ exported ops */

/* out = H in on the full fermion lattice, nrhs fields */
int sfo_hop_full(int L, int T, double theta, int theta_mode, const double* U, int nrhs,
                 const double* in, double* out)
{
    if (check_args(L, T)) return -1;
    geom g = make_geom(L, T, theta, theta_mode);
    for (int r = 0; r < nrhs; ++r)
        hop_full(&g, (const cplx*)U, (const cplx*)in + r * g.Vf * 12, (cplx*)out + r * g.Vf * 12);
    return 0;
}

/* out = D in, D = 1 - kappa H (full lattice) */
int sfo_apply_D(int L, int T, double theta, int theta_mode, double kappa, const double* U,
                int nrhs, const double* in, double* out)
{
    if (check_args(L, T)) return -1;
    geom g = make_geom(L, T, theta, theta_mode);
    for (int r = 0; r < nrhs; ++r) {
        const cplx* pin = (const cplx*)in + r * g.Vf * 12;
        cplx* pout = (cplx*)out + r * g.Vf * 12;
        hop_full(&g, (const cplx*)U, pin, pout);
        for (long k = 0; k < 12 * g.Vf; ++k) pout[k] = pin[k] - kappa * pout[k];
    }
    return 0;
}

/* out_e = Dhat in_e (dagger = 0) or Dhat^dag in_e (dagger = 1) */
int sfo_apply_dhat(int L, int T, double theta, double kappa, const double* U, int dagger,
                   int nrhs, const double* in, double* out)
{
    if (check_args(L, T)) return -1;
    geom g = make_geom(L, T, theta, 0);
    const long Vh = g.Vf / 2;
    cplx* w1 = (cplx*)malloc(sizeof(cplx) * 12 * g.Vf);
    cplx* w2 = (cplx*)malloc(sizeof(cplx) * 12 * g.Vf);
    for (int r = 0; r < nrhs; ++r) {
        const cplx* pin = (const cplx*)in + r * Vh * 12;
        cplx* pout = (cplx*)out + r * Vh * 12;
        if (dagger) dhat_dag(&g, (const cplx*)U, kappa, pin, pout, w1, w2);
        else dhat(&g, (const cplx*)U, kappa, pin, pout, w1, w2);
    }
    free(w1);
    free(w2);
    return 0;
}

/* ------------------------------------------------------------- BiCGStab */

static cplx dotc(long n, const cplx* a, const cplx* b) /* sum conj(a) b */
{
    double re = 0, im = 0;
#pragma omp parallel for reduction(+ : re, im) schedule(static)
    for (long k = 0; k < n; ++k) {
        cplx t = conj(a[k]) * b[k];
        re += creal(t);
        im += cimag(t);
    }
    return re + I * im;
}

static double nrm2(long n, const cplx* a) { return sqrt(creal(dotc(n, a, a))); }

/*
 * Textbook BiCGStab (van der Vorst 1992) for A x = b with A = Dhat or Dhat^dag,
 * x0 = 0.  The iterated residual is only a trigger: when it drops below
 * tol/10, the true residual |b - A x| / |b| is recomputed and the method
 * restarts from it unless that is <= tol.  Returns 0 on convergence, 1 when
 * maxiter was reached.
 */
static int bicgstab1(const geom* g, const cplx* U, double kappa, int dagger, const cplx* b,
                     cplx* x, double tol, int maxiter, int* iters_out, double* resid_out)
{
    const long n = 12 * (g->Vf / 2);
    cplx* r = calloc(n, sizeof(cplx));
    cplx* rh = calloc(n, sizeof(cplx));
    cplx* p = calloc(n, sizeof(cplx));
    cplx* v = calloc(n, sizeof(cplx));
    cplx* s = calloc(n, sizeof(cplx));
    cplx* t = calloc(n, sizeof(cplx));
    cplx* w1 = calloc(12 * g->Vf, sizeof(cplx));
    cplx* w2 = calloc(12 * g->Vf, sizeof(cplx));
#define APPLY(in, out) \
    do { if (dagger) dhat_dag(g, U, kappa, in, out, w1, w2); else dhat(g, U, kappa, in, out, w1, w2); } while (0)

    const double bn = nrm2(n, b);
    int it = 0, status = 1;
    double true_res = 0.0;
    memset(x, 0, sizeof(cplx) * n);
    if (bn == 0.0) { status = 0; goto done; }
    memcpy(r, b, sizeof(cplx) * n);
    while (it < maxiter) {
        /* (re)start */
        memcpy(rh, r, sizeof(cplx) * n);
        memset(p, 0, sizeof(cplx) * n);
        memset(v, 0, sizeof(cplx) * n);
        cplx rho_old = 1.0, alpha = 1.0, omega = 1.0;
        int restart = 0;
        while (it < maxiter && !restart) {
            cplx rho = dotc(n, rh, r);
            cplx beta = (rho / rho_old) * (alpha / omega);
            for (long k = 0; k < n; ++k) p[k] = r[k] + beta * (p[k] - omega * v[k]);
            APPLY(p, v);
            alpha = rho / dotc(n, rh, v);
            for (long k = 0; k < n; ++k) s[k] = r[k] - alpha * v[k];
            APPLY(s, t);
            double tt = creal(dotc(n, t, t));
            omega = (tt > 0) ? dotc(n, t, s) / tt : 0.0;
            for (long k = 0; k < n; ++k) {
                x[k] += alpha * p[k] + omega * s[k];
                r[k] = s[k] - omega * t[k];
            }
            rho_old = rho;
            ++it;
            if (nrm2(n, r) <= 0.1 * tol * bn) restart = 1;
        }
        /* true residual */
        APPLY(x, t);
        for (long k = 0; k < n; ++k) r[k] = b[k] - t[k];
        true_res = nrm2(n, r) / bn;
        if (true_res <= tol) { status = 0; break; }
    }
done:
    if (iters_out) *iters_out = it;
    if (resid_out) *resid_out = true_res;
#undef APPLY
    free(r); free(rh); free(p); free(v); free(s); free(t); free(w1); free(w2);
    return status;
}

/* Solve Dhat x_i = b_i (dagger = 0) or Dhat^dag x_i = b_i (dagger = 1) for each
 * right-hand side in turn (Alg. 1).  iters[i], resid[i] receive the iteration
 * count and the final true relative residual.  Returns the number of
 * right-hand sides that did not converge. */
int sfo_bicgstab(int L, int T, double theta, double kappa, const double* U, int dagger, int nrhs,
                 const double* b, double* x, double tol, int maxiter, int* iters, double* resid)
{
    if (check_args(L, T)) return -1;
    geom g = make_geom(L, T, theta, 0);
    const long Vh = g.Vf / 2;
    int bad = 0;
    for (int r = 0; r < nrhs; ++r)
        bad += bicgstab1(&g, (const cplx*)U, kappa, dagger, (const cplx*)b + r * Vh * 12,
                         (cplx*)x + r * Vh * 12, tol, maxiter, iters ? iters + r : NULL,
                         resid ? resid + r : NULL);
    return bad;
}

/* -------------------------------------------------------------- the force */

/*
 * MD force of Eq. (3) for S = sum_i |Dhat^-1 phi_i|^2 given x_i = Dhat^-1 phi_i
 * and y_i = Dhat^-dag x_i on the even sites (the two solves of Alg. 2).
 *
 * With Xh = (x_e, kappa H_oe x_e) and Yh = (y_e, kappa gamma_5 H_oe gamma_5 y_e)
 * on the full lattice, dS = 2 kappa Re sum_i Yh_i^dag dH Xh_i, so for the
 * link U_mu(x) -> exp(i omega^a T^a) U_mu(x):
 *   F^a_mu(x) = 2 kappa Re sum_i [ Yh(x)^dag (1-gamma_mu) (i T^a U) lambda Xh(x+mu)
 *                                + Yh(x+mu)^dag (1+gamma_mu) (i T^a U)^dag lambda^* Xh(x) ].
 * Each component is evaluated from this per-link formula directly.  Links
 * with an end outside x0 = 1..T-1 carry no fermion force.  F is accumulated
 * (+=) into the caller's array, layout F[gsite][mu][a].
 */
int sfo_force(int L, int T, double theta, double kappa, const double* Ud, int nrhs,
              const double* Xd, const double* Yd, double* F)
{
    if (check_args(L, T)) return -1;
    init_tables();
    geom g = make_geom(L, T, theta, 0);
    const cplx* U = (const cplx*)Ud;
    const long Vh = g.Vf / 2;
    cplx* Xh = malloc(sizeof(cplx) * 12 * g.Vf);
    cplx* Yh = malloc(sizeof(cplx) * 12 * g.Vf);
    cplx* w1 = malloc(sizeof(cplx) * 12 * g.Vf);
    cplx* w2 = malloc(sizeof(cplx) * 12 * g.Vf);
    cplx* tmp = malloc(sizeof(cplx) * 12 * Vh);
    const cplx lam_sp = cexp(I * theta / L);

    for (int r = 0; r < nrhs; ++r) {
        const cplx* xe = (const cplx*)Xd + r * Vh * 12;
        const cplx* ye = (const cplx*)Yd + r * Vh * 12;
        /* Xh: even part x_e, odd part kappa H_oe x_e */
        embed(&g, 0, xe, w1);
        hop_full(&g, U, w1, w2);
        extract(&g, 1, w2, tmp);
        for (long k = 0; k < 12 * Vh; ++k) tmp[k] *= kappa;
        embed(&g, 0, xe, Xh);
        for (long i = 0; i < g.Vf; ++i) {
            int x[4];
            fcoords(&g, i, x);
            if (parity(x) == 1) memcpy(Xh + i * 12, tmp + (i / 2) * 12, sizeof(cplx) * 12);
        }
        /* Yh: even part y_e, odd part kappa gamma_5 H_oe gamma_5 y_e */
        cplx* g5y = malloc(sizeof(cplx) * 12 * Vh);
        gamma5_full(Vh, ye, g5y);
        embed(&g, 0, g5y, w1);
        free(g5y);
        hop_full(&g, U, w1, w2);
        extract(&g, 1, w2, tmp);
        gamma5_full(Vh, tmp, tmp);
        for (long k = 0; k < 12 * Vh; ++k) tmp[k] *= kappa;
        embed(&g, 0, ye, Yh);
        for (long i = 0; i < g.Vf; ++i) {
            int x[4];
            fcoords(&g, i, x);
            if (parity(x) == 1) memcpy(Yh + i * 12, tmp + (i / 2) * 12, sizeof(cplx) * 12);
        }

#pragma omp parallel for schedule(static)
        for (long gi = 0; gi < g.Vg; ++gi) {
            int x[4];
            gcoords(&g, gi, x);
            if (x[0] < 1 || x[0] > T - 1) continue;
            for (int mu = 0; mu < 4; ++mu) {
                int y[4] = {x[0], x[1], x[2], x[3]};
                cplx lam = 1.0;
                if (mu == 0) {
                    y[0] += 1;
                    if (y[0] > T - 1) continue;
                } else {
                    y[mu] = (y[mu] + 1) % L;
                    lam = lam_sp;
                }
                const cplx* Uxm = link(&g, U, x, mu);
                const cplx* Xx = Xh + fidx(&g, x) * 12;
                const cplx* Xy = Xh + fidx(&g, y) * 12;
                const cplx* Yx = Yh + fidx(&g, x) * 12;
                const cplx* Yy = Yh + fidx(&g, y) * 12;
                for (int a = 0; a < 8; ++a) {
                    /* M = i T^a U */
                    cplx M[3][3];
                    for (int c = 0; c < 3; ++c)
                        for (int d = 0; d < 3; ++d) {
                            cplx s = 0;
                            for (int k = 0; k < 3; ++k) s += 0.5 * GELL[a][c][k] * Uxm[k * 3 + d];
                            M[c][d] = I * s;
                        }
                    cplx t1 = 0, t2 = 0;
                    for (int s = 0; s < 4; ++s)
                        for (int q = 0; q < 4; ++q) {
                            cplx pm = (s == q ? 1.0 : 0.0) - GAM[mu][s][q];
                            cplx pp = (s == q ? 1.0 : 0.0) + GAM[mu][s][q];
                            for (int c = 0; c < 3; ++c)
                                for (int d = 0; d < 3; ++d) {
                                    /* Yh(x)^dag (1-g) M Xh(x+mu) */
                                    t1 += conj(Yx[s * 3 + c]) * pm * M[c][d] * Xy[q * 3 + d];
                                    /* Yh(x+mu)^dag (1+g) M^dag Xh(x) */
                                    t2 += conj(Yy[s * 3 + c]) * pp * conj(M[d][c]) * Xx[q * 3 + d];
                                }
                        }
                    F[(gi * 4 + mu) * 8 + a] += 2.0 * kappa * creal(lam * t1 + conj(lam) * t2);
                }
            }
        }
    }
    free(Xh); free(Yh); free(w1); free(w2); free(tmp);
    return 0;
}

/* ------------------------------------------------------ plaquette action */

static void mat_mul(const cplx* A, const cplx* B, cplx* C) /* C = A B */
{
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            cplx s = 0;
            for (int k = 0; k < 3; ++k) s += A[r * 3 + k] * B[k * 3 + c];
            C[r * 3 + c] = s;
        }
}

static void mat_dag(const cplx* A, cplx* B)
{
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) B[r * 3 + c] = conj(A[c * 3 + r]);
}

/*
 * Wilson plaquette action on the SF gauge lattice (Sec. 4: "SU(3) plaquette
 * gauge ... action", beta = 4.52):
 *   S_g = beta sum_p w(p) (1 - Re tr U_p / 3),
 *   U_p = U_mu(x) U_nu(x+mu) U_mu(x+nu)^dag U_nu(x)^dag,
 * over all plaquettes inside x0 = 0..T; w = 1/2 for spatial plaquettes at
 * x0 = 0 and x0 = T, w = c_t = 1 for time-like plaquettes touching a boundary,
 * w = 1 otherwise.
 */
double sfo_plaquette_action(int L, int T, double beta, const double* Ud)
{
    if (check_args(L, T)) return NAN;
    geom g = make_geom(L, T, 0.0, 0);
    const cplx* U = (const cplx*)Ud;
    double S = 0.0;
#pragma omp parallel for reduction(+ : S) schedule(static)
    for (long gi = 0; gi < g.Vg; ++gi) {
        int x[4];
        gcoords(&g, gi, x);
        for (int mu = 0; mu < 4; ++mu)
            for (int nu = mu + 1; nu < 4; ++nu) {
                double w = 1.0;
                if (mu == 0) {
                    if (x[0] > T - 1) continue;   /* time-like plaquette leaves the lattice */
                } else {
                    if (x[0] == 0 || x[0] == T) w = 0.5;
                }
                int xm[4] = {x[0], x[1], x[2], x[3]};
                int xn[4] = {x[0], x[1], x[2], x[3]};
                if (mu == 0) xm[0] += 1; else xm[mu] = (xm[mu] + 1) % L;
                xn[nu] = (xn[nu] + 1) % L; /* nu >= 1 is always spatial */
                cplx A[9], B[9], C[9], D[9], E[9];
                mat_mul(link(&g, U, x, mu), link(&g, U, xm, nu), A);
                mat_dag(link(&g, U, xn, mu), B);
                mat_mul(A, B, C);
                mat_dag(link(&g, U, x, nu), D);
                mat_mul(C, D, E);
                double re_tr = creal(E[0] + E[4] + E[8]);
                S += w * (1.0 - re_tr / 3.0);
            }
    }
    return beta * S;
}

/* ------------------------------------------------------ gauge force */

/* weight of the plaquette with base y0 in the plane {mu, nu} (0 if it is not
 * part of the action): the rules of sfo_plaquette_action */
static double plaq_weight(int T, int y0, int mu, int nu)
{
    if (y0 < 0 || y0 > T) return 0.0;
    if (mu == 0 || nu == 0) return (y0 <= T - 1) ? 1.0 : 0.0;
    return (y0 == 0 || y0 == T) ? 0.5 : 1.0;
}

static void shifted(const geom* g, const int x[4], int nu, int d, int out[4])
{
    out[0] = x[0]; out[1] = x[1]; out[2] = x[2]; out[3] = x[3];
    if (nu == 0) out[0] += d;
    else out[nu] = (out[nu] + d + g->L) % g->L;
}

/*
 * Force of the gauge action for the HMC trajectory around Alg. 2 (the steps
 * either side of the fermion force): F^a_mu(x) = dS_g / d omega^a for
 * U_mu(x) -> exp(i omega^a T^a) U_mu(x).  Every plaquette through U_mu(x),
 * traced from that link, is Re tr(U_mu(x) A) with A its staple, and
 * d/d omega Re tr(e^{i omega T^a} U A) = -Im tr(T^a U A) at omega = 0, so
 *   F^a_mu(x) = (beta / 3) sum_staples w(p) Im tr(T^a U_mu(x) A_p),
 *   up staple   A = U_nu(x+mu) U_mu(x+nu)^dag U_nu(x)^dag        (base x),
 *   down staple A = U_nu(x+mu-nu)^dag U_mu(x-nu)^dag U_nu(x-nu)   (base x-nu).
 * Dynamic links: U_0(x) with x0 = 0..T-1 and U_k(x) with x0 = 1..T-1; the
 * spatial boundary links at x0 = 0, T are fixed and get F = 0.
 */
int sfo_gauge_force(int L, int T, double beta, const double* Ud, double* F)
{
    if (check_args(L, T)) return -1;
    init_tables();
    geom g = make_geom(L, T, 0.0, 0);
    const cplx* U = (const cplx*)Ud;
    memset(F, 0, sizeof(double) * g.Vg * 4 * 8);
#pragma omp parallel for schedule(static)
    for (long gi = 0; gi < g.Vg; ++gi) {
        int x[4];
        gcoords(&g, gi, x);
        for (int mu = 0; mu < 4; ++mu) {
            const int dynamic = (mu == 0) ? (x[0] <= T - 1) : (x[0] >= 1 && x[0] <= T - 1);
            if (!dynamic) continue;
            cplx S[9] = {0};  /* sum of weighted staples */
            for (int nu = 0; nu < 4; ++nu) {
                if (nu == mu) continue;
                int xm[4], xn[4], xmn[4], xnd[4];
                shifted(&g, x, mu, +1, xm);
                /* up */
                const double wu = plaq_weight(T, x[0], mu, nu);
                if (wu != 0.0) {
                    shifted(&g, x, nu, +1, xn);
                    cplx B[9], C[9], D[9], E[9];
                    mat_dag(link(&g, U, xn, mu), B);
                    mat_mul(link(&g, U, xm, nu), B, C);
                    mat_dag(link(&g, U, x, nu), D);
                    mat_mul(C, D, E);
                    for (int k = 0; k < 9; ++k) S[k] += wu * E[k];
                }
                /* down */
                shifted(&g, x, nu, -1, xnd);
                const double wd = plaq_weight(T, xnd[0], mu, nu);
                if (wd != 0.0) {
                    shifted(&g, xm, nu, -1, xmn);
                    cplx B[9], C[9], D[9];
                    mat_dag(link(&g, U, xmn, nu), B);
                    mat_dag(link(&g, U, xnd, mu), C);
                    mat_mul(B, C, D);
                    cplx E[9];
                    mat_mul(D, link(&g, U, xnd, nu), E);
                    for (int k = 0; k < 9; ++k) S[k] += wd * E[k];
                }
            }
            cplx W[9];
            mat_mul(link(&g, U, x, mu), S, W);
            for (int a = 0; a < 8; ++a) {
                cplx tr = 0;  /* tr(lambda^a W) */
                for (int r = 0; r < 3; ++r)
                    for (int c = 0; c < 3; ++c) tr += GELL[a][r][c] * W[c * 3 + r];
                F[(gi * 4 + mu) * 8 + a] = beta / 6.0 * cimag(tr);
            }
        }
    }
    return 0;
}

int sfo_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void sfo_set_num_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}
