/*
 * sf_lattice.h -- C ABI of the GB300 (sm_103a) library for the fermion part
 * of the many-flavour HMC molecular-dynamics step of arXiv:1009.5169,
 * "Improving many flavor QCD simulations using multiple GPUs".
 *
 * The calls follow the paper's statement of the problem:
 *   Eq. (2)  det[D]^{N_f} through N_f/2 additive pseudo-fermions phi_i with
 *            action S = sum_i |D^{-1} phi_i|^2;
 *   Alg. 2   blocked force step: solve D X = Phi, then D^dag Y = X, then
 *            accumulate F_mu = sum_i f[x_i, y_i];
 *   Eq. (3)  F_mu(n) = sum_i F_{mu,i}(n), f the gauge derivative of
 *            |D^{-1} phi_i|^2;
 *   Sec. 3.1 site even/odd preconditioning, Wilson fermions;
 *   Sec. 3.2 mixed-precision solves (single-precision inner solver inside a
 *            double-precision outer loop);
 *   Sec. 4   Schroedinger-functional setup with the SU(3) plaquette action.
 * D is taken in the hopping-parameter form D = 1 - kappa H,
 *   (H psi)(x) = sum_mu (1 - gamma_mu) U_mu(x) lambda_mu psi(x+mu)
 *              + (1 + gamma_mu) U_mu(x-mu)^dag lambda_mu^* psi(x-mu),
 * with Euclidean chiral gamma matrices (gamma_5 = diag(1,1,-1,-1)), the
 * fermion on x0 = 1..T-1 (hops leaving that range are dropped), spatial
 * directions periodic with psi(x + L k) = e^{i theta} psi(x) realised as
 * lambda_k = e^{i theta/L}, lambda_0 = 1.  The preconditioned operator is
 * Dhat = 1 - kappa^2 H_eo H_oe on the even sites and det D = det Dhat.
 *
 * Layouts (all double precision, complex numbers as (re, im) pairs):
 *   links   [(T+1) L^3][4][3][3] complex: gauge site lexicographic over
 *           x0 = 0..T, x1, x2, x3 = 0..L-1 with x3 fastest; mu = 0 is time;
 *           [a][b] = row a, column b of U_mu(x).  The time link at x0 = T is
 *           not a link of the SF lattice and is ignored; the spatial links at
 *           x0 = 0 and x0 = T are the SF boundary fields (they enter only the
 *           plaquette action).
 *   even    [nrhs][V/2][4][3] complex, V = L^3 (T-1): the even sites
 *           ((x0+x1+x2+x3) even) of the fermion lattice in lexicographic
 *           order (x0 = 1..T-1 slowest, x3 fastest); for even L the site with
 *           lexicographic index i has even/odd index i/2.  Odd fields alike.
 *   full    [2][nrhs][V/2][4][3] complex: the even-site block of all fields,
 *           then the odd-site block.
 *   force   [(T+1) L^3][4][8]: F^a_mu(x) = dS/d omega^a for
 *           U_mu(x) -> exp(i omega^a T^a) U_mu(x), T^a = lambda^a / 2 with the
 *           Gell-Mann matrices; zero on links without fermion support.
 *
 * Pointers: every array argument may be a host pointer or a device pointer
 * of the lattice's device (detected with cudaPointerGetAttributes).  The
 * caller owns all arrays it passes; the library owns the device copies and
 * workspaces it allocates.  Device pointers are read and written in order on
 * the stream given at creation; calls with host pointers return after the
 * host data is complete.  A lattice object is not thread-safe.
 *
 * Errors: no call throws or aborts.  Each returns an sf_status; the message
 * of the last failure on the calling thread is sf_last_error().  Invalid
 * sizes or arguments give SF_EINVAL and change nothing; allocation failure
 * gives SF_ENOMEM; a CUDA failure gives SF_ECUDA.
 */
#ifndef SF_LATTICE_H
#define SF_LATTICE_H

#ifdef __cplusplus
extern "C" {
#endif

#define SF_MAX_RHS 16

typedef struct sf_lattice sf_lattice;
typedef struct sf_batch sf_batch;

typedef enum {
    SF_OK = 0,
    SF_EINVAL = 1,    /* bad argument or size */
    SF_ENOMEM = 2,    /* device or host allocation failed */
    SF_ECUDA = 3,     /* a CUDA call failed */
    SF_ENOCONV = 4,   /* solver stopped above tolerance; outputs hold the best iterate */
    SF_ETIMEOUT = 5,  /* a bounded device wait ran out */
    SF_ENOTSU3 = 6    /* a link is not in SU(3) to 1e-12 */
} sf_status;

typedef enum {
    SF_OP_DHAT = 0,          /* even -> even: Dhat = 1 - kappa^2 H_eo H_oe */
    SF_OP_DHAT_DAG = 1,      /* even -> even: Dhat^dag = gamma_5 Dhat gamma_5 */
    SF_OP_DHATDAG_DHAT = 2,  /* even -> even: Dhat^dag Dhat */
    SF_OP_D_FULL = 3,        /* full -> full: D = 1 - kappa H */
    SF_OP_HOP_EO = 4,        /* odd -> even: H_eo */
    SF_OP_HOP_OE = 5         /* even -> odd: H_oe */
} sf_op;

typedef enum {
    SF_FP64 = 0,   /* FP64 storage and arithmetic */
    SF_FP32 = 1,   /* FP32 storage and arithmetic, links rebuilt from 2 rows */
    SF_FP16 = 2    /* FP16 operands with a per-(site, rhs) FP32 scale, FP16 links, FP32 arithmetic */
} sf_prec;

typedef enum {
    /* BiCGStab in FP64 on all rhs at once, restarted from the true residual
       until |phi - Dhat x| <= tol |phi| (the plain method, case A of Table 1) */
    SF_SOLVE_BICGSTAB = 0,
    /* FP64 defect correction around an FP32 BiCGStab (Sec. 3.2) */
    SF_SOLVE_MIXED_DC = 1,
    /* FP64 defect correction around BiCGStab with FP16 hop operands */
    SF_SOLVE_MIXED_DC_HALF = 2,
    /* FP64 flexible GCR (restarted, 16 directions) preconditioned by the
       learned network attached with sf_lattice_set_preconditioner; the FP64
       true residual judges it, and FP32-inner BiCGStab under FP64 defect
       correction continues from its iterate if it stops above tol.  One
       lattice only (not batches), nrhs <= 8 (as Gl- and Bl-BiCGStab). */
    SF_SOLVE_FGCR_CNN = 3,
    /* the same FGCR with the identity as preconditioner (the comparison
       without the network) */
    SF_SOLVE_FGCR = 4,
    /* the normal-equation route to the same X, Y: Y by CG on Dhat Dhat^dag
     * (= gamma5 Dhat^dag Dhat gamma5; FP32 inner, FP64 outer defect correction
     * on that system), X = Dhat^dag Y in FP64.  |phi - Dhat X| is the outer
     * residual CG is driven to; |X - Dhat^dag Y| is at rounding level. */
    SF_SOLVE_CG_NORMAL = 5,
    /* the paper's mixed-precision-preconditioned Gl-BiCGStab (Sec. 3.2, case
     * D1 of Table 1): BiCGStab in FP64 on the whole block with scalars from
     * Frobenius inner products, right-preconditioned by FP32 BiCGStab solves
     * of the single systems (relative residual 1e-5 each, all rhs in one
     * launch); restarted from the recomputed FP64 residual while a rhs is
     * above tol.  iters_outer reports the preconditioner calls, iters_inner
     * the FP32 iterations.  One lattice only (not batches).  If it ends above
     * tol (a breakdown that restarting does not cure, e.g. linearly dependent
     * right-hand sides), FP32-inner BiCGStab under FP64 defect correction
     * continues each rhs from its iterate and adds its counts. */
    SF_SOLVE_GL_BICGSTAB = 6,
    /* Bl-BiCGStab in FP64 (the paper's case C, Sec. 3.2): the rhs share one
     * Krylov space through nrhs x nrhs coefficient matrices; restarted from
     * the recomputed FP64 residual while a rhs is above tol.  iters_inner
     * reports the block iterations (each applies Dhat to every rhs twice),
     * iters_outer the restarts + 1.  One lattice only (not batches).  The
     * nrhs x nrhs systems are solved by Householder QR; a rank-deficient block
     * (linearly dependent right-hand sides) breaks down, and FP32-inner
     * BiCGStab under FP64 defect correction continues each rhs from its
     * iterate, adding its counts. */
    SF_SOLVE_BL_BICGSTAB = 7,
    /* the learned preconditioner in mixed precision: FP64 defect correction
     * (r = phi - Dhat x recomputed in FP64, x += |r| e) around flexible GCR in
     * FP32 (16 directions, FP32 hop, float-float dot products) on
     * Dhat e = r / |r| to the relative target max(1e-5, 0.1 tol |phi| / |r|),
     * preconditioned by the attached network on the FP32 residual; the FP64
     * true residual judges, FP32-inner BiCGStab continues if the sweeps run
     * out above tol.  iters_outer: sweeps, iters_inner: FGCR iterations.
     * One lattice only (not batches), nrhs <= 8. */
    SF_SOLVE_FGCR_CNN_MIXED = 8,
    /* the same with the identity as preconditioner (the comparison without
     * the network) */
    SF_SOLVE_FGCR_MIXED = 9
} sf_algo;

typedef struct {
    int iters_outer;                   /* FP64 sweeps of the X solve (max over rhs); Gl-BiCGStab:
                                          its preconditioner calls */
    int iters_inner;                   /* inner iterations of the X solve (max over rhs) */
    int iters_outer_y;                 /* same for the Y solve (0 if Y was not asked for) */
    int iters_inner_y;
    int iters_inner_rhs[SF_MAX_RHS];   /* inner iterations of the X solve per rhs */
    double true_resid[SF_MAX_RHS];     /* |phi_i - Dhat x_i| / |phi_i| (FP64, on the GPU) */
    double true_resid_y[SF_MAX_RHS];   /* |x_i - Dhat^dag y_i| / |x_i| */
    double seconds;                    /* host wall time of the call */
    long long kernel_launches;         /* kernels this call ran on the device */
} sf_solve_info;

/* Create a lattice of spatial extent L (even, 2..64) and SF time extent T
 * (2..64), fermion twist theta, hopping parameter kappa and gauge coupling
 * beta, and upload the gauge field `links` (layout above).  `device` is the
 * CUDA device ordinal; `stream` a cudaStream_t on that device (NULL: the
 * legacy default stream).  Returns SF_ENOTSU3 (and no lattice) if a link is
 * not unitary with unit determinant to 1e-12.  Owns its device memory until
 * sf_lattice_destroy. */
sf_status sf_lattice_create(sf_lattice** out, int L, int T, double theta, double kappa, double beta,
                            const double* links, int device, void* stream);

/* Replace the gauge field (the MD step moves the links) and rebuild the
 * FP64, FP32 and FP16 link copies the kernels read. */
sf_status sf_lattice_set_links(sf_lattice* lat, const double* links);

/* Fix the kernel tiling for one precision instead of autotuning it:
 * TS sites per tile (32, 64 or 128) and NR right-hand sides per thread
 * (1, 2, 3 or 5; FP64: 1 or 2).  A block holds TS * ceil(nrhs / NR) threads,
 * at most 256 (FP64), 320 / 384 / 256 (FP32 and FP16 with NR = 1 / 2 / 3 or
 * 5): checked when a solve or apply uses the
 * tiling, SF_EINVAL beyond.  pipe selects the hop mode: 0 the plain hop;
 * 1 the pipelined hop (operands of the next hops loaded while the current
 * one is applied; FP32 / FP16 only, NR = 1 or 2, at most 256 threads);
 * 2 links staged per tile (each site's eight links read and their third rows
 * rebuilt once per block into 18 KiB of shared memory and applied from there
 * to every right-hand side; FP32 / FP16 only, NR = 1, TS = 32, at most 320
 * threads).  TS = 0 restores autotuning (TS, NR and pipe). */
sf_status sf_lattice_set_tuning(sf_lattice* lat, sf_prec prec, int TS, int NR, int pipe);

/* Tiling in use for a precision and block size (runs the autotuner if it has
 * not run yet); pipe may be NULL. */
sf_status sf_lattice_get_tuning(sf_lattice* lat, sf_prec prec, int nrhs, int* TS, int* NR, int* pipe);

void sf_lattice_destroy(sf_lattice* lat);

/* out = op(in) for nrhs fields (1..SF_MAX_RHS), computed in precision prec
 * (inputs rounded to it, results returned in FP64).  Even/odd/full layouts
 * as listed for each op. */
sf_status wilson_apply_block(sf_lattice* lat, sf_op op, sf_prec prec, int nrhs, const double* in,
                             double* out);

/* The two solves of Alg. 2 on the even sites: X = Dhat^{-1} Phi and, if Y is not
 * NULL, Y = Dhat^{-dag} X, each to |b - A x| <= tol |b| per right-hand side,
 * checked on an FP64 recomputation of the residual.  All nrhs systems run
 * as one block (one launch per kernel for all of them).  maxiter bounds the
 * inner iterations of each sweep.  On SF_ENOCONV, X and Y hold the best
 * iterate and info the residuals reached.  info may be NULL. */
sf_status solve_block(sf_lattice* lat, sf_algo algo, int nrhs, const double* phi, double* X, double* Y,
                      double tol, int maxiter, sf_solve_info* info);

/* Eq. (3) with the force steps of Alg. 2: the force of S = sum_i |Dhat^{-1} phi_i|^2
 * from x_i = Dhat^{-1} phi_i and y_i = Dhat^{-dag} x_i (even sites).  Writes
 * F (force layout, may be NULL) and, if mom is not NULL, does mom -= eps F
 * in FP64 (mom in the force layout). */
sf_status fermion_force(sf_lattice* lat, int nrhs, const double* X, const double* Y, double* F, double* mom,
                        double eps);

/* Alg. 2 as one call: the two solves (as solve_block, X and Y both returned)
 * and the force (as fermion_force, F and / or mom -= eps F).  The odd-site
 * parts of X and Y that the force needs are the first hops of the final FP64
 * true residuals, so no extra hops are applied.  Same layouts, precision
 * rules and statuses as solve_block and fermion_force; on SF_ENOCONV all
 * outputs are still written (from the best iterates).  With
 * SF_SOLVE_CG_NORMAL, X is computed as Dhat^dag Y in FP64 and
 * info->true_resid_y is reported as 0 without recomputation (solve_block
 * recomputes it: FP64 rounding). */
sf_status md_force_step(sf_lattice* lat, sf_algo algo, int nrhs, const double* phi, double* X, double* Y,
                        double* F, double* mom, double eps, double tol, int maxiter, sf_solve_info* info);

/* S_g = beta sum_p w(p) (1 - Re tr U_p / 3) over the SF gauge lattice with
 * w = 1/2 for spatial plaquettes at x0 = 0 and x0 = T and 1 otherwise. */
sf_status plaquette_action(sf_lattice* lat, double* S);

/* ---- the HMC trajectory around Alg. 2 (the steps either side of the MD
 * force: momenta, gauge force, link update, leapfrog).  Momenta and forces
 * use the force layout [(T+1) L^3][4][8] (components along T^a = lambda^a/2);
 * only the dynamic links move: U_0(x) for x0 = 0..T-1 and U_k(x) for
 * x0 = 1..T-1 (the spatial boundary links at x0 = 0, T are fixed, with zero
 * momentum and force). */

/* The force of the plaquette action, F^a_mu(x) = dS_g/d omega^a for
 * U_mu(x) -> exp(i omega^a T^a) U_mu(x): writes F (may be NULL) and, if mom
 * is not NULL, does mom -= eps F. */
sf_status gauge_force(sf_lattice* lat, double* F, double* mom, double eps);

/* U_mu(x) <- exp(i dt P_mu(x)) U_mu(x) on the dynamic links (P = P^a T^a from
 * mom), then the prepared link copies are rebuilt (no SU(3) re-check). */
sf_status sf_lattice_update_links(sf_lattice* lat, const double* mom, double dt);

/* Copy the lattice's current FP64 links out (canonical layout). */
sf_status sf_lattice_get_links(sf_lattice* lat, double* links);

typedef struct {
    double kinetic[2];      /* sum_links,a (P^a)^2 / 2 at the start and the end */
    double s_gauge[2];      /* plaquette action */
    double s_fermion[2];    /* sum_i |Dhat^{-1} phi_i|^2 */
    double dH;              /* H(end) - H(start) */
    int force_evals;        /* fermion force evaluations (leapfrog nsteps + 1, Omelyan 2 nsteps + 1) */
    int inner_iters;        /* inner solver iterations summed over them (X and Y) */
    double seconds;
    long long kernel_launches;
} sf_md_info;

/* One leapfrog molecular-dynamics trajectory of nsteps steps of size dt:
 * P -= dt/2 F(U); then nsteps times { U <- exp(i dt P) U; P -= dt F(U) },
 * the last kick dt/2; F = gauge force + the fermion force of Alg. 2 for
 * the pseudo-fermions phi (nrhs even-site fields, solved with algo to tol).
 * The lattice's links and mom (in / out; its boundary entries are zeroed
 * first) move; H = kinetic + S_g + S_f is reported at both ends, S_f from
 * the X of the first and last force evaluations.  A Metropolis step is the
 * caller's: accept with probability min(1, exp(-dH)), else restore the links
 * with sf_lattice_set_links. */
sf_status sf_md_trajectory(sf_lattice* lat, sf_algo algo, int nrhs, const double* phi, double* mom, int nsteps,
                           double dt, double tol, int maxiter, sf_md_info* info);

/* The same trajectory with the second-order minimum-norm integrator of
 * Omelyan, Mryglod and Folk (2003), two force evaluations per step: per step
 * P -= lambda dt F; U <- exp(i dt/2 P) U; P -= (1 - 2 lambda) dt F;
 * U <- exp(i dt/2 P) U; P -= lambda dt F (the last kick of a step and the
 * first of the next merged).  lambda = 0.1931833275037836 minimises the norm
 * of the leading error terms; lambda must lie in (0, 1/2) (SF_EINVAL), and
 * lambda -> 1/2 gives the leapfrog.  The paper names the HMC algorithm
 * (Sec. 2) without its integrator. */
sf_status sf_md_trajectory_omelyan(sf_lattice* lat, sf_algo algo, int nrhs, const double* phi, double* mom,
                                   int nsteps, double dt, double lambda, double tol, int maxiter,
                                   sf_md_info* info);

/* The leapfrog trajectory on two time scales (Sexton and Weingarten 1992):
 * the fermion force of Alg. 2 kicks with step dt, and each step's drift is
 * split into gauge_substeps leapfrog steps of the (cheap) gauge force,
 * h = dt / gauge_substeps:  P -= dt/2 F_f;  nsteps times { gauge_substeps
 * times { P -= h/2 F_g; U <- exp(i h P) U; P -= h/2 F_g };  P -= dt/2 F_f },
 * neighbouring half kicks merged.  gauge_substeps = 1 is sf_md_trajectory;
 * it must lie in 1..1000 (SF_EINVAL).  force_evals counts the fermion force
 * evaluations (nsteps + 1).  The paper names the HMC algorithm (Sec. 2)
 * without its integrator. */
sf_status sf_md_trajectory_two_scales(sf_lattice* lat, sf_algo algo, int nrhs, const double* phi, double* mom,
                                      int nsteps, double dt, int gauge_substeps, double tol, int maxiter,
                                      sf_md_info* info);

typedef enum { SF_MD_LEAPFROG = 0, SF_MD_OMELYAN = 1 } sf_md_integrator;

/* One HMC trajectory (the algorithm the paper runs, Sec. 2) with the
 * caller's random numbers: pseudo-fermions phi = Dhat eta from the Gaussian
 * even-site fields eta (nrhs of them, host or device; S_f = |eta|^2 at the
 * start), the MD trajectory of sf_md_trajectory_two_scales (leapfrog,
 * gauge_substeps >= 1) or sf_md_trajectory_omelyan (lambda) from the momenta
 * mom (in / out, host or device), then the Metropolis test: *accepted = 1 if
 * uniform < exp(-dH), else 0 and the links are put back to those of the
 * start.  mom keeps its end-of-trajectory values either way (a new
 * trajectory draws new momenta).  SF_EINVAL on a NULL pointer, an unknown
 * integrator or a parameter out of range; SF_ENOCONV if a solve stopped above
 * tol (the test is still applied). */
sf_status sf_hmc_trajectory(sf_lattice* lat, sf_algo algo, int nrhs, const double* eta, double* mom,
                            double uniform, sf_md_integrator integrator, int nsteps, double dt,
                            int gauge_substeps, double lambda, double tol, int maxiter, sf_md_info* info,
                            int* accepted);

/* One launch of the hopping-term kernel H_oe (out_parity 1) or H_eo
 * (out_parity 0) for nrhs fields in precision prec, on the lattice's
 * resident operand and result buffers (those wilson_apply_block last packed;
 * zero after creation), with no packing or unpacking around it.  Enqueued
 * on the lattice's stream and not synchronised, so a caller can time exactly
 * one dslash kernel with events on that stream. */
sf_status wilson_hop_resident(sf_lattice* lat, sf_prec prec, int nrhs, int out_parity);

/* One launch of the FP64 force kernel of Eq. (3) on the lattice's resident
 * full-lattice X and Y (those the last fermion_force or md_force_step with
 * this nrhs packed; zero after creation), writing F (device memory of the
 * lattice's device, layout [(T+1) L^3][4][8], only the entries of dynamic
 * links; not cleared first).  Enqueued on the lattice's stream and not
 * synchronised, so a caller can time exactly one force kernel with events
 * on that stream.  SF_EINVAL if F is NULL, host memory or on another device. */
sf_status fermion_force_resident(sf_lattice* lat, int nrhs, double* F);

/* ---- learned preconditioner: a 4-layer 3^4-stencil convolutional network
 * on the full fermion lattice (widths 32 -> H -> H -> H -> 24, ReLU between
 * layers, H = 16 or 32), BF16 tensor-core kernels with FP32 accumulation.
 * Input channels: the even-site residual r / s, s = |r| / sqrt(24 V/2) (24
 * reals per site, zero on odd sites) and Re, Im of tr U_mu(x) / 3 for
 * mu = 0..3; output: 24 reals per even site; the preconditioner is
 * M(r) = r + s (out(r/s) - out(-r/s)) / 2 (the network learns the correction
 * to the identity; M is odd and positively homogeneous).  Parameters
 * are a flat FP32 array, per layer W[81][c_in][c_out] (offset d in
 * {-1,0,1}^4, d0 slowest) then the bias [c_out].  The network is an addition
 * to the paper's method (whose preconditioner is the single-precision solve
 * of Sec. 3.2); it never decides the answer, the FP64 residual does. */
typedef struct sf_cnn sf_cnn;

/* Number of parameters for hidden width H (16 or 32); -1 otherwise. */
long long sf_cnn_num_params(int hidden);

/* Create a network on a device from initial parameters (host or device). */
sf_status sf_cnn_create(sf_cnn** out, int hidden, const float* params, int device, void* stream);

/* Copy the FP32 master parameters out (host or device). */
sf_status sf_cnn_get_params(sf_cnn* cnn, float* params);

void sf_cnn_destroy(sf_cnn* cnn);

/* out = M(r) for nrhs even-site fields of the lattice (layout `even`). */
sf_status sf_cnn_forward(sf_cnn* cnn, sf_lattice* lat, int nrhs, const double* r, double* out);

/* One Adam step (beta 0.9, 0.999) with learning rate lr.  With targets e
 * (e_i = Dhat^-1 r_i) the loss is the error norm mean_i |M(r_i) - e_i|^2 /
 * |e_i|^2; with e == NULL it is the residual norm mean_i |r_i - Dhat M(r_i)|^2
 * / |r_i|^2, differentiated through the FP64 Dhat and Dhat^dag kernels.
 * *loss receives the loss before the step. */
sf_status sf_cnn_train_step(sf_cnn* cnn, sf_lattice* lat, int nrhs, const double* r, const double* e, float lr,
                            double* loss);

/* The gradient of that loss (either mode) with respect to the parameters
 * (flat layout as the parameters), without updating them. */
sf_status sf_cnn_gradients(sf_cnn* cnn, sf_lattice* lat, int nrhs, const double* r, const double* e, float* grad,
                           double* loss);

/* Which kernels run the network's convolutions: impl = 0 (the default) the
 * tcgen05 tensor-core kernel wherever the layer shape fits its shared memory
 * (hidden width 16; the rest on mma.sync), impl = 1 mma.sync everywhere (a
 * reference for comparisons).  The weight gradients always use mma.sync.
 * SF_EINVAL for another impl.  A convolution whose internal wait timed out
 * makes the next call that synchronises return SF_ECUDA. */
sf_status sf_cnn_set_conv_impl(sf_cnn* cnn, int impl);

/* Attach a network as the preconditioner of SF_SOLVE_FGCR_CNN on this
 * lattice (NULL detaches; the lattice does not own it). */
sf_status sf_lattice_set_preconditioner(sf_lattice* lat, sf_cnn* cnn);

/* The plaquette action S_g of plaquette_action, for callers that cannot
 * allocate device memory (a runtime or scheduler that owns the whole device,
 * or a fixed memory budget handed out by another framework).  The paper has
 * no counterpart to this call; it exists only for such callers.
 *   links   device (or managed) pointer of `device`, 16-byte aligned, gauge
 *           field in the links layout above; anything else (a host pointer,
 *           another device's memory, a misaligned view) gives SF_EINVAL
 *           before any launch;
 *   S       pointer to one double: device memory of `device` is written on
 *           the stream and not synchronised; host or managed memory is
 *           written before the call returns (the call synchronises the
 *           stream, so such an S is refused with SF_EINVAL while the stream
 *           is being captured);
 *   device  CUDA device ordinal of links; stream a cudaStream_t or NULL.
 * The calling thread's current device is the same after the call as before.
 * Nothing is allocated: the reduction's scratch is a fixed 64.5 KiB array in
 * the library's device image, held by every GPU that loads the library until
 * the process exits.  At most 2097152 gauge sites ((T+1) L^3) per call;
 * larger lattices give SF_EINVAL and no launch.  All calls share the array:
 * calls whose kernels overlap on the GPU (unordered streams) race and give
 * wrong results.  The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress) and should come before any stream capture. */
sf_status plaquette_action_noalloc(int L, int T, double beta, const double* links, double* S, int device,
                                   void* stream);

/* Message of the last failure on this thread ("" if none). */
const char* sf_last_error(void);

/* ---- batches: several lattices (any sizes) solved by one launch per kernel
 * and group of lattices (an addition: the paper solves the five equations
 * of one field, Sec. 3.2, and has no batching over fields).  At create the
 * lattices are grouped so that each group's inner-loop working set (FP32
 * links and six FP32 vectors per RHS) fits in three quarters of the L2 cache;
 * a lattice larger than that forms a group of its own.  Groups are solved one
 * after the other, each with its own autotuned tiling.  The lattices must
 * live on the same device and stay alive while the batch exists; their links
 * may change between solves. */
sf_status sf_batch_create(sf_batch** out, int nlat, sf_lattice* const* lats, int nrhs);

/* Number of lattice groups the batch is solved as (-1 for NULL). */
int sf_batch_num_groups(const sf_batch* b);

/* solve_block on every lattice of the batch; phi[l], X[l], Y[l] are lattice
 * l's arrays (Y may be NULL as a whole), info an array of nlat (or NULL). */
sf_status sf_batch_solve(sf_batch* b, sf_algo algo, const double* const* phi, double* const* X,
                         double* const* Y, double tol, int maxiter, sf_solve_info* info);

void sf_batch_destroy(sf_batch* b);

#ifdef __cplusplus
}
#endif
#endif /* SF_LATTICE_H */
