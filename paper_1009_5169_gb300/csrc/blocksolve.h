// Device-resident outer iterations of the block solvers of Sec. 3.2 (Table 1
// cases C and D1): Bl-BiCGStab with s x s coefficient matrices and
// Gl-BiCGStab with Frobenius-product scalars.  Every scalar, every s x s
// matrix and every stop decision lives in a state struct in device memory;
// the field updates are fused kernels (one pass over the vectors they touch,
// with the reductions the next decision needs), and small finishing kernels
// (one block) form the lattice sums, take the decisions and set the
// conditions of the CUDA graph the host builds around them.  One lattice,
// nrhs <= BLK_MAX right-hand sides, FP64 fields, one thread per (site, rhs)
// (tile 32, one rhs per thread).
#pragma once
#include "sf_kernels.h"

namespace sf {

constexpr int BLK_MAX = 8;                   // right-hand sides of a block solve
constexpr int BLK_NQ_R = 1 + 4 * BLK_MAX;    // quantities per rhs of the R update

struct BlState {
    // n x n complex matrices, element (i, j) at [i * BLK_MAX + j]
    double2 M[BLK_MAX * BLK_MAX];      // R0^H V
    double2 Qh[BLK_MAX * BLK_MAX];     // Q^H of the QR factorisation of M
    double2 Rf[BLK_MAX * BLK_MAX];     // its R (upper triangle)
    double2 Q[BLK_MAX * BLK_MAX];      // R0^H R
    double2 alpha[BLK_MAX * BLK_MAX];  // M^-1 (R0^H R)
    double2 beta[BLK_MAX * BLK_MAX];   // -M^-1 (R0^H T)
    double2 omega;
    double bb[BLK_MAX];                // |phi_j|^2
    double rr[BLK_MAX];                // |R_j|^2 of the last recursive residual
    double stop2, tol2;                // (tol / 2)^2 for the recursive residual, tol^2 for the true one
    int n, iters, maxiter, cycles, max_cycles, stop, fail;
    int body_runs, if_runs;            // executions of the iteration body and of its second half
};

struct GlState {
    double2 rho, alpha, omega, beta;
    double bb[BLK_MAX];
    double rr[BLK_MAX];
    double stop2, tol2, delta2;        // delta: relative residual of a preconditioner call
    int n, iters, max_outer, cycles, max_cycles, calls, stop, fail;   // iters: of the current cycle
    int body_runs, if_runs;
};

// ---- Bl-BiCGStab (partials: BLK_NQ_R * BLK_MAX * max(nblocks) doubles)
// state start: bb = |phi|^2 (device), counters cleared, the cycle loop opened
cudaError_t launch_bl_init(BlState* st, int n, const double* bb, double tol, int maxiter, int max_cycles,
                           cudaGraphConditionalHandle h_cycle, cudaStream_t);
// cycle start from the Gram partials of (R0, R), R0 = R: Q, the stop test, the iteration loop's condition
cudaError_t launch_bl_fin_q(BlState* st, const double* partials, int nblocks, cudaGraphConditionalHandle h_iter,
                            cudaStream_t);
// M = R0^H V from its Gram partials, M = Q R (Householder, one warp), alpha = M^-1 Q
cudaError_t launch_bl_fin_alpha(BlState* st, const double* partials, int nblocks, cudaStream_t);
// S = R - V alpha, X += P alpha, |S_j|^2 partials (skipped once stopped)
cudaError_t launch_bl_s(const LaunchCfg&, BlState* st, FieldPtr R, FieldPtr V, FieldPtr P, FieldPtr S, FieldPtr X,
                        double* partials, cudaStream_t);
// the half-step test on |S|^2; opens the IF node of the second half
cudaError_t launch_bl_fin_s(BlState* st, const double* partials, int nblocks, cudaGraphConditionalHandle h_if,
                            cudaStream_t);
// omega = <T, S>_F / <T, T>_F from the RED_TS partials of T = A S
cudaError_t launch_bl_fin_omega(BlState* st, const double* partials, int nblocks, cudaStream_t);
// X += omega S, R = S - omega T; partials |R_j|^2, <R0_i, R_j>, <R0_i, T_j>
cudaError_t launch_bl_r(const LaunchCfg&, BlState* st, FieldPtr S, FieldPtr T, FieldPtr R0, FieldPtr X, FieldPtr R,
                        double* partials, cudaStream_t);
// the stop test on |R|^2, Q = R0^H R, beta = -M^-1 (R0^H T) from the stored QR factors
cudaError_t launch_bl_fin_r(BlState* st, const double* partials, int nblocks, cudaStream_t);
// P = R + (P - omega V) beta in place (skipped once stopped); sets the iteration loop's condition
cudaError_t launch_bl_p(const LaunchCfg&, BlState* st, FieldPtr P, FieldPtr V, FieldPtr R,
                        cudaGraphConditionalHandle h_iter, cudaStream_t);
// after the FP64 true residual |phi - A X|^2 (rr): another cycle while a rhs is above tol
cudaError_t launch_bl_cycle(BlState* st, const double* rr, cudaGraphConditionalHandle h_cycle, cudaStream_t);

// ---- Gl-BiCGStab
cudaError_t launch_gl_init(GlState* st, int n, const double* bb, double tol, double delta, int max_outer,
                           int max_cycles, OState* ost, cudaGraphConditionalHandle h_cycle, cudaStream_t);
// cycle start: rho = <R0, R>_F and |R_j|^2 (R0 = R) from the k_gl_ts partials of (R0, R)
cudaError_t launch_gl_fin_start(GlState* st, const double* partials, int nblocks, cudaGraphConditionalHandle h_iter,
                                cudaStream_t);
// a preconditioner call on a vector with |in_j|^2 = nin: the outer states of
// the FP32 inner solves (skip a rhs below tol |phi_j|, inner target
// max(delta, 0.1 tol |phi_j| / |in_j|)); counts the call
cudaError_t launch_gl_prep(GlState* st, OState* ost, const double* nin, cudaStream_t);
// alpha = rho / <R0, V>_F from the RED_R0V partials of V = A PH
cudaError_t launch_gl_fin_alpha(GlState* st, const double* partials, int nblocks, cudaStream_t);
// S = R - alpha V, X += alpha PH, |S_j|^2 partials
cudaError_t launch_gl_s(const LaunchCfg&, GlState* st, FieldPtr R, FieldPtr V, FieldPtr PH, FieldPtr S, FieldPtr X,
                        double* partials, cudaStream_t);
cudaError_t launch_gl_fin_s(GlState* st, const double* partials, int nblocks, cudaGraphConditionalHandle h_if,
                            cudaStream_t);
// <T, S> and |T|^2 partials (3 per rhs)
cudaError_t launch_gl_ts(const LaunchCfg&, GlState* st, FieldPtr T, FieldPtr S, double* partials, cudaStream_t);
cudaError_t launch_gl_fin_omega(GlState* st, const double* partials, int nblocks, cudaStream_t);
// X += omega SH, R = S - omega T; partials |R_j|^2, <R0_j, R_j>
cudaError_t launch_gl_r(const LaunchCfg&, GlState* st, FieldPtr S, FieldPtr T, FieldPtr SH, FieldPtr R0,
                        FieldPtr X, FieldPtr R, double* partials, cudaStream_t);
// the stop test, rho' = <R0, R>_F, beta = (rho' / rho)(alpha / omega)
cudaError_t launch_gl_fin_r(GlState* st, const double* partials, int nblocks, cudaStream_t);
// P = R + beta (P - omega V) (skipped once stopped); sets the iteration loop's condition
cudaError_t launch_gl_p(const LaunchCfg&, GlState* st, FieldPtr P, FieldPtr V, FieldPtr R,
                        cudaGraphConditionalHandle h_iter, cudaStream_t);
cudaError_t launch_gl_cycle(GlState* st, const double* rr, cudaGraphConditionalHandle h_cycle, cudaStream_t);

}  // namespace sf
