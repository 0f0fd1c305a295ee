// sf_kernels.h -- host-side launch interface of the sm_103a kernels.
// Each precision configuration (field storage of the Krylov vectors, PV, and
// of the hop operands, PH) is compiled in its own translation unit and
// exposes one table of launchers.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "sf_device.cuh"

namespace sf {

enum class Prec : int { F64 = 0, F32 = 1, F16 = 2 };

// reductions fused into the tail of a D-hat application (RED_CG: |x|^2 of
// the tail's x operand and |out|^2, and the start of a CG step: see k_tail)
enum Red : int { RED_NONE = 0, RED_R0V = 1, RED_TS = 2, RED_NORM = 3, RED_CG = 4 };

// Per (lattice, rhs) state of one Krylov iteration, in device memory.  CG
// keeps gamma = |r|^2 in rho.x and its step length in alpha.x; the *_prev
// fields are the copies the CG step reads while its first block of each
// lattice writes the new values.
struct KState {
    double2 rho, alpha, omega, beta;
    float2 alpha_f, omega_f, beta_f;  // the same coefficients for the FP32 kernels
    double rr;        // |r|^2 of the iterated residual
    double target2;   // iterate while rr > target2
    int active;       // 1 while this rhs iterates
    int iters;        // iterations done in this inner solve
    int maxiter;      // inner cap
    int flags;        // bit 0: breakdown (rho or <r0,v> = 0), bit 1: omega = 0
    double gamma_prev, alpha_prev;  // CG: gamma and alpha of the previous step
    int active_prev, iters_prev;    // CG: active and iters before the current step
};

// Per (lattice, rhs) state of the FP64 defect-correction loop.
struct OState {
    double bb;        // |phi|^2
    double rr;        // |phi - Dhat x|^2 of the last true residual
    double tol2;      // stop when rr <= tol2 * bb
    double delta2_floor;  // inner relative target (squared) the precision can reach
    double delta2;    // inner relative target (squared) of the current sweep
    double inv_norm;  // 1 / |r| used to normalise the inner right-hand side
    int active;       // still above tolerance
    int sweeps;
    int inner_iters;  // cumulative inner iterations
    int pad_;
};

struct LaunchCfg {
    const LatDev* lats;   // device array
    int nlat;
    int nrhs;
    int TS;               // sites per tile (multiple of 32)
    int NR;               // right-hand sides per thread (1, 2, 3 or 5)
    int nblocks;          // total blocks (sum of lattice nblk)
    int pipe;             // hop mode: 0 plain, 1 pipelined (FP32 / FP16, NR <= 2, TS * groups <= 256),
                          // 2 links staged per tile (FP32 / FP16, NR = 1, TS 32 or 64, <= 320 threads)
};

struct SolverCtx {
    KState* st;           // [nlat * nrhs]
    OState* ost;          // [nlat * nrhs]
    double* partials;     // [3 * nrhs * nblocks] per-block partial sums (k_finish adds them)
    int* loop_count;      // [0] iterations of the WHILE loop, [1] their cap, [2] continue flag, [3] solve total
    cudaGraphConditionalHandle cond;
    int use_cond;
};

// Untyped field handle: planes plus (FP16 only) the per-site scales.
struct FieldPtr {
    void* v;
    float* s;
};

// The vectors of the inner BiCGStab (ph, sh: hop-operand copies of p, s when
// the hop operands are stored in another precision).
struct IterFields {
    FieldPtr x, r, r0, p, v, s, t, tmp, ph, sh;
};

struct KrylovOps {
    Prec pv, ph;
    // out(parity) = coef kappa_l^kpow H in  (hop operands, PH storage);
    // with ctx, right-hand sides whose KState is inactive are skipped
    cudaError_t (*hop)(const LaunchCfg&, int out_par, bool dag, FieldPtr in, FieldPtr out, double coef, int kpow,
                       const SolverCtx*, cudaStream_t);
    // out = a xv + coef kappa_l^kpow H hin (+ zv) with an optional fused reduction
    cudaError_t (*tail)(const LaunchCfg&, int out_par, bool dag, int red, FieldPtr hin, FieldPtr xv,
                        FieldPtr zv, FieldPtr out, FieldPtr ra, double a, double coef, int kpow,
                        const SolverCtx*, double* norm_out, cudaStream_t);
    // inner init from the FP64 residual r64
    cudaError_t (*init)(const LaunchCfg&, FieldPtr r64, FieldPtr x, FieldPtr r, FieldPtr r0, FieldPtr p,
                        FieldPtr ph, const SolverCtx*, int maxiter, cudaStream_t);
    cudaError_t (*s_update)(const LaunchCfg&, FieldPtr r, FieldPtr v, FieldPtr s, FieldPtr sh,
                            const SolverCtx*, cudaStream_t);
    cudaError_t (*xr_update)(const LaunchCfg&, FieldPtr x, FieldPtr r, FieldPtr p, FieldPtr s, FieldPtr t,
                             FieldPtr r0, const SolverCtx*, cudaStream_t);
    cudaError_t (*p_update)(const LaunchCfg&, FieldPtr p, FieldPtr ph, FieldPtr r, FieldPtr v,
                            const SolverCtx*, cudaStream_t);
    // x64 += x / inv_norm for outer-active rhs
    cudaError_t (*dc_update)(const LaunchCfg&, FieldPtr x64, FieldPtr x, const SolverCtx*, cudaStream_t);
    // canonical AoS FP64 [lattice block][rhs][Vh][12 complex] <-> this precision
    cudaError_t (*pack)(const LaunchCfg&, const double* aos, FieldPtr out, cudaStream_t);
    cudaError_t (*unpack)(const LaunchCfg&, FieldPtr in, double* aos, cudaStream_t);
    // the same for the hop-operand storage PH
    cudaError_t (*pack_h)(const LaunchCfg&, const double* aos, FieldPtr out, cudaStream_t);
    cudaError_t (*unpack_h)(const LaunchCfg&, FieldPtr in, double* aos, cudaStream_t);
    // one BiCGStab iteration on every active rhs (the body of the iteration
    // graph's WHILE node; the last kernel sets the loop condition), and the
    // number of kernels it launches
    cudaError_t (*iterate)(const LaunchCfg&, bool dag, const IterFields&, const SolverCtx*, cudaStream_t);
    int (*iteration_kernels)(const LaunchCfg&);
    // CG on Dhat Dhat^dag (the normal-equation route): start and one step
    // (single-reduction form; its second kernel sets the loop condition)
    cudaError_t (*init_cg)(const LaunchCfg&, FieldPtr r64, FieldPtr x, FieldPtr r, FieldPtr r0, FieldPtr p,
                           FieldPtr ph, const SolverCtx*, int maxiter, cudaStream_t);
    cudaError_t (*iterate_cg)(const LaunchCfg&, bool dag, const IterFields&, const SolverCtx*, cudaStream_t);
    int (*iteration_kernels_cg)(const LaunchCfg&);
};

// Launch a kernel of this library with programmatic stream serialization
// (it starts with pdl_enter(), see sf_device.cuh) and smem bytes of dynamic
// shared memory.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl_smem(void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                                   Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k, args...);
}

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*k)(KArgs...), dim3 grid, dim3 block, cudaStream_t st, Args... args) {
    return launch_pdl_smem(k, grid, block, 0, st, args...);
}

const KrylovOps& ops_f64();
const KrylovOps& ops_f32();
const KrylovOps& ops_f32h16();

// FP64 defect-correction control: sets OState.active / inv_norm from the
// residual norms; writes the number of active rhs to *n_active.
// In the graph-resident solve (use_cond) it also sets the sweep loop's
// condition (any rhs active) and counts the sweeps that start.
cudaError_t launch_outer_check(int n, OState* ost, const double* rr, const double* bb_or_null, int max_sweeps,
                               int* n_active, cudaStream_t, cudaGraphConditionalHandle cond = 0, int use_cond = 0,
                               int* sweeps_run = nullptr);
// dst = src (src NULL: dst = 0), n doubles, as a kernel (kept a kernel node
// inside the graph-resident solve)
cudaError_t launch_copy_f64(double* dst, const double* src, long long n, int sm_count, cudaStream_t st);
// |f|^2 per (lattice, rhs) of an FP64 field
cudaError_t launch_norm2(const LaunchCfg&, FieldPtr f64, const SolverCtx*, double* out, cudaStream_t);

// link preparation: canonical AoS FP64 gauge field -> kernel layouts
// (writes the link arrays g points at)
cudaError_t launch_link_prep(const LatDev& g, const double* canon, cudaStream_t);
// max |U^dag U - 1| and max |det U - 1| over the gauge field's links
cudaError_t launch_su3_check(int L, int T, const double* canon, unsigned long long* out2, cudaStream_t);
cudaError_t launch_plaquette(int L, int T, double beta, const double* canon, double* partials,
                             unsigned* counter, double* out, cudaStream_t);
// force from the full-lattice FP64 fields Xh = (x_e, x_o), Yh = (y_e, y_o)
cudaError_t launch_force(const LaunchCfg&, FieldPtr xe, FieldPtr xo, FieldPtr ye, FieldPtr yo, double* F,
                         double* mom, double eps, cudaStream_t);

// FGCR building blocks (FP64 fields, one thread per (site, rhs): launch with NR = 1)
cudaError_t launch_dot64(const LaunchCfg&, FieldPtr a, FieldPtr b, const SolverCtx*, double2* out, cudaStream_t);
// y += sum_j coef[j][lattice*nrhs + rhs] x_j, xs: device array of nvec field pointers
cudaError_t launch_multi_axpy64(const LaunchCfg&, int nvec, const double2* const* xs, const double2* coef, FieldPtr y,
                                cudaStream_t);
cudaError_t launch_gamma5_64(long long total_elems, int Vpad, FieldPtr in, FieldPtr out, cudaStream_t);
// Gram block G[i][j] = <a_i, b_j> of one lattice's block vectors -> out
// (device, out[j * 2S + 2 i + (0, 1)], S = 8 for nrhs <= 8 else 16); partials
// holds nrhs * 2S * nblocks doubles; out NULL: the partials only
cudaError_t launch_gram64(const LaunchCfg&, FieldPtr a, FieldPtr b, double* partials, double* out, cudaStream_t);
// HMC trajectory (hmc.cu), canonical links and [(T+1) L^3][4][8] momenta:
// gauge force (F and / or mom -= eps F), U <- exp(i dt P) U on the dynamic
// links, zero momenta on the fixed boundary links, and scale * sum x_i^2
// (part: 304 doubles of scratch)
cudaError_t launch_gauge_force(int L, int T, double beta, const double* canon, double* F, double* mom, double eps,
                               cudaStream_t);
cudaError_t launch_link_update(int L, int T, double* canon, const double* mom, double dt, cudaStream_t);
cudaError_t launch_mom_fix(int L, int T, double* mom, cudaStream_t);
cudaError_t launch_sumsq(long long n, const double* x, double scale, double* part, double* out, cudaStream_t);
// y_j += sum_i x_i coef[i * nrhs + j] (coef on the device; x, y distinct)
cudaError_t launch_block_axpy64(const LaunchCfg&, FieldPtr x, const double2* coef, FieldPtr y, cudaStream_t);

}  // namespace sf

// ---- learned preconditioner (cnn.cu)
struct sf_cnn;
namespace sf {
struct CnnLatticeView {
    LatDev desc;             // the lattice (batch offset 0)
    const double* canon;     // device canonical links (features)
    cudaStream_t stream;
    int nrhs;
};
// z = r + |r| net(r / |r|) on the even sites for FP64 fields r, z of the lattice
cudaError_t cnn_apply_field(sf_cnn* c, const CnnLatticeView& v, FieldPtr r, const double* norms,
                            const double* inv_norms, FieldPtr z);
// forward, loss = mean_b |M(r_b) - e_b|^2 / |e_b|^2, backward into the gradient buffer
cudaError_t cnn_loss_grad(sf_cnn* c, const CnnLatticeView& v, FieldPtr r, FieldPtr e, const double* inv_norms,
                          const double* tnorm2, double* loss_host);
// parameter gradients for d loss / d M(r) = G (FP64 field), coef_b = s_b / 2,
// after a cnn_apply_field on the same r (its activations are reused)
cudaError_t cnn_backward_field(sf_cnn* c, const CnnLatticeView& v, FieldPtr G, const double* coef);
cudaError_t cnn_adam(sf_cnn* c, float lr, cudaStream_t st);
cudaError_t cnn_copy_grad(sf_cnn* c, float* out, cudaStream_t st);
// FP32 vector kernels of the mixed-precision flexible GCR (fgcr32.cu), on
// the FP64 BLAS tiling: <a_i, b_i> per (lattice, rhs) into out (device,
// float-float partial sums, fixed-order lattice sums), y_i += sum_j c[j][i]
// x_j, gamma_5, and the conversions r32 = scale r64, x64 += scale e32.
cudaError_t launch_dot32(const LaunchCfg& c, FieldPtr a, FieldPtr b, const SolverCtx* ctx, double2* out,
                         cudaStream_t st);
cudaError_t launch_multi_axpy32(const LaunchCfg& c, int nvec, const float4* const* xs, const double2* coef, FieldPtr y,
                                cudaStream_t st);
cudaError_t launch_gamma5_32(long long nplanes, int Vpad, FieldPtr in, FieldPtr out, int sm_count, cudaStream_t st);
cudaError_t launch_to32(const LaunchCfg& c, FieldPtr in, const double* scale, FieldPtr out, cudaStream_t st);
cudaError_t launch_add32to64(const LaunchCfg& c, FieldPtr e, const double* scale, FieldPtr x, cudaStream_t st);
// out[j nrhs + i] = <a_j, b_i> for j < nvec (<= 18) on one lattice in one pass
// over b; partials: 2 nvec nrhs c.nblocks doubles of scratch
cudaError_t launch_multidot32(const LaunchCfg& c, int nvec, const float4* const* as, FieldPtr b, double* partials,
                              double2* out, cudaStream_t st);
// the network's M(r) for an FP32 field (as cnn_apply_field)
cudaError_t cnn_apply_field32(sf_cnn* c, const CnnLatticeView& v, FieldPtr r, const double* norms,
                              const double* inv_norms, FieldPtr z);
// after a synchronisation: cudaErrorLaunchTimeout if a tensor-core
// convolution's wait timed out since the last check (clears the flag)
cudaError_t cnn_check(sf_cnn* c);
}  // namespace sf
