// api.cu -- the C ABI of include/sf_lattice.h: lattice objects, solver
// workspaces (one lattice or a batch of lattices of any sizes), the tiling
// autotuner, the graph-captured BiCGStab loop and the FP64 defect-correction
// driver around it.
//
// Solve structure (the two solves of Alg. 2; mixed precision as in Sec. 3.2):
//   x = 0; repeat { r = phi - Dhat x (FP64);  stop if |r| <= tol |phi|;
//                   solve Dhat e = r/|r| with BiCGStab in the inner precision
//                   to max(delta_prec, 0.1 tol |phi|/|r|);  x += |r| e }
// The inner loop is one CUDA graph: a WHILE conditional node whose body holds
// the seven kernels of one BiCGStab iteration for every right-hand side of
// every lattice; its last kernel sets the loop condition from the per-rhs
// convergence flags, so an inner solve costs one graph launch and the host
// synchronises once per outer sweep.
#include <algorithm>
#include <array>
#include <chrono>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <limits>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "blocksolve.h"
#include "sf_kernels.h"
#include "sf_lattice.h"

using namespace sf;

namespace {

thread_local std::string g_err;

struct SfError {
    sf_status st;
    std::string msg;
};

#define CK(x)                                                                                      \
    do {                                                                                           \
        cudaError_t e_ = (x);                                                                      \
        if (e_ != cudaSuccess)                                                                     \
            throw SfError{SF_ECUDA, std::string(#x) + ": " + cudaGetErrorString(e_)};              \
    } while (0)

#define REQUIRE(cond, msg)                                   \
    do {                                                     \
        if (!(cond)) throw SfError{SF_EINVAL, (msg)};        \
    } while (0)

template <class F>
sf_status guarded(F&& f) {
    try {
        f();
        return SF_OK;
    } catch (const SfError& e) {
        g_err = e.msg;
        if (e.st == SF_ECUDA) cudaGetLastError();
        return e.st;
    } catch (const std::bad_alloc&) {
        g_err = "host allocation failed";
        return SF_ENOMEM;
    } catch (...) {
        g_err = "unknown error";
        return SF_ECUDA;
    }
}

void* dmalloc(size_t bytes) {
    void* p = nullptr;
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        throw SfError{SF_ENOMEM, std::string("cudaMalloc(") + std::to_string(bytes) + "): " + cudaGetErrorString(e)};
    }
    return p;
}

struct DevMem {
    void* p = nullptr;
    size_t bytes = 0;
    DevMem() = default;
    DevMem(const DevMem&) = delete;
    DevMem& operator=(const DevMem&) = delete;
    ~DevMem() { release(); }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
    }
    void ensure(size_t b) {
        if (b <= bytes) return;
        release();
        p = dmalloc(b);
        bytes = b;
    }
    template <class T>
    T* as() const { return reinterpret_cast<T*>(p); }
};

bool is_device_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

int prec_index(sf_prec p) { return (int)p; }
const KrylovOps& ops_for(int ci) {
    if (ci == 0) return ops_f64();
    if (ci == 1) return ops_f32();
    return ops_f32h16();
}
Prec vec_prec(int ci) { return ci == 0 ? Prec::F64 : Prec::F32; }
Prec hop_prec(int ci) { return ci == 0 ? Prec::F64 : ci == 1 ? Prec::F32 : Prec::F16; }

// bytes of a field of S (site, rhs) units
size_t field_bytes(Prec p, long long S) {
    if (p == Prec::F64) return (size_t)S * 12 * 16;
    if (p == Prec::F32) return (size_t)S * 6 * 16;
    return (size_t)S * 3 * 16;
}

struct FieldBuf {
    DevMem v, s;
    Prec p = Prec::F64;
    void alloc(Prec pr, long long S) {
        p = pr;
        v.ensure(field_bytes(pr, S));
        CK(cudaMemset(v.p, 0, field_bytes(pr, S)));
        if (pr == Prec::F16) {
            s.ensure((size_t)S * sizeof(float));
            CK(cudaMemset(s.p, 0, (size_t)S * sizeof(float)));
        }
    }
    FieldPtr ptr() const { return FieldPtr{v.p, s.as<float>()}; }
};

int round_up(int a, int b) { return (a + b - 1) / b * b; }

// A named NVTX range for the duration of a scope (host side: visible in a
// profiler's timeline around the work a call enqueues; free without one).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// |r| / |b| from the squared norms; NaN when either is not finite (a
// corrupted input reports as such, not as converged), 0 for a zero b (the
// solution is then exactly zero).
double rel_resid(double rr, double bb) {
    if (!std::isfinite(rr) || !std::isfinite(bb)) return std::numeric_limits<double>::quiet_NaN();
    return bb > 0 ? sqrt(rr / bb) : 0.0;
}

// SF_NO_GRAPH=1 runs the solver loops without CUDA graphs (every kernel
// launched from the host; for profilers that cannot look into conditional
// graph nodes).  SF_SWEEP_GRAPHS=1 keeps one graph per defect-correction
// sweep with the sweeps driven from the host (two synchronisations per
// sweep) instead of the whole solve in one graph.
bool env_flag(const char* name) {
    const char* e = getenv(name);
    return e != nullptr && e[0] != '\0' && e[0] != '0';
}
bool no_graph() {
    static const bool v = env_flag("SF_NO_GRAPH");
    return v;
}
bool sweep_graphs() {
    static const bool v = env_flag("SF_SWEEP_GRAPHS");
    return v;
}

}  // namespace

// ---------------------------------------------------------------- lattice
struct sf_lattice {
    int L = 0, T = 0, Vh = 0, Vpad = 0, device = 0, sm_count = 152;
    double theta = 0, kappa = 0, beta = 0;
    cudaStream_t stream = nullptr;
    DevMem canon, u64, u32, u16;
    DevMem scratch;      // plaquette partials + scalars
    DevMem stage_in, stage_out;  // device staging for host arrays
    DevMem stage_out2;           // a second output staging buffer (md_force_step's Y)
    DevMem stage_f, stage_m;     // force and momentum staging (host F, mom)
    cudaStream_t side = nullptr; // device-to-host copies that overlap the compute stream
    cudaEvent_t side_ev = nullptr;
    cudaEvent_t mom_ev = nullptr;  // md_force_step: the host momenta have reached stage_m
    int tune_TS[3] = {0, 0, 0}, tune_NR[3] = {0, 0, 0}, tune_pipe[3] = {0, 0, 0};
    struct Workspace* ws = nullptr;  // own solver workspace (created on first use)
    sf_cnn* cnn = nullptr;           // learned preconditioner for SF_SOLVE_FGCR_CNN (not owned)

    LatDev base_desc() const {
        LatDev g;
        memset(&g, 0, sizeof g);
        g.L = L;
        g.T = T;
        g.Lh = L / 2;
        g.Vh = Vh;
        g.Vpad = Vpad;
        g.L2 = L * L;
        g.L3 = L * L * L;
        g.divLh = make_fastdiv((uint32_t)(L / 2));
        g.divL = make_fastdiv((uint32_t)L);
        g.L3h = L * L * L / 2;
        g.divTm1 = make_fastdiv((uint32_t)(T - 1));
        g.kappa = kappa;
        g.ph_re = cos(theta / L);
        g.ph_im = sin(theta / L);
        g.ph3_re = cos(3.0 * theta / L);
        g.ph3_im = sin(3.0 * theta / L);
        g.u64 = u64.as<double2>();
        g.u32 = u32.as<float4>();
        g.u16 = u16.as<uint2>();
        return g;
    }
    size_t links_bytes() const { return (size_t)(T + 1) * L * L * L * 4 * 18 * sizeof(double); }
};

// ---------------------------------------------------------------- workspace
// Blocks of one lattice in a launch.  Tiles are numbered time-slice fastest
// (column c of TS spatial sites, then x0), and block b owns the contiguous
// tiles [b ntiles / nblk, (b + 1) ntiles / nblk).  With nblk a multiple of
// the ncol columns, every block owns one segment of x0 slices of one column,
// and all blocks of a wave step through the same slices together: a site's
// x1 neighbours (another column) are read at the same step and its x0
// neighbours (the next tiles of the same block) a step later, so they come
// from L2 (at 32^4, 8 blocks per SM out of phase with the columns read each
// input spinor about 2.1 times from DRAM; in phase, 1.2 times).  nseg
// segments per column give about 36 blocks per SM over the launch, several
// waves of the 4 resident 160-thread blocks, so the last partial wave is a
// small part of the launch (32^4 FP32 hop: 244 us at 12 per SM, 2.5 waves;
// 227-231 us at 36; 16^4 and 24^4 unchanged); small lattices get one tile
// per block.
inline int blocks_for(int L3h, int T, int TS, int sm_count) {
    const int ncol = (L3h + TS - 1) / TS;
    const int ntiles = ncol * (T - 1);
    const int nseg = std::max(1, std::min(T - 1, (36 * sm_count) / ncol));
    return std::min(ntiles, ncol * nseg);
}

// Tilings the kernels of a precision index (0 FP64, 1 FP32, 2 FP16 hop
// operands, 3 FP64 vector kernels) are compiled for: blocks of TS sites x
// ceil(nrhs / NR) right-hand-side groups within the kernels' launch bounds
// (FP64: NR = 1 or 2; FP32 / FP16: NR = 1, 2, 3 or 5).
inline bool tiling_ok(int ci, int TS, int NR, int nrhs, int pipe = 0) {
    const int threads = TS * ((nrhs + NR - 1) / NR);
    if (ci == 1 || ci == 2) {
        if (NR != 1 && NR != 2 && NR != 3 && NR != 5) return false;
        if (pipe == 2) return NR == 1 && TS == 32 && threads <= 320;   // links staged per tile
        if (pipe) return pipe == 1 && NR <= 2 && threads <= 256;
        return threads <= (NR == 1 ? 320 : NR == 2 ? 384 : 256);
    }
    if (pipe) return false;
    if (NR != 1 && NR != 2) return false;
    return threads <= 256;
}

struct GraphEntry {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraphConditionalHandle cond = 0;
    long long pro_k = 0, sweep_k = 0;   // graph-resident solve: kernels of the prologue and of one sweep
    // block solvers: kernels of one cycle, one iteration body, its second
    // half and one preconditioner call (without its inner iterations)
    long long cyc_k = 0, it_k = 0, if_k = 0, call_k = 0;
    ~GraphEntry() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
    }
};

struct Workspace {
    std::vector<sf_lattice*> lats;
    int nlat = 0, nrhs = 0, device = 0, sm_count = 152;
    cudaStream_t stream = nullptr;
    cudaStream_t cap_stream = nullptr;
    cudaStream_t cap_top = nullptr, cap_sweep = nullptr;  // capture streams of the graph-resident solve
    long long S = 0;
    std::vector<long long> soff;

    struct Cfg {
        int TS = 0, NR = 0, nblocks = 0, pipe = 0;
        bool ready = false;
        DevMem lats_dev;
        std::vector<LatDev> host;
        LaunchCfg lc{};
        std::vector<LaunchCfg> per_lat;  // pack / unpack / force on lattice l
    } cfg[4];  // FP64, FP32, FP16 hop configurations; [3] FP64 BLAS (TS = 32, NR = 1)

    FieldBuf phi64, x64, y64, r64, t64o, xo64, yo64, w64;
    struct Inner {
        FieldBuf x, r, r0, p, v, s, t, tmp, ph, sh;
        bool ok = false;
    } inner[3];

    DevMem st, ost, partials, loop_count, nrm_bb, nrm_rr, n_active;
    DevMem io;   // canonical AoS staging for batched pack/unpack
    DevMem aux;  // per-rhs scalars of the learned preconditioner's training
    int* pin = nullptr;  // pinned: [0] n_active, [1] loop_count
    std::map<int, std::unique_ptr<GraphEntry>> graphs;
    struct SolveKey {
        int ci, dag, cg, from_x, maxiter;
        const void *phi, *x, *odd_dag;
        bool operator<(const SolveKey& o) const {
            return std::tie(ci, dag, cg, from_x, maxiter, phi, x, odd_dag) <
                   std::tie(o.ci, o.dag, o.cg, o.from_x, o.maxiter, o.phi, o.x, o.odd_dag);
        }
    };
    std::map<SolveKey, std::unique_ptr<GraphEntry>> solve_graphs;
    long long launches = 0;

    ~Workspace() {
        blk.reset();
        graphs.clear();
        if (pin) cudaFreeHost(pin);
        solve_graphs.clear();
        if (cap_stream) cudaStreamDestroy(cap_stream);
        if (cap_top) cudaStreamDestroy(cap_top);
        if (cap_sweep) cudaStreamDestroy(cap_sweep);
    }

    void setup(const std::vector<sf_lattice*>& ls, int nr) {
        lats = ls;
        nlat = (int)ls.size();
        nrhs = nr;
        device = ls[0]->device;
        sm_count = ls[0]->sm_count;
        stream = ls[0]->stream;
        CK(cudaStreamCreateWithFlags(&cap_stream, cudaStreamNonBlocking));
        CK(cudaStreamCreateWithFlags(&cap_top, cudaStreamNonBlocking));
        CK(cudaStreamCreateWithFlags(&cap_sweep, cudaStreamNonBlocking));
        soff.resize(nlat);
        S = 0;
        for (int l = 0; l < nlat; ++l) {
            soff[l] = S;
            S += (long long)nrhs * ls[l]->Vpad;
        }
        phi64.alloc(Prec::F64, S);
        x64.alloc(Prec::F64, S);
        y64.alloc(Prec::F64, S);
        r64.alloc(Prec::F64, S);
        t64o.alloc(Prec::F64, S);
        w64.alloc(Prec::F64, S);
        const size_t n = (size_t)nlat * nrhs;
        st.ensure(n * sizeof(KState));
        ost.ensure(n * sizeof(OState));
        CK(cudaMemset(st.p, 0, n * sizeof(KState)));
        CK(cudaMemset(ost.p, 0, n * sizeof(OState)));
        // the most blocks any tiling can use: the largest of TS = 32, 64, 128
        long long maxblk = 0;
        for (int l = 0; l < nlat; ++l) {
            const int L3h = ls[l]->L * ls[l]->L * ls[l]->L / 2;
            int m = 0;
            for (int TS : {32, 64, 128}) m = std::max(m, blocks_for(L3h, ls[l]->T, TS, sm_count));
            maxblk += m;
        }
        // per-block partial sums of the reductions (3 rows per rhs at most)
        partials.ensure((size_t)3 * nrhs * maxblk * sizeof(double));
        loop_count.ensure(8 * sizeof(int));  // [0] WHILE iterations, [1] cap, [2] continue flag, [3] solve
                                             // total, [4] sweeps of the graph-resident solve
        nrm_bb.ensure(n * sizeof(double));
        nrm_rr.ensure(n * sizeof(double));
        n_active.ensure(sizeof(int));
        CK(cudaHostAlloc(&pin, 8 * sizeof(int), cudaHostAllocDefault));
    }

    void set_tiling(int ci, int TS, int NR, int pipe = 0) {
        Cfg& c = cfg[ci];
        c.TS = TS;
        c.NR = NR;
        c.pipe = pipe;
        c.host.resize(nlat);
        int blk = 0;
        for (int l = 0; l < nlat; ++l) {
            LatDev g = lats[l]->base_desc();
            g.soff = soff[l];
            g.ntiles = ((g.L3h + TS - 1) / TS) * (g.T - 1);  // time-slice-fastest tiles
            g.nblk = blocks_for(g.L3h, g.T, TS, sm_count);
            g.blk0 = blk;
            blk += g.nblk;
            c.host[l] = g;
        }
        c.nblocks = blk;
        c.lats_dev.ensure(sizeof(LatDev) * nlat);
        CK(cudaMemcpy(c.lats_dev.p, c.host.data(), sizeof(LatDev) * nlat, cudaMemcpyHostToDevice));
        c.lc = LaunchCfg{c.lats_dev.as<LatDev>(), nlat, nrhs, TS, NR, blk, pipe};
        c.per_lat.resize(nlat);
        for (int l = 0; l < nlat; ++l) {
            c.per_lat[l] = LaunchCfg{c.lats_dev.as<LatDev>() + l, 1, nrhs, TS, NR,
                                     std::max(1, (c.host[l].Vh + 127) / 128), 0};
        }
        c.ready = true;
        // graphs bake launch shapes in
        for (int k : {0, 1, 8, 9}) graphs.erase(ci * 2 + k);
        solve_graphs.clear();
        if (this->blk) this->blk->graphs.clear();
    }

    void ensure_inner(int ci) {
        Inner& in = inner[ci];
        if (in.ok) return;
        const Prec pv = vec_prec(ci), ph = hop_prec(ci);
        in.x.alloc(pv, S);
        in.r.alloc(pv, S);
        in.r0.alloc(pv, S);
        in.p.alloc(pv, S);
        in.v.alloc(pv, S);
        in.s.alloc(pv, S);
        in.t.alloc(pv, S);
        in.tmp.alloc(ph, S);
        if (ph != pv) {
            in.ph.alloc(ph, S);
            in.sh.alloc(ph, S);
        }
        in.ok = true;
    }

    SolverCtx ctx(bool with_state) {
        SolverCtx c{};
        c.st = with_state ? st.as<KState>() : nullptr;
        c.ost = ost.as<OState>();
        c.partials = partials.as<double>();
        c.loop_count = loop_count.as<int>();
        c.cond = 0;
        c.use_cond = 0;
        return c;
    }

    FieldPtr hop_in(int ci, const FieldBuf& vec, const FieldBuf& copy) const {
        return hop_prec(ci) == vec_prec(ci) ? vec.ptr() : copy.ptr();
    }

    // one BiCGStab iteration on all rhs: 7 kernels and the lattice sums of its 3 reductions
    void enqueue_iteration(int ci, bool dag, const SolverCtx& k, cudaStream_t s, bool cg = false) {
        Inner& in = inner[ci];
        const IterFields f{in.x.ptr(), in.r.ptr(), in.r0.ptr(), in.p.ptr(), in.v.ptr(),
                           in.s.ptr(), in.t.ptr(), in.tmp.ptr(), in.ph.ptr(), in.sh.ptr()};
        const KrylovOps& o = ops_for(ci);
        CK(cg ? o.iterate_cg(cfg[ci].lc, dag, f, &k, s) : o.iterate(cfg[ci].lc, dag, f, &k, s));
    }

    GraphEntry& graph(int ci, bool dag, bool cg = false) {
        const int key = ci * 2 + (dag ? 1 : 0) + (cg ? 8 : 0);
        auto it = graphs.find(key);
        if (it != graphs.end()) return *it->second;
        auto ge = std::make_unique<GraphEntry>();
        CK(cudaGraphCreate(&ge->graph, 0));
        CK(cudaGraphConditionalHandleCreate(&ge->cond, ge->graph, 1, cudaGraphCondAssignDefault));
        alignas(cudaGraphNodeParams) unsigned char cp_raw[sizeof(cudaGraphNodeParams)];
        memset(cp_raw, 0, sizeof cp_raw);
        cudaGraphNodeParams& cp = *reinterpret_cast<cudaGraphNodeParams*>(cp_raw);
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = ge->cond;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        cudaGraphNode_t node;
        CK(cudaGraphAddNode(&node, ge->graph, nullptr, nullptr, 0, &cp));
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        SolverCtx k = ctx(true);
        k.cond = ge->cond;
        k.use_cond = 1;
        CK(cudaStreamBeginCaptureToGraph(cap_stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
        try {
            enqueue_iteration(ci, dag, k, cap_stream, cg);
        } catch (...) {
            cudaGraph_t dummy;
            cudaStreamEndCapture(cap_stream, &dummy);
            throw;
        }
        CK(cudaStreamEndCapture(cap_stream, &body));
        CK(cudaGraphInstantiate(&ge->exec, ge->graph, 0));
        GraphEntry& ref = *ge;
        graphs[key] = std::move(ge);
        return ref;
    }

    // ---- one sweep's FP64 residual on stream s: r64 = phi - A x and |r|^2 (A =
    // Dhat or Dhat^dag; cg: A = Dhat Dhat^dag with w64 = Dhat^dag x first, its
    // first hop kept in odd_dag).  t64o keeps the first hop of the last
    // product (the odd-site part of the solution).  copy_kernel: the odd_dag
    // copy as a kernel (inside the graph-resident solve).
    void sweep_residual(bool dag, bool cg, const FieldBuf& phi, const FieldBuf& x, FieldBuf* odd_dag, cudaStream_t s,
                        bool copy_kernel) {
        if (cg) {
            const KrylovOps& o64 = ops_f64();
            CK(o64.hop(cfg[0].lc, 1, true, x.ptr(), t64o.ptr(), 1.0, 1, nullptr, s));
            if (odd_dag) {
                if (copy_kernel)
                    CK(launch_copy_f64(odd_dag->v.as<double>(), t64o.v.as<double>(), 24LL * S, sm_count, s));
                else
                    CK(cudaMemcpyAsync(odd_dag->v.p, t64o.v.p, field_bytes(Prec::F64, S), cudaMemcpyDeviceToDevice, s));
                launches += copy_kernel ? 1 : 0;
            }
            CK(o64.tail(cfg[0].lc, 0, true, RED_NONE, t64o.ptr(), x.ptr(), FieldPtr{nullptr, nullptr}, w64.ptr(),
                        FieldPtr{nullptr, nullptr}, 1.0, -1.0, 1, nullptr, nullptr, s));
            launches += 2;
            residual64(false, phi, w64, s);
        } else {
            residual64(dag, phi, x, s);
        }
    }

    // add a conditional node (WHILE or IF) controlled by h after the work
    // captured so far on s; returns its body graph
    static cudaGraph_t add_while(cudaStream_t s, cudaGraphConditionalHandle h,
                                 cudaGraphConditionalNodeType type = cudaGraphCondTypeWhile) {
        cudaStreamCaptureStatus cs;
        cudaGraph_t g = nullptr;
        const cudaGraphNode_t* deps = nullptr;
        size_t nd = 0;
        CK(cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, &deps, nullptr, &nd));
        alignas(cudaGraphNodeParams) unsigned char raw[sizeof(cudaGraphNodeParams)];
        memset(raw, 0, sizeof raw);
        cudaGraphNodeParams& cp = *reinterpret_cast<cudaGraphNodeParams*>(raw);
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = h;
        cp.conditional.type = type;
        cp.conditional.size = 1;
        cudaGraphNode_t node;
        CK(cudaGraphAddNode(&node, g, deps, nullptr, nd, &cp));
        CK(cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
        return cp.conditional.phGraph_out[0];
    }

    static void abandon_capture(cudaStream_t s) {
        cudaGraph_t dummy = nullptr;
        cudaStreamEndCapture(s, &dummy);
        if (dummy) cudaGraphDestroy(dummy);
    }

    // a conditional node after the work captured so far on parent, its body
    // captured on child by fn(child)
    template <class F>
    static void cond_body(cudaStream_t parent, cudaGraphConditionalHandle h, cudaGraphConditionalNodeType type,
                          cudaStream_t child, F&& fn) {
        cudaGraph_t body = add_while(parent, h, type);
        CK(cudaStreamBeginCaptureToGraph(child, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
        try {
            fn(child);
        } catch (...) {
            abandon_capture(child);
            throw;
        }
        CK(cudaStreamEndCapture(child, &body));
    }

    static cudaGraphConditionalHandle new_handle(cudaStream_t s) {
        cudaStreamCaptureStatus cs;
        cudaGraph_t g = nullptr;
        CK(cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, nullptr, nullptr, nullptr));
        cudaGraphConditionalHandle h;
        CK(cudaGraphConditionalHandleCreate(&h, g, 0, 0));
        return h;
    }

    // ---- the whole defect-correction solve as one graph, launched once per
    // solve with one host synchronisation at its end: |phi|^2, the first FP64
    // residual and the check that opens the sweep loop, then a WHILE node over
    // the sweeps whose body holds the inner start, the WHILE node over the
    // inner iterations, the update x += |r| e, the next FP64 residual and the
    // check that decides the next sweep (k_outer_check sets the condition;
    // every rhs stops after max_sweeps sweeps, so the loop ends).
    GraphEntry& solve_graph(int ci, bool dag, bool cg, bool from_x, const FieldBuf& phi, FieldBuf& x,
                            FieldBuf* odd_dag, int maxiter, int max_sweeps, long long& pro_k, long long& sweep_k) {
        const SolveKey key{ci, dag ? 1 : 0, cg ? 1 : 0, from_x ? 1 : 0, maxiter, phi.v.p, x.v.p,
                           odd_dag ? odd_dag->v.p : nullptr};
        auto it = solve_graphs.find(key);
        if (it != solve_graphs.end()) {
            pro_k = it->second->pro_k;
            sweep_k = it->second->sweep_k;
            return *it->second;
        }
        const KrylovOps& o = ops_for(ci);
        const int n = nlat * nrhs;
        const long long saved = launches;   // capturing launches nothing
        auto ge = std::make_unique<GraphEntry>();
        auto abandon = [](cudaStream_t s) {
            cudaGraph_t dummy = nullptr;
            cudaStreamEndCapture(s, &dummy);
            if (dummy) cudaGraphDestroy(dummy);
        };
        CK(cudaStreamBeginCapture(cap_top, cudaStreamCaptureModeThreadLocal));
        try {
            const cudaGraphConditionalHandle h_sweep = new_handle(cap_top);
            launches = 0;
            SolverCtx k0 = ctx(false);
            CK(launch_norm2(cfg[0].lc, phi.ptr(), &k0, nrm_bb.as<double>(), cap_top));
            launches += 2;
            if (!from_x) {   // x = 0: r = phi; the odd-site parts of x (and of Dhat^dag x) are 0
                CK(launch_copy_f64(r64.v.as<double>(), phi.v.as<double>(), 24LL * S, sm_count, cap_top));
                CK(launch_copy_f64(nrm_rr.as<double>(), nrm_bb.as<double>(), n, sm_count, cap_top));
                CK(launch_copy_f64(t64o.v.as<double>(), nullptr, 24LL * S, sm_count, cap_top));
                launches += 3;
                if (cg) {
                    CK(launch_copy_f64(w64.v.as<double>(), nullptr, 24LL * S, sm_count, cap_top));
                    launches += 1;
                    if (odd_dag) {
                        CK(launch_copy_f64(odd_dag->v.as<double>(), nullptr, 24LL * S, sm_count, cap_top));
                        launches += 1;
                    }
                }
            } else {
                sweep_residual(dag, cg, phi, x, odd_dag, cap_top, true);
            }
            CK(launch_outer_check(n, ost.as<OState>(), nrm_rr.as<double>(), nrm_bb.as<double>(), max_sweeps,
                                  n_active.as<int>(), cap_top, h_sweep, 1, loop_count.as<int>() + 4));
            launches += 1;
            ge->pro_k = launches;
            cudaGraph_t body = add_while(cap_top, h_sweep);
            CK(cudaStreamBeginCaptureToGraph(cap_sweep, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
            try {
                launches = 0;
                const cudaGraphConditionalHandle h_iter = new_handle(cap_sweep);
                SolverCtx ki = ctx(true);
                ki.cond = h_iter;
                ki.use_cond = 1;
                Inner& in = inner[ci];
                CK((cg ? o.init_cg : o.init)(cfg[ci].lc, r64.ptr(), in.x.ptr(), in.r.ptr(), in.r0.ptr(), in.p.ptr(),
                                             in.ph.ptr(), &ki, maxiter, cap_sweep));
                cudaGraph_t ibody = add_while(cap_sweep, h_iter);
                CK(cudaStreamBeginCaptureToGraph(cap_stream, ibody, nullptr, nullptr, 0,
                                                 cudaStreamCaptureModeThreadLocal));
                try {
                    enqueue_iteration(ci, dag, ki, cap_stream, cg);
                } catch (...) {
                    abandon(cap_stream);
                    throw;
                }
                CK(cudaStreamEndCapture(cap_stream, &ibody));
                CK(o.dc_update(cfg[ci].lc, x.ptr(), in.x.ptr(), &ki, cap_sweep));
                launches += 3;   // init (+ its sums), dc_update
                sweep_residual(dag, cg, phi, x, odd_dag, cap_sweep, true);
                CK(launch_outer_check(n, ost.as<OState>(), nrm_rr.as<double>(), nullptr, max_sweeps,
                                      n_active.as<int>(), cap_sweep, h_sweep, 1, loop_count.as<int>() + 4));
                launches += 1;
                ge->sweep_k = launches;
            } catch (...) {
                abandon(cap_sweep);
                throw;
            }
            CK(cudaStreamEndCapture(cap_sweep, &body));
        } catch (...) {
            launches = saved;
            abandon(cap_top);
            throw;
        }
        launches = saved;
        CK(cudaStreamEndCapture(cap_top, &ge->graph));
        CK(cudaGraphInstantiate(&ge->exec, ge->graph, 0));
        pro_k = ge->pro_k;
        sweep_k = ge->sweep_k;
        GraphEntry& ref = *ge;
        solve_graphs[key] = std::move(ge);
        return ref;
    }

    // ---- autotuning: time Dhat (hop + fused tail) for each admissible tiling
    void autotune(int ci);

    void ensure_cfg(int ci) {
        if (cfg[ci].ready) return;
        if (ci == 3) {
            set_tiling(3, 32, 1);
            return;
        }
        // explicit tiling of the (single) lattice wins
        if (nlat == 1 && lats[0]->tune_TS[ci] > 0) {
            const int TS = lats[0]->tune_TS[ci], NR = lats[0]->tune_NR[ci], pipe = lats[0]->tune_pipe[ci];
            REQUIRE(tiling_ok(ci, TS, NR, nrhs, pipe),
                    "tiling exceeds the block size of this precision (TS * ceil(nrhs / NR) threads; "
                    "pipelined hop: FP32 / FP16, NR <= 2, at most 256 threads; staged links: FP32 / FP16, "
                    "NR = 1, TS = 32, at most 320 threads)");
            set_tiling(ci, TS, NR, pipe);
            return;
        }
        autotune(ci);
    }

    // FP64: r64 = phi - Dhat x (or Dhat^dag), |r|^2 -> nrm_rr
    void residual64(bool dag, const FieldBuf& phi, const FieldBuf& x, cudaStream_t s) {
        ensure_cfg(0);
        const KrylovOps& o = ops_f64();
        const LaunchCfg& lc = cfg[0].lc;
        SolverCtx k = ctx(false);
        // t64o = kappa H_oe x (dag: kappa gamma5 H_oe gamma5 x) is the odd-site part of the
        // full-lattice solution (Sec. 3.1); r64 = phi - (x - kappa H_eo t64o)
        CK(o.hop(lc, 1, dag, x.ptr(), t64o.ptr(), 1.0, 1, nullptr, s));
        CK(o.tail(lc, 0, dag, RED_NORM, t64o.ptr(), x.ptr(), phi.ptr(), r64.ptr(), FieldPtr{nullptr, nullptr}, -1.0,
                  1.0, 1, &k, nrm_rr.as<double>(), s));
        launches += 3;  // hop, tail, lattice sums
    }

    // The full FP64-outer / inner-precision solve of Dhat x = phi (dag: Dhat^dag).
    // Returns per-rhs (sweeps, inner iterations, true residual).
    struct Result {
        std::vector<int> sweeps, inner;
        std::vector<double> resid;
        bool converged = true;
    };

    // ---- flexible GCR (FP64) with the learned preconditioner
    struct Fgcr {
        static constexpr int M = 16;
        int m = 0;
        FieldBuf z[M], w[M];
        FieldBuf r, g5a, g5b;
        DevMem ptrs, coef, dots, nrm, norms, invn;
    };
    std::unique_ptr<Fgcr> fg;

    void apply_dhat64(bool dag, const FieldBuf& in, FieldBuf& out, cudaStream_t s) {
        const KrylovOps& o = ops_f64();
        const LaunchCfg& lc = cfg[0].lc;
        CK(o.hop(lc, 1, dag, in.ptr(), t64o.ptr(), 1.0, 0, nullptr, s));
        CK(o.tail(lc, 0, dag, RED_NONE, t64o.ptr(), in.ptr(), FieldPtr{nullptr, nullptr}, out.ptr(),
                  FieldPtr{nullptr, nullptr}, 1.0, -1.0, 2, nullptr, nullptr, s));
        launches += 2;
    }

    // per-rhs complex <a, b> -> host
    void dots64(const FieldBuf& a, const FieldBuf& b, double2* dev_out, cudaStream_t s) {
        SolverCtx k = ctx(false);
        CK(launch_dot64(cfg[3].lc, a.ptr(), b.ptr(), &k, dev_out, s));
        launches += 2;
    }

    Result fgcr(bool use_cnn, bool dag, const FieldBuf& phi, FieldBuf& x, double tol, int maxiter);

    // ---- FP64 defect correction around an FP32 flexible GCR (16 directions)
    // preconditioned by the learned network (or the identity)
    struct Fgcr32 {
        static constexpr int M = 16;
        FieldBuf z[M], w[M], r, e, g5a, g5b;
        DevMem ptrs, rptr, coef, dots, norms, invn, scale, mdot;
    };
    std::unique_ptr<Fgcr32> f32;
    Result fgcr_mixed(bool use_cnn, bool dag, const FieldBuf& phi, FieldBuf& x, double tol, int maxiter);

    // ---- Gl-BiCGStab (FP64, Frobenius inner products over the block) with
    // FP32-inner BiCGStab solves as its preconditioner
    struct Gl {
        FieldBuf r, r0, p, v, s, t, ph, sh;
        DevMem ptrs, coef, dots;
    };
    std::unique_ptr<Gl> gl;
    void precondition(bool dag, const FieldBuf& in, FieldBuf& out, double delta, int maxiter,
                      std::vector<int>& iters);
    Result gl_bicgstab(bool dag, const FieldBuf& phi, FieldBuf& x, double tol, int maxiter);
    DevMem gram_partials, gram_out, bcoef;
    // G[i][j] = <a_i, b_j> (one lattice) -> host, row-major s x s
    void gram64(const FieldBuf& a, const FieldBuf& b, std::vector<std::complex<double>>& G);
    // y_j += sum_i x_i C[i][j] (C row-major s x s, host)
    void block_axpy64(const FieldBuf& x, const std::vector<std::complex<double>>& C, FieldBuf& y);
    Result bl_bicgstab(bool dag, const FieldBuf& phi, FieldBuf& x, double tol, int maxiter);
    void ensure_gl();

    // ---- the device-resident forms of both block solvers (blocksolve.cu):
    // one graph per (solver, direction, fields, tol, maxiter), launched once
    // per solve with one synchronisation at its end
    struct Blk {
        DevMem state, partials;
        cudaStream_t cs[2] = {nullptr, nullptr};   // capture streams of the IF bodies and the inner loops
        struct Key {
            int gl, dag;
            const void *phi, *x;
            double tol;
            int maxiter;
            bool operator<(const Key& o) const {
                return std::tie(gl, dag, phi, x, tol, maxiter) < std::tie(o.gl, o.dag, o.phi, o.x, o.tol, o.maxiter);
            }
        };
        std::map<Key, std::unique_ptr<GraphEntry>> graphs;
        ~Blk() {
            graphs.clear();
            for (cudaStream_t c : cs)
                if (c) cudaStreamDestroy(c);
        }
    };
    std::unique_ptr<Blk> blk;
    void ensure_blk();
    // out = M in inside a capture on s (the inner WHILE body on child)
    void capture_precondition(bool dag, const FieldBuf& in, FieldBuf& out, int maxiter, cudaStream_t s,
                              cudaStream_t child);
    Result bl_bicgstab_graph(bool dag, const FieldBuf& phi, FieldBuf& x, double tol, int maxiter);
    Result gl_bicgstab_graph(bool dag, const FieldBuf& phi, FieldBuf& x, double tol, int maxiter);

    // per-rhs |b - A x| / |b| in FP64 (A = Dhat, or Dhat^dag for dag)
    std::vector<double> rel_residual(bool dag, const FieldBuf& b, const FieldBuf& x) {
        ensure_cfg(0);
        SolverCtx k0 = ctx(false);
        CK(launch_norm2(cfg[0].lc, b.ptr(), &k0, nrm_bb.as<double>(), stream));
        launches += 2;
        residual64(dag, b, x, stream);
        const size_t n = (size_t)nlat * nrhs;
        std::vector<double> rr(n), bb(n), out(n);
        CK(cudaMemcpyAsync(rr.data(), nrm_rr.p, n * sizeof(double), cudaMemcpyDeviceToHost, stream));
        CK(cudaMemcpyAsync(bb.data(), nrm_bb.p, n * sizeof(double), cudaMemcpyDeviceToHost, stream));
        CK(cudaStreamSynchronize(stream));
        for (size_t i = 0; i < n; ++i) out[i] = rel_resid(rr[i], bb[i]);
        return out;
    }

    // The normal-equation route to the same pair: Y solves (Dhat Dhat^dag) Y = phi
    // by CG (FP32 inner, FP64 outer), X = Dhat^dag Y (the FP64 product of the final
    // residual, so |phi - Dhat X| is exactly the residual the outer loop judged).
    // rx: the CG sweeps and iterations with |phi - Dhat X| / |phi|; ry: |X - Dhat^dag Y| / |X|.
    // With xo / yo, the odd-site parts of X and Y (kappa H_oe X, kappa g5 H_oe g5 Y) are
    // kept from the final residual's hops.  check_y: recompute |X - Dhat^dag Y| / |X|
    // (X is that very product, so it is at FP64 rounding); otherwise reported as 0.
    void solve_normal(const FieldBuf& phi, double tol, int maxiter, Result& rx, Result& ry, bool check_y,
                      FieldBuf* xo = nullptr, FieldBuf* yo = nullptr) {
        rx = solve(1, false, phi, y64, tol, maxiter, false, xo, true, yo);
        CK(cudaMemcpyAsync(x64.v.p, w64.v.p, field_bytes(Prec::F64, S), cudaMemcpyDeviceToDevice, stream));
        ry = Result();
        const size_t n = (size_t)nlat * nrhs;
        ry.sweeps.assign(n, 0);
        ry.inner.assign(n, 0);
        if (check_y) {
            ry.resid = rel_residual(true, x64, y64);
            for (double r : ry.resid)
                if (!(r <= tol)) ry.converged = false;
        } else {
            ry.resid.assign(n, 0.0);
        }
    }

    // odd (optional): receives the odd-site reconstruction kappa H_oe x of the
    // final x (dag: kappa gamma5 H_oe gamma5 x), the first hop of the last true
    // residual, so the force needs no hop of its own.
    //
    // cg: the normal-equation route -- x solves (Dhat Dhat^dag) x = phi by CG
    // (FP32 inner, FP64 outer on the same system); w64 then holds Dhat^dag x
    // of the final residual (dag and odd are not used).
    Result solve(int ci, bool dag, const FieldBuf& phi, FieldBuf& x, double tol, int maxiter, bool from_x = false,
                 FieldBuf* odd = nullptr, bool cg = false, FieldBuf* odd_dag = nullptr) {
        ensure_cfg(0);
        ensure_cfg(ci);
        ensure_inner(ci);
        const KrylovOps& o = ops_for(ci);
        cudaStream_t s = stream;
        const size_t n = (size_t)nlat * nrhs;
        const double floor_delta = (ci == 0) ? 0.0 : (ci == 1) ? 1e-5 : 2e-3;
        const int max_sweeps = (ci == 0) ? 6 : (ci == 1) ? 12 : 24;
        std::vector<OState> oh(n);
        for (auto& e : oh) {
            memset(&e, 0, sizeof e);
            e.tol2 = tol * tol;
            e.delta2_floor = floor_delta * floor_delta;
        }
        CK(cudaMemcpyAsync(ost.p, oh.data(), n * sizeof(OState), cudaMemcpyHostToDevice, s));
        if (!from_x) CK(cudaMemsetAsync(x.v.p, 0, field_bytes(Prec::F64, S), s));
        pin[2] = maxiter + 8;  // WHILE cap
        pin[5] = 0;            // iterations of this solve
        pin[6] = 0;            // sweeps of the graph-resident solve
        CK(cudaMemcpyAsync(loop_count.as<int>() + 1, pin + 2, sizeof(int), cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(loop_count.as<int>() + 3, pin + 5, 2 * sizeof(int), cudaMemcpyHostToDevice, s));
        if (!no_graph() && !sweep_graphs()) {
            // the whole solve on the device: one graph launch, one synchronisation
            long long pro_k = 0, sweep_k = 0;
            GraphEntry& sg = solve_graph(ci, dag, cg, from_x, phi, x, odd_dag, maxiter, max_sweeps, pro_k, sweep_k);
            CK(cudaGraphLaunch(sg.exec, s));
            if (odd) CK(cudaMemcpyAsync(odd->v.p, t64o.v.p, field_bytes(Prec::F64, S), cudaMemcpyDeviceToDevice, s));
            std::vector<OState> out(n);
            CK(cudaMemcpyAsync(out.data(), ost.p, n * sizeof(OState), cudaMemcpyDeviceToHost, s));
            CK(cudaMemcpyAsync(pin + 5, loop_count.as<int>() + 3, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            launches += pro_k + sweep_k * pin[6] +
                        (long long)(cg ? o.iteration_kernels_cg : o.iteration_kernels)(cfg[ci].lc) * pin[5];
            return result_of(out);
        }
        SolverCtx k0 = ctx(false);
        CK(launch_norm2(cfg[0].lc, phi.ptr(), &k0, nrm_bb.as<double>(), s));
        launches += 2;
        SolverCtx k = ctx(true);
        bool have_odd = false;  // t64o holds kappa H_oe x of the current x
        for (int sweep = 0;; ++sweep) {
            if (sweep == 0 && !from_x) {
                // x = 0: r = phi
                CK(cudaMemcpyAsync(r64.v.p, phi.v.p, field_bytes(Prec::F64, S), cudaMemcpyDeviceToDevice, s));
                CK(cudaMemcpyAsync(nrm_rr.p, nrm_bb.p, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
                have_odd = false;
            } else {
                // cg: w = Dhat^dag x with its first hop kappa gamma5 H_oe gamma5 x (the odd part of
                // x as the adjoint solution), then r = phi - Dhat w (first hop: the odd part of w)
                sweep_residual(dag, cg, phi, x, odd_dag, s, false);
                have_odd = true;
            }
            CK(launch_outer_check((int)n, ost.as<OState>(), nrm_rr.as<double>(),
                                  sweep == 0 ? nrm_bb.as<double>() : nullptr, max_sweeps, n_active.as<int>(), s));
            launches += 1;
            CK(cudaMemcpyAsync(pin, n_active.p, sizeof(int), cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            if (pin[0] == 0) break;
            CK((cg ? o.init_cg : o.init)(cfg[ci].lc, r64.ptr(), inner[ci].x.ptr(), inner[ci].r.ptr(),
                                         inner[ci].r0.ptr(), inner[ci].p.ptr(), inner[ci].ph.ptr(), &k, maxiter, s));
            if (no_graph()) {
                // same kernels launched one by one, the loop condition read back
                // by the host after each iteration (for profilers that cannot
                // see inside conditional graph nodes)
                SolverCtx kn = ctx(true);
                for (;;) {
                    enqueue_iteration(ci, dag, kn, s, cg);
                    CK(cudaMemcpyAsync(pin + 3, loop_count.as<int>() + 2, sizeof(int), cudaMemcpyDeviceToHost, s));
                    CK(cudaStreamSynchronize(s));
                    if (!pin[3]) break;
                }
            } else {
                CK(cudaGraphLaunch(graph(ci, dag, cg).exec, s));
            }
            CK(o.dc_update(cfg[ci].lc, x.ptr(), inner[ci].x.ptr(), &k, s));
            launches += 3;  // init (+ its sums), dc_update
        }
        if (odd) {
            if (have_odd) CK(cudaMemcpyAsync(odd->v.p, t64o.v.p, field_bytes(Prec::F64, S), cudaMemcpyDeviceToDevice, s));
            else CK(cudaMemsetAsync(odd->v.p, 0, field_bytes(Prec::F64, S), s));  // x = 0
        }
        if (cg && !have_odd) {  // x = 0
            CK(cudaMemsetAsync(w64.v.p, 0, field_bytes(Prec::F64, S), s));
            if (odd_dag) CK(cudaMemsetAsync(odd_dag->v.p, 0, field_bytes(Prec::F64, S), s));
        }
        std::vector<OState> out(n);
        CK(cudaMemcpyAsync(out.data(), ost.p, n * sizeof(OState), cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(pin + 5, loop_count.as<int>() + 3, sizeof(int), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        launches += (long long)(cg ? o.iteration_kernels_cg : o.iteration_kernels)(cfg[ci].lc) * pin[5];
        return result_of(out);
    }

    static Result result_of(const std::vector<OState>& out) {
        Result res;
        const size_t n = out.size();
        res.sweeps.resize(n);
        res.inner.resize(n);
        res.resid.resize(n);
        for (size_t i = 0; i < n; ++i) {
            res.sweeps[i] = out[i].sweeps;
            res.inner[i] = out[i].inner_iters;
            res.resid[i] = rel_resid(out[i].rr, out[i].bb);
            const bool ok = (out[i].bb == 0.0) || (out[i].rr <= out[i].tol2 * out[i].bb);
            if (!ok) res.converged = false;
        }
        return res;
    }
};

namespace {

struct TuneKey {
    std::vector<std::pair<int, int>> dims;  // (L, T) of each lattice
    int nrhs, ci, sms;
    bool operator<(const TuneKey& o) const {
        return std::tie(dims, nrhs, ci, sms) < std::tie(o.dims, o.nrhs, o.ci, o.sms);
    }
};
std::mutex g_tune_mu;
std::map<TuneKey, std::array<int, 3>> g_tune_cache;  // TS, NR, pipe

}  // namespace

void Workspace::autotune(int ci) {
    TuneKey key;
    for (auto* l : lats) key.dims.push_back({l->L, l->T});
    key.nrhs = nrhs;
    key.ci = ci;
    key.sms = sm_count;
    {
        std::lock_guard<std::mutex> g(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            set_tiling(ci, it->second[0], it->second[1], it->second[2]);
            return;
        }
    }
    ensure_inner(ci);
    const KrylovOps& o = ops_for(ci);
    const int nrs_all[4] = {1, 2, 3, 5};
    const int tss[3] = {32, 64, 128};
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    // every admissible tiling, timed in three interleaved rounds; each keeps its
    // fastest round (the launches are a few microseconds, so one round is noisy)
    struct Cand {
        int TS, NR, pipe;
        float ms;
    };
    std::vector<Cand> cands;
    for (int pipe = 0; pipe <= 2; ++pipe)
        for (int NR : nrs_all) {
            if (NR > nrhs) continue;
            for (int TS : tss)
                if (tiling_ok(ci, TS, NR, nrhs, pipe)) cands.push_back(Cand{TS, NR, pipe, 1e30f});
        }
    REQUIRE(!cands.empty(), "no tiling of this precision fits the number of right-hand sides");
    const FieldPtr none{nullptr, nullptr};
    for (int round = 0; round < 3; ++round)
        for (Cand& cd : cands) {
            set_tiling(ci, cd.TS, cd.NR, cd.pipe);
            const LaunchCfg& lc = cfg[ci].lc;
            Inner& in = inner[ci];
            auto run = [&]() {
                CK(o.hop(lc, 1, false, hop_in(ci, in.p, in.ph), in.tmp.ptr(), 1.0, 0, nullptr, stream));
                CK(o.tail(lc, 0, false, RED_NONE, in.tmp.ptr(), in.p.ptr(), none, in.v.ptr(), none, 1.0, -1.0, 2,
                          nullptr, nullptr, stream));
            };
            run();
            CK(cudaEventRecord(e0, stream));
            const int reps = 8;
            for (int r = 0; r < reps; ++r) run();
            CK(cudaEventRecord(e1, stream));
            CK(cudaEventSynchronize(e1));
            float ms = 0;
            CK(cudaEventElapsedTime(&ms, e0, e1));
            cd.ms = std::min(cd.ms, ms);
        }
    int bTS = 64, bNR = 1, bpipe = 0;
    float best = 1e30f;
    for (const Cand& cd : cands)
        if (cd.ms < best) {
            best = cd.ms;
            bTS = cd.TS;
            bNR = cd.NR;
            bpipe = cd.pipe;
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (env_flag("SF_TUNE_LOG")) {   // every candidate's best time, for diagnosing a choice
        fprintf(stderr, "sf autotune: %d lattice(s), %d rhs, precision %d:", nlat, nrhs, ci);
        for (const Cand& cd : cands) fprintf(stderr, " [TS %d NR %d mode %d %.1f us]", cd.TS, cd.NR, cd.pipe, cd.ms * 125.0f);
        fprintf(stderr, " -> TS %d NR %d mode %d\n", bTS, bNR, bpipe);
    }
    set_tiling(ci, bTS, bNR, bpipe);
    std::lock_guard<std::mutex> g(g_tune_mu);
    g_tune_cache[key] = {bTS, bNR, bpipe};
}


// ---------------------------------------------------------------- FGCR
// Flexible GCR (restarted, m directions) on Dhat x = phi (dag: Dhat^dag) in
// FP64 with the preconditioner z = M(r): the learned network (with
// M^dag(r) = gamma_5 M(gamma_5 r) for the adjoint system) or the identity.
// Directions are orthogonalised in the Dhat-image with two passes of
// classical Gram-Schmidt.  The answer is judged on a recomputed FP64 residual;
// if FGCR stops above tolerance, FP32-inner BiCGStab under FP64 defect
// correction continues from its iterate.
Workspace::Result Workspace::fgcr(bool use_cnn, bool dag, const FieldBuf& phi, FieldBuf& x, double tol, int maxiter) {
    REQUIRE(nlat == 1, "FGCR runs on a single lattice");
    REQUIRE(nrhs <= 8, "FGCR, Gl-BiCGStab and Bl-BiCGStab take up to 8 right-hand sides (one 32-site row per rhs)");
    ensure_cfg(0);
    ensure_cfg(3);
    sf_cnn* cnn = lats[0]->cnn;
    if (use_cnn) REQUIRE(cnn != nullptr, "no learned preconditioner attached (sf_lattice_set_preconditioner)");
    cudaStream_t s = stream;
    const int n = nrhs, m = Fgcr::M;
    if (!fg) {
        fg.reset(new Fgcr());
        fg->m = m;
        for (int k = 0; k < m; ++k) {
            fg->z[k].alloc(Prec::F64, S);
            fg->w[k].alloc(Prec::F64, S);
        }
        fg->r.alloc(Prec::F64, S);
        fg->g5a.alloc(Prec::F64, S);
        fg->g5b.alloc(Prec::F64, S);
        std::vector<void*> p(2 * m);
        for (int k = 0; k < m; ++k) {
            p[k] = fg->z[k].v.p;
            p[m + k] = fg->w[k].v.p;
        }
        fg->ptrs.ensure(p.size() * sizeof(void*));
        CK(cudaMemcpy(fg->ptrs.p, p.data(), p.size() * sizeof(void*), cudaMemcpyHostToDevice));
        fg->coef.ensure((size_t)2 * m * n * sizeof(double2));
        fg->dots.ensure((size_t)2 * m * n * sizeof(double2));
        fg->norms.ensure((size_t)n * sizeof(double));
        fg->invn.ensure((size_t)n * sizeof(double));
    }
    const double2* const* zp = fg->ptrs.as<const double2*>();
    const double2* const* wp = zp + m;
    const LaunchCfg& bl = cfg[3].lc;
    const size_t fbytes = field_bytes(Prec::F64, S);
    std::vector<double2> hd((size_t)2 * m * n), hc((size_t)2 * m * n);
    auto read_dots = [&](int count) {
        CK(cudaMemcpyAsync(hd.data(), fg->dots.p, (size_t)count * n * sizeof(double2), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
    };
    auto axpy = [&](const double2* const* xs, int nvec, FieldBuf& y) {
        CK(cudaMemcpyAsync(fg->coef.p, hc.data(), (size_t)nvec * n * sizeof(double2), cudaMemcpyHostToDevice, s));
        CK(launch_multi_axpy64(bl, nvec, xs, fg->coef.as<double2>(), y.ptr(), s));
        launches += 1;
    };
    CK(cudaMemsetAsync(x.v.p, 0, fbytes, s));
    CK(cudaMemcpyAsync(fg->r.v.p, phi.v.p, fbytes, cudaMemcpyDeviceToDevice, s));
    dots64(phi, phi, fg->dots.as<double2>(), s);
    read_dots(1);
    std::vector<double> bb(n), rr(n), nw((size_t)m * n);
    std::vector<int> iters(n, 0);
    std::vector<char> done(n);
    for (int i = 0; i < n; ++i) {
        bb[i] = hd[i].x;
        rr[i] = bb[i];
        done[i] = (bb[i] == 0.0);
    }
    auto all_done = [&] {
        for (char d : done)
            if (!d) return false;
        return true;
    };
    const CnnLatticeView view{cfg[0].host[0], lats[0]->canon.as<double>(), s, n};
    std::vector<double> hn(n), hi(n);
    int total = 0, restarts = 0;
    while (!all_done() && total < maxiter) {
        ++restarts;
        for (int k = 0; k < m && !all_done() && total < maxiter; ++k) {
            FieldBuf& zk = fg->z[k];
            FieldBuf& wk = fg->w[k];
            // z_k = M(r)
            if (use_cnn) {
                const double nreal = 24.0 * lats[0]->Vh;
                for (int i = 0; i < n; ++i) {
                    hn[i] = sqrt(rr[i] / nreal);  // RMS scale of r
                    hi[i] = hn[i] > 0 ? 1.0 / hn[i] : 0.0;
                }
                CK(cudaMemcpyAsync(fg->norms.p, hn.data(), n * sizeof(double), cudaMemcpyHostToDevice, s));
                CK(cudaMemcpyAsync(fg->invn.p, hi.data(), n * sizeof(double), cudaMemcpyHostToDevice, s));
                const long long tot = (long long)S * 12;
                if (dag) {
                    CK(launch_gamma5_64(tot, lats[0]->Vpad, fg->r.ptr(), fg->g5a.ptr(), s));
                    CK(cnn_apply_field(cnn, view, fg->g5a.ptr(), fg->norms.as<double>(), fg->invn.as<double>(),
                                       fg->g5b.ptr()));
                    CK(launch_gamma5_64(tot, lats[0]->Vpad, fg->g5b.ptr(), zk.ptr(), s));
                } else {
                    CK(cnn_apply_field(cnn, view, fg->r.ptr(), fg->norms.as<double>(), fg->invn.as<double>(),
                                       zk.ptr()));
                }
                launches += 8;
                CK(cudaStreamSynchronize(s));  // the host arrays above are reused next iteration
                CK(cnn_check(cnn));
            } else {
                CK(cudaMemcpyAsync(zk.v.p, fg->r.v.p, fbytes, cudaMemcpyDeviceToDevice, s));
            }
            // w_k = A z_k, orthogonalised against w_0..w_{k-1} (two passes)
            apply_dhat64(dag, zk, wk, s);
            for (int pass = 0; pass < 2 && k > 0; ++pass) {
                for (int j = 0; j < k; ++j) dots64(fg->w[j], wk, fg->dots.as<double2>() + (size_t)j * n, s);
                read_dots(k);
                for (int j = 0; j < k; ++j)
                    for (int i = 0; i < n; ++i) {
                        const double d = nw[(size_t)j * n + i];
                        const double2 v = hd[(size_t)j * n + i];
                        hc[(size_t)j * n + i] = (d > 0) ? make_double2(-v.x / d, -v.y / d) : make_double2(0, 0);
                    }
                axpy(wp, k, wk);
                axpy(zp, k, zk);
            }
            dots64(wk, wk, fg->dots.as<double2>(), s);
            dots64(wk, fg->r, fg->dots.as<double2>() + n, s);
            read_dots(2);
            for (int i = 0; i < n; ++i) {
                const double d = hd[i].x;
                nw[(size_t)k * n + i] = d;
                const double2 v = hd[n + i];
                hc[i] = (!done[i] && d > 0) ? make_double2(v.x / d, v.y / d) : make_double2(0, 0);
            }
            axpy(zp + k, 1, x);
            for (int i = 0; i < n; ++i) hc[i] = make_double2(-hc[i].x, -hc[i].y);
            axpy(wp + k, 1, fg->r);
            dots64(fg->r, fg->r, fg->dots.as<double2>(), s);
            read_dots(1);
            for (int i = 0; i < n; ++i) {
                if (done[i]) continue;
                rr[i] = hd[i].x;
                iters[i] += 1;
                if (!(rr[i] > 0.01 * tol * tol * bb[i])) done[i] = 1;
            }
            ++total;
        }
    }
    // judge on the FP64 true residual; continue with BiCGStab where FGCR fell short
    residual64(dag, phi, x, s);
    std::vector<double> rt(n);
    CK(cudaMemcpyAsync(rt.data(), nrm_rr.p, n * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    Result res;
    res.sweeps.assign(n, restarts);
    res.inner = iters;
    res.resid.resize(n);
    bool ok = true;
    for (int i = 0; i < n; ++i) {
        res.resid[i] = rel_resid(rt[i], bb[i]);
        if (!(rt[i] <= tol * tol * bb[i])) ok = false;
    }
    if (ok) return res;
    Result fb = solve(1, dag, phi, x, tol, maxiter, /*from_x=*/true);
    for (int i = 0; i < n; ++i) {
        res.sweeps[i] += fb.sweeps[i];
        res.inner[i] += fb.inner[i];
        res.resid[i] = fb.resid[i];
    }
    res.converged = fb.converged;
    return res;
}

// The learned preconditioner in its mixed-precision form: an FP64 defect
// correction (r = phi - Dhat x in FP64, x += |r| e) whose inner solve
// Dhat e = r / |r| is flexible GCR in FP32 -- the FP32 hop and Dhat tail,
// FP32 vectors with float-float dot products, one pass of classical
// Gram-Schmidt on the Dhat-images -- with z = M(r) from the network on the
// FP32 residual (M^dag(r) = gamma5 M(gamma5 r) for the adjoint system), to
// the relative target max(1e-5, 0.1 tol |phi| / |r|) of the FP32 inner solves.
// The FP64 true residual judges; FP32-inner BiCGStab continues if the sweeps
// run out above tol.
Workspace::Result Workspace::fgcr_mixed(bool use_cnn, bool dag, const FieldBuf& phi, FieldBuf& x, double tol,
                                        int maxiter) {
    REQUIRE(nlat == 1, "FGCR runs on a single lattice");
    REQUIRE(nrhs <= 8, "FGCR, Gl-BiCGStab and Bl-BiCGStab take up to 8 right-hand sides (one 32-site row per rhs)");
    ensure_cfg(0);
    ensure_cfg(1);
    ensure_cfg(3);
    ensure_inner(1);
    sf_cnn* cnn = lats[0]->cnn;
    if (use_cnn) REQUIRE(cnn != nullptr, "no learned preconditioner attached (sf_lattice_set_preconditioner)");
    cudaStream_t s = stream;
    const int n = nrhs, m = Fgcr32::M;
    if (!f32) {
        f32.reset(new Fgcr32());
        for (int k = 0; k < m; ++k) {
            f32->z[k].alloc(Prec::F32, S);
            f32->w[k].alloc(Prec::F32, S);
        }
        f32->r.alloc(Prec::F32, S);
        f32->e.alloc(Prec::F32, S);
        f32->g5a.alloc(Prec::F32, S);
        f32->g5b.alloc(Prec::F32, S);
        std::vector<void*> p(2 * m);
        for (int k = 0; k < m; ++k) {
            p[k] = f32->z[k].v.p;
            p[m + k] = f32->w[k].v.p;
        }
        f32->ptrs.ensure(p.size() * sizeof(void*));
        CK(cudaMemcpy(f32->ptrs.p, p.data(), p.size() * sizeof(void*), cudaMemcpyHostToDevice));
        const void* rp = f32->r.v.p;
        f32->rptr.ensure(sizeof(void*));
        CK(cudaMemcpy(f32->rptr.p, &rp, sizeof(void*), cudaMemcpyHostToDevice));
        f32->mdot.ensure((size_t)2 * (m + 2) * n * cfg[3].lc.nblocks * sizeof(double));
        f32->coef.ensure((size_t)2 * m * n * sizeof(double2));
        f32->dots.ensure((size_t)2 * m * n * sizeof(double2));
        f32->norms.ensure((size_t)n * sizeof(double));
        f32->invn.ensure((size_t)n * sizeof(double));
        f32->scale.ensure((size_t)n * sizeof(double));
    }
    Fgcr32& F = *f32;
    const float4* const* zp = F.ptrs.as<const float4*>();
    const float4* const* wp = zp + m;
    const LaunchCfg& bl = cfg[3].lc;
    const LaunchCfg& lc32 = cfg[1].lc;
    const KrylovOps& o32 = ops_f32();
    const FieldPtr none{nullptr, nullptr};
    const size_t fbytes64 = field_bytes(Prec::F64, S), fbytes32 = field_bytes(Prec::F32, S);
    std::vector<double2> hd((size_t)2 * m * n), hc((size_t)2 * m * n);
    auto read_dots = [&](int count) {
        CK(cudaMemcpyAsync(hd.data(), F.dots.p, (size_t)count * n * sizeof(double2), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
    };
    auto axpy = [&](const float4* const* xs, int nvec, FieldBuf& y) {
        CK(cudaMemcpyAsync(F.coef.p, hc.data(), (size_t)nvec * n * sizeof(double2), cudaMemcpyHostToDevice, s));
        CK(launch_multi_axpy32(bl, nvec, xs, F.coef.as<double2>(), y.ptr(), s));
        launches += 1;
    };
    auto apply32 = [&](const FieldBuf& in, FieldBuf& out) {   // out = Dhat in (Dhat^dag for dag), FP32
        CK(o32.hop(lc32, 1, dag, in.ptr(), inner[1].tmp.ptr(), 1.0, 0, nullptr, s));
        CK(o32.tail(lc32, 0, dag, RED_NONE, inner[1].tmp.ptr(), in.ptr(), none, out.ptr(), none, 1.0, -1.0, 2, nullptr,
                    nullptr, s));
        launches += 2;
    };
    auto set_scale = [&](const std::vector<double>& v) {
        CK(cudaMemcpyAsync(F.scale.p, v.data(), n * sizeof(double), cudaMemcpyHostToDevice, s));
    };
    // outer FP64: x = 0, r = phi
    CK(cudaMemsetAsync(x.v.p, 0, fbytes64, s));
    CK(cudaMemcpyAsync(r64.v.p, phi.v.p, fbytes64, cudaMemcpyDeviceToDevice, s));
    {
        SolverCtx k0 = ctx(false);
        CK(launch_norm2(cfg[0].lc, phi.ptr(), &k0, nrm_bb.as<double>(), s));
        launches += 2;
    }
    std::vector<double> bb(n), rr(n);
    CK(cudaMemcpyAsync(bb.data(), nrm_bb.p, n * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    rr = bb;
    const CnnLatticeView view{cfg[0].host[0], lats[0]->canon.as<double>(), s, n};
    const double nreal = 24.0 * lats[0]->Vh;
    const int max_sweeps = 12;
    std::vector<int> iters(n, 0), sweeps(n, 0);
    std::vector<double> nw((size_t)m * n), hn(n), hi(n), rin(n), target(n), sc(n);
    std::vector<char> done(n);
    int total = 0;
    for (int sweep = 0; sweep < max_sweeps && total < maxiter; ++sweep) {
        bool any = false;
        for (int i = 0; i < n; ++i) {
            const bool act = bb[i] > 0 && rr[i] > tol * tol * bb[i] && std::isfinite(rr[i]);
            sc[i] = act ? 1.0 / sqrt(rr[i]) : 0.0;
            done[i] = !act;
            rin[i] = act ? 1.0 : 0.0;
            // the inner relative target: the FP32 floor, or what tol still needs
            target[i] = act ? std::max(1e-5, 0.1 * tol * sqrt(bb[i] / rr[i])) : 0.0;
            if (act) {
                any = true;
                sweeps[i] += 1;
            }
        }
        if (!any) break;
        // inner: Dhat e = r / |r| in FP32
        set_scale(sc);
        CK(launch_to32(bl, r64.ptr(), F.scale.as<double>(), F.r.ptr(), s));
        CK(cudaMemsetAsync(F.e.v.p, 0, fbytes32, s));
        launches += 1;
        auto inner_done = [&] {
            for (char d : done)
                if (!d) return false;
            return true;
        };
        while (!inner_done() && total < maxiter) {
            for (int k = 0; k < m && !inner_done() && total < maxiter; ++k) {
                FieldBuf& zk = F.z[k];
                FieldBuf& wk = F.w[k];
                if (use_cnn) {
                    for (int i = 0; i < n; ++i) {
                        hn[i] = sqrt(rin[i] / nreal);   // RMS scale of the inner residual
                        hi[i] = hn[i] > 0 ? 1.0 / hn[i] : 0.0;
                    }
                    CK(cudaMemcpyAsync(F.norms.p, hn.data(), n * sizeof(double), cudaMemcpyHostToDevice, s));
                    CK(cudaMemcpyAsync(F.invn.p, hi.data(), n * sizeof(double), cudaMemcpyHostToDevice, s));
                    const long long planes = (long long)S / lats[0]->Vpad * 6;
                    if (dag) {
                        CK(launch_gamma5_32(planes, lats[0]->Vpad, F.r.ptr(), F.g5a.ptr(), sm_count, s));
                        CK(cnn_apply_field32(cnn, view, F.g5a.ptr(), F.norms.as<double>(), F.invn.as<double>(),
                                             F.g5b.ptr()));
                        CK(launch_gamma5_32(planes, lats[0]->Vpad, F.g5b.ptr(), zk.ptr(), sm_count, s));
                    } else {
                        CK(cnn_apply_field32(cnn, view, F.r.ptr(), F.norms.as<double>(), F.invn.as<double>(),
                                             zk.ptr()));
                    }
                    launches += 8;
                } else {
                    CK(cudaMemcpyAsync(zk.v.p, F.r.v.p, fbytes32, cudaMemcpyDeviceToDevice, s));
                }
                // w_k = Dhat z_k, orthogonalised against w_0..w_{k-1} (classical
                // Gram-Schmidt, one pass: <w_j, w_k> for all j in one kernel)
                apply32(zk, wk);
                if (k > 0) {
                    CK(launch_multidot32(bl, k, wp, wk.ptr(), F.mdot.as<double>(), F.dots.as<double2>(), s));
                    launches += 2;
                    read_dots(k);
                    for (int j = 0; j < k; ++j)
                        for (int i = 0; i < n; ++i) {
                            const double d = nw[(size_t)j * n + i];
                            const double2 v = hd[(size_t)j * n + i];
                            hc[(size_t)j * n + i] = (d > 0) ? make_double2(-v.x / d, -v.y / d) : make_double2(0, 0);
                        }
                    axpy(wp, k, wk);
                    axpy(zp, k, zk);
                }
                // |w_k|^2 and <w_k, r> in one pass over w_k: <r, w_k>^* = <w_k, r>
                {
                    const float4* const* ab = wp + k;   // a_0 = w_k
                    CK(launch_multidot32(bl, 1, ab, wk.ptr(), F.mdot.as<double>(), F.dots.as<double2>(), s));
                    CK(launch_multidot32(bl, 1, F.rptr.as<const float4*>(), wk.ptr(), F.mdot.as<double>(),
                                         F.dots.as<double2>() + n, s));
                    launches += 4;
                }
                read_dots(2);
                for (int i = 0; i < n; ++i) hd[n + i].y = -hd[n + i].y;   // <r, w_k> -> <w_k, r>
                if (use_cnn) CK(cnn_check(cnn));
                for (int i = 0; i < n; ++i) {
                    const double d = hd[i].x;
                    nw[(size_t)k * n + i] = d;
                    const double2 v = hd[n + i];
                    hc[i] = (!done[i] && d > 0) ? make_double2(v.x / d, v.y / d) : make_double2(0, 0);
                }
                axpy(zp + k, 1, F.e);
                for (int i = 0; i < n; ++i) hc[i] = make_double2(-hc[i].x, -hc[i].y);
                axpy(wp + k, 1, F.r);
                CK(launch_multidot32(bl, 1, F.rptr.as<const float4*>(), F.r.ptr(), F.mdot.as<double>(),
                                     F.dots.as<double2>(), s));
                launches += 2;
                read_dots(1);
                for (int i = 0; i < n; ++i) {
                    if (done[i]) continue;
                    rin[i] = hd[i].x;
                    iters[i] += 1;
                    if (!(rin[i] > target[i] * target[i])) done[i] = 1;
                }
                ++total;
            }
        }
        // x += |r| e, then the FP64 true residual
        for (int i = 0; i < n; ++i) sc[i] = (sweeps[i] > 0 && sc[i] > 0) ? 1.0 / sc[i] : 0.0;
        set_scale(sc);
        CK(launch_add32to64(bl, F.e.ptr(), F.scale.as<double>(), x.ptr(), s));
        launches += 1;
        residual64(dag, phi, x, s);
        CK(cudaMemcpyAsync(rr.data(), nrm_rr.p, n * sizeof(double), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
    }
    Result res;
    res.sweeps = sweeps;
    res.inner = iters;
    res.resid.resize(n);
    bool ok = true;
    for (int i = 0; i < n; ++i) {
        res.resid[i] = rel_resid(rr[i], bb[i]);
        if (!(rr[i] <= tol * tol * bb[i])) ok = false;
    }
    if (ok) return res;
    Result fb = solve(1, dag, phi, x, tol, maxiter, /*from_x=*/true);
    for (int i = 0; i < n; ++i) {
        res.sweeps[i] += fb.sweeps[i];
        res.inner[i] += fb.inner[i];
        res.resid[i] = fb.resid[i];
    }
    res.converged = fb.converged;
    return res;
}

// ---------------------------------------------------------------- Gl-BiCGStab
// the eight FP64 block vectors of Gl- and Bl-BiCGStab
void Workspace::ensure_gl() {
    if (gl) return;
    gl.reset(new Gl());
    FieldBuf* f[8] = {&gl->r, &gl->r0, &gl->p, &gl->v, &gl->s, &gl->t, &gl->ph, &gl->sh};
    std::vector<void*> p(8);
    for (int k = 0; k < 8; ++k) {
        f[k]->alloc(Prec::F64, S);
        p[k] = f[k]->v.p;
    }
    gl->ptrs.ensure(p.size() * sizeof(void*));
    CK(cudaMemcpy(gl->ptrs.p, p.data(), p.size() * sizeof(void*), cudaMemcpyHostToDevice));
    gl->coef.ensure((size_t)2 * nrhs * sizeof(double2));
    gl->dots.ensure((size_t)nrhs * sizeof(double2));
}

// out = M in, the preconditioner of the Gl-BiCGStab outer solver: for each rhs
// one FP32-inner BiCGStab solve of Dhat e = in_i / |in_i| (dag: Dhat^dag) from
// e = 0 to relative residual delta, out_i = |in_i| e (the whole block in one
// graph launch, the rhs independent of each other).  iters[i] += the inner
// iterations of rhs i.
void Workspace::precondition(bool dag, const FieldBuf& in, FieldBuf& out, double delta, int maxiter,
                             std::vector<int>& iters) {
    const int ci = 1;
    ensure_cfg(0);
    ensure_cfg(ci);
    ensure_inner(ci);
    const KrylovOps& o = ops_for(ci);
    cudaStream_t s = stream;
    const size_t n = (size_t)nlat * nrhs;
    // one "sweep" of the outer check with tol2 = 0: active where in_i != 0,
    // inv_norm = 1 / |in_i|, inner target delta
    std::vector<OState> oh(n);
    for (auto& e : oh) {
        memset(&e, 0, sizeof e);
        e.bb = 1.0;
        e.delta2_floor = delta * delta;
    }
    CK(cudaMemcpyAsync(ost.p, oh.data(), n * sizeof(OState), cudaMemcpyHostToDevice, s));
    SolverCtx k0 = ctx(false);
    CK(launch_norm2(cfg[0].lc, in.ptr(), &k0, nrm_rr.as<double>(), s));
    CK(launch_outer_check((int)n, ost.as<OState>(), nrm_rr.as<double>(), nullptr, 1, n_active.as<int>(), s));
    CK(cudaMemsetAsync(out.v.p, 0, field_bytes(Prec::F64, S), s));
    launches += 3;
    GraphEntry& ge = graph(ci, dag, false);
    CK(cudaStreamSynchronize(s));  // pin[] is rewritten below
    pin[2] = maxiter + 8;
    pin[5] = 0;
    CK(cudaMemcpyAsync(loop_count.as<int>() + 1, pin + 2, sizeof(int), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(loop_count.as<int>() + 3, pin + 5, sizeof(int), cudaMemcpyHostToDevice, s));
    SolverCtx k = ctx(true);
    CK(o.init(cfg[ci].lc, in.ptr(), inner[ci].x.ptr(), inner[ci].r.ptr(), inner[ci].r0.ptr(), inner[ci].p.ptr(),
              inner[ci].ph.ptr(), &k, maxiter, s));
    if (no_graph()) {
        for (;;) {
            enqueue_iteration(ci, dag, k, s, false);
            CK(cudaMemcpyAsync(pin + 3, loop_count.as<int>() + 2, sizeof(int), cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            if (!pin[3]) break;
        }
    } else {
        CK(cudaGraphLaunch(ge.exec, s));
    }
    CK(o.dc_update(cfg[ci].lc, out.ptr(), inner[ci].x.ptr(), &k, s));
    launches += 3;
    std::vector<OState> oo(n);
    CK(cudaMemcpyAsync(oo.data(), ost.p, n * sizeof(OState), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(pin + 5, loop_count.as<int>() + 3, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    launches += (long long)o.iteration_kernels(cfg[ci].lc) * pin[5];
    for (size_t i = 0; i < n; ++i) iters[i] += oo[i].inner_iters;
}

// Gl-BiCGStab (Jbilou, Sadok and Tinzefte 2005) on the block Dhat X = Phi
// (dag: Dhat^dag) in FP64, right-preconditioned by M (precondition(): FP32
// BiCGStab solves of the single systems, Sec. 3.2): BiCGStab whose scalars
// come from the Frobenius inner products <A, B>_F = sum_i <a_i, b_i> of the
// whole block, so that one alpha, omega, beta serve all right-hand sides and
// the preconditioner calls are independent per rhs (Sec. 3.2).  Stops when
// every rhs's recursive residual is below tol / 2 (at the half step after
// alpha as well), then judges on the recomputed FP64 residual and restarts
// from it while some rhs is above tol.  Result: sweeps = preconditioner
// calls, inner = FP32 iterations per rhs.
Workspace::Result Workspace::gl_bicgstab(bool dag, const FieldBuf& phi, FieldBuf& x, double tol, int maxiter) {
    REQUIRE(nlat == 1, "Gl-BiCGStab runs on a single lattice");
    REQUIRE(nrhs <= 8, "FGCR, Gl-BiCGStab and Bl-BiCGStab take up to 8 right-hand sides (one 32-site row per rhs)");
    // the device-resident form unless kernels are launched one by one (profilers)
    if (!no_graph()) return gl_bicgstab_graph(dag, phi, x, tol, maxiter);
    ensure_cfg(0);
    ensure_cfg(1);
    ensure_cfg(3);
    cudaStream_t s = stream;
    const int n = nrhs;
    const size_t fbytes = field_bytes(Prec::F64, S);
    ensure_gl();
    enum { kR = 0, kR0, kP, kV, kS, kT, kPH, kSH };
    const double2* const* ptr = gl->ptrs.as<const double2*>();
    const LaunchCfg& bl = cfg[3].lc;
    std::vector<double2> hd(n), hc((size_t)2 * n);
    auto dots = [&](const FieldBuf& a, const FieldBuf& b) {
        dots64(a, b, gl->dots.as<double2>(), s);
        CK(cudaMemcpyAsync(hd.data(), gl->dots.p, n * sizeof(double2), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
    };
    auto frob = [&](const FieldBuf& a, const FieldBuf& b) {
        dots(a, b);
        double2 z = make_double2(0.0, 0.0);
        for (int i = 0; i < n; ++i) {
            z.x += hd[i].x;
            z.y += hd[i].y;
        }
        return z;
    };
    // y += c0 xs[k] (+ c1 xs[k + 1]), the same coefficients for every rhs
    auto axpy = [&](int k, int nvec, double2 c0, double2 c1, FieldBuf& y) {
        for (int i = 0; i < n; ++i) {
            hc[i] = c0;
            hc[(size_t)n + i] = c1;
        }
        CK(cudaMemcpyAsync(gl->coef.p, hc.data(), (size_t)nvec * n * sizeof(double2), cudaMemcpyHostToDevice, s));
        CK(launch_multi_axpy64(bl, nvec, ptr + k, gl->coef.as<double2>(), y.ptr(), s));
        launches += 1;
    };
    auto copy = [&](const FieldBuf& from, FieldBuf& to) {
        CK(cudaMemcpyAsync(to.v.p, from.v.p, fbytes, cudaMemcpyDeviceToDevice, s));
    };
    auto cdiv = [](double2 a, double2 b) {
        const double d = b.x * b.x + b.y * b.y;
        return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
    };
    auto cmul = [](double2 a, double2 b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); };
    auto neg = [](double2 a) { return make_double2(-a.x, -a.y); };
    const double2 zero = make_double2(0.0, 0.0);
    const double delta = 1e-5;  // inner relative residual of a preconditioner call (the FP32 floor)
    const int max_outer = 100, max_restarts = 4;

    CK(cudaMemsetAsync(x.v.p, 0, fbytes, s));
    copy(phi, gl->r);
    dots(phi, phi);
    std::vector<double> bb(n);
    for (int i = 0; i < n; ++i) bb[i] = hd[i].x;
    const double stop2 = 0.25 * tol * tol;  // recursive residual target (tol / 2)
    auto below = [&](const FieldBuf& res) {  // every rhs's |res_i|^2 <= stop2 |phi_i|^2
        dots(res, res);
        for (int i = 0; i < n; ++i)
            if (!(hd[i].x <= stop2 * bb[i])) return false;
        return true;
    };
    Result res;
    res.sweeps.assign(n, 0);
    res.inner.assign(n, 0);
    res.resid.assign(n, 0.0);
    int calls = 0;
    std::vector<double> rt(n);
    for (int cycle = 0;; ++cycle) {
        copy(gl->r, gl->r0);
        copy(gl->r, gl->p);
        double2 rho = frob(gl->r0, gl->r);
        bool done = below(gl->r);
        for (int it = 0; it < max_outer && !done && rho.x != 0.0; ++it) {
            precondition(dag, gl->p, gl->ph, delta, maxiter, res.inner);
            ++calls;
            apply_dhat64(dag, gl->ph, gl->v, s);
            const double2 r0v = frob(gl->r0, gl->v);
            if (r0v.x == 0.0 && r0v.y == 0.0) break;
            const double2 alpha = cdiv(rho, r0v);
            copy(gl->r, gl->s);
            axpy(kV, 1, neg(alpha), zero, gl->s);  // s = r - alpha v
            if (below(gl->s)) {
                axpy(kPH, 1, alpha, zero, x);
                done = true;
                break;
            }
            precondition(dag, gl->s, gl->sh, delta, maxiter, res.inner);
            ++calls;
            apply_dhat64(dag, gl->sh, gl->t, s);
            const double2 ts = frob(gl->t, gl->s);
            const double2 tt = frob(gl->t, gl->t);
            if (tt.x == 0.0) break;
            const double2 omega = make_double2(ts.x / tt.x, ts.y / tt.x);
            axpy(kPH, 2, alpha, omega, x);  // x += alpha ph + omega sh
            copy(gl->s, gl->r);
            axpy(kT, 1, neg(omega), zero, gl->r);  // r = s - omega t
            if (below(gl->r)) {
                done = true;
                break;
            }
            if (omega.x == 0.0 && omega.y == 0.0) break;
            const double2 rho1 = frob(gl->r0, gl->r);
            const double2 beta = cmul(cdiv(rho1, rho), cdiv(alpha, omega));
            rho = rho1;
            axpy(kV, 1, neg(omega), zero, gl->p);  // p - omega v
            copy(gl->r, gl->s);
            axpy(kP, 1, beta, zero, gl->s);  // r + beta (p - omega v)
            copy(gl->s, gl->p);
        }
        // judge on the recomputed FP64 residual; restart from it while above tol
        residual64(dag, phi, x, s);
        CK(cudaMemcpyAsync(rt.data(), nrm_rr.p, n * sizeof(double), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        bool ok = true;
        for (int i = 0; i < n; ++i)
            if (!(bb[i] == 0.0 || rt[i] <= tol * tol * bb[i])) ok = false;
        if (ok || cycle + 1 >= max_restarts) {
            res.converged = ok;
            break;
        }
        copy(r64, gl->r);
    }
    for (int i = 0; i < n; ++i) {
        res.sweeps[i] = calls;
        res.resid[i] = rel_resid(rt[i], bb[i]);
    }
    return res;
}

// ---------------------------------------------------------------- Bl-BiCGStab
namespace {
// Solve A X = B for s x s complex A (row-major) and s x m B by Gaussian
// elimination with partial pivoting; false if a pivot vanishes.
bool small_solve(int s, std::vector<std::complex<double>> A, std::vector<std::complex<double>>& B, int m) {
    for (int k = 0; k < s; ++k) {
        int piv = k;
        for (int i = k + 1; i < s; ++i)
            if (std::abs(A[i * s + k]) > std::abs(A[piv * s + k])) piv = i;
        if (!(std::abs(A[piv * s + k]) > 0.0)) return false;
        if (piv != k) {
            for (int j = 0; j < s; ++j) std::swap(A[k * s + j], A[piv * s + j]);
            for (int j = 0; j < m; ++j) std::swap(B[k * m + j], B[piv * m + j]);
        }
        for (int i = k + 1; i < s; ++i) {
            const std::complex<double> f = A[i * s + k] / A[k * s + k];
            for (int j = k; j < s; ++j) A[i * s + j] -= f * A[k * s + j];
            for (int j = 0; j < m; ++j) B[i * m + j] -= f * B[k * m + j];
        }
    }
    for (int k = s - 1; k >= 0; --k)
        for (int j = 0; j < m; ++j) {
            std::complex<double> v = B[k * m + j];
            for (int i = k + 1; i < s; ++i) v -= A[k * s + i] * B[i * m + j];
            B[k * m + j] = v / A[k * s + k];
        }
    return true;
}
}  // namespace

void Workspace::gram64(const FieldBuf& a, const FieldBuf& b, std::vector<std::complex<double>>& G) {
    const LaunchCfg& c = cfg[3].lc;
    const int n = nrhs, S2 = (n <= 8) ? 16 : 32;
    gram_partials.ensure((size_t)n * S2 * c.nblocks * sizeof(double));
    gram_out.ensure((size_t)n * S2 * sizeof(double));
    CK(launch_gram64(c, a.ptr(), b.ptr(), gram_partials.as<double>(), gram_out.as<double>(), stream));
    launches += 2;
    std::vector<double> h((size_t)n * S2);
    CK(cudaMemcpyAsync(h.data(), gram_out.p, h.size() * sizeof(double), cudaMemcpyDeviceToHost, stream));
    CK(cudaStreamSynchronize(stream));
    G.assign((size_t)n * n, 0.0);
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) G[(size_t)i * n + j] = {h[(size_t)j * S2 + 2 * i], h[(size_t)j * S2 + 2 * i + 1]};
}

void Workspace::block_axpy64(const FieldBuf& x, const std::vector<std::complex<double>>& C, FieldBuf& y) {
    const int n = nrhs;
    std::vector<double2> hc((size_t)n * n);
    for (size_t k = 0; k < hc.size(); ++k) hc[k] = make_double2(C[k].real(), C[k].imag());
    bcoef.ensure(hc.size() * sizeof(double2));
    CK(cudaMemcpyAsync(bcoef.p, hc.data(), hc.size() * sizeof(double2), cudaMemcpyHostToDevice, stream));
    CK(launch_block_axpy64(cfg[3].lc, x.ptr(), bcoef.as<double2>(), y.ptr(), stream));
    launches += 1;
    CK(cudaStreamSynchronize(stream));  // hc leaves scope
}

// Bl-BiCGStab (El Guennouni, Jbilou and Sadok 2003) on the block Dhat X = Phi
// (dag: Dhat^dag) in FP64, the blocked solver of the paper's case C (Sec. 3.2,
// Table 1): the columns share one Krylov space through s x s coefficient
// matrices,
//   V = A P;  alpha = (R0^H V)^-1 (R0^H R);  S = R - V alpha;  T = A S;
//   omega = <T, S>_F / <T, T>_F;  X += P alpha + omega S;  R = S - omega T;
//   beta = -(R0^H V)^-1 (R0^H T);  P = R + (P - omega V) beta,
// with R0 the initial residual block, the s x s systems solved on the host
// by pivoted elimination.  Stops when every column's recursive residual is
// below tol / 2 (also at the half step after alpha), judges on the
// recomputed FP64 residual and restarts from it while a column is above tol.
// Result: sweeps = restarts + 1, inner = block iterations (each applies A to
// all s columns twice).
Workspace::Result Workspace::bl_bicgstab(bool dag, const FieldBuf& phi, FieldBuf& x, double tol, int maxiter) {
    REQUIRE(nlat == 1, "Bl-BiCGStab runs on a single lattice");
    REQUIRE(nrhs <= 8, "FGCR, Gl-BiCGStab and Bl-BiCGStab take up to 8 right-hand sides (one 32-site row per rhs)");
    if (!no_graph()) return bl_bicgstab_graph(dag, phi, x, tol, maxiter);
    ensure_cfg(0);
    ensure_cfg(3);
    cudaStream_t s = stream;
    const int n = nrhs;
    const size_t fbytes = field_bytes(Prec::F64, S);
    ensure_gl();
    using cd = std::complex<double>;
    std::vector<double2> hd(n);
    auto dots = [&](const FieldBuf& a, const FieldBuf& b) {
        dots64(a, b, gl->dots.as<double2>(), s);
        CK(cudaMemcpyAsync(hd.data(), gl->dots.p, n * sizeof(double2), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
    };
    auto copy = [&](const FieldBuf& from, FieldBuf& to) {
        CK(cudaMemcpyAsync(to.v.p, from.v.p, fbytes, cudaMemcpyDeviceToDevice, s));
    };
    auto diag = [&](cd w) {  // w times the identity
        std::vector<cd> D((size_t)n * n, 0.0);
        for (int i = 0; i < n; ++i) D[(size_t)i * n + i] = w;
        return D;
    };
    CK(cudaMemsetAsync(x.v.p, 0, fbytes, s));
    copy(phi, gl->r);
    dots(phi, phi);
    std::vector<double> bb(n);
    for (int i = 0; i < n; ++i) bb[i] = hd[i].x;
    const double stop2 = 0.25 * tol * tol;
    auto below = [&](const FieldBuf& res) {
        dots(res, res);
        for (int i = 0; i < n; ++i)
            if (!(hd[i].x <= stop2 * bb[i])) return false;
        return true;
    };
    Result res;
    res.sweeps.assign(n, 0);
    res.inner.assign(n, 0);
    res.resid.assign(n, 0.0);
    const int max_restarts = 4;
    int iters = 0, cycles = 0;
    std::vector<double> rt(n);
    std::vector<cd> M, Q, N;
    for (int cycle = 0;; ++cycle) {
        ++cycles;
        copy(gl->r, gl->r0);
        copy(gl->r, gl->p);
        bool done = below(gl->r);
        while (!done && iters < maxiter) {
            apply_dhat64(dag, gl->p, gl->v, s);
            gram64(gl->r0, gl->v, M);
            gram64(gl->r0, gl->r, Q);
            std::vector<cd> alpha = Q;
            if (!small_solve(n, M, alpha, n)) break;
            ++iters;
            copy(gl->r, gl->s);
            std::vector<cd> na(alpha);
            for (auto& z : na) z = -z;
            block_axpy64(gl->v, na, gl->s);  // S = R - V alpha
            if (below(gl->s)) {
                block_axpy64(gl->p, alpha, x);
                done = true;
                break;
            }
            apply_dhat64(dag, gl->s, gl->t, s);
            dots(gl->t, gl->s);
            cd ts = 0.0;
            for (int i = 0; i < n; ++i) ts += cd(hd[i].x, hd[i].y);
            dots(gl->t, gl->t);
            double tt = 0.0;
            for (int i = 0; i < n; ++i) tt += hd[i].x;
            if (!(tt > 0.0)) break;
            const cd omega = ts / tt;
            block_axpy64(gl->p, alpha, x);
            block_axpy64(gl->s, diag(omega), x);  // X += P alpha + omega S
            copy(gl->s, gl->r);
            block_axpy64(gl->t, diag(-omega), gl->r);  // R = S - omega T
            if (below(gl->r)) {
                done = true;
                break;
            }
            if (omega == 0.0) break;
            gram64(gl->r0, gl->t, N);
            std::vector<cd> beta = N;
            for (auto& z : beta) z = -z;
            if (!small_solve(n, M, beta, n)) break;
            block_axpy64(gl->v, diag(-omega), gl->p);  // P - omega V
            copy(gl->r, gl->ph);
            block_axpy64(gl->p, beta, gl->ph);  // R + (P - omega V) beta
            copy(gl->ph, gl->p);
        }
        residual64(dag, phi, x, s);
        CK(cudaMemcpyAsync(rt.data(), nrm_rr.p, n * sizeof(double), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        bool ok = true;
        for (int i = 0; i < n; ++i)
            if (!(bb[i] == 0.0 || rt[i] <= tol * tol * bb[i])) ok = false;
        if (ok || cycle + 1 >= max_restarts || iters >= maxiter) {
            res.converged = ok;
            break;
        }
        copy(r64, gl->r);
    }
    for (int i = 0; i < n; ++i) {
        res.sweeps[i] = cycles;
        res.inner[i] = iters;
        res.resid[i] = rel_resid(rt[i], bb[i]);
    }
    return res;
}

// ---------------------------------------------------------------- device-resident block solvers

// A block solve that ends above tol (a breakdown that restarting does not
// cure, e.g. linearly dependent right-hand sides, or the cycle cap) is
// continued from its iterate by FP32-inner BiCGStab under FP64 defect
// correction, column by column; its sweeps and iterations are added.
static void continue_per_rhs(Workspace& w, Workspace::Result& res, bool dag, const FieldBuf& phi, FieldBuf& x,
                             double tol, int maxiter) {
    if (res.converged) return;
    Workspace::Result fb = w.solve(1, dag, phi, x, tol, maxiter, /*from_x=*/true);
    for (size_t i = 0; i < res.sweeps.size(); ++i) {
        res.sweeps[i] += fb.sweeps[i];
        res.inner[i] += fb.inner[i];
        res.resid[i] = fb.resid[i];
    }
    res.converged = fb.converged;
}

void Workspace::ensure_blk() {
    if (!blk) {
        blk.reset(new Blk());
        const size_t sb = std::max(sizeof(BlState), sizeof(GlState));
        blk->state.ensure(sb);
        CK(cudaMemset(blk->state.p, 0, sb));
        for (cudaStream_t& c : blk->cs) CK(cudaStreamCreateWithFlags(&c, cudaStreamNonBlocking));
    }
    const int nb = std::max(cfg[0].lc.nblocks, cfg[3].lc.nblocks);
    const size_t need = (size_t)BLK_NQ_R * BLK_MAX * nb * sizeof(double);
    if (blk->partials.bytes < need) {
        blk->graphs.clear();   // they hold the old buffer
        blk->partials.ensure(need);
    }
}

// Bl-BiCGStab as one graph (the iteration of bl_bicgstab, Sec. 3.2 case C):
//   prologue: |phi|^2, X = 0, R = phi, state start (opens the cycle loop)
//   WHILE cycle: R0 = R, P = R, Q = R0^H R and the stop test
//     WHILE iteration: V = A P; M = R0^H V, M = QR, alpha = M^-1 Q;
//       S = R - V alpha with X += P alpha and |S|^2; the half-step test
//       IF not converged: T = A S with <T, S>, |T|^2; omega; X += omega S,
//         R = S - omega T with |R|^2, R0^H R, R0^H T; the stop test,
//         beta = -M^-1 R0^H T
//       P = R + (P - omega V) beta, and the iteration loop's condition
//     FP64 true residual, another cycle while a rhs is above tol, R = r
Workspace::Result Workspace::bl_bicgstab_graph(bool dag, const FieldBuf& phi, FieldBuf& x, double tol, int maxiter) {
    ensure_cfg(0);
    ensure_cfg(3);
    ensure_gl();
    ensure_blk();
    const int n = nrhs, max_cycles = 4;
    cudaStream_t s = stream;
    BlState* bs = blk->state.as<BlState>();
    double* pt = blk->partials.as<double>();
    const LaunchCfg& bl = cfg[3].lc;
    const int nb0 = cfg[0].lc.nblocks, nb3 = bl.nblocks;
    const long long nel = 24LL * S;   // doubles of one FP64 block vector
    const Blk::Key key{0, dag ? 1 : 0, phi.v.p, x.v.p, tol, maxiter};
    auto it = blk->graphs.find(key);
    if (it == blk->graphs.end()) {
        const KrylovOps& o64 = ops_f64();
        const FieldPtr none{nullptr, nullptr};
        Gl& g = *gl;
        auto ge = std::make_unique<GraphEntry>();
        const long long saved = launches;
        CK(cudaStreamBeginCapture(cap_top, cudaStreamCaptureModeThreadLocal));
        try {
            const cudaGraphConditionalHandle h_cycle = new_handle(cap_top);
            launches = 0;
            SolverCtx k0 = ctx(false);
            CK(launch_norm2(cfg[0].lc, phi.ptr(), &k0, nrm_bb.as<double>(), cap_top));
            CK(launch_copy_f64(x.v.as<double>(), nullptr, nel, sm_count, cap_top));
            CK(launch_copy_f64(g.r.v.as<double>(), phi.v.as<double>(), nel, sm_count, cap_top));
            CK(launch_bl_init(bs, n, nrm_bb.as<double>(), tol, maxiter, max_cycles, h_cycle, cap_top));
            ge->pro_k = launches + 5;
            cond_body(cap_top, h_cycle, cudaGraphCondTypeWhile, cap_sweep, [&](cudaStream_t c1) {
                launches = 0;
                CK(launch_copy_f64(g.r0.v.as<double>(), g.r.v.as<double>(), nel, sm_count, c1));
                CK(launch_copy_f64(g.p.v.as<double>(), g.r.v.as<double>(), nel, sm_count, c1));
                CK(launch_gram64(bl, g.r0.ptr(), g.r.ptr(), pt, nullptr, c1));
                const cudaGraphConditionalHandle h_iter = new_handle(c1);
                CK(launch_bl_fin_q(bs, pt, nb3, h_iter, c1));
                cond_body(c1, h_iter, cudaGraphCondTypeWhile, cap_stream, [&](cudaStream_t c2) {
                    const long long outer = launches;
                    launches = 0;
                    apply_dhat64(dag, g.p, g.v, c2);
                    CK(launch_gram64(bl, g.r0.ptr(), g.v.ptr(), pt, nullptr, c2));
                    CK(launch_bl_fin_alpha(bs, pt, nb3, c2));
                    CK(launch_bl_s(bl, bs, g.r.ptr(), g.v.ptr(), g.p.ptr(), g.s.ptr(), x.ptr(), pt, c2));
                    const cudaGraphConditionalHandle h_if = new_handle(c2);
                    CK(launch_bl_fin_s(bs, pt, nb3, h_if, c2));
                    cond_body(c2, h_if, cudaGraphCondTypeIf, blk->cs[0], [&](cudaStream_t c3) {
                        SolverCtx kp = ctx(false);
                        kp.partials = pt;
                        CK(o64.hop(cfg[0].lc, 1, dag, g.s.ptr(), t64o.ptr(), 1.0, 0, nullptr, c3));
                        CK(o64.tail(cfg[0].lc, 0, dag, RED_TS, t64o.ptr(), g.s.ptr(), none, g.t.ptr(), none, 1.0,
                                    -1.0, 2, &kp, nullptr, c3));
                        CK(launch_bl_fin_omega(bs, pt, nb0, c3));
                        CK(launch_bl_r(bl, bs, g.s.ptr(), g.t.ptr(), g.r0.ptr(), x.ptr(), g.r.ptr(), pt, c3));
                        CK(launch_bl_fin_r(bs, pt, nb3, c3));
                        ge->if_k = 5;
                    });
                    CK(launch_bl_p(bl, bs, g.p.ptr(), g.v.ptr(), g.r.ptr(), h_iter, c2));
                    ge->it_k = launches + 5;
                    launches = outer;
                });
                residual64(dag, phi, x, c1);
                CK(launch_bl_cycle(bs, nrm_rr.as<double>(), h_cycle, c1));
                CK(launch_copy_f64(g.r.v.as<double>(), r64.v.as<double>(), nel, sm_count, c1));
                ge->cyc_k = launches + 6;
            });
        } catch (...) {
            launches = saved;
            abandon_capture(cap_top);
            throw;
        }
        launches = saved;
        CK(cudaStreamEndCapture(cap_top, &ge->graph));
        CK(cudaGraphInstantiate(&ge->exec, ge->graph, 0));
        it = blk->graphs.emplace(key, std::move(ge)).first;
    }
    GraphEntry& ge = *it->second;
    CK(cudaGraphLaunch(ge.exec, s));
    BlState h;
    CK(cudaMemcpyAsync(&h, bs, sizeof h, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    launches += ge.pro_k + ge.cyc_k * h.cycles + ge.it_k * h.body_runs + ge.if_k * h.if_runs;
    Result res;
    res.sweeps.assign(n, h.cycles);
    res.inner.assign(n, h.iters);
    res.resid.assign(n, 0.0);
    res.converged = true;
    for (int i = 0; i < n; ++i) {
        res.resid[i] = rel_resid(h.rr[i], h.bb[i]);
        if (!(h.bb[i] == 0.0 || h.rr[i] <= tol * tol * h.bb[i])) res.converged = false;
    }
    continue_per_rhs(*this, res, dag, phi, x, tol, maxiter);
    return res;
}

// out = M in captured on s: |in|^2, the outer states of the FP32 inner
// solves (k_gl_prep: adaptive targets), out = 0, the inner start, the WHILE
// node over the inner iterations (body on child), out += |in| e
void Workspace::capture_precondition(bool dag, const FieldBuf& in, FieldBuf& out, int maxiter, cudaStream_t s,
                                     cudaStream_t child) {
    const int ci = 1;
    const KrylovOps& o = ops_for(ci);
    Inner& w = inner[ci];
    SolverCtx k0 = ctx(false);
    CK(launch_norm2(cfg[0].lc, in.ptr(), &k0, nrm_rr.as<double>(), s));
    CK(launch_gl_prep(blk->state.as<GlState>(), ost.as<OState>(), nrm_rr.as<double>(), s));
    CK(launch_copy_f64(out.v.as<double>(), nullptr, 24LL * S, sm_count, s));
    const cudaGraphConditionalHandle h_in = new_handle(s);
    SolverCtx k = ctx(true);
    k.cond = h_in;
    k.use_cond = 1;
    CK(o.init(cfg[ci].lc, in.ptr(), w.x.ptr(), w.r.ptr(), w.r0.ptr(), w.p.ptr(), w.ph.ptr(), &k, maxiter, s));
    cond_body(s, h_in, cudaGraphCondTypeWhile, child, [&](cudaStream_t c) { enqueue_iteration(ci, dag, k, c, false); });
    CK(o.dc_update(cfg[ci].lc, out.ptr(), w.x.ptr(), &k, s));
}

// Gl-BiCGStab with its FP32 preconditioner as one graph (the iteration of
// gl_bicgstab, Sec. 3.2 case D1):
//   prologue: |phi|^2, X = 0, R = phi, state start (opens the cycle loop)
//   WHILE cycle: R0 = R, P = R, rho = <R0, R>_F and the stop test
//     WHILE iteration: PH = M P; V = A PH with <R0, V>; alpha = rho / <R0, V>_F;
//       S = R - alpha V with X += alpha PH and |S|^2; the half-step test
//       IF not converged: SH = M S; T = A SH; <T, S>, |T|^2; omega;
//         X += omega SH, R = S - omega T with |R|^2, <R0, R>; the stop test, beta
//       P = R + beta (P - omega V), and the iteration loop's condition
//     FP64 true residual, another cycle while a rhs is above tol, R = r
Workspace::Result Workspace::gl_bicgstab_graph(bool dag, const FieldBuf& phi, FieldBuf& x, double tol, int maxiter) {
    ensure_cfg(0);
    ensure_cfg(1);
    ensure_cfg(3);
    ensure_inner(1);
    ensure_gl();
    ensure_blk();
    const int n = nrhs, max_cycles = 4, max_outer = 100;
    const double delta = 1e-5;   // inner relative residual of a preconditioner call (the FP32 floor)
    cudaStream_t s = stream;
    GlState* gs = blk->state.as<GlState>();
    double* pt = blk->partials.as<double>();
    const LaunchCfg& bl = cfg[3].lc;
    const int nb0 = cfg[0].lc.nblocks, nb3 = bl.nblocks;
    const long long nel = 24LL * S;
    const Blk::Key key{1, dag ? 1 : 0, phi.v.p, x.v.p, tol, maxiter};
    auto it = blk->graphs.find(key);
    if (it == blk->graphs.end()) {
        const KrylovOps& o64 = ops_f64();
        const FieldPtr none{nullptr, nullptr};
        Gl& g = *gl;
        auto ge = std::make_unique<GraphEntry>();
        const long long saved = launches;
        CK(cudaStreamBeginCapture(cap_top, cudaStreamCaptureModeThreadLocal));
        try {
            const cudaGraphConditionalHandle h_cycle = new_handle(cap_top);
            launches = 0;
            SolverCtx k0 = ctx(false);
            CK(launch_norm2(cfg[0].lc, phi.ptr(), &k0, nrm_bb.as<double>(), cap_top));
            CK(launch_copy_f64(x.v.as<double>(), nullptr, nel, sm_count, cap_top));
            CK(launch_copy_f64(g.r.v.as<double>(), phi.v.as<double>(), nel, sm_count, cap_top));
            CK(launch_gl_init(gs, n, nrm_bb.as<double>(), tol, delta, max_outer, max_cycles, ost.as<OState>(),
                              h_cycle, cap_top));
            ge->pro_k = 5;
            ge->call_k = 7;   // norm2 (2), prep, out = 0, inner start (2), update
            cond_body(cap_top, h_cycle, cudaGraphCondTypeWhile, cap_sweep, [&](cudaStream_t c1) {
                launches = 0;
                CK(launch_copy_f64(g.r0.v.as<double>(), g.r.v.as<double>(), nel, sm_count, c1));
                CK(launch_copy_f64(g.p.v.as<double>(), g.r.v.as<double>(), nel, sm_count, c1));
                CK(launch_gl_ts(bl, gs, g.r0.ptr(), g.r.ptr(), pt, c1));
                const cudaGraphConditionalHandle h_iter = new_handle(c1);
                CK(launch_gl_fin_start(gs, pt, nb3, h_iter, c1));
                cond_body(c1, h_iter, cudaGraphCondTypeWhile, cap_stream, [&](cudaStream_t c2) {
                    capture_precondition(dag, g.p, g.ph, maxiter, c2, blk->cs[0]);
                    SolverCtx kp = ctx(false);
                    kp.partials = pt;
                    CK(o64.hop(cfg[0].lc, 1, dag, g.ph.ptr(), t64o.ptr(), 1.0, 0, nullptr, c2));
                    CK(o64.tail(cfg[0].lc, 0, dag, RED_R0V, t64o.ptr(), g.ph.ptr(), none, g.v.ptr(), g.r0.ptr(), 1.0,
                                -1.0, 2, &kp, nullptr, c2));
                    CK(launch_gl_fin_alpha(gs, pt, nb0, c2));
                    CK(launch_gl_s(bl, gs, g.r.ptr(), g.v.ptr(), g.ph.ptr(), g.s.ptr(), x.ptr(), pt, c2));
                    const cudaGraphConditionalHandle h_if = new_handle(c2);
                    CK(launch_gl_fin_s(gs, pt, nb3, h_if, c2));
                    cond_body(c2, h_if, cudaGraphCondTypeIf, blk->cs[1], [&](cudaStream_t c3) {
                        capture_precondition(dag, g.s, g.sh, maxiter, c3, blk->cs[0]);
                        CK(o64.hop(cfg[0].lc, 1, dag, g.sh.ptr(), t64o.ptr(), 1.0, 0, nullptr, c3));
                        CK(o64.tail(cfg[0].lc, 0, dag, RED_NONE, t64o.ptr(), g.sh.ptr(), none, g.t.ptr(), none, 1.0,
                                    -1.0, 2, nullptr, nullptr, c3));
                        CK(launch_gl_ts(bl, gs, g.t.ptr(), g.s.ptr(), pt, c3));
                        CK(launch_gl_fin_omega(gs, pt, nb3, c3));
                        CK(launch_gl_r(bl, gs, g.s.ptr(), g.t.ptr(), g.sh.ptr(), g.r0.ptr(), x.ptr(), g.r.ptr(), pt,
                                       c3));
                        CK(launch_gl_fin_r(gs, pt, nb3, c3));
                    });
                    CK(launch_gl_p(bl, gs, g.p.ptr(), g.v.ptr(), g.r.ptr(), h_iter, c2));
                });
                residual64(dag, phi, x, c1);
                CK(launch_gl_cycle(gs, nrm_rr.as<double>(), h_cycle, c1));
                CK(launch_copy_f64(g.r.v.as<double>(), r64.v.as<double>(), nel, sm_count, c1));
            });
            ge->cyc_k = 3 + 6;   // residual (3), copies (3), Frobenius start (2), cycle check
            ge->it_k = 6;        // hop, tail, alpha, S update, half-step test, P update (the call counted apart)
            ge->if_k = 6;        // hop, tail, <T, S>, omega, R update, stop test
        } catch (...) {
            launches = saved;
            abandon_capture(cap_top);
            throw;
        }
        launches = saved;
        CK(cudaStreamEndCapture(cap_top, &ge->graph));
        CK(cudaGraphInstantiate(&ge->exec, ge->graph, 0));
        it = blk->graphs.emplace(key, std::move(ge)).first;
    }
    GraphEntry& ge = *it->second;
    // the inner solves' WHILE cap and iteration total
    pin[2] = maxiter + 8;
    pin[5] = 0;
    CK(cudaMemcpyAsync(loop_count.as<int>() + 1, pin + 2, sizeof(int), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(loop_count.as<int>() + 3, pin + 5, sizeof(int), cudaMemcpyHostToDevice, s));
    CK(cudaGraphLaunch(ge.exec, s));
    GlState h;
    std::vector<OState> oo(n);
    CK(cudaMemcpyAsync(&h, gs, sizeof h, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(oo.data(), ost.p, n * sizeof(OState), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(pin + 5, loop_count.as<int>() + 3, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    launches += ge.pro_k + ge.cyc_k * h.cycles + ge.it_k * h.body_runs + ge.if_k * h.if_runs +
                ge.call_k * h.calls + (long long)ops_for(1).iteration_kernels(cfg[1].lc) * pin[5];
    Result res;
    res.sweeps.assign(n, h.calls);
    res.inner.resize(n);
    res.resid.assign(n, 0.0);
    res.converged = true;
    for (int i = 0; i < n; ++i) {
        res.inner[i] = oo[i].inner_iters;
        res.resid[i] = rel_resid(h.rr[i], h.bb[i]);
        if (!(h.bb[i] == 0.0 || h.rr[i] <= tol * tol * h.bb[i])) res.converged = false;
    }
    continue_per_rhs(*this, res, dag, phi, x, tol, maxiter);
    return res;
}

// ---------------------------------------------------------------- helpers
namespace {

Workspace& lattice_ws(sf_lattice* lat, int nrhs) {
    if (lat->ws && lat->ws->nrhs == nrhs) return *lat->ws;
    delete lat->ws;
    lat->ws = nullptr;
    auto* w = new Workspace();
    try {
        w->setup({lat}, nrhs);
    } catch (...) {
        delete w;
        throw;
    }
    lat->ws = w;
    return *w;
}

void check_nrhs(int nrhs) { REQUIRE(nrhs >= 1 && nrhs <= SF_MAX_RHS, "nrhs must be in 1..16"); }

// copy a canonical array (host or device) into device memory `dst`
const double* to_device(const double* src, size_t bytes, DevMem& stage, cudaStream_t s) {
    if (is_device_ptr(src)) return src;
    stage.ensure(bytes);
    CK(cudaMemcpyAsync(stage.p, src, bytes, cudaMemcpyHostToDevice, s));
    return stage.as<double>();
}

// where a canonical output goes on the device
double* out_device(double* dst, size_t bytes, DevMem& stage) {
    if (is_device_ptr(dst)) return dst;
    stage.ensure(bytes);
    return stage.as<double>();
}

void finish_out(double* dst, const double* dev, size_t bytes, cudaStream_t s) {
    if (dst != dev) {
        CK(cudaMemcpyAsync(dst, dev, bytes, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
    }
}

void upload_links(sf_lattice* lat, const double* links) {
    REQUIRE(links != nullptr, "links is NULL");
    const size_t bytes = lat->links_bytes();
    if (is_device_ptr(links)) {
        CK(cudaMemcpyAsync(lat->canon.p, links, bytes, cudaMemcpyDeviceToDevice, lat->stream));
    } else {
        CK(cudaMemcpyAsync(lat->canon.p, links, bytes, cudaMemcpyHostToDevice, lat->stream));
    }
    // SU(3) check
    unsigned long long* err = reinterpret_cast<unsigned long long*>(lat->scratch.as<char>());
    CK(launch_su3_check(lat->L, lat->T, lat->canon.as<double>(), err, lat->stream));
    unsigned long long h[2];
    CK(cudaMemcpyAsync(h, err, sizeof h, cudaMemcpyDeviceToHost, lat->stream));
    CK(cudaStreamSynchronize(lat->stream));
    double e1, e2;
    memcpy(&e1, &h[0], 8);
    memcpy(&e2, &h[1], 8);
    if (!(e1 <= 1e-12) || !(e2 <= 1e-12)) {
        char buf[160];
        snprintf(buf, sizeof buf, "links not in SU(3): max|U^dag U - 1| = %.3e, max|det U - 1| = %.3e", e1, e2);
        throw SfError{SF_ENOTSU3, buf};
    }
    const LatDev g = lat->base_desc();
    CK(launch_link_prep(g, lat->canon.as<double>(), lat->stream));
}

}  // namespace

// ================================================================ C ABI
extern "C" {

const char* sf_last_error(void) { return g_err.c_str(); }

}  // extern "C"

namespace sf {
void set_last_error(const std::string& msg) { g_err = msg; }
}  // namespace sf

extern "C" {

sf_status sf_lattice_create(sf_lattice** out, int L, int T, double theta, double kappa, double beta,
                            const double* links, int device, void* stream) {
    return guarded([&] {
        REQUIRE(out != nullptr, "out is NULL");
        *out = nullptr;
        REQUIRE(L >= 2 && L <= 64 && (L % 2) == 0, "L must be even and in 2..64");
        REQUIRE(T >= 2 && T <= 64, "T must be in 2..64");
        REQUIRE(std::isfinite(theta) && std::isfinite(kappa) && std::isfinite(beta), "non-finite parameter");
        int ndev = 0;
        CK(cudaGetDeviceCount(&ndev));
        REQUIRE(device >= 0 && device < ndev, "bad device ordinal");
        CK(cudaSetDevice(device));
        std::unique_ptr<sf_lattice> lat(new sf_lattice());
        lat->L = L;
        lat->T = T;
        lat->theta = theta;
        lat->kappa = kappa;
        lat->beta = beta;
        lat->device = device;
        lat->stream = reinterpret_cast<cudaStream_t>(stream);
        CK(cudaDeviceGetAttribute(&lat->sm_count, cudaDevAttrMultiProcessorCount, device));
        lat->Vh = L * L * L * (T - 1) / 2;
        lat->Vpad = round_up(lat->Vh, 64);
        lat->canon.ensure(lat->links_bytes());
        lat->u64.ensure((size_t)4 * 2 * 9 * lat->Vpad * sizeof(double2));
        lat->u32.ensure((size_t)4 * 2 * 3 * lat->Vpad * sizeof(float4));
        lat->u16.ensure((size_t)4 * 2 * 3 * lat->Vpad * sizeof(uint2));
        lat->scratch.ensure(4096 + 2048 * sizeof(double));
        CK(cudaMemset(lat->scratch.p, 0, lat->scratch.bytes));
        upload_links(lat.get(), links);
        *out = lat.release();
    });
}

sf_status sf_lattice_set_links(sf_lattice* lat, const double* links) {
    return guarded([&] {
        REQUIRE(lat != nullptr, "lattice is NULL");
        CK(cudaSetDevice(lat->device));
        upload_links(lat, links);
    });
}

sf_status sf_lattice_set_tuning(sf_lattice* lat, sf_prec prec, int TS, int NR, int pipe) {
    return guarded([&] {
        REQUIRE(lat != nullptr, "lattice is NULL");
        REQUIRE(prec >= SF_FP64 && prec <= SF_FP16, "bad precision");
        const int ci = prec_index(prec);
        if (TS != 0) {
            REQUIRE(TS == 32 || TS == 64 || TS == 128, "TS must be 32, 64 or 128");
            REQUIRE(NR == 1 || NR == 2 || NR == 3 || NR == 5, "NR must be 1, 2, 3 or 5");
            REQUIRE(!(ci == 0 && NR > 2), "FP64 supports NR = 1 or 2");
            REQUIRE(pipe >= 0 && pipe <= 2, "pipe (the hop mode) must be 0, 1 or 2");
            REQUIRE(pipe != 1 || (ci != 0 && NR <= 2), "the pipelined hop takes FP32 / FP16 operands and NR = 1 or 2");
            REQUIRE(pipe != 2 || (ci != 0 && NR == 1 && TS == 32),
                    "staged links take FP32 / FP16 operands, NR = 1 and TS = 32");
        }
        lat->tune_TS[ci] = TS;
        lat->tune_NR[ci] = NR;
        lat->tune_pipe[ci] = TS != 0 ? pipe : 0;
        if (lat->ws) lat->ws->cfg[ci].ready = false;
    });
}

sf_status sf_lattice_get_tuning(sf_lattice* lat, sf_prec prec, int nrhs, int* TS, int* NR, int* pipe) {
    return guarded([&] {
        REQUIRE(lat != nullptr && TS != nullptr && NR != nullptr, "NULL argument");
        REQUIRE(prec >= SF_FP64 && prec <= SF_FP16, "bad precision");
        check_nrhs(nrhs);
        CK(cudaSetDevice(lat->device));
        Workspace& w = lattice_ws(lat, nrhs);
        const int ci = prec_index(prec);
        w.ensure_cfg(ci);
        *TS = w.cfg[ci].TS;
        *NR = w.cfg[ci].NR;
        if (pipe) *pipe = w.cfg[ci].pipe;
    });
}

void sf_lattice_destroy(sf_lattice* lat) {
    if (!lat) return;
    cudaSetDevice(lat->device);
    if (lat->stream) cudaStreamSynchronize(lat->stream);
    if (lat->side) {
        cudaStreamSynchronize(lat->side);
        cudaStreamDestroy(lat->side);
    }
    if (lat->side_ev) cudaEventDestroy(lat->side_ev);
    if (lat->mom_ev) cudaEventDestroy(lat->mom_ev);
    delete lat->ws;
    delete lat;
}

sf_status wilson_apply_block(sf_lattice* lat, sf_op op, sf_prec prec, int nrhs, const double* in, double* out) {
    NvtxRange nvtx_("sf wilson_apply_block");
    return guarded([&] {
        REQUIRE(lat != nullptr && in != nullptr && out != nullptr, "NULL argument");
        REQUIRE(op >= SF_OP_DHAT && op <= SF_OP_HOP_OE, "bad op");
        REQUIRE(prec >= SF_FP64 && prec <= SF_FP16, "bad precision");
        check_nrhs(nrhs);
        CK(cudaSetDevice(lat->device));
        Workspace& w = lattice_ws(lat, nrhs);
        const int ci = prec_index(prec);
        w.ensure_cfg(ci);
        w.ensure_inner(ci);
        const KrylovOps& o = ops_for(ci);
        const LaunchCfg& lc = w.cfg[ci].lc;
        const LaunchCfg& pl = w.cfg[ci].per_lat[0];
        cudaStream_t s = lat->stream;
        const size_t half = (size_t)nrhs * lat->Vh * 24 * sizeof(double);
        const bool full = (op == SF_OP_D_FULL);
        const size_t in_bytes = full ? 2 * half : half, out_bytes = full ? 2 * half : half;
        const double* din = to_device(in, in_bytes, lat->stage_in, s);
        double* dout = out_device(out, out_bytes, lat->stage_out);
        Workspace::Inner& I = w.inner[ci];
        const FieldPtr none{nullptr, nullptr};
        const bool split = hop_prec(ci) != vec_prec(ci);
        // A = vector-precision copy of the input, Ah = hop-precision copy
        FieldBuf& A = I.x;
        FieldBuf& Ah = split ? I.ph : I.x;
        FieldBuf& B = I.r;   // odd half of a full input
        FieldBuf& Bh = split ? I.sh : I.r;
        auto pack_both = [&](const double* src, FieldBuf& v, FieldBuf& h) {
            CK(o.pack(pl, src, v.ptr(), s));
            if (split) CK(o.pack_h(pl, src, h.ptr(), s));
        };
        switch (op) {
            case SF_OP_HOP_EO:
            case SF_OP_HOP_OE: {
                pack_both(din, A, Ah);
                CK(o.hop(lc, op == SF_OP_HOP_EO ? 0 : 1, false, Ah.ptr(), I.tmp.ptr(), 1.0, 0, nullptr, s));
                CK(o.unpack_h(pl, I.tmp.ptr(), dout, s));
                break;
            }
            case SF_OP_DHAT:
            case SF_OP_DHAT_DAG:
            case SF_OP_DHATDAG_DHAT: {
                pack_both(din, A, Ah);
                const bool d1 = (op == SF_OP_DHAT_DAG);
                CK(o.hop(lc, 1, d1, Ah.ptr(), I.tmp.ptr(), 1.0, 0, nullptr, s));
                CK(o.tail(lc, 0, d1, RED_NONE, I.tmp.ptr(), A.ptr(), none, I.v.ptr(), none, 1.0, -1.0, 2, nullptr,
                          nullptr, s));
                FieldBuf* res = &I.v;
                if (op == SF_OP_DHATDAG_DHAT) {
                    // second application needs the hop-precision copy of the intermediate
                    if (split) {
                        CK(o.unpack(pl, I.v.ptr(), dout, s));
                        CK(o.pack_h(pl, dout, I.sh.ptr(), s));
                    }
                    CK(o.hop(lc, 1, true, split ? I.sh.ptr() : I.v.ptr(), I.tmp.ptr(), 1.0, 0, nullptr, s));
                    CK(o.tail(lc, 0, true, RED_NONE, I.tmp.ptr(), I.v.ptr(), none, I.t.ptr(), none, 1.0, -1.0, 2,
                              nullptr, nullptr, s));
                    res = &I.t;
                }
                CK(o.unpack(pl, res->ptr(), dout, s));
                break;
            }
            case SF_OP_D_FULL: {
                const double* de = din;
                const double* dod = din + (size_t)nrhs * lat->Vh * 24;
                pack_both(de, A, Ah);
                pack_both(dod, B, Bh);
                // even: in_e - kappa H_eo in_o ; odd: in_o - kappa H_oe in_e
                CK(o.tail(lc, 0, false, RED_NONE, Bh.ptr(), A.ptr(), none, I.v.ptr(), none, 1.0, -1.0, 1, nullptr,
                          nullptr, s));
                CK(o.tail(lc, 1, false, RED_NONE, Ah.ptr(), B.ptr(), none, I.t.ptr(), none, 1.0, -1.0, 1, nullptr,
                          nullptr, s));
                CK(o.unpack(pl, I.v.ptr(), dout, s));
                CK(o.unpack(pl, I.t.ptr(), dout + (size_t)nrhs * lat->Vh * 24, s));
                break;
            }
        }
        finish_out(out, dout, out_bytes, s);
        CK(cudaGetLastError());
    });
}

sf_status wilson_hop_resident(sf_lattice* lat, sf_prec prec, int nrhs, int out_parity) {
    return guarded([&] {
        REQUIRE(lat != nullptr, "lattice is NULL");
        REQUIRE(prec >= SF_FP64 && prec <= SF_FP16, "bad precision");
        REQUIRE(out_parity == 0 || out_parity == 1, "out_parity must be 0 or 1");
        check_nrhs(nrhs);
        CK(cudaSetDevice(lat->device));
        Workspace& w = lattice_ws(lat, nrhs);
        const int ci = prec_index(prec);
        w.ensure_cfg(ci);
        w.ensure_inner(ci);
        Workspace::Inner& I = w.inner[ci];
        const bool split = hop_prec(ci) != vec_prec(ci);
        CK(ops_for(ci).hop(w.cfg[ci].lc, out_parity, false, split ? I.ph.ptr() : I.x.ptr(), I.tmp.ptr(), 1.0, 0,
                           nullptr, lat->stream));
    });
}

namespace {

void fill_info(sf_solve_info* info, const Workspace::Result& rx, const Workspace::Result* ry, int l, int nrhs,
               double secs, long long launches) {
    if (!info) return;
    memset(info, 0, sizeof *info);
    for (int i = 0; i < nrhs; ++i) {
        const int k = l * nrhs + i;
        info->iters_outer = std::max(info->iters_outer, rx.sweeps[k]);
        info->iters_inner = std::max(info->iters_inner, rx.inner[k]);
        info->iters_inner_rhs[i] = rx.inner[k];
        info->true_resid[i] = rx.resid[k];
        if (ry) {
            info->iters_outer_y = std::max(info->iters_outer_y, ry->sweeps[k]);
            info->iters_inner_y = std::max(info->iters_inner_y, ry->inner[k]);
            info->true_resid_y[i] = ry->resid[k];
        }
    }
    info->seconds = secs;
    info->kernel_launches = launches;
}

int algo_index(sf_algo a) {
    switch (a) {
        case SF_SOLVE_BICGSTAB: return 0;
        case SF_SOLVE_MIXED_DC: return 1;
        case SF_SOLVE_MIXED_DC_HALF: return 2;
        case SF_SOLVE_FGCR_CNN: return 3;
        case SF_SOLVE_FGCR: return 4;
        case SF_SOLVE_CG_NORMAL: return 5;
        case SF_SOLVE_GL_BICGSTAB: return 6;
        case SF_SOLVE_BL_BICGSTAB: return 7;
        case SF_SOLVE_FGCR_CNN_MIXED: return 8;
        case SF_SOLVE_FGCR_MIXED: return 9;
    }
    throw SfError{SF_EINVAL, "bad algorithm"};
}

}  // namespace

sf_status solve_block(sf_lattice* lat, sf_algo algo, int nrhs, const double* phi, double* X, double* Y, double tol,
                      int maxiter, sf_solve_info* info) {
    NvtxRange nvtx_("sf solve_block");
    bool noconv = false;
    sf_status st = guarded([&] {
        const auto t0 = std::chrono::steady_clock::now();
        REQUIRE(lat != nullptr && phi != nullptr && X != nullptr, "NULL argument");
        check_nrhs(nrhs);
        REQUIRE(tol > 0 && tol < 1, "tol must be in (0, 1)");
        REQUIRE(maxiter >= 1, "maxiter must be >= 1");
        const int ci = algo_index(algo);
        const bool fgcr = (ci == 3 || ci == 4), normal = (ci == 5), glb = (ci == 6), blb = (ci == 7);
        const bool fgcr32 = (ci == 8 || ci == 9);
        CK(cudaSetDevice(lat->device));
        Workspace& w = lattice_ws(lat, nrhs);
        w.launches = 0;
        w.ensure_cfg(0);
        if (!fgcr && !blb && !fgcr32) w.ensure_cfg(normal || glb ? 1 : ci);
        cudaStream_t s = lat->stream;
        const size_t bytes = (size_t)nrhs * lat->Vh * 24 * sizeof(double);
        const LaunchCfg& pl = w.cfg[0].per_lat[0];
        const double* dphi = to_device(phi, bytes, lat->stage_in, s);
        CK(ops_f64().pack(pl, dphi, w.phi64.ptr(), s));
        w.launches += 1;
        auto run = [&](bool dag, const FieldBuf& rhs, FieldBuf& sol) {
            if (glb) return w.gl_bicgstab(dag, rhs, sol, tol, maxiter);
            if (blb) return w.bl_bicgstab(dag, rhs, sol, tol, maxiter);
            if (fgcr32) return w.fgcr_mixed(ci == 8, dag, rhs, sol, tol, maxiter);
            return fgcr ? w.fgcr(ci == 3, dag, rhs, sol, tol, maxiter) : w.solve(ci, dag, rhs, sol, tol, maxiter);
        };
        Workspace::Result rx, ry;
        if (normal) w.solve_normal(w.phi64, tol, maxiter, rx, ry, /*check_y=*/true);
        else rx = run(false, w.phi64, w.x64);
        double* dX = out_device(X, bytes, lat->stage_out);
        CK(ops_f64().unpack(pl, w.x64.ptr(), dX, s));
        w.launches += 1;
        finish_out(X, dX, bytes, s);
        bool have_y = false;
        if (Y) {
            if (!normal) ry = run(true, w.x64, w.y64);
            have_y = true;
            double* dY = out_device(Y, bytes, lat->stage_out);
            CK(ops_f64().unpack(pl, w.y64.ptr(), dY, s));
            w.launches += 1;
            finish_out(Y, dY, bytes, s);
        }
        CK(cudaStreamSynchronize(s));
        const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        fill_info(info, rx, have_y ? &ry : nullptr, 0, nrhs, secs, w.launches);
        if (!rx.converged || (have_y && !ry.converged)) noconv = true;
    });
    if (st == SF_OK && noconv) {
        g_err = "solver stopped above tolerance";
        return SF_ENOCONV;
    }
    return st;
}

namespace {

// Odd-site buffers of the force, allocated on first use.
void ensure_odd(Workspace& w) {
    if (!w.xo64.v.p) {
        w.xo64.alloc(Prec::F64, w.S);
        w.yo64.alloc(Prec::F64, w.S);
    }
}

// The force of Eq. (3) from the workspace's x64, xo64, y64, yo64 (even and
// odd sites of X and Y): F = sum_i f[x_i, y_i] and / or mom -= eps F.
// mom_staged: a host mom was already copied to stage_m on the side stream
// (recorded by mom_ev)
void force_from_workspace(sf_lattice* lat, Workspace& w, double* F, double* mom, double eps,
                          bool mom_staged = false) {
    cudaStream_t s = lat->stream;
    const LaunchCfg& pl = w.cfg[0].per_lat[0];
    const size_t fbytes = (size_t)(lat->T + 1) * lat->L * lat->L * lat->L * 4 * 8 * sizeof(double);
    double* dF = nullptr;
    if (F) {
        dF = out_device(F, fbytes, lat->stage_f);
        CK(cudaMemsetAsync(dF, 0, fbytes, s));
    }
    double* dM = nullptr;
    if (mom) {
        if (is_device_ptr(mom)) {
            dM = mom;
        } else if (mom_staged) {
            CK(cudaStreamWaitEvent(s, lat->mom_ev, 0));
            dM = lat->stage_m.as<double>();
        } else {
            lat->stage_m.ensure(fbytes);
            CK(cudaMemcpyAsync(lat->stage_m.p, mom, fbytes, cudaMemcpyHostToDevice, s));
            dM = lat->stage_m.as<double>();
        }
    }
    CK(launch_force(pl, w.x64.ptr(), w.xo64.ptr(), w.y64.ptr(), w.yo64.ptr(), dF, dM, eps, s));
    w.launches += 1;
    if (F && dF != F) CK(cudaMemcpyAsync(F, dF, fbytes, cudaMemcpyDeviceToHost, s));
    if (mom && dM != mom) CK(cudaMemcpyAsync(mom, dM, fbytes, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    CK(cudaGetLastError());
}

}  // namespace

sf_status fermion_force_resident(sf_lattice* lat, int nrhs, double* F) {
    return guarded([&] {
        REQUIRE(lat != nullptr && F != nullptr, "NULL argument");
        check_nrhs(nrhs);
        cudaPointerAttributes a;
        const bool known = cudaPointerGetAttributes(&a, F) == cudaSuccess;
        if (!known) cudaGetLastError();
        REQUIRE(known && a.type == cudaMemoryTypeDevice && a.device == lat->device,
                "F must be device memory of the lattice's device");
        CK(cudaSetDevice(lat->device));
        Workspace& w = lattice_ws(lat, nrhs);
        w.ensure_cfg(0);
        ensure_odd(w);
        CK(launch_force(w.cfg[0].per_lat[0], w.x64.ptr(), w.xo64.ptr(), w.y64.ptr(), w.yo64.ptr(), F, nullptr, 0.0,
                        lat->stream));
    });
}

sf_status fermion_force(sf_lattice* lat, int nrhs, const double* X, const double* Y, double* F, double* mom,
                        double eps) {
    NvtxRange nvtx_("sf fermion_force");
    return guarded([&] {
        REQUIRE(lat != nullptr && X != nullptr && Y != nullptr, "NULL argument");
        REQUIRE(F != nullptr || mom != nullptr, "F and mom are both NULL");
        check_nrhs(nrhs);
        CK(cudaSetDevice(lat->device));
        Workspace& w = lattice_ws(lat, nrhs);
        w.ensure_cfg(0);
        ensure_odd(w);
        cudaStream_t s = lat->stream;
        const KrylovOps& o = ops_f64();
        const LaunchCfg& lc = w.cfg[0].lc;
        const LaunchCfg& pl = w.cfg[0].per_lat[0];
        const size_t bytes = (size_t)nrhs * lat->Vh * 24 * sizeof(double);
        const double* dX = to_device(X, bytes, lat->stage_in, s);
        CK(o.pack(pl, dX, w.x64.ptr(), s));
        const double* dY = to_device(Y, bytes, lat->stage_in, s);
        CK(o.pack(pl, dY, w.y64.ptr(), s));
        // odd-site reconstruction: Xh_o = kappa H_oe x_e, Yh_o = kappa gamma_5 H_oe gamma_5 y_e
        CK(o.hop(lc, 1, false, w.x64.ptr(), w.xo64.ptr(), 1.0, 1, nullptr, s));
        CK(o.hop(lc, 1, true, w.y64.ptr(), w.yo64.ptr(), 1.0, 1, nullptr, s));
        force_from_workspace(lat, w, F, mom, eps);
    });
}

sf_status md_force_step(sf_lattice* lat, sf_algo algo, int nrhs, const double* phi, double* X, double* Y,
                        double* F, double* mom, double eps, double tol, int maxiter, sf_solve_info* info) {
    NvtxRange nvtx_("sf md_force_step");
    bool noconv = false;
    sf_status st = guarded([&] {
        const auto t0 = std::chrono::steady_clock::now();
        REQUIRE(lat != nullptr && phi != nullptr && X != nullptr && Y != nullptr, "NULL argument");
        REQUIRE(F != nullptr || mom != nullptr, "F and mom are both NULL");
        check_nrhs(nrhs);
        REQUIRE(tol > 0 && tol < 1, "tol must be in (0, 1)");
        REQUIRE(maxiter >= 1, "maxiter must be >= 1");
        const int ci = algo_index(algo);
        const bool fgcr = (ci == 3 || ci == 4), normal = (ci == 5), glb = (ci == 6), blb = (ci == 7);
        const bool fgcr32 = (ci == 8 || ci == 9);
        CK(cudaSetDevice(lat->device));
        Workspace& w = lattice_ws(lat, nrhs);
        w.launches = 0;
        w.ensure_cfg(0);
        if (!fgcr && !blb && !fgcr32) w.ensure_cfg(normal || glb ? 1 : ci);
        ensure_odd(w);
        cudaStream_t s = lat->stream;
        const KrylovOps& o = ops_f64();
        const size_t bytes = (size_t)nrhs * lat->Vh * 24 * sizeof(double);
        const LaunchCfg& pl = w.cfg[0].per_lat[0];
        const double* dphi = to_device(phi, bytes, lat->stage_in, s);
        CK(o.pack(pl, dphi, w.phi64.ptr(), s));
        w.launches += 1;
        // host momenta go to the device on the side stream while the solves run
        const bool host_out = (!is_device_ptr(X) || !is_device_ptr(Y));
        const bool host_mom = (mom != nullptr && !is_device_ptr(mom));
        if ((host_out || host_mom) && !lat->side) {
            CK(cudaStreamCreateWithFlags(&lat->side, cudaStreamNonBlocking));
            CK(cudaEventCreateWithFlags(&lat->side_ev, cudaEventDisableTiming));
        }
        if (host_mom) {
            if (!lat->mom_ev) CK(cudaEventCreateWithFlags(&lat->mom_ev, cudaEventDisableTiming));
            const size_t fbytes = (size_t)(lat->T + 1) * lat->L * lat->L * lat->L * 4 * 8 * sizeof(double);
            lat->stage_m.ensure(fbytes);
            CK(cudaMemcpyAsync(lat->stage_m.p, mom, fbytes, cudaMemcpyHostToDevice, lat->side));
            CK(cudaEventRecord(lat->mom_ev, lat->side));
        }
        // X = Dhat^-1 phi and its odd part; Y = Dhat^-dag X and its odd part
        auto run = [&](bool dag, const FieldBuf& rhs, FieldBuf& sol, FieldBuf& odd) {
            if (!fgcr && !glb && !blb && ci < 8) return w.solve(ci, dag, rhs, sol, tol, maxiter, false, &odd);
            Workspace::Result r = glb     ? w.gl_bicgstab(dag, rhs, sol, tol, maxiter)
                                  : blb   ? w.bl_bicgstab(dag, rhs, sol, tol, maxiter)
                                  : ci >= 8 ? w.fgcr_mixed(ci == 8, dag, rhs, sol, tol, maxiter)
                                            : w.fgcr(ci == 3, dag, rhs, sol, tol, maxiter);
            CK(o.hop(w.cfg[0].lc, 1, dag, sol.ptr(), odd.ptr(), 1.0, 1, nullptr, s));
            w.launches += 1;
            return r;
        };
        Workspace::Result rx, ry;
        if (normal) {
            w.solve_normal(w.phi64, tol, maxiter, rx, ry, /*check_y=*/false, &w.xo64, &w.yo64);
        } else {
            rx = run(false, w.phi64, w.x64, w.xo64);
        }
        // host outputs: X and Y leave on the side stream while the Y solve and
        // the force run on the compute stream
        auto out_async = [&](double* dst, FieldBuf& f, DevMem& stage) {
            double* dv = out_device(dst, bytes, stage);
            CK(o.unpack(pl, f.ptr(), dv, s));
            if (dv != dst) {
                CK(cudaEventRecord(lat->side_ev, s));
                CK(cudaStreamWaitEvent(lat->side, lat->side_ev, 0));
                CK(cudaMemcpyAsync(dst, dv, bytes, cudaMemcpyDeviceToHost, lat->side));
            }
        };
        out_async(X, w.x64, lat->stage_out);
        if (!normal) ry = run(true, w.x64, w.y64, w.yo64);
        out_async(Y, w.y64, lat->stage_out2);
        w.launches += 2;
        force_from_workspace(lat, w, F, mom, eps, host_mom);
        CK(cudaStreamSynchronize(s));
        if (lat->side) CK(cudaStreamSynchronize(lat->side));
        const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        fill_info(info, rx, &ry, 0, nrhs, secs, w.launches);
        if (!rx.converged || !ry.converged) noconv = true;
    });
    // on a failure, copies the side stream still holds from or to the
    // caller's host buffers end before the call returns
    if (st != SF_OK && lat != nullptr && lat->side) cudaStreamSynchronize(lat->side);
    if (st == SF_OK && noconv) {
        g_err = "solver stopped above tolerance";
        return SF_ENOCONV;
    }
    return st;
}

sf_status plaquette_action(sf_lattice* lat, double* S) {
    return guarded([&] {
        REQUIRE(lat != nullptr && S != nullptr, "NULL argument");
        CK(cudaSetDevice(lat->device));
        char* base = lat->scratch.as<char>();
        unsigned* counter = reinterpret_cast<unsigned*>(base + 64);
        double* out = reinterpret_cast<double*>(base + 128);
        double* partials = reinterpret_cast<double*>(base + 4096);
        CK(launch_plaquette(lat->L, lat->T, lat->beta, lat->canon.as<double>(), partials, counter, out,
                            lat->stream));
        double h = 0;
        CK(cudaMemcpyAsync(&h, out, sizeof h, cudaMemcpyDeviceToHost, lat->stream));
        CK(cudaStreamSynchronize(lat->stream));
        *S = h;
    });
}

// ---------------------------------------------------------------- HMC trajectory
namespace {
size_t mom_bytes(const sf_lattice* lat) { return (size_t)(lat->T + 1) * lat->L * lat->L * lat->L * 4 * 8 * sizeof(double); }

// rebuild the prepared link copies from the canonical links
void prepare_links(sf_lattice* lat) {
    const LatDev g = lat->base_desc();
    CK(launch_link_prep(g, lat->canon.as<double>(), lat->stream));
}

// scale * sum of squares of n doubles (device) -> host
double sumsq(sf_lattice* lat, long long n, const double* x, double scale) {
    double* base = reinterpret_cast<double*>(lat->scratch.as<char>() + 4096 + 1024 * sizeof(double));
    CK(launch_sumsq(n, x, scale, base, base + 512, lat->stream));
    double h = 0;
    CK(cudaMemcpyAsync(&h, base + 512, sizeof h, cudaMemcpyDeviceToHost, lat->stream));
    CK(cudaStreamSynchronize(lat->stream));
    return h;
}
}  // namespace

sf_status gauge_force(sf_lattice* lat, double* F, double* mom, double eps) {
    return guarded([&] {
        REQUIRE(lat != nullptr, "lattice is NULL");
        REQUIRE(F != nullptr || mom != nullptr, "F and mom are both NULL");
        CK(cudaSetDevice(lat->device));
        cudaStream_t s = lat->stream;
        const size_t fb = mom_bytes(lat);
        DevMem fs, ms;
        double* dF = nullptr;
        if (F) dF = is_device_ptr(F) ? F : (fs.ensure(fb), fs.as<double>());
        double* dM = nullptr;
        if (mom) {
            if (is_device_ptr(mom)) {
                dM = mom;
            } else {
                ms.ensure(fb);
                CK(cudaMemcpyAsync(ms.p, mom, fb, cudaMemcpyHostToDevice, s));
                dM = ms.as<double>();
            }
        }
        CK(launch_gauge_force(lat->L, lat->T, lat->beta, lat->canon.as<double>(), dF, dM, eps, s));
        if (F && dF != F) CK(cudaMemcpyAsync(F, dF, fb, cudaMemcpyDeviceToHost, s));
        if (mom && dM != mom) CK(cudaMemcpyAsync(mom, dM, fb, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
    });
}

sf_status sf_lattice_update_links(sf_lattice* lat, const double* mom, double dt) {
    return guarded([&] {
        REQUIRE(lat != nullptr && mom != nullptr, "NULL argument");
        CK(cudaSetDevice(lat->device));
        DevMem ms;
        const double* dM = mom;
        if (!is_device_ptr(mom)) {
            ms.ensure(mom_bytes(lat));
            CK(cudaMemcpyAsync(ms.p, mom, mom_bytes(lat), cudaMemcpyHostToDevice, lat->stream));
            dM = ms.as<double>();
        }
        CK(launch_link_update(lat->L, lat->T, lat->canon.as<double>(), dM, dt, lat->stream));
        prepare_links(lat);
        CK(cudaStreamSynchronize(lat->stream));
    });
}

sf_status sf_lattice_get_links(sf_lattice* lat, double* links) {
    return guarded([&] {
        REQUIRE(lat != nullptr && links != nullptr, "NULL argument");
        CK(cudaSetDevice(lat->device));
        CK(cudaMemcpyAsync(links, lat->canon.p, lat->links_bytes(), cudaMemcpyDefault, lat->stream));
        CK(cudaStreamSynchronize(lat->stream));
    });
}

}  // extern "C"

namespace {
// One MD trajectory; lam < 0: the leapfrog with the gauge force on m
// substeps of each step (two time scales; m = 1 the plain leapfrog), else the
// second-order minimum-norm integrator of Omelyan, Mryglod and Folk with
// parameter lam.
sf_status md_trajectory(sf_lattice* lat, sf_algo algo, int nrhs, const double* phi, double* mom, int nsteps,
                        double dt, double lam, int m, double tol, int maxiter, sf_md_info* info) {
    NvtxRange nvtx_("sf md_trajectory");
    bool noconv = false;
    sf_status st = guarded([&] {
        const auto t0 = std::chrono::steady_clock::now();
        REQUIRE(lat != nullptr && phi != nullptr && mom != nullptr, "NULL argument");
        REQUIRE(nsteps >= 1, "nsteps must be >= 1");
        REQUIRE(dt > 0.0, "dt must be positive");
        check_nrhs(nrhs);
        (void)algo_index(algo);
        CK(cudaSetDevice(lat->device));
        cudaStream_t s = lat->stream;
        const size_t fb = mom_bytes(lat);
        const size_t xb = (size_t)nrhs * lat->Vh * 24 * sizeof(double);
        DevMem ms, ps, xs, ys;
        double* dM = mom;
        if (!is_device_ptr(mom)) {
            ms.ensure(fb);
            CK(cudaMemcpyAsync(ms.p, mom, fb, cudaMemcpyHostToDevice, s));
            dM = ms.as<double>();
        }
        const double* dP = phi;
        if (!is_device_ptr(phi)) {
            ps.ensure(xb);
            CK(cudaMemcpyAsync(ps.p, phi, xb, cudaMemcpyHostToDevice, s));
            dP = ps.as<double>();
        }
        xs.ensure(xb);
        ys.ensure(xb);
        long long launches = 0;
        int inner = 0, evals = 0;
        CK(launch_mom_fix(lat->L, lat->T, dM, s));
        const long long nmom = (long long)(fb / sizeof(double));
        // P -= e F_gauge(U)
        auto kick_gauge = [&](double e) {
            CK(launch_gauge_force(lat->L, lat->T, lat->beta, lat->canon.as<double>(), nullptr, dM, e, s));
            launches += 1;
        };
        // P -= e F_fermion(U); returns S_f(U) = sum |X|^2
        auto kick_fermion = [&](double e) {
            sf_solve_info fi;
            const sf_status r = md_force_step(lat, algo, nrhs, dP, xs.as<double>(), ys.as<double>(), nullptr, dM, e,
                                              tol, maxiter, &fi);
            if (r == SF_ENOCONV) noconv = true;
            else if (r != SF_OK) throw SfError{r, g_err};
            launches += fi.kernel_launches;
            inner += fi.iters_inner + fi.iters_inner_y;
            ++evals;
            return sumsq(lat, (long long)(xb / sizeof(double)), xs.as<double>(), 1.0);
        };
        // P -= e (F_gauge + F_fermion)(U); returns S_f(U)
        auto kick = [&](double e) {
            kick_gauge(e);
            return kick_fermion(e);
        };
        auto gauge_action = [&](double* S) {
            const sf_status r = plaquette_action(lat, S);
            if (r != SF_OK) throw SfError{r, g_err};
        };
        sf_md_info out;
        memset(&out, 0, sizeof out);
        out.kinetic[0] = sumsq(lat, nmom, dM, 0.5);
        gauge_action(&out.s_gauge[0]);
        // U <- exp(i e P) U and the prepared copies
        auto drift = [&](double e) {
            CK(launch_link_update(lat->L, lat->T, lat->canon.as<double>(), dM, e, s));
            prepare_links(lat);
            launches += 2;
        };
        double sf_end;
        if (lam < 0.0) {   // leapfrog; the gauge force on m substeps of dt / m (neighbouring half kicks merged)
            const double h = dt / m;
            kick_gauge(0.5 * h);
            out.s_fermion[0] = kick_fermion(0.5 * dt);
            sf_end = out.s_fermion[0];
            for (int k = 0; k < nsteps; ++k) {
                for (int j = 0; j < m; ++j) {
                    drift(h);
                    kick_gauge(k == nsteps - 1 && j == m - 1 ? 0.5 * h : h);
                }
                sf_end = kick_fermion(k == nsteps - 1 ? 0.5 * dt : dt);
            }
        } else {           // kick lam dt, drift dt/2, kick (1 - 2 lam) dt, drift dt/2, kick lam dt
            out.s_fermion[0] = kick(lam * dt);
            sf_end = out.s_fermion[0];
            for (int k = 0; k < nsteps; ++k) {
                drift(0.5 * dt);
                kick((1.0 - 2.0 * lam) * dt);
                drift(0.5 * dt);
                sf_end = kick(k == nsteps - 1 ? lam * dt : 2.0 * lam * dt);
            }
        }
        out.kinetic[1] = sumsq(lat, nmom, dM, 0.5);
        gauge_action(&out.s_gauge[1]);
        out.s_fermion[1] = sf_end;
        out.dH = (out.kinetic[1] - out.kinetic[0]) + (out.s_gauge[1] - out.s_gauge[0]) +
                 (out.s_fermion[1] - out.s_fermion[0]);
        out.force_evals = evals;
        out.inner_iters = inner;
        launches += 5 + 2 * 2 + 2;
        if (dM != mom) CK(cudaMemcpyAsync(mom, dM, fb, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        out.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        out.kernel_launches = launches;
        if (info) *info = out;
    });
    if (st == SF_OK && noconv) {
        g_err = "a solve of the trajectory stopped above tolerance";
        return SF_ENOCONV;
    }
    return st;
}
}  // namespace

extern "C" {

sf_status sf_md_trajectory(sf_lattice* lat, sf_algo algo, int nrhs, const double* phi, double* mom, int nsteps,
                           double dt, double tol, int maxiter, sf_md_info* info) {
    return md_trajectory(lat, algo, nrhs, phi, mom, nsteps, dt, -1.0, 1, tol, maxiter, info);
}

sf_status sf_md_trajectory_two_scales(sf_lattice* lat, sf_algo algo, int nrhs, const double* phi, double* mom,
                                      int nsteps, double dt, int gauge_substeps, double tol, int maxiter,
                                      sf_md_info* info) {
    if (gauge_substeps < 1 || gauge_substeps > 1000) {
        g_err = "gauge_substeps must be in 1..1000";
        return SF_EINVAL;
    }
    return md_trajectory(lat, algo, nrhs, phi, mom, nsteps, dt, -1.0, gauge_substeps, tol, maxiter, info);
}

sf_status sf_md_trajectory_omelyan(sf_lattice* lat, sf_algo algo, int nrhs, const double* phi, double* mom,
                                   int nsteps, double dt, double lambda, double tol, int maxiter, sf_md_info* info) {
    if (!(lambda > 0.0 && lambda < 0.5)) {
        g_err = "lambda must be in (0, 1/2)";
        return SF_EINVAL;
    }
    return md_trajectory(lat, algo, nrhs, phi, mom, nsteps, dt, lambda, 1, tol, maxiter, info);
}

sf_status sf_hmc_trajectory(sf_lattice* lat, sf_algo algo, int nrhs, const double* eta, double* mom, double uniform,
                            sf_md_integrator integrator, int nsteps, double dt, int gauge_substeps, double lambda,
                            double tol, int maxiter, sf_md_info* info, int* accepted) {
    NvtxRange nvtx_("sf hmc_trajectory");
    if (lat == nullptr || eta == nullptr || mom == nullptr || accepted == nullptr) {
        g_err = "NULL argument";
        return SF_EINVAL;
    }
    if (integrator != SF_MD_LEAPFROG && integrator != SF_MD_OMELYAN) {
        g_err = "unknown integrator";
        return SF_EINVAL;
    }
    if (integrator == SF_MD_OMELYAN && !(lambda > 0.0 && lambda < 0.5)) {
        g_err = "lambda must be in (0, 1/2)";
        return SF_EINVAL;
    }
    if (integrator == SF_MD_LEAPFROG && (gauge_substeps < 1 || gauge_substeps > 1000)) {
        g_err = "gauge_substeps must be in 1..1000";
        return SF_EINVAL;
    }
    *accepted = 0;
    DevMem phi, old;
    sf_status st = guarded([&] {
        check_nrhs(nrhs);
        CK(cudaSetDevice(lat->device));
        phi.ensure((size_t)nrhs * lat->Vh * 24 * sizeof(double));
        old.ensure(lat->links_bytes());
        CK(cudaMemcpyAsync(old.p, lat->canon.p, lat->links_bytes(), cudaMemcpyDeviceToDevice, lat->stream));
    });
    if (st != SF_OK) return st;
    // phi = Dhat eta: S_f = |eta|^2 at the start of the trajectory
    st = wilson_apply_block(lat, SF_OP_DHAT, SF_FP64, nrhs, eta, phi.as<double>());
    if (st != SF_OK) return st;
    sf_md_info mi;
    st = md_trajectory(lat, algo, nrhs, phi.as<double>(), mom, nsteps, dt,
                       integrator == SF_MD_OMELYAN ? lambda : -1.0,
                       integrator == SF_MD_OMELYAN ? 1 : gauge_substeps, tol, maxiter, &mi);
    if (st != SF_OK && st != SF_ENOCONV) return st;
    if (info) *info = mi;
    // Metropolis: accept with probability min(1, exp(-dH)) given the caller's uniform number
    const bool acc = uniform < std::exp(std::min(0.0, -mi.dH));
    const sf_status rs = guarded([&] {
        if (!acc) {   // back to the links at the start, and their prepared copies
            CK(cudaMemcpyAsync(lat->canon.p, old.p, lat->links_bytes(), cudaMemcpyDeviceToDevice, lat->stream));
            prepare_links(lat);
        }
        CK(cudaStreamSynchronize(lat->stream));
    });
    if (rs != SF_OK) return rs;
    *accepted = acc ? 1 : 0;
    return st;
}

// ---------------------------------------------------------------- batches
}  // extern "C"

// A batch is solved as groups of its lattices, one launch per kernel and group.
// The groups are formed so that each group's inner-loop working set (FP32 links
// and the six FP32 vectors of every RHS) fits in three quarters of L2: a
// group that spills L2 runs its stencils from HBM, where they go no faster than
// the same lattices solved one after the other (measured: eight 16^4 lattices in
// one launch, 27.9 us per lattice and Dhat against 28.9 us alone), while lattices
// too small to fill the GPU gain from sharing launches (eight 8^4: 3.7x).  Each
// group has its own workspace, so the autotuner picks the tiling per group.
struct sf_batch {
    std::vector<std::unique_ptr<Workspace>> groups;
    std::vector<std::pair<int, int>> where;   // lattice -> (group, index in the group)
    int nlat = 0, nrhs = 0, device = 0;
};

namespace {
size_t solve_working_set(const sf_lattice* l, int nrhs) {
    return (size_t)l->Vpad * (4 * 2 * 3 * 16 + (size_t)nrhs * 6 * 96);
}

// first-fit decreasing: the largest lattices first, each into the first group
// with room; a lattice above the budget gets a group of its own
std::vector<std::vector<int>> group_lattices(const std::vector<sf_lattice*>& v, int nrhs, size_t budget) {
    std::vector<int> order(v.size());
    for (size_t i = 0; i < v.size(); ++i) order[i] = (int)i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        return solve_working_set(v[a], nrhs) > solve_working_set(v[b], nrhs);
    });
    std::vector<std::vector<int>> groups;
    std::vector<size_t> used;
    for (int l : order) {
        const size_t ws = solve_working_set(v[l], nrhs);
        size_t g = 0;
        while (g < groups.size() && used[g] + ws > budget) ++g;
        if (g == groups.size()) {
            groups.emplace_back();
            used.push_back(0);
        }
        groups[g].push_back(l);
        used[g] += ws;
    }
    for (auto& g : groups) std::sort(g.begin(), g.end());   // lattices keep their order inside a group
    return groups;
}

size_t batch_budget(int device) {
    if (const char* e = getenv("SF_BATCH_BUDGET_BYTES")) {   // tests: force several groups
        const long long v = atoll(e);
        if (v > 0) return (size_t)v;
    }
    int l2 = 0;
    CK(cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, device));
    return (size_t)l2 / 4 * 3;
}
}  // namespace

extern "C" {

sf_status sf_batch_create(sf_batch** out, int nlat, sf_lattice* const* lats, int nrhs) {
    return guarded([&] {
        REQUIRE(out != nullptr && lats != nullptr, "NULL argument");
        *out = nullptr;
        REQUIRE(nlat >= 1 && nlat <= 4096, "nlat must be in 1..4096");
        check_nrhs(nrhs);
        std::vector<sf_lattice*> v(lats, lats + nlat);
        for (auto* l : v) {
            REQUIRE(l != nullptr, "NULL lattice");
            REQUIRE(l->device == v[0]->device, "lattices on different devices");
        }
        CK(cudaSetDevice(v[0]->device));
        std::unique_ptr<sf_batch> b(new sf_batch());
        b->nlat = nlat;
        b->nrhs = nrhs;
        b->device = v[0]->device;
        b->where.resize(nlat);
        for (const auto& g : group_lattices(v, nrhs, batch_budget(v[0]->device))) {
            std::vector<sf_lattice*> gl;
            for (int l : g) {
                b->where[l] = {(int)b->groups.size(), (int)gl.size()};
                gl.push_back(v[l]);
            }
            b->groups.emplace_back(new Workspace());
            b->groups.back()->setup(gl, nrhs);
        }
        *out = b.release();
    });
}

sf_status sf_batch_solve(sf_batch* b, sf_algo algo, const double* const* phi, double* const* X, double* const* Y,
                         double tol, int maxiter, sf_solve_info* info) {
    NvtxRange nvtx_("sf sf_batch_solve");
    bool noconv = false;
    sf_status st = guarded([&] {
        const auto t0 = std::chrono::steady_clock::now();
        REQUIRE(b != nullptr && phi != nullptr && X != nullptr, "NULL argument");
        REQUIRE(tol > 0 && tol < 1, "tol must be in (0, 1)");
        REQUIRE(maxiter >= 1, "maxiter must be >= 1");
        const int ci = algo_index(algo);
        REQUIRE(ci < 3 || ci == 5, "batches run the BiCGStab and CG algorithms");
        const bool normal = (ci == 5);
        for (int l = 0; l < b->nlat; ++l) REQUIRE(phi[l] != nullptr && X[l] != nullptr, "NULL array in batch");
        CK(cudaSetDevice(b->device));
        std::vector<Workspace::Result> rxs(b->groups.size()), rys(b->groups.size());
        std::vector<long long> launches(b->groups.size(), 0);
        for (size_t gi = 0; gi < b->groups.size(); ++gi) {
            Workspace& w = *b->groups[gi];
            std::vector<int> members;   // batch indices of the group's lattices, in group order
            for (int l = 0; l < b->nlat; ++l)
                if (b->where[l].first == (int)gi) members.push_back(l);
            w.launches = 0;
            w.ensure_cfg(0);
            w.ensure_cfg(normal ? 1 : ci);
            cudaStream_t s = w.stream;
            for (int k = 0; k < w.nlat; ++k) {
                const int l = members[k];
                const size_t bytes = (size_t)w.nrhs * w.lats[k]->Vh * 24 * sizeof(double);
                const double* d = to_device(phi[l], bytes, w.io, s);
                CK(ops_f64().pack(w.cfg[0].per_lat[k], d, w.phi64.ptr(), s));
                if (d != phi[l]) CK(cudaStreamSynchronize(s));
                w.launches += 1;
            }
            if (normal) {
                w.solve_normal(w.phi64, tol, maxiter, rxs[gi], rys[gi], /*check_y=*/true);
            } else {
                rxs[gi] = w.solve(ci, false, w.phi64, w.x64, tol, maxiter);
                if (Y) rys[gi] = w.solve(ci, true, w.x64, w.y64, tol, maxiter);
            }
            for (int k = 0; k < w.nlat; ++k) {
                const int l = members[k];
                const size_t bytes = (size_t)w.nrhs * w.lats[k]->Vh * 24 * sizeof(double);
                double* dX = out_device(X[l], bytes, w.io);
                CK(ops_f64().unpack(w.cfg[0].per_lat[k], w.x64.ptr(), dX, s));
                finish_out(X[l], dX, bytes, s);
                if (Y && Y[l]) {
                    double* dY = out_device(Y[l], bytes, w.io);
                    CK(ops_f64().unpack(w.cfg[0].per_lat[k], w.y64.ptr(), dY, s));
                    finish_out(Y[l], dY, bytes, s);
                }
            }
            CK(cudaStreamSynchronize(s));
            launches[gi] = w.launches;
            if (!rxs[gi].converged || (Y && !rys[gi].converged)) noconv = true;
        }
        const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (info)
            for (int l = 0; l < b->nlat; ++l) {
                const auto [gi, k] = b->where[l];
                fill_info(info + l, rxs[gi], Y ? &rys[gi] : nullptr, k, b->nrhs, secs, launches[gi]);
            }
    });
    if (st == SF_OK && noconv) {
        g_err = "solver stopped above tolerance";
        return SF_ENOCONV;
    }
    return st;
}

int sf_batch_num_groups(const sf_batch* b) { return b ? (int)b->groups.size() : -1; }

void sf_batch_destroy(sf_batch* b) {
    if (!b) return;
    cudaSetDevice(b->device);
    for (auto& w : b->groups)
        if (w->stream) cudaStreamSynchronize(w->stream);
    delete b;
}

}  // extern "C"

// ---------------------------------------------------------------- learned preconditioner
namespace {
struct CnnIo {
    Workspace* w;
    CnnLatticeView view;
};
CnnIo cnn_io(sf_lattice* lat, int nrhs) {
    Workspace& w = lattice_ws(lat, nrhs);
    w.ensure_cfg(0);
    w.ensure_cfg(3);
    return CnnIo{&w, CnnLatticeView{w.cfg[0].host[0], lat->canon.as<double>(), lat->stream, nrhs}};
}
// per-rhs |f|^2 of an FP64 workspace field (host)
std::vector<double> norms2(Workspace& w, const FieldBuf& f, cudaStream_t s) {
    w.dots64(f, f, w.ost.as<double2>(), s);  // OState scratch is free outside solves
    std::vector<double2> h(w.nrhs);
    CK(cudaMemcpyAsync(h.data(), w.ost.p, w.nrhs * sizeof(double2), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    std::vector<double> out(w.nrhs);
    for (int i = 0; i < w.nrhs; ++i) out[i] = h[i].x;
    return out;
}
}  // namespace

extern "C" {

sf_status sf_lattice_set_preconditioner(sf_lattice* lat, sf_cnn* cnn) {
    return guarded([&] {
        REQUIRE(lat != nullptr, "lattice is NULL");
        lat->cnn = cnn;
    });
}

sf_status sf_cnn_forward(sf_cnn* cnn, sf_lattice* lat, int nrhs, const double* r, double* out) {
    return guarded([&] {
        REQUIRE(cnn != nullptr && lat != nullptr && r != nullptr && out != nullptr, "NULL argument");
        check_nrhs(nrhs);
        CK(cudaSetDevice(lat->device));
        CnnIo io = cnn_io(lat, nrhs);
        Workspace& w = *io.w;
        cudaStream_t s = lat->stream;
        const size_t bytes = (size_t)nrhs * lat->Vh * 24 * sizeof(double);
        const LaunchCfg& pl = w.cfg[0].per_lat[0];
        CK(ops_f64().pack(pl, to_device(r, bytes, lat->stage_in, s), w.phi64.ptr(), s));
        std::vector<double> n2 = norms2(w, w.phi64, s), nn(nrhs), inv(nrhs);
        for (int i = 0; i < nrhs; ++i) {
            nn[i] = sqrt(n2[i] / (24.0 * lat->Vh));  // RMS scale of r
            inv[i] = nn[i] > 0 ? 1.0 / nn[i] : 0.0;
        }
        CK(cudaMemcpyAsync(w.nrm_bb.p, nn.data(), nrhs * sizeof(double), cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(w.nrm_rr.p, inv.data(), nrhs * sizeof(double), cudaMemcpyHostToDevice, s));
        CK(cnn_apply_field(cnn, io.view, w.phi64.ptr(), w.nrm_bb.as<double>(), w.nrm_rr.as<double>(), w.x64.ptr()));
        double* dout = out_device(out, bytes, lat->stage_out);
        CK(ops_f64().unpack(pl, w.x64.ptr(), dout, s));
        finish_out(out, dout, bytes, s);
        CK(cudaStreamSynchronize(s));
        CK(cnn_check(cnn));
    });
}

// one forward + backward on (r, e) pairs: the gradient of the mean relative
// squared error of the network's correction against e = Dhat^-1 r
static void cnn_grad_common(sf_cnn* cnn, sf_lattice* lat, int nrhs, const double* r, const double* e, double* loss,
                            CnnIo& io) {
    Workspace& w = *io.w;
    cudaStream_t s = lat->stream;
    const size_t bytes = (size_t)nrhs * lat->Vh * 24 * sizeof(double);
    const LaunchCfg& pl = w.cfg[0].per_lat[0];
    CK(ops_f64().pack(pl, to_device(r, bytes, lat->stage_in, s), w.phi64.ptr(), s));
    std::vector<double> r2 = norms2(w, w.phi64, s), sc(nrhs), inv(nrhs), third(nrhs);
    for (int i = 0; i < nrhs; ++i) {
        REQUIRE(r2[i] > 0, "a training residual is zero");
        sc[i] = sqrt(r2[i] / (24.0 * lat->Vh));  // RMS scale of r
        inv[i] = 1.0 / sc[i];
    }
    w.aux.ensure((size_t)3 * nrhs * sizeof(double));
    double* d_sc = w.aux.as<double>();
    double* d_inv = d_sc + nrhs;
    double* d_3 = d_sc + 2 * nrhs;
    CK(cudaMemcpyAsync(d_sc, sc.data(), nrhs * sizeof(double), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(d_inv, inv.data(), nrhs * sizeof(double), cudaMemcpyHostToDevice, s));
    if (e) {
        // error norm: mean_i |M(r_i) - e_i|^2 / |e_i|^2
        CK(ops_f64().pack(pl, to_device(e, bytes, lat->stage_in, s), w.y64.ptr(), s));
        std::vector<double> e2 = norms2(w, w.y64, s);
        for (int i = 0; i < nrhs; ++i) {
            third[i] = e2[i] * inv[i] * inv[i];
            REQUIRE(third[i] > 0, "a training target is zero");
        }
        CK(cudaMemcpyAsync(d_3, third.data(), nrhs * sizeof(double), cudaMemcpyHostToDevice, s));
        CK(cnn_loss_grad(cnn, io.view, w.phi64.ptr(), w.y64.ptr(), d_inv, d_3, loss));
        return;
    }
    // residual norm: mean_i |r_i - Dhat M(r_i)|^2 / |r_i|^2, whose gradient in
    // M(r_i) is -2 Dhat^dag (r_i - Dhat M(r_i)) / (n |r_i|^2)
    CK(cnn_apply_field(cnn, io.view, w.phi64.ptr(), d_sc, d_inv, w.x64.ptr()));
    w.residual64(false, w.phi64, w.x64, s);
    w.apply_dhat64(true, w.r64, w.y64, s);
    std::vector<double> res2(nrhs);
    CK(cudaMemcpyAsync(res2.data(), w.nrm_rr.p, nrhs * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    CK(cnn_check(cnn));
    double l = 0.0;
    for (int i = 0; i < nrhs; ++i) {
        l += res2[i] / r2[i] / nrhs;
        third[i] = -sc[i] / (nrhs * r2[i]);
    }
    if (loss) *loss = l;
    CK(cudaMemcpyAsync(d_3, third.data(), nrhs * sizeof(double), cudaMemcpyHostToDevice, s));
    CK(cnn_backward_field(cnn, io.view, w.y64.ptr(), d_3));
}

sf_status sf_cnn_train_step(sf_cnn* cnn, sf_lattice* lat, int nrhs, const double* r, const double* e, float lr,
                            double* loss) {
    return guarded([&] {
        REQUIRE(cnn != nullptr && lat != nullptr && r != nullptr, "NULL argument");
        REQUIRE(lr > 0 && lr < 1, "learning rate must be in (0, 1)");
        check_nrhs(nrhs);
        CK(cudaSetDevice(lat->device));
        CnnIo io = cnn_io(lat, nrhs);
        double l = 0.0;
        cnn_grad_common(cnn, lat, nrhs, r, e, &l, io);
        CK(cnn_adam(cnn, lr, lat->stream));
        CK(cudaStreamSynchronize(lat->stream));
        if (loss) *loss = l;
    });
}

sf_status sf_cnn_gradients(sf_cnn* cnn, sf_lattice* lat, int nrhs, const double* r, const double* e, float* grad,
                           double* loss) {
    return guarded([&] {
        REQUIRE(cnn != nullptr && lat != nullptr && r != nullptr && grad != nullptr, "NULL argument");
        check_nrhs(nrhs);
        CK(cudaSetDevice(lat->device));
        CnnIo io = cnn_io(lat, nrhs);
        double l = 0.0;
        cnn_grad_common(cnn, lat, nrhs, r, e, &l, io);
        CK(cnn_copy_grad(cnn, grad, lat->stream));
        if (loss) *loss = l;
    });
}

}  // extern "C"
