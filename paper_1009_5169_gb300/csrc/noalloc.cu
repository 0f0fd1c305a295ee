// noalloc.cu -- the SF plaquette action without any device allocation.
//
// Some callers cannot call cudaMalloc: a scheduler or runtime that owns all
// of the device memory and hands none out, a process that works inside a
// fixed memory budget set by another framework, or code that must not touch
// the allocator while other work is in flight.  plaquette_action_noalloc
// serves them: the caller passes the gauge field (device memory) and where
// to put the result, and the only scratch the reduction needs -- one partial
// sum per block, a completion counter and the final sum -- lives in the
// file-scope array g_noalloc_scratch below, which every GPU that loads this
// library holds until the process exits (64.5 KiB).
//
// The array is shared by every call: the counter is cleared at the start of
// each call, the partial sums are overwritten, and two calls whose kernels
// overlap on the GPU (different streams, no ordering between them) race on
// it and give wrong results.  Its device address is looked up with
// cudaGetSymbolAddress the first time the entry point runs on a device, with
// that device current; that first call should happen before any stream
// capture begins.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <string>

#include "sf_lattice.h"

namespace {

constexpr int kThreads = 256;
constexpr int kMaxBlocks = 8192;                               // partial sums
constexpr long long kMaxSites = (long long)kMaxBlocks * kThreads;  // gauge sites, one per thread
constexpr size_t kCounterOff = kMaxBlocks * sizeof(double);    // 64 KiB
constexpr size_t kResultOff = kCounterOff + 256;
constexpr size_t kScratchBytes = kResultOff + 256;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

struct cd {
    double re, im;
};
__device__ __forceinline__ cd mul(cd a, cd b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }

__device__ __forceinline__ void load(const double2* U, long long gi, int mu, cd (&m)[3][3]) {
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        const double2 v = __ldg(U + (gi * 4 + mu) * 9 + k);
        m[k / 3][k % 3] = cd{v.x, v.y};
    }
}

// One gauge site per thread: the site's plaquettes with SF weights
// (1/2 for spatial plaquettes at x0 = 0 and x0 = T, 1 otherwise), a block
// partial sum, and the last block to finish sums the partials in block order.
__global__ void __launch_bounds__(kThreads) k_plaquette_noalloc(int L, int T, double beta, const double2* __restrict__ U,
                                                                unsigned char* scratch) {
    double* partials = reinterpret_cast<double*>(scratch);
    unsigned* counter = reinterpret_cast<unsigned*>(scratch + kCounterOff);
    double* result = reinterpret_cast<double*>(scratch + kResultOff);
    __shared__ double sw[kThreads / 32];
    __shared__ int last;
    const long long n = (long long)(T + 1) * L * L * L;
    const long long gi = (long long)blockIdx.x * kThreads + threadIdx.x;
    double acc = 0.0;
    if (gi < n) {
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
                int a[4] = {x[0], x[1], x[2], x[3]}, b[4] = {x[0], x[1], x[2], x[3]};
                if (mu == 0) a[0] += 1; else a[mu] = (a[mu] + 1) % L;
                b[nu] = (b[nu] + 1) % L;
                const long long ga = (((long long)a[0] * L + a[1]) * L + a[2]) * L + a[3];
                const long long gb = (((long long)b[0] * L + b[1]) * L + b[2]) * L + b[3];
                cd P[3][3], Q[3][3], R[3][3], S[3][3];
                load(U, gi, mu, P);   // U_mu(x)
                load(U, ga, nu, Q);   // U_nu(x + mu)
                load(U, gb, mu, R);   // U_mu(x + nu)
                load(U, gi, nu, S);   // U_nu(x)
                double tr = 0.0;
                for (int i = 0; i < 3; ++i)
                    for (int k = 0; k < 3; ++k) {
                        cd pq{0, 0};
                        for (int j = 0; j < 3; ++j) {
                            const cd t = mul(P[i][j], Q[j][k]);
                            pq.re += t.re;
                            pq.im += t.im;
                        }
                        // (R^dag S^dag)_{k i} = sum_l conj(R_{l k}) conj(S_{i l})
                        cd rs{0, 0};
                        for (int l = 0; l < 3; ++l) {
                            const cd c = mul(cd{R[l][k].re, -R[l][k].im}, cd{S[i][l].re, -S[i][l].im});
                            rs.re += c.re;
                            rs.im += c.im;
                        }
                        tr += mul(pq, rs).re;
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
        for (int k = 0; k < kThreads / 32; ++k) s += sw[k];
        partials[blockIdx.x] = s;
        __threadfence();
        last = (atomicAdd(counter, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (last && threadIdx.x < 32) {
        __threadfence();
        double s = 0.0;
        for (int b = threadIdx.x; b < (int)gridDim.x; b += 32) s += __ldcg(partials + b);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
        if (threadIdx.x == 0) *result = beta * s;
    }
}

std::mutex g_mu;
constexpr int kMaxDevices = 64;
unsigned char* g_scratch_addr[kMaxDevices] = {};

// Where a pointer lives: 0 host (pageable or pinned), 1 device memory of
// `device`, 2 managed memory, -1 device memory of another device.
int memory_kind(const void* p, int device) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    if (a.type == cudaMemoryTypeManaged) return 2;
    if (a.type == cudaMemoryTypeDevice) return a.device == device ? 1 : -1;
    return 0;
}

// Puts the calling thread's current device back as it found it.
struct DeviceGuard {
    int prev = -1;
    DeviceGuard() {
        if (cudaGetDevice(&prev) != cudaSuccess) {
            cudaGetLastError();
            prev = -1;
        }
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

}  // namespace

namespace sf {
void set_last_error(const std::string& msg);  // api.cu: the message sf_last_error() returns
}

namespace {
sf_status fail(sf_status st, const std::string& msg) {
    sf::set_last_error(msg);
    return st;
}
}  // namespace

extern "C" sf_status plaquette_action_noalloc(int L, int T, double beta, const double* links, double* S, int device,
                                              void* stream) {
    if (L < 2 || L > 64 || (L % 2) != 0 || T < 2 || T > 64)
        return fail(SF_EINVAL, "L must be even and in 2..64, T in 2..64");
    const long long nsites = (long long)(T + 1) * L * L * L;
    if (nsites > kMaxSites)
        return fail(SF_EINVAL, "the allocation-free plaquette handles at most " + std::to_string(kMaxSites) +
                                   " gauge sites ((T+1) L^3); got " + std::to_string(nsites));
    if (links == nullptr || S == nullptr) return fail(SF_EINVAL, "links or S is NULL");
    if (!std::isfinite(beta)) return fail(SF_EINVAL, "beta is not finite");
    if (device < 0 || device >= kMaxDevices) return fail(SF_EINVAL, "bad device ordinal");
    if (reinterpret_cast<uintptr_t>(links) % 16 != 0)
        return fail(SF_EINVAL, "links must be 16-byte aligned (it is read as pairs of doubles)");
    if (reinterpret_cast<uintptr_t>(S) % alignof(double) != 0) return fail(SF_EINVAL, "S must be 8-byte aligned");
    DeviceGuard restore;   // the caller's current device is put back on every return
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) return fail(SF_ECUDA, std::string("cudaSetDevice: ") + cudaGetErrorString(e));
    const int links_kind = memory_kind(links, device);
    if (links_kind != 1 && links_kind != 2)
        return fail(SF_EINVAL, "links must be device (or managed) memory of device " + std::to_string(device));
    const int s_kind = memory_kind(S, device);
    if (s_kind < 0) return fail(SF_EINVAL, "S is device memory of another device");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const bool s_on_host_side = (s_kind != 1);   // host or managed: the call waits for the value
    if (s_on_host_side) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        e = cudaStreamIsCapturing(st, &cs);
        if (e != cudaSuccess) return fail(SF_ECUDA, std::string("cudaStreamIsCapturing: ") + cudaGetErrorString(e));
        if (cs != cudaStreamCaptureStatusNone)
            return fail(SF_EINVAL, "S must be device memory while the stream is being captured "
                                   "(a host or managed S needs a stream synchronisation)");
    }
    unsigned char* scratch = nullptr;
    {
        std::lock_guard<std::mutex> g(g_mu);
        if (g_scratch_addr[device] == nullptr) {
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess) {
                cudaGetLastError();
                return fail(SF_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            }
            g_scratch_addr[device] = static_cast<unsigned char*>(p);
        }
        scratch = g_scratch_addr[device];
    }
    e = cudaMemsetAsync(scratch + kCounterOff, 0, sizeof(unsigned), st);
    if (e != cudaSuccess) return fail(SF_ECUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
    const int blocks = (int)((nsites + kThreads - 1) / kThreads);
    k_plaquette_noalloc<<<blocks, kThreads, 0, st>>>(L, T, beta, reinterpret_cast<const double2*>(links), scratch);
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail(SF_ECUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
    if (!s_on_host_side) {
        e = cudaMemcpyAsync(S, scratch + kResultOff, sizeof(double), cudaMemcpyDeviceToDevice, st);
    } else {
        e = cudaMemcpyAsync(S, scratch + kResultOff, sizeof(double), cudaMemcpyDefault, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
    if (e != cudaSuccess) return fail(SF_ECUDA, std::string("result copy: ") + cudaGetErrorString(e));
    return SF_OK;
}
