// conv_tc.cu -- the 3^4-stencil convolution of the learned preconditioner on
// the fifth-generation tensor cores: tcgen05.mma (BF16 operands from shared
// memory, FP32 accumulator in tensor memory), issued by one thread per CTA.
//
//   Y[row][co] = bias[co] + sum_{k < 81} sum_ci X[nbr(row, k)][ci] W_k[co][ci]
//
// with the neighbour offsets d_k in {-1,0,1}^4 (d0 slowest), zero across the
// time boundaries x0 = 0, T and periodic in space, rows = (batch, site) with
// the site lexicographic over x0 = 1..T-1, x1, x2, x3 (x3 fastest).
//
// Tiling.  An MMA tile is M = 128 rows: 16 consecutive x2-lines of 8
// consecutive x3-sites at fixed (batch, x0, x1).  A tcgen05.mma costs about
// the same number of cycles for every N up to 64, so the kernel gives each
// instruction three output planes at once: the time offset d0 is folded into
// N.  A persistent CTA takes a work unit (batch, x1, 16-line block, 8-site
// block, 16-channel block) and walks the input time slices x0' = 1..T-1;
// for each of the 27 spatial offsets (d1, d2, d3) one MMA multiplies the
// input tile at (x0', x1 + d1, x2 + d2, x3 + d3) by the weights
// [W(d0 = +1) | W(d0 = 0) | W(d0 = -1)] (N = 48) into the tensor-memory
// accumulators of the output slices x0' - 1, x0', x0' + 1, which are kept
// side by side for all slices of the unit (16 columns each, slices 0 and T
// as discarded guards).  The input slice lives in shared memory as a box
//     [channel chunk kc][x1 - 1 .. x1 + 1][18 lines][10 sites]
// of 16-byte entries (8 BF16 channels), lines and sites with a halo of one
// (periodic images), in three slots (the slice in use and the next two,
// fetched with cp.async meanwhile).  Within the box the 8 sites of a line
// are 8 consecutive 16-byte rows (one core matrix of the canonical K-major
// layout without swizzling), the lines are 160 bytes apart (the stride
// between core matrices along M) and the channel chunks one box block apart
// (the stride along K), so the A operand of every spatial offset is the box
// seen through a shifted descriptor start address.  The weights of all
// offsets stay in shared memory ([offset][kc][48 columns] entries of 16
// bytes, K-major).  Output slice x0' - 2 is complete once the MMAs of input
// slice x0' - 1 are; its rows are read back with tcgen05.ld (warp w holds
// tensor-memory lanes 32 w .. 32 w + 31, i.e. rows) while the MMAs of slice
// x0' run, and bias, ReLU or the ReLU-derivative mask and the conversion are
// applied on the way out.
//
// Waits are bounded: an mbarrier wait that does not complete within about a
// second of clock cycles sets the library's error flag (read back with
// conv_tc_error) and the CTA stops; the tensor-memory columns are released
// on every path.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <utility>

#include "conv_tc.h"

namespace sfcnn {

namespace {

constexpr int TC_THREADS = 256;   // warp 0: MMA issue; warps 1-7: slice fetches; warps 4-7: epilogue
constexpr int BOX_X3 = 10;      // 8 sites + halo
constexpr int BOX_LINES = 18;   // 16 lines + halo
constexpr int SLOTS = 4;        // the slices of the MMAs in flight and the next two
constexpr int PLANE = BOX_LINES * BOX_X3;          // entries of one x1 plane of the box
constexpr int KC_STRIDE = 3 * PLANE;               // entries between channel chunks
constexpr int CB = 16;                             // output channels per unit (one TMEM block)
constexpr int NB = 3 * CB;                         // MMA N: three output slices
constexpr long long TIMEOUT_CYCLES = 2000000000LL;

__device__ int g_conv_tc_error;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// shared-memory matrix descriptor: canonical K-major layout, no swizzle
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both K-major
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, bool valid) {
    const int n = valid ? 16 : 0;   // 0: the 16 bytes are zero-filled
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }
// all but the most recent group complete
__device__ __forceinline__ void cp_async_wait_prev() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(mbar)
                 : "memory");
}

// wait for the mbarrier phase `parity`; false after the time limit
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
    const long long t0 = clock64();
    for (;;) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred P;\n mbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\n selp.b32 %0, 1, 0, P;\n}\n"
            : "=r"(done)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (done) return true;
        if (clock64() - t0 > TIMEOUT_CYCLES) return false;
    }
}

template <int N>
__device__ __forceinline__ void tmem_load_row(uint32_t taddr, float (&v)[N]) {
    static_assert(N == 16 || N == 32, "N");
    uint32_t r[N];
    if constexpr (N == 16) {
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
            : "r"(taddr));
    } else {
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
            "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
              "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]),
              "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]),
              "=r"(r[30]), "=r"(r[31])
            : "r"(taddr));
    }
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
    for (int i = 0; i < N; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ int wrap(int a, int L) { return ((a % L) + L) % L; }

}  // namespace

// The 27 x KS MMAs of one input slice (N = 48: the three output slices of
// d0 = +1, 0, -1), fully unrolled so that every descriptor is a base plus a
// compile-time offset (descriptor units: 16 bytes, the start-address field).
template <int KC, int S>
__device__ __forceinline__ void issue_offset(uint32_t d, uint64_t a0, uint64_t b0) {
    constexpr int d1 = S / 9 - 1, d2 = (S / 3) % 3 - 1, d3 = S % 3 - 1;
    constexpr uint64_t aoff = (uint64_t)((d1 + 1) * PLANE + (d2 + 1) * BOX_X3 + (d3 + 1));
    constexpr uint32_t IDESC = idesc_bf16(128, NB);
#pragma unroll
    for (int ks = 0; ks < KC / 2; ++ks) {
        const uint64_t ad = a0 + aoff + (uint64_t)(2 * ks * KC_STRIDE);
        const uint64_t bd = b0 + (uint64_t)((S * KC + 2 * ks) * NB);
        mma_bf16(d, ad, bd, IDESC, 1u);   // the accumulators are zeroed per unit
    }
}

template <int KC, int... Ss>
__device__ __forceinline__ void issue_all(uint32_t d, uint64_t a0, uint64_t b0, std::integer_sequence<int, Ss...>) {
    (issue_offset<KC, Ss>(d, a0, b0), ...);
}

template <int CIP>
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_conv_tc(ConvTcGeo g, int CI, int CO, int tmem_cols, const __nv_bfloat16* __restrict__ X,
              const __nv_bfloat16* __restrict__ Wf, const float* __restrict__ bias, int relu,
              const __nv_bfloat16* __restrict__ mask, __nv_bfloat16* __restrict__ Yh, float* __restrict__ Yf) {
    constexpr int KC = CIP / 8;                     // 16-byte channel chunks
    constexpr int SLOT_ENTRIES = KC * KC_STRIDE;    // one input slice box
    constexpr int NLOAD = TC_THREADS - 32;          // fetching threads (warps 1-7)
    extern __shared__ __align__(128) uint4 smem[];
    __shared__ int s_abort;
    const int nblk_c = (CO + CB - 1) / CB;          // 16-channel blocks of the output
    const int w_entries = nblk_c * 27 * KC * NB;
    uint4* box = smem;
    uint4* wsm = smem + SLOTS * SLOT_ENTRIES;
    uint64_t* mbar = reinterpret_cast<uint64_t*>(wsm + w_entries);   // [2]: commits of even / odd slices
    uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 2);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool issuer = (tid == 0), loader = (warp >= 1), epi = (warp >= 4);
    const int ltid = tid - 32;                      // index among the fetching threads
    const int L = g.L, T = g.T;
    const int n_x2t = (L + 15) / 16, n_x3b = (L + 7) / 8;
    const long long units = (long long)g.nb * L * n_x2t * n_x3b * nblk_c;

    // weights: entry (cblk, s, kc, n), n = 16 j + c: W_k[16 cblk + c][8 kc .. 8 kc + 7] with
    // k = (2 - j) 27 + s (column block j: d0 = 1 - j, output slice x0' + j - 1); zero padding
    for (int e = tid; e < w_entries; e += TC_THREADS) {
        const int n = e % NB, kc = (e / NB) % KC, sp = (e / (NB * KC)) % 27, cb = e / (NB * KC * 27);
        const int co = cb * CB + (n % CB), k = (2 - n / CB) * 27 + sp;
        uint4 v = make_uint4(0, 0, 0, 0);
        if (co < CO && kc * 8 < CI) v = *reinterpret_cast<const uint4*>(Wf + ((long long)k * CO + co) * CI + kc * 8);
        wsm[e] = v;
    }
    if (tid == 0) {
        s_abort = 0;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(mbar)) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(mbar + 1)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tslot)),
                     "r"(tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;   // output slice o of the unit: columns tmem + 16 o, o = 0..T
    const uint32_t box_a = smem_u32(box), w_a = smem_u32(wsm);
    const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;   // this warp's tensor-memory lane quarter
    uint32_t phase[2] = {0u, 0u};

    // This thread's entries of a slice fetch (e = ltid + NLOAD j): source
    // element offset without the x0 term and box entry, set per unit.
    constexpr int NE = (SLOT_ENTRIES + NLOAD - 1) / NLOAD;
    int src_off[NE], dst_off[NE];
    const int x0_stride = L * L * L * CI;   // elements between time slices
    auto set_unit = [&](int b, int x1, int x2_0, int x3_0) {
#pragma unroll
        for (int j = 0; j < NE; ++j) {
            const int e = ltid + j * NLOAD;
            dst_off[j] = -1;
            src_off[j] = -1;
            if (e >= SLOT_ENTRIES) continue;
            const int x3e = e % BOX_X3, line = (e / BOX_X3) % BOX_LINES, x1i = (e / PLANE) % 3, kc = e / (3 * PLANE);
            dst_off[j] = e;   // = kc * KC_STRIDE + x1i * PLANE + line * BOX_X3 + x3e
            if (kc * 8 < CI) {
                const int y1 = wrap(x1 + x1i - 1, L), y2 = wrap(x2_0 + line - 1, L), y3 = wrap(x3_0 + x3e - 1, L);
                src_off[j] = (b * g.V + (y1 * L + y2) * L + y3) * CI + kc * 8;
            }
        }
    };
    // fetching threads: input slice x0 into ring slot (x0 - 1) % 4
    auto load_slice = [&](int x0) {
        const int xoff = (x0 - 1) * x0_stride, soff = ((x0 - 1) % SLOTS) * SLOT_ENTRIES;
#pragma unroll
        for (int j = 0; j < NE; ++j) {
            if (dst_off[j] < 0) continue;
            const bool valid = src_off[j] >= 0;
            cp_async16(box_a + (uint32_t)(dst_off[j] + soff) * 16u, X + (valid ? src_off[j] + xoff : 0), valid);
        }
        cp_async_commit();
    };
    // wait for the commit of slice x0's MMAs (no barrier: the issuing warp keeps issuing);
    // a timeout raises the abort flag, which every thread reads after the next barrier
    auto wait_slice = [&](int x0) {
        const int m = x0 & 1;
        if (!mbar_wait(smem_u32(mbar + m), phase[m])) {
            s_abort = 1;
            atomicExch(&g_conv_tc_error, 1);
        }
        phase[m] ^= 1u;
        tc_fence_after();
    };
    // write output slice o (complete) of the unit: this thread's row (epilogue warps)
    auto epilogue = [&](int o, int b, int x1, int x2_0, int x3_0, int cb) {
        float v[CB];
        tmem_load_row<CB>(tmem + (uint32_t)(CB * o) + lane_base, v);
        const int row = (warp & 3) * 32 + lane;   // line (row >> 3), site (row & 7)
        const int x2 = x2_0 + (row >> 3), x3 = x3_0 + (row & 7);
        if (x2 >= L || x3 >= L) return;
        const long long orow = (long long)b * g.V + ((((long long)(o - 1) * L + x1) * L + x2) * L + x3);
#pragma unroll
        for (int c = 0; c < CB; c += 2) {
            const int co = cb * CB + c;
            if (co >= CO) break;
            float a = v[c], e2 = v[c + 1];
            if (bias) {
                a += bias[co];
                e2 += bias[co + 1];
            }
            if (relu) {
                a = fmaxf(a, 0.f);
                e2 = fmaxf(e2, 0.f);
            }
            if (mask) {
                const __nv_bfloat162 mk = *reinterpret_cast<const __nv_bfloat162*>(mask + orow * CO + co);
                if (!(__bfloat162float(mk.x) > 0.f)) a = 0.f;
                if (!(__bfloat162float(mk.y) > 0.f)) e2 = 0.f;
            }
            if (Yf) *reinterpret_cast<float2*>(Yf + orow * CO + co) = make_float2(a, e2);
            else *reinterpret_cast<__nv_bfloat162*>(Yh + orow * CO + co) = __floats2bfloat162_rn(a, e2);
        }
    };

    bool ok = true;
    for (long long u = blockIdx.x; u < units && ok; u += gridDim.x) {
        long long r = u;
        const int cb = (int)(r % nblk_c); r /= nblk_c;
        const int x3b = (int)(r % n_x3b); r /= n_x3b;
        const int x2t = (int)(r % n_x2t); r /= n_x2t;
        const int x1 = (int)(r % L); r /= L;
        const int b = (int)r;
        const int x2_0 = x2t * 16, x3_0 = x3b * 8;
        if (loader) {
            set_unit(b, x1, x2_0, x3_0);
            load_slice(1);
            if (T - 1 >= 2) load_slice(2);
        }
        if (epi) {   // zero this warp's lanes of the T + 1 output slices (the MMAs only accumulate)
            uint32_t z[CB];
#pragma unroll
            for (int c = 0; c < CB; ++c) z[c] = 0u;
            for (int o = 0; o <= T; ++o)
                asm volatile(
                    "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};\n" ::"r"(
                        tmem + (uint32_t)(CB * o) + lane_base),
                    "r"(z[0]), "r"(z[1]), "r"(z[2]), "r"(z[3]), "r"(z[4]), "r"(z[5]), "r"(z[6]), "r"(z[7]), "r"(z[8]),
                    "r"(z[9]), "r"(z[10]), "r"(z[11]), "r"(z[12]), "r"(z[13]), "r"(z[14]), "r"(z[15])
                    : "memory");
            asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory");
        }
        const uint64_t b0 = sdesc(w_a + (uint32_t)(cb * 27 * KC * NB) * 16u, NB * 16, 128);
        for (int x0 = 1; x0 <= T - 1; ++x0) {
            if (loader) {   // this thread's part of slice x0 (slice x0 + 1 may still be in flight)
                if (x0 + 1 <= T - 1) cp_async_wait_prev();
                else cp_async_wait_all();
            }
            fence_proxy_async();
            tc_fence_before();
            __syncthreads();
            tc_fence_after();
            if (s_abort) {
                ok = false;
                break;
            }
            if (issuer) {
                const uint64_t a0 = sdesc(box_a + (uint32_t)(((x0 - 1) % SLOTS) * SLOT_ENTRIES) * 16u,
                                          KC_STRIDE * 16, BOX_X3 * 16);
                issue_all<KC>(tmem + (uint32_t)(CB * (x0 - 1)), a0, b0, std::make_integer_sequence<int, 27>{});
                mma_commit(smem_u32(mbar + (x0 & 1)));
            }
            if (warp >= 1 && x0 >= 2) {
                wait_slice(x0 - 1);   // then slice x0 - 2's slot is free and output x0 - 2 complete
                if (x0 + 2 <= T - 1) load_slice(x0 + 2);
                if (epi && x0 >= 3) epilogue(x0 - 2, b, x1, x2_0, x3_0, cb);
            } else if (loader && x0 + 2 <= T - 1) {
                load_slice(x0 + 2);   // x0 = 1: slot 3 is unused yet
            }
        }
        // the unit's last slice: its MMAs, then outputs T - 2 and T - 1
        __syncthreads();
        if (!ok || s_abort) {
            ok = false;
            break;
        }
        if (warp >= 1) {
            wait_slice(T - 1);
            if (epi) {
                if (T - 2 >= 1) epilogue(T - 2, b, x1, x2_0, x3_0, cb);
                epilogue(T - 1, b, x1, x2_0, x3_0, cb);
            }
        } else {
            phase[(T - 1) & 1] ^= 1u;   // the issuing warp's view of the same phase
        }
        tc_fence_before();
        __syncthreads();   // every epilogue read done before the next unit zeroes the accumulators
        tc_fence_after();
        if (s_abort) ok = false;
    }
    // release the tensor memory (every thread's reads are complete: tcgen05.wait::ld)
    cp_async_wait_all();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(tmem_cols) : "memory");
}

template <int CIP>
static size_t conv_tc_smem(int co) {
    const int nblk_c = (co + CB - 1) / CB;
    return (size_t)SLOTS * (CIP / 8) * KC_STRIDE * 16 + (size_t)nblk_c * 27 * (CIP / 8) * NB * 16 + 32;
}

template <int CIP>
static cudaError_t launch_tc(const ConvTcGeo& g, int CI, int CO, const __nv_bfloat16* X, const __nv_bfloat16* W,
                             const float* bias, int relu, const __nv_bfloat16* mask, __nv_bfloat16* Yh, float* Yf,
                             int sm_count, cudaStream_t st) {
    const size_t smem = conv_tc_smem<CIP>(CO);
    if (smem > 225u * 1024u) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(k_conv_tc<CIP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int cols = 32;
    while (cols < (g.T + 1) * CB) cols *= 2;   // a power of two, at most 512 (T <= 31)
    const int nblk_c = (CO + CB - 1) / CB;
    const long long units = (long long)g.nb * g.L * ((g.L + 15) / 16) * ((g.L + 7) / 8) * nblk_c;
    const int per_sm = std::max(1, std::min<int>(512 / cols, (int)((225u * 1024u) / smem)));
    const int grid = (int)std::min<long long>(units, (long long)sm_count * per_sm);
    k_conv_tc<CIP><<<grid, TC_THREADS, smem, st>>>(g, CI, CO, cols, X, W, bias, relu, mask, Yh, Yf);
    return cudaGetLastError();
}

bool conv_tc_supported(int ci, int co) {
    if (ci % 8 != 0 || co % 2 != 0 || ci > 32 || co > 32 || ci < 8 || co < 2) return false;
    const int cip = ci <= 16 ? 16 : 32;
    const size_t smem = cip == 16 ? conv_tc_smem<16>(co) : conv_tc_smem<32>(co);
    return smem <= 225u * 1024u;   // two input slices and the weights of all offsets in shared memory
}

cudaError_t conv_tc(const ConvTcGeo& g, int ci, int co, const __nv_bfloat16* X, const __nv_bfloat16* W,
                    const float* bias, int relu, const __nv_bfloat16* mask, __nv_bfloat16* Yh, float* Yf, int sm_count,
                    cudaStream_t st) {
    if (!conv_tc_supported(ci, co) || g.L < 2 || g.T < 2 || g.T > 31) return cudaErrorInvalidValue;
    if ((long long)g.nb * g.V * 32 >= (1LL << 31)) return cudaErrorInvalidValue;   // 32-bit element offsets
    if (ci <= 16) return launch_tc<16>(g, ci, co, X, W, bias, relu, mask, Yh, Yf, sm_count, st);
    return launch_tc<32>(g, ci, co, X, W, bias, relu, mask, Yh, Yf, sm_count, st);
}

int conv_tc_error(bool reset) {
    int v = 0;
    cudaMemcpyFromSymbol(&v, g_conv_tc_error, sizeof(int));
    if (reset && v) {
        const int z = 0;
        cudaMemcpyToSymbol(g_conv_tc_error, &z, sizeof(int));
    }
    return v;
}

}  // namespace sfcnn
