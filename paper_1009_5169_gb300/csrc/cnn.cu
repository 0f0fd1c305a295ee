// cnn.cu -- the learned preconditioner: a 4-layer 3^4-stencil convolutional
// network on the full SF fermion lattice, trained and applied with
// hand-written BF16 tensor-core kernels with FP32 accumulation -- the
// convolutions on tcgen05 (conv_tc.cu) where the layer shape fits its shared
// memory (hidden width 16), mma.sync m16n8k16 (k_conv below) otherwise and
// for the weight gradients -- used as the preconditioner M of flexible GCR.
//
// Network (widths 32 -> H -> H -> H -> 24, H = 16 or 32):
//   input   channels 0..23: the even-site residual r/s, s = |r|/sqrt(24 V/2)
//           its RMS scale (spin, colour, re/im; zero on odd sites);
//           24..31: Re, Im of tr U_mu(x)/3, mu = 0..3;
//   layer   Y(x) = b + sum_k X(x + d_k) W_k, d_k in {-1,0,1}^4 (81 offsets,
//           d0 slowest), zero across the time boundaries, periodic in space;
//           ReLU after layers 0..2;
//   output  channels 0..23 on the even sites;
//           M(r) = r + s (out(r/s) - out(-r/s)) / 2: the network learns the
//           correction to the identity, the symmetrisation makes M odd and
//           positively homogeneous (both signs run as one batch).
// Layouts: activations [batch][site][channel] BF16 (site lexicographic over
// the fermion lattice, x3 fastest); weights per layer FP32 master
// W[81][ci][co] and bias [co]; BF16 copies Wf[k][co][ci] (forward) and
// Wb[k][ci][co] = W[81-1-k] (backward data: the transposed map with the
// offset reversed).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "conv_tc.h"
#include "krylov_impl.cuh"
#include "sf_lattice.h"

namespace sf {
void set_last_error(const std::string& msg);
}

namespace sfcnn {
using namespace sf;

constexpr int NOFF = 81;
constexpr int CIN0 = 32;
constexpr int COUT = 24;
constexpr int ROWS = 128;   // rows (sites) per forward block
constexpr int PADH = 8;     // smem row padding (halves) against bank conflicts

struct Geo {
    int L, T, V;       // fermion lattice, V = (T-1) L^3
    int nb;            // batch (right-hand sides)
};

__device__ __forceinline__ void site_coords(const Geo& g, int s, int (&x)[4]) {
    x[3] = s % g.L;
    s /= g.L;
    x[2] = s % g.L;
    s /= g.L;
    x[1] = s % g.L;
    x[0] = s / g.L + 1;
}

// neighbour x + d_k of site s (lexicographic), or -1 outside the time range
__device__ __forceinline__ int nbr(const Geo& g, const int (&x)[4], int k) {
    const int d0 = k / 27 - 1, d1 = (k / 9) % 3 - 1, d2 = (k / 3) % 3 - 1, d3 = k % 3 - 1;
    const int y0 = x[0] + d0;
    if (y0 < 1 || y0 > g.T - 1) return -1;
    const int y1 = (x[1] + d1 + g.L) % g.L, y2 = (x[2] + d2 + g.L) % g.L, y3 = (x[3] + d3 + g.L) % g.L;
    return (((y0 - 1) * g.L + y1) * g.L + y2) * g.L + y3;
}

__device__ __forceinline__ uint32_t pack2(__nv_bfloat16 lo, __nv_bfloat16 hi) {
    return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// ------------------------------------------------------------ convolution
// Y[row][co] = sum_k sum_ci X[nbr(row, k)][ci] B_k[co][ci] (+ bias), one
// block per ROWS rows of the (batch x site) matrix, 4 warps of 32 rows.
// Optional epilogues: ReLU, multiply by (mask > 0), FP32 or BF16 output.
template <int CI, int CO>
__global__ void __launch_bounds__(128) k_conv(Geo g, const __nv_bfloat16* __restrict__ X,
                                              const __nv_bfloat16* __restrict__ B, const float* __restrict__ bias,
                                              int relu, const __nv_bfloat16* __restrict__ mask,
                                              __nv_bfloat16* __restrict__ Yh, float* __restrict__ Yf) {
    static_assert(CI % 8 == 0 && CO % 8 == 0, "channel counts");
    constexpr int NT = CO / 8;
    constexpr int CIP = (CI + 15) / 16 * 16;  // K padded to the MMA step with zeros
    __shared__ __align__(16) __nv_bfloat16 As[ROWS][CIP + PADH];
    __shared__ __align__(16) __nv_bfloat16 Bs[CO][CIP + PADH];
    if (CIP != CI) {
        // zero the padding columns once; the per-offset loads never touch them
        for (int q = threadIdx.x; q < ROWS; q += 128)
            for (int c = CI; c < CIP; ++c) As[q][c] = __float2bfloat16(0.f);
        for (int q = threadIdx.x; q < CO; q += 128)
            for (int c = CI; c < CIP; ++c) Bs[q][c] = __float2bfloat16(0.f);
    }
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, gq = lane >> 2, tq = lane & 3;
    const long long nrows = (long long)g.nb * g.V;
    const long long row = (long long)blockIdx.x * ROWS + tid;
    int x[4] = {0, 0, 0, 0};
    int bidx = 0;
    const bool valid = row < nrows;
    if (valid) {
        bidx = (int)(row / g.V);
        site_coords(g, (int)(row - (long long)bidx * g.V), x);
    }
    float acc[2][NT][4];
#pragma unroll
    for (int m = 0; m < 2; ++m)
#pragma unroll
        for (int n = 0; n < NT; ++n)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[m][n][q] = 0.f;
    for (int k = 0; k < NOFF; ++k) {
        // gather the k-th neighbour row of every row of the tile
        const int s = valid ? nbr(g, x, k) : -1;
        uint4* dst = reinterpret_cast<uint4*>(&As[tid][0]);
        if (s >= 0) {
            const uint4* src = reinterpret_cast<const uint4*>(X + ((long long)bidx * g.V + s) * CI);
#pragma unroll
            for (int q = 0; q < CI / 8; ++q) dst[q] = __ldg(src + q);
        } else {
#pragma unroll
            for (int q = 0; q < CI / 8; ++q) dst[q] = make_uint4(0, 0, 0, 0);
        }
        // the offset's weight block [CO][CI]
        const uint4* wsrc = reinterpret_cast<const uint4*>(B + (long long)k * CO * CI);
        for (int q = tid; q < CO * CI / 8; q += 128) {
            const int r = q / (CI / 8), c = q % (CI / 8);
            *reinterpret_cast<uint4*>(&Bs[r][c * 8]) = __ldg(wsrc + q);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < CIP / 16; ++kk) {
            uint32_t a[2][4];
#pragma unroll
            for (int m = 0; m < 2; ++m) {
                const int r0 = warp * 32 + m * 16 + gq;
                const int c0 = kk * 16 + tq * 2;
                a[m][0] = *reinterpret_cast<const uint32_t*>(&As[r0][c0]);
                a[m][1] = *reinterpret_cast<const uint32_t*>(&As[r0 + 8][c0]);
                a[m][2] = *reinterpret_cast<const uint32_t*>(&As[r0][c0 + 8]);
                a[m][3] = *reinterpret_cast<const uint32_t*>(&As[r0 + 8][c0 + 8]);
            }
#pragma unroll
            for (int n = 0; n < NT; ++n) {
                uint32_t b[2];
                const int c0 = kk * 16 + tq * 2;
                b[0] = *reinterpret_cast<const uint32_t*>(&Bs[n * 8 + gq][c0]);
                b[1] = *reinterpret_cast<const uint32_t*>(&Bs[n * 8 + gq][c0 + 8]);
                mma16816(acc[0][n], a[0], b);
                mma16816(acc[1][n], a[1], b);
            }
        }
        __syncthreads();
    }
    // epilogue: rows warp*32 + m*16 + gq (+8), columns n*8 + tq*2 (+1)
#pragma unroll
    for (int m = 0; m < 2; ++m)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const long long r = (long long)blockIdx.x * ROWS + warp * 32 + m * 16 + gq + h * 8;
            if (r >= nrows) continue;
#pragma unroll
            for (int n = 0; n < NT; ++n) {
                const int c = n * 8 + tq * 2;
                float v0 = acc[m][n][2 * h], v1 = acc[m][n][2 * h + 1];
                if (bias) {
                    v0 += bias[c];
                    v1 += bias[c + 1];
                }
                if (relu) {
                    v0 = fmaxf(v0, 0.f);
                    v1 = fmaxf(v1, 0.f);
                }
                if (mask) {
                    const __nv_bfloat162 mk = *reinterpret_cast<const __nv_bfloat162*>(mask + r * CO + c);
                    if (!(__bfloat162float(mk.x) > 0.f)) v0 = 0.f;
                    if (!(__bfloat162float(mk.y) > 0.f)) v1 = 0.f;
                }
                if (Yf) {
                    Yf[r * CO + c] = v0;
                    Yf[r * CO + c + 1] = v1;
                } else {
                    *reinterpret_cast<__nv_bfloat162*>(Yh + r * CO + c) = __floats2bfloat162_rn(v0, v1);
                }
            }
        }
}

// ------------------------------------------------------------ weight gradient
// partial[chunk][k][ci][co] = sum over the chunk's rows of H[nbr(row,k)][ci] dZ[row][co]
constexpr int WG_ROWS = 64;      // rows per smem tile
constexpr int WG_CHUNK = 2048;   // rows per block

template <int CI, int CO>
__global__ void __launch_bounds__(128) k_wgrad(Geo g, const __nv_bfloat16* __restrict__ H,
                                               const __nv_bfloat16* __restrict__ dZ, float* __restrict__ partial) {
    constexpr int MT = CI / 16, NT = CO / 8;
    __shared__ __align__(16) __nv_bfloat16 Hs[WG_ROWS][CI + PADH];
    __shared__ __align__(16) __nv_bfloat16 Zs[WG_ROWS][CO + PADH];
    __shared__ float red[4][CI * CO];
    const int k = blockIdx.y, chunk = blockIdx.x;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, gq = lane >> 2, tq = lane & 3;
    const long long nrows = (long long)g.nb * g.V;
    float acc[MT][NT][4];
#pragma unroll
    for (int m = 0; m < MT; ++m)
#pragma unroll
        for (int n = 0; n < NT; ++n)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[m][n][q] = 0.f;
    const long long r_begin = (long long)chunk * WG_CHUNK;
    for (long long t0 = r_begin; t0 < r_begin + WG_CHUNK && t0 < nrows; t0 += WG_ROWS) {
        // rows t0 .. t0+63: threads 0..63 gather H rows, 64..127 copy dZ rows
        if (tid < WG_ROWS) {
            const long long row = t0 + tid;
            uint4* dst = reinterpret_cast<uint4*>(&Hs[tid][0]);
            int s = -1, b = 0;
            if (row < nrows) {
                b = (int)(row / g.V);
                int x[4];
                site_coords(g, (int)(row - (long long)b * g.V), x);
                s = nbr(g, x, k);
            }
            if (s >= 0) {
                const uint4* src = reinterpret_cast<const uint4*>(H + ((long long)b * g.V + s) * CI);
#pragma unroll
                for (int q = 0; q < CI / 8; ++q) dst[q] = __ldg(src + q);
            } else {
#pragma unroll
                for (int q = 0; q < CI / 8; ++q) dst[q] = make_uint4(0, 0, 0, 0);
            }
        } else {
            const int rr = tid - WG_ROWS;
            const long long row = t0 + rr;
            __nv_bfloat16* dst = &Zs[rr][0];
            if (row < nrows) {
                const __nv_bfloat16* src = dZ + row * CO;
#pragma unroll
                for (int q = 0; q < CO; ++q) dst[q] = src[q];
            } else {
#pragma unroll
                for (int q = 0; q < CO; ++q) dst[q] = __float2bfloat16(0.f);
            }
        }
        __syncthreads();
        // warp w reduces over rows w*16 .. w*16+15 of the tile (one k16 step)
        const int rb = warp * 16;
#pragma unroll
        for (int m = 0; m < MT; ++m) {
            // A[mi = ci][kk = row]: a0a1 = (ci = gq, rows tq*2, tq*2+1) ...
            uint32_t a[4];
            const int ci = m * 16 + gq;
            a[0] = pack2(Hs[rb + tq * 2][ci], Hs[rb + tq * 2 + 1][ci]);
            a[1] = pack2(Hs[rb + tq * 2][ci + 8], Hs[rb + tq * 2 + 1][ci + 8]);
            a[2] = pack2(Hs[rb + tq * 2 + 8][ci], Hs[rb + tq * 2 + 9][ci]);
            a[3] = pack2(Hs[rb + tq * 2 + 8][ci + 8], Hs[rb + tq * 2 + 9][ci + 8]);
#pragma unroll
            for (int n = 0; n < NT; ++n) {
                uint32_t b[2];
                const int co = n * 8 + gq;
                b[0] = pack2(Zs[rb + tq * 2][co], Zs[rb + tq * 2 + 1][co]);
                b[1] = pack2(Zs[rb + tq * 2 + 8][co], Zs[rb + tq * 2 + 9][co]);
                mma16816(acc[m][n], a, b);
            }
        }
        __syncthreads();
    }
    // fixed-order reduction over the 4 warps
#pragma unroll
    for (int m = 0; m < MT; ++m)
#pragma unroll
        for (int n = 0; n < NT; ++n)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int ci = m * 16 + gq + h * 8, co = n * 8 + tq * 2;
                red[warp][ci * CO + co] = acc[m][n][2 * h];
                red[warp][ci * CO + co + 1] = acc[m][n][2 * h + 1];
            }
    __syncthreads();
    float* out = partial + ((long long)chunk * NOFF + k) * CI * CO;
    for (int i = tid; i < CI * CO; i += 128) out[i] = ((red[0][i] + red[1][i]) + red[2][i]) + red[3][i];
}

// sum the chunk partials in order: grad[k][ci][co]
__global__ void k_wgrad_reduce(int nchunk, int n, const float* __restrict__ partial, float* __restrict__ grad) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        float s = 0.f;
        for (int c = 0; c < nchunk; ++c) s += partial[(long long)c * n + i];
        grad[i] = s;
    }
}

// bias gradient: db[co] = sum_rows dZ[row][co] (block partials, fixed order)
__global__ void k_bgrad(long long nrows, int CO_, const __nv_bfloat16* __restrict__ dZ, float* __restrict__ partial) {
    __shared__ float sw[8][32];
    const int co = threadIdx.x & 31, grp = threadIdx.x >> 5;  // 256 threads: 8 groups x 32 channels
    float s = 0.f;
    if (co < CO_) {
        for (long long r = (long long)blockIdx.x * 8 + grp; r < nrows; r += (long long)gridDim.x * 8)
            s += __bfloat162float(dZ[r * CO_ + co]);
    }
    sw[grp][co] = s;
    __syncthreads();
    if (grp == 0 && co < CO_) {
        float t = 0.f;
        for (int q = 0; q < 8; ++q) t += sw[q][co];
        partial[blockIdx.x * 32 + co] = t;
    }
}

__global__ void k_bgrad_reduce(int nblk, int CO_, const float* __restrict__ partial, float* __restrict__ grad) {
    const int co = threadIdx.x;
    if (co >= CO_) return;
    float s = 0.f;
    for (int b = 0; b < nblk; ++b) s += partial[b * 32 + co];
    grad[co] = s;
}

// ------------------------------------------------------------ features / output
// The link features of every fermion site, once per network application:
// LF[s][2 mu], LF[s][2 mu + 1] = Re, Im tr U_mu(x) / 3 (BF16, 16 bytes a site).
__global__ void k_link_features(Geo g, const double2* __restrict__ canon, __nv_bfloat16* __restrict__ LF) {
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < g.V; s += (long long)gridDim.x * blockDim.x) {
        const long long gi = s + (long long)g.L * g.L * g.L;  // gauge site of the fermion site
        __align__(16) __nv_bfloat16 out[8];
#pragma unroll
        for (int mu = 0; mu < 4; ++mu) {
            const double2* U = canon + (gi * 4 + mu) * 9;
            const double2 a = __ldg(U), bb = __ldg(U + 4), c = __ldg(U + 8);
            out[2 * mu] = __float2bfloat16((float)((a.x + bb.x + c.x) / 3.0));
            out[2 * mu + 1] = __float2bfloat16((float)((a.y + bb.y + c.y) / 3.0));
        }
        *reinterpret_cast<uint4*>(LF + s * 8) = *reinterpret_cast<const uint4*>(out);
    }
}

// Input features of the network batch of 2 nrhs entries: entry b < nrhs is
// r_b / s_b, entry nrhs + b is -r_b / s_b (s_b the RMS scale of r_b, passed as
// inv_scale = 1 / s_b), residual channels on the even sites, the link
// features LF on every site.  g.nb = 2 nrhs.
template <typename P>
__global__ void k_features(LatDev gl, Geo g, CField<P> r, const double* __restrict__ inv_scale,
                           const __nv_bfloat16* __restrict__ LF, __nv_bfloat16* __restrict__ X) {
    const long long n = (long long)g.nb * g.V;
    const int nrhs = g.nb / 2;
    for (long long row = blockIdx.x * (long long)blockDim.x + threadIdx.x; row < n;
         row += (long long)gridDim.x * blockDim.x) {
        const int b2 = (int)(row / g.V), s = (int)(row - (long long)b2 * g.V);
        const int b = b2 % nrhs;
        int x[4];
        site_coords(g, s, x);
        const int par = (x[0] + x[1] + x[2] + x[3]) & 1;
        __align__(16) __nv_bfloat16 out[24];
        if (par == 0) {
            const int cb = s >> 1;
            const double sc = (b2 < nrhs ? 1.0 : -1.0) * inv_scale[b];
            cpx<typename P::real> p[4][3];
            load_spinor<P, typename P::real>(r, vbase<P>(gl, b), gl.Vpad, cb, 0, p);
#pragma unroll
            for (int c = 0; c < 12; ++c) {
                out[2 * c] = __float2bfloat16((float)((double)p[c / 3][c % 3].re * sc));
                out[2 * c + 1] = __float2bfloat16((float)((double)p[c / 3][c % 3].im * sc));
            }
        } else {
#pragma unroll
            for (int c = 0; c < 24; ++c) out[c] = __float2bfloat16(0.f);
        }
        uint4* dst = reinterpret_cast<uint4*>(X + row * CIN0);
        const uint4* srcv = reinterpret_cast<const uint4*>(out);
#pragma unroll
        for (int q = 0; q < 3; ++q) dst[q] = srcv[q];
        dst[3] = __ldg(reinterpret_cast<const uint4*>(LF + (long long)s * 8));
    }
}

// z = r + s_b (out_b - out_{nrhs+b}) / 2 on the even sites (out FP32
// [2 nrhs][V][24]); g.nb = 2 nrhs; r and z FP64 or FP32 blocks
template <typename P>
__global__ void k_output(LatDev gl, Geo g, const float* __restrict__ Y, const double* __restrict__ scale,
                         CField<P> r, Field<P> z) {
    using R = typename P::real;
    const int nrhs = g.nb / 2;
    const long long n = (long long)nrhs * gl.Vh;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(i / gl.Vh), cb = (int)(i - (long long)b * gl.Vh);
        const SiteX sx = decode_site(gl, cb, 0);
        const float* yp = Y + ((long long)b * g.V + sx.lex) * COUT;
        const float* ym = Y + ((long long)(nrhs + b) * g.V + sx.lex) * COUT;
        const double sc = 0.5 * scale[b];
        cpx<R> p[4][3];
        load_spinor<P, R>(r, vbase<P>(gl, b), gl.Vpad, cb, 0, p);
#pragma unroll
        for (int c = 0; c < 12; ++c) {
            cpx<R>& q = p[c / 3][c % 3];
            q = cpx<R>{(R)((double)q.re + sc * ((double)yp[2 * c] - (double)ym[2 * c])),
                       (R)((double)q.im + sc * ((double)yp[2 * c + 1] - (double)ym[2 * c + 1]))};
        }
        store_spinor<P, R>(z, vbase<P>(gl, b), gl.Vpad, cb, 0, p);
    }
}

// loss = (1/nrhs) sum_b |rh_b + (out_b - out_{nrhs+b})/2 - t_b|^2 / |t_b|^2 over
// the even sites, rh_b = r_b / s_b, t_b = e_b / s_b; dZ = d loss / d out
// (BF16, zero on odd sites: +d/2 for entry b, -d/2 for entry nrhs + b);
// per-block partial sums of the two norms per entry.  g.nb = 2 nrhs.
__global__ void k_loss(LatDev gl, Geo g, const float* __restrict__ Y, CField<P64> rin, CField<P64> e,
                       const double* __restrict__ inv_scale, const double* __restrict__ tnorm2,
                       __nv_bfloat16* __restrict__ dZ, double* __restrict__ partial) {
    __shared__ double s1[256], s2[256];
    const int nrhs = g.nb / 2;
    const int b = blockIdx.y;
    double a1 = 0.0, a2 = 0.0;
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < g.V; s += (long long)gridDim.x * blockDim.x) {
        const long long rowp = (long long)b * g.V + s, rowm = (long long)(nrhs + b) * g.V + s;
        int x[4];
        site_coords(g, (int)s, x);
        const int par = (x[0] + x[1] + x[2] + x[3]) & 1;
        __nv_bfloat16* dp = dZ + rowp * COUT;
        __nv_bfloat16* dm = dZ + rowm * COUT;
        if (par) {
#pragma unroll
            for (int c = 0; c < COUT; ++c) dp[c] = dm[c] = __float2bfloat16(0.f);
            continue;
        }
        const int cb = (int)(s >> 1);
        const long long base = (gl.soff + (long long)b * gl.Vpad) * 12;
        const double sc = inv_scale[b];
        const double w = 2.0 / (nrhs * tnorm2[b]);
#pragma unroll
        for (int c = 0; c < 12; ++c) {
            const double2 t = __ldg(e.v + base + (long long)c * gl.Vpad + cb);
            const double2 rv = __ldg(rin.v + base + (long long)c * gl.Vpad + cb);
            const double tr = t.x * sc, ti = t.y * sc;
            const double orr = 0.5 * ((double)Y[rowp * COUT + 2 * c] - (double)Y[rowm * COUT + 2 * c]);
            const double oi = 0.5 * ((double)Y[rowp * COUT + 2 * c + 1] - (double)Y[rowm * COUT + 2 * c + 1]);
            const double dr = orr + rv.x * sc - tr, di = oi + rv.y * sc - ti;
            a1 += dr * dr + di * di;
            a2 += tr * tr + ti * ti;
            dp[2 * c] = __float2bfloat16((float)(0.5 * w * dr));
            dp[2 * c + 1] = __float2bfloat16((float)(0.5 * w * di));
            dm[2 * c] = __float2bfloat16((float)(-0.5 * w * dr));
            dm[2 * c + 1] = __float2bfloat16((float)(-0.5 * w * di));
        }
    }
    s1[threadIdx.x] = a1;
    s2[threadIdx.x] = a2;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            s1[threadIdx.x] += s1[threadIdx.x + o];
            s2[threadIdx.x] += s2[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        partial[(b * gridDim.x + blockIdx.x) * 2] = s1[0];
        partial[(b * gridDim.x + blockIdx.x) * 2 + 1] = s2[0];
    }
}

// dZ of the output from an FP64 even-site field G (d loss / d M(r) = G):
// dZ_b = coef_b G, dZ_{nrhs+b} = -coef_b G on the even sites, zero elsewhere
// (coef_b = s_b / 2 from M = r + s (out_+ - out_-) / 2).  g.nb = 2 nrhs.
__global__ void k_dz_from_field(LatDev gl, Geo g, CField<P64> G, const double* __restrict__ coef,
                                __nv_bfloat16* __restrict__ dZ) {
    const int nrhs = g.nb / 2;
    const long long n = (long long)nrhs * g.V;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(i / g.V), s = (int)(i - (long long)b * g.V);
        int x[4];
        site_coords(g, s, x);
        const int par = (x[0] + x[1] + x[2] + x[3]) & 1;
        __nv_bfloat16* dp = dZ + ((long long)b * g.V + s) * COUT;
        __nv_bfloat16* dm = dZ + ((long long)(nrhs + b) * g.V + s) * COUT;
        if (par) {
#pragma unroll
            for (int c = 0; c < COUT; ++c) dp[c] = dm[c] = __float2bfloat16(0.f);
            continue;
        }
        const int cb = s >> 1;
        const long long base = (gl.soff + (long long)b * gl.Vpad) * 12;
        const double cf_ = coef[b];
#pragma unroll
        for (int c = 0; c < 12; ++c) {
            const double2 v = __ldg(G.v + base + (long long)c * gl.Vpad + cb);
            dp[2 * c] = __float2bfloat16((float)(cf_ * v.x));
            dp[2 * c + 1] = __float2bfloat16((float)(cf_ * v.y));
            dm[2 * c] = __float2bfloat16((float)(-cf_ * v.x));
            dm[2 * c + 1] = __float2bfloat16((float)(-cf_ * v.y));
        }
    }
}

// Adam step on the FP32 master parameters; refreshes the BF16 copies
__global__ void k_adam(int n, float* __restrict__ p, const float* __restrict__ grad, float* __restrict__ m1,
                       float* __restrict__ m2, float lr, float b1, float b2, float eps, float c1, float c2) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float gr = grad[i];
        const float a = b1 * m1[i] + (1.f - b1) * gr;
        const float v = b2 * m2[i] + (1.f - b2) * gr * gr;
        m1[i] = a;
        m2[i] = v;
        p[i] -= lr * (a / c1) / (sqrtf(v / c2) + eps);
    }
}

// BF16 copies of one layer: Wf[k][co][ci] = W[k][ci][co], Wb[k][ci][co] = W[80-k][ci][co]
__global__ void k_wcopy(int ci, int co, const float* __restrict__ W, __nv_bfloat16* __restrict__ Wf,
                        __nv_bfloat16* __restrict__ Wb) {
    const int n = NOFF * ci * co;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int k = i / (ci * co), rem = i % (ci * co), a = rem / co, c = rem % co;
        const __nv_bfloat16 v = __float2bfloat16(W[i]);
        Wf[((long long)k * co + c) * ci + a] = v;
        Wb[((long long)(NOFF - 1 - k) * ci + a) * co + c] = v;
    }
}

// ------------------------------------------------------------ host side
struct Buf {
    void* p = nullptr;
    size_t n = 0;
    ~Buf() {
        if (p) cudaFree(p);
    }
    void ensure(size_t bytes) {
        if (bytes <= n) return;
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
        if (cudaMalloc(&p, bytes) != cudaSuccess) {
            cudaGetLastError();
            throw std::bad_alloc();
        }
        n = bytes;
    }
    template <class T>
    T* as() const { return reinterpret_cast<T*>(p); }
};

struct LayerShape {
    int ci, co;
    size_t woff, boff;  // offsets into the flat parameter vector
};

void backward_layers(sf_cnn* c, const Geo& g, __nv_bfloat16* dz, __nv_bfloat16* dz2, cudaStream_t st);

}  // namespace sfcnn

using namespace sfcnn;

struct sf_cnn {
    int hidden = 32, device = 0;
    int conv_impl = 0;    // 0: tcgen05 convolutions where the shape fits, 1: mma.sync everywhere
    int sm_count = 152;
    cudaStream_t stream = nullptr;
    std::vector<LayerShape> layers;
    size_t nparams = 0;
    Buf params, grad, m1, m2, wf, wb;
    long long step = 0;
    // activations for a given geometry
    Buf act[4], out, dz[2], partial, wpart, lpart, lfeat;
    Geo geo{};
    size_t wf_off[4] = {0, 0, 0, 0};
};

namespace sfcnn {

cudaError_t refresh_bf16(sf_cnn* c, cudaStream_t st) {
    for (size_t l = 0; l < c->layers.size(); ++l) {
        const LayerShape& s = c->layers[l];
        k_wcopy<<<64, 256, 0, st>>>(s.ci, s.co, c->params.as<float>() + s.woff,
                                            c->wf.as<__nv_bfloat16>() + c->wf_off[l],
                                            c->wb.as<__nv_bfloat16>() + c->wf_off[l]);
    }
    return cudaGetLastError();
}

template <int CI, int CO>
void conv_launch(const Geo& g, const __nv_bfloat16* X, const __nv_bfloat16* B, const float* bias, int relu,
                 const __nv_bfloat16* mask, __nv_bfloat16* Yh, float* Yf, cudaStream_t st) {
    const long long rows = (long long)g.nb * g.V;
    const int blocks = (int)((rows + ROWS - 1) / ROWS);
    k_conv<CI, CO><<<blocks, 128, 0, st>>>(g, X, B, bias, relu, mask, Yh, Yf);
}

void conv_any(const sf_cnn* c, int ci, int co, const Geo& g, const __nv_bfloat16* X, const __nv_bfloat16* B,
              const float* bias, int relu, const __nv_bfloat16* mask, __nv_bfloat16* Yh, float* Yf, cudaStream_t st) {
    if (c->conv_impl == 0 && conv_tc_supported(ci, co) &&
        conv_tc(ConvTcGeo{g.L, g.T, g.V, g.nb}, ci, co, X, B, bias, relu, mask, Yh, Yf, c->sm_count, st) ==
            cudaSuccess)
        return;
    cudaGetLastError();   // a geometry the tensor-core kernel does not take: mma.sync
#define SFC(A, B_) if (ci == A && co == B_) { conv_launch<A, B_>(g, X, B, bias, relu, mask, Yh, Yf, st); return; }
    SFC(32, 32) SFC(32, 16) SFC(16, 16) SFC(16, 24) SFC(32, 24) SFC(24, 16) SFC(24, 32) SFC(16, 32)
#undef SFC
}

void wgrad_any(int ci, int co, const Geo& g, const __nv_bfloat16* H, const __nv_bfloat16* dZ, float* partial,
               int nchunk, cudaStream_t st) {
    const dim3 grid(nchunk, NOFF);
#define SFW(A, B_) if (ci == A && co == B_) { k_wgrad<A, B_><<<grid, 128, 0, st>>>(g, H, dZ, partial); return; }
    SFW(32, 32) SFW(32, 16) SFW(16, 16) SFW(16, 24) SFW(32, 24)
#undef SFW
}

}  // namespace sfcnn

namespace sfcnn {

void ensure_geo(sf_cnn* c, const Geo& g) {
    const long long rows = (long long)g.nb * g.V;
    const int H = c->hidden;
    c->act[0].ensure((size_t)rows * CIN0 * 2);
    c->lfeat.ensure((size_t)g.V * 8 * 2);
    for (int l = 1; l < 4; ++l) c->act[l].ensure((size_t)rows * H * 2);
    c->out.ensure((size_t)rows * COUT * 4);
    c->dz[0].ensure((size_t)rows * 32 * 2);
    c->dz[1].ensure((size_t)rows * 32 * 2);
    const int nchunk = (int)((rows + WG_CHUNK - 1) / WG_CHUNK);
    c->wpart.ensure((size_t)nchunk * NOFF * 32 * 32 * 4);
    c->lpart.ensure((size_t)g.nb * 1024 * 2 * 8 + 4096 * 4);
    c->partial.ensure((size_t)4096 * 32 * 4);
    c->geo = g;
}

// forward through the network; returns nothing, activations in c->act, output in c->out
void forward(sf_cnn* c, const Geo& g, cudaStream_t st) {
    const __nv_bfloat16* wf = c->wf.as<__nv_bfloat16>();
    const float* P = c->params.as<float>();
    for (int l = 0; l < 4; ++l) {
        const LayerShape& s = c->layers[l];
        const bool last = (l == 3);
        conv_any(c, s.ci, s.co, g, c->act[l].as<__nv_bfloat16>(), wf + c->wf_off[l], P + s.boff, last ? 0 : 1, nullptr,
                 last ? nullptr : c->act[l + 1].as<__nv_bfloat16>(), last ? c->out.as<float>() : nullptr, st);
    }
}

// parameter gradients from dZ of the output (dz, overwritten) and the
// activations kept by the last forward pass
void backward_layers(sf_cnn* c, const Geo& g, __nv_bfloat16* dz, __nv_bfloat16* dz2, cudaStream_t st) {
    const long long rows = (long long)g.nb * g.V;
    const int nchunk = (int)((rows + WG_CHUNK - 1) / WG_CHUNK);
    float* G = c->grad.as<float>();
    const __nv_bfloat16* wb = c->wb.as<__nv_bfloat16>();
    for (int l = 3; l >= 0; --l) {
        const LayerShape& s = c->layers[l];
        // weight and bias gradients of layer l from its input act[l] and dZ_l
        wgrad_any(s.ci, s.co, g, c->act[l].as<__nv_bfloat16>(), dz, c->wpart.as<float>(), nchunk, st);
        const int nw = NOFF * s.ci * s.co;
        k_wgrad_reduce<<<(nw + 255) / 256, 256, 0, st>>>(nchunk, nw, c->wpart.as<float>(), G + s.woff);
        const int bblk = (int)std::min<long long>((rows + 7) / 8, 4096);
        k_bgrad<<<bblk, 256, 0, st>>>(rows, s.co, dz, c->partial.as<float>());
        k_bgrad_reduce<<<1, 32, 0, st>>>(bblk, s.co, c->partial.as<float>(), G + s.boff);
        if (l > 0) {
            // dZ_{l-1} = (W_l^T conv dZ_l) * (act[l] > 0)
            conv_any(c, s.co, s.ci, g, dz, wb + c->wf_off[l], nullptr, 0, c->act[l].as<__nv_bfloat16>(), dz2, nullptr,
                     st);
            std::swap(dz, dz2);
        }
    }
}

}  // namespace sfcnn

extern "C" {

long long sf_cnn_num_params(int hidden) {
    if (hidden != 16 && hidden != 32) return -1;
    const int w[5] = {CIN0, hidden, hidden, hidden, COUT};
    long long n = 0;
    for (int l = 0; l < 4; ++l) n += (long long)NOFF * w[l] * w[l + 1] + w[l + 1];
    return n;
}

sf_status sf_cnn_create(sf_cnn** out, int hidden, const float* params, int device, void* stream) {
    if (!out) return SF_EINVAL;
    *out = nullptr;
    if (hidden != 16 && hidden != 32) {
        sf::set_last_error("hidden width must be 16 or 32");
        return SF_EINVAL;
    }
    if (!params) {
        sf::set_last_error("params is NULL");
        return SF_EINVAL;
    }
    try {
        if (cudaSetDevice(device) != cudaSuccess) {
            cudaGetLastError();
            sf::set_last_error("bad device");
            return SF_EINVAL;
        }
        auto* c = new sf_cnn();
        c->hidden = hidden;
        c->device = device;
        if (cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
            cudaGetLastError();
            c->sm_count = 152;
        }
        c->stream = reinterpret_cast<cudaStream_t>(stream);
        const int w[5] = {CIN0, hidden, hidden, hidden, COUT};
        size_t off = 0, woff = 0;
        for (int l = 0; l < 4; ++l) {
            LayerShape s{w[l], w[l + 1], off, off + (size_t)NOFF * w[l] * w[l + 1]};
            c->layers.push_back(s);
            c->wf_off[l] = woff;
            woff += (size_t)NOFF * w[l] * w[l + 1];
            off = s.boff + w[l + 1];
        }
        c->nparams = off;
        c->params.ensure(off * 4);
        c->grad.ensure(off * 4);
        c->m1.ensure(off * 4);
        c->m2.ensure(off * 4);
        c->wf.ensure(woff * 2);
        c->wb.ensure(woff * 2);
        cudaMemcpyAsync(c->params.p, params, off * 4, cudaMemcpyDefault, c->stream);
        cudaMemsetAsync(c->m1.p, 0, off * 4, c->stream);
        cudaMemsetAsync(c->m2.p, 0, off * 4, c->stream);
        refresh_bf16(c, c->stream);
        cudaError_t e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) {
            delete c;
            sf::set_last_error(std::string("cnn create: ") + cudaGetErrorString(e));
            return SF_ECUDA;
        }
        *out = c;
        return SF_OK;
    } catch (const std::bad_alloc&) {
        sf::set_last_error("allocation failed");
        return SF_ENOMEM;
    }
}

sf_status sf_cnn_get_params(sf_cnn* c, float* params) {
    if (!c || !params) return SF_EINVAL;
    cudaError_t e = cudaMemcpyAsync(params, c->params.p, c->nparams * 4, cudaMemcpyDefault, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        sf::set_last_error(cudaGetErrorString(e));
        return SF_ECUDA;
    }
    return SF_OK;
}

sf_status sf_cnn_set_conv_impl(sf_cnn* c, int impl) {
    if (!c || (impl != 0 && impl != 1)) {
        sf::set_last_error("sf_cnn_set_conv_impl: NULL network or impl not 0 / 1");
        return SF_EINVAL;
    }
    c->conv_impl = impl;
    return SF_OK;
}

void sf_cnn_destroy(sf_cnn* c) {
    if (!c) return;
    cudaSetDevice(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    delete c;
}

}  // extern "C"

namespace sf {

// M(r) for an FP64 field f of the lattice workspace (nrhs fields), into z.
// norms_dev: |r_b| per field (device).  Used by FGCR and sf_cnn_forward.
template <typename P>
static cudaError_t cnn_apply_any(sf_cnn* c, const CnnLatticeView& v, FieldPtr r, const double* norms,
                                 const double* inv_norms, FieldPtr z) {
    using namespace sfcnn;
    Geo g{v.desc.L, v.desc.T, 2 * v.desc.Vh, 2 * v.nrhs};  // entries +r/s and -r/s
    try {
        ensure_geo(c, g);
    } catch (const std::bad_alloc&) {
        return cudaErrorMemoryAllocation;
    }
    const long long rows = (long long)g.nb * g.V;
    int blocks = (int)std::min<long long>((g.V + 255) / 256, 4 * c->sm_count);
    k_link_features<<<blocks, 256, 0, v.stream>>>(g, reinterpret_cast<const double2*>(v.canon),
                                                  c->lfeat.as<__nv_bfloat16>());
    blocks = (int)std::min<long long>((rows + 255) / 256, 8 * c->sm_count);
    k_features<P><<<blocks, 256, 0, v.stream>>>(v.desc, g, cf<P>(r), inv_norms, c->lfeat.as<__nv_bfloat16>(),
                                                 c->act[0].as<__nv_bfloat16>());
    forward(c, g, v.stream);
    blocks = (int)std::min<long long>(((long long)v.nrhs * v.desc.Vh + 255) / 256, 8 * c->sm_count);
    k_output<P><<<blocks, 256, 0, v.stream>>>(v.desc, g, c->out.as<float>(), norms, cf<P>(r), wf<P>(z));
    return cudaGetLastError();
}

cudaError_t cnn_apply_field(sf_cnn* c, const CnnLatticeView& v, FieldPtr r, const double* norms, const double* inv_norms,
                            FieldPtr z) {
    return cnn_apply_any<P64>(c, v, r, norms, inv_norms, z);
}

cudaError_t cnn_apply_field32(sf_cnn* c, const CnnLatticeView& v, FieldPtr r, const double* norms,
                              const double* inv_norms, FieldPtr z) {
    return cnn_apply_any<P32>(c, v, r, norms, inv_norms, z);
}

// forward + loss + backward; grads into c->grad; loss value into *loss (host)
cudaError_t cnn_loss_grad(sf_cnn* c, const CnnLatticeView& v, FieldPtr r, FieldPtr e, const double* inv_norms,
                          const double* tnorm2, double* loss_host) {
    using namespace sfcnn;
    Geo g{v.desc.L, v.desc.T, 2 * v.desc.Vh, 2 * v.nrhs};  // entries +r/s and -r/s
    try {
        ensure_geo(c, g);
    } catch (const std::bad_alloc&) {
        return cudaErrorMemoryAllocation;
    }
    cudaStream_t st = v.stream;
    const long long rows = (long long)g.nb * g.V;
    int blocks = (int)std::min<long long>((g.V + 255) / 256, 4 * c->sm_count);
    k_link_features<<<blocks, 256, 0, st>>>(g, reinterpret_cast<const double2*>(v.canon), c->lfeat.as<__nv_bfloat16>());
    blocks = (int)std::min<long long>((rows + 255) / 256, 8 * c->sm_count);
    k_features<P64><<<blocks, 256, 0, st>>>(v.desc, g, cf<P64>(r), inv_norms, c->lfeat.as<__nv_bfloat16>(),
                                        c->act[0].as<__nv_bfloat16>());
    forward(c, g, st);
    const int lblk = (int)std::min<long long>((g.V + 255) / 256, 1024);
    __nv_bfloat16* dz = c->dz[0].as<__nv_bfloat16>();
    __nv_bfloat16* dz2 = c->dz[1].as<__nv_bfloat16>();
    double* lp = c->lpart.as<double>();
    k_loss<<<dim3(lblk, v.nrhs), 256, 0, st>>>(v.desc, g, c->out.as<float>(), cf<P64>(r), cf<P64>(e), inv_norms, tnorm2,
                                              dz, lp);
    sfcnn::backward_layers(c, g, dz, dz2, st);
    if (loss_host) {
        std::vector<double> h((size_t)lblk * v.nrhs * 2);
        cudaMemcpyAsync(h.data(), lp, h.size() * 8, cudaMemcpyDeviceToHost, st);
        cudaError_t err = cudaStreamSynchronize(st);
        if (err != cudaSuccess) return err;
        double tot = 0.0;
        for (int b = 0; b < v.nrhs; ++b) {
            double a1 = 0.0, a2 = 0.0;
            for (int k = 0; k < lblk; ++k) {
                a1 += h[((size_t)b * lblk + k) * 2];
                a2 += h[((size_t)b * lblk + k) * 2 + 1];
            }
            tot += (a2 > 0 ? a1 / a2 : 0.0);
        }
        *loss_host = tot / v.nrhs;
    }
    return cudaGetLastError();
}

cudaError_t cnn_backward_field(sf_cnn* c, const CnnLatticeView& v, FieldPtr G, const double* coef) {
    using namespace sfcnn;
    Geo g{v.desc.L, v.desc.T, 2 * v.desc.Vh, 2 * v.nrhs};
    const long long rows = (long long)v.nrhs * g.V;
    const int blocks = (int)std::min<long long>((rows + 255) / 256, 4 * 152);
    __nv_bfloat16* dz = c->dz[0].as<__nv_bfloat16>();
    __nv_bfloat16* dz2 = c->dz[1].as<__nv_bfloat16>();
    k_dz_from_field<<<blocks, 256, 0, v.stream>>>(v.desc, g, cf<P64>(G), coef, dz);
    backward_layers(c, g, dz, dz2, v.stream);
    return cudaGetLastError();
}

cudaError_t cnn_adam(sf_cnn* c, float lr, cudaStream_t st) {
    using namespace sfcnn;
    c->step += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - powf(b1, (float)c->step), c2 = 1.f - powf(b2, (float)c->step);
    k_adam<<<256, 256, 0, st>>>((int)c->nparams, c->params.as<float>(), c->grad.as<float>(), c->m1.as<float>(),
                                        c->m2.as<float>(), lr, b1, b2, 1e-8f, c1, c2);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return refresh_bf16(c, st);
}

cudaError_t cnn_check(sf_cnn*) {
    return sfcnn::conv_tc_error(true) ? cudaErrorLaunchTimeout : cudaSuccess;
}

cudaError_t cnn_copy_grad(sf_cnn* c, float* out, cudaStream_t st) {
    cudaError_t e = cudaMemcpyAsync(out, c->grad.p, c->nparams * 4, cudaMemcpyDefault, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return e;
}

}  // namespace sf
