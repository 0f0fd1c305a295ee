// fgcr32.cu -- the FP32 vector kernels of the flexible GCR that runs as the
// inner solver of the FP64 defect correction (the learned preconditioner's
// mixed-precision form): complex dot products per (lattice, rhs) with
// float-float accumulation and fixed-order lattice sums, multi-axpy,
// gamma_5, and the conversions between the FP64 outer and FP32 inner fields.
// Launched with the FP64 BLAS tiling (TS = 32 sites, one rhs per thread row).
#include "krylov_impl.cuh"

namespace sf {

// partials of <a_i, b_i> (complex, sum conj(a) b) for every (lattice, rhs)
__global__ void __launch_bounds__(KB<P64, 1>::MAXT) k_dot32(const LatDev* __restrict__ lats, int nlat, int nrhs,
                                                          CField<P32> a, CField<P32> b, SolverCtx ctx) {
    pdl_enter();
    using A = AccOf<float>::T;
    const int l = find_lattice(lats, nlat, blockIdx.x);
    const LatDev g = lats[l];
    const int r0 = threadIdx.y;
    A red[1][2] = {{acc_zero<A>(), acc_zero<A>()}};
    if (r0 < nrhs) {
        for (int tile = tile_begin(g), te = tile_end(g); tile < te; ++tile) {
            const int cb = tile_cb(g, tile, threadIdx.x);
            if (cb < 0) continue;
            cpx<float> x[4][3], y[4][3];
            load_spinor<P32, float>(a, vbase<P32>(g, r0), g.Vpad, cb, 0, x);
            load_spinor<P32, float>(b, vbase<P32>(g, r0), g.Vpad, cb, 0, y);
            dotc_acc(x, y, red[0][0], red[0][1]);
        }
    }
    block_partials<1, 2>(red, nrhs, ctx.partials);
}

cudaError_t launch_dot32(const LaunchCfg& c, FieldPtr a, FieldPtr b, const SolverCtx* ctx, double2* out,
                         cudaStream_t st) {
    launch_pdl(k_dot32, dim3(c.nblocks), dim3(c.TS, c.nrhs), st, c.lats, c.nlat, c.nrhs, cf<P32>(a), cf<P32>(b), *ctx);
    launch_finish<2, AccOf<float>::T, FIN_DOT, float>(c, *ctx, reinterpret_cast<double*>(out), 0, st);
    return cudaGetLastError();
}

// y_i += sum_j c[j][i] x_j for nvec FP32 vectors x_j (coefficients per (lattice, rhs), device)
__global__ void __launch_bounds__(KB<P64, 1>::MAXT) k_multi_axpy32(const LatDev* __restrict__ lats, int nlat, int nrhs,
                                                                 int nvec, const float4* const* __restrict__ xs,
                                                                 const double2* __restrict__ c, float4* __restrict__ y) {
    pdl_enter();
    const int l = find_lattice(lats, nlat, blockIdx.x);
    const LatDev g = lats[l];
    const int r0 = threadIdx.y;
    if (r0 >= nrhs) return;
    for (int tile = tile_begin(g), te = tile_end(g); tile < te; ++tile) {
        const int cb = tile_cb(g, tile, threadIdx.x);
        if (cb < 0) continue;
        const long long base = vbase<P32>(g, r0) + cb;
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const long long idx = base + (long long)k * g.Vpad;
            float4 acc = y[idx];
            for (int j = 0; j < nvec; ++j) {
                const double2 cd = c[j * nlat * nrhs + l * nrhs + r0];
                const float cr = (float)cd.x, ci = (float)cd.y;
                const float4 xv = xs[j][idx];
                acc.x = fmaf(cr, xv.x, fmaf(-ci, xv.y, acc.x));
                acc.y = fmaf(cr, xv.y, fmaf(ci, xv.x, acc.y));
                acc.z = fmaf(cr, xv.z, fmaf(-ci, xv.w, acc.z));
                acc.w = fmaf(cr, xv.w, fmaf(ci, xv.z, acc.w));
            }
            y[idx] = acc;
        }
    }
}

cudaError_t launch_multi_axpy32(const LaunchCfg& c, int nvec, const float4* const* xs, const double2* coef, FieldPtr y,
                                cudaStream_t st) {
    launch_pdl(k_multi_axpy32, dim3(c.nblocks), dim3(c.TS, c.nrhs), st, c.lats, c.nlat, c.nrhs, nvec, xs, coef,
               reinterpret_cast<float4*>(y.v));
    return cudaGetLastError();
}

// out = gamma_5 in for an FP32 block: float4 planes 3..5 hold spin 2, 3
__global__ void k_gamma5_32(long long nplanes, int Vpad, const float4* __restrict__ in, float4* __restrict__ out) {
    pdl_enter();
    const long long n = nplanes * Vpad;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int k = (int)((i / Vpad) % 6);
        float4 v = in[i];
        if (k >= 3) v = make_float4(-v.x, -v.y, -v.z, -v.w);
        out[i] = v;
    }
}

cudaError_t launch_gamma5_32(long long nplanes, int Vpad, FieldPtr in, FieldPtr out, int sm_count, cudaStream_t st) {
    launch_pdl(k_gamma5_32, dim3(4 * sm_count), dim3(256), st, nplanes, Vpad, reinterpret_cast<const float4*>(in.v),
               reinterpret_cast<float4*>(out.v));
    return cudaGetLastError();
}

// r32 = scale[l nrhs + i] r64 (FP64 block -> FP32 block)
__global__ void __launch_bounds__(KB<P64, 1>::MAXT) k_to32(const LatDev* __restrict__ lats, int nlat, int nrhs,
                                                         CField<P64> in, const double* __restrict__ scale,
                                                         Field<P32> out) {
    pdl_enter();
    const int l = find_lattice(lats, nlat, blockIdx.x);
    const LatDev g = lats[l];
    const int r0 = threadIdx.y;
    if (r0 >= nrhs) return;
    const double sc = scale[l * nrhs + r0];
    for (int tile = tile_begin(g), te = tile_end(g); tile < te; ++tile) {
        const int cb = tile_cb(g, tile, threadIdx.x);
        if (cb < 0) continue;
        cpx<double> x[4][3];
        load_spinor<P64, double>(in, vbase<P64>(g, r0), g.Vpad, cb, 0, x);
        cpx<float> y[4][3];
#pragma unroll
        for (int s = 0; s < 4; ++s)
#pragma unroll
            for (int c = 0; c < 3; ++c) y[s][c] = cpx<float>{(float)(sc * x[s][c].re), (float)(sc * x[s][c].im)};
        store_spinor<P32, float>(out, vbase<P32>(g, r0), g.Vpad, cb, 0, y);
    }
}

cudaError_t launch_to32(const LaunchCfg& c, FieldPtr in, const double* scale, FieldPtr out, cudaStream_t st) {
    launch_pdl(k_to32, dim3(c.nblocks), dim3(c.TS, c.nrhs), st, c.lats, c.nlat, c.nrhs, cf<P64>(in), scale,
               wf<P32>(out));
    return cudaGetLastError();
}

// x64 += scale[l nrhs + i] e32
__global__ void __launch_bounds__(KB<P64, 1>::MAXT) k_add32to64(const LatDev* __restrict__ lats, int nlat, int nrhs,
                                                              CField<P32> e, const double* __restrict__ scale,
                                                              Field<P64> x) {
    pdl_enter();
    const int l = find_lattice(lats, nlat, blockIdx.x);
    const LatDev g = lats[l];
    const int r0 = threadIdx.y;
    if (r0 >= nrhs) return;
    const double sc = scale[l * nrhs + r0];
    if (sc == 0.0) return;
    for (int tile = tile_begin(g), te = tile_end(g); tile < te; ++tile) {
        const int cb = tile_cb(g, tile, threadIdx.x);
        if (cb < 0) continue;
        cpx<float> y[4][3];
        load_spinor<P32, float>(e, vbase<P32>(g, r0), g.Vpad, cb, 0, y);
        cpx<double> xv[4][3];
        load_spinor<P64, double>(CField<P64>{x.v, x.scale}, vbase<P64>(g, r0), g.Vpad, cb, 0, xv);
#pragma unroll
        for (int s = 0; s < 4; ++s)
#pragma unroll
            for (int c = 0; c < 3; ++c)
                xv[s][c] = cpx<double>{xv[s][c].re + sc * (double)y[s][c].re, xv[s][c].im + sc * (double)y[s][c].im};
        store_spinor<P64, double>(x, vbase<P64>(g, r0), g.Vpad, cb, 0, xv);
    }
}

cudaError_t launch_add32to64(const LaunchCfg& c, FieldPtr e, const double* scale, FieldPtr x, cudaStream_t st) {
    launch_pdl(k_add32to64, dim3(c.nblocks), dim3(c.TS, c.nrhs), st, c.lats, c.nlat, c.nrhs, cf<P32>(e), scale,
               wf<P64>(x));
    return cudaGetLastError();
}

}  // namespace sf

namespace sf {

// <a_j, b_i> for j < nvec (FP32 vectors a_j, one b) and every rhs i of one
// lattice: thread (site, rhs) loads b once per site and runs over the a_j;
// per-block partials [(rhs * 2 nvec + 2 j + re/im) * gridDim.x + block],
// float-float within a thread, then a fixed-order shuffle and warp sum.
constexpr int MDOT_MAX = 18;

__global__ void __launch_bounds__(KB<P64, 1>::MAXT) k_multidot32(const LatDev* __restrict__ lats, int nrhs, int nvec,
                                                               const float4* const* __restrict__ as, CField<P32> b,
                                                               double* __restrict__ partials) {
    pdl_enter();
    using A = AccOf<float>::T;
    __shared__ A sw[MAX_WARPS][2 * MDOT_MAX];
    const LatDev g = lats[0];
    const int r0 = threadIdx.y;
    A acc[2 * MDOT_MAX];
#pragma unroll
    for (int q = 0; q < 2 * MDOT_MAX; ++q) acc[q] = acc_zero<A>();
    if (r0 < nrhs) {
        for (int tile = tile_begin(g), te = tile_end(g); tile < te; ++tile) {
            const int cb = tile_cb(g, tile, threadIdx.x);
            if (cb < 0) continue;
            const long long base = vbase<P32>(g, r0) + cb;
            float4 bv[6];
#pragma unroll
            for (int k = 0; k < 6; ++k) bv[k] = __ldg(b.v + base + (long long)k * g.Vpad);
#pragma unroll
            for (int j = 0; j < MDOT_MAX; ++j) {
                if (j >= nvec) break;
                float sr = 0.f, si = 0.f;
#pragma unroll
                for (int k = 0; k < 6; ++k) {
                    const float4 av = __ldg(as[j] + base + (long long)k * g.Vpad);
                    sr = fmaf(av.x, bv[k].x, fmaf(av.y, bv[k].y, fmaf(av.z, bv[k].z, fmaf(av.w, bv[k].w, sr))));
                    si = fmaf(av.x, bv[k].y, fmaf(-av.y, bv[k].x, fmaf(av.z, bv[k].w, fmaf(-av.w, bv[k].z, si))));
                }
                acc[2 * j] = acc_add(acc[2 * j], A{sr, 0.f});
                acc[2 * j + 1] = acc_add(acc[2 * j + 1], A{si, 0.f});
            }
        }
    }
    const int lane = threadIdx.x & 31;
    const int wpr = blockDim.x >> 5;
    const int w = threadIdx.y * wpr + (threadIdx.x >> 5);
#pragma unroll
    for (int q = 0; q < 2 * MDOT_MAX; ++q) {
        if (q >= 2 * nvec) break;
        A v = acc[q];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v = acc_add(v, acc_shfl_down(v, off));
        if (lane == 0) sw[w][q] = v;
    }
    __syncthreads();
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    for (int t = tid; t < nrhs * 2 * nvec; t += blockDim.x * blockDim.y) {
        const int rhs = t / (2 * nvec), q = t % (2 * nvec);
        A s = acc_zero<A>();
        for (int k = 0; k < wpr; ++k) s = acc_add(s, sw[rhs * wpr + k][q]);
        partials[(long long)(rhs * 2 * nvec + q) * gridDim.x + blockIdx.x] = acc_to_double(s);
    }
}

// out[j * nrhs + i] = (re, im) of the lattice sums, one warp per (rhs, quantity)
// row in block order (the same result for every run)
__global__ void k_multidot_finish(int nrhs, int nvec, int nblocks, const double* __restrict__ partials,
                                  double2* __restrict__ out) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int row = w; row < nrhs * 2 * nvec; row += nw) {
        const double* src = partials + (long long)row * nblocks;
        double a = 0.0;
        for (int c = lane; c < nblocks; c += 32) a += src[c];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) a += __shfl_down_sync(0xffffffffu, a, off);
        if (lane == 0) {
            const int rhs = row / (2 * nvec), q = row % (2 * nvec), j = q / 2;
            double* o = reinterpret_cast<double*>(out + (size_t)j * nrhs + rhs);
            o[q & 1] = a;
        }
    }
}

cudaError_t launch_multidot32(const LaunchCfg& c, int nvec, const float4* const* as, FieldPtr b, double* partials,
                              double2* out, cudaStream_t st) {
    if (c.nlat != 1 || nvec < 1 || nvec > MDOT_MAX) return cudaErrorInvalidValue;
    launch_pdl(k_multidot32, dim3(c.nblocks), dim3(c.TS, c.nrhs), st, c.lats, c.nrhs, nvec, as, cf<P32>(b), partials);
    k_multidot_finish<<<1, 1024, 0, st>>>(c.nrhs, nvec, c.nblocks, partials, out);
    return cudaGetLastError();
}

}  // namespace sf
