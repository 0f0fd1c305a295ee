// conv_tc.h -- the tensor-core (tcgen05) 3^4-stencil convolution of the
// learned preconditioner (conv_tc.cu), called by cnn.cu.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace sfcnn {

struct ConvTcGeo {
    int L, T, V;   // fermion lattice, V = (T-1) L^3
    int nb;        // batch
};

// Shapes the kernel takes: ci in {8, 16, 24, 32} input channels (padded to 16
// or 32 per offset), co <= 32 output channels, as long as two input slices
// and the weights of all offsets fit in shared memory (not ci and co both
// above 16).  conv_tc also needs T <= 31 (the output slices of a unit share
// the 512 tensor-memory columns) and fewer than 2^31 / 32 rows; otherwise it
// returns cudaErrorInvalidValue without launching.
bool conv_tc_supported(int ci, int co);

// Y[row][co] = bias + sum_k sum_ci X[nbr(row, k)][ci] W[k][co][ci] over the
// nb x V rows (X BF16 [row][ci]; W BF16 [81][co][ci]); epilogue: ReLU
// (relu != 0), zero where mask[row][co] <= 0 (mask != NULL), BF16 (Yh) or FP32
// (Yf) output [row][co].  Asynchronous on st.
cudaError_t conv_tc(const ConvTcGeo& g, int ci, int co, const __nv_bfloat16* X, const __nv_bfloat16* W,
                    const float* bias, int relu, const __nv_bfloat16* mask, __nv_bfloat16* Yh, float* Yf,
                    int sm_count, cudaStream_t st);

// 1 if a convolution's wait timed out since the last reset (the output of
// that launch is incomplete); reset clears the flag.
int conv_tc_error(bool reset);

}  // namespace sfcnn
