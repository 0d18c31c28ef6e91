// mlp_internal.h -- kernels of the warm-start MLP (not public).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace fga {

enum GemmEpiKind : int {
    EPI_STORE = 0,        // C = acc (FP32)
    EPI_BIAS_RELU = 1,    // C = max(acc + bias, 0)
    EPI_BIAS = 2,         // C = acc + bias
    EPI_BIAS_DENORM = 3,  // C = (acc + bias) * scale + shift
    EPI_RELU_MASK = 4,    // C = acc where mask > 0, else 0
};

struct GemmEpi {
    const float *bias;
    const float *scale;
    const float *shift;
    const __nv_bfloat16 *mask;
    int ldm;
    float *outf;            // FP32 output (may be null)
    __nv_bfloat16 *outb;    // BF16 output (may be null)
    int ldc;
    int *err;               // device word: set to 1 when a wait of the tensor-core path timed out (may be null)
    float *ws;              // split-K workspace for products with few output tiles (may be null)
    long long ws_floats;    // its capacity
};

cudaError_t mlp_gemm(int layout, int epi, int M, int N, int K, const __nv_bfloat16 *A, int lda,
                     const __nv_bfloat16 *B, int ldb, const GemmEpi &ep, cudaStream_t s);
cudaError_t mlp_to_bf16_pad(const float *X, int rows, int cols, int ldo, __nv_bfloat16 *out, cudaStream_t s);
cudaError_t mlp_mse(const float *Y, const float *T, long long n, float scale, float *dYf, __nv_bfloat16 *dYb,
                    double *loss_part, int nparts, cudaStream_t s);
cudaError_t mlp_colsum_f32(const float *X, int rows, int cols, float *out, cudaStream_t s);
cudaError_t mlp_colsum_bf16(const __nv_bfloat16 *X, int rows, int cols, float *out, cudaStream_t s);
cudaError_t mlp_adam(float *w, float *m, float *v, const float *g, int rows, int cols, float lr, float b1, float b2,
                     float eps, float c1, float c2, __nv_bfloat16 *wb, __nv_bfloat16 *wt, cudaStream_t s);
cudaError_t mlp_copy_bf16(const float *w, int rows, int cols, __nv_bfloat16 *wb, __nv_bfloat16 *wt, cudaStream_t s);
cudaError_t mlp_col_stats(float *Y, long long rows, int cols, float *mean, float *stdv, cudaStream_t s);

}  // namespace fga
