// mlp.cu -- the learned warm start's network: a 3-layer ReLU MLP
// (in -> h1 -> h2 -> out) trained and evaluated with BF16 tensor-core GEMMs
// (mma.sync m16n8k16, FP32 accumulation), FP32 master weights and Adam.
//
// GEMM convention: C(m, n) = epilogue( sum_k A(m, k) B(n, k) ), where
// A(m, k) = A[m*lda + k] (K-major) or A[k*lda + m] (M-major), and likewise B.
// Tiles of 64 x 64 x 32 are staged through shared memory (transposed on the
// way in when the operand is not K-major), 4 warps each own 32 x 32.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "mlp_internal.h"

namespace fga {

namespace {

constexpr int BM = 64, BN = 64, BK = 32, PADK = 8;

__device__ __forceinline__ void mma_bf16(float *d, const uint32_t *a, const uint32_t *b) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// Loads a 64 x 32 tile of X(row, k) (row in [r0, r0+64), k in [k0, k0+32))
// into S[row][k].  KMAJ: X(row, k) = X[row*ld + k], else X[k*ld + row].
// Out-of-range elements read as zero.  ld and the contiguous extent must be
// multiples of 8 (16-byte vector loads).
template <bool KMAJ>
__device__ __forceinline__ void load_tile(__nv_bfloat16 (*S)[BK + PADK], const __nv_bfloat16 *X, int ld, int rows,
                                          int K, int r0, int k0) {
    const int t = threadIdx.x;
    if (KMAJ) {
        // 64 rows x 4 vectors of 8 along k
        for (int v = t; v < 64 * 4; v += 128) {
            const int row = v >> 2, kk = (v & 3) * 8;
            const int gr = r0 + row, gk = k0 + kk;
            uint4 val = make_uint4(0, 0, 0, 0);
            if (gr < rows && gk < K) val = *reinterpret_cast<const uint4 *>(X + (long long)gr * ld + gk);
            *reinterpret_cast<uint4 *>(&S[row][kk]) = val;
        }
    } else {
        // 32 k x 8 vectors of 8 along rows
        for (int v = t; v < 32 * 8; v += 128) {
            const int kk = v >> 3, row = (v & 7) * 8;
            const int gr = r0 + row, gk = k0 + kk;
            uint4 val = make_uint4(0, 0, 0, 0);
            if (gr < rows && gk < K) val = *reinterpret_cast<const uint4 *>(X + (long long)gk * ld + gr);
            const __nv_bfloat16 *e = reinterpret_cast<const __nv_bfloat16 *>(&val);
            #pragma unroll
            for (int j = 0; j < 8; ++j) S[row + j][kk] = e[j];
        }
    }
}

template <bool AK, bool BKM, int EPI>
__global__ void __launch_bounds__(128) k_gemm(int M, int N, int K, const __nv_bfloat16 *A, int lda,
                                              const __nv_bfloat16 *B, int ldb, GemmEpi ep) {
    __shared__ __align__(16) __nv_bfloat16 As[BM][BK + PADK];
    __shared__ __align__(16) __nv_bfloat16 Bs[BN][BK + PADK];
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
    const int gid = lane >> 2, tig = lane & 3;
    float acc[2][4][4];
    #pragma unroll
    for (int i = 0; i < 2; ++i)
        #pragma unroll
        for (int j = 0; j < 4; ++j)
            #pragma unroll
            for (int r = 0; r < 4; ++r) acc[i][j][r] = 0.f;
    for (int k0 = 0; k0 < K; k0 += BK) {
        load_tile<AK>(As, A, lda, M, K, m0, k0);
        load_tile<BKM>(Bs, B, ldb, N, K, n0, k0);
        __syncthreads();
        #pragma unroll
        for (int kk = 0; kk < BK; kk += 16) {
            uint32_t af[2][4], bf[4][2];
            #pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int r = wm + i * 16 + gid;
                const int c = kk + 2 * tig;
                af[i][0] = *reinterpret_cast<const uint32_t *>(&As[r][c]);
                af[i][1] = *reinterpret_cast<const uint32_t *>(&As[r + 8][c]);
                af[i][2] = *reinterpret_cast<const uint32_t *>(&As[r][c + 8]);
                af[i][3] = *reinterpret_cast<const uint32_t *>(&As[r + 8][c + 8]);
            }
            #pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int n = wn + j * 8 + gid;
                const int c = kk + 2 * tig;
                bf[j][0] = *reinterpret_cast<const uint32_t *>(&Bs[n][c]);
                bf[j][1] = *reinterpret_cast<const uint32_t *>(&Bs[n][c + 8]);
            }
            #pragma unroll
            for (int i = 0; i < 2; ++i)
                #pragma unroll
                for (int j = 0; j < 4; ++j) mma_bf16(acc[i][j], af[i], bf[j]);
        }
        __syncthreads();
    }
    // epilogue
    #pragma unroll
    for (int i = 0; i < 2; ++i) {
        #pragma unroll
        for (int j = 0; j < 4; ++j) {
            #pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int m = m0 + wm + i * 16 + gid + h * 8;
                const int n = n0 + wn + j * 8 + 2 * tig;
                if (m >= M) continue;
                #pragma unroll
                for (int q = 0; q < 2; ++q) {
                    const int nn = n + q;
                    if (nn >= N) continue;
                    float v = acc[i][j][h * 2 + q];
                    const long long o = (long long)m * ep.ldc + nn;
                    if (EPI == EPI_BIAS_RELU || EPI == EPI_BIAS || EPI == EPI_BIAS_DENORM) {
                        v += ep.bias[nn];
                        if (EPI == EPI_BIAS_RELU) v = fmaxf(v, 0.f);
                        if (EPI == EPI_BIAS_DENORM) v = v * ep.scale[nn] + ep.shift[nn];
                        if (ep.outf) ep.outf[o] = v;
                        if (ep.outb) ep.outb[o] = __float2bfloat16_rn(v);
                    } else if (EPI == EPI_RELU_MASK) {
                        const float h_act = __bfloat162float(ep.mask[(long long)m * ep.ldm + nn]);
                        v = h_act > 0.f ? v : 0.f;
                        if (ep.outb) ep.outb[o] = __float2bfloat16_rn(v);
                        if (ep.outf) ep.outf[o] = v;
                    } else {   // EPI_STORE
                        ep.outf[o] = v;
                    }
                }
            }
        }
    }
}

__global__ void k_to_bf16_pad(const float *X, int rows, int cols, int ldo, __nv_bfloat16 *out) {
    const long long n = (long long)rows * ldo;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(i / ldo), c = (int)(i % ldo);
        out[i] = __float2bfloat16_rn(c < cols ? X[(long long)r * cols + c] : 0.f);
    }
}

// MSE: loss = sum (Y - T)^2 / (rows * cols); dY = 2 (Y - T) / (rows * cols)
__global__ void k_mse(const float *Y, const float *T, long long n, float scale, float *dYf, __nv_bfloat16 *dYb,
                      double *loss_part) {
    double s = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float d = Y[i] - T[i];
        s += (double)d * (double)d;
        const float g = 2.f * d * scale;
        dYf[i] = g;
        dYb[i] = __float2bfloat16_rn(g);
    }
    #pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    __shared__ double w[32];
    if ((threadIdx.x & 31) == 0) w[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += w[i];
        loss_part[blockIdx.x] = t;
    }
}

// column sums of a rows x cols matrix (FP32 or BF16), fixed order per column
template <typename T>
__global__ void k_colsum(const T *X, int rows, int cols, float *out) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= cols) return;
    float s = 0.f;
    for (int r = 0; r < rows; ++r) s += (float)X[(long long)r * cols + c];
    out[c] = s;
}

// Adam on FP32 master weights w (n values), then the BF16 copies: wb in the
// stored [rows x cols] layout and wt = its transpose [cols x rows].
__global__ void k_adam(float *w, float *m, float *v, const float *g, int rows, int cols, float lr, float b1, float b2,
                       float eps, float c1, float c2, __nv_bfloat16 *wb, __nv_bfloat16 *wt) {
    const int n = rows * cols;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
        w[i] = wi;
        if (wb) {
            const __nv_bfloat16 h = __float2bfloat16_rn(wi);
            wb[i] = h;
            if (wt) {
                const int r = i / cols, c = i % cols;
                wt[(long long)c * rows + r] = h;
            }
        }
    }
}

__global__ void k_copy_bf16(const float *w, int rows, int cols, __nv_bfloat16 *wb, __nv_bfloat16 *wt) {
    const int n = rows * cols;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const __nv_bfloat16 h = __float2bfloat16_rn(w[i]);
        wb[i] = h;
        const int r = i / cols, c = i % cols;
        wt[(long long)c * rows + r] = h;
    }
}

// per-column mean and standard deviation (FP64 sums, two passes), then the
// columns standardised in place
__global__ void k_col_stats(float *Y, long long rows, int cols, float *mean, float *stdv) {
    const int c = blockIdx.x;
    double s = 0.0, s2 = 0.0;
    for (long long r = threadIdx.x; r < rows; r += blockDim.x) s += Y[r * cols + c];
    __shared__ double red[256];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    const double mu = red[0] / (double)rows;
    __syncthreads();
    for (long long r = threadIdx.x; r < rows; r += blockDim.x) {
        const double d = Y[r * cols + c] - mu;
        s2 += d * d;
    }
    red[threadIdx.x] = s2;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    double sd = sqrt(red[0] / (double)rows);
    if (!(sd > 1e-8)) sd = 1.0;
    for (long long r = threadIdx.x; r < rows; r += blockDim.x) Y[r * cols + c] = (float)((Y[r * cols + c] - mu) / sd);
    if (threadIdx.x == 0) {
        mean[c] = (float)mu;
        stdv[c] = (float)sd;
    }
}

inline int nblk(long long n, int t) {
    long long b = (n + t - 1) / t;
    return (int)(b < 4096 ? (b < 1 ? 1 : b) : 4096);
}

}  // namespace

template <bool AK, bool BKM, int EPI>
static cudaError_t gemm_t(int M, int N, int K, const __nv_bfloat16 *A, int lda, const __nv_bfloat16 *B, int ldb,
                          const GemmEpi &ep, cudaStream_t s) {
    dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM);
    k_gemm<AK, BKM, EPI><<<grid, 128, 0, s>>>(M, N, K, A, lda, B, ldb, ep);
    return cudaGetLastError();
}

cudaError_t mlp_gemm(int layout, int epi, int M, int N, int K, const __nv_bfloat16 *A, int lda,
                     const __nv_bfloat16 *B, int ldb, const GemmEpi &ep, cudaStream_t s) {
    // layout: bit 0 = A is K-major, bit 1 = B is K-major
#define FGA_GEMM_CASE(L, AKv, BKv)                                                                       \
    if (layout == L) {                                                                                   \
        switch (epi) {                                                                                   \
        case EPI_BIAS_RELU: return gemm_t<AKv, BKv, EPI_BIAS_RELU>(M, N, K, A, lda, B, ldb, ep, s);      \
        case EPI_BIAS: return gemm_t<AKv, BKv, EPI_BIAS>(M, N, K, A, lda, B, ldb, ep, s);                \
        case EPI_BIAS_DENORM: return gemm_t<AKv, BKv, EPI_BIAS_DENORM>(M, N, K, A, lda, B, ldb, ep, s);  \
        case EPI_RELU_MASK: return gemm_t<AKv, BKv, EPI_RELU_MASK>(M, N, K, A, lda, B, ldb, ep, s);      \
        default: return gemm_t<AKv, BKv, EPI_STORE>(M, N, K, A, lda, B, ldb, ep, s);                     \
        }                                                                                                \
    }
    FGA_GEMM_CASE(3, true, true)
    FGA_GEMM_CASE(1, true, false)
    FGA_GEMM_CASE(2, false, true)
    FGA_GEMM_CASE(0, false, false)
#undef FGA_GEMM_CASE
    return cudaErrorInvalidValue;
}

cudaError_t mlp_to_bf16_pad(const float *X, int rows, int cols, int ldo, __nv_bfloat16 *out, cudaStream_t s) {
    k_to_bf16_pad<<<nblk((long long)rows * ldo, 256), 256, 0, s>>>(X, rows, cols, ldo, out);
    return cudaGetLastError();
}

cudaError_t mlp_mse(const float *Y, const float *T, long long n, float scale, float *dYf, __nv_bfloat16 *dYb,
                    double *loss_part, int nparts, cudaStream_t s) {
    k_mse<<<nparts, 256, 0, s>>>(Y, T, n, scale, dYf, dYb, loss_part);
    return cudaGetLastError();
}

cudaError_t mlp_colsum_f32(const float *X, int rows, int cols, float *out, cudaStream_t s) {
    k_colsum<float><<<(cols + 127) / 128, 128, 0, s>>>(X, rows, cols, out);
    return cudaGetLastError();
}

cudaError_t mlp_colsum_bf16(const __nv_bfloat16 *X, int rows, int cols, float *out, cudaStream_t s) {
    k_colsum<__nv_bfloat16><<<(cols + 127) / 128, 128, 0, s>>>(X, rows, cols, out);
    return cudaGetLastError();
}

cudaError_t mlp_adam(float *w, float *m, float *v, const float *g, int rows, int cols, float lr, float b1, float b2,
                     float eps, float c1, float c2, __nv_bfloat16 *wb, __nv_bfloat16 *wt, cudaStream_t s) {
    k_adam<<<nblk((long long)rows * cols, 256), 256, 0, s>>>(w, m, v, g, rows, cols, lr, b1, b2, eps, c1, c2, wb, wt);
    return cudaGetLastError();
}

cudaError_t mlp_copy_bf16(const float *w, int rows, int cols, __nv_bfloat16 *wb, __nv_bfloat16 *wt, cudaStream_t s) {
    k_copy_bf16<<<nblk((long long)rows * cols, 256), 256, 0, s>>>(w, rows, cols, wb, wt);
    return cudaGetLastError();
}

cudaError_t mlp_col_stats(float *Y, long long rows, int cols, float *mean, float *stdv, cudaStream_t s) {
    k_col_stats<<<cols, 256, 0, s>>>(Y, rows, cols, mean, stdv);
    return cudaGetLastError();
}

}  // namespace fga
