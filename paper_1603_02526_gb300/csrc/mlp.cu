// mlp.cu -- the learned warm start's network: a 3-layer ReLU MLP
// (in -> h1 -> h2 -> out) trained and evaluated with BF16 GEMMs on the
// 5th-generation tensor cores (tcgen05.mma, FP32 accumulation in tensor
// memory), FP32 master weights and Adam.
//
// GEMM convention: C(m, n) = epilogue( sum_k A(m, k) B(n, k) ), where
// A(m, k) = A[m*lda + k] (K-major) or A[k*lda + m] (M-major), and likewise B.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "mlp_internal.h"
#include "tc05.cuh"

namespace fga {

namespace {

// Epilogue of one element: v = sum_k A(m, k) B(nn, k).
template <int EPI>
__device__ __forceinline__ float epi_value(const GemmEpi &ep, int m, int nn, float v) {
    if (EPI == EPI_BIAS_RELU || EPI == EPI_BIAS || EPI == EPI_BIAS_DENORM) {
        v += ep.bias[nn];
        if (EPI == EPI_BIAS_RELU) v = fmaxf(v, 0.f);
        if (EPI == EPI_BIAS_DENORM) v = v * ep.scale[nn] + ep.shift[nn];
    } else if (EPI == EPI_RELU_MASK) {
        v = __bfloat162float(ep.mask[(long long)m * ep.ldm + nn]) > 0.f ? v : 0.f;
    }
    return v;
}

// ---------------------------------------------------------------------------
// 5th-generation tensor-core path.  One CTA of 128 threads computes a
// 128 x 128 tile of C with its FP32 accumulator in tensor memory (128 lanes x
// 128 columns).  K advances in blocks of 64 through two shared-memory stages:
// the threads copy a block of A and of B into the no-swizzle K-major
// core-matrix layout, then thread 0 issues four MMAs of K = 16 and commits
// them to the stage's mbarrier; the threads wait on that mbarrier before
// they refill the stage two blocks later, so the copy of block k + 1
// overlaps the MMAs of block k.  The epilogue reads the accumulator back
// with tcgen05.ld, each thread one row of 16 columns at a time.
// ---------------------------------------------------------------------------
constexpr int TBM = 128, TBN = 128, TBK = 64;
constexpr int T_TILE = TBM * TBK * 2;        // bytes of one operand block (A and B alike)
constexpr int T_LBO = TBM * 16;              // K-direction distance of core matrices
constexpr int T_SBO = 128;                   // M/N-direction distance of core matrices
constexpr int T_HDR = 1024;                  // mbarriers and the tensor-memory address
// Slack after the four blocks, larger than the furthest byte a descriptor of
// these tiles can address under either reading of its two byte offsets.
constexpr int T_GUARD = 32768;
constexpr int T_SMEM = T_HDR + 4 * T_TILE + T_GUARD;
constexpr unsigned long long T_TIMEOUT_NS = 1000000000ull;

// Copies rows [r0, r0 + 128) x k [k0, k0 + 64) of X into the block at S
// (element (r, k) at byte (k / 8) T_LBO + (r / 8) T_SBO + (r % 8) 16 + (k % 8) 2).
// KMAJ: X(r, k) = X[r*ld + k], else X[k*ld + r].  Rows >= rows and k >= K read
// as zero; K and ld are multiples of 8, and so is rows for an M-major X.
template <bool KMAJ>
__device__ __forceinline__ void tc_stage(unsigned char *S, const __nv_bfloat16 *X, int ld, int rows, int K, int r0,
                                         int k0) {
    const int t = threadIdx.x;
    if (KMAJ) {
        // v: bits 0..2 row within a group of 8, bits 3..5 16-byte chunk along
        // k, bits 6..9 group of 8 rows.  A warp reads 64 contiguous bytes of
        // each of 8 rows and writes four whole core matrices.
        #pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int v = t + 128 * i;
            const int row = (v >> 6) * 8 + (v & 7), c = (v >> 3) & 7;
            const int gr = r0 + row, gk = k0 + c * 8;
            uint4 val = make_uint4(0, 0, 0, 0);
            if (gr < rows && gk < K) val = __ldg(reinterpret_cast<const uint4 *>(X + (long long)gr * ld + gk));
            *reinterpret_cast<uint4 *>(S + c * T_LBO + (row >> 3) * T_SBO + (row & 7) * 16) = val;
        }
    } else {
        // p: bits 0..2 and 5 group of 8 rows (rc), bits 3..4 pair of k (kp),
        // bits 6..8 group of 8 k (kc).  Each thread reads rows 8 rc .. 8 rc + 7
        // at k and k + 1 (16 bytes each) and stores the 8 (k, k + 1) pairs as
        // 32-bit words, in an order rotated by rc so that the 32 lanes of a
        // warp hit 32 distinct banks.
        #pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int p = t + 128 * i;
            const int rc = (p & 7) | (((p >> 5) & 1) << 3), kp = (p >> 3) & 3, kc = p >> 6;
            const int k = k0 + kc * 8 + 2 * kp, gr = r0 + rc * 8;
            uint4 a = make_uint4(0, 0, 0, 0), b = make_uint4(0, 0, 0, 0);
            if (gr < rows) {
                if (k < K) a = __ldg(reinterpret_cast<const uint4 *>(X + (long long)k * ld + gr));
                if (k + 1 < K) b = __ldg(reinterpret_cast<const uint4 *>(X + (long long)(k + 1) * ld + gr));
            }
            const uint32_t aw[4] = {a.x, a.y, a.z, a.w}, bw[4] = {b.x, b.y, b.z, b.w};
            uint32_t pr[8];
            #pragma unroll
            for (int j = 0; j < 8; ++j) {
                const uint32_t lo = (j & 1) ? (aw[j >> 1] >> 16) : (aw[j >> 1] & 0xFFFFu);
                const uint32_t hi = (j & 1) ? (bw[j >> 1] >> 16) : (bw[j >> 1] & 0xFFFFu);
                pr[j] = lo | (hi << 16);
            }
            // pr[jj] <- pr[(jj + rc) % 8], by three conditional rotations
            #pragma unroll
            for (int sh = 0; sh < 3; ++sh) {
                const bool f = (rc >> sh) & 1;
                uint32_t q[8];
                #pragma unroll
                for (int jj = 0; jj < 8; ++jj) q[jj] = f ? pr[(jj + (1 << sh)) & 7] : pr[jj];
                #pragma unroll
                for (int jj = 0; jj < 8; ++jj) pr[jj] = q[jj];
            }
            unsigned char *base = S + kc * T_LBO + rc * T_SBO + kp * 4;
            #pragma unroll
            for (int jj = 0; jj < 8; ++jj)
                *reinterpret_cast<uint32_t *>(base + ((jj + rc) & 7) * 16) = pr[jj];
        }
    }
}

template <bool AK, bool BKM, int EPI>
__global__ void __launch_bounds__(128, 1) k_gemm_tc(int M, int N, int K, const __nv_bfloat16 *A, int lda,
                                                   const __nv_bfloat16 *B, int ldb, GemmEpi ep) {
    extern __shared__ __align__(1024) unsigned char tsm[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(tsm);   // one per stage
    uint32_t *tslot = reinterpret_cast<uint32_t *>(tsm + 64);
    unsigned char *tiles = tsm + T_HDR;
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int m0 = blockIdx.y * TBM, n0 = blockIdx.x * TBN;
    if (t == 0) {
        tc05::mbar_init(&bar[0], 1);
        tc05::mbar_init(&bar[1], 1);
    }
    if (warp == 0) tc05::tmem_alloc(tslot, TBN);
    tc05::fence_before_sync();
    __syncthreads();
    tc05::fence_after_sync();
    const uint32_t tmem = *tslot;
    constexpr uint32_t idesc = tc05::idesc_bf16_f32<TBM, TBN>();
    const int nk = (K + TBK - 1) / TBK;
    bool ok = true;
    int issued = 0;   // K blocks committed
    for (int kb = 0; kb < nk; ++kb) {
        const int s = kb & 1;
        unsigned char *sa = tiles + s * 2 * T_TILE, *sb = sa + T_TILE;
        if (kb >= 2) {
            // the MMAs of block kb - 2 have finished reading this stage
            const bool w = tc05::mbar_wait(&bar[s], ((kb - 2) >> 1) & 1, T_TIMEOUT_NS);
            if (!__syncthreads_and(w)) {
                ok = false;
                break;
            }
        }
        tc_stage<AK>(sa, A, lda, M, K, m0, kb * TBK);
        tc_stage<BKM>(sb, B, ldb, N, K, n0, kb * TBK);
        tc05::fence_proxy_async_smem();
        __syncthreads();
        if (t == 0) {
            tc05::fence_after_sync();
            const uint32_t a0 = tc05::smem_addr(sa), b0 = tc05::smem_addr(sb);
            #pragma unroll
            for (int j = 0; j < TBK / 16; ++j)
                tc05::mma_bf16(tmem, tc05::smem_desc(a0 + 2 * j * T_LBO, T_LBO, T_SBO),
                               tc05::smem_desc(b0 + 2 * j * T_LBO, T_LBO, T_SBO), idesc, kb > 0 || j > 0);
            tc05::commit(&bar[s]);
        }
        issued = kb + 1;
    }
    // the last commit covers every MMA issued before it
    bool done = true;
    if (issued > 0) done = tc05::mbar_wait(&bar[(issued - 1) & 1], ((issued - 1) >> 1) & 1, T_TIMEOUT_NS);
    done = __syncthreads_and(done) != 0;
    tc05::fence_after_sync();
    if (ok && done && issued > 0) {
        const int m = m0 + warp * 32 + lane;
        const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
        const bool vf = ep.outf && (ep.ldc & 7) == 0 && (reinterpret_cast<uintptr_t>(ep.outf) & 15) == 0;
        const bool vb = ep.outb && (ep.ldc & 7) == 0 && (reinterpret_cast<uintptr_t>(ep.outb) & 15) == 0;
        #pragma unroll 1
        for (int c = 0; c < TBN / 16; ++c) {
            const int nb = n0 + c * 16;
            if (nb >= N) break;   // uniform over the CTA
            float v[16];
            tc05::ld_32x32b_x16(trow + (uint32_t)(c * 16), v);
            if (m >= M) continue;
            const bool full = nb + 16 <= N;
            #pragma unroll
            for (int q = 0; q < 16; ++q) v[q] = (full || nb + q < N) ? epi_value<EPI>(ep, m, nb + q, v[q]) : 0.f;
            const long long o = (long long)m * ep.ldc + nb;
            if (full && vf) {
                #pragma unroll
                for (int q = 0; q < 16; q += 4)
                    *reinterpret_cast<float4 *>(ep.outf + o + q) = make_float4(v[q], v[q + 1], v[q + 2], v[q + 3]);
            } else if (ep.outf) {
                for (int q = 0; q < 16 && nb + q < N; ++q) ep.outf[o + q] = v[q];
            }
            if (full && vb) {
                #pragma unroll
                for (int h = 0; h < 2; ++h) {
                    uint32_t w[4];
                    #pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const __nv_bfloat162 pq = __floats2bfloat162_rn(v[8 * h + 2 * q], v[8 * h + 2 * q + 1]);
                        w[q] = *reinterpret_cast<const uint32_t *>(&pq);
                    }
                    *reinterpret_cast<uint4 *>(ep.outb + o + 8 * h) = make_uint4(w[0], w[1], w[2], w[3]);
                }
            } else if (ep.outb) {
                for (int q = 0; q < 16 && nb + q < N; ++q) ep.outb[o + q] = __float2bfloat16_rn(v[q]);
            }
        }
    } else if (t == 0 && ep.err) {
        atomicOr(ep.err, 1);
    }
    tc05::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc05::tmem_dealloc(tmem, TBN);
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
static cudaError_t gemm_tc_t(int M, int N, int K, const __nv_bfloat16 *A, int lda, const __nv_bfloat16 *B, int ldb,
                             const GemmEpi &ep, cudaStream_t s) {
    cudaError_t e = cudaFuncSetAttribute(k_gemm_tc<AK, BKM, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize, T_SMEM);
    if (e != cudaSuccess) return e;
    dim3 grid((N + TBN - 1) / TBN, (M + TBM - 1) / TBM);
    k_gemm_tc<AK, BKM, EPI><<<grid, 128, T_SMEM, s>>>(M, N, K, A, lda, B, ldb, ep);
    return cudaGetLastError();
}

// Operand rules of the tensor-core path: 16-byte aligned base, K and ld
// multiples of 8, ld covering the contiguous extent; an M-major operand's
// row count a multiple of 8 as well.
static bool operand_ok(const __nv_bfloat16 *X, int ld, int rows, int K, bool kmaj) {
    if (!X || (reinterpret_cast<uintptr_t>(X) & 15) || ld % 8) return false;
    return kmaj ? ld >= K : (rows % 8 == 0 && ld >= rows);
}

cudaError_t mlp_gemm(int layout, int epi, int M, int N, int K, const __nv_bfloat16 *A, int lda,
                     const __nv_bfloat16 *B, int ldb, const GemmEpi &ep, cudaStream_t s) {
    // layout: bit 0 = A is K-major, bit 1 = B is K-major
    if (M < 1 || N < 1 || K < 8 || K % 8 || ep.ldc < N || !operand_ok(A, lda, M, K, layout & 1) ||
        !operand_ok(B, ldb, N, K, (layout >> 1) & 1))
        return cudaErrorInvalidValue;
#define FGA_GEMM_CASE(L, AKv, BKv)                                                                          \
    if (layout == L) {                                                                                      \
        switch (epi) {                                                                                      \
        case EPI_BIAS_RELU: return gemm_tc_t<AKv, BKv, EPI_BIAS_RELU>(M, N, K, A, lda, B, ldb, ep, s);      \
        case EPI_BIAS: return gemm_tc_t<AKv, BKv, EPI_BIAS>(M, N, K, A, lda, B, ldb, ep, s);                \
        case EPI_BIAS_DENORM: return gemm_tc_t<AKv, BKv, EPI_BIAS_DENORM>(M, N, K, A, lda, B, ldb, ep, s);  \
        case EPI_RELU_MASK: return gemm_tc_t<AKv, BKv, EPI_RELU_MASK>(M, N, K, A, lda, B, ldb, ep, s);      \
        default: return gemm_tc_t<AKv, BKv, EPI_STORE>(M, N, K, A, lda, B, ldb, ep, s);                     \
        }                                                                                                   \
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
