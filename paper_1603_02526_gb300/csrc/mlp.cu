// mlp.cu -- the learned warm start's network: a 3-layer ReLU MLP
// (in -> h1 -> h2 -> out) trained and evaluated with BF16 GEMMs on the
// 5th-generation tensor cores (tcgen05.mma, FP32 accumulation in tensor
// memory), FP32 master weights and Adam.
//
// GEMM convention: C(m, n) = epilogue( sum_k A(m, k) B(n, k) ), where
// A(m, k) = A[m*lda + k] (K-major) or A[k*lda + m] (M-major), and likewise B.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cstring>
#include <atomic>
#include <mutex>
#include <unordered_map>

#include "mlp_internal.h"
#include "tc05.cuh"

namespace fga {

namespace {

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
// two stages of A and B (64 KB), widened to 96 KB for the epilogue's
// staging block (4 warps x 32 rows x 132 floats), which reuses them
constexpr int T_SMEM = T_HDR + 6 * T_TILE;
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

// Epilogue of a 128 x 128 tile whose FP32 accumulator sits in tensor memory
// at tmem, staged through shared memory at S (the operand stages, free once
// the MMAs are done; 4 x 32 x T_SROW floats).  Pass 1: warp w reads its 32
// rows (one per lane, 32 columns at a time) and writes them as 16-byte rows
// segments into its own 32 x T_SROW block (a stride of 132 floats keeps the
// eight lanes of each store phase on distinct banks).  Pass 2: row by row,
// lane l takes columns 4l .. 4l + 3 (their bias, scale and shift held in
// registers), applies the element epilogue and stores whole 512-byte (FP32)
// or 256-byte (BF16) row segments.  Every thread of the CTA calls it
// (tcgen05.ld is warp-collective).
constexpr int T_SROW = TBN + 4;
static_assert(4 * 32 * T_SROW * 4 <= T_SMEM - T_HDR, "the epilogue's staging fits in the operand area");

template <int EPI>
__device__ __forceinline__ void tc_epilogue(const GemmEpi &ep, int M, int N, int m0, int n0, uint32_t tmem,
                                            float *S) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float *Sw = S + warp * 32 * T_SROW;
    const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
    #pragma unroll 1
    for (int c = 0; c < TBN / 32; ++c) {
        if (n0 + c * 32 >= N) break;   // uniform over the CTA
        float v[32];
        tc05::ld_32x32b_x32(trow + (uint32_t)(c * 32), v);
        #pragma unroll
        for (int q = 0; q < 32; q += 4)
            *reinterpret_cast<float4 *>(Sw + lane * T_SROW + c * 32 + q) = make_float4(v[q], v[q + 1], v[q + 2], v[q + 3]);
    }
    __syncwarp();
    const int n = n0 + 4 * lane;
    float bias[4] = {0.f, 0.f, 0.f, 0.f}, scale[4] = {1.f, 1.f, 1.f, 1.f}, shift[4] = {0.f, 0.f, 0.f, 0.f};
    #pragma unroll
    for (int j = 0; j < 4; ++j) {
        if (n + j < N) {
            if (EPI == EPI_BIAS_RELU || EPI == EPI_BIAS || EPI == EPI_BIAS_DENORM) bias[j] = ep.bias[n + j];
            if (EPI == EPI_BIAS_DENORM) {
                scale[j] = ep.scale[n + j];
                shift[j] = ep.shift[n + j];
            }
        }
    }
    const bool whole = n + 4 <= N;
    const bool vf = ep.outf && (ep.ldc & 3) == 0 && (reinterpret_cast<uintptr_t>(ep.outf) & 15) == 0;
    const bool vb = ep.outb && (ep.ldc & 3) == 0 && (reinterpret_cast<uintptr_t>(ep.outb) & 7) == 0;
    const bool vm = EPI == EPI_RELU_MASK && (ep.ldm & 3) == 0 && (reinterpret_cast<uintptr_t>(ep.mask) & 7) == 0;
    #pragma unroll 4
    for (int r = 0; r < 32; ++r) {
        const int m = m0 + warp * 32 + r;
        if (m >= M || n >= N) continue;
        const float4 a = *reinterpret_cast<const float4 *>(Sw + r * T_SROW + 4 * lane);
        float o[4] = {a.x, a.y, a.z, a.w};
        if (EPI == EPI_RELU_MASK) {
            float mk[4];
            if (whole && vm) {
                const uint2 w = *reinterpret_cast<const uint2 *>(ep.mask + (long long)m * ep.ldm + n);
                const __nv_bfloat162 lo = *reinterpret_cast<const __nv_bfloat162 *>(&w.x);
                const __nv_bfloat162 hi = *reinterpret_cast<const __nv_bfloat162 *>(&w.y);
                mk[0] = __low2float(lo);
                mk[1] = __high2float(lo);
                mk[2] = __low2float(hi);
                mk[3] = __high2float(hi);
            } else {
                #pragma unroll
                for (int j = 0; j < 4; ++j)
                    mk[j] = n + j < N ? __bfloat162float(ep.mask[(long long)m * ep.ldm + n + j]) : 0.f;
            }
            #pragma unroll
            for (int j = 0; j < 4; ++j) o[j] = mk[j] > 0.f ? o[j] : 0.f;
        } else if (EPI != EPI_STORE) {
            #pragma unroll
            for (int j = 0; j < 4; ++j) {
                float x = o[j] + bias[j];
                if (EPI == EPI_BIAS_RELU) x = fmaxf(x, 0.f);
                if (EPI == EPI_BIAS_DENORM) x = x * scale[j] + shift[j];
                o[j] = x;
            }
        }
        const long long off = (long long)m * ep.ldc + n;
        if (ep.outf) {
            if (whole && vf) {
                *reinterpret_cast<float4 *>(ep.outf + off) = make_float4(o[0], o[1], o[2], o[3]);
            } else {
                #pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (n + j < N) ep.outf[off + j] = o[j];
            }
        }
        if (ep.outb) {
            if (whole && vb) {
                const __nv_bfloat162 p0 = __floats2bfloat162_rn(o[0], o[1]), p1 = __floats2bfloat162_rn(o[2], o[3]);
                uint2 w;
                w.x = *reinterpret_cast<const uint32_t *>(&p0);
                w.y = *reinterpret_cast<const uint32_t *>(&p1);
                *reinterpret_cast<uint2 *>(ep.outb + off) = w;
            } else {
                #pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (n + j < N) ep.outb[off + j] = __float2bfloat16_rn(o[j]);
            }
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
    const int t = threadIdx.x, warp = t >> 5;
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
    // split K: slice blockIdx.z takes the blocks [kbeg, kbeg + nk)
    const int nk_all = (K + TBK - 1) / TBK;
    const int per = (nk_all + (int)gridDim.z - 1) / (int)gridDim.z;
    const int kbeg = (int)blockIdx.z * per;
    const int nk = max(0, min(nk_all, kbeg + per) - kbeg);
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
        tc_stage<AK>(sa, A, lda, M, K, m0, (kbeg + kb) * TBK);
        tc_stage<BKM>(sb, B, ldb, N, K, n0, (kbeg + kb) * TBK);
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
        GemmEpi e = ep;
        if (gridDim.z > 1) e.outf = ep.outf + (long long)blockIdx.z * M * ep.ldc;   // this slice's partial
        tc_epilogue<EPI>(e, M, N, m0, n0, tmem, reinterpret_cast<float *>(tiles));
    } else if (t == 0 && ep.err) {
        atomicOr(ep.err, 1);
    }
    tc05::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc05::tmem_dealloc(tmem, TBN);
}

// ---------------------------------------------------------------------------
// TMA path for two K-major operands (the forward and data-gradient
// products).  Warp-specialised: thread 0 (warp 0) is the producer, which
// fills a ring of T_NS stages with TMA tensor loads (per operand and block
// of 64 k, one box of 128 rows x 128 bytes in the 128-byte swizzled layout,
// every stage on a 1024-byte boundary) completing on the stage's "full"
// mbarrier; thread 32
// (warp 1) issues the MMAs of a stage once it is full and commits them to
// the stage's "empty" mbarrier, which the producer waits on before it
// refills the stage; a final commit to "done" releases the epilogue of all
// four warps.  Every wait is bounded; a wait that gives up sets ep.err,
// and before it leaves the CTA waits (bounded) for every copy it issued.
// ---------------------------------------------------------------------------
constexpr int T_NS = 3;                                   // stages
constexpr int T_SMEM_TMA = T_HDR + T_NS * 2 * T_TILE;     // 97 KB: two CTAs per SM
static_assert(4 * 32 * T_SROW * 4 <= T_SMEM_TMA - T_HDR, "the epilogue's staging fits in the stages");

template <int EPI>
__global__ void __launch_bounds__(128, 1) k_gemm_tma(int M, int N, int K, const __grid_constant__ CUtensorMap tmA,
                                                    const __grid_constant__ CUtensorMap tmB, GemmEpi ep) {
    extern __shared__ __align__(1024) unsigned char tsm[];
    uint64_t *full = reinterpret_cast<uint64_t *>(tsm);   // [T_NS]
    uint64_t *empty = full + T_NS;                        // [T_NS]
    uint64_t *done = empty + T_NS;                        // [1]
    uint32_t *tslot = reinterpret_cast<uint32_t *>(tsm + 128);
    unsigned char *tiles = tsm + T_HDR;
    const int t = threadIdx.x, warp = t >> 5;
    const int m0 = blockIdx.y * TBM, n0 = blockIdx.x * TBN;
    // split K: slice blockIdx.z takes the blocks [kbeg, kbeg + nk)
    const int nk_all = (K + TBK - 1) / TBK;
    const int per = (nk_all + (int)gridDim.z - 1) / (int)gridDim.z;
    const int kbeg = (int)blockIdx.z * per;
    // the swizzled stages must start on 1024-byte boundaries: otherwise no
    // copy and no MMA is issued and the error word is set
    const bool aligned = (tc05::smem_addr(tiles) & 1023u) == 0;
    const int nk = aligned ? max(0, min(nk_all, kbeg + per) - kbeg) : 0;
    if (t == 0 && !aligned && ep.err) atomicOr(ep.err, 1);
    if (t == 0) {
        for (int s = 0; s < T_NS; ++s) {
            tc05::mbar_init(&full[s], 1);
            tc05::mbar_init(&empty[s], 1);
        }
        tc05::mbar_init(done, 1);
        tc05::fence_proxy_async_smem();
    }
    if (warp == 0) tc05::tmem_alloc(tslot, TBN);
    tc05::fence_before_sync();
    __syncthreads();
    tc05::fence_after_sync();
    const uint32_t tmem = *tslot;
    bool ok = true;
    int issued = 0;   // blocks whose copies thread 0 issued
    if (t == 0) {
        for (int kb = 0; kb < nk; ++kb) {
            const int s = kb % T_NS;
            if (kb >= T_NS && !tc05::mbar_wait(&empty[s], ((kb / T_NS) - 1) & 1, T_TIMEOUT_NS)) {
                ok = false;
                break;
            }
            unsigned char *sa = tiles + s * 2 * T_TILE, *sb = sa + T_TILE;
            tc05::mbar_arrive_expect_tx(&full[s], 2 * T_TILE);
            tc05::tma_load_2d(sa, &tmA, (kbeg + kb) * TBK, m0, &full[s]);
            tc05::tma_load_2d(sb, &tmB, (kbeg + kb) * TBK, n0, &full[s]);
            issued = kb + 1;
        }
    } else if (t == 32) {
        constexpr uint32_t idesc = tc05::idesc_bf16_f32<TBM, TBN>();
        for (int kb = 0; kb < nk; ++kb) {
            const int s = kb % T_NS;
            if (!tc05::mbar_wait(&full[s], (kb / T_NS) & 1, T_TIMEOUT_NS)) {
                ok = false;
                break;
            }
            tc05::fence_after_sync();
            const uint32_t a0 = tc05::smem_addr(tiles + s * 2 * T_TILE), b0 = a0 + T_TILE;
            #pragma unroll
            for (int j = 0; j < TBK / 16; ++j)   // K step of 16 bf16 = 32 bytes inside the swizzle atom
                tc05::mma_bf16(tmem, tc05::smem_desc_sw128(a0 + 32 * j), tc05::smem_desc_sw128(b0 + 32 * j), idesc,
                               kb > 0 || j > 0);
            tc05::commit(&empty[s]);
        }
        tc05::commit(done);   // covers every MMA issued above
    }
    __syncwarp();
    const bool fin = tc05::mbar_wait(done, 0, T_TIMEOUT_NS);
    const bool good = __syncthreads_and(ok && fin) != 0;
    tc05::fence_after_sync();
    if (good && nk > 0) {
        GemmEpi e = ep;
        if (gridDim.z > 1) e.outf = ep.outf + (long long)blockIdx.z * M * ep.ldc;   // this slice's partial
        tc_epilogue<EPI>(e, M, N, m0, n0, tmem, reinterpret_cast<float *>(tiles));
    }
    else if (t == 0 && ep.err) atomicOr(ep.err, 1);
    if (t == 0) {
        // every stage's last issued copy has landed before the CTA leaves
        for (int s = 0; s < T_NS && s < issued; ++s) {
            const int uses = (issued - 1 - s) / T_NS + 1;
            tc05::mbar_wait(&full[s], (uses - 1) & 1, T_TIMEOUT_NS);
        }
    }
    tc05::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc05::tmem_dealloc(tmem, TBN);
}

// The split-K slices' sums, added in slice order, through the element
// epilogue EPI: v = sum_z ws[z][m][n], then bias / ReLU / mask /
// de-standardise as in tc_epilogue, stored as FP32 and/or BF16.
template <int EPI>
__global__ void k_split_sum(const float *ws, int S, int M, int N, GemmEpi ep) {
    const long long n_el = (long long)M * N;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n_el; i += (long long)gridDim.x * blockDim.x) {
        float v = 0.f;
        for (int z = 0; z < S; ++z) v += ws[z * n_el + i];
        const int m = (int)(i / N), n = (int)(i % N);
        if (EPI == EPI_BIAS_RELU || EPI == EPI_BIAS || EPI == EPI_BIAS_DENORM) {
            v += ep.bias[n];
            if (EPI == EPI_BIAS_RELU) v = fmaxf(v, 0.f);
            if (EPI == EPI_BIAS_DENORM) v = v * ep.scale[n] + ep.shift[n];
        } else if (EPI == EPI_RELU_MASK) {
            v = __bfloat162float(ep.mask[(long long)m * ep.ldm + n]) > 0.f ? v : 0.f;
        }
        const long long o = (long long)m * ep.ldc + n;
        if (ep.outf) ep.outf[o] = v;
        if (ep.outb) ep.outb[o] = __float2bfloat16_rn(v);
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

// The dynamic shared-memory limit of a kernel, raised once per device.
template <typename F>
static cudaError_t smem_attr_once(F *fn, int bytes, std::atomic<unsigned long long> &done) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = dev < 64 ? 1ull << dev : 0ull;
    if (bit && (done.load(std::memory_order_acquire) & bit)) return cudaSuccess;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess && bit) done.fetch_or(bit, std::memory_order_acq_rel);
    return e;
}

template <bool AK, bool BKM, int EPI>
static cudaError_t gemm_tc_t(int M, int N, int K, const __nv_bfloat16 *A, int lda, const __nv_bfloat16 *B, int ldb,
                             const GemmEpi &ep, cudaStream_t s, int S) {
    static std::atomic<unsigned long long> attr_set{0};
    cudaError_t e = smem_attr_once(k_gemm_tc<AK, BKM, EPI>, T_SMEM, attr_set);
    if (e != cudaSuccess) return e;
    dim3 grid((N + TBN - 1) / TBN, (M + TBM - 1) / TBM, S);
    k_gemm_tc<AK, BKM, EPI><<<grid, 128, T_SMEM, s>>>(M, N, K, A, lda, B, ldb, ep);
    return cudaGetLastError();
}

// cuTensorMapEncodeTiled from the driver, resolved once through the runtime
// (no link-time dependency on the driver library).
static PFN_cuTensorMapEncodeTiled_v12000 encode_tiled() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

// Tensor map of a K-major BF16 operand X(r, k) = X[r*ld + k], rows x K,
// boxes of 64 k x 128 rows (128 bytes x 128) written in the 128-byte
// swizzled layout, zero fill outside.  A map is a
// pure function of (address, rows, K, ld), so maps are kept in a small
// cache: the network's operands live in buffers it owns, and a training
// step reuses the same few dozen maps.
struct MapKey {
    const void *p;
    int rows, K, ld;
    bool operator==(const MapKey &o) const { return p == o.p && rows == o.rows && K == o.K && ld == o.ld; }
};
struct MapKeyHash {
    size_t operator()(const MapKey &k) const {
        size_t h = std::hash<const void *>()(k.p);
        h ^= (size_t)k.rows * 0x9E3779B97F4A7C15ull + (size_t)k.K * 0xC2B2AE3D27D4EB4Full + (size_t)k.ld;
        return h;
    }
};

static cudaError_t kmajor_map(CUtensorMap *m, const __nv_bfloat16 *X, int rows, int K, int ld) {
    static std::mutex mu;
    static std::unordered_map<MapKey, CUtensorMap, MapKeyHash> cache;
    const MapKey key{X, rows, K, ld};
    {
        std::lock_guard<std::mutex> lk(mu);
        auto it = cache.find(key);
        if (it != cache.end()) {
            *m = it->second;
            return cudaSuccess;
        }
    }
    PFN_cuTensorMapEncodeTiled_v12000 fn = encode_tiled();
    if (!fn) return cudaErrorNotSupported;
    const cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * sizeof(__nv_bfloat16)};
    const cuuint32_t box[2] = {(cuuint32_t)TBK, (cuuint32_t)TBM};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16 *>(X), dims, strides, box,
                          estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    std::lock_guard<std::mutex> lk(mu);
    if (cache.size() > 4096) cache.clear();
    cache.emplace(key, *m);
    return cudaSuccess;
}

template <int EPI>
static cudaError_t gemm_tma_t(int M, int N, int K, const __nv_bfloat16 *A, int lda, const __nv_bfloat16 *B, int ldb,
                              const GemmEpi &ep, cudaStream_t s, int S) {
    static std::atomic<unsigned long long> attr_set{0};
    CUtensorMap ta, tb;
    cudaError_t e = kmajor_map(&ta, A, M, K, lda);
    if (e == cudaSuccess) e = kmajor_map(&tb, B, N, K, ldb);
    if (e == cudaSuccess) e = smem_attr_once(k_gemm_tma<EPI>, T_SMEM_TMA, attr_set);
    if (e != cudaSuccess) return e;
    dim3 grid((N + TBN - 1) / TBN, (M + TBM - 1) / TBM, S);
    k_gemm_tma<EPI><<<grid, 128, T_SMEM_TMA, s>>>(M, N, K, ta, tb, ep);
    return cudaGetLastError();
}

// Operand rules of the tensor-core path: 16-byte aligned base, K and ld
// multiples of 8, ld covering the contiguous extent; an M-major operand's
// row count a multiple of 8 as well.
static bool operand_ok(const __nv_bfloat16 *X, int ld, int rows, int K, bool kmaj) {
    if (!X || (reinterpret_cast<uintptr_t>(X) & 15) || ld % 8) return false;
    return kmaj ? ld >= K : (rows % 8 == 0 && ld >= rows);
}

// Split-K factor: about one wave of CTAs when the tile grid is small (the
// products of a training batch), K long enough (at least 8 blocks) for the
// shorter slices to pay for the slice sum, and a workspace for the slices'
// partials is given; every slice non-empty; 1 otherwise.
static int split_factor(int M, int N, int K, const GemmEpi &ep) {
    const int tiles = ((N + TBN - 1) / TBN) * ((M + TBM - 1) / TBM), nk = (K + TBK - 1) / TBK;
    if (!ep.ws || nk < 8) return 1;
    int S = std::min(std::min(nk, 16), std::max(1, 148 / tiles));
    while (S > 1 && (long long)S * M * N > ep.ws_floats) --S;
    if (S > 1) {
        const int per = (nk + S - 1) / S;
        S = (nk + per - 1) / per;
    }
    return S;
}

template <int EPI>
static cudaError_t gemm_launch(int layout, int M, int N, int K, const __nv_bfloat16 *A, int lda,
                               const __nv_bfloat16 *B, int ldb, const GemmEpi &ep, cudaStream_t s, int S) {
    switch (layout) {   // bit 0: A is K-major, bit 1: B is K-major
    case 3: return gemm_tma_t<EPI>(M, N, K, A, lda, B, ldb, ep, s, S);   // TMA-fed, warp-specialised
    case 1: return gemm_tc_t<true, false, EPI>(M, N, K, A, lda, B, ldb, ep, s, S);
    case 2: return gemm_tc_t<false, true, EPI>(M, N, K, A, lda, B, ldb, ep, s, S);
    case 0: return gemm_tc_t<false, false, EPI>(M, N, K, A, lda, B, ldb, ep, s, S);
    }
    return cudaErrorInvalidValue;
}

template <int EPI>
static cudaError_t gemm_epi(int layout, int M, int N, int K, const __nv_bfloat16 *A, int lda, const __nv_bfloat16 *B,
                            int ldb, const GemmEpi &ep, cudaStream_t s) {
    const int S = split_factor(M, N, K, ep);
    if (S <= 1) return gemm_launch<EPI>(layout, M, N, K, A, lda, B, ldb, ep, s, 1);
    // slices write raw sums; the slice sum applies the epilogue
    GemmEpi part;
    std::memset(&part, 0, sizeof part);
    part.outf = ep.ws;
    part.ldc = N;
    part.err = ep.err;
    cudaError_t e = gemm_launch<EPI_STORE>(layout, M, N, K, A, lda, B, ldb, part, s, S);
    if (e != cudaSuccess) return e;
    const long long n_el = (long long)M * N;
    k_split_sum<EPI><<<(int)std::min<long long>((n_el + 255) / 256, 1184), 256, 0, s>>>(ep.ws, S, M, N, ep);
    return cudaGetLastError();
}

cudaError_t mlp_gemm(int layout, int epi, int M, int N, int K, const __nv_bfloat16 *A, int lda,
                     const __nv_bfloat16 *B, int ldb, const GemmEpi &ep, cudaStream_t s) {
    if (layout < 0 || layout > 3 || M < 1 || N < 1 || K < 8 || K % 8 || ep.ldc < N ||
        !operand_ok(A, lda, M, K, layout & 1) || !operand_ok(B, ldb, N, K, (layout >> 1) & 1))
        return cudaErrorInvalidValue;
    switch (epi) {
    case EPI_BIAS_RELU: return gemm_epi<EPI_BIAS_RELU>(layout, M, N, K, A, lda, B, ldb, ep, s);
    case EPI_BIAS: return gemm_epi<EPI_BIAS>(layout, M, N, K, A, lda, B, ldb, ep, s);
    case EPI_BIAS_DENORM: return gemm_epi<EPI_BIAS_DENORM>(layout, M, N, K, A, lda, B, ldb, ep, s);
    case EPI_RELU_MASK: return gemm_epi<EPI_RELU_MASK>(layout, M, N, K, A, lda, B, ldb, ep, s);
    default: return gemm_epi<EPI_STORE>(layout, M, N, K, A, lda, B, ldb, ep, s);
    }
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
