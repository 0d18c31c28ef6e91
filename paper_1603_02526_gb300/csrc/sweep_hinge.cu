// sweep_hinge.cu -- the hinge-bank sweep: Algorithm 2 on a linear
// soft-margin SVM written as a factor graph (Sec. V-C): hinge factors
// c max(0, 1 - y (w.x + b)) on one shared (w, b) plus L2 factors
// (lambda/2)|w|^2, FP32, one rho, alpha = 1, one persistent launch per call.
//
// Displacements (as in the disk-tile sweep): with one rho, m = z + Delta,
// so z <- z + (sum of the edges' displacements) / deg; with alpha = 1,
// n^k = y^k - Delta^k with y^k = 2 z^k - z^{k-1}.  A hinge factor's
// operator moves n along (x, 1): Delta = g (x, 1) with one scalar
// g = gamma y / rho, gamma = min(c, rho t / (|x|^2 + 1)),
// t = 1 - y (n.(x, 1)) (zero when t <= 0).  Its state is g, and n.(x, 1) =
// y.(x, 1) - g (|x|^2 + 1): one dot product with y per factor per
// iteration, then g (x, 1) added into the sums.  An L2 factor's
// displacement is -lambda / (rho + lambda) n, kept per component.
//
// Work: each CTA holds its slice of the data rows in shared memory (256 B
// per row).  A group of 8 lanes works on one factor at a time: lane m holds
// components 4m..4m+3 and 32+4m..32+4m+3 of y and of its running sums, so a
// row is read once per iteration (two 16-byte loads per lane) and the dot
// product needs three shuffles.  The groups' sums are combined per warp
// (two shuffles), per CTA (in shared memory, fixed warp order) and across
// CTAs in the fixed-point accumulators (exact, order-free), each word
// carrying a count of the contributions it holds: a CTA starts its next
// pass once every word counts all CTAs, and only checked passes add a grid
// barrier.  Checks form x, u and the FP64 residual sums from the same
// quantities and store the state.
#include <cuda_runtime.h>
#include <stdint.h>

#include "hinge_internal.h"
#include "residual.cuh"
#include "persist.cuh"

namespace fga {

// Shared memory: data rows, per-factor (y, c, |x|^2 + 1), z / z_prev / y /
// y_prev per component, the warps' staged sums, the L2 state.
struct HingeSmem {
    int X, meta, z, zp, y, yp, stg, l2d, l2s, pv, total;
};
static __host__ __device__ HingeSmem hinge_smem_layout(int rows) {
    HingeSmem L{};
    int o = 0;
    L.X = o;
    o += rows * kHingeD * 4;
    L.meta = o;
    o += rows * 16;
    L.z = o;
    o += 80 * 4;
    L.zp = o;
    o += 80 * 4;
    L.y = o;
    o += 80 * 4;
    L.yp = o;
    o += 80 * 4;
    L.stg = o;
    o += kHingeWarps * 68 * 4;
    L.l2d = o;
    o += kHingeMaxL2 * kHingeD * 4;
    L.l2s = o;
    o += kHingeMaxL2 * kHingeD * 4;
    L.pv = o;   // per variable and word parity: the value seen the last time
    o += 2 * 80 * 8;
    L.total = o;
    return L;
}

int hinge_smem_bytes(int rows) { return hinge_smem_layout(rows).total; }

// Component c (0..7) of lane m: 4m + c for c < 4, 32 + 4m + c - 4 after.
static __device__ __forceinline__ int hcomp(int m, int c) { return (c < 4 ? 4 * m : 28 + 4 * m) + c; }

// One pass over the CTA's hinge factors.  g[k]: state of factor
// gi + k * groups.  Returns in acc/accb the lane's share of the sums.
template <bool GEN>
static __device__ __forceinline__ void hinge_factors(const HingeArgs &a, const PassMode pm, const HingeCta &C, int gi,
                                                     int m, float (&g)[kHingeK], const float *Xs,
                                                     const float4 *metas, const float *zt, const float *zpt,
                                                     const float *yt, const float *ypt, float (&acc)[8],
                                                     float &accb, double &pri) {
    const int MODE = GEN ? pm.mode : (int)T_MID;
    const bool RELOAD = GEN && pm.reload;
    const bool SAVE = GEN && pm.save;
    const bool CHK = MODE == T_CHK || MODE == T_FINAL;
    const int D = a.D;
    // y in registers (every pass); z, z_prev, y_prev read from shared
    // memory by the rare passes that need them
    float yv[8];
    #pragma unroll
    for (int c = 0; c < 8; ++c) yv[c] = yt[hcomp(m, c)];
    const float yb = yt[D];
    #pragma unroll
    for (int c = 0; c < 8; ++c) acc[c] = 0.f;
    accb = 0.f;
    #pragma unroll
    for (int k = 0; k < kHingeK; ++k) {
        const int i = gi + k * kHingeGroups;
        const bool valid = i < C.nf;
        // the slots past the CTA's last row would change nothing (g = 0, no
        // state): stop once no group of the warp has a row left
        if (k > 0 && __all_sync(0xffffffffu, !valid)) break;
        const int f = C.f0 + i;
        float x[8];
        float4 mt = make_float4(0.f, 0.f, 1.f, 0.f);
        if (valid) {
            const float4 xa = *reinterpret_cast<const float4 *>(Xs + (size_t)i * kHingeD + 4 * m);
            const float4 xb = *reinterpret_cast<const float4 *>(Xs + (size_t)i * kHingeD + 32 + 4 * m);
            x[0] = xa.x; x[1] = xa.y; x[2] = xa.z; x[3] = xa.w;
            x[4] = xb.x; x[5] = xb.y; x[6] = xb.z; x[7] = xb.w;
            mt = metas[i];
        } else {
            #pragma unroll
            for (int c = 0; c < 8; ++c) x[c] = 0.f;
        }
        const size_t eb = (size_t)a.hb_e0 + (size_t)f * (D + 1);
        // the dot product with (x, 1): of y, or of n = z - u on the call's
        // first pass
        float p = 0.f;
        if (MODE == T_FIRST) {
            #pragma unroll
            for (int c = 0; c < 8; ++c) {
                const int j = hcomp(m, c);
                if (valid && j < D) p = __fmaf_rn(__fsub_rn(zt[j], a.u[eb + j]), x[c], p);
            }
            if (valid && m == 0) p = __fadd_rn(p, __fsub_rn(zt[D], a.u[eb + D]));
        } else {
            #pragma unroll
            for (int c = 0; c < 8; ++c) p = __fmaf_rn(yv[c], x[c], p);
            if (m == 0) p = __fadd_rn(p, yb);
        }
        p = __fadd_rn(p, __shfl_xor_sync(0xffffffffu, p, 1));
        p = __fadd_rn(p, __shfl_xor_sync(0xffffffffu, p, 2));
        p = __fadd_rn(p, __shfl_xor_sync(0xffffffffu, p, 4));
        const float gk = g[k];
        if (CHK && valid) {
            // residual of iteration it-1: x - z = n^{it-2} + g (x, 1) - z
            // per edge; the state itself is stored only if the CTAs stop
            // here (hinge_state), from g kept in gres and gsave
            const float gp = RELOAD ? 0.f : a.gsave[(size_t)((pm.it - 1) & 1) * a.N + f];
            float sq = 0.f;
            #pragma unroll
            for (int c = 0; c < 9; ++c) {
                const bool isb = c == 8;
                if (isb && m != 0) continue;
                const int j = isb ? D : hcomp(m, c);
                if (!isb && j >= D) continue;
                const float xt = isb ? 1.f : x[c];
                const float no = RELOAD ? __fsub_rn(zpt[j], a.u[eb + j]) : __fsub_rn(ypt[j], __fmul_rn(gp, xt));
                const float d = __fsub_rn(__fadd_rn(no, __fmul_rn(gk, xt)), zt[j]);
                sq = __fmaf_rn(d, d, sq);
            }
            pri += (double)sq;
            if (m == 0) a.gres[f] = gk;
        }
        if (MODE == T_FINAL) continue;
        if (SAVE && valid && m == 0) a.gsave[(size_t)(pm.it & 1) * a.N + f] = gk;
        // the operator: n.(x, 1) = y.(x, 1) - g (|x|^2 + 1); gamma =
        // min(c, t rho / (|x|^2 + 1)) with rho / (|x|^2 + 1) precomputed
        // (mt.w), g = gamma y / rho
        const float nx = MODE == T_FIRST ? p : __fsub_rn(p, __fmul_rn(gk, mt.z));
        const float t = __fsub_rn(1.f, __fmul_rn(mt.x, nx));
        const float gam = t > 0.f ? fminf(mt.y, __fmul_rn(t, mt.w)) : 0.f;
        const float gn = valid ? __fmul_rn(__fmul_rn(gam, mt.x), a.inv_rho) : 0.f;
        g[k] = gn;
        #pragma unroll
        for (int c = 0; c < 8; ++c) acc[c] = __fmaf_rn(gn, x[c], acc[c]);
        accb = __fadd_rn(accb, gn);
    }
}

// The state of the checked iteration it-1 of a pass that stopped (or of
// the call's last iteration): x = n^{it-2} + g (x, 1) and u = z_prev - z +
// g (x, 1) for every hinge edge, with g of iteration it-1 (gres) and of
// it-2 (gsave, or the stored u when it-2 began the call), and the tables
// of the pass.  Lane j of each warp per component, one factor per warp at a
// time.
static __device__ __forceinline__ void hinge_state(const HingeArgs &a, const HingeCta &C, long long it, bool reload,
                                                   const float *Xs, const float *zt, const float *zpt,
                                                   const float *ypt) {
    const int D = a.D;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int i = warp; i < C.nf; i += nw) {
        const int f = C.f0 + i;
        const size_t eb = (size_t)a.hb_e0 + (size_t)f * (D + 1);
        const float gk = a.gres[f];
        const float gp = reload ? 0.f : a.gsave[(size_t)((it - 1) & 1) * a.N + f];
        for (int j = lane; j <= D; j += 32) {
            const float xt = j < D ? Xs[(size_t)i * kHingeD + j] : 1.f;
            const float no = reload ? __fsub_rn(zpt[j], a.u[eb + j]) : __fsub_rn(ypt[j], __fmul_rn(gp, xt));
            const float dl = __fmul_rn(gk, xt);
            a.xout[eb + j] = __fadd_rn(no, dl);
            a.u[eb + j] = __fadd_rn(__fsub_rn(zpt[j], zt[j]), dl);
        }
    }
}

// L2 factors (CTA 0, thread j per component j < D): displacement
// -lambda / (rho + lambda) n, n = y - Delta (z - u on the call's first pass).
// Returns the sum of the factors' new displacements on component j.
template <bool GEN>
static __device__ __forceinline__ float hinge_l2(const HingeArgs &a, const PassMode pm, int j, float *l2d, float *l2s,
                                                 const float *zt, const float *zpt, const float *yt,
                                                 const float *ypt, double &pri) {
    const int MODE = GEN ? pm.mode : (int)T_MID;
    const bool RELOAD = GEN && pm.reload;
    const bool SAVE = GEN && pm.save;
    const bool CHK = MODE == T_CHK || MODE == T_FINAL;
    float S = 0.f;
    for (int f = 0; f < a.nl2; ++f) {
        const float q = __fdiv_rn(-a.lam[f], __fadd_rn(a.rho, a.lam[f]));
        const size_t e = (size_t)a.l2_e0 + (size_t)j * a.l2_nf + f;
        float &dl = l2d[f * kHingeD + j];
        if (CHK) {
            const float no = RELOAD ? __fsub_rn(zpt[j], a.u[e]) : __fsub_rn(ypt[j], l2s[f * kHingeD + j]);
            const float xo = __fadd_rn(no, dl);
            const float uo = __fadd_rn(__fsub_rn(zpt[j], zt[j]), dl);
            const float d = __fsub_rn(xo, zt[j]);
            pri += (double)__fmul_rn(d, d);
            a.xout[e] = xo;
            a.u[e] = uo;
            a.l2res[f * kHingeD + j] = dl;
        }
        if (MODE == T_FINAL) continue;
        if (SAVE) l2s[f * kHingeD + j] = dl;
        const float n = MODE == T_FIRST ? __fsub_rn(zt[j], a.u[e]) : __fsub_rn(yt[j], dl);
        dl = __fmul_rn(q, n);
        S = __fadd_rn(S, dl);
    }
    return S;
}

__global__ void __launch_bounds__(kHingeWarps * 32, 1) k_hinge_sweep(const HingeArgs a) {
    extern __shared__ __align__(16) unsigned char hsm[];
    const HingeCta C = a.cta[blockIdx.x];
    const HingeSmem L = hinge_smem_layout(a.rows_max);
    float *Xs = reinterpret_cast<float *>(hsm + L.X);
    float4 *metas = reinterpret_cast<float4 *>(hsm + L.meta);
    float *zt = reinterpret_cast<float *>(hsm + L.z);
    float *zpt = reinterpret_cast<float *>(hsm + L.zp);
    float *yt = reinterpret_cast<float *>(hsm + L.y);
    float *ypt = reinterpret_cast<float *>(hsm + L.yp);
    float *stg = reinterpret_cast<float *>(hsm + L.stg);
    float *l2d = reinterpret_cast<float *>(hsm + L.l2d);
    float *l2s = reinterpret_cast<float *>(hsm + L.l2s);
    unsigned long long *pv = reinterpret_cast<unsigned long long *>(hsm + L.pv);
    __shared__ double s_res[2];
    __shared__ int s_ok;
    __shared__ int s_dec[2];
    __shared__ ResidualTest s_rt[2];   // primal, dual; read by thread 0 at checks
    if (threadIdx.x == 0) {
        const double E = a.E > 0 ? (double)a.E : 1.0;
        s_rt[0].init(E, a.tol_pri);
        s_rt[1].init(E, a.tol_dual);
    }

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int gi = warp * 4 + (lane >> 3), m = lane & 7;
    const int D = a.D;
    const int NV = D + 1;   // variables: w_0 .. w_{D-1}, b (index D)

    // this CTA's data rows and per-factor constants, once per launch
    {
        const float4 *src = reinterpret_cast<const float4 *>(a.X + (size_t)C.f0 * kHingeD);
        float4 *dst = reinterpret_cast<float4 *>(Xs);
        for (int q = threadIdx.x; q < C.nf * (kHingeD / 4); q += blockDim.x) dst[q] = src[q];
        for (int i = threadIdx.x; i < C.nf; i += blockDim.x) metas[i] = a.meta[C.f0 + i];
    }
    for (int j = threadIdx.x; j < 80; j += blockDim.x) {
        float z0 = 0.f, zp0 = 0.f;
        if (j < NV) {
            const int v = j < D ? a.vw + j : a.vb;
            z0 = a.zin[v];
            zp0 = a.resume ? a.zpin[v] : z0;
        }
        zt[j] = z0;
        zpt[j] = zp0;
        yt[j] = a.resume ? __fmaf_rn(2.f, z0, -zp0) : 0.f;
        ypt[j] = 0.f;
        pv[j] = 0ull;   // the words are zeroed before the launch
        pv[80 + j] = 0ull;
    }
    if (blockIdx.x == 0)
        for (int q = threadIdx.x; q < kHingeMaxL2 * kHingeD; q += blockDim.x) {
            const int f = q / kHingeD, j = q % kHingeD;
            l2d[q] = (a.resume && f < a.nl2 && j < D) ? a.l2res[q] : 0.f;
            l2s[q] = 0.f;
        }
    float g[kHingeK];
    #pragma unroll
    for (int k = 0; k < kHingeK; ++k) {
        const int i = gi + k * kHingeGroups;
        g[k] = (a.resume && i < C.nf) ? a.gres[C.f0 + i] : 0.f;
    }
    __syncthreads();

    const unsigned long long G = (unsigned long long)a.G;
    const float inv_fix = kTileFixInv;
    bool skip = a.skip_block == (int)blockIdx.x;
    const bool res1 = a.resume != 0;
    int nchk = 0;   // checks so far: their residual partials alternate between two buffers
    for (long long it = 1; it <= a.K + 1; ++it) {
        const bool fin = it == a.K + 1;
        const bool pend = it > 1;
        const bool chk = fin || (pend && (a.k0 + it - 1) % a.check_every == 0);
        const bool save = (pend || res1) && !fin && (it == a.K || (a.k0 + it) % a.check_every == 0);
        const bool reload = it == 2 && !res1;
        double pri = 0.0, dual = 0.0;
        if (threadIdx.x == 0) s_ok = 1;
        __syncthreads();
        if (pend && threadIdx.x < NV) {
            // z <- z + sum / deg from the words of the previous pass: every
            // CTA holds every variable, so the word of the previous pass's
            // parity is complete when it counts G contributions more than
            // when this CTA read it two passes before (see kTileCountUnit)
            const int j = threadIdx.x;
            const int par = (int)((it - 1) & 1);
            const unsigned long long *src = a.acc + (size_t)par * NV * kHingeAccStride + (size_t)j * kHingeAccStride;
            const unsigned long long p = pv[par * 80 + j];
            unsigned long long w = ld_relaxed_u64(src);
            if (tile_count(w - p) != (unsigned)G) {
                const unsigned long long t0 = global_ns();
                unsigned int spins = 0;
                for (;;) {
                    w = ld_relaxed_u64(src);
                    if (tile_count(w - p) == (unsigned)G) break;
                    if ((++spins & 63u) == 0u &&
                        (*(volatile int *)&a.sync->error ||
                         global_ns() - t0 > (unsigned long long)a.timeout_ns || spins > (1u << 30))) {
                        atomicCAS(&a.sync->error, 0, kETimeout);
                        s_ok = 0;
                        break;
                    }
                }
            }
            pv[par * 80 + j] = w;
            const float S = __fmul_rn(__ll2float_rn((long long)(w - p - G * kTileCountUnit)), inv_fix);
            const float zo = zt[j];
            const int deg = j < D ? a.deg_w : a.deg_b;
            const float zn = __fadd_rn(zo, __fdiv_rn(S, (float)deg));
            zpt[j] = zo;
            zt[j] = zn;
            ypt[j] = yt[j];
            yt[j] = __fmaf_rn(2.f, zn, -zo);
            if (blockIdx.x == 0) {
                // CTA 0 owns the variables: stores z at checks, adds the dual residual
                if (chk) {
                    const int v = j < D ? a.vw + j : a.vb;
                    a.zout[v] = zn;
                    a.zpout[v] = zo;
                    const double dz = (double)zn - (double)zo;
                    dual += (double)deg * (double)a.rho * (double)a.rho * dz * dz;
                }
            }
        }
        __syncthreads();
        if (!s_ok) return;   // a wait ran out of time (error word set)
        PassMode pm;
        pm.mode = !pend ? (res1 ? T_MID : T_FIRST) : fin ? T_FINAL : chk ? T_CHK : T_MID;
        pm.reload = reload && (chk || fin);
        pm.save = save;
        pm.it = it;
        const bool plain = pm.mode == T_MID && !pm.save;
        float acc[8], accb;
        if (plain) hinge_factors<false>(a, pm, C, gi, m, g, Xs, metas, zt, zpt, yt, ypt, acc, accb, pri);
        else hinge_factors<true>(a, pm, C, gi, m, g, Xs, metas, zt, zpt, yt, ypt, acc, accb, pri);
        if (!fin) {
            // the warp's four groups, then the CTA's warps in order
            #pragma unroll
            for (int c = 0; c < 8; ++c) {
                acc[c] = __fadd_rn(acc[c], __shfl_xor_sync(0xffffffffu, acc[c], 8));
                acc[c] = __fadd_rn(acc[c], __shfl_xor_sync(0xffffffffu, acc[c], 16));
            }
            accb = __fadd_rn(accb, __shfl_xor_sync(0xffffffffu, accb, 8));
            accb = __fadd_rn(accb, __shfl_xor_sync(0xffffffffu, accb, 16));
            if (lane < 8) {
                #pragma unroll
                for (int c = 0; c < 8; ++c) stg[warp * 68 + hcomp(lane, c)] = acc[c];
                if (lane == 0) stg[warp * 68 + 64] = accb;
            }
        }
        __syncthreads();
        if (threadIdx.x < NV) {
            const int j = threadIdx.x;
            float S = 0.f;
            if (!fin) {
                const int js = j < D ? j : 64;
                for (int w = 0; w < kHingeWarps; ++w) S = __fadd_rn(S, stg[w * 68 + js]);
            }
            if (blockIdx.x == 0 && j < D && a.nl2 > 0) {
                const float s2 = plain ? hinge_l2<false>(a, pm, j, l2d, l2s, zt, zpt, yt, ypt, pri)
                                       : hinge_l2<true>(a, pm, j, l2d, l2s, zt, zpt, yt, ypt, pri);
                S = __fadd_rn(S, s2);
            }
            if (!fin && !skip) {
                long long q = 0;
                if (fabsf(S) < kTileFixMax) q = __float2ll_rn(__fmul_rn(S, kTileFixScale));
                else atomicOr(&a.sync->overflow, 1);
                // one contribution: its count and its value in one addition
                red_add_u64(a.acc + (size_t)(it & 1) * NV * kHingeAccStride + (size_t)j * kHingeAccStride,
                            kTileCountUnit + (unsigned long long)q);
            }
        }
        if (chk) {
            // the CTA's two sums as float pairs, one float4 per CTA and check parity
            const float4 bs = block_sum2_ff(pri, dual);
            if (threadIdx.x == 0) reinterpret_cast<float4 *>(a.res)[(size_t)(nchk & 1) * a.G + blockIdx.x] = bs;
        }
        // the grid-wide barrier only where the residual decision needs every
        // CTA's partials; otherwise the next pass's polls are the wait
        if (!chk) {
            skip = false;
            continue;
        }
        ++nchk;
        if (!tile_barrier(a.sync, G * (unsigned long long)nchk, a.timeout_ns, skip)) return;
        skip = false;
        {
            if (threadIdx.x < 32) {
                const float4 *r4 = reinterpret_cast<const float4 *>(a.res) + (size_t)((nchk - 1) & 1) * a.G;
                const float2 tp = warp_sum_partial_ff(r4, a.G, 0);
                const float2 td = warp_sum_partial_ff(r4, a.G, 1);
                if (threadIdx.x == 0) {
                    const bool finite = isfinite(tp.x) && isfinite(td.x) && *(volatile int *)&a.sync->overflow == 0;
                    const bool conv = finite && s_rt[0].pass(tp.x, tp.y) && s_rt[1].pass(td.x, td.y);
                    s_dec[0] = finite;
                    s_dec[1] = conv;
                    if (!finite || conv || fin) {   // the reported values, in FP64
                        s_res[0] = sqrt(((double)tp.x + (double)tp.y) / s_rt[0].E);
                        s_res[1] = sqrt(((double)td.x + (double)td.y) / s_rt[1].E);
                    }
                }
            }
            __syncthreads();
            CheckOut c;
            c.rp = s_res[0];
            c.rd = s_res[1];
            const bool finite = s_dec[0] != 0;
            c.status = finite ? 0 : kENonFinite;
            c.stop = !finite || s_dec[1] != 0;
            if (c.stop || fin) {
                hinge_state(a, C, it, pm.reload, Xs, zt, zpt, ypt);
                if (blockIdx.x == 0 && threadIdx.x == 0) {
                    Ctl *ctl = a.ctl;
                    ctl->iters = it - 1;
                    ctl->r_pri = c.rp;
                    ctl->r_dual = c.rd;
                    int st = c.status;
                    if (st == 0 && !c.stop && (a.tol_pri > 0.0 || a.tol_dual > 0.0)) st = kEBudget;
                    ctl->status = st;
                    ctl->xpar = a.xw;
                    ctl->zpar = a.zw;
                    ctl->checked = 1;
                    __threadfence();
                    *(volatile int *)&ctl->done = 1;
                }
                return;
            }
            __syncthreads();
        }
    }
}

// ---------------------------------------------------------------------------
// Latency floor of one pass on the same grid (a measurement, not part of a
// solve).  MODE 0: the grid-wide barrier alone (what a checked pass adds).
// MODE 1: what an unchecked pass does besides the operators -- every CTA
// adds one contribution (count, value 0) to each of the D + 1 variables'
// words, then polls the words until every CTA's contribution of the pass is
// in.  Needs the words zeroed before the launch.
// ---------------------------------------------------------------------------
template <int MODE>
__global__ void __launch_bounds__(kHingeWarps * 32, 1) k_hinge_floor(const HingeArgs a, long long iters) {
    __shared__ unsigned long long s_pv[2 * 80];
    __shared__ int s_ok;
    const int NV = a.D + 1;
    for (int j = threadIdx.x; j < 2 * 80; j += blockDim.x) s_pv[j] = 0ull;
    __syncthreads();
    const unsigned long long G = (unsigned long long)a.G;
    for (long long it = 1; it <= iters; ++it) {
        if (MODE == 1) {
            const int par = (int)(it & 1);
            if (threadIdx.x == 0) s_ok = 1;
            __syncthreads();
            if (threadIdx.x < NV) {
                const int j = threadIdx.x;
                unsigned long long *w = a.acc + (size_t)par * NV * kHingeAccStride + (size_t)j * kHingeAccStride;
                red_add_u64(w, kTileCountUnit);
                const unsigned long long p = s_pv[par * 80 + j];
                unsigned long long v = ld_relaxed_u64(w);
                const unsigned long long t0 = global_ns();
                unsigned int spins = 0;
                while (tile_count(v - p) != (unsigned)G) {
                    if ((++spins & 63u) == 0u &&
                        (*(volatile int *)&a.sync->error || global_ns() - t0 > (unsigned long long)a.timeout_ns ||
                         spins > (1u << 30))) {
                        atomicCAS(&a.sync->error, 0, kETimeout);
                        s_ok = 0;
                        break;
                    }
                    v = ld_relaxed_u64(w);
                }
                s_pv[par * 80 + j] = v;
            }
            __syncthreads();
            if (!s_ok) return;
        } else if (!tile_barrier(a.sync, G * (unsigned long long)it, a.timeout_ns, false)) {
            return;
        }
    }
}

cudaError_t hinge_floor_launch(const HingeArgs &a, long long iters, int mode, cudaStream_t s) {
    const void *fn = mode == 0 ? (const void *)k_hinge_floor<0> : (const void *)k_hinge_floor<1>;
    void *args[] = {(void *)&a, (void *)&iters};
    return cudaLaunchCooperativeKernel(fn, dim3(a.G), dim3(kHingeWarps * 32), args, 0, s);
}

cudaError_t hinge_sweep_launch(const HingeArgs &a, int smem, cudaStream_t s) {
    cudaError_t e = cudaFuncSetAttribute((const void *)k_hinge_sweep, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    void *args[] = {(void *)&a};
    // cooperative: the grid must be co-resident for the grid-wide barrier
    return cudaLaunchCooperativeKernel((const void *)k_hinge_sweep, dim3(a.G), dim3(kHingeWarps * 32), args,
                                       (size_t)smem, s);
}

}  // namespace fga
