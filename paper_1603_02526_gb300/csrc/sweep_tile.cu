// sweep_tile.cu -- the disk-tile sweep: Algorithm 2 on a circle-packing
// graph (Sec. V-A, Appendix A operators) in FP32, one persistent launch per
// call, the per-edge state of the disk pairs held in registers.
//
// Work: a unit is 32 row disks x 8 column disks of the pair matrix; lane l
// of the warp that owns it holds the u of its 8 pairs (48 values) for the
// whole launch.  x is not stored between iterations: with the deferred
// update of Algorithm 2, iteration k needs x^{k-1} = Prox(z^{k-2} - u^{k-2}),
// which the lane recomputes from u and the z two iterations back (the same
// operations on the same operands, so the same bits).  Per iteration a lane
// then runs, for each of its 8 pairs,
//   u += alpha (x^{k-1} - z^{k-1}),  n = z^{k-1} - u,  x^k = Prox(n),
//   m = x^k + u,
// adds m of its row disk in registers and leaves m of the column disk for a
// fixed shuffle reduce-scatter over the 32 lanes (27 shuffles per unit).
//
// z-update (deterministic, no float atomics): each CTA sums the staged unit
// and local-factor contributions per variable in a fixed order and writes
// one partial per (CTA, variable) into a variable-major array; after the
// grid-wide barrier every CTA sums, for each variable of its z table, that
// variable's partials in CTA order -- every CTA obtains the same bits.  One
// grid barrier per iteration.  The residuals (FP64) ride on the same
// barrier: the check of iteration k-1 is evaluated during iteration k.
#include <cuda_runtime.h>
#include <stdint.h>

#include "sweep.cuh"
#include "tile_internal.h"

namespace fga {

enum TileMode : int { T_FIRST = 0, T_MID = 1, T_CHK = 2, T_FINAL = 3 };

// ---------------------------------------------------------------------------
// operators (Appendix A), FP32, one rho.  Explicit round-to-nearest
// intrinsics pin every rounding, so a recomputed x has the bits of the first
// evaluation whatever the surrounding code.
// ---------------------------------------------------------------------------

// No-collision operator on (c1, r1, c2, r2): with one rho every share of the
// displacement D = max(0, r1 + r2 - |c1 - c2|) is D/4; centres move apart
// along (c2 - c1)/|c2 - c1| ((1, 0) when they coincide), radii shrink.
// D <= 0 gives t = 0 and x = n exactly.
static __device__ __forceinline__ void tile_prox_pair(const float (&n)[6], float (&x)[6]) {
    const float dx = __fsub_rn(n[3], n[0]);
    const float dy = __fsub_rn(n[4], n[1]);
    const float d2 = __fmaf_rn(dx, dx, __fmul_rn(dy, dy));
    const bool pos = d2 > 0.f;
    const float rd = rsqrtf(pos ? d2 : 1.f);
    const float D = __fsub_rn(__fadd_rn(n[2], n[5]), __fmul_rn(d2, rd));
    const float t = __fmul_rn(0.25f, fmaxf(D, 0.f));
    const float hx = pos ? __fmul_rn(dx, rd) : 1.f;
    const float hy = pos ? __fmul_rn(dy, rd) : 0.f;
    x[0] = __fmaf_rn(-t, hx, n[0]);
    x[1] = __fmaf_rn(-t, hy, n[1]);
    x[2] = __fsub_rn(n[2], t);
    x[3] = __fmaf_rn(t, hx, n[3]);
    x[4] = __fmaf_rn(t, hy, n[4]);
    x[5] = __fsub_rn(n[5], t);
}

// Wall: keep the disk in the half-plane Q.(c - V) >= r.  With one rho the
// violation h < 0 is removed by g = -h / (|Q|^2 + 1): c += g Q, r -= g.
static __device__ __forceinline__ void tile_prox_wall(const float (&n)[3], const float *p, float (&x)[3]) {
    const float h = __fsub_rn(__fmaf_rn(p[0], __fsub_rn(n[0], p[2]), __fmul_rn(p[1], __fsub_rn(n[1], p[3]))), n[2]);
    const float g = __fmul_rn(-fminf(h, 0.f), p[4]);
    x[0] = __fmaf_rn(g, p[0], n[0]);
    x[1] = __fmaf_rn(g, p[1], n[1]);
    x[2] = __fsub_rn(n[2], g);
}

// Radius rewards: linear -w r gives n + w / rho; the area reward -r^2 / 2
// gives rho n / (rho - 1).
static __device__ __forceinline__ float tile_prox_radius(int type, float n, float p0) {
    return type == 2 ? __fadd_rn(n, p0) : __fmul_rn(p0, n);
}

// ---------------------------------------------------------------------------
// grid barrier: one counter that only grows; CTA b waits until it reaches
// G x (iterations so far).  Bounded by timeout_ns and a spin count; on
// expiry the CTA sets the error word and every CTA leaves.
// ---------------------------------------------------------------------------
static __device__ __forceinline__ void red_release_add_u64(unsigned long long *p, unsigned long long v) {
    asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
static __device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

static __device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// The CTA's writes before the barrier are ordered by bar.sync and the
// cumulative release of the arrival; the waiting thread polls with relaxed
// loads and takes one acquire load once the count is reached, which orders
// the CTA's later reads (through bar.sync) after every CTA's writes.
static __device__ __forceinline__ bool tile_barrier(TileSync *s, unsigned long long target, long long timeout_ns,
                                                    bool skip) {
    __shared__ int s_err;
    __syncthreads();
    if (threadIdx.x == 0) {
        int err = 0;
        if (!skip) red_release_add_u64(&s->count, 1ull);
        if (ld_relaxed_u64(&s->count) < target) {
            const unsigned long long t0 = global_ns();
            unsigned int spins = 0;
            while (ld_relaxed_u64(&s->count) < target) {
                ++spins;
                if ((spins & 63u) == 0u) {
                    if (*(volatile int *)&s->error) { err = 1; break; }
                    if (global_ns() - t0 > (unsigned long long)timeout_ns || spins > (1u << 30)) {
                        atomicExch(&s->error, kETimeout);
                        err = 1;
                        break;
                    }
                }
            }
        }
        (void)ld_acquire_u64(&s->count);
        if (!err && *(volatile int *)&s->error) err = 1;
        s_err = err;
    }
    __syncthreads();
    return s_err == 0;
}

// ---------------------------------------------------------------------------
// z gather: z of every slot-var from its partials (previous iteration),
// the old z kept as z_prev; owners write z out (checks) and add the dual
// residual rho^2 (z - z_prev)^2 of their variables.
// ---------------------------------------------------------------------------
template <bool CHK>
static __device__ __forceinline__ void tile_gather(const TileArgs &a, int nsv, const int4 *sv, const float *zden,
                                                   float *zt, float *zpt, int rbuf, double &dual) {
    const float4 *src = reinterpret_cast<const float4 *>(a.tpart + (size_t)rbuf * a.ptot);
    for (int i = threadIdx.x; i < nsv; i += blockDim.x) {
        const int4 d = sv[i];
        float S = 0.f;
        int p = d.y >> 2;
        const int pe = d.z >> 2;
        for (; p + 4 <= pe; p += 4) {
            float4 t[4];
            #pragma unroll
            for (int j = 0; j < 4; ++j) t[j] = __ldcg(src + p + j);
            #pragma unroll
            for (int j = 0; j < 4; ++j) {
                S = __fadd_rn(S, t[j].x);
                S = __fadd_rn(S, t[j].y);
                S = __fadd_rn(S, t[j].z);
                S = __fadd_rn(S, t[j].w);
            }
        }
        for (; p < pe; ++p) {
            const float4 t = __ldcg(src + p);
            S = __fadd_rn(S, t.x);
            S = __fadd_rn(S, t.y);
            S = __fadd_rn(S, t.z);
            S = __fadd_rn(S, t.w);
        }
        const float zn = __fdiv_rn(S, zden[i]);
        const int s = i / 3, q = i - 3 * s;
        const float zo = zt[4 * s + q];
        zpt[4 * s + q] = zo;
        zt[4 * s + q] = zn;
        if (CHK && d.w < 0) {
            a.zout[d.x] = zn;
            const double dz = (double)zn - (double)zo;
            dual += __ldg(a.srho2 + d.x) * dz * dz;
        }
    }
}

// ---------------------------------------------------------------------------
// one unit (one warp): the iteration of Algorithm 2 on its <= 256 pairs
// ---------------------------------------------------------------------------
template <int MODE>
static __device__ __forceinline__ void tile_unit(const TileArgs &a, int unit, int lane, int rs, unsigned msk,
                                                 float (&u)[8][6], const float4 *z4, const float4 *zp4, float *stg_w,
                                                 double &pri) {
    const uint4 cw = __ldg(reinterpret_cast<const uint4 *>(a.colslot) + unit);
    const unsigned cs[8] = {cw.x & 0xffffu, cw.x >> 16, cw.y & 0xffffu, cw.y >> 16,
                            cw.z & 0xffffu, cw.z >> 16, cw.w & 0xffffu, cw.w >> 16};
    const float4 zr = z4[rs];
    float4 zrp = make_float4(0.f, 0.f, 0.f, 0.f);
    if (MODE != T_FIRST) zrp = zp4[rs];
    const size_t ubase = (size_t)a.pair_ebase + (size_t)unit * kUnitEdges + lane;
    float ar0 = 0.f, ar1 = 0.f, ar2 = 0.f;
    float col[8][3];
    const float al = a.alpha;
    #pragma unroll
    for (int c = 0; c < 8; ++c) {
        const bool on = (msk >> c) & 1u;
        const float4 zc = z4[cs[c]];
        const float z[6] = {zr.x, zr.y, zr.z, zc.x, zc.y, zc.z};
        if (MODE != T_FIRST) {
            // deferred update of the previous iteration, x^{k-1} recomputed
            const float4 zcp = zp4[cs[c]];
            const float zp[6] = {zrp.x, zrp.y, zrp.z, zcp.x, zcp.y, zcp.z};
            float no[6], xo[6];
            #pragma unroll
            for (int k = 0; k < 6; ++k) no[k] = __fsub_rn(zp[k], u[c][k]);
            tile_prox_pair(no, xo);
            #pragma unroll
            for (int k = 0; k < 6; ++k) {
                const float d = __fsub_rn(xo[k], z[k]);
                if (MODE >= T_CHK && on) {
                    const double dd = (double)xo[k] - (double)z[k];
                    pri += dd * dd;
                }
                u[c][k] = on ? __fmaf_rn(al, d, u[c][k]) : u[c][k];
            }
            if (MODE >= T_CHK) {
                #pragma unroll
                for (int k = 0; k < 6; ++k) {
                    a.xout[ubase + (c * 6 + k) * 32] = xo[k];
                    a.u[ubase + (c * 6 + k) * 32] = u[c][k];
                }
            }
        }
        if (MODE != T_FINAL) {
            float n[6], x[6];
            #pragma unroll
            for (int k = 0; k < 6; ++k) n[k] = __fsub_rn(z[k], u[c][k]);
            tile_prox_pair(n, x);
            float m[6];
            #pragma unroll
            for (int k = 0; k < 6; ++k) m[k] = on ? __fadd_rn(x[k], u[c][k]) : 0.f;
            ar0 = __fadd_rn(ar0, m[0]);
            ar1 = __fadd_rn(ar1, m[1]);
            ar2 = __fadd_rn(ar2, m[2]);
            col[c][0] = m[3];
            col[c][1] = m[4];
            col[c][2] = m[5];
        }
    }
    if (MODE == T_FINAL) return;
    // row disks: one partial per lane
    stg_w[lane] = ar0;
    stg_w[32 + lane] = ar1;
    stg_w[64 + lane] = ar2;
    // column disks: reduce-scatter over the lanes.  Step s halves the
    // columns a lane keeps and adds the partner's value of the kept ones.
    const unsigned FULL = 0xffffffffu;
    const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4;
    float h4[4][3];
    #pragma unroll
    for (int i = 0; i < 4; ++i) {
        #pragma unroll
        for (int q = 0; q < 3; ++q) {
            const float keep = b4 ? col[i + 4][q] : col[i][q];
            const float send = b4 ? col[i][q] : col[i + 4][q];
            h4[i][q] = __fadd_rn(keep, __shfl_xor_sync(FULL, send, 16));
        }
    }
    float h2[2][3];
    #pragma unroll
    for (int i = 0; i < 2; ++i) {
        #pragma unroll
        for (int q = 0; q < 3; ++q) {
            const float keep = b3 ? h4[i + 2][q] : h4[i][q];
            const float send = b3 ? h4[i][q] : h4[i + 2][q];
            h2[i][q] = __fadd_rn(keep, __shfl_xor_sync(FULL, send, 8));
        }
    }
    float h1[3];
    #pragma unroll
    for (int q = 0; q < 3; ++q) {
        const float keep = b2 ? h2[1][q] : h2[0][q];
        const float send = b2 ? h2[0][q] : h2[1][q];
        h1[q] = __fadd_rn(keep, __shfl_xor_sync(FULL, send, 4));
        h1[q] = __fadd_rn(h1[q], __shfl_xor_sync(FULL, h1[q], 2));
        h1[q] = __fadd_rn(h1[q], __shfl_xor_sync(FULL, h1[q], 1));
    }
    // lane holds the full sums of column 4 b4 + 2 b3 + b2; lanes 0..2 of
    // each group of four write one component each
    const int cc = (b4 ? 4 : 0) + (b3 ? 2 : 0) + (b2 ? 1 : 0);
    const int q = lane & 3;
    if (q < 3) stg_w[96 + q * 8 + cc] = q == 0 ? h1[0] : q == 1 ? h1[1] : h1[2];
}

// ---------------------------------------------------------------------------
// walls and radius rewards (one thread each, u in global memory)
// ---------------------------------------------------------------------------
template <int MODE>
static __device__ __forceinline__ void tile_local(const TileArgs &a, const TileLocal &L, float *ul, const float *zt,
                                                  const float *zpt, float *stg, double &pri) {
    const float al = a.alpha;
    if (L.type == 1) {
        float u[3], z[3];
        #pragma unroll
        for (int k = 0; k < 3; ++k) {
            u[k] = ul[k];
            z[k] = zt[4 * L.slot + k];
        }
        if (MODE != T_FIRST) {
            float no[3], xo[3];
            #pragma unroll
            for (int k = 0; k < 3; ++k) no[k] = __fsub_rn(zpt[4 * L.slot + k], u[k]);
            tile_prox_wall(no, L.p, xo);
            #pragma unroll
            for (int k = 0; k < 3; ++k) {
                const float d = __fsub_rn(xo[k], z[k]);
                if (MODE >= T_CHK) {
                    const double dd = (double)xo[k] - (double)z[k];
                    pri += dd * dd;
                }
                u[k] = __fmaf_rn(al, d, u[k]);
                ul[k] = u[k];
                if (MODE >= T_CHK) {
                    a.xout[L.e0 + k] = xo[k];
                    a.u[L.e0 + k] = u[k];
                }
            }
        }
        if (MODE != T_FINAL) {
            float n[3], x[3];
            #pragma unroll
            for (int k = 0; k < 3; ++k) n[k] = __fsub_rn(z[k], u[k]);
            tile_prox_wall(n, L.p, x);
            #pragma unroll
            for (int k = 0; k < 3; ++k) stg[L.stg + k] = __fadd_rn(x[k], u[k]);
        }
    } else {
        float u = ul[0];
        const float z = zt[4 * L.slot + 2];
        if (MODE != T_FIRST) {
            const float xo = tile_prox_radius(L.type, __fsub_rn(zpt[4 * L.slot + 2], u), L.p[0]);
            const float d = __fsub_rn(xo, z);
            if (MODE >= T_CHK) {
                const double dd = (double)xo - (double)z;
                pri += dd * dd;
            }
            u = __fmaf_rn(al, d, u);
            ul[0] = u;
            if (MODE >= T_CHK) {
                a.xout[L.e0] = xo;
                a.u[L.e0] = u;
            }
        }
        if (MODE != T_FINAL) {
            const float x = tile_prox_radius(L.type, __fsub_rn(z, u), L.p[0]);
            stg[L.stg] = __fadd_rn(x, u);
        }
    }
}

// Walls and rewards go to every warp in turn (item i: warp i mod warps,
// lane i / warps), after the warp's unit.
template <int MODE>
static __device__ __forceinline__ void tile_work(const TileArgs &a, int nloc, const TileLocal *loc, float *uloc,
                                                 bool has_unit, int unit, int lane, int rs, unsigned msk,
                                                 float (&u)[8][6], const float4 *z4, const float4 *zp4, float *stg,
                                                 double &pri) {
    const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (has_unit) tile_unit<MODE>(a, unit, lane, rs, msk, u, z4, zp4, stg + warp * kUnitStage, pri);
    const float *zt = reinterpret_cast<const float *>(z4);
    const float *zpt = reinterpret_cast<const float *>(zp4);
    for (int i = lane * nw + warp; i < nloc; i += 32 * nw) tile_local<MODE>(a, loc[i], uloc + 4 * i, zt, zpt, stg, pri);
}

// ---------------------------------------------------------------------------
// the kernel: iterations 1..K of one call, then the deferred update of
// iteration K (with its residual check), in one cooperative launch
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kTileMaxWarps * 32, 1) k_tile_sweep(const TileArgs a) {
    extern __shared__ __align__(16) unsigned char tsm[];
    const TileSmem L = tile_smem_layout(a.smax, a.svmax, a.locmax, a.clmax, a.stgmax);
    float4 *z4 = reinterpret_cast<float4 *>(tsm + L.z4);
    float4 *zp4 = reinterpret_cast<float4 *>(tsm + L.zp4);
    int4 *sv = reinterpret_cast<int4 *>(tsm + L.sv);
    TileLocal *loc = reinterpret_cast<TileLocal *>(tsm + L.loc);
    float *uloc = reinterpret_cast<float *>(tsm + L.uloc);
    float *zden = reinterpret_cast<float *>(tsm + L.zden);
    int *cptr = reinterpret_cast<int *>(tsm + L.cptr);
    int *clist = reinterpret_cast<int *>(tsm + L.clist);
    float *stg = reinterpret_cast<float *>(tsm + L.stg);
    float *zt = reinterpret_cast<float *>(z4);
    float *zpt = reinterpret_cast<float *>(zp4);
    __shared__ double s_res[2];

    const TileCta C = a.cta[blockIdx.x];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const bool has_unit = warp < C.nunit;
    const int unit = C.unit0 + warp;
    int rs = 0;
    unsigned msk = 0u;
    float u[8][6];
    if (has_unit) {
        rs = a.rowslot[unit * 32 + lane];
        msk = a.mask[unit * 32 + lane];
        const size_t ubase = (size_t)a.pair_ebase + (size_t)unit * kUnitEdges + lane;
        #pragma unroll
        for (int c = 0; c < 8; ++c) {
            #pragma unroll
            for (int k = 0; k < 6; ++k) u[c][k] = a.u[ubase + (c * 6 + k) * 32];
        }
    } else {
        #pragma unroll
        for (int c = 0; c < 8; ++c) {
            #pragma unroll
            for (int k = 0; k < 6; ++k) u[c][k] = 0.f;
        }
    }
    // the CTA's tables, once per launch
    const int cbase = a.cptr[C.sv0];
    for (int i = threadIdx.x; i < C.nsv; i += blockDim.x) {
        const int4 d = a.sv[C.sv0 + i];
        sv[i] = d;
        zden[i] = a.zden[C.sv0 + i];
        const int s = i / 3, q = i - 3 * s;
        zt[4 * s + q] = a.zin[d.x];
    }
    for (int i = threadIdx.x; i <= C.nsv; i += blockDim.x) cptr[i] = a.cptr[C.sv0 + i] - cbase;
    const int ncl = a.cptr[C.sv0 + C.nsv] - cbase;
    for (int j = threadIdx.x; j < ncl; j += blockDim.x) clist[j] = a.clist[cbase + j];
    for (int i = threadIdx.x; i < C.nloc; i += blockDim.x) {
        const TileLocal l = a.loc[C.loc0 + i];
        loc[i] = l;
        uloc[4 * i] = a.u[l.e0];
        if (l.type == 1) {
            uloc[4 * i + 1] = a.u[l.e0 + 1];
            uloc[4 * i + 2] = a.u[l.e0 + 2];
        }
    }
    __syncthreads();

    const unsigned long long G = (unsigned long long)a.G;
    bool skip = a.skip_block == (int)blockIdx.x;
    for (long long it = 1; it <= a.K + 1; ++it) {
        const bool fin = it == a.K + 1;
        const bool pend = it > 1;
        const bool chk = fin || (pend && (a.k0 + it - 1) % a.check_every == 0);
        double pri = 0.0, dual = 0.0;
        if (pend) {
            if (chk) tile_gather<true>(a, C.nsv, sv, zden, zt, zpt, (int)((it - 1) & 1), dual);
            else tile_gather<false>(a, C.nsv, sv, zden, zt, zpt, (int)((it - 1) & 1), dual);
        }
        __syncthreads();
        if (!pend) tile_work<T_FIRST>(a, C.nloc, loc, uloc, has_unit, unit, lane, rs, msk, u, z4, zp4, stg, pri);
        else if (fin) tile_work<T_FINAL>(a, C.nloc, loc, uloc, has_unit, unit, lane, rs, msk, u, z4, zp4, stg, pri);
        else if (chk) tile_work<T_CHK>(a, C.nloc, loc, uloc, has_unit, unit, lane, rs, msk, u, z4, zp4, stg, pri);
        else tile_work<T_MID>(a, C.nloc, loc, uloc, has_unit, unit, lane, rs, msk, u, z4, zp4, stg, pri);
        __syncthreads();
        if (!fin) {
            // one partial per (CTA, variable): staged contributions in list order
            float *dst = a.tpart + (size_t)(it & 1) * a.ptot;
            for (int i = threadIdx.x; i < C.nsv; i += blockDim.x) {
                const int j1 = cptr[i + 1];
                float S = 0.f;
                for (int j = cptr[i]; j < j1; ++j) S = __fadd_rn(S, stg[clist[j]]);
                __stcg(dst + (sv[i].w & 0x7fffffff), S);
            }
        }
        if (chk) {
            const double sp = block_sum(pri);
            const double sd = block_sum(dual);
            if (threadIdx.x == 0) {
                double *r = a.res + (size_t)(it & 1) * 2 * a.G;
                r[blockIdx.x] = sp;
                r[a.G + blockIdx.x] = sd;
            }
        }
        if (!tile_barrier(a.sync, G * (unsigned long long)it, a.timeout_ns, skip)) return;
        skip = false;
        if (chk) {
            if (threadIdx.x < 32) {
                const double *r = a.res + (size_t)(it & 1) * 2 * a.G;
                const double sp = warp_sum_partials(r, a.G);
                const double sd = warp_sum_partials(r + a.G, a.G);
                if (threadIdx.x == 0) {
                    const double E = a.E > 0 ? (double)a.E : 1.0;
                    s_res[0] = sqrt(sp / E);
                    s_res[1] = sqrt(sd / E);
                }
            }
            __syncthreads();
            CheckOut c;
            c.rp = s_res[0];
            c.rd = s_res[1];
            const bool finite = isfinite(c.rp) && isfinite(c.rd);
            c.status = finite ? 0 : kENonFinite;
            c.stop = !finite || (c.rp <= a.tol_pri && c.rd <= a.tol_dual);
            if (c.stop || fin) {
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

int tile_max_warps() {
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, (const void *)k_tile_sweep) != cudaSuccess) return 0;
    const int w = fa.maxThreadsPerBlock / 32;
    return w < kTileMaxWarps ? w : kTileMaxWarps;
}

int tile_smem_bytes(const TilePlan &P) {
    return tile_smem_layout(P.smax, P.svmax, P.locmax, P.clmax, P.stgmax).total;
}

cudaError_t tile_sweep_launch(const TileArgs &a, int block, int smem, cudaStream_t s) {
    cudaError_t e = cudaFuncSetAttribute((const void *)k_tile_sweep, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    void *args[] = {(void *)&a};
    // cooperative: the grid must be co-resident for the grid-wide barrier
    return cudaLaunchCooperativeKernel((const void *)k_tile_sweep, dim3(a.G), dim3(block), args, (size_t)smem, s);
}

}  // namespace fga
