// sweep_tile.cu -- the disk-tile sweep: Algorithm 2 on a circle-packing
// graph (Sec. V-A, Appendix A operators) in FP32, one persistent launch per
// call, the per-edge state of the disk pairs held in registers.
//
// Displacements.  Write each operator's result as x = n + Delta.  With one
// rho, m = x + u = z + Delta (since n = z - u), so the z-update of Algorithm
// 2 is z_b <- z_b + (sum of Delta over the edges of b) / deg(b): the CTAs
// reduce displacements, which are zero for every factor that is already
// satisfied.  A disk pair's displacement has three numbers (a, b, t):
// Delta = (-a, -b, -t, a, b, -t) on (c1, r1, c2, r2).
//
// Two forms of the per-pair state, both kept in registers by the lane that
// owns the pair for the whole launch:
//  * alpha = 1: u^k = z^{k-1} - z^k + Delta^k, hence n^k = y^k - Delta^k
//    with y^k = 2 z^k - z^{k-1} per variable: the pair's state is its
//    displacement (3 values), and an iteration is one operator evaluation.
//  * any alpha: the pair keeps its 6 u values; x^{k-1} (needed by the
//    deferred u-update) is recomputed from u and z^{k-2} -- the same
//    operations on the same operands, so the same bits -- instead of being
//    stored.
// Walls and radius rewards (few) keep u in shared memory in both forms.
//
// Work: a unit is 32 row disks x 8 column disks of the pair matrix, one warp
// each; a lane adds its row disk's displacements in registers and leaves
// those of the column disks to a fixed shuffle reduce-scatter over the 32
// lanes (21 shuffles of sums, then 6 of a butterfly, per unit).
//
// z-update (deterministic, no float atomics): each CTA sums the staged unit
// and local-factor contributions per variable in a fixed order and adds
// that partial, as a 64-bit fixed-point integer together with a count of
// one, into the variable's word; integer addition is exact and associative,
// so every CTA reads the same sum whatever the order of the additions.  A
// CTA starts its next pass once each of its variables' words counts all the
// variable's holders (tile_gather): there is no grid-wide barrier on an
// unchecked pass.  A checked pass adds one, so that every CTA decides on the
// same residual sums (FP64): the check of iteration k-1 is evaluated during
// iteration k.
#include <cuda_runtime.h>
#include <stdint.h>

#include "persist.cuh"
#include "residual.cuh"
#include "sweep.cuh"
#include "tile_internal.h"

namespace fga {


// ---------------------------------------------------------------------------
// operators (Appendix A), FP32, one rho; explicit round-to-nearest
// intrinsics pin every rounding.
// ---------------------------------------------------------------------------

// No-collision operator: from dx, dy = n_c2 - n_c1 and sr = n_r1 + n_r2, the
// displacement (a, b, t): t = qw max(0, sr - |(dx, dy)|) with qw = 1/4 (the
// four equal shares of one rho; 0 for an empty pair slot), (a, b) = t times
// the unit vector along (dx, dy), or (t, 0) when the centres coincide.
static __device__ __forceinline__ void pair_disp(float dx, float dy, float sr, float qw, float &a, float &b,
                                                 float &t) {
    const float d2 = __fmaf_rn(dx, dx, __fmul_rn(dy, dy));
    const bool pos = d2 > 0.f;
    const float rd = rsqrtf(pos ? d2 : 1.f);
    const float D = __fsub_rn(sr, __fmul_rn(d2, rd));
    t = __fmul_rn(qw, fmaxf(D, 0.f));
    const float tr = __fmul_rn(t, rd);
    a = pos ? __fmul_rn(tr, dx) : t;
    b = __fmul_rn(tr, dy);
}

// Wall: keep the disk in the half-plane Q.(c - V) >= r.  With one rho the
// violation h < 0 is removed by g = -h / (|Q|^2 + 1): Delta = g (Qx, Qy, -1).
static __device__ __forceinline__ void wall_disp(const float (&n)[3], const float *p, float (&dl)[3]) {
    const float h = __fsub_rn(__fmaf_rn(p[0], __fsub_rn(n[0], p[2]), __fmul_rn(p[1], __fsub_rn(n[1], p[3]))), n[2]);
    const float g = __fmul_rn(-fminf(h, 0.f), p[4]);
    dl[0] = __fmul_rn(g, p[0]);
    dl[1] = __fmul_rn(g, p[1]);
    dl[2] = -g;
}

// Radius rewards: linear -w r: Delta = w / rho (p0); the area reward
// -r^2 / 2: x = rho n / (rho - 1), Delta = n / (rho - 1) (p0 = 1 / (rho - 1)).
static __device__ __forceinline__ float radius_disp(int type, float n, float p0) {
    return type == 2 ? p0 : __fmul_rn(p0, n);
}

// ---------------------------------------------------------------------------
// z gather: z <- z + (sum of the variable's partials) / deg, the old z kept
// as z_prev and, for the alpha = 1 form, y = 2 z - z_prev (the old y kept as
// y_prev).  Each variable's new partials are the difference between its
// accumulator word of the previous pass's parity and the value that word
// had when read two passes before (pv); the thread polls the word until
// that difference counts all the variable's holders, which is the only wait
// between the CTAs of an unchecked pass.  Owners write z
// out (checks) and add the dual residual rho^2 (z - z_prev)^2 of their
// variables.  Returns false when a poll ran out of time (the error word is
// then set and the launch ends).
// ---------------------------------------------------------------------------
template <bool CHK, bool A1>
static __device__ __forceinline__ bool tile_gather(const TileArgs &a, int nsv, const int4 *sv, const float *zden,
                                                   float *zt, float *zpt, float *yt, float *ypt,
                                                   unsigned long long *pv, int par, double &dual) {
    bool ok = true;
    const unsigned long long *src = a.acc + (size_t)par * a.ptot;
    pv += (size_t)par * nsv;
    for (int i = threadIdx.x; i < nsv; i += blockDim.x) {
        const int4 d = sv[i];
        const unsigned long long p = pv[i], want = (unsigned long long)d.y;
        unsigned long long w = ld_relaxed_u64(src + d.x);
        if (tile_count(w - p) != (unsigned)want) {
            const unsigned long long t0 = global_ns();
            unsigned int spins = 0;
            for (;;) {
                w = ld_relaxed_u64(src + d.x);
                if (tile_count(w - p) == (unsigned)want) break;
                if ((++spins & 63u) == 0u) {
                    if (*(volatile int *)&a.sync->error ||
                        global_ns() - t0 > (unsigned long long)a.timeout_ns || spins > (1u << 30)) {
                        atomicCAS(&a.sync->error, 0, kETimeout);
                        ok = false;
                        break;
                    }
                }
            }
            if (!ok) break;
        }
        pv[i] = w;
        const long long q = (long long)(w - p - want * kTileCountUnit);
        const float S = __fmul_rn(__ll2float_rn(q), kTileFixInv);
        const int s = i / 3, qq = i - 3 * s, o = 4 * s + qq;
        const float zo = zt[o];
        const float zn = __fadd_rn(zo, __fdiv_rn(S, zden[i]));
        zpt[o] = zo;
        zt[o] = zn;
        if (A1) {
            ypt[o] = yt[o];
            yt[o] = __fmaf_rn(2.f, zn, -zo);
        }
        if (CHK && d.w < 0) {
            a.zout[d.x] = zn;
            if (A1) a.zpout[d.x] = zo;
            const double dz = (double)zn - (double)zo;
            dual += __ldg(a.srho2 + d.x) * dz * dz;
        }
    }
    return ok;
}

// Register slot j of lane l holds column j ^ mp, mp = (l >> 2) & 7, of the
// unit; csp packs the z-table slots of the lane's register slots (two
// 16-bit values per word).  An empty pair slot has weight w = 0: its share
// qw = w / 4 makes its displacement exactly 0, and in the u form its u
// stays 0.
static __device__ __forceinline__ unsigned col_slot(const unsigned (&csp)[4], int c) {
    return (c & 1) ? (csp[c >> 1] >> 16) : (csp[c >> 1] & 0xffffu);
}

// Row displacements of the lane's pairs to the staging area, column ones
// reduce-scattered over the lanes.  The partner at distance 16 (8, 4)
// holds the same columns in its upper half (quarter, eighth) of slots that
// this lane holds in its lower one, so each step adds the partner's upper
// values to the lane's lower ones; the lane ends with the sums of column
// (lane >> 2) & 7.
static __device__ __forceinline__ void stage_unit(int lane, float ar0, float ar1, float ar2, const float (&col)[8][3],
                                                  float *stg_w) {
    stg_w[lane] = ar0;
    stg_w[32 + lane] = ar1;
    stg_w[64 + lane] = ar2;
    const unsigned FULL = 0xffffffffu;
    float h4[4][3];
    #pragma unroll
    for (int i = 0; i < 4; ++i) {
        #pragma unroll
        for (int q = 0; q < 3; ++q) h4[i][q] = __fadd_rn(col[i][q], __shfl_xor_sync(FULL, col[i + 4][q], 16));
    }
    float h2[2][3];
    #pragma unroll
    for (int i = 0; i < 2; ++i) {
        #pragma unroll
        for (int q = 0; q < 3; ++q) h2[i][q] = __fadd_rn(h4[i][q], __shfl_xor_sync(FULL, h4[i + 2][q], 8));
    }
    float h1[3];
    #pragma unroll
    for (int q = 0; q < 3; ++q) {
        h1[q] = __fadd_rn(h2[0][q], __shfl_xor_sync(FULL, h2[1][q], 4));
        h1[q] = __fadd_rn(h1[q], __shfl_xor_sync(FULL, h1[q], 2));
        h1[q] = __fadd_rn(h1[q], __shfl_xor_sync(FULL, h1[q], 1));
    }
    const int cc = (lane >> 2) & 7;
    const int q = lane & 3;
    if (q < 3) stg_w[96 + q * 8 + cc] = q == 0 ? h1[0] : q == 1 ? h1[1] : h1[2];
}

// ---------------------------------------------------------------------------
// one unit, alpha = 1: state D[c] = (a, b, t) of each pair.  In pass `it`
// (>= 2) D holds Delta^{it-1}.  A pass that checks also needs Delta^{it-2}:
// the pass before stores it to a.dsave (SAVE); when the previous pass was
// the call's first, the stored u is read again instead (RELOAD).
// ---------------------------------------------------------------------------
template <bool GEN>
static __device__ __forceinline__ void tile_unit_a1(const TileArgs &a, const PassMode pm, int unit, int lane, int rs, unsigned msk,
                                                    const unsigned (&csp)[4], float (&D)[8][3], const float4 *z4,
                                                    const float4 *zp4, const float4 *y4, const float4 *yp4,
                                                    float *stg_w, double &pri) {
    const int MODE = GEN ? pm.mode : (int)T_MID;
    const bool RELOAD = GEN && pm.reload;
    const bool SAVE = GEN && pm.save;
    const bool CHK = MODE == T_CHK || MODE == T_FINAL;
    const size_t ubase = (size_t)a.pair_ebase + (size_t)unit * kUnitEdges + lane;
    const size_t dbase = (size_t)unit * (kUnitEdges / 2) + lane;
    float4 zr = make_float4(0.f, 0.f, 0.f, 0.f), zpr = zr, yr = zr, ypr = zr;
    if (MODE == T_FIRST || CHK) zr = z4[rs];
    if (CHK) zpr = zp4[rs];
    if (CHK && !RELOAD) ypr = yp4[rs];
    if (MODE == T_MID || MODE == T_CHK) yr = y4[rs];
    float ar0 = 0.f, ar1 = 0.f, ar2 = 0.f;
    float col[8][3];
    #pragma unroll
    for (int c = 0; c < 8; ++c) {
        const unsigned slot = col_slot(csp, c);
        const float w = ((msk >> c) & 1u) ? 1.f : 0.f;
        if (CHK) {
            // iteration it-1: x = n^{it-2} + Delta^{it-1}, u = z_prev - z + Delta^{it-1}
            const float4 zc = z4[slot], zpc = zp4[slot];
            const float z[6] = {zr.x, zr.y, zr.z, zc.x, zc.y, zc.z};
            const float zp[6] = {zpr.x, zpr.y, zpr.z, zpc.x, zpc.y, zpc.z};
            float no[6];
            if (RELOAD) {
                #pragma unroll
                for (int k = 0; k < 6; ++k) no[k] = __fsub_rn(zp[k], a.u[ubase + (c * 6 + k) * 32]);
            } else {
                const float4 ypc = yp4[slot];
                const float pa = a.dsave[dbase + (c * 3) * 32], pb = a.dsave[dbase + (c * 3 + 1) * 32],
                            pt = a.dsave[dbase + (c * 3 + 2) * 32];
                no[0] = __fadd_rn(ypr.x, pa);
                no[1] = __fadd_rn(ypr.y, pb);
                no[2] = __fadd_rn(ypr.z, pt);
                no[3] = __fsub_rn(ypc.x, pa);
                no[4] = __fsub_rn(ypc.y, pb);
                no[5] = __fadd_rn(ypc.z, pt);
            }
            const float dl[6] = {-D[c][0], -D[c][1], -D[c][2], D[c][0], D[c][1], -D[c][2]};
            float sq = 0.f;
            #pragma unroll
            for (int k = 0; k < 6; ++k) {
                const float xo = __fadd_rn(no[k], dl[k]);
                const float d = __fsub_rn(xo, z[k]);
                sq = __fmaf_rn(d, d, sq);
                // x and u of the pairs are stored by the call's last pass and
                // by a check that also saves (its dsave then no longer holds
                // the displacements of it-2); any other check that stops the
                // call stores them afterwards (tile_store_a1), so that checks
                // that go on write nothing but the displacements
                if (MODE == T_FINAL || SAVE) {
                    a.xout[ubase + (c * 6 + k) * 32] = xo;
                    a.u[ubase + (c * 6 + k) * 32] = __fadd_rn(__fsub_rn(zp[k], z[k]), dl[k]);
                }
            }
            // the pair's squared differences in FP32, the sum over pairs in
            // FP64 (the FP64 pipe is narrow on this part)
            pri += (double)__fmul_rn(sq, w);
            // the displacements of the stored state, for a later call to
            // resume from (with the z before it, written by the owners)
            #pragma unroll
            for (int j = 0; j < 3; ++j) a.dres[dbase + (c * 3 + j) * 32] = D[c][j];
        }
        if (MODE == T_FINAL) continue;
        if (SAVE) {
            #pragma unroll
            for (int j = 0; j < 3; ++j) a.dsave[dbase + (c * 3 + j) * 32] = D[c][j];
        }
        float dx, dy, sr;
        if (MODE == T_FIRST) {
            // n = z - u from the stored u
            const float4 zc = z4[slot];
            float n[6];
            const float z[6] = {zr.x, zr.y, zr.z, zc.x, zc.y, zc.z};
            #pragma unroll
            for (int k = 0; k < 6; ++k) n[k] = __fsub_rn(z[k], a.u[ubase + (c * 6 + k) * 32]);
            dx = __fsub_rn(n[3], n[0]);
            dy = __fsub_rn(n[4], n[1]);
            sr = __fadd_rn(n[2], n[5]);
        } else {
            // n = y - Delta: n_c2 - n_c1 = (y_c2 - y_c1) - 2 (a, b), n_r1 + n_r2 = y_r1 + y_r2 + 2 t
            const float4 yc = y4[slot];
            dx = __fmaf_rn(-2.f, D[c][0], __fsub_rn(yc.x, yr.x));
            dy = __fmaf_rn(-2.f, D[c][1], __fsub_rn(yc.y, yr.y));
            sr = __fmaf_rn(2.f, D[c][2], __fadd_rn(yr.z, yc.z));
        }
        float pa, pb, pt;
        pair_disp(dx, dy, sr, __fmul_rn(0.25f, w), pa, pb, pt);
        D[c][0] = pa;
        D[c][1] = pb;
        D[c][2] = pt;
        ar0 = __fsub_rn(ar0, pa);
        ar1 = __fsub_rn(ar1, pb);
        ar2 = __fsub_rn(ar2, pt);
        col[c][0] = pa;
        col[c][1] = pb;
        col[c][2] = -pt;
    }
    if (MODE != T_FINAL) stage_unit(lane, ar0, ar1, ar2, col, stg_w);
}

// ---------------------------------------------------------------------------
// alpha = 1, after a check that stops the call: the stored state of
// iteration it-1 (x and u of the unit's pair edges), from the displacements
// of iteration it-1 (dres, written by the check pass), those of it-2 (dsave,
// or the stored u when it-2 was the call's start: RELOAD) and the pass's z
// tables -- the same operations on the same operands as a check pass that
// stores them (so the same bits).
// ---------------------------------------------------------------------------
static __device__ __forceinline__ void tile_store_a1(const TileArgs &a, bool reload, int unit, int lane, int rs,
                                                     const unsigned (&csp)[4], const float4 *z4, const float4 *zp4,
                                                     const float4 *yp4) {
    const size_t ubase = (size_t)a.pair_ebase + (size_t)unit * kUnitEdges + lane;
    const size_t dbase = (size_t)unit * (kUnitEdges / 2) + lane;
    const float4 zr = z4[rs], zpr = zp4[rs];
    const float4 ypr = reload ? make_float4(0.f, 0.f, 0.f, 0.f) : yp4[rs];
    #pragma unroll 2
    for (int c = 0; c < 8; ++c) {
        const unsigned slot = col_slot(csp, c);
        const float4 zc = z4[slot], zpc = zp4[slot];
        const float z[6] = {zr.x, zr.y, zr.z, zc.x, zc.y, zc.z};
        const float zp[6] = {zpr.x, zpr.y, zpr.z, zpc.x, zpc.y, zpc.z};
        float no[6];
        if (reload) {
            #pragma unroll
            for (int k = 0; k < 6; ++k) no[k] = __fsub_rn(zp[k], a.u[ubase + (c * 6 + k) * 32]);
        } else {
            const float4 ypc = yp4[slot];
            const float pa = a.dsave[dbase + (c * 3) * 32], pb = a.dsave[dbase + (c * 3 + 1) * 32],
                        pt = a.dsave[dbase + (c * 3 + 2) * 32];
            no[0] = __fadd_rn(ypr.x, pa);
            no[1] = __fadd_rn(ypr.y, pb);
            no[2] = __fadd_rn(ypr.z, pt);
            no[3] = __fsub_rn(ypc.x, pa);
            no[4] = __fsub_rn(ypc.y, pb);
            no[5] = __fadd_rn(ypc.z, pt);
        }
        const float da = a.dres[dbase + (c * 3) * 32], db = a.dres[dbase + (c * 3 + 1) * 32],
                    dt = a.dres[dbase + (c * 3 + 2) * 32];
        const float dl[6] = {-da, -db, -dt, da, db, -dt};
        #pragma unroll
        for (int k = 0; k < 6; ++k) {
            a.xout[ubase + (c * 6 + k) * 32] = __fadd_rn(no[k], dl[k]);
            a.u[ubase + (c * 6 + k) * 32] = __fadd_rn(__fsub_rn(zp[k], z[k]), dl[k]);
        }
    }
}

// ---------------------------------------------------------------------------
// one unit, any alpha: state u[c][k]; x^{it-1} recomputed from u and z_prev
// ---------------------------------------------------------------------------
template <bool GEN>
static __device__ __forceinline__ void tile_unit_u(const TileArgs &a, const PassMode pm, int unit, int lane, int rs, unsigned msk,
                                                   const unsigned (&csp)[4], float (&u)[8][6], const float4 *z4,
                                                   const float4 *zp4, float *stg_w, double &pri) {
    const int MODE = GEN ? pm.mode : (int)T_MID;
    const float4 zr = z4[rs];
    float4 zrp = make_float4(0.f, 0.f, 0.f, 0.f);
    if (MODE != T_FIRST) zrp = zp4[rs];
    const size_t ubase = (size_t)a.pair_ebase + (size_t)unit * kUnitEdges + lane;
    float ar0 = 0.f, ar1 = 0.f, ar2 = 0.f;
    float col[8][3];
    const float al = a.alpha;
    #pragma unroll
    for (int c = 0; c < 8; ++c) {
        const unsigned slot = col_slot(csp, c);
        const float w = ((msk >> c) & 1u) ? 1.f : 0.f;
        const float qw = __fmul_rn(0.25f, w);
        const float4 zc = z4[slot];
        const float z[6] = {zr.x, zr.y, zr.z, zc.x, zc.y, zc.z};
        if (MODE != T_FIRST) {
            // deferred update of the previous iteration, x^{it-1} recomputed
            const float4 zcp = zp4[slot];
            const float zp[6] = {zrp.x, zrp.y, zrp.z, zcp.x, zcp.y, zcp.z};
            float no[6];
            #pragma unroll
            for (int k = 0; k < 6; ++k) no[k] = __fsub_rn(zp[k], u[c][k]);
            float oa, ob, ot;
            pair_disp(__fsub_rn(no[3], no[0]), __fsub_rn(no[4], no[1]), __fadd_rn(no[2], no[5]), qw, oa, ob, ot);
            const float dl[6] = {-oa, -ob, -ot, oa, ob, -ot};
            const float aw = __fmul_rn(al, w);
            float sq = 0.f;
            #pragma unroll
            for (int k = 0; k < 6; ++k) {
                const float xo = __fadd_rn(no[k], dl[k]);
                const float d = __fsub_rn(xo, z[k]);
                if (MODE >= T_CHK) {
                    sq = __fmaf_rn(d, d, sq);
                    a.xout[ubase + (c * 6 + k) * 32] = xo;
                }
                u[c][k] = __fmaf_rn(aw, d, u[c][k]);
                if (MODE >= T_CHK) a.u[ubase + (c * 6 + k) * 32] = u[c][k];
            }
            if (MODE >= T_CHK) pri += (double)__fmul_rn(sq, w);
        }
        if (MODE != T_FINAL) {
            float n[6];
            #pragma unroll
            for (int k = 0; k < 6; ++k) n[k] = __fsub_rn(z[k], u[c][k]);
            float pa, pb, pt;
            pair_disp(__fsub_rn(n[3], n[0]), __fsub_rn(n[4], n[1]), __fadd_rn(n[2], n[5]), qw, pa, pb, pt);
            ar0 = __fsub_rn(ar0, pa);
            ar1 = __fsub_rn(ar1, pb);
            ar2 = __fsub_rn(ar2, pt);
            col[c][0] = pa;
            col[c][1] = pb;
            col[c][2] = -pt;
        }
    }
    if (MODE != T_FINAL) stage_unit(lane, ar0, ar1, ar2, col, stg_w);
}

// ---------------------------------------------------------------------------
// walls and radius rewards (one thread each, u in shared memory, any alpha)
// ---------------------------------------------------------------------------
template <bool GEN>
static __device__ __forceinline__ void tile_local(const TileArgs &a, const PassMode pm, const TileLocal &L, float *ul, const float *zt,
                                                  const float *zpt, float *stg, double &pri) {
    const int MODE = GEN ? pm.mode : (int)T_MID;
    const float al = a.alpha;
    if (L.type == 1) {
        float u[3], z[3];
        #pragma unroll
        for (int k = 0; k < 3; ++k) {
            u[k] = ul[k];
            z[k] = zt[4 * L.slot + k];
        }
        if (MODE != T_FIRST) {
            float no[3], dl[3];
            #pragma unroll
            for (int k = 0; k < 3; ++k) no[k] = __fsub_rn(zpt[4 * L.slot + k], u[k]);
            wall_disp(no, L.p, dl);
            #pragma unroll
            for (int k = 0; k < 3; ++k) {
                const float xo = __fadd_rn(no[k], dl[k]);
                const float d = __fsub_rn(xo, z[k]);
                if (MODE >= T_CHK) {
                    const double dd = (double)xo - (double)z[k];
                    pri += dd * dd;
                }
                u[k] = __fmaf_rn(al, d, u[k]);
                ul[k] = u[k];
                if (MODE >= T_CHK) {
                    a.xout[L.e0 + k] = xo;
                    a.u[L.e0 + k] = u[k];
                }
            }
        }
        if (MODE != T_FINAL) {
            float n[3], dl[3];
            #pragma unroll
            for (int k = 0; k < 3; ++k) n[k] = __fsub_rn(z[k], u[k]);
            wall_disp(n, L.p, dl);
            #pragma unroll
            for (int k = 0; k < 3; ++k) stg[L.stg + k] = dl[k];
        }
    } else {
        float u = ul[0];
        const float z = zt[4 * L.slot + 2];
        if (MODE != T_FIRST) {
            const float no = __fsub_rn(zpt[4 * L.slot + 2], u);
            const float xo = __fadd_rn(no, radius_disp(L.type, no, L.p[0]));
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
        if (MODE != T_FINAL) stg[L.stg] = radius_disp(L.type, __fsub_rn(z, u), L.p[0]);
    }
}

// The same for alpha = 1 in displacement form.  A wall's displacement is
// g (Qx, Qy, -1): its state is g; the linear reward's is the constant
// w / rho (no state); the area reward's is n / (rho - 1): its state is that
// value.  ul: [0..2] the u stored at the start of the call (read again by
// the first check, RELOAD), [3] the state, [4] the state kept for the next
// check (SAVE).  Check passes store x, u and the state as in tile_unit_a1.
template <bool GEN>
static __device__ __forceinline__ void tile_local_a1(const TileArgs &a, const PassMode pm, const TileLocal &L, int li, float *ul,
                                                     const float *zt, const float *zpt, const float *yt,
                                                     const float *ypt, float *stg, double &pri) {
    const int MODE = GEN ? pm.mode : (int)T_MID;
    const bool RELOAD = GEN && pm.reload;
    const bool SAVE = GEN && pm.save;
    const bool CHK = MODE == T_CHK || MODE == T_FINAL;
    const int o = 4 * L.slot;
    if (L.type == 1) {
        const float *p = L.p;
        if (CHK) {
            const float g = ul[3];
            const float dl[3] = {__fmul_rn(g, p[0]), __fmul_rn(g, p[1]), -g};
            float no[3];
            if (RELOAD) {
                #pragma unroll
                for (int k = 0; k < 3; ++k) no[k] = __fsub_rn(zpt[o + k], ul[k]);
            } else {
                const float gp = ul[4];
                no[0] = __fsub_rn(ypt[o], __fmul_rn(gp, p[0]));
                no[1] = __fsub_rn(ypt[o + 1], __fmul_rn(gp, p[1]));
                no[2] = __fadd_rn(ypt[o + 2], gp);
            }
            #pragma unroll
            for (int k = 0; k < 3; ++k) {
                const float xo = __fadd_rn(no[k], dl[k]);
                const float uo = __fadd_rn(__fsub_rn(zpt[o + k], zt[o + k]), dl[k]);
                const float d = __fsub_rn(xo, zt[o + k]);
                pri += (double)__fmul_rn(d, d);
                a.xout[L.e0 + k] = xo;
                a.u[L.e0 + k] = uo;
            }
            a.lres[li] = g;
        }
        if (MODE == T_FINAL) return;
        if (SAVE) ul[4] = ul[3];
        float n[3];
        if (MODE == T_FIRST) {
            #pragma unroll
            for (int k = 0; k < 3; ++k) n[k] = __fsub_rn(zt[o + k], ul[k]);
        } else {
            const float g = ul[3];
            n[0] = __fsub_rn(yt[o], __fmul_rn(g, p[0]));
            n[1] = __fsub_rn(yt[o + 1], __fmul_rn(g, p[1]));
            n[2] = __fadd_rn(yt[o + 2], g);
        }
        float dl[3];
        wall_disp(n, p, dl);
        ul[3] = -dl[2];
        #pragma unroll
        for (int k = 0; k < 3; ++k) stg[L.stg + k] = dl[k];
    } else {
        const bool quad = L.type == 3;
        if (CHK) {
            const float dl = quad ? ul[3] : L.p[0];
            float no;
            if (RELOAD) no = __fsub_rn(zpt[o + 2], ul[0]);
            else no = __fsub_rn(ypt[o + 2], quad ? ul[4] : L.p[0]);
            const float xo = __fadd_rn(no, dl);
            const float uo = __fadd_rn(__fsub_rn(zpt[o + 2], zt[o + 2]), dl);
            const float d = __fsub_rn(xo, zt[o + 2]);
            pri += (double)__fmul_rn(d, d);
            a.xout[L.e0] = xo;
            a.u[L.e0] = uo;
            a.lres[li] = ul[3];
        }
        if (MODE == T_FINAL) return;
        if (!quad) {
            stg[L.stg] = L.p[0];
            return;
        }
        if (SAVE) ul[4] = ul[3];
        const float n = MODE == T_FIRST ? __fsub_rn(zt[o + 2], ul[0]) : __fsub_rn(yt[o + 2], ul[3]);
        const float dl = __fmul_rn(L.p[0], n);
        ul[3] = dl;
        stg[L.stg] = dl;
    }
}

// Walls and rewards go to every warp in turn (item i: warp i mod warps,
// lane i / warps), after the warp's unit.
template <bool GEN, bool A1>
static __device__ __forceinline__ void tile_locals(const TileArgs &a, const PassMode pm, const TileCta &C, const TileLocal *loc,
                                                   float *uloc, int lane, const float4 *z4, const float4 *zp4,
                                                   const float4 *y4, const float4 *yp4, float *stg, double &pri) {
    const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const float *zt = reinterpret_cast<const float *>(z4);
    const float *zpt = reinterpret_cast<const float *>(zp4);
    const float *yt = reinterpret_cast<const float *>(y4);
    const float *ypt = reinterpret_cast<const float *>(yp4);
    for (int i = lane * nw + warp; i < C.nloc; i += 32 * nw) {
        if constexpr (A1)
            tile_local_a1<GEN>(a, pm, loc[i], C.loc0 + i, uloc + 8 * i, zt, zpt, yt, ypt, stg, pri);
        else
            tile_local<GEN>(a, pm, loc[i], uloc + 8 * i, zt, zpt, stg, pri);
    }
}

// Per-lane state of its pairs, for either form.
template <bool A1>
struct PairState;
template <>
struct PairState<true> {
    float D[8][3];
};
template <>
struct PairState<false> {
    float u[8][6];
};

// A unit's lane descriptors: the z-table slot of the lane's row disk, the
// mask of its pairs, and the slots of its register slots' column disks.
static __device__ __forceinline__ void unit_desc(const TileArgs &a, int unit, int lane, int &rs, unsigned &msk,
                                                 unsigned (&csp)[4]) {
    rs = a.rowslot[unit * 32 + lane];
    msk = a.mask[unit * 32 + lane];
    const int mp = (lane >> 2) & 7;
    #pragma unroll
    for (int j = 0; j < 4; ++j)
        csp[j] = (unsigned)a.colslot[unit * 8 + ((2 * j) ^ mp)] | ((unsigned)a.colslot[unit * 8 + ((2 * j + 1) ^ mp)] << 16);
}

// Several units per warp (MULTI): a unit's pair state lives in device
// memory between passes (alpha = 1: its displacements in dlive; any alpha:
// its u in the edge array) and is loaded into registers for the unit's turn.
template <bool A1>
static __device__ __forceinline__ void state_load(const TileArgs &a, int unit, int lane, PairState<A1> &ps) {
    if constexpr (A1) {
        const size_t dbase = (size_t)unit * (kUnitEdges / 2) + lane;
        #pragma unroll
        for (int c = 0; c < 8; ++c) {
            #pragma unroll
            for (int k = 0; k < 3; ++k) ps.D[c][k] = a.dlive[dbase + (c * 3 + k) * 32];
        }
    } else {
        const size_t ubase = (size_t)a.pair_ebase + (size_t)unit * kUnitEdges + lane;
        #pragma unroll
        for (int c = 0; c < 8; ++c) {
            #pragma unroll
            for (int k = 0; k < 6; ++k) ps.u[c][k] = a.u[ubase + (c * 6 + k) * 32];
        }
    }
}
template <bool A1>
static __device__ __forceinline__ void state_store(const TileArgs &a, int unit, int lane, const PairState<A1> &ps) {
    if constexpr (A1) {
        const size_t dbase = (size_t)unit * (kUnitEdges / 2) + lane;
        #pragma unroll
        for (int c = 0; c < 8; ++c) {
            #pragma unroll
            for (int k = 0; k < 3; ++k) a.dlive[dbase + (c * 3 + k) * 32] = ps.D[c][k];
        }
    } else {
        const size_t ubase = (size_t)a.pair_ebase + (size_t)unit * kUnitEdges + lane;
        #pragma unroll
        for (int c = 0; c < 8; ++c) {
            #pragma unroll
            for (int k = 0; k < 6; ++k) a.u[ubase + (c * 6 + k) * 32] = ps.u[c][k];
        }
    }
}

template <bool GEN, bool A1, bool MULTI>
static __device__ __forceinline__ void tile_pass(const TileArgs &a, const PassMode pm, const TileCta &C, const TileLocal *loc, float *uloc,
                                                 bool has_unit, int unit, int lane, int rs, unsigned msk,
                                                 const unsigned (&csp)[4], PairState<A1> &ps, const float4 *z4,
                                                 const float4 *zp4, const float4 *y4, const float4 *yp4, float *stg,
                                                 double &pri) {
    if constexpr (MULTI) {
        // the warp's units in turn: unit w, w + warps, ... of the CTA
        const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
        const int MODE = GEN ? pm.mode : (int)T_MID;
        for (int lu = warp; lu < C.nunit; lu += nw) {
            const int un = C.unit0 + lu;
            int rs_u;
            unsigned msk_u, csp_u[4];
            unit_desc(a, un, lane, rs_u, msk_u, csp_u);
            PairState<A1> pu;
            state_load<A1>(a, un, lane, pu);
            float *stg_w = stg + lu * kUnitStage;
            if constexpr (A1)
                tile_unit_a1<GEN>(a, pm, un, lane, rs_u, msk_u, csp_u, pu.D, z4, zp4, y4, yp4, stg_w, pri);
            else
                tile_unit_u<GEN>(a, pm, un, lane, rs_u, msk_u, csp_u, pu.u, z4, zp4, stg_w, pri);
            if (MODE != T_FINAL) state_store<A1>(a, un, lane, pu);
        }
    } else {
        float *stg_w = stg + (threadIdx.x >> 5) * kUnitStage;
        if (has_unit) {
            if constexpr (A1)
                tile_unit_a1<GEN>(a, pm, unit, lane, rs, msk, csp, ps.D, z4, zp4, y4, yp4, stg_w, pri);
            else
                tile_unit_u<GEN>(a, pm, unit, lane, rs, msk, csp, ps.u, z4, zp4, stg_w, pri);
        }
    }
    tile_locals<GEN, A1>(a, pm, C, loc, uloc, lane, z4, zp4, y4, yp4, stg, pri);
}

// ---------------------------------------------------------------------------
// the kernel: iterations 1..K of one call, then the deferred update of
// iteration K (with its residual check), in one cooperative launch
// ---------------------------------------------------------------------------
// MULTI: more units than warps in a CTA (larger graphs): each warp takes
// its units in turn, their state in device memory between passes.
template <bool A1, bool MULTI>
__global__ void __launch_bounds__(kTileMaxWarps * 32, 1) k_tile_sweep(const TileArgs a) {
    extern __shared__ __align__(16) unsigned char tsm[];
    const TileSmem L = tile_smem_layout(a.smax, a.svmax, a.locmax, a.clmax, a.stgmax);
    float4 *z4 = reinterpret_cast<float4 *>(tsm + L.z4);
    float4 *zp4 = reinterpret_cast<float4 *>(tsm + L.zp4);
    float4 *y4 = reinterpret_cast<float4 *>(tsm + L.y4);
    float4 *yp4 = reinterpret_cast<float4 *>(tsm + L.yp4);
    int4 *sv = reinterpret_cast<int4 *>(tsm + L.sv);
    TileLocal *loc = reinterpret_cast<TileLocal *>(tsm + L.loc);
    float *uloc = reinterpret_cast<float *>(tsm + L.uloc);
    float *zden = reinterpret_cast<float *>(tsm + L.zden);
    int *cptr = reinterpret_cast<int *>(tsm + L.cptr);
    unsigned short *clist = reinterpret_cast<unsigned short *>(tsm + L.clist);   // positions < 2^16
    float *stg = reinterpret_cast<float *>(tsm + L.stg);
    unsigned long long *pv = reinterpret_cast<unsigned long long *>(tsm + L.pv);
    float *zt = reinterpret_cast<float *>(z4);
    float *zpt = reinterpret_cast<float *>(zp4);
    float *yt = reinterpret_cast<float *>(y4);
    float *ypt = reinterpret_cast<float *>(yp4);
    __shared__ double s_res[2];
    __shared__ int s_dec[2];
    __shared__ ResidualTest s_rt[2];   // primal, dual; read by thread 0 at checks
    if (threadIdx.x == 0) {
        const double E = a.E > 0 ? (double)a.E : 1.0;
        s_rt[0].init(E, a.tol_pri);
        s_rt[1].init(E, a.tol_dual);
    }

    const TileCta C = a.cta[blockIdx.x];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const bool has_unit = !MULTI && warp < C.nunit;
    const int unit = C.unit0 + warp;
    int rs = 0;
    unsigned msk = 0u;
    unsigned csp[4] = {0u, 0u, 0u, 0u};
    PairState<A1> ps;
    if (has_unit) unit_desc(a, unit, lane, rs, msk, csp);
    if constexpr (MULTI) {
        // a call that resumes the previous one takes up its displacements
        if constexpr (A1) {
            for (int lu = warp; lu < C.nunit; lu += (int)(blockDim.x >> 5)) {
                const size_t dbase = (size_t)(C.unit0 + lu) * (kUnitEdges / 2) + lane;
                for (int j = 0; j < 24; ++j)
                    a.dlive[dbase + j * 32] = a.resume ? a.dres[dbase + j * 32] : 0.f;
            }
        }
    } else if constexpr (A1) {
        // a call that resumes the previous one takes up its displacements
        const size_t dbase = (size_t)unit * (kUnitEdges / 2) + lane;
        #pragma unroll
        for (int c = 0; c < 8; ++c) {
            #pragma unroll
            for (int k = 0; k < 3; ++k) ps.D[c][k] = (a.resume && has_unit) ? a.dres[dbase + (c * 3 + k) * 32] : 0.f;
        }
    } else {
        const size_t ubase = (size_t)a.pair_ebase + (size_t)unit * kUnitEdges + lane;
        #pragma unroll
        for (int c = 0; c < 8; ++c) {
            #pragma unroll
            for (int k = 0; k < 6; ++k) ps.u[c][k] = has_unit ? a.u[ubase + (c * 6 + k) * 32] : 0.f;
        }
    }
    // the CTA's tables, once per launch
    const int cbase = a.cptr[C.sv0];
    for (int i = threadIdx.x; i < C.nsv; i += blockDim.x) {
        const int4 d = a.sv[C.sv0 + i];
        sv[i] = d;
        pv[i] = 0ull;   // the words are zeroed before the launch
        pv[C.nsv + i] = 0ull;
        zden[i] = a.zden[C.sv0 + i];
        const int s = i / 3, q = i - 3 * s;
        const float z0 = a.zin[d.x];
        zt[4 * s + q] = z0;
        if (A1 && a.resume) {
            const float zp0 = a.zpin[d.x];
            zpt[4 * s + q] = zp0;
            yt[4 * s + q] = __fmaf_rn(2.f, z0, -zp0);
        } else {
            yt[4 * s + q] = 0.f;
        }
    }
    for (int i = threadIdx.x; i <= C.nsv; i += blockDim.x) cptr[i] = a.cptr[C.sv0 + i] - cbase;
    const int ncl = a.cptr[C.sv0 + C.nsv] - cbase;
    for (int j = threadIdx.x; j < ncl; j += blockDim.x) clist[j] = (unsigned short)a.clist[cbase + j];
    for (int i = threadIdx.x; i < C.nloc; i += blockDim.x) {
        const TileLocal l = a.loc[C.loc0 + i];
        loc[i] = l;
        uloc[8 * i] = a.u[l.e0];
        if (l.type == 1) {
            uloc[8 * i + 1] = a.u[l.e0 + 1];
            uloc[8 * i + 2] = a.u[l.e0 + 2];
        }
        uloc[8 * i + 3] = (A1 && a.resume) ? a.lres[C.loc0 + i] : 0.f;
        uloc[8 * i + 4] = 0.f;
    }
    __syncthreads();

    const unsigned long long G = (unsigned long long)a.G;
    bool skip = a.skip_block == (int)blockIdx.x;
    // resuming (alpha = 1): the first pass is an ordinary one, from the
    // displacements and the two z of the previous call's last iteration
    const bool res1 = A1 && a.resume;
    __shared__ int s_ok;
    int nchk = 0;   // checks so far: their residual partials alternate between two buffers
    for (long long it = 1; it <= a.K + 1; ++it) {
        const bool fin = it == a.K + 1;
        const bool pend = it > 1;
        const bool chk = fin || (pend && (a.k0 + it - 1) % a.check_every == 0);
        // the next pass checks: keep the displacements this pass replaces
        const bool save = A1 && (pend || res1) && !fin && (it == a.K || (a.k0 + it) % a.check_every == 0);
        const bool reload = it == 2 && !res1;
        double pri = 0.0, dual = 0.0;
        if (threadIdx.x == 0) s_ok = 1;
        __syncthreads();
        if (pend) {
            const int par = (int)((it - 1) & 1);   // the words the previous pass added into
            const bool ok = chk ? tile_gather<true, A1>(a, C.nsv, sv, zden, zt, zpt, yt, ypt, pv, par, dual)
                                : tile_gather<false, A1>(a, C.nsv, sv, zden, zt, zpt, yt, ypt, pv, par, dual);
            if (!ok) s_ok = 0;
        }
        __syncthreads();
        if (!s_ok) return;   // a wait ran out of time (error word set)
        PassMode pm;
        pm.mode = !pend ? (res1 ? T_MID : T_FIRST) : fin ? T_FINAL : chk ? T_CHK : T_MID;
        pm.reload = reload && (chk || fin);
        pm.save = save;
        pm.it = it;
        if (pm.mode == T_MID && !pm.save)
            tile_pass<false, A1, MULTI>(a, pm, C, loc, uloc, has_unit, unit, lane, rs, msk, csp, ps, z4, zp4, y4, yp4, stg,
                                        pri);
        else
            tile_pass<true, A1, MULTI>(a, pm, C, loc, uloc, has_unit, unit, lane, rs, msk, csp, ps, z4, zp4, y4, yp4, stg,
                                       pri);
        __syncthreads();
        if (!fin) {
            // one partial per (CTA, variable): staged contributions in list
            // order, added in fixed point into the variable's accumulator
            unsigned long long *dst = a.acc + (size_t)(it & 1) * a.ptot;
            bool ovf = false;
            for (int i = threadIdx.x; i < C.nsv; i += blockDim.x) {
                const int j1 = cptr[i + 1];
                float S = 0.f;
                // eight list entries, then eight staged values, then the
                // adds (two dependent loads per eight contributions)
                for (int j = cptr[i]; j < j1; j += 8) {
                    int idx[8];
                    #pragma unroll
                    for (int t = 0; t < 8; ++t) idx[t] = j + t < j1 ? (int)clist[j + t] : -1;
                    float v[8];
                    #pragma unroll
                    for (int t = 0; t < 8; ++t) v[t] = idx[t] >= 0 ? stg[idx[t]] : 0.f;
                    #pragma unroll
                    for (int t = 0; t < 8; ++t) S = __fadd_rn(S, v[t]);
                }
                long long q = 0;
                if (fabsf(S) < kTileFixMax) q = __float2ll_rn(__fmul_rn(S, kTileFixScale));
                else ovf = true;
                // one contribution: its count and its value in one addition
                red_add_u64(dst + sv[i].x, kTileCountUnit + (unsigned long long)q);
            }
            if (ovf) atomicOr(&a.sync->overflow, 1);
        }
        if (chk) {
            // the CTA's sums through float pairs (csrc/residual.cuh), stored as doubles
            const float4 bs = block_sum2_ff(pri, dual);
            const double sp = (double)bs.x + (double)bs.y;
            const double sd = (double)bs.z + (double)bs.w;
            if (threadIdx.x == 0) {
                double *r = a.res + (size_t)(nchk & 1) * 2 * a.G;
                r[blockIdx.x] = sp;
                r[a.G + blockIdx.x] = sd;
            }
        }
        // the grid-wide barrier only where the residual decision needs
        // every CTA's partials; otherwise the next pass's polls are the wait
        if (!chk) continue;
        ++nchk;
        if (!tile_barrier(a.sync, G * (unsigned long long)nchk, a.timeout_ns, skip)) return;
        skip = false;
        {
            if (threadIdx.x < 32) {
                const double *r = a.res + (size_t)((nchk - 1) & 1) * 2 * a.G;
                const double sp = warp_sum_partials(r, a.G);
                const double sd = warp_sum_partials(r + a.G, a.G);
                if (threadIdx.x == 0) {
                    const bool finite = isfinite(sp) && isfinite(sd) && *(volatile int *)&a.sync->overflow == 0;
                    const bool conv = finite && s_rt[0].pass(sp) && s_rt[1].pass(sd);
                    s_dec[0] = finite;
                    s_dec[1] = conv;
                    if (!finite || conv || fin) {   // the reported values
                        s_res[0] = sqrt(sp / s_rt[0].E);
                        s_res[1] = sqrt(sd / s_rt[1].E);
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
                // a check that stops the call stores its state now (alpha = 1;
                // a check that also saved has stored it in the pass)
                if (A1 && !fin && !pm.save) {
                    if constexpr (MULTI) {
                        for (int lu = warp; lu < C.nunit; lu += (int)(blockDim.x >> 5)) {
                            int rs_u;
                            unsigned msk_u, csp_u[4];
                            unit_desc(a, C.unit0 + lu, lane, rs_u, msk_u, csp_u);
                            tile_store_a1(a, pm.reload, C.unit0 + lu, lane, rs_u, csp_u, z4, zp4, yp4);
                        }
                    } else if (has_unit) {
                        tile_store_a1(a, pm.reload, unit, lane, rs, csp, z4, zp4, yp4);
                    }
                }
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
// MODE 1: what an unchecked pass costs besides the operators -- every CTA
// adds one contribution to each variable it holds (count and a value of 0),
// then polls its variables' words until every holder's contribution of the
// pass is counted.  Needs the accumulator words zeroed before the launch.
// ---------------------------------------------------------------------------
template <int MODE>
__global__ void __launch_bounds__(kTileMaxWarps * 32, 1) k_tile_floor(const TileArgs a, long long iters) {
    extern __shared__ __align__(16) unsigned char tsm[];
    const TileSmem L = tile_smem_layout(a.smax, a.svmax, a.locmax, a.clmax, a.stgmax);
    int4 *sv = reinterpret_cast<int4 *>(tsm + L.sv);
    unsigned long long *pv = reinterpret_cast<unsigned long long *>(tsm + L.pv);
    const TileCta C = a.cta[blockIdx.x];
    for (int i = threadIdx.x; i < C.nsv; i += blockDim.x) {
        sv[i] = a.sv[C.sv0 + i];
        pv[i] = 0ull;
        pv[C.nsv + i] = 0ull;
    }
    __shared__ int s_ok;
    __syncthreads();
    const unsigned long long G = (unsigned long long)a.G;
    for (long long it = 1; it <= iters; ++it) {
        if (MODE == 1) {
            // the pass's contributions into the words of its parity, then
            // the wait for every holder's
            unsigned long long *acc = a.acc + (size_t)(it & 1) * a.ptot;
            unsigned long long *pp = pv + (size_t)(it & 1) * C.nsv;
            for (int i = threadIdx.x; i < C.nsv; i += blockDim.x) red_add_u64(acc + sv[i].x, kTileCountUnit);
            if (threadIdx.x == 0) s_ok = 1;
            __syncthreads();
            for (int i = threadIdx.x; i < C.nsv; i += blockDim.x) {
                const unsigned long long p = pp[i];
                const unsigned want = (unsigned)sv[i].y;
                unsigned long long w = ld_relaxed_u64(acc + sv[i].x);
                const unsigned long long t0 = global_ns();
                unsigned int spins = 0;
                while (tile_count(w - p) != want) {
                    if ((++spins & 63u) == 0u &&
                        (*(volatile int *)&a.sync->error || global_ns() - t0 > (unsigned long long)a.timeout_ns)) {
                        atomicCAS(&a.sync->error, 0, kETimeout);
                        s_ok = 0;
                        break;
                    }
                    w = ld_relaxed_u64(acc + sv[i].x);
                }
                pp[i] = w;
            }
            __syncthreads();
            if (!s_ok) return;
        } else if (!tile_barrier(a.sync, G * (unsigned long long)it, a.timeout_ns, false)) {
            return;
        }
    }
}

cudaError_t tile_floor_launch(const TileArgs &a, long long iters, int mode, int block, int smem, cudaStream_t s) {
    const void *fn = mode == 0 ? (const void *)k_tile_floor<0> : (const void *)k_tile_floor<1>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    void *args[] = {(void *)&a, (void *)&iters};
    return cudaLaunchCooperativeKernel(fn, dim3(a.G), dim3(block), args, (size_t)smem, s);
}

static const void *tile_kernel(bool a1, bool multi) {
    if (multi) return a1 ? (const void *)k_tile_sweep<true, true> : (const void *)k_tile_sweep<false, true>;
    return a1 ? (const void *)k_tile_sweep<true, false> : (const void *)k_tile_sweep<false, false>;
}

int tile_max_warps() {
    int w = kTileMaxWarps;
    for (bool a1 : {true, false}) {
        for (bool multi : {false, true}) {
            cudaFuncAttributes fa;
            if (cudaFuncGetAttributes(&fa, tile_kernel(a1, multi)) != cudaSuccess) return 0;
            if (fa.maxThreadsPerBlock / 32 < w) w = fa.maxThreadsPerBlock / 32;
        }
    }
    return w;
}

int tile_smem_bytes(const TilePlan &P) {
    return tile_smem_layout(P.smax, P.svmax, P.locmax, P.clmax, P.stgmax).total;
}

cudaError_t tile_sweep_launch(const TileArgs &a, int block, int smem, cudaStream_t s) {
    const void *fn = tile_kernel(a.alpha == 1.0f, a.dlive != nullptr);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    void *args[] = {(void *)&a};
    // cooperative: the grid must be co-resident for the grid-wide barrier
    return cudaLaunchCooperativeKernel(fn, dim3(a.G), dim3(block), args, (size_t)smem, s);
}

}  // namespace fga
