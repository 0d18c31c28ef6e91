// sweep.cuh -- device code of the factor-graph ADMM sweep (Algorithm 2).
//
// Included by sweep_f32.cu (FP32 messages, FMA contraction allowed) and by
// sweep_f64.cu (FP64, compiled with -fmad=false so that every product and
// sum is rounded on its own, as in a plain serial FP64 loop).
//
// Iteration structure inside one call (k = iterations done so far):
//   phase F(k): deferred u- and n-updates of iteration k-1
//               (u += alpha (x - z), n = z - u), then the x-update
//               x = Prox(n) of every factor (Eq. PO), then m = x + u and
//               rho*m scattered into the variable-major array;
//   phase Z(k): z_b = sum(rho m) / sum(rho) per variable.
// x and m are double-buffered so that the state after iteration k-1 is
// still intact when phase F(k) finds, from the residuals it computed, that
// iteration k-1 already met the tolerances.  Phases are separated by a
// grid-wide barrier (persistent kernel) or by kernel boundaries (unfused).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "fga_internal.h"

namespace fga {

// Status codes (same numbers as the public header).
constexpr int kETimeout = -5;
constexpr int kENonFinite = -6;
constexpr int kEBudget = -7;

// ---------------------------------------------------------------------------
// memory helpers
// ---------------------------------------------------------------------------
// Data written by other CTAs inside the same launch (z, the variable-major
// array, hub partials, residual partials) is read through L2 only, since L1
// is not coherent across SMs.
template <typename R>
__device__ __forceinline__ R ldg_l2(const R *p) { return __ldcg(p); }

static __device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

static __device__ __forceinline__ unsigned int ld_acquire_u32(const unsigned int *p) {
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

static __device__ __forceinline__ void st_release_u32(unsigned int *p, unsigned int v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

static __device__ __forceinline__ unsigned int atom_add_acq_rel(unsigned int *p, unsigned int v) {
    unsigned int old;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

// Grid-wide barrier with a time limit.  One thread per CTA arrives on a
// counter; the last arrival resets the counter and bumps the generation.
// Every wait is bounded by timeout_ns (globaltimer) and by a spin count; on
// expiry the CTA records FGA_ETIMEOUT in the barrier's error word and
// returns false, and every other CTA stops waiting as soon as it sees the
// error word.  The caller then leaves the kernel.  `skip` suppresses this
// CTA's arrival (fault-injection test of the time limit).
static __device__ __noinline__ bool grid_barrier(Barrier *b, unsigned int nblk, unsigned int &gen,
                                          long long timeout_ns, bool skip) {
    __shared__ int s_err;
    __syncthreads();
    if (threadIdx.x == 0) {
        int err = 0;
        if (!skip) {
            __threadfence();
            unsigned int prev = atom_add_acq_rel(&b->count, 1u);
            if (prev == nblk - 1) {
                atomicExch(&b->count, 0u);
                __threadfence();
                st_release_u32(&b->gen, gen + 1);
            }
        }
        const unsigned long long t0 = global_ns();
        const unsigned long long lim = (unsigned long long)timeout_ns;
        unsigned int spins = 0;
        while (ld_acquire_u32(&b->gen) == gen) {
            ++spins;
            if ((spins & 63u) == 0u) {
                if (*(volatile int *)&b->error) { err = 1; break; }
                if (global_ns() - t0 > lim || spins > (1u << 30)) {
                    atomicExch(&b->error, kETimeout);
                    err = 1;
                    break;
                }
            }
        }
        if (!err && *(volatile int *)&b->error) err = 1;
        gen += 1;
        s_err = err;
    }
    __syncthreads();
    return s_err == 0;
}

// Deterministic block sum of one double per thread (fixed shuffle tree,
// then warp results in warp order).  Result valid in thread 0.
static __device__ __forceinline__ double block_sum(double v) {
    __shared__ double s_w[32];
    #pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) s_w[w] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        for (int i = 0; i < nw; ++i) t += s_w[i];
    }
    return t;
}

// Sum of the first n values of an array written by all CTAs, in a fixed
// order; every caller obtains the same bits.  Called by a full warp.
static __device__ __forceinline__ double warp_sum_partials(const double *p, int n) {
    const int l = threadIdx.x & 31;
    double s = 0.0;
    for (int i = l; i < n; i += 32) s += ldg_l2(p + i);
    #pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    return s;
}

// ---------------------------------------------------------------------------
// proximal operators (Eq. PO).  Operation order matches a plain serial
// implementation of the same formulas, so that in FP64 with contraction off
// the results are the correctly rounded values of the same expression tree.
// ---------------------------------------------------------------------------

// Appendix A no-collision, (c1, r1, c2, r2): move the centres apart along
// nhat = (c2-c1)/|c2-c1| and shrink both radii, the total displacement
// D = r1 + r2 - |c1 - c2| split in proportion to 1/rho.
template <typename R>
__device__ __forceinline__ void prox_pack_pair(const R *n, const R *rho, R *x) {
    const R dx = n[3] - n[0];
    const R dy = n[4] - n[1];
    const R d = sqrt(dx * dx + dy * dy);
    const R D = n[2] + n[5] - d;
    if (!(D > R(0))) {
        #pragma unroll
        for (int k = 0; k < 6; ++k) x[k] = n[k];
        return;
    }
    R hx = R(1), hy = R(0);
    if (d > R(0)) {
        hx = dx / d;
        hy = dy / d;
    }
    const R wc1 = R(1) / rho[0], wr1 = R(1) / rho[2];
    const R wc2 = R(1) / rho[3], wr2 = R(1) / rho[5];
    const R W = wc1 + wr1 + wc2 + wr2;
    const R tc1 = (D * wc1) / W, tr1 = (D * wr1) / W;
    const R tc2 = (D * wc2) / W, tr2 = (D * wr2) / W;
    x[0] = n[0] - tc1 * hx;
    x[1] = n[1] - tc1 * hy;
    x[2] = n[2] - tr1;
    x[3] = n[3] + tc2 * hx;
    x[4] = n[4] + tc2 * hy;
    x[5] = n[5] - tr2;
}

// Appendix A wall: disk (c, r) inside the half-plane Q.(c - V) >= r.
template <typename R>
__device__ __forceinline__ void prox_pack_wall(const R *n, const R *rho, R Qx, R Qy, R Vx, R Vy, R *x) {
    const R h = Qx * (n[0] - Vx) + Qy * (n[1] - Vy) - n[2];
    if (h >= R(0)) {
        x[0] = n[0];
        x[1] = n[1];
        x[2] = n[2];
        return;
    }
    const R wc = R(1) / rho[0], wr = R(1) / rho[2];
    const R den = wc * (Qx * Qx + Qy * Qy) + wr;
    const R lam = -h / den;
    const R sc = lam * wc;
    x[0] = n[0] + sc * Qx;
    x[1] = n[1] + sc * Qy;
    x[2] = n[2] - lam * wr;
}

// ---------------------------------------------------------------------------
// per-edge pre/post steps of phase F
// ---------------------------------------------------------------------------
template <typename R>
struct EdgeIO {
    const R *xin;   // x after the previous iteration
    R *xout;        // x of this iteration
    R *mout;        // m of this iteration (may be null)
    const R *zc;    // z after the previous iteration
    // fast z-order only: the current chunk's z per slot and its rho*m buffer
    // (shared memory), indexed through lslot / lpos
    const R *zl;
    R *pb;
    int fast;
};

template <typename R>
__device__ __forceinline__ R edge_rho(const SweepArgs<R> &a, long long e) {
    return a.rho_e ? a.rho_e[e] : a.rho_u;
}

// z of the variable at the far end of edge e.
template <typename R>
__device__ __forceinline__ R edge_z(const SweepArgs<R> &a, const EdgeIO<R> &io, long long e) {
    return io.fast ? io.zl[a.lslot[e]] : ldg_l2(io.zc + a.svar[e]);
}

// Deferred u-update of the previous iteration (when MODE != F_PROX) and the
// n-update; returns n and leaves the current u in `u`.
template <typename R, int MODE>
__device__ __forceinline__ R edge_pre(const SweepArgs<R> &a, const EdgeIO<R> &io, long long e, R &u,
                                      double &pri) {
    const R z = edge_z(a, io, e);
    u = a.u[e];
    if (MODE != F_PROX) {
        const R al = a.alpha_e ? a.alpha_e[e] : a.alpha_u;
        const R xo = io.xin[e];
        const R d = xo - z;
        const double dd = (double)xo - (double)z;
        pri += dd * dd;
        u = u + al * d;
        a.u[e] = u;
    }
    return z - u;
}

// m-update, then rho*m either scattered into the variable-major array
// (canonical order) or parked in the chunk's shared-memory buffer at the
// edge's slot-sorted position (fast order).
template <typename R>
__device__ __forceinline__ void edge_post(const SweepArgs<R> &a, const EdgeIO<R> &io, long long e, R x, R u) {
    io.xout[e] = x;
    const R m = x + u;
    if (io.mout) io.mout[e] = m;
    const R p = edge_rho(a, e) * m;
    if (io.fast) io.pb[a.lpos[e]] = p;
    else a.pvm[a.pos[e]] = p;
}

// ---------------------------------------------------------------------------
// per-type work items
// ---------------------------------------------------------------------------
template <typename R, int MODE>
__device__ __forceinline__ void item_pack_pair(const SweepArgs<R> &a, const BucketDev<R> &B, const EdgeIO<R> &io,
                                               long long f, double &pri) {
    R n[6], u[6], rho[6];
    long long e[6];
    #pragma unroll
    for (int k = 0; k < 6; ++k) {
        e[k] = B.ebase + k * B.nf + f;
        n[k] = edge_pre<R, MODE>(a, io, e[k], u[k], pri);
        rho[k] = edge_rho(a, e[k]);
    }
    if (MODE == F_U_ONLY) return;
    R x[6];
    prox_pack_pair(n, rho, x);
    #pragma unroll
    for (int k = 0; k < 6; ++k) edge_post(a, io, e[k], x[k], u[k]);
}

template <typename R, int MODE>
__device__ __forceinline__ void item_pack_wall(const SweepArgs<R> &a, const BucketDev<R> &B, const EdgeIO<R> &io,
                                               long long f, double &pri) {
    R n[3], u[3], rho[3];
    long long e[3];
    #pragma unroll
    for (int k = 0; k < 3; ++k) {
        e[k] = B.ebase + k * B.nf + f;
        n[k] = edge_pre<R, MODE>(a, io, e[k], u[k], pri);
        rho[k] = edge_rho(a, e[k]);
    }
    if (MODE == F_U_ONLY) return;
    const R *p = B.prm;
    const long long nf = B.nf;
    R x[3];
    prox_pack_wall(n, rho, p[f], p[nf + f], p[2 * nf + f], p[3 * nf + f], x);
    #pragma unroll
    for (int k = 0; k < 3; ++k) edge_post(a, io, e[k], x[k], u[k]);
}

// Hinge c max(0, 1 - y (w.x + b)) on (w in R^D, b): two passes over the
// factor's edges (the first computes the margin, the second writes x).
template <typename R, int MODE>
__device__ __forceinline__ void item_svm_hinge(const SweepArgs<R> &a, const BucketDev<R> &B, const EdgeIO<R> &io,
                                               long long f, double &pri) {
    const int D = B.arity - 1;
    const long long nf = B.nf;
    const R *p = B.prm;
    R dot = R(0), s = R(0), nb = R(0), rb = R(1);
    for (int j = 0; j < D; ++j) {
        const long long e = B.ebase + j * nf + f;
        R u;
        const R n = edge_pre<R, MODE>(a, io, e, u, pri);
        const R xi = p[j * nf + f];
        dot += n * xi;
        s += (xi * xi) / edge_rho(a, e);
    }
    {
        const long long e = B.ebase + (long long)D * nf + f;
        R u;
        nb = edge_pre<R, MODE>(a, io, e, u, pri);
        rb = edge_rho(a, e);
    }
    if (MODE == F_U_ONLY) return;
    dot += nb;
    s += R(1) / rb;
    const R y = p[(long long)D * nf + f];
    const R c = p[(long long)(D + 1) * nf + f];
    const R t = R(1) - y * dot;
    const bool active = t > R(0);
    R gy = R(0);
    if (active) {
        R gam = t / s;
        if (gam > c) gam = c;
        gy = gam * y;
    }
    for (int j = 0; j <= D; ++j) {
        const long long e = B.ebase + j * nf + f;
        const R u = a.u[e];
        const R n = edge_z(a, io, e) - u;
        R x = n;
        if (active) x = (j < D) ? n + (gy * p[j * nf + f]) / edge_rho(a, e) : n + gy / edge_rho(a, e);
        edge_post(a, io, e, x, u);
    }
}

// Appendix B dynamics: v = P n with P the rho-weighted projector onto
// {x' = A x + B u}, precomputed per distinct (A, B, rho).  AC = compile-time
// arity (n kept in registers), or 0 for any arity (n re-formed from u and z
// for each output row).
template <typename R, int MODE, int AC>
__device__ __forceinline__ void item_mpc_dyn(const SweepArgs<R> &a, const BucketDev<R> &B, const EdgeIO<R> &io,
                                             long long f, double &pri) {
    if constexpr (AC > 0) {
        R n[AC], u[AC];
        #pragma unroll
        for (int k = 0; k < AC; ++k) n[k] = edge_pre<R, MODE>(a, io, B.ebase + k * B.nf + f, u[k], pri);
        if (MODE == F_U_ONLY) return;
        const R *P = B.pmat + (long long)B.pidx[f] * AC * AC;
        #pragma unroll 2
        for (int i = 0; i < AC; ++i) {
            R acc = R(0);
            #pragma unroll
            for (int j = 0; j < AC; ++j) acc += __ldg(P + i * AC + j) * n[j];
            edge_post(a, io, B.ebase + i * B.nf + f, acc, u[i]);
        }
    } else {
        const int A = B.arity;
        for (int k = 0; k < A; ++k) {
            R u;
            edge_pre<R, MODE>(a, io, B.ebase + k * B.nf + f, u, pri);
        }
        if (MODE == F_U_ONLY) return;
        const R *P = B.pmat + (long long)B.pidx[f] * A * A;
        for (int i = 0; i < A; ++i) {
            R acc = R(0);
            for (int j = 0; j < A; ++j) {
                const long long e = B.ebase + j * B.nf + f;
                acc += __ldg(P + i * A + j) * (edge_z(a, io, e) - a.u[e]);
            }
            const long long e = B.ebase + i * B.nf + f;
            edge_post(a, io, e, acc, a.u[e]);
        }
    }
}

// Elementwise types: one work item per scalar edge; li = k * nf + f.
template <typename R, int MODE>
__device__ __forceinline__ void item_elementwise(const SweepArgs<R> &a, const BucketDev<R> &B, const EdgeIO<R> &io,
                                                 long long li, double &pri) {
    const long long e = B.ebase + li;
    R u;
    const R n = edge_pre<R, MODE>(a, io, e, u, pri);
    if (MODE == F_U_ONLY) return;
    const long long f = li % B.nf;
    const R rho = edge_rho(a, e);
    R x;
    switch (B.type) {
    case 2:  // PACK_RADIUS_LIN: f = -w r
        x = n + B.prm[f] / rho;
        break;
    case 3:  // PACK_RADIUS_QUAD: f = -r^2/2
        x = (rho * n) / (rho - R(1));
        break;
    case 5:  // SVM_L2: f = lambda/2 |w|^2
        x = (rho * n) / (rho + B.prm[f]);
        break;
    case 7:  // MPC_QUAD: f = 1/2 q v^2, q per scalar component
        x = (rho * n) / (B.prm[li] + rho);
        break;
    case 8: {  // MPC_BOX
        const R lo = B.prm[f], hi = B.prm[B.nf + f];
        x = n;
        if (x < lo) x = lo;
        if (x > hi) x = hi;
        break;
    }
    default:  // 9, FIX
        x = B.prm[li];
        break;
    }
    edge_post(a, io, e, x, u);
}

template <typename R, int MODE>
__device__ __forceinline__ void process_in_bucket(const SweepArgs<R> &a, const BucketDev<R> &B, const EdgeIO<R> &io,
                                                  long long li, double &pri) {
    switch (B.type) {
    case 0: item_pack_pair<R, MODE>(a, B, io, li, pri); break;
    case 1: item_pack_wall<R, MODE>(a, B, io, li, pri); break;
    case 4: item_svm_hinge<R, MODE>(a, B, io, li, pri); break;
    case 6:
        if (B.arity == 28) item_mpc_dyn<R, MODE, 28>(a, B, io, li, pri);
        else item_mpc_dyn<R, MODE, 0>(a, B, io, li, pri);
        break;
    default: item_elementwise<R, MODE>(a, B, io, li, pri); break;
    }
}

template <typename R, int MODE>
__device__ __forceinline__ void process_item(const SweepArgs<R> &a, const EdgeIO<R> &io, long long it, double &pri) {
    int b = 0;
    while (b + 1 < a.nb && it >= a.bk[b + 1].item0) ++b;
    process_in_bucket<R, MODE>(a, a.bk[b], io, it - a.bk[b].item0, pri);
}

// Canonical order: every work item on its own, rho*m scattered to the
// variable-major array.  Fast order: CTAs walk their chunks; a chunk's
// variables ("slots") get their z staged in shared memory, every edge's
// rho*m lands in shared memory sorted by slot, and each slot's sum over the
// chunk (edges in slot order, fixed shuffle tree) is written to the
// variable-major partial array.  Both orders are deterministic.
template <typename R, int MODE>
__device__ __forceinline__ void phase_f(const SweepArgs<R> &a, EdgeIO<R> io, double &pri) {
    if (!io.fast) {
        const long long stride = (long long)gridDim.x * blockDim.x;
        for (long long it = (long long)blockIdx.x * blockDim.x + threadIdx.x; it < a.nitems_f; it += stride)
            process_item<R, MODE>(a, io, it, pri);
        return;
    }
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R *pb = reinterpret_cast<R *>(smem_raw);
    R *zl = pb + kChunkEdges;
    io.pb = pb;
    io.zl = zl;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    for (int c = blockIdx.x; c < a.nchunks; c += gridDim.x) {
        const ChunkDev ch = a.chunks[c];
        for (int s = threadIdx.x; s < ch.nslots; s += blockDim.x) zl[s] = ldg_l2(io.zc + a.slot_var[ch.sbase + s]);
        __syncthreads();
        const BucketDev<R> &B = a.bk[ch.bucket];
        for (int i = threadIdx.x; i < ch.nitems; i += blockDim.x)
            process_in_bucket<R, MODE>(a, B, io, ch.f0 + i, pri);
        __syncthreads();
        if (MODE != F_U_ONLY) {
            const int *lr = a.lrow + ch.lrbase;
            for (int sl = warp; sl < ch.nslots; sl += nwarps) {
                const int beg = lr[sl], end = lr[sl + 1];
                R S = R(0);
                for (int k = beg + lane; k < end; k += 32) S += pb[k];
                #pragma unroll
                for (int o = 16; o > 0; o >>= 1) S += __shfl_xor_sync(0xffffffffu, S, o);
                if (lane == 0) a.part[a.ppos[ch.sbase + sl]] = S;
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// phase Z: z_b = sum_k pvm[k] / srho_b over the variable's row.
// ---------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ void z_store(const SweepArgs<R> &a, int b, R S, const R *zo, R *zn, bool chk,
                                        double &dual) {
    const R zold = zo[b];
    R znew = zold;
    if (a.srho[b] > R(0)) znew = S / a.srho[b];   // a variable without edges keeps z
    zn[b] = znew;
    if (chk) {
        const double dz = (double)znew - (double)zold;
        dual += a.srho2[b] * dz * dz;
    }
}

template <typename R>
__device__ __forceinline__ void phase_z(const SweepArgs<R> &a, const R *zo, R *zn, bool chk, double &dual) {
    const long long gtid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long gstride = (long long)gridDim.x * blockDim.x;
    if (a.zorder == 0) {
        // canonical: one thread per variable, edges one by one in creation order
        for (long long b = gtid; b < a.nz; b += gstride) {
            R S = R(0);
            for (int k = a.row[b]; k < a.row[b + 1]; ++k) S += ldg_l2(a.pvm + k);
            z_store(a, (int)b, S, zo, zn, chk, dual);
        }
        return;
    }
    // fast: sums of the chunk partials, row by row (variable-major)
    const R *src = a.part;
    const int *row = a.prow;
    // low-degree variables one thread each ...
    for (long long i = gtid; i < a.n_small; i += gstride) {
        const int b = a.small_vars[i];
        R S = R(0);
        for (int k = row[b]; k < row[b + 1]; ++k) S += ldg_l2(src + k);
        z_store(a, b, S, zo, zn, chk, dual);
    }
    // ... the others one warp per item (a whole row, or one piece of a hub
    // row whose pieces are combined in piece order by the last warp done).
    const int lane = threadIdx.x & 31;
    const long long wid = gtid >> 5, nw = gstride >> 5;
    for (long long w = wid; w < a.n_witems; w += nw) {
        const int4 wi = a.witems[w];
        R S = R(0);
        for (int k = lane; k < wi.z; k += 32) S += ldg_l2(src + wi.y + k);
        #pragma unroll
        for (int o = 16; o > 0; o >>= 1) S += __shfl_xor_sync(0xffffffffu, S, o);
        if (wi.w < 0) {
            if (lane == 0) z_store(a, wi.x, S, zo, zn, chk, dual);
            continue;
        }
        const int h = wi.w;
        const int piece = (wi.y - row[wi.x]) / kPiece;
        const int np = a.hub_npieces[h];
        unsigned int ticket = 0;
        if (lane == 0) {
            a.hub_part[a.hub_off[h] + piece] = S;
            __threadfence();
            ticket = atomicAdd(&a.hub_ticket[h], 1u);
        }
        ticket = __shfl_sync(0xffffffffu, ticket, 0);
        if (ticket == (unsigned int)(np - 1)) {
            __threadfence();
            R T = R(0);
            for (int k = lane; k < np; k += 32) T += ldg_l2(a.hub_part + a.hub_off[h] + k);
            #pragma unroll
            for (int o = 16; o > 0; o >>= 1) T += __shfl_xor_sync(0xffffffffu, T, o);
            if (lane == 0) {
                a.hub_ticket[h] = 0u;
                z_store(a, wi.x, T, zo, zn, chk, dual);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// residual check (identical in every CTA of the persistent kernel)
// ---------------------------------------------------------------------------
struct CheckOut {
    double rp, rd;
    bool stop;
    int status;
};

template <typename R>
__device__ __forceinline__ CheckOut residual_check(const SweepArgs<R> &a, int nparts, int dual_buf) {
    __shared__ double s_r[2];
    if (threadIdx.x < 32) {
        const double sp = warp_sum_partials(a.res_pri, nparts);
        const double sd = warp_sum_partials(a.res_dual + (long long)dual_buf * a.gmax, nparts);
        if (threadIdx.x == 0) {
            const double E = a.E > 0 ? (double)a.E : 1.0;
            s_r[0] = sqrt(sp / E);
            s_r[1] = sqrt(sd / E);
        }
    }
    __syncthreads();
    CheckOut c;
    c.rp = s_r[0];
    c.rd = s_r[1];
    __syncthreads();
    const bool finite = isfinite(c.rp) && isfinite(c.rd);
    c.status = finite ? 0 : kENonFinite;
    c.stop = !finite || (c.rp <= a.tol_pri && c.rd <= a.tol_dual);
    return c;
}

template <typename R>
__device__ __forceinline__ void write_ctl(const SweepArgs<R> &a, long long iters, const CheckOut &c, int xp, int zp,
                                          bool budget_end) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        Ctl *ctl = a.ctl;
        ctl->iters = iters;
        ctl->r_pri = c.rp;
        ctl->r_dual = c.rd;
        int st = c.status;
        if (st == 0 && budget_end && !(c.rp <= a.tol_pri && c.rd <= a.tol_dual) &&
            (a.tol_pri > 0.0 || a.tol_dual > 0.0))
            st = kEBudget;
        ctl->status = st;
        ctl->xpar = xp;
        ctl->zpar = zp;
        ctl->checked = 1;
        __threadfence();
        *(volatile int *)&ctl->done = 1;
    }
}

template <typename R>
__device__ __forceinline__ EdgeIO<R> make_io(const SweepArgs<R> &a, int xp, int zp) {
    EdgeIO<R> io;
    io.xin = a.x[xp];
    io.xout = a.x[xp ^ 1];
    io.mout = a.m[xp ^ 1];
    io.zc = a.z[zp];
    io.zl = nullptr;
    io.pb = nullptr;
    io.fast = a.zorder;
    return io;
}

// ---------------------------------------------------------------------------
// the persistent kernel: a whole call in one launch
// ---------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(256, 3) k_sweep_persistent(const SweepArgs<R> a) {
    unsigned int gen = 0;
    const unsigned int G = gridDim.x;
    bool skip = (a.skip_block == (int)blockIdx.x);
    int xp = a.xpar0, zp = a.zpar0;
    for (long long it = 1; it <= a.K; ++it) {
        const bool pend = it > 1;
        const bool chk = pend && ((a.k0 + it - 1) % a.check_every == 0);
        const EdgeIO<R> io = make_io(a, xp, zp);
        double pri = 0.0;
        if (pend) phase_f<R, F_U_PROX>(a, io, pri);
        else phase_f<R, F_PROX>(a, io, pri);
        if (chk) {
            const double s = block_sum(pri);
            if (threadIdx.x == 0) a.res_pri[blockIdx.x] = s;
        }
        if (!grid_barrier(a.bar, G, gen, a.timeout_ns, skip)) return;
        skip = false;
        if (chk) {
            const CheckOut c = residual_check(a, G, (int)((it - 1) & 1));
            if (c.stop) {
                write_ctl(a, it - 1, c, xp, zp, false);
                return;
            }
        }
        xp ^= 1;
        const bool chkz = ((a.k0 + it) % a.check_every == 0) || it == a.K;
        double dual = 0.0;
        phase_z(a, a.z[zp], a.z[zp ^ 1], chkz, dual);
        if (chkz) {
            const double s = block_sum(dual);
            if (threadIdx.x == 0) a.res_dual[(long long)(it & 1) * a.gmax + blockIdx.x] = s;
        }
        if (!grid_barrier(a.bar, G, gen, a.timeout_ns, false)) return;
        zp ^= 1;
    }
    if (a.K <= 0) return;
    // u-update of the last iteration, and its residual check
    EdgeIO<R> io = make_io(a, xp, zp);
    double pri = 0.0;
    phase_f<R, F_U_ONLY>(a, io, pri);
    const double s = block_sum(pri);
    if (threadIdx.x == 0) a.res_pri[blockIdx.x] = s;
    if (!grid_barrier(a.bar, G, gen, a.timeout_ns, skip)) return;
    const CheckOut c = residual_check(a, G, (int)(a.K & 1));
    write_ctl(a, a.K, c, xp, zp, true);
}

// ---------------------------------------------------------------------------
// unfused launches: one kernel per phase; each exits at once when an
// earlier check of this call has stopped it.
// ---------------------------------------------------------------------------
template <typename R, int MODE>
__global__ void __launch_bounds__(256) k_phase_f(const SweepArgs<R> a, int xp, int zp, int chk) {
    if (*(volatile int *)&a.ctl->done) return;
    const EdgeIO<R> io = make_io(a, xp, zp);
    double pri = 0.0;
    phase_f<R, MODE>(a, io, pri);
    if (chk) {
        const double s = block_sum(pri);
        if (threadIdx.x == 0) a.res_pri[blockIdx.x] = s;
    }
}

template <typename R>
__global__ void __launch_bounds__(256) k_phase_z(const SweepArgs<R> a, int zp, long long it, int chk) {
    if (*(volatile int *)&a.ctl->done) return;
    double dual = 0.0;
    phase_z(a, a.z[zp], a.z[zp ^ 1], chk != 0, dual);
    if (chk) {
        const double s = block_sum(dual);
        if (threadIdx.x == 0) a.res_dual[(long long)(it & 1) * a.gmax + blockIdx.x] = s;
    }
}

template <typename R>
__global__ void __launch_bounds__(32) k_check(const SweepArgs<R> a, long long it_checked, int xp, int zp,
                                              int final_check, int nparts) {
    if (*(volatile int *)&a.ctl->done) return;
    const CheckOut c = residual_check(a, nparts, (int)(it_checked & 1));
    if (c.stop || final_check) write_ctl(a, it_checked, c, xp, zp, final_check != 0 && !c.stop);
}

}  // namespace fga
