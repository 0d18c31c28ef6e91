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

// ---- cp.async (global -> shared, one element, zero when !valid) -------------
template <typename R>
static __device__ __forceinline__ void cp_async_zfill(R *dst, const R *src, bool valid) {
    const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst));
    if (sizeof(R) == 8)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(d), "l"(src), "r"(valid ? 8 : 0) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(d), "l"(src), "r"(valid ? 4 : 0) : "memory");
}
static __device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
static __device__ __forceinline__ void cp_async_wait_group() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// ---- mbarrier + bulk asynchronous copy (global -> shared) --------------------
static __device__ __forceinline__ unsigned smem_u32(const void *p) {
    return (unsigned)__cvta_generic_to_shared(p);
}
static __device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
static __device__ __forceinline__ void mbar_inval(unsigned long long *bar) {
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}
static __device__ __forceinline__ void mbar_fence_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
static __device__ __forceinline__ void mbar_expect_tx(unsigned long long *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
static __device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// 1-D bulk copy of `bytes` (a multiple of 16; both addresses 16-byte
// aligned) from global to this CTA's shared memory, completing on `bar`.
static __device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, unsigned long long *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
static __device__ __forceinline__ void fence_proxy_async_shared() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
static __device__ __forceinline__ void fence_proxy_async_global() {
    asm volatile("fence.proxy.async.global;" ::: "memory");
}

static __device__ __forceinline__ void red_release_add_u64(unsigned long long *p, unsigned long long v) {
    asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
// Fire-and-forget integer addition at L2 (no value returned to the thread).
static __device__ __forceinline__ void red_add_u64(unsigned long long *p, unsigned long long v) {
    asm volatile("red.relaxed.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
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

// Grid-wide barrier with a time limit.  The barrier's first eight bytes
// (count and gen, zeroed before each launch) are one 64-bit counter that
// only grows: thread 0 of each CTA arrives with a fire-and-forget release
// addition and waits, polling with relaxed loads, until the counter reaches
// nblk x (barriers passed so far, `gen` + 1); one acquire load then orders
// the CTA's later reads (through bar.sync) after every CTA's writes.  No
// arrival returns a value and no last arrival has to release the others,
// which makes a barrier of several hundred CTAs cheaper than a counter that
// is reset each time.  Every wait is bounded by timeout_ns (globaltimer) and
// by a spin count; on expiry the CTA records FGA_ETIMEOUT in the barrier's
// error word and returns false, and every other CTA stops waiting as soon as
// it sees the error word.  The caller then leaves the kernel.  `skip`
// suppresses this CTA's arrival (fault-injection test of the time limit).
static __device__ __noinline__ bool grid_barrier(Barrier *b, unsigned int nblk, unsigned int &gen,
                                          long long timeout_ns, bool skip) {
    __shared__ int s_err;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long *cnt = reinterpret_cast<unsigned long long *>(&b->count);
        const unsigned long long target = (unsigned long long)nblk * ((unsigned long long)gen + 1ull);
        int err = 0;
        if (!skip) red_release_add_u64(cnt, 1ull);
        if (ld_relaxed_u64(cnt) < target) {
            const unsigned long long t0 = global_ns();
            const unsigned long long lim = (unsigned long long)timeout_ns;
            unsigned int spins = 0;
            while (ld_relaxed_u64(cnt) < target) {
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
        }
        (void)ld_acquire_u64(cnt);
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

// FP32 variant of the same projection: the direction and length come from
// one approximate reciprocal square root, and with a uniform rho every
// share w_k / W is 1/4.  (FP32 results are compared with the FP64 oracle
// through tolerances, never bit for bit.)
__device__ __forceinline__ void prox_pack_pair_f32(const float *n, const float *rho, bool uniform, float *x) {
    const float dx = n[3] - n[0];
    const float dy = n[4] - n[1];
    const float d2 = dx * dx + dy * dy;
    const float rd = d2 > 0.f ? rsqrtf(d2) : 0.f;
    const float D = n[2] + n[5] - d2 * rd;
    if (!(D > 0.f)) {
        #pragma unroll
        for (int k = 0; k < 6; ++k) x[k] = n[k];
        return;
    }
    float hx = 1.f, hy = 0.f;
    if (d2 > 0.f) {
        hx = dx * rd;
        hy = dy * rd;
    }
    float tc1, tr1, tc2, tr2;
    if (uniform) {
        tc1 = tr1 = tc2 = tr2 = 0.25f * D;
    } else {
        const float wc1 = 1.f / rho[0], wr1 = 1.f / rho[2], wc2 = 1.f / rho[3], wr2 = 1.f / rho[5];
        const float iW = D / (wc1 + wr1 + wc2 + wr2);
        tc1 = wc1 * iW;
        tr1 = wr1 * iW;
        tc2 = wc2 * iW;
        tr2 = wr2 * iW;
    }
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
// edge access.  Storage index of scalar edge k of factor f in bucket B:
// factor-major (B.aos: the factor's edges are adjacent, ebase + f*arity + k)
// or edge-major (ebase + k*nf + f).  Indices are 32-bit (|E| < 2^31).
// ---------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ int bedge(const BucketDev<R> &B, int f, int k) {
    return B.aos ? B.ebase + f * B.arity + k : B.ebase + k * B.nf + f;
}

template <typename R>
struct EdgeIO {
    const R *xin;   // x after the previous iteration
    R *xout;        // x of this iteration
    R *mout;        // m of this iteration (may be null)
    const R *zc;    // z after the previous iteration
    // fast order only: the current chunk's z per slot and its rho*m buffer
    // (shared memory), addressed through lidx = slot | position << 16
    const R *zl;
    R *pb;
};

template <typename R>
__device__ __forceinline__ R edge_rho(const SweepArgs<R> &a, int e) {
    return a.rho_e ? a.rho_e[e] : a.rho_u;
}

// The z order an edge access is compiled for (the FAST template argument of
// the functions below): canonical rows, fast-order chunks, scatter columns.
enum EdgeOrder : int { EO_CANON = 0, EO_CHUNK = 1, EO_SCATTER = 2 };

// Where the rho*m of edge e goes in pvm outside the fast order: its slot in
// the variable-major rows (canonical), or its column or overflow slot
// (scatter); returns the edge's scalar variable.
template <typename R, int FAST>
__device__ __forceinline__ int edge_dest(const SweepArgs<R> &a, int e, unsigned &dst) {
    if constexpr (FAST == EO_SCATTER) {
        const unsigned v = a.ev[e];
        const unsigned c = v >> kEvColShift, b = v & kEvVarMask;
        dst = c != kEvOverflow ? c * (unsigned)a.nz + b : a.ovf0 + (unsigned)a.pos[e];
        return (int)b;
    }
    dst = (unsigned)a.pos[e];
    return a.svar[e];
}

// z at the far end of edge e; `ix` receives what edge_put needs later.
template <typename R, int FAST>
__device__ __forceinline__ R edge_z(const SweepArgs<R> &a, const EdgeIO<R> &io, int e, unsigned &ix) {
    if constexpr (FAST == EO_CHUNK) {
        ix = a.lidx[e];
        return io.zl[ix & 0xffffu];
    }
    return ldg_l2(io.zc + edge_dest<R, FAST>(a, e, ix));
}

template <typename R, int FAST>
__device__ __forceinline__ void edge_put(const SweepArgs<R> &a, const EdgeIO<R> &io, unsigned ix, R p) {
    if constexpr (FAST == EO_CHUNK) io.pb[ix >> 16] = p;
    else a.pvm[ix] = p;
}

// Deferred u-update of the previous iteration (when MODE != F_PROX) and the
// n-update, given z and the current u; returns n, updates u.
template <typename R, int MODE>
__device__ __forceinline__ R update_un(const SweepArgs<R> &a, const EdgeIO<R> &io, int e, R z, R xo, R &u,
                                       double &pri) {
    if (MODE != F_PROX) {
        const R al = a.alpha_e ? a.alpha_e[e] : a.alpha_u;
        const R d = xo - z;
        if constexpr (fmode_checks(MODE)) {
            const double dd = (double)xo - (double)z;
            pri += dd * dd;
        }
        // three weights: an edge whose last message had zero or infinite
        // weight restarts from u = 0
        u = (a.wcls && a.wcls[e] != 1) ? R(0) : u + al * d;
    }
    return z - u;
}

// Three-weight mode: the weight class of the messages an item just sent,
// read back by the thread that wrote them -- infinite for FIX (its rho m
// slot then holds m itself), zero on an edge of a constraint-type factor
// (disk pair, wall, box, hinge, margin) whose x equals its n, standard
// otherwise (standard classes are set once by fga_init).
template <typename R>
__device__ __forceinline__ void twa_mark(const SweepArgs<R> &a, const BucketDev<R> &B, const EdgeIO<R> &io, int li) {
    const int t = B.type;
    const bool cons = t == 0 || t == 1 || t == 4 || t == 8 || t == 10;
    if (!cons && t != 9) return;
    const int ne = B.per_edge ? 1 : B.arity;
    for (int k = 0; k < ne; ++k) {
        const int e = B.per_edge ? B.ebase + li : bedge(B, li, k);
        const R u = a.u[e], x = io.xout[e];
        unsigned char c;
        if (t == 9) {
            c = 2;
            a.pvm[a.pos[e]] = x + u;
        } else {
            const R n = ldg_l2(io.zc + a.svar[e]) - u;
            c = x == n ? 0 : 1;
        }
        a.wcls[e] = c;
        a.pwcls[a.pos[e]] = c;
    }
}

// One scalar edge, start of phase F: returns n; u holds the updated u
// (already stored when MODE != F_PROX).
template <typename R, int MODE, int FAST>
__device__ __forceinline__ R edge_pre(const SweepArgs<R> &a, const EdgeIO<R> &io, int e, R &u, unsigned &ix,
                                      double &pri) {
    const R z = edge_z<R, FAST>(a, io, e, ix);
    u = a.u[e];
    const R xo = MODE != F_PROX ? io.xin[e] : R(0);
    const R n = update_un<R, MODE>(a, io, e, z, xo, u, pri);
    if (MODE != F_PROX) a.u[e] = u;
    return n;
}

// The same in two halves, so that an item issues the loads of several of
// its edges before the first store (a store to u may alias a later load as
// far as the compiler knows, so edge_pre in a loop over edges makes every
// edge's loads wait for the previous edge's store): edge_load reads z at
// the far end, u and the previous x; edge_update runs the deferred u-update
// and the n-update and stores u.  The arithmetic is edge_pre's.
template <typename R, int MODE, int FAST>
__device__ __forceinline__ void edge_load(const SweepArgs<R> &a, const EdgeIO<R> &io, int e, R &z, R &u, R &xo,
                                          unsigned &ix) {
    z = edge_z<R, FAST>(a, io, e, ix);
    u = a.u[e];
    xo = MODE != F_PROX ? io.xin[e] : R(0);
}

template <typename R, int MODE>
__device__ __forceinline__ R edge_update(const SweepArgs<R> &a, const EdgeIO<R> &io, int e, R z, R xo, R &u,
                                         double &pri) {
    const R n = update_un<R, MODE>(a, io, e, z, xo, u, pri);
    if (MODE != F_PROX) a.u[e] = u;
    return n;
}

// One scalar edge, end of phase F: x, m = x + u, rho*m to the z-reduction.
template <typename R, int FAST>
__device__ __forceinline__ void edge_post(const SweepArgs<R> &a, const EdgeIO<R> &io, int e, unsigned ix, R x, R u) {
    io.xout[e] = x;
    const R m = x + u;
    if (io.mout) io.mout[e] = m;
    edge_put<R, FAST>(a, io, ix, edge_rho(a, e) * m);
}

// 6 consecutive values with three 2-element vector accesses (the pair
// bucket is factor-major with an even base, so e0 = ebase + 6 f is even).
template <typename T, typename V2>
__device__ __forceinline__ void load6(const T *p, T *v) {
    const V2 *q = reinterpret_cast<const V2 *>(p);
    #pragma unroll
    for (int i = 0; i < 3; ++i) {
        const V2 t = q[i];
        v[2 * i] = t.x;
        v[2 * i + 1] = t.y;
    }
}
template <typename T, typename V2>
__device__ __forceinline__ void store6(T *p, const T *v) {
    V2 *q = reinterpret_cast<V2 *>(p);
    #pragma unroll
    for (int i = 0; i < 3; ++i) {
        V2 t;
        t.x = v[2 * i];
        t.y = v[2 * i + 1];
        q[i] = t;
    }
}
template <typename R> struct Vec2;
template <> struct Vec2<float> { using T = float2; };
template <> struct Vec2<double> { using T = double2; };

// ---------------------------------------------------------------------------
// per-type work items
// ---------------------------------------------------------------------------
template <typename R, int MODE, int FAST>
__device__ __forceinline__ void item_pack_pair(const SweepArgs<R> &a, const BucketDev<R> &B, const EdgeIO<R> &io,
                                               int f, double &pri) {
    using V = typename Vec2<R>::T;
    const int e0 = B.ebase + 6 * f;
    R u[6], z[6], xo[6], rho[6], n[6];
    unsigned ix[6];
    load6<R, V>(a.u + e0, u);
    if (MODE != F_PROX) load6<R, V>(io.xin + e0, xo);
    if constexpr (FAST == EO_CHUNK) {
        load6<unsigned, uint2>(a.lidx + e0, ix);
        #pragma unroll
        for (int k = 0; k < 6; ++k) z[k] = io.zl[ix[k] & 0xffffu];
    } else if constexpr (FAST == EO_CANON) {
        int sv[6], ps[6];
        load6<int, int2>(a.svar + e0, sv);
        load6<int, int2>(a.pos + e0, ps);
        #pragma unroll
        for (int k = 0; k < 6; ++k) {
            z[k] = ldg_l2(io.zc + sv[k]);
            ix[k] = (unsigned)ps[k];
        }
    } else {
        #pragma unroll
        for (int k = 0; k < 6; ++k) z[k] = edge_z<R, FAST>(a, io, e0 + k, ix[k]);
    }
    if (a.rho_e) load6<R, V>(a.rho_e + e0, rho);
    else {
        #pragma unroll
        for (int k = 0; k < 6; ++k) rho[k] = a.rho_u;
    }
    #pragma unroll
    for (int k = 0; k < 6; ++k) n[k] = update_un<R, MODE>(a, io, e0 + k, z[k], xo[k], u[k], pri);
    if (MODE != F_PROX) store6<R, V>(a.u + e0, u);
    if (MODE == F_U_ONLY) return;
    R x[6];
    if constexpr (sizeof(R) == 4) prox_pack_pair_f32(n, rho, a.rho_e == nullptr, x);
    else prox_pack_pair(n, rho, x);
    store6<R, V>(io.xout + e0, x);
    R m[6];
    #pragma unroll
    for (int k = 0; k < 6; ++k) m[k] = x[k] + u[k];
    if (io.mout) store6<R, V>(io.mout + e0, m);
    #pragma unroll
    for (int k = 0; k < 6; ++k) edge_put<R, FAST>(a, io, ix[k], rho[k] * m[k]);
}

// The same, with u, x and the slot/position indices read from a bulk-copy
// stage in shared memory (su, sx, si point at this pair's six entries).
template <typename R, int MODE>
__device__ __forceinline__ void item_pack_pair_staged(const SweepArgs<R> &a, const BucketDev<R> &B,
                                                      const EdgeIO<R> &io, int f, const R *su, const R *sx,
                                                      const unsigned *si, double &pri) {
    using V = typename Vec2<R>::T;
    const int e0 = B.ebase + 6 * f;
    R u[6], z[6], xo[6], rho[6], n[6];
    unsigned ix[6];
    #pragma unroll
    for (int k = 0; k < 6; ++k) {
        u[k] = su[k];
        xo[k] = MODE != F_PROX ? sx[k] : R(0);
        ix[k] = si[k];
        z[k] = io.zl[ix[k] & 0xffffu];
    }
    if (a.rho_e) load6<R, V>(a.rho_e + e0, rho);
    else {
        #pragma unroll
        for (int k = 0; k < 6; ++k) rho[k] = a.rho_u;
    }
    #pragma unroll
    for (int k = 0; k < 6; ++k) n[k] = update_un<R, MODE>(a, io, e0 + k, z[k], xo[k], u[k], pri);
    if (MODE != F_PROX) store6<R, V>(a.u + e0, u);
    if (MODE == F_U_ONLY) return;
    R x[6];
    if constexpr (sizeof(R) == 4) prox_pack_pair_f32(n, rho, a.rho_e == nullptr, x);
    else prox_pack_pair(n, rho, x);
    store6<R, V>(io.xout + e0, x);
    R m[6];
    #pragma unroll
    for (int k = 0; k < 6; ++k) m[k] = x[k] + u[k];
    if (io.mout) store6<R, V>(io.mout + e0, m);
    #pragma unroll
    for (int k = 0; k < 6; ++k) edge_put<R, EO_CHUNK>(a, io, ix[k], rho[k] * m[k]);
}

// Bounded wait on a stage barrier; false (and the grid's error word set)
// if the copy did not land within about a second.
static __device__ __forceinline__ bool stage_wait(unsigned long long *bar, unsigned parity, Barrier *gb) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (unsigned spin = 0; spin < (1u << 26); ++spin) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((spin & 255u) == 0u && global_ns() - t0 > 1000000000ull) break;
    }
    atomicExch(&gb->error, kETimeout);
    return false;
}

template <typename R, int MODE, int FAST>
__device__ __forceinline__ void item_pack_wall(const SweepArgs<R> &a, const BucketDev<R> &B, const EdgeIO<R> &io,
                                               int f, double &pri) {
    R n[3], u[3], rho[3];
    unsigned ix[3];
    int e[3];
    #pragma unroll
    for (int k = 0; k < 3; ++k) {
        e[k] = bedge(B, f, k);
        n[k] = edge_pre<R, MODE, FAST>(a, io, e[k], u[k], ix[k], pri);
        rho[k] = edge_rho(a, e[k]);
    }
    if (MODE == F_U_ONLY) return;
    const R *p = B.prm;
    const int nf = B.nf;
    R x[3];
    prox_pack_wall(n, rho, p[f], p[nf + f], p[2 * nf + f], p[3 * nf + f], x);
    #pragma unroll
    for (int k = 0; k < 3; ++k) edge_post<R, FAST>(a, io, e[k], ix[k], x[k], u[k]);
}

// Hinge c max(0, 1 - y (w.x + b)) on (w in R^D, b), one thread per factor:
// two passes over the factor's edges (the first computes the margin in the
// order of a serial loop, the second writes x).  Parameters factor-major:
// p[f*(D+2) + j] = x_j, then y, c.
template <typename R, int MODE, int FAST>
__device__ __forceinline__ void item_svm_hinge(const SweepArgs<R> &a, const BucketDev<R> &B, const EdgeIO<R> &io,
                                               int f, double &pri) {
    const int D = B.arity - 1;
    const R *p = B.prm + (long long)f * (D + 2);
    R dot = R(0), s = R(0), nb = R(0), rb = R(1);
    for (int j = 0; j < D; ++j) {
        const int e = bedge(B, f, j);
        R u;
        unsigned ix;
        const R n = edge_pre<R, MODE, FAST>(a, io, e, u, ix, pri);
        const R xi = p[j];
        dot += n * xi;
        s += (xi * xi) / edge_rho(a, e);
    }
    {
        const int e = bedge(B, f, D);
        R u;
        unsigned ix;
        nb = edge_pre<R, MODE, FAST>(a, io, e, u, ix, pri);
        rb = edge_rho(a, e);
    }
    if (MODE == F_U_ONLY) return;
    dot += nb;
    s += R(1) / rb;
    const R y = p[D];
    const R c = p[D + 1];
    const R t = R(1) - y * dot;
    const bool active = t > R(0);
    R gy = R(0);
    if (active) {
        R gam = t / s;
        if (gam > c) gam = c;
        gy = gam * y;
    }
    for (int j = 0; j <= D; ++j) {
        const int e = bedge(B, f, j);
        const R u = a.u[e];
        unsigned ix;
        const R n = edge_z<R, FAST>(a, io, e, ix) - u;
        R x = n;
        if (active) x = (j < D) ? n + (gy * p[j]) / edge_rho(a, e) : n + gy / edge_rho(a, e);
        edge_post<R, FAST>(a, io, e, ix, x, u);
    }
}

// The same operator with one warp per factor (fast and scatter orders): lane l owns the
// edges j = l, l + 32, ...; the margin and the weight sum are reduced with a
// fixed shuffle tree; one pass, the factor's edges and data point read
// contiguously (factor-major storage).
template <typename R, int MODE, int FAST = EO_CHUNK>
__device__ __forceinline__ void item_svm_hinge_warp(const SweepArgs<R> &a, const BucketDev<R> &B, const EdgeIO<R> &io,
                                                    int f, double &pri) {
    constexpr int JMAX = 4;   // up to 128 edges per factor kept in registers
    const int D = B.arity - 1;
    const int lane = threadIdx.x & 31;
    const R *p = B.prm + (long long)f * (D + 2);
    const int e0 = B.ebase + f * B.arity;
    R n[JMAX], u[JMAX], rho[JMAX], xi[JMAX];
    unsigned ix[JMAX];
    R dot = R(0), s = R(0);
    #pragma unroll
    for (int q = 0; q < JMAX; ++q) {
        const int j = lane + 32 * q;
        if (j > D) continue;
        const int e = e0 + j;
        n[q] = edge_pre<R, MODE, FAST>(a, io, e, u[q], ix[q], pri);
        rho[q] = edge_rho(a, e);
        xi[q] = j < D ? p[j] : R(1);
        dot += n[q] * xi[q];
        s += (xi[q] * xi[q]) / rho[q];
    }
    if (MODE == F_U_ONLY) return;
    #pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        dot += __shfl_xor_sync(0xffffffffu, dot, o);
        s += __shfl_xor_sync(0xffffffffu, s, o);
    }
    const R y = p[D];
    const R c = p[D + 1];
    const R t = R(1) - y * dot;
    R gy = R(0);
    if (t > R(0)) {
        R gam = t / s;
        if (gam > c) gam = c;
        gy = gam * y;
    }
    #pragma unroll
    for (int q = 0; q < JMAX; ++q) {
        const int j = lane + 32 * q;
        if (j > D) continue;
        const R x = n[q] + (gy * xi[q]) / rho[q];
        edge_post<R, FAST>(a, io, e0 + j, ix[q], x, u[q]);
    }
}

// Appendix C one-point margin: the indicator of y (w.x + b) >= 1 - xi on
// (w in R^D, b, xi), one thread per factor.  The prox is the rho-weighted
// projection onto the half-space a.v >= 1 with a = (y x, y, 1):
// v = n + lambda a / rho, lambda = (1 - a.n)^+ / sum_k a_k^2 / rho_k.  Two
// passes over the factor's edges (the first forms a.n and the weight sum in
// the order of a serial loop, the second writes x).  Parameters
// factor-major: p[f*(D+1) + j] = x_j, then y.
template <typename R, int MODE, int FAST>
__device__ __forceinline__ void item_svm_margin(const SweepArgs<R> &a, const BucketDev<R> &B, const EdgeIO<R> &io,
                                                int f, double &pri) {
    const int D = B.arity - 2;
    const R *p = B.prm + (long long)f * (D + 1);
    const R y = p[D];
    R an = R(0), awa = R(0);
    for (int j = 0; j < D + 2; ++j) {
        const int e = bedge(B, f, j);
        R u;
        unsigned ix;
        const R n = edge_pre<R, MODE, FAST>(a, io, e, u, ix, pri);
        const R aj = j < D ? y * p[j] : (j == D ? y : R(1));
        an += aj * n;
        awa += (aj * aj) / edge_rho(a, e);
    }
    if (MODE == F_U_ONLY) return;
    const R viol = R(1) - an;
    const R lam = viol > R(0) ? viol / awa : R(0);
    for (int j = 0; j < D + 2; ++j) {
        const int e = bedge(B, f, j);
        const R u = a.u[e];
        unsigned ix;
        const R n = edge_z<R, FAST>(a, io, e, ix) - u;
        const R aj = j < D ? y * p[j] : (j == D ? y : R(1));
        edge_post<R, FAST>(a, io, e, ix, n + (lam * aj) / edge_rho(a, e), u);
    }
}

// The margin operator with one warp per factor (fast and scatter orders): lane l owns
// the edges j = l, l + 32, ...; a.n and the weight sum are reduced with a
// fixed shuffle tree; one pass, the factor's edges and data point read
// contiguously (factor-major storage).
template <typename R, int MODE, int FAST = EO_CHUNK>
__device__ __forceinline__ void item_svm_margin_warp(const SweepArgs<R> &a, const BucketDev<R> &B,
                                                     const EdgeIO<R> &io, int f, double &pri) {
    constexpr int JMAX = 4;   // up to 128 edges per factor kept in registers
    const int D = B.arity - 2;
    const int lane = threadIdx.x & 31;
    const R *p = B.prm + (long long)f * (D + 1);
    const R y = p[D];
    const int e0 = B.ebase + f * B.arity;
    R n[JMAX], u[JMAX], rho[JMAX], av[JMAX];
    unsigned ix[JMAX];
    R an = R(0), awa = R(0);
    #pragma unroll
    for (int q = 0; q < JMAX; ++q) {
        const int j = lane + 32 * q;
        if (j > D + 1) continue;
        const int e = e0 + j;
        n[q] = edge_pre<R, MODE, FAST>(a, io, e, u[q], ix[q], pri);
        rho[q] = edge_rho(a, e);
        av[q] = j < D ? y * p[j] : (j == D ? y : R(1));
        an += av[q] * n[q];
        awa += (av[q] * av[q]) / rho[q];
    }
    if (MODE == F_U_ONLY) return;
    #pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        an += __shfl_xor_sync(0xffffffffu, an, o);
        awa += __shfl_xor_sync(0xffffffffu, awa, o);
    }
    const R viol = R(1) - an;
    const R lam = viol > R(0) ? viol / awa : R(0);
    #pragma unroll
    for (int q = 0; q < JMAX; ++q) {
        const int j = lane + 32 * q;
        if (j > D + 1) continue;
        edge_post<R, FAST>(a, io, e0 + j, ix[q], n[q] + (lam * av[q]) / rho[q], u[q]);
    }
}

// Appendix C equality of two copies v1, v2 in R^D: both become the
// rho-weighted mean of the two messages, component by component.  One work
// item per component pair: li = j * nf + f with edge-major storage (the
// pairs of consecutive items sit side by side), li = f * D + j with
// factor-major storage (scatter order: consecutive items take consecutive
// components of one copy).
template <typename R, int MODE, int FAST>
__device__ __forceinline__ void item_equal(const SweepArgs<R> &a, const BucketDev<R> &B, const EdgeIO<R> &io, int li,
                                           double &pri) {
    const int D = B.arity >> 1;
    const int j = B.aos ? li % D : li / B.nf, f = B.aos ? li / D : li - j * B.nf;
    const int e1 = bedge(B, f, j), e2 = bedge(B, f, D + j);
    R u1, u2;
    unsigned i1, i2;
    const R n1 = edge_pre<R, MODE, FAST>(a, io, e1, u1, i1, pri);
    const R n2 = edge_pre<R, MODE, FAST>(a, io, e2, u2, i2, pri);
    if (MODE == F_U_ONLY) return;
    const R r1 = edge_rho(a, e1), r2 = edge_rho(a, e2);
    const R v = (r1 * n1 + r2 * n2) / (r1 + r2);
    edge_post<R, FAST>(a, io, e1, i1, v, u1);
    edge_post<R, FAST>(a, io, e2, i2, v, u2);
}

// NB equality items of one thread, li = i0 + q * step: the loads of all of
// them first (as items_elementwise).
template <typename R, int MODE, int FAST, int NB>
__device__ __forceinline__ void items_equal(const SweepArgs<R> &a, const BucketDev<R> &B, const EdgeIO<R> &io, int i0,
                                            int step, double &pri) {
    const int D = B.arity >> 1;
    R z[NB][2], u[NB][2], xo[NB][2];
    unsigned ix[NB][2];
    int e[NB][2];
    #pragma unroll
    for (int q = 0; q < NB; ++q) {
        const int li = i0 + q * step;
        if (li >= B.nitems) continue;
        const int j = B.aos ? li % D : li / B.nf, f = B.aos ? li / D : li - j * B.nf;
        e[q][0] = bedge(B, f, j);
        e[q][1] = bedge(B, f, D + j);
        #pragma unroll
        for (int k = 0; k < 2; ++k) edge_load<R, MODE, FAST>(a, io, e[q][k], z[q][k], u[q][k], xo[q][k], ix[q][k]);
    }
    #pragma unroll
    for (int q = 0; q < NB; ++q) {
        if (i0 + q * step >= B.nitems) break;
        const R n1 = edge_update<R, MODE>(a, io, e[q][0], z[q][0], xo[q][0], u[q][0], pri);
        const R n2 = edge_update<R, MODE>(a, io, e[q][1], z[q][1], xo[q][1], u[q][1], pri);
        if (MODE == F_U_ONLY) continue;
        const R r1 = edge_rho(a, e[q][0]), r2 = edge_rho(a, e[q][1]);
        const R v = (r1 * n1 + r2 * n2) / (r1 + r2);
        edge_post<R, FAST>(a, io, e[q][0], ix[q][0], v, u[q][0]);
        edge_post<R, FAST>(a, io, e[q][1], ix[q][1], v, u[q][1]);
    }
}

// Appendix B dynamics: v = P n with P the rho-weighted projector onto
// {x' = A x + B u}, precomputed per distinct (A, B, rho).  AC = compile-time
// arity (n kept in registers), or 0 for any arity (n re-formed from u and z
// for each output row).
template <typename R, int MODE, int FAST, int AC>
__device__ __forceinline__ void item_mpc_dyn(const SweepArgs<R> &a, const BucketDev<R> &B, const EdgeIO<R> &io,
                                             int f, double &pri) {
    if constexpr (AC > 0) {
        R n[AC], u[AC];
        unsigned ix[AC];
        // the loads of CH edges at a time before their updates (CH divides
        // AC; small groups keep the register demand within the kernel's)
        constexpr int CH = AC % 4 == 0 ? 4 : AC % 3 == 0 ? 3 : 1;
        #pragma unroll
        for (int k0 = 0; k0 < AC; k0 += CH) {
            R z[CH], xo[CH];
            #pragma unroll
            for (int t = 0; t < CH; ++t)
                edge_load<R, MODE, FAST>(a, io, bedge(B, f, k0 + t), z[t], u[k0 + t], xo[t], ix[k0 + t]);
            #pragma unroll
            for (int t = 0; t < CH; ++t)
                n[k0 + t] = edge_update<R, MODE>(a, io, bedge(B, f, k0 + t), z[t], xo[t], u[k0 + t], pri);
        }
        if (MODE == F_U_ONLY) return;
        const R *P = B.pmat + (long long)B.pidx[f] * AC * AC;
        #pragma unroll 2
        for (int i = 0; i < AC; ++i) {
            R acc = R(0);
            #pragma unroll
            for (int j = 0; j < AC; ++j) acc += __ldg(P + i * AC + j) * n[j];
            edge_post<R, FAST>(a, io, bedge(B, f, i), ix[i], acc, u[i]);
        }
    } else {
        const int A = B.arity;
        for (int k = 0; k < A; ++k) {
            R u;
            unsigned ix;
            edge_pre<R, MODE, FAST>(a, io, bedge(B, f, k), u, ix, pri);
        }
        if (MODE == F_U_ONLY) return;
        const R *P = B.pmat + (long long)B.pidx[f] * A * A;
        for (int i = 0; i < A; ++i) {
            R acc = R(0);
            unsigned ix;
            for (int j = 0; j < A; ++j) {
                const int e = bedge(B, f, j);
                acc += __ldg(P + i * A + j) * (edge_z<R, FAST>(a, io, e, ix) - a.u[e]);
            }
            const int e = bedge(B, f, i);
            edge_z<R, FAST>(a, io, e, ix);
            edge_post<R, FAST>(a, io, e, ix, acc, a.u[e]);
        }
    }
}

// Elementwise types: one work item per scalar edge, item li at storage
// edge ebase + li: component k of factor f at li = k * nf + f (edge-major)
// or li = f * arity + k (factor-major, scatter order).  Parameters SoA:
// prm[j * nf + f]; per-component parameters at j = k.
template <typename R>
__device__ __forceinline__ R elementwise_x(const BucketDev<R> &B, int li, R n, R rho) {
    const int f = B.aos ? li / B.arity : li % B.nf;
    const int pk = B.aos ? (li - f * B.arity) * B.nf + f : li;   // per-component parameter index
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
        x = (rho * n) / (B.prm[pk] + rho);
        break;
    case 8: {  // MPC_BOX
        const R lo = B.prm[f], hi = B.prm[B.nf + f];
        x = n;
        if (x < lo) x = lo;
        if (x > hi) x = hi;
        break;
    }
    case 11: {  // SVM_SLACK: f = lambda xi on xi >= 0
        const R v = n - B.prm[f] / rho;
        x = v > R(0) ? v : R(0);
        break;
    }
    default:  // 9, FIX
        x = B.prm[pk];
        break;
    }
    return x;
}

template <typename R, int MODE, int FAST>
__device__ __forceinline__ void item_elementwise(const SweepArgs<R> &a, const BucketDev<R> &B, const EdgeIO<R> &io,
                                                 int li, double &pri) {
    const int e = B.ebase + li;
    R u;
    unsigned ix;
    const R n = edge_pre<R, MODE, FAST>(a, io, e, u, ix, pri);
    if (MODE == F_U_ONLY) return;
    edge_post<R, FAST>(a, io, e, ix, elementwise_x(B, li, n, edge_rho(a, e)), u);
}

// NB elementwise items of one thread, li = i0 + q * step (q < NB, those
// below B.nitems): the loads of all NB items first, then their updates and
// operators in order (the same arithmetic, item by item, as NB calls of
// item_elementwise).
template <typename R, int MODE, int FAST, int NB>
__device__ __forceinline__ void items_elementwise(const SweepArgs<R> &a, const BucketDev<R> &B, const EdgeIO<R> &io,
                                                  int i0, int step, double &pri) {
    R z[NB], u[NB], xo[NB];
    unsigned ix[NB];
    #pragma unroll
    for (int q = 0; q < NB; ++q) {
        const int li = i0 + q * step;
        if (li < B.nitems) edge_load<R, MODE, FAST>(a, io, B.ebase + li, z[q], u[q], xo[q], ix[q]);
    }
    #pragma unroll
    for (int q = 0; q < NB; ++q) {
        const int li = i0 + q * step;
        if (li >= B.nitems) break;
        const int e = B.ebase + li;
        const R n = edge_update<R, MODE>(a, io, e, z[q], xo[q], u[q], pri);
        if (MODE == F_U_ONLY) continue;
        edge_post<R, FAST>(a, io, e, ix[q], elementwise_x(B, li, n, edge_rho(a, e)), u[q]);
    }
}

// KIND 0: every factor type; KIND 1: graphs without hinge, dynamics, margin
// and equality factors (packing); KIND 2: graphs with margin or equality
// factors but no hinge or dynamics factors (the paper-form SVM); KIND 3:
// dynamics factors of up to 9 edges (4 states, 1 input) and elementwise
// factors, no hinge, margin or equality (the long-horizon MPC): without the
// 28-edge dynamics path the kernel needs fewer registers and fits 4 CTAs
// per SM.  Each kernel is compiled without the paths its graphs lack, so
// that their register demand does not limit it.
template <typename R, int MODE, int FAST, int KIND>
__device__ __forceinline__ void process_in_bucket(const SweepArgs<R> &a, const BucketDev<R> &B, const EdgeIO<R> &io,
                                                  int li, double &pri) {
    // user-supplied operators run their own kernels (run-time compiled)
    if (B.type >= kUserType0) return;
    switch (B.type) {
    case 0: item_pack_pair<R, MODE, FAST>(a, B, io, li, pri); break;
    case 1: item_pack_wall<R, MODE, FAST>(a, B, io, li, pri); break;
    case 4:
        if constexpr (KIND == 0) item_svm_hinge<R, MODE, FAST>(a, B, io, li, pri);
        break;
    case 6:
        if constexpr (KIND == 0) {
            if (B.arity == 28) item_mpc_dyn<R, MODE, FAST, 28>(a, B, io, li, pri);
            else if (B.arity == 9) item_mpc_dyn<R, MODE, FAST, 9>(a, B, io, li, pri);   // 4 states, 1 input
            else item_mpc_dyn<R, MODE, FAST, 0>(a, B, io, li, pri);
        } else if constexpr (KIND == 3) {
            if (B.arity == 9) item_mpc_dyn<R, MODE, FAST, 9>(a, B, io, li, pri);
            else item_mpc_dyn<R, MODE, FAST, 0>(a, B, io, li, pri);
        }
        break;
    case 10:
        if constexpr (KIND != 1) item_svm_margin<R, MODE, FAST>(a, B, io, li, pri);
        break;
    case 12:
        if constexpr (KIND != 1) item_equal<R, MODE, FAST>(a, B, io, li, pri);
        break;
    default: item_elementwise<R, MODE, FAST>(a, B, io, li, pri); break;
    }
}

// Issues one stage of bulk copies (u, x when needed, index) for the disk
// pairs [fs, fs + ns) into `buf`, completing on `bar`.
template <typename R, int MODE>
__device__ __forceinline__ void issue_pair_stage(const SweepArgs<R> &a, const EdgeIO<R> &io, const BucketDev<R> &B,
                                                 const ChunkSmem &L, unsigned char *buf, unsigned long long *bar,
                                                 int fs, int ns) {
    const unsigned br = (unsigned)align16(6 * ns * (int)sizeof(R));
    const unsigned bi = (unsigned)align16(6 * ns * 4);
    const int e0 = B.ebase + 6 * fs;
    mbar_expect_tx(bar, br + (MODE != F_PROX ? br : 0u) + bi);
    bulk_g2s(buf + L.stage_u, a.u + e0, br, bar);
    if (MODE != F_PROX) bulk_g2s(buf + L.stage_x, io.xin + e0, br, bar);
    bulk_g2s(buf + L.stage_i, a.lidx + e0, bi, bar);
}

// Canonical order: every work item on its own, rho*m scattered to the
// variable-major array.  Fast order: CTAs walk their chunks; a chunk's
// variables ("slots") get their z staged in shared memory, every edge's
// rho*m lands in shared memory sorted by slot, and each slot's sum over the
// chunk (edges in slot order) is written to the variable-major partial
// array.  Both orders are deterministic.
// BATCH (the one-launch-per-phase kernels): elementwise and equality
// items of the scatter order with the loads of two items (two edges) in
// flight together; the persistent kernel, compiled for three or four
// resident CTAs per SM, keeps one item at a time (the batches' extra
// registers would spill there).
template <typename R, int MODE, int KIND_, bool BATCH = false>
__device__ __forceinline__ void phase_f(const SweepArgs<R> &a, EdgeIO<R> io, double &pri) {
    constexpr int KIND = kind_types(KIND_);
    if constexpr (kind_scatter(KIND_)) {
        // scatter order: bucket after bucket over the whole grid, each
        // edge's rho*m straight to its column (or overflow slot); hinge and
        // margin factors one warp each, every other item one thread
        const int gtid = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
        const int wid = gtid >> 5, nw = stride >> 5;
        for (int b = 0; b < a.nb; ++b) {
            const BucketDev<R> &B = a.bk[b];
            if (B.type >= kUserType0) continue;
            if (KIND == 0 && B.type == 4 && B.arity <= 128) {
                for (int i = wid; i < B.nitems; i += nw)
                    item_svm_hinge_warp<R, MODE, EO_SCATTER>(a, B, io, i, pri);
            } else if ((KIND == 0 || KIND == 2) && B.type == 10 && B.arity >= 16 && B.arity <= 128) {
                for (int i = wid; i < B.nitems; i += nw)
                    item_svm_margin_warp<R, MODE, EO_SCATTER>(a, B, io, i, pri);
            } else if (BATCH && B.per_edge) {
                // elementwise buckets: two items per thread with their loads
                // in flight together (the same items, in the same order, as
                // one at a time)
                for (int i = gtid; i < B.nitems; i += 2 * stride)
                    items_elementwise<R, MODE, EO_SCATTER, 2>(a, B, io, i, stride, pri);
            } else if (BATCH && KIND != 1 && B.type == 12) {
                for (int i = gtid; i < B.nitems; i += stride) items_equal<R, MODE, EO_SCATTER, 1>(a, B, io, i, stride, pri);
            } else {
                for (int i = gtid; i < B.nitems; i += stride)
                    process_in_bucket<R, MODE, EO_SCATTER, KIND>(a, B, io, i, pri);
            }
        }
        return;
    }
    if (a.zorder == 0) {
        const int stride = gridDim.x * blockDim.x;
        for (int it = blockIdx.x * blockDim.x + threadIdx.x; it < a.nitems_f; it += stride) {
            int b = 0;
            while (b + 1 < a.nb && it >= a.bk[b + 1].item0) ++b;
            process_in_bucket<R, MODE, EO_CANON, KIND>(a, a.bk[b], io, it - a.bk[b].item0, pri);
            if (MODE != F_U_ONLY && a.wcls) twa_mark<R>(a, a.bk[b], io, it - a.bk[b].item0);
        }
        return;
    }
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr ChunkSmem L = chunk_smem((int)sizeof(R));
    R *pb = reinterpret_cast<R *>(smem_raw + L.pb);
    R *zl = reinterpret_cast<R *>(smem_raw + L.zl);
    int *lr_s = reinterpret_cast<int *>(smem_raw + L.lr);
    int *pp_s = reinterpret_cast<int *>(smem_raw + L.pp);
    unsigned long long *sbar = reinterpret_cast<unsigned long long *>(smem_raw + L.bar);
    io.pb = pb;
    io.zl = zl;
    if (threadIdx.x == 0) {
        mbar_init(&sbar[0], 1);
        mbar_init(&sbar[1], 1);
        mbar_fence_init();
    }
    __syncthreads();
    unsigned parity = 0u;   // bit b: phase of stage barrier b
    bool staged_ok = true;
    for (int c = blockIdx.x; c < a.nchunks; c += gridDim.x) {
        const ChunkDev ch = a.chunks[c];
        const int *lr = a.lrow + ch.lrbase;
        for (int s = threadIdx.x; s <= ch.nslots; s += blockDim.x) {
            lr_s[s] = lr[s] + s;   // segment s starts after s pad elements
            if (s < ch.nslots) {
                zl[s] = ldg_l2(io.zc + a.slot_var[ch.sbase + s]);
                pp_s[s] = a.ppos[ch.sbase + s];
            }
        }
        __syncthreads();
        const BucketDev<R> &B = a.bk[ch.bucket];
        const int f0 = (int)ch.f0;
        if (B.type == 0) {
            // disk pairs: double-buffered bulk copies of (u, x, index) for
            // kStagePairs factors at a time
            const int nst = (ch.nitems + kStagePairs - 1) / kStagePairs;
            if (threadIdx.x == 0) {
                fence_proxy_async_shared();
                issue_pair_stage<R, MODE>(a, io, B, L, smem_raw + L.st, &sbar[0], f0, min(kStagePairs, ch.nitems));
                if (nst > 1)
                    issue_pair_stage<R, MODE>(a, io, B, L, smem_raw + L.st + L.stage_bytes, &sbar[1],
                                              f0 + kStagePairs, min(kStagePairs, ch.nitems - kStagePairs));
            }
            for (int st = 0; st < nst; ++st) {
                const int b = st & 1;
                if (staged_ok) staged_ok = stage_wait(&sbar[b], (parity >> b) & 1u, a.bar);
                parity ^= 1u << b;
                const unsigned char *buf = smem_raw + L.st + b * L.stage_bytes;
                const R *su = reinterpret_cast<const R *>(buf + L.stage_u);
                const R *sx = reinterpret_cast<const R *>(buf + L.stage_x);
                const unsigned *si = reinterpret_cast<const unsigned *>(buf + L.stage_i);
                const int ns = min(kStagePairs, ch.nitems - st * kStagePairs);
                if (staged_ok) {
                    for (int i = threadIdx.x; i < ns; i += blockDim.x)
                        item_pack_pair_staged<R, MODE>(a, B, io, f0 + st * kStagePairs + i, su + 6 * i, sx + 6 * i,
                                                       si + 6 * i, pri);
                }
                __syncthreads();
                if (threadIdx.x == 0 && st + 2 < nst && staged_ok) {
                    fence_proxy_async_shared();
                    issue_pair_stage<R, MODE>(a, io, B, L, smem_raw + L.st + b * L.stage_bytes, &sbar[b],
                                              f0 + (st + 2) * kStagePairs,
                                              min(kStagePairs, ch.nitems - (st + 2) * kStagePairs));
                }
            }
        } else if (KIND == 0 && B.type == 4 && B.arity <= 128) {
            const int warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
            for (int i = warp; i < ch.nitems; i += nwarps) item_svm_hinge_warp<R, MODE>(a, B, io, f0 + i, pri);
        } else if (KIND == 2 && B.type == 10 && B.arity >= 16 && B.arity <= 128) {
            // a warp per margin factor once a factor fills half a warp;
            // smaller factors keep one thread each
            const int warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
            for (int i = warp; i < ch.nitems; i += nwarps) item_svm_margin_warp<R, MODE>(a, B, io, f0 + i, pri);
        } else {
            for (int i = threadIdx.x; i < ch.nitems; i += blockDim.x)
                process_in_bucket<R, MODE, EO_CHUNK, KIND>(a, B, io, f0 + i, pri);
        }
        __syncthreads();
        if (MODE != F_U_ONLY) {
            // one thread per slot, its segment in order (segments are padded
            // by one element, so equal-length neighbours sit in different
            // banks)
            for (int sl = threadIdx.x; sl < ch.nslots; sl += blockDim.x) {
                const int beg = lr_s[sl], end = lr_s[sl + 1] - 1;
                R S = R(0);
                for (int k = beg; k < end; ++k) S += pb[k];
                a.part[pp_s[sl]] = S;
            }
        }
        __syncthreads();
    }
    // u and x written here are read back by bulk copies (async proxy) in the
    // next phase F
    fence_proxy_async_global();
    __syncthreads();
    // after a stage wait ran out a copy may still be in flight: the barriers
    // are then left alone (the grid-wide error word ends the launch)
    if (threadIdx.x == 0 && staged_ok) {
        mbar_inval(&sbar[0]);
        mbar_inval(&sbar[1]);
    }
}

// ---------------------------------------------------------------------------
// phase Z: z_b = sum_k pvm[k] / srho_b over the variable's row.
// ---------------------------------------------------------------------------
template <typename R, bool CHK>
__device__ __forceinline__ void z_store(const SweepArgs<R> &a, int b, R S, const R *zo, R *zn, double &dual) {
    const R zold = zo[b];
    R znew = zold;
    if (a.srho[b] > R(0)) znew = S / a.srho[b];   // a variable without edges keeps z
    zn[b] = znew;
    if constexpr (CHK) {
        const double dz = (double)znew - (double)zold;
        dual += a.srho2[b] * dz * dz;
    }
}

// Shard mode (SHARD = true): instead of z, phase Z writes this shard's
// running sums of rho m, s_out[b] = s_in[b] + (the shard's terms of b).  In
// the canonical order the shard's terms are added one by one onto s_in[b]
// (so shards taken in creation order reproduce the serial sum exactly); in
// the fast order the shard's own sum is added to s_in[b] once.  s_in may
// be null (start from zero).
template <typename R, bool SHARD>
__device__ __forceinline__ R shard_start(const R *s_in, long long b) {
    if constexpr (SHARD) return s_in ? s_in[b] : R(0);
    return R(0);
}

template <typename R, bool CHK, bool SHARD = false, bool SCAT = false>
__device__ __forceinline__ void phase_z(const SweepArgs<R> &a, const R *zo, R *zn, double &dual,
                                        const R *s_in = nullptr, R *s_out = nullptr) {
    const long long gtid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long gstride = (long long)gridDim.x * blockDim.x;
    auto finish = [&](int b, R S) {
        if constexpr (SHARD) s_out[b] = S;
        else z_store<R, CHK>(a, b, S, zo, zn, dual);
    };
    auto finish_sum = [&](int b, R S) {   // fast order: one sum per shard
        if constexpr (SHARD) s_out[b] = s_in ? s_in[b] + S : S;
        else z_store<R, CHK>(a, b, S, zo, zn, dual);
    };
    if (!SCAT && !SHARD && a.zorder == 0 && a.wcls) {
        // canonical, three weights: per variable, in creation order, the
        // infinite-weight messages (m), the others (rho m) and among them
        // the standard ones; z from the first non-empty group
        for (long long b = gtid; b < a.nz; b += gstride) {
            R S = R(0), Rr = R(0), Ss = R(0), Rs = R(0), Si = R(0), Ni = R(0);
            auto add = [&](int k, R v, int c) {
                if (c == 2) {
                    Si += v;
                    Ni += R(1);
                } else {
                    const R r = a.prho ? a.prho[k] : a.rho_u;
                    S += v;
                    Rr += r;
                    if (c == 1) {
                        Ss += v;
                        Rs += r;
                    }
                }
            };
            const int k1 = a.row[b + 1];
            int k = a.row[b];
            // eight messages and classes loaded together, then added one by
            // one in creation order (the same sums as one at a time)
            for (; k + 8 <= k1; k += 8) {
                R v[8];
                int c[8];
                #pragma unroll
                for (int t = 0; t < 8; ++t) {
                    v[t] = ldg_l2(a.pvm + k + t);
                    c[t] = a.pwcls[k + t];
                }
                #pragma unroll
                for (int t = 0; t < 8; ++t) add(k + t, v[t], c[t]);
            }
            for (; k < k1; ++k) add(k, ldg_l2(a.pvm + k), a.pwcls[k]);
            const R zold = zo[b];
            R znew = zold;
            if (Ni > R(0)) znew = Si / Ni;
            else if (Rs > R(0)) znew = Ss / Rs;
            else if (Rr > R(0)) znew = S / Rr;
            zn[b] = znew;
            if constexpr (CHK) {
                const double dz = (double)znew - (double)zold;
                dual += a.srho2[b] * dz * dz;
            }
        }
        return;
    }
    if (!SCAT && a.zorder == 0) {
        // canonical.  Rows of at most kZShort values: one thread per
        // variable over the whole grid, its values added one by one in
        // creation order straight from the variable-major array.
        for (long long b = gtid; b < a.nz; b += gstride) {
            const int k0 = a.row[b], k1 = a.row[b + 1];
            if (k1 - k0 > kZShort) continue;
            R S = shard_start<R, SHARD>(s_in, b);
            for (int k = k0; k < k1; ++k) S += ldg_l2(a.pvm + k);
            finish((int)b, S);
        }
        // Longer rows: warp 0 of a CTA takes 32 consecutive variables, one
        // per lane; the warp copies 32 values of each of the 32 rows at a
        // time into shared memory (cp.async, zero past a row's end; two
        // buffers, the next block in flight while this one is added) and
        // each lane adds its own row's values one by one in creation order.
        // One lane per variable keeps every FP64 addition of a warp useful.
        // Both paths add in the same order, so the sums are the same.
        if ((threadIdx.x >> 5) == 0) {
            extern __shared__ __align__(16) unsigned char zs_raw[];
            R *zbuf = reinterpret_cast<R *>(zs_raw);   // [2][32 rows][kZRow]
            const int lane = threadIdx.x & 31;
            for (long long base = (long long)blockIdx.x * 32; base < a.nz; base += (long long)gridDim.x * 32) {
                const long long b = base + lane;
                const int k0r = b < a.nz ? a.row[b] : 0, lenr = b < a.nz ? a.row[b + 1] - k0r : 0;
                const bool valid = b < a.nz && lenr > kZShort;   // short rows are done above
                const int k0 = valid ? k0r : 0, len = valid ? lenr : 0;
                int maxlen = len;
                #pragma unroll
                for (int o = 16; o > 0; o >>= 1) maxlen = max(maxlen, __shfl_xor_sync(0xffffffffu, maxlen, o));
                const int nch = (maxlen + 31) / 32;
                R S = valid ? shard_start<R, SHARD>(s_in, b) : R(0);
                auto issue = [&](int c) {
                    R *buf = zbuf + (c & 1) * 32 * kZRow;
                    #pragma unroll 4
                    for (int j = 0; j < 32; ++j) {
                        const int kj0 = __shfl_sync(0xffffffffu, k0, j), lj = __shfl_sync(0xffffffffu, len, j);
                        const int t = c * 32 + lane;
                        cp_async_zfill<R>(buf + j * kZRow + lane, a.pvm + (t < lj ? kj0 + t : 0), t < lj);
                    }
                    cp_async_commit();
                };
                if (nch > 0) issue(0);
                for (int c = 0; c < nch; ++c) {
                    if (c + 1 < nch) {
                        issue(c + 1);
                        cp_async_wait_group<1>();
                    } else {
                        cp_async_wait_group<0>();
                    }
                    __syncwarp();
                    const R *row = zbuf + (c & 1) * 32 * kZRow + lane * kZRow;
                    const int n = min(32, len - c * 32);
                    for (int t = 0; t < n; ++t) S += row[t];
                    __syncwarp();
                }
                if (valid) finish((int)b, S);
            }
        }
        return;
    }
    // scatter order: a variable's columns, added in column (= creation)
    // order; the loads of all columns are issued before the additions
    constexpr bool scat = SCAT;
    auto colsum = [&](int b) {
        R v[kColMax];
        #pragma unroll
        for (int c = 0; c < kColMax; ++c) v[c] = c < a.colw ? ldg_l2(a.pvm + (size_t)c * a.nz + b) : R(0);
        R S = R(0);
        #pragma unroll
        for (int c = 0; c < kColMax; ++c)
            if (c < a.colw) S += v[c];
        return S;
    };
    if constexpr (scat && !SHARD) {
        // NB variables per thread: every load of the NB (overflow flags,
        // columns, old z, rho sums) before their stores; the same additions
        // in the same order as colsum and z_store
        constexpr int NB = 4;
        for (long long b0 = gtid; b0 < a.nz; b0 += NB * gstride) {
            int bb[NB];
            bool ok[NB];
            #pragma unroll
            for (int q = 0; q < NB; ++q) {
                const long long b = b0 + q * gstride;
                bb[q] = (int)b;
                ok[q] = b < a.nz && !a.zovf[b];
            }
            R S[NB];
            #pragma unroll
            for (int q = 0; q < NB; ++q) S[q] = R(0);
            for (int c0 = 0; c0 < a.colw; c0 += 4) {
                R v[NB][4];
                #pragma unroll
                for (int q = 0; q < NB; ++q) {
                    #pragma unroll
                    for (int t = 0; t < 4; ++t)
                        v[q][t] = (ok[q] && c0 + t < a.colw) ? ldg_l2(a.pvm + (size_t)(c0 + t) * a.nz + bb[q]) : R(0);
                }
                #pragma unroll
                for (int q = 0; q < NB; ++q) {
                    #pragma unroll
                    for (int t = 0; t < 4; ++t)
                        if (c0 + t < a.colw) S[q] += v[q][t];
                }
            }
            R zold[NB], sr[NB];
            #pragma unroll
            for (int q = 0; q < NB; ++q) {
                zold[q] = ok[q] ? zo[bb[q]] : R(0);
                sr[q] = ok[q] ? a.srho[bb[q]] : R(0);
            }
            #pragma unroll
            for (int q = 0; q < NB; ++q) {
                if (!ok[q]) continue;
                R znew = zold[q];
                if (sr[q] > R(0)) znew = S[q] / sr[q];   // a variable without edges keeps z
                zn[bb[q]] = znew;
                if constexpr (CHK) {
                    const double dz = (double)znew - (double)zold[q];
                    dual += a.srho2[bb[q]] * dz * dz;
                }
            }
        }
    } else if constexpr (scat) {
        for (long long b = gtid; b < a.nz; b += gstride)
            if (!a.zovf[b]) finish_sum((int)b, colsum((int)b));
    }
    // fast: sums of the chunk partials, row by row (variable-major); scatter:
    // the overflow rows, the columns added first
    const R *src = scat ? a.pvm + a.ovf0 : a.part;
    const int *row = a.prow;
    // low-degree variables one thread each (fast order; none in scatter) ...
    for (long long i = gtid; i < a.n_small; i += gstride) {
        const int b = a.small_vars[i];
        R S = R(0);
        for (int k = row[b]; k < row[b + 1]; ++k) S += ldg_l2(src + k);
        finish_sum(b, S);
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
            if (lane == 0) finish_sum(wi.x, scat ? colsum(wi.x) + S : S);
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
                finish_sum(wi.x, scat ? colsum(wi.x) + T : T);
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
    return io;
}

// ---------------------------------------------------------------------------
// the persistent kernel: a whole call in one launch
// ---------------------------------------------------------------------------
template <typename R, int KIND>
__global__ void __launch_bounds__(256, (sizeof(R) == 4 && (kind_types(KIND) == 1 || kind_types(KIND) == 3)) ? 4 : 3)
    k_sweep_persistent(const SweepArgs<R> a) {
    constexpr bool SCAT = kind_scatter(KIND);
    unsigned int gen = 0;
    const unsigned int G = gridDim.x;
    bool skip = (a.skip_block == (int)blockIdx.x);
    int xp = a.xpar0, zp = a.zpar0;
    for (long long it = 1; it <= a.K; ++it) {
        const bool pend = it > 1;
        const bool chk = pend && ((a.k0 + it - 1) % a.check_every == 0);
        const EdgeIO<R> io = make_io(a, xp, zp);
        double pri = 0.0;
        if (chk) phase_f<R, F_U_PROX_CHK, KIND>(a, io, pri);
        else if (pend) phase_f<R, F_U_PROX, KIND>(a, io, pri);
        else phase_f<R, F_PROX, KIND>(a, io, pri);
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
        if (chkz) phase_z<R, true, false, SCAT>(a, a.z[zp], a.z[zp ^ 1], dual);
        else phase_z<R, false, false, SCAT>(a, a.z[zp], a.z[zp ^ 1], dual);
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
    phase_f<R, F_U_ONLY, KIND>(a, io, pri);
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
template <typename R, int MODE, int KIND>
__global__ void __launch_bounds__(256) k_phase_f(const SweepArgs<R> a, int xp, int zp) {
    if (*(volatile int *)&a.ctl->done) return;
    const EdgeIO<R> io = make_io(a, xp, zp);
    double pri = 0.0;
    phase_f<R, MODE, KIND, true>(a, io, pri);
    if constexpr (fmode_checks(MODE)) {
        const double s = block_sum(pri);
        if (threadIdx.x == 0) a.res_pri[blockIdx.x] = s;
    }
}

template <typename R, bool SCAT>
__global__ void __launch_bounds__(256) k_phase_z(const SweepArgs<R> a, int zp, long long it, int chk) {
    if (*(volatile int *)&a.ctl->done) return;
    double dual = 0.0;
    if (chk) phase_z<R, true, false, SCAT>(a, a.z[zp], a.z[zp ^ 1], dual);
    else phase_z<R, false, false, SCAT>(a, a.z[zp], a.z[zp ^ 1], dual);
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

// ---------------------------------------------------------------------------
// shard mode (the graph holds a contiguous slice of the factors; z needs the
// rho m sums of every shard): phase F as above, then these kernels.
// ---------------------------------------------------------------------------
// This shard's running sums s_out = s_in + its terms (see phase_z).
template <typename R>
__global__ void __launch_bounds__(256) k_shard_sums(const SweepArgs<R> a, const R *s_in, R *s_out) {
    double unused = 0.0;
    phase_z<R, false, true>(a, nullptr, nullptr, unused, s_in, s_out);
}

// Rank-ordered sum of G shards' own sums: total[b] = ((p_0 + p_1) + p_2) ...
template <typename R>
__global__ void __launch_bounds__(256) k_shard_add_parts(const R *parts, int G, long long nz, R *total) {
    for (long long b = (long long)blockIdx.x * blockDim.x + threadIdx.x; b < nz;
         b += (long long)gridDim.x * blockDim.x) {
        R S = parts[b];
        for (int r = 1; r < G; ++r) S += parts[(long long)r * nz + b];
        total[b] = S;
    }
}

// z from the graph-wide sums (the graph's srho / srho2 hold the totals of
// every shard); with CHK the dual residual's per-CTA partial sums.
template <typename R, bool CHK>
__global__ void __launch_bounds__(256) k_shard_z(const SweepArgs<R> a, const R *total, int zp) {
    double dual = 0.0;
    for (long long b = (long long)blockIdx.x * blockDim.x + threadIdx.x; b < a.nz;
         b += (long long)gridDim.x * blockDim.x)
        z_store<R, CHK>(a, (int)b, total[b], a.z[zp], a.z[zp ^ 1], dual);
    if constexpr (CHK) {
        const double s = block_sum(dual);
        if (threadIdx.x == 0) a.res_dual[blockIdx.x] = s;
    }
}

// n per-CTA partials added into one FP64 value by a fixed shuffle tree
// (deterministic); one warp.
template <typename R>
__global__ void __launch_bounds__(32) k_shard_total(const double *part, int n, double *out) {
    const double s = warp_sum_partials(part, n);
    if (threadIdx.x == 0) *out = s;
}

}  // namespace fga
