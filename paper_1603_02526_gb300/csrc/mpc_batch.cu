// mpc_batch.cu -- batched ragged MPC: many small factor graphs (Sec. V-B,
// Appendix B) solved by Algorithm 2 in one persistent launch.
//
// Each CTA takes instances from a work counter (longest horizons first),
// keeps the instance's whole state (x, u, n per edge; z per variable; the
// dynamics projector) in shared memory, and
// iterates with CTA-local synchronisation only:
//   X   x-update: dynamics rows v = P n, quadratic costs rho n / (w + rho),
//       boxes clamp, fixed x_0
//   Z   per variable: z_b = sum rho (x + u) / sum rho over its 2 or 3 edges,
//       then on those edges u += alpha (x - z_b), n = z_b - u (+ the primal
//       and dual residual partials on check iterations)
// and stops when both RMS residuals of a checked iteration (FP64 sums of
// the threads' partials) meet the tolerances, or at the iteration budget.
// The stored state is then exactly the state after the reported number of
// iterations.
#include <cuda_runtime.h>

#include <cmath>

#include "mpc_internal.h"
#include "residual.cuh"

namespace fga {

namespace {

constexpr int kENonFinite = -6;
constexpr int kEBudget = -7;

struct Shape {
    int nx, nu, S, A, T, E, V;
    __device__ int dyn(int t) const { return nx + t * A; }
    __device__ int quad(int t) const { return nx + A * T + t * S; }
    __device__ int quadT() const { return nx + A * T + S * T; }
    __device__ int box(int t) const { return 2 * nx + A * T + S * T + t * nu; }
};

__device__ __forceinline__ Shape make_shape(int nx, int nu, int T) {
    Shape g;
    g.nx = nx;
    g.nu = nu;
    g.S = nx + nu;
    g.A = 2 * nx + nu;
    g.T = T;
    g.E = 2 * nx + (3 * nx + 3 * nu) * T;
    g.V = g.S * T + nx;
    return g;
}

// scalar variable (z index) of scalar edge e
__device__ __forceinline__ int edge_var(const Shape &g, int e) {
    if (e < g.nx) return e;                                   // FIX(x_0)
    e -= g.nx;
    if (e < g.A * g.T) {                                      // DYN(x_t, u_t, x_t+1)
        const int t = e / g.A, c = e - t * g.A;
        return c < g.S ? t * g.S + c : (t + 1) * g.S + (c - g.S);
    }
    e -= g.A * g.T;
    if (e < g.S * g.T) return e;                              // QUAD(x_t, u_t): t*S + c
    e -= g.S * g.T;
    if (e < g.nx) return g.T * g.S + e;                       // QUAD(x_T)
    e -= g.nx;
    const int t = e / g.nu;                                   // BOX(u_t)
    return t * g.S + g.nx + (e - t * g.nu);
}

// the 2 or 3 edges of scalar variable b, ascending creation order
__device__ __forceinline__ int var_edges(const Shape &g, int b, int *ed) {
    if (b >= g.T * g.S) {                                     // x_T
        const int c = b - g.T * g.S;
        ed[0] = g.dyn(g.T - 1) + g.S + c;
        ed[1] = g.quadT() + c;
        return 2;
    }
    const int t = b / g.S, c = b - t * g.S;
    if (c < g.nx) {                                           // x_t
        ed[0] = t == 0 ? c : g.dyn(t - 1) + g.S + c;
        ed[1] = g.dyn(t) + c;
        ed[2] = g.quad(t) + c;
        return 3;
    }
    const int cu = c - g.nx;                                  // u_t
    ed[0] = g.dyn(t) + g.nx + cu;
    ed[1] = g.quad(t) + g.nx + cu;
    ed[2] = g.box(t) + cu;
    return 3;
}

// The same edges as var_edges, computed with selects (no divergence
// between state and input variables in a warp): x_t (t >= 1) has
// DYN_{t-1}, DYN_t, QUAD_t; x_0 has FIX, DYN_0, QUAD_0; u_t has DYN_t,
// QUAD_t, BOX_t; x_T has DYN_{T-1}, QUAD_T.  Ascending in every case.
__device__ __forceinline__ int var_edges_sel(const Shape &g, int b, int *ed) {
    const int t = b / g.S, c = b - t * g.S;
    const bool is_u = c >= g.nx, last = t == g.T;
    const int prev = t == 0 ? c : g.dyn(t - 1) + g.S + c;
    ed[0] = is_u ? g.dyn(t) + c : prev;
    ed[1] = last ? g.quadT() + c : (is_u ? g.quad(t) + c : g.dyn(t) + c);
    ed[2] = is_u ? g.box(t) + (c - g.nx) : g.quad(t) + c;
    return last ? 2 : 3;
}

struct CheckOut {
    bool stop;
    int status;
    double rp, rd;
};

// Four consecutive values from a 16-byte aligned shared-memory address.
__device__ __forceinline__ void ld4(const float *p, float *v) {
    const float4 t = *reinterpret_cast<const float4 *>(p);
    v[0] = t.x;
    v[1] = t.y;
    v[2] = t.z;
    v[3] = t.w;
}
__device__ __forceinline__ void ld4(const double *p, double *v) {
    const double2 a = *reinterpret_cast<const double2 *>(p), b = *reinterpret_cast<const double2 *>(p + 2);
    v[0] = a.x;
    v[1] = a.y;
    v[2] = b.x;
    v[3] = b.y;
}

// Residual check of one iteration.  Each thread's squared primal and dual
// residual partials are summed by a fixed tree (warps by shuffles, then the
// warps in order by thread 0, which alone decides); every thread returns
// the same decision.  FP64 state sums in FP64.  FP32 state sums in float
// pairs (TwoSum), which carry the sum to about 2^-44 relative: an FP64-class
// sum without the FP64 pipe, whose dependent adds cost about 64 cycles
// each here; the reported norms are formed in FP64 from the pair.  red
// holds at least 34 doubles (up to 16 warps) and flag 2 ints.
template <int NT>
__device__ __forceinline__ CheckOut block_check(float pri, float dual, const ResidualTest &tp_,
                                                const ResidualTest &td_, double tol_pri, double tol_dual, bool last,
                                                double *red, int *flag) {
    float pl = 0.f, dl = 0.f;
    #pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float ah = __shfl_xor_sync(0xffffffffu, pri, o), alo = __shfl_xor_sync(0xffffffffu, pl, o);
        const float bh = __shfl_xor_sync(0xffffffffu, dual, o), blo = __shfl_xor_sync(0xffffffffu, dl, o);
        ff_add(pri, pl, ah, alo);
        ff_add(dual, dl, bh, blo);
    }
    float *rf = reinterpret_cast<float *>(red);
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        rf[w] = pri;
        rf[16 + w] = pl;
        rf[32 + w] = dual;
        rf[48 + w] = dl;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        float ph = rf[0], plo = rf[16], dh = rf[32], dlo = rf[48];
        for (int i = 1; i < NT / 32; ++i) {
            ff_add(ph, plo, rf[i], rf[16 + i]);
            ff_add(dh, dlo, rf[32 + i], rf[48 + i]);
        }
        const bool finite = isfinite(ph) && isfinite(dh);
        const bool conv = finite && tp_.pass(ph, plo) && td_.pass(dh, dlo);
        const bool stop = !finite || conv || last;
        if (stop) {
            red[32] = sqrt(((double)ph + (double)plo) / tp_.E);
            red[33] = sqrt(((double)dh + (double)dlo) / td_.E);
        }
        flag[0] = stop;
        flag[1] = !finite ? kENonFinite : (conv || (tol_pri <= 0.0 && tol_dual <= 0.0)) ? 0 : kEBudget;
    }
    __syncthreads();
    CheckOut c;
    c.stop = flag[0] != 0;
    c.status = flag[1];
    c.rp = red[32];
    c.rd = red[33];
    return c;
}

template <int NT>
__device__ __forceinline__ CheckOut block_check(double pri, double dual, const ResidualTest &tp_,
                                                const ResidualTest &td_, double tol_pri, double tol_dual, bool last,
                                                double *red, int *flag) {
    #pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        pri += __shfl_xor_sync(0xffffffffu, pri, o);
        dual += __shfl_xor_sync(0xffffffffu, dual, o);
    }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        red[w] = pri;
        red[16 + w] = dual;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double tp = 0.0, td = 0.0;
        for (int i = 0; i < NT / 32; ++i) {
            tp += red[i];
            td += red[16 + i];
        }
        const bool finite = isfinite(tp) && isfinite(td);
        const bool conv = finite && tp_.pass(tp) && td_.pass(td);
        const bool stop = !finite || conv || last;
        if (stop) {
            red[32] = sqrt(tp / tp_.E);
            red[33] = sqrt(td / td_.E);
        }
        flag[0] = stop;
        flag[1] = !finite ? kENonFinite : (conv || (tol_pri <= 0.0 && tol_dual <= 0.0)) ? 0 : kEBudget;
    }
    __syncthreads();
    CheckOut c;
    c.stop = flag[0] != 0;
    c.status = flag[1];
    c.rp = red[32];
    c.rd = red[33];
    return c;
}

}  // namespace

int mpc_smem_bytes(int rsize, int nx, int nu, int tmax, int threads) {
    (void)threads;
    const int A = 2 * nx + nu;
    const int E = 2 * nx + (3 * nx + 3 * nu) * tmax;
    const int V = (nx + nu) * tmax + nx;
    int b = (3 * E + V + A * (A + 1) + 3 * nx + 2 * nu) * rsize;
    b = (b + 15) & ~15;
    return b + 72 * (int)sizeof(double);
}

// NXC, NUC: the state and input sizes when known at compile time (the
// index arithmetic then divides by constants, and each thread keeps one row
// of the dynamics projector in registers), 0 for sizes given at run time.
template <typename R, int NT, int NXC, int NUC>
__global__ void __launch_bounds__(NT) k_mpc_batch(const MpcArgs<R> a) {
    extern __shared__ __align__(16) unsigned char sm[];
    __shared__ int s_k;
    __shared__ int s_flag[2];
    constexpr int AC = 2 * NXC + NUC;             // dynamics factor arity (compile time), 0 if unknown
    constexpr int GC = AC ? NT / (AC ? AC : 1) : 0;   // dynamics factors a pass covers, one row per thread
    // 16-byte loads of a dynamics factor's n: the factor starts at nx + t A
    // within n, n at 2 E values from a 16-byte aligned base, E even when
    // nx + nu is; so nx, nu multiples of 4 (float) or 2 (double) suffice
    constexpr bool VEC = AC != 0 && AC % 4 == 0 &&
                         (sizeof(R) == 4 ? (NXC % 4 == 0 && NUC % 4 == 0) : (NXC % 2 == 0 && NUC % 2 == 0));
    const int nx = NXC ? NXC : a.nx, nu = NUC ? NUC : a.nu, A = 2 * nx + nu, LP = A + 1;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_k = (int)atomicAdd(a.queue, 1u);
        __syncthreads();
        const int k = s_k;
        if (k >= a.n_inst) return;
        const int inst = a.order[k];
        const Shape g = make_shape(nx, nu, a.T[inst]);
        R *x = reinterpret_cast<R *>(sm);
        R *u = x + g.E;
        R *nb = u + g.E;
        R *z = nb + g.E;
        R *P = z + g.V;
        R *q = P + A * LP;
        R *r = q + nx;
        R *x0 = r + nu;
        R *cw = x0 + nx;                 // rho / (w + rho) per cost component (nx states, nu inputs)
        const int nvals = 3 * g.E + g.V + A * LP + 3 * nx + 2 * nu;
        double *red = reinterpret_cast<double *>(sm + ((nvals * (int)sizeof(R) + 15) & ~15));
        const long long eo = a.eoff[inst], zof = a.zoff[inst];
        const int sy = a.sys[inst];
        for (int e = threadIdx.x; e < g.E; e += NT) {
            x[e] = a.x[eo + e];
            u[e] = a.u[eo + e];
        }
        for (int b = threadIdx.x; b < g.V; b += NT) z[b] = a.z[zof + b];
        for (int j = threadIdx.x; j < A * A; j += NT) P[(j / A) * LP + (j % A)] = a.P[(long long)sy * A * A + j];
        for (int j = threadIdx.x; j < nx; j += NT) {
            q[j] = a.q[sy * nx + j];
            x0[j] = a.x0[(long long)inst * nx + j];
        }
        for (int j = threadIdx.x; j < nu; j += NT) r[j] = a.r[sy * nu + j];
        for (int j = threadIdx.x; j < nx + nu; j += NT) {
            const R w = j < nx ? a.q[sy * nx + j] : a.r[sy * nu + j - nx];
            cw[j] = a.rho / (w + a.rho);
        }
        __syncthreads();
        // n = z - u of the stored state
        for (int e = threadIdx.x; e < g.E; e += NT) nb[e] = z[edge_var(g, e)] - u[e];
        // this thread's projector row (compile-time sizes): row prow of the
        // dynamics factors pgrp, pgrp + GC, ...
        const int prow = AC ? (int)threadIdx.x % (AC ? AC : 1) : 0;
        const int pgrp = AC ? (int)threadIdx.x / (AC ? AC : 1) : 0;
        R Pr[AC ? AC : 1];
        if (AC) {
            #pragma unroll
            for (int j = 0; j < (AC ? AC : 1); ++j) Pr[j] = pgrp < GC ? P[prow * LP + j] : R(0);
        }
        __syncthreads();

        const R rho = a.rho, alpha = a.alpha;
        ResidualTest rtp, rtd;   // used by thread 0
        if (threadIdx.x == 0) {
            rtp.init((double)g.E, a.tol_pri);
            rtd.init((double)g.E, a.tol_dual);
        }
        long long done = 0;
        int status = 0;
        double rp = nan(""), rd = nan("");
        const long long K = a.max_iters;
        const int ce = a.check_every;
        const int nrow = g.T * A;
        const int new_ = g.E - nrow;   // elementwise edges: FIX (first nx), then costs and boxes
        int rm = 1 % ce;   // it mod check_every, kept by counting (no 64-bit division per iteration)
        // The elementwise operators (FIX, costs, boxes) need only their own
        // edge's n, so the Z phase of an unchecked iteration applies them to
        // the n it has just formed (x of the next iteration, the same
        // formulas); ew_pending marks an x not advanced that way (the first
        // iteration, and after a checked one, whose stored x must stay).
        bool ew_pending = true;
        for (long long it = 1; it <= K; ++it) {
            // X: x-update.  Dynamics rows v = P n, then the elementwise edges.
            if (AC) {
                if (pgrp < GC) {
                    for (int t = pgrp; t < g.T; t += GC) {
                        const R *n = nb + g.dyn(t);
                        R s0 = R(0), s1 = R(0), s2 = R(0), s3 = R(0);
                        if (VEC) {
                            // n is 16-byte aligned here (see VEC): one vector load per 4 (float) or 2 (double) values
                            #pragma unroll
                            for (int j = 0; j < (AC ? AC : 4); j += 4) {
                                R v[4];
                                ld4(n + j, v);
                                s0 += Pr[j] * v[0];
                                s1 += Pr[j + 1] * v[1];
                                s2 += Pr[j + 2] * v[2];
                                s3 += Pr[j + 3] * v[3];
                            }
                        } else {
                            #pragma unroll
                            for (int j = 0; j + 3 < (AC ? AC : 1); j += 4) {
                                s0 += Pr[j] * n[j];
                                s1 += Pr[j + 1] * n[j + 1];
                                s2 += Pr[j + 2] * n[j + 2];
                                s3 += Pr[j + 3] * n[j + 3];
                            }
                            #pragma unroll
                            for (int j = (AC ? AC : 1) & ~3; j < (AC ? AC : 1); ++j) s0 += Pr[j] * n[j];
                        }
                        x[g.dyn(t) + prow] = (s0 + s1) + (s2 + s3);
                    }
                }
            } else {
                for (int item = threadIdx.x; item < nrow; item += NT) {
                    const int t = item / A, row = item - t * A;
                    const R *n = nb + g.dyn(t);
                    const R *Pp = P + row * LP;
                    R acc = R(0);
                    for (int j = 0; j < A; ++j) acc += Pp[j] * n[j];
                    x[g.dyn(t) + row] = acc;
                }
            }
            for (int i = ew_pending ? (int)threadIdx.x : new_; i < new_; i += NT) {
                if (i < nx) {
                    x[i] = x0[i];
                    continue;
                }
                const int e = i + nrow;
                const R n = nb[e];
                R v;
                if (e < g.quadT()) {
                    v = cw[(e - g.quad(0)) % g.S] * n;
                } else if (e < g.box(0)) {
                    v = cw[e - g.quadT()] * n;
                } else {
                    v = n;
                    if (v < a.lo) v = a.lo;
                    if (v > a.hi) v = a.hi;
                }
                x[e] = v;
            }
            __syncthreads();
            // Z: rho-weighted mean over each variable's edges, then on those
            // edges u += alpha (x - z) and n = z - u (each edge belongs to one
            // variable), with the residual partials on check iterations.
            const bool chk = rm == 0 || it == K;
            ew_pending = chk;
            R pri_r = R(0), dual_r = R(0);
            for (int b = threadIdx.x; b < g.V; b += NT) {
                int ed[3];
                const int ne = var_edges_sel(g, b, ed);
                const int tb = b / g.S, cb = b - tb * g.S;
                const bool ub = cb >= nx;             // an input variable u_t
                R xe[3], ue[3];
                #pragma unroll
                for (int j = 0; j < 3; ++j) {
                    xe[j] = j < ne ? x[ed[j]] : R(0);
                    ue[j] = j < ne ? u[ed[j]] : R(0);
                }
                R znew;
                if (sizeof(R) == 4) {
                    // one rho: z = sum (x + u) / deg, by a multiply with 1 / deg
                    R S = (xe[0] + ue[0]) + (xe[1] + ue[1]);
                    if (ne == 3) S += xe[2] + ue[2];
                    znew = S * (ne == 3 ? R(1) / R(3) : R(0.5));
                } else {
                    // FP64: the definition's sums and division, in edge order
                    R S = rho * (xe[0] + ue[0]) + rho * (xe[1] + ue[1]), Rs = rho + rho;
                    if (ne == 3) {
                        S += rho * (xe[2] + ue[2]);
                        Rs += rho;
                    }
                    znew = S / Rs;
                }
                const R zold = z[b];
                z[b] = znew;
                R nn[3];
                #pragma unroll
                for (int j = 0; j < 3; ++j) {
                    if (j < ne) {
                        const R d = xe[j] - znew;
                        const R un = ue[j] + alpha * d;
                        u[ed[j]] = un;
                        nn[j] = znew - un;
                        nb[ed[j]] = nn[j];
                        if (chk) pri_r += d * d;
                    }
                }
                if (!chk) {
                    // next x of this variable's cost edge (QUAD_t, or QUAD_T for
                    // x_T: the second edge of u_t and x_T, the third of x_t) and
                    // of u_t's box edge; x_0's FIX edge keeps x_0
                    const int qj = (ub || ne == 2) ? 1 : 2;
                    x[ed[qj]] = cw[cb] * nn[qj];
                    if (ub) {
                        R v = nn[2];
                        if (v < a.lo) v = a.lo;
                        if (v > a.hi) v = a.hi;
                        x[ed[2]] = v;
                    }
                }
                if (chk) {
                    const R dz = znew - zold;
                    dual_r += (R)ne * rho * rho * dz * dz;
                }
            }
            rm = rm + 1 == ce ? 0 : rm + 1;
            if (chk) {
                const CheckOut c = block_check<NT>(pri_r, dual_r, rtp, rtd, a.tol_pri, a.tol_dual, it == K, red,
                                                         s_flag);
                if (c.stop) {
                    done = it;
                    status = c.status;
                    rp = c.rp;
                    rd = c.rd;
                    break;
                }
            }
            __syncthreads();
        }
        // store the state of the instance
        __syncthreads();
        for (int e = threadIdx.x; e < g.E; e += NT) {
            a.x[eo + e] = x[e];
            a.u[eo + e] = u[e];
        }
        for (int b = threadIdx.x; b < g.V; b += NT) a.z[zof + b] = z[b];
        if (threadIdx.x == 0) {
            a.iters[inst] = done;
            a.status[inst] = status;
            a.rpri[inst] = rp;
            a.rdual[inst] = rd;
        }
    }
}

template <typename R>
static const void *mpc_kernel(int threads, bool fixed) {
    // 224 and 448 threads: 8 and 16 dynamics factors of 28 rows per pass,
    // every lane busy in the x phase for 12 states and 4 inputs
    if (fixed)
        return threads == 64    ? (const void *)k_mpc_batch<R, 64, 12, 4>
               : threads == 128 ? (const void *)k_mpc_batch<R, 128, 12, 4>
               : threads == 224 ? (const void *)k_mpc_batch<R, 224, 12, 4>
               : threads == 256 ? (const void *)k_mpc_batch<R, 256, 12, 4>
               : threads == 448 ? (const void *)k_mpc_batch<R, 448, 12, 4>
                                : (const void *)k_mpc_batch<R, 512, 12, 4>;
    return threads == 64    ? (const void *)k_mpc_batch<R, 64, 0, 0>
           : threads == 128 ? (const void *)k_mpc_batch<R, 128, 0, 0>
           : threads == 224 ? (const void *)k_mpc_batch<R, 224, 0, 0>
           : threads == 256 ? (const void *)k_mpc_batch<R, 256, 0, 0>
           : threads == 448 ? (const void *)k_mpc_batch<R, 448, 0, 0>
                            : (const void *)k_mpc_batch<R, 512, 0, 0>;
}

template <typename R>
cudaError_t mpc_launch(const MpcArgs<R> &a, int threads, int grid, int smem, cudaStream_t s) {
    // the benchmark's sizes (12 states, 4 inputs) have their own instance
    const bool fixed = a.nx == 12 && a.nu == 4;
    const void *fn = mpc_kernel<R>(threads, fixed);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    void *args[] = {(void *)&a};
    return cudaLaunchKernel(fn, dim3(grid), dim3(threads), args, (size_t)smem, s);
}

// Resident CTAs per SM, the smaller of the two instances' (the grid takes
// work from a counter, so a grid larger than the resident one only waits).
template <typename R>
int mpc_max_blocks_per_sm(int threads, int smem) {
    int best = -1;
    for (bool fixed : {true, false}) {
        const void *fn = mpc_kernel<R>(threads, fixed);
        if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess) return 0;
        int n = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, threads, (size_t)smem) != cudaSuccess) return 0;
        best = best < 0 ? n : (n < best ? n : best);
    }
    return best;
}

// ---------------------------------------------------------------------------
// warm start: from a predicted trajectory and multipliers to (z, u).
// pred row of instance i (stride ld): [T x S values: step t = (x_{t+1}, u_t)]
// then [T x S values: step t = (lambda_t, mu_t)], lambda_t the multiplier of
// the dynamics constraint M v = 0 (M = [A B -I]) and mu_t of the input box.
// At an ADMM fixed point every edge's scaled dual is u = -(1/rho) times the
// factor's (sub)gradient at z, which gives
//   DYN_t:  u = -(1/rho) M^T lambda_t      QUAD: u = -(1/rho) w (.) z
//   BOX_t:  u = -mu_t / rho                FIX:  minus the other u's of x_0
// x is set to z (the first iteration carries no pending u-update).
// ---------------------------------------------------------------------------
template <typename R>
__global__ void k_mpc_warm(const MpcArgs<R> a, const R *Am, const R *Bm, const float *pred, long long ld) {
    const int inst = blockIdx.x;
    if (inst >= a.n_inst) return;
    const int nx = a.nx, nu = a.nu;
    const Shape g = make_shape(nx, nu, a.T[inst]);
    const long long eo = a.eoff[inst], zof = a.zoff[inst];
    const int sy = a.sys[inst];
    const float *pz = pred + (long long)inst * ld;
    const float *pl = pz + (long long)g.T * g.S;
    const R *Ai = Am + (long long)sy * nx * nx, *Bi = Bm + (long long)sy * nx * nu;
    const R *q = a.q + (long long)sy * nx, *r = a.r + (long long)sy * nu;
    const R irho = R(1) / a.rho;
    R *z = a.z + zof, *u = a.u + eo, *x = a.x + eo;
    // z: x_0 from the instance, then (u_t, x_{t+1}) from the prediction
    for (int j = threadIdx.x; j < nx; j += blockDim.x) z[j] = a.x0[(long long)inst * nx + j];
    for (int j = threadIdx.x; j < g.T * g.S; j += blockDim.x) {
        const int t = j / g.S, c = j - t * g.S;
        if (c < nx) z[(t + 1) * g.S + c] = (R)pz[j];
        else z[t * g.S + c] = (R)pz[j];
    }
    __syncthreads();
    for (int t = threadIdx.x; t < g.T; t += blockDim.x) {
        const float *lam = pl + (long long)t * g.S;
        R *ud = u + g.dyn(t);
        // M^T lambda = [A^T lambda; B^T lambda; -lambda]
        for (int c = 0; c < nx; ++c) {
            R s = R(0);
            for (int i = 0; i < nx; ++i) s += Ai[i * nx + c] * (R)lam[i];
            ud[c] = -irho * s;
        }
        for (int c = 0; c < nu; ++c) {
            R s = R(0);
            for (int i = 0; i < nx; ++i) s += Bi[i * nu + c] * (R)lam[i];
            ud[nx + c] = -irho * s;
        }
        for (int c = 0; c < nx; ++c) ud[g.S + c] = irho * (R)lam[c];
        R *uq = u + g.quad(t);
        for (int c = 0; c < nx; ++c) uq[c] = -irho * q[c] * z[t * g.S + c];
        for (int c = 0; c < nu; ++c) uq[nx + c] = -irho * r[c] * z[t * g.S + nx + c];
        R *ub = u + g.box(t);
        for (int c = 0; c < nu; ++c) ub[c] = -irho * (R)lam[nx + c];
    }
    for (int c = threadIdx.x; c < nx; c += blockDim.x) u[g.quadT() + c] = -irho * q[c] * z[g.T * g.S + c];
    __syncthreads();
    for (int c = threadIdx.x; c < nx; c += blockDim.x) u[c] = -(u[g.dyn(0) + c] + u[g.quad(0) + c]);
    for (int e = threadIdx.x; e < g.E; e += blockDim.x) x[e] = z[edge_var(g, e)];
}

template <typename R>
cudaError_t mpc_warm_start_impl(const MpcArgs<R> &a, const R *Am, const R *Bm, const float *pred, long long ld,
                                cudaStream_t s) {
    k_mpc_warm<R><<<a.n_inst, 64, 0, s>>>(a, Am, Bm, pred, ld);
    return cudaGetLastError();
}

// Training targets from a solved batch: z-part (x_{t+1}, u_t) and the
// multipliers lambda_t = -rho K u_dyn_t (K = (M M^T)^{-1} M, per system) and
// mu_t = -rho u_box_t, the inverse of the warm-start map.
template <typename R>
__global__ void k_mpc_targets(const MpcArgs<R> a, const R *K, float *out, long long ld) {
    const int inst = blockIdx.x;
    if (inst >= a.n_inst) return;
    const int nx = a.nx, nu = a.nu, A = 2 * nx + nu;
    const Shape g = make_shape(nx, nu, a.T[inst]);
    const long long eo = a.eoff[inst], zof = a.zoff[inst];
    const int sy = a.sys[inst];
    const R *Ks = K + (long long)sy * nx * A;
    const R *z = a.z + zof, *u = a.u + eo;
    float *oz = out + (long long)inst * ld;
    float *ol = oz + (long long)g.T * g.S;
    for (int j = threadIdx.x; j < g.T * g.S; j += blockDim.x) {
        const int t = j / g.S, c = j - t * g.S;
        oz[j] = (float)(c < nx ? z[(t + 1) * g.S + c] : z[t * g.S + c]);
    }
    for (int j = threadIdx.x; j < g.T * g.S; j += blockDim.x) {
        const int t = j / g.S, c = j - t * g.S;
        if (c < nx) {
            R s = R(0);
            for (int k = 0; k < A; ++k) s += Ks[c * A + k] * u[g.dyn(t) + k];
            ol[j] = (float)(-a.rho * s);
        } else {
            ol[j] = (float)(-a.rho * u[g.box(t) + (c - nx)]);
        }
    }
}

template <typename R>
cudaError_t mpc_targets_impl(const MpcArgs<R> &a, const R *K, float *out, long long ld, cudaStream_t s) {
    k_mpc_targets<R><<<a.n_inst, 64, 0, s>>>(a, K, out, ld);
    return cudaGetLastError();
}

template cudaError_t mpc_launch<float>(const MpcArgs<float> &, int, int, int, cudaStream_t);
template cudaError_t mpc_launch<double>(const MpcArgs<double> &, int, int, int, cudaStream_t);
template int mpc_max_blocks_per_sm<float>(int, int);
template int mpc_max_blocks_per_sm<double>(int, int);
template cudaError_t mpc_warm_start_impl<float>(const MpcArgs<float> &, const float *, const float *, const float *,
                                                long long, cudaStream_t);
template cudaError_t mpc_warm_start_impl<double>(const MpcArgs<double> &, const double *, const double *,
                                                 const float *, long long, cudaStream_t);
template cudaError_t mpc_targets_impl<float>(const MpcArgs<float> &, const float *, float *, long long, cudaStream_t);
template cudaError_t mpc_targets_impl<double>(const MpcArgs<double> &, const double *, float *, long long,
                                              cudaStream_t);

}  // namespace fga
