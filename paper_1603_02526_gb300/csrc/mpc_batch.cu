// mpc_batch.cu -- batched ragged MPC: many small factor graphs (Sec. V-B,
// Appendix B) solved by Algorithm 2 in one persistent launch.
//
// Each CTA takes instances from a work counter (longest horizons first),
// keeps the instance's whole state (x, u, n per edge; z per variable; the
// dynamics projector) in shared memory, and
// iterates with CTA-local synchronisation only:
//   F1  deferred u-update of the previous iteration, n = z - u
//       (+ FP64 primal residual on check iterations)
//   F2  x-update: dynamics rows v = P n, quadratic costs rho n / (w + rho),
//       boxes clamp, fixed x_0
//   Z   z_b = sum rho (x + u) / sum rho over the variable's 2 or 3 edges
//       (+ FP64 dual residual on check iterations)
// and stops when both RMS residuals of a checked iteration meet the
// tolerances, or at the iteration budget.  The stored state is then exactly
// the state after the reported number of iterations.
#include <cuda_runtime.h>

#include <cmath>

#include "mpc_internal.h"

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

// Deterministic block sums of two doubles per thread (fixed shuffle tree,
// then warps in order), broadcast to every thread; red holds 2 x 33 doubles.
template <int NT>
__device__ __forceinline__ void block_sum2_bcast(double &v0, double &v1, double *red) {
    #pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        v0 += __shfl_xor_sync(0xffffffffu, v0, o);
        v1 += __shfl_xor_sync(0xffffffffu, v1, o);
    }
    const int w = threadIdx.x >> 5;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) {
        red[w] = v0;
        red[33 + w] = v1;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t0 = 0.0, t1 = 0.0;
        for (int i = 0; i < NT / 32; ++i) {
            t0 += red[i];
            t1 += red[33 + i];
        }
        red[32] = t0;
        red[65] = t1;
    }
    __syncthreads();
    v0 = red[32];
    v1 = red[65];
}

}  // namespace

int mpc_smem_bytes(int rsize, int nx, int nu, int tmax, int threads) {
    (void)threads;
    const int A = 2 * nx + nu;
    const int E = 2 * nx + (3 * nx + 3 * nu) * tmax;
    const int V = (nx + nu) * tmax + nx;
    int b = (3 * E + V + A * (A + 1) + 2 * nx + nu) * rsize;
    b = (b + 15) & ~15;
    return b + 72 * (int)sizeof(double);
}

// NXC, NUC: the state and input sizes when known at compile time (the
// index arithmetic then divides by constants and the dynamics rows unroll),
// 0 for sizes given at run time.
template <typename R, int NT, int NXC, int NUC>
__global__ void __launch_bounds__(NT) k_mpc_batch(const MpcArgs<R> a) {
    extern __shared__ __align__(16) unsigned char sm[];
    __shared__ int s_k;
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
        const int nvals = 3 * g.E + g.V + A * LP + 2 * nx + nu;
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
        __syncthreads();

        const R rho = a.rho, alpha = a.alpha;
        const double E = (double)g.E;
        long long done = 0;
        int status = 0;
        double rp = nan(""), rd = nan("");
        double dual = 0.0;               // this thread's share of the last checked dual residual
        bool pend = a.first_pending != 0;
        const long long K = a.max_iters;
        const int ce = a.check_every;
        int rm = 1 % ce;   // it mod check_every, kept by counting (no 64-bit division per iteration)
        int rm_prev = 0;   // (it - 1) mod check_every
        for (long long it = 1; K > 0 && it <= K + 1; ++it) {
            const bool last = it == K + 1;
            const bool chk = pend && (rm_prev == 0 || last);
            // F1: u-update of iteration it-1, n-update.  The thread's
            // squared differences are summed in the working precision, the
            // threads' sums in FP64 (the FP64 pipe is narrow on this part).
            R pri_r = R(0);
            for (int e = threadIdx.x; e < g.E; e += NT) {
                const R zb = z[edge_var(g, e)];
                R ue = u[e];
                if (pend) {
                    const R d = x[e] - zb;
                    if (chk) pri_r += d * d;
                    ue = ue + alpha * d;
                    u[e] = ue;
                }
                nb[e] = zb - ue;
            }
            double pri = (double)pri_r;
            if (chk) {
                double sp = pri, sd = dual;
                block_sum2_bcast<NT>(sp, sd, red);
                rp = sqrt(sp / E);
                rd = sqrt(sd / E);
                const bool finite = isfinite(rp) && isfinite(rd);
                if (!finite || (rp <= a.tol_pri && rd <= a.tol_dual) || last) {
                    done = it - 1;
                    status = !finite ? kENonFinite
                                     : ((rp <= a.tol_pri && rd <= a.tol_dual) ||
                                        (a.tol_pri <= 0.0 && a.tol_dual <= 0.0)) ? 0 : kEBudget;
                    break;
                }
            }
            __syncthreads();
            // F2: x-update.  Dynamics rows first (T*A items), then the
            // elementwise edges (FIX, costs, boxes).
            const int nrow = g.T * A;
            const int nitem = nrow + (g.E - nrow);
            for (int item = threadIdx.x; item < nitem; item += NT) {
                if (item < nrow) {
                    const int t = item / A, row = item - t * A;
                    const R *n = nb + g.dyn(t);
                    const R *Pr = P + row * LP;
                    R acc = R(0);
                    #pragma unroll
                    for (int j = 0; j < A; ++j) acc += Pr[j] * n[j];
                    x[g.dyn(t) + row] = acc;
                } else {
                    int e = item - nrow;
                    if (e < nx) {
                        x[e] = x0[e];
                        continue;
                    }
                    e += nrow;
                    const R n = nb[e];
                    R v;
                    if (e < g.quadT()) {
                        const int c = (e - g.quad(0)) % g.S;
                        const R w = c < nx ? q[c] : r[c - nx];
                        v = (rho * n) / (w + rho);
                    } else if (e < g.box(0)) {
                        v = (rho * n) / (q[e - g.quadT()] + rho);
                    } else {
                        v = n;
                        if (v < a.lo) v = a.lo;
                        if (v > a.hi) v = a.hi;
                    }
                    x[e] = v;
                }
            }
            __syncthreads();
            // Z: rho-weighted mean over each variable's edges
            const bool chkz = rm == 0 || it == K;
            R dual_r = R(0);
            for (int b = threadIdx.x; b < g.V; b += NT) {
                int ed[3];
                const int ne = var_edges(g, b, ed);
                R S = R(0), Rs = R(0);
                for (int j = 0; j < ne; ++j) {
                    S += rho * (x[ed[j]] + u[ed[j]]);
                    Rs += rho;
                }
                const R zold = z[b];
                const R znew = S / Rs;
                z[b] = znew;
                if (chkz) {
                    const R dz = znew - zold;
                    dual_r += (R)ne * rho * rho * dz * dz;
                }
            }
            dual = (double)dual_r;
            pend = true;
            rm_prev = rm;
            rm = rm + 1 == ce ? 0 : rm + 1;
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
    if (fixed)
        return threads == 64    ? (const void *)k_mpc_batch<R, 64, 12, 4>
               : threads == 128 ? (const void *)k_mpc_batch<R, 128, 12, 4>
                                : (const void *)k_mpc_batch<R, 256, 12, 4>;
    return threads == 64    ? (const void *)k_mpc_batch<R, 64, 0, 0>
           : threads == 128 ? (const void *)k_mpc_batch<R, 128, 0, 0>
                            : (const void *)k_mpc_batch<R, 256, 0, 0>;
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
