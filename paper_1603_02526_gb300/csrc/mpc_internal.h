// mpc_internal.h -- descriptors of the batched MPC solver (not public).
#pragma once

#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

namespace fga {

// One MPC instance is the factor graph of Sec. V-B / Appendix B with
// horizon T: variables x_0, u_0, x_1, ..., u_{T-1}, x_T (z index of x_t is
// t*S, of u_t is t*S + nx, S = nx + nu) and factors, in creation order,
//   FIX(x_0) | DYN(x_t, u_t, x_{t+1}) t < T | QUAD(x_t, u_t) t < T |
//   QUAD(x_T) | BOX(u_t) t < T
// i.e. E = 2 nx + 3 (nx + nu) T scalar edges, V = S T + nx scalar variables.
template <typename R>
struct MpcArgs {
    int n_inst, nx, nu;
    const int *T;             // horizon per instance
    const long long *zoff;    // first scalar variable of every instance
    const long long *eoff;    // first scalar edge of every instance
    const int *sys;           // system index of every instance
    const int *order;         // instances in the order they are handed out
    const R *P;               // per system: (2nx+nu) x (2nx+nu) projector onto the dynamics
    const R *q;               // per system: nx state weights
    const R *r;               // per system: nu input weights
    const R *x0;              // per instance: nx
    R lo, hi, rho, alpha;
    R *z, *u, *x;             // state in global memory (loaded / stored per solve)
    long long *iters;         // per instance: iterations done
    int *status;              // per instance: 0, FGA_EBUDGET or FGA_ENONFINITE
    double *rpri, *rdual;     // per instance: RMS residuals of the last check
    unsigned *queue;          // work counter (zeroed before every launch)
    long long max_iters;
    double tol_pri, tol_dual;
    int check_every;
    int first_pending;        // 1: the stored x/u carry a pending u-update (resume)
};

struct MpcConfig {
    int threads;              // CTA size (64, 128 or 256)
    int check_every;          // residual check interval
};

// dynamic shared memory for instances up to horizon tmax
int mpc_smem_bytes(int rsize, int nx, int nu, int tmax, int threads);

template <typename R>
cudaError_t mpc_launch(const MpcArgs<R> &a, int threads, int grid, int smem, cudaStream_t s);
template <typename R>
int mpc_max_blocks_per_sm(int threads, int smem);
// One lane per time step (mpc_warp.cu; FP32, 12 states, 4 inputs, horizons
// up to 64): work items (two instances of at most 32 steps, or one of
// 33..64 steps, inst[1] = -2), the launch, and its resident CTAs per SM.
bool mpc_warp_items(const int *T, int n, std::vector<int2> &items);
cudaError_t mpc_warp_launch(const MpcArgs<float> &a, const int2 *items, int n_items, int grid, cudaStream_t s);
int mpc_warp_max_blocks_per_sm();
constexpr int kMpcWarpThreads = 64;   // CTA size of the per-step kernel

template <typename R>
cudaError_t mpc_warm_start_impl(const MpcArgs<R> &a, const R *Am, const R *Bm, const float *pred, long long ld,
                                cudaStream_t s);
template <typename R>
cudaError_t mpc_targets_impl(const MpcArgs<R> &a, const R *K, float *out, long long ld, cudaStream_t s);

}  // namespace fga
