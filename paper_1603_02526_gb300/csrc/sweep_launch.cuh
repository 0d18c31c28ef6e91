// sweep_launch.cuh -- host launchers of the sweep kernels for one real type.
// Included once per precision (sweep_f32.cu, sweep_f64.cu).
#pragma once

#include "sweep.cuh"

namespace fga {

template <typename R, int KIND>
static cudaError_t allow_smem_k(int smem) {
    // kernels that take the chunk buffers may need more than the default 48 KB;
    // ask for the largest shared-memory carveout so several CTAs fit per SM
    cudaError_t e = cudaFuncSetAttribute((const void *)k_sweep_persistent<R, KIND>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute((const void *)k_sweep_persistent<R, KIND>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute((const void *)k_phase_f<R, F_PROX, KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             smem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute((const void *)k_phase_f<R, F_U_PROX, KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             smem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute((const void *)k_phase_f<R, F_U_PROX_CHK, KIND>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute((const void *)k_phase_f<R, F_U_ONLY, KIND>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}

template <typename R>
static cudaError_t allow_smem(int smem, int kind) {
    switch (kind) {
    case 1: return allow_smem_k<R, 1>(smem);
    case 2: return allow_smem_k<R, 2>(smem);
    case 3: return allow_smem_k<R, 3>(smem);
    case kKindScatter + 0: return allow_smem_k<R, kKindScatter + 0>(smem);
    case kKindScatter + 1: return allow_smem_k<R, kKindScatter + 1>(smem);
    case kKindScatter + 2: return allow_smem_k<R, kKindScatter + 2>(smem);
    case kKindScatter + 3: return allow_smem_k<R, kKindScatter + 3>(smem);
    default: return allow_smem_k<R, 0>(smem);
    }
}

template <typename R>
static const void *persistent_fn(int kind) {
    switch (kind) {
    case 1: return (const void *)k_sweep_persistent<R, 1>;
    case 2: return (const void *)k_sweep_persistent<R, 2>;
    case 3: return (const void *)k_sweep_persistent<R, 3>;
    case kKindScatter + 0: return (const void *)k_sweep_persistent<R, kKindScatter + 0>;
    case kKindScatter + 1: return (const void *)k_sweep_persistent<R, kKindScatter + 1>;
    case kKindScatter + 2: return (const void *)k_sweep_persistent<R, kKindScatter + 2>;
    case kKindScatter + 3: return (const void *)k_sweep_persistent<R, kKindScatter + 3>;
    default: return (const void *)k_sweep_persistent<R, 0>;
    }
}

template <typename R>
cudaError_t sweep_persistent(const SweepArgs<R> &a, int grid, int block, int smem, int kind, cudaStream_t s) {
    cudaError_t e = allow_smem<R>(smem, kind);
    if (e != cudaSuccess) return e;
    void *args[] = {(void *)&a};
    // Cooperative launch: the runtime refuses a grid that cannot be
    // co-resident, so the grid-wide barrier can never wait on a CTA that
    // was not scheduled.
    return cudaLaunchCooperativeKernel(persistent_fn<R>(kind), dim3(grid), dim3(block), args, (size_t)smem, s);
}

template <typename R, int KIND>
static void phase_f_k(const SweepArgs<R> &a, int mode, int xp, int zp, int grid, int block, int smem,
                      cudaStream_t s) {
    if (mode == F_PROX) k_phase_f<R, F_PROX, KIND><<<grid, block, smem, s>>>(a, xp, zp);
    else if (mode == F_U_PROX) k_phase_f<R, F_U_PROX, KIND><<<grid, block, smem, s>>>(a, xp, zp);
    else if (mode == F_U_PROX_CHK) k_phase_f<R, F_U_PROX_CHK, KIND><<<grid, block, smem, s>>>(a, xp, zp);
    else k_phase_f<R, F_U_ONLY, KIND><<<grid, block, smem, s>>>(a, xp, zp);
}

template <typename R>
cudaError_t sweep_phase_f(const SweepArgs<R> &a, int mode, int xp, int zp, int grid, int block, int smem, int kind,
                          cudaStream_t s) {
    cudaError_t e = allow_smem<R>(smem, kind);
    if (e != cudaSuccess) return e;
    switch (kind) {
    case 1: phase_f_k<R, 1>(a, mode, xp, zp, grid, block, smem, s); break;
    case 2: phase_f_k<R, 2>(a, mode, xp, zp, grid, block, smem, s); break;
    case 3: phase_f_k<R, 3>(a, mode, xp, zp, grid, block, smem, s); break;
    case kKindScatter + 0: phase_f_k<R, kKindScatter + 0>(a, mode, xp, zp, grid, block, smem, s); break;
    case kKindScatter + 1: phase_f_k<R, kKindScatter + 1>(a, mode, xp, zp, grid, block, smem, s); break;
    case kKindScatter + 2: phase_f_k<R, kKindScatter + 2>(a, mode, xp, zp, grid, block, smem, s); break;
    case kKindScatter + 3: phase_f_k<R, kKindScatter + 3>(a, mode, xp, zp, grid, block, smem, s); break;
    default: phase_f_k<R, 0>(a, mode, xp, zp, grid, block, smem, s); break;
    }
    return cudaGetLastError();
}

template <typename R>
cudaError_t sweep_phase_z(const SweepArgs<R> &a, int zp, long long it, int chk, int grid, int block,
                          cudaStream_t s) {
    if (a.zorder == 4) k_phase_z<R, true><<<grid, block, 0, s>>>(a, zp, it, chk);
    else k_phase_z<R, false><<<grid, block, a.zorder == 0 ? canonical_z_smem((int)sizeof(R)) : 0, s>>>(a, zp, it, chk);
    return cudaGetLastError();
}

template <typename R>
cudaError_t sweep_check(const SweepArgs<R> &a, long long it_checked, int xp, int zp, int final_check,
                        int grid_partials, cudaStream_t s) {
    k_check<R><<<1, 32, 0, s>>>(a, it_checked, xp, zp, final_check, grid_partials);
    return cudaGetLastError();
}

template <typename R>
cudaError_t shard_sums(const SweepArgs<R> &a, const R *s_in, R *s_out, int grid, int block, cudaStream_t s) {
    k_shard_sums<R><<<grid, block, a.zorder == 0 ? canonical_z_smem((int)sizeof(R)) : 0, s>>>(a, s_in, s_out);
    return cudaGetLastError();
}

template <typename R>
cudaError_t shard_add_parts(const R *parts, int G, long long nz, R *total, int grid, cudaStream_t s) {
    k_shard_add_parts<R><<<grid, 256, 0, s>>>(parts, G, nz, total);
    return cudaGetLastError();
}

template <typename R>
cudaError_t shard_z(const SweepArgs<R> &a, const R *total, int zp, int chk, int grid, int block, cudaStream_t s) {
    if (chk) k_shard_z<R, true><<<grid, block, 0, s>>>(a, total, zp);
    else k_shard_z<R, false><<<grid, block, 0, s>>>(a, total, zp);
    return cudaGetLastError();
}

template <typename R>
cudaError_t shard_total(const double *part, int n, double *out, cudaStream_t s) {
    k_shard_total<R><<<1, 32, 0, s>>>(part, n, out);
    return cudaGetLastError();
}

template <typename R>
int sweep_max_blocks_per_sm(int block, int smem, int kind) {
    if (allow_smem<R>(smem, kind) != cudaSuccess) return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, persistent_fn<R>(kind), block, (size_t)smem) != cudaSuccess)
        return 0;
    return n;
}

}  // namespace fga
