// FP32 instantiation of the sweep (FMA contraction allowed).
#include "sweep_launch.cuh"

namespace fga {
template cudaError_t sweep_persistent<float>(const SweepArgs<float> &, int, int, int, int, cudaStream_t);
template cudaError_t sweep_phase_f<float>(const SweepArgs<float> &, int, int, int, int, int, int, int,
                                          cudaStream_t);
template cudaError_t sweep_phase_z<float>(const SweepArgs<float> &, int, long long, int, int, int, cudaStream_t);
template cudaError_t sweep_check<float>(const SweepArgs<float> &, long long, int, int, int, int, cudaStream_t);
template int sweep_max_blocks_per_sm<float>(int, int, int);
template cudaError_t shard_sums<float>(const SweepArgs<float> &, const float *, float *, int, int, cudaStream_t);
template cudaError_t shard_add_parts<float>(const float *, int, long long, float *, int, cudaStream_t);
template cudaError_t shard_z<float>(const SweepArgs<float> &, const float *, int, int, int, int, cudaStream_t);
template cudaError_t shard_total<float>(const double *, int, double *, cudaStream_t);
}  // namespace fga
