// FP32 instantiation of the sweep (FMA contraction allowed).
#include "sweep_launch.cuh"

namespace fga {
template cudaError_t sweep_persistent<float>(const SweepArgs<float> &, int, int, int, int, cudaStream_t);
template cudaError_t sweep_phase_f<float>(const SweepArgs<float> &, int, int, int, int, int, int, int,
                                          cudaStream_t);
template cudaError_t sweep_phase_z<float>(const SweepArgs<float> &, int, long long, int, int, int, cudaStream_t);
template cudaError_t sweep_check<float>(const SweepArgs<float> &, long long, int, int, int, int, cudaStream_t);
template int sweep_max_blocks_per_sm<float>(int, int, int);
}  // namespace fga
