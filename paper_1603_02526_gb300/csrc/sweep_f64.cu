// FP64 instantiation of the sweep.  Built with -fmad=false: no product is
// fused into an add, so each operation is rounded exactly as in a plain
// serial FP64 loop over the same expression.
#include "sweep_launch.cuh"

namespace fga {
template cudaError_t sweep_persistent<double>(const SweepArgs<double> &, int, int, int, int, cudaStream_t);
template cudaError_t sweep_phase_f<double>(const SweepArgs<double> &, int, int, int, int, int, int, int,
                                          cudaStream_t);
template cudaError_t sweep_phase_z<double>(const SweepArgs<double> &, int, long long, int, int, int, cudaStream_t);
template cudaError_t sweep_check<double>(const SweepArgs<double> &, long long, int, int, int, int, cudaStream_t);
template int sweep_max_blocks_per_sm<double>(int, int, int);
template cudaError_t shard_sums<double>(const SweepArgs<double> &, const double *, double *, int, int, cudaStream_t);
template cudaError_t shard_add_parts<double>(const double *, int, long long, double *, int, cudaStream_t);
template cudaError_t shard_z<double>(const SweepArgs<double> &, const double *, int, int, int, int, cudaStream_t);
template cudaError_t shard_total<double>(const double *, int, double *, cudaStream_t);
}  // namespace fga
