// Per-iteration pass kernels, FP32 vectors.
#include "engine_iter.cuh"

namespace ld {
template int iteration_launch<float>(const Solve &, int, cudaStream_t);
template int iteration_occupancy<float>(int, int, bool, int, bool, int *);
}  // namespace ld
