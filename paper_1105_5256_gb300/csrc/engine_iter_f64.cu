// Per-iteration pass kernels, FP64 vectors.
#include "engine_iter.cuh"

namespace ld {
template int iteration_launch<double>(const Solve &, int, cudaStream_t);
template int iteration_occupancy<double>(int, int, bool, int, bool, int *);
}  // namespace ld
