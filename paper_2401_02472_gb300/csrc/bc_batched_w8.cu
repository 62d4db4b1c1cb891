// Batched-form kernels for 256 sources per batch.
#include "bc_batched_launch.cuh"

namespace sp {
template sp_status launch_batched_w<8>(const BatchedLaunch& L, LaunchResult* result);
}  // namespace sp
