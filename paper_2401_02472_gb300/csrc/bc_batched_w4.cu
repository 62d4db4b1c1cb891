// Batched-form kernels for 128 sources per batch.
#include "bc_batched_launch.cuh"

namespace sp {
template sp_status launch_batched_w<4>(const BatchedLaunch& L, LaunchResult* result);
}  // namespace sp
