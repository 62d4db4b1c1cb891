// Batched-form kernels for 32 sources per batch.
#include "bc_batched_launch.cuh"

namespace sp {
template sp_status launch_batched_w<1>(const BatchedLaunch& L, LaunchResult* result);
}  // namespace sp
