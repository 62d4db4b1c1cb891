// Width dispatch of the batched form.
#include "internal.h"

namespace sp {

sp_status run_batched(const BatchedLaunch& L, LaunchResult* result) {
    switch (L.width) {
        case 32: return launch_batched_w<1>(L, result);
        case 64: return launch_batched_w<2>(L, result);
        case 128: return launch_batched_w<4>(L, result);
        case 256: return launch_batched_w<8>(L, result);
        default: return fail(SP_ERR_INVALID_ARG, "batch width must be 32, 64, 128 or 256");
    }
}

}  // namespace sp
