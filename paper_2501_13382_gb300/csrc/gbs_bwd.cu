// gbs_bwd.cu -- adjoint of the Gaussian beam sum (placeholder until implemented).
#include "gbt_internal.h"

namespace gbt {

size_t bwd_workspace_bytes(const TraceDev &, const gbt_sum_args &) { return 256; }

void bwd_launch(const TraceDev &, const SceneDev &, const gbt_sum_args &, const float *, float *,
                float *, double *, void *, cudaStream_t)
{
    fail(GBT_ERR_UNSUPPORTED, "gbt_sum_backward is not built yet");
}

}  // namespace gbt
