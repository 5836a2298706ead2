// proj_tc.cu -- tensor-core a-projection (FP16 single pass, BF16 three-product split).
#include "cyc_impl.h"

namespace cyc {

bool tc_supported(int) { return false; }
ProjPlan tc_plan(int, int, int64_t, int) { return ProjPlan{1, 0}; }
size_t tc_max_partials(int, int, int) { return 1; }
cudaError_t tc_launch(const ProjArgs&, int, cudaStream_t) { return cudaErrorNotSupported; }

}  // namespace cyc
