// fx_plan_wide.cu -- the batched path's streaming kernels on the wide strips,
// compiled apart from the other classes.
#include "fx_plan_kernels.cuh"

namespace fx {

const void *plan_fast_kernel_wide(const KParams &kp, int g) { return fast_kernel_of<kWideRm>(kp, g); }
const void *plan_redo_kernel_wide(const KParams &kp) { return redo_kernel_of<kWideRm>(kp); }

}  // namespace fx

namespace fx {
FX_CHECK_COUNTER(checked_count_plan_wide)
}  // namespace fx
