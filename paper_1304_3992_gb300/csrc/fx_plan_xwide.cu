// fx_plan_xwide.cu -- the batched path's streaming kernels on the extra-wide strips,
// compiled apart from the other classes.
#include "fx_plan_kernels.cuh"

namespace fx {

const void *plan_fast_kernel_xwide(const KParams &kp, int g) { return fast_kernel_of<kXWideRm>(kp, g); }
const void *plan_redo_kernel_xwide(const KParams &kp) { return redo_kernel_of<kXWideRm>(kp); }

}  // namespace fx

namespace fx {
FX_CHECK_COUNTER(checked_count_plan_xwide)
}  // namespace fx
