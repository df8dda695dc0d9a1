// fx_plan_compact.cu -- the batched path's streaming kernels on the compact strips,
// compiled apart from the other classes.
#include "fx_plan_kernels.cuh"

namespace fx {

const void *plan_fast_kernel_compact(const KParams &kp, int g) { return fast_kernel_of<kCompactRm>(kp, g); }
const void *plan_redo_kernel_compact(const KParams &kp) { return redo_kernel_of<kCompactRm>(kp); }

}  // namespace fx

namespace fx {
FX_CHECK_COUNTER(checked_count_plan_compact)
}  // namespace fx
