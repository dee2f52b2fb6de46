// FP64 mode instantiation of the fused trace kernels.  Compiled with -fmad=false: every
// product and sum is rounded on its own, as in the plain restatement of the method.
#include "mcv_kernels.cuh"

namespace mcv {
MCV_DEFINE_TRACE_ENTRY_POINTS(double, f64)
}  // namespace mcv
