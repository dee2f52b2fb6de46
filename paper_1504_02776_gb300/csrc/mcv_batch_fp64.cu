// FP64 mode instantiation of the batched kernels, built without FMA contraction like the
// other FP64 kernels (mcv_fp64.cu).
#include "mcv_kernels.cuh"

namespace mcv {
MCV_DEFINE_BATCH_ENTRY_POINTS(double, f64, false)
}  // namespace mcv
