// FP32 fast mode instantiation of the batched kernels (FMA contraction on).
#include "mcv_kernels.cuh"

namespace mcv {
MCV_DEFINE_BATCH_ENTRY_POINTS(float, f32, false)
}  // namespace mcv
