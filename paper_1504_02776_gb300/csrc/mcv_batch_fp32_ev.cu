// FP32 fast mode instantiation of the batched kernels that append to event lists.
#include "mcv_kernels.cuh"

namespace mcv {
MCV_DEFINE_BATCH_ENTRY_POINTS(float, f32_ev, true)
}  // namespace mcv
