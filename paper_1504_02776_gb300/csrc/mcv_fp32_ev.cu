// FP32 fast mode instantiation of the fused waves that append to an event list.
#include "mcv_kernels.cuh"

namespace mcv {
MCV_DEFINE_EVENT_ENTRY_POINTS(float, f32)
}  // namespace mcv
