// FP32 fast mode instantiation of the fused trace kernels (FMA contraction on).
#include "mcv_kernels.cuh"

namespace mcv {
MCV_DEFINE_TRACE_ENTRY_POINTS(float, f32)
}  // namespace mcv
