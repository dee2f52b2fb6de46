// FP32 fast mode instantiation of the source, detector and adjoint kernels.
#include "mcv_kernels.cuh"

namespace mcv {
MCV_DEFINE_AUX_ENTRY_POINTS(float, f32)
}  // namespace mcv
