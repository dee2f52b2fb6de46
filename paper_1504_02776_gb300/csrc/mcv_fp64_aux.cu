// FP64 mode instantiation of the source, detector and adjoint kernels (-fmad=false).
#include "mcv_kernels.cuh"

namespace mcv {
MCV_DEFINE_AUX_ENTRY_POINTS(double, f64)
}  // namespace mcv
