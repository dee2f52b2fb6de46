// FP64 mode instantiation of the fused waves that append to an event list (-fmad=false).
#include "mcv_kernels.cuh"

namespace mcv {
MCV_DEFINE_EVENT_ENTRY_POINTS(double, f64)
}  // namespace mcv
