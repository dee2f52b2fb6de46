// FP64 mode instantiation of the batched kernels that append to event lists (-fmad=false).
#include "mcv_kernels.cuh"

namespace mcv {
MCV_DEFINE_BATCH_ENTRY_POINTS(double, f64_ev, true)
}  // namespace mcv
