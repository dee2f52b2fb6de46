// FP64 mode instantiation of the hot-path kernels.  Built with -fmad=false: every product
// and sum is rounded on its own, as in the plain restatement the results are checked
// against, so the two differ only through the math library's transcendental functions.
#include "mcv_kernels.cuh"

namespace mcv {
MCV_DEFINE_ENTRY_POINTS(double, f64)
}  // namespace mcv
