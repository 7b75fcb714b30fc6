// FP64 instantiation of the inner-CG kernels (cg_impl.cuh).
#include "cg_impl.cuh"

namespace mrcg {

MRCG_CG_PRECISION_ENTRY_POINTS(double, f64)

}  // namespace mrcg
