// FP32 instantiation of every kernel launcher (mixed-precision path: fields
// in FP32, reductions and scalars in FP64).
#include "rd_launch_impl.cuh"

namespace rd {
template struct Launch<float>;
}  // namespace rd
