// FP64 instantiation of every kernel launcher (plain FP64 path).
#include "rd_launch_impl.cuh"

namespace rd {
template struct Launch<double>;
}  // namespace rd
