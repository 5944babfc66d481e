// Kernel instantiations for fp64 units (one translation unit per element type).
#include "sf_launch_impl.cuh"

namespace sfgb {
SFGB_INSTANTIATE(double)
}  // namespace sfgb
