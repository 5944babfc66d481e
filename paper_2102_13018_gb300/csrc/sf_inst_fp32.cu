// Kernel instantiations for fp32 units (one translation unit per element type).
#include "sf_launch_impl.cuh"

namespace sfgb {
SFGB_INSTANTIATE(float)
}  // namespace sfgb
