// Kernel instantiations for int32 units (one translation unit per element type).
#include "sf_launch_impl.cuh"

namespace sfgb {
SFGB_INSTANTIATE(int32_t)
}  // namespace sfgb
