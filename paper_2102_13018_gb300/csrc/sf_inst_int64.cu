// Kernel instantiations for int64 units (one translation unit per element type).
#include "sf_launch_impl.cuh"

namespace sfgb {
SFGB_INSTANTIATE(int64_t)
}  // namespace sfgb
