// Kernel instantiations for bf16 units (one translation unit per element type).
#include "sf_launch_impl.cuh"

namespace sfgb {
SFGB_INSTANTIATE(bf16)
}  // namespace sfgb
