// Fused-step instantiations for float32 b and w storage.
#define SPG_BF16_FLAG false
#include "spg_step_kernel.cuh"

namespace spg {
SPG_DEFINE_DISPATCH(false, f32)
}  // namespace spg
