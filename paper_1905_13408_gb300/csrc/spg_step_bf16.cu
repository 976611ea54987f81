// Fused-step instantiations for bfloat16 b and w storage.
#define SPG_BF16_FLAG true
#include "spg_step_kernel.cuh"

namespace spg {
SPG_DEFINE_DISPATCH(true, bf16)
}  // namespace spg
