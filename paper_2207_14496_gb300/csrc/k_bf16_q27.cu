// Step kernels instantiated for storage bf16, D3Q27.
// FP32 arithmetic on offsets f_i - w_i; cell mass, excess mass and reductions
// stay FP64.
#include "fsl_kernels.cuh"

namespace fsl {
const Launch* launch_bf16_q27() { return Kernels<27, SBF16>::table(); }
}  // namespace fsl
