// Step kernels instantiated for storage fp16, D3Q27.
// FP32 arithmetic on offsets f_i - w_i; cell mass, excess mass and reductions
// stay FP64.
#include "fsl_kernels.cuh"

namespace fsl {
const Launch* launch_fp16_q27() { return Kernels<27, SF16>::table(); }
}  // namespace fsl
