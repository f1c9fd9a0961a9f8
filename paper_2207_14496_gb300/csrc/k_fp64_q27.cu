// Step kernels instantiated for storage fp64, D3Q27.
// Built with -fmad=false: no multiply-add contraction, so the FP64 results follow
// the source's operation order exactly (bit-reproducible against a plain FP64
// evaluation).
#include "fsl_kernels.cuh"

namespace fsl {
const Launch* launch_fp64_q27() { return Kernels<27, SF64>::table(); }
}  // namespace fsl
