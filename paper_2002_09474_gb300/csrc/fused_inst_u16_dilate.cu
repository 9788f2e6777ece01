// Instantiations of the fused kernel for u16 pixels, dilate (op 1).
#include "fused_kernel.cuh"

namespace morph {
FusedKernelFn fused_kernel_u16_dilate(int cfg) { return pick_fused_kernel<uint16_t, 1>(cfg); }
FusedPipeKernelFn fused_pipe_kernel_u16_dilate(int cfg) { return pick_fused_pipe_kernel<uint16_t, 1>(cfg); }
}  // namespace morph
