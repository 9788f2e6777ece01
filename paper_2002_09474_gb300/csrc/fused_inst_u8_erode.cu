// Instantiations of the fused kernel for u8 pixels, erode (op 0).
#include "fused_kernel.cuh"

namespace morph {
FusedKernelFn fused_kernel_u8_erode(int cfg) { return pick_fused_kernel<uint8_t, 0>(cfg); }
FusedPipeKernelFn fused_pipe_kernel_u8_erode(int cfg) { return pick_fused_pipe_kernel<uint8_t, 0>(cfg); }
}  // namespace morph
