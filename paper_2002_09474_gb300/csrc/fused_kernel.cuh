// The single-image fused kernel template (one CTA per output tile) and the
// table of its tile-shape instantiations.
#pragma once

#include "morph_internal.h"
#include "morph_tile.cuh"

namespace morph {

// At least 5 resident CTAs per SM for 8-bit pixels (registers capped at 96,
// a few bytes spilled: measured 5-8% faster at 3 x 3 to 7 x 7 on 4096^2
// than 4 CTAs at 120 registers), 4 for 16-bit pixels (5 measured 2-4%
// slower there).
template <typename T, int OP, int TX, int TY>
__global__ void __launch_bounds__(kThreads, sizeof(T) == 1 ? 5 : 4) fused_kernel(const __grid_constant__ CUtensorMap tin,
                                                            const __grid_constant__ CUtensorMap tout,
                                                            const ImgArgs a, const Geom g) {
  __shared__ __align__(8) uint64_t bar;
  extern __shared__ __align__(128) uint4 smem[];
  if (a.tma_ld && threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_barrier_init();
  }
  __syncthreads();
  pdl_wait();
  uint32_t phase = 0;
  run_tile<T, OP, TX, TY>(a, &tin, &tout, blockIdx.x * TX, blockIdx.y * TY, g, smem, &bar, phase, a.err);
  pdl_launch_dependents();
}

// Persistent form: a grid of (SMs x resident CTAs) CTAs walks the tiles in
// row-major order, tile blockIdx.x + i * gridDim.x on iteration i.  Two
// copies of region A (see make_geom's `pipe` layout) let the TMA load of the
// next tile run while the current one is computed, and the TMA store of a
// tile stays in flight until the next tile begins.  Needs a.tma_ld.
template <typename T, int OP, int TX, int TY>
__global__ void __launch_bounds__(kThreads, 3) fused_pipe_kernel(const __grid_constant__ CUtensorMap tin,
                                                                 const __grid_constant__ CUtensorMap tout,
                                                                 const ImgArgs a, const Geom g, int ntx,
                                                                 int ntiles) {
  __shared__ __align__(8) uint64_t bar[2];
  extern __shared__ __align__(128) uint4 smem[];
  if (static_cast<int>(blockIdx.x) >= ntiles) return;  // whole CTA
  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_barrier_init();
  }
  __syncthreads();
  pdl_wait();
  run_tiles_pipelined<T, OP, TX, TY>(a, &tin, &tout, g, smem, bar, ntx, ntiles, blockIdx.x, gridDim.x);
  pdl_launch_dependents();
}

template <typename T, int OP>
FusedKernelFn pick_fused_kernel(int cfg) {
  switch (cfg) {
    case kTile128x64: return fused_kernel<T, OP, 128, 64>;
    case kTile64x64: return fused_kernel<T, OP, 64, 64>;
    case kTile64x128: return fused_kernel<T, OP, 64, 128>;
    case kTile256x32: return fused_kernel<T, OP, 256, 32>;
    case kTile32x32: return fused_kernel<T, OP, 32, 32>;
    case kTile128x128: return fused_kernel<T, OP, 128, 128>;
    case kTile256x64: return fused_kernel<T, OP, 256, 64>;
    case kTile32x128: return fused_kernel<T, OP, 32, 128>;
  }
  return nullptr;
}

template <typename T, int OP>
FusedPipeKernelFn pick_fused_pipe_kernel(int cfg) {
  switch (cfg) {
    case kTile128x64: return fused_pipe_kernel<T, OP, 128, 64>;
    case kTile64x64: return fused_pipe_kernel<T, OP, 64, 64>;
    case kTile64x128: return fused_pipe_kernel<T, OP, 64, 128>;
    case kTile256x32: return fused_pipe_kernel<T, OP, 256, 32>;
    case kTile32x32: return fused_pipe_kernel<T, OP, 32, 32>;
    case kTile128x128: return fused_pipe_kernel<T, OP, 128, 128>;
    case kTile256x64: return fused_pipe_kernel<T, OP, 256, 64>;
    case kTile32x128: return fused_pipe_kernel<T, OP, 32, 128>;
  }
  return nullptr;
}

}  // namespace morph
