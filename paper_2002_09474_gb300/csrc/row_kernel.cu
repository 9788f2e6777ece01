// The row-pass kernel (w x 1 windows): instantiations and launch.  Device
// code in morph_row.cuh.
#include <cstring>
#include <mutex>

#include "morph_internal.h"
#include "morph_row.cuh"

namespace morph {

template <typename T, int OP, bool BLK>
__global__ void __launch_bounds__(kRowThreads, 2) row_kernel(const __grid_constant__ CUtensorMap tin,
                                                             const RowArgs a, const RowGeom g) {
  __shared__ __align__(8) uint64_t bar;
  extern __shared__ __align__(128) uint8_t rsmem[];
  if (a.tma_ld && threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_barrier_init();
  }
  __syncthreads();
  pdl_wait();
  uint32_t phase = 0;
  row_tile<T, OP, BLK>(a, &tin, blockIdx.x, g, rsmem, &bar, phase);
  pdl_launch_dependents();
}

namespace {

using RowFn = void (*)(const CUtensorMap, const RowArgs, const RowGeom);

RowFn row_kernel_for(int esz, int op, bool blk) {
  if (esz == 1) {
    if (op == 0) return blk ? row_kernel<uint8_t, 0, true> : row_kernel<uint8_t, 0, false>;
    return blk ? row_kernel<uint8_t, 1, true> : row_kernel<uint8_t, 1, false>;
  }
  if (op == 0) return blk ? row_kernel<uint16_t, 0, true> : row_kernel<uint16_t, 0, false>;
  return blk ? row_kernel<uint16_t, 1, true> : row_kernel<uint16_t, 1, false>;
}

}  // namespace

bool row_fits(const FusedLaunch& L) { return row_geom(L.esz, L.wx, L.ax).smem <= kMaxSmemBytes; }

cudaError_t row_launch(const FusedLaunch& L, bool blocked, cudaStream_t stream) {
  const int E = L.esz;
  const RowGeom g = row_geom(E, L.wx, L.ax);
  if (g.smem > kMaxSmemBytes) return cudaErrorInvalidConfiguration;
  RowArgs a;
  a.src = static_cast<const uint8_t*>(L.src);
  a.dst = static_cast<uint8_t*>(L.dst);
  a.sp = L.sp;
  a.dp = L.dp;
  a.W = L.W;
  a.H = L.H;
  a.w = L.wx;
  a.a = L.ax;
  a.ntx = cdiv(L.W, g.txp);
  a.nty = cdiv(L.H, g.ty);
  a.blocked = blocked ? 1 : 0;
  a.ld_vec = (reinterpret_cast<uintptr_t>(L.src) % 4 == 0) && (L.sp % 4 == 0);
  const int sv = 8 * E;  // bytes of one 8-pixel row segment
  a.st_vec = (reinterpret_cast<uintptr_t>(L.dst) % sv == 0) && (L.dp % sv == 0);
  a.err = device_error_word();
  if (!a.err) return cudaErrorInvalidDevice;
  CUtensorMap tin;
  memset(&tin, 0, sizeof(tin));
  a.tma_ld = encode_tensor_map_2d(&tin, L.src, E, L.W, L.H, L.sp, 128 / E, g.ty) ? 1 : 0;
  RowFn k = row_kernel_for(E, L.op, blocked);
  static std::mutex mu;
  static const void* opted[64][8] = {};
  {
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lock(mu);
    const int slot = (E - 1) * 4 + L.op * 2 + (blocked ? 1 : 0);
    if (opted[dev & 63][slot] != reinterpret_cast<const void*>(k)) {
      cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmemBytes);
      if (e != cudaSuccess) return e;
      opted[dev & 63][slot] = reinterpret_cast<const void*>(k);
    }
  }
  return launch_pdl(L.pdl, k, dim3(a.ntx * a.nty), dim3(kRowThreads), g.smem, stream, tin, a, g);
}

}  // namespace morph
