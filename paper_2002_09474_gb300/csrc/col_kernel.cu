// The column-pass kernel (1 x w windows): instantiations, tile-height choice
// and launch.  Device code in morph_col.cuh.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include "morph_col.cuh"
#include "morph_geom.h"
#include "morph_internal.h"

namespace morph {

template <typename T, int OP, bool BLK>
__global__ void __launch_bounds__(kColThreads, 4) col_kernel(const __grid_constant__ CUtensorMap tin,
                                                             const ColArgs a) {
  __shared__ __align__(8) uint64_t bars[kColMaxBoxes];
  extern __shared__ __align__(128) uint8_t csmem[];
  if (a.tma_ld && threadIdx.x == 0) {
    for (int b = 0; b < kColMaxBoxes; ++b) mbar_init(&bars[b], 1);
    fence_barrier_init();
  }
  __syncthreads();
  pdl_wait();
  col_tile<T, OP, BLK>(a, &tin, blockIdx.x, csmem, reinterpret_cast<uint32_t*>(csmem + kColBytes * a.ihp), bars);
  pdl_launch_dependents();
}

namespace {

using ColFn = void (*)(const CUtensorMap, const ColArgs);

ColFn col_kernel_for(int esz, int op, bool blk) {
  if (esz == 1) {
    if (op == 0) return blk ? col_kernel<uint8_t, 0, true> : col_kernel<uint8_t, 0, false>;
    return blk ? col_kernel<uint8_t, 1, true> : col_kernel<uint8_t, 1, false>;
  }
  if (op == 0) return blk ? col_kernel<uint16_t, 0, true> : col_kernel<uint16_t, 0, false>;
  return blk ? col_kernel<uint16_t, 1, true> : col_kernel<uint16_t, 1, false>;
}

int sm_count() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  return n;
}

}  // namespace

cudaError_t col_launch(const FusedLaunch& L, bool blocked, cudaStream_t stream) {
  const int E = L.esz;
  const int sms = sm_count();
  if (sms <= 0) return cudaErrorInvalidDevice;
  const int ty = col_pick_ty(E, L.W, L.H, L.wy, sms, kMaxSmemBytes);
  const ColGeom g = col_geom(E, ty, L.wy);
  if (g.smem > kMaxSmemBytes || !g.ok) return cudaErrorInvalidConfiguration;
  ColArgs a;
  a.src = static_cast<const uint8_t*>(L.src);
  a.dst = static_cast<uint8_t*>(L.dst);
  a.sp = L.sp;
  a.dp = L.dp;
  a.W = L.W;
  a.H = L.H;
  a.w = L.wy;
  a.a = L.ay;
  a.ty = g.ty;
  a.ih = g.ih;
  a.ihp = g.ihp;
  a.ntx = cdiv(L.W * E, kColBytes);
  a.ntiles = a.ntx * cdiv(L.H, g.ty);
  a.blocked = blocked ? 1 : 0;
  a.ld_vec = (reinterpret_cast<uintptr_t>(L.src) % 4 == 0) && (L.sp % 4 == 0);
  a.st_vec = (reinterpret_cast<uintptr_t>(L.dst) % 4 == 0) && (L.dp % 4 == 0);
  a.err = device_error_word();
  if (!a.err) return cudaErrorInvalidDevice;
  CUtensorMap tin;
  memset(&tin, 0, sizeof(tin));
  a.tma_ld = encode_tensor_map_2d(&tin, L.src, E, L.W, L.H, L.sp, kColBytes / E, kColBox) ? 1 : 0;
  ColFn k = col_kernel_for(E, L.op, blocked);
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
  return launch_pdl(L.pdl, k, dim3(a.ntiles), dim3(kColThreads), g.smem, stream, tin, a);
}

}  // namespace morph
