// The warp-tiled van Herk/Gil-Werman kernel of the pass along y (1 x w
// windows): instantiations, launch shape and launch.  Device code in
// morph_colv.cuh.
#include <cstring>
#include <mutex>

#include "morph_colv.cuh"
#include "morph_geom.h"
#include "morph_internal.h"
#include "plan.h"

namespace morph {

template <typename T, int OP>
__global__ void __launch_bounds__(128) colv_kernel(const __grid_constant__ CUtensorMap tin, const ColvArgs a) {
  extern __shared__ __align__(128) uint8_t vsmem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int task = blockIdx.x * a.wpc + warp;
  if (task >= a.ntask) return;
  uint8_t* tile = vsmem + warp * colv_tile_bytes(a.nbox);
  uint64_t* bars = reinterpret_cast<uint64_t*>(vsmem + a.wpc * colv_tile_bytes(a.nbox)) + warp * kCvMaxBox;
  if (a.tma_ld) {
    if (lane == 0) {
      for (int b = 0; b < a.nbox; ++b) mbar_init(&bars[b], 1);
      fence_barrier_init();
    }
    __syncwarp();
  }
  colv_tile<T, OP>(a, &tin, task, lane, tile, bars);
}

namespace {

using ColvFn = void (*)(const CUtensorMap, const ColvArgs);

ColvFn colv_kernel_for(int esz, int op) {
  if (esz == 1) return op == 0 ? colv_kernel<uint8_t, 0> : colv_kernel<uint8_t, 1>;
  return op == 0 ? colv_kernel<uint16_t, 0> : colv_kernel<uint16_t, 1>;
}

int sm_count_v() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  return n;
}

}  // namespace

bool colv_fits(const FusedLaunch& L) {
  return L.wy >= 2 && colv_plan(L.esz, L.W, L.H, L.wy, 152, kMaxSmemBytes, tuning().colv_rows).ok;
}

cudaError_t colv_launch(const FusedLaunch& L, cudaStream_t stream) {
  const int E = L.esz;
  const int sms = sm_count_v();
  if (sms <= 0) return cudaErrorInvalidDevice;
  const ColvPlan p = colv_plan(E, L.W, L.H, L.wy, sms, kMaxSmemBytes, tuning().colv_rows);
  if (!p.ok) return cudaErrorInvalidConfiguration;
  ColvArgs a;
  a.src = static_cast<const uint8_t*>(L.src);
  a.dst = static_cast<uint8_t*>(L.dst);
  a.sp = L.sp;
  a.dp = L.dp;
  a.W = L.W;
  a.H = L.H;
  a.w = L.wy;
  a.a = L.ay;
  a.L = p.L;
  a.nbox = p.nbox;
  a.ns = cdiv(L.W * E, kCvBytes);
  a.ntask = p.ntask;
  a.wpc = p.wpc;
  a.ld_vec = (reinterpret_cast<uintptr_t>(L.src) % 4 == 0) && (L.sp % 4 == 0);
  a.st_vec = (reinterpret_cast<uintptr_t>(L.dst) % 4 == 0) && (L.dp % 4 == 0);
  a.err = device_error_word();
  if (!a.err) return cudaErrorInvalidDevice;
  CUtensorMap tin;
  memset(&tin, 0, sizeof(tin));
  a.tma_ld = encode_tensor_map_2d(&tin, L.src, E, L.W, L.H, L.sp, kCvBytes / E, kCvBox) ? 1 : 0;
  ColvFn k = colv_kernel_for(E, L.op);
  static std::mutex mu;
  static const void* opted[64][4] = {};
  {
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lock(mu);
    const int slot = (E - 1) * 2 + L.op;
    if (opted[dev & 63][slot] != reinterpret_cast<const void*>(k)) {
      cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmemBytes);
      if (e != cudaSuccess) return e;
      opted[dev & 63][slot] = reinterpret_cast<const void*>(k);
    }
  }
  const int grid = cdiv(p.ntask, p.wpc);
  note_launch();
  k<<<grid, 32 * p.wpc, p.smem, stream>>>(tin, a);
  return cudaGetLastError();
}

}  // namespace morph
