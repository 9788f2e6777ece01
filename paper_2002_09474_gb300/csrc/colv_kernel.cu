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

template <typename T, int OP, int LB>
__global__ void __launch_bounds__(128) colv_kernel(const __grid_constant__ CUtensorMap tin, const ColvArgs a) {
  extern __shared__ __align__(128) uint8_t vsmem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int task = blockIdx.x * a.wpc + warp;
  if (task >= a.ntask) return;
  uint8_t* tile = vsmem + warp * colv_tile_bytes(a.nbox, LB);
  uint64_t* bars = reinterpret_cast<uint64_t*>(vsmem + a.wpc * colv_tile_bytes(a.nbox, LB)) + warp * a.nbox;
  if (a.tma_ld) {
    if (lane == 0) {
      for (int b = 0; b < a.nbox; ++b) mbar_init(&bars[b], 1);
      fence_barrier_init();
    }
    __syncwarp();
  }
  pdl_wait();
  colv_tile<T, OP, LB>(a, &tin, task, lane, tile, bars);
  pdl_launch_dependents();
}

namespace {

using ColvFn = void (*)(const CUtensorMap, const ColvArgs);

int sm_count_v() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  return n;
}

ColvFn colv_kernel_for(int esz, int op, int lb) {
  if (lb == 8) {
    if (esz == 1) return op == 0 ? colv_kernel<uint8_t, 0, 8> : colv_kernel<uint8_t, 1, 8>;
    return op == 0 ? colv_kernel<uint16_t, 0, 8> : colv_kernel<uint16_t, 1, 8>;
  }
  if (esz == 1) return op == 0 ? colv_kernel<uint8_t, 0, 4> : colv_kernel<uint8_t, 1, 4>;
  return op == 0 ? colv_kernel<uint16_t, 0, 4> : colv_kernel<uint16_t, 1, 4>;
}

}  // namespace

// Bytes per lane: forced by the tuning, else 8
// (two independent scan chains per lane) for windows of at most 16 rows on
// images at least 512 bytes wide (measured on the GB300 at 4096^2, 1 x 9 to
// 1 x 21: 3-10% faster up to 16 rows, slower from 17), else 4.
int colv_lane_bytes(const FusedLaunch& L) {
  const int f = tuning().colv_lb;
  if (f == 4 || f == 8) return f;
  if (L.wy <= 16 && static_cast<long long>(L.W) * L.esz >= 512) return 8;
  return 4;
}

// Tile height: forced by the tuning, else the one the autotuner measured
// for this pixel type and window class (on images of at least 12 Mpixels:
// it measures at 16 Mpixels), else the built-in rule.
ColvPlan colv_plan_for(const FusedLaunch& L) {
  const Tuning& t = tuning();
  int rows = t.colv_rows;
  if (rows == 0 && static_cast<long long>(L.W) * L.H >= (12ll << 20)) {
    const int fam = t.colv_fam_tuned[L.esz - 1][colv_tune_class(L.wy)];
    if (fam > 0) rows = colv_family_rows(fam, L.wy);
  }
  return colv_plan(L.esz, L.W, L.H, L.wy, kMaxSmemBytes, rows, colv_lane_bytes(L), sm_count_v());
}

bool colv_fits(const FusedLaunch& L) { return L.wy >= 2 && colv_plan_for(L).ok; }

cudaError_t colv_launch(const FusedLaunch& L, cudaStream_t stream) {
  const int E = L.esz;
  const ColvPlan p = colv_plan_for(L);
  if (!p.ok) return cudaErrorInvalidConfiguration;
  const int sb = colv_strip_bytes(p.lb);
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
  a.ns = cdiv(L.W * E, sb);
  a.ntask = p.ntask;
  a.wpc = p.wpc;
  a.ld_vec = (reinterpret_cast<uintptr_t>(L.src) % p.lb == 0) && (L.sp % p.lb == 0);
  a.st_vec = (reinterpret_cast<uintptr_t>(L.dst) % p.lb == 0) && (L.dp % p.lb == 0);
  a.err = device_error_word();
  if (!a.err) return cudaErrorInvalidDevice;
  CUtensorMap tin;
  memset(&tin, 0, sizeof(tin));
  a.tma_ld = encode_tensor_map_2d(&tin, L.src, E, L.W, L.H, L.sp, sb / E, kCvBox) ? 1 : 0;
  ColvFn k = colv_kernel_for(E, L.op, p.lb);
  static std::mutex mu;
  static const void* opted[64][16] = {};
  {
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lock(mu);
    const int slot = (E - 1) * 4 + L.op * 2 + (p.lb == 8 ? 1 : 0);
    if (opted[dev & 63][slot] != reinterpret_cast<const void*>(k)) {
      cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmemBytes);
      if (e != cudaSuccess) return e;
      opted[dev & 63][slot] = reinterpret_cast<const void*>(k);
    }
  }
  const int grid = cdiv(p.ntask, p.wpc);
  return launch_pdl(L.pdl, k, dim3(grid), dim3(32 * p.wpc), p.smem, stream, tin, a);
}

}  // namespace morph
