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

template <typename T, int OP, int NWL, bool RG>
__global__ void __launch_bounds__(128) colv_kernel(const __grid_constant__ CUtensorMap tin, const ColvArgs a) {
  extern __shared__ __align__(128) uint8_t vsmem[];
  pdl_launch_dependents();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int task = blockIdx.x * a.wpc + warp;
  if (task >= a.ntask) return;
  uint8_t* tile = vsmem + warp * colv_tile_bytes(a.nbox, NWL);
  uint64_t* bars = reinterpret_cast<uint64_t*>(vsmem + a.wpc * colv_tile_bytes(a.nbox, NWL)) + warp * a.nbox;
  if (a.tma_ld) {
    if (lane == 0) {
      for (int b = 0; b < a.nbox; ++b) mbar_init(&bars[b], 1);
      fence_barrier_init();
    }
    __syncwarp();
  }
  pdl_wait();
  colv_tile<T, OP, NWL, RG>(a, &tin, task, lane, tile, bars);
}

// The shared-tile form (w > LW): thread 0 issues the CTA tile's boxes, every
// warp then makes its LW output rows.  Thread 0 waits for every box before
// the CTA exits, so no copy is in flight into released shared memory.
template <typename T, int OP, int LW>
__global__ void __launch_bounds__(256) colw_kernel(const __grid_constant__ CUtensorMap tin, const ColwArgs a) {
  extern __shared__ __align__(128) uint8_t wsmem[];
  constexpr int E = sizeof(T);
  uint64_t* bars = reinterpret_cast<uint64_t*>(wsmem + a.nbox * kCvBoxBytes);
  const int ctile = blockIdx.x;
  pdl_launch_dependents();
  pdl_wait();
  if (threadIdx.x == 0) {
    for (int b = 0; b < a.nbox; ++b) mbar_init(&bars[b], 1);
    fence_barrier_init();
    const int s = ctile % a.ns;
    const int ysc = (ctile / a.ns) * (a.nw * LW) - a.a;
    for (int b = 0; b < a.nbox; ++b) {
      mbar_arrive_expect_tx(&bars[b], static_cast<uint32_t>(kCvBoxBytes));
      tma_load_2d(wsmem + b * kCvBoxBytes, &tin, &bars[b], s * (kCvBytes / E), ysc + b * kCvBox);
    }
  }
  __syncthreads();
  colw_warp<T, OP, LW>(a, ctile, threadIdx.x >> 5, threadIdx.x & 31, wsmem, bars);
  if (threadIdx.x == 0)
    for (int b = 0; b < a.nbox; ++b) mbar_wait_bounded(&bars[b], 0);
}

namespace {

using ColvFn = void (*)(const CUtensorMap, const ColvArgs);
using ColwFn = void (*)(const CUtensorMap, const ColwArgs);

ColwFn colw_kernel_for(int esz, int op, int lw) {
  if (lw == 64) {
    if (esz == 1) return op == 0 ? colw_kernel<uint8_t, 0, 64> : colw_kernel<uint8_t, 1, 64>;
    return op == 0 ? colw_kernel<uint16_t, 0, 64> : colw_kernel<uint16_t, 1, 64>;
  }
  if (esz == 1) return op == 0 ? colw_kernel<uint8_t, 0, 32> : colw_kernel<uint8_t, 1, 32>;
  return op == 0 ? colw_kernel<uint16_t, 0, 32> : colw_kernel<uint16_t, 1, 32>;
}

int sm_count_w() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  return n;
}

ColvFn colv_kernel_for(int esz, int op, int nwl, bool ring) {
  if (ring) {
    if (esz == 1) return op == 0 ? colv_kernel<uint8_t, 0, 1, true> : colv_kernel<uint8_t, 1, 1, true>;
    return op == 0 ? colv_kernel<uint16_t, 0, 1, true> : colv_kernel<uint16_t, 1, 1, true>;
  }
  if (nwl == 2) {
    if (esz == 1) return op == 0 ? colv_kernel<uint8_t, 0, 2, false> : colv_kernel<uint8_t, 1, 2, false>;
    return op == 0 ? colv_kernel<uint16_t, 0, 2, false> : colv_kernel<uint16_t, 1, 2, false>;
  }
  if (esz == 1) return op == 0 ? colv_kernel<uint8_t, 0, 1, false> : colv_kernel<uint8_t, 1, 1, false>;
  return op == 0 ? colv_kernel<uint16_t, 0, 1, false> : colv_kernel<uint16_t, 1, 1, false>;
}

// Words per lane: 2 when forced (colv mode 4), and by default for windows
// of at most 16 rows on images at least 512 bytes wide (measured on the
// GB300 at 4096^2, 1 x 9 to 1 x 21: two independent scan chains per lane
// 3-10% faster up to 16 rows, slower from 17); else 1.
int colv_words(const FusedLaunch& L) {
  const int m = tuning().colv_mode;
  if (m == 4) return 2;
  if ((m == -1 || m == 1) && L.wy <= 16 && static_cast<long long>(L.W) * L.esz >= 512) return 2;
  return 1;
}

// The ring form (colv mode 6): rows a TMA box can load.
bool colv_ring_on(const FusedLaunch& L) {
  if (tuning().colv_mode != 6) return false;
  CUtensorMap probe;
  return encode_tensor_map_2d(&probe, L.src, L.esz, L.W, L.H, L.sp, kCvBytes / L.esz, kCvBox);
}

// The warp tile plan: rows forced by the tuning, else the built-in rule.
ColvPlan colv_plan_for(const FusedLaunch& L, bool ring) {
  if (ring) return colv_ring_plan(L.esz, L.W, L.H, L.wy, kMaxSmemBytes, tuning().colv_rows, sm_count_w());
  return colv_plan(L.esz, L.W, L.H, L.wy, kMaxSmemBytes, tuning().colv_rows, colv_words(L), sm_count_w());
}


}  // namespace

// Rows per warp of the shared-tile form for a window (0: not applicable).
int colw_rows(int w) { return w > 64 ? 64 : w > 32 ? 32 : 0; }

bool colw_fits(const FusedLaunch& L) {
  const int lw = colw_rows(L.wy);
  if (!lw) return false;
  CUtensorMap probe;
  if (!encode_tensor_map_2d(&probe, L.src, L.esz, L.W, L.H, L.sp, kCvBytes / L.esz, kCvBox)) return false;
  return colw_plan(L.esz, L.W, L.H, L.wy, lw, 152, kMaxSmemBytes, 16).ok;
}

cudaError_t colw_launch(const FusedLaunch& L, cudaStream_t stream) {
  const int E = L.esz, lw = colw_rows(L.wy);
  const int sms = sm_count_w();
  if (sms <= 0) return cudaErrorInvalidDevice;
  if (!lw) return cudaErrorInvalidConfiguration;
  ColwFn k = colw_kernel_for(E, L.op, lw);
  static std::mutex mu;
  static const void* opted[64][8] = {};
  static int max_warps[64][8] = {};  // resident warps per SM the registers allow
  int mw = 0;
  {
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lock(mu);
    const int slot = (E - 1) * 4 + L.op * 2 + (lw == 64 ? 1 : 0);
    if (opted[dev & 63][slot] != reinterpret_cast<const void*>(k)) {
      cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmemBytes);
      if (e != cudaSuccess) return e;
      cudaFuncAttributes fa;
      e = cudaFuncGetAttributes(&fa, k);
      if (e != cudaSuccess) return e;
      const int regs = (fa.numRegs + 7) / 8 * 8;
      int w = regs > 0 ? 65536 / (regs * 32) : 64;
      max_warps[dev & 63][slot] = w < 1 ? 1 : w > 64 ? 64 : w;
      opted[dev & 63][slot] = reinterpret_cast<const void*>(k);
    }
    mw = max_warps[dev & 63][slot];
  }
  const ColwPlan p = colw_plan(E, L.W, L.H, L.wy, lw, sms, kMaxSmemBytes, mw);
  if (!p.ok) return cudaErrorInvalidConfiguration;
  ColwArgs a;
  a.src = static_cast<const uint8_t*>(L.src);
  a.dst = static_cast<uint8_t*>(L.dst);
  a.sp = L.sp;
  a.dp = L.dp;
  a.W = L.W;
  a.H = L.H;
  a.w = L.wy;
  a.a = L.ay;
  a.nw = p.nw;
  a.nbox = p.nbox;
  a.ns = cdiv(L.W * E, kCvBytes);
  a.ntile = p.ntile;
  a.st_vec = (reinterpret_cast<uintptr_t>(L.dst) % 4 == 0) && (L.dp % 4 == 0);
  a.err = device_error_word();
  if (!a.err) return cudaErrorInvalidDevice;
  CUtensorMap tin;
  memset(&tin, 0, sizeof(tin));
  if (!encode_tensor_map_2d(&tin, L.src, E, L.W, L.H, L.sp, kCvBytes / E, kCvBox))
    return cudaErrorInvalidConfiguration;
  return launch_pdl(L.pdl, k, dim3(p.ntile), dim3(32 * p.nw), p.smem, stream, tin, a);
}

bool colv_fits(const FusedLaunch& L) {
  return L.wy >= 2 && colv_plan_for(L, colv_ring_on(L)).ok;
}

cudaError_t colv_launch(const FusedLaunch& L, cudaStream_t stream) {
  const int E = L.esz;
  const bool ring = colv_ring_on(L);
  const ColvPlan p = colv_plan_for(L, ring);
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
  a.ns = cdiv(L.W * E, kCvBytes * p.nwl);
  a.ntask = p.ntask;
  a.wpc = p.wpc;
  a.ld_vec = (reinterpret_cast<uintptr_t>(L.src) % 4 == 0) && (L.sp % 4 == 0);
  a.st_vec = (reinterpret_cast<uintptr_t>(L.dst) % (4 * p.nwl) == 0) && (L.dp % (4 * p.nwl) == 0);
  a.err = device_error_word();
  if (!a.err) return cudaErrorInvalidDevice;
  // ring form: the tile's rows cycle through the plan's boxes (when the
  // whole tile fits in fewer, nothing wraps)
  a.nring = ring ? p.nbox : 0;
  a.ring_mul = ring ? ((1 << 20) + p.nbox - 1) / p.nbox : 0;
  CUtensorMap tin;
  memset(&tin, 0, sizeof(tin));
  a.tma_ld = encode_tensor_map_2d(&tin, L.src, E, L.W, L.H, L.sp, kCvBytes * p.nwl / E, kCvBox) ? 1 : 0;
  if (ring && !a.tma_ld) return cudaErrorInvalidConfiguration;
  ColvFn k = colv_kernel_for(E, L.op, p.nwl, ring);
  static std::mutex mu;
  static const void* opted[64][16] = {};
  {
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lock(mu);
    const int slot = (E - 1) * 8 + L.op * 4 + (p.nwl == 2 ? 2 : 0) + (ring ? 1 : 0);
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
