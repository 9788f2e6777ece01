// The strip-streaming van Herk/Gil-Werman kernel of the pass along y (1 x w
// windows): instantiations, launch shape and launch.  Device code in
// morph_cols.cuh.
#include <cstring>
#include <mutex>

#include "morph_cols.cuh"
#include "morph_geom.h"
#include "morph_internal.h"
#include "plan.h"

namespace morph {

template <typename T, int OP>
__global__ void __launch_bounds__(128) cols_kernel(const __grid_constant__ CUtensorMap tin, const ColsArgs a) {
  extern __shared__ __align__(128) uint8_t csmem[];
  pdl_launch_dependents();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int task = blockIdx.x * a.wpc + warp;
  if (task >= a.ntask) return;
  uint8_t* ws = csmem + warp * cols_warp_smem(a.rs);
  uint64_t* bars = cols_bars(ws, a.rs);
  if (lane == 0) {
    for (int b = 0; b < 2 * kCsSlots; ++b) mbar_init(&bars[b], 1);
    fence_barrier_init();
  }
  __syncwarp();
  pdl_wait();
  cols_task<T, OP>(a, &tin, task, lane, ws);
}

namespace {

using ColsFn = void (*)(const CUtensorMap, const ColsArgs);

ColsFn cols_kernel_for(int esz, int op) {
  if (esz == 1) return op == 0 ? cols_kernel<uint8_t, 0> : cols_kernel<uint8_t, 1>;
  return op == 0 ? cols_kernel<uint16_t, 0> : cols_kernel<uint16_t, 1>;
}

int sm_count_s() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  return n;
}

// Opts the kernel into the full shared memory once per device and returns
// the resident warps per SM its registers allow (0 on error).
int cols_prepare(ColsFn k, int esz, int op) {
  static std::mutex mu;
  static const void* opted[64][4] = {};
  static int max_warps[64][4] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  std::lock_guard<std::mutex> lock(mu);
  const int slot = (esz - 1) * 2 + op;
  if (opted[dev & 63][slot] != reinterpret_cast<const void*>(k)) {
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmemBytes) != cudaSuccess) return 0;
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, k) != cudaSuccess) return 0;
    const int regs = (fa.numRegs + 7) / 8 * 8;
    const int w = regs > 0 ? 65536 / (regs * 32) : 64;
    max_warps[dev & 63][slot] = w < 1 ? 1 : w > 64 ? 64 : w;
    opted[dev & 63][slot] = reinterpret_cast<const void*>(k);
  }
  return max_warps[dev & 63][slot];
}

}  // namespace

bool cols_fits(const FusedLaunch& L) {
  if (L.wy < 9 || L.wy > kCsMaxW) return false;
  CUtensorMap probe;
  if (!encode_tensor_map_2d(&probe, L.src, L.esz, L.W, L.H, L.sp, 128 / L.esz, kCsBox)) return false;
  return cols_plan(L.esz, L.W, L.H, L.wy, kMaxSmemBytes, 152, 64, tuning().colv_rows).ok;
}

cudaError_t cols_launch(const FusedLaunch& L, cudaStream_t stream) {
  const int E = L.esz;
  const int sms = sm_count_s();
  if (sms <= 0) return cudaErrorInvalidDevice;
  ColsFn k = cols_kernel_for(E, L.op);
  const int mw = cols_prepare(k, E, L.op);
  if (mw <= 0) return cudaErrorInvalidConfiguration;
  const ColsPlan p = cols_plan(E, L.W, L.H, L.wy, kMaxSmemBytes, sms, mw, tuning().colv_rows);
  if (!p.ok) return cudaErrorInvalidConfiguration;
  ColsArgs a;
  a.dst = static_cast<uint8_t*>(L.dst);
  a.dp = L.dp;
  a.W = L.W;
  a.H = L.H;
  a.w = L.wy;
  a.a = L.ay;
  a.Lo = p.Lo;
  a.ns = cdiv(L.W * E, 128);
  a.ntask = p.ntask;
  a.wpc = p.wpc;
  a.rs = p.rs;
  a.st_vec = (reinterpret_cast<uintptr_t>(L.dst) % 4 == 0) && (L.dp % 4 == 0);
  a.err = device_error_word();
  if (!a.err) return cudaErrorInvalidDevice;
  CUtensorMap tin;
  memset(&tin, 0, sizeof(tin));
  if (!encode_tensor_map_2d(&tin, L.src, E, L.W, L.H, L.sp, 128 / E, kCsBox)) return cudaErrorInvalidConfiguration;
  return launch_pdl(L.pdl, k, dim3(cdiv(p.ntask, p.wpc)), dim3(32 * p.wpc), p.smem, stream, tin, a);
}

}  // namespace morph
