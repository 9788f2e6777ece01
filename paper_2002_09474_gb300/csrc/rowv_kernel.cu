// The register-blocked van Herk/Gil-Werman kernel of the pass along x (w x 1
// windows, 9 <= w <= 256): instantiations, launch shape and launch.  Device
// code in morph_rowv.cuh.
#include <cstring>
#include <mutex>

#include "morph_geom.h"
#include "morph_internal.h"
#include "morph_rowv.cuh"
#include "plan.h"

namespace morph {

constexpr int kRvWarps = 4;  // warps per CTA

template <typename T, int OP>
__global__ void __launch_bounds__(32 * kRvWarps, 4) rowv_kernel(const RowvArgs a) {
  extern __shared__ __align__(128) uint8_t rvsmem[];
  pdl_launch_dependents();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int task = blockIdx.x * kRvWarps + warp;
  if (task >= a.ntask) return;
  pdl_wait();
  rowv_task<T, OP>(a, task, lane, rvsmem + warp * rv_warp_smem(sizeof(T)));
}

namespace {

using RowvFn = void (*)(const RowvArgs);

RowvFn rowv_kernel_for(int esz, int op) {
  if (esz == 1) return op == 0 ? rowv_kernel<uint8_t, 0> : rowv_kernel<uint8_t, 1>;
  return op == 0 ? rowv_kernel<uint16_t, 0> : rowv_kernel<uint16_t, 1>;
}

int sm_count_r() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  return n;
}

}  // namespace


bool rowv_fits(const FusedLaunch& L) {
  const int al = 8 * L.esz;  // row alignment the vector loads and stores need
  return L.wx >= 9 && L.wx <= 256 && L.wy == 1 && reinterpret_cast<uintptr_t>(L.src) % al == 0 &&
         L.sp % al == 0;
}

cudaError_t rowv_launch(const FusedLaunch& L, cudaStream_t stream) {
  const int sms = sm_count_r();
  if (sms <= 0) return cudaErrorInvalidDevice;
  if (!rowv_fits(L)) return cudaErrorInvalidConfiguration;
  const int smem = kRvWarps * rv_warp_smem(L.esz);
  RowvFn k = rowv_kernel_for(L.esz, L.op);
  static std::mutex mu;
  static const void* opted[64][4] = {};
  static int resident[64][4] = {};  // CTAs per SM
  int wps = 0;                        // resident warps per SM
  {
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lock(mu);
    const int slot = (L.esz - 1) * 2 + L.op;
    if (opted[dev & 63][slot] != reinterpret_cast<const void*>(k)) {
      cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
      if (e != cudaSuccess) return e;
      int n = 0;
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, 32 * kRvWarps, smem);
      if (e != cudaSuccess) return e;
      resident[dev & 63][slot] = n > 0 ? n : 1;
      opted[dev & 63][slot] = reinterpret_cast<const void*>(k);
    }
    wps = kRvWarps * resident[dev & 63][slot];
  }
  const RowvPlan p = rowv_plan(L.W, L.H, sms, wps, tuning().rowv_seg);
  if (!p.ok) return cudaErrorInvalidConfiguration;
  RowvArgs a;
  a.src = static_cast<const uint8_t*>(L.src);
  a.dst = static_cast<uint8_t*>(L.dst);
  a.sp = L.sp;
  a.dp = L.dp;
  a.W = L.W;
  a.H = L.H;
  a.w = L.wx;
  a.a = L.ax;
  a.seg = p.seg;
  a.nseg = p.nseg;
  a.ntask = p.ntask;
  const int al = 8 * L.esz;
  a.st_vec = (reinterpret_cast<uintptr_t>(L.dst) % al == 0) && (L.dp % al == 0);
  return launch_pdl(L.pdl, k, dim3(cdiv(p.ntask, kRvWarps)), dim3(32 * kRvWarps), smem, stream, a);
}

}  // namespace morph
