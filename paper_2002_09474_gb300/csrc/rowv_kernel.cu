// The register-blocked van Herk/Gil-Werman kernel of the pass along x (w x 1
// windows, 9 <= w <= 256): instantiations for 4 and 8 rows per warp, launch
// shape and launch.  Device code in morph_rowv.cuh.
#include <cstring>
#include <mutex>

#include "morph_geom.h"
#include "morph_internal.h"
#include "morph_rowv.cuh"
#include "plan.h"

namespace morph {

constexpr int kRvWarps = 4;  // warps per CTA

// Registers: at most 128 a thread with 8 rows per warp (4 CTAs of 4 warps),
// 80 with 4 rows (6 CTAs), 64 with 2 rows (8 CTAs).
template <typename T, int OP, int RR>
__global__ void __launch_bounds__(32 * kRvWarps, RR == 8 ? 4 : RR == 4 ? 6 : 8) rowv_kernel(const RowvArgs a) {
  extern __shared__ __align__(128) uint8_t rvsmem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int task = blockIdx.x * kRvWarps + warp;
  if (task >= a.ntask) return;
  pdl_wait();
  rowv_task<T, OP, RR>(a, task, lane, rvsmem + warp * rv_warp_smem(sizeof(T), RR));
  pdl_launch_dependents();
}

namespace {

using RowvFn = void (*)(const RowvArgs);

RowvFn rowv_kernel_for(int esz, int op, int rr) {
  if (rr == 2) {
    if (esz == 1) return op == 0 ? rowv_kernel<uint8_t, 0, 2> : rowv_kernel<uint8_t, 1, 2>;
    return op == 0 ? rowv_kernel<uint16_t, 0, 2> : rowv_kernel<uint16_t, 1, 2>;
  }
  if (rr == 8) {
    if (esz == 1) return op == 0 ? rowv_kernel<uint8_t, 0, 8> : rowv_kernel<uint8_t, 1, 8>;
    return op == 0 ? rowv_kernel<uint16_t, 0, 8> : rowv_kernel<uint16_t, 1, 8>;
  }
  if (esz == 1) return op == 0 ? rowv_kernel<uint8_t, 0, 4> : rowv_kernel<uint8_t, 1, 4>;
  return op == 0 ? rowv_kernel<uint16_t, 0, 4> : rowv_kernel<uint16_t, 1, 4>;
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

// Rows per warp: forced by the tuning mode (2: 8 rows, 3: 4 rows, 4: 2
// rows), else as the autotuner measured for this pixel type, else 2 -- measured on the GB300 at 4096^2 (u8 / u16, 101 x 1):
// 8 rows 22.1 / 29.2 us, 4 rows 17.2 / 22.3 us, 2 rows 14.8 / 16.1 us; fewer
// rows per warp lower the registers (64) and shared memory (3.6-4.2 KB) a
// warp needs, and the extra resident warps hide the latency.
int rowv_rows(int esz) {
  const Tuning& t = tuning();
  const int m = t.rowv_mode;
  if (m >= 2) return m == 2 ? 8 : m == 3 ? 4 : 2;
  const int r = t.rowv_rr[esz - 1];
  return r == 4 || r == 8 ? r : 2;
}

cudaError_t rowv_launch(const FusedLaunch& L, cudaStream_t stream) {
  const int sms = sm_count_r();
  if (sms <= 0) return cudaErrorInvalidDevice;
  if (!rowv_fits(L)) return cudaErrorInvalidConfiguration;
  const int rr = rowv_rows(L.esz);
  const int smem = kRvWarps * rv_warp_smem(L.esz, rr);
  RowvFn k = rowv_kernel_for(L.esz, L.op, rr);
  static std::mutex mu;
  static const void* opted[64][16] = {};
  static int resident[64][16] = {};  // CTAs per SM
  int wps = 0;                        // resident warps per SM
  {
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lock(mu);
    const int slot = (L.esz - 1) * 4 + L.op * 2 + (rr == 8 ? 1 : 0) + (rr == 2 ? 8 : 0);
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
  const RowvPlan p = rowv_plan(L.W, L.H, rr, sms, wps, tuning().rowv_seg);
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
