// Single-image fused erosion/dilation kernel: one CTA per output tile.
#include <cstring>
#include <mutex>

#include <cudaTypedefs.h>

#include "morph_internal.h"
#include "batch.h"
#include "fused_kernel.cuh"

namespace morph {

// Device error word of the fused kernels (kernels get its address).
__device__ int g_fused_err;

namespace {

using KernelFn = FusedKernelFn;

KernelFn kernel_for(int esz, int op, int cfg) {
  if (cfg < 0 || cfg >= kNumTileCfg) return nullptr;
  if (esz == 1) return op == 0 ? fused_kernel_u8_erode(cfg) : fused_kernel_u8_dilate(cfg);
  return op == 0 ? fused_kernel_u16_erode(cfg) : fused_kernel_u16_dilate(cfg);
}

FusedPipeKernelFn pipe_kernel_for(int esz, int op, int cfg) {
  if (cfg < 0 || cfg >= kNumTileCfg) return nullptr;
  if (esz == 1) return op == 0 ? fused_pipe_kernel_u8_erode(cfg) : fused_pipe_kernel_u8_dilate(cfg);
  return op == 0 ? fused_pipe_kernel_u16_erode(cfg) : fused_pipe_kernel_u16_dilate(cfg);
}

// Raises a kernel's dynamic shared-memory limit once per device.
cudaError_t allow_smem(const void* fn) {
  static std::mutex mu;
  static const void* done[64][64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  const void** row = done[dev & 63];
  for (int i = 0; i < 64; ++i) {
    if (row[i] == fn) return cudaSuccess;
    if (!row[i]) {
      e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmemBytes);
      if (e == cudaSuccess) row[i] = fn;
      return e;
    }
  }
  return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmemBytes);
}

// CTAs of a persistent launch: resident CTAs per SM x SMs, at most one per tile.
int persistent_grid(const void* fn, int smem, int ntiles) {
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kThreads, smem) != cudaSuccess) return 0;
  if (per_sm < 1) return 0;
  const long long n = static_cast<long long>(sms) * per_sm;
  return static_cast<int>(n < ntiles ? n : ntiles);
}

// Address of g_fused_err on the current device (cached per device).
int* fused_err_ptr() {
  static int* ptrs[64] = {};
  static std::mutex mu;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lock(mu);
  if (!ptrs[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_fused_err) != cudaSuccess) return nullptr;
    ptrs[dev] = static_cast<int*>(p);
  }
  return ptrs[dev];
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

}  // namespace

bool encode_tensor_map_2d(CUtensorMap* map, const void* base, int esz, int W, int H, long long pitch,
                          int box_w, int box_h) {
  auto fn = encode_fn();
  if (!fn) return false;
  if ((reinterpret_cast<uintptr_t>(base) & 15) || (pitch & 15) || pitch >= (1ll << 40)) return false;
  if (box_w < 1 || box_w > 256 || box_h < 1 || box_h > 256 || (box_w * esz) % 16) return false;
  // A box larger than the tensor is not used: the kernels' transfer counts
  // assume full boxes.
  if (box_w > W || box_h > H) return false;
  cuuint64_t dims[2] = {static_cast<cuuint64_t>(W), static_cast<cuuint64_t>(H)};
  cuuint64_t strides[1] = {static_cast<cuuint64_t>(pitch)};
  cuuint32_t box[2] = {static_cast<cuuint32_t>(box_w), static_cast<cuuint32_t>(box_h)};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, esz == 1 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_UINT16, 2,
                  const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

void fill_img_args(const FusedLaunch& L, const Geom& g, int TX, int TY, ImgArgs* ap, CUtensorMap* tin,
                   CUtensorMap* tout) {
  ImgArgs& a = *ap;
  a.src = static_cast<const uint8_t*>(L.src);
  a.dst = static_cast<uint8_t*>(L.dst);
  a.sp = L.sp;
  a.dp = L.dp;
  a.W = L.W;
  a.H = L.H;
  a.wx = L.wx;
  a.wy = L.wy;
  a.ax = L.ax;
  a.ay = L.ay;
  a.blk_y = L.vhgw_col && L.wy > 1;
  a.blk_x = L.vhgw_row && L.wx > 1;
  a.err = fused_err_ptr();
  a.ld_vec = (reinterpret_cast<uintptr_t>(L.src) % 4 == 0) && (L.sp % 4 == 0);
  a.st_vec = (reinterpret_cast<uintptr_t>(L.dst) % 4 == 0) && (L.dp % 4 == 0);
  a.st_vec16 = (reinterpret_cast<uintptr_t>(L.dst) % 16 == 0) && (L.dp % 16 == 0);
  memset(tin, 0, sizeof(*tin));
  memset(tout, 0, sizeof(*tout));
  a.tma_ld = encode_tensor_map_2d(tin, L.src, L.esz, L.W, L.H, L.sp, 128 / L.esz, g.bh) ? 1 : 0;
  // TMA stores only with 128-byte box rows (tiles at least 128 bytes wide),
  // the form proven on the GPU; the kernel uses them for whole tiles only.
  a.tma_st = (TX * L.esz >= 128) && encode_tensor_map_2d(tout, L.dst, L.esz, L.W, L.H, L.dp, 128 / L.esz, TY);
}

int fused_smem_bytes(const FusedLaunch& L) {
  if (L.cfg < 0 || L.cfg >= kNumTileCfg) return 0;
  return make_geom(L.esz, tile_tx(L.cfg), tile_ty(L.cfg), L.wx, L.wy, L.ax, L.vhgw_col, L.vhgw_row).smem_bytes;
}

int fused_pipe_smem_bytes(const FusedLaunch& L) {
  if (L.cfg < 0 || L.cfg >= kNumTileCfg) return 0;
  return make_geom(L.esz, tile_tx(L.cfg), tile_ty(L.cfg), L.wx, L.wy, L.ax, L.vhgw_col, L.vhgw_row, true)
      .smem_bytes;
}

cudaError_t fused_launch(const FusedLaunch& L, cudaStream_t stream) {
  const int TX = tile_tx(L.cfg), TY = tile_ty(L.cfg);
  const Geom g = make_geom(L.esz, TX, TY, L.wx, L.wy, L.ax, L.vhgw_col, L.vhgw_row);
  if (g.smem_bytes > kMaxSmemBytes) return cudaErrorInvalidConfiguration;
  ImgArgs a;
  CUtensorMap tin, tout;
  fill_img_args(L, g, TX, TY, &a, &tin, &tout);
  if (!a.err) return cudaErrorInvalidDevice;
  const int ntx = cdiv(L.W, TX), nty = cdiv(L.H, TY);
  if (L.pipe && a.tma_ld) {
    const Geom gp = make_geom(L.esz, TX, TY, L.wx, L.wy, L.ax, L.vhgw_col, L.vhgw_row, true);
    FusedPipeKernelFn k = pipe_kernel_for(L.esz, L.op, L.cfg);
    if (k && gp.smem_bytes <= kMaxSmemBytes && gp.bh == g.bh) {
      cudaError_t e = allow_smem(reinterpret_cast<const void*>(k));
      if (e != cudaSuccess) return e;
      const int grid = persistent_grid(reinterpret_cast<const void*>(k), gp.smem_bytes, ntx * nty);
      if (grid > 0) {
        return launch_pdl(L.pdl, k, dim3(grid), dim3(kThreads), gp.smem_bytes, stream, tin, tout, a, gp, ntx, ntx * nty);
      }
    }
  }
  KernelFn k = kernel_for(L.esz, L.op, L.cfg);
  if (!k) return cudaErrorInvalidValue;
  cudaError_t e = allow_smem(reinterpret_cast<const void*>(k));
  if (e != cudaSuccess) return e;
  dim3 grid(ntx, nty);
  return launch_pdl(L.pdl, k, grid, dim3(kThreads), g.smem_bytes, stream, tin, tout, a, g);
}

int* device_error_word() { return fused_err_ptr(); }

int fused_take_device_error() {
  int v = 0, z = 0;
  if (cudaMemcpyFromSymbol(&v, g_fused_err, sizeof(int)) != cudaSuccess) return -1;
  if (v) cudaMemcpyToSymbol(g_fused_err, &z, sizeof(int));
  return v;
}

}  // namespace morph
