// Single-image fused erosion/dilation kernel: one CTA per output tile.
#include <cstring>
#include <mutex>

#include <cudaTypedefs.h>

#include "morph_internal.h"
#include "morph_tile.cuh"

namespace morph {

__device__ int g_fused_err;

template <typename T, int OP, int TX, int TY>
__global__ void __launch_bounds__(kThreads, 2) fused_kernel(const __grid_constant__ CUtensorMap tin,
                                                         const __grid_constant__ CUtensorMap tout,
                                                         const ImgArgs a, const Geom g) {
  __shared__ __align__(8) uint64_t bar;
  extern __shared__ __align__(128) uint4 smem[];
  if (a.tma_ld && threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_barrier_init();
  }
  __syncthreads();
  uint32_t phase = 0;
  run_tile<T, OP, TX, TY>(a, &tin, &tout, blockIdx.x * TX, blockIdx.y * TY, g, smem, &bar, phase,
                          &g_fused_err);
}

namespace {

using KernelFn = void (*)(const CUtensorMap, const CUtensorMap, const ImgArgs, const Geom);

template <typename T, int OP>
KernelFn pick_kernel(int cfg) {
  switch (cfg) {
    case kTile128x64: return fused_kernel<T, OP, 128, 64>;
    case kTile64x64: return fused_kernel<T, OP, 64, 64>;
    case kTile64x128: return fused_kernel<T, OP, 64, 128>;
    case kTile256x32: return fused_kernel<T, OP, 256, 32>;
    case kTile32x32: return fused_kernel<T, OP, 32, 32>;
    case kTile32x128: return fused_kernel<T, OP, 32, 128>;
  }
  return nullptr;
}

KernelFn kernel_for(int esz, int op, int cfg) {
  if (esz == 1) return op == 0 ? pick_kernel<uint8_t, 0>(cfg) : pick_kernel<uint8_t, 1>(cfg);
  return op == 0 ? pick_kernel<uint16_t, 0>(cfg) : pick_kernel<uint16_t, 1>(cfg);
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

int fused_smem_bytes(const FusedLaunch& L) {
  if (L.cfg < 0 || L.cfg >= kNumTileCfg) return 0;
  return make_geom(L.esz, tile_tx(L.cfg), tile_ty(L.cfg), L.wx, L.wy, L.ax, L.vhgw_col, L.vhgw_row).smem_bytes;
}

cudaError_t fused_launch(const FusedLaunch& L, cudaStream_t stream) {
  const int TX = tile_tx(L.cfg), TY = tile_ty(L.cfg);
  const Geom g = make_geom(L.esz, TX, TY, L.wx, L.wy, L.ax, L.vhgw_col, L.vhgw_row);
  if (g.smem_bytes > kMaxSmemBytes) return cudaErrorInvalidConfiguration;
  KernelFn k = kernel_for(L.esz, L.op, L.cfg);
  if (!k) return cudaErrorInvalidValue;
  static bool opted[2][2][kNumTileCfg] = {};
  bool& done = opted[L.esz - 1][L.op][L.cfg];
  if (!done) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmemBytes);
    if (e != cudaSuccess) return e;
    done = true;
  }
  ImgArgs a;
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
  a.ld_vec = (reinterpret_cast<uintptr_t>(L.src) % 4 == 0) && (L.sp % 4 == 0);
  a.st_vec = (reinterpret_cast<uintptr_t>(L.dst) % 4 == 0) && (L.dp % 4 == 0);
  CUtensorMap tin, tout;
  memset(&tin, 0, sizeof(tin));
  memset(&tout, 0, sizeof(tout));
  a.tma_ld = encode_tensor_map_2d(&tin, L.src, L.esz, L.W, L.H, L.sp, 128 / L.esz, g.bh) ? 1 : 0;
  const int sbox = TX * L.esz < 128 ? TX * L.esz : 128;
  a.tma_st = encode_tensor_map_2d(&tout, L.dst, L.esz, L.W, L.H, L.dp, sbox / L.esz, TY) ? 1 : 0;
  dim3 grid(cdiv(L.W, TX), cdiv(L.H, TY));
  k<<<grid, kThreads, g.smem_bytes, stream>>>(tin, tout, a, g);
  return cudaGetLastError();
}

int fused_take_device_error() {
  int v = 0, z = 0;
  if (cudaMemcpyFromSymbol(&v, g_fused_err, sizeof(int)) != cudaSuccess) return -1;
  if (v) cudaMemcpyToSymbol(g_fused_err, &z, sizeof(int));
  return v;
}

}  // namespace morph
