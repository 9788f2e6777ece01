// Host-side interfaces between the C-ABI layer and the kernel translation
// units (not part of the public ABI).
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

namespace morph {

// Output tile shapes the fused kernel is built for (TX x TY pixels): square,
// tall (for long windows along y) and wide (for long windows along x).
enum TileCfg : int {
  kTile128x64 = 0,
  kTile64x64 = 1,
  kTile64x128 = 2,
  kTile256x32 = 3,
  kTile32x32 = 4,
  kTile128x128 = 5,
  kTile256x64 = 6,
  kTile32x128 = 7,
  kNumTileCfg = 8
};
inline int tile_tx(int cfg) {
  static const int tx[kNumTileCfg] = {128, 64, 64, 256, 32, 128, 256, 32};
  return tx[cfg];
}
inline int tile_ty(int cfg) {
  static const int ty[kNumTileCfg] = {64, 64, 128, 32, 32, 128, 64, 128};
  return ty[cfg];
}

// Largest dynamic shared memory a CTA may use on sm_103a (bytes).
constexpr int kMaxSmemBytes = 227 * 1024 - 1024;  // leave room for static smem

// One single-image launch of the fused kernel, fully resolved.
struct FusedLaunch {
  int esz;             // 1 or 2
  int op;              // 0 erode, 1 dilate
  int cfg;             // TileCfg
  const void* src;
  void* dst;
  long long sp, dp;
  int W, H;
  int wx, wy, ax, ay;  // clipped window
  bool vhgw_col, vhgw_row;
  bool pipe;           // persistent input-prefetching kernel (set by the planner)
  bool pdl;            // launch with programmatic stream serialisation (the
                       // second launch of the two-launch form)
};

// Shared-memory bytes the fused kernel needs for this launch (0 if the
// configuration is invalid).
int fused_smem_bytes(const FusedLaunch& L);
// The same for the persistent, prefetching form (two region-A slots).
int fused_pipe_smem_bytes(const FusedLaunch& L);
// Kernel entry of one (pixel type, op, tile configuration); defined in the
// instantiation units fused_inst_*.cu.
struct ImgArgs;
struct Geom;
using FusedKernelFn = void (*)(const CUtensorMap, const CUtensorMap, const ImgArgs, const Geom);
FusedKernelFn fused_kernel_u8_erode(int cfg);
FusedKernelFn fused_kernel_u8_dilate(int cfg);
FusedKernelFn fused_kernel_u16_erode(int cfg);
FusedKernelFn fused_kernel_u16_dilate(int cfg);
// The persistent, input-prefetching form (fused_pipe_kernel).
using FusedPipeKernelFn = void (*)(const CUtensorMap, const CUtensorMap, const ImgArgs, const Geom, int, int);
FusedPipeKernelFn fused_pipe_kernel_u8_erode(int cfg);
FusedPipeKernelFn fused_pipe_kernel_u8_dilate(int cfg);
FusedPipeKernelFn fused_pipe_kernel_u16_erode(int cfg);
FusedPipeKernelFn fused_pipe_kernel_u16_dilate(int cfg);

// Counts one kernel launch enqueued by the library (morph_launch_count).
void note_launch();

// Launches kernel k; with pdl, with programmatic stream serialisation: it
// may then be scheduled while the previous kernel on the stream finishes
// (its CTAs wait in griddepcontrol.wait before touching memory).  Counts the
// launch.
template <typename... Params, typename... Args>
cudaError_t launch_pdl(bool pdl, void (*k)(Params...), dim3 grid, dim3 block, size_t smem, cudaStream_t stream,
                       Args&&... args) {
  note_launch();
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, k, static_cast<Args&&>(args)...);
}

// Enqueues the fused kernel; returns a cudaError_t.
cudaError_t fused_launch(const FusedLaunch& L, cudaStream_t stream);
// Reads and clears the fused kernels' device error word.
int fused_take_device_error();
// Device address of that word on the current device (nullptr on failure).
int* device_error_word();

// The column-pass kernel for 1 x wy windows (blocked: van Herk/Gil-Werman
// blocks, needs wy >= 9; else the direct method).
cudaError_t col_launch(const FusedLaunch& L, bool blocked, cudaStream_t stream);

// The warp-tiled van Herk/Gil-Werman kernel of the pass along y (any wy >= 2),
// when its warp tile fits in shared memory (colv_fits).
bool colv_fits(const FusedLaunch& L);
cudaError_t colv_launch(const FusedLaunch& L, cudaStream_t stream);

// dst -= sub for row_bytes bytes of each of H rows (pixels of esz bytes; the
// gradient's dilation minus erosion, which never wraps).
cudaError_t sub_launch(void* dst, long long dp, const void* sub, long long sp, int row_bytes, int H, int esz,
                       cudaStream_t stream);

// The one-pass opening (kind 0), closing (1) or gradient (2) for windows of
// at most 9 pixels a side on images at least as large as the window
// (comp_fits; morph_comp.cuh).  The anchor is the first step's; the second
// step of an opening or closing takes the reflected element.
bool comp_fits(int W, int H, int wx, int wy);
cudaError_t comp_launch(const void* src, long long sp, void* dst, long long dp, int W, int H, int esz, int kind,
                        int wx, int wy, int ax, int ay, bool pdl, cudaStream_t stream);

// One warp waits, bounded, on an mbarrier phase nothing completes, and
// records kDevErrTmaTimeout when the wait gives up (selftest.cu).
cudaError_t selftest_wait_timeout(cudaStream_t stream);

// The register-blocked van Herk/Gil-Werman kernel of the pass along x
// (9 <= wx <= 256, rows aligned to 8 * esz bytes; rowv_fits).
bool rowv_fits(const FusedLaunch& L);
cudaError_t rowv_launch(const FusedLaunch& L, cudaStream_t stream);

// The row-pass kernel for wx x 1 windows (blocked needs wx >= 9), when its
// tile fits in shared memory (row_fits).
bool row_fits(const FusedLaunch& L);
cudaError_t row_launch(const FusedLaunch& L, bool blocked, cudaStream_t stream);

// Enqueues the tiled transpose kernel: dst (W rows of H pixels) = src^T.
cudaError_t transpose_launch(const void* src, long long sp, void* dst, long long dp, int W, int H, int esz,
                             cudaStream_t stream);

// Encodes a 2-D tiled tensor map over a pitched image (driver entry point
// resolved through the runtime).  Returns false if TMA cannot describe it.
bool encode_tensor_map_2d(CUtensorMap* map, const void* base, int esz, int W, int H, long long pitch,
                          int box_w, int box_h);

}  // namespace morph
