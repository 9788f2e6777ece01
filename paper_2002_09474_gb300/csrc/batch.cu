// Batched erosion/dilation: many independent images of different sizes,
// windows, pixel types and operations in ONE persistent kernel launch.
//
// The host lays out, in device memory, one record per image (its arguments,
// tile geometry and TMA tensor maps) and the running count of tiles before
// each image.  Persistent CTAs (as many as fit on the GPU at once) take tile
// indices from an atomic counter, find the tile's image by binary search and
// run the same tile body as the single-image kernel.  All images of a batch
// share one output-tile shape, chosen so that every image's tile fits in
// shared memory.
#include <cstring>
#include <mutex>
#include <vector>

#include "batch.h"
#include "fused_kernel.cuh"
#include "plan.h"

namespace morph {

// Scheduling / error words of the batch kernels (kernels get their address).
__device__ int g_batch_err;

namespace {

template <int TX, int TY>
__global__ void __launch_bounds__(kThreads, 2) batch_kernel(const BatchImage* __restrict__ imgs,
                                                            const CUtensorMap* __restrict__ maps,
                                                            int nimg, int ntiles, int* counter, int* err) {
  __shared__ __align__(8) uint64_t bar;
  __shared__ int s_tile;
  extern __shared__ __align__(128) uint4 smem[];
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_barrier_init();
  }
  uint32_t phase = 0;
  for (;;) {
    __syncthreads();  // every thread has read the previous s_tile
    if (threadIdx.x == 0) s_tile = atomicAdd(counter, 1);
    __syncthreads();
    const int t = s_tile;
    if (t >= ntiles) break;
    // image of tile t: the last image whose first tile is <= t
    int lo = 0, hi = nimg - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (imgs[mid].tile0 <= t) lo = mid;
      else hi = mid - 1;
    }
    const BatchImage& im = imgs[lo];
    const int local = t - im.tile0;
    const int x0 = (local % im.tiles_x) * TX, y0 = (local / im.tiles_x) * TY;
    if (y0 >= im.a.H) {  // cannot happen for a consistent record
      if (threadIdx.x == 0) atomicExch(err, kDevErrBadTile);
      continue;
    }
    const CUtensorMap* tin = maps + 2 * lo;
    const CUtensorMap* tout = maps + 2 * lo + 1;
    bool ok;
    if (im.esz == 1)
      ok = im.op == 0 ? run_tile<uint8_t, 0, TX, TY>(im.a, tin, tout, x0, y0, im.g, smem, &bar, phase, err)
                      : run_tile<uint8_t, 1, TX, TY>(im.a, tin, tout, x0, y0, im.g, smem, &bar, phase, err);
    else
      ok = im.op == 0 ? run_tile<uint16_t, 0, TX, TY>(im.a, tin, tout, x0, y0, im.g, smem, &bar, phase, err)
                      : run_tile<uint16_t, 1, TX, TY>(im.a, tin, tout, x0, y0, im.g, smem, &bar, phase, err);
    if (!ok) break;  // a bounded wait gave up; the error word is set
  }
}

using BatchKernelFn = void (*)(const BatchImage*, const CUtensorMap*, int, int, int*, int*);

BatchKernelFn batch_kernel_for(int cfg) {
  switch (cfg) {
    case kTile128x64: return batch_kernel<128, 64>;
    case kTile64x64: return batch_kernel<64, 64>;
    case kTile32x32: return batch_kernel<32, 32>;
  }
  return nullptr;
}

int* batch_err_ptr() {
  static int* ptrs[64] = {};
  static std::mutex mu;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lock(mu);
  if (!ptrs[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_batch_err) != cudaSuccess) return nullptr;
    ptrs[dev] = static_cast<int*>(p);
  }
  return ptrs[dev];
}

}  // namespace

// Tile shapes a batch may use (one for all of its images).
static const int kBatchCfgs[] = {kTile128x64, kTile64x64, kTile32x32};

int batch_prepare(const BatchImageIn* in, int n, BatchHost* out) {
  out->cfg = -1;
  out->smem = 0;
  out->ntiles = 0;
  // the tile shape with the lowest summed cost that fits every image
  double best = 1e300;
  for (int cfg : kBatchCfgs) {
    double cost = 0;
    int smem = 0;
    bool fits = true;
    for (int i = 0; i < n && fits; ++i) {
      FusedLaunch L = in[i].L;
      L.cfg = cfg;
      const int b = fused_smem_bytes(L);
      if (b <= 0 || b > kMaxSmemBytes) fits = false;
      smem = smem > b ? smem : b;
      cost += tile_cost(L, cfg);
    }
    if (fits && cost < best) {
      best = cost;
      out->cfg = cfg;
      out->smem = smem;
    }
  }
  if (out->cfg < 0) return -1;
  const int TX = tile_tx(out->cfg), TY = tile_ty(out->cfg);
  out->imgs.resize(n);
  out->maps.assign(2 * static_cast<size_t>(n), CUtensorMap{});
  int tiles = 0;
  for (int i = 0; i < n; ++i) {
    const FusedLaunch& L = in[i].L;
    BatchImage& b = out->imgs[i];
    memset(&b, 0, sizeof(b));
    b.esz = L.esz;
    b.op = L.op;
    b.g = make_geom(L.esz, TX, TY, L.wx, L.wy, L.ax, L.vhgw_col, L.vhgw_row);
    fill_img_args(L, b.g, TX, TY, &b.a, &out->maps[2 * i], &out->maps[2 * i + 1]);
    b.tiles_x = cdiv(L.W, TX);
    b.tile0 = tiles;
    tiles += b.tiles_x * cdiv(L.H, TY);
  }
  out->ntiles = tiles;
  return 0;
}

cudaError_t batch_configure(BatchHost* h) {
  BatchKernelFn k = batch_kernel_for(h->cfg);
  if (!k) return cudaErrorInvalidValue;
  static bool opted[64][kNumTileCfg] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (!opted[dev & 63][h->cfg]) {
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmemBytes);
    if (e != cudaSuccess) return e;
    opted[dev & 63][h->cfg] = true;
  }
  int per_sm = 0, sms = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kThreads, h->smem);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  h->grid = per_sm * sms;
  if (h->grid > h->ntiles) h->grid = h->ntiles;
  if (h->grid < 1) h->grid = 1;
  h->err = batch_err_ptr();
  return h->err ? cudaSuccess : cudaErrorInvalidDevice;
}

cudaError_t batch_enqueue(const BatchHost& h, const BatchImage* d_imgs, const CUtensorMap* d_maps, int* d_counter,
                          cudaStream_t stream) {
  BatchKernelFn k = batch_kernel_for(h.cfg);
  if (!k || h.grid < 1 || !h.err) return cudaErrorInvalidValue;
  cudaError_t e = cudaMemsetAsync(d_counter, 0, sizeof(int), stream);
  if (e != cudaSuccess) return e;
  note_launch();
  k<<<h.grid, kThreads, h.smem, stream>>>(d_imgs, d_maps, static_cast<int>(h.imgs.size()), h.ntiles, d_counter,
                                          h.err);
  return cudaGetLastError();
}

cudaError_t batch_enqueue_raw(int cfg, int smem, int grid, int* err, int nimg, int ntiles,
                              const BatchImage* d_imgs, const CUtensorMap* d_maps, int* d_counter,
                              cudaStream_t stream) {
  BatchKernelFn k = batch_kernel_for(cfg);
  if (!k || grid < 1 || !err) return cudaErrorInvalidValue;
  cudaError_t e = cudaMemsetAsync(d_counter, 0, sizeof(int), stream);
  if (e != cudaSuccess) return e;
  note_launch();
  k<<<grid, kThreads, smem, stream>>>(d_imgs, d_maps, nimg, ntiles, d_counter, err);
  return cudaGetLastError();
}

int batch_take_device_error() {
  int v = 0, z = 0;
  if (cudaMemcpyFromSymbol(&v, g_batch_err, sizeof(int)) != cudaSuccess) return -1;
  if (v) cudaMemcpyToSymbol(g_batch_err, &z, sizeof(int));
  return v;
}

}  // namespace morph
