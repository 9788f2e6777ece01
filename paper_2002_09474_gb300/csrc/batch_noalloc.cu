// morph_batch_noalloc: the batched persistent launch for callers that may not
// allocate memory.  Its device scratch is a fixed array in this file; the
// host-side staging copy and working arrays are fixed-size statics too, so a
// call allocates nothing on the device or the host.
#include <algorithm>
#include <cstring>
#include <mutex>

#include "../../include/morph.h"
#include "batch.h"
#include "plan.h"

namespace morph {

int validate(const void* src, size_t sp, const void* dst, size_t dp, int W, int H, int dtype, int op, int wx,
             int wy, int ax, int ay);
void clip_window(int n, int w, int a, int* w_out, int* a_out);

namespace {

constexpr int kMaxImages = MORPH_NOALLOC_MAX_IMAGES;

// Layout of the scratch: tensor maps (64-byte aligned), image records, the
// tile counter.
struct NoallocScratch {
  CUtensorMap maps[2 * kMaxImages];
  BatchImage imgs[kMaxImages];
  int counter;
};

// The device scratch.  In host code this name is only a stand-in for the
// symbol; its device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[sizeof(NoallocScratch)];

// Host-side working storage of one call (shared by all calls).
NoallocScratch g_stage;
BatchImageIn g_in[kMaxImages];
struct Range {
  uintptr_t lo, hi;
  int is_dst;
};
Range g_ranges[2 * kMaxImages];

// Device address of g_noalloc_scratch per device, looked up once per device
// with that device current.
void* g_scratch_ptr[64] = {};
std::mutex g_setup_mu;

void* scratch_for_current_device() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lock(g_setup_mu);
  if (!g_scratch_ptr[dev]) {
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess) return nullptr;
    g_scratch_ptr[dev] = ptr;
  }
  return g_scratch_ptr[dev];
}

int esz_code(int dtype) { return dtype == MORPH_U8 ? 1 : dtype == MORPH_U16 ? 2 : 0; }

// Same checks and plan as the allocating morph_batch, on fixed arrays.
int plan_fixed(const morph_desc* d, int n) {
  for (int i = 0; i < n; ++i) {
    const morph_desc& e = d[i];
    if (e.src_pitch < 0 || e.dst_pitch < 0) return MORPH_ERR_PITCH;
    const int rc = validate(e.src, static_cast<size_t>(e.src_pitch), e.dst, static_cast<size_t>(e.dst_pitch),
                            e.width, e.height, e.dtype, e.op, e.wx, e.wy, e.anchor_x, e.anchor_y);
    if (rc != MORPH_OK) return rc;
    FusedLaunch& L = g_in[i].L;
    L = FusedLaunch();
    L.esz = esz_code(e.dtype);
    L.op = e.op;
    L.src = e.src;
    L.dst = e.dst;
    L.sp = e.src_pitch;
    L.dp = e.dst_pitch;
    L.W = e.width;
    L.H = e.height;
    clip_window(e.width, e.wx, e.anchor_x, &L.wx, &L.ax);
    clip_window(e.height, e.wy, e.anchor_y, &L.wy, &L.ay);
    if (!plan_single(&L)) return MORPH_ERR_WINDOW;
    const uintptr_t s0 = reinterpret_cast<uintptr_t>(e.src), d0 = reinterpret_cast<uintptr_t>(e.dst);
    const uintptr_t row = static_cast<uintptr_t>(e.width) * L.esz;
    g_ranges[2 * i] = {s0, s0 + static_cast<uintptr_t>(e.height - 1) * e.src_pitch + row, 0};
    g_ranges[2 * i + 1] = {d0, d0 + static_cast<uintptr_t>(e.height - 1) * e.dst_pitch + row, 1};
  }
  std::sort(g_ranges, g_ranges + 2 * n, [](const Range& a, const Range& b) { return a.lo < b.lo; });
  uintptr_t reach_any = 0, reach_dst = 0;
  for (int i = 0; i < 2 * n; ++i) {
    const Range& r = g_ranges[i];
    if (r.lo < reach_dst) return MORPH_ERR_ALIAS;
    if (r.is_dst && r.lo < reach_any) return MORPH_ERR_ALIAS;
    reach_any = std::max(reach_any, r.hi);
    if (r.is_dst) reach_dst = std::max(reach_dst, r.hi);
  }
  return MORPH_OK;
}

}  // namespace
}  // namespace morph

using namespace morph;

extern "C" int morph_batch_noalloc(const morph_desc* descs_host, int n, void* stream) {
  if (!descs_host) return MORPH_ERR_NULL;
  if (n < 1) return MORPH_ERR_ARG;
  if (n > kMaxImages) return MORPH_ERR_LIMIT;
  uint8_t* scratch = static_cast<uint8_t*>(scratch_for_current_device());
  if (!scratch) return MORPH_ERR_CUDA;
  int rc = plan_fixed(descs_host, n);
  if (rc != MORPH_OK) return rc;
  // tile shape shared by the batch: the cheapest that fits every image
  static const int cfgs[] = {kTile128x64, kTile64x64, kTile32x32};
  int cfg = -1, smem = 0;
  double best = 1e300;
  for (int c : cfgs) {
    double cost = 0;
    int need = 0;
    bool fits = true;
    for (int i = 0; i < n && fits; ++i) {
      FusedLaunch L = g_in[i].L;
      L.cfg = c;
      const int b = fused_smem_bytes(L);
      if (b <= 0 || b > kMaxSmemBytes) fits = false;
      need = need > b ? need : b;
      cost += tile_cost(L, c);
    }
    if (fits && cost < best) {
      best = cost;
      cfg = c;
      smem = need;
    }
  }
  if (cfg < 0) return MORPH_ERR_WINDOW;
  const int TX = tile_tx(cfg), TY = tile_ty(cfg);
  int tiles = 0;
  for (int i = 0; i < n; ++i) {
    const FusedLaunch& L = g_in[i].L;
    BatchImage& b = g_stage.imgs[i];
    memset(&b, 0, sizeof(b));
    b.esz = L.esz;
    b.op = L.op;
    b.g = make_geom(L.esz, TX, TY, L.wx, L.wy, L.ax, L.vhgw_col, L.vhgw_row);
    fill_img_args(L, b.g, TX, TY, &b.a, &g_stage.maps[2 * i], &g_stage.maps[2 * i + 1]);
    b.tiles_x = cdiv(L.W, TX);
    b.tile0 = tiles;
    tiles += b.tiles_x * cdiv(L.H, TY);
  }
  BatchHost h;  // default-constructed: its containers stay empty (no allocation)
  h.cfg = cfg;
  h.smem = smem;
  h.ntiles = tiles;
  if (batch_configure(&h) != cudaSuccess) return MORPH_ERR_CUDA;
  NoallocScratch* dev = reinterpret_cast<NoallocScratch*>(scratch);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemcpyAsync(dev->maps, g_stage.maps, sizeof(CUtensorMap) * 2 * n, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(dev->imgs, g_stage.imgs, sizeof(BatchImage) * n, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = batch_enqueue_raw(cfg, smem, h.grid, h.err, n, tiles, dev->imgs, dev->maps, &dev->counter, st);
  return e == cudaSuccess ? MORPH_OK : MORPH_ERR_CUDA;
}
