// Batched erosion/dilation: many independent images of different sizes,
// windows, pixel types and operations in a few launches.
//
// Each image goes where a single call of it would: windows whose passes take
// the direct method (and images too small for the single-pass kernels) into
// one persistent launch of the fused tile kernel; 1-D windows taking van
// Herk/Gil-Werman into a batched launch of their pass's kernel; 2-D windows
// whose passes both take van Herk/Gil-Werman into the batched pass along x,
// writing an intermediate image, and then the batched pass along y reading
// it (section 5: the element is separable).  The host lays out, in device
// memory, one record per image and pass (its arguments, TMA tensor maps and
// the running count of work items before it); a warp or CTA finds its
// record by binary search over those counts and runs the single-image
// kernel's own device code on it.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

#include "batch.h"
#include "fused_kernel.cuh"
#include "plan.h"

namespace morph {

int validate(const void* src, size_t sp, const void* dst, size_t dp, int W, int H, int dtype, int op, int wx,
             int wy, int ax, int ay);
void clip_window(int n, int w, int a, int* w_out, int* a_out);

// Scheduling / error words of the batch kernels (kernels get their address).
__device__ int g_batch_err;

namespace {

// ---- kernels -----------------------------------------------------------------

// Record of work item t: the last record whose first item is <= t.
template <typename R>
__device__ __forceinline__ int find_record(const R* recs, int n, int t, int R::*first) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (recs[mid].*first <= t) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

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
    const int i = find_record(imgs, nimg, t, &BatchImage::tile0);
    const BatchImage& im = imgs[i];
    const int local = t - im.tile0;
    const int x0 = (local % im.tiles_x) * TX, y0 = (local / im.tiles_x) * TY;
    if (y0 >= im.a.H) {  // cannot happen for a consistent record
      if (threadIdx.x == 0) atomicExch(err, kDevErrBadTile);
      continue;
    }
    const CUtensorMap* tin = maps + 2 * i;
    const CUtensorMap* tout = maps + 2 * i + 1;
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

// The pass along x of every record: one warp per task (kBatchRR rows and a
// segment of one image), each warp with the shared memory of the widest
// pixel type.
__global__ void __launch_bounds__(32 * 4, 8) batch_rowv_kernel(const BatchRowv* __restrict__ recs, int nrec,
                                                               int ntask) {
  extern __shared__ __align__(128) uint8_t bsmem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int t = blockIdx.x * 4 + warp;
  if (t >= ntask) return;
  const int i = find_record(recs, nrec, t, &BatchRowv::task0);
  const BatchRowv& r = recs[i];
  uint8_t* ws = bsmem + warp * rv_warp_smem(2, kBatchRR);
  const int local = t - r.task0;
  if (r.esz == 1) {
    if (r.op == 0) rowv_task<uint8_t, 0, kBatchRR>(r.a, local, lane, ws);
    else rowv_task<uint8_t, 1, kBatchRR>(r.a, local, lane, ws);
  } else {
    if (r.op == 0) rowv_task<uint16_t, 0, kBatchRR>(r.a, local, lane, ws);
    else rowv_task<uint16_t, 1, kBatchRR>(r.a, local, lane, ws);
  }
}

// The pass along y of one tile class: one warp (one CTA) per warp tile, the
// shared memory sized for the class's largest tile (nbox boxes).
__global__ void __launch_bounds__(32) batch_colv_kernel(const BatchColv* __restrict__ recs,
                                                        const CUtensorMap* __restrict__ maps, int nrec, int ntask,
                                                        int nbox) {
  extern __shared__ __align__(128) uint8_t bsmem[];
  const int lane = threadIdx.x;
  const int t = blockIdx.x;
  if (t >= ntask) return;
  const int i = find_record(recs, nrec, t, &BatchColv::task0);
  const BatchColv& r = recs[i];
  uint64_t* bars = reinterpret_cast<uint64_t*>(bsmem + colv_tile_bytes(nbox, 4));
  if (r.a.tma_ld) {
    if (lane == 0) {
      for (int b = 0; b < r.a.nbox; ++b) mbar_init(&bars[b], 1);
      fence_barrier_init();
    }
    __syncwarp();
  }
  const int local = t - r.task0;
  const CUtensorMap* tin = maps + r.map;
  if (r.esz == 1) {
    if (r.op == 0) colv_tile<uint8_t, 0, 4>(r.a, tin, local, lane, bsmem, bars);
    else colv_tile<uint8_t, 1, 4>(r.a, tin, local, lane, bsmem, bars);
  } else {
    if (r.op == 0) colv_tile<uint16_t, 0, 4>(r.a, tin, local, lane, bsmem, bars);
    else colv_tile<uint16_t, 1, 4>(r.a, tin, local, lane, bsmem, bars);
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

int esz_code(int dtype) { return dtype == MORPH_U8 ? 1 : dtype == MORPH_U16 ? 2 : 0; }

}  // namespace

// ---- host side -----------------------------------------------------------------

// SMs of the current device (looked up once per device).
static int batch_sms() {
  static int sms[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 1;
  if (!sms[dev]) {
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) return 1;
    sms[dev] = n;
  }
  return sms[dev];
}

// Arguments of the pass along x in a batch: kBatchRR rows per warp task,
// whole rows per task, or, with fill_gpu (a batch with too few tasks to fill
// the GPU), segments as a single call of the image would take them on the
// batched kernel's residency (4 warps a CTA, 8 CTAs an SM); false where the
// kernel does not take the launch (9 <= wx <= 256, wy = 1, rows aligned to
// 8 bytes per pixel byte).
bool rowv_batch_args(const FusedLaunch& L, RowvArgs* a, bool fill_gpu) {
  const int al = 8 * L.esz;
  if (L.wx < 9 || L.wx > 256 || L.wy != 1) return false;
  if (reinterpret_cast<uintptr_t>(L.src) % al || L.sp % al) return false;
  const RowvPlan p = fill_gpu ? rowv_plan(L.W, L.H, kBatchRR, batch_sms(), kBatchRowvWps, 0)
                              : rowv_plan(L.W, L.H, kBatchRR, 1, 1, L.W);
  if (!p.ok) return false;
  memset(a, 0, sizeof(*a));
  a->src = static_cast<const uint8_t*>(L.src);
  a->dst = static_cast<uint8_t*>(L.dst);
  a->sp = L.sp;
  a->dp = L.dp;
  a->W = L.W;
  a->H = L.H;
  a->w = L.wx;
  a->a = L.ax;
  a->seg = p.seg;
  a->nseg = p.nseg;
  a->ntask = p.ntask;
  a->st_vec = (reinterpret_cast<uintptr_t>(L.dst) % al == 0) && (L.dp % al == 0);
  return true;
}

// Arguments of the pass along y in a batch: one warp per CTA, 4 bytes per
// lane, the built-in tile height (with fill_gpu, shorter where the image has
// too few tiles to fill the GPU, as a single call's); false where its warp
// tile does not fit or its source is not one TMA can load (base and pitch
// multiples of 16 bytes: the kernel's plain loads are latency-bound at its
// one-warp-per-CTA occupancy).
bool colv_batch_args(const FusedLaunch& L, ColvArgs* a, CUtensorMap* map, bool fill_gpu) {
  if (L.wy < 2 || L.wx != 1) return false;
  if (!tma_loadable(L.src, L.sp)) return false;
  const ColvPlan p = colv_plan(L.esz, L.W, L.H, L.wy, kMaxSmemBytes, 0, 4, fill_gpu ? batch_sms() : 0);
  if (!p.ok || p.nbox > kCvMaxBox) return false;
  memset(a, 0, sizeof(*a));
  a->src = static_cast<const uint8_t*>(L.src);
  a->dst = static_cast<uint8_t*>(L.dst);
  a->sp = L.sp;
  a->dp = L.dp;
  a->W = L.W;
  a->H = L.H;
  a->w = L.wy;
  a->a = L.ay;
  a->L = p.L;
  a->nbox = p.nbox;
  a->ns = cdiv(L.W * L.esz, colv_strip_bytes(4));
  a->ntask = a->ns * cdiv(L.H, p.L);
  a->wpc = 1;
  a->ld_vec = (reinterpret_cast<uintptr_t>(L.src) % 4 == 0) && (L.sp % 4 == 0);
  a->st_vec = (reinterpret_cast<uintptr_t>(L.dst) % 4 == 0) && (L.dp % 4 == 0);
  a->err = device_error_word();
  if (!a->err) return false;
  memset(map, 0, sizeof(*map));
  a->tma_ld = encode_tensor_map_2d(map, L.src, L.esz, L.W, L.H, L.sp, colv_strip_bytes(4) / L.esz, kCvBox) ? 1 : 0;
  return true;
}


int plan_batch_into(const morph_desc* d, int n, BatchImageIn* out, BatchRange* ranges) {
  if (!d) return MORPH_ERR_NULL;
  if (n < 1) return MORPH_ERR_ARG;
  for (int i = 0; i < n; ++i) {
    const morph_desc& e = d[i];
    if (e.src_pitch < 0 || e.dst_pitch < 0) return MORPH_ERR_PITCH;
    const int rc = validate(e.src, static_cast<size_t>(e.src_pitch), e.dst, static_cast<size_t>(e.dst_pitch),
                            e.width, e.height, e.dtype, e.op, e.wx, e.wy, e.anchor_x, e.anchor_y);
    if (rc != MORPH_OK) return rc;
    FusedLaunch& L = out[i].L;
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
    ranges[2 * i] = {s0, s0 + static_cast<uintptr_t>(e.height - 1) * e.src_pitch + row, 0};
    ranges[2 * i + 1] = {d0, d0 + static_cast<uintptr_t>(e.height - 1) * e.dst_pitch + row, 1};
  }
  std::sort(ranges, ranges + 2 * n, [](const BatchRange& a, const BatchRange& b) { return a.lo < b.lo; });
  // sweep: a destination may not overlap any range that starts before it ends
  uintptr_t reach_any = 0, reach_dst = 0;
  for (int i = 0; i < 2 * n; ++i) {
    const BatchRange& r = ranges[i];
    if (r.lo < reach_dst) return MORPH_ERR_ALIAS;            // overlaps an earlier destination
    if (r.is_dst && r.lo < reach_any) return MORPH_ERR_ALIAS;  // a destination overlaps anything earlier
    reach_any = std::max(reach_any, r.hi);
    if (r.is_dst) reach_dst = std::max(reach_dst, r.hi);
  }
  return MORPH_OK;
}

// Tile shapes the fused group may use (one for all of its images).
static const int kBatchCfgs[] = {kTile128x64, kTile64x64, kTile32x32};

int batch_prepare_fused(const FusedLaunch* const* Ls, int n, int* cfg_out, int* smem_out, int* ntiles_out,
                        BatchImage* imgs, CUtensorMap* maps) {
  // the tile shape with the lowest summed cost that fits every image
  double best = 1e300;
  int cfg = -1, smem = 0;
  for (int c : kBatchCfgs) {
    double cost = 0;
    int need = 0;
    bool fits = true;
    for (int i = 0; i < n && fits; ++i) {
      FusedLaunch L = *Ls[i];
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
  if (cfg < 0) return -1;
  const int TX = tile_tx(cfg), TY = tile_ty(cfg);
  int tiles = 0;
  for (int i = 0; i < n; ++i) {
    const FusedLaunch& L = *Ls[i];
    BatchImage& b = imgs[i];
    memset(&b, 0, sizeof(b));
    b.esz = L.esz;
    b.op = L.op;
    b.g = make_geom(L.esz, TX, TY, L.wx, L.wy, L.ax, L.vhgw_col, L.vhgw_row);
    fill_img_args(L, b.g, TX, TY, &b.a, &maps[2 * i], &maps[2 * i + 1]);
    b.tiles_x = cdiv(L.W, TX);
    b.tile0 = tiles;
    tiles += b.tiles_x * cdiv(L.H, TY);
  }
  *cfg_out = cfg;
  *smem_out = smem;
  *ntiles_out = tiles;
  return 0;
}

namespace {

enum BatchForm { kFormFused = 0, kFormX = 1, kFormY = 2, kFormXY = 3, kFormFY = 4 };

// Pass-along-x launch of L (wy must be 1) in a batch.
FusedLaunch x_part(const FusedLaunch& L) {
  FusedLaunch A = L;
  A.wy = 1;
  A.ay = 0;
  return A;
}
FusedLaunch y_part(const FusedLaunch& L) {
  FusedLaunch B = L;
  B.wx = 1;
  B.ax = 0;
  return B;
}
size_t inter_pitch(const FusedLaunch& L) { return (static_cast<size_t>(L.W) * L.esz + 15) / 16 * 16; }

// The form an image takes in a batch: the single-pass kernels wherever a
// pass takes van Herk/Gil-Werman and their kernels accept it, the fused
// kernel otherwise.  The intermediate of a 2-D window is 16-byte pitched,
// so both passes of it always qualify once the source does.
int batch_form(const FusedLaunch& L) {
  const bool vx = L.wx > 1 && L.vhgw_row, vy = L.wy > 1 && L.vhgw_col;
  RowvArgs ra;
  ColvArgs ca;
  CUtensorMap m;
  if (L.wx > 1 && L.wy > 1) {
    // two passes when the pass along x takes van Herk/Gil-Werman; a direct
    // pass along y then runs on the pass-along-y kernel too (exact for any
    // window), instead of a fused tile carrying the pass along x's halo
    // (2000 uneven images: those images took half of the fused launch's
    // time)
    FusedLaunch A = x_part(L), B = y_part(L);
    // the pass along y reads a 16-byte-pitched intermediate
    B.src = reinterpret_cast<const void*>(static_cast<uintptr_t>(256));
    B.sp = static_cast<long long>(inter_pitch(L));
    A.dst = reinterpret_cast<void*>(static_cast<uintptr_t>(256));
    A.dp = B.sp;
    if (vx) return rowv_batch_args(A, &ra) && colv_batch_args(B, &ca, &m) ? kFormXY : kFormFused;
    // a direct pass along x (the pass-along-x kernel needs 9 pixels) with a
    // pass along y above the crossover: the pass along x as a 1-D record of
    // the fused group, the pass along y on its kernel
    if (vy) return colv_batch_args(B, &ca, &m) ? kFormFY : kFormFused;
    return kFormFused;
  }
  if (L.wy == 1 && vx) return rowv_batch_args(L, &ra) ? kFormX : kFormFused;
  if (L.wx == 1 && vy) return colv_batch_args(L, &ca, &m) ? kFormY : kFormFused;
  return kFormFused;
}

}  // namespace

bool batch_runs_alone(const FusedLaunch& L) {
  // a pass that takes van Herk/Gil-Werman whose source the batched
  // single-pass kernels cannot load fast: its single call has kernels that
  // can (the row and column kernels), where the fused kernel's tile would
  // carry the window's whole halo
  const bool vx = L.wx > 1 && L.vhgw_row, vy = L.wy > 1 && L.vhgw_col;
  if (!vx && !vy) return false;
  if (L.wx > 1 && L.wy > 1 && (!vx || !vy)) return false;  // a direct pass: the fused kernel
  return batch_form(L) == kFormFused;
}

namespace {

int colv_class(int nbox) {
  for (int c = 0; c < kColvClasses; ++c)
    if (nbox <= kColvClassBoxes[c]) return c;
  return -1;
}

}  // namespace

int batch_prepare(const BatchImageIn* in, int n, BatchHost* out) {
  *out = BatchHost();
  // Forms, and the warp tasks of the single-pass groups in their long-task
  // shapes (whole rows; the built-in tile height): a group whose tasks do
  // not fill the GPU takes the shorter tasks a single call would.
  std::vector<int> forms(n);
  long long tx = 0, ty = 0, ty_slots = 0;
  for (int i = 0; i < n; ++i) {
    const FusedLaunch& L = in[i].L;
    forms[i] = batch_form(L);
    if (forms[i] == kFormFused) continue;
    if (forms[i] == kFormX || forms[i] == kFormXY) tx += (L.H + kBatchRR - 1) / kBatchRR;
    if (forms[i] != kFormX) {
      const ColvPlan p = colv_plan(L.esz, L.W, L.H, L.wy, kMaxSmemBytes, 0, 4, 0);
      if (!p.ok) return -1;
      ty += static_cast<long long>(cdiv(L.W * L.esz, colv_strip_bytes(4))) * cdiv(L.H, p.L);
      ty_slots = std::max<long long>(ty_slots, static_cast<long long>(batch_sms()) * p.wps);
    }
  }
  const bool fill_x = tx < static_cast<long long>(batch_sms()) * kBatchRowvWps;
  const bool fill_y = 5 * ty < 3 * ty_slots;
  std::vector<const FusedLaunch*> fused;
  // storage of the 1-D pass-along-x records of the fused group (reserved,
  // so that pointers into it stay valid)
  std::vector<FusedLaunch> xparts;
  xparts.reserve(n);
  std::vector<BatchColv> cols_by_class[kColvClasses];
  std::vector<CUtensorMap> maps_by_class[kColvClasses];
  std::vector<int> inter_class;  // class of each intermediate's pass-along-y record (index in .col until sorted)
  size_t inter = 0;
  for (int i = 0; i < n; ++i) {
    const FusedLaunch& L = in[i].L;
    const int form = forms[i];
    if (form == kFormFused) {
      fused.push_back(&L);
      continue;
    }
    int fused_x = -1;
    if (form == kFormFY) {  // placeholder destination until bound
      FusedLaunch A = x_part(L);
      A.dst = reinterpret_cast<void*>(static_cast<uintptr_t>(256));
      A.dp = static_cast<long long>(inter_pitch(L));
      xparts.push_back(A);
      fused_x = static_cast<int>(fused.size());
      fused.push_back(&xparts.back());
      out->fused_x.push_back(A);
    }
    if (form == kFormX || form == kFormXY) {
      BatchRowv r;
      memset(&r, 0, sizeof(r));
      FusedLaunch A = form == kFormXY ? x_part(L) : L;
      if (form == kFormXY) {  // placeholder destination until bound
        A.dst = reinterpret_cast<void*>(static_cast<uintptr_t>(256));
        A.dp = static_cast<long long>(inter_pitch(L));
      }
      if (!rowv_batch_args(A, &r.a, fill_x)) return -1;
      r.esz = L.esz;
      r.op = L.op;
      r.task0 = out->row_tasks;
      out->row_tasks += r.a.ntask;
      out->rows.push_back(r);
    }
    if (form == kFormY || form == kFormXY || form == kFormFY) {
      const bool split = form != kFormY;
      BatchColv c;
      memset(&c, 0, sizeof(c));
      CUtensorMap m;
      memset(&m, 0, sizeof(m));
      FusedLaunch B = split ? y_part(L) : L;
      if (split) {
        B.src = reinterpret_cast<const void*>(static_cast<uintptr_t>(256));
        B.sp = static_cast<long long>(inter_pitch(L));
      }
      if (!colv_batch_args(B, &c.a, &m, fill_y)) return -1;
      c.esz = L.esz;
      c.op = L.op;
      const int k = colv_class(c.a.nbox);
      if (k < 0) return -1;
      if (split) {
        BatchHost::Inter t;
        t.row = form == kFormXY ? static_cast<int>(out->rows.size()) - 1 : -1;
        t.fused = fused_x;
        t.col = static_cast<int>(cols_by_class[k].size());
        t.off = inter;
        t.pitch = static_cast<long long>(inter_pitch(L));
        t.W = L.W;
        t.H = L.H;
        t.esz = L.esz;
        out->inters.push_back(t);
        inter_class.push_back(k);
        inter += (inter_pitch(L) * static_cast<size_t>(L.H) + 255) / 256 * 256;
      }
      cols_by_class[k].push_back(c);
      maps_by_class[k].push_back(m);
    }
  }
  out->inter_bytes = inter;
  for (int k = 0; k < kColvClasses; ++k) {
    out->col_first[k] = static_cast<int>(out->cols.size());
    out->col_count[k] = static_cast<int>(cols_by_class[k].size());
    int tasks = 0;
    for (BatchColv& c : cols_by_class[k]) {
      c.task0 = tasks;
      tasks += c.a.ntask;
      c.map = static_cast<int>(out->col_maps.size());
      out->cols.push_back(c);
      out->col_maps.push_back(maps_by_class[k][&c - cols_by_class[k].data()]);
    }
    out->col_tasks[k] = tasks;
  }
  for (size_t j = 0; j < out->inters.size(); ++j) out->inters[j].col += out->col_first[inter_class[j]];
  if (!fused.empty()) {
    out->imgs.resize(fused.size());
    out->maps.assign(2 * fused.size(), CUtensorMap{});
    if (batch_prepare_fused(fused.data(), static_cast<int>(fused.size()), &out->cfg, &out->smem, &out->ntiles,
                            out->imgs.data(), out->maps.data()) != 0)
      return -1;
  }
  return 0;
}

int batch_bind_intermediates(void* inter, BatchHost* h) {
  uint8_t* base = static_cast<uint8_t*>(inter);
  size_t fx = 0;  // next of h->fused_x
  for (const BatchHost::Inter& t : h->inters) {
    uint8_t* p = base + t.off;
    if (t.fused >= 0) {
      // the fused record of the pass along x, filled again with its output
      if (fx >= h->fused_x.size() || t.fused >= static_cast<int>(h->imgs.size())) return -1;
      FusedLaunch A = h->fused_x[fx++];
      A.dst = p;
      A.dp = t.pitch;
      BatchImage& b = h->imgs[t.fused];
      fill_img_args(A, b.g, tile_tx(h->cfg), tile_ty(h->cfg), &b.a, &h->maps[2 * t.fused], &h->maps[2 * t.fused + 1]);
    } else {
      RowvArgs& ra = h->rows[t.row].a;
      ra.dst = p;
      ra.dp = t.pitch;
    }
    BatchColv& c = h->cols[t.col];
    c.a.src = p;
    c.a.sp = t.pitch;
    CUtensorMap& m = h->col_maps[c.map];
    memset(&m, 0, sizeof(m));
    c.a.tma_ld = encode_tensor_map_2d(&m, p, t.esz, t.W, t.H, t.pitch, colv_strip_bytes(4) / t.esz, kCvBox) ? 1 : 0;
  }
  return 0;
}

namespace {

template <typename K>
cudaError_t opt_in(K k, int smem, bool* done) {
  if (*done) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess) *done = true;
  return e;
}

}  // namespace

cudaError_t batch_fused_grid(int cfg, int smem, int ntiles, int* grid, int** err) {
  BatchKernelFn k = batch_kernel_for(cfg);
  if (!k) return cudaErrorInvalidValue;
  static bool opted[64][kNumTileCfg] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = opt_in(k, kMaxSmemBytes, &opted[dev & 63][cfg]);
  if (e != cudaSuccess) return e;
  int per_sm = 0, sms = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kThreads, smem);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  int g = per_sm * sms;
  if (g > ntiles) g = ntiles;
  *grid = g < 1 ? 1 : g;
  *err = batch_err_ptr();
  return *err ? cudaSuccess : cudaErrorInvalidDevice;
}

cudaError_t batch_configure(BatchHost* h) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (!h->imgs.empty()) {
    e = batch_fused_grid(h->cfg, h->smem, h->ntiles, &h->grid, &h->err);
    if (e != cudaSuccess) return e;
  } else {
    h->err = batch_err_ptr();
  }
  static bool opted_r[64] = {}, opted_c[64] = {};
  e = opt_in(batch_rowv_kernel, 4 * rv_warp_smem(2, kBatchRR), &opted_r[dev & 63]);
  if (e != cudaSuccess) return e;
  return opt_in(batch_colv_kernel, kMaxSmemBytes, &opted_c[dev & 63]);
}

BatchDev batch_dev_layout(const BatchHost& h) {
  auto up = [](size_t v) { return (v + 255) / 256 * 256; };
  BatchDev L;
  L.maps_off = 0;
  L.imgs_off = up(h.maps.size() * sizeof(CUtensorMap));
  L.counter_off = up(L.imgs_off + h.imgs.size() * sizeof(BatchImage));
  L.rows_off = L.counter_off + 256;
  L.col_maps_off = up(L.rows_off + h.rows.size() * sizeof(BatchRowv));
  L.cols_off = up(L.col_maps_off + h.col_maps.size() * sizeof(CUtensorMap));
  L.inter_off = up(L.cols_off + h.cols.size() * sizeof(BatchColv));
  L.bytes = L.inter_off + h.inter_bytes;
  return L;
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

cudaError_t batch_enqueue(const BatchHost& h, uint8_t* base, const BatchDev& L, cudaStream_t stream) {
  cudaError_t e = cudaSuccess;
  if (!h.imgs.empty()) {
    e = batch_enqueue_raw(h.cfg, h.smem, h.grid, h.err, static_cast<int>(h.imgs.size()), h.ntiles,
                          reinterpret_cast<const BatchImage*>(base + L.imgs_off),
                          reinterpret_cast<const CUtensorMap*>(base + L.maps_off),
                          reinterpret_cast<int*>(base + L.counter_off), stream);
    if (e != cudaSuccess) return e;
  }
  if (!h.rows.empty()) {
    note_launch();
    batch_rowv_kernel<<<cdiv(h.row_tasks, 4), 32 * 4, 4 * rv_warp_smem(2, kBatchRR), stream>>>(
        reinterpret_cast<const BatchRowv*>(base + L.rows_off), static_cast<int>(h.rows.size()), h.row_tasks);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  for (int k = 0; k < kColvClasses; ++k) {
    if (!h.col_count[k]) continue;
    note_launch();
    const int nbox = kColvClassBoxes[k];
    batch_colv_kernel<<<h.col_tasks[k], 32, colv_smem_bytes(nbox, 1, 4), stream>>>(
        reinterpret_cast<const BatchColv*>(base + L.cols_off) + h.col_first[k],
        reinterpret_cast<const CUtensorMap*>(base + L.col_maps_off), h.col_count[k], h.col_tasks[k], nbox);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return e;
}

int batch_take_device_error() {
  int v = 0, z = 0;
  if (cudaMemcpyFromSymbol(&v, g_batch_err, sizeof(int)) != cudaSuccess) return -1;
  if (v) cudaMemcpyToSymbol(g_batch_err, &z, sizeof(int));
  return v;
}

}  // namespace morph
