// C ABI (include/morph.h): argument checks, exact window clipping, method and
// tile choice (section 5.3's crossover), launches, host staging.
#include <algorithm>
#include <atomic>
#include <cstring>
#include <mutex>
#include <vector>

#include "../../include/morph.h"
#include "../../include/morph_tuning.h"
#include "batch.h"
#include "morph_internal.h"
#include "plan.h"

using namespace morph;

namespace {

int esz_of(int dtype) { return dtype == MORPH_U8 ? 1 : dtype == MORPH_U16 ? 2 : 0; }

// Byte ranges [p, p + (H-1)*pitch + W*esz) of source and destination overlap?
bool overlaps(const void* a, size_t ap, const void* b, size_t bp, int W, int H, int esz) {
  const uintptr_t a0 = reinterpret_cast<uintptr_t>(a), b0 = reinterpret_cast<uintptr_t>(b);
  const uintptr_t a1 = a0 + static_cast<uintptr_t>(H - 1) * ap + static_cast<uintptr_t>(W) * esz;
  const uintptr_t b1 = b0 + static_cast<uintptr_t>(H - 1) * bp + static_cast<uintptr_t>(W) * esz;
  return a0 < b1 && b0 < a1;
}

}  // namespace

namespace morph {

int validate(const void* src, size_t sp, const void* dst, size_t dp, int W, int H, int dtype, int op, int wx,
             int wy, int ax, int ay) {
  if (!src || !dst) return MORPH_ERR_NULL;
  const int esz = esz_of(dtype);
  if (!esz || (op != MORPH_ERODE && op != MORPH_DILATE)) return MORPH_ERR_DTYPE;
  if (W < 1 || H < 1 || W > (1 << 30) || H > (1 << 30)) return MORPH_ERR_SIZE;
  if (wx < 1 || wy < 1) return MORPH_ERR_WINDOW;
  if (ax < 0 || ax >= wx || ay < 0 || ay >= wy) return MORPH_ERR_ANCHOR;
  if (sp < static_cast<size_t>(W) * esz || dp < static_cast<size_t>(W) * esz) return MORPH_ERR_PITCH;
  // 16-bit pixels must be 2-byte aligned in every row.
  if (esz == 2 && ((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst) | sp | dp) & 1))
    return MORPH_ERR_PITCH;
  if (overlaps(src, sp, dst, dp, W, H, esz)) return MORPH_ERR_ALIAS;
  return MORPH_OK;
}

// A window never needs more than n-1 cells on either side of its anchor on an
// axis of n pixels: every output pixel's clipped window is unchanged when the
// part beyond n-1 cells is cut off.  So (w, a) -> (a' + e' + 1, a') with
// a' = min(a, n-1), e' = min(w-1-a, n-1) gives identical results.
void clip_window(int n, int w, int a, int* w_out, int* a_out) {
  const int before = std::min(a, n - 1);
  const int after = std::min(w - 1 - a, n - 1);
  *a_out = before;
  *w_out = before + after + 1;
}

namespace {

constexpr int kMaxDevices = 64;

// Stream-ordered scratch (intermediate images, batch records) comes from a
// memory pool of the library's own per device, whose release threshold keeps
// freed memory mapped for the next call.  The device's default pool gives
// freed memory back to the driver at every synchronisation, after which the
// next large allocation maps new pages on the calling thread: milliseconds
// for a few hundred MB, and a stall of whatever loop issues the calls.
// morph_release_staging trims the pools.
std::mutex g_pool_mu;
cudaMemPool_t g_pool[kMaxDevices] = {};

cudaError_t scratch_pool(cudaMemPool_t* out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_pool_mu);
  if (!g_pool[dev]) {
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool = nullptr;
    e = cudaMemPoolCreate(&pool, &props);
    if (e != cudaSuccess) return e;
    uint64_t keep = ~0ull;
    e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    if (e != cudaSuccess) {
      cudaMemPoolDestroy(pool);
      return e;
    }
    g_pool[dev] = pool;
  }
  *out = g_pool[dev];
  return cudaSuccess;
}

// Pool memory, freed with cudaFreeAsync.  Under stream capture the
// allocation becomes a node of the graph (cudaMallocAsync), which owns it.
cudaError_t scratch_malloc(void** p, size_t bytes, cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaError_t e = cudaStreamIsCapturing(st, &cs);
  if (e != cudaSuccess) return e;
  if (cs != cudaStreamCaptureStatusNone) return cudaMallocAsync(p, bytes, st);
  cudaMemPool_t pool = nullptr;
  e = scratch_pool(&pool);
  if (e != cudaSuccess) return e;
  return cudaMallocFromPoolAsync(p, bytes, pool, st);
}

// Stream-ordered scratch image of `rows` rows of `row_bytes` (pitch rounded
// to 16 bytes so that TMA can describe it).
struct Scratch {
  void* p = nullptr;
  size_t pitch = 0;
  cudaStream_t st = nullptr;
  bool alloc(size_t row_bytes, int rows, cudaStream_t s) {
    st = s;
    pitch = (row_bytes + 15) / 16 * 16;
    return scratch_malloc(&p, pitch * static_cast<size_t>(rows), s) == cudaSuccess;
  }
  ~Scratch() {
    if (p) cudaFreeAsync(p, st);
  }
};

// The warp-tiled pass along y and the register-blocked pass along x: used
// when forced (mode >= 1) and they accept the launch; in auto mode (-1)
// wherever the van Herk/Gil-Werman method is chosen, where both were
// measured faster than the column and row kernels on the GB300 (4096^2
// images, CUDA-graph timing): along y 10-25% at 51, 101 and 127 rows, along
// x 19-26% (u8) and 41-59% (u16) at 21, 101 and 127 columns.
bool use_colv(const FusedLaunch& L) {
  const int m = tuning().colv_mode;
  if (m == 0) return false;
  // in auto mode only on sources TMA can describe: its plain loads are
  // latency-bound at its occupancy (GB300, 1 x 101 at 4096^2, u8: 10.6 us
  // aligned, 138 us from an unaligned base, where the column kernel takes
  // 20.7 us)
  return (m >= 1 || (L.vhgw_col && tma_loadable(L.src, L.sp))) && colv_fits(L);
}
bool use_rowv(const FusedLaunch& L) {
  const int m = tuning().rowv_mode;
  if (m == 0) return false;
  return (m >= 1 || L.vhgw_row) && rowv_fits(L);
}

int launch_one(FusedLaunch L, cudaStream_t stream) {
  if (!plan_single(&L)) return MORPH_ERR_WINDOW;
  if (tuning().pdl_mode == 1) L.pdl = true;
  if (L.wx == 1 && L.wy > 1 && use_colv(L)) {
    return colv_launch(L, stream) == cudaSuccess ? MORPH_OK : MORPH_ERR_CUDA;
  }
  if (L.wx == 1 && L.wy > 1 && tuning().col_mode != 0)
    return col_launch(L, L.vhgw_col && L.wy >= 9, stream) == cudaSuccess ? MORPH_OK : MORPH_ERR_CUDA;
  if (L.wy == 1 && L.wx > 1 && use_rowv(L))
    return rowv_launch(L, stream) == cudaSuccess ? MORPH_OK : MORPH_ERR_CUDA;
  if (L.wy == 1 && L.wx > 1 && tuning().row_mode != 0 && row_fits(L))
    return row_launch(L, L.vhgw_row && L.wx >= 9, stream) == cudaSuccess ? MORPH_OK : MORPH_ERR_CUDA;
  return fused_launch(L, stream) == cudaSuccess ? MORPH_OK : MORPH_ERR_CUDA;
}

// The pass along x in the paper's baseline form (section 5.2.1): transpose,
// the same pass along y, transpose back -- here through the standalone
// transpose kernels and HBM, where the fused kernel transposes 8x8 blocks in
// registers.  A 2-D window first runs its 1 x wy pass into a scratch image.
int launch_transposed_x(const FusedLaunch& L, cudaStream_t stream) {
  const int W = L.W, H = L.H, e = L.esz;
  const void* xs = L.src;
  long long xsp = L.sp;
  Scratch ya, tb, tc;
  if (L.wy > 1) {
    if (!ya.alloc(static_cast<size_t>(W) * e, H, stream)) return MORPH_ERR_NOMEM;
    FusedLaunch A = L;
    A.wx = 1;
    A.ax = 0;
    A.dst = ya.p;
    A.dp = static_cast<long long>(ya.pitch);
    const int rc = launch_one(A, stream);
    if (rc != MORPH_OK) return rc;
    xs = ya.p;
    xsp = A.dp;
  }
  // tb, tc: H pixels per row, W rows (the transposed image)
  if (!tb.alloc(static_cast<size_t>(H) * e, W, stream) || !tc.alloc(static_cast<size_t>(H) * e, W, stream))
    return MORPH_ERR_NOMEM;
  if (transpose_launch(xs, xsp, tb.p, static_cast<long long>(tb.pitch), W, H, e, stream) != cudaSuccess)
    return MORPH_ERR_CUDA;
  FusedLaunch B = L;
  B.W = H;
  B.H = W;
  B.wx = 1;
  B.ax = 0;
  B.wy = L.wx;
  B.ay = L.ax;
  B.src = tb.p;
  B.sp = static_cast<long long>(tb.pitch);
  B.dst = tc.p;
  B.dp = static_cast<long long>(tc.pitch);
  const int rc = launch_one(B, stream);
  if (rc != MORPH_OK) return rc;
  return transpose_launch(tc.p, static_cast<long long>(tc.pitch), L.dst, L.dp, H, W, e, stream) == cudaSuccess
             ? MORPH_OK
             : MORPH_ERR_CUDA;
}

}  // namespace

int launch_planned(FusedLaunch L, cudaStream_t stream) {
  if (L.wx > 1 && tuning().xpass_transpose[L.esz - 1]) return launch_transposed_x(L, stream);
  if (!plan_split(L)) return launch_one(L, stream);
  // Split form (section 5's separability): one 1-D pass into an
  // intermediate image, then the other from it (the pass along x first by
  // default).  The intermediate is a
  // stream-ordered allocation (16-byte rows, so both launches can use TMA).
  Scratch tmp;
  if (!tmp.alloc(static_cast<size_t>(L.W) * L.esz, L.H, stream)) return MORPH_ERR_NOMEM;
  FusedLaunch A = L, B = L;
  if (tuning().split_order == 1) {  // the pass along x first
    A.wy = 1;
    A.ay = 0;
    B.wx = 1;
    B.ax = 0;
  } else {
    A.wx = 1;
    A.ax = 0;
    B.wy = 1;
    B.ay = 0;
  }
  A.dst = tmp.p;
  A.dp = static_cast<long long>(tmp.pitch);
  B.src = tmp.p;
  B.sp = static_cast<long long>(tmp.pitch);
  int rc = launch_one(A, stream);
  if (rc == MORPH_OK) rc = launch_one(B, stream);
  return rc;
}

namespace {
std::atomic<long long> g_launches{0};
}  // namespace

void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

int run_single(const void* src, size_t sp, void* dst, size_t dp, int W, int H, int dtype, int op, int wx,
               int wy, int ax, int ay, cudaStream_t stream) {
  int rc = validate(src, sp, dst, dp, W, H, dtype, op, wx, wy, ax, ay);
  if (rc != MORPH_OK) return rc;
  FusedLaunch L;
  memset(&L, 0, sizeof(L));
  L.esz = esz_of(dtype);
  L.op = op;
  L.src = src;
  L.dst = dst;
  L.sp = static_cast<long long>(sp);
  L.dp = static_cast<long long>(dp);
  L.W = W;
  L.H = H;
  clip_window(W, wx, ax, &L.wx, &L.ax);
  clip_window(H, wy, ay, &L.wy, &L.ay);
  return launch_planned(L, stream);
}

// Device staging buffers of morph_apply_host: one input/output pair per
// device, grown on demand and kept until morph_release_staging.
struct Staging {
  void* in = nullptr;
  void* out = nullptr;
  size_t bytes = 0;
};
Staging g_staging[kMaxDevices];
std::mutex g_staging_mu;

int stage_buffers(size_t bytes, void** in, void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return MORPH_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_staging_mu);
  Staging& s = g_staging[dev];
  if (s.bytes < bytes) {
    if (s.in) cudaFree(s.in);
    if (s.out) cudaFree(s.out);
    s = Staging();
    if (cudaMalloc(&s.in, bytes) != cudaSuccess) return MORPH_ERR_NOMEM;
    if (cudaMalloc(&s.out, bytes) != cudaSuccess) {
      cudaFree(s.in);
      s.in = nullptr;
      return MORPH_ERR_NOMEM;
    }
    s.bytes = bytes;
  }
  *in = s.in;
  *out = s.out;
  return MORPH_OK;
}

// Copy/compute pipeline of morph_apply_host_batch, one per device: three
// staging slots (input and output image each), three streams (copies in,
// filtering, copies out) and the events that order a slot's stages, so the
// copy in of image i+1, the filtering of image i and the copy out of image
// i-1 run at the same time.
constexpr int kPipeSlots = 3;
struct Pipeline {
  std::mutex mu;
  void* in[kPipeSlots] = {};
  void* out[kPipeSlots] = {};
  size_t bytes = 0;
  cudaStream_t st[3] = {};
  cudaEvent_t start = nullptr;
  cudaEvent_t in_done[kPipeSlots] = {}, comp_done[kPipeSlots] = {}, out_done[kPipeSlots] = {};
  bool ready = false;
};
Pipeline g_pipe[kMaxDevices];

void free_pipeline_buffers(Pipeline& p) {
  for (int k = 0; k < kPipeSlots; ++k) {
    if (p.in[k]) cudaFree(p.in[k]);
    if (p.out[k]) cudaFree(p.out[k]);
    p.in[k] = p.out[k] = nullptr;
  }
  p.bytes = 0;
}

int pipeline_for_current_device(size_t bytes, Pipeline** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return MORPH_ERR_CUDA;
  Pipeline& p = g_pipe[dev];
  std::lock_guard<std::mutex> lock(p.mu);
  if (!p.ready) {
    for (int k = 0; k < 3; ++k)
      if (cudaStreamCreateWithFlags(&p.st[k], cudaStreamNonBlocking) != cudaSuccess) return MORPH_ERR_CUDA;
    if (cudaEventCreateWithFlags(&p.start, cudaEventDisableTiming) != cudaSuccess) return MORPH_ERR_CUDA;
    for (int k = 0; k < kPipeSlots; ++k)
      if (cudaEventCreateWithFlags(&p.in_done[k], cudaEventDisableTiming) != cudaSuccess ||
          cudaEventCreateWithFlags(&p.comp_done[k], cudaEventDisableTiming) != cudaSuccess ||
          cudaEventCreateWithFlags(&p.out_done[k], cudaEventDisableTiming) != cudaSuccess)
        return MORPH_ERR_CUDA;
    p.ready = true;
  }
  if (p.bytes < bytes) {
    for (int k = 0; k < 3; ++k) cudaStreamSynchronize(p.st[k]);
    free_pipeline_buffers(p);
    for (int k = 0; k < kPipeSlots; ++k)
      if (cudaMalloc(&p.in[k], bytes) != cudaSuccess || cudaMalloc(&p.out[k], bytes) != cudaSuccess) {
        free_pipeline_buffers(p);
        return MORPH_ERR_NOMEM;
      }
    p.bytes = bytes;
  }
  *out = &p;
  return MORPH_OK;
}

void release_pipelines() {
  int cur = 0;
  cudaGetDevice(&cur);
  for (int d = 0; d < kMaxDevices; ++d) {
    Pipeline& p = g_pipe[d];
    std::lock_guard<std::mutex> lock(p.mu);
    if (!p.bytes) continue;
    cudaSetDevice(d);
    for (int k = 0; k < 3; ++k) cudaStreamSynchronize(p.st[k]);
    free_pipeline_buffers(p);
  }
  cudaSetDevice(cur);
}

int plan_batch(const morph_desc* d, int n, std::vector<BatchImageIn>* out) {
  if (!d) return MORPH_ERR_NULL;
  if (n < 1) return MORPH_ERR_ARG;
  out->resize(n);
  std::vector<BatchRange> ranges(2 * static_cast<size_t>(n));
  return plan_batch_into(d, n, out->data(), ranges.data());
}

// Pinned host staging of batch records, per device: slots used in turn, each
// with the event of the copy that last read it, so records travel by truly
// asynchronous copies (a copy from pageable memory would wait for the
// stream's earlier work and stall the caller).  A call takes a slot whose
// previous copy has run; while every slot is still queued behind other
// work it adds one (up to kStageSlotsMax), and only then waits.  Slots grow
// on demand.
constexpr int kStageSlotsMax = 64;
struct RecordStage {
  std::mutex mu;
  void* buf[kStageSlotsMax] = {};
  size_t cap[kStageSlotsMax] = {};
  cudaEvent_t ev[kStageSlotsMax] = {};
  int used = 0, next = 0;
};
RecordStage g_rstage[kMaxDevices];

// Copies `bytes` of host records at `src` to device `dst` on `st` through
// the pinned staging slots.
cudaError_t stage_records(void* dst, const void* const* parts, const size_t* sizes, const size_t* offs, int nparts,
                          size_t bytes, cudaStream_t st) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  RecordStage& rs = g_rstage[dev];
  std::lock_guard<std::mutex> lock(rs.mu);
  int k = -1;
  for (int i = 0; i < rs.used && k < 0; ++i) {
    const int j = (rs.next + i) % rs.used;
    e = cudaEventQuery(rs.ev[j]);
    if (e == cudaSuccess) k = j;
    else if (e != cudaErrorNotReady) return e;
  }
  if (k < 0 && rs.used < kStageSlotsMax) {
    e = cudaEventCreateWithFlags(&rs.ev[rs.used], cudaEventDisableTiming);
    if (e != cudaSuccess) return e;
    k = rs.used++;
  }
  if (k < 0) {
    k = rs.next % rs.used;
    e = cudaEventSynchronize(rs.ev[k]);  // the slot's previous copy has run
    if (e != cudaSuccess) return e;
  }
  rs.next = (k + 1) % rs.used;
  if (rs.cap[k] < bytes) {
    if (rs.buf[k]) cudaFreeHost(rs.buf[k]);
    rs.buf[k] = nullptr;
    rs.cap[k] = 0;
    const size_t want = bytes < (1u << 16) ? (1u << 16) : bytes * 2;
    e = cudaHostAlloc(&rs.buf[k], want, cudaHostAllocDefault);
    if (e != cudaSuccess) return e;
    rs.cap[k] = want;
  }
  uint8_t* h = static_cast<uint8_t*>(rs.buf[k]);
  for (int i = 0; i < nparts; ++i)
    if (sizes[i]) memcpy(h + offs[i], parts[i], sizes[i]);
  e = cudaMemcpyAsync(dst, h, bytes, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return e;
  return cudaEventRecord(rs.ev[k], st);
}

// The records of a prepared batch into its device block (layout L) on `st`.
cudaError_t upload_batch(const BatchHost& h, const BatchDev& L, uint8_t* base, cudaStream_t st) {
  const void* parts[5] = {h.maps.data(), h.imgs.data(), h.rows.data(), h.col_maps.data(), h.cols.data()};
  const size_t sizes[5] = {h.maps.size() * sizeof(CUtensorMap), h.imgs.size() * sizeof(BatchImage),
                           h.rows.size() * sizeof(BatchRowv), h.col_maps.size() * sizeof(CUtensorMap),
                           h.cols.size() * sizeof(BatchColv)};
  const size_t offs[5] = {L.maps_off, L.imgs_off, L.rows_off, L.col_maps_off, L.cols_off};
  return stage_records(base, parts, sizes, offs, 5, L.inter_off, st);
}

struct BatchPlan {
  int device = 0;
  BatchHost host;
  void* dmem = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

namespace {

// Takes out of a planned batch `in` the images that run as their own single
// call (batch_runs_alone, or at least the tuned number of pixels); their
// descriptor indices go to `alone`, and `in` keeps the rest, in order, for
// the batched launches.
void split_alone(const morph_desc* d, std::vector<BatchImageIn>* in, std::vector<int>* alone) {
  const long long lim = tuning().batch_alone;
  size_t k = 0;
  for (size_t i = 0; i < in->size(); ++i) {
    if ((lim > 0 && static_cast<long long>(d[i].width) * d[i].height >= lim) || batch_runs_alone((*in)[i].L)) {
      alone->push_back(static_cast<int>(i));
    } else {
      (*in)[k++] = (*in)[i];
    }
  }
  in->resize(k);
}

// The single calls of the images split off above, on `st`.
int run_alone(const morph_desc* d, const std::vector<int>& alone, cudaStream_t st) {
  for (int i : alone) {
    const morph_desc& e = d[i];
    const int rc = run_single(e.src, static_cast<size_t>(e.src_pitch), e.dst, static_cast<size_t>(e.dst_pitch),
                              e.width, e.height, e.dtype, e.op, e.wx, e.wy, e.anchor_x, e.anchor_y, st);
    if (rc != MORPH_OK) return rc;
  }
  return MORPH_OK;
}

}  // namespace

}  // namespace morph

// ---------------------------------------------------------------------------
// Exported entry points
// ---------------------------------------------------------------------------
extern "C" {

int morph_apply(const void* src, size_t src_pitch, void* dst, size_t dst_pitch, int width, int height,
                int dtype, int op, int wx, int wy, int anchor_x, int anchor_y, void* stream) {
  return run_single(src, src_pitch, dst, dst_pitch, width, height, dtype, op, wx, wy, anchor_x, anchor_y,
                    static_cast<cudaStream_t>(stream));
}

int morph_composite(const void* src, size_t src_pitch, void* dst, size_t dst_pitch, int width, int height,
                    int dtype, int kind, int wx, int wy, int anchor_x, int anchor_y, void* stream) {
  if (kind != MORPH_OPEN && kind != MORPH_CLOSE && kind != MORPH_GRADIENT) return MORPH_ERR_ARG;
  int rc = validate(src, src_pitch, dst, dst_pitch, width, height, dtype, MORPH_ERODE, wx, wy, anchor_x, anchor_y);
  if (rc != MORPH_OK) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int esz = esz_of(dtype);
  // one pass over the image, both steps in shared memory (no intermediate
  // image): forced (mode 1) wherever it fits; by default for the gradient
  // of windows up to 5 x 5, where it was measured faster on the GB300 than
  // two calls and the subtraction pass (4096^2, u8 / u16, us: 3 x 3
  // 37.7 / 41.4 against 46.1 / 55.3, 5 x 5 42.3 / 46.2 against 50.8 /
  // 57.2).  Its 16-bit-lane passes issue more instructions per pixel than
  // the tile kernel's, so openings and closings (four passes) and larger
  // windows measured slower than two calls (u8 3 x 3 opening 49.6 against
  // 41.4 us).
  const int cm = tuning().comp_mode;
  if (cm != 0 && comp_fits(width, height, wx, wy) &&
      (cm == 1 || (kind == MORPH_GRADIENT && wx <= 5 && wy <= 5)))
    return comp_launch(src, static_cast<long long>(src_pitch), dst, static_cast<long long>(dst_pitch), width, height,
                       esz, kind, wx, wy, anchor_x, anchor_y, tuning().pdl_mode == 1, st) == cudaSuccess
               ? MORPH_OK
               : MORPH_ERR_CUDA;
  // the intermediate (opening, closing) or the erosion (gradient), ordered
  // on the caller's stream and freed there
  Scratch t;
  if (!t.alloc(static_cast<size_t>(width) * esz, height, st)) return MORPH_ERR_NOMEM;
  const int rx = wx - 1 - anchor_x, ry = wy - 1 - anchor_y;  // the reflected element's anchor
  if (kind == MORPH_GRADIENT) {
    // The subtraction is an elementwise pass after the dilation.  Folding
    // it into the store of the dilation's pass along y (each output minus
    // the erosion's pixel, read from global memory there) was measured
    // 1.2-4x slower on the GB300 than this pass: each row's stores then
    // wait on a global load inside the scan.
    rc = run_single(src, src_pitch, t.p, t.pitch, width, height, dtype, MORPH_ERODE, wx, wy, anchor_x, anchor_y, st);
    if (rc == MORPH_OK)
      rc = run_single(src, src_pitch, dst, dst_pitch, width, height, dtype, MORPH_DILATE, wx, wy, anchor_x, anchor_y,
                      st);
    if (rc == MORPH_OK &&
        sub_launch(dst, static_cast<long long>(dst_pitch), t.p, static_cast<long long>(t.pitch), width * esz, height,
                   esz, st) != cudaSuccess)
      rc = MORPH_ERR_CUDA;
    return rc;
  }
  const int first = kind == MORPH_OPEN ? MORPH_ERODE : MORPH_DILATE;
  const int second = kind == MORPH_OPEN ? MORPH_DILATE : MORPH_ERODE;
  rc = run_single(src, src_pitch, t.p, t.pitch, width, height, dtype, first, wx, wy, anchor_x, anchor_y, st);
  if (rc == MORPH_OK) rc = run_single(t.p, t.pitch, dst, dst_pitch, width, height, dtype, second, wx, wy, rx, ry, st);
  return rc;
}

int morph_copy_2d(void* dst, size_t dst_pitch, const void* src, size_t src_pitch, size_t width_bytes, int height,
                  void* stream) {
  if (!dst || !src) return MORPH_ERR_NULL;
  if (height < 1) return MORPH_ERR_SIZE;
  if (dst_pitch < width_bytes || src_pitch < width_bytes) return MORPH_ERR_PITCH;
  if (width_bytes == 0) return MORPH_OK;
  return cudaMemcpy2DAsync(dst, dst_pitch, src, src_pitch, width_bytes, static_cast<size_t>(height), cudaMemcpyDefault,
                           static_cast<cudaStream_t>(stream)) == cudaSuccess
             ? MORPH_OK
             : MORPH_ERR_CUDA;
}

int morph_copy_batch(const morph_copy_desc* copies, int n, void* stream) {
  if (n < 0) return MORPH_ERR_ARG;
  if (n > 0 && !copies) return MORPH_ERR_NULL;
  for (int i = 0; i < n; ++i)
    if (copies[i].bytes && (!copies[i].dst || !copies[i].src)) return MORPH_ERR_NULL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  for (int i = 0; i < n; ++i) {
    if (!copies[i].bytes) continue;
    if (cudaMemcpyAsync(copies[i].dst, copies[i].src, static_cast<size_t>(copies[i].bytes), cudaMemcpyDefault, st) !=
        cudaSuccess)
      return MORPH_ERR_CUDA;
  }
  return MORPH_OK;
}

int morph_selftest_wait_timeout(void* stream) {
  return selftest_wait_timeout(static_cast<cudaStream_t>(stream)) == cudaSuccess ? MORPH_OK : MORPH_ERR_CUDA;
}

int morph_erode(const uint8_t* src, int width, int height, size_t pitch, int wx, int wy, int anchor_x,
                int anchor_y, uint8_t* dst, void* stream) {
  return morph_apply(src, pitch, dst, pitch, width, height, MORPH_U8, MORPH_ERODE, wx, wy, anchor_x, anchor_y,
                     stream);
}

int morph_dilate(const uint8_t* src, int width, int height, size_t pitch, int wx, int wy, int anchor_x,
                 int anchor_y, uint8_t* dst, void* stream) {
  return morph_apply(src, pitch, dst, pitch, width, height, MORPH_U8, MORPH_DILATE, wx, wy, anchor_x,
                     anchor_y, stream);
}

int morph_erode_u16(const uint16_t* src, int width, int height, size_t pitch, int wx, int wy, int anchor_x,
                    int anchor_y, uint16_t* dst, void* stream) {
  return morph_apply(src, pitch, dst, pitch, width, height, MORPH_U16, MORPH_ERODE, wx, wy, anchor_x,
                     anchor_y, stream);
}

int morph_dilate_u16(const uint16_t* src, int width, int height, size_t pitch, int wx, int wy, int anchor_x,
                     int anchor_y, uint16_t* dst, void* stream) {
  return morph_apply(src, pitch, dst, pitch, width, height, MORPH_U16, MORPH_DILATE, wx, wy, anchor_x,
                     anchor_y, stream);
}

static int transpose_any(const void* src, int width, int height, size_t src_pitch, void* dst, size_t dst_pitch,
                         int esz, void* stream) {
  if (!src || !dst) return MORPH_ERR_NULL;
  if (width < 1 || height < 1 || width > (1 << 30) || height > (1 << 30)) return MORPH_ERR_SIZE;
  if (src_pitch < static_cast<size_t>(width) * esz || dst_pitch < static_cast<size_t>(height) * esz)
    return MORPH_ERR_PITCH;
  if (esz == 2 &&
      ((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst) | src_pitch | dst_pitch) & 1))
    return MORPH_ERR_PITCH;
  // source: height rows; destination: width rows of height pixels
  const uintptr_t s0 = reinterpret_cast<uintptr_t>(src), d0 = reinterpret_cast<uintptr_t>(dst);
  const uintptr_t s1 = s0 + static_cast<uintptr_t>(height - 1) * src_pitch + static_cast<uintptr_t>(width) * esz;
  const uintptr_t d1 = d0 + static_cast<uintptr_t>(width - 1) * dst_pitch + static_cast<uintptr_t>(height) * esz;
  if (s0 < d1 && d0 < s1) return MORPH_ERR_ALIAS;
  return transpose_launch(src, static_cast<long long>(src_pitch), dst, static_cast<long long>(dst_pitch), width,
                          height, esz, static_cast<cudaStream_t>(stream)) == cudaSuccess
             ? MORPH_OK
             : MORPH_ERR_CUDA;
}

int transpose_u8(const uint8_t* src, int width, int height, size_t src_pitch, uint8_t* dst, size_t dst_pitch,
                 void* stream) {
  return transpose_any(src, width, height, src_pitch, dst, dst_pitch, 1, stream);
}

int transpose_u16(const uint16_t* src, int width, int height, size_t src_pitch, uint16_t* dst, size_t dst_pitch,
                  void* stream) {
  return transpose_any(src, width, height, src_pitch, dst, dst_pitch, 2, stream);
}

int morph_batch(const morph_desc* descs_host, int n, void* stream) {
  std::vector<BatchImageIn> in;
  int rc = plan_batch(descs_host, n, &in);
  if (rc != MORPH_OK) return rc;
  std::vector<int> alone;
  split_alone(descs_host, &in, &alone);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (!in.empty()) {
    BatchHost h;
    if (batch_prepare(in.data(), static_cast<int>(in.size()), &h) != 0) return MORPH_ERR_WINDOW;
    if (batch_configure(&h) != cudaSuccess) return MORPH_ERR_CUDA;
    const BatchDev L = batch_dev_layout(h);
    // Stream-ordered scratch from the library's pool (records, then the 2-D
    // images' intermediates): allocated and freed in the stream's order, so
    // concurrent batches on different streams never share it.
    void* dmem = nullptr;
    if (scratch_malloc(&dmem, L.bytes, st) != cudaSuccess) return MORPH_ERR_NOMEM;
    uint8_t* base = static_cast<uint8_t*>(dmem);
    batch_bind_intermediates(base + L.inter_off, &h);
    cudaError_t e = upload_batch(h, L, base, st);
    if (e == cudaSuccess) e = batch_enqueue(h, base, L, st);
    cudaFreeAsync(dmem, st);
    if (e != cudaSuccess) return MORPH_ERR_CUDA;
  }
  return run_alone(descs_host, alone, st);
}

int morph_batch_plan_create(const morph_desc* descs_host, int n, void** plan) {
  if (!plan) return MORPH_ERR_NULL;
  *plan = nullptr;
  std::vector<BatchImageIn> in;
  int rc = plan_batch(descs_host, n, &in);
  if (rc != MORPH_OK) return rc;
  std::vector<int> alone;
  split_alone(descs_host, &in, &alone);
  BatchPlan* p = new BatchPlan();
  cudaGetDevice(&p->device);
  if (batch_prepare(in.data(), static_cast<int>(in.size()), &p->host) != 0) {
    delete p;
    return MORPH_ERR_WINDOW;
  }
  if (batch_configure(&p->host) != cudaSuccess) {
    delete p;
    return MORPH_ERR_CUDA;
  }
  const BatchDev L = batch_dev_layout(p->host);
  if (cudaMalloc(&p->dmem, L.bytes) != cudaSuccess) {
    delete p;
    return MORPH_ERR_NOMEM;
  }
  uint8_t* base = static_cast<uint8_t*>(p->dmem);
  batch_bind_intermediates(base + L.inter_off, &p->host);
  // Records at fixed addresses, then the launches captured into a graph.
  cudaStream_t cs = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = upload_batch(p->host, L, base, cs);
  if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
  if (e == cudaSuccess) e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    // the large images' single calls join the graph (their scratch images
    // become allocation nodes of it)
    cudaError_t le = batch_enqueue(p->host, base, L, cs);
    int arc = MORPH_OK;
    if (le == cudaSuccess) arc = run_alone(descs_host, alone, cs);
    e = cudaStreamEndCapture(cs, &p->graph);
    if (le != cudaSuccess) e = le;
    else if (arc != MORPH_OK && e == cudaSuccess) e = cudaErrorUnknown;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&p->exec, p->graph, 0);
  if (cs) cudaStreamDestroy(cs);
  if (e != cudaSuccess) {
    morph_batch_plan_destroy(p);
    return MORPH_ERR_CUDA;
  }
  *plan = p;
  return MORPH_OK;
}

int morph_batch_plan_launch(void* plan, void* stream) {
  if (!plan) return MORPH_ERR_NULL;
  BatchPlan* p = static_cast<BatchPlan*>(plan);
  return cudaGraphLaunch(p->exec, static_cast<cudaStream_t>(stream)) == cudaSuccess ? MORPH_OK : MORPH_ERR_CUDA;
}

int morph_batch_plan_destroy(void* plan) {
  if (!plan) return MORPH_ERR_NULL;
  BatchPlan* p = static_cast<BatchPlan*>(plan);
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(p->device);
  if (p->exec) cudaGraphExecDestroy(p->exec);
  if (p->graph) cudaGraphDestroy(p->graph);
  if (p->dmem) cudaFree(p->dmem);
  cudaSetDevice(cur);
  delete p;
  return MORPH_OK;
}

int morph_set_tuning(int dtype, int cross_row, int cross_col, int tile_cfg) {
  const int esz = esz_of(dtype);
  if (!esz) return MORPH_ERR_DTYPE;
  if (tile_cfg < -1 || tile_cfg >= kNumTileCfg) return MORPH_ERR_ARG;
  Tuning& t = tuning();
  if (cross_row >= 0) t.cross_row[esz - 1] = cross_row;
  if (cross_col >= 0) t.cross_col[esz - 1] = cross_col;
  if (tile_cfg >= -1) t.forced_cfg[esz - 1] = tile_cfg;
  return MORPH_OK;
}

int morph_set_split_order(int order) {
  if (order < 0 || order > 1) return MORPH_ERR_ARG;
  tuning().split_order = order;
  return MORPH_OK;
}

int morph_set_pdl(int on) {
  if (on < 0 || on > 1) return MORPH_ERR_ARG;
  tuning().pdl_mode = on;
  return MORPH_OK;
}

int morph_set_split(int mode) {
  if (mode < -1 || mode > 1) return MORPH_ERR_ARG;
  tuning().split_mode = mode;
  return MORPH_OK;
}

int morph_set_composite_kernel(int mode) {
  if (mode < -1 || mode > 1) return MORPH_ERR_ARG;
  tuning().comp_mode = mode;
  return MORPH_OK;
}

int morph_set_batch_alone(long long min_pixels) {
  tuning().batch_alone = min_pixels < 0 ? kBatchAlonePixels : min_pixels;
  return MORPH_OK;
}

int morph_set_xpass(int dtype, int mode) {
  const int esz = esz_of(dtype);
  if (!esz) return MORPH_ERR_DTYPE;
  if (mode < 0 || mode > 1) return MORPH_ERR_ARG;
  tuning().xpass_transpose[esz - 1] = mode;
  return MORPH_OK;
}

int morph_set_column_kernel(int mode) {
  if (mode < -1 || mode > 1) return MORPH_ERR_ARG;
  tuning().col_mode = mode;
  return MORPH_OK;
}

int morph_set_row_kernel(int mode) {
  if (mode < -1 || mode > 1) return MORPH_ERR_ARG;
  tuning().row_mode = mode;
  return MORPH_OK;
}

int morph_set_colv(int mode, int rows, int lane_bytes) {
  if (mode < -1 || mode > 1 || rows < 0 || rows > 1024 ||
      (lane_bytes != 0 && lane_bytes != 4 && lane_bytes != 8))
    return MORPH_ERR_ARG;
  tuning().colv_mode = mode;
  tuning().colv_rows = rows;
  tuning().colv_lb = lane_bytes;
  return MORPH_OK;
}

int morph_set_rowv(int mode, int seg) {
  if (mode < -1 || mode > 4 || seg < 0 || seg > (1 << 20)) return MORPH_ERR_ARG;
  tuning().rowv_mode = mode;
  tuning().rowv_seg = seg;
  return MORPH_OK;
}

int morph_set_pipeline(int mode) {
  if (mode < -1 || mode > 1) return MORPH_ERR_ARG;
  tuning().pipe_mode = mode;
  return MORPH_OK;
}

int morph_reset_tuning(void) {
  reset_tuning_defaults();
  return MORPH_OK;
}

int morph_apply_host(const void* src, size_t src_pitch, void* dst, size_t dst_pitch, int width, int height,
                     int dtype, int op, int wx, int wy, int anchor_x, int anchor_y, void* stream) {
  // Host buffers may overlap-check like device ones; the staging copies do not.
  int rc = validate(src, src_pitch, dst, dst_pitch, width, height, dtype, op, wx, wy, anchor_x, anchor_y);
  if (rc != MORPH_OK) return rc;
  const int esz = esz_of(dtype);
  const size_t row = static_cast<size_t>(width) * esz;
  const size_t pitch = (row + 15) / 16 * 16;  // 16-byte rows: the TMA path
  void *din = nullptr, *dout = nullptr;
  rc = stage_buffers(pitch * static_cast<size_t>(height), &din, &dout);
  if (rc != MORPH_OK) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (cudaMemcpy2DAsync(din, pitch, src, src_pitch, row, height, cudaMemcpyHostToDevice, st) != cudaSuccess)
    return MORPH_ERR_CUDA;
  rc = run_single(din, pitch, dout, pitch, width, height, dtype, op, wx, wy, anchor_x, anchor_y, st);
  if (rc != MORPH_OK) return rc;
  if (cudaMemcpy2DAsync(dst, dst_pitch, dout, pitch, row, height, cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return MORPH_ERR_CUDA;
  return cudaStreamSynchronize(st) == cudaSuccess ? MORPH_OK : MORPH_ERR_CUDA;
}

int morph_apply_host_batch(const morph_desc* descs, int n, void* stream) {
  if (!descs) return MORPH_ERR_NULL;
  if (n < 1) return MORPH_ERR_ARG;
  size_t most = 0;  // largest staging image (16-byte rows)
  for (int i = 0; i < n; ++i) {
    const morph_desc& d = descs[i];
    const int rc = validate(d.src, static_cast<size_t>(d.src_pitch), d.dst, static_cast<size_t>(d.dst_pitch),
                            d.width, d.height, d.dtype, d.op, d.wx, d.wy, d.anchor_x, d.anchor_y);
    if (rc != MORPH_OK) return rc;
    const size_t pitch = (static_cast<size_t>(d.width) * esz_of(d.dtype) + 15) / 16 * 16;
    most = std::max(most, pitch * static_cast<size_t>(d.height));
  }
  Pipeline* pl = nullptr;
  int rc = pipeline_for_current_device(most, &pl);
  if (rc != MORPH_OK) return rc;
  std::lock_guard<std::mutex> lock(pl->mu);
  cudaStream_t caller = static_cast<cudaStream_t>(stream);
  // the pipeline's streams start after work already queued on the caller's
  if (cudaEventRecord(pl->start, caller) != cudaSuccess) return MORPH_ERR_CUDA;
  for (int k = 0; k < 3; ++k)
    if (cudaStreamWaitEvent(pl->st[k], pl->start, 0) != cudaSuccess) return MORPH_ERR_CUDA;
  for (int i = 0; i < n && rc == MORPH_OK; ++i) {
    const morph_desc& d = descs[i];
    const int slot = i % kPipeSlots;
    const size_t row = static_cast<size_t>(d.width) * esz_of(d.dtype);
    const size_t pitch = (row + 15) / 16 * 16;
    // copy in once the slot's previous image has been copied out
    if (i >= kPipeSlots && cudaStreamWaitEvent(pl->st[0], pl->out_done[slot], 0) != cudaSuccess) rc = MORPH_ERR_CUDA;
    if (rc == MORPH_OK && cudaMemcpy2DAsync(pl->in[slot], pitch, d.src, static_cast<size_t>(d.src_pitch), row,
                                            d.height, cudaMemcpyHostToDevice, pl->st[0]) != cudaSuccess)
      rc = MORPH_ERR_CUDA;
    if (rc == MORPH_OK && cudaEventRecord(pl->in_done[slot], pl->st[0]) != cudaSuccess) rc = MORPH_ERR_CUDA;
    // filter once it is in (and once the slot's previous output is out)
    if (rc == MORPH_OK && cudaStreamWaitEvent(pl->st[1], pl->in_done[slot], 0) != cudaSuccess) rc = MORPH_ERR_CUDA;
    if (rc == MORPH_OK && i >= kPipeSlots && cudaStreamWaitEvent(pl->st[1], pl->out_done[slot], 0) != cudaSuccess)
      rc = MORPH_ERR_CUDA;
    if (rc == MORPH_OK)
      rc = run_single(pl->in[slot], pitch, pl->out[slot], pitch, d.width, d.height, d.dtype, d.op, d.wx, d.wy,
                      d.anchor_x, d.anchor_y, pl->st[1]);
    if (rc == MORPH_OK && cudaEventRecord(pl->comp_done[slot], pl->st[1]) != cudaSuccess) rc = MORPH_ERR_CUDA;
    // copy out once it is filtered
    if (rc == MORPH_OK && cudaStreamWaitEvent(pl->st[2], pl->comp_done[slot], 0) != cudaSuccess) rc = MORPH_ERR_CUDA;
    if (rc == MORPH_OK && cudaMemcpy2DAsync(d.dst, static_cast<size_t>(d.dst_pitch), pl->out[slot], pitch, row,
                                            d.height, cudaMemcpyDeviceToHost, pl->st[2]) != cudaSuccess)
      rc = MORPH_ERR_CUDA;
    if (rc == MORPH_OK && cudaEventRecord(pl->out_done[slot], pl->st[2]) != cudaSuccess) rc = MORPH_ERR_CUDA;
  }
  // everything queued so far must finish before the call returns, errors or not
  for (int k = 0; k < 3; ++k) cudaStreamSynchronize(pl->st[k]);
  if (rc != MORPH_OK) return rc;
  return cudaStreamSynchronize(caller) == cudaSuccess ? MORPH_OK : MORPH_ERR_CUDA;
}

int morph_release_staging(void) {
  release_pipelines();
  {
    // unused pool memory back to the driver (blocks still in use stay)
    std::lock_guard<std::mutex> lock(g_pool_mu);
    for (int d = 0; d < kMaxDevices; ++d)
      if (g_pool[d]) cudaMemPoolTrimTo(g_pool[d], 0);
  }
  std::lock_guard<std::mutex> lock(g_staging_mu);
  int cur = 0;
  cudaGetDevice(&cur);
  for (int d = 0; d < kMaxDevices; ++d) {
    Staging& s = g_staging[d];
    if (!s.in && !s.out) continue;
    cudaSetDevice(d);
    if (s.in) cudaFree(s.in);
    if (s.out) cudaFree(s.out);
    s = Staging();
  }
  cudaSetDevice(cur);
  return MORPH_OK;
}

const char* morph_status_string(int status) {
  switch (status) {
    case MORPH_OK: return "ok";
    case MORPH_ERR_NULL: return "null pointer";
    case MORPH_ERR_SIZE: return "invalid image size";
    case MORPH_ERR_WINDOW: return "invalid or unsupported window size";
    case MORPH_ERR_ANCHOR: return "anchor outside the window";
    case MORPH_ERR_PITCH: return "pitch smaller than a row";
    case MORPH_ERR_ALIAS: return "source and destination overlap";
    case MORPH_ERR_CUDA: return "CUDA error";
    case MORPH_ERR_NOMEM: return "out of memory";
    case MORPH_ERR_DTYPE: return "unknown dtype or op";
    case MORPH_ERR_ARG: return "invalid argument";
    case MORPH_ERR_DEVICE: return "device-side error reported by a kernel";
    case MORPH_ERR_LIMIT: return "more images than the no-allocation entry point accepts";
  }
  return "unknown status";
}

long long morph_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

int morph_device_error(void) {
  if (cudaDeviceSynchronize() != cudaSuccess) return MORPH_ERR_CUDA;
  const int a = fused_take_device_error();
  const int b = batch_take_device_error();
  return a ? a : b;
}

}  // extern "C"
