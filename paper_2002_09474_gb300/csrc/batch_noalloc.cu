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

// Host-side working storage of one call (shared by all calls).  The staged
// records are page-locked once per process (cudaHostRegister pins memory the
// library already has; it allocates none), so their copy to the device is
// truly asynchronous; a call waits, before overwriting them, for the copy of
// the previous call to have run (g_stage_done).
alignas(4096) NoallocScratch g_stage;
BatchImageIn g_in[kMaxImages];
const FusedLaunch* g_lp[kMaxImages];
BatchRange g_ranges[2 * kMaxImages];
bool g_stage_pinned = false;
cudaEvent_t g_stage_done[64] = {};
int g_stage_dev = -1;  // device of the last call's copy (its event)

// Device address of g_noalloc_scratch per device, looked up once per device
// with that device current; the staging copy is page-locked on the first
// call, and each device's event created on its first call.
void* g_scratch_ptr[64] = {};
std::mutex g_setup_mu;

void* scratch_for_current_device(int* dev_out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lock(g_setup_mu);
  if (!g_scratch_ptr[dev]) {
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess) return nullptr;
    if (cudaEventCreateWithFlags(&g_stage_done[dev], cudaEventDisableTiming) != cudaSuccess) return nullptr;
    g_scratch_ptr[dev] = ptr;
  }
  if (!g_stage_pinned) {
    // a failure leaves the staging pageable: the copy then waits for the
    // stream's earlier work, but the results are the same
    g_stage_pinned = cudaHostRegister(&g_stage, sizeof(g_stage), cudaHostRegisterDefault) == cudaSuccess;
    if (!g_stage_pinned) cudaGetLastError();
  }
  *dev_out = dev;
  return g_scratch_ptr[dev];
}

}  // namespace
}  // namespace morph

using namespace morph;

extern "C" int morph_batch_noalloc(const morph_desc* descs_host, int n, void* stream) {
  if (!descs_host) return MORPH_ERR_NULL;
  if (n < 1) return MORPH_ERR_ARG;
  if (n > kMaxImages) return MORPH_ERR_LIMIT;
  int dev = 0;
  uint8_t* scratch = static_cast<uint8_t*>(scratch_for_current_device(&dev));
  if (!scratch) return MORPH_ERR_CUDA;
  // the same checks and plan as morph_batch, into the fixed arrays
  int rc = plan_batch_into(descs_host, n, g_in, g_ranges);
  if (rc != MORPH_OK) return rc;
  // the previous call's copy of g_stage must have run before it is rewritten
  if (g_stage_dev >= 0 && cudaEventSynchronize(g_stage_done[g_stage_dev]) != cudaSuccess) return MORPH_ERR_CUDA;
  // every image in the fused persistent kernel (no intermediate images: the
  // single-pass kernels' two-launch form would need scratch of image size)
  for (int i = 0; i < n; ++i) g_lp[i] = &g_in[i].L;
  int cfg = -1, smem = 0, tiles = 0;
  if (batch_prepare_fused(g_lp, n, &cfg, &smem, &tiles, g_stage.imgs, g_stage.maps) != 0) return MORPH_ERR_WINDOW;
  int grid = 0;
  int* err = nullptr;
  if (batch_fused_grid(cfg, smem, tiles, &grid, &err) != cudaSuccess) return MORPH_ERR_CUDA;
  NoallocScratch* d = reinterpret_cast<NoallocScratch*>(scratch);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemcpyAsync(d->maps, g_stage.maps, sizeof(CUtensorMap) * 2 * n, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d->imgs, g_stage.imgs, sizeof(BatchImage) * n, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaEventRecord(g_stage_done[dev], st);
  if (e == cudaSuccess) g_stage_dev = dev;
  if (e == cudaSuccess) e = batch_enqueue_raw(cfg, smem, grid, err, n, tiles, d->imgs, d->maps, &d->counter, st);
  return e == cudaSuccess ? MORPH_OK : MORPH_ERR_CUDA;
}
