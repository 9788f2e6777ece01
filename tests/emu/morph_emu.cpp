// CPU emulator of the fused erosion/dilation tile kernel -- TEST
// INFRASTRUCTURE ONLY.
//
// Compiles the kernel's own tile code (paper_2002_09474_gb300/csrc/
// morph_tile.cuh) for the host with MORPH_HOST_EMU set, runs every CTA as
// kThreads std::threads meeting at a real barrier for __syncthreads, and
// models the TMA unit and the mbarrier transaction count in software.  Built
// with AddressSanitizer, so any shared-memory access outside a CTA's exact
// dynamic allocation and any global access outside the image buffers stops
// the run.  It also checks the rules the hardware does not check for us:
// TMA coordinates 16-byte aligned, no store box starting outside the tensor,
// boxes no larger than the tensor, transfer counts that match the expected
// bytes.  On half of the cases (by seed) a TMA load lands only when a thread
// waits on its mbarrier for the phase it completes, so a missing or
// wrong-phase wait reads stale shared memory, and loads still in flight when
// a CTA ends are an error; on the other half loads land when issued, so a
// buffer refilled before its last read shows up.  Results are compared with
// the brute-force oracle.
//
// Input, one case per line on stdin:
//   esz op W H spad soff dpad doff wx wy ax ay cfg cross_x cross_y seed kern
// (pads/offsets in bytes; cfg -1 = the planner's choice; kern 0 = one CTA
// per tile, 1 = the persistent two-slot kernel with 3 CTAs when the input is
// TMA-loadable, 2 = the column kernel for 1 x wy windows, its tile height
// planned for 152 SMs on odd seeds and 3 SMs on even ones, 3 = the row
// kernel for wx x 1 windows, 4 = the warp-tiled van Herk/Gil-Werman kernel
// of the pass along y for 1 x wy windows, its tile height planned for 152
// SMs on odd seeds and 3 SMs on even ones, 5 = the register-blocked van
// Herk/Gil-Werman kernel of the pass along x for wx x 1 windows, when the
// source rows allow it, its segment planned for 152 SMs on odd seeds and 3
// SMs on even ones; the warp-tiled kernel's strip width varies with the
// seed: 4 or 8 bytes per lane; 6 = the one-pass composite, op then being
// the kind: 0 opening, 1 closing, 2 gradient).
// Output: one line per case, "OK ..." or "FAIL ...".
#define MORPH_HOST_EMU 1

#include <atomic>
#include <map>
#include <memory>
#include <mutex>
#include <barrier>
#include <chrono>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include <unistd.h>

#include <cuda.h>
#include <cuda_runtime.h>

// ---- device-language shim (host definitions of what the tile code uses) ----
thread_local uint3 emu_threadIdx;
#define threadIdx emu_threadIdx

struct EmuCta {
  std::barrier<>* bar = nullptr;
  std::barrier<>* wbar[8] = {};  // one per warp (__syncwarp)
  std::atomic<int> orflag{0};
  std::atomic<int> anyfalse[8] = {};  // per warp (__all_sync)
  uint32_t shfl[8][32] = {};           // per warp (__shfl_sync)
  // mbarriers by address: a phase completes when its arrivals are in and
  // its transaction count is back to zero; the phase bit then flips.
  struct Mbar {
    int count = 1, pending = 1;
    long long tx = 0;
    int phase_bit = 0;
  };
  std::mutex mu;
  std::map<const void*, Mbar> mbars;
  // TMA loads not yet landed (deferred mode): each lands when a thread waits
  // on its barrier for the phase it completes
  struct PendingLoad {
    void* dst;
    CUtensorMap map;
    int x, y;
    uint64_t* bar;
  };
  std::vector<PendingLoad> pending;
  const uint8_t* smem = nullptr;
  size_t smem_size = 0;
  std::atomic<int> errors{0};
  std::string first_error;
  std::atomic<int> partial_stores{0};
};
thread_local EmuCta* g_cta = nullptr;
// Deferred mode (chosen per case): a TMA load copies nothing when it is
// issued, only when a thread waits on its mbarrier for the phase it
// completes, so a read that does not wait, or waits for the wrong phase,
// sees stale shared memory; and a CTA that ends with loads in flight is an
// error.  Immediate mode copies at issue, so a buffer refilled before its
// last read shows up instead.
bool g_tma_deferred = false;

static void emu_error(const char* what) {
  if (g_cta->errors.fetch_add(1) == 0) g_cta->first_error = what;
}
// Errors of a CTA that has ended, counting TMA loads still in flight.
static int cta_end_errors(EmuCta& cta) {
  if (!cta.pending.empty()) {
    if (cta.errors.fetch_add(1) == 0) cta.first_error = "TMA loads still in flight when the CTA ended";
  }
  return cta.errors.load();
}

static inline void __syncthreads() { g_cta->bar->arrive_and_wait(); }
static inline void __syncwarp() { g_cta->wbar[threadIdx.x >> 5]->arrive_and_wait(); }
// every lane of the warp takes part (full mask): lane src's v
static inline unsigned int __shfl_sync(unsigned, unsigned int v, int src) {
  uint32_t* x = g_cta->shfl[threadIdx.x >> 5];
  x[threadIdx.x & 31] = v;
  __syncwarp();
  const unsigned int r = x[src & 31];
  __syncwarp();
  return r;
}
// every lane of the warp takes part (full mask): true when no lane's p is false
static inline bool __all_sync(unsigned, bool p) {
  std::atomic<int>& f = g_cta->anyfalse[threadIdx.x >> 5];
  if (!p) f.store(1);
  __syncwarp();
  const bool r = f.load() == 0;
  __syncwarp();
  if ((threadIdx.x & 31) == 0) f.store(0);
  __syncwarp();
  return r;
}
static inline int __syncthreads_or(int p) {
  if (p) g_cta->orflag.store(1);
  g_cta->bar->arrive_and_wait();
  const int r = g_cta->orflag.load();
  g_cta->bar->arrive_and_wait();
  if (threadIdx.x == 0) g_cta->orflag.store(0);
  g_cta->bar->arrive_and_wait();
  return r;
}
static inline unsigned int __vminu2(unsigned int a, unsigned int b) {
  const unsigned lo = (a & 0xFFFFu) < (b & 0xFFFFu) ? (a & 0xFFFFu) : (b & 0xFFFFu);
  const unsigned hi = (a >> 16) < (b >> 16) ? (a >> 16) : (b >> 16);
  return lo | (hi << 16);
}
static inline unsigned int __vmaxu2(unsigned int a, unsigned int b) {
  const unsigned lo = (a & 0xFFFFu) > (b & 0xFFFFu) ? (a & 0xFFFFu) : (b & 0xFFFFu);
  const unsigned hi = (a >> 16) > (b >> 16) ? (a >> 16) : (b >> 16);
  return lo | (hi << 16);
}
// Per-lane subtraction of two 16-bit lanes, modulo 2^16 in each lane.
static inline unsigned int __vsub2(unsigned int a, unsigned int b) {
  const unsigned lo = ((a & 0xFFFFu) - (b & 0xFFFFu)) & 0xFFFFu;
  const unsigned hi = ((a >> 16) - (b >> 16)) & 0xFFFFu;
  return lo | (hi << 16);
}
// Byte selection from the 8-byte value {y, x}: result byte i is byte
// (s >> 4i) & 7 (bit 3 of each selector nibble replicates that byte's sign).
static inline unsigned int __byte_perm(unsigned int x, unsigned int y, unsigned int s) {
  const uint64_t v = (static_cast<uint64_t>(y) << 32) | x;
  unsigned int r = 0;
  for (int i = 0; i < 4; ++i) {
    const unsigned sel = (s >> (4 * i)) & 0xF;
    unsigned byte = static_cast<unsigned>(v >> (8 * (sel & 7))) & 0xFFu;
    if (sel & 8) byte = (byte & 0x80u) ? 0xFFu : 0u;
    r |= byte << (8 * i);
  }
  return r;
}
template <typename T>
static inline T __ldg(const T* p) {
  return *p;
}
static inline int atomicExch(int* p, int v) { return __atomic_exchange_n(p, v, __ATOMIC_SEQ_CST); }
static inline unsigned int __funnelshift_r(unsigned int lo, unsigned int hi, unsigned int s) {
  const uint64_t v = (static_cast<uint64_t>(hi) << 32) | lo;
  return static_cast<unsigned int>(v >> (s & 31));
}

#include "morph_tile.cuh"
#include "morph_col.cuh"
#include "morph_row.cuh"
#include "morph_colv.cuh"
#include "morph_rowv.cuh"
#include "morph_comp.cuh"

// ---- TMA / mbarrier model ------------------------------------------------------
struct EmuMap {
  const uint8_t* base;
  uint8_t* wbase;
  int esz, W, H;
  long long pitch;
  int bw, bh;  // box, in elements
};
static_assert(sizeof(EmuMap) <= sizeof(CUtensorMap), "map too large");

static void check_smem(const void* p, size_t bytes, size_t align, const char* what) {
  const uint8_t* b = static_cast<const uint8_t*>(p);
  if (b < g_cta->smem || b + bytes > g_cta->smem + g_cta->smem_size) emu_error(what);
  if ((b - g_cta->smem) % align) emu_error("TMA shared-memory address misaligned");
}

namespace morph {
static void mbar_check_complete(EmuCta::Mbar& m) {  // caller holds g_cta->mu
  if (m.pending == 0 && m.tx == 0) {
    m.phase_bit ^= 1;
    m.pending = m.count;
  }
}
void mbar_init(uint64_t* bar, uint32_t count) {
  std::lock_guard<std::mutex> l(g_cta->mu);
  EmuCta::Mbar& m = g_cta->mbars[bar];
  m.count = m.pending = static_cast<int>(count);
  m.tx = 0;
  m.phase_bit = 0;
}
void fence_barrier_init() {}
void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  std::lock_guard<std::mutex> l(g_cta->mu);
  auto it = g_cta->mbars.find(bar);
  if (it == g_cta->mbars.end()) {
    emu_error("arrive on an uninitialised mbarrier");
    return;
  }
  it->second.tx += bytes;
  it->second.pending -= 1;
  mbar_check_complete(it->second);
}
static void land_tma_load(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y);  // holds g_cta->mu
bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  std::lock_guard<std::mutex> l(g_cta->mu);
  auto it = g_cta->mbars.find(bar);
  if (it == g_cta->mbars.end()) {
    emu_error("wait on an uninitialised mbarrier");
    return true;
  }
  if (it->second.phase_bit == static_cast<int>(parity)) {  // the phase waited for: its loads land now
    std::vector<EmuCta::PendingLoad> keep;
    std::vector<EmuCta::PendingLoad> land;
    for (auto& p : g_cta->pending) (p.bar == bar ? land : keep).push_back(p);
    g_cta->pending.swap(keep);
    for (auto& p : land) land_tma_load(p.dst, &p.map, p.bar, p.x, p.y);
  }
  return it->second.phase_bit != static_cast<int>(parity);
}
bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
  const auto t0 = std::chrono::steady_clock::now();
  while (!mbar_try_wait(bar, parity)) {
    if (std::chrono::steady_clock::now() - t0 > std::chrono::seconds(5)) {
      std::lock_guard<std::mutex> l(g_cta->mu);
      emu_error(g_cta->mbars[bar].tx < 0 ? "TMA delivered more bytes than expected"
                                         : "TMA transfer count never reached the expected bytes (the wait times out)");
      return false;
    }
    std::this_thread::yield();
  }
  return true;
}
void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
  const EmuMap* m = reinterpret_cast<const EmuMap*>(map);
  if ((static_cast<long long>(x) * m->esz) % 16) emu_error("TMA load x not 16-byte aligned");
  if (m->bw > m->W || m->bh > m->H) emu_error("TMA box larger than the tensor");
  const size_t row = static_cast<size_t>(m->bw) * m->esz;
  check_smem(dst, row * m->bh, 128, "TMA load box outside shared memory");
  std::lock_guard<std::mutex> l(g_cta->mu);
  if (g_tma_deferred) {
    EmuCta::PendingLoad p{dst, {}, x, y, bar};
    memcpy(&p.map, map, sizeof(CUtensorMap));
    g_cta->pending.push_back(p);
    return;
  }
  land_tma_load(dst, map, bar, x, y);
}
static void land_tma_load(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
  const EmuMap* m = reinterpret_cast<const EmuMap*>(map);
  const size_t row = static_cast<size_t>(m->bw) * m->esz;
  uint8_t* d = static_cast<uint8_t*>(dst);
  for (int r = 0; r < m->bh; ++r)
    for (int c = 0; c < m->bw; ++c) {
      const int gx = x + c, gy = y + r;
      for (int b = 0; b < m->esz; ++b) {
        uint8_t v = 0;
        if (gx >= 0 && gx < m->W && gy >= 0 && gy < m->H) v = m->base[gy * m->pitch + gx * m->esz + b];
        d[r * row + c * m->esz + b] = v;
      }
    }
  EmuCta::Mbar& mb = g_cta->mbars[bar];
  mb.tx -= static_cast<long long>(row) * m->bh;
  mbar_check_complete(mb);
}
void fence_proxy_async_smem() {}
void prefetch_tensormap(const CUtensorMap*) {}
void tma_store_2d(const CUtensorMap* map, const void* src, int x, int y) {
  const EmuMap* m = reinterpret_cast<const EmuMap*>(map);
  if (x < 0 || y < 0) emu_error("TMA store starts at a negative coordinate");
  if (x >= m->W || y >= m->H) emu_error("TMA store starts outside the tensor");
  if ((static_cast<long long>(x) * m->esz) % 16) emu_error("TMA store x not 16-byte aligned");
  if (m->bw > m->W || m->bh > m->H) emu_error("TMA store box larger than the tensor");
  if (x + m->bw > m->W || y + m->bh > m->H) g_cta->partial_stores++;
  const size_t row = static_cast<size_t>(m->bw) * m->esz;
  check_smem(src, row * m->bh, 128, "TMA store box outside shared memory");
  const uint8_t* s = static_cast<const uint8_t*>(src);
  for (int r = 0; r < m->bh; ++r)
    for (int c = 0; c < m->bw; ++c) {
      const int gx = x + c, gy = y + r;
      if (gx < m->W && gy < m->H)
        for (int b = 0; b < m->esz; ++b) m->wbase[gy * m->pitch + gx * m->esz + b] = s[r * row + c * m->esz + b];
    }
}
void cp_async8(void* smem, const void* gmem) {
  if (reinterpret_cast<uintptr_t>(gmem) % 8) emu_error("cp.async source not 8-byte aligned");
  check_smem(smem, 8, 8, "cp.async destination outside shared memory");
  memcpy(smem, gmem, 8);
}
void cp_async16(void* smem, const void* gmem) {
  if (reinterpret_cast<uintptr_t>(gmem) % 16) emu_error("cp.async source not 16-byte aligned");
  check_smem(smem, 16, 16, "cp.async destination outside shared memory");
  memcpy(smem, gmem, 16);
}
void cp_async_commit() {}
void bulk_commit() {}
void bulk_wait_read_all() {}
void bulk_wait_all() {}
}  // namespace morph

// ---- host side: planner (linked from plan.cpp) ----------------------------------
#include "morph_internal.h"
#include "plan.h"
namespace morph {
int fused_smem_bytes(const FusedLaunch& L) {
  if (L.cfg < 0 || L.cfg >= kNumTileCfg) return 0;
  return make_geom(L.esz, tile_tx(L.cfg), tile_ty(L.cfg), L.wx, L.wy, L.ax, L.vhgw_col, L.vhgw_row).smem_bytes;
}
int fused_pipe_smem_bytes(const FusedLaunch& L) {
  if (L.cfg < 0 || L.cfg >= kNumTileCfg) return 0;
  return make_geom(L.esz, tile_tx(L.cfg), tile_ty(L.cfg), L.wx, L.wy, L.ax, L.vhgw_col, L.vhgw_row, true)
      .smem_bytes;
}
}  // namespace morph

extern "C" int oracle_morph(const void* src, int esz, int W, int H, long long pitch, int wx, int wy, int ax,
                            int ay, int op, void* dst, long long dpitch);

using namespace morph;

using CtaFn = void (*)(const ImgArgs&, const CUtensorMap*, const CUtensorMap*, int, int, const Geom&, uint4*,
                       uint64_t*, uint32_t&, int*);

template <typename T, int OP, int TX, int TY>
void cta_body(const ImgArgs& a, const CUtensorMap* tin, const CUtensorMap* tout, int x0, int y0, const Geom& g,
              uint4* smem, uint64_t* bar, uint32_t& phase, int* err) {
  run_tile<T, OP, TX, TY>(a, tin, tout, x0, y0, g, smem, bar, phase, err);
}

using PipeFn = void (*)(const ImgArgs&, const CUtensorMap*, const CUtensorMap*, const Geom&, uint4*, uint64_t*,
                       int, int, int, int);

template <typename T, int OP, int TX, int TY>
void pipe_body(const ImgArgs& a, const CUtensorMap* tin, const CUtensorMap* tout, const Geom& g, uint4* smem,
               uint64_t* bar, int ntx, int ntiles, int cta, int ncta) {
  run_tiles_pipelined<T, OP, TX, TY>(a, tin, tout, g, smem, bar, ntx, ntiles, cta, ncta);
}

template <typename T, int OP>
PipeFn pick_pipe(int cfg) {
  switch (cfg) {
    case kTile128x64: return pipe_body<T, OP, 128, 64>;
    case kTile64x64: return pipe_body<T, OP, 64, 64>;
    case kTile64x128: return pipe_body<T, OP, 64, 128>;
    case kTile256x32: return pipe_body<T, OP, 256, 32>;
    case kTile32x32: return pipe_body<T, OP, 32, 32>;
    case kTile128x128: return pipe_body<T, OP, 128, 128>;
    case kTile256x64: return pipe_body<T, OP, 256, 64>;
    case kTile32x128: return pipe_body<T, OP, 32, 128>;
  }
  return nullptr;
}

template <typename T, int OP>
CtaFn pick(int cfg) {
  switch (cfg) {
    case kTile128x64: return cta_body<T, OP, 128, 64>;
    case kTile64x64: return cta_body<T, OP, 64, 64>;
    case kTile64x128: return cta_body<T, OP, 64, 128>;
    case kTile256x32: return cta_body<T, OP, 256, 32>;
    case kTile32x32: return cta_body<T, OP, 32, 32>;
    case kTile128x128: return cta_body<T, OP, 128, 128>;
    case kTile256x64: return cta_body<T, OP, 256, 64>;
    case kTile32x128: return cta_body<T, OP, 32, 128>;
  }
  return nullptr;
}

static void clip_window(int n, int w, int a, int* w_out, int* a_out) {
  const int before = a < n - 1 ? a : n - 1;
  const int after = (w - 1 - a) < n - 1 ? (w - 1 - a) : n - 1;
  *a_out = before;
  *w_out = before + after + 1;
}

// A pool of kThreads workers that run one CTA's body per pool_run call.
#include <functional>
static std::function<void(int)> g_job;
static std::barrier<>* g_start = nullptr;
static std::barrier<>* g_done = nullptr;
static bool g_quit = false;
static int g_active = kThreads;  // threads of the current CTA
static void pool_init() {
  static std::barrier<> start(kColThreads + 1), done(kColThreads + 1);
  g_start = &start;
  g_done = &done;
  for (int t = 0; t < kColThreads; ++t)
    std::thread([t] {
      for (;;) {
        g_start->arrive_and_wait();
        if (g_quit) return;
        if (t < g_active) g_job(t);
        g_done->arrive_and_wait();
      }
    }).detach();
}
static void pool_run(std::function<void(int)> job, int nthreads = kThreads) {
  g_job = std::move(job);
  g_active = nthreads;
  g_start->arrive_and_wait();
  g_done->arrive_and_wait();
}

using ColFnE = bool (*)(const ColArgs&, const CUtensorMap*, int, uint8_t*, uint32_t*, uint64_t*);
template <typename T, int OP>
ColFnE pick_col(bool blk) {
  return blk ? col_tile<T, OP, true> : col_tile<T, OP, false>;
}

using RowFnE = bool (*)(const RowArgs&, const CUtensorMap*, int, const RowGeom&, uint8_t*, uint64_t*, uint32_t&);
template <typename T, int OP>
RowFnE pick_row(bool blk) {
  return blk ? row_tile<T, OP, true> : row_tile<T, OP, false>;
}

static uint64_t splitmix(uint64_t& s) {
  uint64_t z = (s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Planner queries (a line starting with "P"), answered with the default
// tuning, one line each:
//   P split esz W H wx wy      -> split 0|1           (plan_split)
//   P single esz W H wx wy     -> single ok vhgw_col vhgw_row cfg ctas_per_sm
//   P colvrows esz w           -> colvrows L          (built-in tile height)
//   P colv esz W H w lb        -> colv ok L nbox wpc ntask wps   (152 SMs)
//   P rowv W H rr wps          -> rowv ok seg nseg ntask         (152 SMs)
//   P ctas smem_bytes          -> ctas n
static void planner_query(const char* s) {
  char what[32];
  int n = 0;
  if (sscanf(s, "%31s%n", what, &n) != 1) return;
  s += n;
  reset_tuning_defaults();
  if (!strcmp(what, "split") || !strcmp(what, "single")) {
    int esz = 1, W = 1, H = 1, wx = 1, wy = 1;
    sscanf(s, "%d %d %d %d %d", &esz, &W, &H, &wx, &wy);
    FusedLaunch L{};
    L.esz = esz;
    L.W = W;
    L.H = H;
    L.wx = wx;
    L.wy = wy;
    L.ax = wx / 2;
    L.ay = wy / 2;
    if (what[1] == 'p') {
      printf("split %d\n", plan_split(L) ? 1 : 0);
    } else {
      const bool ok = plan_single(&L);
      printf("single %d %d %d %d %d\n", ok ? 1 : 0, L.vhgw_col ? 1 : 0, L.vhgw_row ? 1 : 0, L.cfg,
             ok ? ctas_per_sm(fused_smem_bytes(L)) : 0);
    }
  } else if (!strcmp(what, "colvrows")) {
    int esz = 1, w = 2;
    sscanf(s, "%d %d", &esz, &w);
    printf("colvrows %d\n", colv_default_rows(esz, w));
  } else if (!strcmp(what, "colv")) {
    int esz = 1, W = 1, H = 1, w = 2, lb = 4;
    sscanf(s, "%d %d %d %d %d", &esz, &W, &H, &w, &lb);
    const ColvPlan p = colv_plan(esz, W, H, w, kMaxSmemBytes, 0, lb, 152);
    printf("colv %d %d %d %d %d %d\n", p.ok ? 1 : 0, p.L, p.nbox, p.wpc, p.ntask, p.wps);
  } else if (!strcmp(what, "rowv")) {
    int W = 1, H = 1, rr = 2, wps = 32;
    sscanf(s, "%d %d %d %d", &W, &H, &rr, &wps);
    const RowvPlan p = rowv_plan(W, H, rr, 152, wps, 0);
    printf("rowv %d %d %d %d\n", p.ok ? 1 : 0, p.seg, p.nseg, p.ntask);
  } else if (!strcmp(what, "ctas")) {
    int b = 0;
    sscanf(s, "%d", &b);
    printf("ctas %d\n", ctas_per_sm(b));
  } else {
    printf("unknown %s\n", what);
  }
  fflush(stdout);
}

int main() {
  int esz, op, W, H, spad, soff, dpad, doff, wx, wy, ax, ay, cfg, crx, cry, kern;
  unsigned long long seed;
  int failures = 0, cases = 0;
  pool_init();
  char line[512];
  while (fgets(line, sizeof line, stdin)) {
    if (line[0] == 'P') {
      planner_query(line + 1);
      continue;
    }
    if (sscanf(line, "%d %d %d %d %d %d %d %d %d %d %d %d %d %d %d %llu %d", &esz, &op, &W, &H, &spad, &soff,
               &dpad, &doff, &wx, &wy, &ax, &ay, &cfg, &crx, &cry, &seed, &kern) != 17)
      break;
    const int pipe = kern == 1;
    ++cases;
    g_tma_deferred = (seed >> 2) & 1;
    const long long sp = static_cast<long long>(W) * esz + spad, dp = static_cast<long long>(W) * esz + dpad;
    // Exact-size buffers: ASan flags any byte outside [offset, last pixel].
    const size_t sbytes = soff + (H - 1) * sp + static_cast<size_t>(W) * esz;
    const size_t dbytes = doff + (H - 1) * dp + static_cast<size_t>(W) * esz;
    uint8_t* sbuf = static_cast<uint8_t*>(aligned_alloc(256, (sbytes + 255) / 256 * 256));
    uint8_t* dbuf = static_cast<uint8_t*>(aligned_alloc(256, (dbytes + 255) / 256 * 256));
    // aligned_alloc rounds the size up; poison nothing extra ourselves but
    // check guard bytes below.
    uint64_t st = seed;
    for (size_t i = 0; i < sbytes; ++i) sbuf[i] = static_cast<uint8_t>(splitmix(st));
    memset(dbuf, 0xA5, dbytes);
    const uint8_t* src = sbuf + soff;
    uint8_t* dst = dbuf + doff;

    Tuning& t = tuning();
    reset_tuning_defaults();
    if (crx >= 0) t.cross_row[esz - 1] = crx;
    if (cry >= 0) t.cross_col[esz - 1] = cry;
    t.forced_cfg[esz - 1] = cfg;
    FusedLaunch L{};
    L.esz = esz;
    L.op = op;
    L.src = src;
    L.dst = dst;
    L.sp = sp;
    L.dp = dp;
    L.W = W;
    L.H = H;
    clip_window(W, wx, ax, &L.wx, &L.ax);
    clip_window(H, wy, ay, &L.wy, &L.ay);
    if (!plan_single(&L)) {
      printf("FAIL case %d: no plan\n", cases);
      ++failures;
      continue;
    }
    const int TX = tile_tx(L.cfg), TY = tile_ty(L.cfg);
    const Geom g1 = make_geom(esz, TX, TY, L.wx, L.wy, L.ax, L.vhgw_col, L.vhgw_row);
    const Geom gp = make_geom(esz, TX, TY, L.wx, L.wy, L.ax, L.vhgw_col, L.vhgw_row, true);
    ImgArgs a{};
    a.src = src;
    a.dst = dst;
    a.sp = sp;
    a.dp = dp;
    a.W = W;
    a.H = H;
    a.wx = L.wx;
    a.wy = L.wy;
    a.ax = L.ax;
    a.ay = L.ay;
    a.blk_y = L.vhgw_col && L.wy > 1;
    a.blk_x = L.vhgw_row && L.wx > 1;
    a.ld_vec = (reinterpret_cast<uintptr_t>(src) % 4 == 0) && (sp % 4 == 0);
    a.st_vec = (reinterpret_cast<uintptr_t>(dst) % 4 == 0) && (dp % 4 == 0);
    a.st_vec16 = (reinterpret_cast<uintptr_t>(dst) % 16 == 0) && (dp % 16 == 0);
    int errword = 0;
    a.err = &errword;
    // the launcher's TMA decisions (same rules as encode_tensor_map_2d)
    auto tma_ok = [&](const void* base, long long pitch, int bw, int bh) {
      return !(reinterpret_cast<uintptr_t>(base) & 15) && !(pitch & 15) && bw >= 1 && bw <= 256 && bh >= 1 &&
             bh <= 256 && (bw * esz) % 16 == 0 && bw <= W && bh <= H;
    };
    CUtensorMap tin{}, tout{};
    EmuMap mi{src, nullptr, esz, W, H, sp, g1.box / esz, g1.bh};
    const int sbox = TX * esz < 128 ? TX * esz : 128;
    EmuMap mo{nullptr, dst, esz, W, H, dp, sbox / esz, TY};
    a.tma_ld = tma_ok(src, sp, mi.bw, mi.bh);
    a.tma_st = TX * esz >= 128 && tma_ok(dst, dp, mo.bw, mo.bh);
    memcpy(&tin, &mi, sizeof(mi));
    memcpy(&tout, &mo, sizeof(mo));
    const bool use_col = kern == 2 && L.wx == 1 && L.wy > 1;
    const RowGeom rg = row_geom(esz, L.wx, L.ax);
    const bool use_row = kern == 3 && L.wy == 1 && L.wx > 1 && rg.smem <= kMaxSmemBytes;
    const bool use_pipe = !use_col && !use_row && pipe && a.tma_ld && gp.smem_bytes <= kMaxSmemBytes;
    const Geom& g = use_pipe ? gp : g1;
    CtaFn fn = esz == 1 ? (op == 0 ? pick<uint8_t, 0>(L.cfg) : pick<uint8_t, 1>(L.cfg))
                        : (op == 0 ? pick<uint16_t, 0>(L.cfg) : pick<uint16_t, 1>(L.cfg));
    PipeFn pfn = esz == 1 ? (op == 0 ? pick_pipe<uint8_t, 0>(L.cfg) : pick_pipe<uint8_t, 1>(L.cfg))
                          : (op == 0 ? pick_pipe<uint16_t, 0>(L.cfg) : pick_pipe<uint16_t, 1>(L.cfg));
    const int gx = cdiv(W, TX), gy = cdiv(H, TY);
    const int ntiles = gx * gy, ncta = use_pipe ? (ntiles < 3 ? ntiles : 3) : ntiles;
    int errors = 0, partial = 0;
    std::string first;
    int col_ty = 0;
    if (use_col) {
      // the column kernel, planned and launched as col_launch does
      const bool blk = L.vhgw_col && L.wy >= 9;
      const int ty = col_pick_ty(esz, W, H, L.wy, (seed & 1) ? 152 : 3, kMaxSmemBytes);
      const ColGeom cg = col_geom(esz, ty, L.wy);
      col_ty = ty;
      ColArgs c{};
      c.src = src;
      c.dst = dst;
      c.sp = sp;
      c.dp = dp;
      c.W = W;
      c.H = H;
      c.w = L.wy;
      c.a = L.ay;
      c.ty = cg.ty;
      c.ih = cg.ih;
      c.ihp = cg.ihp;
      c.ntx = cdiv(W * esz, kColBytes);
      c.ntiles = c.ntx * cdiv(H, cg.ty);
      c.blocked = blk;
      c.ld_vec = a.ld_vec;
      c.st_vec = (reinterpret_cast<uintptr_t>(dst) % 4 == 0) && (dp % 4 == 0);
      c.err = &errword;
      c.tma_ld = tma_ok(src, sp, kColBytes / esz, kColBox);
      EmuMap mc{src, nullptr, esz, W, H, sp, kColBytes / esz, kColBox};
      CUtensorMap tc{};
      memcpy(&tc, &mc, sizeof(mc));
      ColFnE cf = esz == 1 ? (op == 0 ? pick_col<uint8_t, 0>(blk) : pick_col<uint8_t, 1>(blk))
                           : (op == 0 ? pick_col<uint16_t, 0>(blk) : pick_col<uint16_t, 1>(blk));
      for (int t = 0; t < c.ntiles; ++t) {
        EmuCta cta;
        std::barrier<> bar(kColThreads);
        cta.bar = &bar;
        uint8_t* sm = static_cast<uint8_t*>(aligned_alloc(128, (cg.smem + 127) / 128 * 128));
        cta.smem = sm;
        cta.smem_size = cg.smem;
        uint64_t mbars[kColMaxBoxes] = {};
        pool_run(
            [&](int tid) {
              g_cta = &cta;
              emu_threadIdx = make_uint3(tid, 0, 0);
              if (tid == 0)
                for (int b = 0; b < kColMaxBoxes; ++b) mbar_init(&mbars[b], 1);
              __syncthreads();
              cf(c, &tc, t, sm, reinterpret_cast<uint32_t*>(sm + kColBytes * cg.ihp), mbars);
            },
            kColThreads);
        free(sm);
        errors += cta_end_errors(cta);
        if (cta.errors.load() && first.empty()) first = cta.first_error;
      }
      a.tma_ld = c.tma_ld;
    }
    if (use_row) {
      // the row kernel, launched as row_launch does
      const bool blk = L.vhgw_row && L.wx >= 9;
      RowArgs ra{};
      ra.src = src;
      ra.dst = dst;
      ra.sp = sp;
      ra.dp = dp;
      ra.W = W;
      ra.H = H;
      ra.w = L.wx;
      ra.a = L.ax;
      ra.ntx = cdiv(W, rg.txp);
      ra.nty = cdiv(H, rg.ty);
      ra.blocked = blk;
      ra.ld_vec = a.ld_vec;
      ra.st_vec = (reinterpret_cast<uintptr_t>(dst) % (8 * esz) == 0) && (dp % (8 * esz) == 0);
      ra.err = &errword;
      ra.tma_ld = tma_ok(src, sp, 128 / esz, rg.ty);
      EmuMap mr{src, nullptr, esz, W, H, sp, 128 / esz, rg.ty};
      CUtensorMap tr{};
      memcpy(&tr, &mr, sizeof(mr));
      RowFnE rf = esz == 1 ? (op == 0 ? pick_row<uint8_t, 0>(blk) : pick_row<uint8_t, 1>(blk))
                           : (op == 0 ? pick_row<uint16_t, 0>(blk) : pick_row<uint16_t, 1>(blk));
      for (int t = 0; t < ra.ntx * ra.nty; ++t) {
        EmuCta cta;
        std::barrier<> bar(kRowThreads);
        cta.bar = &bar;
        uint8_t* sm = static_cast<uint8_t*>(aligned_alloc(128, (rg.smem + 127) / 128 * 128));
        cta.smem = sm;
        cta.smem_size = rg.smem;
        uint64_t mbar = 0;
        pool_run(
            [&](int tid) {
              g_cta = &cta;
              emu_threadIdx = make_uint3(tid, 0, 0);
              uint32_t phase = 0;
              if (tid == 0) mbar_init(&mbar, 1);
              __syncthreads();
              rf(ra, &tr, t, rg, sm, &mbar, phase);
            },
            kRowThreads);
        free(sm);
        errors += cta_end_errors(cta);
        if (cta.errors.load() && first.empty()) first = cta.first_error;
      }
      a.tma_ld = ra.tma_ld;
    }
    const bool use_colv = kern == 4 && L.wx == 1 && L.wy > 1;
    if (use_colv) {
      // the warp-tiled pass along y, planned and launched as colv_launch does;
      // bytes per lane by seed: 4 or 8
      const int lb = (seed / 2) % 2 ? 8 : 4;
      const int sbytes = colv_strip_bytes(lb);
      const int forced = (seed & 1) ? 0 : 1 + static_cast<int>(seed % 200);
      const ColvPlan p = colv_plan(esz, W, H, L.wy, kMaxSmemBytes, forced, lb, (seed % 3) ? 152 : 3);
      if (!p.ok) {
        printf("FAIL case %d: no colv plan\n", cases);
        ++failures;
        continue;
      }
      col_ty = p.L;
      ColvArgs c{};
      c.src = src;
      c.dst = dst;
      c.sp = sp;
      c.dp = dp;
      c.W = W;
      c.H = H;
      c.w = L.wy;
      c.a = L.ay;
      c.L = p.L;
      c.nbox = p.nbox;
      c.ns = cdiv(W * esz, sbytes);
      c.ntask = p.ntask;
      c.wpc = p.wpc;
      c.ld_vec = (reinterpret_cast<uintptr_t>(src) % lb == 0) && (sp % lb == 0);
      c.st_vec = (reinterpret_cast<uintptr_t>(dst) % lb == 0) && (dp % lb == 0);
      c.err = &errword;
      c.tma_ld = tma_ok(src, sp, sbytes / esz, kCvBox);
      EmuMap mc{src, nullptr, esz, W, H, sp, sbytes / esz, kCvBox};
      CUtensorMap tc{};
      memcpy(&tc, &mc, sizeof(mc));
      using VFn = bool (*)(const ColvArgs&, const CUtensorMap*, int, int, uint8_t*, uint64_t*);
      VFn vf = lb == 8 ? (esz == 1 ? (op == 0 ? colv_tile<uint8_t, 0, 8> : colv_tile<uint8_t, 1, 8>)
                                   : (op == 0 ? colv_tile<uint16_t, 0, 8> : colv_tile<uint16_t, 1, 8>))
                         : (esz == 1 ? (op == 0 ? colv_tile<uint8_t, 0, 4> : colv_tile<uint8_t, 1, 4>)
                                     : (op == 0 ? colv_tile<uint16_t, 0, 4> : colv_tile<uint16_t, 1, 4>));
      const int nthr = 32 * c.wpc;
      for (int blk = 0; blk < cdiv(c.ntask, c.wpc); ++blk) {
        EmuCta cta;
        std::barrier<> bar(nthr);
        cta.bar = &bar;
        std::barrier<>* wbv[8] = {};  // per warp (__syncwarp)
        for (int wi = 0; wi < c.wpc; ++wi) cta.wbar[wi] = wbv[wi] = new std::barrier<>(32);
        uint8_t* sm = static_cast<uint8_t*>(aligned_alloc(128, (p.smem + 127) / 128 * 128));
        cta.smem = sm;
        cta.smem_size = p.smem;
        pool_run(
            [&](int tid) {
              g_cta = &cta;
              emu_threadIdx = make_uint3(tid, 0, 0);
              const int warp = tid >> 5, lane = tid & 31, task = blk * c.wpc + warp;
              if (task >= c.ntask) return;
              uint8_t* tile = sm + warp * colv_tile_bytes(c.nbox, lb);
              uint64_t* bars = reinterpret_cast<uint64_t*>(sm + c.wpc * colv_tile_bytes(c.nbox, lb)) + warp * c.nbox;
              if (c.tma_ld && lane == 0)
                for (int b = 0; b < c.nbox; ++b) mbar_init(&bars[b], 1);
              // lanes wait on the barriers only after lane 0 initialised them
              // (a warp-wide __syncwarp in the kernel)
              while (c.tma_ld && lane != 0) {
                bool ready;
                {
                  std::lock_guard<std::mutex> l(g_cta->mu);
                  ready = g_cta->mbars.count(&bars[c.nbox - 1]) != 0;
                }
                if (ready) break;
                std::this_thread::yield();
              }
              vf(c, &tc, task, lane, tile, bars);
            },
            nthr);
        for (int wi = 0; wi < c.wpc; ++wi) delete wbv[wi];
        free(sm);
        errors += cta_end_errors(cta);
        if (cta.errors.load() && first.empty()) first = cta.first_error;
      }
      a.tma_ld = c.tma_ld;
    }
    const int ral = 8 * esz;
    const bool use_rowv = kern == 5 && L.wy == 1 && L.wx >= 9 && L.wx <= 256 &&
                          reinterpret_cast<uintptr_t>(src) % ral == 0 && sp % ral == 0;
    if (use_rowv) {
      const int rr = (seed / 2) % 3 == 0 ? 8 : (seed / 2) % 3 == 1 ? 4 : 2;  // rows per warp
      const RowvPlan p = rowv_plan(W, H, rr, (seed & 1) ? 152 : 3, 12, (seed % 3 == 0) ? 256 * static_cast<int>(1 + seed % 5) : 0);
      col_ty = p.seg;
      RowvArgs ra{};
      ra.src = src;
      ra.dst = dst;
      ra.sp = sp;
      ra.dp = dp;
      ra.W = W;
      ra.H = H;
      ra.w = L.wx;
      ra.a = L.ax;
      ra.seg = p.seg;
      ra.nseg = p.nseg;
      ra.ntask = p.ntask;
      ra.st_vec = (reinterpret_cast<uintptr_t>(dst) % ral == 0) && (dp % ral == 0);
      using RvFn = void (*)(const RowvArgs&, int, int, uint8_t*);
      RvFn rf = rr == 8 ? (esz == 1 ? (op == 0 ? rowv_task<uint8_t, 0, 8> : rowv_task<uint8_t, 1, 8>)
                                    : (op == 0 ? rowv_task<uint16_t, 0, 8> : rowv_task<uint16_t, 1, 8>))
              : rr == 4 ? (esz == 1 ? (op == 0 ? rowv_task<uint8_t, 0, 4> : rowv_task<uint8_t, 1, 4>)
                                    : (op == 0 ? rowv_task<uint16_t, 0, 4> : rowv_task<uint16_t, 1, 4>))
                        : (esz == 1 ? (op == 0 ? rowv_task<uint8_t, 0, 2> : rowv_task<uint8_t, 1, 2>)
                                    : (op == 0 ? rowv_task<uint16_t, 0, 2> : rowv_task<uint16_t, 1, 2>));
      const int wpc = 4;
      for (int blk = 0; blk < cdiv(p.ntask, wpc); ++blk) {
        EmuCta cta;
        std::barrier<> bar(32 * wpc);
        std::vector<std::unique_ptr<std::barrier<>>> wb;
        for (int w = 0; w < wpc; ++w) {
          wb.emplace_back(new std::barrier<>(32));
          cta.wbar[w] = wb.back().get();
        }
        cta.bar = &bar;
        const size_t smb = static_cast<size_t>(wpc) * rv_warp_smem(esz, rr);
        uint8_t* sm = static_cast<uint8_t*>(aligned_alloc(128, (smb + 127) / 128 * 128));
        cta.smem = sm;
        cta.smem_size = smb;
        pool_run(
            [&](int tid) {
              g_cta = &cta;
              emu_threadIdx = make_uint3(tid, 0, 0);
              const int warp = tid >> 5, lane = tid & 31, task = blk * wpc + warp;
              if (task >= p.ntask) return;
              rf(ra, task, lane, sm + warp * rv_warp_smem(esz, rr));
            },
            32 * wpc);
        free(sm);
        errors += cta_end_errors(cta);
        if (cta.errors.load() && first.empty()) first = cta.first_error;
      }
    }
    const bool use_comp = kern == 6;
    if (use_comp) {
      CompArgs ca{};
      ca.src = src;
      ca.dst = dst;
      ca.sp = sp;
      ca.dp = dp;
      ca.W = W;
      ca.H = H;
      ca.wx = wx;
      ca.wy = wy;
      ca.ax = ax;
      ca.ay = ay;
      ca.tiles_x = cdiv(W, kCompTX);
      const int ntile = ca.tiles_x * cdiv(H, kCompTY);
      using CompFn = void (*)(const CompArgs&, int, int, uint32_t*);
      // the halo class the launcher picks (2, 4 or 8), and on odd seeds the
      // widest one (8), which every window fits
      const int halo = (wx > wy ? wx : wy) - 1;
      const int hb = (seed & 1) ? 8 : halo <= 2 ? 2 : halo <= 4 ? 4 : 8;
#define MORPH_COMP_PICK(HB)                                                                                    \
  (esz == 1 ? (op == 0 ? comp_tile<uint8_t, 0, HB> : op == 1 ? comp_tile<uint8_t, 1, HB> : comp_tile<uint8_t, 2, HB>) \
            : (op == 0 ? comp_tile<uint16_t, 0, HB> : op == 1 ? comp_tile<uint16_t, 1, HB> : comp_tile<uint16_t, 2, HB>))
      CompFn cf = hb == 2 ? MORPH_COMP_PICK(2) : hb == 4 ? MORPH_COMP_PICK(4) : MORPH_COMP_PICK(8);
#undef MORPH_COMP_PICK
      for (int tile = 0; tile < ntile; ++tile) {
        EmuCta cta;
        std::barrier<> bar(kCompThreads);
        cta.bar = &bar;
        const size_t smb = sizeof(uint32_t) * kCompSmemWords;
        uint32_t* sm = static_cast<uint32_t*>(aligned_alloc(128, smb));
        cta.smem = reinterpret_cast<const uint8_t*>(sm);
        cta.smem_size = smb;
        pool_run(
            [&](int tid) {
              g_cta = &cta;
              emu_threadIdx = make_uint3(tid, 0, 0);
              cf(ca, tile, tid, sm);
            },
            kCompThreads);
        free(sm);
        errors += cta_end_errors(cta);
        if (cta.errors.load() && first.empty()) first = cta.first_error;
      }
    }
    for (int c = 0; c < (use_col || use_row || use_colv || use_rowv || use_comp ? 0 : ncta); ++c) {
      const int bx = c % gx, by = c / gx;
      EmuCta cta;
      std::barrier<> bar(kThreads);
      cta.bar = &bar;
      uint4* smem = static_cast<uint4*>(aligned_alloc(128, (g.smem_bytes + 127) / 128 * 128));
      cta.smem = reinterpret_cast<const uint8_t*>(smem);
      cta.smem_size = g.smem_bytes;
      uint64_t mbar[2] = {0, 0};
      pool_run([&](int tid) {
        g_cta = &cta;
        emu_threadIdx = make_uint3(tid, 0, 0);
        uint32_t phase = 0;
        if (use_pipe) {
          if (tid == 0) {
            mbar_init(&mbar[0], 1);
            mbar_init(&mbar[1], 1);
          }
          __syncthreads();
          pfn(a, &tin, &tout, g, smem, mbar, gx, ntiles, c, ncta);
        } else {
          if (tid == 0) mbar_init(&mbar[0], 1);
          __syncthreads();
          fn(a, &tin, &tout, bx * TX, by * TY, g, smem, &mbar[0], phase, a.err);
        }
      });
      free(smem);
      errors += cta_end_errors(cta);
      partial += cta.partial_stores.load();
      if (cta.errors.load() && first.empty()) first = cta.first_error;
    }
    // compare with the oracle, and check the bytes between rows are untouched
    std::vector<uint8_t> want(static_cast<size_t>(W) * H * esz);
    if (use_comp) {
      // the composite from the oracle's erosion and dilation (section 2)
      const long long wp = static_cast<long long>(W) * esz;
      std::vector<uint8_t> mid(want.size()), other(want.size());
      if (op == 2) {
        oracle_morph(src, esz, W, H, sp, wx, wy, ax, ay, 1, want.data(), wp);
        oracle_morph(src, esz, W, H, sp, wx, wy, ax, ay, 0, other.data(), wp);
        for (size_t i = 0; i < want.size(); i += esz) {
          if (esz == 1) {
            want[i] = static_cast<uint8_t>(want[i] - other[i]);
          } else {
            uint16_t d, e;
            memcpy(&d, &want[i], 2);
            memcpy(&e, &other[i], 2);
            d = static_cast<uint16_t>(d - e);
            memcpy(&want[i], &d, 2);
          }
        }
      } else {
        oracle_morph(src, esz, W, H, sp, wx, wy, ax, ay, op == 0 ? 0 : 1, mid.data(), wp);
        oracle_morph(mid.data(), esz, W, H, wp, wx, wy, wx - 1 - ax, wy - 1 - ay, op == 0 ? 1 : 0, want.data(), wp);
      }
    } else {
      oracle_morph(src, esz, W, H, sp, wx, wy, ax, ay, op, want.data(), static_cast<long long>(W) * esz);
    }
    long long bad = 0, guard = 0;
    for (int y = 0; y < H; ++y) {
      if (memcmp(dst + y * dp, want.data() + static_cast<size_t>(y) * W * esz, static_cast<size_t>(W) * esz)) ++bad;
      if (y < H - 1)
        for (long long b = static_cast<long long>(W) * esz; b < dp; ++b)
          if (dst[y * dp + b] != 0xA5) ++guard;
    }
    for (int b = 0; b < doff; ++b)
      if (dbuf[b] != 0xA5) ++guard;
    const bool ok = !errors && !bad && !guard && !errword;
    if (!ok) ++failures;
    printf("%s case %d esz %d op %d %dx%d win %dx%d a %d,%d cfg %d tile %dx%d blk %d,%d tma %d,%d kern %d "
           "col_ty %d partial_st %d rows_bad %lld guard %lld dev_err %d %s\n",
           ok ? "OK" : "FAIL", cases, esz, op, W, H, wx, wy, ax, ay, L.cfg, TX, TY, a.blk_x, a.blk_y, a.tma_ld,
           a.tma_st, use_comp ? 6 : use_rowv ? 5 : use_colv ? kern : use_row ? 3 : use_col ? 2 : use_pipe ? 1 : 0, col_ty, partial, bad, guard, errword, first.c_str());
    fflush(stdout);
    free(sbuf);
    free(dbuf);
  }
  fprintf(stderr, "%d cases, %d failures\n", cases, failures);
  // The pool's threads still wait on a static barrier: leave without running
  // static destructors under them.
  fflush(stdout);
  fflush(stderr);
  _exit(failures ? 1 : 0);
}
