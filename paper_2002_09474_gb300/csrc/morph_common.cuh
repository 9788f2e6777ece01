// Device helpers shared by the morphology kernels (sm_103a).
//
// Pixels travel packed in 32-bit words: four 8-bit pixels or two 16-bit
// pixels, lowest address in the lowest byte.  One packed min/max handles a
// whole word, the GPU counterpart of the paper's 16-lane vminq_u8/vmaxq_u8
// (section 3, section 5.1.1).
#pragma once

#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

namespace morph {

// Codes a kernel writes to its device error word.
enum : int {
  kDevErrNone = 0,
  kDevErrTmaTimeout = 1,  // a TMA load did not complete within the wait limit
  kDevErrBadTile = 2,     // a work item named a tile outside its image
};

// Wall-clock limit of every bounded wait (nanoseconds, %globaltimer).
constexpr unsigned long long kWaitLimitNs = 2000000000ull;

template <typename T> struct Pix;
template <> struct Pix<uint8_t> {
  static constexpr int PK = 4;          // pixels per 32-bit word
  static constexpr uint32_t MAXV = 0xFFu;
};
template <> struct Pix<uint16_t> {
  static constexpr int PK = 2;
  static constexpr uint32_t MAXV = 0xFFFFu;
};

// Identity of the operation on a packed word: all ones never lowers a min
// (erosion), zero never raises a max (dilation).
template <int OP> __host__ __device__ constexpr uint32_t ident_word() {
  return OP == 0 ? 0xFFFFFFFFu : 0u;
}

// In-register transpose of a PK x PK block of pixels held as PK words.
// On entry v[i] holds row i (pixel j in lane j); on exit v[j] holds column j
// (row i in lane i).  4x4 bytes: two butterfly rounds of byte permutes, first
// interleaving bytes of row pairs, then 16-bit halves of those pairs -- the
// same two-level 2x2 block transpose as the paper's vtrn-based 8x8.16 and
// 16x16.8 transposes (section 4), on 4-byte registers.
__device__ __forceinline__ void transpose_block(uint32_t (&v)[4]) {
  const uint32_t a0 = __byte_perm(v[0], v[1], 0x5140);  // r0.b0 r1.b0 r0.b1 r1.b1
  const uint32_t a1 = __byte_perm(v[0], v[1], 0x7362);  // r0.b2 r1.b2 r0.b3 r1.b3
  const uint32_t b0 = __byte_perm(v[2], v[3], 0x5140);  // r2.b0 r3.b0 r2.b1 r3.b1
  const uint32_t b1 = __byte_perm(v[2], v[3], 0x7362);  // r2.b2 r3.b2 r2.b3 r3.b3
  v[0] = __byte_perm(a0, b0, 0x5410);                   // column 0
  v[1] = __byte_perm(a0, b0, 0x7632);                   // column 1
  v[2] = __byte_perm(a1, b1, 0x5410);                   // column 2
  v[3] = __byte_perm(a1, b1, 0x7632);                   // column 3
}
// 2x2 block of 16-bit pixels.
__device__ __forceinline__ void transpose_block(uint32_t (&v)[2]) {
  const uint32_t c0 = __byte_perm(v[0], v[1], 0x5410);  // r0.p0 r1.p0
  const uint32_t c1 = __byte_perm(v[0], v[1], 0x7632);  // r0.p1 r1.p1
  v[0] = c0;
  v[1] = c1;
}

// ---------------------------------------------------------------------------
// Shared-memory / TMA / mbarrier wrappers (inline PTX).
// ---------------------------------------------------------------------------
#ifndef MORPH_HOST_EMU
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

// Makes the barrier initialisation visible to the TMA unit (async proxy).
__device__ __forceinline__ void fence_barrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_test_wait(uint64_t* bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return done != 0;
}

__device__ __forceinline__ unsigned long long global_timer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return done != 0;
}

// Waits for the barrier phase with the given parity to complete; gives up
// after kWaitLimitNs and returns false.  try_wait suspends the thread in
// hardware until the phase completes or a short system time limit passes.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_timer_ns();
  while (!mbar_try_wait(bar, parity)) {
    if (global_timer_ns() - t0 > kWaitLimitNs) return false;
  }
  return true;
}

// 2-D tiled TMA load of one box into shared memory, completing on `bar`.
// x must be a multiple of 16 bytes / element size (caller's contract).
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4}], [%2];" ::"r"(smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_addr(bar)), "r"(x), "r"(y)
      : "memory");
}

// Orders this thread's generic-proxy shared-memory accesses before later
// async-proxy (TMA) accesses to the same memory.
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void prefetch_tensormap(const CUtensorMap* map) {
  asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

// 2-D tiled TMA store of one box from shared memory (bulk-group completion).
__device__ __forceinline__ void tma_store_2d(const CUtensorMap* map, const void* src, int x, int y) {
  asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.tile.bulk_group [%0, {%2, %3}], [%1];" ::"l"(
                   reinterpret_cast<uint64_t>(map)),
               "r"(smem_addr(src)), "r"(x), "r"(y)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read_all() {
  asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// Programmatic dependent launch: a kernel launched with programmatic stream
// serialisation may start while the previous kernel on its stream is still
// running.  Each kernel of this library lets its successor be scheduled once
// every one of its CTAs has finished its work (launch_dependents at the end,
// so the successor's CTAs take SMs only as this grid drains), and waits for
// its predecessor to finish and flush its memory (wait) before touching
// global memory; without such a launch both are no-ops.
__device__ __forceinline__ void pdl_launch_dependents() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Per-thread asynchronous copies global -> shared (8 or 16 bytes, both
// addresses aligned to the size), grouped by commit; wait_group<N> returns
// once at most N of this thread's groups are still in flight.
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_addr(smem)), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(smem)), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

#else
// Host stand-ins with the same signatures, defined by the CPU emulator of the
// kernels (tests/emu); only compiled when MORPH_HOST_EMU is set.
void mbar_init(uint64_t* bar, uint32_t count);
void fence_barrier_init();
void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes);
bool mbar_try_wait(uint64_t* bar, uint32_t parity);
bool mbar_wait_bounded(uint64_t* bar, uint32_t parity);
void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y);
void fence_proxy_async_smem();
void prefetch_tensormap(const CUtensorMap* map);
void tma_store_2d(const CUtensorMap* map, const void* src, int x, int y);
void bulk_commit();
void bulk_wait_read_all();
void bulk_wait_all();
inline void pdl_launch_dependents() {}
inline void pdl_wait() {}
void cp_async8(void* smem, const void* gmem);
void cp_async16(void* smem, const void* gmem);
void cp_async_commit();
template <int N>
void cp_async_wait() {}

#endif

}  // namespace morph
