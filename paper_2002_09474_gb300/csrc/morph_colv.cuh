// Pass along y (a 1 x w element; the paper's "horizontal pass", section 5.1)
// by van Herk/Gil-Werman (section 5.1.1) with blocks of w rows, one warp per
// work item.
//
// A warp owns a strip 128 bytes wide (lane l: bytes 4l .. 4l+3 of every row,
// four u8 or two u16 pixels) and L consecutive output rows.  Its L + w - 1
// input rows arrive in shared memory as TMA boxes of 32 rows, each on its
// own mbarrier, all issued when the warp starts; the scans begin as soon as
// the first boxes land.  Warps never share shared memory and never
// synchronise: lanes touch only their own 4-byte column.
//
// Blocks of w rows are aligned to the end of the tile: the last block ends
// at output row L, the first one is partial when w does not divide L.  For a
// block [E - w, E):
//   h-scan  rows E-1 down to E-w:  h[r] = op(S[r], h[r+1]), written over S[r]
//           in place (the suffix the paper keeps in its second buffer);
//           h[E-w] is the whole block, which is output E-w.
//   g-scan  rows E .. E+w-2:  g = op(g, S[e]); output e-w+1 = op(h[e-w+1], g).
// Every row is scanned once each way, whatever the tile height, so halo rows
// cost shared memory and L2 traffic but no arithmetic beyond the partial
// first block.
//
// 8-bit pixels ride in 16-bit lanes without unpacking: min/max.u16x2 of two
// words sets each lane's high byte to the min/max of the high bytes whatever
// the low bytes hold.  The raw word carries pixels 1 and 3 in its high
// bytes, the word shifted left by 8 carries pixels 0 and 2; one byte permute
// puts the four results back together.  16-bit pixels use the raw word.
#pragma once

#include "morph_common.cuh"

namespace morph {

constexpr int kCvBytes = 128;  // strip width (bytes)
constexpr int kCvBox = 32;     // rows per TMA box
constexpr int kCvMaxBox = 56;  // boxes per warp tile at most (1792 rows)
constexpr int kCvBoxBytes = kCvBytes * kCvBox;

struct ColvArgs {
  const uint8_t* src;
  uint8_t* dst;
  long long sp, dp;  // pitches in bytes
  int W, H;          // pixels
  int w, a;          // window along y and its anchor, clipped to the image
  int L;             // output rows per warp tile
  int nbox;          // shared-memory boxes per warp tile: ceil((L + w - 1) / 32)
  int ns;            // strips across: ceil(W * esz / 128)
  int ntask;         // warp tiles: ns * ceil(H / L)
  int wpc;           // warps per CTA
  int tma_ld;        // 1: input boxes arrive by TMA
  int ld_vec;        // 1: rows allow aligned 32-bit loads
  int st_vec;        // 1: rows allow aligned 32-bit stores
  int* err;          // device error word
};

// Shared memory of one CTA: wpc warp tiles, then wpc * kCvMaxBox mbarriers.
__host__ __device__ inline int colv_tile_bytes(int nbox) { return nbox * kCvBoxBytes; }
__host__ __device__ inline int colv_smem_bytes(int nbox, int wpc) {
  return wpc * colv_tile_bytes(nbox) + wpc * kCvMaxBox * 8;
}

// Two 16-bit-lane carriers of one 32-bit word (u8: odd pixels in v[0], even
// pixels in v[1]; u16: the word itself in v[0]).
template <int E>
struct Cw {
  uint32_t v[E == 1 ? 2 : 1];
};

template <int E>
__device__ __forceinline__ Cw<E> cw_of(uint32_t raw) {
  Cw<E> c;
  c.v[0] = raw;
  if (E == 1) c.v[E == 1 ? 1 : 0] = raw << 8;
  return c;
}
template <int E>
__device__ __forceinline__ uint32_t cw_word(const Cw<E>& c) {
  // bytes: even.b1 (pixel 0), odd.b1 (pixel 1), even.b3 (pixel 2), odd.b3 (pixel 3)
  if (E == 1) return __byte_perm(c.v[E == 1 ? 1 : 0], c.v[0], 0x7351);
  return c.v[0];
}
template <int OP, int E>
__device__ __forceinline__ Cw<E> cw_op(const Cw<E>& a, const Cw<E>& b) {
  Cw<E> r;
#pragma unroll
  for (int i = 0; i < (E == 1 ? 2 : 1); ++i) r.v[i] = OP == 0 ? __vminu2(a.v[i], b.v[i]) : __vmaxu2(a.v[i], b.v[i]);
  return r;
}

// Stores output word `word` of row y at pixel px0 (the lane's first pixel).
template <typename T>
__device__ __forceinline__ void colv_store(const ColvArgs& a, int y, int px0, uint32_t word, bool fast) {
  constexpr int E = sizeof(T), PPW = 4 / E;
  uint8_t* row = a.dst + static_cast<long long>(y) * a.dp;
  if (fast) {
    *reinterpret_cast<uint32_t*>(row + static_cast<long long>(px0) * E) = word;
  } else {
#pragma unroll
    for (int t = 0; t < PPW; ++t)
      if (px0 + t < a.W) reinterpret_cast<T*>(row)[px0 + t] = static_cast<T>(word >> (8 * E * t));
  }
}

// One warp tile.  tile: this warp's shared memory (nbox boxes); bars: its
// kCvMaxBox mbarriers, initialised with count 1.  lane: 0..31.  Returns false
// when a bounded wait gave up (error word set by lane 0).
template <typename T, int OP>
__device__ __forceinline__ bool colv_tile(const ColvArgs& a, const CUtensorMap* tin, int task, int lane,
                                          uint8_t* tile, uint64_t* bars) {
  constexpr int E = sizeof(T), PPW = 4 / E;
  using C = Cw<E>;
  const uint32_t IDW = ident_word<OP>();
  const int s = task % a.ns;                  // strip
  const int y0 = (task / a.ns) * a.L;         // first output row
  const int Lr = a.L < a.H - y0 ? a.L : a.H - y0;  // output rows of this tile
  const int w = a.w;
  const int ys = y0 - a.a;                    // image row of tile row 0
  const int nin = Lr + w - 1;                 // input rows
  const int nb = (nin + kCvBox - 1) / kCvBox;  // boxes to fill
  const int px0 = s * (kCvBytes / E) + lane * PPW;
  const bool col_in = px0 < a.W;
  const bool fast = a.st_vec && px0 + PPW <= a.W;
  uint8_t* col = tile + 4 * lane;

  auto LD = [&](int r) { return *reinterpret_cast<const uint32_t*>(col + r * kCvBytes); };
  auto ST = [&](int r, uint32_t v) { *reinterpret_cast<uint32_t*>(col + r * kCvBytes) = v; };

  int have = 0;  // boxes landed (and fixed up)
  if (a.tma_ld) {
    if (lane == 0) {
      fence_proxy_async_smem();
      for (int b = 0; b < nb; ++b) {
        mbar_arrive_expect_tx(&bars[b], static_cast<uint32_t>(kCvBoxBytes));
        tma_load_2d(tile + b * kCvBoxBytes, tin, &bars[b], s * (kCvBytes / E), ys + b * kCvBox);
      }
    }
  } else {
    for (int r = 0; r < nin; ++r) {
      const int y = ys + r;
      uint32_t v = IDW;
      if (y >= 0 && y < a.H && col_in) {
        const uint8_t* row = a.src + static_cast<long long>(y) * a.sp;
        if (a.ld_vec && px0 + PPW <= a.W) {
          v = *reinterpret_cast<const uint32_t*>(row + static_cast<long long>(px0) * E);
        } else {
#pragma unroll
          for (int t = 0; t < PPW; ++t)
            if (px0 + t < a.W) {
              const uint32_t sh = 8 * E * t, m = (E == 1 ? 0xFFu : 0xFFFFu) << sh;
              v = (v & ~m) | (static_cast<uint32_t>(reinterpret_cast<const T*>(row)[px0 + t]) << sh);
            }
        }
      }
      ST(r, v);
    }
    have = nb;
  }

  // Makes rows [0, rows) available: waits for their boxes; for erosion,
  // rows outside the image (TMA fills them with 0) become the identity.
  auto ensure = [&](int rows) -> bool {
    const int need = (rows + kCvBox - 1) / kCvBox;
    for (; have < need; ++have) {
      if (!mbar_wait_bounded(&bars[have], 0)) {
        if (lane == 0) {
          atomicExch(a.err, kDevErrTmaTimeout);
          for (int b = have + 1; b < nb; ++b) mbar_wait_bounded(&bars[b], 0);  // let copies in flight land
        }
        return false;
      }
      if (OP == 0) {
        const int r0 = have * kCvBox;
        if (ys + r0 < 0 || ys + r0 + kCvBox > a.H)
          for (int r = r0; r < r0 + kCvBox; ++r)
            if (ys + r < 0 || ys + r >= a.H) ST(r, IDW);
      }
    }
    return true;
  };

  const int beta = Lr % w;
  for (int E0 = beta ? beta : w; E0 <= Lr; E0 += w) {
    const int lo = E0 - w > 0 ? E0 - w : 0;
    if (!ensure(E0 + w - 1)) return false;
    // h-scan, in place
    C h = cw_of<E>(LD(E0 - 1));
    ST(E0 - 1, cw_word<E>(h));
#pragma unroll 4
    for (int r = E0 - 2; r >= lo; --r) {
      h = cw_op<OP, E>(h, cw_of<E>(LD(r)));
      ST(r, cw_word<E>(h));
    }
    if (E0 - w >= 0 && col_in) colv_store<T>(a, y0 + E0 - w, px0, cw_word<E>(h), fast);
    // g-scan; rows before w-1 (partial first block only) emit nothing
    C g = cw_of<E>(LD(E0));
    int e = E0;
    const int e_emit = E0 > w - 1 ? E0 : w - 1;
    for (; e < e_emit; ) {
      ++e;
      g = cw_op<OP, E>(g, cw_of<E>(LD(e)));
    }
    // here g covers rows E0 .. e
    if (col_in) {
      if (fast) {
        uint8_t* out = a.dst + static_cast<long long>(y0 + e - w + 1) * a.dp + static_cast<long long>(px0) * E;
#pragma unroll 4
        for (; e <= E0 + w - 2; ++e) {
          const C o = cw_op<OP, E>(cw_of<E>(LD(e - w + 1)), g);
          *reinterpret_cast<uint32_t*>(out) = cw_word<E>(o);
          out += a.dp;
          if (e + 1 <= E0 + w - 2) g = cw_op<OP, E>(g, cw_of<E>(LD(e + 1)));
        }
      } else {
        for (; e <= E0 + w - 2; ++e) {
          const C o = cw_op<OP, E>(cw_of<E>(LD(e - w + 1)), g);
          colv_store<T>(a, y0 + e - w + 1, px0, cw_word<E>(o), false);
          if (e + 1 <= E0 + w - 2) g = cw_op<OP, E>(g, cw_of<E>(LD(e + 1)));
        }
      }
    }
  }
  return true;
}

}  // namespace morph

namespace morph {

// Launch shape of the pass along y: output rows per warp tile (L), warps per
// CTA, shared memory.  The model: each warp tile costs its L rows plus the
// g-scan rows of a partial first block plus a fixed start-up; tiles run in
// waves of (SMs x resident warps); an SM issues at full rate only with about
// 8 warps busy.
struct ColvPlan {
  int L, nbox, wpc, ntask, smem;
  bool ok;
};

inline ColvPlan colv_plan(int esz, int W, int H, int w, int sms, int max_smem, int forced_L) {
  ColvPlan best{0, 0, 0, 0, 0, false};
  if (w < 2 || sms < 1) return best;
  const int ns = (W * esz + kCvBytes - 1) / kCvBytes;
  int hmax = (H + 7) / 8 * 8;
  if (hmax > 1024) hmax = 1024;
  int want = 0;  // a forced tile height, at most the image's height
  if (forced_L > 0) {
    want = (forced_L + 7) / 8 * 8;
    if (want > hmax) want = hmax;
  }
  double best_cost = 1e300;
  for (int L = 8; L <= hmax; L += 8) {
    if (want > 0 && L != want) continue;
    const int nbox = (L + w - 1 + kCvBox - 1) / kCvBox;
    if (nbox > kCvMaxBox) break;
    int wpc = 4;
    while (wpc > 1 && colv_smem_bytes(nbox, wpc) > max_smem) wpc /= 2;
    const int smem = colv_smem_bytes(nbox, wpc);
    if (smem > max_smem) break;
    int ctas = 233472 / (smem + 1024);
    if (ctas > 32) ctas = 32;
    if (ctas * wpc > 64) ctas = 64 / wpc;
    if (ctas < 1) ctas = 1;
    const int wps = ctas * wpc;
    const long long ntask = static_cast<long long>(ns) * ((H + L - 1) / L);
    const double per_sm = static_cast<double>(ntask) / sms;
    const double waves = static_cast<double>(static_cast<long long>((per_sm + wps - 1) / wps));
    const double busy = per_sm < wps ? per_sm : wps;
    const int beta = L % w;
    const double extra = beta ? (w - 1 - beta) : 0;
    const double work = L + 0.25 * extra + 32.0;
    const double eff = busy >= 8 ? 1.0 : busy / 8.0;
    const double cost = waves * work / eff;
    if (cost < best_cost) {
      best_cost = cost;
      best = ColvPlan{L, nbox, wpc, static_cast<int>(ntask), smem, true};
    }
  }
  return best;
}

}  // namespace morph
