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
  int st_vec;        // 1: rows allow aligned stores of a lane's words (4 * words per lane bytes)
  int* err;          // device error word
  int nring;         // ring form: boxes of the ring (the tile's rows cycle through them)
  int ring_mul;      // ceil(2^20 / nring): floor(b / nring) = (b * ring_mul) >> 20 for b < 2^10
};

// Shared memory of one CTA: wpc warp tiles (boxes of 32 rows of 128 * nwl
// bytes), then wpc * nbox mbarriers.
__host__ __device__ inline int colv_tile_bytes(int nbox, int nwl = 1) { return nbox * kCvBoxBytes * nwl; }
__host__ __device__ inline int colv_smem_bytes(int nbox, int wpc, int nwl = 1) {
  return wpc * colv_tile_bytes(nbox, nwl) + wpc * nbox * 8;
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

// NWL 32-bit words of one row of a lane's column (NWL = 1 or 2).
template <int NWL>
struct Wd {
  uint32_t v[NWL];
};
template <int NWL>
__device__ __forceinline__ Wd<NWL> wd_ld(const uint8_t* p) {
  Wd<NWL> w;
  if (NWL == 2) {
    const uint2 u = *reinterpret_cast<const uint2*>(p);
    w.v[0] = u.x;
    w.v[NWL - 1] = u.y;
  } else {
    w.v[0] = *reinterpret_cast<const uint32_t*>(p);
  }
  return w;
}
template <int NWL>
__device__ __forceinline__ void wd_st(uint8_t* p, const Wd<NWL>& w) {
  if (NWL == 2)
    *reinterpret_cast<uint2*>(p) = make_uint2(w.v[0], w.v[NWL - 1]);
  else
    *reinterpret_cast<uint32_t*>(p) = w.v[0];
}

// One warp tile.  tile: this warp's shared memory (nbox boxes of 32 rows of
// 128 * NWL bytes); bars: its nbox mbarriers, initialised with count 1.
// lane: 0..31, owning bytes 4 NWL lane .. 4 NWL lane + 4 NWL - 1 of each row
// of the strip.  Two words per lane give each lane two independent scan
// chains.  Returns false when a bounded wait gave up (error word set by lane
// 0).
//
// Ring form (RG, TMA-loaded rows, one word per lane): the tile's rows cycle
// through a.nring boxes.  Row r is last read at g-scan step r + w - 1 (as
// the suffix h), so once the g-scan has passed 32 (b - nring) + 30 + w, box
// b can be loaded into the slot of box b - nring.  Every wait then finds its
// box issued when nring >= ceil((w + 39) / 32) (the h-scan of a block waits
// for rows below E0 with the g-scan done to E0 - 2; a g-scan batch at e
// waits for rows to e + 7 with the g-scan done to e - 2 at worst); one box
// more lets a load run ahead.  The shared memory then no longer grows with
// the tile height L.
template <typename T, int OP, int NWL = 1, bool RG = false>
__device__ __forceinline__ bool colv_tile(const ColvArgs& a, const CUtensorMap* tin, int task, int lane,
                                          uint8_t* tile, uint64_t* bars) {
  static_assert(!RG || NWL == 1, "the ring form has one word per lane");
  static_assert(kCvBox == 32, "rows per box");
  constexpr int E = sizeof(T), PPW = 4 / E;
  constexpr int SB = kCvBytes * NWL, BOXB = SB * kCvBox;  // strip bytes, box bytes
  using C = Cw<E>;
  using Wv = Wd<NWL>;
  const uint32_t IDW = ident_word<OP>();
  const int s = task % a.ns;                  // strip
  const int y0 = (task / a.ns) * a.L;         // first output row
  const int Lr = a.L < a.H - y0 ? a.L : a.H - y0;  // output rows of this tile
  const int w = a.w;
  const int ys = y0 - a.a;                    // image row of tile row 0
  const int nin = Lr + w - 1;                 // input rows
  const int nb = (nin + kCvBox - 1) / kCvBox;  // boxes to fill
  const int px0 = s * (SB / E) + lane * PPW * NWL;  // the lane's first pixel
  const bool col_in = px0 < a.W;
  const bool fast = a.st_vec && px0 + PPW * NWL <= a.W;
  uint8_t* col = tile + 4 * NWL * lane;

  const int NR = RG ? a.nring : 0;
  auto slot_of = [&](int b) { return RG ? b - ((b * a.ring_mul) >> 20) * NR : b; };
  auto rowp = [&](int r) { return RG ? col + slot_of(r >> 5) * BOXB + (r & 31) * SB : col + r * SB; };
  auto LD = [&](int r) { return wd_ld<NWL>(rowp(r)); };
  auto ST = [&](int r, const Wv& v) { wd_st<NWL>(rowp(r), v); };
  Wv IDV;
#pragma unroll
  for (int i = 0; i < NWL; ++i) IDV.v[i] = IDW;

  int have = 0;  // boxes landed (and fixed up)
  int nxt = RG && NR < nb ? NR : nb;  // boxes issued
  auto issue = [&](int b) {  // lane 0
    const int sl = slot_of(b);
    mbar_arrive_expect_tx(&bars[sl], static_cast<uint32_t>(BOXB));
    tma_load_2d(tile + sl * BOXB, tin, &bars[sl], s * (SB / E), ys + b * kCvBox);
  };
  if (a.tma_ld) {
    if (lane == 0) {
      fence_proxy_async_smem();
      for (int b = 0; b < nxt; ++b) issue(b);
    }
  } else {
    for (int r = 0; r < nin; ++r) {
      const int y = ys + r;
      Wv v = IDV;
      if (y >= 0 && y < a.H) {
        const uint8_t* row = a.src + static_cast<long long>(y) * a.sp;
#pragma unroll
        for (int i = 0; i < NWL; ++i) {
          const int p0 = px0 + i * PPW;
          if (a.ld_vec && p0 + PPW <= a.W) {
            v.v[i] = *reinterpret_cast<const uint32_t*>(row + static_cast<long long>(p0) * E);
          } else {
#pragma unroll
            for (int t = 0; t < PPW; ++t)
              if (p0 + t < a.W) {
                const uint32_t sh = 8 * E * t, m = (E == 1 ? 0xFFu : 0xFFFFu) << sh;
                v.v[i] = (v.v[i] & ~m) | (static_cast<uint32_t>(reinterpret_cast<const T*>(row)[p0 + t]) << sh);
              }
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
      const uint32_t par = RG ? static_cast<uint32_t>(((have * a.ring_mul) >> 20) & 1) : 0u;
      bool got = mbar_wait_bounded(&bars[slot_of(have)], par);
      if (RG) got = __all_sync(0xffffffffu, got);
      if (!got) {
        if (lane == 0) {
          atomicExch(a.err, kDevErrTmaTimeout);
          for (int b = have + 1; b < nxt; ++b)  // let copies in flight land
            mbar_wait_bounded(&bars[slot_of(b)], RG ? static_cast<uint32_t>(((b * a.ring_mul) >> 20) & 1) : 0u);
        }
        return false;
      }
      if (OP == 0) {
        const int r0 = have * kCvBox;
        if (ys + r0 < 0 || ys + r0 + kCvBox > a.H)
          for (int r = r0; r < r0 + kCvBox; ++r)
            if (ys + r < 0 || ys + r >= a.H) ST(r, IDV);
      }
    }
    return true;
  };
  // Ring form: loads the boxes whose slots the g-scan, done to row e_done,
  // has freed.  The h-scan's in-place stores went to those slots, so every
  // lane orders them before the copy (proxy fence), then lane 0 issues.
  auto release = [&](int e_done) {
    while (nxt < nb && 32 * (nxt - NR) + 30 + w <= e_done) {
      fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) issue(nxt);
      ++nxt;
    }
  };
  // stores output row y from the lane's words
  auto store = [&](int y, const Wv& v, bool vec) {
    if (vec) {
      wd_st<NWL>(a.dst + static_cast<long long>(y) * a.dp + static_cast<long long>(px0) * E, v);
    } else {
#pragma unroll
      for (int i = 0; i < NWL; ++i)
        if (px0 + i * PPW < a.W) colv_store<T>(a, y, px0 + i * PPW, v.v[i], false);
    }
  };

  // Rows move between shared memory and registers 8 at a time: the 8 loads
  // of a batch issue together, so a scan waits for shared-memory latency
  // once per batch rather than once per row (the in-place stores of the
  // h-scan would otherwise order every load after the previous store).
  constexpr int kB = 8;
  C IDC;
#pragma unroll
  for (int i = 0; i < (E == 1 ? 2 : 1); ++i) IDC.v[i] = IDW;
  const int beta = Lr % w;
  for (int E0 = beta ? beta : w; E0 <= Lr; E0 += w) {
    const int lo = E0 - w > 0 ? E0 - w : 0;
    if (!ensure(RG ? E0 : E0 + w - 1)) return false;
    // h-scan, rows E0-1 down to lo, in place
    C h[NWL];
#pragma unroll
    for (int i = 0; i < NWL; ++i) h[i] = IDC;
    int r = E0 - 1;
    for (; r - (kB - 1) >= lo; r -= kB) {
      Wv x[kB];
#pragma unroll
      for (int t = 0; t < kB; ++t) x[t] = LD(r - t);
#pragma unroll
      for (int t = 0; t < kB; ++t)
#pragma unroll
        for (int i = 0; i < NWL; ++i) {
          h[i] = cw_op<OP, E>(h[i], cw_of<E>(x[t].v[i]));
          x[t].v[i] = cw_word<E>(h[i]);
        }
#pragma unroll
      for (int t = 0; t < kB; ++t) ST(r - t, x[t]);
    }
    for (; r >= lo; --r) {
      Wv x = LD(r);
#pragma unroll
      for (int i = 0; i < NWL; ++i) {
        h[i] = cw_op<OP, E>(h[i], cw_of<E>(x.v[i]));
        x.v[i] = cw_word<E>(h[i]);
      }
      ST(r, x);
    }
    if (E0 - w >= 0 && col_in) {
      Wv o;
#pragma unroll
      for (int i = 0; i < NWL; ++i) o.v[i] = cw_word<E>(h[i]);
      store(y0 + E0 - w, o, fast);
    }
    // g-scan over rows E0 .. E0+w-2; row e closes the window of output
    // e-w+1, so rows before w-1 (a partial first block only) emit nothing
    C g[NWL];
#pragma unroll
    for (int i = 0; i < NWL; ++i) g[i] = IDC;
    const int e_emit = E0 > w - 1 ? E0 : w - 1;
    const int last = E0 + w - 2;
    int e = E0;
    if (RG && !ensure(e_emit)) return false;
    for (; e < e_emit; ++e) {
      const Wv x = LD(e);
#pragma unroll
      for (int i = 0; i < NWL; ++i) g[i] = cw_op<OP, E>(g[i], cw_of<E>(x.v[i]));
    }
    if (!RG && !col_in) continue;
    // emission of output e-w+1 from the g-prefix and h-suffix; the vector
    // form walks one output pointer down the rows (the branch and the row
    // address stay out of the scan)
    auto emit = [&](const Wv& xe, const Wv& xh) {
      Wv o;
#pragma unroll
      for (int i = 0; i < NWL; ++i) {
        g[i] = cw_op<OP, E>(g[i], cw_of<E>(xe.v[i]));
        o.v[i] = cw_word<E>(cw_op<OP, E>(cw_of<E>(xh.v[i]), g[i]));
      }
      return o;
    };
    if (RG) {
      // every lane runs the same loops (the releases synchronise the
      // warp); only the store differs
      uint8_t* out = a.dst + static_cast<long long>(y0 + e - w + 1) * a.dp + static_cast<long long>(px0) * E;
      for (; e + (kB - 1) <= last; e += kB) {
        if (!ensure(e + kB)) return false;
        Wv xe[kB], xh[kB];
#pragma unroll
        for (int t = 0; t < kB; ++t) {
          xe[t] = LD(e + t);
          xh[t] = LD(e + t - w + 1);
        }
#pragma unroll
        for (int t = 0; t < kB; ++t) {
          const Wv o = emit(xe[t], xh[t]);
          if (fast)
            wd_st<NWL>(out, o);
          else if (col_in)
            store(y0 + e + t - w + 1, o, false);
          out += a.dp;
        }
        release(e + kB - 1);
      }
      for (; e <= last; ++e) {
        if (!ensure(e + 1)) return false;
        const Wv o = emit(LD(e), LD(e - w + 1));
        if (fast)
          wd_st<NWL>(out, o);
        else if (col_in)
          store(y0 + e - w + 1, o, false);
        out += a.dp;
        release(e);
      }
    } else if (fast) {
      uint8_t* out = a.dst + static_cast<long long>(y0 + e - w + 1) * a.dp + static_cast<long long>(px0) * E;
      for (; e + (kB - 1) <= last; e += kB) {
        Wv xe[kB], xh[kB];
#pragma unroll
        for (int t = 0; t < kB; ++t) {
          xe[t] = LD(e + t);
          xh[t] = LD(e + t - w + 1);
        }
#pragma unroll
        for (int t = 0; t < kB; ++t) {
          wd_st<NWL>(out, emit(xe[t], xh[t]));
          out += a.dp;
        }
      }
      for (; e <= last; ++e) {
        wd_st<NWL>(out, emit(LD(e), LD(e - w + 1)));
        out += a.dp;
      }
    } else {
      for (; e <= last; ++e) store(y0 + e - w + 1, emit(LD(e), LD(e - w + 1)), false);
    }
  }
  return true;
}

}  // namespace morph

namespace morph {

// Launch shape of the pass along y: output rows per warp tile (L), warps per
// CTA, shared memory.  A tile of L rows scans L rows backwards and, per block
// it touches, w - 1 rows forwards -- L + ceil(L / w) * (w - 1) row steps,
// fewest per output when L is a multiple of w -- while taller tiles leave
// fewer warps resident, and fewer tiles leave SMs idle.  The default L was
// measured on the GB300 (CUDA-graph timing of 1 x w windows, w from 9 to
// 127, on 2048^2, 4096 x 2048 and 4096^2 images of both pixel types, tile
// heights 9 to 256).  Below 32 rows: the largest multiple of w whose L + w -
// 1 input rows fill one 32-row box (w <= 16) or two.  From 32 rows: for
// 8-bit pixels 2w (at most 256), for 16-bit pixels w itself from 120 rows,
// else 2w (at most 256) from 64 rows, else 64; but if those tiles are fewer
// than 0.6 times the warps resident on the whole GPU, 64 rows, or 32 when 64
// still leaves too few.  Over the 54 measured cases the rule's total is 2%
// above that of the best height per case (the former fixed rule: 17%), and
// no case is more than 14% slower than its best.  Warps per CTA: the choice
// that keeps the most warps resident per SM, the smallest CTA among ties (a
// CTA's shared memory returns only when its last warp ends; 3-4% faster for
// u8 at 51 and 101 rows on the GB300).
struct ColvPlan {
  int L, nbox, wpc, ntask, smem, nwl;
  bool ok;
  int wps;  // warps resident per SM
};

// cap_box > 0: at most that many boxes per warp (the ring form).
inline ColvPlan colv_shape(int esz, int W, int H, int w, int max_smem, int L, int nwl, int cap_box = 0) {
  ColvPlan p{0, 0, 0, 0, 0, nwl, false};
  const int ns = (W * esz + kCvBytes * nwl - 1) / (kCvBytes * nwl);
  int nbox = (L + w - 1 + kCvBox - 1) / kCvBox;
  if (cap_box > 0 && nbox > cap_box) nbox = cap_box;
  if (nbox > kCvMaxBox) return p;
  int wpc = 0, wps = 0;
  for (int c = 1; c <= 4; c *= 2) {
    if (colv_smem_bytes(nbox, c, nwl) > max_smem) continue;
    int ctas = 233472 / (colv_smem_bytes(nbox, c, nwl) + 1024);
    if (ctas > 32) ctas = 32;
    if (ctas * c > 64) ctas = 64 / c;
    if (ctas * c > wps) {
      wps = ctas * c;
      wpc = c;
    }
  }
  if (wpc == 0) return p;
  const long long ntask = static_cast<long long>(ns) * ((H + L - 1) / L);
  if (ntask > (1ll << 30)) return p;
  return ColvPlan{L, nbox, wpc, static_cast<int>(ntask), colv_smem_bytes(nbox, wpc, nwl), nwl, true, wps};
}

inline int colv_default_rows(int esz, int w) {
  if (w < 32) {
    const int rows = w <= 16 ? kCvBox : 2 * kCvBox;  // input rows of the tile
    const int k = (rows - w + 1) / w;
    return w * (k > 1 ? k : 1);
  }
  const int two = 2 * w < 256 ? 2 * w : 256;
  if (esz == 1) return w >= 32 ? two : 64;
  if (w >= 120 && w <= 256) return w;
  return w >= 64 ? two : 64;
}

// nwl: 32-bit words per lane (1, or 2 for strips 256 bytes wide).
// sms: the GPU's SM count for the rule on too few tiles (0: rule off).
inline ColvPlan colv_plan(int esz, int W, int H, int w, int max_smem, int forced_L, int nwl = 1, int sms = 0) {
  ColvPlan p{0, 0, 0, 0, 0, nwl, false, 0};
  if (w < 2 || W < 1 || H < 1) return p;
  const int hmax = H < 1024 ? H : 1024;
  auto fit = [&](int L) {
    if (L > hmax) L = hmax;
    ColvPlan q{0, 0, 0, 0, 0, nwl, false, 0};
    // very long windows: shorter tiles until one fits
    for (; L >= 1; L -= 8) {
      q = colv_shape(esz, W, H, w, max_smem, L, nwl);
      if (q.ok) break;
    }
    return q;
  };
  if (forced_L > 0) return fit(forced_L);
  p = fit(colv_default_rows(esz, w));
  if (w < 32 || sms <= 0) return p;
  auto enough = [&](const ColvPlan& q) { return q.ok && 5ll * q.ntask >= 3ll * sms * q.wps; };
  if (!p.ok || enough(p)) return p;
  for (int L : {64, 32}) {
    const ColvPlan q = fit(L);
    if (!q.ok) continue;
    p = q;
    if (enough(q)) break;
  }
  return p;
}


// The ring form's plan: nring = ceil((w + 39) / 32) + 1 boxes per warp
// (see colv_tile), tiles of L = k w rows (whole blocks), k the largest of 1
// .. 8 (L <= 1024) whose tiles still give at least 0.6 x the warps resident
// on the whole GPU; forced_L > 0 overrides.  Needs TMA-loaded rows.
inline int colv_ring_boxes(int w) { return (w + 39 + kCvBox - 1) / kCvBox + 1; }
inline ColvPlan colv_ring_plan(int esz, int W, int H, int w, int max_smem, int forced_L, int sms) {
  ColvPlan p{0, 0, 0, 0, 0, 1, false, 0};
  if (w < 2 || W < 1 || H < 1) return p;
  const int nr = colv_ring_boxes(w);
  const int hmax = H < 1024 ? H : 1024;
  if (forced_L > 0) return colv_shape(esz, W, H, w, max_smem, forced_L < hmax ? forced_L : hmax, 1, nr);
  p = colv_shape(esz, W, H, w, max_smem, w < hmax ? w : hmax, 1, nr);
  if (!p.ok || sms <= 0) return p;
  for (int k = 8; k >= 2; --k) {
    const int L = k * w;
    if (L > hmax) continue;
    const ColvPlan q = colv_shape(esz, W, H, w, max_smem, L, 1, nr);
    if (q.ok && 5ll * q.ntask >= 3ll * sms * q.wps) return q;
  }
  return p;
}

}  // namespace morph

namespace morph {

// ---------------------------------------------------------------------------
// Shared-tile form for long windows (w > LW): the warps of a CTA share one
// input tile -- NW x LW output rows of a 128-byte strip plus the window's
// w - 1 halo rows, loaded once -- and each warp keeps the block suffix of its
// LW output rows in registers instead of writing it over the input.  With
// w > LW a warp's LW outputs start their windows inside one block of w rows
// (the partial block at the top of its tile), so
//   h-scan  rows LW-1 .. 0 into registers h[0..LW-1]
//   g-scan  rows LW .. LW+w-2; row w-1+o closes output o = op(h[o], g).
// Sharing the halo rows lets about twice as many warps stay resident per SM
// as the in-place form, and loads each halo row once per CTA.
// ---------------------------------------------------------------------------
struct ColwArgs {
  const uint8_t* src;
  uint8_t* dst;
  long long sp, dp;
  int W, H;
  int w, a;    // window (w > LW) and anchor, clipped to the image
  int nw;      // warps per CTA (output rows per CTA: nw * LW)
  int nbox;    // 32-row boxes per CTA tile: ceil((nw * LW + w - 1) / 32)
  int ns;      // strips across
  int ntile;   // CTA tiles: ns * ceil(H / (nw * LW))
  int st_vec;  // 1: rows allow aligned 32-bit stores
  int* err;
};

__host__ __device__ inline int colw_smem_bytes(int nbox) { return nbox * kCvBoxBytes + nbox * 8; }

// One warp of a CTA tile.  tile: the CTA's input tile; bars: its nbox
// mbarriers (count 1), the boxes issued by the CTA's thread 0.  False when a
// bounded wait gave up.
template <typename T, int OP, int LW>
__device__ __forceinline__ bool colw_warp(const ColwArgs& a, int ctile, int warp, int lane, const uint8_t* tile,
                                          uint64_t* bars) {
  constexpr int E = sizeof(T), PPW = 4 / E;
  using C = Cw<E>;
  const uint32_t IDW = ident_word<OP>();
  const int s = ctile % a.ns;
  const int yc = (ctile / a.ns) * (a.nw * LW);  // first output row of the CTA tile
  const int y0 = yc + warp * LW;                // this warp's first output row
  if (y0 >= a.H) return true;
  const int w = a.w;
  const int ysc = yc - a.a;                     // image row of CTA tile row 0
  const int r0 = warp * LW;                     // this warp's tile row 0
  const int px0 = s * (kCvBytes / E) + lane * PPW;
  const bool col_in = px0 < a.W;
  const bool fast = a.st_vec && px0 + PPW <= a.W;
  const uint8_t* col = tile + 4 * lane;
  // rows outside the image read as the identity (TMA fills them with 0)
  const bool edge = ysc + r0 < 0 || ysc + r0 + LW + w - 1 > a.H;
  auto LD = [&](int r) -> uint32_t {  // r: row of this warp's tile
    const uint32_t v = *reinterpret_cast<const uint32_t*>(col + (r0 + r) * kCvBytes);
    if (!edge) return v;
    const int y = ysc + r0 + r;
    return (y < 0 || y >= a.H) ? IDW : v;
  };
  int have = 0;
  auto ensure = [&](int rows) -> bool {  // this warp's tile rows [0, rows) landed
    const int need = (r0 + rows + kCvBox - 1) / kCvBox;
    for (; have < need; ++have)
      if (!mbar_wait_bounded(&bars[have], 0)) {
        if (lane == 0) atomicExch(a.err, kDevErrTmaTimeout);
        return false;
      }
    return true;
  };
  C IDC;
#pragma unroll
  for (int i = 0; i < (E == 1 ? 2 : 1); ++i) IDC.v[i] = IDW;

  // h-scan into registers
  if (!ensure(LW)) return false;
  uint32_t h[LW];
  {
    C acc = IDC;
#pragma unroll
    for (int t = LW - 1; t >= 0; --t) {
      acc = cw_op<OP, E>(acc, cw_of<E>(LD(t)));
      h[t] = cw_word<E>(acc);
    }
  }
  // g-scan: rows LW .. w-2 emit nothing
  C g = IDC;
  int e = LW;
  constexpr int kB = 8;
  for (; e + kB <= w - 1; e += kB) {
    if (!ensure(e + kB)) return false;
    uint32_t x[kB];
#pragma unroll
    for (int t = 0; t < kB; ++t) x[t] = LD(e + t);
#pragma unroll
    for (int t = 0; t < kB; ++t) g = cw_op<OP, E>(g, cw_of<E>(x[t]));
  }
  for (; e < w - 1; ++e) {
    if (!ensure(e + 1)) return false;
    g = cw_op<OP, E>(g, cw_of<E>(LD(e)));
  }
  // rows w-1 .. w-2+LW close outputs 0 .. LW-1
  const int nout = a.H - y0 < LW ? a.H - y0 : LW;
  if (!ensure(w - 1 + LW)) return false;
  uint8_t* out = a.dst + static_cast<long long>(y0) * a.dp + static_cast<long long>(px0) * E;
#pragma unroll
  for (int o0 = 0; o0 < LW; o0 += kB) {
    uint32_t x[kB];
#pragma unroll
    for (int t = 0; t < kB; ++t) x[t] = LD(w - 1 + o0 + t);
#pragma unroll
    for (int t = 0; t < kB; ++t) {
      const int o = o0 + t;
      g = cw_op<OP, E>(g, cw_of<E>(x[t]));
      const uint32_t v = cw_word<E>(cw_op<OP, E>(cw_of<E>(h[o]), g));
      if (col_in && o < nout) {
        if (fast) {
          *reinterpret_cast<uint32_t*>(out + static_cast<long long>(o) * a.dp) = v;
        } else {
          T* row = reinterpret_cast<T*>(a.dst + static_cast<long long>(y0 + o) * a.dp);
#pragma unroll
          for (int q = 0; q < PPW; ++q)
            if (px0 + q < a.W) row[px0 + q] = static_cast<T>(v >> (8 * E * q));
        }
      }
    }
  }
  return true;
}

// Launch shape of the shared-tile form: warps per CTA (1..8) so that the
// CTA tiles come closest to filling whole waves of resident CTAs, preferring
// more warps (fewer halo rows per output).
struct ColwPlan {
  int nw, nbox, ntile, smem;
  bool ok;
};
inline ColwPlan colw_plan(int esz, int W, int H, int w, int LW, int sms, int max_smem, int max_warps) {
  ColwPlan best{0, 0, 0, 0, false};
  if (w <= LW || sms < 1) return best;
  const int ns = (W * esz + kCvBytes - 1) / kCvBytes;
  double best_cost = 1e300;
  for (int nw = 8; nw >= 1; --nw) {
    const int rows = nw * LW + w - 1;
    const int nbox = (rows + kCvBox - 1) / kCvBox;
    const int smem = colw_smem_bytes(nbox);
    if (smem > max_smem) continue;
    int ctas = 233472 / (smem + 1024);
    if (ctas > 32) ctas = 32;
    if (ctas * nw > max_warps) ctas = max_warps / nw;  // registers
    if (ctas < 1) continue;
    const long long ntile = static_cast<long long>(ns) * ((H + nw * LW - 1) / (nw * LW));
    const double waves = static_cast<double>((ntile + static_cast<long long>(sms) * ctas - 1) /
                                             (static_cast<long long>(sms) * ctas));
    // per-CTA time ~ its warps' scans (LW + w - 1 rows each, in parallel)
    // plus its load (rows) spread over the SM; prefer fewer waves
    const double cost = waves * (LW + w - 1 + 0.25 * rows / nw * ctas / 4.0);
    if (cost < best_cost) {
      best_cost = cost;
      best = ColwPlan{nw, nbox, static_cast<int>(ntile), smem, true};
    }
  }
  return best;
}

}  // namespace morph
