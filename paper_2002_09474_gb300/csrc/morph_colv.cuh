// Pass along y (a 1 x w element; the paper's "horizontal pass", section 5.1)
// by van Herk/Gil-Werman (section 5.1.1) with blocks of w rows, one warp per
// work item.
//
// A warp owns a strip of 32 lanes x LB bytes (lane l: bytes LB l .. LB l +
// LB - 1 of every row; LB = 4 by default, 8 for two words per lane) and L
// consecutive output rows.  Its
// L + w - 1 input rows arrive in shared memory as TMA boxes of 32 rows, each
// on its own mbarrier, all issued when the warp starts; the scans begin as
// soon as the first boxes land.  Warps never share shared memory and never
// synchronise: lanes touch only their own column.
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
// the low bytes hold.  A 32-bit word of four pixels is carried as the raw
// word (pixels 1 and 3 in the high bytes) and the word shifted left by 8
// (pixels 0 and 2); one byte permute puts the four results back together.
// 16-bit pixels use the raw word.
#pragma once

#include "morph_common.cuh"

namespace morph {

constexpr int kCvBox = 32;     // rows per TMA box
constexpr int kCvMaxBox = 56;  // boxes per warp tile at most (1792 rows)

struct ColvArgs {
  const uint8_t* src;
  uint8_t* dst;
  long long sp, dp;  // pitches in bytes
  int W, H;          // pixels
  int w, a;          // window along y and its anchor, clipped to the image
  int L;             // output rows per warp tile
  int nbox;          // shared-memory boxes per warp tile: ceil((L + w - 1) / 32)
  int ns;            // strips across: ceil(W * esz / strip bytes)
  int ntask;         // warp tiles: ns * ceil(H / L)
  int wpc;           // warps per CTA
  int tma_ld;        // 1: input boxes arrive by TMA
  int ld_vec;        // 1: rows allow aligned loads of a lane's bytes
  int st_vec;        // 1: rows allow aligned stores of a lane's bytes
  int* err;          // device error word
};

// Strip bytes of a lane width, shared memory of one CTA: wpc warp tiles
// (boxes of 32 rows of 32 * lb bytes), then wpc * nbox mbarriers.
__host__ __device__ constexpr int colv_strip_bytes(int lb) { return 32 * lb; }
__host__ __device__ inline int colv_tile_bytes(int nbox, int lb = 4) { return nbox * kCvBox * colv_strip_bytes(lb); }
__host__ __device__ inline int colv_smem_bytes(int nbox, int wpc, int lb = 4) {
  return wpc * colv_tile_bytes(nbox, lb) + wpc * nbox * 8;
}

// 16-bit-lane carriers of one word: u8: odd pixels in v[0], even pixels in
// v[1]; u16: the word itself.
template <int E>
struct Cw {
  static constexpr int N = E == 1 ? 2 : 1;
  uint32_t v[N];
};

template <int E>
__device__ __forceinline__ Cw<E> cw_of(uint32_t raw) {
  Cw<E> c;
  c.v[0] = raw;
  if (E == 1) c.v[Cw<E>::N - 1] = raw << 8;
  return c;
}
template <int E>
__device__ __forceinline__ uint32_t cw_word(const Cw<E>& c) {
  // bytes: even.b1 (pixel 0), odd.b1 (pixel 1), even.b3 (pixel 2), odd.b3 (pixel 3)
  if (E == 1) return __byte_perm(c.v[Cw<E>::N - 1], c.v[0], 0x7351);
  return c.v[0];
}
template <int OP, int E>
__device__ __forceinline__ Cw<E> cw_op(const Cw<E>& a, const Cw<E>& b) {
  Cw<E> r;
#pragma unroll
  for (int i = 0; i < Cw<E>::N; ++i) r.v[i] = OP == 0 ? __vminu2(a.v[i], b.v[i]) : __vmaxu2(a.v[i], b.v[i]);
  return r;
}

// A lane's bytes of one row: LB = 4 (one word) or 8 (two).
template <int LB>
struct Wd {
  static constexpr int N = LB / 4;
  uint32_t v[N];
};
template <int LB>
__device__ __forceinline__ Wd<LB> wd_ld(const uint8_t* p) {
  Wd<LB> w;
  if (LB == 8) {
    const uint2 u = *reinterpret_cast<const uint2*>(p);
    w.v[0] = u.x;
    w.v[Wd<LB>::N - 1] = u.y;
  } else {
    w.v[0] = *reinterpret_cast<const uint32_t*>(p);
  }
  return w;
}
template <int LB>
__device__ __forceinline__ void wd_st(uint8_t* p, const Wd<LB>& w) {
  if (LB == 8)
    *reinterpret_cast<uint2*>(p) = make_uint2(w.v[0], w.v[Wd<LB>::N - 1]);
  else
    *reinterpret_cast<uint32_t*>(p) = w.v[0];
}

// One warp tile.  tile: this warp's shared memory (nbox boxes of 32 rows of
// 32 * LB bytes); bars: its nbox mbarriers, initialised with count 1.
// lane: 0..31, owning bytes LB lane .. LB lane + LB - 1 of each row of the
// strip.  Two words per lane give each lane two independent scan chains.
// Returns false when a bounded wait gave up (error word set by lane 0).
template <typename T, int OP, int LB = 4>
__device__ __forceinline__ bool colv_tile(const ColvArgs& a, const CUtensorMap* tin, int task, int lane,
                                          uint8_t* tile, uint64_t* bars) {
  constexpr int E = sizeof(T);
  static_assert(LB == 4 || LB == 8, "4 or 8 bytes per lane");
  constexpr int NW = Wd<LB>::N;                // words per lane
  constexpr int PPW = 4 / E;                   // pixels per word
  constexpr int SB = colv_strip_bytes(LB), BOXB = SB * kCvBox;  // strip bytes, box bytes
  using C = Cw<E>;
  using Wv = Wd<LB>;
  const uint32_t IDW = ident_word<OP>();
  const int s = task % a.ns;                  // strip
  const int y0 = (task / a.ns) * a.L;         // first output row
  const int Lr = a.L < a.H - y0 ? a.L : a.H - y0;  // output rows of this tile
  const int w = a.w;
  const int ys = y0 - a.a;                    // image row of tile row 0
  const int nin = Lr + w - 1;                 // input rows
  const int nb = (nin + kCvBox - 1) / kCvBox;  // boxes to fill
  const int px0 = s * (SB / E) + lane * (LB / E);  // the lane's first pixel
  const bool col_in = px0 < a.W;
  const bool fast = a.st_vec && px0 + LB / E <= a.W;
  uint8_t* col = tile + LB * lane;

  auto rowp = [&](int r) { return col + r * SB; };
  auto LD = [&](int r) { return wd_ld<LB>(rowp(r)); };
  auto ST = [&](int r, const Wv& v) { wd_st<LB>(rowp(r), v); };
  Wv IDV;
#pragma unroll
  for (int i = 0; i < NW; ++i) IDV.v[i] = IDW;

  int have = 0;  // boxes landed (and fixed up)
  if (a.tma_ld) {
    if (lane == 0) {
      fence_proxy_async_smem();
      for (int b = 0; b < nb; ++b) {
        mbar_arrive_expect_tx(&bars[b], static_cast<uint32_t>(BOXB));
        tma_load_2d(tile + b * BOXB, tin, &bars[b], s * (SB / E), ys + b * kCvBox);
      }
    }
  } else {
    for (int r = 0; r < nin; ++r) {
      const int y = ys + r;
      Wv v = IDV;
      if (y >= 0 && y < a.H) {
        const uint8_t* row = a.src + static_cast<long long>(y) * a.sp;
#pragma unroll
        for (int i = 0; i < NW; ++i) {
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
      if (!mbar_wait_bounded(&bars[have], 0u)) {
        if (lane == 0) {
          atomicExch(a.err, kDevErrTmaTimeout);
          for (int b = have + 1; b < nb; ++b) mbar_wait_bounded(&bars[b], 0u);  // let copies in flight land
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
  // stores output row y from the lane's words
  auto store = [&](int y, const Wv& v, bool vec) {
    uint8_t* row = a.dst + static_cast<long long>(y) * a.dp;
    if (vec) {
      wd_st<LB>(row + static_cast<long long>(px0) * E, v);
    } else {
#pragma unroll
      for (int i = 0; i < NW; ++i)
#pragma unroll
        for (int t = 0; t < PPW; ++t)
          if (px0 + i * PPW + t < a.W)
            reinterpret_cast<T*>(row)[px0 + i * PPW + t] = static_cast<T>(v.v[i] >> (8 * E * t));
    }
  };

  // Rows move between shared memory and registers 8 at a time: the 8 loads
  // of a batch issue together, so a scan waits for shared-memory latency
  // once per batch rather than once per row (the in-place stores of the
  // h-scan would otherwise order every load after the previous store).
  constexpr int kB = 8;
  C IDC;
#pragma unroll
  for (int i = 0; i < C::N; ++i) IDC.v[i] = IDW;
  const int beta = Lr % w;
  for (int E0 = beta ? beta : w; E0 <= Lr; E0 += w) {
    const int lo = E0 - w > 0 ? E0 - w : 0;
    if (!ensure(E0 + w - 1)) return false;
    // h-scan, rows E0-1 down to lo, in place
    C h[NW];
#pragma unroll
    for (int i = 0; i < NW; ++i) h[i] = IDC;
    int r = E0 - 1;
    for (; r - (kB - 1) >= lo; r -= kB) {
      Wv x[kB];
#pragma unroll
      for (int t = 0; t < kB; ++t) x[t] = LD(r - t);
#pragma unroll
      for (int t = 0; t < kB; ++t)
#pragma unroll
        for (int i = 0; i < NW; ++i) {
          h[i] = cw_op<OP, E>(h[i], cw_of<E>(x[t].v[i]));
          x[t].v[i] = cw_word<E>(h[i]);
        }
#pragma unroll
      for (int t = 0; t < kB; ++t) ST(r - t, x[t]);
    }
    for (; r >= lo; --r) {
      Wv x = LD(r);
#pragma unroll
      for (int i = 0; i < NW; ++i) {
        h[i] = cw_op<OP, E>(h[i], cw_of<E>(x.v[i]));
        x.v[i] = cw_word<E>(h[i]);
      }
      ST(r, x);
    }
    if (E0 - w >= 0 && col_in) {
      Wv o;
#pragma unroll
      for (int i = 0; i < NW; ++i) o.v[i] = cw_word<E>(h[i]);
      store(y0 + E0 - w, o, fast);
    }
    // g-scan over rows E0 .. E0+w-2; row e closes the window of output
    // e-w+1, so rows before w-1 (a partial first block only) emit nothing
    C g[NW];
#pragma unroll
    for (int i = 0; i < NW; ++i) g[i] = IDC;
    const int e_emit = E0 > w - 1 ? E0 : w - 1;
    const int last = E0 + w - 2;
    int e = E0;
    for (; e < e_emit; ++e) {
      const Wv x = LD(e);
#pragma unroll
      for (int i = 0; i < NW; ++i) g[i] = cw_op<OP, E>(g[i], cw_of<E>(x.v[i]));
    }
    if (!col_in) continue;
    // emission of output e-w+1 from the g-prefix and h-suffix; the vector
    // form walks one output pointer down the rows (the branch and the row
    // address stay out of the scan)
    auto emit = [&](const Wv& xe, const Wv& xh) {
      Wv o;
#pragma unroll
      for (int i = 0; i < NW; ++i) {
        g[i] = cw_op<OP, E>(g[i], cw_of<E>(xe.v[i]));
        o.v[i] = cw_word<E>(cw_op<OP, E>(cw_of<E>(xh.v[i]), g[i]));
      }
      return o;
    };
    if (fast) {
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
          wd_st<LB>(out, emit(xe[t], xh[t]));
          out += a.dp;
        }
      }
      for (; e <= last; ++e) {
        wd_st<LB>(out, emit(LD(e), LD(e - w + 1)));
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
  int L, nbox, wpc, ntask, smem, lb;
  bool ok;
  int wps;  // warps resident per SM
};

// lb: bytes per lane (4 or 8).
inline ColvPlan colv_shape(int esz, int W, int H, int w, int max_smem, int L, int lb) {
  ColvPlan p{0, 0, 0, 0, 0, lb, false};
  const int sb = colv_strip_bytes(lb);
  const int ns = (W * esz + sb - 1) / sb;
  const int nbox = (L + w - 1 + kCvBox - 1) / kCvBox;
  if (nbox > kCvMaxBox) return p;
  int wpc = 0, wps = 0;
  for (int c = 1; c <= 4; c *= 2) {
    if (colv_smem_bytes(nbox, c, lb) > max_smem) continue;
    int ctas = 233472 / (colv_smem_bytes(nbox, c, lb) + 1024);
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
  return ColvPlan{L, nbox, wpc, static_cast<int>(ntask), colv_smem_bytes(nbox, wpc, lb), lb, true, wps};
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

// lb: bytes per lane (4; 8 for strips 256 bytes wide).  sms: the GPU's SM count for the rule on too
// few tiles (0: rule off).
inline ColvPlan colv_plan(int esz, int W, int H, int w, int max_smem, int forced_L, int lb = 4, int sms = 0) {
  ColvPlan p{0, 0, 0, 0, 0, lb, false, 0};
  if (w < 2 || W < 1 || H < 1) return p;
  const int hmax = H < 1024 ? H : 1024;
  auto fit = [&](int L) {
    if (L > hmax) L = hmax;
    ColvPlan q{0, 0, 0, 0, 0, lb, false, 0};
    // very long windows: shorter tiles until one fits
    for (; L >= 1; L -= 8) {
      q = colv_shape(esz, W, H, w, max_smem, L, lb);
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


}  // namespace morph

