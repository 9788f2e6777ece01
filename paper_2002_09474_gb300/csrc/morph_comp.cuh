// Opening, closing and the morphological gradient in one pass over the image
// (section 2: operations built from erosion, dilation and arithmetic), for
// windows of at most kCompMaxW pixels a side, each 1-D pass by the direct
// method (sections 5.1.2 and 5.2.2).  One CTA loads its output tile and the
// halo both steps need, runs the four 1-D passes (or, for the gradient, the
// min and the max of two) in shared memory, and writes the tile: each pixel
// crosses HBM once in and once out, where two calls move the intermediate
// image out and back in.
//
// Pixels live in shared memory as 16-bit lanes, two per 32-bit word (pixel
// pairs 2k, 2k+1 of a region row), so one __vminu2/__vmaxu2 handles two
// pixels of either type.  Region rows have kCompRowW words.
//
// Edges: the first step reads the image with clamped coordinates (the
// nearest in-image pixel), which for a min or max over a window that
// contains an in-image pixel is the same as leaving out-of-image pixels out.
// The intermediate image of an opening or closing has no pixels outside the
// image, so its out-of-image positions are set to the second step's
// identity before that step reads them.
#pragma once

#include <cstdint>

#include "morph_common.cuh"

namespace morph {

constexpr int kCompMaxW = 9;               // largest window side
constexpr int kCompHalo = kCompMaxW - 1;   // largest halo on one side
constexpr int kCompTX = 128;               // output tile, pixels (even)
constexpr int kCompTY = 32;
constexpr int kCompThreads = 256;
constexpr int kCompRowW = (kCompTX + 2 * kCompHalo) / 2;  // words per region row
constexpr int kCompInRows = kCompTY + 2 * kCompHalo;       // input region rows
constexpr int kCompMidRows = kCompTY + kCompHalo;          // rows after the first pass along y
constexpr int kCompSmemWords = kCompRowW * (kCompInRows + kCompMidRows + kCompTY);
enum { kCompOpen = 0, kCompClose = 1, kCompGradient = 2 };

struct CompArgs {
  const uint8_t* src;
  uint8_t* dst;
  long long sp, dp;    // bytes per row
  int W, H;
  int wx, wy, ax, ay;  // the element and the first step's anchor (the gradient's only one)
  int tiles_x;         // tiles per image row
};

template <int OP> __device__ __forceinline__ uint32_t comp_op(uint32_t a, uint32_t b) {
  return OP == 0 ? __vminu2(a, b) : __vmaxu2(a, b);
}

// Region rows [ry, ry + nrows), pixels [rx, rx + 2 nw) into buf, each pixel
// the image's at the clamped coordinates.  Warp w takes rows w, w + 8, ...;
// every load of a thread is issued before its first store, so that they are
// all in flight together (a store between them would order each load after
// it).
template <typename T>
__device__ __forceinline__ void comp_load(const CompArgs& a, int rx, int ry, int nw, int nrows, uint32_t* buf,
                                          int tid) {
  constexpr int RPW = (kCompInRows + kCompThreads / 32 - 1) / (kCompThreads / 32);  // rows per warp
  constexpr int KPL = (kCompRowW + 31) / 32;                                       // words per lane and row
  const int warp = tid >> 5, lane = tid & 31;
  const bool inside = rx >= 0 && rx + 2 * nw <= a.W;  // no column clamping in this region
  uint32_t v[RPW][KPL];
#pragma unroll
  for (int i = 0; i < RPW; ++i) {
    const int r = warp + i * (kCompThreads / 32);
    if (r >= nrows) continue;
    int gy = ry + r;
    gy = gy < 0 ? 0 : (gy >= a.H ? a.H - 1 : gy);
    const T* row = reinterpret_cast<const T*>(a.src + static_cast<long long>(gy) * a.sp);
#pragma unroll
    for (int j = 0; j < KPL; ++j) {
      const int k = lane + 32 * j;
      if (k >= nw) continue;
      int g0 = rx + 2 * k, g1 = g0 + 1;
      if (!inside) {
        g0 = g0 < 0 ? 0 : (g0 >= a.W ? a.W - 1 : g0);
        g1 = g1 < 0 ? 0 : (g1 >= a.W ? a.W - 1 : g1);
      }
      v[i][j] = static_cast<uint32_t>(row[g0]) | (static_cast<uint32_t>(row[g1]) << 16);
    }
  }
#pragma unroll
  for (int i = 0; i < RPW; ++i) {
    const int r = warp + i * (kCompThreads / 32);
    if (r >= nrows) continue;
#pragma unroll
    for (int j = 0; j < KPL; ++j) {
      const int k = lane + 32 * j;
      if (k < nw) buf[r * kCompRowW + k] = v[i][j];
    }
  }
}

// The loops over a window below run to HB, a compile-time bound on the
// halo (2, 4 or 8): the compiler unrolls them, and a step beyond the actual
// halo h is a predicated instruction that still issues, so the bound is
// kept close to h.

// Pass along y: out[r][k] = op(in[r .. r + h][k]), rows r in [0, nout),
// every word of the row (those past the region's compute unused values
// inside the buffer).  A thread makes 8 consecutive rows of one word from
// 8 + h loaded rows.  Reads rows up to 8 ceil(nout / 8) + h - 1 of `in`.
template <int OP, int HB>
__device__ __forceinline__ void comp_ypass(const uint32_t* in, uint32_t* out, int nout, int h, int tid) {
  constexpr int R = 8;
  const int items = (nout + R - 1) / R * kCompRowW;
  for (int i = tid; i < items; i += kCompThreads) {
    const int g = i / kCompRowW, k = i - g * kCompRowW, r0 = g * R;
    uint32_t v[R + HB];
#pragma unroll
    for (int j = 0; j < R + HB; ++j)
      if (j < R + h) v[j] = in[(r0 + j) * kCompRowW + k];
#pragma unroll
    for (int rr = 0; rr < R; ++rr) {
      uint32_t acc = v[rr];
#pragma unroll
      for (int d = 1; d <= HB; ++d)
        if (d <= h) acc = comp_op<OP>(acc, v[rr + d]);
      if (r0 + rr < nout) out[(r0 + rr) * kCompRowW + k] = acc;
    }
  }
}

// The gradient's pass along y: the min of the same rows into lo, the max
// into hi.
template <int HB>
__device__ __forceinline__ void comp_ypass_minmax(const uint32_t* in, uint32_t* lo, uint32_t* hi, int nout, int h,
                                                  int tid) {
  constexpr int R = 8;
  const int items = (nout + R - 1) / R * kCompRowW;
  for (int i = tid; i < items; i += kCompThreads) {
    const int g = i / kCompRowW, k = i - g * kCompRowW, r0 = g * R;
    uint32_t v[R + HB];
#pragma unroll
    for (int j = 0; j < R + HB; ++j)
      if (j < R + h) v[j] = in[(r0 + j) * kCompRowW + k];
#pragma unroll
    for (int rr = 0; rr < R; ++rr) {
      uint32_t mn = v[rr], mx = v[rr];
#pragma unroll
      for (int d = 1; d <= HB; ++d)
        if (d <= h) {
          mn = __vminu2(mn, v[rr + d]);
          mx = __vmaxu2(mx, v[rr + d]);
        }
      if (r0 + rr < nout) {
        lo[(r0 + rr) * kCompRowW + k] = mn;
        hi[(r0 + rr) * kCompRowW + k] = mx;
      }
    }
  }
}

// Pass along x of one word: pixels (2k, 2k+1) of a region row folded over
// pixels (2k + d, 2k + 1 + d), d in [0, h]; reads words k .. k + (h+1)/2.
template <int OP, int HB>
__device__ __forceinline__ uint32_t comp_xword(const uint32_t* row, int h) {
  uint32_t w[HB / 2 + 1];
#pragma unroll
  for (int j = 0; j <= HB / 2; ++j)
    if (2 * j <= h + 1) w[j] = row[j];
  uint32_t acc = w[0];
#pragma unroll
  for (int d = 1; d <= HB; ++d)
    if (d <= h) acc = comp_op<OP>(acc, (d & 1) ? __byte_perm(w[d >> 1], w[(d >> 1) + 1], 0x5432) : w[d >> 1]);
  return acc;
}

// The first step's pass along x into the intermediate region (nrows rows,
// nwo words), whose pixel (row r, pixel i) is the image's (xb + i, yb + r):
// positions outside the image get the identity of the second step (OP2).
template <int OP1, int OP2, int HB>
__device__ __forceinline__ void comp_xpass_mid(const CompArgs& a, const uint32_t* in, uint32_t* out, int nrows,
                                               int nwo, int h, int xb, int yb, int tid) {
  const int warp = tid >> 5, lane = tid & 31;
  const uint32_t id2 = ident_word<OP2>();
  // the whole region inside the image (most tiles): nothing to mask
  const bool all_in = xb >= 0 && xb + 2 * nwo <= a.W && yb >= 0 && yb + nrows <= a.H;
  for (int r = warp; r < nrows; r += kCompThreads / 32) {
    const int gy = yb + r;
    const bool row_in = gy >= 0 && gy < a.H;
    for (int k = lane; k < nwo; k += 32) {
      uint32_t v = comp_xword<OP1, HB>(in + r * kCompRowW + k, h);
      const int gx = xb + 2 * k;
      if (all_in) {
      } else if (!row_in) {
        v = id2;
      } else {
        if (gx < 0 || gx >= a.W) v = (v & 0xFFFF0000u) | (id2 & 0x0000FFFFu);
        if (gx + 1 < 0 || gx + 1 >= a.W) v = (v & 0x0000FFFFu) | (id2 & 0xFFFF0000u);
      }
      out[r * kCompRowW + k] = v;
    }
  }
}

// Writes result word v (pixels x, x + 1) into image row `row` where inside
// (x is even; pair: the row's pixel pairs start at even addresses of their
// size, so a u8 pair is one 16-bit store and a u16 pair one 32-bit store).
template <typename T>
__device__ __forceinline__ void comp_store(const CompArgs& a, T* row, bool pair, int x, uint32_t v) {
  if (x >= a.W) return;
  if (pair && x + 1 < a.W) {
    if (sizeof(T) == 1)
      *reinterpret_cast<uint16_t*>(row + x) = static_cast<uint16_t>((v & 0xFFu) | ((v >> 8) & 0xFF00u));
    else
      *reinterpret_cast<uint32_t*>(row + x) = v;
    return;
  }
  row[x] = static_cast<T>(v & 0xFFFFu);
  if (x + 1 < a.W) row[x + 1] = static_cast<T>(v >> 16);
}

// Row y of the output (nullptr when below the image) and whether its pixel
// pairs are aligned for one store each.
template <typename T>
__device__ __forceinline__ T* comp_row(const CompArgs& a, int y, bool* pair) {
  if (y >= a.H) return nullptr;
  T* row = reinterpret_cast<T*>(a.dst + static_cast<long long>(y) * a.dp);
  *pair = !(reinterpret_cast<uintptr_t>(row) & (2 * sizeof(T) - 1));
  return row;
}

// One output tile.  smem: kCompSmemWords words.  HB >= both halos.
template <typename T, int KIND, int HB>
__device__ __forceinline__ void comp_tile(const CompArgs& a, int tile, int tid, uint32_t* smem) {
  uint32_t* s_in = smem;
  uint32_t* s_mid = smem + kCompRowW * kCompInRows;
  uint32_t* s_out = s_mid + kCompRowW * kCompMidRows;
  const int x0 = (tile % a.tiles_x) * kCompTX, y0 = (tile / a.tiles_x) * kCompTY;
  const int hx = a.wx - 1, hy = a.wy - 1;
  const int warp = tid >> 5, lane = tid & 31;
  constexpr int kOutW = kCompTX / 2;
  if (KIND == kCompGradient) {
    // both results from one region: rows y0 - ay .., pixels x0 - ax ..
    comp_load<T>(a, x0 - a.ax, y0 - a.ay, (kCompTX + hx + 1) / 2, kCompTY + hy, s_in, tid);
    __syncthreads();
    comp_ypass_minmax<HB>(s_in, s_mid, s_out, kCompTY, hy, tid);
    __syncthreads();
    for (int r = warp; r < kCompTY; r += kCompThreads / 32) {
      bool pair = false;
      T* row = comp_row<T>(a, y0 + r, &pair);
      if (!row) continue;
#pragma unroll
      for (int k = lane; k < kOutW; k += 32) {
        const uint32_t mn = comp_xword<0, HB>(s_mid + r * kCompRowW + k, hx);
        const uint32_t mx = comp_xword<1, HB>(s_out + r * kCompRowW + k, hx);
        comp_store<T>(a, row, pair, x0 + 2 * k, __vsub2(mx, mn));  // mx >= mn in both lanes
      }
    }
    return;
  }
  constexpr int OP1 = KIND == kCompOpen ? 0 : 1, OP2 = 1 - OP1;
  // input region rows y0 - hy .., pixels x0 - hx ..; the intermediate's
  // region starts at (x0 - hx + ax, y0 - hy + ay), its pixel (r, i) the first
  // step over input pixels i .. i + hx of rows r .. r + hy
  const int nw_in = (kCompTX + 2 * hx + 1) / 2, nw_mid = (kCompTX + hx + 1) / 2;
  comp_load<T>(a, x0 - hx, y0 - hy, nw_in, kCompTY + 2 * hy, s_in, tid);
  __syncthreads();
  comp_ypass<OP1, HB>(s_in, s_mid, kCompTY + hy, hy, tid);
  __syncthreads();
  comp_xpass_mid<OP1, OP2, HB>(a, s_mid, s_in, kCompTY + hy, nw_mid, hx, x0 - hx + a.ax, y0 - hy + a.ay, tid);
  __syncthreads();
  comp_ypass<OP2, HB>(s_in, s_out, kCompTY, hy, tid);
  __syncthreads();
  for (int r = warp; r < kCompTY; r += kCompThreads / 32) {
    bool pair = false;
    T* row = comp_row<T>(a, y0 + r, &pair);
    if (!row) continue;
#pragma unroll
    for (int k = lane; k < kOutW; k += 32)
      comp_store<T>(a, row, pair, x0 + 2 * k, comp_xword<OP2, HB>(s_out + r * kCompRowW + k, hx));
  }
}

}  // namespace morph
