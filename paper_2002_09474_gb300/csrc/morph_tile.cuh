// Fused two-pass erosion/dilation of one output tile (sm_103a).
//
// A CTA computes a TX x TY tile of D (paper section 2) in shared memory:
//
//   1. TMA load of the input window of the tile (TX+wx-1 columns, TY+wy-1
//      rows, column start rounded down to 16 bytes) into S0 -- or plain
//      loads when the image is not TMA-aligned.  Pixels outside the image
//      become the operation's identity (section 2's window ignores them).
//   2. Working copy in 16-bit lanes: every word holds two pixels, so one
//      min.u16x2 / max.u16x2 handles two pixels (8-bit pixels are widened
//      once; on sm_103a the byte-wise __vminu4 costs several instructions,
//      the 16x2 form one).
//   3. Pass along y (1 x wy element, the paper's "horizontal pass" of
//      section 5.1): each thread scans one word column downwards, either
//      directly with outputs sharing the common rows (the paired-row idea of
//      section 5.1.2, generalised to G outputs) or by van Herk/Gil-Werman
//      (section 5.1.1).  Results leave through 2x2 register transposes into
//      S1T, where a row is one pixel column x and a word holds two image rows.
//   4. Pass along x (wx x 1 element, section 5.2) on S1T: the same vertical
//      scan, now along x -- the paper's "transpose, vertical pass,
//      transpose" (sections 1 and 5.2.1) done in registers and shared memory.
//      Results transpose back into row-major S2.
//   5. Coalesced 32-bit stores of S2, clipped to the image.
//
// Each image pixel crosses HBM once in and once out; the halos of
// neighbouring tiles are re-read from L2.
#pragma once

#include "morph_common.cuh"

namespace morph {

constexpr int kThreads = 256;  // threads per CTA of every tile kernel
constexpr int kGroup = 4;      // outputs per thread along the scan direction

// 16-bit-lane min/max (both pixel types run in this form).
template <int OP> __device__ __forceinline__ uint32_t op2(uint32_t a, uint32_t b) {
  return OP == 0 ? __vminu2(a, b) : __vmaxu2(a, b);
}

// Walks a row-major n0 x n1 index space with a fixed stride without a
// division per step (a runtime-divisor % or / costs ~20 instructions).
struct Strided2D {
  int c, r, dc, dr, n0;
  __device__ __forceinline__ Strided2D(int n0_, int start, int step) : n0(n0_) {
    c = start % n0;
    r = start / n0;
    dc = step % n0;
    dr = step / n0;
  }
  __device__ __forceinline__ void next() {
    c += dc;
    r += dr;
    if (c >= n0) {
      c -= n0;
      ++r;
    }
  }
};

// ---------------------------------------------------------------------------
// Tile geometry, computed identically on the host (shared-memory size) and on
// the device (addressing).  Sizes in 32-bit words unless named otherwise.
// ---------------------------------------------------------------------------
struct Geom {
  int esz;       // bytes per pixel
  int ox;        // first needed pixel, counted from the 16-byte-aligned load start
  int lead;      // pixels between the load start and x0 (ox + anchor_x)
  int iw_pix;    // pixels needed per input row, from the load start
  int nw;        // 16-bit-lane words per working row (2 pixels each)
  int c0;        // first working word the passes need (words left of it hold only padding)
  int nbx;       // 128-byte TMA boxes across a row
  int ih;        // input rows: TY + wy - 1
  int nby, bh;   // TMA boxes down the tile and their height
  int ihp;       // rows allocated per box column (nby * bh)
  int p1;        // S1T row pitch (words): TY/2 row pairs + 1
  int off_s0, off_w, off_s1t, off_h, off_s2;  // word offsets in dynamic smem
  int smem_bytes;
};

__host__ __device__ inline int cdiv(int a, int b) { return (a + b - 1) / b; }
__host__ __device__ inline int round_up(int a, int b) { return cdiv(a, b) * b; }

// vhgw_any: either pass uses van Herk/Gil-Werman (needs the H scratch).
__host__ __device__ inline Geom make_geom(int esz, int TX, int TY, int wx, int wy, int ax,
                                          bool vhgw_col, bool vhgw_row) {
  Geom g;
  g.esz = esz;
  const int al = 16 / esz;                   // pixels per 16 bytes
  g.lead = round_up(ax, al);                 // load start = x0 - lead, 16-byte aligned
  g.ox = g.lead - ax;
  g.iw_pix = g.ox + TX + wx - 1;
  g.nw = (esz == 1) ? 2 * cdiv(g.iw_pix, 4) : cdiv(g.iw_pix, 2);
  g.c0 = (esz == 1) ? 2 * (g.ox / 4) : g.ox / 2;
  g.nbx = cdiv(g.iw_pix * esz, 128);
  g.ih = TY + wy - 1;
  g.nby = cdiv(g.ih, 256);
  g.bh = cdiv(g.ih, g.nby);
  g.ihp = g.nby * g.bh;
  g.p1 = TY / 2 + 1;
  const int s0 = g.nbx * g.ihp * 32;         // TMA landing buffer (box layout)
  const int w = (esz == 1) ? g.ih * g.nw : 0; // widened copy (8-bit only)
  const int s1t = 2 * g.nw * g.p1;           // one row per pixel column
  int h = 0;
  if (vhgw_col) h = TY * g.nw;
  if (vhgw_row && TX * g.p1 > h) h = TX * g.p1;
  const int s2 = TY * (TX * esz / 4);
  // Regions (each 32-word = 128-byte aligned):
  //  8-bit : A = S0 then S1T, B = widened copy then S2, C = H
  //  16-bit: A = S0 (working copy) then S2, B = S1T, C = H
  int a, b;
  if (esz == 1) {
    a = s0 > s1t ? s0 : s1t;
    b = w > s2 ? w : s2;
    g.off_s0 = 0;
    g.off_s1t = 0;
    g.off_w = round_up(a, 32);
    g.off_s2 = g.off_w;
    g.off_h = g.off_w + round_up(b, 32);
  } else {
    a = s0 > s2 ? s0 : s2;
    b = s1t;
    g.off_s0 = 0;
    g.off_w = 0;
    g.off_s2 = 0;
    g.off_s1t = round_up(a, 32);
    g.off_h = g.off_s1t + round_up(b, 32);
  }
  g.smem_bytes = 4 * (g.off_h + round_up(h, 32));
  return g;
}

// Per-launch description of one image.
struct ImgArgs {
  const uint8_t* src;
  uint8_t* dst;
  long long sp, dp;    // pitches in bytes
  int W, H;            // pixels
  int wx, wy, ax, ay;  // window and anchor (already clipped to the image)
  int vhgw_col, vhgw_row;
  int tma;             // 1: S0 arrives by TMA through the tensor map
  int ld_vec;          // 1: src rows allow aligned 32-bit loads
  int st_vec;          // 1: dst rows allow aligned 32-bit stores
};

// out[j] = op over rows j .. j+w-1 of the column at p (row stride `stride`),
// j = 0..G-1.  For w >= G the G windows share rows G-1 .. w-1 (the "core"),
// which is scanned once; each output adds a suffix of the rows before the
// core and a prefix of the rows after it.  With G = 2 this is exactly the
// paper's paired-row loop (section 5.1.2): w-1 shared rows, one extra row per
// output.
template <int OP, int G>
__device__ __forceinline__ void direct_group(const uint32_t* __restrict__ p, int stride, int w,
                                             uint32_t (&out)[G]) {
  if (w >= G) {
    uint32_t core = p[(G - 1) * stride];
    const uint32_t* q = p + G * stride;
#pragma unroll 4
    for (int k = G; k < w; ++k, q += stride) core = op2<OP>(core, *q);
    uint32_t left[G];  // left[j] = op(rows j .. G-2), j <= G-2
    left[G - 2] = p[(G - 2) * stride];
#pragma unroll
    for (int j = G - 3; j >= 0; --j) left[j] = op2<OP>(left[j + 1], p[j * stride]);
    uint32_t right = p[w * stride];  // op(rows w .. w+j-1), j >= 1
    out[0] = op2<OP>(core, left[0]);
#pragma unroll
    for (int j = 1; j < G - 1; ++j) {
      out[j] = op2<OP>(op2<OP>(core, left[j]), right);
      right = op2<OP>(right, p[(w + j) * stride]);
    }
    out[G - 1] = op2<OP>(core, right);
  } else {
    // w < G: load the G+w-1 <= 2G-2 rows once, then combine.
    uint32_t r[2 * G - 2];
#pragma unroll
    for (int k = 0; k < 2 * G - 2; ++k) r[k] = (k < G + w - 1) ? p[k * stride] : 0u;
#pragma unroll
    for (int j = 0; j < G; ++j) {
      uint32_t v = r[j];
#pragma unroll
      for (int k = 1; k < G; ++k)
        if (k < w) v = op2<OP>(v, r[j + k]);
      out[j] = v;
    }
  }
}

// van Herk/Gil-Werman on one block [lo, hi) of a column (rows relative to
// the pass's first input row): h, the running op from the block's last row
// upwards, goes to hcol for rows < nout; g, the running op from the block's
// first row downwards, replaces the column in place.  A window starting at
// row s then is op(h[s], g[s+w-1]) (section 5.1.1).
template <int OP>
__device__ __forceinline__ void vhgw_block(uint32_t* __restrict__ col, int stride, int lo, int hi,
                                           uint32_t* __restrict__ hcol, int hstride, int nout) {
  uint32_t h = col[(hi - 1) * stride];
  if (hi - 1 < nout) hcol[(hi - 1) * hstride] = h;
#pragma unroll 4
  for (int r = hi - 2; r >= lo; --r) {
    h = op2<OP>(h, col[r * stride]);
    if (r < nout) hcol[r * hstride] = h;
  }
  uint32_t g = col[lo * stride];
#pragma unroll 4
  for (int r = lo + 1; r < hi; ++r) {
    g = op2<OP>(g, col[r * stride]);
    col[r * stride] = g;
  }
}

// Address of 32-bit word c of row r in a TMA box-layout buffer (128-byte
// boxes stacked per box column, `ihp` rows each).
__device__ __forceinline__ int box_word(int r, int c, int ihp) {
  return (c >> 5) * (ihp * 32) + r * 32 + (c & 31);
}

template <typename T> __device__ __forceinline__ uint32_t load_px(const uint8_t* row, int x) {
  return reinterpret_cast<const T*>(row)[x];
}

// One tile.  `bar`/`phase` track the TMA barrier across tiles of a CTA.
// Returns false when a bounded wait gave up (the error word is set).
template <typename T, int OP, int TX, int TY>
__device__ __forceinline__ bool run_tile(const ImgArgs& a, const CUtensorMap* tin, int x0, int y0,
                                         const Geom& g, uint32_t* smem, uint64_t* bar,
                                         uint32_t& phase, int* err) {
  constexpr int E = sizeof(T);
  constexpr int PPW = 4 / E;  // pixels per 32-bit word in S0/S2
  constexpr int G = kGroup;
  constexpr uint32_t PXMASK = (E == 1) ? 0xFFu : 0xFFFFu;
  const int tid = threadIdx.x;
  const int xs = x0 - g.lead;  // first loaded pixel column (16-byte aligned)
  const int ys = y0 - a.ay;    // first loaded row
  uint32_t* s0 = smem + g.off_s0;
  const uint32_t IDW = ident_word<OP>();
  const int nwi = cdiv(g.iw_pix * E, 4);  // S0 words per row that matter
  const int wi0 = (E == 1) ? g.c0 / 2 : g.c0;  // first S0 word that matters

  // ---- 1. load ----------------------------------------------------------------
  const bool border = xs < 0 || ys < 0 || xs + g.iw_pix > a.W || ys + g.ih > a.H;
  if (a.tma) {
    if (tid == 0) {
      fence_proxy_async_smem();
      mbar_arrive_expect_tx(bar, static_cast<uint32_t>(g.nbx * g.nby * 128 * g.bh));
      for (int bx = 0; bx < g.nbx; ++bx)
        for (int by = 0; by < g.nby; ++by)
          tma_load_2d(s0 + (bx * g.ihp + by * g.bh) * 32, tin, bar, xs + bx * (128 / E), ys + by * g.bh);
    }
    const bool ok = mbar_wait_bounded(bar, phase);
    phase ^= 1u;
    if (__syncthreads_or(!ok)) {
      if (tid == 0) atomicExch(err, kDevErrTmaTimeout);
      return false;
    }
    // TMA fills out-of-image pixels with 0: the identity of max, not of min.
    if (OP == 0 && border) {
      for (Strided2D i(nwi - wi0, tid, kThreads); i.r < g.ih; i.next()) {
        const int c = wi0 + i.c, r = i.r;
        const int y = ys + r;
        uint32_t* pw = s0 + box_word(r, c, g.ihp);
        if (y < 0 || y >= a.H) {
          *pw = IDW;
        } else {
          uint32_t v = *pw;
#pragma unroll
          for (int t = 0; t < PPW; ++t) {
            const int x = xs + c * PPW + t;
            if (x < 0 || x >= a.W) v |= PXMASK << (8 * E * t);
          }
          *pw = v;
        }
      }
      __syncthreads();
    }
  } else {
    for (Strided2D i(nwi - wi0, tid, kThreads); i.r < g.ih; i.next()) {
      const int c = wi0 + i.c, r = i.r;
      const int y = ys + r;
      uint32_t v = IDW;
      if (y >= 0 && y < a.H) {
        const uint8_t* row = a.src + static_cast<long long>(y) * a.sp;
        const int xp = xs + c * PPW;
        if (a.ld_vec && xp >= 0 && xp + PPW <= a.W) {
          v = *reinterpret_cast<const uint32_t*>(row + static_cast<long long>(xp) * E);
        } else {
#pragma unroll
          for (int t = 0; t < PPW; ++t) {
            const int x = xp + t;
            if (x >= 0 && x < a.W) {
              const uint32_t sh = 8 * E * t;
              v = (v & ~(PXMASK << sh)) | (load_px<T>(row, x) << sh);
            }
          }
        }
      }
      s0[box_word(r, c, g.ihp)] = v;
    }
    __syncthreads();
  }

  // ---- 2. working copy in 16-bit lanes ----------------------------------------
  // Column c of the working buffer starts at wcol(c); rows are wstride apart.
  uint32_t* wbuf;
  int wstride;
  if (E == 1) {
    wbuf = smem + g.off_w;
    wstride = g.nw;
    for (Strided2D i(g.nw / 2 - wi0, tid, kThreads); i.r < g.ih; i.next()) {
      const int q = wi0 + i.c, r = i.r;
      const uint32_t v = s0[box_word(r, q, g.ihp)];
      uint2 pr;
      pr.x = __byte_perm(v, 0u, 0x4140);  // pixels 0,1 -> 16-bit lanes
      pr.y = __byte_perm(v, 0u, 0x4342);  // pixels 2,3
      *reinterpret_cast<uint2*>(wbuf + r * g.nw + 2 * q) = pr;
    }
    __syncthreads();
  } else {
    wbuf = s0;
    wstride = 32;
  }
  auto wcol = [&](int c) -> uint32_t* {
    return E == 1 ? wbuf + c : wbuf + (c >> 5) * (g.ihp * 32) + (c & 31);
  };

  // ---- 3. pass along y (window wy), results transposed into S1T -----------------
  uint32_t* s1t = smem + g.off_s1t;
  uint32_t* hb = smem + g.off_h;
  constexpr int NSG = TY / G;  // row groups per column
  const int ncw = g.nw - g.c0;  // working columns the passes need
  if (a.vhgw_col) {
    const int nblk = cdiv(g.ih, a.wy);
    for (Strided2D i(ncw, tid, kThreads); i.r < nblk; i.next()) {
      const int c = g.c0 + i.c;
      const int lo = i.r * a.wy;
      const int hi = min(lo + a.wy, g.ih);
      vhgw_block<OP>(wcol(c), wstride, lo, hi, hb + c, g.nw, TY);
    }
    __syncthreads();
  }
  for (Strided2D i(ncw, tid, kThreads); i.r < NSG; i.next()) {
    const int c = g.c0 + i.c;
    const int r0 = i.r * G;
    uint32_t o[G];
    const uint32_t* col = wcol(c);
    if (a.vhgw_col) {
#pragma unroll
      for (int j = 0; j < G; ++j)
        o[j] = op2<OP>(hb[(r0 + j) * g.nw + c], col[(r0 + j + a.wy - 1) * wstride]);
    } else {
      direct_group<OP, G>(col + r0 * wstride, wstride, a.wy, o);
    }
#pragma unroll
    for (int pr = 0; pr < G / 2; ++pr) {
      uint32_t v[2] = {o[2 * pr], o[2 * pr + 1]};
      transpose_block(v);  // v[t] = pixel 2c+t of rows r0+2pr, r0+2pr+1
      const int sp = r0 / 2 + pr;
      s1t[(2 * c) * g.p1 + sp] = v[0];
      s1t[(2 * c + 1) * g.p1 + sp] = v[1];
    }
  }
  __syncthreads();

  // ---- 4. pass along x (window wx) on S1T, results back to row-major S2 ---------
  uint32_t* s2 = smem + g.off_s2;
  constexpr int NSP = TY / 2;                // row pairs
  constexpr int NXQ = TX / G;                // output pixel groups
  constexpr int P2 = TX * E / 4;             // S2 row pitch (words)
  constexpr int SWM = (P2 < 32 ? P2 : 32) - 1;  // S2 bank swizzle mask
  uint32_t* s1x = s1t + g.ox * g.p1;         // row 0 = first needed pixel column
  if (a.vhgw_row) {
    const int nx = TX + a.wx - 1;
    const int nblk = cdiv(nx, a.wx);
    for (int it = tid; it < NSP * nblk; it += kThreads) {
      const int sp = it % NSP, k = it / NSP;
      const int lo = k * a.wx;
      const int hi = min(lo + a.wx, nx);
      vhgw_block<OP>(s1x + sp, g.p1, lo, hi, hb + sp, g.p1, TX);
    }
    __syncthreads();
  }
  for (int it = tid; it < NSP * NXQ; it += kThreads) {
    const int sp = it % NSP, xq = it / NSP;
    const int xo = xq * G;
    uint32_t o[G];
    if (a.vhgw_row) {
#pragma unroll
      for (int j = 0; j < G; ++j)
        o[j] = op2<OP>(hb[(xo + j) * g.p1 + sp], s1x[(xo + j + a.wx - 1) * g.p1 + sp]);
    } else {
      direct_group<OP, G>(s1x + xo * g.p1 + sp, g.p1, a.wx, o);
    }
    // o[j] = pixel xo+j of rows 2sp, 2sp+1 -> row-major pixel pairs
    uint32_t rw[2][G / 2];
#pragma unroll
    for (int pr = 0; pr < G / 2; ++pr) {
      uint32_t v[2] = {o[2 * pr], o[2 * pr + 1]};
      transpose_block(v);  // v[i] = pixels xo+2pr, xo+2pr+1 of row 2sp+i
      rw[0][pr] = v[0];
      rw[1][pr] = v[1];
    }
    const int sw = sp & SWM;
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const int s = 2 * sp + i;
      if (E == 1) {
        // narrow the 4 pixels held in two 16-bit-lane words to one byte word
        s2[s * P2 + (xq ^ sw)] = __byte_perm(rw[i][0], rw[i][1], 0x6420);
      } else {
#pragma unroll
        for (int pr = 0; pr < G / 2; ++pr) s2[s * P2 + ((xq * (G / 2) + pr) ^ sw)] = rw[i][pr];
      }
    }
  }
  __syncthreads();

  // ---- 5. store S2, clipped to the image -----------------------------------------
  for (int it = tid; it < TY * P2; it += kThreads) {
    const int xw = it % P2, s = it / P2;
    const int y = y0 + s;
    const int x = x0 + xw * PPW;
    if (y >= a.H || x >= a.W) continue;
    const uint32_t v = s2[s * P2 + (xw ^ ((s >> 1) & SWM))];
    uint8_t* row = a.dst + static_cast<long long>(y) * a.dp;
    if (a.st_vec && x + PPW <= a.W) {
      *reinterpret_cast<uint32_t*>(row + static_cast<long long>(x) * E) = v;
    } else {
#pragma unroll
      for (int t = 0; t < PPW; ++t)
        if (x + t < a.W) reinterpret_cast<T*>(row)[x + t] = static_cast<T>(v >> (8 * E * t));
    }
  }
  __syncthreads();
  return true;
}

}  // namespace morph
