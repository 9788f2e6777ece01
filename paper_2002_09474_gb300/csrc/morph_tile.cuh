// Fused two-pass erosion/dilation of one output tile (sm_103a).
//
// A CTA computes a TX x TY tile of D (paper section 2) in shared memory.
// Work units are "octets": 8 consecutive pixels of one row, held in registers
// as four 32-bit words of two 16-bit lanes, so one min.u16x2 / max.u16x2
// handles two pixels (on sm_103a the byte-wise __vminu4 costs several
// instructions, the 16x2 form one).  8-bit pixels are widened on the fly when
// read from shared memory and narrowed again before the final store.
//
//   1. TMA 2-D load of the tile's input window -- TX+wx-1 columns (start
//      rounded down to 16 bytes) by TY+wy-1 rows -- into S0, or plain loads
//      when the image is not TMA-aligned.  Pixels outside the image become the
//      operation's identity (the section 2 window ignores them).
//   2. Pass along y (1 x wy element; the paper's "horizontal pass" of
//      section 5.1) on octet columns of S0, by one of two methods:
//        direct  -- each thread makes 8 consecutive outputs, which share the
//                   rows common to their windows (the paired-row loop of
//                   section 5.1.2, generalised from 2 to 8 outputs);
//        blocked -- van Herk/Gil-Werman's decomposition (section 5.1.1): a
//                   window is a suffix of the block it starts in plus a
//                   prefix of the block it ends in.  Blocks here are 8 rows
//                   held in registers rather than w rows; the whole blocks
//                   that lie inside a window are folded from per-block
//                   totals (w/64 extra operations per output), and both scan
//                   phases run fully in parallel.  With 8-row blocks and
//                   w = 8 this is exactly the paper's method.
//      Each thread's 8x8-pixel result block is transposed in registers
//      (2x2 byte-permute butterflies, the GPU form of the vtrn transposes of
//      section 4) into S1T, where a row is one pixel column.
//   3. Pass along x (wx x 1 element, section 5.2) on S1T with the same two
//      methods -- the paper's "transpose, vertical pass, transpose" (sections
//      1 and 5.2.1) -- and the 8x8 results transposed back into row-major S2.
//   4. S2 leaves by a TMA 2-D store when the tile lies wholly inside the
//      image, otherwise by plain stores checked pixel by pixel.
// A window of width 1 skips its pass and the transposes around it.
// Each image pixel crosses HBM once in and once out; tile halos are re-read
// from L2.
#pragma once

#include "morph_common.cuh"
#include "morph_geom.h"

namespace morph {

constexpr int kThreads = 128;  // threads per CTA of every tile kernel

// ---------------------------------------------------------------------------
// Packed helpers on octets (uint4 = 8 pixels in 16-bit lanes)
// ---------------------------------------------------------------------------
template <int OP> __device__ __forceinline__ uint32_t op2(uint32_t a, uint32_t b) {
  return OP == 0 ? __vminu2(a, b) : __vmaxu2(a, b);
}
template <int OP> __device__ __forceinline__ uint4 op4(uint4 a, uint4 b) {
  return make_uint4(op2<OP>(a.x, b.x), op2<OP>(a.y, b.y), op2<OP>(a.z, b.z), op2<OP>(a.w, b.w));
}
// 8 bytes -> 8 pixels in 16-bit lanes, and back.
__device__ __forceinline__ uint4 widen8(uint2 b) {
  return make_uint4(__byte_perm(b.x, 0u, 0x4140), __byte_perm(b.x, 0u, 0x4342),
                    __byte_perm(b.y, 0u, 0x4140), __byte_perm(b.y, 0u, 0x4342));
}
__device__ __forceinline__ uint2 narrow8(uint4 w) {
  return make_uint2(__byte_perm(w.x, w.y, 0x6420), __byte_perm(w.z, w.w, 0x6420));
}
__device__ __forceinline__ uint32_t word_of(const uint4& v, int j) {
  return j == 0 ? v.x : j == 1 ? v.y : j == 2 ? v.z : v.w;
}
__device__ __forceinline__ void set_word(uint4& v, int j, uint32_t w) {
  if (j == 0) v.x = w;
  else if (j == 1) v.y = w;
  else if (j == 2) v.z = w;
  else v.w = w;
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

// Per-launch description of one image.
struct ImgArgs {
  const uint8_t* src;
  uint8_t* dst;
  long long sp, dp;    // pitches in bytes
  int W, H;            // pixels
  int wx, wy, ax, ay;  // window and anchor (already clipped to the image)
  int blk_y, blk_x;    // 1: the pass uses the blocked method (window >= 8)
  int tma_ld;          // 1: S0 arrives by TMA through the input tensor map
  int tma_st;          // 1: S2 leaves by TMA through the output tensor map
  int ld_vec;          // 1: src rows allow aligned 32-bit loads
  int st_vec;          // 1: dst rows allow aligned 32-bit stores
  int st_vec16;        // 1: dst rows allow aligned 16-byte stores
  int* err;            // device error word (set when a bounded wait gives up)
};

// ---------------------------------------------------------------------------
// Direct method: out[j] = op over rows r0+j .. r0+j+w-1, j = 0..G-1.  For
// w >= G the G windows share rows r0+G-1 .. r0+w-1 (scanned once); each adds
// a suffix of the rows before and a prefix of the rows after.  With G = 2 this
// is the paper's paired-row loop (section 5.1.2).
// ---------------------------------------------------------------------------
template <int OP, int G, class In>
__device__ __forceinline__ void direct_group(const In& in, int r0, int w, uint4 (&out)[G]) {
  if (w >= G) {
    uint4 core = in(r0 + G - 1);
#pragma unroll 2
    for (int k = G; k < w; ++k) core = op4<OP>(core, in(r0 + k));
    // out[j] = core + suffix(rows r0+j .. r0+G-2) + prefix(rows r0+w .. r0+w+j-1)
    uint4 acc = in(r0 + G - 2);
    out[G - 2] = op4<OP>(core, acc);
#pragma unroll
    for (int j = G - 3; j >= 0; --j) {
      acc = op4<OP>(acc, in(r0 + j));
      out[j] = op4<OP>(core, acc);
    }
    acc = in(r0 + w);
    out[G - 1] = op4<OP>(core, acc);
#pragma unroll
    for (int j = 1; j < G - 1; ++j) {
      out[j] = op4<OP>(out[j], acc);
      acc = op4<OP>(acc, in(r0 + w + j));
      if (j == G - 2) out[G - 1] = op4<OP>(out[G - 1], acc);
    }
  } else {
    // w < G: read the G+w-1 rows once; r[j] becomes op(r[j] .. r[j+w-1]) in
    // place (later j only read rows above j, still unmodified).
    uint4 r[2 * G - 2];
#pragma unroll
    for (int k = 0; k < 2 * G - 2; ++k)
      if (k < G + w - 1) r[k] = in(r0 + k);
#pragma unroll
    for (int j = 0; j < G; ++j) {
#pragma unroll
      for (int k = 1; k < G; ++k)
        if (k < w) r[j] = op4<OP>(r[j], r[j + k]);
      out[j] = r[j];
    }
  }
}

// ---------------------------------------------------------------------------
// Shared-memory views.  Each gives row r of one 16-byte column as 8 pixels in
// 16-bit lanes.
// ---------------------------------------------------------------------------
// Octet k of the TMA landing buffer (128-byte boxes, `ihp` rows per box column).
// Byte offset of byte b of row r in the TMA landing buffer: one box per row
// (box = the row) or 128-byte boxes stacked per box column of `ihp` rows.
__device__ __forceinline__ int s0_off(int r, int b, const Geom& g) {
  return g.nbx == 1 ? r * g.box + b : (b >> 7) * (g.ihp * 128) + r * 128 + (b & 127);
}

template <typename T>
struct S0Col {
  const uint8_t* base;
  int stride;
  __device__ __forceinline__ S0Col(const uint8_t* s0, int k, const Geom& g) {
    base = s0 + s0_off(0, k * 8 * static_cast<int>(sizeof(T)), g);
    stride = g.nbx == 1 ? g.box : 128;
  }
  __device__ __forceinline__ uint4 operator()(int r) const {
    if (sizeof(T) == 1) return widen8(*reinterpret_cast<const uint2*>(base + r * stride));
    return *reinterpret_cast<const uint4*>(base + r * stride);
  }
};

// S1T row ox + xr (xr counted from the first needed pixel column), chunk c of
// 8 image rows; the chunk index is XOR-swizzled by xr/8 so that the
// 8-row-strided writes of the transposes hit distinct banks.
template <int MT>
struct TCol {
  const uint4* base;  // S1T + ox * ntc
  int ntc, c;
  __device__ __forceinline__ uint4 operator()(int xr) const {
    return base[xr * ntc + (c ^ ((xr >> 3) & MT))];
  }
};

// A block-aligned run of S1T rows whose swizzled chunk is fixed: row i at
// base[i * stride].
struct TColB {
  const uint4* base;
  int stride;
  __device__ __forceinline__ uint4 operator()(int i) const { return base[i * stride]; }
};

// S2 (output tile, original pixel type), octet k: rows of `SBOX`-byte boxes.
template <typename T, int TX, int TY>
struct S2Col {
  uint8_t* base;
  static constexpr int SBOX = (TX * sizeof(T) < 128) ? TX * sizeof(T) : 128;
  __device__ __forceinline__ S2Col(uint8_t* s2, int k) {
    const int byte = k * 8 * static_cast<int>(sizeof(T));
    base = s2 + (byte / SBOX) * (TY * SBOX) + (byte % SBOX);
  }
  __device__ __forceinline__ void store(int r, uint4 v) const {
    if (sizeof(T) == 1)
      *reinterpret_cast<uint2*>(base + r * SBOX) = narrow8(v);
    else
      *reinterpret_cast<uint4*>(base + r * SBOX) = v;
  }
};

// In-register transpose of an 8x8-pixel block: v[i] holds row i (word j =
// pixels 2j, 2j+1); on exit t[p] holds pixel column p (word q = rows 2q, 2q+1).
__device__ __forceinline__ void transpose8(const uint4 (&v)[8], uint4 (&t)[8]) {
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      uint32_t p[2] = {word_of(v[2 * q], j), word_of(v[2 * q + 1], j)};
      transpose_block(p);
      set_word(t[2 * j], q, p[0]);
      set_word(t[2 * j + 1], q, p[1]);
    }
}

// ---------------------------------------------------------------------------
// Blocked large-window method.  The scanned column is cut into blocks of 8
// rows (block j = rows 8j .. 8j+7).  Phase 1 (one thread per block) loads the
// block into registers and stores its suffix op S (rows of blocks j < nout/8),
// its prefix op P (blocks jlo <= j < jhi: rows w-1 .. w-2+nout, kept from row
// 8*jlo on) and its total T[j].  Phase 2 (one thread per 8 outputs) gives
//   out[s] = op(S[s], P[s+w-1], T[j] for the blocks strictly inside),
// a window starting in one block and ending in a later one (w >= 8).
// ---------------------------------------------------------------------------
struct BlkGeo {
  int nrows;  // input rows of the pass (rows >= nrows read as the identity)
  int nout;   // outputs (a multiple of 8)
  int w;      // window
  int jlo;    // first block whose prefix is kept: (w-1)/8
  int jhi;    // one past the last: ceil((w-1+nout)/8)
};
__device__ __forceinline__ BlkGeo blk_geo(int nrows, int nout, int w) {
  BlkGeo b;
  b.nrows = nrows;
  b.nout = nout;
  b.w = w;
  b.jlo = (w - 1) / kBlk;
  b.jhi = (w - 1 + nout + kBlk - 1) / kBlk;
  return b;
}

// BlkGeo for a phase-1 call that passes rows relative to block j (block 0 of
// the shifted view is block j of the pass).
__device__ __forceinline__ BlkGeo bg_shift(const BlkGeo& b, int j) {
  BlkGeo s = b;
  s.nrows = b.nrows - kBlk * j;
  s.nout = b.nout - kBlk * j;
  s.jlo = b.jlo - j;
  s.jhi = b.jhi - j;
  return s;
}

// Phase 1 for block j.  sp/pp/tp: where rows 8j.. of S / P and T[j] go,
// consecutive rows `stride` uint4 apart.
template <int OP, class In>
__device__ __forceinline__ void blocked_scan(const In& in, int j, const BlkGeo& b, uint4* sp, uint4* pp,
                                             uint4* tp, int stride) {
  const uint32_t id = ident_word<OP>();
  uint4 v[kBlk];
  const int r0 = j * kBlk;
  if (r0 + kBlk <= b.nrows) {
#pragma unroll
    for (int i = 0; i < kBlk; ++i) v[i] = in(r0 + i);
  } else {
#pragma unroll
    for (int i = 0; i < kBlk; ++i) v[i] = (r0 + i < b.nrows) ? in(r0 + i) : make_uint4(id, id, id, id);
  }
  if (j >= b.jlo && j < b.jhi) {
    uint4 p = v[0];
    pp[0] = p;
#pragma unroll
    for (int i = 1; i < kBlk; ++i) {
      p = op4<OP>(p, v[i]);
      pp[i * stride] = p;
    }
  }
  uint4 sfx = v[kBlk - 1];
  const bool keep_s = r0 < b.nout;
  if (keep_s) sp[(kBlk - 1) * stride] = sfx;
#pragma unroll
  for (int i = kBlk - 2; i >= 0; --i) {
    sfx = op4<OP>(sfx, v[i]);
    if (keep_s) sp[i * stride] = sfx;
  }
  *tp = sfx;
}

// Phase 2 for outputs s = 8k .. 8k+7.  The window of output 8k+i ends in
// block ce0 for i < isplit and in block ce0+1 after; ld gives S row s
// (s_at), P for output i (p_at) and T[j] (t_at).
template <int OP, class Ld>
__device__ __forceinline__ void blocked_combine(const Ld& ld, int k, int w, uint4 (&out)[kBlk]) {
  const uint32_t id = ident_word<OP>();
  const int e0 = k * kBlk + w - 1;
  const int ce0 = e0 / kBlk;
  const int isplit = kBlk * (ce0 + 1) - e0;
  uint4 ma = make_uint4(id, id, id, id);  // totals of blocks k+1 .. ce0-1
  for (int j = k + 1; j < ce0; ++j) ma = op4<OP>(ma, ld.t_at(j));
  const uint4 mb = (ce0 > k) ? op4<OP>(ma, ld.t_at(ce0)) : ma;  // ... k+1 .. ce0
#pragma unroll
  for (int i = 0; i < kBlk; ++i) {
    const uint4 m = (i < isplit) ? ma : mb;
    out[i] = op4<OP>(op4<OP>(ld.s_at(i), ld.p_at(i, isplit)), m);
  }
}

// Phase-2 view of the y-pass scratch (row-major, octet column c).
struct YLd {
  const uint4 *s, *p, *t;  // S row 8k, P row for output 8k, T row 0 -- all at column c
  int pitch;
  __device__ __forceinline__ uint4 s_at(int i) const { return s[i * pitch]; }
  __device__ __forceinline__ uint4 p_at(int i, int) const { return p[i * pitch]; }
  __device__ __forceinline__ uint4 t_at(int j) const { return t[j * pitch]; }
};

// Phase-2 view of the x-pass scratch: rows of NTC chunks, chunk c stored at
// c ^ ((row/8) & MT) so that lanes working on consecutive 8-row groups hit
// distinct banks.
template <int MT>
struct XLd {
  const uint4 *sb, *pb, *tb;
  int c, ntc, k, prow0;  // prow0: P buffer row of output 8k
  __device__ __forceinline__ uint4 s_at(int i) const {
    return sb[(kBlk * k + i) * ntc + (c ^ (k & MT))];
  }
  __device__ __forceinline__ uint4 p_at(int i, int) const {
    const int r = prow0 + i;
    return pb[r * ntc + (c ^ ((r >> 3) & MT))];
  }
  __device__ __forceinline__ uint4 t_at(int j) const { return tb[j * ntc + (c ^ (j & MT))]; }
};

template <typename T> __device__ __forceinline__ uint32_t load_px(const uint8_t* row, int x) {
  return reinterpret_cast<const T*>(row)[x];
}

// ---------------------------------------------------------------------------
// One tile, in three parts: tile_issue_load (thread 0 starts the TMA copy of
// the tile's input window into S0), the wait on its barrier, and tile_body
// (identity fix-up or plain loads, both passes, store).  `shift` moves the
// region-A buffers to the second slot of a pipelined layout (0 otherwise).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4* tile_buf(uint4* smem, const Geom& g, int off, int bit, int shift) {
  return smem + off + ((g.in_a & bit) ? shift : 0);
}

// Thread 0 only.  The caller has ordered every earlier generic-proxy access
// to this S0 before the call (barrier, and a proxy fence after writes).
template <typename T>
__device__ __forceinline__ void tile_issue_load(const ImgArgs& a, const CUtensorMap* tin, int x0, int y0,
                                                const Geom& g, uint8_t* s0, uint64_t* bar) {
  constexpr int E = sizeof(T);
  const int xs = x0 - g.lead;
  const int ys = y0 - a.ay;
  mbar_arrive_expect_tx(bar, static_cast<uint32_t>(g.nbx * g.nby * g.box * g.bh));
  for (int bx = 0; bx < g.nbx; ++bx)
    for (int by = 0; by < g.nby; ++by)
      tma_load_2d(s0 + (bx * g.ihp + by * g.bh) * g.box, tin, bar, xs + bx * (g.box / E), ys + by * g.bh);
}

// All threads: waits for the tile's input.  False when the bounded wait gave
// up (the error word is set).
__device__ __forceinline__ bool tile_wait_load(uint64_t* bar, uint32_t& phase, int* err) {
  const bool ok = mbar_wait_bounded(bar, phase);
  phase ^= 1u;
  if (__syncthreads_or(!ok)) {
    if (threadIdx.x == 0) atomicExch(err, kDevErrTmaTimeout);
    return false;
  }
  return true;
}

// async_store: a TMA store of S2 is left in flight (the caller waits for its
// reads before S2's space is reused) and the tile ends with a proxy fence,
// so the next TMA load may overwrite any buffer this tile wrote.
template <typename T, int OP, int TX, int TY>
__device__ __forceinline__ void tile_body(const ImgArgs& a, const CUtensorMap* tout, int x0, int y0,
                                          const Geom& g, uint4* smem, int shift, bool async_store) {
  constexpr int E = sizeof(T);
  constexpr int PPW = 4 / E;   // pixels per 32-bit word of S0/S2
  constexpr int NTC = TY / 8;  // 8-row chunks per S1T row
  constexpr int NXO = TX / 8;  // output octets per row
  constexpr int MT = (NTC < 8 ? NTC : 8) - 1;
  constexpr int SBOX = S2Col<T, TX, TY>::SBOX;
  constexpr uint32_t PXMASK = (E == 1) ? 0xFFu : 0xFFFFu;
  const int tid = threadIdx.x;
  const int xs = x0 - g.lead;  // first loaded pixel column (16-byte aligned)
  const int ys = y0 - a.ay;    // first loaded row
  uint8_t* s0 = reinterpret_cast<uint8_t*>(tile_buf(smem, g, g.off_s0, kInAS0, shift));
  const uint32_t IDW = ident_word<OP>();

  // ---- 1. load fix-up, or plain loads -------------------------------------------
  const int w_lo = g.k0 * 2 * E, w_hi = g.noct * 2 * E;  // S0 words the passes read
  const bool border = xs < 0 || ys < 0 || xs + g.noct * 8 > a.W || ys + g.ih > a.H;
  if (a.tma_ld) {
    // TMA fills out-of-image pixels with 0: the identity of max, not of min.
    if (OP == 0 && border) {
      for (Strided2D i(w_hi - w_lo, tid, kThreads); i.r < g.ih; i.next()) {
        const int c = w_lo + i.c, r = i.r;
        const int y = ys + r;
        uint32_t* pw = reinterpret_cast<uint32_t*>(s0 + s0_off(r, 4 * c, g));
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
    for (Strided2D i(w_hi - w_lo, tid, kThreads); i.r < g.ih; i.next()) {
      const int c = w_lo + i.c, r = i.r;
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
      *reinterpret_cast<uint32_t*>(s0 + s0_off(r, 4 * c, g)) = v;
    }
    __syncthreads();
  }

  uint8_t* s2 = reinterpret_cast<uint8_t*>(tile_buf(smem, g, g.off_s2, kInAS2, shift));
  uint4* s1t = tile_buf(smem, g, g.off_s1t, kInAS1T, shift);
  const int nk = g.noct - g.k0;  // octet columns of S0 the pass along y covers

  // Emits the 8 y-pass outputs rows 8k..8k+7 of octet column c.
  auto emit_y = [&](int c, int k, const uint4 (&o)[kBlk]) {
    if (a.wx == 1) {
      const S2Col<T, TX, TY> out(s2, c);
#pragma unroll
      for (int i = 0; i < kBlk; ++i) out.store(kBlk * k + i, o[i]);
    } else {
      uint4 t[kBlk];
      transpose8(o, t);
      // S1T row 8c+px is pixel column xr = 8c+px-ox (relative to the first
      // needed one); its chunk k is stored at k ^ ((xr/8) & MT).  Rows with
      // xr < 0 are never read.
      const int xr0 = kBlk * c - g.ox;
      const int split = (xr0 & 7) ? kBlk - (xr0 & 7) : kBlk;
      const int ca = k ^ ((xr0 >> 3) & MT), cb = k ^ (((xr0 + 7) >> 3) & MT);
      uint4* row = s1t + (kBlk * c) * NTC;
#pragma unroll
      for (int px = 0; px < kBlk; ++px)
        if (xr0 + px >= 0) row[px * NTC + (px < split ? ca : cb)] = t[px];
    }
  };

  // ---- 2. pass along y --------------------------------------------------------
  if (a.wy == 1 && a.wx > 1) {
    for (Strided2D i(nk, tid, kThreads); i.r < NTC; i.next()) {  // transpose only
      const int c = g.k0 + i.c, k = i.r;
      const S0Col<T> col(s0, c, g);
      uint4 o[kBlk];
#pragma unroll
      for (int q = 0; q < kBlk; ++q) o[q] = col(kBlk * k + q);
      emit_y(c, k, o);
    }
  } else if (a.blk_y) {
    const BlkGeo bg = blk_geo(g.ih, TY, a.wy);
    uint4* sy = tile_buf(smem, g, g.off_sy, kInAY, shift);
    uint4* py = tile_buf(smem, g, g.off_py, kInAY, shift);
    uint4* ty = tile_buf(smem, g, g.off_ty, kInAY, shift);
    const int pitch = g.noct;
    for (Strided2D i(nk, tid, kThreads); i.r < g.nchy; i.next()) {
      const int c = g.k0 + i.c, j = i.r;
      blocked_scan<OP>(S0Col<T>(s0, c, g), j, bg, sy + (kBlk * j) * pitch + c,
                       py + (kBlk * (j - bg.jlo)) * pitch + c, ty + j * pitch + c, pitch);
    }
    __syncthreads();
    for (Strided2D i(nk, tid, kThreads); i.r < NTC; i.next()) {
      const int c = g.k0 + i.c, k = i.r;
      const YLd ld{sy + (kBlk * k) * pitch + c, py + (kBlk * k + a.wy - 1 - kBlk * bg.jlo) * pitch + c,
                   ty + c, pitch};
      uint4 o[kBlk];
      blocked_combine<OP>(ld, k, a.wy, o);
      emit_y(c, k, o);
    }
  } else {
    for (Strided2D i(nk, tid, kThreads); i.r < NTC; i.next()) {
      const int c = g.k0 + i.c;
      uint4 o[kBlk];
      direct_group<OP, kBlk>(S0Col<T>(s0, c, g), kBlk * i.r, a.wy, o);
      emit_y(c, i.r, o);
    }
  }
  __syncthreads();

  // ---- 3. pass along x on S1T, results transposed back into S2 -------------------
  if (a.wx > 1) {
    const uint4* s1x = s1t + g.ox * NTC;
    auto emit_x = [&](int c, int k, const uint4 (&o)[kBlk]) {
      uint4 rw[kBlk];
      transpose8(o, rw);  // o[pixel] (rows in words) -> rw[row] (pixels in words)
      const S2Col<T, TX, TY> out(s2, k);
#pragma unroll
      for (int r = 0; r < kBlk; ++r) out.store(kBlk * c + r, rw[r]);
    };
    if (a.blk_x) {
      const BlkGeo bg = blk_geo(g.nrx, TX, a.wx);
      uint4* sx = tile_buf(smem, g, g.off_sx, kInAX, shift);
      uint4* px = tile_buf(smem, g, g.off_px, kInAX, shift);
      uint4* tx = tile_buf(smem, g, g.off_tx, kInAX, shift);
      for (int it = tid; it < NTC * g.nchx; it += kThreads) {
        const int c = it % NTC, j = it / NTC;
        const int cs = c ^ (j & MT);                 // S rows 8j.. (block-aligned)
        const int cp = c ^ ((j - bg.jlo) & MT);      // P rows 8(j-jlo)..
        const TColB in{s1x + (kBlk * j) * NTC + cs, NTC};
        blocked_scan<OP>(in, 0, bg_shift(bg, j), sx + (kBlk * j) * NTC + cs,
                         px + (kBlk * (j - bg.jlo)) * NTC + cp, tx + j * NTC + (c ^ (j & MT)), NTC);
      }
      __syncthreads();
      for (int it = tid; it < NXO * NTC; it += kThreads) {
        const int k = it % NXO, c = it / NXO;
        const XLd<MT> ld{sx, px, tx, c, NTC, k, kBlk * k + a.wx - 1 - kBlk * bg.jlo};
        uint4 o[kBlk];
        blocked_combine<OP>(ld, k, a.wx, o);
        emit_x(c, k, o);
      }
    } else {
      for (int it = tid; it < NXO * NTC; it += kThreads) {
        const int k = it % NXO, c = it / NXO;
        uint4 o[kBlk];
        direct_group<OP, kBlk>(TCol<MT>{s1x, NTC, c}, kBlk * k, a.wx, o);
        emit_x(c, k, o);
      }
    }
  }

  // ---- 4. store S2 ---------------------------------------------------------------
  // The TMA store is used only for tiles that lie wholly inside the image;
  // tiles on the right or bottom edge take the plain, per-pixel-checked path.
  if (a.tma_st && x0 + TX <= a.W && y0 + TY <= a.H) {
    fence_proxy_async_smem();  // make this thread's S2 writes visible to the TMA unit
    __syncthreads();
    if (tid == 0) {
      for (int bx = 0; bx < TX * E / SBOX; ++bx) tma_store_2d(tout, s2 + bx * TY * SBOX, x0 + bx * (SBOX / E), y0);
      bulk_commit();
      if (!async_store) bulk_wait_read_all();
    }
    __syncthreads();
  } else {
    __syncthreads();
    // 16-byte vectors where the row allows, 32-bit words or pixels at the edge
    constexpr int NV = TX * E / 16;  // 16-byte vectors per output row
    constexpr int VPX = 16 / E;      // pixels per vector
    for (int it = tid; it < TY * NV; it += kThreads) {
      const int xv = it % NV, s = it / NV;
      const int y = y0 + s;
      const int x = x0 + xv * VPX;
      if (y >= a.H || x >= a.W) continue;
      const int byte = xv * 16;
      const uint8_t* sp = s2 + (byte / SBOX) * (TY * SBOX) + s * SBOX + byte % SBOX;
      uint8_t* row = a.dst + static_cast<long long>(y) * a.dp;
      if (a.st_vec16 && x + VPX <= a.W) {
        *reinterpret_cast<uint4*>(row + static_cast<long long>(x) * E) = *reinterpret_cast<const uint4*>(sp);
        continue;
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int xq = x + q * PPW;
        if (xq >= a.W) break;
        const uint32_t v = reinterpret_cast<const uint32_t*>(sp)[q];
        if (a.st_vec && xq + PPW <= a.W) {
          *reinterpret_cast<uint32_t*>(row + static_cast<long long>(xq) * E) = v;
        } else {
#pragma unroll
          for (int t = 0; t < PPW; ++t)
            if (xq + t < a.W) reinterpret_cast<T*>(row)[xq + t] = static_cast<T>(v >> (8 * E * t));
        }
      }
    }
    if (async_store) fence_proxy_async_smem();
    __syncthreads();
  }
}

// A whole tile in one CTA with one S0 (the batched kernel's form).
// `bar`/`phase` track the TMA barrier across tiles of a CTA.  Returns false
// when a bounded wait gave up (the error word is set).
template <typename T, int OP, int TX, int TY>
__device__ __forceinline__ bool run_tile(const ImgArgs& a, const CUtensorMap* tin, const CUtensorMap* tout,
                                         int x0, int y0, const Geom& g, uint4* smem, uint64_t* bar,
                                         uint32_t& phase, int* err) {
  if (a.tma_ld) {
    if (threadIdx.x == 0) {
      fence_proxy_async_smem();
      tile_issue_load<T>(a, tin, x0, y0, g, reinterpret_cast<uint8_t*>(smem + g.off_s0), bar);
    }
    if (!tile_wait_load(bar, phase, err)) return false;
  }
  tile_body<T, OP, TX, TY>(a, tout, x0, y0, g, smem, 0, false);
  return true;
}

// The persistent form: this CTA computes tiles cta, cta + ncta, ... (row-major
// over ntx tile columns) in a pipelined layout (make_geom with `pipe`).  The
// TMA load of the next tile goes into the other region-A slot while the
// current tile is computed; a tile's TMA store stays in flight until the
// next tile begins.  Needs a.tma_ld; bar[0..1] initialised with count 1.
template <typename T, int OP, int TX, int TY>
__device__ __forceinline__ void run_tiles_pipelined(const ImgArgs& a, const CUtensorMap* tin,
                                                    const CUtensorMap* tout, const Geom& g, uint4* smem,
                                                    uint64_t* bar, int ntx, int ntiles, int cta, int ncta) {
  const int tid = threadIdx.x;
  int t = cta;
  if (t >= ntiles) return;
  uint8_t* s0a = reinterpret_cast<uint8_t*>(smem + g.off_s0);
  uint8_t* s0b = s0a + 16 * g.a_slot;
  if (tid == 0) tile_issue_load<T>(a, tin, (t % ntx) * TX, (t / ntx) * TY, g, s0a, &bar[0]);
  uint32_t ph0 = 0, ph1 = 0;
  for (int i = 0; t < ntiles; ++i, t += ncta) {
    const int slot = i & 1;
    const int next = t + ncta;
    if (tid == 0) {
      bulk_wait_read_all();  // the previous tile's TMA store has read its S2
      if (next < ntiles)
        tile_issue_load<T>(a, tin, (next % ntx) * TX, (next / ntx) * TY, g, slot ? s0a : s0b,
                           slot ? &bar[0] : &bar[1]);
    }
    const bool ok = slot ? tile_wait_load(&bar[1], ph1, a.err) : tile_wait_load(&bar[0], ph0, a.err);
    if (!ok) {
      // let the other slot's copy land before the CTA's memory goes away
      if (tid == 0 && next < ntiles) mbar_wait_bounded(slot ? &bar[0] : &bar[1], slot ? ph0 : ph1);
      break;
    }
    tile_body<T, OP, TX, TY>(a, tout, (t % ntx) * TX, (t / ntx) * TY, g, smem, slot * g.a_slot, true);
  }
  if (tid == 0) bulk_wait_all();
}

}  // namespace morph
