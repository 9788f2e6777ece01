// Row pass: erosion/dilation by a w x 1 element (the pass along x; the
// paper's "vertical pass" of section 5.2) as a kernel of its own.
//
// A CTA of 256 threads computes a tile 256 bytes wide (256 u8 or 128 u16
// pixels) and TY rows tall (64 for u8, 128 for u16).  Its input -- the tile's
// columns plus the window's halo, as 128-byte TMA boxes -- lands in RAW.
//
//   Phase 1: each 8 x 8-pixel block of the input (8 rows of one 8-pixel
//     column group; groups aligned to the first window start, the load start
//     being rounded down to 16 bytes for TMA) is widened to 16-bit lanes and
//     transposed in registers (2x2 byte-permute butterflies -- section 4's
//     transposes), so that one 16-byte word holds one pixel column of 8
//     rows; the words go to S1T, one per (column, row octet), XOR-swizzled
//     so that both phases access shared memory without bank conflicts.  For
//     the blocked method the block's total goes to TOT.
//   Phase 2: each thread makes the 8 x 8 outputs of one (row octet, column
//     block) pair from S1T in registers -- the direct method (section 5.2.2,
//     8 outputs sharing their common columns) or van Herk/Gil-Werman
//     (section 5.2.1) as out[8k+i] = op(S_k[i], T_{k+1..k+q-1}, Q_k[i]) --
//     transposes them back and stores 8 contiguous pixels per row.
//
// This is the paper's "transpose, pass, transpose" without a trip through
// memory.
#pragma once

#include "morph_tile.cuh"

namespace morph {

constexpr int kRowThreads = 256;  // threads per CTA of the row kernel
constexpr int kRowBytes = 256;    // output tile width in bytes

struct RowArgs {
  const uint8_t* src;
  uint8_t* dst;
  long long sp, dp;  // pitches in bytes
  int W, H;          // pixels
  int w, a;          // window along x and its anchor, clipped to the image
  int ntx, nty;      // tiles across and down
  int blocked;       // 1: van Herk/Gil-Werman blocks (w >= 9); 0: direct
  int tma_ld;        // 1: RAW arrives by TMA
  int ld_vec;        // 1: rows allow aligned 32-bit loads
  int st_vec;        // 1: rows allow aligned 8-byte (u8) / 16-byte (u16) stores
  int* err;          // device error word
};

// Tile geometry (host and device).  Offsets in bytes.
struct RowGeom {
  int txp, ty, nro, nkb;  // tile pixels across, rows, row octets, output column blocks
  int lead, ox;           // load start = x0 - lead (16-byte aligned); first window start in RAW
  int nb;                 // 8-pixel column blocks in S1T (covering txp + w - 1 columns)
  int npl, nbx;           // RAW pixels per row and its 128-byte boxes
  int off_s1t, off_tot, smem;
};

__host__ __device__ inline RowGeom row_geom(int esz, int w, int ax) {
  RowGeom g;
  g.txp = kRowBytes / esz;
  g.ty = esz == 1 ? 64 : 128;
  g.nro = g.ty / 8;
  g.nkb = g.txp / 8;
  const int al = 16 / esz;  // pixels per 16 bytes
  g.lead = (ax + al - 1) / al * al;
  g.ox = g.lead - ax;
  g.nb = (g.txp + w - 1 + 7) / 8;
  const int need = g.ox + 8 * g.nb + 8;  // the last block's funnel read ends here
  const int box = 128 / esz;
  g.npl = (need + box - 1) / box * box;
  g.nbx = g.npl / box;
  g.off_s1t = g.nbx * 128 * g.ty;
  g.off_tot = g.off_s1t + 8 * g.nb * g.nro * 16;
  g.smem = g.off_tot + g.nb * g.nro * 16;
  return g;
}

// S1T / TOT word of (pixel column p or block m, row octet ro).
__device__ __forceinline__ int row_slot(int p, int ro, int nro) { return p * nro + (ro ^ ((p >> 3) & 7)); }
__device__ __forceinline__ int tot_slot(int m, int ro, int nro) { return m * nro + (ro ^ (m & 7)); }

// RAW byte offset of byte b of row r (boxes of 128 bytes stacked per box column).
__device__ __forceinline__ int raw_off(int r, int b, int ty) { return (b >> 7) * (ty * 128) + r * 128 + (b & 127); }

// 8 pixels (8 * E bytes) of RAW row r starting at pixel p = 8m + sh, sh the
// tile's uniform sub-block shift, as 16-bit lanes.
template <int E>
__device__ __forceinline__ uint4 raw_octet(const uint8_t* raw, int r, int m, int sh, int ty) {
  if (E == 1) {
    const int b = 8 * m;
    const uint2 lo = *reinterpret_cast<const uint2*>(raw + raw_off(r, b, ty));
    uint2 v = lo;
    if (sh) {
      const uint2 hi = *reinterpret_cast<const uint2*>(raw + raw_off(r, b + 8, ty));
      const int s = 8 * (sh & 3);
      const uint32_t a0 = sh < 4 ? lo.x : lo.y, a1 = sh < 4 ? lo.y : hi.x, a2 = sh < 4 ? hi.x : hi.y;
      v = make_uint2(__funnelshift_r(a0, a1, s), __funnelshift_r(a1, a2, s));
    }
    return widen8(v);
  } else {
    const int b = 16 * m;
    const uint4 lo = *reinterpret_cast<const uint4*>(raw + raw_off(r, b, ty));
    if (!sh) return lo;
    const uint4 hi = *reinterpret_cast<const uint4*>(raw + raw_off(r, b + 16, ty));
    // 16-bit pixels: shift by sh pixels = 2*sh bytes across the 8 words
    const uint32_t wv[8] = {lo.x, lo.y, lo.z, lo.w, hi.x, hi.y, hi.z, hi.w};
    const int wq = sh >> 1, s = 16 * (sh & 1);
    uint32_t o[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      uint32_t x0 = wv[0], x1 = wv[1];
#pragma unroll
      for (int c = 1; c < 4; ++c)
        if (wq == c) {
          x0 = wv[i + c];
          x1 = wv[i + c + 1];
        }
      if (wq == 0) {
        x0 = wv[i];
        x1 = wv[i + 1];
      }
      o[i] = __funnelshift_r(x0, x1, s);
    }
    return make_uint4(o[0], o[1], o[2], o[3]);
  }
}

// One tile.  bar: mbarrier initialised with count 1 (TMA path); phase its
// parity.  False when the bounded wait gave up (error word set).
template <typename T, int OP, bool BLK>
__device__ __forceinline__ bool row_tile(const RowArgs& a, const CUtensorMap* tin, int tile, const RowGeom& g,
                                         uint8_t* smem, uint64_t* bar, uint32_t& phase) {
  constexpr int E = sizeof(T), PPW = 4 / E;
  const int tid = threadIdx.x;
  const int x0 = (tile % a.ntx) * g.txp;  // first output column
  const int y0 = (tile / a.ntx) * g.ty;   // first row
  const int xs = x0 - g.lead;             // first RAW column (16-byte aligned)
  const uint32_t IDW = ident_word<OP>();
  uint8_t* raw = smem;
  uint4* s1t = reinterpret_cast<uint4*>(smem + g.off_s1t);
  uint4* tot = reinterpret_cast<uint4*>(smem + g.off_tot);

  // ---- RAW ------------------------------------------------------------------------
  if (a.tma_ld) {
    if (tid == 0) {
      fence_proxy_async_smem();
      mbar_arrive_expect_tx(bar, static_cast<uint32_t>(g.nbx * 128 * g.ty));
      for (int bx = 0; bx < g.nbx; ++bx) tma_load_2d(raw + bx * 128 * g.ty, tin, bar, xs + bx * (128 / E), y0);
    }
    const bool ok = mbar_wait_bounded(bar, phase);
    phase ^= 1u;
    if (__syncthreads_or(!ok)) {
      if (tid == 0) atomicExch(a.err, kDevErrTmaTimeout);
      return false;
    }
  } else {
    const int nwr = g.npl * E / 4;  // 32-bit words per RAW row
    for (Strided2D i(nwr, tid, kRowThreads); i.r < g.ty; i.next()) {
      const int c = i.c, r = i.r, y = y0 + r;
      uint32_t v = IDW;
      if (y < a.H) {
        const uint8_t* row = a.src + static_cast<long long>(y) * a.sp;
        const int px = xs + c * PPW;
        if (a.ld_vec && px >= 0 && px + PPW <= a.W) {
          v = *reinterpret_cast<const uint32_t*>(row + static_cast<long long>(px) * E);
        } else {
#pragma unroll
          for (int t = 0; t < PPW; ++t)
            if (px + t >= 0 && px + t < a.W) {
              const uint32_t sh = 8 * E * t, m = (E == 1 ? 0xFFu : 0xFFFFu) << sh;
              v = (v & ~m) | (static_cast<uint32_t>(reinterpret_cast<const T*>(row)[px + t]) << sh);
            }
        }
      }
      *reinterpret_cast<uint32_t*>(raw + raw_off(r, 4 * c, g.ty)) = v;
    }
    __syncthreads();
  }

  // ---- phase 1: transpose 8x8 blocks into S1T (and block totals) --------------------
  const int mb0 = g.ox >> 3, sh = g.ox & 7;  // S1T block m starts at RAW pixel 8(m + mb0) + sh
  const int nbr = (g.nb + 31) & ~31;         // blocks rounded to whole warps
  for (int i = tid; i < g.nro * nbr; i += kRowThreads) {
    const int ro = i / nbr, m = i % nbr;  // ro is warp-uniform
    if (m >= g.nb) continue;
    uint4 v[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) v[t] = raw_octet<E>(raw, 8 * ro + t, m + mb0, sh, g.ty);
    // columns of this block outside the image take the identity
    const int gx = xs + g.ox + 8 * m;
    if (gx < 0 || gx + 8 > a.W) {
      uint4 keep;
      uint32_t kw[4];
#pragma unroll
      for (int d = 0; d < 4; ++d) {
        const int p0 = gx + 2 * d, p1 = p0 + 1;
        kw[d] = ((p0 >= 0 && p0 < a.W) ? 0x0000FFFFu : 0u) | ((p1 >= 0 && p1 < a.W) ? 0xFFFF0000u : 0u);
      }
      keep = make_uint4(kw[0], kw[1], kw[2], kw[3]);
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        v[t].x = (v[t].x & keep.x) | (IDW & ~keep.x);
        v[t].y = (v[t].y & keep.y) | (IDW & ~keep.y);
        v[t].z = (v[t].z & keep.z) | (IDW & ~keep.z);
        v[t].w = (v[t].w & keep.w) | (IDW & ~keep.w);
      }
    }
    uint4 c[8];
    transpose8(v, c);  // c[p] = pixel column 8m+p, rows 8ro .. 8ro+7
#pragma unroll
    for (int p = 0; p < 8; ++p) s1t[row_slot(8 * m + p, ro, g.nro)] = c[p];
    if (BLK) {
      uint4 t = c[0];
#pragma unroll
      for (int p = 1; p < 8; ++p) t = op4<OP>(t, c[p]);
      tot[tot_slot(m, ro, g.nro)] = t;
    }
  }
  __syncthreads();

  // ---- phase 2: one (row octet, column block) per thread --------------------------------
  const int ro = tid / g.nkb, k = tid % g.nkb;
  const uint4 id4 = make_uint4(IDW, IDW, IDW, IDW);
  auto col = [&](int p) { return s1t[row_slot(p, ro, g.nro)]; };
  uint4 o[8];
  if (BLK) {
    const int q = (a.w - 1) >> 3, r = (a.w - 1) & 7;
    uint4 s[8];
    s[7] = col(8 * k + 7);
#pragma unroll
    for (int t = 6; t >= 0; --t) s[t] = op4<OP>(col(8 * k + t), s[t + 1]);
    uint4 m = id4;
    for (int j = k + 1; j < k + q; ++j) m = op4<OP>(m, tot[tot_slot(j, ro, g.nro)]);
    const int b = 8 * (k + q);
    uint4 h = id4;
    for (int t = 0; t < r; ++t) h = op4<OP>(h, col(b + t));
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      h = op4<OP>(h, col(b + r + t));
      o[t] = op4<OP>(op4<OP>(s[t], m), h);
    }
  } else {
    direct_group<OP, 8>(col, 8 * k, a.w, o);
  }
  uint4 rw[8];
  transpose8(o, rw);  // rw[t] = row 8ro+t, pixels 8k .. 8k+7
  const int xo = x0 + 8 * k;
  const int yo = y0 + 8 * ro;
  if (a.st_vec && x0 + g.txp <= a.W && y0 + g.ty <= a.H) {
    uint8_t* out = a.dst + static_cast<long long>(yo) * a.dp + static_cast<long long>(xo) * E;
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      if (E == 1)
        *reinterpret_cast<uint2*>(out + t * a.dp) = narrow8(rw[t]);
      else
        *reinterpret_cast<uint4*>(out + t * a.dp) = rw[t];
    }
  } else if (xo < a.W) {
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      if (yo + t >= a.H) break;
      uint8_t* row = a.dst + static_cast<long long>(yo + t) * a.dp;
      uint32_t wd[4];
      if (E == 1) {
        const uint2 n = narrow8(rw[t]);
        wd[0] = n.x;
        wd[1] = n.y;
      } else {
        wd[0] = rw[t].x;
        wd[1] = rw[t].y;
        wd[2] = rw[t].z;
        wd[3] = rw[t].w;
      }
#pragma unroll
      for (int px = 0; px < 8; ++px)
        if (xo + px < a.W) reinterpret_cast<T*>(row)[xo + px] = static_cast<T>(wd[px / PPW] >> (8 * E * (px % PPW)));
    }
  }
  return true;
}

}  // namespace morph
