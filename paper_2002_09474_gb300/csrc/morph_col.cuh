// Column pass: erosion/dilation by a 1 x w element (the pass along y; the
// paper's "horizontal pass" of section 5.1) as a kernel of its own.
//
// A CTA of 256 threads computes a tile 128 bytes wide (32 lanes x one 32-bit
// word of a row: 4 u8 or 2 u16 pixels per lane) and `ty` rows tall.  The
// tile's input rows (ty + w - 1) arrive in shared memory as TMA boxes of 64
// rows, each on its own mbarrier, all issued at the start; the outputs are
// made 64 rows (8 groups of 8) at a time, each chunk as soon as the boxes it
// reads have landed, so loads, arithmetic and stores overlap within the CTA.
// (Plain loads of the whole tile when the image is not TMA-aligned.)  Pixels
// of a word are processed in 16-bit lanes (u8 widened on the fly), so one
// min/max.u16x2 handles two.  Columns never mix, so no halo along x is
// loaded.
//
//   direct (w <= crossover): each thread makes 8 consecutive outputs of its
//     column that share the rows common to their windows (section 5.1.2's
//     paired rows, generalised from 2 to 8 outputs).
//   blocked (w >= 9): van Herk/Gil-Werman (section 5.1.1) on blocks of 8
//     rows.  The output rows 8k .. 8k+7 have windows that start in block k
//     and end in block k+q, q = (w-1) div 8, so
//        out[8k+i] = op( S_k[i], T_{k+1} .. T_{k+q-1}, Q_k[i] )
//     with S_k[i] the suffix of block k from row i, T_j the total of block j
//     and Q_k[i] the prefix from row 8(k+q) to the window's last row.  The
//     totals are computed once per tile into shared memory; S_k and Q_k are
//     computed in registers by the thread that makes the outputs.
//
// Outputs leave straight from registers: a warp writes 128 contiguous bytes
// of one row per store.
#pragma once

#include "morph_common.cuh"

namespace morph {

constexpr int kColThreads = 256;  // threads per CTA of the column kernel
constexpr int kColBytes = 128;    // tile width in bytes
constexpr int kColBox = 64;       // rows per TMA box (one mbarrier each)
constexpr int kColMaxBoxes = 32;  // boxes per tile at most

// Per-launch description.
struct ColArgs {
  const uint8_t* src;
  uint8_t* dst;
  long long sp, dp;  // pitches in bytes
  int W, H;          // pixels
  int w, a;          // window along y and its anchor, clipped to the image
  int ty;            // output rows per tile (multiple of 8)
  int ih;            // input rows per tile: ty + w - 1
  int ihp;           // rows of the shared-memory input tile (whole boxes)
  int ntx;           // tiles across
  int ntiles;        // tiles in the image
  int blocked;       // 1: van Herk/Gil-Werman blocks; 0: direct
  int tma_ld;        // 1: the input tile arrives by TMA
  int ld_vec;        // 1: rows allow aligned 32-bit loads
  int st_vec;        // 1: rows allow aligned 32-bit stores
  int* err;          // device error word
};

// Shared memory of one CTA: the input tile, then the block totals.
__host__ __device__ inline int col_tot_rows(int ty, int w) { return ty / 8 + (w - 1) / 8; }
__host__ __device__ inline int col_smem_bytes(int esz, int ty, int w, int ihp) {
  const int nw = 2 / esz;  // 32-bit words per lane after widening
  return kColBytes * ihp + col_tot_rows(ty, w) * 32 * nw * 4;
}

// Geometry of one tile height: input rows, the shared-memory rows (whole
// 64-row boxes), shared memory.  Valid while the boxes fit kColMaxBoxes.
struct ColGeom {
  int ty, ih, nb, ihp, smem;
  bool ok;
};
inline ColGeom col_geom(int esz, int ty, int w) {
  ColGeom g;
  g.ty = ty;
  g.ih = ty + w - 1;
  g.nb = (g.ih + kColBox - 1) / kColBox;
  g.ihp = g.nb * kColBox;
  g.smem = col_smem_bytes(esz, ty, w, g.ihp);
  g.ok = g.nb <= kColMaxBoxes;
  return g;
}

// Tile height: fewest waves of resident CTAs times the rows a tile loads
// (its outputs, plus the window's halo rows at about a third of the weight)
// plus a fixed cost per tile.  Heights are multiples of 8 up to 1024 and fit
// `max_smem` bytes.
inline int col_pick_ty(int esz, int W, int H, int w, int sms, int max_smem) {
  const int ntx = (W * esz + kColBytes - 1) / kColBytes;
  int hmax = (H + 7) / 8 * 8;
  if (hmax > 1024) hmax = 1024;
  double best = 1e300;
  int best_ty = 8;
  for (int ty = 8; ty <= hmax; ty += 8) {
    const ColGeom g = col_geom(esz, ty, w);
    if (g.smem > max_smem || !g.ok) break;
    int per_sm = 232448 / (g.smem + 1024);
    if (per_sm > 4) per_sm = 4;  // registers: 4 CTAs of 256 threads
    if (per_sm < 1) per_sm = 1;
    const double ntiles = static_cast<double>(ntx) * ((H + ty - 1) / ty);
    const double slots = static_cast<double>(sms) * per_sm;
    const double waves = static_cast<double>(static_cast<long long>((ntiles + slots - 1) / slots));
    const double cost = waves * (ty + 0.35 * (w - 1) + 24.0);
    if (cost < best) {
      best = cost;
      best_ty = ty;
    }
  }
  return best_ty;
}

// Two pixels per 32-bit word in 16-bit lanes; NW words per lane.
template <int NW>
struct CV {
  uint32_t v[NW];
};

template <int OP, int NW>
__device__ __forceinline__ CV<NW> cop(const CV<NW>& a, const CV<NW>& b) {
  CV<NW> r;
#pragma unroll
  for (int i = 0; i < NW; ++i) r.v[i] = OP == 0 ? __vminu2(a.v[i], b.v[i]) : __vmaxu2(a.v[i], b.v[i]);
  return r;
}

template <int OP, int NW>
__device__ __forceinline__ CV<NW> cident() {
  CV<NW> r;
#pragma unroll
  for (int i = 0; i < NW; ++i) r.v[i] = ident_word<OP>();
  return r;
}

// One row of the lane's column from the input tile.
template <int E>
__device__ __forceinline__ CV<2 / E> crow(const uint8_t* col, int r) {
  const uint32_t raw = *reinterpret_cast<const uint32_t*>(col + r * kColBytes);
  CV<2 / E> o;
  if (E == 1) {
    o.v[0] = __byte_perm(raw, 0u, 0x4140);
    o.v[1 % (2 / E)] = __byte_perm(raw, 0u, 0x4342);
  } else {
    o.v[0] = raw;
  }
  return o;
}

template <int E>
__device__ __forceinline__ uint32_t cnarrow(const CV<2 / E>& x) {
  if (E == 1) return __byte_perm(x.v[0], x.v[1 % (2 / E)], 0x6420);
  return x.v[0];
}

// Stores output row y of the lane's word (px0 = its first pixel).
template <typename T>
__device__ __forceinline__ void cstore(const ColArgs& a, int y, int px0, uint32_t word) {
  constexpr int E = sizeof(T), PPW = 4 / E;
  uint8_t* row = a.dst + static_cast<long long>(y) * a.dp;
  if (a.st_vec && px0 + PPW <= a.W) {
    *reinterpret_cast<uint32_t*>(row + static_cast<long long>(px0) * E) = word;
  } else {
#pragma unroll
    for (int t = 0; t < PPW; ++t)
      if (px0 + t < a.W) reinterpret_cast<T*>(row)[px0 + t] = static_cast<T>(word >> (8 * E * t));
  }
}

// One tile.  bars: kColMaxBoxes mbarriers initialised with count 1 (TMA
// path).  False when a bounded wait gave up (error word set).
template <typename T, int OP, bool BLK>
__device__ __forceinline__ bool col_tile(const ColArgs& a, const CUtensorMap* tin, int tile, uint8_t* s0,
                                         uint32_t* tot, uint64_t* bars) {
  constexpr int E = sizeof(T), NW = 2 / E, PPW = 4 / E;
  using V = CV<NW>;
  const int tid = threadIdx.x;
  const int x0 = (tile % a.ntx) * (kColBytes / E);  // first pixel column of the tile
  const int y0 = (tile / a.ntx) * a.ty;              // first output row
  const int ys = y0 - a.a;                           // first input row
  const uint32_t IDW = ident_word<OP>();
  const int rows_out = a.ty < a.H - y0 ? a.ty : a.H - y0;
  const int ngroups = (rows_out + 7) >> 3;
  const int need_rows = 8 * ngroups + a.w - 1;  // input rows this tile reads
  const int q = (a.w - 1) >> 3, r = (a.w - 1) & 7;
  // every word of the tile lies inside the image and rows take 32-bit stores
  const bool fast = a.st_vec && x0 + kColBytes / E <= a.W;

  // ---- start the loads -----------------------------------------------------------
  const int nbl = (need_rows + kColBox - 1) / kColBox;  // TMA boxes to load
  if (a.tma_ld) {
    if (tid == 0) {
      fence_proxy_async_smem();
      for (int b = 0; b < nbl; ++b) {
        mbar_arrive_expect_tx(&bars[b], static_cast<uint32_t>(kColBox * kColBytes));
        tma_load_2d(s0 + b * kColBox * kColBytes, tin, &bars[b], x0, ys + b * kColBox);
      }
    }
  } else {
    for (int i = tid; i < need_rows * 32; i += kColThreads) {
      const int rr = i >> 5, l = i & 31, y = ys + rr;
      const int px = x0 + l * PPW;
      uint32_t v = IDW;
      if (y >= 0 && y < a.H) {
        const uint8_t* row = a.src + static_cast<long long>(y) * a.sp;
        if (a.ld_vec && px + PPW <= a.W) {
          v = *reinterpret_cast<const uint32_t*>(row + static_cast<long long>(px) * E);
        } else {
#pragma unroll
          for (int t = 0; t < PPW; ++t)
            if (px + t < a.W) {
              const uint32_t sh = 8 * E * t, m = (E == 1 ? 0xFFu : 0xFFFFu) << sh;
              v = (v & ~m) | (static_cast<uint32_t>(reinterpret_cast<const T*>(row)[px + t]) << sh);
            }
        }
      }
      *reinterpret_cast<uint32_t*>(s0 + rr * kColBytes + 4 * l) = v;
    }
    __syncthreads();
  }

  // ---- 64 output rows at a time ------------------------------------------------------
  int have = 0;   // boxes waited for
  int tdone = 1;  // block totals T_j known for 1 <= j < tdone
  for (int k0 = 0; k0 < ngroups; k0 += 8) {
    const int k1 = k0 + 8 < ngroups ? k0 + 8 : ngroups;
    if (a.tma_ld) {
      const int nb_need = (8 * k1 + a.w - 1 + kColBox - 1) / kColBox;
      bool ok = true;
      for (int b = have; b < nb_need; ++b) ok = ok && mbar_wait_bounded(&bars[b], 0);
      if (__syncthreads_or(!ok)) {
        if (tid == 0) {
          atomicExch(a.err, kDevErrTmaTimeout);
          for (int b = have; b < nbl; ++b) mbar_wait_bounded(&bars[b], 0);  // let copies in flight land
        }
        return false;
      }
      // TMA fills rows outside the image with 0, the identity of max only.
      if (OP == 0 && (ys + have * kColBox < 0 || ys + nb_need * kColBox > a.H)) {
        for (int i = tid; i < (nb_need - have) * kColBox * 32; i += kColThreads) {
          const int rr = have * kColBox + (i >> 5), y = ys + rr;
          if (y < 0 || y >= a.H) *reinterpret_cast<uint32_t*>(s0 + rr * kColBytes + 4 * (i & 31)) = IDW;
        }
        __syncthreads();
      }
      have = nb_need;
    }
    if (BLK) {
      // totals of the blocks strictly inside this chunk's windows: j < k1 + q - 1
      const int tneed = k1 + q - 1;
      for (int i = tid; i < (tneed - tdone) * 32; i += kColThreads) {
        const int j = tdone + (i >> 5), l = i & 31;
        const uint8_t* col = s0 + 4 * l + 8 * j * kColBytes;
        V t = crow<E>(col, 0);
#pragma unroll
        for (int k = 1; k < 8; ++k) t = cop<OP>(t, crow<E>(col, k));
        if (NW == 2)
          *reinterpret_cast<uint2*>(tot + (j * 32 + l) * 2) = make_uint2(t.v[0], t.v[1 % NW]);
        else
          tot[j * 32 + l] = t.v[0];
      }
      if (tneed > tdone) tdone = tneed;
      __syncthreads();
      for (int i = tid; i < (k1 - k0) * 32; i += kColThreads) {
        const int k = k0 + (i >> 5), l = i & 31;
        const uint8_t* col = s0 + 4 * l;
        // suffix of block k
        V s[8];
        s[7] = crow<E>(col, 8 * k + 7);
#pragma unroll
        for (int t = 6; t >= 0; --t) s[t] = cop<OP>(crow<E>(col, 8 * k + t), s[t + 1]);
        // whole blocks k+1 .. k+q-1
        V m = cident<OP, NW>();
        for (int j = k + 1; j < k + q; ++j) {
          V t;
          if (NW == 2) {
            const uint2 u = *reinterpret_cast<const uint2*>(tot + (j * 32 + l) * 2);
            t.v[0] = u.x;
            t.v[1 % NW] = u.y;
          } else {
            t.v[0] = tot[j * 32 + l];
          }
          m = cop<OP>(m, t);
        }
        // prefix from row 8(k+q): its first r rows, then one more row per output
        const int b = 8 * (k + q);
        V h = cident<OP, NW>();
        for (int t = 0; t < r; ++t) h = cop<OP>(h, crow<E>(col, b + t));
        const int px0 = x0 + l * PPW;
        if (fast) {
          uint8_t* out = a.dst + static_cast<long long>(y0 + 8 * k) * a.dp + static_cast<long long>(px0) * E;
#pragma unroll
          for (int t = 0; t < 8; ++t) {
            h = cop<OP>(h, crow<E>(col, b + r + t));
            const V o = cop<OP>(cop<OP>(s[t], m), h);
            if (8 * k + t < rows_out) *reinterpret_cast<uint32_t*>(out + t * a.dp) = cnarrow<E>(o);
          }
        } else {
          const bool col_in = px0 < a.W;
#pragma unroll
          for (int t = 0; t < 8; ++t) {
            h = cop<OP>(h, crow<E>(col, b + r + t));
            const V o = cop<OP>(cop<OP>(s[t], m), h);
            if (col_in && 8 * k + t < rows_out) cstore<T>(a, y0 + 8 * k + t, px0, cnarrow<E>(o));
          }
        }
      }
    } else {
      const int w = a.w;
      for (int i = tid; i < (k1 - k0) * 32; i += kColThreads) {
        const int k = k0 + (i >> 5), l = i & 31;
        const uint8_t* col = s0 + 4 * l;
        const int r0 = 8 * k;
        V out[8];
        if (w >= 8) {
          // the 8 windows share rows r0+7 .. r0+w-1
          V core = crow<E>(col, r0 + 7);
          for (int t = 8; t < w; ++t) core = cop<OP>(core, crow<E>(col, r0 + t));
          V acc = crow<E>(col, r0 + 6);  // suffix of rows r0+j .. r0+6
          out[6] = cop<OP>(core, acc);
#pragma unroll
          for (int j = 5; j >= 0; --j) {
            acc = cop<OP>(acc, crow<E>(col, r0 + j));
            out[j] = cop<OP>(core, acc);
          }
          out[7] = core;
          acc = crow<E>(col, r0 + w);  // prefix of rows r0+w .. r0+w+j-1
#pragma unroll
          for (int j = 1; j < 8; ++j) {
            out[j] = cop<OP>(out[j], acc);
            if (j < 7) acc = cop<OP>(acc, crow<E>(col, r0 + w + j));
          }
        } else {
          // w < 8: rows r0 .. r0+w+6 once, each output folds its w rows
          V rw[15];
#pragma unroll
          for (int t = 0; t < 15; ++t)
            if (t < 7 + w) rw[t] = crow<E>(col, r0 + t);
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            V o = rw[j];
#pragma unroll
            for (int t = 1; t < 8; ++t)
              if (t < w) o = cop<OP>(o, rw[j + t]);
            out[j] = o;
          }
        }
        const int px0 = x0 + l * PPW;
        if (fast) {
          uint8_t* o = a.dst + static_cast<long long>(y0 + r0) * a.dp + static_cast<long long>(px0) * E;
#pragma unroll
          for (int t = 0; t < 8; ++t)
            if (r0 + t < rows_out) *reinterpret_cast<uint32_t*>(o + t * a.dp) = cnarrow<E>(out[t]);
        } else if (px0 < a.W) {
#pragma unroll
          for (int t = 0; t < 8; ++t)
            if (r0 + t < rows_out) cstore<T>(a, y0 + r0 + t, px0, cnarrow<E>(out[t]));
        }
      }
    }
  }
  return true;
}

}  // namespace morph
