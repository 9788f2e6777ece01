// Pass along x (a w x 1 element; the paper's "vertical pass", section 5.2) by
// van Herk/Gil-Werman with 8-pixel blocks, one warp per RR rows (2, 4 or
// 8) and a segment of columns, the block data in registers.
//
// The warp walks its segment in chunks of 256 pixels.  In a chunk, lane l
// owns block k = 32c + l: the 8 input columns whose pixels start the windows
// of outputs x = xs + 8k .. xs + 8k + 7 (xs the segment's first output, so
// the block starts at input column xs - a + 8k).  It loads the block's 8 rows
// (each warp copy reads 256 contiguous bytes of one row) and transposes them
// in registers into 8 column vectors, one per pixel column, each RR/2 32-bit
// words holding the RR rows in 16-bit lanes -- the paper's transpose of
// section 4, so that the pass along x becomes a pass over registers, two rows
// per instruction.  Fewer rows per warp (RR = 2 by default) cut the
// registers and shared memory a warp needs, so more warps stay resident.
//
// With q = (w - 1) div 8 and r = (w - 1) mod 8, output 8k + i takes the
// window from offset i of block k to offset r + i of block k + q:
//    out = op( S_k[i], T_{k+1} .. T_{k+q-1}, P_{k+q}[r + i] )
// with S the suffix within block k, T a block's total and P_j[n] the prefix
// of block j up to offset n (for n > 7: op(T_j, P_{j+1}[n - 8])).  This is
// van Herk/Gil-Werman's suffix/prefix decomposition (section 5.1.1) with
// blocks of 8 and the whole blocks between folded from their totals.  Every
// lane writes its block's prefixes (the last one is its total) to a ring in
// shared memory; the outputs of chunk c are made once chunk c + 1's
// prefixes are there.  The whole blocks are folded by warp-shuffle doubling
// over the two chunks' totals (from the ring for short windows), and the
// suffix is scanned in registers, seeded with that fold.
//
// 8-bit pixels are widened by duplicating each byte into both halves of its
// 16-bit lane (p * 257), which min/max.u16x2 preserve; the transposes do the
// widening for free.  Needs w >= 9 (q >= 1) and w <= 256 (the window ends
// within the next chunk), rows aligned to 8 bytes (u8) or 16 bytes (u16).
#pragma once

#include "morph_common.cuh"

namespace morph {

constexpr int kRvChunk = 256;  // pixels per chunk (32 lanes x 8)
constexpr int kRvRing = 64;    // prefix ring: two chunks of blocks
// Input chunks in flight or in use per warp: 3 for u8 (copies run two
// chunks ahead), 2 for u16 (one chunk ahead; each chunk is twice the bytes).
__host__ __device__ constexpr int rv_slots(int esz) { return esz == 1 ? 3 : 2; }
// Shared memory per warp: the prefix ring (kRvRing records, one per block:
// its 8 prefixes of RR/2 words, padded by 16 bytes so that a quarter warp's
// 16-byte accesses to consecutive records hit distinct banks), then the
// input slots of RR rows x 33 entries of 8 pixels.
__host__ __device__ constexpr int rv_rec_bytes(int rr) { return 16 * rr + 16; }
__host__ __device__ constexpr int rv_raw_off(int rr) { return kRvRing * rv_rec_bytes(rr); }
__host__ __device__ constexpr int rv_warp_smem(int esz, int rr) {
  return rv_raw_off(rr) + rv_slots(esz) * rr * 33 * 8 * esz;
}

struct RowvArgs {
  const uint8_t* src;
  uint8_t* dst;
  long long sp, dp;  // pitches in bytes
  int W, H;          // pixels
  int w, a;          // window along x and its anchor, clipped to the image (9 <= w <= 256)
  int seg;           // output columns per segment (multiple of 256)
  int nseg;          // segments across: ceil(W / seg)
  int ntask;         // warp tasks: ceil(H / RR) * nseg
  int st_vec;        // 1: output rows allow aligned 8 * esz-byte stores
};

// RR rows of one pixel column: word j holds rows 2j (low lane) and 2j+1.
template <int RR>
struct RVec {
  uint32_t w[RR / 2];
};

template <int OP, int RR>
__device__ __forceinline__ RVec<RR> rv_op(const RVec<RR>& a, const RVec<RR>& b) {
  RVec<RR> r;
#pragma unroll
  for (int j = 0; j < RR / 2; ++j) r.w[j] = OP == 0 ? __vminu2(a.w[j], b.w[j]) : __vmaxu2(a.w[j], b.w[j]);
  return r;
}
template <int OP, int RR>
__device__ __forceinline__ RVec<RR> rv_ident() {
  RVec<RR> r;
#pragma unroll
  for (int j = 0; j < RR / 2; ++j) r.w[j] = ident_word<OP>();
  return r;
}
// Shared-memory slots hold whole vectors (8 or 16 bytes).
template <int RR>
__device__ __forceinline__ RVec<RR> rv_lds(const RVec<RR>* p) {
  return *p;
}

// 8 pixels of one row starting at pixel column B (any integer), as 8 * E
// bytes in the low words of `o` (u8: o[0..1], u16: o[0..3]); pixels outside
// [0, W) take the identity.  dl = B mod 8 (the same for every lane).
template <typename T, int OP>
__device__ __forceinline__ void rv_load_row(const uint8_t* row, int B, int dl, int W, uint32_t (&o)[4]) {
  constexpr int E = sizeof(T);
  const uint32_t IDW = ident_word<OP>();
  const int B8 = B - dl;  // multiple of 8 pixels
  if (B8 >= 0 && B8 + 16 <= W) {
    if (E == 1) {
      const uint2 x = *reinterpret_cast<const uint2*>(row + B8);
      uint2 y = make_uint2(0u, 0u);
      if (dl) y = *reinterpret_cast<const uint2*>(row + B8 + 8);
      const int s = 8 * (dl & 3);
      const uint32_t a0 = dl < 4 ? x.x : x.y, a1 = dl < 4 ? x.y : y.x, a2 = dl < 4 ? y.x : y.y;
      o[0] = __funnelshift_r(a0, a1, s);
      o[1] = __funnelshift_r(a1, a2, s);
      o[2] = o[3] = 0u;
    } else {
      const uint4 x = *reinterpret_cast<const uint4*>(row + 2 * B8);
      uint4 y = make_uint4(0u, 0u, 0u, 0u);
      if (dl) y = *reinterpret_cast<const uint4*>(row + 2 * B8 + 16);
      const int s = 16 * (dl & 1);
      uint32_t v[8] = {x.x, x.y, x.z, x.w, y.x, y.y, y.z, y.w};
      // shift by dl/2 words (uniform), then by s bits
      switch (dl >> 1) {
        case 0:
#pragma unroll
          for (int h = 0; h < 4; ++h) o[h] = __funnelshift_r(v[h], v[h + 1], s);
          break;
        case 1:
#pragma unroll
          for (int h = 0; h < 4; ++h) o[h] = __funnelshift_r(v[h + 1], v[h + 2], s);
          break;
        case 2:
#pragma unroll
          for (int h = 0; h < 4; ++h) o[h] = __funnelshift_r(v[h + 2], v[h + 3], s);
          break;
        default:
#pragma unroll
          for (int h = 0; h < 4; ++h) o[h] = __funnelshift_r(v[h + 3], v[h + 4], s);
          break;
      }
    }
  } else {
    o[0] = o[1] = o[2] = o[3] = IDW;
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const int x = B + t;
      if (x >= 0 && x < W) {
        const uint32_t v = reinterpret_cast<const T*>(row)[x];
        const int wi = t * E / 4, sh = 8 * ((t * E) & 3);
        const uint32_t m = (E == 1 ? 0xFFu : 0xFFFFu) << sh;
        o[wi] = (o[wi] & ~m) | (v << sh);
      }
    }
  }
}

// Transposes RR rows of 8 pixels (R[r]: u8 words 0..1 or u16 words 0..3) into
// column vectors: V[p] = pixel column p; u8 bytes are duplicated into their
// 16-bit lane.
template <typename T, int RR>
__device__ __forceinline__ void rv_transpose_in(const uint32_t (&R)[RR][4], RVec<RR> (&V)[8]) {
  constexpr int E = sizeof(T);
#pragma unroll
  for (int p = 0; p < 8; ++p) {
#pragma unroll
    for (int j = 0; j < RR / 2; ++j) {
      if (E == 1) {
        // bytes p%4 of rows 2j and 2j+1, each duplicated into its 16-bit lane
        const uint32_t sel = (p & 3) * 0x11u + (4 + (p & 3)) * 0x1100u;
        V[p].w[j] = __byte_perm(R[2 * j][p >> 2], R[2 * j + 1][p >> 2], sel);
      } else {
        V[p].w[j] = __byte_perm(R[2 * j][p >> 1], R[2 * j + 1][p >> 1], (p & 1) ? 0x7632u : 0x5410u);
      }
    }
  }
}

// Loads block k (RR rows from y0, 8 pixels from column B) directly from
// global memory and transposes it.
template <typename T, int OP, int RR>
__device__ __forceinline__ void rv_load_block(const RowvArgs& a, int y0, int B, int dl, RVec<RR> (&V)[8]) {
  uint32_t R[RR][4];
#pragma unroll
  for (int r = 0; r < RR; ++r) {
    if (y0 + r < a.H) {
      rv_load_row<T, OP>(a.src + static_cast<long long>(y0 + r) * a.sp, B, dl, a.W, R[r]);
    } else {
      R[r][0] = R[r][1] = R[r][2] = R[r][3] = ident_word<OP>();
    }
  }
  rv_transpose_in<T, RR>(R, V);
}

// Writes the RR x 8 output block (column vectors O) at rows y0.., columns
// x.. (columns < xe), transposed back to rows.
template <typename T, int RR>
__device__ __forceinline__ void rv_store_block(const RowvArgs& a, int y0, int x, int xe, const RVec<RR> (&O)[8]) {
  constexpr int E = sizeof(T);
  uint32_t Rw[RR][4];
#pragma unroll
  for (int j = 0; j < RR / 2; ++j) {
    if (E == 1) {
#pragma unroll
      for (int g = 0; g < 2; ++g) {
        const uint32_t A = __byte_perm(O[4 * g].w[j], O[4 * g + 1].w[j], 0x6240);
        const uint32_t Bq = __byte_perm(O[4 * g + 2].w[j], O[4 * g + 3].w[j], 0x6240);
        Rw[2 * j][g] = __byte_perm(A, Bq, 0x5410);
        Rw[2 * j + 1][g] = __byte_perm(A, Bq, 0x7632);
      }
    } else {
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        Rw[2 * j][h] = __byte_perm(O[2 * h].w[j], O[2 * h + 1].w[j], 0x5410);
        Rw[2 * j + 1][h] = __byte_perm(O[2 * h].w[j], O[2 * h + 1].w[j], 0x7632);
      }
    }
  }
  const bool full = a.st_vec && x + 8 <= xe;
#pragma unroll
  for (int r = 0; r < RR; ++r) {
    if (y0 + r >= a.H) break;
    uint8_t* row = a.dst + static_cast<long long>(y0 + r) * a.dp;
    if (full) {
      if (E == 1)
        *reinterpret_cast<uint2*>(row + x) = make_uint2(Rw[r][0], Rw[r][1]);
      else
        *reinterpret_cast<uint4*>(row + 2 * x) = make_uint4(Rw[r][0], Rw[r][1], Rw[r][2], Rw[r][3]);
    } else {
#pragma unroll
      for (int t = 0; t < 8; ++t)
        if (x + t < xe)
          reinterpret_cast<T*>(row)[x + t] = static_cast<T>(Rw[r][t * E / 4] >> (8 * ((t * E) & 3)));
    }
  }
}

// Prefix n of a block's ring record.
template <int RR>
__device__ __forceinline__ RVec<RR> rv_rec_get(const uint8_t* rec, int n) {
  return *reinterpret_cast<const RVec<RR>*>(rec + n * (RR / 2) * 4);
}

// Outputs of one block for a compile-time r: S (suffixes, seeded with the
// fold of the whole blocks), rq and rq1 the records of blocks k+q and
// k+q+1; output i is op(S[i], P_{k+q}[r+i]) or op(S[i], T_{k+q},
// P_{k+q+1}[r+i-8]).  Each prefix is loaded where it is used, so few stay
// live at once.
template <int R, int OP, int RR>
__device__ __forceinline__ void rv_combine_r(RVec<RR> (&S)[8], const uint8_t* rq, const uint8_t* rq1) {
  RVec<RR> tq;
  if (R > 0) tq = rv_rec_get<RR>(rq, 7);
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    if (i + R < 8)
      S[i] = rv_op<OP, RR>(S[i], rv_rec_get<RR>(rq, i + R));
    else
      S[i] = rv_op<OP, RR>(S[i], rv_op<OP, RR>(tq, rv_rec_get<RR>(rq1, i + R - 8)));
  }
}
template <int OP, int RR>
__device__ __forceinline__ void rv_combine(int r, RVec<RR> (&S)[8], const uint8_t* rq, const uint8_t* rq1) {
  switch (r) {
    case 0: rv_combine_r<0, OP, RR>(S, rq, rq1); break;
    case 1: rv_combine_r<1, OP, RR>(S, rq, rq1); break;
    case 2: rv_combine_r<2, OP, RR>(S, rq, rq1); break;
    case 3: rv_combine_r<3, OP, RR>(S, rq, rq1); break;
    case 4: rv_combine_r<4, OP, RR>(S, rq, rq1); break;
    case 5: rv_combine_r<5, OP, RR>(S, rq, rq1); break;
    case 6: rv_combine_r<6, OP, RR>(S, rq, rq1); break;
    default: rv_combine_r<7, OP, RR>(S, rq, rq1); break;
  }
}

// One warp task: rows RR * (task / nseg) .. +RR-1, output columns of segment
// task % nseg.  ws: this warp's shared memory (rv_warp_smem bytes): the
// prefix ring (the record of block b at b mod kRvRing), then the input
// slots.
//
// Input chunks travel by per-lane asynchronous copies one (u16) or two (u8)
// chunks ahead of use: lane l copies the 8 pixels at the aligned column of
// its block start (entry l of each row), lane 31 also the 8 after the chunk
// (entry 32); a block's pixels are entries l and l+1 shifted by the uniform
// B mod 8.  Chunks that reach outside the image (or rows past its bottom)
// are loaded directly instead, pixel by pixel where needed.
template <typename T, int OP, int RR>
__device__ __forceinline__ void rowv_task(const RowvArgs& a, int task, int lane, uint8_t* ws) {
  constexpr int E = sizeof(T), EB = 8 * E;  // bytes per entry
  constexpr int NS = rv_slots(E), D = NS - 1;  // input slots, chunks copied ahead
  using V = RVec<RR>;
  constexpr int RB = rv_rec_bytes(RR);
  uint8_t* raw = ws + rv_raw_off(RR);
  auto rec = [&](int b) { return ws + (b & (kRvRing - 1)) * RB; };
  const int y0 = RR * (task / a.nseg);
  const int xs = (task % a.nseg) * a.seg;
  const int xe = xs + a.seg < a.W ? xs + a.seg : a.W;
  const int nck = (xe - xs + kRvChunk - 1) / kRvChunk;  // output chunks
  const int X0 = xs - a.a;                                // input column of block 0
  const int dl = ((X0 % 8) + 8) % 8;
  const int q = (a.w - 1) >> 3, r = (a.w - 1) & 7;
  const bool rows_in = y0 + RR <= a.H;

  // The chunks whose copies stay inside the image form one interval
  // [jf0, jf1] (the chunk start grows with j); the others load directly.
  const int cs0 = X0 - dl;  // aligned input column of chunk 0's block 0
  const int jf0 = cs0 >= 0 ? 0 : (-cs0 + kRvChunk - 1) / kRvChunk;
  const int jf1 = rows_in ? (a.W - kRvChunk - 8 - cs0 >= 0 ? (a.W - kRvChunk - 8 - cs0) / kRvChunk : -1) : -1;
  auto fast_chunk = [&](int j) { return j >= jf0 && j <= jf1; };
  // this lane's entry in slot 0, row 0; slots and rows at fixed strides
  constexpr int kRowStride = 33 * EB, kSlotStride = RR * kRowStride;
  uint8_t* const ent = raw + lane * EB;
  // this lane's source in chunk 0, row 0 (rows at the pitch; only chunks
  // with every row inside the image are copied)
  const uint8_t* const gsrc = a.src + static_cast<long long>(y0) * a.sp + static_cast<long long>(cs0 + 8 * lane) * E;
  int slot_issue = 0, slot_build = 0;  // j mod NS of the next issue and build
  auto issue = [&](int j) {
    if (j <= nck && fast_chunk(j)) {
      uint8_t* d = ent + slot_issue * kSlotStride;
      const long long off = static_cast<long long>(kRvChunk) * j * E;
#pragma unroll
      for (int rr = 0; rr < RR; ++rr) {
        const uint8_t* g = gsrc + off + rr * a.sp;
        if (E == 1) cp_async8(d + rr * kRowStride, g); else cp_async16(d + rr * kRowStride, g);
        if (lane == 31) {
          if (E == 1) cp_async8(d + rr * kRowStride + EB, g + EB); else cp_async16(d + rr * kRowStride + EB, g + EB);
        }
      }
    }
    cp_async_commit();
    slot_issue = slot_issue + 1 == NS ? 0 : slot_issue + 1;
  };
  // Block data of chunk j from its input slot: V[p] = pixel column p.
  auto build = [&](int j, V (&Vb)[8]) {
    const int slot = slot_build;
    slot_build = slot_build + 1 == NS ? 0 : slot_build + 1;
    if (!fast_chunk(j)) {
      rv_load_block<T, OP, RR>(a, y0, X0 + kRvChunk * j + 8 * lane, dl, Vb);
      return;
    }
    uint32_t R[RR][4];
#pragma unroll
    for (int rr = 0; rr < RR; ++rr) {
      const uint8_t* p0 = ent + slot * kSlotStride + rr * kRowStride;
      const uint8_t* p1 = p0 + EB;
      if (E == 1) {
        const uint2 x = *reinterpret_cast<const uint2*>(p0), y = *reinterpret_cast<const uint2*>(p1);
        const int sh = 8 * (dl & 3);
        const uint32_t a0 = dl < 4 ? x.x : x.y, a1 = dl < 4 ? x.y : y.x, a2 = dl < 4 ? y.x : y.y;
        R[rr][0] = __funnelshift_r(a0, a1, sh);
        R[rr][1] = __funnelshift_r(a1, a2, sh);
        R[rr][2] = R[rr][3] = 0u;
      } else {
        const uint4 x = *reinterpret_cast<const uint4*>(p0), y = *reinterpret_cast<const uint4*>(p1);
        const uint32_t v[8] = {x.x, x.y, x.z, x.w, y.x, y.y, y.z, y.w};
        const int sh = 16 * (dl & 1);
        switch (dl >> 1) {
          case 0:
#pragma unroll
            for (int h = 0; h < 4; ++h) R[rr][h] = __funnelshift_r(v[h], v[h + 1], sh);
            break;
          case 1:
#pragma unroll
            for (int h = 0; h < 4; ++h) R[rr][h] = __funnelshift_r(v[h + 1], v[h + 2], sh);
            break;
          case 2:
#pragma unroll
            for (int h = 0; h < 4; ++h) R[rr][h] = __funnelshift_r(v[h + 2], v[h + 3], sh);
            break;
          default:
#pragma unroll
            for (int h = 0; h < 4; ++h) R[rr][h] = __funnelshift_r(v[h + 3], v[h + 4], sh);
            break;
        }
      }
    }
    rv_transpose_in<T, RR>(R, Vb);
  };
  auto prefixes = [&](const V (&Vb)[8], int k) {  // returns the block total
    // each 16-byte group of prefixes is stored as soon as it is complete
    constexpr int NW = RR / 2, PG = 4 / NW > 0 ? 4 / NW : 1;  // prefixes per 16 bytes
    uint4* out = reinterpret_cast<uint4*>(rec(k));
    V P = Vb[0];
    uint32_t g[4];
#pragma unroll
    for (int n = 0; n < 8; ++n) {
      if (n) P = rv_op<OP, RR>(P, Vb[n]);
#pragma unroll
      for (int j = 0; j < NW; ++j) g[((n % PG) * NW + j) & 3] = P.w[j];
      if (NW <= 4 && (n % PG) == PG - 1) {
#pragma unroll
        for (int c = 0; c < (NW > 4 ? NW / 4 : 1); ++c) out[n / PG] = make_uint4(g[0], g[1], g[2], g[3]);
      }
    }
    return P;
  };
  auto shfl = [&](const V& v, int src) {
    V o;
#pragma unroll
    for (int t = 0; t < RR / 2; ++t) o.w[t] = __shfl_sync(0xffffffffu, v.w[t], src);
    return o;
  };
  auto pick = [&](bool c, const V& x, const V& y) {
    V o;
#pragma unroll
    for (int t = 0; t < RR / 2; ++t) o.w[t] = c ? x.w[t] : y.w[t];
    return o;
  };
  const V ID = rv_ident<OP, RR>();
  V Tprev = ID;  // block totals of the previous chunk (lane l: block 32(j-1) + l)
  // the fold's doubling levels (p = 1 .. 2^(nlev-1), the largest power of
  // two p with 2p <= q - 1 reached) and the lanes its two gathers read
  int nlev = 0, pmax = 1;
  while (2 * pmax <= q - 1) {
    pmax *= 2;
    ++nlev;
  }
  if (nlev == 0) nlev = 1;  // q >= 5 always takes at least the first level
  const int g1_src = (lane + 1) & 31, g2_src = (lane + q - pmax) & 31;
  const bool g1_in = lane + 1 < 32, g2_in = lane + q - pmax < 32;

  // One step: chunk j's block data into Vnew (and its prefixes into the
  // ring), then the outputs of chunk j-1 from Vold.  Steps alternate the two
  // arrays, so no block data is copied between them.
  auto step = [&](int j, const V (&Vold)[8], V (&Vnew)[8]) {
    issue(j + D);
    cp_async_wait<D>();
    __syncwarp();
    build(j, Vnew);
    const V Tnew = prefixes(Vnew, kRvChunk / 8 * j + lane);
    __syncwarp();
    if (j >= 1) {
      // outputs of chunk j-1: block k
      const int k = 32 * (j - 1) + lane;
      // fold of the whole blocks k+1 .. k+q-1.  For q >= 5 by doubling over
      // the 64 totals of chunks j-1 (lo) and j (hi) held in the lanes:
      // after the levels, element i holds the fold of totals i .. i+p-1 (p
      // the largest power of two <= q-1), and the fold of k+1 .. k+q-1 is
      // that of elements k+1 and k+q-p (q-1 <= 2p, so the two overlap or
      // meet; the last total used is element 62 at most).  Shorter folds
      // read the ring (a sparse table of pairwise folds in shared memory
      // was measured slower: its warp synchronisations cost more than the
      // loads they save).
      V m = ID;
      if (q >= 5) {
        V lo = Tprev, hi = Tnew;
        auto level = [&](int p) {
          const int src = (lane + p) & 31;
          const bool in = lane + p < 32;
          const V al = shfl(lo, src), ah = shfl(hi, src);
          lo = rv_op<OP, RR>(lo, pick(in, al, ah));
          hi = rv_op<OP, RR>(hi, pick(in, ah, ID));
        };
        // levels p = 1, 2, 4, 8 while 2p <= q - 1 (q <= 31: at most 4),
        // unrolled: the level count is the same for the whole task
        level(1);
        if (nlev >= 2) level(2);
        if (nlev >= 3) level(4);
        if (nlev >= 4) level(8);
        auto gather = [&](int src, bool in) {
          const V al = shfl(lo, src), ah = shfl(hi, src);
          return pick(in, al, ah);
        };
        m = rv_op<OP, RR>(gather(g1_src, g1_in), gather(g2_src, g2_in));
      } else {
        for (int t = 1; t < q; ++t) m = rv_op<OP, RR>(m, rv_rec_get<RR>(rec(k + t), 7));
      }
      V S[8];  // suffixes of block k, seeded with m
      S[7] = rv_op<OP, RR>(Vold[7], m);
#pragma unroll
      for (int i = 6; i >= 0; --i) S[i] = rv_op<OP, RR>(Vold[i], S[i + 1]);
      // the prefixes of blocks k+q and k+q+1 (two records), combined
      // by a compile-time offset r
      rv_combine<OP, RR>(r, S, rec(k + q), rec(k + q + 1));
      const int x = xs + 8 * k;
      if (x < xe) rv_store_block<T, RR>(a, y0, x, xe, S);
    }
    Tprev = Tnew;
    __syncwarp();
  };
  V VA[8], VB[8];
  for (int j = 0; j < D; ++j) issue(j);
  for (int j = 0; j <= nck; j += 2) {
    step(j, VB, VA);
    if (j + 1 <= nck) step(j + 1, VA, VB);
  }
  cp_async_wait<0>();
}

// Launch shape: segment length (a multiple of 256) and warp tasks.  Each task
// walks its segment chunk by chunk, one chunk ahead, so a task's time is
// about (its chunks + 1) chunk latencies; a second wave of tasks costs a
// whole task time.  So: the shortest segment whose tasks all fit in one
// wave of (SMs x resident warps), else the longest (one segment per row).
struct RowvPlan {
  int seg, nseg, ntask;
  bool ok;
};
inline RowvPlan rowv_plan(int W, int H, int rr, int sms, int wps, int forced_seg) {
  RowvPlan best{0, 0, 0, false};
  if (W < 1 || H < 1 || sms < 1) return best;
  const int wmax = (W + kRvChunk - 1) / kRvChunk * kRvChunk;
  const long long slots = static_cast<long long>(sms) * wps;
  const long long bands = (H + rr - 1) / rr;
  int seg = wmax;
  if (forced_seg > 0) {
    seg = (forced_seg + kRvChunk - 1) / kRvChunk * kRvChunk;
    if (seg > wmax) seg = wmax;
  } else {
    for (int s = kRvChunk; s <= wmax; s += kRvChunk)
      if (bands * ((W + s - 1) / s) <= slots) {
        seg = s;
        break;
      }
  }
  const int nseg = (W + seg - 1) / seg;
  const long long ntask = bands * nseg;
  if (ntask > (1ll << 30)) return best;
  return RowvPlan{seg, nseg, static_cast<int>(ntask), true};
}

}  // namespace morph
