// Pass along y (a 1 x w element; the paper's "horizontal pass", section 5.2)
// by van Herk/Gil-Werman with 8-row blocks, streaming down a strip: the
// strip-streaming form, whose shared memory does not grow with w.
//
// One warp owns a strip 128 bytes wide (lane l owns bytes 4l .. 4l+3 of
// every row) and a band of output rows.  Input rows relative to the band's
// first window row are cut into 8-row blocks j.  With w - 1 = 8q + r
// (0 <= r <= 7), the outputs whose windows end in block j are
// t = 8j + i - (w - 1), i = 0..7, and the window of t splits into
//    Z : rows 8j - w + 1 + i .. 8(j-q) + 7 - r   (a suffix of 8 rows Z_j)
//    M : rows 8(j-q) + 8 - r .. 8j - 1           (the last r rows of block
//                                                 j-q, then blocks j-q+1 ..
//                                                 j-1 whole)
//    P : rows 8j .. 8j + i                       (a prefix of block j)
// so out = op(suffix_i(Z_j), M_j, prefix_i(block j)): the paper's
// suffix/prefix decomposition (section 5.1.1) with blocks of 8, the whole
// blocks between folded from their totals.  Each lane keeps, per block, the
// block total and the fold of its last r rows in a small ring in shared
// memory (its own column only, so no lane waits on another).  The 8 rows Z_j
// are the input read a second time, w - 1 rows behind: a second stream of
// TMA boxes that runs in step with the first, one box per 2 blocks, served
// mostly from L2.  Both streams keep kCsSlots boxes of 16 rows in flight or
// in use, each box on its own mbarrier, so a warp holds 2 x kCsSlots x 2 KB
// of rows whatever w is, and its band can be tall.
//
// Measured on the GB300 (4096^2 and 2048^2, 1 x 15 to 1 x 127, CUDA-graph
// timing) this form is exact but 1.5-3x slower than the warp-tiled kernel
// (morph_colv.cuh), and its time grows with the band height: one warp walks
// its strip 8 rows per step, and each step's work (two block scans, the
// fold of the block totals, eight emissions) is a serial chain that the few
// warps per SM do not hide.  Four slots per stream instead of two were
// slower still (fewer warps resident).  It is therefore opt-in.
//
// 8-bit pixels are not unpacked: min/max.u16x2 on the raw word decides the
// odd pixels in the high bytes, and on the word shifted left by 8 the even
// pixels.  Needs 9 <= w <= 256 (q >= 1; the ring holds q + 1 entries), rows
// that a TMA box can load (16-byte aligned base and pitch, an image at least
// 128 bytes wide and 16 rows high).
#pragma once

#include "morph_colv.cuh"

namespace morph {

constexpr int kCsBox = 16;                  // rows per TMA box
constexpr int kCsBpb = kCsBox / 8;          // 8-row blocks per box
constexpr int kCsBoxBytes = kCsBox * 128;   // one box of a 128-byte strip
constexpr int kCsSlots = 2;                 // boxes per stream in flight or in use
constexpr int kCsMaxW = 256;

// Ring entries per lane: a power of two >= q + 1.
__host__ __device__ inline int cols_ring(int w) {
  const int q = (w - 1) >> 3;
  int rs = 4;
  while (rs < q + 1) rs <<= 1;
  return rs;
}
// Shared memory of one warp: the front and second-read slots, the two rings
// (block totals, folds of a block's last r rows; rs rows of 128 bytes each),
// then 2 kCsSlots mbarriers; rounded to 128 bytes.
__host__ __device__ inline int cols_warp_smem(int rs) {
  return (2 * kCsSlots * kCsBoxBytes + 2 * rs * 128 + 2 * kCsSlots * 8 + 127) / 128 * 128;
}
__host__ __device__ inline uint64_t* cols_bars(uint8_t* ws, int rs) {
  return reinterpret_cast<uint64_t*>(ws + 2 * kCsSlots * kCsBoxBytes + 2 * rs * 128);
}

struct ColsArgs {
  uint8_t* dst;
  long long dp;   // output pitch in bytes
  int W, H;       // pixels
  int w, a;       // window rows and anchor (9 <= w <= 256, 0 <= a < w)
  int Lo;         // output rows per warp band (multiple of 8)
  int ns;         // strips across: ceil(W * esz / 128)
  int ntask;      // ns * ceil(H / Lo)
  int wpc;        // warps per CTA
  int rs;         // ring entries per lane (cols_ring(w))
  int st_vec;     // 1: output rows allow aligned 32-bit stores
  int* err;       // device error word
};

// Stores output word `word` of row y at pixel px0 (the lane's first pixel).
template <typename T>
__device__ __forceinline__ void cols_store(const ColsArgs& a, int y, int px0, uint32_t word, bool fast) {
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

// One warp band.  ws: this warp's shared memory (cols_warp_smem bytes, the
// 2 kCsSlots mbarriers at cols_bars initialised with count 1).  lane: 0..31.
// Returns false when a bounded wait gave up (error word set; the warp then
// waits, bounded, for its copies in flight before returning).
template <typename T, int OP>
__device__ __forceinline__ bool cols_task(const ColsArgs& a, const CUtensorMap* tin, int task, int lane,
                                          uint8_t* ws) {
  constexpr int E = sizeof(T), PPW = 4 / E, S = kCsSlots;
  using C = Cw<E>;
  const uint32_t IDW = ident_word<OP>();
  C IDC;
#pragma unroll
  for (int i = 0; i < (E == 1 ? 2 : 1); ++i) IDC.v[i] = IDW;
  const int s = task % a.ns;
  const int y0 = (task / a.ns) * a.Lo;
  const int Lr = a.Lo < a.H - y0 ? a.Lo : a.H - y0;  // output rows of this band
  const int w = a.w, q = (w - 1) >> 3, r = (w - 1) & 7;
  const int ys = y0 - a.a;              // image row of front row 0
  const int zs = ys - r;                // image row of second-read row 0 (block j - q starts at 8(j - q))
  const int jmax = (Lr + w - 2) >> 3;   // last block whose windows end in the band
  const int NF = jmax / kCsBpb + 1, NZ = (jmax - q) / kCsBpb + 1;  // boxes per stream
  const int mask = a.rs - 1;
  uint8_t* fsl = ws;
  uint8_t* zsl = ws + S * kCsBoxBytes;
  uint32_t* ringT = reinterpret_cast<uint32_t*>(ws + 2 * S * kCsBoxBytes);
  uint32_t* ringS = ringT + a.rs * 32;
  uint64_t* bars = cols_bars(ws, a.rs);  // [0, S): front slots, [S, 2S): second-read slots
  const int px0 = s * (128 / E) + lane * PPW;
  const bool col_in = px0 < a.W;
  const bool fast = a.st_vec && px0 + PPW <= a.W;
  const int xbox = s * (128 / E);

  auto issue = [&](bool front, int b) {  // lane 0
    uint64_t* bar = &bars[(front ? 0 : S) + b % S];
    mbar_arrive_expect_tx(bar, static_cast<uint32_t>(kCsBoxBytes));
    tma_load_2d((front ? fsl : zsl) + (b % S) * kCsBoxBytes, tin, bar, xbox, (front ? ys : zs) + b * kCsBox);
  };
  int nf = NF < S ? NF : S, nz = NZ < S ? NZ : S;  // boxes issued per stream
  int cf = 0, cz = 0;                              // boxes landed per stream
  if (lane == 0) {
    fence_proxy_async_smem();
    for (int b = 0; b < nf; ++b) issue(true, b);
    for (int b = 0; b < nz; ++b) issue(false, b);
  }
  // Waits for box b of a stream (every lane, warp-uniform result); erosion
  // rows outside the image take the identity (the copy fills them with 0,
  // which is already dilation's identity).
  auto land = [&](bool front, int b) -> bool {
    bool got = mbar_wait_bounded(&bars[(front ? 0 : S) + b % S], static_cast<uint32_t>((b / S) & 1));
    got = __all_sync(0xffffffffu, got);
    if (!got) return false;
    const int row0 = (front ? ys : zs) + b * kCsBox;
    if (OP == 0 && (row0 < 0 || row0 + kCsBox > a.H)) {
      uint8_t* slot = (front ? fsl : zsl) + (b % S) * kCsBoxBytes;
      for (int t = 0; t < kCsBox; ++t)
        if (row0 + t < 0 || row0 + t >= a.H) *reinterpret_cast<uint32_t*>(slot + t * 128 + 4 * lane) = IDW;
    }
    return true;
  };
  // Box b's slot is free once every lane has read it: box n = b + S goes
  // there (after a proxy fence when erosion fix-ups wrote into the slot).
  auto refill = [&](bool front, int& n, int N) {
    if (n >= N) return;
    const int row0 = (front ? ys : zs) + (n - S) * kCsBox;
    if (OP == 0 && (row0 < 0 || row0 + kCsBox > a.H)) fence_proxy_async_smem();
    __syncwarp();
    if (lane == 0) issue(front, n);
    ++n;
  };

  bool ok = true;
  for (int j = 0; j <= jmax; ++j) {
    const int fb = j / kCsBpb, fo = j % kCsBpb;
    const uint8_t* fslot = fsl + (fb % S) * kCsBoxBytes + fo * 8 * 128 + 4 * lane;
    if (fo == 0) {
      if (!land(true, fb)) {
        ok = false;
        break;
      }
      ++cf;
    }
    uint32_t x[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) x[t] = *reinterpret_cast<const uint32_t*>(fslot + t * 128);
    if (fo == kCsBpb - 1) refill(true, nf, NF);
    // prefixes of block j; its total; the fold of its last r rows
    C p[8];
    p[0] = cw_of<E>(x[0]);
#pragma unroll
    for (int t = 1; t < 8; ++t) p[t] = cw_op<OP, E>(p[t - 1], cw_of<E>(x[t]));
    C sr = IDC;
#pragma unroll
    for (int t = 7; t >= 1; --t)
      if (t >= 8 - r) sr = cw_op<OP, E>(sr, cw_of<E>(x[t]));
    ringT[(j & mask) * 32 + lane] = cw_word<E>(p[7]);
    ringS[(j & mask) * 32 + lane] = cw_word<E>(sr);
    if (j < q) continue;
    // the second read: rows 8(j - q) - r .. + 7
    const int jz = j - q, zb = jz / kCsBpb, zo = jz % kCsBpb;
    const uint8_t* zslot = zsl + (zb % S) * kCsBoxBytes + zo * 8 * 128 + 4 * lane;
    if (zo == 0) {
      if (!land(false, zb)) {
        ok = false;
        break;
      }
      ++cz;
    }
    uint32_t z[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) z[u] = *reinterpret_cast<const uint32_t*>(zslot + u * 128);
    if (zo == kCsBpb - 1) refill(false, nz, NZ);
    // M: the last r rows of block j - q, then the totals of blocks j-q+1 .. j-1
    // (loads four at a time, so the fold waits on shared memory once per four)
    C m = cw_of<E>(ringS[(jz & mask) * 32 + lane]);
    int b = jz + 1;
    for (; b + 3 < j; b += 4) {
      const uint32_t v0 = ringT[(b & mask) * 32 + lane], v1 = ringT[((b + 1) & mask) * 32 + lane];
      const uint32_t v2 = ringT[((b + 2) & mask) * 32 + lane], v3 = ringT[((b + 3) & mask) * 32 + lane];
      m = cw_op<OP, E>(m, cw_op<OP, E>(cw_op<OP, E>(cw_of<E>(v0), cw_of<E>(v1)), cw_op<OP, E>(cw_of<E>(v2), cw_of<E>(v3))));
    }
    for (; b < j; ++b) m = cw_op<OP, E>(m, cw_of<E>(ringT[(b & mask) * 32 + lane]));
    // suffixes of Z, folded with M
    C sz[8];
    sz[7] = cw_op<OP, E>(cw_of<E>(z[7]), m);
#pragma unroll
    for (int u = 6; u >= 0; --u) sz[u] = cw_op<OP, E>(sz[u + 1], cw_of<E>(z[u]));
    if (!col_in) continue;
    const int t0 = 8 * j - (w - 1);  // output row (in the band) of i = 0
    if (fast && t0 >= 0 && t0 + 8 <= Lr) {
      uint8_t* out = a.dst + static_cast<long long>(y0 + t0) * a.dp + static_cast<long long>(px0) * E;
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        *reinterpret_cast<uint32_t*>(out) = cw_word<E>(cw_op<OP, E>(sz[i], p[i]));
        out += a.dp;
      }
    } else {
#pragma unroll
      for (int i = 0; i < 8; ++i)
        if (t0 + i >= 0 && t0 + i < Lr) cols_store<T>(a, y0 + t0 + i, px0, cw_word<E>(cw_op<OP, E>(sz[i], p[i])), fast);
    }
  }
  if (!ok) {
    if (lane == 0) {
      atomicExch(a.err, kDevErrTmaTimeout);
      for (int b = cf; b < nf; ++b) mbar_wait_bounded(&bars[b % S], static_cast<uint32_t>((b / S) & 1));
      for (int b = cz; b < nz; ++b) mbar_wait_bounded(&bars[S + b % S], static_cast<uint32_t>((b / S) & 1));
    }
    __syncwarp();
    return false;
  }
  return true;
}

// Launch shape: warps per CTA, resident warps per SM (shared memory and a
// register budget), and the band height.  A band of Lo rows reads Lo + w - 1
// rows ahead and Lo rows a second time; taller bands waste less on the w - 1
// rows of warm-up, but fewer bands leave SMs idle.  Default: the tallest of
// 512, 256, 128 and 64 rows whose bands give at least 0.6 x the warps
// resident on the whole GPU (measured on the GB300), else 64.
struct ColsPlan {
  int Lo, wpc, wps, ntask, smem, rs;
  bool ok;
};
inline ColsPlan cols_plan(int esz, int W, int H, int w, int max_smem, int sms, int max_warps, int forced_Lo) {
  ColsPlan p{0, 0, 0, 0, 0, 0, false};
  if (w < 9 || w > kCsMaxW || W < 1 || H < 1 || sms < 1) return p;
  const int rs = cols_ring(w), ws = cols_warp_smem(rs);
  // warps per CTA: the choice that keeps the most warps resident per SM
  int wpc = 0, wps = 0;
  for (int c = 4; c >= 1; c /= 2) {
    if (c * ws > max_smem) continue;
    int ctas = 233472 / (c * ws + 1024);
    if (ctas > 32) ctas = 32;
    int n = ctas * c;
    if (n > max_warps) n = max_warps / c * c;
    if (n > wps) {
      wps = n;
      wpc = c;
    }
  }
  if (wpc == 0) return p;
  const int ns = (W * esz + 127) / 128;
  auto tasks = [&](int Lo) { return static_cast<long long>(ns) * ((H + Lo - 1) / Lo); };
  int Lo = 64;
  if (forced_Lo > 0) {
    Lo = (forced_Lo + 7) / 8 * 8;
  } else {
    for (int c : {512, 256, 128}) {
      if (5 * tasks(c) >= 3ll * sms * wps) {
        Lo = c;
        break;
      }
    }
  }
  const int hmax = (H + 7) / 8 * 8;
  if (Lo > hmax) Lo = hmax;
  if (tasks(Lo) > (1ll << 30)) return p;
  return ColsPlan{Lo, wpc, wps, static_cast<int>(tasks(Lo)), wpc * ws, rs, true};
}

}  // namespace morph
