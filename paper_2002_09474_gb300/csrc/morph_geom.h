// Geometry of one fused-kernel tile (host and device).
#pragma once

#include <cuda_runtime.h>

namespace morph {

__host__ __device__ inline int cdiv(int a, int b) { return (a + b - 1) / b; }
__host__ __device__ inline int round_up(int a, int b) { return cdiv(a, b) * b; }
__host__ __device__ inline int imax(int a, int b) { return a > b ? a : b; }

// Rows (image rows for the pass along y, pixel columns for the pass along x)
// per register block of the large-window method, and outputs per thread of
// both methods: one 8x8-pixel transpose block.
constexpr int kBlk = 8;

// Tile geometry, computed identically on the host (shared-memory size) and on
// the device (addressing).  Offsets and sizes in 16-byte units.
struct Geom {
  int esz;       // bytes per pixel
  int lead;      // load start = x0 - lead, a 16-byte boundary
  int ox;        // first needed pixel, counted from the load start
  int iw_pix;    // pixels needed per input row from the load start: ox + TX + wx - 1
  int noct;      // octets (8 pixels) per input row
  int k0;        // first octet holding needed pixels
  int nbx;       // TMA boxes per input row
  int box;       // bytes per box row (128)
  int ih;        // input rows: TY + wy - 1
  int nby, bh;   // TMA boxes down the tile and their height
  int ihp;       // rows allocated per box column (nby * bh)
  int nchy;      // 8-row blocks of the y pass: ceil(ih / 8)
  int nrx;       // pixel columns the x pass reads: TX + wx - 1
  int nchx;      // 8-column blocks of the x pass: ceil(nrx / 8)
  int t_rows;    // S1T rows allocated
  int off_s0, off_sy, off_py, off_ty, off_s1t, off_sx, off_px, off_tx, off_s2;
  int a_slot;    // pipelined layout: 16-byte units between the two region-A slots (0 otherwise)
  int in_a;      // bit mask of the buffers placed in region A (kInA* bits)
  int smem_bytes;
};

// Buffers of a tile, for Geom::in_a.
constexpr int kInAS0 = 1, kInAY = 2, kInAS1T = 4, kInAX = 8, kInAS2 = 16;

// blk_y / blk_x: the pass uses the blocked large-window method (needs scratch).
// pipe: the persistent kernel's layout -- two copies of region A (S0 and the
// buffers that share its space), so the next tile's input can land in one
// while the current tile is computed in the other, then region B.
__host__ __device__ inline Geom make_geom(int esz, int TX, int TY, int wx, int wy, int ax, bool blk_y,
                                          bool blk_x, bool pipe = false) {
  Geom g;
  g.esz = esz;
  const int al = 16 / esz;  // pixels per 16 bytes
  g.lead = round_up(ax, al);
  g.ox = g.lead - ax;
  g.iw_pix = g.ox + TX + wx - 1;
  g.noct = cdiv(g.iw_pix, 8);
  g.k0 = g.ox / 8;
  // TMA boxes are 128 bytes wide (the form proven on the GPU; row-sized boxes
  // of 32-96 bytes were seen to fault, see the design notes).
  g.nbx = cdiv(g.noct * 8 * esz, 128);
  g.box = 128;
  g.ih = TY + wy - 1;
  g.nby = cdiv(g.ih, 256);
  g.bh = g.nby == 1 ? g.ih : round_up(cdiv(g.ih, g.nby), 8);  // keeps boxes 128-byte aligned
  g.ihp = g.nby * g.bh;
  g.nchy = cdiv(g.ih, kBlk);
  g.nrx = TX + wx - 1;
  g.nchx = cdiv(g.nrx, kBlk);
  g.t_rows = imax(8 * g.noct, g.ox + kBlk * g.nchx);
  blk_y = blk_y && wy > 1;
  blk_x = blk_x && wx > 1;
  const int ntc = TY / 8;
  const int s0 = cdiv(g.nbx * g.ihp * g.box, 16);
  // blocked-method scratch: S (nout rows), P (rows of blocks jlo .. jhi-1,
  // jlo = (w-1)/8, jhi = ceil((w-1+nout)/8)) and one total per block
  const int npy = kBlk * (cdiv(wy - 1 + TY, kBlk) - (wy - 1) / kBlk);
  const int npx = kBlk * (cdiv(wx - 1 + TX, kBlk) - (wx - 1) / kBlk);
  const int sy = blk_y ? TY * g.noct : 0, py = blk_y ? npy * g.noct : 0, ty = blk_y ? g.nchy * g.noct : 0;
  const int ysc = round_up(sy, 8) + round_up(py, 8) + ty;
  const int s1t = (wx > 1) ? g.t_rows * ntc : 0;
  const int sx = blk_x ? TX * ntc : 0, px = blk_x ? npx * ntc : 0, tx = blk_x ? g.nchx * ntc : 0;
  const int xsc = round_up(sx, 8) + round_up(px, 8) + tx;
  const int s2 = TY * TX * esz / 16;
  // Buffers share two regions A (offset 0) and B according to their live
  // ranges: the pass along y reads S0 and writes either its scratch or, for
  // the direct method, its output; the pass along x likewise.
  int a = s0, b = 0;
  int oa = 0;  // offsets within A are 0; within B, `B` marks them
  const int B = -1;
  int where_sy = B, where_s1t, where_sx, where_s2;
  if (wx == 1) {
    if (blk_y) {  // S0 -> y scratch (B) -> S2 (A)
      b = ysc;
      a = imax(a, s2);
      where_s2 = oa;
    } else {  // S0 (A) -> S2 (B)
      b = s2;
      where_s2 = B;
    }
    where_s1t = where_sx = oa;
  } else if (blk_y) {  // S0 -> y scratch (B) -> S1T (A)
    a = imax(a, s1t);
    b = ysc;
    where_s1t = oa;
    if (blk_x) {  // S1T -> x scratch (B) -> S2 (A)
      b = imax(b, xsc);
      a = imax(a, s2);
      where_sx = B;
      where_s2 = oa;
    } else {  // S1T (A) -> S2 (B)
      b = imax(b, s2);
      where_sx = B;
      where_s2 = B;
    }
  } else {  // S0 (A) -> S1T (B), by the direct method or a plain transpose
    b = s1t;
    where_s1t = B;
    if (blk_x) {  // S1T -> x scratch (A) -> S2 (B)
      a = imax(a, xsc);
      b = imax(b, s2);
      where_sx = oa;
      where_s2 = B;
    } else {  // S1T (B) -> S2 (A)
      a = imax(a, s2);
      where_sx = oa;
      where_s2 = oa;
    }
  }
  const int offb = pipe ? 2 * round_up(a, 8) : round_up(a, 8);
  g.a_slot = pipe ? round_up(a, 8) : 0;
  g.in_a = kInAS0 | (where_sy != B ? kInAY : 0) | (where_s1t != B ? kInAS1T : 0) | (where_sx != B ? kInAX : 0) |
           (where_s2 != B ? kInAS2 : 0);
  auto place = [&](int where, int within) { return (where == B ? offb : 0) + within; };
  g.off_s0 = 0;
  g.off_sy = place(where_sy, 0);
  g.off_py = place(where_sy, round_up(sy, 8));
  g.off_ty = place(where_sy, round_up(sy, 8) + round_up(py, 8));
  g.off_s1t = place(where_s1t, 0);
  g.off_sx = place(where_sx, 0);
  g.off_px = place(where_sx, round_up(sx, 8));
  g.off_tx = place(where_sx, round_up(sx, 8) + round_up(px, 8));
  g.off_s2 = place(where_s2, 0);
  g.smem_bytes = 16 * (offb + round_up(b, 8));
  return g;
}

// The geometry of slot 1 of a pipelined layout: region-A buffers moved to the
// second copy of region A.
__host__ __device__ inline Geom geom_slot(const Geom& g, int slot) {
  Geom s = g;
  if (slot) {
    const int d = g.a_slot;
    s.off_s0 += d;
    if (g.in_a & kInAY) {
      s.off_sy += d;
      s.off_py += d;
      s.off_ty += d;
    }
    if (g.in_a & kInAS1T) s.off_s1t += d;
    if (g.in_a & kInAX) {
      s.off_sx += d;
      s.off_px += d;
      s.off_tx += d;
    }
    if (g.in_a & kInAS2) s.off_s2 += d;
  }
  return s;
}

}  // namespace morph
