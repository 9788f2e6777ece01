/*
 * The paper's CPU method on the host -- a CPU BASELINE for the bench only:
 * the GPU library neither links nor calls it, and the tests check it against
 * the oracle.
 *
 * 8-bit erosion (op 0, min) and dilation (op 1, max) by a wx x wy rectangle
 * as two separable passes (section 5), pixels outside the image ignored
 * (identity padding: 255 for min, 0 for max).
 *
 * Vector form (aarch64 NEON, 16 pixels per instruction):
 *  - the pass along y runs down 16-pixel-wide column strips, by the direct
 *    method with two output rows sharing their common rows (section 5.1.2)
 *    or by van Herk/Gil-Werman over blocks of w rows (section 5.1.1);
 *  - the pass along x transposes 16 x 16 blocks (section 4's transposes,
 *    built from 8-, 16-, 32- and 64-bit lane swaps), runs the same pass
 *    along y, and transposes back (section 5.2.1).
 * Scalar form (the paper's baseline): the same two methods pixel by pixel,
 * the pass along x along the rows.  This file is compiled without
 * auto-vectorisation, so the scalar form stays scalar.
 *
 * Transposes for section 4's Table 1: 16 x 16 u8 and 8 x 8 u16 blocks, NEON
 * and scalar.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#if defined(__aarch64__)
#include <arm_neon.h>
#define CM_NEON 1
#else
#define CM_NEON 0
#endif

static inline uint8_t op8(int op, uint8_t a, uint8_t b) { return op ? (a > b ? a : b) : (a < b ? a : b); }

/* ---- scalar passes ------------------------------------------------------ */

/* out row y (y < nout) = op over in rows y .. y + w - 1, columns [0, ncol). */
static void ypass_direct_scalar(const uint8_t* in, long ip, uint8_t* out, long opp, int ncol, int nout, int w,
                                int op) {
  const uint8_t id = op ? 0 : 255;
  for (int y = 0; y < nout; y += 2) {
    for (int x = 0; x < ncol; ++x) {
      /* rows y+1 .. y+w-1 are common to outputs y and y+1 */
      uint8_t c = id;
      for (int r = 1; r < w; ++r) c = op8(op, c, in[(long)(y + r) * ip + x]);
      out[(long)y * opp + x] = op8(op, c, in[(long)y * ip + x]);
      if (y + 1 < nout) out[(long)(y + 1) * opp + x] = op8(op, c, in[(long)(y + w) * ip + x]);
    }
  }
}

/* The same by van Herk/Gil-Werman: blocks of w input rows from row 0; g the
 * prefix from the block's first row, h the suffix to its last;
 * out[y] = op(h[y], g[y + w - 1]).  g, h: nin = nout + w - 1 bytes each. */
static void ypass_vhgw_scalar(const uint8_t* in, long ip, uint8_t* out, long opp, int ncol, int nout, int w, int op,
                              uint8_t* g, uint8_t* h) {
  const int nin = nout + w - 1;
  for (int x = 0; x < ncol; ++x) {
    for (int b = 0; b < nin; b += w) {
      const int e = b + w < nin ? b + w : nin;
      g[b] = in[(long)b * ip + x];
      for (int i = b + 1; i < e; ++i) g[i] = op8(op, g[i - 1], in[(long)i * ip + x]);
      h[e - 1] = in[(long)(e - 1) * ip + x];
      for (int i = e - 2; i >= b; --i) h[i] = op8(op, h[i + 1], in[(long)i * ip + x]);
    }
    for (int y = 0; y < nout; ++y) out[(long)y * opp + x] = op8(op, h[y], g[y + w - 1]);
  }
}

/* The pass along x along the rows: out[y][x] = op over in[y][x .. x + w - 1]. */
static void xpass_direct_scalar(const uint8_t* in, long ip, uint8_t* out, long opp, int nrow, int nout, int w,
                                int op) {
  const uint8_t id = op ? 0 : 255;
  for (int y = 0; y < nrow; ++y) {
    const uint8_t* r = in + (long)y * ip;
    for (int x = 0; x < nout; x += 2) {
      uint8_t c = id;
      for (int k = 1; k < w; ++k) c = op8(op, c, r[x + k]);
      out[(long)y * opp + x] = op8(op, c, r[x]);
      if (x + 1 < nout) out[(long)y * opp + x + 1] = op8(op, c, r[x + w]);
    }
  }
}

static void xpass_vhgw_scalar(const uint8_t* in, long ip, uint8_t* out, long opp, int nrow, int nout, int w, int op,
                              uint8_t* g, uint8_t* h) {
  const int nin = nout + w - 1;
  for (int y = 0; y < nrow; ++y) {
    const uint8_t* r = in + (long)y * ip;
    for (int b = 0; b < nin; b += w) {
      const int e = b + w < nin ? b + w : nin;
      g[b] = r[b];
      for (int i = b + 1; i < e; ++i) g[i] = op8(op, g[i - 1], r[i]);
      h[e - 1] = r[e - 1];
      for (int i = e - 2; i >= b; --i) h[i] = op8(op, h[i + 1], r[i]);
    }
    for (int x = 0; x < nout; ++x) out[(long)y * opp + x] = op8(op, h[x], g[x + w - 1]);
  }
}

/* ---- NEON passes and transposes ------------------------------------------ */
#if CM_NEON
static inline uint8x16_t vop(int op, uint8x16_t a, uint8x16_t b) { return op ? vmaxq_u8(a, b) : vminq_u8(a, b); }

/* ncol a multiple of 16 */
static void ypass_direct_neon(const uint8_t* in, long ip, uint8_t* out, long opp, int ncol, int nout, int w, int op) {
  const uint8x16_t id = vdupq_n_u8(op ? 0 : 255);
  for (int x = 0; x < ncol; x += 16) {
    for (int y = 0; y < nout; y += 2) {
      uint8x16_t c = id;
      for (int r = 1; r < w; ++r) c = vop(op, c, vld1q_u8(in + (long)(y + r) * ip + x));
      vst1q_u8(out + (long)y * opp + x, vop(op, c, vld1q_u8(in + (long)y * ip + x)));
      if (y + 1 < nout) vst1q_u8(out + (long)(y + 1) * opp + x, vop(op, c, vld1q_u8(in + (long)(y + w) * ip + x)));
    }
  }
}

/* g, h: nin vectors each */
static void ypass_vhgw_neon(const uint8_t* in, long ip, uint8_t* out, long opp, int ncol, int nout, int w, int op,
                            uint8x16_t* g, uint8x16_t* h) {
  const int nin = nout + w - 1;
  for (int x = 0; x < ncol; x += 16) {
    for (int b = 0; b < nin; b += w) {
      const int e = b + w < nin ? b + w : nin;
      g[b] = vld1q_u8(in + (long)b * ip + x);
      for (int i = b + 1; i < e; ++i) g[i] = vop(op, g[i - 1], vld1q_u8(in + (long)i * ip + x));
      h[e - 1] = vld1q_u8(in + (long)(e - 1) * ip + x);
      for (int i = e - 2; i >= b; --i) h[i] = vop(op, h[i + 1], vld1q_u8(in + (long)i * ip + x));
    }
    for (int y = 0; y < nout; ++y) vst1q_u8(out + (long)y * opp + x, vop(op, h[y], g[y + w - 1]));
  }
}

/* 16 x 16 bytes: d row i = s column i.  Four rounds of lane swaps between
 * row pairs 1, 2, 4 and 8 apart, on 8-, 16-, 32- and 64-bit lanes: round k
 * turns transposed 2^(k-1)-blocks into transposed 2^k-blocks. */
static void tr16_neon(const uint8_t* s, long sp, uint8_t* d, long dp) {
  uint8x16_t r[16];
  for (int i = 0; i < 16; ++i) r[i] = vld1q_u8(s + (long)i * sp);
  for (int i = 0; i < 16; i += 2) {
    const uint8x16x2_t t = vtrnq_u8(r[i], r[i + 1]);
    r[i] = t.val[0];
    r[i + 1] = t.val[1];
  }
  for (int i = 0; i < 16; i += 4)
    for (int j = 0; j < 2; ++j) {
      const uint16x8x2_t t = vtrnq_u16(vreinterpretq_u16_u8(r[i + j]), vreinterpretq_u16_u8(r[i + j + 2]));
      r[i + j] = vreinterpretq_u8_u16(t.val[0]);
      r[i + j + 2] = vreinterpretq_u8_u16(t.val[1]);
    }
  for (int i = 0; i < 16; i += 8)
    for (int j = 0; j < 4; ++j) {
      const uint32x4x2_t t = vtrnq_u32(vreinterpretq_u32_u8(r[i + j]), vreinterpretq_u32_u8(r[i + j + 4]));
      r[i + j] = vreinterpretq_u8_u32(t.val[0]);
      r[i + j + 4] = vreinterpretq_u8_u32(t.val[1]);
    }
  for (int j = 0; j < 8; ++j) {
    const uint64x2_t a = vreinterpretq_u64_u8(r[j]), b = vreinterpretq_u64_u8(r[j + 8]);
    r[j] = vreinterpretq_u8_u64(vtrn1q_u64(a, b));
    r[j + 8] = vreinterpretq_u8_u64(vtrn2q_u64(a, b));
  }
  for (int i = 0; i < 16; ++i) vst1q_u8(d + (long)i * dp, r[i]);
}

/* 8 x 8 16-bit pixels (pitches in pixels): three rounds on 16-, 32- and
 * 64-bit lanes. */
static void tr8_u16_neon(const uint16_t* s, long sp, uint16_t* d, long dp) {
  uint16x8_t r[8];
  for (int i = 0; i < 8; ++i) r[i] = vld1q_u16(s + (long)i * sp);
  for (int i = 0; i < 8; i += 2) {
    const uint16x8x2_t t = vtrnq_u16(r[i], r[i + 1]);
    r[i] = t.val[0];
    r[i + 1] = t.val[1];
  }
  for (int i = 0; i < 8; i += 4)
    for (int j = 0; j < 2; ++j) {
      const uint32x4x2_t t = vtrnq_u32(vreinterpretq_u32_u16(r[i + j]), vreinterpretq_u32_u16(r[i + j + 2]));
      r[i + j] = vreinterpretq_u16_u32(t.val[0]);
      r[i + j + 2] = vreinterpretq_u16_u32(t.val[1]);
    }
  for (int j = 0; j < 4; ++j) {
    const uint64x2_t a = vreinterpretq_u64_u16(r[j]), b = vreinterpretq_u64_u16(r[j + 4]);
    r[j] = vreinterpretq_u16_u64(vtrn1q_u64(a, b));
    r[j + 4] = vreinterpretq_u16_u64(vtrn2q_u64(a, b));
  }
  for (int i = 0; i < 8; ++i) vst1q_u16(d + (long)i * dp, r[i]);
}
#endif

static void tr16_scalar(const uint8_t* s, long sp, uint8_t* d, long dp) {
  for (int i = 0; i < 16; ++i)
    for (int j = 0; j < 16; ++j) d[(long)j * dp + i] = s[(long)i * sp + j];
}

static void tr8_u16_scalar(const uint16_t* s, long sp, uint16_t* d, long dp) {
  for (int i = 0; i < 8; ++i)
    for (int j = 0; j < 8; ++j) d[(long)j * dp + i] = s[(long)i * sp + j];
}

/* ---- exported ------------------------------------------------------------ */

int cm_has_neon(void) { return CM_NEON; }

static long up16(long v) { return (v + 15) / 16 * 16; }

/*
 * dst = erosion (op 0) or dilation (op 1) of the W x H u8 image src by the
 * wx x wy rectangle with anchor (ax, ay): method 0 direct, 1 van
 * Herk/Gil-Werman (both passes); vec 1 the NEON form, 0 the scalar form.
 * Returns 0, -1 for bad arguments or no NEON, -2 when memory runs out.
 */
int cm_morph_u8(const uint8_t* src, long sp, uint8_t* dst, long dp, int W, int H, int wx, int wy, int ax, int ay,
                int op, int method, int vec) {
  if (!src || !dst || W < 1 || H < 1 || wx < 1 || wy < 1 || ax < 0 || ax >= wx || ay < 0 || ay >= wy) return -1;
  if (vec && !CM_NEON) return -1;
  const uint8_t id = op ? 0 : 255;
  /* identity-padded copy: ax columns left, wx-1-ax right, ay rows above,
   * wy-1-ay below; width rounded up to 16 */
  const long PW = up16(W + wx - 1), PH = H + wy - 1;
  const long HR = up16(H), WR = up16(W);
  const long nbuf = PW * (PH > HR ? PH : HR);
  const long ntmp = (PW > WR ? PW : WR) * HR;
  const long nin_max = (PH > PW ? PH : PW) + 16;
  uint8_t* P = (uint8_t*)malloc(nbuf);
  uint8_t* V = (uint8_t*)malloc(nbuf);
  uint8_t* T = (uint8_t*)malloc(ntmp + PW * HR);
  uint8_t* gh = (uint8_t*)malloc(2 * 16 * nin_max);
  if (!P || !V || !T || !gh) {
    free(P);
    free(V);
    free(T);
    free(gh);
    return -2;
  }
  memset(P, id, nbuf);
  memset(V, id, nbuf);
  memset(T, id, ntmp + PW * HR);
  for (int y = 0; y < H; ++y) memcpy(P + (long)(y + ay) * PW + ax, src + (long)y * sp, W);
  int rc = 0;
  if (!vec) {
    /* scalar: pass along y into V (H rows of PW), pass along x along the rows */
    if (method) ypass_vhgw_scalar(P, PW, V, PW, (int)PW, H, wy, op, gh, gh + nin_max);
    else ypass_direct_scalar(P, PW, V, PW, (int)PW, H, wy, op);
    if (method) xpass_vhgw_scalar(V, PW, T, WR, H, W, wx, op, gh, gh + nin_max);
    else xpass_direct_scalar(V, PW, T, WR, H, W, wx, op);
    for (int y = 0; y < H; ++y) memcpy(dst + (long)y * dp, T + (long)y * WR, W);
  } else {
#if CM_NEON
    uint8x16_t* gv = (uint8x16_t*)malloc(2 * sizeof(uint8x16_t) * nin_max);
    if (!gv) rc = -2;
    if (!rc) {
      /* pass along y: V = H (rows padded to HR) x PW */
      if (method) ypass_vhgw_neon(P, PW, V, PW, (int)PW, H, wy, op, gv, gv + nin_max);
      else ypass_direct_neon(P, PW, V, PW, (int)PW, H, wy, op);
      /* transpose V (HR rows of PW) into T1 (PW rows of HR) */
      uint8_t* T1 = T;
      uint8_t* U = T + PW * HR;  /* WR rows of HR */
      for (long by = 0; by < HR; by += 16)
        for (long bx = 0; bx < PW; bx += 16) tr16_neon(V + by * PW + bx, PW, T1 + bx * HR + by, HR);
      /* pass along x as a pass along y over T1: U row x = op over T1 rows x .. x + wx - 1 */
      if (method) ypass_vhgw_neon(T1, HR, U, HR, (int)HR, W, wx, op, gv, gv + nin_max);
      else ypass_direct_neon(T1, HR, U, HR, (int)HR, W, wx, op);
      /* transpose U (WR rows of HR) back into P (HR rows of WR) */
      for (long by = 0; by < WR; by += 16)
        for (long bx = 0; bx < HR; bx += 16) tr16_neon(U + by * HR + bx, HR, P + bx * WR + by, WR);
      for (int y = 0; y < H; ++y) memcpy(dst + (long)y * dp, P + (long)y * WR, W);
    }
    free(gv);
#endif
  }
  free(P);
  free(V);
  free(T);
  free(gh);
  return rc;
}

/*
 * Transposes n blocks (kind 0: 16 x 16 u8, blocks of 256 bytes; kind 1: 8 x 8
 * u16, blocks of 128 bytes), block i of src into block i of dst, each block
 * rows contiguous; vec 1 NEON, 0 scalar.  Returns 0, or -1.
 */
int cm_transpose_blocks(int kind, int vec, const void* src, void* dst, long n) {
  if (vec && !CM_NEON) return -1;
  if (kind == 0) {
    const uint8_t* s = (const uint8_t*)src;
    uint8_t* d = (uint8_t*)dst;
    for (long i = 0; i < n; ++i) {
#if CM_NEON
      if (vec) {
        tr16_neon(s + 256 * i, 16, d + 256 * i, 16);
        continue;
      }
#endif
      tr16_scalar(s + 256 * i, 16, d + 256 * i, 16);
    }
    return 0;
  }
  if (kind == 1) {
    const uint16_t* s = (const uint16_t*)src;
    uint16_t* d = (uint16_t*)dst;
    for (long i = 0; i < n; ++i) {
#if CM_NEON
      if (vec) {
        tr8_u16_neon(s + 64 * i, 8, d + 64 * i, 8);
        continue;
      }
#endif
      tr8_u16_scalar(s + 64 * i, 8, d + 64 * i, 8);
    }
    return 0;
  }
  return -1;
}
