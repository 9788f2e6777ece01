// Matrix transpose (paper section 4): dst[x][y] = src[y][x] for 8-bit and
// 16-bit images.  The paper transposes 8x8 16-bit and 16x16 8-bit blocks
// with NEON vtrn butterflies in registers; here a CTA moves a 64x64-pixel tile
// through shared memory with 16-byte coalesced loads, and each thread
// transposes one 4x4-pixel block in registers with the same two-level
// butterfly (byte permutes: 2x2 blocks of bytes, then of 16-bit pairs) before
// writing four output rows.
#include "morph_common.cuh"
#include "morph_geom.h"
#include "morph_internal.h"

namespace morph {

namespace {

constexpr int kT = 64;           // tile side in pixels
constexpr int kTThreads = 256;   // one 4x4 block per thread

template <typename T>
struct TrArgs {
  const uint8_t* src;
  uint8_t* dst;
  long long sp, dp;
  int W, H;
  int ld16;  // src rows allow aligned 16-byte loads
  int st4;   // dst rows allow aligned 4*sizeof(T)-byte stores
};

// 4x4 transpose of 16-bit pixels held as 4 rows of two words each
// (row i: w[i][0] = pixels 0,1, w[i][1] = pixels 2,3).
__device__ __forceinline__ void transpose4x4_u16(uint32_t (&w)[4][2]) {
  uint32_t a[2];
  uint32_t o[4][2];
  // 2x2 blocks of 16-bit pixels, then exchange the off-diagonal 2x2 blocks
#pragma unroll
  for (int h = 0; h < 2; ++h) {  // left (pixels 0,1) / right (pixels 2,3) half
#pragma unroll
    for (int p = 0; p < 2; ++p) {  // row pairs (0,1) / (2,3)
      a[0] = w[2 * p][h];
      a[1] = w[2 * p + 1][h];
      transpose_block(a);  // a[0] = pixel 2h of rows 2p,2p+1; a[1] = pixel 2h+1
      o[2 * h][p] = a[0];
      o[2 * h + 1][p] = a[1];
    }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    w[i][0] = o[i][0];
    w[i][1] = o[i][1];
  }
}

template <typename T>
__global__ void __launch_bounds__(kTThreads) transpose_kernel(const TrArgs<T> a) {
  constexpr int E = sizeof(T);
  constexpr int RB = kT * E;       // tile row bytes
  constexpr int PITCH = RB + 4 * E;  // padded smem row (bytes; keeps 4E-byte blocks aligned)
  __shared__ __align__(16) uint8_t tile[kT * PITCH];
  const int x0 = blockIdx.x * kT, y0 = blockIdx.y * kT;
  const int tid = threadIdx.x;

  // load kT rows of kT pixels (16-byte chunks)
  constexpr int CPR = RB / 16;  // chunks per row
  for (int it = tid; it < kT * CPR; it += kTThreads) {
    const int r = it / CPR, c = it % CPR;
    const int y = y0 + r;
    const int xp = x0 + c * (16 / E);  // first pixel of the chunk
    uint8_t* d = tile + r * PITCH + c * 16;
    if (y >= a.H || xp >= a.W) continue;
    const uint8_t* s = a.src + static_cast<long long>(y) * a.sp + static_cast<long long>(xp) * E;
    if (a.ld16 && xp + 16 / E <= a.W) {
      const uint4 v = *reinterpret_cast<const uint4*>(s);
      uint32_t* dw = reinterpret_cast<uint32_t*>(d);
      dw[0] = v.x;
      dw[1] = v.y;
      dw[2] = v.z;
      dw[3] = v.w;
    } else {
      for (int b = 0; b < 16 && xp + b / E < a.W; ++b) d[b] = s[b];
    }
  }
  __syncthreads();

  // one 4x4 block per thread: rows 4by.., pixel columns 4bx..
  const int by = tid % (kT / 4), bx = tid / (kT / 4);
  uint32_t out[4][2];
  if (E == 1) {
    uint32_t v[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) v[i] = *reinterpret_cast<const uint32_t*>(tile + (4 * by + i) * PITCH + 4 * bx);
    transpose_block(v);  // v[j] = pixel column 4bx+j of rows 4by..4by+3
#pragma unroll
    for (int j = 0; j < 4; ++j) out[j][0] = v[j];
  } else {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const uint2 v = *reinterpret_cast<const uint2*>(tile + (4 * by + i) * PITCH + 8 * bx);
      out[i][0] = v.x;
      out[i][1] = v.y;
    }
    transpose4x4_u16(out);  // out[j] = pixel column 4bx+j of rows 4by..4by+3
  }
  // output row x = x0 + 4bx + j holds, from column y0 + 4by, four pixels
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int x = x0 + 4 * bx + j;
    const int y = y0 + 4 * by;
    if (x >= a.W || y >= a.H) continue;
    uint8_t* d = a.dst + static_cast<long long>(x) * a.dp + static_cast<long long>(y) * E;
    if (a.st4 && y + 4 <= a.H) {
      if (E == 1)
        *reinterpret_cast<uint32_t*>(d) = out[j][0];
      else
        *reinterpret_cast<uint2*>(d) = make_uint2(out[j][0], out[j][1]);
    } else {
      for (int i = 0; i < 4 && y + i < a.H; ++i) {
        const uint32_t wv = out[j][(i * E) / 4];
        const int sh = ((i * E) % 4) * 8;
        if (E == 1)
          d[i] = static_cast<uint8_t>(wv >> sh);
        else
          reinterpret_cast<uint16_t*>(d)[i] = static_cast<uint16_t>(wv >> sh);
      }
    }
  }
}

}  // namespace

cudaError_t transpose_launch(const void* src, long long sp, void* dst, long long dp, int W, int H, int esz,
                             cudaStream_t stream) {
  dim3 grid(cdiv(W, kT), cdiv(H, kT));
  const uintptr_t s = reinterpret_cast<uintptr_t>(src), d = reinterpret_cast<uintptr_t>(dst);
  if (esz == 1) {
    TrArgs<uint8_t> a{static_cast<const uint8_t*>(src), static_cast<uint8_t*>(dst), sp, dp, W, H,
                      (s % 16 == 0) && (sp % 16 == 0), (d % 4 == 0) && (dp % 4 == 0)};
    note_launch();
    transpose_kernel<uint8_t><<<grid, kTThreads, 0, stream>>>(a);
  } else {
    TrArgs<uint16_t> a{static_cast<const uint8_t*>(src), static_cast<uint8_t*>(dst), sp, dp, W, H,
                       (s % 16 == 0) && (sp % 16 == 0), (d % 8 == 0) && (dp % 8 == 0)};
    note_launch();
    transpose_kernel<uint16_t><<<grid, kTThreads, 0, stream>>>(a);
  }
  return cudaGetLastError();
}

}  // namespace morph
