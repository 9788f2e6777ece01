// Elementwise step of the composite operations (section 2: opening, closing
// and the morphological gradient are erosions, dilations and arithmetic):
// dst -= sub, pixel by pixel, for the gradient dilate - erode.  The operands
// are a dilation and an erosion of the same image by the same element, so
// dst >= sub in every pixel and no lane's subtraction wraps.
#include <cstdint>

#include "morph_common.cuh"
#include "morph_comp.cuh"
#include "morph_internal.h"

namespace morph {

namespace {

constexpr int kSubThreads = 256;

// One thread per 16-byte chunk of a row: the vector form when both rows'
// chunks are 16-byte aligned, pixel by pixel otherwise.
template <int E>
__global__ void __launch_bounds__(kSubThreads) sub_kernel(uint8_t* dst, long long dp, const uint8_t* sub,
                                                          long long sp, int row_bytes, int H) {
  pdl_launch_dependents();
  pdl_wait();
  const int nch = (row_bytes + 15) / 16;
  const long long total = static_cast<long long>(nch) * H;
  for (long long i = static_cast<long long>(blockIdx.x) * kSubThreads + threadIdx.x; i < total;
       i += static_cast<long long>(gridDim.x) * kSubThreads) {
    const int y = static_cast<int>(i / nch), c = static_cast<int>(i % nch);
    uint8_t* d = dst + static_cast<long long>(y) * dp + 16ll * c;
    const uint8_t* s = sub + static_cast<long long>(y) * sp + 16ll * c;
    const int n = row_bytes - 16 * c < 16 ? row_bytes - 16 * c : 16;
    if (n == 16 && !((reinterpret_cast<uintptr_t>(d) | reinterpret_cast<uintptr_t>(s)) & 15)) {
      uint4 a = *reinterpret_cast<const uint4*>(d);
      const uint4 b = *reinterpret_cast<const uint4*>(s);
      if (E == 1) {
        a.x = __vsub4(a.x, b.x);
        a.y = __vsub4(a.y, b.y);
        a.z = __vsub4(a.z, b.z);
        a.w = __vsub4(a.w, b.w);
      } else {
        a.x = __vsub2(a.x, b.x);
        a.y = __vsub2(a.y, b.y);
        a.z = __vsub2(a.z, b.z);
        a.w = __vsub2(a.w, b.w);
      }
      *reinterpret_cast<uint4*>(d) = a;
    } else if (E == 1) {
      for (int t = 0; t < n; ++t) d[t] = static_cast<uint8_t>(d[t] - s[t]);
    } else {
      for (int t = 0; t < n; t += 2)
        *reinterpret_cast<uint16_t*>(d + t) =
            static_cast<uint16_t>(*reinterpret_cast<const uint16_t*>(d + t) - *reinterpret_cast<const uint16_t*>(s + t));
    }
  }
}

// One CTA per output tile of the one-pass composite (morph_comp.cuh); HB
// bounds both halos (2, 4 or 8).
template <typename T, int KIND, int HB>
__global__ void __launch_bounds__(kCompThreads) comp_kernel(const CompArgs a) {
  __shared__ uint32_t smem[kCompSmemWords];
  pdl_wait();
  comp_tile<T, KIND, HB>(a, blockIdx.x, threadIdx.x, smem);
  pdl_launch_dependents();
}

using CompFn = void (*)(const CompArgs);

template <typename T, int HB>
CompFn comp_kernel_for(int kind) {
  return kind == kCompOpen    ? comp_kernel<T, kCompOpen, HB>
         : kind == kCompClose ? comp_kernel<T, kCompClose, HB>
                              : comp_kernel<T, kCompGradient, HB>;
}

template <typename T>
CompFn comp_kernel_for(int kind, int halo) {
  return halo <= 2 ? comp_kernel_for<T, 2>(kind) : halo <= 4 ? comp_kernel_for<T, 4>(kind) : comp_kernel_for<T, 8>(kind);
}

}  // namespace

bool comp_fits(int W, int H, int wx, int wy) {
  return wx >= 1 && wy >= 1 && wx <= kCompMaxW && wy <= kCompMaxW && W >= wx && H >= wy;
}

cudaError_t comp_launch(const void* src, long long sp, void* dst, long long dp, int W, int H, int esz, int kind,
                        int wx, int wy, int ax, int ay, bool pdl, cudaStream_t stream) {
  if (!comp_fits(W, H, wx, wy) || kind < kCompOpen || kind > kCompGradient) return cudaErrorInvalidValue;
  CompArgs a;
  a.src = static_cast<const uint8_t*>(src);
  a.dst = static_cast<uint8_t*>(dst);
  a.sp = sp;
  a.dp = dp;
  a.W = W;
  a.H = H;
  a.wx = wx;
  a.wy = wy;
  a.ax = ax;
  a.ay = ay;
  a.tiles_x = (W + kCompTX - 1) / kCompTX;
  const long long tiles = static_cast<long long>(a.tiles_x) * ((H + kCompTY - 1) / kCompTY);
  if (tiles > 0x7FFFFFFFll) return cudaErrorInvalidValue;
  const int halo = (wx > wy ? wx : wy) - 1;
  CompFn k = esz == 1 ? comp_kernel_for<uint8_t>(kind, halo) : comp_kernel_for<uint16_t>(kind, halo);
  return launch_pdl(pdl, k, dim3(static_cast<unsigned>(tiles)), dim3(kCompThreads), 0, stream, a);
}

cudaError_t sub_launch(void* dst, long long dp, const void* sub, long long sp, int row_bytes, int H, int esz,
                       cudaStream_t stream) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return cudaErrorInvalidDevice;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return cudaErrorInvalidDevice;
  const long long total = static_cast<long long>((row_bytes + 15) / 16) * H;
  long long blocks = (total + kSubThreads - 1) / kSubThreads;
  const long long cap = static_cast<long long>(sms) * 8;  // a few waves at most; the loop strides
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  auto* d = static_cast<uint8_t*>(dst);
  auto* s = static_cast<const uint8_t*>(sub);
  if (esz == 1)
    return launch_pdl(false, sub_kernel<1>, dim3(static_cast<unsigned>(blocks)), dim3(kSubThreads), 0, stream, d, dp,
                      s, sp, row_bytes, H);
  return launch_pdl(false, sub_kernel<2>, dim3(static_cast<unsigned>(blocks)), dim3(kSubThreads), 0, stream, d, dp, s,
                    sp, row_bytes, H);
}

}  // namespace morph
