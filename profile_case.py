"""Runs one erosion/dilation class a few times through the C ABI, for
profiler captures of a single kernel, e.g.

  python profile_case.py --dtype u8 --wx 1 --wy 101 --op erode --reps 3
  ncu --clock-control none -k regex:colv_kernel -s 2 -c 1 --set full -o prof \
      python profile_case.py --dtype u8 --wx 1 --wy 101 --reps 3

Inputs are seeded uniform images; nothing is checked or printed except a
one-line summary (launch count, mean event time of the launches).

`--packed-minmax` instead times the packed min intrinsics on their own (8
independent accumulators a thread, one intrinsic each per step): the 4-byte
form `__vminu4` against the 2 x 16-bit form `__vminu2`, the choice between
byte lanes and 16-bit lanes in every kernel, and `__vminu2` against the PTX
instruction `min.u16x2` written inline.  Under ncu,
`smsp__inst_executed.sum` of each launch divided by the warp-intrinsics it
prints gives the instructions each form issues:

  ncu --clock-control none --metrics smsp__inst_executed.sum -k regex:packed_minmax -c 2 \
      python profile_case.py --packed-minmax --reps 1
"""
from __future__ import annotations

import argparse
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


PACKED_MINMAX_SRC = r"""
#include <cstdint>
#include <cuda_runtime.h>

__device__ __forceinline__ uint32_t min_u16x2_ptx(uint32_t a, uint32_t b) {
  uint32_t r;
  asm("min.u16x2 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
  return r;
}

// 0: __vminu4 (4 bytes), 1: __vminu2 (2 x 16 bits), 2: the PTX instruction
// min.u16x2 written inline (sm_90 and later)
template <int FORM>
__global__ void packed_minmax_kernel(const uint32_t* in, uint32_t* out, int iters) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t a[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) a[i] = in[t] * (2654435761u + 2u * i);
  for (int k = 0; k < iters; ++k) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const uint32_t b = a[(i + 1) & 7];
      a[i] = FORM == 0 ? __vminu4(a[i], b) : FORM == 1 ? __vminu2(a[i], b) : min_u16x2_ptx(a[i], b);
    }
  }
  uint32_t r = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i) r ^= a[i];
  out[t] = r;
}

extern "C" int packed_minmax_launch(int form, const void* in, void* out, int iters, int blocks, int threads,
                                    void* stream) {
  const uint32_t* i = static_cast<const uint32_t*>(in);
  uint32_t* o = static_cast<uint32_t*>(out);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (form == 0)
    packed_minmax_kernel<0><<<blocks, threads, 0, s>>>(i, o, iters);
  else if (form == 1)
    packed_minmax_kernel<1><<<blocks, threads, 0, s>>>(i, o, iters);
  else
    packed_minmax_kernel<2><<<blocks, threads, 0, s>>>(i, o, iters);
  return static_cast<int>(cudaGetLastError());
}
"""


def packed_minmax(reps: int) -> int:
    """Times __vminu4 against __vminu2 (one launch per form and repetition)."""
    import ctypes
    import subprocess

    import torch

    bdir = os.path.join(ROOT, "_build")
    os.makedirs(bdir, exist_ok=True)
    cu, so = os.path.join(bdir, "packed_minmax.cu"), os.path.join(bdir, "packed_minmax.so")
    with open(cu, "w") as f:
        f.write(PACKED_MINMAX_SRC)
    subprocess.run(["nvcc", "-O3", "-shared", "-Xcompiler", "-fPIC", "-gencode", "arch=compute_103a,code=sm_103a",
                    "-lineinfo", cu, "-o", so], check=True)
    lib = ctypes.CDLL(so)
    lib.packed_minmax_launch.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_int, ctypes.c_void_p]
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    blocks, threads, iters = sms * 8, 256, 2048
    n = blocks * threads
    src = torch.randint(0, 2**31 - 1, (n,), dtype=torch.int32, device="cuda")
    dst = torch.empty_like(src)
    stream = torch.cuda.current_stream()
    warp_ops = (n // 32) * iters * 8
    best = {}
    for form, name in ((0, "__vminu4"), (1, "__vminu2"), (2, "min.u16x2")):
        times = []
        for r in range(3 + reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            rc = lib.packed_minmax_launch(form, src.data_ptr(), dst.data_ptr(), iters, blocks, threads,
                                          ctypes.c_void_p(stream.cuda_stream))
            e1.record(stream)
            torch.cuda.synchronize()
            if rc != 0:
                raise RuntimeError("packed_minmax_launch: CUDA error %d" % rc)
            if r >= 3:
                times.append(e0.elapsed_time(e1) * 1e-3)
        best[name] = min(times)
        print("packed_minmax %s: %d warp-intrinsics a launch, best %.1f us, %.2f T thread-ops/s" % (
            name, warp_ops, best[name] * 1e6, warp_ops * 32 / best[name] * 1e-12))
    print("packed_minmax time ratio __vminu4 / __vminu2: %.2f, __vminu2 / min.u16x2: %.2f" % (
        best["__vminu4"] / best["__vminu2"], best["__vminu2"] / best["min.u16x2"]))
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--dtype", choices=("u8", "u16"), default="u8")
    ap.add_argument("--width", type=int, default=4096)
    ap.add_argument("--height", type=int, default=4096)
    ap.add_argument("--wx", type=int, default=3)
    ap.add_argument("--wy", type=int, default=3)
    ap.add_argument("--op", choices=("erode", "dilate"), default="erode")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--cross-row", type=int, default=-1, help="force the x-pass crossover")
    ap.add_argument("--cross-col", type=int, default=-1, help="force the y-pass crossover")
    ap.add_argument("--tile", type=int, default=-1, help="force a tile configuration first")
    ap.add_argument("--colv", type=int, default=-1,
                    help="force the warp-tiled pass along y with this many rows per tile (0: model)")
    ap.add_argument("--rowv", type=int, default=-1,
                    help="force the register-blocked pass along x with this segment (0: model)")
    ap.add_argument("--kind", choices=("open", "close", "gradient"), default=None,
                    help="run morph_composite of this kind instead of one erosion or dilation")
    ap.add_argument("--one-pass", action="store_true",
                    help="with --kind: force the one-pass composite kernel (windows up to 9 x 9)")
    ap.add_argument("--colv-lanes", type=int, default=0,
                    help="bytes per lane of the warp-tiled pass along y (0: built-in rule; 4 or 8)")
    ap.add_argument("--packed-minmax", action="store_true",
                    help="time __vminu4 against __vminu2 on their own instead of a filter call")
    args = ap.parse_args(argv)
    if args.packed_minmax:
        return packed_minmax(args.reps)

    import torch
    from paper_2002_09474_gb300 import build as libbuild, synth
    libbuild.build()
    from paper_2002_09474_gb300 import morph

    dt = np.uint8 if args.dtype == "u8" else np.uint16
    code = morph.MORPH_U8 if dt == np.uint8 else morph.MORPH_U16
    morph.morph_set_tuning(code, args.cross_row, args.cross_col, args.tile)
    if args.colv >= 0 or args.colv_lanes:
        morph.morph_set_colv(1, max(args.colv, 0), args.colv_lanes)
    if args.rowv >= 0:
        morph.morph_set_rowv(1, args.rowv)
    img = synth.uniform_image(args.width, args.height, dt, seed=1)
    src = torch.from_numpy(img).cuda()
    dst = torch.empty_like(src)
    op = morph.MORPH_ERODE if args.op == "erode" else morph.MORPH_DILATE
    kinds = {"open": morph.MORPH_OPEN, "close": morph.MORPH_CLOSE, "gradient": morph.MORPH_GRADIENT}
    if args.one_pass:
        morph.morph_set_composite_kernel(1)
    times = []
    for _ in range(args.reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        if args.kind:
            morph.composite(src, dst, kinds[args.kind], args.wx, args.wy)
        else:
            morph.apply(src, dst, args.wx, args.wy, op=op)
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    morph.check_device_error()
    print("profile_case %s %dx%d %dx%d %s: %d calls, last %.1f us" % (
        args.dtype, args.width, args.height, args.wx, args.wy, args.kind or args.op, args.reps,
        times[-1] * 1e3))
    return 0


if __name__ == "__main__":
    sys.exit(main())
