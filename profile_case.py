"""Runs one erosion/dilation class a few times through the C ABI, for
profiler captures of a single kernel, e.g.

  python profile_case.py --dtype u8 --wx 1 --wy 101 --op erode --reps 3
  ncu --clock-control none -k regex:colv_kernel -s 2 -c 1 --set full -o prof \
      python profile_case.py --dtype u8 --wx 1 --wy 101 --reps 3

Inputs are seeded uniform images; nothing is checked or printed except a
one-line summary (launch count, mean event time of the launches).
"""
from __future__ import annotations

import argparse
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


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
    args = ap.parse_args(argv)

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
