"""Launch cases for the CPU emulator of the fused kernel (the same shapes,
windows, anchors, methods, tile shapes and pitches as the GPU parity tests).
Prints one case per line: esz op W H spad soff dpad doff wx wy ax ay cfg
cross_x cross_y seed kern.  Every case whose source is TMA-loadable (16-byte
pitch and offset) also appears in the persistent two-slot form (kern 1), and
every 1 x wy case (wy > 1) also through the column kernel (kern 2), every
wx x 1 case (wx > 1) also through the row kernel (kern 3), and every 1 x wy
case also through the warp-tiled van Herk/Gil-Werman kernel of the pass
along y (kern 4, its strip width varying with the seed); kern 5 is the
register-blocked pass along x; kern 6 the one-pass composite (op is then
the kind: opening, closing, gradient).  --only K keeps the cases of kernel K."""
import itertools
import sys

DIRECT, BLOCKED = 1000000, 0


def aligned_pad(w, esz):
    return (16 - (w * esz) % 16) % 16


def cases(full=True):
    seed = 1
    out = []

    def add(esz, op, w, h, spad, soff, dpad, doff, wx, wy, ax, ay, cfg, cx, cy):
        nonlocal seed
        out.append((esz, op, w, h, spad, soff, dpad, doff, wx, wy, ax, ay, cfg, cx, cy, seed))
        seed += 1

    shapes = [(1, 1), (2, 3), (5, 17), (33, 7), (67, 130), (129, 257), (200, 300)]
    wins = [(1, 1), (3, 3), (2, 5), (7, 1), (1, 9), (4, 4), (8, 8), (9, 16), (17, 8), (15, 15),
            (31, 7), (64, 65), (61, 61)]
    methods = {"direct": (DIRECT, DIRECT), "vhgw": (BLOCKED, BLOCKED), "mixed": (BLOCKED, DIRECT)}
    for esz in (1, 2):
        for m, (cx, cy) in methods.items():
            for (h, w) in shapes:
                for n, (wx, wy) in enumerate(wins):
                    for op in (0, 1):
                        pad = aligned_pad(w, esz) if (n + op) % 2 else 0
                        add(esz, op, w, h, pad, 0, pad, 0, wx, wy, wx // 2, wy // 2, -1, cx, cy)
        for cfg in range(8):
            for c in (DIRECT, BLOCKED):
                for (wx, wy, ax, ay) in ((3, 5, 1, 2), (8, 2, 7, 0), (21, 51, 10, 25), (101, 1, 50, 0),
                                         (1, 33, 0, 16), (127, 127, 63, 63)):
                    for op in (0, 1):
                        for pad in (0, aligned_pad(301, esz)):
                            add(esz, op, 301, 177, pad, 0, pad, 0, wx, wy, ax, ay, cfg, c, c)
        for c in (DIRECT, BLOCKED):
            for (wx, wy) in ((4, 3), (6, 6), (5, 2)):
                for ax, ay in itertools.product(range(wx), range(wy)):
                    add(esz, 0, 70, 45, aligned_pad(70, esz), 0, aligned_pad(70, esz), 0, wx, wy, ax, ay,
                        -1, c, c)
        for pad, off, dpad, doff in [(0, 0, 0, 0), (aligned_pad(150, esz), 0, 32, 0), (13 * esz, 0, 13 * esz, 0),
                                     (6, 4, 2, 8), (esz, esz, 3 * esz, esz)]:
            for (wx, wy) in ((3, 3), (17, 9), (40, 40)):
                for op in (0, 1):
                    add(esz, op, 150, 90, pad, off, dpad, doff, wx, wy, wx // 2, wy // 2, -1, -1, -1)
        for (wx, wy, ax, ay) in ((75, 47, 37, 23), (200, 3, 0, 1), (3, 500, 2, 499), (1000, 1000, 1, 998)):
            for op in (0, 1):
                add(esz, op, 37, 23, aligned_pad(37, esz), 0, 0, 0, wx, wy, ax, ay, -1, -1, -1)
        if full:
            for cfg in range(8):
                for c in (DIRECT, BLOCKED):
                    for (wx, wy) in ((3, 3), (1, 17), (17, 1), (21, 51)):
                        for op in (0, 1):
                            add(esz, op, 512, 256, 0, 0, 0, 0, wx, wy, wx // 2, wy // 2, cfg, c, c)
    both = []
    for c in out:
        both.append(c + (0,))
        esz, w, spad, soff, wx, wy = c[0], c[2], c[4], c[5], c[8], c[9]
        if (w * esz + spad) % 16 == 0 and soff % 16 == 0:
            both.append(c + (1,))
    # the column kernel: every 1 x wy case, plus tall images and long windows
    col = [c for c in out if c[8] == 1 and c[9] > 1]
    seed = 100000
    for esz in (1, 2):
        for (w, h) in ((128, 1000), (300, 2100), (64, 700), (1, 900), (257, 33)):
            for wy in (2, 7, 8, 9, 10, 16, 17, 31, 63, 101, 255, 700):
                for op in (0, 1):
                    for cross in (0, 1000000):
                        pad = aligned_pad(w, esz) if (wy + op) % 2 else 0
                        col.append((esz, op, w, h, pad, 0, pad, 0, 1, wy, 0, wy // 2, -1, cross, cross, seed))
                        seed += 1
    for c in col:
        both.append(c + (2,))
    # the row kernel: every wx x 1 case, plus wide images, long windows, all
    # anchor extremes, unaligned pitches and offsets
    row = [c for c in out if c[9] == 1 and c[8] > 1]
    for esz in (1, 2):
        for (w, h) in ((256, 64), (257, 65), (1000, 70), (2100, 9), (7, 130), (513, 128)):
            for wx in (2, 3, 8, 9, 10, 17, 31, 63, 101, 255, 700):
                for ax in sorted({0, wx // 2, wx - 1}):
                    for op in (0, 1):
                        for cross in (0, 1000000):
                            n = len(row)
                            if n % 3 == 0:
                                pad, off, dpad, doff = aligned_pad(w, esz), 0, aligned_pad(w, esz), 0
                            elif n % 3 == 1:
                                pad, off, dpad, doff = 0, 0, 0, 0
                            else:
                                pad, off, dpad, doff = 3 * esz, esz, 5 * esz, 2 * esz
                            row.append((esz, op, w, h, pad, off, dpad, doff, wx, 1, ax, 0, -1, cross, cross, seed))
                            seed += 1
    for c in row:
        both.append(c + (3,))
    # the warp-tiled pass along y: every 1 x wy case, plus tall images, long
    # windows, anchor extremes, unaligned pitches and offsets
    colv = [c for c in out if c[8] == 1 and c[9] > 1]
    for esz in (1, 2):
        for (w, h) in ((128, 1000), (300, 2100), (64, 700), (1, 900), (257, 33), (190, 41)):
            for wy in (2, 3, 7, 8, 9, 16, 17, 31, 63, 101, 255, 700):
                for ay in sorted({0, wy // 2, wy - 1}):
                    for op in (0, 1):
                        n = len(colv)
                        if n % 3 == 0:
                            pad, off, dpad, doff = aligned_pad(w, esz), 0, aligned_pad(w, esz), 0
                        elif n % 3 == 1:
                            pad, off, dpad, doff = 0, 0, 0, 0
                        else:
                            pad, off, dpad, doff = 3 * esz, esz, 5 * esz, 2 * esz
                        colv.append((esz, op, w, h, pad, off, dpad, doff, 1, wy, 0, ay, -1, -1, -1, seed))
                        seed += 1
    for c in colv:
        both.append(c + (4,))
    # the register-blocked pass along x: the row kernel's cases, plus aligned
    # rows (so that the kernel takes them) of ragged widths and heights
    rowv = [c for c in row if 9 <= c[8] <= 256]
    for esz in (1, 2):
        for (w, h) in ((256, 64), (257, 65), (1000, 70), (2100, 9), (1500, 130), (513, 13), (40, 20)):
            for wx in (9, 10, 16, 17, 31, 63, 101, 127, 255, 256):
                for ax in sorted({0, wx // 2, wx - 1}):
                    for op in (0, 1):
                        n = len(rowv)
                        pad = (16 - (w * esz) % 16) % 16
                        dpad, doff = (pad, 0) if n % 2 else (esz, 3 * esz)
                        rowv.append((esz, op, w, h, pad, 0, dpad, doff, wx, 1, ax, 0, -1, -1, -1, seed))
                        seed += 1
    for c in rowv:
        both.append(c + (5,))
    # the one-pass composite (op: 0 opening, 1 closing, 2 gradient): windows
    # up to 9 x 9, every anchor of some windows, ragged and tiny images
    # (never smaller than the window), unaligned pitches and offsets
    comp = []
    for esz in (1, 2):
        for (w, h) in ((128, 32), (129, 33), (300, 70), (9, 9), (17, 5), (5, 40), (257, 95), (64, 31)):
            for (wx, wy) in ((1, 1), (3, 3), (2, 5), (9, 9), (1, 9), (9, 1), (4, 8), (7, 6)):
                if wx > w or wy > h:
                    continue
                for kind in (0, 1, 2):
                    n = len(comp)
                    ax, ay = [(0, wx // 2, wx - 1)[n % 3], (wy - 1, 0, wy // 2)[n % 3]]
                    if n % 3 == 0:
                        pad, off, dpad, doff = aligned_pad(w, esz), 0, aligned_pad(w, esz), 0
                    elif n % 3 == 1:
                        pad, off, dpad, doff = 0, 0, 0, 0
                    else:
                        pad, off, dpad, doff = 3 * esz, esz, 5 * esz, 2 * esz
                    comp.append((esz, kind, w, h, pad, off, dpad, doff, wx, wy, ax, ay, -1, -1, -1, seed))
                    seed += 1
        for (wx, wy) in ((4, 3), (5, 5)):
            for ax, ay in itertools.product(range(wx), range(wy)):
                comp.append((esz, (ax + ay) % 3, 70, 45, 0, 0, 0, 0, wx, wy, ax, ay, -1, -1, -1, seed))
                seed += 1
    for c in comp:
        both.append(c + (6,))
    return both


if __name__ == "__main__":
    only = int(sys.argv[sys.argv.index("--only") + 1]) if "--only" in sys.argv else None
    for c in cases(full="--quick" not in sys.argv):
        if only is None or c[-1] == only:
            print(*c)
