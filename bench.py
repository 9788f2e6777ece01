"""Benchmark: erosion/dilation throughput (Gpixel/s) and fraction of the HBM
roofline on the 4096x4096 workload, through the C ABI.

Workload (one step): 4096x4096 images in uint8 and uint16, each a uniform
random image and a smooth gradient with noise (synthetic, seeded); windows
1x101, 101x1, 21x51 and 127x127 (wx x wy, anchor at the centre); erosion and
dilation of each -- 32 single-image calls.  Every call reads a different copy
of its input (8 rotating copies per image), so inputs come from HBM, not L2
(129 MB).  Inputs are resident in device memory when timing starts.

Reported (one JSON line on rank 0):
  value        whole-job Gpixel/s (output pixels of all ranks / max time)
  roofline     the dominant kernel class: algorithmic bytes (read + write one
               image) / its mean CUDA-event launch time, against the measured
               HBM copy bandwidth
  e2e          the same step through morph_apply_host_batch with pinned host buffers
               (host->device and device->host copies inside the timed region)
  cpu_baseline the brute-force CPU oracle on a bounded sample of the step,
               (separable) the oracle's separable van Herk/Gil-Werman
               checker on the whole step, all cores and one core, and
               (paper_method) the paper's own NEON method against its scalar
               form on the host's Arm cores, one thread
  breakdown    per (dtype, window) class: mean us per call, Gpixel/s, GB/s
  batched      2000 uneven u8 images (sides 64..2048, windows 1..63): images/s
               of the batch plan (one CUDA graph) vs the 2000 per-image calls
               captured in a CUDA graph
  transposes   transpose_u8/u16 of a 4096x4096 image: Gpixel/s, HBM fraction
  serving      Poisson request streams (1k, 2k, 5k, 10k, 20k req/s, 10 s each)
               through the continuous-batching server (4 GB admission
               budget): p50/p99 latency and throughput
``--impl reference`` times the CPU oracle alone (the reference arm).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2002_09474_gb300 import synth  # noqa: E402

SIDE = 4096
WINDOWS = synth.C3_WINDOWS  # (wx, wy)
OPS = (0, 1)                # erode, dilate
DTYPES = (np.uint8, np.uint16)
IMAGES = ("uniform", "gradient")
ROTATE = 8                  # input copies per image (defeats L2 reuse)
STEP_STREAMS = 2            # streams the step's independent calls run on (one per image kind)
METRIC = "erosion/dilation Gpixel/s (4096x4096 u8+u16, 4 windows, erode+dilate)"
UNIT = "Gpixel/s"
KERNEL_SOURCES = None  # every file of the CUDA library's sources


def workload_config():
    return {"workload": "4096x4096 u8+u16 (uniform, gradient+noise), windows 1x101 101x1 21x51 "
                        "127x127, erode+dilate: 32 calls per step",
            "image": [SIDE, SIDE], "windows_wx_wy": [list(w) for w in WINDOWS],
            "dtypes": ["u8", "u16"], "ops": ["erode", "dilate"], "calls_per_step": 32,
            "l2": "inputs rotate over %d copies per image (>1 GB between reuses of a copy)" % ROTATE}


def step_runs():
    """The 32 calls of one step: (dtype, image kind, (wx, wy), op)."""
    return [(dt, kind, w, op) for dt in DTYPES for kind in IMAGES for w in WINDOWS for op in OPS]


def make_image(dtype, kind):
    seed = 3 if dtype == np.uint8 else 4
    if kind == "uniform":
        return synth.uniform_image(SIDE, SIDE, dtype, seed=seed)
    return synth.gradient_image(SIDE, SIDE, dtype, seed=seed + 100)


def kernel_hash() -> str:
    """Hash of the CUDA library's sources: the committed DRAM traffic is
    reported only while it was measured on these exact kernels."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2002_09474_gb300", "csrc")
    for f in sorted(os.listdir(csrc)):
        if f.endswith((".cu", ".cuh", ".cpp", ".h")):
            with open(os.path.join(csrc, f), "rb") as fh:
                h.update(f.encode() + b"\0" + fh.read())
    return h.hexdigest()[:16]


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def load_traffic(kernel_class: str):
    """DRAM bytes per call of a class (all its launches) from the committed
    ncu summary, if it was taken on the current kernel sources: (back to
    back, the way the step runs the calls; each launch after a cache flush),
    or (None, None)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            t = json.load(f)
    except (OSError, ValueError):
        return None, None
    if t.get("kernel_hash") != kernel_hash():
        return None, None
    v = t.get("classes", {}).get(kernel_class)
    if not isinstance(v, dict):
        return None, None
    return v.get("back_to_back"), v.get("cache_flushed")


# ---------------------------------------------------------------------------
# clocks
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "100", "-i", self.gpu_id],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.2)
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def gpu_id_for_smi(torch) -> str:
    try:
        u = torch.cuda.get_device_properties(torch.cuda.current_device()).uuid
        s = str(u)
        return s if s.startswith("GPU-") else "GPU-" + s
    except Exception:
        vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
        return vis.split(",")[0] if vis else "0"


# ---------------------------------------------------------------------------
# CPU oracle baseline (bounded sample)
# ---------------------------------------------------------------------------
def oracle_sample(images, target_ops: float = 1.5e9, seed: int = 7):
    """Times the brute-force oracle on sampled output pixels of every call of
    the step and extrapolates the step's CPU time.  Returns (Gpixel/s,
    threads, seconds spent, description)."""
    import oracle
    g = synth.rng(seed)
    est_step_s = 0.0
    spent = 0.0
    npts_total = 0
    for (dt, kind, (wx, wy), op) in step_runs():
        img = images[(dt, kind)]
        n = int(max(256, min(SIDE * SIDE, target_ops / (wx * wy))))
        xs = g.integers(0, SIDE, size=n)
        ys = g.integers(0, SIDE, size=n)
        t0 = time.perf_counter()
        oracle.morph_points(img, wx, wy, wx // 2, wy // 2, op, xs, ys)
        dt_s = time.perf_counter() - t0
        spent += dt_s
        npts_total += n
        est_step_s += dt_s * (SIDE * SIDE) / n
    step_px = len(step_runs()) * SIDE * SIDE
    desc = ("brute-force oracle (section 2 definition) at %d random output pixels of the "
            "step's 32 calls (about %.1e window cells per call), step time extrapolated by "
            "pixel count" % (npts_total, target_ops))
    return step_px / est_step_s / 1e9, oracle.num_threads(), spent, desc


PAPER_ARM_CONTEXT = ("paper's own ratios, Samsung Exynos 5422 (ARM, one thread, gcc with NEON intrinsics), "
                     "context only: NEON erosion/dilation 3x its scalar van Herk/Gil-Werman; NEON 8x8 u16 "
                     "transpose 5.7x scalar (114 -> 20 ns), 16x16 u8 transpose 12x (565 -> 47 ns)")


def paper_method_sample() -> dict:
    """The paper's CPU method (cpu_method/) on the host's Arm cores, one
    thread: its NEON form against its scalar form for 8-bit erosion of an
    800 x 600 image (the paper's image size) at square windows 3, 15, 31 and
    61, both passes by the direct method and both by van Herk/Gil-Werman; and
    section 4's block transposes (ns per block, 100k blocks).  Every form's
    output is checked against the oracle first.  The paper's own ratios are
    quoted beside it as context."""
    import cpu_method as cm
    import oracle
    if not cm.has_neon():
        return {"unavailable": "the NEON form needs an aarch64 host"}

    def per_call(fn, min_s=0.2):
        fn()
        n, t0 = 0, time.perf_counter()
        while True:
            fn()
            n += 1
            dt = time.perf_counter() - t0
            if dt >= min_s:
                return dt / n

    img = synth.uniform_image(800, 600, np.uint8, seed=11)
    out = {"image": "800x600 u8 uniform, erosion, one thread"}
    for w in (3, 15, 31, 61):
        want = oracle.morph(img, w, w, w // 2, w // 2, "erode")
        row = {}
        for method in ("direct", "vhgw"):
            for vec in (False, True):
                if not np.array_equal(cm.morph(img, w, w, op="erode", method=method, vector=vec), want):
                    raise RuntimeError("paper CPU method differs from the oracle")
                t = per_call(lambda: cm.morph(img, w, w, op="erode", method=method, vector=vec))
                row["%s_%s_ms" % (method, "neon" if vec else "scalar")] = round(t * 1e3, 3)
            row["%s_neon_over_scalar" % method] = round(row["%s_scalar_ms" % method] / row["%s_neon_ms" % method], 2)
        out["%dx%d" % (w, w)] = row
    g = synth.rng(12)
    for kind, blocks in (("u8_16x16", g.integers(0, 256, (100000, 16, 16), dtype=np.uint8)),
                         ("u16_8x8", g.integers(0, 65536, (100000, 8, 8), dtype=np.uint16))):
        k = "u8" if kind.startswith("u8") else "u16"
        ts = {}
        for vec in (False, True):
            if not np.array_equal(cm.transpose_blocks(k, blocks[:64], vec), blocks[:64].transpose(0, 2, 1)):
                raise RuntimeError("paper CPU transpose differs")
            ts[vec] = per_call(lambda: cm.transpose_blocks(k, blocks, vec)) / blocks.shape[0]
        out["transpose_" + kind] = {"scalar_ns": round(ts[False] * 1e9, 1), "neon_ns": round(ts[True] * 1e9, 1),
                                    "neon_over_scalar": round(ts[False] / ts[True], 2)}
    out["paper_context"] = ("paper (Samsung Exynos 5422, one thread): NEON erosion/dilation about 3x its scalar "
                            "van Herk/Gil-Werman; NEON 8x8 u16 transpose 5.7x scalar (114 -> 20 ns), 16x16 u8 "
                            "transpose 12x (565 -> 47 ns)")
    return out


def separable_sample(images):
    """The fair CPU speed baseline: the oracle's separable van Herk/Gil-Werman
    checker (sections 5 and 5.1.1: two 1-D passes, O(1) operations per pixel
    and pass, whatever the window) on the step's own full-size images.  All
    cores: every call of the step; one core: one call per window class (u8
    and u16 uniform erosion), extrapolated by pixel count.  Returns a dict
    for cpu_baseline."""
    import oracle
    cores = oracle.num_threads()
    t0 = time.perf_counter()
    for (dt, kind, (wx, wy), op) in step_runs():
        oracle.sep_vhgw(images[(dt, kind)], wx, wy, wx // 2, wy // 2, op)
    t_all = time.perf_counter() - t0
    step_px = len(step_runs()) * SIDE * SIDE
    prev = oracle.set_threads(1)
    try:
        t1, n1 = 0.0, 0
        for dt in DTYPES:
            for (wx, wy) in WINDOWS:
                t = time.perf_counter()
                oracle.sep_vhgw(images[(dt, "uniform")], wx, wy, wx // 2, wy // 2, 0)
                t1 += time.perf_counter() - t
                n1 += 1
    finally:
        oracle.set_threads(prev)
    one_core = n1 * SIDE * SIDE / t1 / 1e9
    return {"value": round(step_px / t_all / 1e9, 5), "unit": UNIT, "cores": cores,
            "kind": "oracle (separable van Herk/Gil-Werman checker)",
            "single_core_value": round(one_core, 5), "seconds": round(t_all + t1, 1),
            "sample": "all cores: the full step (32 calls at 4096x4096); one core: %d calls (each window "
                      "class, u8 and u16, uniform image, erosion)" % n1,
            "paper_context": PAPER_ARM_CONTEXT}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    images = {(dt, k): make_image(dt, k) for dt in DTYPES for k in IMAGES}
    for _ in range(args.warmup):
        oracle_sample(images, target_ops=5e7)
    vals, spent_total, desc, cores = [], 0.0, "", 1
    t0 = time.perf_counter()
    for _ in range(args.steps):
        v, cores, spent, desc = oracle_sample(images, target_ops=5e7)
        vals.append(v)
        spent_total += spent
    wall = time.perf_counter() - t0
    value = statistics.mean(vals)
    step_px = len(step_runs()) * SIDE * SIDE
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": step_px / (value * 1e9) * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u8+u16", "data": "synthetic",
            "config": workload_config(),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0},
            "wall_s": wall}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def measure_small_images(torch, morph, reps: int = 7) -> dict:
    """The small single-image workloads, as CUDA-graph replays of 32 calls
    over 8 input buffers: a 640 x 480 u8 uniform image eroded by 3 x 3
    (latency-bound: 0.3 MB), and the 1920 x 1080 u8 document-like page eroded
    and dilated by 3, 7, 15, 31 and 61 square windows."""
    def time_calls(img, wx, wy, op):
        h, w = img.shape
        srcs = [torch.from_numpy(img).cuda() for _ in range(8)]
        dsts = [torch.empty_like(srcs[0]) for _ in range(8)]

        def calls():
            sh = torch.cuda.current_stream().cuda_stream
            for i in range(32):
                rc = morph.morph_apply(srcs[i % 8].data_ptr(), w, dsts[i % 8].data_ptr(), w, w, h, morph.MORPH_U8, op,
                                       wx, wy, wx // 2, wy // 2, sh)
                if rc != 0:
                    raise morph.MorphError("morph_apply", rc)
        calls()
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            calls()
        for _ in range(2):
            g.replay()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            g.replay()
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1) * 1e3 / 32)
        us = sorted(ts)[len(ts) // 2]
        return {"us_per_call": round(us, 2), "gpix_s": round(w * h / us / 1e3, 1)}

    out = {"640x480_u8_erode_3x3": time_calls(synth.uniform_image(640, 480, np.uint8, seed=1), 3, 3,
                                               morph.MORPH_ERODE)}
    doc = synth.document_image(1920, 1080, seed=2)
    for k in (3, 7, 15, 31, 61):
        for op, name in ((morph.MORPH_ERODE, "erode"), (morph.MORPH_DILATE, "dilate")):
            out["1920x1080_doc_%s_%dx%d" % (name, k, k)] = time_calls(doc, k, k, op)
    return out


def measure_composite(torch, morph, reps: int = 7, peak: float = 6800.0) -> dict:
    """Opening, closing and gradient of a 4096 x 4096 image (u8 and u16;
    3 x 3 and 9 x 9, which take the one-pass kernel, 21 x 51 and 127 x 127,
    which take two calls through an intermediate) as one morph_composite
    call, against the same steps as separate calls into a caller buffer
    (opening and closing: two morph_apply calls; gradient: two calls and a
    torch subtraction).  Both are timed as CUDA-graph replays of 8 calls;
    the results are checked identical first.  Algorithmic bytes: read and
    write the image once (frac_of_hbm against the measured copy peak)."""
    out = {}
    for dt, tdt, code, name in ((np.uint8, torch.uint8, morph.MORPH_U8, "u8"),
                                (np.uint16, torch.uint16, morph.MORPH_U16, "u16")):
        img = synth.uniform_image(SIDE, SIDE, dt, seed=960)
        esz = np.dtype(dt).itemsize
        srcs = [torch.from_numpy(img).cuda() for _ in range(4)]
        dsts = [torch.empty_like(srcs[0]) for _ in range(4)]
        tmp = torch.empty_like(srcs[0])
        pitch = SIDE * esz
        for (wx, wy) in ((3, 3), (9, 9), (21, 51), (127, 127)):
            ax, ay = wx // 2, wy // 2
            rx, ry = wx - 1 - ax, wy - 1 - ay
            for kind, kname in ((morph.MORPH_OPEN, "open"), (morph.MORPH_CLOSE, "close"),
                                (morph.MORPH_GRADIENT, "gradient")):
                first = morph.MORPH_DILATE if kind == morph.MORPH_CLOSE else morph.MORPH_ERODE
                second = morph.MORPH_ERODE if kind == morph.MORPH_CLOSE else morph.MORPH_DILATE
                sa, sb = (ax, ay) if kind == morph.MORPH_GRADIENT else (rx, ry)

                def one(i, sh):
                    rc = morph.morph_composite(srcs[i % 4].data_ptr(), pitch, dsts[i % 4].data_ptr(), pitch, SIDE,
                                               SIDE, code, kind, wx, wy, ax, ay, sh)
                    if rc != 0:
                        raise morph.MorphError("morph_composite", rc)

                def sep(i, sh):
                    s, d = srcs[i % 4], dsts[i % 4]
                    a_src = s.data_ptr()
                    b_src = a_src if kind == morph.MORPH_GRADIENT else tmp.data_ptr()
                    for (sp_, dp_, op, x_, y_) in ((a_src, tmp.data_ptr(), first, ax, ay),
                                                   (b_src, d.data_ptr(), second, sa, sb)):
                        rc = morph.morph_apply(sp_, pitch, dp_, pitch, SIDE, SIDE, code, op, wx, wy, x_, y_, sh)
                        if rc != 0:
                            raise morph.MorphError("morph_apply", rc)
                    if kind == morph.MORPH_GRADIENT:
                        # dilation minus erosion on the current stream (u16 through
                        # int16 views: the same bits, and dilate >= erode)
                        dv, tv = (d, tmp) if d.dtype == torch.uint8 else (d.view(torch.int16), tmp.view(torch.int16))
                        torch.sub(dv, tv, out=dv)

                st = torch.cuda.current_stream()
                one(0, st.cuda_stream)
                torch.cuda.synchronize()
                ref = dsts[0].clone()
                sep(0, st.cuda_stream)
                torch.cuda.synchronize()
                if not torch.equal(ref, dsts[0]):
                    raise RuntimeError("composite differs from separate calls")
                times = {}
                for label, fn in (("composite", one), ("separate", sep)):
                    g = torch.cuda.CUDAGraph()
                    with torch.cuda.graph(g):
                        for i in range(8):
                            fn(i, torch.cuda.current_stream().cuda_stream)
                    for _ in range(2):
                        g.replay()
                    torch.cuda.synchronize()
                    ts = []
                    for _ in range(reps):
                        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                        e0.record()
                        g.replay()
                        e1.record()
                        torch.cuda.synchronize()
                        ts.append(e0.elapsed_time(e1) * 1e3 / 8)
                    times[label] = round(sorted(ts)[len(ts) // 2], 2)
                out["%s_%s_%dx%d" % (name, kname, wx, wy)] = {
                    "us_per_call": times["composite"], "separate_calls_us": times["separate"],
                    "gpix_s": round(SIDE * SIDE / times["composite"] / 1e3, 1),
                    "frac_of_hbm": round(2 * esz * SIDE * SIDE / (times["composite"] * 1e3) / peak, 3)}
        del srcs, dsts, tmp
    return out


def measure_transposes(torch, morph, peak: float, peak_kind: str, reps: int = 9) -> dict:
    """transpose_u8 / transpose_u16 (section 4) of a 4096 x 4096 image, as
    CUDA-graph replays of 8 calls over 8 input copies (inputs larger than L2
    in total): us per call, Gpixel/s and the fraction of the HBM roofline
    (algorithmic bytes: read and write the image once).  The output is
    checked against torch's transpose first.  The paper's Table 1 figures are
    quoted beside them as context."""
    out = {}
    for dt, tdt, fn, name in ((np.uint8, torch.uint8, morph.transpose_u8, "u8"),
                              (np.uint16, torch.uint16, morph.transpose_u16, "u16")):
        esz = np.dtype(dt).itemsize
        base = torch.from_numpy(synth.uniform_image(SIDE, SIDE, dt, seed=970)).cuda()
        srcs = [base] + [base.clone() for _ in range(7)]
        dsts = [torch.empty_like(base) for _ in range(2)]
        pitch = SIDE * esz

        def calls():
            sh = torch.cuda.current_stream().cuda_stream
            for i in range(8):
                rc = fn(srcs[i].data_ptr(), SIDE, SIDE, pitch, dsts[i % 2].data_ptr(), pitch, sh)
                if rc != 0:
                    raise morph.MorphError(fn.__name__, rc)
        calls()
        torch.cuda.synchronize()
        if not torch.equal(dsts[1], srcs[7].t()):
            raise RuntimeError("%s differs from torch's transpose" % fn.__name__)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            calls()
        for _ in range(2):
            g.replay()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            g.replay()
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1) * 1e3 / 8)
        us = sorted(ts)[len(ts) // 2]
        gbs = 2 * esz * SIDE * SIDE / (us * 1e-6) / 1e9
        out["%s_4096x4096" % name] = {"us_per_call": round(us, 2), "gpix_s": round(SIDE * SIDE / us / 1e3, 1),
                                      "gb_s": round(gbs, 1), "frac_of_%s_hbm" % peak_kind: round(gbs / peak, 3)}
        del srcs, dsts, base, g
    out["paper_context"] = ("Table 1, Samsung Exynos 5422 (ARM NEON): 8x8 u16 transpose 114 -> 20 ns "
                            "(5.7x over scalar), 16x16 u8 transpose 565 -> 47 ns (12x); a single 8x8 or "
                            "16x16 block, not a whole image")
    return out


def measure_batched(torch, morph, reps: int = 5) -> dict:
    """2000 uneven u8 images (inputs 2.2 GB, larger than L2): one batch plan
    (its launches captured once in a CUDA graph) against the same 2000
    images as per-image morph_apply calls, also captured once in a CUDA
    graph, both replayed on one stream; plus morph_batch called directly.
    Rows are pitched to 128 bytes, as a pitched allocation lays them out.
    Identical output is checked on every image before timing."""
    import ctypes
    specs = synth.batch_specs(2000, seed=5)
    pix = synth.batch_pixels(specs, seed=5)
    pitches = [(sp.width + 127) // 128 * 128 for sp in specs]
    srcs, outs, alone = [], [], []
    for p, sp, pt in zip(pix, specs, pitches):
        s = torch.empty((sp.height, pt), dtype=torch.uint8, device="cuda")
        s[:, :sp.width] = torch.from_numpy(p).cuda()
        srcs.append(s)
        outs.append(torch.empty_like(s))
        alone.append(torch.empty_like(s))
    del pix
    arr = (morph.MorphDesc * len(specs))()
    for d, s, o, sp, pt in zip(arr, srcs, outs, specs, pitches):
        d.src, d.dst, d.width, d.height = s.data_ptr(), o.data_ptr(), sp.width, sp.height
        d.src_pitch = d.dst_pitch = pt
        d.wx, d.wy, d.anchor_x, d.anchor_y, d.op = sp.wx, sp.wy, sp.ax, sp.ay, sp.op
        d.dtype = morph.MORPH_U8
    stream = torch.cuda.current_stream()
    plan = ctypes.c_void_p()
    rc = morph.morph_batch_plan_create(arr, len(specs), ctypes.byref(plan))
    if rc != 0:
        raise morph.MorphError("morph_batch_plan_create", rc)

    def per_image_calls():
        sh = torch.cuda.current_stream().cuda_stream
        for s, a, sp, pt in zip(srcs, alone, specs, pitches):
            rc = morph.morph_apply(s.data_ptr(), pt, a.data_ptr(), pt, sp.width, sp.height,
                                   morph.MORPH_U8, sp.op, sp.wx, sp.wy, sp.ax, sp.ay, sh)
            if rc != 0:
                raise morph.MorphError("morph_apply", rc)

    def graph():
        rc = morph.morph_batch_plan_launch(plan, stream.cuda_stream)
        if rc != 0:
            raise morph.MorphError("morph_batch_plan_launch", rc)

    def batch_call():
        rc = morph.morph_batch(arr, len(specs), stream.cuda_stream)
        if rc != 0:
            raise morph.MorphError("morph_batch", rc)

    def timed(fn):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    try:
        graph()
        per_image_calls()
        torch.cuda.synchronize()
        same = all(torch.equal(o[:, :sp.width], a[:, :sp.width]) for o, a, sp in zip(outs, alone, specs))
        n0 = morph.morph_launch_count()
        g_img = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g_img):
            per_image_calls()
        per_image_launches = morph.morph_launch_count() - n0
        t_img = timed(g_img.replay)
        t_graph = timed(graph)
        t_batch = timed(batch_call)
        del g_img
    finally:
        morph.morph_batch_plan_destroy(plan)
    morph.check_device_error()
    n = len(specs)
    px = sum(sp.width * sp.height for sp in specs)
    return {"workload": "2000 u8 images, sides uniform 64..2048, windows uniform 1..63, "
                        "random erode/dilate (seed 5), rows pitched to 128 bytes",
            "pixels": px, "identical_to_per_image": bool(same),
            "graph_images_s": round(n / (t_graph * 1e-3), 1),
            "per_image_images_s": round(n / (t_img * 1e-3), 1),
            "morph_batch_images_s": round(n / (t_batch * 1e-3), 1),
            "graph_gpix_s": round(px / (t_graph * 1e-3) / 1e9, 2),
            "per_image_gpix_s": round(px / (t_img * 1e-3) / 1e9, 2),
            "graph_vs_per_image": round(t_img / t_graph, 3),
            "per_image_form": "the 2000 morph_apply calls captured once in a CUDA graph (%d kernel launches), "
                              "replayed" % per_image_launches,
            "ms": {"graph": round(t_graph, 3), "per_image_graph": round(t_img, 3),
                   "morph_batch": round(t_batch, 3)}}


def measure_serving(torch, rates=(5000.0,), duration_s: float = 3.0, host_copies: bool = False) -> list:
    """Poisson request streams through the continuous-batching server, 4 GB
    admission budget.  Inputs pre-staged in device memory (host-to-device
    copies excluded), or, with host_copies, pinned host images copied in and
    results copied back to pinned host buffers inside each request's latency
    (HostCopyExecutor).  A short run at the same rate warms the pools first;
    the timed requests are generated before it, so that the timed run starts
    on a busy GPU (an idle GPU's clocks take tens of milliseconds to come
    back up)."""
    from paper_2002_09474_gb300 import serve
    if host_copies:
        pool_img, pool_dev = serve.host_arena(torch, seed=6)
        ex = serve.HostCopyExecutor(n_streams=4)
        make = serve.make_host_requests
    else:
        pool_img, pool_dev = serve.source_pool(torch, seed=6)
        ex = serve.GpuExecutor(n_streams=4)
        make = serve.make_requests
    out = []
    for rate in rates:
        rs = make(rate, duration_s, pool_img, pool_dev, seed=6)
        warm = make(rate, min(0.5, duration_s), pool_img, pool_dev, seed=60)
        serve.Server(ex, budget_bytes=4 << 30).run(warm, timeout_s=300)
        st = serve.Server(ex, budget_bytes=4 << 30).run(rs, timeout_s=300)
        torch.cuda.synchronize()
        d = st.summary()
        d.update({"rate_req_s": rate, "duration_s": duration_s, "requests": len(rs),
                  "p50_ms": round(d["p50_ms"], 3), "p99_ms": round(d["p99_ms"], 3),
                  "throughput_req_s": round(d["throughput_req_s"], 1), "gpix_s": round(d["gpix_s"], 2)})
        out.append(d)
    return out


def measure_host_link(torch, step_px: int, io_bytes: int, nbytes: int = 256 << 20, reps: int = 5) -> dict:
    """Pinned host <-> device copy rates in this run (CUDA events, median of
    `reps` after 3 warm-ups): host to device alone, device to host alone, and
    both at once on two streams.  They bound the end-to-end figure: a step
    moves `io_bytes` each way, so it takes at least the longest of the three
    copy times, whatever the kernels do."""
    h_in = torch.empty(nbytes, dtype=torch.uint8).pin_memory()
    h_out = torch.empty(nbytes, dtype=torch.uint8).pin_memory()
    d_in = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    d_out = torch.zeros(nbytes, dtype=torch.uint8, device="cuda")
    s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()

    def timed(h2d: bool, d2h: bool) -> float:
        times = []
        for r in range(3 + reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            out_done = torch.cuda.Event()
            torch.cuda.synchronize()
            e0.record(s_in)
            s_out.wait_event(e0)
            if h2d:
                with torch.cuda.stream(s_in):
                    d_in.copy_(h_in, non_blocking=True)
            if d2h:
                with torch.cuda.stream(s_out):
                    h_out.copy_(d_out, non_blocking=True)
            out_done.record(s_out)
            s_in.wait_event(out_done)
            e1.record(s_in)
            torch.cuda.synchronize()
            if r >= 3:
                times.append(e0.elapsed_time(e1) * 1e-3)
        return float(np.median(times))

    t_in, t_out, t_both = timed(True, False), timed(False, True), timed(True, True)
    step_floor = max(io_bytes / (nbytes / t_in), io_bytes / (nbytes / t_out), 2 * io_bytes / (2 * nbytes / t_both))
    return {"bytes": nbytes, "h2d_gbs": round(nbytes / t_in / 1e9, 1), "d2h_gbs": round(nbytes / t_out / 1e9, 1),
            "both_gbs": round(2 * nbytes / t_both / 1e9, 1),
            "ceiling": round(step_px / step_floor / 1e9, 1),
            "note": "pinned copies of 256 MB timed with CUDA events; ceiling = the step's pixels over its "
                    "copy time in and out at these rates (Gpixel/s)"}


def reduce_over_ranks(torch, dist, value: float, op: str) -> float:
    """max or sum of a float over all ranks (identity without a process group)."""
    if dist is None or not dist.is_initialized():
        return value
    t = torch.tensor([value], dtype=torch.float64,
                     device="cuda" if dist.get_backend() == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def run_gpu(args):
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        dist = None
        torch.cuda.set_device(0)

    from paper_2002_09474_gb300 import build as libbuild
    libbuild.build()
    from paper_2002_09474_gb300 import morph

    # the library's autotuner (crossovers, form of the pass along x), as a
    # user would run it once per device; its cache lives outside the repo
    import tempfile
    tune_path = os.path.join(tempfile.gettempdir(), "morph_tune_%d.json" % local)
    rc = morph.morph_autotune(tune_path)
    if rc != 0:
        raise morph.MorphError("morph_autotune", rc)

    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()
    sh = stream.cuda_stream
    host_imgs = {(dt, k): make_image(dt, k) for dt in DTYPES for k in IMAGES}
    tdt = {np.uint8: torch.uint8, np.uint16: torch.uint16}
    srcs = {}
    for key, im in host_imgs.items():
        base = torch.from_numpy(im).to(dev)
        srcs[key] = [base] + [base.clone() for _ in range(ROTATE - 1)]
    dsts = {dt: [torch.empty((SIDE, SIDE), dtype=tdt[dt], device=dev) for _ in range(ROTATE)]
            for dt in DTYPES}
    runs = step_runs()
    ctr = {"src": {k: 0 for k in srcs}, "dst": {dt: 0 for dt in DTYPES}}

    def launch(run, sh):
        dt, kind, (wx, wy), op = run
        key = (dt, kind)
        i = ctr["src"][key]
        ctr["src"][key] = (i + 1) % ROTATE
        j = ctr["dst"][dt]
        ctr["dst"][dt] = (j + 1) % ROTATE
        s, d = srcs[key][i], dsts[dt][j]
        code = morph.MORPH_U8 if dt == np.uint8 else morph.MORPH_U16
        pitch = SIDE * np.dtype(dt).itemsize
        rc = morph.morph_apply(s.data_ptr(), pitch, d.data_ptr(), pitch, SIDE, SIDE, code, op,
                               wx, wy, wx // 2, wy // 2, sh)
        if rc != 0:
            raise morph.MorphError("morph_apply", rc)

    # eager calls first: per-device set-up happens outside any capture
    for r in runs:
        launch(r, sh)
    torch.cuda.synchronize()

    def capture(calls, nstreams=1, stream_of=None):
        """The calls, through the C ABI, captured once into a CUDA graph,
        issued on `nstreams` streams (call n on stream_of(n, call), default
        round-robin) forked from and joined back to the capture stream;
        returns (graph, kernel launches per replay)."""
        n0 = morph.morph_launch_count()
        g = torch.cuda.CUDAGraph()
        side = [torch.cuda.Stream() for _ in range(nstreams)]
        with torch.cuda.graph(g):
            cs = torch.cuda.current_stream()
            fork = torch.cuda.Event()
            fork.record(cs)
            for s in side:
                s.wait_event(fork)
            for n, r in enumerate(calls):
                k = stream_of(n, r) if stream_of else n % nstreams
                launch(r, side[k].cuda_stream)
            for s in side:
                join = torch.cuda.Event()
                join.record(s)
                cs.wait_event(join)
        return g, morph.morph_launch_count() - n0

    # one step (32 calls) as one graph: replays carry no host launch cost.
    # The calls are independent images: the uniform and the gradient image
    # of each class go on two streams, the same sequence of classes on each,
    # so that one call's kernels fill the SMs the other's leave idle in
    # their first and last waves.
    g_step, launches_per_step = capture(runs, STEP_STREAMS,
                                        lambda n, r: IMAGES.index(r[1]) % STEP_STREAMS)
    for _ in range(args.warmup):
        g_step.replay()
    torch.cuda.synchronize()

    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(gpu_id_for_smi(torch))
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    t_start.record(stream)
    for _ in range(args.steps):
        g_step.replay()
    t_end.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    if dist is not None:
        dist.barrier()
    elapsed_ms = t_start.elapsed_time(t_end)
    max_ms = reduce_over_ranks(torch, dist, elapsed_ms, "max")
    step_px = len(runs) * SIDE * SIDE
    total_px = reduce_over_ranks(torch, dist, float(step_px * args.steps), "sum")
    value = total_px / (max_ms * 1e-3) / 1e9
    del g_step

    # per-class time: each (dtype, window) class's calls of two steps as a
    # graph of its own, replayed and timed with events on this stream
    peak, peak_kind = load_peaks()
    breakdown = {}
    dom, dom_total = None, -1.0
    reps = max(3, min(20, args.steps))
    for dt in DTYPES:
        for w in WINDOWS:
            calls = [r for r in runs if r[0] == dt and r[2] == w] * 2
            g, nl = capture(calls)
            for _ in range(2):
                g.replay()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(reps):
                g.replay()
            e1.record(stream)
            torch.cuda.synchronize()
            mean_ms = e0.elapsed_time(e1) / (reps * len(calls))
            del g
            esz = np.dtype(dt).itemsize
            name = "%s_%dx%d" % ("u8" if dt == np.uint8 else "u16", w[0], w[1])
            gbs = 2 * esz * SIDE * SIDE / (mean_ms * 1e-3) / 1e9
            breakdown[name] = {"us_per_call": round(mean_ms * 1e3, 2),
                               "kernels_per_call": nl // len(calls),
                               "gpix_s": round(SIDE * SIDE / (mean_ms * 1e-3) / 1e9, 1),
                               "gb_s": round(gbs, 1), "frac_of_%s_hbm" % peak_kind: round(gbs / peak, 3)}
            class_total = mean_ms * len(calls) / 2
            if class_total > dom_total:
                dom_total, dom = class_total, (name, gbs)

    # end to end through the host-buffer entry point
    pinned_in = {k: torch.from_numpy(v).pin_memory() for k, v in host_imgs.items()}
    pinned_out = {dt: torch.empty((SIDE, SIDE), dtype=tdt[dt]).pin_memory() for dt in DTYPES}
    e2e_steps = max(3, args.steps // 10)

    # the step's 32 calls as one pipelined host-buffer call: copies in,
    # filtering and copies out of consecutive images overlap
    e2e_descs = (morph.MorphDesc * len(runs))()
    for dsc, (dt, kind, (wx, wy), op) in zip(e2e_descs, runs):
        pitch = SIDE * np.dtype(dt).itemsize
        dsc.src, dsc.dst = pinned_in[(dt, kind)].data_ptr(), pinned_out[dt].data_ptr()
        dsc.width = dsc.height = SIDE
        dsc.src_pitch = dsc.dst_pitch = pitch
        dsc.wx, dsc.wy, dsc.anchor_x, dsc.anchor_y, dsc.op = wx, wy, wx // 2, wy // 2, op
        dsc.dtype = morph.MORPH_U8 if dt == np.uint8 else morph.MORPH_U16

    def e2e_step():
        rc = morph.morph_apply_host_batch(e2e_descs, len(runs), sh)
        if rc != 0:
            raise morph.MorphError("morph_apply_host_batch", rc)
    e2e_step()
    if dist is not None:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        e2e_step()
    e2e_s = reduce_over_ranks(torch, dist, time.perf_counter() - t0, "max")
    e2e_px = reduce_over_ranks(torch, dist, float(step_px * e2e_steps), "sum")
    io_bytes = sum(SIDE * SIDE * np.dtype(dt).itemsize for dt, _, _, _ in runs)
    morph.morph_release_staging()
    morph.check_device_error()
    try:
        host_link = measure_host_link(torch, step_px, io_bytes)
    except Exception as exc:  # a copy-rate probe must not cost the bench line
        host_link = {"error": repr(exc)}

    extras = {}
    if not args.no_extras:
        extras["transposes"] = measure_transposes(torch, morph, peak, peak_kind)
        extras["batched"] = measure_batched(torch, morph)
        extras["composite"] = measure_composite(torch, morph, peak=peak)
        extras["small_images"] = measure_small_images(torch, morph)
        extras["serving"] = measure_serving(torch, rates=args.serving_rates,
                                            duration_s=args.serving_seconds)
        extras["serving_host_copies"] = measure_serving(torch, rates=args.serving_rates,
                                                        duration_s=args.serving_seconds, host_copies=True)

    if rank == 0:
        traffic_b2b, traffic_cold = load_traffic(dom[0])
        line = {"metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": round(max_ms / args.steps, 4), "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "u8+u16 (integer min/max)",
                "data": "synthetic (seeded uniform and gradient+noise images)",
                "config": dict(workload_config(), parallelism="replicas" if world > 1 else "single"),
                "roofline": {"bound": "hbm", "kernel": dom[0], "achieved": round(dom[1], 1),
                             "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
                             "frac": round(dom[1] / peak, 4),
                             "traffic": traffic_b2b, "traffic_cache_flushed": traffic_cold,
                             "traffic_note": "DRAM read+write bytes per call of the class (both launches), "
                                             "ncu: back to back as the step runs them (--cache-control "
                                             "none), and with caches flushed before each launch"},
                "e2e": {"value": round(e2e_px / e2e_s / 1e9, 3), "unit": UNIT,
                        "h2d_bytes_per_step": io_bytes, "d2h_bytes_per_step": io_bytes,
                        "api": "morph_apply_host_batch (the step's 32 images, copies overlapped "
                               "with filtering), pinned host buffers",
                        "host_link": host_link},
                "gpu_launches": launches_per_step * args.steps,
                "timing": "the step's 32 calls captured once into a CUDA graph (on %d streams, one per "
                          "image kind) and replayed; per-class times from single-stream graphs" % STEP_STREAMS,
                "clocks": clk,
                "breakdown": breakdown}
        line.update(extras)
        if not args.no_cpu_baseline:
            v, cores, spent, desc = oracle_sample(host_imgs)
            line["cpu_baseline"] = {"value": round(v, 6), "unit": UNIT, "cores": cores,
                                    "kind": "oracle", "sample": desc, "seconds": round(spent, 1),
                                    "separable": separable_sample(host_imgs),
                                    "paper_method": paper_method_sample()}
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true",
                    help="skip the CPU oracle sample (for profiler runs)")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the batched and serving measurements (for profiler runs)")
    ap.add_argument("--serving-rates", type=float, nargs="+",
                    default=[1000.0, 2000.0, 5000.0, 10000.0, 20000.0],
                    help="request rates of the serving measurement (req/s)")
    ap.add_argument("--serving-seconds", type=float, default=10.0,
                    help="length of each serving run after warm-up")
    args = ap.parse_args(argv)
    if args.warmup < 3 and args.impl == "ours":
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
