"""The kernels' own tile code, emulated on the CPU, against the oracle.

`tests/emu/morph_emu.cpp` compiles the device code of every kernel for the
host (threads of a CTA meeting at real barriers; TMA copies, mbarriers and
cp.async modelled; every access checked by AddressSanitizer and the
alignment sanitizer) and compares each launch's output with the oracle,
bit for bit.  The full case list takes minutes of several cores; this test
runs an evenly spread sample of every kernel's cases (shapes, windows,
anchors, methods, tile shapes, pitches and offsets), built without
optimisation so that the build stays short.
"""
from __future__ import annotations

import hashlib
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
EMU = os.path.join(ROOT, "tests", "emu")
CSRC = os.path.join(ROOT, "paper_2002_09474_gb300", "csrc")
ORACLE_C = os.path.join(ROOT, "oracle", "morph_oracle.c")
BUILD = os.path.join(EMU, "_build")
CUDA_INC = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")

PER_KERNEL = 20  # cases per kernel family (7 families)
WORKERS = max(2, min(8, os.cpu_count() or 2))


def _sources():
    files = [os.path.join(EMU, "morph_emu.cpp"), ORACLE_C, os.path.join(CSRC, "plan.cpp")]
    files += [os.path.join(CSRC, f) for f in sorted(os.listdir(CSRC)) if f.endswith((".cuh", ".h"))]
    return files


def _build() -> str:
    h = hashlib.sha256()
    for f in _sources():
        with open(f, "rb") as fh:
            h.update(os.path.basename(f).encode() + b"\0" + fh.read())
    exe = os.path.join(BUILD, "morph_emu_sample_" + h.hexdigest()[:12])
    if os.path.exists(exe):
        return exe
    os.makedirs(BUILD, exist_ok=True)
    for f in os.listdir(BUILD):  # binaries of earlier sources
        if f.startswith("morph_emu_sample_"):
            os.remove(os.path.join(BUILD, f))
    obj = exe + "_oracle.o"
    subprocess.run(["gcc", "-O0", "-fsanitize=address", "-c", ORACLE_C, "-o", obj], check=True)
    tmp = exe + ".tmp"
    subprocess.run(
        ["g++", "-std=c++20", "-O0", "-fsanitize=address,alignment", "-fno-sanitize-recover=alignment",
         "-I", CSRC, "-I", CUDA_INC, os.path.join(EMU, "morph_emu.cpp"), os.path.join(CSRC, "plan.cpp"), obj,
         "-o", tmp, "-lpthread"],
        check=True,
    )
    os.replace(tmp, exe)
    return exe


def _sample() -> list[str]:
    out = subprocess.run([sys.executable, os.path.join(EMU, "cases.py"), "--quick"], check=True,
                         capture_output=True, text=True).stdout.splitlines()
    by_kern: dict[str, list[str]] = {}
    for line in out:
        by_kern.setdefault(line.split()[-1], []).append(line)
    assert sorted(by_kern) == [str(k) for k in range(7)], sorted(by_kern)
    picked = []
    for k in sorted(by_kern):
        lines = by_kern[k]
        n = min(PER_KERNEL, len(lines))
        picked += [lines[(i * len(lines)) // n] for i in range(n)]
    return picked


@pytest.mark.skipif(shutil.which("g++") is None or shutil.which("gcc") is None, reason="needs gcc and g++")
@pytest.mark.skipif(not os.path.exists(os.path.join(CUDA_INC, "cuda.h")), reason="needs the CUDA headers")
def test_emulated_kernels_equal_the_oracle():
    exe = _build()
    env = dict(os.environ, ASAN_OPTIONS="detect_leaks=0")

    def run(case):
        r = subprocess.run([exe], input=case + "\n", capture_output=True, text=True, env=env, timeout=600)
        return case, r.returncode, r.stdout + r.stderr

    with ThreadPoolExecutor(WORKERS) as ex:
        results = list(ex.map(run, _sample()))
    bad = [f"{case}\n{out.strip()[-2000:]}" for case, rc, out in results
           if rc != 0 or "1 cases, 0 failures" not in out]
    assert not bad, "\n".join(bad[:5])


# The planner's documented decisions, answered by the same binary (plan.cpp
# and the launch-shape rules of morph_colv.cuh and morph_rowv.cuh compiled
# for the host, default tuning: crossovers 9 on both axes).
PLANNER = [
    # two launches for a 2-D window when both passes take van Herk/Gil-Werman
    # on at least 2 Mpixels ...
    ("P split 2 4096 4096 127 127", "split 1"),
    ("P split 1 4096 4096 15 15", "split 1"),
    ("P split 1 2048 1024 15 15", "split 1"),
    ("P split 1 2047 1024 15 15", "split 0"),
    ("P split 1 1024 1024 15 15", "split 0"),
    # ... when one of them does, from 4 Mpixels ...
    ("P split 1 2048 2048 5 40", "split 1"),
    ("P split 1 2048 2048 40 5", "split 1"),
    ("P split 1 2048 2047 5 40", "split 0"),
    ("P split 1 1448 1448 5 40", "split 0"),
    ("P split 2 1448 1448 40 5", "split 0"),
    # ... and never for direct-method windows (9 is the crossover) or 1-D ones
    ("P split 1 4096 4096 9 9", "split 0"),
    ("P split 2 4096 4096 3 3", "split 0"),
    ("P split 1 4096 4096 1 101", "split 0"),
    ("P split 1 4096 4096 101 1", "split 0"),
    # the method per pass: van Herk/Gil-Werman above the crossover, windows of
    # at least 8 (its block)
    ("P single 1 512 512 9 10", "single 1 1 0 {cfg} {ctas}"),
    ("P single 1 512 512 10 9", "single 1 0 1 {cfg} {ctas}"),
    # built-in tile heights of the pass along y: below 32 rows the largest
    # multiple of w filling one 32-row box (w <= 16) or two; from 32 rows 2w
    # (u8, at most 256), for u16 w from 120 rows, 2w from 64, else 64
    ("P colvrows 1 9", "colvrows 18"),
    ("P colvrows 1 16", "colvrows 16"),
    ("P colvrows 1 17", "colvrows 34"),
    ("P colvrows 1 31", "colvrows 31"),
    ("P colvrows 1 101", "colvrows 202"),
    ("P colvrows 1 127", "colvrows 254"),
    ("P colvrows 1 200", "colvrows 256"),
    ("P colvrows 2 51", "colvrows 64"),
    ("P colvrows 2 101", "colvrows 202"),
    ("P colvrows 2 127", "colvrows 127"),
    # a 4096^2 u16 1 x 101 call: 64 strips x 21 bands of 202 rows, ten 32-row
    # boxes per warp tile, one warp per CTA, 5 warps per SM
    ("P colv 2 4096 4096 101 4", "colv 1 202 10 1 1344 5"),
    # the pass along x: the shortest segment whose tasks fit one wave of
    # 152 SMs x 32 warps (4096^2, 2 rows a warp: 2048 bands, 2 segments)
    ("P rowv 4096 4096 2 32", "rowv 1 2048 2 4096"),
    ("P rowv 8192 8192 2 32", "rowv 1 8192 1 4096"),
    # CTAs of the fused kernel per SM in the cost model: shared memory, at
    # most 4 (registers)
    ("P ctas 36864", "ctas 4"),
    ("P ctas 70000", "ctas 3"),
    ("P ctas 120000", "ctas 1"),
]


@pytest.mark.skipif(shutil.which("g++") is None or shutil.which("gcc") is None, reason="needs gcc and g++")
@pytest.mark.skipif(not os.path.exists(os.path.join(CUDA_INC, "cuda.h")), reason="needs the CUDA headers")
def test_planner_decisions():
    exe = _build()
    env = dict(os.environ, ASAN_OPTIONS="detect_leaks=0")
    r = subprocess.run([exe], input="\n".join(q for q, _ in PLANNER) + "\n", capture_output=True, text=True,
                       env=env, timeout=120)
    assert r.returncode == 0, r.stderr[-2000:]
    got = [line for line in r.stdout.splitlines() if line.strip()]
    assert len(got) == len(PLANNER), got
    for (q, want), line in zip(PLANNER, got):
        if "{cfg}" in want:  # the tile shape and its CTAs are the cost model's: only the methods are pinned
            assert line.split()[:4] == want.split()[:4], (q, line)
        else:
            assert line == want, (q, line)
