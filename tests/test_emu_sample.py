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
