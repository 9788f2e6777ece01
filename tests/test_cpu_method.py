"""The paper's CPU method (cpu_method/, a CPU baseline for the bench) against
the oracle: both methods of both passes, scalar form everywhere, the NEON
form on aarch64 hosts; and its block transposes against numpy's."""
import numpy as np
import pytest

import cpu_method as cm
import oracle
from paper_2002_09474_gb300 import synth

FORMS = [False] + ([True] if cm.has_neon() else [])


@pytest.mark.parametrize("vector", FORMS)
@pytest.mark.parametrize("method", ["direct", "vhgw"])
def test_paper_cpu_method_matches_oracle(vector, method):
    g = synth.rng(1200)
    for (h, w) in ((1, 1), (5, 3), (17, 16), (37, 50), (120, 161)):
        img = synth.uniform_image(w, h, np.uint8, gen=g)
        for (wx, wy, ax, ay) in ((1, 1, 0, 0), (3, 3, 1, 1), (4, 7, 0, 6), (15, 31, 14, 0), (61, 9, 30, 4),
                                 (2, 40, 1, 20)):
            for op in ("erode", "dilate"):
                want = oracle.morph(img, wx, wy, ax, ay, op)
                got = cm.morph(img, wx, wy, ax, ay, op, method, vector)
                np.testing.assert_array_equal(got, want, err_msg=str((h, w, wx, wy, ax, ay, op, method, vector)))


@pytest.mark.parametrize("vector", FORMS)
def test_paper_cpu_transposes(vector):
    g = synth.rng(1201)
    b8 = g.integers(0, 256, (33, 16, 16), dtype=np.uint8)
    np.testing.assert_array_equal(cm.transpose_blocks("u8", b8, vector), b8.transpose(0, 2, 1))
    b16 = g.integers(0, 65536, (33, 8, 8), dtype=np.uint16)
    np.testing.assert_array_equal(cm.transpose_blocks("u16", b16, vector), b16.transpose(0, 2, 1))


def test_paper_cpu_rejects_bad_arguments():
    img = np.zeros((4, 4), np.uint8)
    with pytest.raises(RuntimeError):
        cm.morph(img, 3, 3, 3, 1)  # anchor outside the window
    if not cm.has_neon():
        with pytest.raises(RuntimeError):
            cm.morph(img, 3, 3, vector=True)
