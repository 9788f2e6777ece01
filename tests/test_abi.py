"""The C-ABI library loads, exports every entry point include/morph.h and
include/morph_tuning.h declare, and rejects bad arguments before touching a GPU (CPU only: every
call below fails validation, so no CUDA work is issued)."""
import ctypes

import pytest

from paper_2002_09474_gb300 import morph as m

FAKE = 0x100000        # a pointer value that is never dereferenced
FAKE2 = 0x7000000


def test_every_declared_symbol_is_exported():
    decl = m.declared_functions()
    assert len(decl) >= 30 and "morph_set_colv" in decl and "morph_copy_batch" in decl
    missing = [f for f in decl if not m.exported(f)]
    assert not missing, missing


def test_status_strings():
    for code in range(0, -12, -1):
        s = m.status_string(code)
        assert s and s != "unknown status", code
    assert m.status_string(-99) == "unknown status"


@pytest.mark.parametrize("dtype,esz", [(m.MORPH_U8, 1), (m.MORPH_U16, 2)])
def test_single_image_validation(dtype, esz):
    W, H = 64, 32
    p = W * esz
    ok = dict(src=FAKE, sp=p, dst=FAKE2, dp=p, w=W, h=H, dt=dtype, op=0, wx=3, wy=3, ax=1, ay=1)

    def call(**kw):
        a = dict(ok, **kw)
        return m.morph_apply(a["src"], a["sp"], a["dst"], a["dp"], a["w"], a["h"], a["dt"], a["op"],
                             a["wx"], a["wy"], a["ax"], a["ay"], 0)
    assert call(src=0) == -1
    assert call(dst=0) == -1
    assert call(w=0) == -2 and call(h=-1) == -2
    assert call(wx=0) == -3 and call(wy=-2) == -3
    assert call(ax=3) == -4 and call(ay=-1) == -4
    assert call(sp=p - 1) == -5 and call(dp=1) == -5
    assert call(dst=FAKE + 10) == -6            # overlapping source and destination
    assert call(dt=7) == -9 and call(op=2) == -9
    if esz == 2:
        assert call(sp=p + 1) == -5             # 16-bit rows must stay 2-byte aligned
        assert call(src=FAKE + 1) == -5


def test_typed_wrappers_validate():
    assert m.morph_erode(0, 10, 10, 10, 3, 3, 1, 1, FAKE2, 0) == -1
    assert m.morph_dilate(FAKE, 10, 10, 5, 3, 3, 1, 1, FAKE2, 0) == -5
    assert m.morph_erode_u16(FAKE, 10, 10, 20, 3, 3, 5, 1, FAKE2, 0) == -4
    assert m.morph_dilate_u16(FAKE, 10, 10, 20, 0, 3, 0, 1, FAKE2, 0) == -3


def test_transpose_validation():
    assert m.transpose_u8(0, 8, 8, 8, FAKE2, 8, 0) == -1
    assert m.transpose_u8(FAKE, 8, 4, 7, FAKE2, 8, 0) == -5      # src pitch < width
    assert m.transpose_u8(FAKE, 8, 4, 8, FAKE2, 3, 0) == -5      # dst pitch < height
    assert m.transpose_u8(FAKE, 8, 4, 8, FAKE + 8, 8, 0) == -6   # overlap
    assert m.transpose_u16(FAKE, 8, 4, 17, FAKE2, 8, 0) == -5     # odd pitch for 16-bit
    assert m.transpose_u8(FAKE, 0, 4, 8, FAKE2, 8, 0) == -2


def _desc(src, dst, w=16, h=8, pitch=16, wx=3, wy=3, op=0, dtype=0):
    d = m.MorphDesc()
    d.src, d.dst, d.width, d.height = src, dst, w, h
    d.src_pitch = d.dst_pitch = pitch
    d.wx, d.wy, d.anchor_x, d.anchor_y = wx, wy, wx // 2, wy // 2
    d.op, d.dtype = op, dtype
    return d


def test_descriptor_layout_matches_header(tmp_path):
    """The ctypes mirror of morph_desc has the C compiler's size and offsets."""
    import os
    import subprocess
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    c = tmp_path / "layout.c"
    c.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "morph.h"\n'
                 'int main(void){printf("%zu %zu %zu %zu %zu %zu\\n", sizeof(morph_desc),'
                 ' offsetof(morph_desc, width), offsetof(morph_desc, src_pitch),'
                 ' offsetof(morph_desc, wx), offsetof(morph_desc, op), offsetof(morph_desc, dtype));'
                 'return 0;}\n')
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", inc, str(c), "-o", str(exe)])
    got = [int(v) for v in subprocess.check_output([str(exe)]).split()]
    want = [ctypes.sizeof(m.MorphDesc), m.MorphDesc.width.offset, m.MorphDesc.src_pitch.offset,
            m.MorphDesc.wx.offset, m.MorphDesc.op.offset, m.MorphDesc.dtype.offset]
    assert got == want


def test_batch_validation():
    arr = (m.MorphDesc * 3)(_desc(FAKE, FAKE2), _desc(FAKE + 4096, FAKE2 + 4096),
                            _desc(FAKE + 8192, FAKE2 + 8192))
    assert m.morph_batch(arr, 0, 0) == -10
    assert m.morph_batch(None, 3, 0) == -1
    bad = (m.MorphDesc * 2)(_desc(FAKE, FAKE2), _desc(FAKE + 4096, FAKE2 + 64))  # two dsts overlap
    assert m.morph_batch(bad, 2, 0) == -6
    bad2 = (m.MorphDesc * 2)(_desc(FAKE, FAKE2), _desc(FAKE2, FAKE + 8192))      # dst of 0 = src of 1
    assert m.morph_batch(bad2, 2, 0) == -6
    bad3 = (m.MorphDesc * 2)(_desc(FAKE, FAKE2), _desc(FAKE + 4096, FAKE2 + 4096, wx=0))
    assert m.morph_batch(bad3, 2, 0) == -3
    plan = ctypes.c_void_p()
    assert m.morph_batch_plan_create(bad, 2, ctypes.byref(plan)) == -6 and not plan.value
    assert m.morph_batch_plan_launch(None, 0) == -1
    assert m.morph_batch_plan_destroy(None) == -1


def test_tuning_arguments():
    assert m.morph_set_tuning(5, 1, 1, -1) == -9
    assert m.morph_set_tuning(0, 1, 1, 99) == -10
    assert m.morph_set_tuning(0, -1, -1, -1) == 0
    assert m.morph_set_pipeline(2) == -10 and m.morph_set_pipeline(-2) == -10
    assert m.morph_set_pipeline(0) == 0 and m.morph_set_pipeline(-1) == 0
    assert m.morph_set_xpass(5, 0) == -9 and m.morph_set_xpass(0, 2) == -10 and m.morph_set_xpass(1, -1) == -10
    assert m.morph_set_xpass(0, 1) == 0 and m.morph_set_xpass(0, 0) == 0
    assert m.morph_set_batch_alone(0) == 0 and m.morph_set_batch_alone(-1) == 0
    assert m.morph_set_composite_kernel(2) == -10 and m.morph_set_composite_kernel(-2) == -10
    assert m.morph_set_composite_kernel(0) == 0 and m.morph_set_composite_kernel(-1) == 0
    assert m.morph_set_column_kernel(3) == -10 and m.morph_set_column_kernel(-1) == 0
    assert m.morph_set_row_kernel(-3) == -10 and m.morph_set_row_kernel(-1) == 0
    assert m.morph_set_colv(2, 0, 0) == -10 and m.morph_set_colv(-2, 0, 0) == -10
    assert m.morph_set_colv(-1, -1, 0) == -10 and m.morph_set_colv(-1, 0, 2) == -10
    assert m.morph_set_colv(-1, 2000, 0) == -10 and m.morph_set_colv(-1, 0, 0) == 0
    assert m.morph_set_rowv(5, 0) == -10 and m.morph_set_rowv(-1, -2) == -10
    assert m.morph_set_rowv(-1, 0) == 0
    assert m.morph_set_split_order(2) == -10 and m.morph_set_split_order(1) == 0
    assert m.morph_set_pdl(2) == -10 and m.morph_set_pdl(1) == 0 and m.morph_set_pdl(0) == 0
    assert m.morph_reset_tuning() == 0


def test_composite_and_copy_arguments():
    """Argument checks of morph_composite and morph_copy_2d come before any
    CUDA call (no GPU needed)."""
    u8 = m.MORPH_U8
    assert m.morph_composite(FAKE, 640, FAKE2, 640, 640, 480, u8, 3, 3, 3, 1, 1, 0) == -10   # unknown kind
    assert m.morph_composite(FAKE, 640, FAKE2, 640, 640, 480, u8, -1, 3, 3, 1, 1, 0) == -10
    assert m.morph_composite(None, 640, FAKE2, 640, 640, 480, u8, 0, 3, 3, 1, 1, 0) == -1    # null
    assert m.morph_composite(FAKE, 640, FAKE2, 640, 640, 480, u8, 1, 0, 3, 0, 1, 0) == -3    # window
    assert m.morph_composite(FAKE, 640, FAKE2, 640, 640, 480, u8, 2, 3, 3, 3, 1, 0) == -4    # anchor
    assert m.morph_composite(FAKE, 600, FAKE2, 640, 640, 480, u8, 0, 3, 3, 1, 1, 0) == -5    # pitch
    assert m.morph_composite(FAKE, 640, FAKE + 640, 640, 640, 480, u8, 0, 3, 3, 1, 1, 0) == -6  # overlap
    assert m.morph_composite(FAKE, 640, FAKE2, 640, 640, 0, u8, 0, 3, 3, 1, 1, 0) == -2      # size
    assert m.morph_composite(FAKE, 640, FAKE2, 640, 640, 480, 7, 0, 3, 3, 1, 1, 0) == -9     # dtype
    assert m.morph_copy_2d(None, 64, FAKE, 64, 64, 2, 0) == -1
    assert m.morph_copy_2d(FAKE2, 64, None, 64, 64, 2, 0) == -1
    assert m.morph_copy_2d(FAKE2, 64, FAKE, 64, 64, 0, 0) == -2
    assert m.morph_copy_2d(FAKE2, 32, FAKE, 64, 64, 2, 0) == -5
    assert m.morph_copy_2d(FAKE2, 64, FAKE, 32, 64, 2, 0) == -5
    # the batched copy: every entry checked before anything is queued
    cps = (m.MorphCopyDesc * 2)()
    cps[0].dst, cps[0].src, cps[0].bytes = FAKE2, FAKE, 64
    cps[1].dst, cps[1].src, cps[1].bytes = None, FAKE, 64
    assert m.morph_copy_batch(cps, 2, 0) == -1
    assert m.morph_copy_batch(cps, -1, 0) == -10
    assert m.morph_copy_batch(None, 1, 0) == -1
    assert m.morph_copy_batch(None, 0, 0) == 0
