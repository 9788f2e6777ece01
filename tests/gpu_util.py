"""Helpers for the GPU tests: pitched device images with guard bytes."""
from __future__ import annotations

import numpy as np
import pytest

CANARY = 0xA5


def need_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


class DeviceImage:
    """A height x width image inside a larger byte buffer: `pad` extra bytes
    per row, `offset` bytes before the first row, guard bytes around all of
    it filled with CANARY (to catch writes outside the image)."""

    def __init__(self, torch, h: int, w: int, dtype, pad: int = 0, offset: int = 0,
                 guard: int = 256, fill: np.ndarray | None = None):
        self.h, self.w = h, w
        self.dtype = np.dtype(dtype)
        self.esz = self.dtype.itemsize
        self.pitch = w * self.esz + pad
        self.offset = guard + offset
        total = self.offset + self.pitch * h + guard
        host = np.full(total, CANARY, np.uint8)
        if fill is not None:
            assert fill.shape == (h, w) and fill.dtype == self.dtype
            raw = fill.view(np.uint8).reshape(h, w * self.esz)
            for y in range(h):
                s = self.offset + y * self.pitch
                host[s:s + w * self.esz] = raw[y]
        self.host_init = host
        self.buf = torch.from_numpy(host).cuda()
        self.ptr = self.buf.data_ptr() + self.offset

    def read(self) -> np.ndarray:
        host = self.buf.cpu().numpy()
        out = np.empty((self.h, self.w * self.esz), np.uint8)
        for y in range(self.h):
            s = self.offset + y * self.pitch
            out[y] = host[s:s + self.w * self.esz]
        return out.view(self.dtype).reshape(self.h, self.w)

    def untouched_outside(self) -> bool:
        """True if no byte outside the image's pixels changed."""
        host = self.buf.cpu().numpy()
        mask = np.ones(host.size, bool)
        for y in range(self.h):
            s = self.offset + y * self.pitch
            mask[s:s + self.w * self.esz] = False
        return bool((host[mask] == self.host_init[mask]).all())
