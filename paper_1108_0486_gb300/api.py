"""Torch-facing wrapper of the C ABI.

PyTorch supplies device memory (output tensors) and the CUDA stream; every
random number is produced by the library's kernels through the C entry
points in ``_lib``.
"""
from __future__ import annotations

import numpy as np
import torch

from . import _lib as L

TYPES = {"u32": L.XG_U32, "uniform": L.XG_UNIFORM_F32, "normal": L.XG_NORMAL_F32}
LAUNCHES = [(4, 8), (8, 4), (16, 2), (16, 4), (32, 2)]


def _stream_handle(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


class Streams:
    """A context of n independent xorgens streams resident on the GPU.

    param_set 0 is (r,s,a,b,c,d) = (128,95,17,12,13,15), param_set 1 the
    paper's (128,65,15,14,12,17).  ``weyl=False`` outputs the GF(2)-linear part
    alone (for testing).
    """

    def __init__(self, n: int, param_set: int = 0, weyl: bool = True, stream=None,
                 seeds=None):
        self.n = int(n)
        self.param_set = param_set
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.ctx = L.xg_create_streams(self.n, param_set, weyl, _stream_handle(self.stream))
        if seeds is not None:
            self.seed(seeds)

    def close(self):
        if getattr(self, "ctx", None):
            L.xg_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # ---- state ---------------------------------------------------------
    def seed(self, seeds, first: int = 0):
        s = np.ascontiguousarray(np.asarray(seeds, dtype=np.uint32).ravel())
        L.xg_seed(self.ctx, first, s.size, s.ctypes.data)
        return self

    def get_state(self, stream: int):
        ring = np.zeros(128, dtype=np.uint32)
        w = L.xg_get_state(self.ctx, stream, ring.ctypes.data)
        return ring, w

    def set_state(self, stream: int, ring, weyl: int):
        r = np.ascontiguousarray(np.asarray(ring, dtype=np.uint32))
        assert r.size == 128
        L.xg_set_state(self.ctx, stream, r.ctypes.data, weyl)

    def set_launch(self, kind: str, tpg: int = 0, wpl: int = 0):
        L.xg_set_launch(self.ctx, TYPES[kind], tpg, wpl)

    def get_launch(self, kind: str):
        return L.xg_get_launch(self.ctx, TYPES[kind])

    # ---- generation -----------------------------------------------------
    def _gen(self, fn, dtype, n, first, count, out, ld):
        count = self.n - first if count is None else count
        if out is None:
            ld = n if ld is None else ld
            out = torch.empty((count, ld), dtype=dtype, device="cuda")
        else:
            ld = out.stride(0) if (ld is None and out.dim() == 2) else (ld if ld is not None else n)
        fn(self.ctx, first, count, n, out.data_ptr(), ld)
        return out

    def u32(self, n: int, first: int = 0, count=None, out=None, ld=None):
        """n words per stream as int32 bit patterns, shape (count, ld)."""
        return self._gen(L.xg_generate_u32, torch.int32, n, first, count, out, ld)

    def uniform(self, n: int, first: int = 0, count=None, out=None, ld=None):
        return self._gen(L.xg_generate_uniform, torch.float32, n, first, count, out, ld)

    def normal(self, n: int, first: int = 0, count=None, out=None, ld=None):
        return self._gen(L.xg_generate_normal, torch.float32, n, first, count, out, ld)

    def generate(self, kind: str, n: int, **kw):
        return {"u32": self.u32, "uniform": self.uniform, "normal": self.normal}[kind](n, **kw)

    def normal_sum(self, n: int, first: int = 0, count=None, out=None):
        count = self.n - first if count is None else count
        if out is None:
            out = torch.empty(count, dtype=torch.float32, device="cuda")
        L.xg_generate_normal_sum(self.ctx, first, count, n, out.data_ptr())
        return out

    # ---- conversions of given words ------------------------------------
    def transform_uniform(self, words: torch.Tensor, out=None):
        out = torch.empty(words.numel(), dtype=torch.float32, device="cuda") if out is None else out
        L.xg_transform_uniform(self.ctx, words.data_ptr(), words.numel(), out.data_ptr())
        return out

    def transform_normal(self, words: torch.Tensor, out=None):
        out = torch.empty(words.numel(), dtype=torch.float32, device="cuda") if out is None else out
        L.xg_transform_normal(self.ctx, words.data_ptr(), words.numel(), out.data_ptr())
        return out


def as_u32(t: torch.Tensor) -> np.ndarray:
    """Copy an int32 bit-pattern tensor to host as numpy uint32."""
    return t.detach().cpu().numpy().view(np.uint32)
