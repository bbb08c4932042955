"""Torch-facing wrapper of the C ABI.

PyTorch supplies device memory (output tensors) and the CUDA stream; every
random number is produced by the library's kernels through the C entry
points in ``_lib``.
"""
from __future__ import annotations

import numpy as np
import torch
import torch.utils.dlpack

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

    def checkpoint(self, first: int = 0, count=None) -> dict:
        """Every stream's state in [first, first + count) as host arrays:
        rings (count, 128) uint32, weyl (count,) uint32, pos (count,) uint64."""
        count = self.n - first if count is None else count
        rings = np.zeros((count, 128), dtype=np.uint32)
        weyl = np.zeros(count, dtype=np.uint32)
        pos = np.zeros(count, dtype=np.uint64)
        L.xg_get_states(self.ctx, first, count, rings.ctypes.data, weyl.ctypes.data, pos.ctypes.data)
        return {"first": first, "rings": rings, "weyl": weyl, "pos": pos}

    def restore(self, ckpt: dict, first=None, positions: bool = True):
        """Load a checkpoint (from this or another context of the same
        parameter set) into streams [first, first + count)."""
        first = ckpt["first"] if first is None else first
        rings = np.ascontiguousarray(ckpt["rings"], dtype=np.uint32)
        weyl = np.ascontiguousarray(ckpt["weyl"], dtype=np.uint32)
        pos = np.ascontiguousarray(ckpt["pos"], dtype=np.uint64)
        L.xg_set_states(self.ctx, first, weyl.size, rings.ctypes.data, weyl.ctypes.data,
                        pos.ctypes.data if positions else 0)

    def set_launch(self, kind: str, tpg: int = 0, wpl: int = 0):
        L.xg_set_launch(self.ctx, TYPES[kind], tpg, wpl)

    def get_launch(self, kind: str):
        return L.xg_get_launch(self.ctx, TYPES[kind])

    def autotune(self, kind: str, n_per_stream: int, nstreams: int = 0) -> dict:
        """Pick the fastest launch for this type on this workload shape."""
        return L.xg_autotune(self.ctx, TYPES[kind], nstreams, n_per_stream)

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


    # ---- batches and serving -------------------------------------------
    def batch(self, items):
        """One persistent-kernel launch for items (stream, kind, count, out)
        with out a device tensor (or None for count 0)."""
        L.xg_generate_batch(self.ctx, [(int(s), TYPES[k] if isinstance(k, str) else int(k), int(c),
                                        0 if o is None else o.data_ptr()) for s, k, c, o in items])

    def set_batch_shape(self, kind, tpg: int, wpl: int):
        """Batch-kernel shape for single calls of one type: (32,2), (16,4) or (8,4)."""
        L.xg_set_batch_shape(self.ctx, TYPES[kind] if isinstance(kind, str) else int(kind), tpg, wpl)

    def get_batch_shape(self, kind):
        return L.xg_get_batch_shape(self.ctx, TYPES[kind] if isinstance(kind, str) else int(kind))

    def autotune_batch(self, items) -> dict:
        """Pick the batch-kernel shape per type on this batch (streams do not
        advance; the outputs are written).  Returns {kind: (tpg, wpl, ms)}."""
        res = L.xg_autotune_batch(self.ctx, [(int(s), TYPES[k] if isinstance(k, str) else int(k), int(c),
                                              0 if o is None else o.data_ptr()) for s, k, c, o in items])
        return {name: res[TYPES[name]] for name in TYPES}

    def set_batch_split(self, piece_words: int):
        """0: automatic, 1: never cut long calls in batches, else the piece length."""
        L.xg_set_batch_split(self.ctx, piece_words)

    def jump(self, words: int, first: int = 0, count=None):
        """Advance streams by `words` positions without generating them."""
        count = self.n - first if count is None else count
        L.xg_jump(self.ctx, first, count, words)

    def seed_substreams(self, seed: int, log2_spacing: int, first: int = 0, count=None):
        """Streams first + i start at position i * 2^log2_spacing of the one
        sequence seeded by `seed` (disjoint blocks of one period)."""
        count = self.n - first if count is None else count
        L.xg_seed_substreams(self.ctx, first, count, seed, log2_spacing)

    def serve(self, mem_cap_bytes: int = 0, max_batch: int = 0, lanes: int = 0) -> "Server":
        return Server(self, mem_cap_bytes, max_batch, lanes)


class Server:
    """The request server of a Streams context (continuous batching)."""

    def __init__(self, streams: Streams, mem_cap_bytes=0, max_batch=0, lanes=0):
        self.streams = streams
        self.ctx = streams.ctx
        L.xg_server_start(self.ctx, mem_cap_bytes, max_batch, lanes)
        self.running = True

    def submit(self, stream: int, kind, count: int, out: torch.Tensor | None = None) -> int:
        t = TYPES[kind] if isinstance(kind, str) else int(kind)
        return L.xg_submit(self.ctx, stream, t, count, 0 if out is None else out.data_ptr())

    def submit_many(self, requests, tickets=None):
        """Submit (stream, kind, count[, out]) tuples in one call; returns the
        tickets of the admitted ones (all of them unless the cap refused one)."""
        rows = []
        for r in requests:
            k = TYPES[r[1]] if isinstance(r[1], str) else int(r[1])
            out = r[3] if len(r) > 3 else None
            rows.append((int(r[0]), k, int(r[2]), 0 if out is None else out.data_ptr()))
        rec = L.make_requests(rows)
        t = np.zeros(len(rows), dtype=np.uint64)
        n = L.xg_submit_many(self.ctx, rec, 0, len(rows), t)
        return [int(v) for v in t[:n]]

    def poll(self, ticket: int):
        return L.xg_poll(self.ctx, ticket)

    def wait(self, ticket: int, timeout_ms: int = 10000) -> int:
        return L.xg_wait(self.ctx, ticket, timeout_ms)

    def release(self, ticket: int):
        L.xg_release(self.ctx, ticket)

    def cancel(self, ticket: int):
        """Cancel a request not yet launched (XGError XG_EINVAL if it is)."""
        L.xg_cancel(self.ctx, ticket)

    def times(self, ticket: int):
        return L.xg_ticket_times(self.ctx, ticket)

    def stats(self) -> dict:
        return L.xg_server_stats_get(self.ctx)

    def collect(self, max_n: int = 4096, release: bool = False):
        """Finished tickets: (ticket, t_submit, t_launch, t_done, status, d_result)."""
        return L.xg_collect(self.ctx, max_n, release)

    def result(self, ticket: int, kind, count: int, timeout_ms: int = 10000) -> torch.Tensor:
        """Wait for a ticket and view its output as a tensor (no copy)."""
        ptr = self.wait(ticket, timeout_ms)
        dt = torch.int32 if (kind == "u32" or kind == L.XG_U32) else torch.float32
        return device_view(ptr, count, dt)

    def stop(self):
        if self.running:
            L.xg_server_stop(self.ctx)
            self.running = False

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.stop()


# ---- DLPack view of library-owned device memory ------------------------------
import ctypes as _ct


class _DLDevice(_ct.Structure):
    _fields_ = [("device_type", _ct.c_int), ("device_id", _ct.c_int)]


class _DLDataType(_ct.Structure):
    _fields_ = [("code", _ct.c_uint8), ("bits", _ct.c_uint8), ("lanes", _ct.c_uint16)]


class _DLTensor(_ct.Structure):
    _fields_ = [("data", _ct.c_void_p), ("device", _DLDevice), ("ndim", _ct.c_int),
                ("dtype", _DLDataType), ("shape", _ct.POINTER(_ct.c_int64)),
                ("strides", _ct.POINTER(_ct.c_int64)), ("byte_offset", _ct.c_uint64)]


_DELETER = _ct.CFUNCTYPE(None, _ct.c_void_p)


class _DLManagedTensor(_ct.Structure):
    _fields_ = [("dl_tensor", _DLTensor), ("manager_ctx", _ct.c_void_p), ("deleter", _DELETER)]


_keep = {}


@_DELETER
def _dl_deleter(p):
    _keep.pop(p, None)


def device_view(ptr: int, count: int, dtype=torch.float32) -> torch.Tensor:
    """A 1-D tensor over `count` 4-byte elements at device pointer ptr.  The
    memory stays owned by the library (valid until the ticket is released)."""
    code = 0 if dtype == torch.int32 else 2  # kDLInt / kDLFloat
    shape = (_ct.c_int64 * 1)(count)
    mt = _DLManagedTensor()
    mt.dl_tensor = _DLTensor(ptr, _DLDevice(2, torch.cuda.current_device()), 1,
                             _DLDataType(code, 32, 1), shape, None, 0)
    mt.manager_ctx = None
    mt.deleter = _dl_deleter
    addr = _ct.addressof(mt)
    _keep[addr] = (mt, shape)
    PyCapsule_New = _ct.pythonapi.PyCapsule_New
    PyCapsule_New.restype = _ct.py_object
    PyCapsule_New.argtypes = [_ct.c_void_p, _ct.c_char_p, _ct.c_void_p]
    cap = PyCapsule_New(addr, b"dltensor", None)
    return torch.utils.dlpack.from_dlpack(cap)


def as_u32(t: torch.Tensor) -> np.ndarray:
    """Copy an int32 bit-pattern tensor to host as numpy uint32."""
    return t.detach().cpu().numpy().view(np.uint32)


TYPES_W64 = {"u64": L.XG_W64_U64, "uniform": L.XG_W64_UNIFORM_F64}
LAUNCHES_W64 = [(4, 8), (8, 4), (16, 2), (32, 1)]


class Streams64:
    """A context of n independent 64-bit-word xorgens streams on the GPU
    ((r,s,a,b,c,d) = (64,55,42,27,25,22)), with raw 64-bit outputs and FP64
    uniforms.  Outputs: u64 as int64 bit patterns, uniforms as float64."""

    def __init__(self, n: int, weyl: bool = True, stream=None, seeds=None):
        self.n = int(n)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.ctx = L.xg_w64_create(self.n, weyl, _stream_handle(self.stream))
        if seeds is not None:
            self.seed(seeds)

    @staticmethod
    def params():
        return L.xg_w64_params()

    def close(self):
        if getattr(self, "ctx", None):
            L.xg_w64_destroy(self.ctx)
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

    def seed(self, seeds, first: int = 0):
        s = np.ascontiguousarray(np.asarray(seeds, dtype=np.uint32).ravel())
        L.xg_w64_seed(self.ctx, first, s.size, s.ctypes.data)
        return self

    def get_state(self, stream: int):
        ring = np.zeros(64, dtype=np.uint64)
        w = L.xg_w64_get_state(self.ctx, stream, ring.ctypes.data)
        return ring, w

    def set_state(self, stream: int, ring, weyl: int):
        r = np.ascontiguousarray(np.asarray(ring, dtype=np.uint64))
        assert r.size == 64
        L.xg_w64_set_state(self.ctx, stream, r.ctypes.data, weyl)

    def set_launch(self, kind: str, tpg: int = 0, wpl: int = 0, block: int = 0):
        L.xg_w64_set_launch(self.ctx, TYPES_W64[kind], tpg, wpl, block)

    def autotune(self, kind: str, n_per_stream: int, nstreams: int = 0) -> dict:
        return L.xg_w64_autotune(self.ctx, TYPES_W64[kind], nstreams, n_per_stream)

    def jump(self, words: int, first: int = 0, count=None):
        """Advance streams by `words` positions without generating them."""
        count = self.n - first if count is None else count
        L.xg_w64_jump(self.ctx, first, count, words)

    def seed_substreams(self, seed: int, log2_spacing: int, first: int = 0, count=None):
        """Streams first + i start at position i * 2^log2_spacing of the one
        sequence seeded by `seed`."""
        count = self.n - first if count is None else count
        L.xg_w64_seed_substreams(self.ctx, first, count, seed, log2_spacing)

    def set_split(self, piece_words: int):
        """0: automatic, 1: never cut long calls on few streams, else the piece length."""
        L.xg_w64_set_split(self.ctx, piece_words)

    def _gen(self, fn, dtype, n, first, count, out, ld):
        count = self.n - first if count is None else count
        if out is None:
            ld = n if ld is None else ld
            out = torch.empty((count, ld), dtype=dtype, device="cuda")
        else:
            ld = out.stride(0) if (ld is None and out.dim() == 2) else (ld if ld is not None else n)
        fn(self.ctx, first, count, n, out.data_ptr(), ld)
        return out

    def u64(self, n: int, first: int = 0, count=None, out=None, ld=None):
        """n words per stream as int64 bit patterns, shape (count, ld)."""
        return self._gen(L.xg_w64_generate_u64, torch.int64, n, first, count, out, ld)

    def uniform(self, n: int, first: int = 0, count=None, out=None, ld=None):
        """n FP64 uniforms in [0, 1) per stream."""
        return self._gen(L.xg_w64_generate_uniform_f64, torch.float64, n, first, count, out, ld)

    def generate(self, kind: str, n: int, **kw):
        return {"u64": self.u64, "uniform": self.uniform}[kind](n, **kw)

    def transform_uniform(self, words: torch.Tensor, out=None):
        """FP64 uniforms of given 64-bit words (an int64 device tensor)."""
        out = torch.empty(words.numel(), dtype=torch.float64, device="cuda") if out is None else out
        L.xg_w64_transform_uniform_f64(self.ctx, words.data_ptr(), words.numel(), out.data_ptr())
        return out
