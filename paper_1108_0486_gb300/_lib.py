"""ctypes binding of the C ABI in include/xorgens_gb300.h.

Argument marshalling only: every function here forwards to the entry point
of the same name in the in-tree shared library and raises XGError when it
returns a nonzero status.  Loading fails loudly when the library has not been
built; nothing here computes random numbers itself.
"""
from __future__ import annotations

import ctypes
import os
import threading

from .build import LIB_PATH

XG_OK, XG_EINVAL, XG_ENOMEM, XG_EAGAIN, XG_ETIMEDOUT, XG_ECUDA, XG_ENOTFOUND, XG_EDEVICE, XG_ECANCELED = range(9)
XG_U32, XG_UNIFORM_F32, XG_NORMAL_F32 = 0, 1, 2
STATUS_NAMES = {0: "XG_OK", 1: "XG_EINVAL", 2: "XG_ENOMEM", 3: "XG_EAGAIN", 4: "XG_ETIMEDOUT",
                5: "XG_ECUDA", 6: "XG_ENOTFOUND", 7: "XG_EDEVICE", 8: "XG_ECANCELED"}


class XGError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


_lock = threading.Lock()
_lib = None

u32, u64, vp, i32 = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_int
P_u32, P_u64, P_vp, P_i32 = (ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(ctypes.c_uint64),
                             ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_int))

class XgItem(ctypes.Structure):
    _fields_ = [("stream", ctypes.c_uint32), ("type", ctypes.c_uint32),
                ("count", ctypes.c_uint64), ("out", ctypes.c_void_p)]


class XgRequest(ctypes.Structure):
    _fields_ = [("stream", ctypes.c_uint32), ("type", ctypes.c_uint32),
                ("count", ctypes.c_uint64), ("d_out", ctypes.c_void_p)]


class XgServerConfig(ctypes.Structure):
    _fields_ = [("mem_cap_bytes", ctypes.c_uint64), ("max_batch", ctypes.c_uint32),
                ("lanes", ctypes.c_uint32)]


class XgCompletion(ctypes.Structure):
    _fields_ = [("ticket", ctypes.c_uint64), ("t_submit_ns", ctypes.c_uint64),
                ("t_launch_ns", ctypes.c_uint64), ("t_done_ns", ctypes.c_uint64),
                ("status", ctypes.c_int32), ("pad", ctypes.c_uint32), ("d_result", ctypes.c_void_p)]


class XgServerStats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in (
        "submitted", "completed", "refused", "queued", "in_flight", "batches", "items_launched",
        "outstanding_bytes", "now_ns", "host_launch_ns")]


# name -> argtypes (all return xg_status unless listed in _RESTYPES)
SIGNATURES = {
    "xg_create_streams": [P_vp, u32, u32, u32, vp],
    "xg_destroy": [vp],
    "xg_set_stream": [vp, vp],
    "xg_num_streams": [vp, P_u32],
    "xg_seed": [vp, u32, u32, vp],
    "xg_get_state": [vp, u32, vp, P_u32],
    "xg_set_state": [vp, u32, vp, u32],
    "xg_get_states": [vp, u32, u32, vp, vp, vp],
    "xg_set_states": [vp, u32, u32, vp, vp, vp],
    "xg_generate_u32": [vp, u32, u32, u64, vp, u64],
    "xg_generate_uniform": [vp, u32, u32, u64, vp, u64],
    "xg_generate_normal": [vp, u32, u32, u64, vp, u64],
    "xg_generate_normal_sum": [vp, u32, u32, u64, vp],
    "xg_transform_uniform": [vp, vp, u64, vp],
    "xg_transform_normal": [vp, vp, u64, vp],
    "xg_generate_batch": [vp, vp, u32],
    "xg_generate_batch_noalloc": [vp, vp, u32],
    "xg_set_batch_split": [vp, u64],
    "xg_set_batch_shape": [vp, i32, u32, u32],
    "xg_get_batch_shape": [vp, i32, P_u32, P_u32],
    "xg_autotune_batch": [vp, vp, u32, vp, vp, vp],
    "xg_jump": [vp, u32, u32, u64],
    "xg_server_start": [vp, vp],
    "xg_server_stop": [vp],
    "xg_submit": [vp, vp, P_u64],
    "xg_submit_many": [vp, vp, u32, vp, P_u32],
    "xg_poll": [vp, u64, P_i32, P_vp],
    "xg_wait": [vp, u64, u32, P_vp],
    "xg_release": [vp, u64],
    "xg_cancel": [vp, u64],
    "xg_ticket_times": [vp, u64, P_u64, P_u64, P_u64],
    "xg_server_stats_get": [vp, vp],
    "xg_collect": [vp, vp, u32, P_u32, i32],
    "xg_set_launch": [vp, i32, u32, u32],
    "xg_get_launch": [vp, i32, P_u32, P_u32],
    "xg_autotune": [vp, i32, u32, u64, P_u32, P_u32, P_u32, ctypes.POINTER(ctypes.c_float)],
    "xg_last_error": [],
    "xg_version": [],
    # 64-bit words (include/xorgens_w64.h)
    "xg_w64_params": [P_u32, P_u64],
    "xg_w64_create": [P_vp, u32, u32, vp],
    "xg_w64_destroy": [vp],
    "xg_w64_set_stream": [vp, vp],
    "xg_w64_seed": [vp, u32, u32, vp],
    "xg_w64_get_state": [vp, u32, vp, P_u64],
    "xg_w64_set_state": [vp, u32, vp, u64],
    "xg_w64_generate_u64": [vp, u32, u32, u64, vp, u64],
    "xg_w64_generate_uniform_f64": [vp, u32, u32, u64, vp, u64],
    "xg_w64_transform_uniform_f64": [vp, vp, u64, vp],
    "xg_w64_set_launch": [vp, i32, u32, u32, u32],
    "xg_w64_autotune": [vp, i32, u32, u64, P_u32, P_u32, P_u32, ctypes.POINTER(ctypes.c_float)],
    "xg_w64_jump": [vp, u32, u32, u64],
    "xg_seed_substreams": [vp, u32, u32, u32, u32],
    "xg_w64_seed_substreams": [vp, u32, u32, u32, u32],
    "xg_w64_set_split": [vp, u64],
}
_RESTYPES = {"xg_last_error": ctypes.c_char_p, "xg_version": ctypes.c_char_p}


def lib() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(
                    f"{LIB_PATH} is missing: build the CUDA library first "
                    "(python -c 'import __graft_entry__ as g; g.build()')")
            L = ctypes.CDLL(LIB_PATH)
            for name, args in SIGNATURES.items():
                fn = getattr(L, name)
                fn.argtypes = args
                fn.restype = _RESTYPES.get(name, ctypes.c_int)
            _lib = L
    return _lib


def last_error() -> str:
    return lib().xg_last_error().decode()


def check(status: int) -> None:
    if status != XG_OK:
        raise XGError(status, last_error())


def call(name: str, *args) -> None:
    check(getattr(lib(), name)(*args))


# ---- functions with the C names (argument marshalling only) -------------

def xg_create_streams(n_streams: int, param_set: int = 0, weyl_on: bool = True,
                      cuda_stream: int = 0) -> int:
    h = ctypes.c_void_p()
    call("xg_create_streams", ctypes.byref(h), n_streams, param_set, int(bool(weyl_on)),
         ctypes.c_void_p(cuda_stream))
    return h.value


def xg_destroy(ctx: int) -> None:
    call("xg_destroy", ctypes.c_void_p(ctx))


def xg_set_stream(ctx: int, cuda_stream: int) -> None:
    call("xg_set_stream", ctypes.c_void_p(ctx), ctypes.c_void_p(cuda_stream))


def xg_num_streams(ctx: int) -> int:
    n = ctypes.c_uint32()
    call("xg_num_streams", ctypes.c_void_p(ctx), ctypes.byref(n))
    return n.value


def xg_seed(ctx: int, first: int, count: int, host_seeds_ptr: int) -> None:
    call("xg_seed", ctypes.c_void_p(ctx), first, count, ctypes.c_void_p(host_seeds_ptr))


def xg_get_state(ctx: int, stream: int, host_ring_ptr: int) -> int:
    w = ctypes.c_uint32()
    call("xg_get_state", ctypes.c_void_p(ctx), stream, ctypes.c_void_p(host_ring_ptr), ctypes.byref(w))
    return w.value


def xg_set_state(ctx: int, stream: int, host_ring_ptr: int, weyl: int) -> None:
    call("xg_set_state", ctypes.c_void_p(ctx), stream, ctypes.c_void_p(host_ring_ptr), weyl & 0xFFFFFFFF)


def xg_get_states(ctx, first, count, rings_ptr, weyl_ptr, pos_ptr=0) -> None:
    call("xg_get_states", ctypes.c_void_p(ctx), first, count, ctypes.c_void_p(rings_ptr),
         ctypes.c_void_p(weyl_ptr), ctypes.c_void_p(pos_ptr or None))


def xg_set_states(ctx, first, count, rings_ptr, weyl_ptr, pos_ptr=0) -> None:
    call("xg_set_states", ctypes.c_void_p(ctx), first, count, ctypes.c_void_p(rings_ptr),
         ctypes.c_void_p(weyl_ptr), ctypes.c_void_p(pos_ptr or None))


def xg_generate_u32(ctx, first, nstreams, n_per_stream, out_ptr, ld) -> None:
    call("xg_generate_u32", ctypes.c_void_p(ctx), first, nstreams, n_per_stream, ctypes.c_void_p(out_ptr), ld)


def xg_generate_uniform(ctx, first, nstreams, n_per_stream, out_ptr, ld) -> None:
    call("xg_generate_uniform", ctypes.c_void_p(ctx), first, nstreams, n_per_stream, ctypes.c_void_p(out_ptr), ld)


def xg_generate_normal(ctx, first, nstreams, n_per_stream, out_ptr, ld) -> None:
    call("xg_generate_normal", ctypes.c_void_p(ctx), first, nstreams, n_per_stream, ctypes.c_void_p(out_ptr), ld)


def xg_generate_normal_sum(ctx, first, nstreams, n_per_stream, sums_ptr) -> None:
    call("xg_generate_normal_sum", ctypes.c_void_p(ctx), first, nstreams, n_per_stream, ctypes.c_void_p(sums_ptr))


def xg_transform_uniform(ctx, words_ptr, n, out_ptr) -> None:
    call("xg_transform_uniform", ctypes.c_void_p(ctx), ctypes.c_void_p(words_ptr), n, ctypes.c_void_p(out_ptr))


def xg_transform_normal(ctx, words_ptr, n, out_ptr) -> None:
    call("xg_transform_normal", ctypes.c_void_p(ctx), ctypes.c_void_p(words_ptr), n, ctypes.c_void_p(out_ptr))


def make_items(items):
    """A ctypes xg_item array from (stream, type, count, out_ptr) tuples (build
    it once to reuse it across calls)."""
    if isinstance(items, ctypes.Array):
        return items
    import numpy as np
    a = np.asarray(items, dtype=np.uint64).reshape(-1, 4)
    rec = np.zeros(a.shape[0], dtype=[("stream", "<u4"), ("type", "<u4"), ("count", "<u8"),
                                     ("out", "<u8")])
    rec["stream"], rec["type"], rec["count"], rec["out"] = a[:, 0], a[:, 1], a[:, 2], a[:, 3]
    arr = (XgItem * a.shape[0])()
    ctypes.memmove(arr, rec.ctypes.data, rec.nbytes)
    return arr


def xg_generate_batch(ctx, items) -> None:
    """items: sequence of (stream, type, count, out_ptr), or a make_items() array."""
    arr = make_items(items)
    call("xg_generate_batch", ctypes.c_void_p(ctx), arr, len(arr))


def xg_generate_batch_noalloc(ctx, items) -> None:
    """items: sequence of (stream, type, count, out_ptr), or a make_items()
    array; at most 1024."""
    arr = make_items(items)
    call("xg_generate_batch_noalloc", ctypes.c_void_p(ctx), arr, len(arr))


def xg_set_batch_shape(ctx, type_, tpg, wpl) -> None:
    call("xg_set_batch_shape", ctypes.c_void_p(ctx), int(type_), tpg, wpl)


def xg_get_batch_shape(ctx, type_):
    t, w = ctypes.c_uint32(), ctypes.c_uint32()
    call("xg_get_batch_shape", ctypes.c_void_p(ctx), int(type_), ctypes.byref(t), ctypes.byref(w))
    return t.value, w.value


def xg_autotune_batch(ctx, items):
    """Per output type: (tpg, wpl, median ms) of the fastest batch shape on
    the given batch (ms 0 for a type absent from it)."""
    arr = make_items(items)
    tpg = (ctypes.c_uint32 * 3)()
    wpl = (ctypes.c_uint32 * 3)()
    ms = (ctypes.c_float * 3)()
    call("xg_autotune_batch", ctypes.c_void_p(ctx), arr, len(arr), tpg, wpl, ms)
    return [(tpg[k], wpl[k], ms[k]) for k in range(3)]


def xg_set_batch_split(ctx, piece_words) -> None:
    call("xg_set_batch_split", ctypes.c_void_p(ctx), piece_words)


def xg_jump(ctx, first, nstreams, words) -> None:
    call("xg_jump", ctypes.c_void_p(ctx), first, nstreams, words)


def xg_seed_substreams(ctx, first, count, seed, log2_spacing) -> None:
    call("xg_seed_substreams", ctypes.c_void_p(ctx), first, count, seed, log2_spacing)


def xg_server_start(ctx, mem_cap_bytes=0, max_batch=0, lanes=0) -> None:
    cfg = XgServerConfig(mem_cap_bytes, max_batch, lanes)
    call("xg_server_start", ctypes.c_void_p(ctx), ctypes.byref(cfg))


def xg_server_stop(ctx) -> None:
    call("xg_server_stop", ctypes.c_void_p(ctx))


def xg_submit(ctx, stream, out_type, count, d_out=0) -> int:
    req = XgRequest(stream, out_type, count, d_out)
    t = ctypes.c_uint64()
    call("xg_submit", ctypes.c_void_p(ctx), ctypes.byref(req), ctypes.byref(t))
    return t.value


def make_requests(reqs):
    """A numpy record array laid out as xg_request[] from (stream, type,
    count, d_out) tuples (build it once, submit slices of it)."""
    import numpy as np
    a = np.asarray(reqs, dtype=np.uint64).reshape(-1, 4)
    rec = np.zeros(a.shape[0], dtype=[("stream", "<u4"), ("type", "<u4"), ("count", "<u8"),
                                     ("d_out", "<u8")])
    rec["stream"], rec["type"], rec["count"], rec["d_out"] = a[:, 0], a[:, 1], a[:, 2], a[:, 3]
    assert rec.itemsize == ctypes.sizeof(XgRequest)
    return rec


def xg_submit_many(ctx, rec, first, n, tickets):
    """Submit rec[first:first+n] (from make_requests); tickets (numpy uint64)
    receives their tickets at the same positions.  Returns how many were
    admitted (an XG_EAGAIN refusal is not raised: fewer than n come back)."""
    acc = ctypes.c_uint32()
    st = lib().xg_submit_many(ctypes.c_void_p(ctx), ctypes.c_void_p(rec.ctypes.data + first * rec.itemsize), n,
                              ctypes.c_void_p(tickets.ctypes.data + first * 8), ctypes.byref(acc))
    if st not in (XG_OK, XG_EAGAIN):
        check(st)
    return acc.value


def xg_poll(ctx, ticket):
    done, ptr = ctypes.c_int(), ctypes.c_void_p()
    call("xg_poll", ctypes.c_void_p(ctx), ticket, ctypes.byref(done), ctypes.byref(ptr))
    return bool(done.value), ptr.value


def xg_wait(ctx, ticket, timeout_ms=10000):
    ptr = ctypes.c_void_p()
    call("xg_wait", ctypes.c_void_p(ctx), ticket, timeout_ms, ctypes.byref(ptr))
    return ptr.value


def xg_release(ctx, ticket) -> None:
    call("xg_release", ctypes.c_void_p(ctx), ticket)


def xg_cancel(ctx, ticket) -> None:
    call("xg_cancel", ctypes.c_void_p(ctx), ticket)


def xg_ticket_times(ctx, ticket):
    a, b, c = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
    call("xg_ticket_times", ctypes.c_void_p(ctx), ticket, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c))
    return a.value, b.value, c.value


def xg_collect(ctx, max_n=4096, release=False, buf=None):
    """Finished tickets as a list of (ticket, t_submit, t_launch, t_done, status, d_result)."""
    arr = buf if buf is not None else (XgCompletion * max_n)()
    n = ctypes.c_uint32()
    call("xg_collect", ctypes.c_void_p(ctx), arr, len(arr), ctypes.byref(n), int(bool(release)))
    return [(c.ticket, c.t_submit_ns, c.t_launch_ns, c.t_done_ns, c.status, c.d_result)
            for c in arr[: n.value]]


COMPLETION_DTYPE = [("ticket", "<u8"), ("t_submit_ns", "<u8"), ("t_launch_ns", "<u8"), ("t_done_ns", "<u8"),
                    ("status", "<i4"), ("pad", "<u4"), ("d_result", "<u8")]


def xg_collect_into(ctx, buf, release=False) -> int:
    """xg_collect into a numpy record array of COMPLETION_DTYPE; returns the
    number of records written (no per-record Python objects)."""
    assert buf.itemsize == ctypes.sizeof(XgCompletion)
    n = ctypes.c_uint32()
    call("xg_collect", ctypes.c_void_p(ctx), ctypes.c_void_p(buf.ctypes.data), len(buf), ctypes.byref(n),
         int(bool(release)))
    return n.value


def xg_server_stats_get(ctx) -> dict:
    st = XgServerStats()
    call("xg_server_stats_get", ctypes.c_void_p(ctx), ctypes.byref(st))
    return {n: getattr(st, n) for n, _ in XgServerStats._fields_}


def xg_set_launch(ctx, out_type, tpg, wpl) -> None:
    call("xg_set_launch", ctypes.c_void_p(ctx), out_type, tpg, wpl)


def xg_get_launch(ctx, out_type):
    t, w = ctypes.c_uint32(), ctypes.c_uint32()
    call("xg_get_launch", ctypes.c_void_p(ctx), out_type, ctypes.byref(t), ctypes.byref(w))
    return t.value, w.value


def xg_autotune(ctx, out_type, nstreams, n_per_stream):
    t, w, b, ms = ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_float()
    call("xg_autotune", ctypes.c_void_p(ctx), out_type, nstreams, n_per_stream, ctypes.byref(t),
         ctypes.byref(w), ctypes.byref(b), ctypes.byref(ms))
    return {"tpg": t.value, "wpl": w.value, "block": b.value, "ms": ms.value}


def xg_version() -> str:
    return lib().xg_version().decode()


# ---- 64-bit words --------------------------------------------------------
XG_W64_U64, XG_W64_UNIFORM_F64 = 0, 1


def xg_w64_params():
    v = (ctypes.c_uint32 * 6)()
    om = ctypes.c_uint64()
    call("xg_w64_params", v, ctypes.byref(om))
    return tuple(v), om.value


def xg_w64_create(n_streams: int, weyl_on: bool = True, cuda_stream: int = 0) -> int:
    h = ctypes.c_void_p()
    call("xg_w64_create", ctypes.byref(h), n_streams, int(bool(weyl_on)), ctypes.c_void_p(cuda_stream))
    return h.value


def xg_w64_destroy(ctx: int) -> None:
    call("xg_w64_destroy", ctypes.c_void_p(ctx))


def xg_w64_set_stream(ctx: int, cuda_stream: int) -> None:
    call("xg_w64_set_stream", ctypes.c_void_p(ctx), ctypes.c_void_p(cuda_stream))


def xg_w64_seed(ctx: int, first: int, count: int, host_seeds_ptr: int) -> None:
    call("xg_w64_seed", ctypes.c_void_p(ctx), first, count, ctypes.c_void_p(host_seeds_ptr))


def xg_w64_get_state(ctx: int, stream: int, host_ring_ptr: int) -> int:
    w = ctypes.c_uint64()
    call("xg_w64_get_state", ctypes.c_void_p(ctx), stream, ctypes.c_void_p(host_ring_ptr), ctypes.byref(w))
    return w.value


def xg_w64_set_state(ctx: int, stream: int, host_ring_ptr: int, weyl: int) -> None:
    call("xg_w64_set_state", ctypes.c_void_p(ctx), stream, ctypes.c_void_p(host_ring_ptr), weyl)


def xg_w64_generate_u64(ctx, first, nstreams, n_per_stream, out_ptr, ld) -> None:
    call("xg_w64_generate_u64", ctypes.c_void_p(ctx), first, nstreams, n_per_stream, ctypes.c_void_p(out_ptr), ld)


def xg_w64_generate_uniform_f64(ctx, first, nstreams, n_per_stream, out_ptr, ld) -> None:
    call("xg_w64_generate_uniform_f64", ctypes.c_void_p(ctx), first, nstreams, n_per_stream,
         ctypes.c_void_p(out_ptr), ld)


def xg_w64_transform_uniform_f64(ctx, words_ptr, n, out_ptr) -> None:
    call("xg_w64_transform_uniform_f64", ctypes.c_void_p(ctx), ctypes.c_void_p(words_ptr), n,
         ctypes.c_void_p(out_ptr))


def xg_w64_set_launch(ctx, out_type, tpg, wpl, block=0) -> None:
    call("xg_w64_set_launch", ctypes.c_void_p(ctx), out_type, tpg, wpl, block)


def xg_w64_jump(ctx, first, nstreams, words) -> None:
    call("xg_w64_jump", ctypes.c_void_p(ctx), first, nstreams, words)


def xg_w64_set_split(ctx, piece_words) -> None:
    call("xg_w64_set_split", ctypes.c_void_p(ctx), piece_words)


def xg_w64_seed_substreams(ctx, first, count, seed, log2_spacing) -> None:
    call("xg_w64_seed_substreams", ctypes.c_void_p(ctx), first, count, seed, log2_spacing)


def xg_w64_autotune(ctx, out_type, nstreams, n_per_stream):
    t, w, b, ms = ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_float()
    call("xg_w64_autotune", ctypes.c_void_p(ctx), out_type, nstreams, n_per_stream, ctypes.byref(t),
         ctypes.byref(w), ctypes.byref(b), ctypes.byref(ms))
    return {"tpg": t.value, "wpl": w.value, "block": b.value, "ms": ms.value}
