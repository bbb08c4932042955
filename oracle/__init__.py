"""xorgens oracle -- TEST INFRASTRUCTURE ONLY.

Plain, slow, serial CPU implementation of the xorgens generator of
Nandapalan, Brent, Murray and Rendell (arXiv:1108.0486): the recurrence and
circular buffer of Sec. 2, the Weyl generator and output combination of
Sec. 1.5 Eq. (1), and this project's uniform / Box-Muller conversions (FP64).
The arithmetic lives in ``xorgens_oracle.c`` (generator) and ``gf2.c``
(Berlekamp-Massey and Rabin's irreducibility test, used only to pin the
recurrence); this module compiles them with gcc and wraps them with ctypes.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s cpu_baseline /
reference legs may import this package.  It shares no code with the GPU
library and never imports it.

Parity status (each pin lives in ``tests/test_oracle_pins.py``):
  * recurrence, circular buffer   -- pinned (irreducible degree-4096 minimal
    polynomial for both published parameter sets, impulse responses in closed
    form, lag dependency, GF(2) linearity, tiny sets by brute-force period)
  * Weyl word and Eq. (1)         -- pinned (closed form of omega, invariant
    out_k - x_k = h(w_0 + k omega))
  * uniform conversion            -- pinned (exact closed form)
  * Box-Muller in FP64            -- pinned (special points, against
    math.sin/cos on the reduced angle, moments)
  * seeding (project definition)  -- parity unpinned: the paper defers to the
    xorgens package, which is not available; only determinism and
    distinctness are checked.
"""
from __future__ import annotations

import contextlib
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SOURCES = ("xorgens_oracle.c", "gf2.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_LIB_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

# The parameter sets named in the paper and used by the library:
#   (128, 95, 17, 12, 13, 15): default set of this library,
#   (128, 65, 15, 14, 12, 17): the set the paper reports results for (Sec. 2).
PARAM_SETS = {
    0: (128, 95, 17, 12, 13, 15),
    1: (128, 65, 15, 14, 12, 17),
}


class _Gen(ctypes.Structure):
    _fields_ = [
        ("w", ctypes.c_uint32), ("r", ctypes.c_uint32), ("s", ctypes.c_uint32),
        ("a", ctypes.c_uint32), ("b", ctypes.c_uint32), ("c", ctypes.c_uint32),
        ("d", ctypes.c_uint32), ("weyl_on", ctypes.c_uint32), ("mask", ctypes.c_uint32),
        ("omega", ctypes.c_uint32), ("gamma", ctypes.c_uint32), ("i", ctypes.c_uint32),
        ("weyl", ctypes.c_uint32), ("k", ctypes.c_uint64), ("x", ctypes.c_uint32 * 256),
    ]


def build(force: bool = False, plant: int = 0) -> str:
    """Compile the oracle's C sources into a shared library (gcc, -O2).
    plant != 0 builds a variant with a deliberate mistake (tests only)."""
    os.makedirs(_LIB_DIR, exist_ok=True)
    srcs = [os.path.join(_HERE, s) for s in _SOURCES]
    path = _LIB_PATH if plant == 0 else os.path.join(_LIB_DIR, f"liboracle_plant{plant}.so")
    if not force and os.path.exists(path):
        newest = max(os.path.getmtime(s) for s in srcs)
        if os.path.getmtime(path) >= newest:
            return path
    tmp = path + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", f"-DXGO_PLANT={int(plant)}", "-fPIC",
           "-shared", "-o", tmp, *srcs, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, path)
    return path


def _declare(L):
    u32, u64, p = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_void_p
    G = ctypes.POINTER(_Gen)
    L.xgo_sizeof.restype = ctypes.c_size_t
    assert L.xgo_sizeof() == ctypes.sizeof(_Gen), "oracle struct layout mismatch"
    L.xgo_omega.argtypes = [u32]; L.xgo_omega.restype = u32
    L.xgo_init.argtypes = [G, u32, u32, u32, u32, u32, u32, u32, u32]
    L.xgo_init.restype = ctypes.c_int
    L.xgo_set_state.argtypes = [G, p, u32]
    L.xgo_get_state.argtypes = [G, p, p]
    L.xgo_step.argtypes = [G]; L.xgo_step.restype = u32
    L.xgo_next.argtypes = [G]; L.xgo_next.restype = u32
    L.xgo_combine.argtypes = [G, u32, u32]; L.xgo_combine.restype = u32
    L.xgo_seed32.argtypes = [G, u32]; L.xgo_seed32.restype = ctypes.c_int
    L.xgo_uniform.argtypes = [u32]; L.xgo_uniform.restype = ctypes.c_float
    L.xgo_normal_pair.argtypes = [u32, u32, p, p]
    L.xgo_normal_pairs.argtypes = [p, u64, p]
    for f in ("xgo_fill_u32", "xgo_fill_raw", "xgo_fill_uniform", "xgo_fill_normal"):
        getattr(L, f).argtypes = [G, u64, p]
    L.xgo_sum_normal.argtypes = [G, u64]; L.xgo_sum_normal.restype = ctypes.c_double
    L.xgo_streams.argtypes = [u32, u32, u32, u32, u32, u32, u32, p, u32, u64,
                              ctypes.c_int, p]
    L.xgo_streams.restype = ctypes.c_int
    L.xgo_cycle_length.argtypes = [G, u64]; L.xgo_cycle_length.restype = u64
    L.xgo_berlekamp_massey.argtypes = [p, ctypes.c_int, p]
    L.xgo_berlekamp_massey.restype = ctypes.c_int
    L.xgo_poly_irreducible.argtypes = [p, ctypes.c_int]
    L.xgo_poly_irreducible.restype = ctypes.c_int
    return L


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _declare(ctypes.CDLL(build()))
    return _lib


@contextlib.contextmanager
def planted(plant: int):
    """Temporarily route every oracle call to a variant built with a
    deliberate mistake (XGO_PLANT in xorgens_oracle.c); for the tests that
    check that the pins catch such mistakes."""
    global _lib
    lib()
    with _lock:
        saved = _lib
        _lib = _declare(ctypes.CDLL(build(plant=plant)))
    try:
        yield
    finally:
        with _lock:
            _lib = saved


def _ptr(a: np.ndarray) -> int:
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data


def omega(w: int = 32) -> int:
    return int(lib().xgo_omega(w))


class Xorgens:
    """One serial xorgens generator (w-bit words, parameters {r,s,a,b,c,d})."""

    def __init__(self, r=128, s=95, a=17, b=12, c=13, d=15, w=32, weyl=True):
        self.g = _Gen()
        if lib().xgo_init(ctypes.byref(self.g), w, r, s, a, b, c, d, int(bool(weyl))):
            raise ValueError("invalid xorgens parameters")

    @classmethod
    def param_set(cls, idx: int = 0, weyl=True) -> "Xorgens":
        return cls(*PARAM_SETS[idx], weyl=weyl)

    @property
    def r(self) -> int:
        return self.g.r

    def seed(self, seed: int) -> "Xorgens":
        if lib().xgo_seed32(ctypes.byref(self.g), seed & 0xFFFFFFFF):
            raise ValueError("seeding needs w = 32")
        return self

    def set_state(self, x_oldest_first, weyl: int) -> "Xorgens":
        x = np.ascontiguousarray(np.asarray(x_oldest_first, dtype=np.uint32))
        assert x.size == self.g.r
        lib().xgo_set_state(ctypes.byref(self.g), _ptr(x), weyl & 0xFFFFFFFF)
        return self

    def get_state(self):
        x = np.zeros(self.g.r, dtype=np.uint32)
        w = np.zeros(1, dtype=np.uint32)
        lib().xgo_get_state(ctypes.byref(self.g), _ptr(x), _ptr(w))
        return x, int(w[0])

    def step(self) -> int:
        """Advance the recurrence (and Weyl word); return x_k."""
        return int(lib().xgo_step(ctypes.byref(self.g)))

    def next(self) -> int:
        return int(lib().xgo_next(ctypes.byref(self.g)))

    @property
    def weyl(self) -> int:
        return int(self.g.weyl)

    def u32(self, n: int) -> np.ndarray:
        out = np.empty(n, dtype=np.uint32)
        lib().xgo_fill_u32(ctypes.byref(self.g), n, _ptr(out))
        return out

    def raw(self, n: int) -> np.ndarray:
        out = np.empty(n, dtype=np.uint32)
        lib().xgo_fill_raw(ctypes.byref(self.g), n, _ptr(out))
        return out

    def uniform(self, n: int) -> np.ndarray:
        out = np.empty(n, dtype=np.float32)
        lib().xgo_fill_uniform(ctypes.byref(self.g), n, _ptr(out))
        return out

    def normal64(self, n: int) -> np.ndarray:
        out = np.empty(n, dtype=np.float64)
        lib().xgo_fill_normal(ctypes.byref(self.g), n, _ptr(out))
        return out

    def sum_normal64(self, n: int) -> float:
        return float(lib().xgo_sum_normal(ctypes.byref(self.g), n))

    def cycle_length(self, limit: int) -> int:
        return int(lib().xgo_cycle_length(ctypes.byref(self.g), limit))

    def clone(self) -> "Xorgens":
        o = Xorgens.__new__(Xorgens)
        o.g = _Gen()
        ctypes.pointer(o.g)[0] = self.g
        return o


def uniform_of(words: np.ndarray) -> np.ndarray:
    """Uniform conversion applied word by word through the oracle."""
    f = lib().xgo_uniform
    return np.array([f(int(v)) for v in np.asarray(words).ravel()], dtype=np.float32)


def normal_pair64(o1: int, o2: int):
    z1 = np.zeros(1); z2 = np.zeros(1)
    lib().xgo_normal_pair(o1 & 0xFFFFFFFF, o2 & 0xFFFFFFFF, _ptr(z1), _ptr(z2))
    return float(z1[0]), float(z2[0])


def normal_pairs64(words) -> np.ndarray:
    """FP64 Box-Muller of consecutive word pairs (2i, 2i+1)."""
    w = np.ascontiguousarray(np.asarray(words, dtype=np.uint32).ravel())
    assert w.size % 2 == 0
    out = np.empty(w.size, dtype=np.float64)
    lib().xgo_normal_pairs(_ptr(w), w.size // 2, _ptr(out))
    return out


def streams(seeds, n: int, kind: str = "u32", param_set: int = 0, weyl=True) -> np.ndarray:
    """n outputs from each freshly seeded stream, shape (len(seeds), n)."""
    seeds = np.ascontiguousarray(np.asarray(seeds, dtype=np.uint32))
    dt = {"u32": np.uint32, "uniform": np.float32, "normal": np.float64}[kind]
    k = {"u32": 0, "uniform": 1, "normal": 2}[kind]
    out = np.empty((seeds.size, n), dtype=dt)
    rc = lib().xgo_streams(*PARAM_SETS[param_set], int(bool(weyl)), _ptr(seeds),
                           seeds.size, n, k, _ptr(out))
    if rc:
        raise ValueError("oracle stream generation failed")
    return out


def berlekamp_massey(bits) -> np.ndarray:
    """Connection polynomial C (coefficients low to high, length L+1)."""
    b = np.ascontiguousarray(np.asarray(bits, dtype=np.uint8) & 1)
    conn = np.zeros(b.size + 1, dtype=np.uint8)
    L = lib().xgo_berlekamp_massey(_ptr(b), b.size, _ptr(conn))
    if L < 0:
        raise MemoryError
    return conn[: L + 1].copy()


def is_irreducible(coeffs) -> bool:
    c = np.ascontiguousarray(np.asarray(coeffs, dtype=np.uint8) & 1)
    n = c.size - 1
    rc = lib().xgo_poly_irreducible(_ptr(c), n)
    if rc < 0:
        raise ValueError("polynomial must be monic of degree >= 1")
    return bool(rc)
