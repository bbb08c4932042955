"""Derive the FP32 polynomial coefficients of the GPU Box-Muller transform.

The kernels evaluate, in binary32 with fused multiply-adds,
  * ln(1 + t) = t + t^2 Q(t)          for t in [sqrt(1/2) - 1, sqrt(2) - 1],
  * sin(pi x / 4) = x S(x^2)           for x in [-1, 1],
  * cos(pi x / 4) = 1 + x^2 C(x^2)     for x in [-1, 1],
and this script computes Q, S and C as weighted minimax polynomials with the
Remez exchange algorithm (E. Ya. Remez, 1934), in 60-digit arithmetic
(mpmath), then rounds them to binary32.  The weights make the error relative
to the function each polynomial finally produces.  The constant terms 1 (in
cos) and t (in the log) are kept outside the fitted polynomials so that the
results are exact at x = 0 and t = 0.

Run:  python derive_normal_coeffs.py      (prints the C++ constants)
"""
import struct

import mpmath as mp

mp.mp.dps = 60


def remez(f, w, a, b, deg, grid=6000, iters=40):
    """Weighted minimax polynomial p of degree deg minimising max |(f-p) w|."""
    n = deg + 2
    xs = [(a + b) / 2 - (b - a) / 2 * mp.cos(mp.pi * k / (n - 1)) for k in range(n)]
    pts = [a + (b - a) * mp.mpf(k) / grid for k in range(grid + 1)]
    best = None
    for _ in range(iters):
        A = mp.matrix(n, n)
        y = mp.matrix(n, 1)
        for i, x in enumerate(xs):
            for j in range(deg + 1):
                A[i, j] = x ** j
            A[i, deg + 1] = (-1) ** i / w(x)
            y[i] = f(x)
        sol = mp.lu_solve(A, y)
        c = [sol[j] for j in range(deg + 1)]

        def err(x):
            return (f(x) - mp.polyval(c[::-1], x)) * w(x)

        ev = [err(x) for x in pts]
        emax = max(abs(e) for e in ev)
        if best is None or emax < best[1]:
            best = (c, emax)
        # local extrema of the error, then keep an alternating set of n of them
        ext = [0] + [k for k in range(1, grid) if (ev[k] - ev[k - 1]) * (ev[k + 1] - ev[k]) <= 0] + [grid]
        sel = []
        for k in ext:
            if sel and mp.sign(ev[sel[-1]]) == mp.sign(ev[k]):
                if abs(ev[k]) > abs(ev[sel[-1]]):
                    sel[-1] = k
            else:
                sel.append(k)
        while len(sel) > n:
            sel.pop(0 if abs(ev[sel[0]]) < abs(ev[sel[-1]]) else -1)
        if len(sel) < n:
            break
        xs = [pts[k] for k in sel]
    return best


def f32(x):
    return struct.unpack("<f", struct.pack("<f", float(x)))[0]


def hexf(x):
    return float(x).hex()


def main():
    # ln(1+t) = t + t^2 Q(t); weight so that the error is relative to ln(1+t)
    lo, hi = mp.sqrt(mp.mpf(1) / 2) - 1, mp.sqrt(mp.mpf(2)) - 1
    Qf = lambda t: (mp.log1p(t) - t) / t ** 2 if t != 0 else mp.mpf(-1) / 2
    Qw = lambda t: t ** 2 / mp.log1p(t) if t != 0 else mp.mpf(0)
    Q, eQ = remez(Qf, lambda t: abs(Qw(t)) + mp.mpf(10) ** -40, lo, hi, 8)
    # sin(pi x/4) = x S(x^2), y = x^2 in [0, 1]; relative weight
    Sf = lambda y: mp.sin(mp.pi / 4 * mp.sqrt(y)) / mp.sqrt(y) if y > 0 else mp.pi / 4
    S, eS = remez(Sf, lambda y: 1 / Sf(y), mp.mpf(0), mp.mpf(1), 3)
    # cos(pi x/4) = 1 + y C(y); weight y / cos so that the error is relative to cos
    Cf = lambda y: (mp.cos(mp.pi / 4 * mp.sqrt(y)) - 1) / y if y > 0 else -(mp.pi / 4) ** 2 / 2
    C, eC = remez(Cf, lambda y: (y + mp.mpf(10) ** -40) / mp.cos(mp.pi / 4 * mp.sqrt(y)),
                  mp.mpf(0), mp.mpf(1), 3)
    # -2 ln 2 split so that e * HI is exact for |e| <= 24 (HI keeps 16 significant bits)
    n2l = -2 * mp.log(2)
    HI = mp.mpf(int(n2l * 2 ** 15)) / 2 ** 15
    LO = n2l - HI
    print(f"// minimax relative errors: Q {mp.nstr(eQ, 3)}, S {mp.nstr(eS, 3)}, C {mp.nstr(eC, 3)}")
    for name, cs in (("kLogQ", Q), ("kSinS", S), ("kCosC", C)):
        print(f"constexpr float {name}[{len(cs)}] = {{" +
              ", ".join(f"{hexf(f32(v))}f" for v in cs) + "};")
    print(f"constexpr float kNeg2Ln2Hi = {hexf(f32(HI))}f;")
    print(f"constexpr float kNeg2Ln2Lo = {hexf(f32(LO))}f;")
    assert f32(HI) == float(HI)


if __name__ == "__main__":
    main()
