"""Search for a 64-bit-word xorgens parameter set (r, s, a, b, c, d) with
r = 64 words, so that n = r w = 4096 as for the paper's 32-bit sets, whose
linear part has a primitive characteristic polynomial (period 2^4096 - 1,
Sec. 1.5).  Uses only the oracle.  Test infrastructure: it wrote the record
tests/golden/w64_param_set.txt that the tests and the library's constants
follow.

Candidates (this project's choices, not the paper's):
  * s odd (gcd(r, s) = 1) with 41 <= s <= 55, so that 32-word rounds fit
    (a round reads only words at least s back) and s stays away from r/2;
  * shifts a, b, c, d in [16, 48] -- near w/2, as in the published 32-bit
    sets -- with a != c and b != d.
For each candidate: the minimal polynomial of bit 0 of the raw words
(Berlekamp-Massey on 2n + 64 bits) must have degree n; a screen for factors
of degree <= 32; Rabin's test; then the order of z must be 2^n - 1.  Among
the primitive ones the set whose polynomial has weight (number of nonzero
coefficients) closest to n/2 is chosen: a sparse characteristic polynomial is
a known weakness of linear generators.

    python oracle/search_w64_params.py --tries 30000 --procs 6 --write tests/golden/w64_param_set.txt
"""
from __future__ import annotations

import argparse
import multiprocessing as mp
import os
import sys
import time

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import oracle  # noqa: E402

N = 4096


def candidates(tries: int, seed: int = 1108):
    rng = np.random.default_rng(seed)
    seen = set()
    while len(seen) < tries:
        s = int(rng.choice(np.arange(41, 57, 2)))
        a, b, c, d = (int(v) for v in rng.integers(16, 49, size=4))
        if a == c or b == d:
            continue
        t = (64, s, a, b, c, d)
        if t in seen:
            continue
        seen.add(t)
        yield t


def examine(params):
    g = oracle.Xorgens64(*params, weyl=False).seed(1)
    bits = (g.raw(2 * N + 64) & np.uint64(1)).astype(np.uint8)
    P = oracle.minimal_polynomial_of_bits(bits)
    if P.size - 1 != N:
        return params, "degree", None
    if oracle.small_factor(P, 32):
        return params, "small", None
    if not oracle.is_irreducible(P):
        return params, "reducible", None
    if not oracle.is_primitive(P):
        return params, "not primitive", None
    return params, "primitive", int(P.sum())


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--tries", type=int, default=6000)
    ap.add_argument("--procs", type=int, default=os.cpu_count() or 1)
    ap.add_argument("--write", default=None, help="write the chosen set's record to this path")
    args = ap.parse_args()
    oracle.lib()
    t0 = time.time()
    found = []
    counts = {}
    ctx = mp.get_context("spawn")
    with ctx.Pool(args.procs) as pool:
        for params, verdict, weight in pool.imap_unordered(examine, candidates(args.tries), chunksize=8):
            counts[verdict] = counts.get(verdict, 0) + 1
            if verdict == "primitive":
                found.append((abs(weight - N // 2), weight, params))
                print(f"primitive {params} weight {weight}", flush=True)
    found.sort()
    print(f"examined {sum(counts.values())} in {time.time() - t0:.0f} s: {counts}")
    if found:
        _, weight, params = found[0]
        print(f"chosen {params} weight {weight}")
        if args.write:
            write_record(args.write, args.tries, args.procs, counts, found, params, weight)


def write_record(path, tries, procs, counts, found, params, weight):
    """The record the tests read (tests/golden/w64_param_set.txt)."""
    lines = [
        "# 64-bit-word xorgens parameter set used by oracle/ and the library (w = 64).",
        "# The paper gives no 64-bit set (Sec. 1.5 states the family for general w);",
        "# this record was written by",
        f"#     python oracle/search_w64_params.py --tries {tries} --procs {procs} --write {path}",
        f"# which examined {sum(counts.values())} candidates (seeded PCG64 1108): "
        f"{counts.get('degree', 0)} had a minimal",
        f"# polynomial of degree < 4096, {counts.get('small', 0)} a factor of degree <= 32, "
        f"{counts.get('reducible', 0)} failed",
        f"# Rabin's test, {counts.get('not primitive', 0)} were irreducible but not primitive, "
        f"{counts.get('primitive', 0)} primitive:",
    ]
    for _, w, p in sorted(found, key=lambda f: f[2]):
        mark = "   <- chosen: weight closest to 2048" if p == params else ""
        lines.append(f"#     ({','.join(str(v) for v in p)}) weight {w}{mark}")
    lines += ["# The tests recheck primitivity (order of z = 2^4096 - 1) and the weight.",
              f"params {','.join(str(v) for v in params)}", f"weight {weight}", ""]
    with open(path, "w") as f:
        f.write("\n".join(lines))


if __name__ == "__main__":
    main()
