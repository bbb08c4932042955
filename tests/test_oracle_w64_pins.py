"""Pins for the 64-bit-word oracle (w = 64) and for the primitivity test.

As for the 32-bit oracle, each test checks against something independent of
the oracle's code: closed forms of the shift operators on bit sets, exact
integer arithmetic, brute-force orders of z on small polynomials, the
complete factorisation of 2^4096 - 1, and library routines.
"""
import math
import os
import random

import numpy as np
import pytest

import oracle as O
from test_oracle_pins import _order_of_z

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
MASK64 = (1 << 64) - 1


def _w64_golden():
    d = {}
    with open(os.path.join(GOLDEN, "w64_param_set.txt")) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if line:
                k, v = line.split(None, 1)
                d[k] = v.strip()
    return d


def _miller_rabin(n, rounds=24, seed=4096):
    if n < 2:
        return False
    for p in (2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37):
        if n % p == 0:
            return n == p
    d, s = n - 1, 0
    while d % 2 == 0:
        d //= 2
        s += 1
    rng = random.Random(seed)
    for _ in range(rounds):
        x = pow(rng.randrange(2, n - 1), d, n)
        if x in (1, n - 1):
            continue
        for _ in range(s - 1):
            x = x * x % n
            if x == n - 1:
                break
        else:
            return False
    return True


# ------------------------------------------------------ primitivity test

def test_fermat_factorisation_of_2_4096_minus_1():
    """2^4096 - 1 = F_0 F_1 ... F_11; the factor lists multiply out exactly,
    every factor is a (probable) prime, and every factor of F_k (k >= 2) has
    the form j 2^(k+2) + 1 (Euler and Lucas)."""
    allq = []
    for k in range(12):
        fs = O.fermat_factors(k)
        assert math.prod(fs) == (1 << (1 << k)) + 1
        for q in fs:
            assert _miller_rabin(q), (k, q)
            if k >= 2:
                assert (q - 1) % (1 << (k + 2)) == 0, (k, q)
        allq += fs
    assert math.prod(allq) == (1 << 4096) - 1
    assert len(set(allq)) == len(allq) == 25


def test_primitivity_small_textbook_cases():
    # z^4 + z + 1: primitive (order 15); z^4 + z^3 + z^2 + z + 1: irreducible,
    # order 5 (it divides z^5 - 1); z^4 + z^2 + 1 = (z^2 + z + 1)^2: reducible
    assert O.is_primitive([1, 1, 0, 0, 1])
    assert O.is_irreducible([1, 1, 1, 1, 1]) and not O.is_primitive([1, 1, 1, 1, 1])
    assert O.has_order([1, 1, 1, 1, 1], 5, [5])
    assert not O.is_primitive([1, 0, 1, 0, 1])


def test_zpow_against_brute_force_on_degree_8():
    """z^e mod P by the oracle's powering routine equals repeated
    multiplication by z, and is_primitive agrees with the brute-force order of
    z, for every monic P of degree 8 with P(0) = 1."""
    n = 8
    rng = np.random.default_rng(3)
    for p_low in range(1, 1 << n, 2):
        p_int = p_low | (1 << n)
        coeffs = [(p_int >> i) & 1 for i in range(n + 1)]
        order = _order_of_z(p_int, n, 1 << n)
        assert O.is_primitive(coeffs) == (order == (1 << n) - 1), p_int
        e = int(rng.integers(0, 5000))
        a = 1
        for _ in range(e):
            a <<= 1
            if (a >> n) & 1:
                a ^= p_int
        got = O.zpow(coeffs, e)
        assert sum(int(v) << i for i, v in enumerate(got)) == a, (p_int, e)


def test_primitivity_agrees_with_brute_force_periods_of_tiny_sets():
    """w = 8, r = 2, s = 1 generators (16-bit state): the oracle's
    primitivity test on the minimal polynomial says 'primitive' exactly when
    the brute-force cycle length is 2^16 - 1 (2^16 - 1 = 3 * 5 * 17 * 257)."""
    seen = {True: 0, False: 0}
    for a in range(1, 8):
        for b in range(1, 8):
            for c in (1, 3, 5, 7):
                for d in (1, 3, 5, 7):
                    g = O.Xorgens(2, 1, a, b, c, d, w=8, weyl=False).set_state([1, 0], 0)
                    cyc = g.cycle_length(1 << 16)
                    P = O.minimal_polynomial_of_bits(g.clone().raw(64) & 1)
                    prim = P.size - 1 == 16 and O.is_primitive(P)
                    assert prim == (cyc == (1 << 16) - 1), (a, b, c, d, cyc)
                    seen[prim] += 1
    assert seen[True] > 0 and seen[False] > 0


@pytest.mark.parametrize("ps", [0, 1])
def test_published_32bit_sets_are_primitive(ps):
    """Table 1: period 2^4128 = 2^32 (2^4096 - 1 + 1) -- the linear part has
    the full period 2^4096 - 1, i.e. a primitive characteristic polynomial."""
    g = O.Xorgens.param_set(ps, weyl=False).seed(3)
    P = O.minimal_polynomial_of_bits(g.raw(2 * 4096 + 64) & 1)
    assert P.size - 1 == 4096
    assert O.is_primitive(P)


# ------------------------------------------------------ 64-bit generator

def test_omega64_nearest_odd_to_golden_closed_form():
    """Sec. 1.5: omega is the odd integer nearest 2^(w-1) (sqrt 5 - 1).  With
    w = 64: |omega - t| < 1 with omega odd, checked by exact integers:
    (omega + 2^63 - 1)^2 < 5 * 2^126 < (omega + 2^63 + 1)^2.  It is the
    familiar golden-ratio constant 2^64 / phi."""
    om = O.omega64()
    assert om & 1
    assert (om + (1 << 63) - 1) ** 2 < 5 << 126 < (om + (1 << 63) + 1) ** 2
    assert om == 0x9E3779B97F4A7C15


def test_param_set_w64_matches_golden_record():
    k = _w64_golden()
    assert O.PARAM_SET_W64 == tuple(int(v) for v in k["params"].split(","))


def _unit_response64(p, q, j):
    """e_j (I + L^p)(I + R^q) on 64-bit words as a set of bit positions."""
    s = {j}
    if j + p < 64:
        s ^= {j + p}
    s ^= {i - q for i in s if i >= q}
    return sum(1 << i for i in s)


def test_w64_impulse_response_closed_form():
    """Sec. 2 recurrence with w = 64: one bit in x_{k-r} (resp. x_{k-s}) gives
    the closed form of the left (resp. right) operator pair; other slots 0."""
    r, s, a, b, c, d = O.PARAM_SET_W64
    for j in range(64):
        for slot, expect in ((0, _unit_response64(a, b, j)), (r - s, _unit_response64(c, d, j)),
                             (1, 0), (r - 1, 0), (r - s + 1, 0)):
            x = np.zeros(r, dtype=np.uint64)
            x[slot] = np.uint64(1 << j)
            g = O.Xorgens64(r, s, a, b, c, d, weyl=False).set_state(x, 0)
            assert g.step() == expect, (j, slot)


def test_w64_lag_dependency():
    """Flipping state word j first changes output j+1 (lag r) or, for
    j >= r - s, output j + 1 - (r - s) (lag s)."""
    r, s, a, b, c, d = O.PARAM_SET_W64
    rng = np.random.default_rng(64)
    x0 = rng.integers(0, 2**63, r, dtype=np.uint64) * np.uint64(2) + np.uint64(1)
    base = O.Xorgens64(r, s, a, b, c, d, weyl=False).set_state(x0, 0).raw(2 * r)
    for j in range(r):
        x1 = x0.copy()
        x1[j] ^= np.uint64(1 << (j % 64))
        pert = O.Xorgens64(r, s, a, b, c, d, weyl=False).set_state(x1, 0).raw(2 * r)
        first = int(np.flatnonzero(pert != base)[0]) + 1
        assert first == (j + 1 if j < r - s else j + 1 - (r - s)), j


def test_w64_gf2_linearity():
    r, s, a, b, c, d = O.PARAM_SET_W64
    rng = np.random.default_rng(65)
    xa = rng.integers(0, 2**64 - 1, r, dtype=np.uint64, endpoint=True)
    xb = rng.integers(0, 2**64 - 1, r, dtype=np.uint64, endpoint=True)
    mk = lambda x: O.Xorgens64(r, s, a, b, c, d, weyl=False).set_state(x, 0)
    assert np.array_equal(mk(xa ^ xb).raw(3000), mk(xa).raw(3000) ^ mk(xb).raw(3000))


def test_w64_minimal_polynomial_primitive_degree_4096():
    """The chosen set's linear part has period 2^4096 - 1: the minimal
    polynomial of output bits 0 and 63 has degree r w = 4096 and is primitive
    (z has order 2^4096 - 1, checked against all 25 prime factors)."""
    r, s, a, b, c, d = O.PARAM_SET_W64
    g = O.Xorgens64(r, s, a, b, c, d, weyl=False).seed(11)
    raw = g.raw(2 * 4096 + 64)
    P0 = O.minimal_polynomial_of_bits(raw & np.uint64(1))
    P63 = O.minimal_polynomial_of_bits(raw >> np.uint64(63))
    assert P0.size - 1 == 4096 and np.array_equal(P0, P63)
    assert O.is_irreducible(P0)
    assert O.is_primitive(P0)
    assert int(P0.sum()) == int(_w64_golden()["weight"])


def test_w64_weyl_combination_invariant():
    """Eq. (1) with w = 64, gamma = 32: out_k - x_k = w_k xor (w_k >> 32) with
    w_k = w_0 + k omega mod 2^64 (Weyl word advanced before use)."""
    r, s, a, b, c, d = O.PARAM_SET_W64
    rng = np.random.default_rng(66)
    x = rng.integers(0, 2**64 - 1, r, dtype=np.uint64, endpoint=True)
    w0 = 0x0123456789ABCDEF
    out = O.Xorgens64(r, s, a, b, c, d, weyl=True).set_state(x, w0).u64(2000)
    raw = O.Xorgens64(r, s, a, b, c, d, weyl=False).set_state(x, w0).raw(2000)
    om = 0x9E3779B97F4A7C15
    for k in range(1, 2001):
        wk = (w0 + k * om) & MASK64
        assert (int(out[k - 1]) - int(raw[k - 1])) & MASK64 == wk ^ (wk >> 32), k


def test_w64_uniform_closed_form():
    """(o >> 11) 2^-53, exact: compared with Python's exact rationals."""
    from fractions import Fraction
    rng = np.random.default_rng(67)
    words = [0, 1, (1 << 11) - 1, 1 << 11, MASK64, 1 << 63] + \
        [int(v) for v in rng.integers(0, 2**64 - 1, 2000, dtype=np.uint64, endpoint=True)]
    got = O.uniform64_of(words)
    for o, u in zip(words, got):
        assert Fraction(float(u)) == Fraction(o >> 11, 1 << 53)
    assert got[4] == 1.0 - 2.0**-53 and got[3] == 2.0**-53 and got[0] == 0.0


def test_w64_split_invariance_and_state_roundtrip():
    p = O.PARAM_SET_W64
    g = O.Xorgens64(*p).seed(5)
    whole = g.clone().u64(1000)
    h = g.clone()
    parts = np.concatenate([h.u64(1), h.u64(300), h.u64(699)])
    assert np.array_equal(whole, parts)
    x, w = g.get_state()
    g2 = O.Xorgens64(*p).set_state(x, w)
    assert np.array_equal(g2.u64(500), g.clone().u64(500))


def test_w64_seeding_determinism_and_distinct_streams():
    """Seeding is this project's definition (pinned above): also deterministic,
    distinct seeds give distinct streams, seed 0 is valid."""
    a = O.streams64([0, 1, 2, 0xFFFFFFFF], 256)
    b = O.streams64([0, 1, 2, 0xFFFFFFFF], 256)
    assert np.array_equal(a, b)
    assert len({row.tobytes() for row in a}) == 4
    assert all(np.any(row != 0) for row in a)
    u = O.streams64([9], 100000, kind="uniform")[0]
    assert 0.0 <= u.min() and u.max() < 1.0 and abs(u.mean() - 0.5) < 0.005


def test_w64_seed_xorshift_is_marsaglia_13_7_17_full_period():
    """The 64-bit oracle's own copy of the seed expander: Marsaglia's
    (13, 7, 17) as a product of shift matrices, of order 2^64 - 1."""
    from test_oracle_pins import _check_xorshift
    _check_xorshift(O.xorshift64_w64)


def test_w64_seed_procedure_recovered_through_the_warm_up():
    """Undo the 4r = 256-word warm-up of a seeded 64-bit state: the ring and
    w_0 before it are xorshift outputs 65 .. 129 of v, whole 64-bit words,
    oldest first (matrix powers of the xorshift, not the oracle's loop)."""
    from test_oracle_pins import MASK64, SEED_CASES, _expected_seed_words, _undo_steps
    r, s, a, b, c, d = O.PARAM_SET_W64
    om = O.omega64()
    for seed in SEED_CASES:
        x, w = O.Xorgens64(*O.PARAM_SET_W64).seed(seed).get_state()
        ring0 = _undo_steps(x, r, s, a, b, c, d, 4 * r, MASK64)
        w0 = (w - 4 * r * om) & MASK64
        assert ring0 + [w0] == _expected_seed_words(seed, r + 1, 64), f"seed {seed:#x}"


def test_w64_outputs_after_jump_equal_stepping():
    for J in (0, 1, 63, 64, 4097, 100003, (1 << 21) + 5):
        for weyl in (False, True):
            got = O.u64_after_jump(11, J, 24, weyl=weyl)
            g = O.Xorgens64(*O.PARAM_SET_W64, weyl=weyl).seed(11)
            ref = g.u64(J + 24)[J:] if weyl else g.raw(J + 24)[J:]
            assert np.array_equal(got, ref), (J, weyl)
