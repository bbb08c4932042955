"""GPU path against the CPU oracle, through the C ABI.

u32 words and uniforms must match bit for bit; FP32 normals must be within
4 ulp of the FP64 oracle rounded to FP32 (ulp taken at the rounded value).
Sizes span several rounds, tiles and a ragged tail; the full-size workloads
(16384 streams x 2^16 words) are checked on sampled streams.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_1108_0486_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

LAUNCHES = [(4, 8), (8, 4), (16, 2), (16, 4), (32, 2)]
KINDS = ["u32", "uniform", "normal"]
NORMAL_TOL_ULP = 4.0


@pytest.fixture(scope="module", autouse=True)
def _device():
    torch.cuda.set_device(0)
    yield
    torch.cuda.synchronize()


def Streams(*a, **k):
    from paper_1108_0486_gb300 import Streams as S
    return S(*a, **k)


def u32np(t):
    from paper_1108_0486_gb300 import as_u32
    return as_u32(t)


def ulp_error(z_gpu, z64):
    z64 = np.asarray(z64, dtype=np.float64)
    z32 = z64.astype(np.float32)
    ulp = np.spacing(np.abs(z32)).astype(np.float64)
    return np.abs(np.asarray(z_gpu, dtype=np.float64) - z64) / ulp


def convert_oracle(words, kind, n):
    """Oracle outputs of one call of n outputs from the given words."""
    if kind == "u32":
        return words[..., :n]
    if kind == "uniform":
        return O.uniform_of(words[..., :n]).reshape(words[..., :n].shape)
    nw = n + (n & 1)
    z = O.normal_pairs64(words[..., :nw]).reshape(words[..., :nw].shape)
    return z[..., :n]


def words_per_call(kind, n):
    return n + (n & 1) if kind == "normal" else n


def check(kind, got, ref):
    if kind == "normal":
        err = ulp_error(got, ref)
        assert float(err.max()) <= NORMAL_TOL_ULP, f"max normal error {err.max():.3f} ulp"
    elif kind == "uniform":
        assert np.array_equal(np.asarray(got, dtype=np.float32), ref)
    else:
        assert np.array_equal(np.asarray(got).view(np.uint32), ref)


def host(kind, t):
    return u32np(t) if kind == "u32" else t.cpu().numpy()


# --------------------------------------------------------------------------

def test_single_stream_2p20_words_bit_exact():
    cfg = W.SINGLE_STREAM
    with Streams(1, seeds=[cfg["seed"]]) as st:
        got = u32np(st.u32(cfg["n"]))[0]
    ref = O.Xorgens.param_set(0).seed(cfg["seed"]).u32(cfg["n"])
    assert np.array_equal(got, ref)


def test_golden_first_words():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden",
                        "xorgens_128_95_seed12345678_u32_first1024.txt")
    ref = np.array([int(l, 16) for l in open(path) if not l.startswith("#")], dtype=np.uint32)
    with Streams(1, seeds=[0x12345678]) as st:
        assert np.array_equal(u32np(st.u32(1024))[0], ref)


@pytest.mark.parametrize("ps", [0, 1])
@pytest.mark.parametrize("tpg,wpl", LAUNCHES)
@pytest.mark.parametrize("kind", KINDS)
def test_multi_stream_parity(ps, tpg, wpl, kind):
    """300 streams (ragged last block and group), n = 4133 (ragged rounds)."""
    seeds = W.seeds(300)
    n = 4133
    with Streams(300, param_set=ps, seeds=seeds) as st:
        st.set_launch(kind, tpg, wpl)
        got = host(kind, st.generate(kind, n))
    ref = convert_oracle(O.streams(seeds, words_per_call(kind, n), param_set=ps), kind, n)
    check(kind, got, ref)


@pytest.mark.parametrize("ps", [0, 1])
def test_split_invariance_mixed_types_and_launches(ps):
    """Any sequence of calls, of any sizes, types and launch configurations,
    reads consecutive words of each stream."""
    rng = np.random.default_rng(7 + ps)
    seeds = W.seeds(70, start=1000)
    calls = []
    for _ in range(40):
        kind = KINDS[rng.integers(0, 3)]
        n = int(rng.choice([1, 2, 3, 31, 32, 33, 63, 64, 65, 127, 128, 129, 500, 1001]))
        calls.append((kind, n, LAUNCHES[rng.integers(0, len(LAUNCHES))]))
    total = sum(words_per_call(k, n) for k, n, _ in calls)
    ref_words = O.streams(seeds, total, param_set=ps)
    off = 0
    with Streams(70, param_set=ps, seeds=seeds) as st:
        for kind, n, (tpg, wpl) in calls:
            st.set_launch(kind, tpg, wpl)
            got = host(kind, st.generate(kind, n))
            nw = words_per_call(kind, n)
            check(kind, got, convert_oracle(ref_words[:, off:off + nw], kind, n))
            off += nw


def test_ld_padding_and_unaligned_rows():
    """ld = n + 3 (rows not 16-byte aligned: scalar-store path); the padding
    between rows stays untouched."""
    seeds = W.seeds(50)
    n, ld = 777, 780 + 3
    for kind in KINDS:
        with Streams(50, seeds=seeds) as st:
            dt = torch.int32 if kind == "u32" else torch.float32
            out = torch.full((50, ld), -7, dtype=dt, device="cuda")
            st.generate(kind, n, out=out, ld=ld)
            h = host(kind, out)
        ref = convert_oracle(O.streams(seeds, words_per_call(kind, n)), kind, n)
        check(kind, h[:, :n], ref)
        pad = h[:, n:].view(np.int32) if kind == "u32" else h[:, n:]
        assert np.all(pad == -7)


def test_weyl_off_is_raw_part_and_gf2_linear():
    seeds = W.seeds(8, start=40)
    with Streams(8, weyl=False, seeds=seeds) as st:
        got = u32np(st.u32(3000))
    ref = np.stack([O.Xorgens.param_set(0, weyl=False).seed(int(s)).u32(3000) for s in seeds])
    assert np.array_equal(got, ref)
    rng = np.random.default_rng(3)
    xa = rng.integers(0, 2**32, 128, dtype=np.uint64).astype(np.uint32)
    xb = rng.integers(0, 2**32, 128, dtype=np.uint64).astype(np.uint32)
    with Streams(3, weyl=False) as st:
        st.set_state(0, xa, 0)
        st.set_state(1, xb, 0)
        st.set_state(2, xa ^ xb, 0)
        y = u32np(st.u32(5000))
    assert np.array_equal(y[2], y[0] ^ y[1])


def test_state_checkpoint_matches_oracle_state():
    seeds = W.seeds(4, start=9)
    with Streams(4, seeds=seeds) as st:
        for n in (1, 100, 33, 64, 1000):
            st.u32(n)
        ring, w = st.get_state(2)
        g = O.Xorgens.param_set(0).seed(int(seeds[2]))
        g.u32(1 + 100 + 33 + 64 + 1000)
        ref_ring, ref_w = g.get_state()
        assert np.array_equal(ring, ref_ring) and w == ref_w
        # restore into another stream and continue identically
        st.set_state(0, ring, w)
        a = u32np(st.u32(700))
        assert np.array_equal(a[0], a[2])
        assert np.array_equal(a[0], g.u32(700))


def test_bulk_checkpoint_restore_and_migrate():
    """xg_get_states / xg_set_states: the checkpoint equals the oracle's
    state, restoring it replays the same continuation, and loading it into
    another context (other seeds) makes that one continue identically."""
    S = 300
    seeds = W.seeds(S, start=901)
    with Streams(S, seeds=seeds) as st:
        st.uniform(1777)                                   # pend != 0 afterwards
        ck = st.checkpoint()
        for i in (0, 7, S - 1):
            g = O.Xorgens.param_set(0).seed(int(seeds[i]))
            g.u32(1777)
            ring, w = g.get_state()
            assert np.array_equal(ck["rings"][i], ring) and int(ck["weyl"][i]) == w
        assert np.all(ck["pos"] == 1777)
        ref = u32np(st.u32(2049))
        st.restore(ck)
        assert np.array_equal(u32np(st.u32(2049)), ref)
        part = st.checkpoint(first=100, count=50)
    with Streams(S, seeds=W.seeds(S, start=5)) as other:
        other.restore(ck)
        assert np.array_equal(u32np(other.u32(2049)), ref)
        assert np.all(other.checkpoint()["pos"] == 1777 + 2049)
        other.restore(part, first=0, positions=False)      # a slice into other streams
        got = u32np(other.u32(10, first=0, count=50))
    g = O.Xorgens.param_set(0).seed(int(seeds[100]))
    g.u32(1777 + 2049)                                     # where the slice was taken
    assert np.array_equal(got[0], g.u32(10))


def test_reseed_equals_fresh_context():
    seeds = W.seeds(20)
    with Streams(20, seeds=seeds) as st:
        st.u32(999)
        st.seed(seeds)
        a = u32np(st.u32(500))
    with Streams(20, seeds=seeds) as st2:
        b = u32np(st2.u32(500))
    assert np.array_equal(a, b)


# ---- the normal transform --------------------------------------------------

def _transform(words):
    with Streams(1) as st:
        t = torch.from_numpy(words.view(np.int32)).cuda()
        z = st.transform_normal(t)
        return z.cpu().numpy()


def test_normal_radius_all_m1():
    """Every u1 = m1 2^-24, m1 = 1 .. 2^24, at angle 0 (z1 = R, z2 = 0),
    including the FP64 tail branch m1 <= 62."""
    m1 = np.arange(1, (1 << 24) + 1, dtype=np.uint64)
    words = np.empty(2 * m1.size, dtype=np.uint32)
    words[0::2] = ((m1 - 1) << 8).astype(np.uint32) | 0x5A
    words[1::2] = 0x3C  # m2 = 0
    z = _transform(words)
    ref = O.normal_pairs64(words)
    err = ulp_error(z, ref)
    assert float(err.max()) <= NORMAL_TOL_ULP, err.max()
    assert np.all(z[1::2] == 0.0)


def test_normal_angle_all_m2():
    """Every u2 = m2 2^-24 at a fixed radius; quarter turns exact."""
    m2 = np.arange(0, 1 << 24, dtype=np.uint64)
    words = np.empty(2 * m2.size, dtype=np.uint32)
    words[0::2] = np.uint32((3_000_000 - 1) << 8)
    words[1::2] = (m2 << 8).astype(np.uint32)
    z = _transform(words)
    ref = O.normal_pairs64(words)
    err = ulp_error(z, ref)
    assert float(err.max()) <= NORMAL_TOL_ULP, err.max()
    assert np.all(z[ref == 0.0] == 0.0)


def test_normal_bits_same_at_every_launch():
    """The (32,2) launch runs the normal transform two pairs at a time with
    packed FP32x2 instructions; the other launches one pair at a time.  Every
    launch gives the same bits (ragged lengths, odd counts, both sets); the
    fused sums are checked per launch by test_fused_normal_sum."""
    for ps in (0, 1):
        seeds = W.seeds(50, start=311)
        outs = []
        for tpg, wpl in LAUNCHES:
            with Streams(50, param_set=ps, seeds=seeds) as st:
                st.set_launch("normal", tpg, wpl)
                z = [st.normal(n).cpu().numpy() for n in (1, 257, 4096 + 3, 20000)]
            outs.append(z)
        ref_z = outs[-1]
        for z, (tpg, wpl) in zip(outs, LAUNCHES):
            for a, b in zip(z, ref_z):
                assert np.array_equal(a.view(np.uint32), b.view(np.uint32)), (ps, tpg, wpl)


def test_normal_transform_packed_and_scalar_agree():
    """The stand-alone transform (two pairs per thread, packed) on an odd
    number of pairs (the last one alone) against the oracle, and against
    the same words run as one pair per call."""
    rng = np.random.default_rng(21)
    words = rng.integers(0, 2**32, 2 * 100001, dtype=np.uint64).astype(np.uint32)
    words[:64] = (np.arange(64, dtype=np.uint32) << 8)   # the FP64 tail in some quads
    z = _transform(words)
    err = ulp_error(z, O.normal_pairs64(words))
    assert float(err.max()) <= NORMAL_TOL_ULP, err.max()
    single = np.concatenate([_transform(words[2 * i:2 * i + 2]) for i in (0, 1, 2, 63, 64, 99999, 100000)])
    assert np.array_equal(single.view(np.uint32),
                          np.concatenate([z[2 * i:2 * i + 2] for i in (0, 1, 2, 63, 64, 99999, 100000)]).view(np.uint32))


def test_normal_random_pairs():
    rng = np.random.default_rng(11)
    words = rng.integers(0, 2**32, 1 << 25, dtype=np.uint64).astype(np.uint32)
    z = _transform(words)
    err = ulp_error(z, O.normal_pairs64(words))
    assert float(err.max()) <= NORMAL_TOL_ULP, err.max()


def test_uniform_transform_all_words_sampled():
    rng = np.random.default_rng(12)
    words = np.concatenate([np.arange(0, 1 << 20, dtype=np.uint32) << 12,
                            rng.integers(0, 2**32, 1 << 20, dtype=np.uint64).astype(np.uint32),
                            np.array([0xFFFFFFFF, 0, 0xFF, 0x100], dtype=np.uint32)])
    with Streams(1) as st:
        f = st.transform_uniform(torch.from_numpy(words.view(np.int32)).cuda()).cpu().numpy()
    assert np.array_equal(f, O.uniform_of(words))


# ---- the fused sum --------------------------------------------------------

def fused_order_sum(z, tpg, wpl):
    """The kernel's documented order: each lane sums its words in sequence,
    then a butterfly over lane offsets tpg/2 .. 1 (all in FP32)."""
    n = z.size
    rw = tpg * wpl
    nw = n + (n & 1)
    nr = -(-nw // rw)
    zz = np.zeros(nr * rw, dtype=np.float32)
    zz[:n] = z
    per_lane = zz.reshape(nr, tpg, wpl).transpose(1, 0, 2).reshape(tpg, nr * wpl)
    acc = np.add.accumulate(per_lane, axis=1, dtype=np.float32)[:, -1]
    off = tpg // 2
    while off >= 1:
        acc = (acc + acc[np.arange(tpg) ^ off]).astype(np.float32)
        off //= 2
    return acc[0]


@pytest.mark.parametrize("tpg,wpl", LAUNCHES)
def test_fused_normal_sum(tpg, wpl):
    seeds = W.seeds(40, start=77)
    n = 5001
    with Streams(40, seeds=seeds) as a, Streams(40, seeds=seeds) as b:
        a.set_launch("normal", tpg, wpl)
        b.set_launch("normal", tpg, wpl)
        z = a.normal(n).cpu().numpy()
        s = b.normal_sum(n).cpu().numpy()
        # both contexts advanced identically
        assert np.array_equal(u32np(a.u32(64)), u32np(b.u32(64)))
    for i in range(40):
        assert s[i] == fused_order_sum(z[i], tpg, wpl), i
    # against the FP64 oracle sum: each term within 4 ulp plus FP32 rounding
    # of the additions (n terms per lane at most, log2(tpg) butterfly steps)
    for i in range(0, 40, 7):
        z64 = O.Xorgens.param_set(0).seed(int(seeds[i])).normal64(n)
        absum = float(np.abs(z64).sum())
        m = n // tpg + int(math.log2(tpg)) + 2
        bound = absum * (NORMAL_TOL_ULP * 2.0**-23 + m * 2.0**-24 / (1 - m * 2.0**-24))
        assert abs(float(s[i]) - float(z64.sum())) <= bound


def test_fused_normal_sum_full_size_sampled():
    """The fused sum on the full normals workload (16384 streams x 2^16, the
    bench's launch): sampled streams against the FP64 oracle sum within the
    rounding bound of the FP32 summation order."""
    S, n = W.NORMALS["streams"], W.NORMALS["n"]
    seeds = W.seeds(S)
    with Streams(S, seeds=seeds) as st:
        st.autotune("normal", n)
        tpg, _ = st.get_launch("normal")
        s = st.normal_sum(n).cpu().numpy()
    m = n // tpg + int(math.log2(tpg)) + 2
    for i in (0, 1, 777, 8191, 12000, S - 1):
        z64 = O.Xorgens.param_set(0).seed(int(seeds[i])).normal64(n)
        bound = float(np.abs(z64).sum()) * (NORMAL_TOL_ULP * 2.0**-23 + m * 2.0**-24 / (1 - m * 2.0**-24))
        assert abs(float(s[i]) - float(z64.sum())) <= bound, i
    torch.cuda.empty_cache()


# ---- host output -----------------------------------------------------------

def test_host_output_matches_device_output():
    from paper_1108_0486_gb300 import _lib as L
    seeds = W.seeds(33)
    n = 10_000
    for kind, fn, dt in (("u32", L.xg_generate_u32, np.uint32),
                         ("uniform", L.xg_generate_uniform, np.float32),
                         ("normal", L.xg_generate_normal, np.float32)):
        with Streams(33, seeds=seeds) as a, Streams(33, seeds=seeds) as b:
            dev = host(kind, a.generate(kind, n))
            h = np.full((33, n), 0, dtype=dt)
            fn(b.ctx, 0, 33, n, h.ctypes.data, n)
            if kind == "u32":
                assert np.array_equal(h, dev)
            else:
                assert np.array_equal(h.view(np.uint32), dev.view(np.uint32))


# ---- full-size workloads (sampled) -------------------------------------------

def test_many_streams_full_size_sampled():
    """16384 streams x 2^16 u32 words (4 GiB), then as many uniforms, in the
    default launch; 48 sampled streams compared word for word."""
    cfg = W.MANY_STREAMS
    S, n = cfg["streams"], cfg["n"]
    seeds = W.seeds(S)
    rng = np.random.default_rng(5)
    pick = np.unique(np.concatenate([[0, 1, S - 1], rng.integers(0, S, 45)]))
    with Streams(S, seeds=seeds) as st:
        buf = torch.empty((S, n), dtype=torch.int32, device="cuda")
        st.u32(n, out=buf)
        got_u = u32np(buf[torch.from_numpy(pick).cuda()])
        fbuf = buf.view(torch.float32)
        st.uniform(n, out=fbuf)
        got_f = fbuf[torch.from_numpy(pick).cuda()].cpu().numpy()
        del buf, fbuf
    ref = O.streams(seeds[pick], 2 * n)
    assert np.array_equal(got_u, ref[:, :n])
    assert np.array_equal(got_f, O.uniform_of(ref[:, n:]).reshape(len(pick), n))


def test_normals_full_size_sampled():
    """2^30 normals over 16384 streams; 16 sampled streams within 4 ulp, and
    the whole output has mean ~0 and variance ~1."""
    cfg = W.NORMALS
    S, n = cfg["streams"], cfg["n"]
    seeds = W.seeds(S)
    pick = np.array([0, 5, 100, 2048, 4097, 8191, 8192, 10000, 12345, 16000, 16380, 16383,
                     3, 777, 9999, 15000])
    with Streams(S, seeds=seeds) as st:
        z = st.normal(n)
        mean = float(z.double().mean())
        var = float(z.double().var())
        got = z[torch.from_numpy(pick).cuda()].cpu().numpy()
        del z
    N = S * n
    assert abs(mean) < 6 / math.sqrt(N) and abs(var - 1) < 6 * math.sqrt(2 / N)
    ref = O.streams(seeds[pick], n, kind="normal")
    err = ulp_error(got, ref)
    assert float(err.max()) <= NORMAL_TOL_ULP


# ---- argument errors --------------------------------------------------------

def test_argument_errors():
    from paper_1108_0486_gb300 import XGError, _lib as L
    with Streams(10, seeds=W.seeds(10)) as st:
        out = torch.empty((10, 100), dtype=torch.int32, device="cuda")
        with pytest.raises(XGError) as e:
            L.xg_generate_u32(st.ctx, 5, 10, 100, out.data_ptr(), 100)  # range
        assert e.value.status == L.XG_EINVAL
        with pytest.raises(XGError):
            L.xg_generate_u32(st.ctx, 0, 10, 100, out.data_ptr(), 50)   # ld < n
        with pytest.raises(XGError):
            L.xg_generate_u32(st.ctx, 0, 10, 100, 0, 100)               # null
        with pytest.raises(XGError):
            st.set_launch("u32", 8, 8)                                    # unsupported
        words = torch.zeros(64, dtype=torch.int32, device="cuda")
        res = torch.empty(64, dtype=torch.float32, device="cuda")
        with pytest.raises(XGError) as e:
            L.xg_transform_normal(st.ctx, words.data_ptr(), 63, res.data_ptr())   # odd count
        assert e.value.status == L.XG_EINVAL
        with pytest.raises(XGError):
            L.xg_transform_normal(st.ctx, words.data_ptr() + 4, 32, res.data_ptr())  # not 8-byte aligned
        with pytest.raises(XGError):
            L.xg_transform_uniform(st.ctx, words.data_ptr() + 2, 16, res.data_ptr())  # not 4-byte aligned
        # zero-size calls are no-ops and do not advance the streams
        L.xg_generate_u32(st.ctx, 0, 10, 0, out.data_ptr(), 100)
        L.xg_generate_u32(st.ctx, 0, 0, 100, out.data_ptr(), 100)
        a = u32np(st.u32(10))
    ref = O.streams(W.seeds(10), 10)
    assert np.array_equal(a, ref)


def test_single_stream_beyond_2p32_words():
    """One call of 2^32 + 5 words on one stream (16 GiB; the counts pass
    32 bits): the head equals the oracle, the tail and a piece from the
    middle equal the oracle's jump to the same place (z^J modulo the minimal
    polynomial), and the position is the whole count."""
    n = (1 << 32) + 5
    with Streams(1, seeds=[77]) as st:
        out = torch.empty(n, dtype=torch.int32, device="cuda")
        st.u32(n, out=out.view(1, n))
        head = u32np(out[:1024])
        tail = u32np(out[n - 1024:])
        mid = u32np(out[(1 << 31) + 12345:(1 << 31) + 12345 + 256])
        pos = int(st.checkpoint()["pos"][0])
        del out
    assert pos == n
    assert np.array_equal(head, O.Xorgens.param_set(0).seed(77).u32(1024))
    assert np.array_equal(tail, O.u32_after_jump(77, n - 1024, 1024))
    assert np.array_equal(mid, O.u32_after_jump(77, (1 << 31) + 12345, 256))
    torch.cuda.empty_cache()


def test_four_million_streams():
    """2^22 streams in one context (3.3 GB of state): seeding and a short
    call on all of them; the last streams equal the oracle."""
    S = 1 << 22
    seeds = np.arange(1, S + 1, dtype=np.uint32)
    with Streams(S, seeds=seeds) as st:
        got = u32np(st.u32(40))
    for i in (0, S // 2 + 3, S - 1):
        assert np.array_equal(got[i], O.streams([int(seeds[i])], 40)[0]), i
    torch.cuda.empty_cache()
