"""64-bit-word generators on the GPU against the 64-bit oracle: raw u64
outputs and FP64 uniforms bit-exact, for every launch shape, ragged lengths,
split calls, state save/restore, host outputs and the bench's full size
(sampled rows)."""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def api():
    from paper_1108_0486_gb300 import api as A
    return A


def _u(t):
    return t.cpu().numpy().view(np.uint64)


def test_parameter_set_matches_oracle(api):
    params, omega = api.Streams64.params()
    assert params == O.PARAM_SET_W64
    assert omega == O.omega64()


@pytest.mark.parametrize("launch", [(4, 8), (8, 4), (16, 2), (32, 1)])
@pytest.mark.parametrize("n", [1, 31, 32, 33, 1000, 4099])
def test_u64_and_uniform_bit_exact(api, launch, n):
    seeds = list(range(100, 137))
    st = api.Streams64(len(seeds), seeds=seeds)
    st.set_launch("u64", *launch)
    st.set_launch("uniform", *launch)
    got = _u(st.u64(n))
    assert np.array_equal(got, O.streams64(seeds, n))
    # the streams continue: next n as uniforms equal the oracle's words n..2n
    gu = st.uniform(n).cpu().numpy()
    ref = O.streams64(seeds, 2 * n)[:, n:]
    assert np.array_equal(gu, O.uniform64_of(ref).reshape(gu.shape))


def test_weyl_off_is_the_raw_recurrence(api):
    seeds = [7, 8, 9]
    st = api.Streams64(3, weyl=False, seeds=seeds)
    got = _u(st.u64(777))
    for i, s in enumerate(seeds):
        g = O.Xorgens64(*O.PARAM_SET_W64, weyl=False).seed(s)
        assert np.array_equal(got[i], g.raw(777))


def test_split_calls_concatenate(api):
    seeds = list(range(1, 65))
    rng = np.random.default_rng(9)
    cuts = sorted(int(v) for v in rng.integers(1, 5000, 6))
    st = api.Streams64(64, seeds=seeds)
    pieces, prev = [], 0
    for k, c in enumerate(cuts + [5000]):
        if c == prev:
            continue
        kind = "u64" if k % 2 == 0 else "uniform"
        t = st.generate(kind, c - prev)
        pieces.append(("u64" if kind == "u64" else "f64", t.cpu().numpy()))
        prev = c
    ref = O.streams64(seeds, 5000)
    off = 0
    for kind, arr in pieces:
        w = arr.shape[1]
        if kind == "u64":
            assert np.array_equal(arr.view(np.uint64), ref[:, off:off + w])
        else:
            assert np.array_equal(arr, O.uniform64_of(ref[:, off:off + w]).reshape(arr.shape))
        off += w


def test_state_roundtrip_and_oracle_state(api):
    st = api.Streams64(4, seeds=[11, 12, 13, 14])
    st.u64(1234)
    ring, w = st.get_state(2)
    g = O.Xorgens64(*O.PARAM_SET_W64).seed(13)
    g.u64(1234)
    x, wo = g.get_state()
    assert np.array_equal(ring, x) and w == wo
    nxt = _u(st.u64(300, first=2, count=1))[0]
    st.set_state(2, ring, w)
    again = _u(st.u64(300, first=2, count=1))[0]
    assert np.array_equal(nxt, again) and np.array_equal(nxt, g.u64(300))


def test_host_output_matches_device(api):
    seeds = list(range(40, 48))
    a = api.Streams64(8, seeds=seeds)
    b = api.Streams64(8, seeds=seeds)
    dev = _u(a.u64(3001))
    host = np.zeros((8, 3001), dtype=np.uint64)
    from paper_1108_0486_gb300 import _lib as L
    L.xg_w64_generate_u64(b.ctx, 0, 8, 3001, host.ctypes.data, 3001)
    assert np.array_equal(dev, host)


def test_full_size_sampled_rows(api):
    """16384 streams x 2^16 words (the bench's 64-bit row), autotuned launch:
    whole rows of sampled streams bit-exact with the oracle."""
    n_streams, n = 16384, 1 << 16
    seeds = np.arange(1, n_streams + 1, dtype=np.uint32)
    st = api.Streams64(n_streams, seeds=seeds)
    st.autotune("uniform", n)
    out = st.uniform(n)
    for row in (0, 1, 4095, 8191, 16383):
        ref = O.uniform64_of(O.streams64([int(seeds[row])], n)[0])
        assert np.array_equal(out[row].cpu().numpy(), ref), row


def test_uniform_conversion_edge_words(api):
    """The conversion alone on words that take each path of the kernel's
    integer construction (leading one in either half, zero, extremes)."""
    edge = [0, 1, (1 << 11) - 1, 1 << 11, (1 << 11) + 1, (1 << 43) - 1, 1 << 43, (1 << 43) + 1,
            (1 << 44) - 1, 1 << 63, (1 << 64) - 1, 0x9E3779B97F4A7C15]
    edge += [1 << j for j in range(64)] + [(1 << j) - 1 for j in range(1, 65)]
    rng = np.random.default_rng(12)
    rand = rng.integers(0, 2**64 - 1, 100000, dtype=np.uint64, endpoint=True)
    small = rand >> rng.integers(0, 64, rand.size, dtype=np.uint64)
    words = np.concatenate([np.array(edge, dtype=np.uint64), rand, small])
    st = api.Streams64(1)
    got = st.transform_uniform(torch.from_numpy(words.view(np.int64)).cuda()).cpu().numpy()
    assert np.array_equal(got, O.uniform64_of(words))


def test_argument_errors(api):
    from paper_1108_0486_gb300 import _lib as L
    st = api.Streams64(4, seeds=[1, 2, 3, 4])
    with pytest.raises(L.XGError):
        st.set_launch("u64", 8, 8)
    with pytest.raises(L.XGError):
        st.u64(10, first=3, count=2)
    buf = torch.empty(16, dtype=torch.int32, device="cuda")
    with pytest.raises(L.XGError):   # 4-byte aligned, not 8: refused on the host
        L.xg_w64_generate_u64(st.ctx, 0, 1, 4, buf.data_ptr() + 4, 4)
    with pytest.raises(L.XGError) as e:
        st.jump(5, first=2, count=3)   # streams out of range
    assert e.value.status == L.XG_EINVAL
    # a zero jump and an empty range are no-ops
    st.jump(0)
    st.jump(12345, first=4, count=0)
    assert np.array_equal(_u(st.u64(64)), O.streams64([1, 2, 3, 4], 64))


# ---- jump-ahead -------------------------------------------------------------

@pytest.mark.parametrize("J", [1, 31, 32, 33, 64, 1000, 4099, 123457])
def test_jump_equals_stepping(api, J):
    """Jumping J words lands where generating J words does (the oracle
    steps one word at a time), from a position with words pending."""
    seeds = list(range(300, 337))
    st = api.Streams64(len(seeds), seeds=seeds)
    st.u64(5)
    st.jump(J)
    got = _u(st.u64(256))
    ref = O.streams64(seeds, 5 + J + 256)[:, 5 + J:]
    assert np.array_equal(got, ref)


def test_jump_weyl_off_and_subrange(api):
    """With the Weyl generator off the jump is the raw recurrence's; only
    the streams named move."""
    seeds = [21, 22, 23, 24, 25]
    st = api.Streams64(5, weyl=False, seeds=seeds)
    st.jump(777, first=1, count=3)
    got = _u(st.u64(100))
    for i, s in enumerate(seeds):
        g = O.Xorgens64(*O.PARAM_SET_W64, weyl=False).seed(s)
        if 1 <= i <= 3:
            g.raw(777)
        assert np.array_equal(got[i], g.raw(100)), i


def test_jump_far_against_the_oracle(api):
    """64-bit jumps far past stepping distance against the oracle's jump by
    z^J modulo the minimal polynomial, Weyl generator on and off."""
    seeds = [31, 32]
    for J in ((1 << 32) + 5, (1 << 40) + 12345, 1 << 63):
        for weyl in (True, False):
            st = api.Streams64(2, weyl=weyl, seeds=seeds)
            st.jump(J)
            got = _u(st.u64(48))
            for i, sd in enumerate(seeds):
                assert np.array_equal(got[i], O.u64_after_jump(sd, J, 48, weyl=weyl)), (J, weyl, i)


def test_jump_tensor_cores_against_the_table_kernel_and_the_oracle(api, monkeypatch):
    """1500 64-bit streams: the tensor-core path equals the table kernel and
    the oracle's jump."""
    J = (1 << 50) + 777
    seeds = list(range(900, 2400))
    out = []
    for tc in ("1", "0"):
        monkeypatch.setenv("XG_JUMP_TENSOR_CORES", tc)
        st = api.Streams64(len(seeds), seeds=seeds)
        st.jump(J)
        out.append(_u(st.u64(24)))
    assert np.array_equal(out[0], out[1])
    for i in (0, 1023, 1499):
        assert np.array_equal(out[0][i], O.u64_after_jump(seeds[i], J, 24)), i


def test_jump_many_streams_multiplies_the_powers_first(api, monkeypatch):
    """4200 64-bit streams and five set bits: the product of the powers
    applied once, on both GF(2) paths, equal to the oracle's jump."""
    J = (1 << 40) + (1 << 33) + 0b10101
    seeds = list(range(5, 4205))
    for tc in ("1", "0"):
        monkeypatch.setenv("XG_JUMP_TENSOR_CORES", tc)
        st = api.Streams64(len(seeds), seeds=seeds)
        st.jump(J)
        got = _u(st.u64(16))
        for i in (0, 4100, 4199):
            assert np.array_equal(got[i], O.u64_after_jump(seeds[i], J, 16)), (tc, i)


def test_jump_composes_at_large_distances(api):
    """M^a M^b = M^(a+b) for distances up to 2^63, and the Weyl word
    advances by the distance times omega mod 2^64: jumping a then b gives
    the outputs of jumping a + b at once."""
    seeds = list(range(1, 17))
    for a, b in ((1 << 40, (1 << 40) + 12345), ((1 << 63) - 1, 1), (3 << 61, 987654321)):
        x = api.Streams64(16, seeds=seeds)
        y = api.Streams64(16, seeds=seeds)
        x.jump(a)
        x.jump(b)
        y.jump(a + b)
        assert np.array_equal(_u(x.u64(300)), _u(y.u64(300)))


@pytest.mark.parametrize("q,count", [(5, 37), (0, 9), (12, 20)])
def test_substreams_are_consecutive_blocks(api, q, count):
    """Stream i of seed_substreams starts at word i 2^q of the one sequence
    of the seed (the oracle run serially)."""
    seed = 0x0BADF00D
    st = api.Streams64(count + 2, seeds=list(range(1, count + 3)))
    st.seed_substreams(seed, q, first=1, count=count)
    got = _u(st.u64(1 << q, first=1, count=count))
    ref = O.streams64([seed], count << q)[0]
    assert np.array_equal(got.reshape(-1), ref)
    # the neighbours keep their own seeds
    assert np.array_equal(_u(st.u64(3, first=0, count=1))[0], O.streams64([1], 3)[0])


def test_substreams_far_apart_equal_jumps(api):
    seed = 4242
    a = api.Streams64(4)
    b = api.Streams64(4, seeds=[seed] * 4)
    a.seed_substreams(seed, 37)
    for i in range(1, 4):
        b.jump(i << 37, first=i, count=1)
    got = _u(a.u64(200))
    assert np.array_equal(got, _u(b.u64(200)))
    for i in (1, 3):
        assert np.array_equal(got[i][:40], O.u64_after_jump(seed, i << 37, 40)), i
    from paper_1108_0486_gb300 import _lib as L
    with pytest.raises(L.XGError):
        a.seed_substreams(seed, 63, count=3)


@pytest.mark.parametrize("split", [0, 1 << 10])
def test_long_calls_on_few_streams_are_cut_exactly(api, split):
    """Calls of 2^18 words and more on few streams run as jump-ahead pieces;
    outputs and the states left behind equal the serial stream's."""
    seeds = [5, 6, 7]
    n = (1 << 18) + 12345
    st = api.Streams64(3, seeds=seeds)
    st.set_split(split)
    out = torch.empty((3, n + 3), dtype=torch.int64, device="cuda")   # ld > n
    st.u64(n, out=out[:, :n], ld=n + 3)
    f = st.uniform(n)
    tail = _u(st.u64(1000))
    ref = O.streams64(seeds, 2 * n + 1000)
    assert np.array_equal(_u(out[:, :n]), ref[:, :n])
    assert np.array_equal(f.cpu().numpy(), O.uniform64_of(ref[:, n:2 * n]).reshape(3, n))
    assert np.array_equal(tail, ref[:, 2 * n:])


def test_long_single_stream_cut_and_uncut_agree(api):
    a = api.Streams64(1, seeds=[77])
    b = api.Streams64(1, seeds=[77])
    b.set_split(1)
    n = 1 << 20
    assert np.array_equal(_u(a.u64(n)), _u(b.u64(n)))
    assert np.array_equal(_u(a.u64(333)), _u(b.u64(333)))
    from paper_1108_0486_gb300 import _lib as L
    with pytest.raises(L.XGError):
        a.set_split(100)   # not a power of two
