"""Batched persistent kernel and request server against the oracle and
against the plain one-launch-per-call path."""
import threading
import time

import numpy as np
import pytest

import oracle as O
from paper_1108_0486_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

KINDS = ["u32", "uniform", "normal"]
TOL = 4.0


@pytest.fixture(scope="module", autouse=True)
def _device():
    torch.cuda.set_device(0)
    yield
    torch.cuda.synchronize()


def Streams(*a, **k):
    from paper_1108_0486_gb300 import Streams as S
    return S(*a, **k)


def nwords(kind, n):
    return n + (n & 1) if kind == "normal" else n


def oracle_call(words, kind, n):
    if kind == "u32":
        return words[:n]
    if kind == "uniform":
        return O.uniform_of(words[:n])
    return O.normal_pairs64(words[:nwords(kind, n)])[:n]


def check(kind, got_tensor, ref):
    if kind == "u32":
        assert np.array_equal(got_tensor.cpu().numpy().view(np.uint32), ref)
    elif kind == "uniform":
        assert np.array_equal(got_tensor.cpu().numpy(), ref)
    else:
        z = got_tensor.cpu().numpy().astype(np.float64)
        z32 = ref.astype(np.float32)
        err = np.abs(z - ref) / np.spacing(np.abs(z32)).astype(np.float64)
        assert float(err.max()) <= TOL, err.max()


def alloc(kind, n):
    return torch.empty(max(n, 1), dtype=torch.int32 if kind == "u32" else torch.float32, device="cuda")


def random_items(rng, n_streams, n_items, max_len=40000):
    items = []
    for _ in range(n_items):
        s = int(rng.integers(0, n_streams))
        k = KINDS[int(rng.integers(0, 3))]
        n = int(np.exp(rng.uniform(0, np.log(max_len))))
        items.append((s, k, n))
    return items


def oracle_per_item(seeds, items, ps=0):
    """The oracle outputs of each item, streams advancing in item order."""
    total = {}
    for s, k, n in items:
        total[s] = total.get(s, 0) + nwords(k, n)
    words = {s: O.Xorgens.param_set(ps).seed(int(seeds[s])).u32(t) for s, t in total.items()}
    off = {s: 0 for s in total}
    refs = []
    for s, k, n in items:
        w = words[s][off[s]:off[s] + nwords(k, n)]
        off[s] += nwords(k, n)
        refs.append(oracle_call(w, k, n))
    return refs


# ----------------------------------------------------------------- batch

@pytest.mark.parametrize("ps", [0, 1])
def test_batch_mixed_types_uneven_lengths_and_chains(ps):
    rng = np.random.default_rng(21 + ps)
    seeds = W.seeds(150, start=500)
    items = random_items(rng, 150, 400)  # many streams appear several times
    outs = [alloc(k, n) for _, k, n in items]
    with Streams(150, param_set=ps, seeds=seeds) as st:
        st.batch([(s, k, n, o) for (s, k, n), o in zip(items, outs)])
        torch.cuda.synchronize()
    for (s, k, n), o, ref in zip(items, outs, oracle_per_item(seeds, items, ps)):
        check(k, o[:n], ref)


SHAPES = [(32, 2), (16, 4), (8, 4)]


@pytest.mark.parametrize("ps", [0, 1])
@pytest.mark.parametrize("shape", SHAPES)
def test_batch_shapes_against_the_oracle(ps, shape, monkeypatch):
    """u32 and uniform calls alone on their stream run 1, 2 or 4 streams per
    warp (normals and chains of several calls stay one per warp), with
    ragged lengths, unaligned outputs (which must not be grouped) and calls
    cut into pieces: every output against the oracle.  The group length
    limit is lifted (a batch this small would otherwise group nothing)."""
    monkeypatch.setenv("XG_BATCH_GROUP_MAX_WORDS", str(1 << 40))
    rng = np.random.default_rng(70 + ps)
    S = 120
    seeds = W.seeds(S, start=3000)
    items = random_items(rng, S, 160, max_len=20000)
    big = torch.zeros(1 << 22, dtype=torch.int32, device="cuda")
    outs, off = [], 0
    for j, (_, k, n) in enumerate(items):
        off += 1 if j % 7 == 3 else 0          # some outputs 4-byte aligned only
        o = big[off:off + max(n, 1)]
        outs.append(o if k == "u32" else o.view(torch.float32))
        off = (off + max(n, 1) + 3) // 4 * 4 + 4
    with Streams(S, param_set=ps, seeds=seeds) as st:
        for k in ("u32", "uniform"):
            st.set_batch_shape(k, *shape)
            assert st.get_batch_shape(k) == shape
        st.set_batch_split(2048)
        st.batch([(s, k, n, o) for (s, k, n), o in zip(items, outs)])
        torch.cuda.synchronize()
        after = st.u32(40).cpu().numpy().view(np.uint32)
    refs = oracle_per_item(seeds, items, ps)
    for (s, k, n), o, ref in zip(items, outs, refs):
        if n:
            check(k, o[:n], ref)
    # every stream ends where the oracle does
    total = {}
    for s_, k, n in items:
        total[s_] = total.get(s_, 0) + nwords(k, n)
    for s_ in (0, 5, S - 1):
        ref = O.Xorgens.param_set(ps).seed(int(seeds[s_])).u32(total.get(s_, 0) + 40)[-40:]
        assert np.array_equal(after[s_], ref)


def test_batch_shape_argument_errors():
    from paper_1108_0486_gb300 import XGError, _lib as L
    with Streams(4, seeds=[1, 2, 3, 4]) as st:
        with pytest.raises(XGError):
            st.set_batch_shape("u32", 4, 8)
        with pytest.raises(XGError):
            st.set_batch_shape("normal", 8, 4)
        st.set_batch_shape("normal", 32, 2)
        assert st.get_batch_shape("normal") == (32, 2)


def test_autotune_batch_keeps_streams_and_picks_supported_shapes():
    rng = np.random.default_rng(8)
    S = 256
    seeds = W.seeds(S)
    items = [(s, KINDS[int(rng.integers(0, 3))], int(rng.integers(1000, 60000))) for s in range(S)]
    outs = [alloc(k, n) for _, k, n in items]
    with Streams(S, seeds=seeds) as st:
        res = st.autotune_batch([(s, k, n, o) for (s, k, n), o in zip(items, outs)])
        for k in ("u32", "uniform"):
            assert tuple(res[k][:2]) in SHAPES and res[k][2] > 0
            assert st.get_batch_shape(k) == tuple(res[k][:2])
        assert tuple(res["normal"][:2]) == (32, 2)
        # the streams did not advance: a batch now gives the oracle's first words
        st.batch([(s, k, n, o) for (s, k, n), o in zip(items, outs)])
        torch.cuda.synchronize()
    refs = oracle_per_item(seeds, items)
    for j in (0, 1, 100, 255):
        s, k, n = items[j]
        check(k, outs[j][:n], refs[j])


def test_batch_equals_plain_calls_bitwise():
    rng = np.random.default_rng(5)
    seeds = W.seeds(64)
    items = random_items(rng, 64, 200)
    outs = [alloc(k, n) for _, k, n in items]
    with Streams(64, seeds=seeds) as a, Streams(64, seeds=seeds) as b:
        a.batch([(s, k, n, o) for (s, k, n), o in zip(items, outs)])
        for (s, k, n), o in zip(items, outs):
            ref = b.generate(k, n, first=s, count=1)[0, :n]
            assert torch.equal(o[:n], ref)
        # both contexts end in the same state
        assert torch.equal(a.u32(100), b.u32(100))


def test_batch_unaligned_outputs_and_zero_counts():
    seeds = W.seeds(10)
    items = [(0, "u32", 1001), (1, "uniform", 77), (2, "normal", 33), (3, "u32", 0), (0, "u32", 5)]
    big = torch.zeros(4096, dtype=torch.int32, device="cuda")
    outs = [big[1:1002], big[1100:1177].view(torch.float32), big[1201:1234].view(torch.float32),
            None, big[3001:3006]]
    with Streams(10, seeds=seeds) as st:
        st.batch([(s, k, n, o) for (s, k, n), o in zip(items, outs)])
        torch.cuda.synchronize()
    refs = oracle_per_item(seeds, items)
    for (s, k, n), o, ref in zip(items, outs, refs):
        if n:
            check(k, o[:n], ref)


def test_batch_uneven_workload_sampled():
    """4096 streams, one item each, lengths log-uniform in [2^10, 2^24],
    mixed types (about 29 GB of outputs), in one launch; sampled items
    (the longest, the shortest and a few others) against the oracle."""
    items = W.batched_uneven()
    seeds = W.seeds(len(items))
    outs = [alloc(KINDS[it.kind], it.count) for it in items]
    with Streams(len(items), seeds=seeds) as st:
        st.batch([(it.stream, it.kind, it.count, o) for it, o in zip(items, outs)])
        torch.cuda.synchronize()
    counts = np.array([it.count for it in items])
    pick = list(np.argsort(counts)[[0, 1, len(items) // 2, -2, -1]]) + [7, 1234, 4095]
    for i in pick:
        it = items[i]
        k = KINDS[it.kind]
        words = O.Xorgens.param_set(0).seed(int(seeds[it.stream])).u32(nwords(k, it.count))
        check(k, outs[i][:it.count], oracle_call(words, k, it.count))


# ---------------------------------------------------------------- server

def test_server_results_same_alone_and_in_the_mix():
    """Requests from 4 client threads, arriving while others run; each
    result equals the same request run alone through the plain path."""
    rng = np.random.default_rng(9)
    S = 300
    seeds = W.seeds(S, start=77)
    reqs = random_items(rng, S, 600, max_len=200000)
    outs = [alloc(k, n) for _, k, n in reqs]
    tickets = [None] * len(reqs)
    with Streams(S, seeds=seeds) as st:
        srv = st.serve(lanes=8, max_batch=64)

        def client(idx):
            for i in idx:
                s, k, n = reqs[i]
                tickets[i] = srv.submit(s, k, n, out=outs[i])

        parts = np.array_split(np.arange(len(reqs)), 4)
        th = [threading.Thread(target=client, args=(p,)) for p in parts]
        for t in th:
            t.start()
        for t in th:
            t.join()
        for t in tickets:
            srv.wait(t, 60000)
        stats = srv.stats()
        for t in tickets:
            srv.release(t)
        srv.stop()
    assert stats["completed"] == len(reqs) and stats["batches"] >= 2
    # per stream, submission order is ticket order
    order = np.argsort(np.array(tickets))
    with Streams(S, seeds=seeds) as alone:
        for i in order:
            s, k, n = reqs[i]
            ref = alone.generate(k, n, first=s, count=1)[0, :n]
            assert torch.equal(outs[i][:n], ref), (i, s, k, n)
    # and against the oracle for a sample
    ordered = [reqs[i] for i in order]
    refs = oracle_per_item(seeds, ordered)
    for j in range(0, len(ordered), 37):
        s, k, n = ordered[j]
        check(k, outs[order[j]][:n], refs[j])


def test_server_pool_buffers_and_release():
    seeds = W.seeds(20)
    reqs = [(i % 20, KINDS[i % 3], 1000 + 37 * i) for i in range(60)]
    with Streams(20, seeds=seeds) as st:
        srv = st.serve(mem_cap_bytes=64 << 20)
        tickets = [srv.submit(s, k, n) for s, k, n in reqs]
        results = [srv.result(t, k, n).clone() for t, (_, k, n) in zip(tickets, reqs)]
        assert srv.stats()["outstanding_bytes"] == sum(4 * n for _, _, n in reqs)
        for t in tickets:
            srv.release(t)
        assert srv.stats()["outstanding_bytes"] == 0
        srv.stop()
    refs = oracle_per_item(seeds, reqs)
    for (s, k, n), r, ref in zip(reqs, results, refs):
        check(k, r[:n], ref)


def test_server_submit_and_collect_on_two_threads():
    """One thread submits in bulk under a small memory cap (resubmitting the
    refused tail), another drains completions with xg_collect, copies each
    pooled result and releases it, as the header allows; every result
    equals the same request run alone."""
    from paper_1108_0486_gb300 import _lib as L
    from paper_1108_0486_gb300.api import device_view
    rng = np.random.default_rng(21)
    S = 64
    seeds = W.seeds(S, start=5)
    reqs = random_items(rng, S, 400, max_len=60000)
    got = {}
    ticket_of = [None] * len(reqs)
    done_submitting = threading.Event()
    refused = threading.Event()
    errors = []
    with Streams(S, seeds=seeds) as st:
        srv = st.serve(mem_cap_bytes=2 << 20, lanes=4, max_batch=32)
        req_of = {}
        book = threading.Lock()

        def submitter():
            try:
                i = 0
                while i < len(reqs):
                    # xg_submit_many admits a prefix of the chunk; the cap
                    # refused the rest, which goes again
                    with book:   # tickets are recorded before any can be collected
                        ts = srv.submit_many(reqs[i:i + 16])
                        for j, t in enumerate(ts):
                            req_of[t] = i + j
                            ticket_of[i + j] = t
                    if len(ts) < len(reqs[i:i + 16]):
                        refused.set()
                    if not ts:
                        time.sleep(0.0002)
                    i += len(ts)
            except Exception as e:  # noqa: BLE001 - reported by the main thread
                errors.append(e)
            finally:
                done_submitting.set()

        def collector():
            try:
                # start draining once the cap has pushed back (or all is in)
                while not (refused.is_set() or done_submitting.is_set()):
                    time.sleep(0.0005)
                while not (done_submitting.is_set() and len(got) == sum(t is not None for t in ticket_of)):
                    with book:
                        comps = srv.collect(64, release=False)
                    if not comps:
                        time.sleep(0.0001)
                    for (t, _, _, _, status, ptr) in comps:
                        assert status == L.XG_OK
                        s_, k, n = reqs[req_of[t]]
                        dt = torch.int32 if k == "u32" else torch.float32
                        got[t] = device_view(ptr, n, dt).clone()
                        torch.cuda.synchronize()
                        srv.release(t)
            except Exception as e:  # noqa: BLE001
                errors.append(e)

        th = [threading.Thread(target=submitter), threading.Thread(target=collector)]
        for t in th:
            t.start()
        for t in th:
            t.join(300)
        stats = srv.stats()
        srv.stop()
    assert not errors, errors
    assert len(got) == len(reqs) and stats["outstanding_bytes"] == 0
    assert stats["refused"] > 0          # the cap did push back
    order = np.argsort(np.array(ticket_of, dtype=np.uint64))
    with Streams(S, seeds=seeds) as alone:
        for i in order:
            s_, k, n = reqs[i]
            ref = alone.generate(k, n, first=s_, count=1)[0, :n]
            assert torch.equal(got[ticket_of[i]], ref), (i, s_, k, n)


def test_server_admission_by_memory():
    from paper_1108_0486_gb300 import XGError, _lib as L
    with Streams(8, seeds=W.seeds(8)) as st:
        srv = st.serve(mem_cap_bytes=1 << 20)  # 1 MiB: 262144 outputs
        t1 = srv.submit(0, "u32", 200000)
        with pytest.raises(XGError) as e:
            srv.submit(1, "u32", 100000)
        assert e.value.status == L.XG_EAGAIN
        # larger than the cap itself: never admissible, so not a retry case
        with pytest.raises(XGError) as e:
            srv.submit(2, "u32", 262145)
        assert e.value.status == L.XG_EINVAL and "cap" in str(e.value)
        srv.wait(t1)
        srv.release(t1)
        t2 = srv.submit(1, "u32", 100000)
        srv.wait(t2)
        assert srv.stats()["refused"] == 1
        srv.release(t2)
        srv.stop()


def test_server_owns_the_context_while_running():
    from paper_1108_0486_gb300 import XGError, _lib as L
    with Streams(4, seeds=W.seeds(4)) as st:
        srv = st.serve()
        with pytest.raises(XGError):
            st.u32(10)
        with pytest.raises(XGError) as e:
            srv.poll(123456)
        assert e.value.status == L.XG_ENOTFOUND
        srv.stop()
        st.u32(10)  # plain calls work again


# -------------------------------------------------------------- autotuner

@pytest.mark.parametrize("kind", KINDS)
def test_autotune_picks_a_supported_launch_and_leaves_streams_in_place(kind):
    from paper_1108_0486_gb300.api import LAUNCHES
    seeds = W.seeds(2000, start=3)
    with Streams(2000, seeds=seeds) as st:
        st.u32(77)  # a position that is not a multiple of the round width
        best = st.autotune(kind, 4096)
        assert (best["tpg"], best["wpl"]) in LAUNCHES and best["block"] in (32, 64, 128, 256)
        assert st.get_launch(kind) == (best["tpg"], best["wpl"])
        got = st.generate(kind, 3001)
    ref = O.streams(seeds, 77 + nwords(kind, 3001))[:, 77:]
    for i in (0, 999, 1999):
        check(kind, got[i, :3001], oracle_call(ref[i], kind, 3001))


# ------------------------------------------------------------ jump-ahead

@pytest.mark.parametrize("ps", [0, 1])
def test_jump_matches_stepping(ps):
    seeds = W.seeds(6, start=40)
    for J in (1, 63, 64, 4095, 4096, 65537, 1_000_003, (1 << 22) + 3):
        with Streams(6, param_set=ps, seeds=seeds) as st:
            st.u32(7)          # not at a round boundary
            st.jump(J)
            got = st.u32(500).cpu().numpy().view(np.uint32)
        for i in (0, 5):
            ref = O.Xorgens.param_set(ps).seed(int(seeds[i])).u32(7 + J + 500)[7 + J:]
            assert np.array_equal(got[i], ref), (ps, J, i)


@pytest.mark.parametrize("ps", [0, 1])
def test_jump_far_against_the_oracle(ps):
    """Jumps far past any stepping distance against the oracle's own jump,
    which takes z^J modulo the minimal polynomial of the Sec. 2 recurrence
    (a different route from the GPU's powers of the transition matrix):
    Weyl generator on and off, all 32 bits of every word."""
    seeds = W.seeds(3, start=500)
    for J in ((1 << 32) + 5, (1 << 40) + 12345, 1 << 63, (1 << 64) - 1):
        for weyl in (True, False):
            with Streams(3, param_set=ps, seeds=seeds, weyl=weyl) as st:
                st.jump(J)
                got = st.u32(64).cpu().numpy().view(np.uint32)
            for i in (0, 2):
                ref = O.u32_after_jump(int(seeds[i]), J, 64, param_set=ps, weyl=weyl)
                assert np.array_equal(got[i], ref), (ps, J, weyl, i)


def test_jump_from_a_pending_position_against_the_oracle():
    """A jump from a position inside a round (words pending), then a cut
    call across a 2^21-word piece boundary, all against the oracle."""
    seeds = W.seeds(2, start=900)
    J = (1 << 45) + 77
    with Streams(2, seeds=seeds) as st:
        st.u32(13)
        st.jump(J)
        got = st.u32((1 << 21) + 300).cpu().numpy().view(np.uint32)
    for i in range(2):
        ref = O.u32_after_jump(int(seeds[i]), 13 + J, 64)
        assert np.array_equal(got[i][:64], ref)
        ref = O.u32_after_jump(int(seeds[i]), 13 + J + (1 << 21) - 32, 332)
        assert np.array_equal(got[i][(1 << 21) - 32:], ref)


# ---- the tensor-core path of the jump-ahead (tcgen05, FP8 0/1 operands) ----

def _jump_states(S, J, ps=0, monkeypatch=None, tc=True, seeds=None):
    if monkeypatch is not None:
        monkeypatch.setenv("XG_JUMP_TENSOR_CORES", "1" if tc else "0")
    seeds = W.seeds(S, start=7000) if seeds is None else seeds
    with Streams(S, param_set=ps, seeds=seeds) as st:
        st.u32(5)                      # words pending: the jump starts inside a round
        st.jump(J)
        ck = st.checkpoint()
        words = st.u32(48).cpu().numpy().view(np.uint32)
    return ck, words, seeds


@pytest.mark.parametrize("ps", [0, 1])
def test_jump_tensor_cores_against_the_table_kernel_and_the_oracle(ps, monkeypatch):
    """2304 streams (nine tiles of 256 states, the last one partly padding
    after 2048 + 256): the tensor-core application equals the table kernel
    bit for bit on every stream, and sampled streams equal the oracle's
    jump (z^J modulo the minimal polynomial)."""
    J = (1 << 40) + 12345
    S = 2304 - 100
    a, wa, seeds = _jump_states(S, J, ps, monkeypatch, tc=True)
    b, wb, _ = _jump_states(S, J, ps, monkeypatch, tc=False)
    assert np.array_equal(a["rings"], b["rings"]) and np.array_equal(a["weyl"], b["weyl"])
    assert np.array_equal(wa, wb)
    for i in (0, 255, 256, 1777, S - 1):
        assert np.array_equal(wa[i], O.u32_after_jump(int(seeds[i]), 5 + J, 48, param_set=ps)), i


@pytest.mark.parametrize("tc", [True, False])
def test_jump_many_streams_multiplies_the_powers_first(tc, monkeypatch):
    """More than 4096 streams and several set bits: the powers are
    multiplied first (b - 1 products of 4096-column matrices) and the
    product applied once; equal to the oracle's jump, on the tensor cores
    and on the table kernel."""
    J = (1 << 44) + (1 << 30) + 777
    S = 4500
    a, wa, seeds = _jump_states(S, J, 0, monkeypatch, tc=tc)
    for i in (0, 2222, 4096, S - 1):
        assert np.array_equal(wa[i], O.u32_after_jump(int(seeds[i]), 5 + J, 48)), (tc, i)
    assert np.array_equal(a["pos"], np.full(S, 5 + J, dtype=np.uint64))


def test_jump_tensor_cores_small_and_partial_tiles(monkeypatch):
    """With the threshold lowered, 1, 37 and 300 states run on the tensor
    cores (one partly filled tile, and a second one nearly empty)."""
    monkeypatch.setenv("XG_GF2_TC_MIN_STATES", "1")
    for S in (1, 37, 300):
        a, wa, seeds = _jump_states(S, (1 << 63) + 99, 0, monkeypatch, tc=True)
        b, wb, _ = _jump_states(S, (1 << 63) + 99, 0, monkeypatch, tc=False)
        assert np.array_equal(a["rings"], b["rings"]), S
        assert np.array_equal(wa[S - 1], O.u32_after_jump(int(seeds[S - 1]), 5 + (1 << 63) + 99, 48)), S


def test_substreams_and_cut_calls_on_the_tensor_cores(monkeypatch):
    """Doubling steps of 1024 and more pairs: 3000 substreams of one
    sequence, and one call of 2^20 words cut into 16384 pieces of 64 words
    (its prologue's last steps apply a power to 1024 .. 8192 pieces)."""
    monkeypatch.setenv("XG_JUMP_TENSOR_CORES", "1")
    seed = 0xC0FFEE
    with Streams(3000) as st:
        st.seed_substreams(seed, 20)
        got = st.u32(32).cpu().numpy().view(np.uint32)
    for i in (1, 1024, 2047, 2999):
        assert np.array_equal(got[i], O.u32_after_jump(seed, i << 20, 32)), i
    with Streams(2, seeds=[11, 12]) as st:
        st.set_batch_split(64)
        n = 1 << 20
        out = torch.empty(n, dtype=torch.int32, device="cuda")
        st.batch([(0, "u32", n, out)])
        torch.cuda.synchronize()
        tail = st.u32(16, first=0, count=1).cpu().numpy().view(np.uint32)[0]
    ref = O.Xorgens.param_set(0).seed(11).u32(n + 16)
    assert np.array_equal(out.cpu().numpy().view(np.uint32), ref[:n])
    assert np.array_equal(tail, ref[n:])


def test_jump_composes_for_large_distances():
    seeds = W.seeds(4)
    a, b = (1 << 40) + 12345, (1 << 37) + 999
    with Streams(4, seeds=seeds) as x, Streams(4, seeds=seeds) as y:
        x.jump(a)
        x.jump(b)
        y.jump(a + b)
        assert torch.equal(x.u32(300), y.u32(300))
        x.jump(1 << 63)
        y.jump(1 << 62)
        y.jump(1 << 62)
        assert torch.equal(x.normal(301), y.normal(301))


@pytest.mark.parametrize("ps,q,count", [(0, 6, 37), (1, 6, 37), (0, 10, 100), (0, 0, 9)])
def test_substreams_are_consecutive_blocks_of_one_sequence(ps, q, count):
    """Stream i of seed_substreams starts at word i 2^q of the one seeded
    sequence (the oracle run serially): with 2^q-word blocks, the streams'
    outputs laid end to end are that sequence; positions are i 2^q."""
    seed = 0x12345678
    with Streams(count + 3, param_set=ps, seeds=W.seeds(count + 3)) as st:
        st.seed_substreams(seed, q, first=2, count=count)
        pos = st.checkpoint(first=2, count=count)["pos"]
        got = st.u32(1 << q, first=2, count=count).cpu().numpy().view(np.uint32)
        other = st.u32(5, first=0, count=2).cpu().numpy().view(np.uint32)
    ref = O.Xorgens.param_set(ps).seed(seed).u32(count << q)
    assert np.array_equal(got.reshape(-1), ref)
    assert np.array_equal(pos, np.arange(count, dtype=np.uint64) << np.uint64(q))
    # the streams outside the range keep their own seeds
    assert np.array_equal(other, O.streams(W.seeds(count + 3)[:2], 5, param_set=ps))


@pytest.mark.parametrize("q", [30, 40])
def test_substreams_far_apart_equal_jumps(q):
    """At 2^q-word spacing stream i equals the seeded stream jumped by i 2^q,
    Weyl word included (2^30 omega is not 0 mod 2^32; normals use every bit)."""
    seed = 99
    with Streams(5) as a, Streams(5, seeds=[seed] * 5) as b:
        a.seed_substreams(seed, q)
        for i in range(1, 5):
            b.jump(i << q, first=i, count=1)
        assert np.array_equal(a.checkpoint()["weyl"], b.checkpoint()["weyl"])
        assert torch.equal(a.normal(333), b.normal(333))
        got = a.u32(64).cpu().numpy().view(np.uint32)
    # and against the oracle's jump: stream i is the sequence from word i 2^q
    for i in (1, 4):
        assert np.array_equal(got[i], O.u32_after_jump(seed, (i << q) + 334, 64)), i


def test_substreams_weyl_off_and_errors():
    from paper_1108_0486_gb300 import XGError, _lib as L
    with Streams(8, weyl=False) as st:
        st.seed_substreams(5, 7)
        got = st.u32(128).cpu().numpy().view(np.uint32)
        with pytest.raises(XGError) as e:      # 2 * 2^63 does not fit in 64 bits
            st.seed_substreams(5, 63, count=3)
        assert e.value.status == L.XG_EINVAL
        with pytest.raises(XGError):
            st.seed_substreams(5, 4, first=6, count=3)   # out of range
        st.seed_substreams(5, 63, count=2)           # 1 * 2^63 fits
    ref = O.Xorgens.param_set(0, weyl=False).seed(5).u32(8 * 128)
    assert np.array_equal(got.reshape(-1), ref)


@pytest.mark.parametrize("piece", [64, 1024])
def test_batch_cut_into_pieces_equals_uncut(piece):
    rng = np.random.default_rng(31)
    seeds = W.seeds(90)
    items = [(i, KINDS[i % 3], int(rng.integers(1, 60000))) for i in range(90)]
    items += [(90 // 2, "u32", 5000), (3, "normal", 777)]  # streams with two items stay whole
    with Streams(90, seeds=seeds) as a, Streams(90, seeds=seeds) as b:
        a.set_batch_split(piece)
        b.set_batch_split(1)
        oa = [alloc(k, n) for _, k, n in items]
        ob = [alloc(k, n) for _, k, n in items]
        a.batch([(s, k, n, o) for (s, k, n), o in zip(items, oa)])
        b.batch([(s, k, n, o) for (s, k, n), o in zip(items, ob)])
        for (s, k, n), x, y in zip(items, oa, ob):
            assert torch.equal(x[:n], y[:n]), (s, k, n)
        assert torch.equal(a.u32(129), b.u32(129))  # same state afterwards
    refs = oracle_per_item(seeds, items)
    for j in (0, 1, 2, 50, 89, 90, 91):
        s, k, n = items[j]
        check(k, oa[j][:n], refs[j])


def test_server_with_cut_requests():
    rng = np.random.default_rng(13)
    S = 64
    seeds = W.seeds(S, start=200)
    reqs = random_items(rng, S, 150, max_len=300000)
    outs = [alloc(k, n) for _, k, n in reqs]
    with Streams(S, seeds=seeds) as st:
        st.set_batch_split(4096)
        srv = st.serve(lanes=4, max_batch=32)
        tickets = [srv.submit(s, k, n, out=o) for (s, k, n), o in zip(reqs, outs)]
        for t in tickets:
            srv.wait(t, 60000)
        for t in tickets:
            srv.release(t)
        srv.stop()
    refs = oracle_per_item(seeds, reqs)
    for (s, k, n), o, ref in zip(reqs, outs, refs):
        check(k, o[:n], ref)


# ------------------------------------------------- failure detection (host)

def test_server_survives_failed_launches(monkeypatch):
    """Host-side fault injection: the first two batch launches fail before
    reaching the GPU.  Their requests report XG_EDEVICE, leave their streams
    untouched, and the server goes on serving."""
    from paper_1108_0486_gb300 import XGError, _lib as L
    monkeypatch.setenv("XG_INJECT_LAUNCH_FAILURES", "2")
    seeds = W.seeds(3)
    outs = [alloc("u32", 1000) for _ in range(4)]
    with Streams(3, seeds=seeds) as st:
        srv = st.serve(lanes=1, max_batch=1)
        failed = 0
        for i in range(2):
            t = srv.submit(i, "u32", 1000, out=outs[i])
            with pytest.raises(XGError) as e:
                srv.wait(t, 10000)
            assert e.value.status == L.XG_EDEVICE
            srv.release(t)
            failed += 1
        t = srv.submit(0, "u32", 1000, out=outs[2])
        srv.wait(t, 10000)
        t2 = srv.submit(0, "u32", 1000, out=outs[3])
        srv.wait(t2, 10000)
        srv.stop()
    assert failed == 2
    ref = O.Xorgens.param_set(0).seed(int(seeds[0])).u32(2000)
    assert np.array_equal(outs[2].cpu().numpy().view(np.uint32), ref[:1000])
    assert np.array_equal(outs[3].cpu().numpy().view(np.uint32), ref[1000:])


def test_collect_drains_finished_requests():
    seeds = W.seeds(16)
    with Streams(16, seeds=seeds) as st:
        srv = st.serve()
        tickets = {srv.submit(i, KINDS[i % 3], 5000 + i) for i in range(16)}
        got = []
        for _ in range(2000):
            got += srv.collect(release=True)
            if len(got) == 16:
                break
            import time
            time.sleep(0.001)
        assert {g[0] for g in got} == tickets and all(g[4] == 0 for g in got)
        assert all(g[1] <= g[2] <= g[3] for g in got)  # submit <= launch <= done
        assert srv.stats()["outstanding_bytes"] == 0
        srv.stop()


def test_server_serving_workload_sampled():
    """The serving workload's request generator (65536 streams, sizes
    log-uniform in [2^10, 2^22], 60/30/10 normal/uniform/u32, PCG64 seed 486)
    over a 0.05 s window (~1000 requests, ~2 GB), submitted back to back into
    the library pool; every 50th request (a 2% sample) is checked against the
    oracle with its stream advanced by the earlier requests on it."""
    S = 65536
    reqs = W.serving_requests(n_streams=S, rate=20000.0, duration=0.05)
    seeds = W.seeds(S)
    with Streams(S, seeds=seeds) as st:
        srv = st.serve(mem_cap_bytes=16 << 30)
        tickets = [srv.submit(r.stream, r.kind, r.count) for r in reqs]
        sample = list(range(0, len(reqs), 50))
        got = {i: srv.result(tickets[i], reqs[i].kind, reqs[i].count).clone() for i in sample}
        for t in tickets:
            srv.wait(t, 60000)
            srv.release(t)
        srv.stop()
    assert len(reqs) > 500 and len(sample) >= 10
    for i in sample:
        r = reqs[i]
        k = KINDS[r.kind]
        before = sum(nwords(KINDS[q.kind], q.count) for q in reqs[:i] if q.stream == r.stream)
        words = O.Xorgens.param_set(0).seed(int(seeds[r.stream])).u32(before + nwords(k, r.count))
        check(k, got[i][:r.count], oracle_call(words[before:], k, r.count))


def test_submit_many_admits_in_order_and_matches_the_oracle():
    seeds = W.seeds(50, start=5)
    reqs = [(i % 50, KINDS[i % 3], 500 + 91 * i) for i in range(120)]
    with Streams(50, seeds=seeds) as st:
        srv = st.serve()
        tickets = srv.submit_many(reqs)
        assert len(tickets) == len(reqs) and tickets == sorted(tickets)
        outs = [srv.result(t, k, n).clone() for t, (_, k, n) in zip(tickets, reqs)]
        for t in tickets:
            srv.release(t)
        srv.stop()
    for (s, k, n), o, ref in zip(reqs, outs, oracle_per_item(seeds, reqs)):
        check(k, o[:n], ref)


def test_submit_many_partial_admission_and_invalid_requests():
    from paper_1108_0486_gb300 import _lib as L
    with Streams(4, seeds=[1, 2, 3, 4]) as st:
        srv = st.serve(mem_cap_bytes=1 << 20)
        # 400 KB each: the third would pass the 1 MiB cap
        t = srv.submit_many([(0, "u32", 100000), (1, "u32", 100000), (2, "u32", 100000)])
        assert len(t) == 2
        with pytest.raises(L.XGError):     # stream 9 does not exist: nothing admitted
            srv.submit_many([(3, "u32", 10), (9, "u32", 10)])
        assert srv.stats()["submitted"] == 2
        for x in t:
            srv.wait(x, 60000)
            srv.release(x)
        assert len(srv.submit_many([(2, "u32", 100000), (3, "u32", 10)])) == 2
        srv.stop()


def test_server_trace_records_every_batch(tmp_path, monkeypatch):
    path = tmp_path / "trace.csv"
    monkeypatch.setenv("XG_SERVER_TRACE", str(path))
    with Streams(8, seeds=W.seeds(8)) as st:
        srv = st.serve(lanes=2)
        tickets = [srv.submit(i % 8, KINDS[i % 3], 5000 + i) for i in range(24)]
        for t in tickets:
            srv.wait(t, 60000)
            srv.release(t)
        batches = srv.stats()["batches"]
        srv.stop()
    lines = path.read_text().splitlines()
    assert lines[0].startswith("lane,items,units,words")
    assert lines[1].startswith("# loop iterations")
    rows = [l.split(",") for l in lines[2:]]
    assert len(rows) == batches and sum(int(r[1]) for r in rows) == 24
    assert all(float(r[7]) >= 0 for r in rows)


def test_server_with_the_paper_parameter_set():
    """The request server on a context of the paper's set (128,65,15,14,12,17)
    gives the oracle's outputs of that set."""
    seeds = W.seeds(30, start=300)
    reqs = [(i % 30, KINDS[i % 3], 700 + 53 * i) for i in range(90)]
    with Streams(30, param_set=1, seeds=seeds) as st:
        srv = st.serve(lanes=4)
        tickets = srv.submit_many(reqs)
        outs = [srv.result(t, k, n).clone() for t, (_, k, n) in zip(tickets, reqs)]
        for t in tickets:
            srv.release(t)
        srv.stop()
    for (s, k, n), o, ref in zip(reqs, outs, oracle_per_item(seeds, reqs, ps=1)):
        check(k, o[:n], ref)


def test_contexts_on_concurrent_cuda_streams():
    """Two contexts generating at the same time on their own CUDA streams
    (and a batch on a third) give the same outputs as alone."""
    s1, s2, s3 = (torch.cuda.Stream() for _ in range(3))
    seeds_a, seeds_b = W.seeds(64, start=1), W.seeds(64, start=1000)
    with Streams(64, seeds=seeds_a, stream=s1) as a, Streams(64, seeds=seeds_b, stream=s2) as b, \
            Streams(8, seeds=W.seeds(8, start=77), stream=s3) as c:
        outs_c = [alloc(KINDS[i % 3], 200000 + i) for i in range(8)]
        with torch.cuda.stream(s1):
            ua = a.u32(50000)
        with torch.cuda.stream(s2):
            nb = b.normal(50000)
        c.batch([(i, KINDS[i % 3], 200000 + i, outs_c[i]) for i in range(8)])
        torch.cuda.synchronize()
        ua, nb = ua.clone(), nb.clone()
    with Streams(64, seeds=seeds_a) as a2, Streams(64, seeds=seeds_b) as b2:
        assert torch.equal(ua, a2.u32(50000))
        assert torch.equal(nb, b2.normal(50000))
    refs = oracle_per_item(W.seeds(8, start=77), [(i, KINDS[i % 3], 200000 + i) for i in range(8)])
    for i in range(8):
        check(KINDS[i % 3], outs_c[i][:200000 + i], refs[i])


def test_server_cancel_queued_requests():
    """Requests queued behind a long one on the same stream can be
    cancelled: they never run, the stream's later requests read the words
    they would have read, poll/wait report XG_ECANCELED, xg_collect reports
    them, and release returns their bytes.  A finished request cannot be
    cancelled."""
    from paper_1108_0486_gb300 import XGError, _lib as L
    seeds = W.seeds(2, start=500)
    sizes = [1 << 25, 5000, 6000, 7000, 8000, 9000]
    with Streams(2, seeds=seeds) as st:
        st.set_batch_split(1)   # no cutting: the first request is one warp's 20 ms
        srv = st.serve(lanes=4)
        tickets = [srv.submit(0, "u32", n) for n in sizes]
        # the first request keeps stream 0 busy for far longer than this
        srv.cancel(tickets[2])
        srv.cancel(tickets[4])
        with pytest.raises(XGError) as e:
            srv.cancel(tickets[2])            # already cancelled
        assert e.value.status == L.XG_EINVAL
        kept = [0, 1, 3, 5]
        outs = {i: srv.result(tickets[i], "u32", sizes[i], timeout_ms=60000).clone() for i in kept}
        for i in (2, 4):
            with pytest.raises(XGError) as e:
                srv.wait(tickets[i])
            assert e.value.status == L.XG_ECANCELED
        with pytest.raises(XGError) as e:
            srv.cancel(tickets[0])            # finished
        assert e.value.status == L.XG_EINVAL
        done = {}
        for _ in range(200):
            for (t, _, _, _, status, _) in srv.collect(64):
                done[t] = status
            if len(done) == len(sizes):
                break
            time.sleep(0.005)
        assert {done[tickets[i]] for i in (2, 4)} == {L.XG_ECANCELED}
        assert all(done[tickets[i]] == L.XG_OK for i in kept)
        for t in tickets:
            srv.release(t)
        assert srv.stats()["outstanding_bytes"] == 0
        srv.stop()
    seq = O.Xorgens.param_set(0).seed(int(seeds[0])).u32(sum(sizes[i] for i in kept))
    off = 0
    for i in kept:
        assert np.array_equal(outs[i].cpu().numpy().view(np.uint32), seq[off:off + sizes[i]]), i
        off += sizes[i]


def test_tensor_core_wait_that_runs_out_reports_a_device_error(monkeypatch):
    """The failure path of the tensor-core kernel's bounded waits.  With
    XG_TC_TEST_STALL=1 its first CTA arms the first stage's barrier but starts
    none of that stage's copies, so the waits on the stage give up after 2 s;
    the kernel then waits (bounded) for its copies in flight, frees its TMEM
    and returns.  The jump reports XG_EDEVICE, and the context and the GPU
    keep working: the same context, reseeded, jumps to the oracle's words."""
    from paper_1108_0486_gb300 import _lib as L
    monkeypatch.setenv("XG_GF2_TC_MIN_STATES", "1")
    monkeypatch.setenv("XG_JUMP_TENSOR_CORES", "1")
    seeds = W.seeds(4, start=9100)
    J = (1 << 40) + 3
    with Streams(4, seeds=seeds) as st:
        monkeypatch.setenv("XG_TC_TEST_STALL", "1")
        with pytest.raises(L.XGError) as err:
            st.jump(1 << 20)
        assert err.value.status == L.XG_EDEVICE and "gave up waiting" in str(err.value)
        monkeypatch.delenv("XG_TC_TEST_STALL")
        st.seed(seeds)
        st.jump(J)
        got = st.u32(32).cpu().numpy().view(np.uint32)
    for i in range(4):
        assert np.array_equal(got[i], O.u32_after_jump(int(seeds[i]), J, 32)), i
