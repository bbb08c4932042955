"""xg_generate_batch_noalloc: the batched generation entry point for callers
that must not allocate device memory while they run (its scratch is a fixed
device array inside the library).  Checked through the C ABI against
xg_generate_batch on two calls in a row.  This file is collected last."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

KINDS = ["u32", "uniform", "normal"]


def _items(rng, n_streams, n_items):
    out = []
    for _ in range(n_items):
        s = int(rng.integers(0, n_streams))
        k = int(rng.integers(0, 3))
        n = int(np.exp(rng.uniform(0, np.log(30000))))
        out.append((s, k, n))
    return out


def _alloc(items):
    return [torch.full((max(n, 1),), -1, dtype=torch.int32, device="cuda") for _, _, n in items]


def test_noalloc_batch_matches_batch_on_two_calls():
    from paper_1108_0486_gb300 import Streams, _lib as L
    torch.cuda.set_device(0)
    rng = np.random.default_rng(2024)
    seeds = np.arange(1, 97, dtype=np.uint32)
    with Streams(96, seeds=seeds) as a, Streams(96, seeds=seeds) as b:
        for call in range(2):
            items = _items(rng, 96, 300)  # streams repeat: chains of calls
            ref = _alloc(items)
            got = _alloc(items)
            L.xg_generate_batch(a.ctx, [(s, k, n, o.data_ptr()) for (s, k, n), o in zip(items, ref)])
            L.xg_generate_batch_noalloc(b.ctx, [(s, k, n, o.data_ptr()) for (s, k, n), o in zip(items, got)])
            torch.cuda.synchronize()
            for (s, k, n), r, g in zip(items, ref, got):
                # u32 and uniform: bit-exact; normals: the same kernel code, so also bit-exact
                # (well within the 4-ulp tolerance of the other tests)
                assert torch.equal(r[:n], g[:n]), (call, s, KINDS[k], n)
        # the streams ended in the same state
        assert torch.equal(a.u32(64), b.u32(64))


def test_noalloc_rejects_more_than_the_maximum():
    from paper_1108_0486_gb300 import Streams, XGError, _lib as L
    torch.cuda.set_device(0)
    with Streams(4, seeds=[1, 2, 3, 4]) as st:
        out = torch.empty(8, dtype=torch.int32, device="cuda")
        with pytest.raises(XGError) as e:
            L.xg_generate_batch_noalloc(st.ctx, [(0, 0, 1, out.data_ptr())] * 1025)
        assert e.value.status == L.XG_EINVAL and "1024" in str(e.value)
