"""xg_generate_batch_noalloc: the batched generation entry point for callers
that must not allocate device memory while they run (their memory belongs to
another allocator, or their loop cannot take cudaMalloc's implicit
synchronisation).  Its scratch is a fixed device array inside the library.
Checked through the C ABI against xg_generate_batch on two calls in a row, at
the item limit, and for allocation: free device memory does not change across
calls.  This file is collected last."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

KINDS = ["u32", "uniform", "normal"]


def _items(rng, n_streams, n_items, max_len=30000):
    out = []
    for _ in range(n_items):
        s = int(rng.integers(0, n_streams))
        k = int(rng.integers(0, 3))
        n = int(np.exp(rng.uniform(0, np.log(max_len))))
        out.append((s, k, n))
    return out


def _alloc(items):
    return [torch.full((max(n, 1),), -1, dtype=torch.int32, device="cuda") for _, _, n in items]


def _compare(L, a, b, items, tag):
    ref = _alloc(items)
    got = _alloc(items)
    L.xg_generate_batch(a.ctx, [(s, k, n, o.data_ptr()) for (s, k, n), o in zip(items, ref)])
    L.xg_generate_batch_noalloc(b.ctx, [(s, k, n, o.data_ptr()) for (s, k, n), o in zip(items, got)])
    torch.cuda.synchronize()
    for (s, k, n), r, g in zip(items, ref, got):
        # u32 and uniform: bit-exact; normals: the same kernel code, so also
        # bit-exact (well within the 4-ulp tolerance of the other tests)
        assert torch.equal(r[:n], g[:n]), (tag, s, KINDS[k], n)


def test_noalloc_batch_matches_batch_on_two_calls():
    from paper_1108_0486_gb300 import Streams, _lib as L
    torch.cuda.set_device(0)
    rng = np.random.default_rng(2024)
    seeds = np.arange(1, 97, dtype=np.uint32)
    with Streams(96, seeds=seeds) as a, Streams(96, seeds=seeds) as b:
        for call in range(2):
            _compare(L, a, b, _items(rng, 96, 300), call)  # streams repeat: chains of calls
        # the streams ended in the same state
        assert torch.equal(a.u32(64), b.u32(64))


def test_noalloc_at_the_item_limit():
    """Exactly 1024 items: on 1024 distinct streams (half the planner's
    stream table filled), then all on one stream (one chain of 1024 calls)."""
    from paper_1108_0486_gb300 import Streams, _lib as L
    torch.cuda.set_device(0)
    rng = np.random.default_rng(1024)
    seeds = np.arange(1, 1025, dtype=np.uint32)
    with Streams(1024, seeds=seeds) as a, Streams(1024, seeds=seeds) as b:
        distinct = [(s, int(rng.integers(0, 3)), int(rng.integers(1, 3000))) for s in range(1024)]
        _compare(L, a, b, distinct, "distinct")
        one = [(7, int(rng.integers(0, 3)), int(rng.integers(1, 300))) for _ in range(1024)]
        _compare(L, a, b, one, "one stream")
        assert torch.equal(a.u32(32), b.u32(32))


def test_noalloc_allocates_no_device_memory():
    """Free device memory (cudaMemGetInfo) and torch's allocator are unchanged
    across two calls; everything the calls use exists before them."""
    from paper_1108_0486_gb300 import Streams, _lib as L
    torch.cuda.set_device(0)
    rng = np.random.default_rng(7)
    with Streams(64, seeds=np.arange(1, 65, dtype=np.uint32)) as st:
        batches = [_items(rng, 64, 200) for _ in range(3)]
        outs = [_alloc(items) for items in batches]
        args = [[(s, k, n, o.data_ptr()) for (s, k, n), o in zip(items, out)]
                for items, out in zip(batches, outs)]
        L.xg_generate_batch_noalloc(st.ctx, args[0])
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        torch_before = torch.cuda.memory_stats().get("allocation.all.allocated", 0)
        for a in args[1:]:
            L.xg_generate_batch_noalloc(st.ctx, a)
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        assert free1 == free0
        assert torch.cuda.memory_stats().get("allocation.all.allocated", 0) == torch_before


def test_noalloc_rejects_more_than_the_maximum():
    from paper_1108_0486_gb300 import Streams, XGError, _lib as L
    torch.cuda.set_device(0)
    with Streams(4, seeds=[1, 2, 3, 4]) as st:
        out = torch.empty(8, dtype=torch.int32, device="cuda")
        with pytest.raises(XGError) as e:
            L.xg_generate_batch_noalloc(st.ctx, [(0, 0, 1, out.data_ptr())] * 1025)
        assert e.value.status == L.XG_EINVAL and "1024" in str(e.value)
