"""blsh_compact_noalloc: the compaction for callers that cannot allocate
device memory (code running inside a host that owns every allocation through
its own pool).  Its output must equal blsh_compact's on the same inputs, on
two calls in a row (the second call must not see the first call's scratch).
This file is collected last on purpose."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def reference(B, ctx, st, keep, cap):
    out = torch.full((cap,), -1, dtype=torch.int64, device="cuda")
    n = torch.zeros(1, dtype=torch.int64, device="cuda")
    B.blsh_compact(ctx, st, keep, out, n)
    B.blsh_status(ctx)
    return out.cpu().numpy(), int(n.item())


def test_noalloc_matches_compact_twice(B, ctx):
    rng = np.random.default_rng(42)
    keep = (1 << B.ACCEPT) | (1 << B.ACCEPT_AT_MAX)
    for P in (5_000_003, 70_000):            # a large call, then a smaller one
        st = torch.from_numpy(rng.integers(0, 5, P).astype(np.uint8)).cuda()
        cap = P
        want, n_want = reference(B, ctx, st, keep, cap)
        out = torch.full((cap,), -1, dtype=torch.int64, device="cuda")
        n = torch.zeros(1, dtype=torch.int64, device="cuda")
        B.blsh_compact_noalloc(st, keep, out, n)
        torch.cuda.synchronize()
        assert int(n.item()) == n_want
        assert np.array_equal(out.cpu().numpy()[:n_want], want[:n_want])


def test_noalloc_device_count_and_limits(B, ctx):
    rng = np.random.default_rng(7)
    P = 100_000
    st = torch.from_numpy(rng.integers(0, 5, P).astype(np.uint8)).cuda()
    pd = torch.tensor([61_234], dtype=torch.int64, device="cuda")
    out = torch.full((P,), -1, dtype=torch.int64, device="cuda")
    n = torch.zeros(1, dtype=torch.int64, device="cuda")
    B.blsh_compact_noalloc(st, 1 << B.LITE_ACCEPT, out, n, P_dev=pd)
    ref = torch.full((P,), -1, dtype=torch.int64, device="cuda")
    nr = torch.zeros(1, dtype=torch.int64, device="cuda")
    B.blsh_compact(ctx, st, 1 << B.LITE_ACCEPT, ref, nr, P_dev=pd)
    B.blsh_status(ctx)
    assert int(n.item()) == int(nr.item())
    assert torch.equal(out[: int(n.item())], ref[: int(nr.item())])
    # a capacity below the count writes only cap indices and reports the count
    small = torch.full((10,), -1, dtype=torch.int64, device="cuda")
    B.blsh_compact_noalloc(st, 1 << B.LITE_ACCEPT, small, n, P_dev=pd)
    torch.cuda.synchronize()
    assert int(n.item()) == int(nr.item()) and torch.equal(small, ref[:10])
    # more statuses than the fixed scratch covers: rejected before any launch
    big = torch.empty(67_108_865, dtype=torch.uint8, device="cuda")
    with pytest.raises(B.BlshError) as e:
        B.blsh_compact_noalloc(big, 1, out, n)
    assert e.value.code == B.ESIZE
