"""Hot calls allocate nothing and never synchronise: the verification plane and
Lite's squared-norm buffer are sized once by blsh_ctx_reserve, so a CUDA
graph captured at a larger N than any earlier call still takes the plane and
norm routes, with outputs equal to the oracle's.  Without a reservation the
same calls read the rows and form the norms per pair (same outputs)."""
import numpy as np
import pytest
import torch

import oracle as O
import synth

pytestmark = pytest.mark.gpu


def workload(N, n_random, seed=5):
    """Cosine signatures of 2,048 bits (> 64 MB for N = 300,000, so the plane
    applies) and short sparse rows.  Objects come in triples whose signatures
    differ in a few bits; the three pairs of every triple survive Lite's
    pruning (as many survivors as rows: the norm pass applies), and n_random
    random pairs are added."""
    rng = np.random.default_rng(seed)
    W, G = 64, N // 3
    base = rng.integers(0, 1 << 32, size=(G, W), dtype=np.uint64).astype(np.uint32)
    sig = np.repeat(base, 3, axis=0)
    for member in (1, 2):                       # one bit flipped in words 0..3
        for c in range(4):
            sig[member::3, c] ^= np.uint32(1) << rng.integers(0, 32, G).astype(np.uint32)
    g3 = 3 * np.arange(G, dtype=np.uint32)
    trip = np.concatenate([np.stack([g3, g3 + 1], 1), np.stack([g3, g3 + 2], 1), np.stack([g3 + 1, g3 + 2], 1)])
    rand = rng.integers(0, 3 * G, size=(n_random, 2)).astype(np.uint32)
    rand.sort(axis=1)
    pairs = np.concatenate([trip, rand]).astype(np.uint32)
    lens = rng.integers(3, 9, 3 * G)
    rows = [np.sort(rng.choice(2000, int(n), replace=False)).astype(np.uint32) for n in lens]
    vals = [rng.uniform(0.1, 1.0, len(r)).astype(np.float32) for r in rows]
    vals = [(v / np.sqrt(np.sum(v.astype(np.float64) ** 2))).astype(np.float32) for v in vals]
    indptr = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    csr = synth.CSR(indptr, np.concatenate(rows), np.concatenate(vals), 2000)
    return sig, pairs, csr


def dev_inputs(sig, pairs, csr, dev):
    t32 = lambda a: torch.from_numpy(np.ascontiguousarray(a).view(np.int32)).to(dev)
    return (t32(sig), t32(pairs), torch.from_numpy(csr.indptr).to(dev), t32(csr.indices),
            torch.from_numpy(csr.values).to(dev))


def outputs(P, levels, dev):
    return dict(status=torch.full((P,), 77, dtype=torch.uint8, device=dev),
                n_used=torch.zeros(P, dtype=torch.int16, device=dev),
                m=torch.zeros(P, dtype=torch.int16, device=dev),
                est=torch.full((P,), float("nan"), dtype=torch.float32, device=dev),
                hist=torch.zeros(levels, dtype=torch.int64, device=dev),
                lst=torch.full((P,), 77, dtype=torch.uint8, device=dev),
                sim=torch.full((P,), float("nan"), dtype=torch.float64, device=dev))


def call(B, ctx, tab, sig, pairs, ip, ix, vals, o):
    B.blsh_verify_both(ctx, tab, pairs, sig, o["status"], o["n_used"], o["m"], o["est"], o["hist"], ip, ix, vals,
                       o["lst"], o["sim"])


def check(o, want, lite):
    assert np.array_equal(o["status"].cpu().numpy(), want.status)
    assert np.array_equal(o["n_used"].cpu().numpy().view(np.uint16), want.n_used)
    assert np.array_equal(o["m"].cpu().numpy().view(np.uint16), want.m)
    est = o["est"].cpu().numpy()
    assert np.array_equal(np.isnan(est), np.isnan(want.est))
    ok = ~np.isnan(want.est)
    assert np.max(np.abs(est[ok] - want.est[ok]), initial=0) <= 1e-6
    assert np.array_equal(o["lst"].cpu().numpy(), lite.status)
    sim = o["sim"].cpu().numpy()
    assert np.array_equal(np.isnan(sim), np.isnan(lite.sim))
    assert np.array_equal(sim[~np.isnan(sim)], lite.sim[~np.isnan(lite.sim)])


@pytest.mark.parametrize("reserve", [True, False], ids=["reserved", "unreserved"])
def test_graph_at_larger_N_than_any_earlier_call(B, reserve):
    dev = torch.device("cuda", 0)
    sig, pairs, csr = workload(300_000, 50_000)
    N, P = sig.shape[0], len(pairs)
    p = O.Params(kind=1, t=0.7, k=32, n_max=2048, h=128)
    tab_o = O.tables(p)
    want = O.verify(tab_o, pairs, sig)
    lite = O.verify_lite(tab_o, pairs, sig, csr)
    assert int((lite.status != O.PRUNED).sum()) > N // 2       # the norm pass applies
    ctx = B.Context(0)
    if reserve:
        B.blsh_ctx_reserve(ctx, N)
    tab = B.blsh_tables_build(ctx, B.make_params(kind=1, t=0.7, k=32, n_max=2048, h=128))
    sig_d, pairs_d, ip, ix, vals = dev_inputs(sig, pairs, csr, dev)
    # an eager call over a small prefix of the objects first
    n0 = 2000
    small = pairs[(pairs[:, 1] < n0)]
    sp = torch.from_numpy(small.view(np.int32)).to(dev)
    o0 = outputs(len(small), tab.levels, dev)
    call(B, ctx, tab, sig_d[:n0], sp, ip[: n0 + 1], ix, vals, o0)
    assert B.blsh_status(ctx) == 0
    check(o0, O.verify(tab_o, small, sig[:n0]), O.verify_lite(tab_o, small, sig[:n0], csr))
    # then a graph captured over all N objects
    o = outputs(P, tab.levels, dev)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    before = B.blsh_launch_count(ctx)
    with torch.cuda.graph(g, stream=s):
        call(B, ctx, tab, sig_d, pairs_d, ip, ix, vals, o)
    launched = B.blsh_launch_count(ctx) - before
    # plane copy, verification, survivor collection, row norms, queued and
    # in-place exact passes; without the reservation no plane copy and no norms
    assert launched == (6 if reserve else 4)
    g.replay()
    torch.cuda.synchronize()
    assert B.blsh_status(ctx) == 0
    check(o, want, lite)
    # a second replay gives the same outputs
    for v in o.values():
        v.fill_(77 if v.dtype == torch.uint8 else float("nan") if v.is_floating_point() else 0)
    g.replay()
    torch.cuda.synchronize()
    check(o, want, lite)


def test_reserve_arguments(B):
    ctx = B.Context(0)
    assert B.blsh_ctx_reserved(ctx) == 0
    with pytest.raises(B.BlshError) as e:
        B.blsh_ctx_reserve(ctx, -1)
    assert e.value.code == B.EINVAL
    B.blsh_ctx_reserve(ctx, 1000)
    B.blsh_ctx_reserve(ctx, 10)          # never shrinks
    assert B.blsh_ctx_reserved(ctx) == 1000
    B.blsh_ctx_reserve(ctx, 0)           # releases
    assert B.blsh_ctx_reserved(ctx) == 0
