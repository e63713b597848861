"""GPU parity: the Section 4.3 tables and Algorithm 1 against the CPU oracle.

Tables: minMatches and the concentration bitmap bit-exact, estimates within
1e-6.  Verification: per-pair status, hashes used, agreements bit-exact and
estimates within 1e-6, for every launch plan (the plan may only change
speed), for ragged pair counts spanning several CTAs, and for the edge cases
(no pairs, one pair, identical and disjoint signatures, pairs naming an
object >= N)."""
import numpy as np
import pytest
import torch

import oracle as O
import synth

pytestmark = pytest.mark.gpu
EST_TOL = 1e-6

TABLE_PARAMS = [
    dict(kind=0, n_max=256, k=32, t=0.7),
    dict(kind=0, n_max=512, k=64, t=0.5),
    dict(kind=0, n_max=384, k=128, t=0.8, eps=0.01, delta=0.03, gamma=0.05),
    dict(kind=0, n_max=256, k=32, t=0.6, alpha=2.0, beta=5.0),
    dict(kind=1, n_max=2048, k=32, t=0.7),
    dict(kind=1, n_max=1024, k=32, t=0.8),
    dict(kind=1, n_max=4096, k=128, t=0.6),
    dict(kind=1, n_max=512, k=64, t=0.5, eps=0.05),
]


def oracle_params(d):
    return O.Params(kind=d["kind"], t=d.get("t", 0.7), eps=d.get("eps", 0.03), delta=d.get("delta", 0.05),
                    gamma=d.get("gamma", 0.03), alpha=d.get("alpha", 1.0), beta=d.get("beta", 1.0), k=d["k"],
                    n_max=d["n_max"], h=min(d["n_max"], 64 if d["kind"] == 0 else 128))


def gpu_tables(B, ctx, d):
    p = B.make_params(kind=d["kind"], t=d.get("t", 0.7), eps=d.get("eps", 0.03), delta=d.get("delta", 0.05),
                      gamma=d.get("gamma", 0.03), alpha=d.get("alpha", 1.0), beta=d.get("beta", 1.0), k=d["k"],
                      n_max=d["n_max"])
    return B.blsh_tables_build(ctx, p)


@pytest.mark.parametrize("d", TABLE_PARAMS, ids=lambda d: "-".join(f"{k}{v}" for k, v in d.items()))
def test_tables_bit_exact(B, ctx, d):
    tab = gpu_tables(B, ctx, d)
    assert tab.build_status == B.OK
    g = B.blsh_tables_download(tab)
    o = O.tables(oracle_params(d))
    assert g["near_ties"] == 0
    assert np.array_equal(g["min_matches"], o.min_matches)
    assert np.array_equal(g["conc"], o.conc)
    L = o.min_matches.shape[0]
    for j in range(L):
        n = (j + 1) * d["k"]
        assert np.max(np.abs(g["est"][j, : n + 1] - o.est[j, : n + 1])) <= EST_TOL
        pr_o, pr_g = o.prune_prob[j, : n + 1], g["prune_prob"][j, : n + 1]
        assert np.allclose(pr_g, pr_o, rtol=1e-10, atol=1e-14)
        mm = o.min_matches[j]
        assert np.allclose(g["conc_prob"][j, mm: n + 1], o.conc_prob[j, mm: n + 1], rtol=1e-10, atol=1e-13)


def test_tables_reject_bad_params(B, ctx):
    for bad in (dict(k=48), dict(n_max=100), dict(t=1.5), dict(eps=0.0), dict(n_max=8192)):
        d = dict(kind=0, n_max=256, k=32, t=0.7)
        d.update(bad)
        with pytest.raises(B.BlshError) as e:
            gpu_tables(B, ctx, d)
        assert e.value.code == B.EINVAL


def run_verify(B, ctx, tab, pairs, sig, plan=None, P_dev=None, cap=None):
    dev = torch.device("cuda")
    pairs_t = torch.from_numpy(np.ascontiguousarray(pairs, np.uint32).view(np.int32)).to(dev)
    if cap is not None and cap > len(pairs):
        pairs_t = torch.cat([pairs_t, torch.zeros((cap - len(pairs), 2), dtype=torch.int32, device=dev)])
    sig_t = torch.from_numpy(np.ascontiguousarray(sig, np.uint32).view(np.int32)).to(dev)
    P = pairs_t.shape[0]
    status = torch.full((P,), 77, dtype=torch.uint8, device=dev)
    n_used = torch.zeros(P, dtype=torch.int16, device=dev)
    m = torch.zeros(P, dtype=torch.int16, device=dev)
    est = torch.full((P,), float('nan'), dtype=torch.float32, device=dev)   # entries not written stay NaN
    hist = torch.zeros(tab.levels, dtype=torch.int64, device=dev)
    pd = None if P_dev is None else torch.tensor([P_dev], dtype=torch.int64, device=dev)
    B.blsh_verify(ctx, tab, pairs_t, sig_t, status, n_used, m, est, hist, P_dev=pd, plan=plan)
    rc = B.blsh_status(ctx)
    return rc, status.cpu().numpy(), n_used.cpu().numpy().view(np.uint16), m.cpu().numpy().view(np.uint16), \
        est.cpu().numpy(), hist.cpu().numpy()


def assert_same(res, want, hist, p):
    rc, st, nu, m, est, h = res
    assert rc == 0
    assert np.array_equal(st, want.status)
    assert np.array_equal(nu, want.n_used)
    assert np.array_equal(m, want.m)
    assert np.array_equal(np.isnan(est), np.isnan(want.est))
    ok = ~np.isnan(want.est)
    assert np.max(np.abs(est[ok] - want.est[ok]), initial=0) <= EST_TOL
    assert np.array_equal(h, O.stop_hist(want.n_used, p.k, p.levels).astype(np.int64))


def all_plans(B, kind, k):
    plans = []
    groups = [1] if kind == 1 else [g for g in (1, 4, 8, 16, 32) if {1: 32, 4: 32, 8: 32, 16: 64, 32: 128}[g] <= k]
    for g in groups:
        for block in (128, 512):
            plans.append(B.blsh_plan(B.PLAN_PLAIN, g, block, 32, 0))
            for grab in (1, 37, 256):
                plans.append(B.blsh_plan(B.PLAN_PERSISTENT, g, block, grab, 0))
    plans.append(B.blsh_plan(B.PLAN_PERSISTENT, groups[-1], 256, 64, 1))
    return plans


def model_signatures(kind, n_max, P, seed):
    rng = np.random.default_rng(seed)
    sims = np.concatenate([rng.uniform(0, 1, P // 2), rng.uniform(0.55, 0.97, P - P // 2 - 2), [1.0, 0.0]])
    if kind == 1:
        sims = np.clip(sims, 0.5, 1.0)
    return synth.bernoulli_signatures(sims, n_max, "jaccard" if kind == 0 else "cosine", seed=seed)


@pytest.mark.parametrize("d", [TABLE_PARAMS[0], TABLE_PARAMS[1], TABLE_PARAMS[2], TABLE_PARAMS[4],
                               TABLE_PARAMS[6]], ids=lambda d: f"kind{d['kind']}-k{d['k']}-n{d['n_max']}")
def test_verify_every_plan_matches_oracle(B, ctx, d):
    p = oracle_params(d)
    sig, pairs = model_signatures(d["kind"], d["n_max"], 3001, seed=d["k"] + d["kind"])
    rng = np.random.default_rng(1)
    pairs = np.concatenate([pairs, rng.integers(0, sig.shape[0], size=(2000, 2)).astype(np.uint32)])
    want = O.verify(O.tables(p), pairs, sig)
    tab = gpu_tables(B, ctx, d)
    for plan in all_plans(B, d["kind"], d["k"]):
        assert_same(run_verify(B, ctx, tab, pairs, sig, plan=plan), want, None, p)
    assert_same(run_verify(B, ctx, tab, pairs, sig), want, None, p)


@pytest.mark.parametrize("d", [TABLE_PARAMS[4], TABLE_PARAMS[7]], ids=["k32-n2048", "k64-n512"])
def test_verify_large_signature_set_matches_oracle(B, ctx, d):
    """Cosine signature sets too large for L2 (> 64 MB) are verified with the
    first two words of every row read from a dense plane once the context
    has reserved it (blsh_ctx_reserve), and from the rows without one: the
    same outputs as the oracle either way, every plan."""
    p = oracle_params(d)
    sig, pairs = model_signatures(1, d["n_max"], 3001, seed=11)
    W = sig.shape[1]
    rows = (64 << 20) // (4 * W) + 4096                   # just past the plane threshold
    rng = np.random.default_rng(2)
    big = rng.integers(0, 1 << 32, size=(rows, W), dtype=np.uint64).astype(np.uint32)
    big[-sig.shape[0]:] = sig                             # the model pairs at the end of the set
    pairs = pairs + np.uint32(rows - sig.shape[0])
    pairs = np.concatenate([pairs, rng.integers(0, rows, size=(20000, 2)).astype(np.uint32)])
    want = O.verify(O.tables(p), pairs, big)
    ctx = B.Context(0)          # a context of its own: no reservation yet
    tab = gpu_tables(B, ctx, d)
    B.blsh_timing_begin(ctx)
    res = run_verify(B, ctx, tab, pairs, big)
    assert [n for n, _ in B.blsh_timing_end(ctx)] == ["verify_kernel"]     # rows read directly
    assert_same(res, want, None, p)
    B.blsh_ctx_reserve(ctx, rows)
    assert B.blsh_ctx_reserved(ctx) == rows
    for plan in (B.blsh_plan(B.PLAN_PLAIN, 1, 128, 32, 0), B.blsh_plan(B.PLAN_PERSISTENT, 1, 256, 37, 0)):
        assert_same(run_verify(B, ctx, tab, pairs, big, plan=plan), want, None, p)
    B.blsh_timing_begin(ctx)
    res = run_verify(B, ctx, tab, pairs, big)
    assert [n for n, _ in B.blsh_timing_end(ctx)] == ["plane_copy_kernel", "verify_kernel"]
    assert_same(res, want, None, p)


def test_autotune_k_outputs_are_the_chosen_ks(B, ctx):
    """The batching pattern's tuner chooses k among 32, 64 and 128 together
    with the plan; later calls with the returned tables give the oracle's
    outputs for that k (and Lite's h rounded up to a whole chunk)."""
    sig, pairs = model_signatures(0, 256, 20001, seed=21)
    dev = torch.device("cuda")
    pairs_t = torch.from_numpy(pairs.view(np.int32)).to(dev)
    sig_t = torch.from_numpy(sig.view(np.int32)).to(dev)
    P = len(pairs)
    st = torch.zeros(P, dtype=torch.uint8, device=dev)
    nu = torch.zeros(P, dtype=torch.int16, device=dev)
    params = B.make_params(kind=0, t=0.6, k=32, n_max=256, h=64)
    tab, plan, ms = B.blsh_autotune_k(ctx, params, (32, 64, 128), pairs_t, sig_t, st, nu)
    k = tab.params.k
    assert k in (32, 64, 128) and sorted(ms) == [32, 64, 128] and all(v > 0 for v in ms.values())
    assert tab.params.h == (128 if k == 128 else 64)
    assert plan.mode in (B.PLAN_PLAIN, B.PLAN_PERSISTENT) and plan.block in (128, 256, 512)
    p = O.Params(kind=0, t=0.6, k=k, n_max=256, h=tab.params.h)
    want = O.verify(O.tables(p), pairs, sig)
    assert_same(run_verify(B, ctx, tab, pairs, sig), want, None, p)
    for bad in ((48,), (32, 512), ()):
        with pytest.raises((B.BlshError, ValueError)):
            B.blsh_autotune_k(ctx, params, bad, pairs_t, sig_t, st, nu)
    with pytest.raises(B.BlshError):          # 128 does not divide n_max = 320
        B.blsh_autotune_k(ctx, B.make_params(kind=0, t=0.6, k=32, n_max=320), (32, 128), pairs_t, sig_t, st, nu)


def test_verify_device_count_and_capacity(B, ctx):
    d = TABLE_PARAMS[4]
    p = oracle_params(d)
    sig, pairs = model_signatures(1, 2048, 1000, seed=5)
    want = O.verify(O.tables(p), pairs[:777], sig)
    tab = gpu_tables(B, ctx, d)
    for plan in (None, B.blsh_plan(B.PLAN_PLAIN, 1, 256, 32, 0)):
        rc, st, nu, m, est, h = run_verify(B, ctx, tab, pairs, sig, plan=plan, P_dev=777, cap=1000)
        assert rc == 0
        assert np.array_equal(st[:777], want.status) and np.all(st[777:] == 77)
        assert np.array_equal(nu[:777], want.n_used)


def test_verify_edge_cases(B, ctx):
    d = TABLE_PARAMS[0]
    p = oracle_params(d)
    tab = gpu_tables(B, ctx, d)
    sig, pairs = model_signatures(0, 256, 64, seed=9)
    # no pairs
    rc, st, *_ = run_verify(B, ctx, tab, pairs[:0], sig)
    assert rc == 0 and len(st) == 0
    # one pair; identical; disjoint
    for q in (0, len(pairs) - 2, len(pairs) - 1):
        want = O.verify(O.tables(p), pairs[q:q + 1], sig)
        assert_same(run_verify(B, ctx, tab, pairs[q:q + 1], sig), want, None, p)
    # a pair naming an object >= N is flagged; the others are still exact
    bad = pairs.copy()
    bad[5] = (0, sig.shape[0])
    bad[9] = (sig.shape[0] + 3, 1)
    want = O.verify(O.tables(p), bad, sig)
    rc, st, nu, m, est, h = run_verify(B, ctx, tab, bad, sig)
    assert rc == B.ERANGE
    assert st[5] == B.BAD_PAIR and st[9] == B.BAD_PAIR
    ok = np.ones(len(bad), bool); ok[[5, 9]] = False
    assert np.array_equal(st[ok], want.status[ok]) and np.array_equal(m[ok], want.m[ok])
    assert B.blsh_status(ctx) == 0          # the error was cleared


def test_verify_rejects_bad_arguments(B, ctx):
    tab = gpu_tables(B, ctx, TABLE_PARAMS[0])
    sig, pairs = model_signatures(0, 256, 8, seed=1)
    dev = torch.device("cuda")
    st = torch.zeros(len(pairs), dtype=torch.uint8, device=dev)
    short = torch.zeros((sig.shape[0], 128), dtype=torch.int32, device=dev)   # fewer than n_max words
    with pytest.raises(B.BlshError) as e:
        B.blsh_verify(ctx, tab, torch.from_numpy(pairs.view(np.int32)).to(dev), short, st)
    assert e.value.code == B.EINVAL
    with pytest.raises(B.BlshError):
        B.blsh_verify(ctx, tab, torch.from_numpy(pairs.view(np.int32)).to(dev),
                      torch.from_numpy(sig.view(np.int32)).to(dev), st,
                      plan=B.blsh_plan(B.PLAN_PERSISTENT, 3, 256, 32, 0))


def test_autotune_picks_a_valid_plan(B, ctx):
    d = TABLE_PARAMS[0]
    p = oracle_params(d)
    sig, pairs = model_signatures(0, 256, 20000, seed=3)
    tab = gpu_tables(B, ctx, d)
    dev = torch.device("cuda")
    pt = torch.from_numpy(pairs.view(np.int32)).to(dev)
    stt = torch.from_numpy(sig.view(np.int32)).to(dev)
    st = torch.zeros(len(pairs), dtype=torch.uint8, device=dev)
    best = B.blsh_autotune(ctx, tab, pt, stt, st)
    assert best.mode in (0, 1) and best.group in (1, 4, 8, 16, 32)
    want = O.verify(O.tables(p), pairs, sig)
    assert_same(run_verify(B, ctx, tab, pairs, sig), want, None, p)   # now with the tuned plan


def test_lite_form_every_cosine_plan(B, ctx):
    """Algorithm 2's pruning pass runs in whichever plan the context holds."""
    d = TABLE_PARAMS[4]
    p = oracle_params(d)
    sig, pairs = model_signatures(1, 2048, 4001, seed=12)
    csr = synth.CSR(np.zeros(sig.shape[0] + 1, np.int64), np.zeros(0, np.uint32), np.zeros(0, np.float32), 1)
    want = O.verify_lite(O.tables(p), pairs, sig, csr)
    tab = gpu_tables(B, ctx, d)
    dev = torch.device("cuda")
    pt = torch.from_numpy(pairs.view(np.int32)).to(dev)
    stt = torch.from_numpy(sig.view(np.int32)).to(dev)
    ip = torch.zeros(sig.shape[0] + 1, dtype=torch.int64, device=dev)
    ix = torch.zeros(1, dtype=torch.int32, device=dev)
    val = torch.zeros(1, dtype=torch.float32, device=dev)
    st = torch.zeros(len(pairs), dtype=torch.uint8, device=dev)
    sim = torch.full((len(pairs),), float('nan'), dtype=torch.float64, device=dev)
    B.blsh_autotune(ctx, tab, pt, stt, st)          # stores some plan for these tables
    B.blsh_verify_lite(ctx, tab, pt, stt, ip, ix, val, st, sim)
    assert B.blsh_status(ctx) == 0
    assert np.array_equal(st.cpu().numpy(), want.status)
    # each launch form explicitly: the plain one runs the two-pass kernel,
    # where a survivor of the pruning loop is decided, not open
    for plan in (B.blsh_plan(B.PLAN_PLAIN, 1, 256, 32, 0), B.blsh_plan(B.PLAN_PERSISTENT, 1, 256, 64, 0)):
        B.blsh_set_plan(ctx, tab, plan)
        st.fill_(77)
        B.blsh_verify_lite(ctx, tab, pt, stt, ip, ix, val, st, sim)
        assert B.blsh_status(ctx) == 0
        assert np.array_equal(st.cpu().numpy(), want.status)


@pytest.mark.parametrize("kind", [0, 1])
@pytest.mark.parametrize("mode", [0, 1])
def test_verify_both_matches_oracle_and_separate_calls(B, ctx, kind, mode):
    """The fused pass gives Algorithm 1's and Algorithm 2's outputs exactly,
    in both launch forms, with bad pairs and a device pair count."""
    dev = torch.device("cuda")
    if kind == 0:
        objs = synth.jaccard_sets(n_sets=2000, vocab=10000, mean_size=50, n_groups=200, seed=21)
        a, b = synth.minhash_coeffs(256, seed=22)
        sig = O.minhash(objs, a, b)
        pairs = np.concatenate([O.lsh_candidates(sig, O.JACCARD, 8, 32), synth.random_pairs(2000, 3001, seed=23)])
        d = dict(kind=0, n_max=256, k=32, t=0.7)
    else:
        objs = synth.tfidf_vectors(n_docs=3000, dim=30000, mean_nnz=80, n_groups=150, seed=24)
        sig = O.srp_sparse(objs, synth.gaussian_matrix(30000, 512, seed=25))
        pairs = np.concatenate([O.lsh_candidates(sig, O.COSINE, 8, 30), synth.random_pairs(3000, 3001, seed=26)])
        d = dict(kind=1, n_max=512, k=32, t=0.7)
    pairs = pairs.copy()
    pairs[5, 1] = objs.n + 3                     # a pair naming an object >= N
    P = len(pairs)
    p = oracle_params(d)
    tab_o = O.tables(p)
    want = O.verify(tab_o, pairs, sig)
    lite = O.verify_lite(tab_o, pairs, sig, objs)
    tab = gpu_tables(B, ctx, d)
    B.blsh_set_plan(ctx, tab, B.blsh_plan(mode, 1 if kind == 1 else 8, 256, 64, 0))
    t32 = lambda x: torch.from_numpy(np.ascontiguousarray(x, np.uint32).view(np.int32)).to(dev)
    ip = torch.from_numpy(objs.indptr).to(dev)
    ix = t32(objs.indices)
    val = None if objs.values is None else torch.from_numpy(objs.values).to(dev)
    cap = P + 100
    pt = torch.cat([t32(pairs), torch.zeros((100, 2), dtype=torch.int32, device=dev)])
    pd = torch.tensor([P], dtype=torch.int64, device=dev)
    st = torch.full((cap,), 77, dtype=torch.uint8, device=dev)
    nu = torch.zeros(cap, dtype=torch.int16, device=dev)
    m = torch.zeros(cap, dtype=torch.int16, device=dev)
    est = torch.full((cap,), float('nan'), dtype=torch.float32, device=dev)
    hist = torch.zeros(tab.levels, dtype=torch.int64, device=dev)
    lst = torch.full((cap,), 77, dtype=torch.uint8, device=dev)
    lnu = torch.zeros(cap, dtype=torch.int16, device=dev)
    sim = torch.full((cap,), float('nan'), dtype=torch.float64, device=dev)
    B.blsh_verify_both(ctx, tab, pt, t32(sig), st, nu, m, est, hist, ip, ix, val, lst, sim, lite_n_used=lnu, P_dev=pd)
    assert B.blsh_status(ctx) == B.ERANGE
    assert B.blsh_status(ctx) == 0
    assert np.array_equal(st.cpu().numpy()[:P], want.status) and np.all(st.cpu().numpy()[P:] == 77)
    assert np.array_equal(nu.cpu().numpy().view(np.uint16)[:P], want.n_used)
    assert np.array_equal(m.cpu().numpy().view(np.uint16)[:P], want.m)
    e = est.cpu().numpy()[:P]
    ok = ~np.isnan(want.est)
    assert np.array_equal(np.isnan(e), ~ok) and np.max(np.abs(e[ok] - want.est[ok]), initial=0) <= EST_TOL
    good = np.arange(P) != 5
    assert np.array_equal(hist.cpu().numpy(), O.stop_hist(want.n_used[good], p.k, p.levels).astype(np.int64))
    assert np.array_equal(lst.cpu().numpy()[:P], lite.status) and np.all(lst.cpu().numpy()[P:] == 77)
    assert np.array_equal(lnu.cpu().numpy().view(np.uint16)[:P], lite.n_used)
    g = sim.cpu().numpy()[:P]
    assert np.array_equal(np.isnan(g), np.isnan(lite.sim))
    okl = ~np.isnan(lite.sim)
    assert np.array_equal(g[okl], lite.sim[okl])
    assert (lite.status == O.LITE_ACCEPT).sum() > 10 and (want.status != O.PRUNED).sum() > 10


@pytest.mark.parametrize("kind", [0, 1])
def test_capped_then_resume_equals_full(B, ctx, kind):
    """Lazy hashing: the capped pass (first 128 or 512 hashes) and the resume
    pass give exactly the outputs of the single fused pass, and the need
    flags mark exactly the objects of the pairs that needed more hashes."""
    dev = torch.device("cuda")
    if kind == 0:
        objs = synth.jaccard_sets(n_sets=2000, vocab=10000, mean_size=50, n_groups=200, seed=41)
        a, b = synth.minhash_coeffs(256, seed=42)
        sig = O.minhash(objs, a, b)
        pairs = np.concatenate([O.lsh_candidates(sig, O.JACCARD, 8, 32), synth.random_pairs(2000, 3001, seed=43)])
        d, limit = dict(kind=0, n_max=256, k=32, t=0.7), 128
    else:
        objs = synth.tfidf_vectors(n_docs=3000, dim=30000, mean_nnz=80, n_groups=150, seed=44)
        sig = O.srp_sparse(objs, synth.gaussian_matrix(30000, 2048, seed=45))
        pairs = np.concatenate([O.lsh_candidates(sig, O.COSINE, 8, 30), synth.random_pairs(3000, 3001, seed=46)])
        d, limit = dict(kind=1, n_max=2048, k=32, t=0.7), 256
    P = len(pairs)
    tab = gpu_tables(B, ctx, d)
    t32 = lambda x: torch.from_numpy(np.ascontiguousarray(x, np.uint32).view(np.int32)).to(dev)
    ip = torch.from_numpy(objs.indptr).to(dev)
    ix = t32(objs.indices)
    val = None if objs.values is None else torch.from_numpy(objs.values).to(dev)
    pt, st = t32(pairs), t32(sig)

    def buffers():
        return (torch.zeros(P, dtype=torch.uint8, device=dev), torch.zeros(P, dtype=torch.int16, device=dev),
                torch.zeros(P, dtype=torch.int16, device=dev),
                torch.full((P,), float("nan"), dtype=torch.float32, device=dev),
                torch.zeros(tab.levels, dtype=torch.int64, device=dev), torch.zeros(P, dtype=torch.uint8, device=dev),
                torch.full((P,), float("nan"), dtype=torch.float64, device=dev))
    full = buffers()
    B.blsh_verify_both(ctx, tab, pt, st, *full[:5], ip, ix, val, full[5], full[6])
    lazy = buffers()
    need = torch.zeros(objs.n, dtype=torch.uint8, device=dev)
    B.blsh_verify_both_capped(ctx, tab, limit, pt, st, *lazy[:5], ip, ix, val, lazy[5], lazy[6], need)
    assert B.blsh_status(ctx) == 0
    capped = lazy[0].cpu().numpy() == B.NEEDS_HASHES
    assert capped.any() and not capped.all()
    marked = np.zeros(objs.n, bool)
    marked[pairs[capped].reshape(-1)] = True
    assert np.array_equal(need.cpu().numpy() == 1, marked)
    B.blsh_verify_resume(ctx, tab, pt, st, lazy[0], lazy[1], lazy[2], lazy[3], lazy[4])
    assert B.blsh_status(ctx) == 0
    for f, g in zip(full, lazy):
        a_, b_ = f.cpu().numpy(), g.cpu().numpy()
        if a_.dtype.kind == "f":
            assert np.array_equal(np.isnan(a_), np.isnan(b_)) and np.array_equal(a_[~np.isnan(a_)], b_[~np.isnan(b_)])
        else:
            assert np.array_equal(a_, b_)


@pytest.mark.parametrize("off", [0, 1, 2], ids=["aligned", "shift1", "shift2"])
def test_first_pass_forms_match_oracle(B, ctx, off):
    """The two-pass cosine form (k = 32, plain plan): with the pair list and
    every output array aligned for four-pair stores the first pass takes four
    pairs a lane, otherwise one; both give the oracle's outputs, for pair
    counts that leave every remainder mod 4, with an object index >= N in
    one pair (its quad goes pair by pair) and a device pair count."""
    d = TABLE_PARAMS[4]
    p = oracle_params(d)
    sig, pairs = model_signatures(1, d["n_max"], 4003, seed=31)
    rng = np.random.default_rng(3)
    pairs = np.concatenate([pairs, rng.integers(0, sig.shape[0], size=(3000, 2)).astype(np.uint32)])
    pairs[17] = (1, sig.shape[0] + 5)
    tab = gpu_tables(B, ctx, d)
    dev = torch.device("cuda")
    plan = B.blsh_plan(B.PLAN_PLAIN, 1, 256, 32, 0)
    sig_t = torch.from_numpy(sig.view(np.int32)).to(dev)
    for P in (len(pairs), len(pairs) - 1, len(pairs) - 2, len(pairs) - 3, 3, 1):
        want = O.verify(O.tables(p), pairs[:P], sig)
        cap = P + 8
        pt = torch.zeros((cap + off, 2), dtype=torch.int32, device=dev)
        pt[off:off + P] = torch.from_numpy(pairs[:P].view(np.int32)).to(dev)
        st = torch.full((cap + off,), 77, dtype=torch.uint8, device=dev)
        nu = torch.zeros(cap + off, dtype=torch.int16, device=dev)
        m = torch.zeros(cap + off, dtype=torch.int16, device=dev)
        est = torch.full((cap + off,), float("nan"), dtype=torch.float32, device=dev)
        hist = torch.zeros(tab.levels, dtype=torch.int64, device=dev)
        pd = torch.tensor([P], dtype=torch.int64, device=dev)
        B.blsh_verify(ctx, tab, pt[off:], sig_t, st[off:], nu[off:], m[off:], est[off:], hist, P_dev=pd, plan=plan)
        rc = B.blsh_status(ctx)
        if P > 17:
            assert rc == B.ERANGE
            assert B.blsh_status(ctx) == 0
        else:
            assert rc == 0
        s = st.cpu().numpy()[off:]
        assert np.array_equal(s[:P], want.status) and np.all(s[P:] == 77) and np.all(st.cpu().numpy()[:off] == 77)
        good = np.array([not (P > 17 and q == 17) for q in range(P)], bool)
        assert np.array_equal(nu.cpu().numpy().view(np.uint16)[off:off + P][good], want.n_used[good])
        assert np.array_equal(m.cpu().numpy().view(np.uint16)[off:off + P][good], want.m[good])
        e = est.cpu().numpy()[off:off + P]
        ok = ~np.isnan(want.est)
        assert np.array_equal(np.isnan(e), ~ok) and np.max(np.abs(e[ok] - want.est[ok]), initial=0) <= EST_TOL
        assert np.array_equal(hist.cpu().numpy(), O.stop_hist(want.n_used[good], p.k, p.levels).astype(np.int64))
