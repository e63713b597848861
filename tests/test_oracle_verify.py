"""Pins for the oracle's Algorithm 1 (BayesLSH) and Algorithm 2
(BayesLSH-Lite).

The decision procedure is re-implemented here "online", as the algorithms are
printed: Pr[S>=t|M] and the concentration are recomputed with scipy at every
chunk, no tables (Section 4.3 claims the tables change nothing).  The paper's
probabilistic guarantees (Section 1) are checked by Monte Carlo under the model
they are stated for.
"""
import math

import numpy as np
import pytest

import oracle as O
import synth

sp = pytest.importorskip("scipy.special")


def c2r(c):
    return 1.0 - math.acos(c) / math.pi


def online_prune(p, m, n):
    if p.kind == O.JACCARD:
        return float(sp.betainc(n - m + p.beta, m + p.alpha, 1.0 - p.t))
    a, b = m + 1.0, n - m + 1.0
    den = float(sp.betainc(b, a, 0.5))
    return 0.0 if den == 0.0 else float(sp.betainc(b, a, 1 - c2r(p.t))) / den


def online_est(p, m, n):
    if p.kind == O.JACCARD:
        return min(1.0, max(0.0, (m + p.alpha - 1.0) / (n + p.alpha + p.beta - 2.0)))
    return math.cos(math.pi * (1.0 - max(m / n, 0.5)))


def online_conc(p, m, n):
    s = online_est(p, m, n)
    if p.kind == O.JACCARD:
        a, b = m + p.alpha, n - m + p.beta
        return float(sp.betainc(a, b, min(1.0, s + p.delta)) - sp.betainc(a, b, max(0.0, s - p.delta)))
    a, b = m + 1.0, n - m + 1.0
    rhi, rlo = c2r(min(1.0, s + p.delta)), max(0.5, c2r(max(-1.0, s - p.delta)))
    return (float(sp.betainc(b, a, 1 - rlo)) - float(sp.betainc(b, a, 1 - rhi))) / float(sp.betainc(b, a, 0.5))


def hashes_agree(p, sx, sy):
    if p.kind == O.JACCARD:
        return sx[: p.n_max] == sy[: p.n_max]
    bx = np.unpackbits(sx.view(np.uint8), bitorder="little")[: p.n_max]
    by = np.unpackbits(sy.view(np.uint8), bitorder="little")[: p.n_max]
    return bx == by


def online_algorithm1(p, sig, pairs):
    out = []
    for x, y in pairs:
        agree = hashes_agree(p, sig[x], sig[y])
        n = m = 0
        while True:
            m += int(agree[n: n + p.k].sum())
            n += p.k
            if online_prune(p, m, n) < p.eps:
                st = O.PRUNED
                break
            if online_conc(p, m, n) >= 1 - p.gamma:
                st = O.ACCEPT
                break
            if n == p.n_max:
                st = O.ACCEPT_AT_MAX
                break
        out.append((st, n, m, online_est(p, m, n)))
    return out


@pytest.mark.parametrize("kind,n_max,k", [(O.JACCARD, 256, 32), (O.JACCARD, 256, 64), (O.COSINE, 2048, 32),
                                          (O.COSINE, 1024, 128)])
def test_algorithm1_equals_online_inference(kind, n_max, k):
    p = O.Params(kind=kind, n_max=n_max, k=k, t=0.7)
    rng = np.random.default_rng(7)
    sims = np.concatenate([rng.uniform(0, 1, 300), rng.uniform(0.6, 0.95, 300), [1.0, 0.0]])
    if kind == O.COSINE:
        sims = np.clip(sims, 0.5, 1.0)
    sig, pairs = synth.bernoulli_signatures(sims, n_max, "jaccard" if kind == O.JACCARD else "cosine", seed=11)
    tab = O.tables(p)
    res = O.verify(tab, pairs, sig)
    want = online_algorithm1(p, sig, pairs)
    assert res.bad == 0
    for q, (st, n, m, est) in enumerate(want):
        assert (res.status[q], res.n_used[q], res.m[q]) == (st, n, m), q
        if st == O.PRUNED:                     # no estimate is output for a pruned pair
            assert np.isnan(res.est[q])
        else:
            assert res.est[q] == pytest.approx(est, abs=1e-15)
    assert set(res.status.tolist()) >= {O.PRUNED, O.ACCEPT}


def test_identical_and_disjoint_pairs():
    """Identical signatures: never pruned (Pr >= eps at m = n).  Signatures
    that never agree: pruned after the first chunk."""
    for kind, nm in ((O.JACCARD, 256), (O.COSINE, 2048)):
        p = O.Params(kind=kind, n_max=nm)
        tab = O.tables(p)
        sig, pairs = synth.bernoulli_signatures(np.array([1.0, 0.0]), nm,
                                                "jaccard" if kind == O.JACCARD else "cosine", seed=3)
        r = O.verify(tab, pairs, sig)
        assert r.status[0] == O.ACCEPT and r.m[0] == r.n_used[0]
        assert r.status[1] == O.PRUNED and r.n_used[1] == p.k and r.m[1] == 0


def test_out_of_range_pairs_are_flagged():
    p = O.Params(kind=O.JACCARD, n_max=64)
    tab = O.tables(p)
    sig, _ = synth.bernoulli_signatures(np.array([0.5]), 64, "jaccard")
    r = O.verify(tab, np.array([[0, 1], [0, 2], [5, 1]], np.uint32), sig)
    assert r.bad == 2 and r.status.tolist()[1:] == [255, 255]


@pytest.mark.parametrize("kind", [O.JACCARD, O.COSINE])
def test_bayesian_guarantees_monte_carlo(kind):
    """Section 1 guarantees, under the model they are derived for: the
    similarity drawn from the prior, each hash agreeing with probability
    sim (Eq. lshmain).  A pruned pair had Pr[S >= t] < eps when it was
    pruned, so at most a fraction eps of pruned pairs are true pairs; a
    concentrated estimate is within delta with probability >= 1 - gamma."""
    p = O.Params(kind=kind, n_max=256 if kind == O.JACCARD else 2048, t=0.7)
    rng = np.random.default_rng(2024 + kind)
    P = 20000
    if kind == O.JACCARD:
        s = rng.uniform(0, 1, P)                 # Beta(1,1) prior
        r = s
    else:
        r = rng.uniform(0.5, 1, P)               # uniform prior on r in [0.5, 1]
        s = np.cos(np.pi * (1 - r))
    sig, pairs = synth.bernoulli_signatures(r, p.n_max, "jaccard" if kind == O.JACCARD else "cosine", seed=99)
    res = O.verify(O.tables(p), pairs, sig)
    pruned = res.status == O.PRUNED
    fn = np.mean(s[pruned] >= p.t)
    sd = math.sqrt(p.eps * (1 - p.eps) / pruned.sum())
    assert fn <= p.eps + 3 * sd
    conc = res.status == O.ACCEPT
    err = np.mean(np.abs(res.est[conc] - s[conc]) >= p.delta)
    sd = math.sqrt(p.gamma * (1 - p.gamma) / conc.sum())
    assert conc.sum() > 500 and err <= p.gamma + 3 * sd
    # and true pairs well above the threshold are almost never pruned
    hi = s >= p.t + 0.1
    assert np.mean(pruned[hi]) < p.eps


def test_lite_equals_online_algorithm2():
    p = O.Params(kind=O.JACCARD, n_max=256, h=64, t=0.5)
    sets = synth.jaccard_sets(n_sets=300, vocab=400, mean_size=40, n_groups=60, seed=5)
    a, b = synth.minhash_coeffs(256, seed=8)
    sig = O.minhash(sets, a, b)
    pairs = synth.random_pairs(300, 3000, seed=4)
    # add the planted near-duplicates: every pair that shares many elements
    cand = O.lsh_candidates(sig, O.JACCARD, 4, 16)
    pairs = np.concatenate([pairs, cand])
    tab = O.tables(p)
    res = O.verify_lite(tab, pairs, sig, sets)
    kept = 0
    for q, (x, y) in enumerate(pairs):
        agree = sig[x] == sig[y]
        n = m = 0
        pruned = False
        while n < p.h:
            m += int(agree[n: n + p.k].sum()); n += p.k
            if online_prune(p, m, n) < p.eps:
                pruned = True
                break
        assert res.n_used[q] == n
        if pruned:
            assert res.status[q] == O.PRUNED and np.isnan(res.sim[q])
            continue
        A, B = set(sets.row(x).tolist()), set(sets.row(y).tolist())
        s = len(A & B) / len(A | B)
        assert res.sim[q] == s
        assert res.status[q] == (O.LITE_ACCEPT if s > p.t else O.LITE_REJECT)
        kept += s > p.t
    assert kept > 20


def test_lite_cosine_exact_similarity():
    vecs = synth.tfidf_vectors(n_docs=400, dim=3000, mean_nnz=60, n_groups=80, seed=9)
    R = synth.gaussian_matrix(3000, 256, seed=10)
    sig = O.srp_sparse(vecs, R)
    p = O.Params(kind=O.COSINE, n_max=256, h=128, t=0.5)
    pairs = np.concatenate([synth.random_pairs(400, 2000, seed=1), O.lsh_candidates(sig, O.COSINE, 8, 12)])
    res = O.verify_lite(O.tables(p), pairs, sig, vecs)
    dense = np.zeros((400, 3000))
    for i in range(400):
        ix, v = vecs.row(i)
        dense[i, ix] = v
    surv = res.status != O.PRUNED
    assert surv.sum() > 50
    for q in np.nonzero(surv)[0]:
        x, y = pairs[q]
        want = dense[x] @ dense[y] / (np.linalg.norm(dense[x]) * np.linalg.norm(dense[y]))
        assert res.sim[q] == pytest.approx(want, abs=1e-12)
        assert res.status[q] == (O.LITE_ACCEPT if res.sim[q] > p.t else O.LITE_REJECT)


def test_exact_similarity_edge_cases():
    e = np.zeros(0, np.uint32)
    assert O.exact_jaccard(np.array([1, 2, 3]), np.array([1, 2, 3])) == 1.0
    assert O.exact_jaccard(np.array([1, 2]), np.array([3, 4])) == 0.0
    assert O.exact_jaccard(e, e) == 0.0
    assert O.exact_jaccard(np.array([1, 5, 9, 11]), np.array([2, 5, 11])) == 2 / 5
    ix = np.array([3, 7], np.uint32)
    v = np.array([0.6, 0.8], np.float32)
    assert O.exact_cosine(ix, v, ix, v) == pytest.approx(1.0, abs=1e-7)
    assert O.exact_cosine(ix, v, e, np.zeros(0, np.float32)) == 0.0
    assert O.exact_cosine(ix, v, ix, -v) == pytest.approx(-1.0, abs=1e-7)
    # order independence: the fixed-point sum does not depend on the order of
    # the terms, so reversing both rows gives the same bits
    rng = np.random.default_rng(0)
    idx = np.sort(rng.choice(10000, 500, replace=False)).astype(np.uint32)
    a = rng.standard_normal(500).astype(np.float32); a /= np.float32(np.linalg.norm(a))
    b = rng.standard_normal(500).astype(np.float32); b /= np.float32(np.linalg.norm(b))
    s1 = O.exact_cosine(idx, a, idx, b)
    assert s1 == pytest.approx(float(a.astype(np.float64) @ b.astype(np.float64)) /
                               (np.linalg.norm(a.astype(np.float64)) * np.linalg.norm(b.astype(np.float64))), abs=1e-13)


def test_compact_and_stop_hist():
    rng = np.random.default_rng(3)
    st = rng.integers(0, 5, 1000).astype(np.uint8)
    keep = (1 << O.ACCEPT) | (1 << O.ACCEPT_AT_MAX)
    assert np.array_equal(O.compact(st, keep), np.nonzero((st == 1) | (st == 2))[0])
    nu = (rng.integers(1, 9, 1000) * 32).astype(np.uint16)
    h = O.stop_hist(nu, 32, 8)
    assert h.tolist() == np.bincount(nu // 32 - 1, minlength=8).tolist()
