"""Pins of the oracle's AllPairs-style candidate generator (prefix filtering;
Section 5.1's comparison algorithm, Bayardo et al. 2007): hand-worked
examples, completeness against brute-force exact similarities (the property
that makes the filter an exact candidate generator), candidates sharing a
feature, monotonicity in t, the closed form at t -> 0 (every shared feature
indexed), and long rows indexing every feature."""
import json
import os

import numpy as np
import pytest

import oracle as O
import synth

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "allpairs_examples.json")))


def csr_of(rows, dim, values=None):
    indptr = np.concatenate([[0], np.cumsum([len(r) for r in rows])]).astype(np.int64)
    idx = np.concatenate([np.asarray(r, np.uint32) for r in rows]) if rows else np.zeros(0, np.uint32)
    val = None if values is None else np.concatenate([np.asarray(v, np.float32) for v in values])
    return synth.CSR(indptr, idx, val, dim)


def indexed_sets(csr, flags):
    return [sorted(int(f) for f, z in zip(csr.indices[a:b], flags[a:b]) if z)
            for a, b in zip(csr.indptr[:-1], csr.indptr[1:])]


@pytest.mark.parametrize("case", GOLD["sets"]["cases"], ids=lambda c: f"t{c['t']}")
def test_hand_worked_sets(case):
    g = GOLD["sets"]
    csr = csr_of(g["rows"], g["dim"])
    assert indexed_sets(csr, O.allpairs_indexed(csr, case["t"], O.JACCARD)) == case["indexed"]
    assert O.allpairs_candidates(csr, case["t"], O.JACCARD).tolist() == case["candidates"]


@pytest.mark.parametrize("case", GOLD["cosine"]["cases"], ids=lambda c: f"t{c['t']}")
def test_hand_worked_cosine(case):
    g = GOLD["cosine"]
    csr = csr_of([[f for f, _ in r] for r in g["rows"]], g["dim"], [[v for _, v in r] for r in g["rows"]])
    assert indexed_sets(csr, O.allpairs_indexed(csr, case["t"], O.COSINE)) == case["indexed"]
    assert O.allpairs_candidates(csr, case["t"], O.COSINE).tolist() == case["candidates"]


def exact_cosine_pairs(csr, t):
    X = np.zeros((csr.n, csr.dim))
    for i in range(csr.n):
        a, b = csr.indptr[i], csr.indptr[i + 1]
        X[i, csr.indices[a:b]] = csr.values[a:b]
    G = X @ X.T
    xs, ys = np.nonzero(np.triu(G >= t, 1))
    return set(zip(xs.tolist(), ys.tolist())), X


def exact_jaccard_pairs(csr, t):
    S = [set(csr.indices[a:b].tolist()) for a, b in zip(csr.indptr[:-1], csr.indptr[1:])]
    out = set()
    for x in range(len(S)):
        for y in range(x + 1, len(S)):
            u = len(S[x] | S[y])
            if u and len(S[x] & S[y]) / u >= t:
                out.add((x, y))
    return out, S


@pytest.mark.parametrize("t", [0.3, 0.5, 0.7, 0.9])
def test_complete_for_cosine(t):
    vecs = synth.tfidf_vectors(n_docs=400, dim=3000, mean_nnz=30, n_groups=60, seed=int(t * 10))
    true, X = exact_cosine_pairs(vecs, t)
    cand = set(map(tuple, O.allpairs_candidates(vecs, t, O.COSINE).tolist()))
    assert true <= cand and len(true) > 0
    # every candidate shares a feature
    share = (X != 0).astype(np.int32) @ (X != 0).astype(np.int32).T
    assert all(share[x, y] > 0 for x, y in cand)


@pytest.mark.parametrize("t", [0.3, 0.5, 0.7, 0.75])
def test_complete_for_sets(t):
    sets = synth.jaccard_sets(n_sets=300, vocab=1500, mean_size=25, n_groups=50, seed=int(t * 10))
    true, S = exact_jaccard_pairs(sets, t)
    cand = set(map(tuple, O.allpairs_candidates(sets, t, O.JACCARD).tolist()))
    assert true <= cand and len(true) > 0
    assert all(S[x] & S[y] for x, y in cand)


def test_monotone_in_t_and_closed_form_at_zero():
    vecs = synth.tfidf_vectors(n_docs=300, dim=2000, mean_nnz=20, n_groups=30, seed=4)
    prev = None
    for t in (0.9, 0.7, 0.5, 0.3, 0.1):
        cand = set(map(tuple, O.allpairs_candidates(vecs, t, O.COSINE).tolist()))
        if prev is not None:
            assert prev <= cand
        prev = cand
    # t -> 0: every feature indexed, so the candidates are the pairs sharing a feature
    _, X = exact_cosine_pairs(vecs, 1.0)
    share = (X != 0).astype(np.int32) @ (X != 0).astype(np.int32).T
    xs, ys = np.nonzero(np.triu(share > 0, 1))
    assert set(map(tuple, O.allpairs_candidates(vecs, 1e-12, O.COSINE).tolist())) == set(zip(xs.tolist(), ys.tolist()))
    sets = synth.jaccard_sets(n_sets=200, vocab=800, mean_size=15, n_groups=20, seed=5)
    flags = O.allpairs_indexed(sets, 1e-12, O.JACCARD)
    assert flags.all()


def test_long_rows_index_every_feature():
    rng = np.random.default_rng(3)
    rows = [np.sort(rng.choice(20000, 5000, replace=False)), np.sort(rng.choice(20000, 40, replace=False))]
    vals = [np.full(5000, 1 / np.sqrt(5000)), np.full(40, 1 / np.sqrt(40))]
    csr = csr_of(rows, 20000, vals)
    flags = O.allpairs_indexed(csr, 0.9, O.COSINE)
    assert flags[:5000].all() and not flags[5000:].all()
