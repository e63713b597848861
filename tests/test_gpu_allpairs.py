"""GPU parity of the AllPairs-style prefix-filter candidate generator (the
candidate source Section 5.1 pairs with BayesLSH besides LSH): the candidate
list equal to the oracle's, pair for pair and in the same order, for tf-idf
vectors and sets, with rows of every length class (up to 32 elements, up to
4096, longer); the count-only protocol; truncation of the pairs and an
undersized key buffer reported; small inputs."""
import numpy as np
import pytest
import torch

import oracle as O
import synth

pytestmark = pytest.mark.gpu
dev = torch.device("cuda")


def with_long_rows(csr, n_long, length, seed, values):
    """csr with n_long rows of `length` elements appended (longer than the
    shared-memory sort: every feature indexed)."""
    rng = np.random.default_rng(seed)
    rows = [np.sort(rng.choice(csr.dim, length, replace=False)).astype(np.uint32) for _ in range(n_long)]
    indptr = np.concatenate([csr.indptr, csr.indptr[-1] + np.cumsum([length] * n_long)]).astype(np.int64)
    indices = np.concatenate([csr.indices] + rows).astype(np.uint32)
    vals = None
    if values:
        v = [rng.uniform(0.1, 1.0, length) for _ in range(n_long)]
        v = [(x / np.linalg.norm(x)).astype(np.float32) for x in v]
        vals = np.concatenate([csr.values] + v).astype(np.float32)
    return synth.CSR(indptr, indices, vals, csr.dim)


def run(B, ctx, csr, t, kind, max_dups=None, cap=None):
    ip = torch.from_numpy(csr.indptr).to(dev)
    ix = torch.from_numpy(csr.indices.view(np.int32)).to(dev)
    val = None if kind == O.JACCARD else torch.from_numpy(csr.values).to(dev)
    N, nnz = csr.n, int(csr.indptr[-1])
    n_pairs = torch.zeros(1, dtype=torch.int64, device=dev)
    n_dups = torch.zeros(1, dtype=torch.int64, device=dev)
    ws = torch.zeros(B.blsh_allpairs_workspace(N, nnz, csr.dim, 0), dtype=torch.uint8, device=dev)
    B.blsh_allpairs_candidates(ctx, ip, ix, val, csr.dim, t, kind, None, n_pairs, ws, 0, n_dups)
    assert B.blsh_status(ctx) == 0
    dups = int(n_dups.item())
    assert int(n_pairs.item()) == 0
    md = dups if max_dups is None else max_dups
    ws = torch.zeros(B.blsh_allpairs_workspace(N, nnz, csr.dim, md), dtype=torch.uint8, device=dev)
    c = (dups if cap is None else cap) or 1
    pairs = torch.full((c, 2), -1, dtype=torch.int32, device=dev)
    B.blsh_allpairs_candidates(ctx, ip, ix, val, csr.dim, t, kind, pairs, n_pairs, ws, md, n_dups)
    rc = B.blsh_status(ctx)
    return rc, dups, int(n_pairs.item()), pairs.cpu().numpy().view(np.uint32)


@pytest.mark.parametrize("t", [0.3, 0.5, 0.7, 0.9])
def test_cosine_matches_oracle(B, ctx, t):
    vecs = synth.tfidf_vectors(n_docs=3000, dim=30000, mean_nnz=80, n_groups=150, seed=5)
    vecs = with_long_rows(vecs, 3, 5000, seed=6, values=True)
    lens = np.diff(vecs.indptr)
    assert (lens <= 32).any() and ((lens > 32) & (lens <= 4096)).any() and (lens > 4096).any()
    want = O.allpairs_candidates(vecs, t, O.COSINE)
    rc, dups, n, got = run(B, ctx, vecs, t, O.COSINE)
    assert rc == 0 and n == len(want) and dups >= n
    assert np.array_equal(got[:n], want)


@pytest.mark.parametrize("t", [0.3, 0.5, 0.7, 0.8])
def test_sets_match_oracle(B, ctx, t):
    sets = synth.jaccard_sets(n_sets=3000, vocab=10000, mean_size=50, n_groups=200, seed=1)
    sets = with_long_rows(sets, 2, 4500, seed=7, values=False)
    want = O.allpairs_candidates(sets, t, O.JACCARD)
    rc, dups, n, got = run(B, ctx, sets, t, O.JACCARD)
    assert rc == 0 and n == len(want)
    assert np.array_equal(got[:n], want)


def test_truncation_and_small_inputs(B, ctx):
    sets = synth.jaccard_sets(n_sets=800, vocab=3000, mean_size=30, n_groups=80, seed=3)
    want = O.allpairs_candidates(sets, 0.5, O.JACCARD)
    assert len(want) > 20
    # fewer pairs than the candidates: the first cap written, the count reported
    rc, dups, n, got = run(B, ctx, sets, 0.5, O.JACCARD, cap=len(want) - 7)
    assert rc == B.ETRUNC and n == len(want)
    assert np.array_equal(got[: len(want) - 7], want[: len(want) - 7])
    # a key buffer below the count: no pairs, truncation reported
    rc, dups, n, got = run(B, ctx, sets, 0.5, O.JACCARD, max_dups=10)
    assert rc == B.ETRUNC and n == 0
    assert B.blsh_status(ctx) == 0
    # one row, and rows without elements
    one = synth.CSR(np.array([0, 3], np.int64), np.array([1, 5, 9], np.uint32), None, 10)
    assert run(B, ctx, one, 0.5, O.JACCARD)[2] == 0
    empty = synth.CSR(np.array([0, 0, 2, 2, 4], np.int64), np.array([1, 2, 1, 2], np.uint32), None, 4)
    rc, dups, n, got = run(B, ctx, empty, 0.5, O.JACCARD)
    assert rc == 0 and got[:n].tolist() == O.allpairs_candidates(empty, 0.5, O.JACCARD).tolist() == [[1, 3]]
