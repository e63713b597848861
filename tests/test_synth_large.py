"""The device-side generator of the 5e6-vector workload, run on the CPU at a
small size: the recipe's invariants (row lengths, sorted distinct term ids
per row, unit norms, planted groups sharing terms, determinism)."""
import numpy as np
import torch

import synth


def _draw(seed=3):
    return synth.large_tfidf_device(n_docs=3000, dim=1 << 16, nnz_min=5, nnz_max=400, n_groups=200, seed=seed,
                                    device=torch.device("cpu"))


def test_rows_are_sorted_distinct_unit_vectors():
    indptr, indices, values = _draw()
    ip = indptr.numpy()
    ix = indices.numpy().view(np.uint32)
    v = values.numpy().astype(np.float64)
    assert ip[0] == 0 and np.all(np.diff(ip) >= 1)
    lens = np.diff(ip)
    assert lens.max() <= 400                   # merged draws only shrink a row
    assert ix.max() < (1 << 16)
    for r in range(0, 3000, 7):
        row = ix[ip[r]:ip[r + 1]]
        assert np.all(np.diff(row.astype(np.int64)) > 0)
        nrm = np.sqrt((v[ip[r]:ip[r + 1]] ** 2).sum())
        assert nrm == 0.0 or abs(nrm - 1.0) < 1e-6


def test_lengths_follow_the_power_law_and_groups_share_terms():
    indptr, indices, _ = _draw()
    ip = indptr.numpy()
    ix = indices.numpy().view(np.uint32)
    lens = np.diff(ip)
    # p(l) ~ l^-2 on [5, 400]: about half the rows are shorter than 10
    assert 0.35 < float((lens < 10).mean()) < 0.6
    # the first rows are planted groups: a variant keeps 60-90% of its base's draws,
    # so consecutive rows overlap far more than random rows do
    def jac(a, b):
        a, b = set(a.tolist()), set(b.tolist())
        return len(a & b) / max(1, len(a | b))
    near = np.mean([jac(ix[ip[r]:ip[r + 1]], ix[ip[r + 1]:ip[r + 2]]) for r in range(0, 400)])
    far = np.mean([jac(ix[ip[r]:ip[r + 1]], ix[ip[r + 1500]:ip[r + 1501]]) for r in range(0, 400)])
    assert near > 0.2 and far < 0.1


def test_seeded():
    a = _draw(5)
    b = _draw(5)
    c = _draw(6)
    assert all(torch.equal(x, y) for x, y in zip(a, b))
    assert not torch.equal(a[1][:1000], c[1][:1000])
