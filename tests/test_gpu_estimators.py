"""GPU parity for the classical estimator (Section 3, the "LSH Approx" mode)
and the method-of-moments prior (Section 4.1)."""
import numpy as np
import pytest
import torch

import oracle as O
import synth

pytestmark = pytest.mark.gpu
dev = torch.device("cuda")


def t32(a):
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int32)).to(dev)


@pytest.mark.parametrize("kind,n,W", [(0, 360, 360), (0, 256, 256), (1, 2048, 64), (1, 70, 4)])
def test_mle_matches_oracle(B, ctx, kind, n, W):
    rng = np.random.default_rng(n)
    sims = rng.uniform(0.5 if kind else 0.0, 1.0, 5003)
    sig, pairs = synth.bernoulli_signatures(sims, 32 * W if kind else W, "cosine" if kind else "jaccard", seed=n)
    m_o, est_o, keep_o = O.estimate_mle(kind, n, 0.7, pairs, sig)
    P = len(pairs)
    m = torch.zeros(P, dtype=torch.int16, device=dev)
    est = torch.zeros(P, dtype=torch.float32, device=dev)
    keep = torch.zeros(P, dtype=torch.uint8, device=dev)
    B.blsh_estimate_mle(ctx, kind, n, 0.7, t32(pairs), t32(sig), m, est, keep)
    assert B.blsh_status(ctx) == 0
    assert np.array_equal(m.cpu().numpy().view(np.uint16), m_o)
    assert np.array_equal(keep.cpu().numpy(), keep_o)
    assert np.max(np.abs(est.cpu().numpy() - est_o)) <= 1e-6


def test_prior_matches_oracle(B, ctx):
    sets = synth.jaccard_sets(n_sets=3000, vocab=8000, mean_size=60, n_groups=300, seed=3)
    a, b = synth.minhash_coeffs(256, seed=4)
    sig = O.minhash(sets, a, b)
    cand = O.lsh_candidates(sig, O.JACCARD, 4, 16)
    rng = np.random.default_rng(0)
    sample = cand[rng.choice(len(cand), min(5000, len(cand)), replace=False)]
    want_sims = np.array([O.exact_jaccard(sets.row(int(x)), sets.row(int(y))) for x, y in sample])
    want = O.fit_beta_prior(want_sims)
    out, sims = B.blsh_fit_beta_prior(ctx, t32(sample), torch.from_numpy(sets.indptr).to(dev),
                                      t32(sets.indices))
    assert B.blsh_status(ctx) == 0
    assert np.array_equal(sims.cpu().numpy(), want_sims)             # bit-identical doubles
    assert out[4] == want[4]
    for g, w in zip(out[:4], want[:4]):
        assert g == pytest.approx(w, rel=1e-12)
    # the fitted prior builds tables like any other Beta
    tab = B.blsh_tables_build(ctx, B.make_params(kind=0, t=0.7, alpha=out[2], beta=out[3], n_max=256))
    o = O.tables(O.Params(kind=0, t=0.7, alpha=out[2], beta=out[3], n_max=256))
    g = B.blsh_tables_download(tab)
    assert g["near_ties"] == 0
    assert np.array_equal(g["min_matches"], o.min_matches) and np.array_equal(g["conc"], o.conc)


def test_mle_device_count_and_bad_pairs(B, ctx):
    sig, pairs = synth.bernoulli_signatures(np.linspace(0, 1, 300), 256, "jaccard", seed=9)
    pairs = pairs.copy()
    pairs[7, 1] = 600                 # one past the last row
    pairs[250, 0] = 0xFFFFFFFF
    P = len(pairs)
    m = torch.full((P,), 0x5A5A, dtype=torch.int16, device=dev)
    keep = torch.full((P,), 77, dtype=torch.uint8, device=dev)
    est = torch.zeros(P, dtype=torch.float32, device=dev)
    pd = torch.tensor([200], dtype=torch.int64, device=dev)
    B.blsh_estimate_mle(ctx, 0, 256, 0.5, t32(pairs), t32(sig), m, est, keep, P_dev=pd)
    assert B.blsh_status(ctx) == B.ERANGE
    assert B.blsh_status(ctx) == 0
    m_o, est_o, keep_o = O.estimate_mle(0, 256, 0.5, pairs[:200], sig)
    k = keep.cpu().numpy()
    assert k[7] == B.BAD_PAIR and np.isnan(est.cpu().numpy()[7])
    ok = np.arange(200) != 7
    assert np.array_equal(m.cpu().numpy().view(np.uint16)[:200][ok], m_o[ok])
    assert np.array_equal(k[:200][ok], keep_o[ok])
    assert np.all(k[200:] == 77) and np.all(m.cpu().numpy()[200:] == 0x5A5A)     # beyond *P_dev: untouched


def test_prior_many_random_pairs(B, ctx):
    """A large sample (many CTAs in the similarity pass, long strided sums in
    the moments pass), including self-pairs (similarity 1)."""
    sets = synth.jaccard_sets(n_sets=4000, vocab=30000, mean_size=100, n_groups=100, seed=5)
    pairs = synth.random_pairs(4000, 60000, seed=6)
    pairs[::997, 1] = pairs[::997, 0]
    want_sims = np.array([O.exact_jaccard(sets.row(int(x)), sets.row(int(y))) for x, y in pairs])
    want = O.fit_beta_prior(want_sims)
    out, sims = B.blsh_fit_beta_prior(ctx, t32(pairs), torch.from_numpy(sets.indptr).to(dev), t32(sets.indices))
    assert B.blsh_status(ctx) == 0
    assert np.array_equal(sims.cpu().numpy(), want_sims)
    assert out[4] == want[4]
    for g, w in zip(out[:4], want[:4]):
        assert g == pytest.approx(w, rel=1e-12)
