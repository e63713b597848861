"""Pins for the oracle's inference tables (Section 4.3: minMatches and the
(m,n) concentration cache; Sections 4.1 / 4.2 for the quantities inside).

The tables are recomputed here from the paper's formulas with scipy (Boost's
incomplete beta) and, near the decision boundaries, with mpmath at 40 digits.
Neither shares code with the oracle.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle as O

sp = pytest.importorskip("scipy.special")
GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def c2r(c):
    return 1.0 - math.acos(c) / math.pi


def r2c(r):
    return math.cos(math.pi * (1.0 - r))


def ref_prune(p, m, n):
    """Pr[S >= t | M(m,n)] straight from Sections 4.1 / 4.2 with scipy."""
    if p.kind == O.JACCARD:
        return float(sp.betainc(n - m + p.beta, m + p.alpha, 1.0 - p.t))
    a, b = m + 1.0, n - m + 1.0
    den = float(sp.betainc(b, a, 0.5))
    if den == 0.0:
        return 0.0
    return float(sp.betainc(b, a, 1.0 - c2r(p.t))) / den


def ref_est(p, m, n):
    if p.kind == O.JACCARD:
        return min(1.0, max(0.0, (m + p.alpha - 1.0) / (n + p.alpha + p.beta - 2.0)))
    return r2c(max(m / n, 0.5))


def ref_conc(p, m, n):
    s = ref_est(p, m, n)
    if p.kind == O.JACCARD:
        a, b = m + p.alpha, n - m + p.beta
        hi, lo = min(1.0, s + p.delta), max(0.0, s - p.delta)
        return float(sp.betainc(a, b, hi) - sp.betainc(a, b, lo))
    a, b = m + 1.0, n - m + 1.0
    rhi = c2r(min(1.0, s + p.delta))
    rlo = max(0.5, c2r(max(-1.0, s - p.delta)))
    den = float(sp.betainc(b, a, 0.5))
    return (float(sp.betainc(b, a, 1 - rlo)) - float(sp.betainc(b, a, 1 - rhi))) / den


PARAMS = [
    O.Params(kind=O.JACCARD, n_max=256),
    O.Params(kind=O.JACCARD, n_max=512, k=64, t=0.5),
    O.Params(kind=O.JACCARD, n_max=256, alpha=2.0, beta=5.0, t=0.6),
    O.Params(kind=O.JACCARD, n_max=384, k=128, t=0.8, eps=0.01, delta=0.03, gamma=0.05),
    O.Params(kind=O.COSINE, n_max=2048),
    O.Params(kind=O.COSINE, n_max=1024, t=0.8),
    O.Params(kind=O.COSINE, n_max=512, k=64, t=0.5, eps=0.05),
]


@pytest.mark.parametrize("p", PARAMS, ids=lambda p: f"kind{p.kind}-k{p.k}-n{p.n_max}-t{p.t}-a{p.alpha}")
def test_tables_against_independent_inference(p):
    tab = O.tables(p)
    assert tab.scan_matches_search, "linear scan and binary search disagree (Section 4.3)"
    near = 0
    for j in range(p.levels):
        n = (j + 1) * p.k
        pr = np.array([ref_prune(p, m, n) for m in range(n + 1)])
        # Pr[S >= t | M] grows with m for fixed n (Section 4.3) -- where it is not 0.
        nz = pr > 1e-300
        assert np.all(np.diff(pr[nz]) >= -1e-15)
        ok = np.nonzero(pr >= p.eps)[0]
        want_mm = int(ok[0]) if len(ok) else n + 1
        assert abs(pr[want_mm - 1] - p.eps) > 1e-9 if 0 < want_mm <= n else True
        assert tab.min_matches[j] == want_mm, (n, tab.min_matches[j], want_mm)
        # The oracle's probabilities agree with the library's to 1e-9 (absolute).
        got = tab.prune_prob[j, : n + 1]
        assert np.allclose(got, pr, rtol=1e-9, atol=1e-12)
        for m in range(want_mm, n + 1):
            c = ref_conc(p, m, n)
            if abs(c - (1 - p.gamma)) < 1e-9:
                near += 1
                continue
            assert tab.conc[j, m] == (1 if c >= 1 - p.gamma else 0), (n, m, c)
            assert tab.conc_prob[j, m] == pytest.approx(c, abs=1e-9)
        assert np.all(tab.conc[j, :want_mm] == 0)
        for m in range(n + 1):
            assert tab.est[j, m] == pytest.approx(ref_est(p, m, n), abs=1e-15)
    assert near == 0


def test_boundaries_with_mpmath():
    """minMatches and the first concentrated m, checked at 40 digits."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40

    def prune(p, m, n):
        if p.kind == O.JACCARD:
            return mp.betainc(m + p.alpha, n - m + p.beta, mp.mpf(p.t), 1, regularized=True)
        tr = 1 - mp.acos(mp.mpf(p.t)) / mp.pi
        f = lambda r: r ** m * (1 - r) ** (n - m)
        return mp.betainc(m + 1, n - m + 1, tr, 1) / mp.betainc(m + 1, n - m + 1, mp.mpf("0.5"), 1)

    for p in (O.Params(kind=O.JACCARD, n_max=256), O.Params(kind=O.COSINE, n_max=2048)):
        tab = O.tables(p)
        for j in list(range(0, p.levels, max(1, p.levels // 6))) + [p.levels - 1]:
            n = (j + 1) * p.k
            mm = int(tab.min_matches[j])
            assert prune(p, mm, n) >= p.eps
            if mm > 0:
                assert prune(p, mm - 1, n) < p.eps


def test_tables_cross_check_values():
    """Table entries computed independently with scipy's regularised
    incomplete beta; a check that the readings of Sections 4.1-4.3 are the
    intended ones."""
    tj = O.tables(O.Params(kind=O.JACCARD, n_max=256))
    assert tj.min_matches.tolist() == [18, 38, 59, 80, 102, 123, 144, 166]
    c = np.nonzero(tj.conc[7])[0]
    assert (c.min(), c.max()) == (216, 256)
    c = np.nonzero(tj.conc[2])[0]
    assert c.min() == 94 and not tj.conc[:2].any()
    tc = O.tables(O.Params(kind=O.COSINE, n_max=2048))
    assert [int(tc.min_matches[j]) for j in range(8)] == [20, 42, 64, 87, 110, 133, 156, 179]
    assert [int(tc.min_matches[j]) for j in (15, 31, 63)] == [364, 739, 1493]
    assert np.nonzero(tc.conc[0])[0].tolist() == [32]
    c = np.nonzero(tc.conc[63])[0]
    assert (c.min(), c.max()) == (1498, 2048)


def test_min_matches_tracks_threshold():
    for p, target in ((O.Params(kind=O.JACCARD, n_max=4096, k=128), 0.7),
                      (O.Params(kind=O.COSINE, n_max=4096, k=128), c2r(0.7))):
        tab = O.tables(p)
        n = np.arange(1, p.levels + 1) * p.k
        assert np.all(np.diff(tab.min_matches) > 0)
        frac = tab.min_matches / n
        assert np.all(frac < target)               # eps-pruning is conservative
        assert abs(frac[-1] - target) < 3 * math.sqrt(target * (1 - target) / n[-1])


def test_mode_is_argmax_of_posterior():
    """Equation map: the table's estimate maximises the posterior density,
    found here by a fine grid search."""
    grid = np.linspace(1e-6, 1 - 1e-6, 400001)
    for alpha, beta, m, n in [(1, 1, 20, 32), (2, 5, 40, 64), (3, 1.5, 100, 128), (1, 1, 0, 32)]:
        p = O.Params(kind=O.JACCARD, alpha=alpha, beta=beta, n_max=128)
        tab = O.tables(p)
        logpdf = (m + alpha - 1) * np.log(grid) + (n - m + beta - 1) * np.log1p(-grid)
        assert tab.est[n // 32 - 1, m] == pytest.approx(grid[np.argmax(logpdf)], abs=1e-5)
    rgrid = np.linspace(0.5, 1 - 1e-7, 500001)
    p = O.Params(kind=O.COSINE, n_max=128)
    tab = O.tables(p)
    for m, n in [(24, 32), (80, 96), (128, 128), (10, 32)]:
        logpdf = m * np.log(rgrid) + (n - m) * np.log1p(-rgrid)
        assert tab.est[n // 32 - 1, m] == pytest.approx(r2c(rgrid[np.argmax(logpdf)]), abs=1e-4)


def test_appendix_schedule_concentrates():
    """Appendix: a pair with cosine 0.70 (r = 0.75) observed at 24/32, 48/64,
    96/128 agreements; the posterior mode stays at r = 0.75 and its
    concentration grows with n."""
    g = GOLD["appendix_schedule"]
    assert abs(c2r(g["cosine"]) - g["r"]) < g["r_tolerance"]
    assert c2r(GOLD["r_of_orthogonal"]["cosine"]) == GOLD["r_of_orthogonal"]["r"]
    p = O.Params(kind=O.COSINE, n_max=128, t=0.5)
    tab = O.tables(p)
    prev = 0.0
    for m, n in g["mn"]:
        assert m / n == g["r"]
        assert tab.est[n // 32 - 1, m] == pytest.approx(r2c(0.75), abs=1e-15)
        cp = tab.conc_prob[n // 32 - 1, m]
        assert cp > prev
        prev = cp


def test_concentration_goes_to_one():
    """At a fixed match fraction the posterior concentrates as n grows."""
    for kind, frac in ((O.JACCARD, 0.8), (O.COSINE, 0.85)):
        p = O.Params(kind=kind, n_max=4096, k=128, t=0.5)
        tab = O.tables(p)
        vals = [tab.conc_prob[j, int(frac * (j + 1) * 128)] for j in range(p.levels)]
        assert all(b >= a - 1e-12 for a, b in zip(vals, vals[1:]))
        assert vals[-1] > 0.999


def test_experiment_parameters_are_defaults():
    g = GOLD["experiment_parameters"]
    p = O.Params()
    assert (p.eps, p.gamma, p.delta, p.k, p.h) == (g["eps"], g["gamma"], g["delta"], g["k"], g["h_jaccard"])


def test_lsh_band_formula():
    # Section 2: l = ceil(log eps / log(1 - t^k)); e.g. t^k = 1/2 needs
    # ceil(log2(1/eps)) bands.
    assert O.lsh_bands_for(0.5 ** (1 / 8), 8, 0.03) == math.ceil(math.log2(1 / 0.03))
    assert O.lsh_bands_for(0.7, 8, 0.03) == 60
