"""GPU parity for the producers and the output step: minhash, sign random
projections (sparse and dense), LSH banding, Lite's exact similarity, and the
stable compaction -- all bit-exact against the CPU oracle."""
import numpy as np
import pytest
import torch

import oracle as O
import synth

pytestmark = pytest.mark.gpu
dev = torch.device("cuda")


def t32(a):
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int32)).to(dev)


def csr_dev(csr):
    out = [torch.from_numpy(csr.indptr).to(dev), t32(csr.indices.astype(np.uint32))]
    out.append(None if csr.values is None else torch.from_numpy(csr.values).to(dev))
    return out


@pytest.mark.parametrize("n_hashes", [32, 96, 256, 512])
def test_minhash_bit_exact(B, ctx, n_hashes):
    sets = synth.jaccard_sets(n_sets=1500, vocab=50000, mean_size=50, n_groups=100, seed=n_hashes)
    # add an empty set and long ones: one chunk, several chunks (10,000 and
    # 25,000 elements), and element ids just below 2^32
    rows = [sets.row(i) for i in range(sets.n)] + [np.zeros(0, np.int64), np.arange(0, 3000 * 7, 7),
                                                     np.arange(5, 10000 * 3 + 5, 3), np.arange(0, 25000),
                                                     np.arange(2 ** 32 - 15000, 2 ** 32 - 1, 3)]
    lens = np.array([len(r) for r in rows])
    csr = synth.CSR(np.concatenate([[0], np.cumsum(lens)]).astype(np.int64),
                    np.concatenate(rows).astype(np.uint32), None, 2 ** 32)
    a, b = synth.minhash_coeffs(n_hashes, seed=7)
    want = O.minhash(csr, a, b)
    ip, ix, _ = csr_dev(csr)
    sig = torch.zeros((csr.n, n_hashes), dtype=torch.int32, device=dev)
    B.blsh_minhash(ctx, ip, ix, n_hashes, t32(a), t32(b), sig)
    assert B.blsh_status(ctx) == 0
    assert np.array_equal(sig.cpu().numpy().view(np.uint32), want)


@pytest.mark.parametrize("bits", [64, 96, 384, 1536, 2048, 4096])
def test_srp_sparse_bit_exact(B, ctx, bits):
    vecs = synth.tfidf_vectors(n_docs=900, dim=20000, mean_nnz=80, n_groups=50, seed=bits)
    R = synth.gaussian_matrix(20000, bits, seed=11)
    want = O.srp_sparse(vecs, R)
    ip, ix, val = csr_dev(vecs)
    sig = torch.zeros((vecs.n, bits // 32), dtype=torch.int32, device=dev)
    B.blsh_srp_sparse(ctx, ip, ix, val, torch.from_numpy(R).to(dev), sig)
    rc, counters = B.blsh_status(ctx, counters=True)
    assert rc == 0
    assert np.array_equal(sig.cpu().numpy().view(np.uint32), want)


def test_srp_sparse_exact_ties_and_zero_rows(B, ctx):
    # rows whose projections are exactly zero (a zero row; x and -x at the same
    # index twice would be merged, so use two terms with cancelling products)
    R = np.ones((4, 32), np.float32)
    R[1] = -1
    csr = synth.CSR(np.array([0, 0, 2, 3], np.int64), np.array([0, 1, 2], np.uint32),
                    np.array([0.5, 0.5, -0.25], np.float32), 4)
    want = O.srp_sparse(csr, R)
    ip, ix, val = csr_dev(csr)
    sig = torch.zeros((3, 1), dtype=torch.int32, device=dev)
    B.blsh_srp_sparse(ctx, ip, ix, val, torch.from_numpy(R).to(dev), sig)
    rc, c = B.blsh_status(ctx, counters=True)
    assert rc == 0
    got = sig.cpu().numpy().view(np.uint32)
    assert np.array_equal(got, want)
    assert got[0, 0] == 0xFFFFFFFF and got[1, 0] == 0xFFFFFFFF and got[2, 0] == 0
    assert c[3] == 64 and c[2] >= 64


@pytest.mark.parametrize("n_docs", [3, 1100])
def test_srp_sparse_recheck_queue(B, ctx, n_docs):
    """Signs the FP32 bound cannot decide go through the recheck queue (and,
    past its 2^20 entries, through the in-line recheck): rows whose dots are
    exactly zero for every bit, or cancel to a few ulps."""
    bits = 2048
    rng = np.random.default_rng(n_docs)
    R = rng.standard_normal((6, bits)).astype(np.float32)
    R[1] = -R[0]
    R[3] = -R[2] * np.float32(1.0000001)
    rows, vals = [], []
    for i in range(n_docs):
        if i % 3 == 0:
            rows.append([0, 1]); vals.append([0.5, 0.5])          # exactly 0 for every bit
        elif i % 3 == 1:
            rows.append([2, 3]); vals.append([0.25, 0.25])        # nearly cancelling
        else:
            rows.append([0, 4, 5]); vals.append([0.3, 0.6, -0.2])
    csr = synth.CSR(np.concatenate([[0], np.cumsum([len(r) for r in rows])]).astype(np.int64),
                    np.concatenate(rows).astype(np.uint32), np.concatenate(vals).astype(np.float32), 6)
    want = O.srp_sparse(csr, R)
    ip, ix, val = csr_dev(csr)
    sig = torch.zeros((n_docs, bits // 32), dtype=torch.int32, device=dev)
    B.blsh_srp_sparse(ctx, ip, ix, val, torch.from_numpy(R).to(dev), sig)
    rc, c = B.blsh_status(ctx, counters=True)
    assert rc == 0
    assert np.array_equal(sig.cpu().numpy().view(np.uint32), want)
    n_zero_rows = (n_docs + 2) // 3
    assert c[3] >= n_zero_rows * bits and c[2] >= n_zero_rows * bits


@pytest.mark.parametrize("n,d,bits,tc,margin", [
    (3000, 64, 128, False, 0.0),      # CUDA-core path (bits not a multiple of 256)
    (300, 64, 256, True, 0.0),        # tensor cores, one K stage, ragged last row tile
    (3000, 256, 1024, True, 0.0),     # tensor cores, four K stages, four bit tiles
    (3000, 256, 1024, True, 1e-3),    # the precision workload's margin (wider than the error bound)
    (1000, 128, 512, True, 0.0),
])
def test_srp_dense_bit_exact(B, ctx, n, d, bits, tc, margin):
    X = synth.gaussian_mixture(n_points=n, dim=d, n_centers=50, seed=d)
    X[5] = 0.0                                            # a zero row: every dot is exactly 0
    R = synth.gaussian_matrix(d, bits, seed=5)
    want = O.srp_dense(X, R)
    sig = torch.zeros((n, bits // 32), dtype=torch.int32, device=dev)
    nws = B.blsh_srp_dense_workspace(n, d, bits)
    assert (nws > 0) == tc
    ws = torch.zeros(max(nws, 1), dtype=torch.uint8, device=dev) if tc else None
    B.blsh_srp_dense(ctx, torch.from_numpy(X).to(dev), torch.from_numpy(R).to(dev), sig, margin=margin, workspace=ws)
    rc, c = B.blsh_status(ctx, counters=True)
    assert rc == 0
    got = sig.cpu().numpy().view(np.uint32)
    bad = np.nonzero(got != want)
    assert np.array_equal(got, want), (len(bad[0]), bad[0][:5], bad[1][:5])
    assert c[3] >= bits                                   # the zero row went through the exact recheck
    if tc:
        # the tensor cores decided almost every sign themselves: only products
        # within the margin (well under 5% of them here) plus the zero row
        assert c[2] < 0.05 * n * bits + bits


def gpu_candidates(B, ctx, sig, kind, rows, bands, cap=None, ws_bytes=None):
    N = sig.shape[0]
    if ws_bytes is None:
        ws_bytes = B.blsh_lsh_candidates_workspace(N, kind, rows, bands)
    ws = torch.zeros(ws_bytes, dtype=torch.uint8, device=dev)
    n = torch.zeros(1, dtype=torch.int64, device=dev)
    if cap is None:
        # count-only call first (capacity 0), then the real one
        B.blsh_lsh_candidates(ctx, t32(sig), kind, rows, bands, None, n, ws)
        rc0 = B.blsh_status(ctx)
        assert rc0 == (B.ETRUNC if int(n.item()) > 0 else 0)
        cap = max(1, int(n.item()))
    pairs = torch.zeros((cap, 2), dtype=torch.int32, device=dev)
    B.blsh_lsh_candidates(ctx, t32(sig), kind, rows, bands, pairs, n, ws)
    rc = B.blsh_status(ctx)
    k = int(n.item())
    return rc, k, pairs[: min(k, cap)].cpu().numpy().view(np.uint32)


def sorted_pairs(p):
    p = np.asarray(p, np.uint64)
    key = (p[:, 0] << np.uint64(32)) | p[:, 1]
    return np.sort(key)


def test_banding_jaccard_bit_exact(B, ctx):
    sets = synth.jaccard_sets(n_sets=2000, vocab=10000, mean_size=50, n_groups=200, seed=1)
    a, b = synth.minhash_coeffs(256, seed=2)
    sig = O.minhash(sets, a, b)
    for rows, bands in ((8, 32), (4, 16), (1, 3)):
        want = O.lsh_candidates(sig, O.JACCARD, rows, bands)
        rc, n, got = gpu_candidates(B, ctx, sig, 0, rows, bands)
        assert rc == 0 and n == len(want)
        assert np.all(got[:, 0] < got[:, 1])
        assert np.array_equal(sorted_pairs(got), sorted_pairs(want))


def test_banding_jaccard_wide_and_fallback(B, ctx):
    """Many bands: up to 32 bands take the class-id path, more bands the
    per-pair hash check."""
    sets = synth.jaccard_sets(n_sets=1500, vocab=3000, mean_size=40, n_groups=200, seed=5)
    a, b = synth.minhash_coeffs(256, seed=6)
    sig = O.minhash(sets, a, b)
    for rows, bands in ((3, 32), (2, 40), (2, 100)):
        want = O.lsh_candidates(sig, O.JACCARD, rows, bands)
        rc, n, got = gpu_candidates(B, ctx, sig, 0, rows, bands)
        assert rc == 0 and n == len(want)
        assert np.array_equal(sorted_pairs(got), sorted_pairs(want))


def test_banding_jaccard_key_collision(B, ctx):
    """146089 and 154344 have the same top 32 bits of the one-row band hash,
    so their objects share a sort key; they must not become candidates of
    each other (the class ids compare the hashes themselves)."""
    sig = np.zeros((600, 4), np.uint32)
    sig[:200, :] = 146089
    sig[200:400, :] = 154344
    sig[400:, :] = np.arange(1, 201, dtype=np.uint32)[:, None] * 7919
    sig = sig[np.random.default_rng(0).permutation(600)]
    for rows, bands in ((1, 1), (1, 2), (1, 4)):
        want = O.lsh_candidates(sig, O.JACCARD, rows, bands)
        assert len(want) == 2 * 200 * 199 // 2
        rc, n, got = gpu_candidates(B, ctx, sig, 0, rows, bands)
        assert rc == 0 and n == len(want)
        assert np.array_equal(sorted_pairs(got), sorted_pairs(want))


def test_banding_cosine_bit_exact(B, ctx):
    vecs = synth.tfidf_vectors(n_docs=3000, dim=30000, mean_nnz=80, n_groups=100, seed=3)
    sig = O.srp_sparse(vecs, synth.gaussian_matrix(30000, 512, seed=4))
    # (2, 3) and (1, 4): buckets of 750 and 1,500 objects, longer than the
    # staged window of the cosine emission kernel; (12, 40) and (17, 30):
    # packed key rows of 80 and 120 bytes (the wide-row form of that kernel)
    for rows, bands in ((8, 35), (12, 20), (32, 4), (5, 7), (2, 3), (1, 4), (12, 40), (17, 30)):
        want = O.lsh_candidates(sig, O.COSINE, rows, bands)
        rc, n, got = gpu_candidates(B, ctx, sig, 1, rows, bands)
        assert rc == 0 and n == len(want)
        assert np.array_equal(sorted_pairs(got), sorted_pairs(want))


def test_banding_keep_record_same_output(B, ctx):
    """The emission's count pass records which pairs it keeps, in the
    workspace's last 64 N bands bytes, and its write pass replays the record
    instead of testing again; a workspace without that area, or with only part
    of it (the positions past its end are tested again), must give the same
    pairs in the same order, and the oracle's set."""
    vecs = synth.tfidf_vectors(n_docs=3000, dim=30000, mean_nnz=80, n_groups=100, seed=3)
    csig = O.srp_sparse(vecs, synth.gaussian_matrix(30000, 512, seed=4))
    sets = synth.jaccard_sets(n_sets=2000, vocab=10000, mean_size=50, n_groups=200, seed=1)
    a, b = synth.minhash_coeffs(256, seed=2)
    jsig = O.minhash(sets, a, b)
    for kind, sig, rows, bands in ((1, csig, 8, 35), (1, csig, 2, 3), (1, csig, 12, 40), (1, csig, 17, 30),
                                   (1, csig, 5, 7), (0, jsig, 8, 32)):
        N = sig.shape[0]
        full = B.blsh_lsh_candidates_workspace(N, kind, rows, bands)
        rec = 64 * N * bands
        outs = []
        for extra in (rec, 0, 4096, rec // 40):
            rc, n, got = gpu_candidates(B, ctx, sig, kind, rows, bands, ws_bytes=full - rec + extra)
            assert rc == 0
            outs.append(got)
        for got in outs[1:]:
            assert np.array_equal(got, outs[0])
        want = O.lsh_candidates(sig, O.JACCARD if kind == 0 else O.COSINE, rows, bands)
        assert len(outs[0]) == len(want) and np.array_equal(sorted_pairs(outs[0]), sorted_pairs(want))
    with pytest.raises(B.BlshError):          # short of the part before the record
        gpu_candidates(B, ctx, csig, 1, 8, 35, ws_bytes=B.blsh_lsh_candidates_workspace(3000, 1, 8, 35)
                       - 64 * 3000 * 35 - 256)


def test_banding_buckets_and_truncation(B, ctx):
    # 300 identical rows (one bucket of 44,850 pairs) plus distinct ones
    sig = np.arange(1000 * 8, dtype=np.uint32).reshape(1000, 8)
    sig[:300] = 5
    want = O.lsh_candidates(sig, O.JACCARD, 4, 2)
    rc, n, got = gpu_candidates(B, ctx, sig, 0, 4, 2)
    assert rc == 0 and n == len(want) == 300 * 299 // 2
    assert np.array_equal(sorted_pairs(got), sorted_pairs(want))
    rc, n, got = gpu_candidates(B, ctx, sig, 0, 4, 2, cap=1000)
    assert rc == B.ETRUNC and n == len(want) and len(got) == 1000
    rc, n, got = gpu_candidates(B, ctx, sig[:1], 0, 4, 2)
    assert rc == 0 and n == 0


def test_lite_jaccard_bit_exact(B, ctx):
    sets = synth.jaccard_sets(n_sets=2000, vocab=10000, mean_size=50, n_groups=200, seed=1)
    a, b = synth.minhash_coeffs(256, seed=2)
    sig = O.minhash(sets, a, b)
    pairs = np.concatenate([O.lsh_candidates(sig, O.JACCARD, 8, 32), synth.random_pairs(2000, 5000, seed=3)])
    p = O.Params(kind=O.JACCARD, n_max=256, h=64, t=0.7)
    want = O.verify_lite(O.tables(p), pairs, sig, sets)
    tab = B.blsh_tables_build(ctx, B.make_params(kind=0, t=0.7, n_max=256, h=64))
    ip, ix, _ = csr_dev(sets)
    P = len(pairs)
    st = torch.zeros(P, dtype=torch.uint8, device=dev)
    sim = torch.full((P,), float('nan'), dtype=torch.float64, device=dev)   # entries not written stay NaN
    nu = torch.zeros(P, dtype=torch.int16, device=dev)
    B.blsh_verify_lite(ctx, tab, t32(pairs), t32(sig), ip, ix, None, st, sim, nu)
    assert B.blsh_status(ctx) == 0
    assert np.array_equal(st.cpu().numpy(), want.status)
    assert np.array_equal(nu.cpu().numpy().view(np.uint16), want.n_used)
    g = sim.cpu().numpy()
    assert np.array_equal(np.isnan(g), np.isnan(want.sim))
    ok = ~np.isnan(g)
    assert np.array_equal(g[ok], want.sim[ok])          # bit-identical doubles
    assert (want.status == O.LITE_ACCEPT).sum() > 50


def test_lite_cosine_bit_exact(B, ctx):
    vecs = synth.tfidf_vectors(n_docs=3000, dim=30000, mean_nnz=80, n_groups=150, seed=5)
    sig = O.srp_sparse(vecs, synth.gaussian_matrix(30000, 256, seed=6))
    pairs = np.concatenate([O.lsh_candidates(sig, O.COSINE, 8, 30), synth.random_pairs(3000, 3000, seed=1)])
    p = O.Params(kind=O.COSINE, n_max=256, h=128, t=0.7)
    want = O.verify_lite(O.tables(p), pairs, sig, vecs)
    tab = B.blsh_tables_build(ctx, B.make_params(kind=1, t=0.7, n_max=256, h=128))
    ip, ix, val = csr_dev(vecs)
    P = len(pairs)
    st = torch.zeros(P, dtype=torch.uint8, device=dev)
    sim = torch.full((P,), float('nan'), dtype=torch.float64, device=dev)   # entries not written stay NaN
    B.blsh_verify_lite(ctx, tab, t32(pairs), t32(sig), ip, ix, val, st, sim)
    assert B.blsh_status(ctx) == 0
    assert np.array_equal(st.cpu().numpy(), want.status)
    g = sim.cpu().numpy()
    ok = ~np.isnan(want.sim)
    assert np.array_equal(np.isnan(g), ~ok)
    assert np.array_equal(g[ok], want.sim[ok])
    assert (want.status == O.LITE_ACCEPT).sum() > 50


def test_lite_cosine_fixed_point_edges(B, ctx):
    """Lite's exact cosine on rows built to exercise the fixed-point products:
    ties at half (1.5 and 2.5 after scaling), negative terms, subnormals,
    products far below 2^-60, rows longer than the shared-memory stage (600
    and 700 terms), and signed unit-norm rows of mixed magnitudes."""
    rng = np.random.default_rng(7)
    rows, vals = [], []
    t = np.float32(2.0 ** -30)
    rows.append(np.arange(8)); vals.append(np.array([1.5 * 2 ** -30, 2.5 * 2 ** -30, -2.5 * 2 ** -30, 3.5 * 2 ** -30,
                                                     1e-40, -3e-39, 0.25, -0.5], np.float32))
    rows.append(np.arange(8)); vals.append(np.array([t, t, t, -t, 1e-38, 2e-38, 1e-20, 0.125], np.float32))
    for n in (600, 700, 40, 90):
        idx = np.sort(rng.choice(1000, n, replace=False))
        v = rng.standard_normal(n) * rng.choice([1e-12, 1e-3, 1.0], n)
        rows.append(idx); vals.append((v / np.linalg.norm(v)).astype(np.float32))   # rows of norm 1
    lens = [len(r) for r in rows]
    csr = synth.CSR(np.concatenate([[0], np.cumsum(lens)]).astype(np.int64), np.concatenate(rows).astype(np.uint32),
                    np.concatenate(vals).astype(np.float32), 1000)
    n_obj = len(rows)
    sig = np.zeros((n_obj, 8), np.uint32)                 # identical signatures: every pair survives pruning
    pairs = np.array([(i, j) for i in range(n_obj) for j in range(i + 1, n_obj)], np.uint32)
    p = O.Params(kind=O.COSINE, n_max=256, h=128, t=0.1)
    want = O.verify_lite(O.tables(p), pairs, sig, csr)
    assert np.all(want.status != O.PRUNED)
    tab = B.blsh_tables_build(ctx, B.make_params(kind=1, t=0.1, n_max=256, h=128))
    ip, ix, val = csr_dev(csr)
    st = torch.zeros(len(pairs), dtype=torch.uint8, device=dev)
    sim = torch.full((len(pairs),), float('nan'), dtype=torch.float64, device=dev)
    B.blsh_verify_lite(ctx, tab, t32(pairs), t32(sig), ip, ix, val, st, sim)
    assert B.blsh_status(ctx) == 0
    assert np.array_equal(st.cpu().numpy(), want.status)
    assert np.array_equal(sim.cpu().numpy(), want.sim)     # bit-identical doubles


def test_lite_survivors_beyond_queue(B, ctx):
    """8.5 million survivors (identical signatures): more than the survivor
    queue holds (2^23), so the rest go through the in-place pass."""
    sets = synth.jaccard_sets(n_sets=3000, vocab=400, mean_size=12, n_groups=300, seed=11)
    sig = np.zeros((sets.n, 64), np.uint32)
    pairs = synth.random_pairs(sets.n, 8_500_000, seed=12)
    p = O.Params(kind=O.JACCARD, n_max=64, h=64, t=0.3)
    want = O.verify_lite(O.tables(p), pairs, sig, sets)
    assert np.all(want.status != O.PRUNED)
    tab = B.blsh_tables_build(ctx, B.make_params(kind=0, t=0.3, n_max=64, h=64))
    ip, ix, _ = csr_dev(sets)
    P = len(pairs)
    st = torch.zeros(P, dtype=torch.uint8, device=dev)
    sim = torch.full((P,), float('nan'), dtype=torch.float64, device=dev)   # entries not written stay NaN
    B.blsh_verify_lite(ctx, tab, t32(pairs), t32(sig), ip, ix, None, st, sim)
    assert B.blsh_status(ctx) == 0
    assert np.array_equal(st.cpu().numpy(), want.status)
    assert np.array_equal(sim.cpu().numpy(), want.sim)


def test_lite_cosine_every_route_with_and_without_norms(B):
    """Lite's exact cosine through every route of the exact pass: rows of up
    to 32 terms (held in registers), up to 512 (staged in shared memory) and
    longer (searched in global memory), paired with each other; 8.5 million
    survivors, so both the queued pass and the in-place pass run; once with
    the rows' squared norms formed once per call (a reserved context: the
    survivors outnumber half the rows) and once formed per pair.
    Bit-identical similarities."""
    rng = np.random.default_rng(21)
    n_obj = 3000
    kind = rng.random(n_obj)
    lens = np.where(kind < 0.7, rng.integers(3, 33, n_obj),
                    np.where(kind < 0.95, rng.integers(33, 513, n_obj), rng.integers(513, 800, n_obj)))
    rows = [np.sort(rng.choice(5000, int(n), replace=False)).astype(np.uint32) for n in lens]
    vals = []
    for n in lens:
        v = rng.standard_normal(int(n)) * rng.choice([1e-6, 1e-2, 1.0], int(n))
        vals.append((v / np.linalg.norm(v)).astype(np.float32))
    csr = synth.CSR(np.concatenate([[0], np.cumsum(lens)]).astype(np.int64), np.concatenate(rows),
                    np.concatenate(vals), 5000)
    sig = np.zeros((n_obj, 8), np.uint32)                 # identical signatures: every pair survives pruning
    pairs = synth.random_pairs(n_obj, 8_500_000, seed=22)
    p = O.Params(kind=O.COSINE, n_max=256, h=128, t=0.05)
    want = O.verify_lite(O.tables(p), pairs, sig, csr)
    assert np.all(want.status != O.PRUNED) and (want.status == O.LITE_ACCEPT).any()
    ip, ix, val = csr_dev(csr)
    P = len(pairs)
    for reserve in (True, False):
        c = B.Context(0)
        if reserve:
            B.blsh_ctx_reserve(c, n_obj)
        tab = B.blsh_tables_build(c, B.make_params(kind=1, t=0.05, n_max=256, h=128))
        st = torch.zeros(P, dtype=torch.uint8, device=dev)
        sim = torch.full((P,), float('nan'), dtype=torch.float64, device=dev)
        B.blsh_verify_lite(c, tab, t32(pairs), t32(sig), ip, ix, val, st, sim)
        assert B.blsh_status(c) == 0
        assert np.array_equal(st.cpu().numpy(), want.status)
        assert np.array_equal(sim.cpu().numpy(), want.sim)


@pytest.mark.parametrize("P", [0, 1, 31, 4097, 1_000_003])
def test_compact_stable_and_exact(B, ctx, P):
    rng = np.random.default_rng(P)
    st = rng.integers(0, 5, P).astype(np.uint8)
    if P > 10:
        st[::7] = 255
    keep = (1 << 1) | (1 << 2) | (1 << 4)
    want = O.compact(st, keep)
    out = torch.full((max(P, 1),), -1, dtype=torch.int64, device=dev)
    n = torch.zeros(1, dtype=torch.int64, device=dev)
    B.blsh_compact(ctx, torch.from_numpy(st).to(dev), keep, out, n)
    assert B.blsh_status(ctx) == 0
    assert int(n.item()) == len(want)
    assert np.array_equal(out[: len(want)].cpu().numpy(), want)
    if len(want) > 3:
        small = torch.zeros(3, dtype=torch.int64, device=dev)
        B.blsh_compact(ctx, torch.from_numpy(st).to(dev), keep, small, n)
        assert B.blsh_status(ctx) == B.ETRUNC
        assert np.array_equal(small.cpu().numpy(), want[:3]) and int(n.item()) == len(want)


def test_srp_sparse_cols_selected_rows(B, ctx):
    """Columns [128, 640) of 2,048 for a third of the rows: those words equal
    the oracle's, every other word keeps its sentinel."""
    vecs = synth.tfidf_vectors(n_docs=900, dim=20000, mean_nnz=80, n_groups=50, seed=31)
    R = synth.gaussian_matrix(20000, 2048, seed=32)
    want = O.srp_sparse(vecs, R)
    ip, ix, val = csr_dev(vecs)
    mask = (np.arange(vecs.n) % 3 == 1).astype(np.uint8)
    sig = torch.full((vecs.n, 64), 0x5A5A5A5A, dtype=torch.int32, device=dev)
    B.blsh_srp_sparse_cols(ctx, ip, ix, val, torch.from_numpy(R).to(dev), sig, 128, 512,
                           row_mask=torch.from_numpy(mask).to(dev))
    assert B.blsh_status(ctx) == 0
    got = sig.cpu().numpy().view(np.uint32)
    sel = mask == 1
    assert np.array_equal(got[sel][:, 4:20], want[sel][:, 4:20])
    assert np.all(got[sel][:, :4] == 0x5A5A5A5A) and np.all(got[sel][:, 20:] == 0x5A5A5A5A)
    assert np.all(got[~sel] == 0x5A5A5A5A)
    # all rows, the whole width in two ranges: the full signatures
    B.blsh_srp_sparse_cols(ctx, ip, ix, val, torch.from_numpy(R).to(dev), sig, 0, 512)
    B.blsh_srp_sparse_cols(ctx, ip, ix, val, torch.from_numpy(R).to(dev), sig, 512, 1536)
    assert B.blsh_status(ctx) == 0
    assert np.array_equal(sig.cpu().numpy().view(np.uint32), want)


@pytest.mark.parametrize("cols", [(0, 384, 1664), (0, 128, 1920), (256, 640, 1152)])
def test_srp_sparse_cols_ragged_rows_and_split_ranges(B, ctx, cols):
    """Rows of 0, 1, 7, 31, 32, 33, 200 and 1,500 nonzeros (the kernel reads
    a row's entries 32 at a time and issues several gathers together), and
    column ranges that take more than one launch (1,664 = 13 x 128 columns):
    bit-exact to the oracle."""
    rng = np.random.default_rng(sum(cols))
    dim, bits = 5000, 2048
    lengths = [0, 1, 7, 31, 32, 33, 200, 1500, 64, 95]
    indptr = np.concatenate([[0], np.cumsum(lengths)]).astype(np.int64)
    indices = np.concatenate([np.sort(rng.choice(dim, n, replace=False)) for n in lengths]).astype(np.uint32)
    values = rng.standard_normal(int(indptr[-1])).astype(np.float32)
    vecs = synth.CSR(indptr, indices, values, dim)
    R = synth.gaussian_matrix(dim, bits, seed=33)
    want = O.srp_sparse(vecs, R)
    ip, ix, val = csr_dev(vecs)
    Rd = torch.from_numpy(R).to(dev)
    sig = torch.full((len(lengths), bits // 32), 0x5A5A5A5A, dtype=torch.int32, device=dev)
    c0, c1, c2 = cols
    B.blsh_srp_sparse_cols(ctx, ip, ix, val, Rd, sig, c0, c1 - c0)
    B.blsh_srp_sparse_cols(ctx, ip, ix, val, Rd, sig, c1, c2)
    assert B.blsh_status(ctx) == 0
    got = sig.cpu().numpy().view(np.uint32)
    w0, w1 = c0 // 32, (c1 + c2) // 32
    assert np.array_equal(got[:, w0:w1], want[:, w0:w1])
    assert np.all(got[:, :w0] == 0x5A5A5A5A) and np.all(got[:, w1:] == 0x5A5A5A5A)
