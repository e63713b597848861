"""Pins for the oracle's hash families (minhash, Section 4.1; sign random
projections, Section 4.2), LSH banding (Section 2) and the output steps.

Each is checked against a brute-force restatement in Python or numpy and
against the LSH property Pr[h(x) = h(y)] = sim (Eq. lshmain)."""
import math
from collections import defaultdict

import numpy as np
import pytest

import oracle as O
import synth


def test_minhash_brute_force():
    sets = synth.jaccard_sets(n_sets=50, vocab=500, mean_size=20, n_groups=5, seed=1)
    a, b = synth.minhash_coeffs(64, seed=2)
    sig = O.minhash(sets, a, b)
    p = (1 << 31) - 1
    for i in range(sets.n):
        xs = [int(v) for v in sets.row(i)]
        for j in range(64):
            assert sig[i, j] == min((int(a[j]) * x + int(b[j])) % p for x in xs)


def test_minhash_empty_set_and_bijection():
    csr = synth.CSR(np.array([0, 0, 3], np.int64), np.array([5, 6, 2 ** 24 - 1], np.uint32), None, 2 ** 24)
    a, b = synth.minhash_coeffs(16, seed=3)
    sig = O.minhash(csr, a, b)
    assert np.all(sig[0] == 0xFFFFFFFF)
    # h_j is a bijection of [0, p): distinct elements never tie
    x = np.arange(0, 100000, dtype=np.uint64)
    h = (np.uint64(a[0]) * x + np.uint64(b[0])) % np.uint64((1 << 31) - 1)
    assert len(np.unique(h)) == len(x)


def test_minhash_collision_rate_is_jaccard():
    rng = np.random.default_rng(5)
    A = np.sort(rng.choice(100000, 300, replace=False))
    B = np.sort(np.concatenate([A[:200], rng.choice(np.setdiff1d(np.arange(100000), A), 100, replace=False)]))
    J = len(np.intersect1d(A, B)) / len(np.union1d(A, B))
    csr = synth.CSR(np.array([0, len(A), len(A) + len(B)], np.int64), np.concatenate([A, B]).astype(np.uint32),
                    None, 100000)
    a, b = synth.minhash_coeffs(20000, seed=6)
    sig = O.minhash(csr, a, b)
    rate = np.mean(sig[0] == sig[1])
    assert abs(rate - J) < 4 * math.sqrt(J * (1 - J) / 20000) + 0.01


def test_srp_sparse_brute_force_and_dense():
    vecs = synth.tfidf_vectors(n_docs=60, dim=800, mean_nnz=30, n_groups=5, seed=2)
    R = synth.gaussian_matrix(800, 128, seed=3)
    sig = O.srp_sparse(vecs, R)
    dense = np.zeros((60, 800), np.float32)
    for i in range(60):
        ix, v = vecs.row(i)
        dense[i, ix] = v
    dots = dense.astype(np.float64) @ R.astype(np.float64)
    bits = np.unpackbits(sig.view(np.uint8), axis=1, bitorder="little")
    sure = np.abs(dots) > 1e-12
    assert np.array_equal(bits[sure], (dots >= 0)[sure])
    sig_d, dd = O.srp_dense(dense, R, want_dots=True)
    assert np.allclose(dd, dots, atol=1e-12)
    bits_d = np.unpackbits(sig_d.view(np.uint8), axis=1, bitorder="little")
    assert np.array_equal(bits_d[sure], bits[sure])


def test_srp_zero_row_and_bit_layout():
    R = np.array([[1.0, -1.0] * 16], np.float32)         # d = 1, 32 bits
    sig = O.srp_dense(np.array([[0.0], [2.0], [-3.0]], np.float32), R)
    assert sig[0, 0] == 0xFFFFFFFF                       # dot = 0 gives bit 1
    assert sig[1, 0] == 0x55555555                       # bit j of word j/32 at position j%32
    assert sig[2, 0] == 0xAAAAAAAA


def test_srp_collision_rate_is_angle():
    rng = np.random.default_rng(8)
    d = 64
    x = rng.standard_normal(d)
    y = x + 1.2 * rng.standard_normal(d)
    X = np.stack([x, y]).astype(np.float32)
    R = synth.gaussian_matrix(d, 32 * 640, seed=9)
    sig = O.srp_dense(X, R)
    bits = np.unpackbits(sig.view(np.uint8), axis=1, bitorder="little")
    xx, yy = X.astype(np.float64)
    r = 1 - math.acos(xx @ yy / (np.linalg.norm(xx) * np.linalg.norm(yy))) / math.pi
    n = bits.shape[1]
    assert abs(np.mean(bits[0] == bits[1]) - r) < 4 * math.sqrt(r * (1 - r) / n)


@pytest.mark.parametrize("theta_deg", [30, 60, 90, 120])
def test_counter_code_collision_rate_is_angle(theta_deg):
    """Section 4.2's guarantee Pr[h(x) = h(y)] = 1 - theta/pi for the hash
    family the 5e6-vector workload uses: the signs of projections onto the
    decoded two-byte counter codes (Section 4.3 encoding of Irwin-Hall
    samples).  Over 102,400 hashes (25 disjoint blocks of 64 code rows x
    4,096 bits) of a pair at a known angle in 64 dimensions, the collision
    rate lies within binomial 4 sigma of 1 - theta/pi.  A wrong decode offset
    or scale, a dropped sign or a biased sum would move it away."""
    rng = np.random.default_rng(theta_deg)
    d, bits, blocks = 64, 4096, 25
    theta = math.radians(theta_deg)
    x = rng.standard_normal(d)
    x /= np.linalg.norm(x)
    z = rng.standard_normal(d)
    z -= (z @ x) * x
    z /= np.linalg.norm(z)
    y = math.cos(theta) * x + math.sin(theta) * z
    X = np.stack([x, y]).astype(np.float32)
    xx, yy = X.astype(np.float64)
    r = 1 - math.acos(np.clip(xx @ yy / (np.linalg.norm(xx) * np.linalg.norm(yy)), -1, 1)) / math.pi
    csr = synth.CSR(np.array([0, d, 2 * d], np.int64), np.tile(np.arange(d, dtype=np.uint32), 2),
                    X.reshape(-1), d)
    agree = n = 0
    for blk in range(blocks):
        Rq = O.gaussian_codes(17, d, bits, row0=blk * d)
        sig = O.srp_sparse_q16(csr, Rq)
        b = np.unpackbits(sig.view(np.uint8), axis=1, bitorder="little")
        agree += int((b[0] == b[1]).sum())
        n += bits
    assert abs(agree / n - r) < 4 * math.sqrt(r * (1 - r) / n)


def brute_candidates(sig, kind, rows, bands):
    out = set()
    for b in range(bands):
        buckets = defaultdict(list)
        for i in range(sig.shape[0]):
            if kind == O.JACCARD:
                key = tuple(sig[i, b * rows:(b + 1) * rows].tolist())
            else:
                bits = np.unpackbits(sig[i].view(np.uint8), bitorder="little")
                key = tuple(bits[b * rows:(b + 1) * rows].tolist())
            buckets[key].append(i)
        for ids in buckets.values():
            for u in range(len(ids)):
                for v in range(u + 1, len(ids)):
                    out.add((ids[u], ids[v]))
    return sorted(out)


def test_banding_brute_force():
    sets = synth.jaccard_sets(n_sets=400, vocab=600, mean_size=30, n_groups=60, seed=4)
    a, b = synth.minhash_coeffs(64, seed=5)
    sig = O.minhash(sets, a, b)
    got = O.lsh_candidates(sig, O.JACCARD, 4, 16)
    assert [tuple(r) for r in got.tolist()] == brute_candidates(sig, O.JACCARD, 4, 16)
    vecs = synth.tfidf_vectors(n_docs=300, dim=2000, mean_nnz=40, n_groups=40, seed=6)
    sigc = O.srp_sparse(vecs, synth.gaussian_matrix(2000, 128, seed=7))
    got = O.lsh_candidates(sigc, O.COSINE, 8, 10)
    assert len(got) > 100
    assert [tuple(r) for r in got.tolist()] == brute_candidates(sigc, O.COSINE, 8, 10)


def test_banding_edge_cases():
    sig = np.zeros((5, 8), np.uint32)                    # all identical: every pair
    assert len(O.lsh_candidates(sig, O.JACCARD, 8, 1)) == 10
    sig = np.arange(40, dtype=np.uint32).reshape(5, 8)   # all distinct: none
    assert len(O.lsh_candidates(sig, O.JACCARD, 4, 2)) == 0
    assert len(O.lsh_candidates(np.zeros((1, 8), np.uint32), O.JACCARD, 4, 2)) == 0


# ---- two-byte Gaussian storage (Section 4.3) ----

def test_quantize_hand_values():
    x = np.array([0.0, 1.0, -0.5, -8.0, 7.99, 2.0 ** -13, -2.0 ** -60, 2.0 ** -60, 8.0 - 2.0 ** -12], np.float32)
    q, n = O.quantize_gaussian(x)
    # floor((x + 8) * 4096): 32768, 36864, 30720, 0, floor(15.99 * 4096) = 65495 (x is the float
    # nearest 7.99), 32768, 32767 (just below 8 * 4096), 32768, 65535
    want = [32768, 36864, 30720, 0, int(np.floor((np.float64(np.float32(7.99)) + 8) * 4096)), 32768, 32767,
            32768, 65535]
    assert q.tolist() == want and n == 0


def test_quantize_clamps_and_counts():
    q, n = O.quantize_gaussian(np.array([8.0, -8.5, 100.0, np.nan, -1e30], np.float32))
    assert q.tolist() == [65535, 0, 65535, 0, 0] and n == 5


def test_quantize_error_bound_brute_force():
    """Each value decodes to the grid point at or just below it: 0 <= x - r < 2^-12."""
    x = np.random.default_rng(0).standard_normal(200000).astype(np.float32)
    q, n = O.quantize_gaussian(x)
    assert n == 0
    grid = q.astype(np.float64) / 4096.0 - 8.0
    d = x.astype(np.float64) - grid
    assert d.min() >= 0.0 and d.max() < 2.0 ** -12
    assert np.array_equal(O.dequantize_gaussian(q[:1000]), grid[:1000])


def test_srp_q16_exact_sign_brute_force():
    """The two-byte projection's bits against exactly rounded sums (fsum) of
    the decoded products, wherever the sum is not within a rounding of 0."""
    vecs = synth.tfidf_vectors(n_docs=60, dim=500, mean_nnz=30, seed=8)
    Rq, _ = O.quantize_gaussian(synth.gaussian_matrix(500, 64, seed=9))
    sig = O.srp_sparse_q16(vecs, Rq)
    checked = 0
    for i in range(vecs.n):
        s, e = vecs.indptr[i], vecs.indptr[i + 1]
        for j in range(64):
            terms = [float(vecs.values[k]) * (int(Rq[vecs.indices[k], j]) / 4096.0 - 8.0) for k in range(s, e)]
            exact = math.fsum(terms)
            if abs(exact) > 1e-12 * (sum(abs(t) for t in terms) + 1e-300):
                assert ((int(sig[i, j // 32]) >> (j % 32)) & 1) == (exact >= 0.0)
                checked += 1
    assert checked > 0.99 * vecs.n * 64


def test_srp_q16_matches_float_path_on_grid_values():
    """R whose entries lie on the two-byte grid: the float projection of the
    decoded matrix and the two-byte projection are the same function."""
    vecs = synth.tfidf_vectors(n_docs=200, dim=3000, mean_nnz=40, seed=10)
    Rq, _ = O.quantize_gaussian(synth.gaussian_matrix(3000, 128, seed=11))
    R = (Rq.astype(np.float64) / 4096.0 - 8.0).astype(np.float32)
    assert np.array_equal(R.astype(np.float64), Rq.astype(np.float64) / 4096.0 - 8.0)   # exact in float32
    assert np.array_equal(O.srp_sparse_q16(vecs, Rq), O.srp_sparse(vecs, R))


# ---- counter-generated two-byte Gaussian codes (Section 4.3 storage) ----

def test_splitmix64_published_outputs():
    """The first outputs of SplitMix64 from seed 0, as published with the
    generator's reference code."""
    want = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F, 0xF88BB8A8724C81EC]
    assert [O.splitmix64_at(0, k) for k in range(4)] == want


def test_gaussian_code_of_the_first_entry_by_hand():
    """Entry (0, 0) of seed 0 uses the first three published outputs: the sum
    of their twelve 16-bit pieces, centred and floored onto the 1/4096 grid
    of the two-byte encoding."""
    outs = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    S = sum((o >> (16 * h)) & 0xFFFF for o in outs for h in range(4))
    assert S == 397544
    code = (S - 393210) // 16 + 32768          # floor((x + 8) 2^16 / 16), x = (S - 393210) / 2^16
    assert code == 33038
    assert O.gaussian_codes(0, 1, 32)[0, 0] == code


def test_gaussian_codes_are_standard_normal_to_irwin_hall_accuracy():
    """Decoded values of a million codes: mean (the floor onto the grid
    shifts it by 7.5/16 of a step), variance 1, excess kurtosis -0.1 (the
    Irwin-Hall sum of twelve uniforms), no correlation between neighbours,
    everything inside +-6."""
    q = O.gaussian_codes(12345, 500, 2048)
    x = q.astype(np.float64) / 4096.0 - 8.0
    n = x.size
    assert abs(x.mean() - (-7.5 / 16 / 4096)) < 5.0 / np.sqrt(n)
    var = x.var()
    assert abs(var - 1.0) < 0.01
    kurt = ((x - x.mean()) ** 4).mean() / var ** 2 - 3.0
    assert abs(kurt - (-0.1)) < 0.03
    flat = x.ravel()
    assert abs(np.corrcoef(flat[:-1], flat[1:])[0, 1]) < 0.005
    assert q.min() >= 8192 and q.max() <= 57343


def test_gaussian_codes_depend_on_seed_and_position_only():
    a = O.gaussian_codes(7, 40, 128)
    assert np.array_equal(a, O.gaussian_codes(7, 40, 128))
    assert np.array_equal(a[:10, :64], O.gaussian_codes(7, 10, 128)[:, :64])
    assert (a != O.gaussian_codes(8, 40, 128)).mean() > 0.99


def test_gaussian_code_rows_from_any_offset():
    whole = O.gaussian_codes(99, 30, 64)
    assert np.array_equal(O.gaussian_codes(99, 7, 64, row0=11), whole[11:18])
