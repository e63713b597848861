"""GPU parity for the two-byte storage of the projection matrix (Section
4.3): the codes and the sparse projection over them, bit-exact against the
oracle."""
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
    return (torch.from_numpy(csr.indptr).to(dev), t32(csr.indices.astype(np.uint32)),
            torch.from_numpy(csr.values).to(dev))


def test_quantize_bit_exact(B, ctx):
    x = synth.gaussian_matrix(3001, 77, seed=3).ravel()            # ragged length
    x[:6] = [0.0, -2.0 ** -60, 2.0 ** -60, -8.0, 8.0 - 2.0 ** -12, 1.0]
    want, n_out = O.quantize_gaussian(x)
    assert n_out == 0
    q = B.blsh_quantize_gaussian(ctx, torch.from_numpy(x).to(dev))
    assert B.blsh_status(ctx) == 0
    assert np.array_equal(q.cpu().numpy().view(np.uint16), want)


def test_quantize_out_of_range_reported(B, ctx):
    x = np.array([0.5, 8.0, -9.0, np.nan, 3.0], np.float32)
    want, n_out = O.quantize_gaussian(x)
    q = B.blsh_quantize_gaussian(ctx, torch.from_numpy(x).to(dev))
    assert B.blsh_status(ctx) == B.ENUMERIC
    assert B.blsh_status(ctx) == 0
    assert np.array_equal(q.cpu().numpy().view(np.uint16), want) and n_out == 3


@pytest.mark.parametrize("bits", [64, 96, 256, 768, 2048, 4096])
def test_srp_q16_bit_exact(B, ctx, bits):
    vecs = synth.tfidf_vectors(n_docs=700, dim=20000, mean_nnz=80, n_groups=50, seed=bits + 1)
    Rq, _ = O.quantize_gaussian(synth.gaussian_matrix(20000, bits, seed=12))
    want = O.srp_sparse_q16(vecs, Rq)
    ip, ix, val = csr_dev(vecs)
    sig = torch.zeros((vecs.n, bits // 32), dtype=torch.int32, device=dev)
    Rq_d = torch.from_numpy(Rq.view(np.int16)).to(dev)
    B.blsh_srp_sparse_q16(ctx, ip, ix, val, Rq_d, sig)
    assert B.blsh_status(ctx) == 0
    assert np.array_equal(sig.cpu().numpy().view(np.uint32), want)


@pytest.mark.parametrize("n_docs", [3, 1100])
def test_srp_q16_zero_and_cancelling_rows(B, ctx, n_docs):
    """Exactly zero sums (every bit through the FP64 recheck, past the queue's
    capacity for 1100 rows) and sums that cancel to a few ulps."""
    bits = 2048
    rng = np.random.default_rng(n_docs)
    Rq = rng.integers(0, 65536, size=(6, bits), dtype=np.int64).astype(np.uint16)
    Rq[1] = (65536 - Rq[0].astype(np.int64)).clip(0, 65535)        # decodes to -r0 (except at code 0)
    Rq[3] = Rq[2]
    rows, vals = [], []
    for i in range(n_docs):
        if i % 3 == 0:
            rows.append([0, 1]); vals.append([0.5, 0.5])
        elif i % 3 == 1:
            rows.append([2, 3]); vals.append([0.25, -0.25])         # exactly zero
        else:
            rows.append([0, 4, 5]); vals.append([0.3, 0.6, -0.2])
    csr = synth.CSR(np.concatenate([[0], np.cumsum([len(r) for r in rows])]).astype(np.int64),
                    np.concatenate(rows).astype(np.uint32), np.concatenate(vals).astype(np.float32), 6)
    want = O.srp_sparse_q16(csr, Rq)
    ip, ix, val = csr_dev(csr)
    sig = torch.zeros((n_docs, bits // 32), dtype=torch.int32, device=dev)
    B.blsh_srp_sparse_q16(ctx, ip, ix, val, torch.from_numpy(Rq.view(np.int16)).to(dev), sig)
    rc, c = B.blsh_status(ctx, counters=True)
    assert rc == 0
    assert np.array_equal(sig.cpu().numpy().view(np.uint32), want)
    assert c[3] >= (n_docs // 3) * bits


def test_srp_q16_matches_float_path_on_grid_values(B, ctx):
    """The float projection over the decoded matrix gives the same bits."""
    vecs = synth.tfidf_vectors(n_docs=500, dim=8000, mean_nnz=60, seed=14)
    Rq, _ = O.quantize_gaussian(synth.gaussian_matrix(8000, 1024, seed=15))
    R = (Rq.astype(np.float64) / 4096.0 - 8.0).astype(np.float32)
    ip, ix, val = csr_dev(vecs)
    s1 = torch.zeros((vecs.n, 32), dtype=torch.int32, device=dev)
    s2 = torch.zeros_like(s1)
    B.blsh_srp_sparse_q16(ctx, ip, ix, val, torch.from_numpy(Rq.view(np.int16)).to(dev), s1)
    B.blsh_srp_sparse(ctx, ip, ix, val, torch.from_numpy(R).to(dev), s2)
    assert B.blsh_status(ctx) == 0
    assert torch.equal(s1, s2)


@pytest.mark.parametrize("seed,dim,bits", [(0, 1, 8), (1, 777, 2048), (2 ** 63 + 5, 3, 1032)])
def test_gaussian_codes_bit_exact(B, ctx, seed, dim, bits):
    """Codes generated on the device from the counter equal the oracle's."""
    got = B.blsh_gaussian_codes(ctx, seed, dim, bits)
    assert B.blsh_status(ctx) == 0
    assert np.array_equal(got.cpu().numpy().view(np.uint16), O.gaussian_codes(seed, dim, bits))


def test_gaussian_codes_large_sampled(B, ctx):
    """A 2^20 x 2,048 code matrix (4 GB of codes; counters past 2^32): sampled
    rows equal the oracle's, and the decoded values have unit variance."""
    dim, bits, seed = 1 << 20, 2048, 77
    got = B.blsh_gaussian_codes(ctx, seed, dim, bits)
    assert B.blsh_status(ctx) == 0
    for r in (0, 1, 65535, 524287, dim - 1):
        assert np.array_equal(got[r].cpu().numpy().view(np.uint16), O.gaussian_codes(seed, 1, bits, row0=r)[0])
    x = got[::997].cpu().numpy().view(np.uint16).astype(np.float64) / 4096.0 - 8.0
    assert abs(x.var() - 1.0) < 0.01
    del got


def test_srp_q16_on_generated_codes(B, ctx):
    """The sparse projection over device-generated codes equals the oracle's
    over its own codes for the same seed."""
    vecs = synth.tfidf_vectors(n_docs=600, dim=30000, mean_nnz=80, n_groups=40, seed=21)
    Rq = B.blsh_gaussian_codes(ctx, 1234, 30000, 2048)
    want = O.srp_sparse_q16(vecs, O.gaussian_codes(1234, 30000, 2048))
    ip, ix, val = csr_dev(vecs)
    sig = torch.zeros((vecs.n, 64), dtype=torch.int32, device=dev)
    B.blsh_srp_sparse_q16(ctx, ip, ix, val, Rq, sig)
    assert B.blsh_status(ctx) == 0
    assert np.array_equal(sig.cpu().numpy().view(np.uint32), want)


@pytest.mark.parametrize("cols", [(0, 512), (384, 1664), (128, 1024)])
def test_srp_q16_cols_selected_rows(B, ctx, cols):
    """A column range of the two-byte projection for every third row (1,664
    columns take two launches): those words equal the oracle's, the rest keep
    their sentinel."""
    vecs = synth.tfidf_vectors(n_docs=900, dim=20000, mean_nnz=80, n_groups=50, seed=33)
    Rq = O.gaussian_codes(5, 20000, 2048)
    want = O.srp_sparse_q16(vecs, Rq)
    ip, ix, val = csr_dev(vecs)
    mask = (np.arange(vecs.n) % 3 == 1).astype(np.uint8)
    sig = torch.full((vecs.n, 64), 0x5A5A5A5A, dtype=torch.int32, device=dev)
    c0, cn = cols
    B.blsh_srp_sparse_q16_cols(ctx, ip, ix, val, torch.from_numpy(Rq.view(np.int16)).to(dev), sig, c0, cn,
                               row_mask=torch.from_numpy(mask).to(dev))
    assert B.blsh_status(ctx) == 0
    got = sig.cpu().numpy().view(np.uint32)
    sel = mask == 1
    w0, w1 = c0 // 32, (c0 + cn) // 32
    assert np.array_equal(got[sel][:, w0:w1], want[sel][:, w0:w1])
    assert np.all(got[sel][:, :w0] == 0x5A5A5A5A) and np.all(got[sel][:, w1:] == 0x5A5A5A5A)
    assert np.all(got[~sel] == 0x5A5A5A5A)
