"""Host-side logic of bench.py without a GPU: the algorithmic-byte model the
roofline divides by, and the lazy-hashing prefix rule."""
import types

import numpy as np
import pytest
import torch

import bench
import paper_1110_1328_gb300 as B
import synth


def test_csr_rows_bytes_by_hand():
    # rows {0: [1, 3], 1: [3], 2: []} over 4 terms, 128 columns of float R
    indptr = np.array([0, 2, 3, 3], np.int64)
    indices = np.array([1, 3, 3], np.uint32)
    # 3 nonzeros (8 B each), 3 rows (16 B + 16 B of signature each), 2 distinct terms x 512 B
    assert bench.csr_rows_bytes(indptr, indices, None, 128, 4) == 3 * 8 + 3 * (16 + 16) + 2 * 512
    # only row 1: one nonzero, one row, one distinct term
    mask = np.array([False, True, False])
    assert bench.csr_rows_bytes(indptr, indices, mask, 128, 4) == 8 + (16 + 16) + 512
    # two-byte codes halve the R bytes
    assert bench.csr_rows_bytes(indptr, indices, None, 128, 2) == 3 * 8 + 3 * 32 + 2 * 256


def _fake_pipe(w, P, lazy):
    rng = np.random.default_rng(0)
    return types.SimpleNamespace(P=P, N=w["n"], lazy_bits=lazy, with_lite=True, dense=False,
                                 pairs=torch.from_numpy(rng.integers(0, w["n"], (P, 2)).astype(np.int32)))


def test_kernel_work_covers_every_timed_kernel_of_a_cosine_step():
    w = dict(bench.WORKLOADS["cosine-small"], n=500)
    objs = synth.tfidf_vectors(n_docs=500, dim=5000, mean_nnz=40, n_groups=20, seed=1)
    P = 10_000
    rng = np.random.default_rng(1)
    st = rng.integers(0, 4, P).astype(np.uint8)
    nu = (rng.integers(4, 64, P) * 32).astype(np.uint16)
    lst = rng.integers(0, 4, P).astype(np.uint8)
    need = rng.random(500) < 0.1
    work = bench.kernel_work(B, _fake_pipe(w, P, 512), w, objs, st, nu, lst, need)
    for k in ("srp_sparse4_kernel", "verify_kernel", "verify_resume_kernel", "emit_warp_kernel (count pass)",
              "emit_warp_kernel (write pass)", "digit_scatter_kernel", "compact_write", "lite_queue_kernel"):
        assert work[k][1] == "B" and work[k][0] > 0
    # the resume kernel reads the chunks of the open pairs only; the capped
    # kernel at most lazy_bits / k chunks of each pair
    capped = np.minimum(nu.astype(np.int64), 512) // 32
    assert work["verify_kernel"][0] >= int(capped.sum()) * 8
    # gathered bytes of the two SRP launches: every nonzero's row slice
    nnz_rows = np.diff(objs.indptr)
    want = int(nnz_rows.sum()) * 512 * 4 + int(nnz_rows[need].sum()) * (2048 - 512) * 4
    assert work["srp_sparse4_kernel gathered"][0] == want


def test_lazy_prefix_must_cover_the_banded_hashes():
    prop = bench.Pipeline.lazy_bits.fget
    w = dict(bench.WORKLOADS["cosine-small"])                 # 8 x 35 bands read 280 bits
    ok = types.SimpleNamespace(w=dict(w, lazy_bits=512), kind=1, dense=False, with_lite=True)
    assert prop(ok) == 512
    assert prop(types.SimpleNamespace(w=dict(w, lazy_bits=0), kind=1, dense=False, with_lite=True)) == 0
    assert prop(types.SimpleNamespace(w=dict(w, lazy_bits=2048), kind=1, dense=False, with_lite=True)) == 0
    with pytest.raises(ValueError):
        prop(types.SimpleNamespace(w=dict(w, lazy_bits=256), kind=1, dense=False, with_lite=True))
    # no lazy hashing without the fused Lite pass, for dense rows or two-byte R
    assert prop(types.SimpleNamespace(w=dict(w, lazy_bits=512), kind=1, dense=False, with_lite=False)) == 0
    assert prop(types.SimpleNamespace(w=dict(w, lazy_bits=512), kind=1, dense=True, with_lite=True)) == 0


def _recorded_names():
    """Kernel names the library gives its timing records (the strings passed
    to BLSH_LAUNCHED / blsh_time_stop, directly or through a name variable)."""
    import os
    import re
    root = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_1110_1328_gb300", "csrc")
    names = set()
    for f in os.listdir(root):
        if f.endswith((".cu", ".cuh")):
            src = open(os.path.join(root, f)).read()
            for call in re.findall(r"(?:BLSH_LAUNCHED|blsh_time_stop)\(ctx, ([^;]*)\);", src):
                names.update(re.findall(r'"([^"]+)"', call))
            names.update(re.findall(r'const char \*name = [^;]*?"([^"]+)"', src))
            names.update(re.findall(r'const char \*name = [^;]*?: "([^"]+)"', src))
    return names


@pytest.mark.parametrize("workload", ["cosine-small", "cosine-small-q16", "jaccard-small", "allpairs-cosine"])
def test_modelled_kernels_are_the_recorded_ones(workload):
    """Every kernel the byte model names is a name the library records, so
    the roofline finds its bytes."""
    w = dict(bench.WORKLOADS[workload])
    if w["kind"] == 1:
        w["n"] = 300
        objs = synth.tfidf_vectors(n_docs=300, dim=3000, mean_nnz=30, n_groups=10, seed=2)
    else:
        w["n"] = 300
        objs = synth.jaccard_sets(n_sets=300, vocab=2000, mean_size=20, n_groups=10, seed=2)
    P = 1000
    rng = np.random.default_rng(0)
    st = rng.integers(0, 4, P).astype(np.uint8)
    nu = (rng.integers(1, 8, P) * w["k"]).astype(np.uint16)
    lst = rng.integers(0, 4, P).astype(np.uint8)
    pipe = _fake_pipe(w, P, 512 if workload == "cosine-small" else 0)
    pipe.with_lite = "lite" in w.get("stages", ("lite",))
    if w.get("candidates") == "allpairs":
        pipe.allpairs, pipe.nnz, pipe.dim, pipe.max_dups = True, int(objs.indptr[-1]), objs.dim, 5 * P
    work = bench.kernel_work(B, pipe, w, objs, st, nu, lst, rng.random(300) < 0.1)
    names = _recorded_names()
    missing = [k for k in work if not k.endswith(" gathered") and k not in names]
    assert not missing, missing


def _fake_large_pipe(n_docs=3000, P=20_000, lazy=512, seed=3, n_groups=200):
    """A stand-in for bench.LargePipeline on the CPU: the workload's generator
    at a small size, random candidate pairs and random per-pair outputs."""
    w = dict(bench.WORKLOADS["large-mixed"], n=n_docs, dim=1 << 16, lazy_bits=lazy)
    indptr, indices, values = synth.large_tfidf_device(n_docs=n_docs, dim=1 << 16, nnz_min=5, nnz_max=400,
                                                       n_groups=n_groups, seed=seed, device=torch.device("cpu"))
    rng = np.random.default_rng(seed)
    pr = np.sort(rng.integers(0, n_docs, (P, 2)), axis=1).astype(np.int32)
    levels = w["n_max"] // w["k"]
    pipe = types.SimpleNamespace(
        torch=torch, B=B, w=w, dev=torch.device("cpu"), indptr=indptr, indices=indices, values=values, N=n_docs,
        nnz=int(indptr[-1]), P=P, bits=w["bits"], lazy_bits=lazy, pairs=torch.from_numpy(pr), ranges=[(0, P)],
        status=torch.from_numpy(rng.integers(0, 3, P).astype(np.uint8)),
        n_used=torch.from_numpy((rng.integers(1, levels + 1, P) * w["k"]).astype(np.int16)),
        lstatus=torch.from_numpy(rng.choice([0, 3, 4], P).astype(np.uint8)),
        need=torch.from_numpy((rng.random(n_docs) < 0.2).astype(np.uint8)))
    return w, pipe


def test_large_kernel_work_by_hand():
    w, pipe = _fake_large_pipe()
    work = bench.large_kernel_work(pipe)
    L, bits, k = 512, w["bits"], w["k"]
    nu = pipe.n_used.numpy().astype(np.int64)
    st = pipe.status.numpy()
    kept = (st == B.ACCEPT) | (st == B.ACCEPT_AT_MAX)
    resumed = nu > L
    want_v = pipe.P * 14 + 4 * int((kept & ~resumed).sum()) + int(np.minimum(nu // k, L // k).sum()) * (k // 4)
    assert work["verify_kernel"] == (want_v, "B")
    want_r = pipe.P + int(resumed.sum()) * 13 + 4 * int((kept & resumed).sum()) + int((nu[resumed] // k).sum()) * 8
    assert work["verify_resume_kernel"] == (want_r, "B")
    # projection: the prefix of every row, the rest of the rows marked in need
    ip, ix = pipe.indptr.numpy(), pipe.indices.numpy()
    need = pipe.need.numpy().astype(bool)
    sel = np.concatenate([np.arange(ip[i], ip[i + 1]) for i in np.flatnonzero(need)])
    want_p = (pipe.nnz * 8 + pipe.N * (16 + L // 8) + len(np.unique(ix)) * L * 2
              + len(sel) * 8 + int(need.sum()) * (16 + (bits - L) // 8) + len(np.unique(ix[sel])) * (bits - L) * 2)
    assert work["srp_sparse4_kernel (two-byte codes)"] == (want_p, "B")
    for name in ("lite_queue_kernel", "emit_warp_kernel (write pass)", "compact_write", "band_keys_kernel"):
        assert work[name][0] > 0


def test_large_oracle_sample_times_and_extrapolation():
    """The cpu_baseline leg's sampling on a small stand-in: the oracle's inputs
    come from the sampled rows (terms renumbered, its own codes), the timings
    are positive, and the extrapolation scales each part by its own unit."""
    import oracle as O
    w, pipe = _fake_large_pipe(n_docs=600, P=3000, n_groups=50)
    w = dict(w, bits=256, n_max=256, h=128)
    inp = bench.large_oracle_inputs(pipe, w, seed=1, n_pairs=500, n_hash=100, threads=2)
    assert inp["hash_csr"].n == 100 and len(inp["pairs"]) == 500
    assert inp["pair_sig"].shape == (inp["pair_csr"].n, 8)
    t1 = bench.large_oracle_times(O, w, inp, threads=1, min_verify_s=0.0)
    t2 = bench.large_oracle_times(O, w, inp, threads=2, min_verify_s=0.0)
    for t in (t1, t2):
        assert t["hash_s"] > 0 and t["verify_s"] > 0 and t["pairs"] == 500 and t["objects"] == 100
    T = bench.extrapolate({"hash_s": 2.0, "band_s": 1.0, "verify_s": 3.0, "nnz": 10, "objects": 5, "pairs": 30},
                          N=50, nnz=100, P=300)
    assert T == 100 * 0.2 + 50 * 0.2 + 300 * 0.1
