"""GPU parity at the benchmark's full sizes, in the launch configuration
bench.py times (its Pipeline: the autotuned verification plan, device-side
pair counts, and a CUDA-graph replay of the whole step).

cosine-small (20,000 tf-idf vectors, 2,048 SRP bits, ~2.7e7 candidate pairs)
and jaccard-small (2,000 sets, 256 minhashes) are compared with the oracle in
full: signatures, the candidate set, every pair's Algorithm 1 and Algorithm 2
outcome, and both output sets.  The 1,000,000-node Chung-Lu workload, the
1,000,000-point dense workload and the 5,000,000-vector mixed workload (also
streamed in several batches with its checkpoint record) are compared on
samples the oracle computes one by one, plus properties that hold at any
size."""
import numpy as np
import pytest
import torch

import bench
import oracle as O
import synth

pytestmark = pytest.mark.gpu


def u32(t):
    return t.cpu().numpy().view(np.uint32)


def run_pipeline(B, name, graph=True):
    w = dict(bench.WORKLOADS[name])
    objs, hashp = bench.make_inputs(w)
    pipe = bench.Pipeline(B, torch, w, objs, hashp, torch.device("cuda", 0))
    if graph:
        g = torch.cuda.CUDAGraph()
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            pipe.step()
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        with torch.cuda.graph(g):
            pipe.step()
        # poison the outputs, then replay: the graph must recompute everything
        pipe.status.fill_(77)
        pipe.lstatus.fill_(77)
        pipe.sig.fill_(0)
        pipe.need.fill_(0)
        g.replay()
    else:
        pipe.step()
    torch.cuda.synchronize()
    assert B.blsh_status(pipe.ctx) == 0
    return w, objs, hashp, pipe


def check_outputs_against_oracle(B, w, objs, pipe, sig_o, pairs_gpu):
    P = len(pairs_gpu)
    p = O.Params(kind=w["kind"], t=w["t"], k=w["k"], n_max=w["n_max"], h=w["h"])
    tab = O.tables(p)
    want = O.verify(tab, pairs_gpu, sig_o)
    assert want.bad == 0
    assert np.array_equal(pipe.status[:P].cpu().numpy(), want.status)
    assert np.array_equal(pipe.n_used[:P].cpu().numpy().view(np.uint16), want.n_used)
    assert np.array_equal(pipe.m[:P].cpu().numpy().view(np.uint16), want.m)
    # estimates are outputs of kept pairs only (the entries of pruned pairs
    # are not written, and the pipeline's buffers are reused across calls)
    est = pipe.est[:P].cpu().numpy()
    ok = ~np.isnan(want.est)
    assert not np.isnan(est[ok]).any()
    assert np.max(np.abs(est[ok] - want.est[ok]), initial=0) <= 1e-6
    assert np.array_equal(pipe.hist.cpu().numpy(), O.stop_hist(want.n_used, p.k, p.levels).astype(np.int64))
    lite = O.verify_lite(tab, pairs_gpu, sig_o, objs)
    assert np.array_equal(pipe.lstatus[:P].cpu().numpy(), lite.status)
    sim = pipe.sim[:P].cpu().numpy()
    ok = ~np.isnan(lite.sim)   # survivors only
    assert np.array_equal(sim[ok], lite.sim[ok])
    n1, n2 = [int(x) for x in pipe.n_out.cpu()]
    keep1 = O.compact(want.status, (1 << O.ACCEPT) | (1 << O.ACCEPT_AT_MAX))
    keep2 = O.compact(lite.status, 1 << O.LITE_ACCEPT)
    assert (n1, n2) == (len(keep1), len(keep2))
    assert np.array_equal(pipe.out1[:n1].cpu().numpy(), keep1)
    assert np.array_equal(pipe.out2[:n2].cpu().numpy(), keep2)
    return want, lite


@pytest.mark.parametrize("name", ["jaccard-small", "cosine-small"])
def test_full_pipeline_matches_oracle(B, name):
    w, objs, hashp, pipe = run_pipeline(B, name)
    if w["kind"] == 1:
        sig_o = O.srp_sparse(objs, hashp)
    else:
        sig_o = O.minhash(objs, hashp[0], hashp[1])
    if pipe.lazy_bits:
        # lazy hashing: the first lazy_bits hashes of every object, all of them
        # for the objects of pairs that needed more (and at least some did)
        lw = pipe.lazy_bits // 32
        need = pipe.need.cpu().numpy() == 1
        assert need.any()
        assert np.array_equal(u32(pipe.sig)[:, :lw], sig_o[:, :lw])
        assert np.array_equal(u32(pipe.sig)[need], sig_o[need])
    else:
        assert np.array_equal(u32(pipe.sig), sig_o)
    pairs_o = O.lsh_candidates(sig_o, w["kind"], w["rows"], w["bands"])
    P = pipe.P
    pairs_gpu = u32(pipe.pairs[:P])
    assert P == len(pairs_o)
    key = lambda a: np.sort((a[:, 0].astype(np.uint64) << np.uint64(32)) | a[:, 1])
    assert np.array_equal(key(pairs_gpu), key(pairs_o))
    want, lite = check_outputs_against_oracle(B, w, objs, pipe, sig_o, pairs_gpu)
    assert (want.status == O.PRUNED).any() and (want.status != O.PRUNED).any()
    assert (lite.status == O.LITE_ACCEPT).sum() > 10


def test_allpairs_pipeline_matches_oracle(B):
    """cosine-small's vectors with candidates from the AllPairs-style prefix
    filter instead of banding, in bench's launch configuration (CUDA-graph
    replay): the candidate list equal to the oracle's, pair for pair and in
    order, and every pair's Algorithm 1 and 2 outcome and both output sets
    equal to the oracle's."""
    w, objs, hashp, pipe = run_pipeline(B, "allpairs-cosine")
    sig_o = O.srp_sparse(objs, hashp)
    pairs_o = O.allpairs_candidates(objs, w["t"], O.COSINE)
    P = pipe.P
    assert P == len(pairs_o) and P > 1_000_000
    pairs_gpu = u32(pipe.pairs[:P])
    assert np.array_equal(pairs_gpu, pairs_o)
    want, lite = check_outputs_against_oracle(B, w, objs, pipe, sig_o, pairs_gpu)
    assert (lite.status == O.LITE_ACCEPT).sum() > 10


def test_batching_workload_sampled(B):
    """1,000,000 Chung-Lu adjacency sets, ~1e8 candidate pairs: sampled
    oracle checks (signature rows, pairs' outcomes) and properties of the
    candidate set."""
    w, objs, hashp, pipe = run_pipeline(B, "batching", graph=False)
    P = pipe.P
    assert P > 1_000_000
    rng = np.random.default_rng(0)
    # signature rows: oracle minhash of 3,000 random rows
    rows = np.sort(rng.choice(objs.n, 3000, replace=False))
    sub = synth.CSR(np.concatenate([[0], np.cumsum(np.diff(objs.indptr)[rows])]).astype(np.int64),
                    np.concatenate([objs.row(int(i)) for i in rows]).astype(np.uint32), None, objs.dim)
    sig_sub = O.minhash(sub, hashp[0], hashp[1])
    assert np.array_equal(u32(pipe.sig[torch.from_numpy(rows).cuda()]), sig_sub)
    # sampled pairs: every outcome recomputed by the oracle from its own hashes
    pairs = u32(pipe.pairs[:P])
    q = np.sort(rng.choice(P, 20000, replace=False))
    sp = pairs[q]
    assert np.all(sp[:, 0] < sp[:, 1])
    ids, inv = np.unique(sp.reshape(-1), return_inverse=True)
    sub = synth.CSR(np.concatenate([[0], np.cumsum(np.diff(objs.indptr)[ids])]).astype(np.int64),
                    np.concatenate([objs.row(int(i)) for i in ids]).astype(np.uint32), None, objs.dim)
    sig_o = O.minhash(sub, hashp[0], hashp[1])
    local = inv.reshape(-1, 2).astype(np.uint32)
    # each sampled pair collides on a whole band of the oracle's hashes
    r, bands = w["rows"], w["bands"]
    band_eq = np.stack([(sig_o[local[:, 0], b * r:(b + 1) * r] == sig_o[local[:, 1], b * r:(b + 1) * r]).all(1)
                        for b in range(bands)], 1)
    assert band_eq.any(1).all()
    p = O.Params(kind=0, t=w["t"], k=w["k"], n_max=w["n_max"], h=w["h"])
    tab = O.tables(p)
    want = O.verify(tab, local, sig_o)
    assert np.array_equal(pipe.status[:P].cpu().numpy()[q], want.status)
    assert np.array_equal(pipe.m[:P].cpu().numpy().view(np.uint16)[q], want.m)
    lite = O.verify_lite(tab, local, sig_o, sub)
    assert np.array_equal(pipe.lstatus[:P].cpu().numpy()[q], lite.status)
    sim = pipe.sim[:P].cpu().numpy()[q]
    ok = ~np.isnan(lite.sim)
    assert np.array_equal(sim[ok], lite.sim[ok])
    # the candidate list has no duplicates
    key = np.sort((pairs[:, 0].astype(np.uint64) << np.uint64(32)) | pairs[:, 1])
    assert np.all(np.diff(key) > 0)
    # stop histogram and status counts agree
    st = pipe.status[:P].cpu().numpy()
    assert int(pipe.hist.sum()) == P and not np.any(st == 77)


def test_precision_workload_sampled(B):
    """1,000,000 dense 256-d embeddings, 1,024 bits by the tensor-core
    projection, about 6e8 candidate pairs: sampled signature rows bit-exact
    to the oracle's FP64 signs, sampled pairs' outcomes recomputed by the
    oracle, and the candidate list free of duplicates."""
    w, objs, R, pipe = run_pipeline(B, "precision", graph=False)
    P = pipe.P
    assert P > 100_000_000
    rng = np.random.default_rng(1)
    rows = np.sort(rng.choice(objs.n, 2000, replace=False))
    assert np.array_equal(u32(pipe.sig[torch.from_numpy(rows).cuda()]), O.srp_dense(objs.X[rows], R))
    q = np.sort(rng.choice(P, 4000, replace=False))
    sp = u32(pipe.pairs[torch.from_numpy(q).cuda()])
    assert np.all(sp[:, 0] < sp[:, 1])
    ids, inv = np.unique(sp.reshape(-1), return_inverse=True)
    sig_o = O.srp_dense(objs.X[ids], R)
    local = inv.reshape(-1, 2).astype(np.uint32)
    r, bands = w["rows"], w["bands"]

    def band_bits(s, b):
        return (s[:, (b * r) // 32] >> np.uint32((b * r) % 32)) & np.uint32((1 << r) - 1)

    band_eq = np.stack([band_bits(sig_o[local[:, 0]], b) == band_bits(sig_o[local[:, 1]], b) for b in range(bands)], 1)
    assert band_eq.any(1).all()
    p = O.Params(kind=1, t=w["t"], k=w["k"], n_max=w["n_max"], h=w["h"])
    want = O.verify(O.tables(p), local, sig_o)
    qd = torch.from_numpy(q).cuda()
    assert np.array_equal(pipe.status[qd].cpu().numpy(), want.status)
    assert np.array_equal(pipe.m[qd].cpu().numpy().view(np.uint16), want.m)
    est = pipe.est[qd].cpu().numpy()
    ok = ~np.isnan(want.est)   # kept pairs only
    assert np.max(np.abs(est[ok] - want.est[ok]), initial=0) <= 1e-6
    # no duplicates (sorted on the device: object ids are below 2^31)
    dp = pipe.pairs[:P].long()
    key, _ = torch.sort((dp[:, 0] << 32) | dp[:, 1])
    assert bool((key[1:] > key[:-1]).all())


@pytest.fixture(scope="module")
def large_pipe(B):
    """The 5e6-vector mixed workload in bench's launch configuration: one
    batch, lazy hashing, the autotuned plan, one CUDA-graph replay of the
    whole step after its outputs were poisoned."""
    w = dict(bench.WORKLOADS["large-mixed"])
    dev = torch.device("cuda", 0)
    pipe = bench.LargePipeline(B, torch, w, dev)
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        pipe.step()
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    with torch.cuda.graph(g):
        pipe.step()
    pipe.status.fill_(77)
    pipe.lstatus.fill_(77)
    pipe.sig.fill_(0)
    pipe.n_out.fill_(-1)
    g.replay()
    torch.cuda.synchronize()
    assert B.blsh_status(pipe.ctx) == 0
    yield w, pipe
    del g


def large_oracle_view(pipe, w, ids):
    """The sampled objects' rows with their terms renumbered 0..T-1, and the
    oracle's own codes for those terms."""
    dev = pipe.dev
    indptr = pipe.indptr.cpu().numpy()
    rows = [np.arange(indptr[i], indptr[i + 1]) for i in ids]
    sel = torch.from_numpy(np.concatenate(rows)).to(dev)
    terms = pipe.indices[sel].cpu().numpy().view(np.uint32)
    vals = pipe.values[sel].cpu().numpy()
    uterm, tinv = np.unique(terms, return_inverse=True)
    local = synth.CSR(np.concatenate([[0], np.cumsum([len(r) for r in rows])]).astype(np.int64),
                      tinv.astype(np.uint32), vals, len(uterm))
    Rq = np.stack([O.gaussian_codes(w["r_seed"], 1, w["bits"], row0=int(t))[0] for t in uterm])
    return local, Rq


def test_large_mixed_workload_sampled(B, large_pipe):
    """5,000,000 tf-idf vectors over a 2^24-term vocabulary, R generated on
    the device as two-byte codes (68.7 GB), about 1e9 candidates verified by
    Algorithms 1 and 2 with lazy hashing (the first 256 bits of every object,
    the rest of the objects of the pairs left open): sampled pairs' outcomes
    of both algorithms recomputed by the oracle from its own full signatures,
    sampled signature rows bit-exact (the prefix of every row, and all bits
    of the rows the step hashed in full), every sampled pair colliding in a
    band, the candidate list free of duplicates, and the kept counts equal to
    the statuses."""
    w, pipe = large_pipe
    dev = pipe.dev
    P, L = pipe.P, pipe.lazy_bits
    assert P > 100_000_000 and len(pipe.ranges) == 1 and pipe.batch >= P and 0 < L < w["bits"]
    rng = np.random.default_rng(3)
    q = np.sort(rng.choice(P, 3000, replace=False))
    qd = torch.from_numpy(q).to(dev)
    sp = u32(pipe.pairs[qd])
    assert np.all(sp[:, 0] < sp[:, 1])
    # pairs the lazy prefix left open, so that the resumed path is covered
    open_q = torch.nonzero(pipe.n_used[:P].to(torch.int64) & 0xFFFF > L).flatten()
    assert open_q.numel() > 0
    extra_q = open_q[torch.randperm(open_q.numel(), device=dev)[:500]].sort().values.cpu().numpy()
    q = np.union1d(q, extra_q)
    qd = torch.from_numpy(q).to(dev)
    sp = u32(pipe.pairs[qd])
    extra = rng.choice(pipe.N, 300, replace=False)
    ids, inv = np.unique(np.concatenate([sp.reshape(-1), extra]), return_inverse=True)
    local, Rq = large_oracle_view(pipe, w, ids)
    sig_o = O.srp_sparse_q16(local, Rq)
    ids_d = torch.from_numpy(ids).to(dev)
    got = u32(pipe.sig[ids_d])
    pw = L // 32
    assert np.array_equal(got[:, :pw], sig_o[:, :pw])                 # every object's prefix
    full = pipe.need[ids_d].cpu().numpy().astype(bool)
    assert full.any() and np.array_equal(got[full], sig_o[full])     # the rows hashed in full
    lp = inv[: 2 * len(q)].reshape(-1, 2).astype(np.uint32)
    r, bands = w["rows"], w["bands"]

    def band_bits(s, b):
        return (s[:, (b * r) // 32] >> np.uint32((b * r) % 32)) & np.uint32((1 << r) - 1)

    band_eq = np.stack([band_bits(sig_o[lp[:, 0]], b) == band_bits(sig_o[lp[:, 1]], b) for b in range(bands)], 1)
    assert band_eq.any(1).all()
    p = O.Params(kind=1, t=w["t"], k=w["k"], n_max=w["n_max"], h=w["h"])
    tab = O.tables(p)
    want = O.verify(tab, lp, sig_o)
    assert np.array_equal(pipe.status[qd].cpu().numpy(), want.status)
    assert np.array_equal(pipe.n_used[qd].cpu().numpy().view(np.uint16), want.n_used)
    assert np.array_equal(pipe.m[qd].cpu().numpy().view(np.uint16), want.m)
    est = pipe.est[qd].cpu().numpy()
    ok = ~np.isnan(want.est)
    assert np.max(np.abs(est[ok] - want.est[ok]), initial=0) <= 1e-6
    lite = O.verify_lite(tab, lp, sig_o, local)
    assert np.array_equal(pipe.lstatus[qd].cpu().numpy(), lite.status)
    sim = pipe.sim[qd].cpu().numpy()
    ok = ~np.isnan(lite.sim)
    assert np.array_equal(sim[ok], lite.sim[ok])
    # each distinct pair once (sorted on the device)
    dp = pipe.pairs[:P].long()
    key, _ = torch.sort((dp[:, 0] << 32) | dp[:, 1])
    assert bool((key[1:] > key[:-1]).all())
    del key, dp
    # the kept counts and output sets are those of the statuses
    st = pipe.status[:P]
    k1 = torch.nonzero((st == B.ACCEPT) | (st == B.ACCEPT_AT_MAX)).flatten()
    k2 = torch.nonzero(pipe.lstatus[:P] == B.LITE_ACCEPT).flatten()
    assert pipe.kept_counts() == [k1.numel(), k2.numel()]
    assert torch.equal(pipe.out1[: k1.numel()], k1) and torch.equal(pipe.out2[: k2.numel()], k2)
    # the stop histogram counts every pair once
    assert int(pipe.hist.sum().item()) == P


def test_large_mixed_streamed_in_batches(B, large_pipe, tmp_path):
    """The same candidates verified in several device batches (a cap below
    P), eagerly with the checkpoint record, interrupted while the second
    batch is being recorded and resumed (that batch is then redone): every
    batch's statuses, hashes used, agreements,
    estimates and Lite outcomes equal those of the single-batch step, the
    pairs at and around every batch boundary agree with the oracle, and the
    kept counts and stop histogram add up."""
    from paper_1110_1328_gb300.batches import Checkpoint
    w, pipe = large_pipe
    dev = pipe.dev
    P = pipe.P
    ref = {n: getattr(pipe, n)[:P].clone() for n in ("status", "n_used", "m", "lstatus")}
    ref_est, ref_sim = pipe.est[:P].clone(), pipe.sim[:P].clone()
    ref_kept, ref_hist = pipe.kept_counts(), pipe.hist.sum(0).cpu()
    pipe.set_batch(P // 3 + 12_345)
    assert len(pipe.ranges) == 3
    boundary = set()
    for b0, n in pipe.ranges:
        boundary.update(q for q in range(b0 - 2, b0 + 3) if 0 <= q < P)
        boundary.update(q for q in range(b0 + n - 2, b0 + n + 2) if 0 <= q < P)
    boundary = np.array(sorted(boundary))
    seen, got_b = [], {}

    class Stop(Exception):
        pass

    def on_batch(b, b0, n, stop_after=None):
        torch.cuda.synchronize()
        for name in ("status", "n_used", "m", "lstatus"):
            assert torch.equal(getattr(pipe, name)[:n], ref[name][b0:b0 + n]), (b, name)
        kept = (ref["status"][b0:b0 + n] == B.ACCEPT) | (ref["status"][b0:b0 + n] == B.ACCEPT_AT_MAX)
        assert torch.equal(pipe.est[:n][kept], ref_est[b0:b0 + n][kept])
        surv = (ref["lstatus"][b0:b0 + n] == B.LITE_ACCEPT) | (ref["lstatus"][b0:b0 + n] == B.LITE_REJECT)
        assert torch.equal(pipe.sim[:n][surv], ref_sim[b0:b0 + n][surv])
        sel = boundary[(boundary >= b0) & (boundary < b0 + n)]
        got_b.update({int(q): (int(pipe.status[q - b0]), int(pipe.lstatus[q - b0])) for q in sel})
        seen.append(b)
        if stop_after is not None and b == stop_after:
            raise Stop()

    ck = Checkpoint(str(tmp_path / "large.json"))
    with pytest.raises(Stop):
        pipe.verify_streamed(ck, on_batch=lambda b, b0, n: on_batch(b, b0, n, stop_after=1))
    assert ck.load(ck_job := json_job(pipe)).next_batch == 1
    rec = pipe.verify_streamed(ck, on_batch=on_batch)
    assert seen == [0, 1, 1, 2]
    assert rec.next_batch == 3 and rec.kept == ref_kept and rec.hist == [int(x) for x in ref_hist]
    assert ck_job == rec.job
    # the boundary pairs against the oracle
    qd = torch.from_numpy(boundary).to(dev)
    sp = u32(pipe.pairs[qd])
    ids, inv = np.unique(sp.reshape(-1), return_inverse=True)
    local, Rq = large_oracle_view(pipe, w, ids)
    sig_o = O.srp_sparse_q16(local, Rq)
    lp = inv.reshape(-1, 2).astype(np.uint32)
    tab = O.tables(O.Params(kind=1, t=w["t"], k=w["k"], n_max=w["n_max"], h=w["h"]))
    want, lite = O.verify(tab, lp, sig_o), O.verify_lite(tab, lp, sig_o, local)
    for i, q in enumerate(boundary):
        assert got_b[int(q)] == (int(want.status[i]), int(lite.status[i])), q
    # the captured-step path over the same batches gives the same counts
    pipe.step()
    assert B.blsh_status(pipe.ctx) == 0
    assert pipe.kept_counts() == ref_kept


def json_job(pipe):
    w = pipe.w
    return {"workload": "large-mixed", "n": pipe.N, "seed": w["seed"], "r_seed": w["r_seed"], "P": pipe.P,
            "batch": pipe.batch, "lazy_bits": pipe.lazy_bits}
