"""Per-launch device timing (blsh_timing_begin / blsh_timing_end): each
launch through a recording context gives one record, named for its kernel,
in launch order; graph capture and a context that is not recording give
none."""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu
dev = torch.device("cuda")


def _minhash_inputs():
    sets = synth.jaccard_sets(n_sets=4000, vocab=20000, mean_size=50, n_groups=400, seed=5)
    a, b = synth.minhash_coeffs(256, seed=6)
    args = (torch.from_numpy(sets.indptr).to(dev), torch.from_numpy(sets.indices.view(np.int32)).to(dev),
            torch.from_numpy(a.view(np.int32)).to(dev), torch.from_numpy(b.view(np.int32)).to(dev))
    sig = torch.zeros((len(sets.indptr) - 1, 256), dtype=torch.int32, device=dev)
    return args, sig


def test_records_each_launch_in_order(B, ctx):
    (indptr, indices, a, b), sig = _minhash_inputs()
    status = torch.full((1 << 20,), 3, dtype=torch.uint8, device=dev)
    out = torch.zeros(1 << 20, dtype=torch.int64, device=dev)
    n_out = torch.zeros(1, dtype=torch.int64, device=dev)
    B.blsh_minhash(ctx, indptr, indices, 256, a, b, sig)          # not recording: no records
    B.blsh_timing_begin(ctx)
    B.blsh_minhash(ctx, indptr, indices, 256, a, b, sig)
    B.blsh_compact(ctx, status, 1 << 3, out, n_out)
    rec = B.blsh_timing_end(ctx)
    assert B.blsh_status(ctx) == 0
    assert [n for n, _ in rec] == ["minhash_kernel", "minhash_big_kernel", "compact_count", "compact_write"]
    assert all(t > 0.0 for _, t in rec)
    assert int(n_out.item()) == 1 << 20
    # recording is off again
    B.blsh_minhash(ctx, indptr, indices, 256, a, b, sig)
    B.blsh_timing_begin(ctx, 8)
    assert B.blsh_timing_end(ctx) == []


def test_capacity_and_graph_capture(B, ctx):
    (indptr, indices, a, b), sig = _minhash_inputs()
    B.blsh_timing_begin(ctx, 3)
    for _ in range(3):
        B.blsh_minhash(ctx, indptr, indices, 256, a, b, sig)        # 6 launches, 3 records kept
    rec = B.blsh_timing_end(ctx)
    assert [n for n, _ in rec] == ["minhash_kernel", "minhash_big_kernel", "minhash_kernel"]
    # launches captured into a graph are not recorded (events stay off the capture)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        B.blsh_minhash(ctx, indptr, indices, 256, a, b, sig, stream=s)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    B.blsh_timing_begin(ctx)
    with torch.cuda.graph(g):
        B.blsh_minhash(ctx, indptr, indices, 256, a, b, sig)
    g.replay()
    torch.cuda.synchronize()
    assert B.blsh_timing_end(ctx) == []
    assert B.blsh_status(ctx) == 0


def test_rejects_bad_sizes(B, ctx):
    with pytest.raises(B.BlshError):
        B.blsh_timing_begin(ctx, 0)
    with pytest.raises(B.BlshError):
        B.blsh_timing_begin(ctx, 1 << 17)
