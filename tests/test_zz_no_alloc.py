"""blsh_compact_noalloc: the stable compaction for callers that cannot allocate
device memory (code running inside a host application that owns every device
allocation through its own memory pool, or a plug-in for which allocating
outside that pool is forbidden), so cannot create a blsh_ctx.

Its output must equal blsh_compact's and the oracle's on the same inputs, on
two calls in a row (the second call must not see the first call's scratch),
and a new CUDA context (after cudaDeviceReset) must get its own scratch
address.  The file's name makes pytest collect it last, so that a run which
stops at the first failure has run every other test before this one."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

import oracle as O

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def reference(B, ctx, st, keep, cap, P_dev=None):
    out = torch.full((cap,), -1, dtype=torch.int64, device="cuda")
    n = torch.zeros(1, dtype=torch.int64, device="cuda")
    B.blsh_compact(ctx, st, keep, out, n, P_dev=P_dev)
    assert B.blsh_status(ctx) == 0
    return out.cpu().numpy(), int(n.item())


def noalloc(B, st, keep, cap, P_dev=None):
    out = torch.full((max(cap, 1),), -1, dtype=torch.int64, device="cuda")
    n = torch.full((1,), -7, dtype=torch.int64, device="cuda")
    B.blsh_compact_noalloc(st, keep, out[:cap], n, P_dev=P_dev)
    torch.cuda.synchronize()
    return out.cpu().numpy(), int(n.item())


def test_noalloc_matches_compact_and_oracle_twice(B, ctx):
    rng = np.random.default_rng(42)
    keep = (1 << B.ACCEPT) | (1 << B.ACCEPT_AT_MAX)
    for P in (5_000_003, 70_000):            # a large call, then a smaller one
        st_h = rng.integers(0, 5, P).astype(np.uint8)
        st = torch.from_numpy(st_h).cuda()
        want = O.compact(st_h, keep)
        ref, n_ref = reference(B, ctx, st, keep, P)
        out, n = noalloc(B, st, keep, P)
        assert n == n_ref == len(want)
        assert np.array_equal(out[:n], want) and np.array_equal(ref[:n], want)


def test_noalloc_device_count_capacity_stream_and_limits(B, ctx):
    rng = np.random.default_rng(7)
    P = 100_000
    st_h = rng.integers(0, 5, P).astype(np.uint8)
    st = torch.from_numpy(st_h).cuda()
    mask = 1 << B.LITE_ACCEPT
    # the count read on the device (clamped to P)
    pd = torch.tensor([61_234], dtype=torch.int64, device="cuda")
    want = O.compact(st_h[:61_234], mask)
    out, n = noalloc(B, st, mask, P, P_dev=pd)
    assert n == len(want) and np.array_equal(out[:n], want)
    # a capacity below the count writes only cap indices and reports the count
    small, n = noalloc(B, st, mask, 10, P_dev=pd)
    assert n == len(want) and np.array_equal(small[:10], want[:10])
    # no statuses at all, and a device-side count of zero: one tile launched,
    # nothing kept
    empty = torch.zeros(0, dtype=torch.uint8, device="cuda")
    out, n = noalloc(B, empty, mask, 0)
    assert n == 0
    zero = torch.zeros(1, dtype=torch.int64, device="cuda")
    out, n = noalloc(B, st, mask, P, P_dev=zero)
    assert n == 0 and np.all(out == -1)
    # on a stream other than the default one
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        out2 = torch.full((P,), -1, dtype=torch.int64, device="cuda")
        n2 = torch.zeros(1, dtype=torch.int64, device="cuda")
        B.blsh_compact_noalloc(st, mask, out2, n2)
    s.synchronize()
    want = O.compact(st_h, mask)
    assert int(n2.item()) == len(want) and np.array_equal(out2.cpu().numpy()[: len(want)], want)
    # more statuses than the fixed scratch covers: rejected before any launch
    big = torch.empty(67_108_865, dtype=torch.uint8, device="cuda")
    with pytest.raises(B.BlshError) as e:
        B.blsh_compact_noalloc(big, 1, out2, n2)
    assert e.value.code == B.ESIZE


# Runs in a fresh process with the CUDA runtime alone (no torch, whose own
# allocations would not survive the reset): the entry point on
# runtime-allocated buffers, cudaDeviceReset (which ends this process's
# primary context), then the entry point again in the new context.
_RESET_SCRIPT = r"""
import ctypes as C, json, sys
import numpy as np
sys.path.insert(0, sys.argv[1])
from paper_1110_1328_gb300 import build as b
L = C.CDLL(b.LIB)
rt_path = [ln.split()[-1] for ln in open('/proc/self/maps') if 'libcudart.so' in ln][0]
rt = C.CDLL(rt_path)
L.blsh_compact_noalloc.argtypes = [C.c_void_p, C.c_int64, C.c_void_p, C.c_uint32, C.c_void_p, C.c_int64,
                                   C.c_void_p, C.c_void_p]
L.blsh_compact_noalloc.restype = C.c_int
rt.cudaMalloc.argtypes = [C.POINTER(C.c_void_p), C.c_size_t]
rt.cudaMemcpy.argtypes = [C.c_void_p, C.c_void_p, C.c_size_t, C.c_int]
rt.cudaFree.argtypes = [C.c_void_p]
st = np.load(sys.argv[2])
P, mask = st.size, int(sys.argv[3])
def run():
    d_st, d_out, d_n = C.c_void_p(), C.c_void_p(), C.c_void_p()
    assert rt.cudaMalloc(C.byref(d_st), P) == 0 and rt.cudaMalloc(C.byref(d_out), 8 * P) == 0
    assert rt.cudaMalloc(C.byref(d_n), 8) == 0
    assert rt.cudaMemcpy(d_st, st.ctypes.data, P, 1) == 0
    rc = L.blsh_compact_noalloc(d_st, P, None, mask, d_out, P, d_n, None)
    assert rt.cudaDeviceSynchronize() == 0
    n = np.zeros(1, np.int64)
    assert rt.cudaMemcpy(n.ctypes.data, d_n, 8, 2) == 0
    out = np.zeros(int(n[0]), np.int64)
    if n[0]:
        assert rt.cudaMemcpy(out.ctypes.data, d_out, 8 * int(n[0]), 2) == 0
    for p in (d_st, d_out, d_n):
        rt.cudaFree(p)
    return rc, out.tolist()
assert rt.cudaSetDevice(0) == 0
r1 = run()
assert rt.cudaDeviceReset() == 0
assert rt.cudaSetDevice(0) == 0
r2 = run()
print(json.dumps({"rc": [r1[0], r2[0]], "out": [r1[1], r2[1]]}))
"""


def test_noalloc_after_device_reset_new_context(B, tmp_path):
    rng = np.random.default_rng(11)
    st = rng.integers(0, 5, 200_003).astype(np.uint8)
    path = tmp_path / "status.npy"
    np.save(path, st)
    mask = (1 << B.ACCEPT) | (1 << B.ACCEPT_AT_MAX)
    r = subprocess.run([sys.executable, "-c", _RESET_SCRIPT, ROOT, str(path), str(mask)], capture_output=True,
                       text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    res = json.loads(r.stdout.strip().splitlines()[-1])
    want = O.compact(st, mask).tolist()
    assert res["rc"] == [0, 0]
    assert res["out"][0] == want and res["out"][1] == want
