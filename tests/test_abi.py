"""The C ABI without a GPU: the library builds, loads and exports every entry
point that include/blsh.h declares; host-side argument checks."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    src = open(os.path.join(ROOT, "include", "blsh.h")).read()
    return sorted(set(re.findall(r"^BLSH_API[^(]*?\b(blsh_\w+)\(", src, flags=re.M)))


def test_header_declares_the_boundary():
    names = declared()
    for need in ("blsh_minhash", "blsh_srp_sparse", "blsh_srp_dense", "blsh_lsh_candidates", "blsh_verify",
                 "blsh_verify_lite", "blsh_tables_build", "blsh_compact", "blsh_autotune", "blsh_status"):
        assert need in names


def test_library_exports_every_declared_symbol(B):
    lib = C.CDLL(B.lib_path())
    missing = [n for n in declared() if not hasattr(lib, n)]
    assert not missing
    # the binding declares each symbol's signature and has a Python function
    # of the same name for each
    import paper_1110_1328_gb300 as pkg
    assert not [n for n in declared() if not hasattr(pkg.lib(), n)]
    assert not [n for n in declared() if not callable(getattr(pkg, n, None))]
    assert B.lib().blsh_version().startswith(b"libblsh")
    assert pkg.blsh_version().startswith("libblsh") and pkg.blsh_strerror(B.ERANGE) == "pair index out of range"
    assert pkg.blsh_last_error(None) == "no context"


def test_host_checks_without_device(B):
    lib = B.lib()
    n = C.c_size_t()
    # per (object, band): two key buffers, two id buffers, the pair counts
    # and a 4-byte class id (up to 32 bands) or an 8-byte band hash (more)
    assert lib.blsh_lsh_candidates_workspace(1000, B.JACCARD, 8, 32, C.byref(n)) == 0
    assert n.value >= 1000 * 32 * (8 + 8 + 4 + 4 + 8 + 4)
    assert lib.blsh_lsh_candidates_workspace(1000, B.JACCARD, 2, 40, C.byref(n)) == 0
    assert n.value >= 1000 * 40 * (8 + 8 + 4 + 4 + 8 + 8)
    assert lib.blsh_lsh_candidates_workspace(-1, B.JACCARD, 8, 32, C.byref(n)) == B.EINVAL
    assert lib.blsh_lsh_candidates_workspace(10, 7, 8, 32, C.byref(n)) == B.EINVAL
    assert lib.blsh_strerror(B.ERANGE) == b"pair index out of range"
    # every entry point rejects a NULL context before touching the GPU
    assert lib.blsh_verify(None, None, None, 0, None, None, 0, 0, None, None, None, None, None, None) == B.EINVAL
    assert lib.blsh_compact(None, None, 0, None, 0, None, 0, None, None) == B.EINVAL
    assert lib.blsh_minhash(None, None, None, 0, 32, None, None, None, None) == B.EINVAL
    assert lib.blsh_gaussian_codes(None, 1, 10, 128, None, None) == B.EINVAL
    assert lib.blsh_srp_sparse_q16_cols(None, None, None, None, 0, None, 1, 128, 0, 128, None, None, None) == B.EINVAL
    assert lib.blsh_srp_sparse_cols(None, None, None, None, 0, None, 1, 128, 0, 128, None, None, None) == B.EINVAL
    assert lib.blsh_verify_both_capped(None, None, 128, None, 0, None, None, 0, 0, None, None, None, None, None,
                                       None, None, None, None, None, None, None, None) == B.EINVAL
    assert lib.blsh_verify_resume(None, None, None, 0, None, None, 0, 0, None, None, None, None, None,
                                  None) == B.EINVAL
    assert lib.blsh_timing_begin(None, 16) == B.EINVAL
    n_rec = C.c_int32(-1)
    assert lib.blsh_timing_end(None, 0, None, None, C.byref(n_rec)) == B.EINVAL
    assert lib.blsh_launch_count(None) == -1


def test_ctx_create_fails_cleanly_without_gpu(B):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = C.c_void_p()
    assert B.lib().blsh_ctx_create(C.byref(h), 0) == B.EDEVICE
    with pytest.raises(B.BlshError):
        B.Context(0)


def test_oracle_is_not_imported_by_the_product():
    pkg = os.path.join(ROOT, "paper_1110_1328_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text and "blsh_oracle" not in text
