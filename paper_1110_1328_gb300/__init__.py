"""Python binding of libblsh, the GB300 (sm_103a) BayesLSH verification library.

Argument marshalling only: every function here has the name of a C entry
point of ``include/blsh.h``, takes torch tensors (device memory) and passes
their data pointers, sizes and the current CUDA stream to the library.  All
computation runs in the library's CUDA kernels; there is no CPU fallback, and
importing a function fails loudly when the library has not been built.
"""
from __future__ import annotations

import ctypes as C
import os

import torch

from . import build as _build

JACCARD, COSINE = 0, 1
PRUNED, ACCEPT, ACCEPT_AT_MAX, LITE_REJECT, LITE_ACCEPT, BAD_PAIR = 0, 1, 2, 3, 4, 255
NEEDS_HASHES = 253
PLAN_PLAIN, PLAN_PERSISTENT = 0, 1
OK, EINVAL, ERANGE, ETRUNC, ENOMEM, EDEVICE, ENUMERIC, ESIZE = range(8)

_lib = None


class BlshError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"libblsh error {code}: {msg}")
        self.code = code


class blsh_params(C.Structure):
    _fields_ = [("kind", C.c_int32), ("k", C.c_int32), ("n_max", C.c_int32), ("h", C.c_int32),
                ("t", C.c_double), ("eps", C.c_double), ("delta", C.c_double), ("gamma", C.c_double),
                ("alpha", C.c_double), ("beta", C.c_double)]


class blsh_plan(C.Structure):
    _fields_ = [("mode", C.c_int32), ("group", C.c_int32), ("block", C.c_int32), ("grab", C.c_int32),
                ("ctas_per_sm", C.c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


def lib_path() -> str:
    return _build.LIB


def lib():
    """Loads libblsh.so (build it with paper_1110_1328_gb300.build.build())."""
    global _lib
    if _lib is None:
        if not os.path.exists(_build.LIB):
            raise ImportError(f"libblsh is not built ({_build.LIB} missing); run __graft_entry__.build()")
        L = C.CDLL(_build.LIB)
        p, i32, i64, u32, sz = C.c_void_p, C.c_int32, C.c_int64, C.c_uint32, C.c_size_t
        sig = {
            "blsh_version": ([], C.c_char_p),
            "blsh_strerror": ([C.c_int], C.c_char_p),
            "blsh_ctx_create": ([p, C.c_int], C.c_int),
            "blsh_ctx_destroy": ([p], C.c_int),
            "blsh_ctx_reserve": ([p, i64], C.c_int),
            "blsh_ctx_reserved": ([p], C.c_int64),
            "blsh_last_error": ([p], C.c_char_p),
            "blsh_status": ([p, p, p], C.c_int),
            "blsh_launch_count": ([p], C.c_int64),
            "blsh_timing_begin": ([p, i32], C.c_int),
            "blsh_timing_end": ([p, i32, p, p, p], C.c_int),
            "blsh_tables_build": ([p, p, p, p], C.c_int),
            "blsh_tables_destroy": ([p], C.c_int),
            "blsh_tables_download": ([p, p, p, p, p, p, p, p, p], C.c_int),
            "blsh_minhash": ([p, p, p, i64, i32, p, p, p, p], C.c_int),
            "blsh_srp_sparse": ([p, p, p, p, i64, p, i64, i32, p, p], C.c_int),
            "blsh_srp_sparse_cols": ([p, p, p, p, i64, p, i64, i32, i32, i32, p, p, p], C.c_int),
            "blsh_srp_sparse_q16": ([p, p, p, p, i64, p, i64, i32, p, p], C.c_int),
            "blsh_srp_sparse_q16_cols": ([p, p, p, p, i64, p, i64, i32, i32, i32, p, p, p], C.c_int),
            "blsh_quantize_gaussian": ([p, p, i64, p, p], C.c_int),
            "blsh_gaussian_codes": ([p, C.c_uint64, i64, i32, p, p], C.c_int),
            "blsh_srp_dense": ([p, p, i64, i32, p, i32, C.c_float, p, p, sz, p], C.c_int),
            "blsh_srp_dense_workspace": ([i64, i32, i32, p], C.c_int),
            "blsh_lsh_candidates_workspace": ([i64, i32, i32, i32, p], C.c_int),
            "blsh_lsh_candidates": ([p, p, i64, i32, i32, i32, i32, p, i64, p, p, sz, p], C.c_int),
            "blsh_allpairs_workspace": ([i64, i64, i64, i64, p], C.c_int),
            "blsh_allpairs_candidates": ([p, p, p, p, i64, i64, i64, C.c_double, i32, i64, p, i64, p, p, p, sz, p],
                                         C.c_int),
            "blsh_verify": ([p, p, p, i64, p, p, i64, i32, p, p, p, p, p, p], C.c_int),
            "blsh_verify_plan": ([p, p, p, p, i64, p, p, i64, i32, p, p, p, p, p, p], C.c_int),
            "blsh_verify_lite": ([p, p, p, i64, p, p, i64, i32, p, p, p, p, p, p, p], C.c_int),
            "blsh_verify_both": ([p, p, p, i64, p, p, i64, i32, p, p, p, p, p, p, p, p, p, p, p, p], C.c_int),
            "blsh_verify_both_capped": ([p, p, i32, p, i64, p, p, i64, i32, p, p, p, p, p, p, p, p, p, p, p, p, p], C.c_int),
            "blsh_verify_resume": ([p, p, p, i64, p, p, i64, i32, p, p, p, p, p, p], C.c_int),
            "blsh_set_plan": ([p, p, p], C.c_int),
            "blsh_autotune": ([p, p, p, i64, p, i64, i32, p, p, p, p, p, p], C.c_int),
            "blsh_autotune_k": ([p, p, p, i32, p, i64, p, i64, i32, p, p, p, p, p, p, p, p], C.c_int),
            "blsh_compact": ([p, p, i64, p, u32, p, i64, p, p], C.c_int),
            "blsh_compact_noalloc": ([p, i64, p, u32, p, i64, p, p], C.c_int),
            "blsh_estimate_mle": ([p, i32, i32, C.c_double, p, i64, p, p, i64, i32, p, p, p, p], C.c_int),
            "blsh_fit_beta_prior": ([p, p, i64, p, p, i64, p, p, p, p], C.c_int),
        }
        for name, (args, res) in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def exported_symbols() -> list[str]:
    """Names of the C entry points this binding declares."""
    lib()
    return sorted(n for n in dir(_lib) if n.startswith("blsh_"))


# ---------------------------------------------------------------------------
# marshalling helpers
# ---------------------------------------------------------------------------

def _ptr(t):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor):
        raise TypeError("expected a torch tensor")
    if t.numel() and not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return t.data_ptr() or None


def _dev(t, dtype=None):
    if t is not None:
        if not t.is_cuda:
            raise ValueError("libblsh takes device tensors")
        if dtype is not None and t.dtype != dtype:
            raise TypeError(f"expected {dtype}, got {t.dtype}")
    return _ptr(t)


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


def _check(rc: int, ctx=None):
    if rc != OK:
        msg = lib().blsh_last_error(ctx.handle if ctx is not None else None)
        raise BlshError(rc, (msg or b"").decode() or lib().blsh_strerror(rc).decode())


class Context:
    """Owns a blsh_ctx (device scratch, autotuned plans)."""

    def __init__(self, device: int | None = None):
        if device is None:
            device = torch.cuda.current_device()
        self.device = device
        h = C.c_void_p()
        rc = lib().blsh_ctx_create(C.byref(h), device)
        if rc != OK:
            raise BlshError(rc, "blsh_ctx_create failed (a GB300 / sm_103 device is required)")
        self.handle = h

    def close(self):
        if self.handle:
            lib().blsh_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Tables:
    """Owns a blsh_tables (the Section 4.3 tables on the device)."""

    def __init__(self, handle, params):
        self.handle = handle
        self.params = params

    @property
    def levels(self) -> int:
        return self.params.n_max // self.params.k

    def close(self):
        if self.handle:
            lib().blsh_tables_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def make_params(kind=JACCARD, t=0.7, eps=0.03, delta=0.05, gamma=0.03, alpha=1.0, beta=1.0, k=32, n_max=256,
                h=None) -> blsh_params:
    if h is None:
        h = 64 if kind == JACCARD else 128
    h = min(n_max, (h + k - 1) // k * k)      # Lite's h: a multiple of k, at most n_max
    return blsh_params(kind, k, n_max, h, t, eps, delta, gamma, alpha, beta)


# ---------------------------------------------------------------------------
# entry points (same names as the C ABI)
# ---------------------------------------------------------------------------

def blsh_ctx_create(device: int | None = None) -> Context:
    return Context(device)


def blsh_ctx_destroy(ctx: Context) -> None:
    ctx.close()


def blsh_ctx_reserve(ctx: Context, max_objects: int) -> None:
    """Set-up: the context's per-object buffers (verification plane, Lite
    norms) for up to max_objects rows, so hot calls never allocate."""
    _check(lib().blsh_ctx_reserve(ctx.handle, int(max_objects)), ctx)


def blsh_ctx_reserved(ctx: Context) -> int:
    return int(lib().blsh_ctx_reserved(ctx.handle))


def blsh_tables_destroy(tab: "Tables") -> None:
    tab.close()


def blsh_last_error(ctx: Context | None) -> str:
    return (lib().blsh_last_error(ctx.handle if ctx is not None else None) or b"").decode()


def blsh_strerror(rc: int) -> str:
    return (lib().blsh_strerror(int(rc)) or b"").decode()


def blsh_version() -> str:
    return lib().blsh_version().decode()


def blsh_status(ctx: Context, stream=None, counters: bool = False):
    buf = (C.c_uint64 * 4)()
    rc = lib().blsh_status(ctx.handle, _stream(stream), buf)
    if counters:
        return rc, list(buf)
    return rc


def blsh_launch_count(ctx: Context) -> int:
    return int(lib().blsh_launch_count(ctx.handle))


def blsh_timing_begin(ctx: Context, max_launches: int = 4096) -> None:
    """Switches per-launch device timing on for the kernels launched through ctx."""
    _check(lib().blsh_timing_begin(ctx.handle, int(max_launches)), ctx)


def blsh_timing_end(ctx: Context, max_records: int = 4096) -> list[tuple[str, float]]:
    """(kernel name, device ms) of each launch recorded since blsh_timing_begin,
    in launch order; switches timing off."""
    names = (C.c_char_p * max_records)()
    ms = (C.c_float * max_records)()
    n = C.c_int32(0)
    _check(lib().blsh_timing_end(ctx.handle, int(max_records), names, ms, C.byref(n)), ctx)
    return [(names[i].decode(), float(ms[i])) for i in range(n.value)]


def blsh_tables_build(ctx: Context, params: blsh_params, stream=None) -> Tables:
    h = C.c_void_p()
    rc = lib().blsh_tables_build(ctx.handle, C.byref(params), C.byref(h), _stream(stream))
    if rc not in (OK, ENUMERIC) or not h:
        _check(rc, ctx)
    t = Tables(h, params)
    t.build_status = rc
    return t


def blsh_tables_download(tab: Tables):
    import numpy as np
    p = tab.params
    L, W = p.n_max // p.k, p.n_max + 1
    levels = C.c_int32()
    ties = C.c_int32()
    mm = np.zeros(L, np.int32)
    conc = np.zeros((L, W), np.uint8)
    est = np.zeros((L, W), np.float32)
    pr = np.zeros((L, W), np.float64)
    cp = np.zeros((L, W), np.float64)
    par = blsh_params()
    rc = lib().blsh_tables_download(tab.handle, C.byref(par), C.byref(levels), C.byref(ties),
                                    mm.ctypes.data, conc.ctypes.data, est.ctypes.data, pr.ctypes.data,
                                    cp.ctypes.data)
    _check(rc)
    return {"min_matches": mm, "conc": conc, "est": est, "prune_prob": pr, "conc_prob": cp,
            "near_ties": ties.value, "levels": levels.value}


def blsh_minhash(ctx: Context, indptr, indices, n_hashes: int, a, b, sig, stream=None):
    N = indptr.numel() - 1
    idx = indices if indices.numel() else torch.zeros(1, dtype=torch.int32, device=indptr.device)
    rc = lib().blsh_minhash(ctx.handle, _dev(indptr, torch.int64), _dev(idx), N, n_hashes, _dev(a), _dev(b),
                            _dev(sig), _stream(stream))
    _check(rc, ctx)


def blsh_srp_sparse(ctx: Context, indptr, indices, values, R, sig, stream=None):
    N = indptr.numel() - 1
    dim, bits = R.shape
    idx = indices if indices.numel() else torch.zeros(1, dtype=torch.int32, device=indptr.device)
    val = values if values.numel() else torch.zeros(1, dtype=torch.float32, device=indptr.device)
    rc = lib().blsh_srp_sparse(ctx.handle, _dev(indptr, torch.int64), _dev(idx), _dev(val, torch.float32), N,
                               _dev(R, torch.float32), dim, bits, _dev(sig), _stream(stream))
    _check(rc, ctx)


def blsh_srp_sparse_cols(ctx: Context, indptr, indices, values, R, sig, col_begin: int, col_count: int,
                         row_mask=None, stream=None):
    """Columns [col_begin, col_begin + col_count) of the sparse projection, for
    the rows row_mask (uint8 tensor) selects (all when None)."""
    N = indptr.numel() - 1
    dim, bits = R.shape
    idx = indices if indices.numel() else torch.zeros(1, dtype=torch.int32, device=indptr.device)
    val = values if values.numel() else torch.zeros(1, dtype=torch.float32, device=indptr.device)
    rc = lib().blsh_srp_sparse_cols(ctx.handle, _dev(indptr, torch.int64), _dev(idx), _dev(val, torch.float32), N,
                                    _dev(R, torch.float32), dim, bits, col_begin, col_count,
                                    _dev(row_mask, torch.uint8), _dev(sig), _stream(stream))
    _check(rc, ctx)


def blsh_quantize_gaussian(ctx: Context, x, q=None, stream=None):
    """Two-byte codes of Gaussian samples (Section 4.3); returns q (int16
    tensor holding the uint16 codes, same shape as x)."""
    if q is None:
        q = torch.empty(x.shape, dtype=torch.int16, device=x.device)
    rc = lib().blsh_quantize_gaussian(ctx.handle, _dev(x, torch.float32), x.numel(), _dev(q), _stream(stream))
    _check(rc, ctx)
    return q


def blsh_gaussian_codes(ctx: Context, seed: int, dim: int, bits: int, stream=None):
    """Two-byte Gaussian codes R [dim][bits] generated on the device from a
    counter (SplitMix64 + Irwin-Hall); returns an int16 tensor holding the
    uint16 codes."""
    codes = torch.empty((dim, bits), dtype=torch.int16, device=torch.device("cuda", ctx.device))
    _check(lib().blsh_gaussian_codes(ctx.handle, int(seed) & (2 ** 64 - 1), int(dim), int(bits), _dev(codes),
                                     _stream(stream)), ctx)
    return codes


def blsh_srp_sparse_q16(ctx: Context, indptr, indices, values, Rq, sig, stream=None):
    """blsh_srp_sparse with R as two-byte codes Rq [dim][bits] (Section 4.3)."""
    N = indptr.numel() - 1
    dim, bits = Rq.shape
    idx = indices if indices.numel() else torch.zeros(1, dtype=torch.int32, device=indptr.device)
    val = values if values.numel() else torch.zeros(1, dtype=torch.float32, device=indptr.device)
    rc = lib().blsh_srp_sparse_q16(ctx.handle, _dev(indptr, torch.int64), _dev(idx), _dev(val, torch.float32), N,
                                   _dev(Rq), dim, bits, _dev(sig), _stream(stream))
    _check(rc, ctx)


def blsh_srp_sparse_q16_cols(ctx: Context, indptr, indices, values, Rq, sig, col_begin: int, col_count: int,
                             row_mask=None, stream=None):
    """Columns [col_begin, col_begin + col_count) of blsh_srp_sparse_q16's
    signatures for the rows row_mask (uint8 [N], or None: all) selects."""
    N = indptr.numel() - 1
    dim, bits = Rq.shape
    rc = lib().blsh_srp_sparse_q16_cols(ctx.handle, _dev(indptr, torch.int64), _dev(indices),
                                        _dev(values, torch.float32), N, _dev(Rq), dim, bits, int(col_begin),
                                        int(col_count), _dev(row_mask, torch.uint8), _dev(sig), _stream(stream))
    _check(rc, ctx)


def blsh_srp_dense_workspace(N: int, d: int, bits: int) -> int:
    n = C.c_size_t()
    _check(lib().blsh_srp_dense_workspace(N, d, bits, C.byref(n)))
    return n.value


def blsh_srp_dense(ctx: Context, X, R, sig, margin: float = 0.0, workspace=None, stream=None):
    N, d = X.shape
    bits = R.shape[1]
    nbytes = 0 if workspace is None else workspace.numel() * workspace.element_size()
    rc = lib().blsh_srp_dense(ctx.handle, _dev(X, torch.float32), N, d, _dev(R, torch.float32), bits,
                              float(margin), _dev(sig), _dev(workspace), nbytes, _stream(stream))
    _check(rc, ctx)


def blsh_lsh_candidates_workspace(N: int, kind: int, rows: int, bands: int) -> int:
    n = C.c_size_t()
    _check(lib().blsh_lsh_candidates_workspace(N, kind, rows, bands, C.byref(n)))
    return n.value


def blsh_lsh_candidates(ctx: Context, sig, kind: int, rows: int, bands: int, pairs, n_pairs, workspace,
                        stream=None):
    N, W = sig.shape
    cap = pairs.shape[0] if pairs is not None else 0
    rc = lib().blsh_lsh_candidates(ctx.handle, _dev(sig), N, W, kind, rows, bands,
                                   _dev(pairs) if cap else None, cap, _dev(n_pairs, torch.int64),
                                   _dev(workspace), workspace.numel() * workspace.element_size(),
                                   _stream(stream))
    _check(rc, ctx)


def blsh_allpairs_workspace(N: int, nnz: int, dim: int, max_dups: int) -> int:
    n = C.c_size_t()
    _check(lib().blsh_allpairs_workspace(N, nnz, dim, max_dups, C.byref(n)))
    return n.value


def blsh_allpairs_candidates(ctx: Context, indptr, indices, values, dim: int, t: float, kind: int, pairs, n_pairs,
                             workspace, max_dups: int = 0, n_dups=None, nnz: int | None = None, stream=None):
    """AllPairs-style prefix-filter candidates (pairs=None: count-only call,
    n_dups receives the number of candidate keys to size max_dups).  nnz:
    the nonzero count (default: the length of indices)."""
    N = indptr.numel() - 1
    if nnz is None:
        nnz = indices.numel()
    cap = pairs.shape[0] if pairs is not None else 0
    idx = indices if indices.numel() else torch.zeros(1, dtype=torch.int32, device=indptr.device)
    rc = lib().blsh_allpairs_candidates(ctx.handle, _dev(indptr, torch.int64), _dev(idx),
                                        None if values is None else _dev(values, torch.float32), N, int(nnz), int(dim),
                                        float(t), int(kind), int(max_dups), _dev(pairs) if cap else None, cap,
                                        _dev(n_pairs, torch.int64), _dev(n_dups, torch.int64), _dev(workspace),
                                        workspace.numel() * workspace.element_size(), _stream(stream))
    _check(rc, ctx)


def blsh_verify(ctx: Context, tab: Tables, pairs, sig, status, n_used=None, m=None, est=None, stop_hist=None,
                P_dev=None, plan: blsh_plan | None = None, stream=None):
    P = pairs.shape[0]
    N, W = sig.shape
    args = (_dev(pairs), P, _dev(P_dev, torch.int64), _dev(sig), N, W, _dev(status, torch.uint8),
            _dev(n_used), _dev(m), _dev(est, torch.float32), _dev(stop_hist), _stream(stream))
    if plan is None:
        rc = lib().blsh_verify(ctx.handle, tab.handle, *args)
    else:
        rc = lib().blsh_verify_plan(ctx.handle, tab.handle, C.byref(plan), *args)
    _check(rc, ctx)


def blsh_verify_plan(ctx, tab, plan, pairs, sig, status, n_used=None, m=None, est=None, stop_hist=None,
                     P_dev=None, stream=None):
    blsh_verify(ctx, tab, pairs, sig, status, n_used, m, est, stop_hist, P_dev, plan, stream)


def blsh_verify_lite(ctx: Context, tab: Tables, pairs, sig, indptr, indices, values, status, sim, n_used=None,
                     P_dev=None, stream=None):
    P = pairs.shape[0]
    N, W = sig.shape
    rc = lib().blsh_verify_lite(ctx.handle, tab.handle, _dev(pairs), P, _dev(P_dev, torch.int64), _dev(sig), N, W,
                                _dev(indptr, torch.int64), _dev(indices), _dev(values, torch.float32),
                                _dev(status, torch.uint8), _dev(n_used), _dev(sim, torch.float64),
                                _stream(stream))
    _check(rc, ctx)


def blsh_set_plan(ctx: Context, tab: Tables, plan: blsh_plan):
    """Make `plan` the launch plan used for these tables."""
    _check(lib().blsh_set_plan(ctx.handle, tab.handle, C.byref(plan)), ctx)


def blsh_verify_both(ctx: Context, tab: Tables, pairs, sig, status, n_used, m, est, stop_hist, indptr, indices,
                     values, lite_status, sim, lite_n_used=None, P_dev=None, stream=None):
    """Algorithms 1 and 2 over the same pairs in one pass (outputs of
    blsh_verify and blsh_verify_lite)."""
    P = pairs.shape[0]
    N, W = sig.shape
    rc = lib().blsh_verify_both(ctx.handle, tab.handle, _dev(pairs), P, _dev(P_dev, torch.int64), _dev(sig), N, W,
                                _dev(status, torch.uint8), _dev(n_used), _dev(m), _dev(est, torch.float32),
                                _dev(stop_hist), _dev(indptr, torch.int64), _dev(indices),
                                None if values is None else _dev(values, torch.float32),
                                _dev(lite_status, torch.uint8), _dev(lite_n_used), _dev(sim, torch.float64),
                                _stream(stream))
    _check(rc, ctx)


def blsh_verify_both_capped(ctx: Context, tab: Tables, hash_limit: int, pairs, sig, status, n_used, m, est,
                            stop_hist, indptr, indices, values, lite_status, sim, need, lite_n_used=None,
                            P_dev=None, stream=None):
    """blsh_verify_both over the first hash_limit hashes; undecided pairs get
    NEEDS_HASHES and mark their objects in need (uint8 [N])."""
    P = pairs.shape[0]
    N, W = sig.shape
    rc = lib().blsh_verify_both_capped(ctx.handle, tab.handle, hash_limit, _dev(pairs), P, _dev(P_dev, torch.int64),
                                       _dev(sig), N, W, _dev(status, torch.uint8), _dev(n_used), _dev(m),
                                       _dev(est, torch.float32), _dev(stop_hist), _dev(indptr, torch.int64),
                                       _dev(indices), None if values is None else _dev(values, torch.float32),
                                       _dev(lite_status, torch.uint8), _dev(lite_n_used), _dev(sim, torch.float64),
                                       _dev(need, torch.uint8), _stream(stream))
    _check(rc, ctx)


def blsh_verify_resume(ctx: Context, tab: Tables, pairs, sig, status, n_used=None, m=None, est=None,
                       stop_hist=None, P_dev=None, stream=None):
    """Finish the NEEDS_HASHES pairs over all n_max hashes."""
    P = pairs.shape[0]
    N, W = sig.shape
    rc = lib().blsh_verify_resume(ctx.handle, tab.handle, _dev(pairs), P, _dev(P_dev, torch.int64), _dev(sig), N, W,
                                  _dev(status, torch.uint8), _dev(n_used), _dev(m), _dev(est, torch.float32),
                                  _dev(stop_hist), _stream(stream))
    _check(rc, ctx)


def blsh_autotune(ctx: Context, tab: Tables, pairs, sig, status, n_used=None, m=None, est=None,
                  stream=None) -> blsh_plan:
    P = pairs.shape[0]
    N, W = sig.shape
    best = blsh_plan()
    rc = lib().blsh_autotune(ctx.handle, tab.handle, _dev(pairs), P, _dev(sig), N, W, _dev(status, torch.uint8),
                             _dev(n_used), _dev(m), _dev(est, torch.float32), C.byref(best), _stream(stream))
    _check(rc, ctx)
    return best


def blsh_autotune_k(ctx: Context, params: blsh_params, ks, pairs, sig, status, n_used=None, m=None, est=None,
                    stream=None):
    """The chunk size k in ks and the launch plan, tuned together; returns
    (the chosen k's Tables, the plan, {k: best ms per call})."""
    P = pairs.shape[0]
    N, W = sig.shape
    ks = [int(k) for k in ks]
    karr = (C.c_int32 * len(ks))(*ks)
    ms = (C.c_float * len(ks))()
    best = blsh_plan()
    h = C.c_void_p()
    rc = lib().blsh_autotune_k(ctx.handle, C.byref(params), karr, len(ks), _dev(pairs), P, _dev(sig), N, W,
                               _dev(status, torch.uint8), _dev(n_used), _dev(m), _dev(est, torch.float32),
                               C.byref(h), C.byref(best), ms, _stream(stream))
    _check(rc, ctx)
    par = blsh_params()
    lv, ties = C.c_int32(), C.c_int32()
    _check(lib().blsh_tables_download(h, C.byref(par), C.byref(lv), C.byref(ties), None, None, None, None, None))
    return Tables(h, par), best, {kk: float(v) for kk, v in zip(ks, ms)}


def blsh_compact(ctx: Context, status, keep_mask: int, out_idx, n_out, P_dev=None, stream=None):
    P = status.numel()
    cap = out_idx.numel() if out_idx is not None else 0
    rc = lib().blsh_compact(ctx.handle, _dev(status, torch.uint8), P, _dev(P_dev, torch.int64), keep_mask,
                            _dev(out_idx, torch.int64) if cap else None, cap, _dev(n_out, torch.int64),
                            _stream(stream))
    _check(rc, ctx)


def blsh_compact_noalloc(status, keep_mask: int, out_idx, n_out, P_dev=None, stream=None):
    """The stable compaction without a context and without any allocation
    (scratch in a fixed array of the library; see include/blsh.h)."""
    P = status.numel()
    cap = out_idx.numel() if out_idx is not None else 0
    rc = lib().blsh_compact_noalloc(_dev(status, torch.uint8), P, _dev(P_dev, torch.int64), keep_mask,
                                    _dev(out_idx, torch.int64) if cap else None, cap, _dev(n_out, torch.int64),
                                    _stream(stream))
    if rc != OK:
        raise BlshError(rc, lib().blsh_strerror(rc).decode())


def blsh_estimate_mle(ctx: Context, kind: int, n_hashes: int, t: float, pairs, sig, m=None, est=None, keep=None,
                      P_dev=None, stream=None):
    """The fixed-n maximum-likelihood estimate (Section 3) and [est > t]."""
    P = pairs.shape[0]
    N, W = sig.shape
    rc = lib().blsh_estimate_mle(ctx.handle, kind, n_hashes, float(t), _dev(pairs), P, _dev(P_dev, torch.int64),
                                 _dev(sig), N, W, _dev(m), _dev(est, torch.float32), _dev(keep, torch.uint8),
                                 _stream(stream))
    _check(rc, ctx)


def blsh_fit_beta_prior(ctx: Context, pairs, indptr, indices, sims=None, stream=None):
    """Method-of-moments Beta prior from exact similarities of sampled pairs
    (Section 4.1).  Returns (mean, var, alpha, beta, fallback) and the sims."""
    r = pairs.shape[0]
    N = indptr.numel() - 1
    if sims is None:
        sims = torch.empty(r, dtype=torch.float64, device=pairs.device)
    out_dev = torch.empty(5, dtype=torch.float64, device=pairs.device)
    out = (C.c_double * 5)()
    rc = lib().blsh_fit_beta_prior(ctx.handle, _dev(pairs), r, _dev(indptr, torch.int64), _dev(indices), N,
                                   _dev(sims, torch.float64), _dev(out_dev), out, _stream(stream))
    _check(rc, ctx)
    return tuple(out), sims
