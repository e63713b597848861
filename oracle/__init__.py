"""CPU oracle for BayesLSH candidate verification -- TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its Python binding) never does.

The arithmetic lives in ``blsh_oracle.c`` (plain C, FP64, one pair and one
chunk at a time, compiled with FP contraction off so x86 and Arm give the same
bits).  This module only compiles it, loads it with ctypes and marshals numpy
arrays.  Every function cites the passage of the paper it follows.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "blsh_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libblsh_oracle.so")

JACCARD, COSINE = 0, 1
PRUNED, ACCEPT, ACCEPT_AT_MAX, LITE_REJECT, LITE_ACCEPT = 0, 1, 2, 3, 4

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle into a shared library (gcc, -O2, no FP contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
                               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB_PATH)
        d, i, p, i64 = C.c_double, C.c_int, C.c_void_p, C.c_int64
        L.orc_ibeta.argtypes = [d, d, d]; L.orc_ibeta.restype = d
        L.orc_log_ibeta.argtypes = [d, d, d]; L.orc_log_ibeta.restype = d
        L.orc_tables.argtypes = [i, d, d, d, d, d, d, i, i, p, p, p, p, p]; L.orc_tables.restype = i
        L.orc_verify.argtypes = [i, i, i, p, p, p, p, i64, p, i64, i, p, p, p, p]; L.orc_verify.restype = i64
        L.orc_verify_lite.argtypes = [i, i, i, p, p, i64, p, i64, i, p, p, p, d, p, p, p]
        L.orc_verify_lite.restype = i64
        L.orc_exact_jaccard.argtypes = [p, i64, p, i64]; L.orc_exact_jaccard.restype = d
        L.orc_exact_cosine.argtypes = [p, p, i64, p, p, i64]; L.orc_exact_cosine.restype = d
        L.orc_minhash.argtypes = [p, p, i64, i, p, p, p]; L.orc_minhash.restype = None
        L.orc_srp_sparse.argtypes = [p, p, p, i64, p, i, p]; L.orc_srp_sparse.restype = None
        L.orc_srp_dense.argtypes = [p, i64, i, p, i, p, p]; L.orc_srp_dense.restype = None
        L.orc_lsh_candidates.argtypes = [p, i64, i, i, i, i, p, i64]; L.orc_lsh_candidates.restype = i64
        L.orc_compact.argtypes = [p, i64, C.c_uint32, p]; L.orc_compact.restype = i64
        L.orc_allpairs_indexed.argtypes = [p, p, p, i64, i64, d, i, p]; L.orc_allpairs_indexed.restype = i
        L.orc_allpairs_candidates.argtypes = [p, p, p, i64, i64, d, i, p, i64]
        L.orc_allpairs_candidates.restype = i64
        L.orc_stop_hist.argtypes = [p, i64, i, i, p]; L.orc_stop_hist.restype = None
        L.orc_estimate_mle.argtypes = [i, i, d, p, i64, p, i, p, p, p]; L.orc_estimate_mle.restype = None
        L.orc_fit_beta_prior.argtypes = [p, i64, p]; L.orc_fit_beta_prior.restype = None
        L.orc_quantize_gaussian.argtypes = [p, i64, p]; L.orc_quantize_gaussian.restype = i64
        L.orc_dequantize_gaussian.argtypes = [C.c_uint16]; L.orc_dequantize_gaussian.restype = d
        L.orc_srp_sparse_q16.argtypes = [p, p, p, i64, p, i, p]; L.orc_srp_sparse_q16.restype = None
        L.orc_splitmix64_at.argtypes = [C.c_uint64, C.c_uint64]; L.orc_splitmix64_at.restype = C.c_uint64
        L.orc_gaussian_codes.argtypes = [C.c_uint64, i64, i64, i, p]; L.orc_gaussian_codes.restype = None
        _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


# --------------------------------------------------------------------------
# Incomplete beta and inference (Sections 4.1, 4.2)
# --------------------------------------------------------------------------

def ibeta(a: float, b: float, x: float) -> float:
    """Regularised incomplete beta I_x(a,b) (Section 4.1, "Inference")."""
    return lib().orc_ibeta(float(a), float(b), float(x))


def log_ibeta(a: float, b: float, x: float) -> float:
    return lib().orc_log_ibeta(float(a), float(b), float(x))


@dataclass
class Params:
    """Parameters of Algorithms 1 and 2 (t, eps, delta, gamma; Section 5.1
    sets k = 32, h = 64 for Jaccard and 128 for cosine) and the Jaccard Beta
    prior (Section 4.1)."""
    kind: int = JACCARD
    t: float = 0.7
    eps: float = 0.03
    delta: float = 0.05
    gamma: float = 0.03
    alpha: float = 1.0
    beta: float = 1.0
    k: int = 32
    n_max: int = 256
    h: int = 64

    @property
    def levels(self) -> int:
        return self.n_max // self.k


@dataclass
class Tables:
    """Section 4.3: min_matches[j] = minMatches(n_j) with n_j = (j+1) k;
    conc[j][m] = 1 iff m >= minMatches(n_j) and the estimate after m of n_j
    matches is concentrated; est[j][m] = the posterior mode S^(m, n_j)."""
    params: Params
    min_matches: np.ndarray    # int32 [L]
    conc: np.ndarray           # uint8 [L][n_max+1]
    est: np.ndarray            # float64 [L][n_max+1]
    prune_prob: np.ndarray     # float64 [L][n_max+1] (Pr[S>=t|M], NaN where m > n)
    conc_prob: np.ndarray      # float64 [L][n_max+1] (NaN where not evaluated)
    scan_matches_search: bool  # linear scan and binary search agree


def tables(p: Params) -> Tables:
    """minMatches and the concentration cache for n = k, 2k, ..., n_max
    (Section 4.3, "Pre-computation of minimum matches", "Cache results of
    inference")."""
    L, W = p.levels, p.n_max + 1
    mm = np.zeros(L, np.int32)
    conc = np.zeros((L, W), np.uint8)
    est = np.zeros((L, W), np.float64)
    pr = np.zeros((L, W), np.float64)
    cp = np.zeros((L, W), np.float64)
    rc = lib().orc_tables(p.kind, p.t, p.eps, p.delta, p.gamma, p.alpha, p.beta, p.k, p.n_max,
                          _ptr(mm), _ptr(conc), _ptr(est), _ptr(pr), _ptr(cp))
    if rc == -1:
        raise ValueError("n_max must be a positive multiple of k")
    return Tables(p, mm, conc, est, pr, cp, rc == 0)


# --------------------------------------------------------------------------
# Algorithms 1 and 2
# --------------------------------------------------------------------------

@dataclass
class VerifyResult:
    status: np.ndarray   # uint8 [P]
    n_used: np.ndarray   # uint16 [P]
    m: np.ndarray        # uint16 [P]
    est: np.ndarray      # float64 [P]
    bad: int             # pairs naming an object >= N


def verify(tab: Tables, pairs: np.ndarray, sig: np.ndarray) -> VerifyResult:
    """Algorithm 1 (BayesLSH) over every pair, chunk by chunk, with the
    Section 4.3 tables."""
    p = tab.params
    pairs = _c(pairs, np.uint32).reshape(-1, 2)
    sig = _c(sig, np.uint32)
    P, N, Wd = len(pairs), sig.shape[0], sig.shape[1]
    need = p.n_max if p.kind == JACCARD else p.n_max // 32
    if Wd < need:
        raise ValueError("signature rows shorter than n_max hashes")
    st = np.zeros(P, np.uint8); nu = np.zeros(P, np.uint16); m = np.zeros(P, np.uint16)
    est = np.zeros(P, np.float64)
    bad = lib().orc_verify(p.kind, p.k, p.n_max, _ptr(tab.min_matches), _ptr(tab.conc), _ptr(tab.est),
                           _ptr(pairs), P, _ptr(sig), N, Wd, _ptr(st), _ptr(nu), _ptr(m), _ptr(est))
    return VerifyResult(st, nu, m, est, int(bad))


@dataclass
class LiteResult:
    status: np.ndarray   # uint8 [P]
    n_used: np.ndarray   # uint16 [P]
    sim: np.ndarray      # float64 [P], NaN for pruned pairs
    bad: int


def verify_lite(tab: Tables, pairs: np.ndarray, sig: np.ndarray, csr) -> LiteResult:
    """Algorithm 2 (BayesLSH-Lite): prune with up to h hashes, then the exact
    similarity of the survivors, kept iff s > t."""
    p = tab.params
    pairs = _c(pairs, np.uint32).reshape(-1, 2)
    sig = _c(sig, np.uint32)
    P, N, Wd = len(pairs), sig.shape[0], sig.shape[1]
    if p.h % p.k != 0 or p.h > p.n_max:
        raise ValueError("h must be a multiple of k and at most n_max")
    indptr = _c(csr.indptr, np.int64); idx = _c(csr.indices, np.uint32)
    vals = None if csr.values is None else _c(csr.values, np.float32)
    st = np.zeros(P, np.uint8); nu = np.zeros(P, np.uint16); sim = np.zeros(P, np.float64)
    bad = lib().orc_verify_lite(p.kind, p.k, p.h, _ptr(tab.min_matches), _ptr(pairs), P, _ptr(sig), N, Wd,
                                _ptr(indptr), _ptr(idx), _ptr(vals), p.t, _ptr(st), _ptr(nu), _ptr(sim))
    return LiteResult(st, nu, sim, int(bad))


def exact_jaccard(a: np.ndarray, b: np.ndarray) -> float:
    a = _c(a, np.uint32); b = _c(b, np.uint32)
    return lib().orc_exact_jaccard(_ptr(a), len(a), _ptr(b), len(b))


def exact_cosine(ia, va, ib, vb) -> float:
    ia = _c(ia, np.uint32); ib = _c(ib, np.uint32); va = _c(va, np.float32); vb = _c(vb, np.float32)
    return lib().orc_exact_cosine(_ptr(ia), _ptr(va), len(ia), _ptr(ib), _ptr(vb), len(ib))


# --------------------------------------------------------------------------
# Hashes and candidate generation
# --------------------------------------------------------------------------

def minhash(csr, a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """sig[i][j] = min over x in S_i of (a_j x + b_j) mod (2^31 - 1)
    (Section 4.1, "LSH family")."""
    a = _c(a, np.uint32); b = _c(b, np.uint32)
    indptr = _c(csr.indptr, np.int64); idx = _c(csr.indices, np.uint32)
    N = len(indptr) - 1
    sig = np.zeros((N, len(a)), np.uint32)
    lib().orc_minhash(_ptr(indptr), _ptr(idx), N, len(a), _ptr(a), _ptr(b), _ptr(sig))
    return sig


def srp_sparse(csr, R: np.ndarray) -> np.ndarray:
    """Bit j of row i = [x_i . r_j >= 0] (Section 4.2, "LSH family"), FP64
    sums in row order; R is [dim][bits] float32."""
    R = _c(R, np.float32)
    bits = R.shape[1]
    if bits % 32:
        raise ValueError("bits must be a multiple of 32")
    indptr = _c(csr.indptr, np.int64); idx = _c(csr.indices, np.uint32); val = _c(csr.values, np.float32)
    N = len(indptr) - 1
    sig = np.zeros((N, bits // 32), np.uint32)
    lib().orc_srp_sparse(_ptr(indptr), _ptr(idx), _ptr(val), N, _ptr(R), bits, _ptr(sig))
    return sig


def quantize_gaussian(x: np.ndarray):
    """Two-byte storage of Gaussian samples (Section 4.3): q = floor((x + 8)
    2^16 / 16), clamped to [0, 65535].  Returns (q, number clamped)."""
    x = _c(x, np.float32)
    q = np.zeros(x.shape, np.uint16)
    n = lib().orc_quantize_gaussian(_ptr(x), x.size, _ptr(q))
    return q, int(n)


def dequantize_gaussian(q: np.ndarray) -> np.ndarray:
    """q * 16 / 2^16 - 8 (Section 4.3)."""
    f = lib().orc_dequantize_gaussian
    return np.array([f(int(v)) for v in np.asarray(q).ravel()], np.float64).reshape(np.shape(q))


def splitmix64_at(seed: int, k: int) -> int:
    """Output k of the SplitMix64 stream started at `seed` (Steele, Lea and
    Flood 2014)."""
    return int(lib().orc_splitmix64_at(seed & (2 ** 64 - 1), k))


def gaussian_codes(seed: int, dim: int, bits: int, row0: int = 0) -> np.ndarray:
    """Two-byte codes (Section 4.3) of rows row0 .. row0+dim-1 of an R
    [.][bits] generated from a counter: entry c = t bits + j from SplitMix64
    outputs 3c..3c+2 of `seed`, twelve 16-bit integers summed (Irwin-Hall),
    x = (S - 393210) / 65536, code floor((x + 8) 2^16 / 16)."""
    codes = np.zeros((dim, bits), np.uint16)
    lib().orc_gaussian_codes(seed & (2 ** 64 - 1), row0, dim, bits, _ptr(codes))
    return codes


def srp_sparse_q16(csr, Rq: np.ndarray) -> np.ndarray:
    """Sparse SRP with R stored in two bytes per entry (Section 4.3): bit j of
    row i = [sum of x_e r(e, j) >= 0], r decoded from Rq [dim][bits] uint16,
    FP64 sums in row order."""
    Rq = _c(Rq, np.uint16)
    bits = Rq.shape[1]
    if bits % 32:
        raise ValueError("bits must be a multiple of 32")
    indptr = _c(csr.indptr, np.int64); idx = _c(csr.indices, np.uint32); val = _c(csr.values, np.float32)
    N = len(indptr) - 1
    sig = np.zeros((N, bits // 32), np.uint32)
    lib().orc_srp_sparse_q16(_ptr(indptr), _ptr(idx), _ptr(val), N, _ptr(Rq), bits, _ptr(sig))
    return sig


def srp_dense(X: np.ndarray, R: np.ndarray, want_dots: bool = False):
    """The same for dense rows X [N][d], R [d][bits]."""
    X = _c(X, np.float32); R = _c(R, np.float32)
    N, d = X.shape
    bits = R.shape[1]
    sig = np.zeros((N, bits // 32), np.uint32)
    dots = np.zeros((N, bits), np.float64) if want_dots else None
    lib().orc_srp_dense(_ptr(X), N, d, _ptr(R), bits, _ptr(sig), _ptr(dots))
    return (sig, dots) if want_dots else sig


def lsh_candidates(sig: np.ndarray, kind: int, rows: int, bands: int) -> np.ndarray:
    """Distinct pairs (x < y) that agree on all `rows` hashes of at least one
    of `bands` bands (Section 2, "Candidate generation via LSH"), sorted."""
    sig = _c(sig, np.uint32)
    N, Wd = sig.shape
    n = lib().orc_lsh_candidates(_ptr(sig), N, Wd, kind, rows, bands, None, 0)
    if n < 0:
        raise MemoryError("oracle banding ran out of memory")
    out = np.zeros((max(n, 1), 2), np.uint32)
    n2 = lib().orc_lsh_candidates(_ptr(sig), N, Wd, kind, rows, bands, _ptr(out), n)
    assert n2 == n
    return out[:n]


def allpairs_indexed(csr, t: float, kind: int) -> np.ndarray:
    """Per nonzero: 1 if its feature is an indexed feature of its row under
    AllPairs' prefix filter (features by decreasing frequency; the row's
    unindexed prefix bounds its contribution below t), else 0.  The
    comparison algorithm of Section 5.1 (Bayardo et al. 2007)."""
    indptr = _c(csr.indptr, np.int64); idx = _c(csr.indices, np.uint32)
    val = None if kind == JACCARD else _c(csr.values, np.float32)
    out = np.zeros(max(int(indptr[-1]), 1), np.uint8)
    if lib().orc_allpairs_indexed(_ptr(indptr), _ptr(idx), _ptr(val), len(indptr) - 1, int(csr.dim), float(t),
                                  kind, _ptr(out)) != 0:
        raise MemoryError("orc_allpairs_indexed")
    return out[: int(indptr[-1])]


def allpairs_candidates(csr, t: float, kind: int) -> np.ndarray:
    """AllPairs-style candidates: distinct pairs (x, y), x < y, with an indexed
    feature of x present in y, sorted by (x, y) (uint32 [P][2])."""
    indptr = _c(csr.indptr, np.int64); idx = _c(csr.indices, np.uint32)
    val = None if kind == JACCARD else _c(csr.values, np.float32)
    N = len(indptr) - 1
    n = lib().orc_allpairs_candidates(_ptr(indptr), _ptr(idx), _ptr(val), N, int(csr.dim), float(t), kind, None, 0)
    if n < 0:
        raise MemoryError("orc_allpairs_candidates")
    out = np.zeros((max(n, 1), 2), np.uint32)
    lib().orc_allpairs_candidates(_ptr(indptr), _ptr(idx), _ptr(val), N, int(csr.dim), float(t), kind, _ptr(out), n)
    return out[:n]


def lsh_bands_for(t: float, rows: int, eps: float) -> int:
    """l = ceil(log eps / log(1 - t^rows)) signatures of `rows` hashes each
    give an expected false-negative rate eps at similarity t (Section 2)."""
    return int(math.ceil(math.log(eps) / math.log(1.0 - t ** rows)))


def compact(status: np.ndarray, keep_mask: int) -> np.ndarray:
    """Indices of pairs whose status is in keep_mask, in input order."""
    status = _c(status, np.uint8)
    out = np.zeros(len(status), np.int64)
    n = lib().orc_compact(_ptr(status), len(status), keep_mask, _ptr(out))
    return out[:n]


def stop_hist(n_used: np.ndarray, k: int, levels: int) -> np.ndarray:
    """Number of pairs that stopped after chunk j (n = (j+1) k)."""
    n_used = _c(n_used, np.uint16)
    h = np.zeros(levels, np.uint64)
    lib().orc_stop_hist(_ptr(n_used), len(n_used), k, levels, _ptr(h))
    return h


def estimate_mle(kind: int, n: int, t: float, pairs: np.ndarray, sig: np.ndarray):
    """Section 3: m of the first n hashes agree, estimate m/n (Jaccard) or
    cos(pi (1 - m/n)) (cosine); Section 2: keep iff the estimate exceeds t."""
    pairs = _c(pairs, np.uint32).reshape(-1, 2)
    sig = _c(sig, np.uint32)
    P = len(pairs)
    m = np.zeros(P, np.uint16); est = np.zeros(P, np.float64); keep = np.zeros(P, np.uint8)
    lib().orc_estimate_mle(kind, n, t, _ptr(pairs), P, _ptr(sig), sig.shape[1], _ptr(m), _ptr(est), _ptr(keep))
    return m, est, keep


def fit_beta_prior(sims: np.ndarray):
    """Section 4.1: method-of-moments Beta(alpha, beta) from sampled
    similarities; returns (mean, var, alpha, beta, fallback)."""
    sims = _c(sims, np.float64)
    out = np.zeros(5, np.float64)
    lib().orc_fit_beta_prior(_ptr(sims), len(sims), _ptr(out))
    return tuple(out.tolist())
