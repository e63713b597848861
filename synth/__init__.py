"""Seeded synthetic workloads for BayesLSH candidate verification.

This module only draws random inputs: sets, sparse and dense vectors, the
coefficients of the minhash functions, the Gaussian projection vectors of the
sign-random-projection hashes and lists of candidate pairs.  It holds none of
the method's arithmetic (no hashing, no inference, no verification).  The CPU
oracle and the CUDA library both receive these arrays as inputs, so the random
numbers the method draws are fixed outside either of them.

The shapes follow the paper's workloads (Section 5, Table 1: tf-idf text with
average length 76-786 over 47k-344k dimensions; graph adjacency lists with
power-law degrees).  The paper's datasets themselves are not used.

Every generator is seeded.  Integer streams come from splitmix64 (Steele, Lea
and Flood, "Fast splittable pseudorandom number generators", 2014) or from
numpy's PCG64 generator.
"""
from __future__ import annotations

import math
import os
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass

import numpy as np

P31 = (1 << 31) - 1          # prime modulus of the minhash family (a*x+b) mod p
_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Outputs offset+1 .. offset+n of the splitmix64 counter stream for `seed`.

    Output i is mix(seed + i * 0x9E3779B97F4A7C15), mix being the
    published finaliser (xor-shift 30, multiply, xor-shift 27, multiply,
    xor-shift 31).  All arithmetic wraps modulo 2^64.
    """
    with np.errstate(over="ignore"):
        i = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + i * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniform01(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Doubles in [0, 1) with 53 random bits each, from splitmix64."""
    z = splitmix64(seed, n, offset)
    return (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def minhash_coeffs(n_hashes: int, seed: int) -> tuple[np.ndarray, np.ndarray]:
    """Coefficients of n_hashes functions h_j(x) = (a_j x + b_j) mod (2^31 - 1).

    a_j is drawn from [1, p-1] and b_j from [0, p-1] (reduction of 64-bit
    draws, bias below 2^-32).  Returned as uint32 arrays.
    """
    z = splitmix64(seed, 2 * n_hashes)
    a = (np.uint64(1) + z[0::2] % np.uint64(P31 - 1)).astype(np.uint32)
    b = (z[1::2] % np.uint64(P31)).astype(np.uint32)
    return a, b


def gaussian_matrix(rows: int, cols: int, seed: int, row_offset: int = 0,
                    chunk_rows: int = 4096) -> np.ndarray:
    """Standard normal float32 matrix [rows][cols] by Box-Muller in float64.

    Entry (r, c) uses splitmix64 draws 2*((row_offset+r)*cols+c) and the one
    after it: u1 in (0, 1], u2 in [0, 1), g = sqrt(-2 ln u1) cos(2 pi u2),
    rounded to float32.  Row r depends only on (seed, row_offset + r), so any
    row range can be regenerated on its own.
    """
    out = np.empty((rows, cols), dtype=np.float32)
    chunk_rows = max(1, min(chunk_rows, (1 << 20) // max(cols, 1)))

    def fill(r0):
        r1 = min(rows, r0 + chunk_rows)
        cnt = (r1 - r0) * cols
        z = splitmix64(seed, 2 * cnt, offset=2 * (row_offset + r0) * cols)
        u1 = ((z[0::2] >> np.uint64(11)).astype(np.float64) + 1.0) * (2.0 ** -53)
        u2 = (z[1::2] >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
        g = np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)
        out[r0:r1] = g.reshape(r1 - r0, cols).astype(np.float32)

    starts = range(0, rows, chunk_rows)
    if rows * cols >= (1 << 22):
        # numpy releases the GIL inside these ufuncs; chunks are independent
        with ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 1)) as ex:
            list(ex.map(fill, starts))
    else:
        for r0 in starts:
            fill(r0)
    return out


@dataclass
class CSR:
    """Rows of a sparse matrix: row i holds indices[indptr[i]:indptr[i+1]]
    (strictly increasing uint32) and, for real-valued rows, the float32
    values at the same positions."""
    indptr: np.ndarray            # int64 [N+1]
    indices: np.ndarray           # uint32 [nnz]
    values: np.ndarray | None     # float32 [nnz] or None for binary sets
    dim: int

    @property
    def n(self) -> int:
        return len(self.indptr) - 1

    def row(self, i: int):
        s, e = int(self.indptr[i]), int(self.indptr[i + 1])
        if self.values is None:
            return self.indices[s:e]
        return self.indices[s:e], self.values[s:e]


def _csr_from_rows(rows, dim, values=None) -> CSR:
    lens = np.fromiter((len(r) for r in rows), dtype=np.int64, count=len(rows))
    indptr = np.zeros(len(rows) + 1, dtype=np.int64)
    np.cumsum(lens, out=indptr[1:])
    idx = np.concatenate(rows).astype(np.uint32) if rows else np.zeros(0, np.uint32)
    vals = None
    if values is not None:
        vals = np.concatenate(values).astype(np.float32) if values else np.zeros(0, np.float32)
    return CSR(indptr, idx, vals, dim)


def _perturb(base: np.ndarray, frac: float, vocab: int, rng) -> np.ndarray:
    """Replace round(frac*|base|) elements of a set by fresh ids not in it."""
    nrep = int(round(frac * len(base)))
    keep = rng.permutation(base)[: len(base) - nrep]
    fresh = []
    taken = set(base.tolist())
    while len(fresh) < nrep:
        c = int(rng.integers(vocab))
        if c not in taken:
            taken.add(c)
            fresh.append(c)
    return np.unique(np.concatenate([keep, np.array(fresh, dtype=np.int64)]))


def jaccard_sets(n_sets: int = 2000, vocab: int = 10000, mean_size: float = 50.0,
                 sigma: float = 0.8, n_groups: int = 200, group_size=(2, 5),
                 frac=(0.1, 0.4), seed: int = 1) -> CSR:
    """Binary sets over a vocabulary, with planted near-duplicate groups.

    Sizes are lognormal with the given mean (mu = ln(mean) - sigma^2/2),
    clamped to [1, vocab].  Each of n_groups groups has 2-5 members derived
    from one base set by replacing a fraction f ~ U[frac] of its elements
    with fresh ids, so member-to-base Jaccard is (1-f)/(1+f).  The remaining
    sets are independent uniform draws.  Row order is shuffled.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    mu = math.log(mean_size) - sigma * sigma / 2.0

    def size():
        return int(min(vocab, max(1, round(rng.lognormal(mu, sigma)))))

    rows = []
    for _ in range(n_groups):
        if len(rows) >= n_sets:
            break
        base = np.sort(rng.choice(vocab, size=max(2, size()), replace=False))
        rows.append(base)
        for _ in range(int(rng.integers(group_size[0], group_size[1] + 1)) - 1):
            if len(rows) >= n_sets:
                break
            rows.append(_perturb(base, float(rng.uniform(*frac)), vocab, rng))
    while len(rows) < n_sets:
        rows.append(np.sort(rng.choice(vocab, size=size(), replace=False)))
    order = rng.permutation(len(rows))
    return _csr_from_rows([rows[i] for i in order], vocab)


def _zipf_terms(rng, cdf, perm, nnz):
    """nnz distinct term ids with Zipf rank probabilities, mapped by perm."""
    got: list[int] = []
    seen = set()
    while len(got) < nnz:
        draw = np.searchsorted(cdf, rng.random(2 * (nnz - len(got)) + 8), side="right")
        for r in draw.tolist():
            if r not in seen:
                seen.add(r)
                got.append(r)
                if len(got) == nnz:
                    break
    return perm[np.array(got, dtype=np.int64)]


def tfidf_vectors(n_docs: int = 20000, dim: int = 100000, zipf_s: float = 1.1,
                  mean_nnz: float = 80.0, sigma: float = 0.8, n_groups: int = 200,
                  group_size=(2, 5), frac=(0.1, 0.4), seed: int = 2) -> CSR:
    """tf-idf-like sparse float32 vectors, L2-normalised, with planted groups.

    Term ranks follow Zipf(zipf_s) over dim ranks, drawn without replacement
    within a document and mapped to ids by a fixed random permutation.  nnz is
    lognormal with the given mean.  Term frequency tf = 1 + Geometric(0.5);
    weight = log(1+tf) * ln(N/df) (df counted over the generated corpus,
    floored at 1), then each row is scaled to unit L2 norm (in float64,
    rounded to float32).  Group members copy a base document's terms and
    replace a fraction f ~ U[frac] of them with fresh Zipf draws; their tf
    values are redrawn.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    ranks = np.arange(1, dim + 1, dtype=np.float64)
    pmf = ranks ** (-zipf_s)
    cdf = np.cumsum(pmf / pmf.sum())
    cdf[-1] = 1.0
    perm = rng.permutation(dim)
    mu = math.log(mean_nnz) - sigma * sigma / 2.0

    def nnz():
        return int(min(dim, max(1, round(rng.lognormal(mu, sigma)))))

    term_rows = []
    for _ in range(n_groups):
        if len(term_rows) >= n_docs:
            break
        base = _zipf_terms(rng, cdf, perm, max(2, nnz()))
        term_rows.append(base)
        for _ in range(int(rng.integers(group_size[0], group_size[1] + 1)) - 1):
            if len(term_rows) >= n_docs:
                break
            f = float(rng.uniform(*frac))
            nrep = int(round(f * len(base)))
            keep = rng.permutation(base)[: len(base) - nrep]
            taken = set(keep.tolist())
            extra = [t for t in _zipf_terms(rng, cdf, perm, nrep + 16).tolist() if t not in taken]
            term_rows.append(np.concatenate([keep, np.array(extra[:nrep], dtype=np.int64)]))
    while len(term_rows) < n_docs:
        term_rows.append(_zipf_terms(rng, cdf, perm, nnz()))
    order = rng.permutation(len(term_rows))
    term_rows = [np.sort(term_rows[i]) for i in order]
    df = np.zeros(dim, dtype=np.int64)
    for r in term_rows:
        df[r] += 1
    idf = np.log(len(term_rows) / np.maximum(df, 1))
    vals = []
    for r in term_rows:
        tf = 1 + rng.geometric(0.5, size=len(r))
        w = np.log1p(tf) * idf[r]
        nrm = math.sqrt(float(np.dot(w, w)))
        if nrm == 0.0:
            w = np.ones(len(r))
            nrm = math.sqrt(len(r))
        vals.append((w / nrm).astype(np.float32))
    return _csr_from_rows(term_rows, dim, vals)


def chung_lu_sets(n_nodes: int = 1_000_000, exponent: float = 2.1, mean_degree: float = 30.0,
                  i0: float = 10.0, seed: int = 3) -> CSR:
    """Adjacency sets of a Chung-Lu random graph with power-law degrees.

    Node weights w_i = (i + i0)^(-1/(exponent-1)) scaled to the given mean
    degree; n_nodes*mean_degree/2 edges are drawn with both endpoints
    proportional to w; self-loops and duplicate edges are dropped.  A node
    left without edges gets one, to a node drawn proportional to w, so that
    no adjacency set is empty (graph datasets list only nodes with edges).
    Row i is the sorted neighbour set of node i.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    w = (np.arange(n_nodes, dtype=np.float64) + i0) ** (-1.0 / (exponent - 1.0))
    cdf = np.cumsum(w / w.sum())
    cdf[-1] = 1.0
    m = int(n_nodes * mean_degree / 2)
    u = np.searchsorted(cdf, rng.random(m), side="right").astype(np.int64)
    v = np.searchsorted(cdf, rng.random(m), side="right").astype(np.int64)
    keep = u != v
    u, v = u[keep], v[keep]
    a = np.minimum(u, v)
    b = np.maximum(u, v)
    key = np.unique(a * n_nodes + b)
    a, b = key // n_nodes, key % n_nodes
    lonely = np.setdiff1d(np.arange(n_nodes, dtype=np.int64), np.concatenate([a, b]))
    if lonely.size:
        partner = np.searchsorted(cdf, rng.random(lonely.size), side="right").astype(np.int64)
        partner = np.where(partner == lonely, (partner + 1) % n_nodes, partner)
        key = np.unique(np.concatenate([key, np.minimum(lonely, partner) * n_nodes + np.maximum(lonely, partner)]))
        a, b = key // n_nodes, key % n_nodes
    src = np.concatenate([a, b])
    dst = np.concatenate([b, a])
    order = np.lexsort((dst, src))
    src, dst = src[order], dst[order]
    indptr = np.zeros(n_nodes + 1, dtype=np.int64)
    np.cumsum(np.bincount(src, minlength=n_nodes), out=indptr[1:])
    return CSR(indptr, dst.astype(np.uint32), None, n_nodes)


def gaussian_mixture(n_points: int = 1_000_000, dim: int = 256, n_centers: int = 10000,
                     sigma_within: float = 0.15, seed: int = 4) -> np.ndarray:
    """Dense float32 points [n][dim]: a centre uniform on the unit sphere plus
    N(0, sigma_within^2/dim * I) noise (so the noise norm is about
    sigma_within).  Centres are chosen with equal weights."""
    rng = np.random.Generator(np.random.PCG64(seed))
    centers = rng.standard_normal((n_centers, dim))
    centers /= np.linalg.norm(centers, axis=1, keepdims=True)
    out = np.empty((n_points, dim), dtype=np.float32)
    step = 65536
    scale = sigma_within / math.sqrt(dim)
    for s in range(0, n_points, step):
        e = min(n_points, s + step)
        c = rng.integers(n_centers, size=e - s)
        out[s:e] = (centers[c] + scale * rng.standard_normal((e - s, dim))).astype(np.float32)
    return out


def random_pairs(n_objects: int, n_pairs: int, seed: int = 5) -> np.ndarray:
    """n_pairs uniform pairs (x, y) with x < y, uint32 [n_pairs][2]
    (duplicates possible)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    x = rng.integers(n_objects, size=n_pairs, dtype=np.int64)
    y = rng.integers(n_objects - 1, size=n_pairs, dtype=np.int64)
    y = np.where(y >= x, y + 1, y)
    return np.stack([np.minimum(x, y), np.maximum(x, y)], axis=1).astype(np.uint32)


def bernoulli_signatures(sims: np.ndarray, n_hashes: int, kind: str, seed: int = 6):
    """Signature pairs whose hashes agree independently with probability
    sims[i] (the LSH model: Pr[h(x) = h(y)] = sim).

    Returns (sig, pairs): sig has 2*len(sims) rows, pair i is (2i, 2i+1).
    For kind 'jaccard' rows hold n_hashes uint32 values; for 'cosine' rows
    hold n_hashes/32 uint32 words of packed bits (bit j in word j/32, bit
    j%32).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    P = len(sims)
    agree = rng.random((P, n_hashes)) < np.asarray(sims, dtype=np.float64)[:, None]
    if kind == "jaccard":
        x = rng.integers(0, P31, size=(P, n_hashes), dtype=np.int64)
        y = np.where(agree, x, (x + 1 + rng.integers(0, P31 - 1, size=(P, n_hashes))) % P31)
        sig = np.empty((2 * P, n_hashes), dtype=np.uint32)
        sig[0::2], sig[1::2] = x, y
    else:
        assert n_hashes % 32 == 0
        xb = rng.random((P, n_hashes)) < 0.5
        yb = np.where(agree, xb, ~xb)
        w = np.uint64(1) << np.arange(32, dtype=np.uint64)

        def pack(bits):
            b = bits.reshape(P, n_hashes // 32, 32).astype(np.uint64)
            return (b * w).sum(axis=2).astype(np.uint32)
        sig = np.empty((2 * P, n_hashes // 32), dtype=np.uint32)
        sig[0::2], sig[1::2] = pack(xb), pack(yb)
    pairs = np.stack([np.arange(0, 2 * P, 2), np.arange(1, 2 * P, 2)], axis=1).astype(np.uint32)
    return sig, pairs


def large_tfidf_device(n_docs: int = 5_000_000, dim: int = 1 << 24, zipf_s: float = 1.1,
                       nnz_min: int = 5, nnz_max: int = 20000, nnz_exp: float = 2.0,
                       n_groups: int = 100_000, group_size=(2, 5), frac=(0.1, 0.4), seed: int = 9,
                       device=None):
    """tf-idf-like sparse vectors at a scale the host cannot draw quickly
    (5e6 documents, ~2e8 nonzeros), drawn on the GPU with torch's seeded
    generator and returned as device tensors (indptr int64 [N+1], indices
    int32 holding uint32 term ids, values float32).

    Row lengths follow a power law p(l) ~ l^-nnz_exp on [nnz_min, nnz_max]
    (inverse CDF of the continuous law, floored).  Term ranks follow
    Zipf(zipf_s) over dim ranks by the inverse CDF of the continuous law
    (rank = floor((1 + u (dim^(1-s) - 1))^(1/(1-s)))), mapped to ids by a
    fixed random permutation; repeated draws within a row merge into one term
    whose tf is the number of draws plus a Geometric(0.5) extra.  The first
    rows form n_groups planted groups: a base document followed by 1..4
    variants that redraw a fraction f ~ U[frac] of its draws.  weight =
    log(1+tf) ln(N/df), each row scaled to unit L2 norm (in float64, rounded
    to float32; a row whose weights are all 0 keeps them).
    """
    import torch

    dev = torch.device("cuda", 0) if device is None else device
    g = torch.Generator(device=dev)
    g.manual_seed(seed)
    f64 = torch.float64

    def lengths(k):
        u = torch.rand(k, generator=g, device=dev, dtype=f64)
        e = 1.0 - nnz_exp
        lo, hi = float(nnz_min), float(nnz_max + 1)
        x = (lo ** e + u * (hi ** e - lo ** e)) ** (1.0 / e)
        return x.floor().clamp(nnz_min, nnz_max).to(torch.int64)

    perm = torch.randperm(dim, generator=g, device=dev)

    def terms(k):
        u = torch.rand(k, generator=g, device=dev, dtype=f64)
        e = 1.0 - zipf_s
        r = (1.0 + u * (float(dim) ** e - 1.0)) ** (1.0 / e)
        return perm[(r.floor().clamp(1, dim) - 1).to(torch.int64)]

    # group structure: rows [0, n_grouped) are groups (base first), the rest independent
    sizes = torch.randint(group_size[0], group_size[1] + 1, (n_groups,), generator=g, device=dev)
    starts = torch.cumsum(sizes, 0) - sizes
    n_grouped = int(sizes.sum().item())
    if n_grouped > n_docs:
        raise ValueError("planted groups exceed the document count")
    member = torch.arange(n_grouped, device=dev)
    group_of = torch.repeat_interleave(torch.arange(n_groups, device=dev), sizes)
    base_row = starts[group_of]                          # row of each grouped member's base
    is_base = member == base_row
    # draws of every base and independent row
    own = torch.ones(n_docs, dtype=torch.bool, device=dev)
    own[:n_grouped] = is_base
    lens = lengths(n_docs)
    lens = torch.where(own, lens, lens[torch.cat([base_row, torch.arange(n_grouped, n_docs, device=dev)])])
    row_of = torch.repeat_interleave(torch.arange(n_docs, device=dev), lens)
    total = row_of.numel()
    ids = terms(total)
    # variants copy their base's draws and redraw a fraction f of them
    first = torch.cumsum(lens, 0) - lens
    var = ~own
    if bool(var.any()):
        f = torch.empty(n_docs, device=dev, dtype=f64).uniform_(frac[0], frac[1], generator=g)
        pos = torch.arange(total, device=dev) - first[row_of]          # draw index within the row
        src_row = torch.cat([base_row, torch.arange(n_grouped, n_docs, device=dev)])[row_of]
        copied = ids[first[src_row] + pos]
        keep = torch.rand(total, generator=g, device=dev, dtype=f64) >= f[row_of]
        ids = torch.where(var[row_of] & keep, copied, ids)
    # merge repeated terms within a row; tf = draws + Geometric(0.5)
    key, draws = torch.unique(row_of * dim + ids, sorted=True, return_counts=True)
    rows = key // dim
    ids = key - rows * dim
    u = torch.rand(key.numel(), generator=g, device=dev, dtype=f64).clamp_min(1e-300)
    tf = draws.to(f64) + torch.floor(torch.log(u) / math.log(0.5))
    df = torch.bincount(ids, minlength=dim)
    w = torch.log1p(tf) * torch.log(n_docs / df[ids].clamp_min(1).to(f64))
    nrm = torch.zeros(n_docs, dtype=f64, device=dev).index_add_(0, rows, w * w).sqrt()
    w = torch.where(nrm[rows] > 0, w / nrm[rows].clamp_min(1e-300), w)
    indptr = torch.zeros(n_docs + 1, dtype=torch.int64, device=dev)
    indptr[1:] = torch.cumsum(torch.bincount(rows, minlength=n_docs), 0)
    return indptr, ids.to(torch.int32), w.to(torch.float32)
