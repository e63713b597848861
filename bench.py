#!/usr/bin/env python
"""Benchmark of BayesLSH candidate verification on GB300.

A step is one pass of the whole verification path over one batch of
synthetic objects, every stage in libblsh's CUDA kernels:
  sign random projections of the sparse rows (the first lazy_bits bits of
  every object; Section 3's lazy hashing) -> LSH banding candidates ->
  Algorithms 1 (BayesLSH) and 2 (Lite) over every candidate in one pass,
  Algorithm 1 stopping at the computed hashes -> the remaining hashes of the
  objects of the pairs still open -> Algorithm 1 finished for those pairs ->
  compaction of both output sets.
The inference tables (Section 4.3) are built once per parameter set before the
timed region (their build time is reported separately).

Default workload (large-mixed): 5,000,000 tf-idf-like sparse float32 vectors
over a 2^24-term vocabulary (Zipf(1.1) term ids, power-law lengths on
[5, 20,000], 100,000 planted near-duplicate groups; drawn on the GPU), 2,048
SRP bits over a projection matrix stored as two-byte Gaussian codes generated
on the device (68.7 GB), banding 16 bits x 5 bands (about 1e9 candidates),
t = 0.6, eps = 0.03, delta = 0.05, gamma = 0.03, k = 32, Lite h = 128, the
first 256 bits hashed for every object; candidates verified in device-resident
batches sized by free HBM (--batch-pairs caps them).

Output: one JSON line (rank 0).  `value` is candidate pairs verified per
second for the whole job; `e2e` the same through the public API with the
objects copied from pinned host memory and the output sets copied back inside
the timed region; `cpu_baseline` the oracle on the host cores on a seeded
sample, extrapolated to the whole step.

  python bench.py [--steps K] [--warmup W] [--workload NAME] [--impl ours|reference]
                  [--lazy-bits L] [--batch-pairs B] [--profile-step] [--no-graph] [--no-cpu-baseline]

Other workloads: cosine-small (20,000 tf-idf vectors, dim 100,000), jaccard-small,
batching (1M Chung-Lu sets), precision (1M dense points, tensor-core
projection), cosine-small-q16 (two-byte R), verify-large (Algorithm 1 alone at
HBM scale), sweep (the gamma/delta/eps study), and the small *-profile shapes
for ncu captures.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "candidate pairs verified/s at fixed t,ε,δ,γ; verify HBM GB/s vs peak; hashes/s"

WORKLOADS = {
    "cosine-small": dict(kind=1, n=20000, dim=100000, mean_nnz=80.0, bits=2048, rows=8, bands=35, t=0.7,
                         n_max=2048, k=32, h=128, seed=2, lazy_bits=512,
                         text="cosine, BayesLSH + Lite: N=20,000 tf-idf sparse float32 vectors, dim 100,000, "
                              "Zipf(1.1) term ids, lognormal nnz (mean 80), 2,048 SRP bits, banding 8x35, "
                              "t=0.7, eps=0.03, delta=0.05, gamma=0.03, k=32, h=128"),
    "cosine-small-q16": dict(kind=1, n=20000, dim=100000, mean_nnz=80.0, bits=2048, rows=8, bands=35, t=0.7,
                             n_max=2048, k=32, h=128, seed=2, r_format="q16",
                             text="cosine-small with the projection matrix stored as two-byte codes "
                                  "(Section 4.3): N=20,000 tf-idf vectors, dim 100,000, 2,048 SRP bits, "
                                  "banding 8x35, t=0.7"),
    "allpairs-cosine": dict(kind=1, n=20000, dim=100000, mean_nnz=80.0, bits=2048, rows=8, bands=35, t=0.7,
                            n_max=2048, k=32, h=128, seed=2, lazy_bits=512, candidates="allpairs",
                            text="cosine-small's 20,000 tf-idf vectors with candidates from AllPairs-style prefix "
                                 "filtering (Section 5.1's other candidate generator) instead of LSH banding, "
                                 "then BayesLSH + Lite over them: 2,048 SRP bits, t=0.7"),
    "cosine-profile": dict(kind=1, n=6000, dim=30000, mean_nnz=80.0, bits=2048, rows=8, bands=35, t=0.7,
                           n_max=2048, k=32, h=128, seed=2,
                           text="cosine-small shape at 6,000 vectors over dim 30,000 (R = 245 MB > L2), for "
                                "ncu captures"),
    "verify-large": dict(kind=1, gpu_only=True, n=5_000_000, bits=2048, pairs=200_000_000, t=0.7, n_max=2048, k=32, h=128,
                         seed=9, text="verification only: 5,000,000 random 2,048-bit signatures (1.3 GB) and "
                                      "200,000,000 uniform random candidate pairs (HBM-resident, no reuse)"),
    "large-mixed": dict(kind=1, gpu_only=True, n=5_000_000, dim=1 << 24, bits=2048, rows=16, bands=5, t=0.6,
                        n_max=2048, k=32, h=128, seed=9, r_seed=31, lazy_bits=256,
                        text="cosine, BayesLSH + Lite on N=5,000,000 tf-idf sparse float32 vectors over a 2^24-term "
                             "vocabulary (Zipf(1.1) ranks, power-law lengths l^-2 on [5, 20,000], 100,000 planted "
                             "near-duplicate groups; drawn on the GPU), 2,048 SRP bits over R as two-byte Gaussian "
                             "codes generated on the device (68.7 GB), banding 16x5, t=0.6, eps=0.03, delta=0.05, "
                             "gamma=0.03, k=32, h=128; candidates verified in device-resident batches sized by "
                             "free HBM"),
    "large-profile": dict(kind=1, gpu_only=True, n=600_000, dim=1 << 19, bits=1024, rows=16, bands=5, t=0.6,
                          n_max=1024, k=32, h=128, seed=9, r_seed=31, lazy_bits=256, n_groups=10000,
                          text="large-mixed shape for ncu captures: 600,000 tf-idf vectors over 2^19 terms, 1,024 "
                               "bits from device-generated two-byte codes (1.1 GB; the code rows the nonzeros touch "
                               "exceed L2), the 256-bit lazy prefix, banding 16x5, t=0.6"),
    "verify-profile": dict(kind=1, gpu_only=True, n=1_500_000, bits=2048, pairs=50_000_000, t=0.7, n_max=2048,
                           k=32, h=128, seed=9,
                           text="verify-large shape for ncu captures: 1,500,000 random 2,048-bit signatures (384 MB) "
                                "and 50,000,000 random pairs"),
    "jaccard-small": dict(kind=0, n=2000, vocab=10000, n_hashes=256, rows=8, bands=32, t=0.7, n_max=256, k=32,
                          h=64, seed=1,
                          text="jaccard, BayesLSH + Lite: N=2,000 sets over vocab 10,000, lognormal sizes "
                               "(mean 50), 200 planted groups, 256 minhashes, banding 8x32, t=0.7"),
    "precision": dict(kind=1, dense=True, n=1_000_000, d=256, n_centers=10000, sigma=0.15, bits=1024, rows=16,
                      bands=64, t=0.8, n_max=1024, k=32, h=128, margin=1e-3, seed=4,
                      stages=("hash", "band", "verify", "compact"),
                      text="cosine, BayesLSH + Lite on dense rows: N=1,000,000 float32 embeddings, d=256, "
                           "10,000-component Gaussian mixture (noise norm 0.15), 1,024 SRP bits by the BF16 "
                           "tensor-core projection with FP32/FP64 recheck below 1e-3 |x||r|, banding 16x64, t=0.8 "
                           "(BayesLSH; no Lite pass)"),
    "sweep": dict(kind=1, seed=2, gpu_only=True, text="cosine-small candidates (2.66e7 pairs), gamma, delta, epsilon each "
                                         "over 0.01..0.09 with the others at 0.05, t = 0.7"),
    "precision-profile": dict(kind=1, dense=True, n=200_000, d=256, n_centers=2000, sigma=0.15, bits=1024, rows=16,
                              bands=64, t=0.8, n_max=1024, k=32, h=128, margin=1e-3, seed=4,
                              stages=("hash", "band", "verify", "compact"),
                              text="precision shape at 200,000 points (X = 205 MB > L2), for ncu captures"),
    "batching": dict(kind=0, n=1_000_000, n_hashes=256, rows=3, bands=32, t=0.5, n_max=256, k=32, h=64, seed=3,
                     tune_k=(32, 64, 128),
                     text="jaccard, BayesLSH + Lite: Chung-Lu graph N=1,000,000, exponent 2.1, mean degree 30, "
                          "256 minhashes, banding 3x32 (power-law buckets, about 1e8 candidate pairs), t=0.5"),
}


# ---------------------------------------------------------------------------
# workload
# ---------------------------------------------------------------------------

def dense_csr(X: np.ndarray) -> synth.CSR:
    """Dense rows as CSR (every coordinate present), for Lite's exact cosine."""
    N, d = X.shape
    return synth.CSR(np.arange(0, N * d + 1, d, dtype=np.int64), np.tile(np.arange(d, dtype=np.uint32), N),
                     X.reshape(-1), d)


def make_inputs(w: dict, rank: int = 0):
    seed = w["seed"] + 1000 * rank
    if w.get("dense"):
        X = synth.gaussian_mixture(n_points=w["n"], dim=w["d"], n_centers=w["n_centers"],
                                   sigma_within=w["sigma"], seed=seed)
        R = synth.gaussian_matrix(w["d"], w["bits"], seed=seed + 1)
        objs = dense_csr(X)
        objs.X = X
        return objs, R
    if w["kind"] == 1:
        objs = synth.tfidf_vectors(n_docs=w["n"], dim=w["dim"], mean_nnz=w["mean_nnz"], seed=seed)
        R = synth.gaussian_matrix(w["dim"], w["bits"], seed=seed + 1)
        return objs, R
    if "vocab" in w:
        objs = synth.jaccard_sets(n_sets=w["n"], vocab=w["vocab"], seed=seed)
    else:
        objs = synth.chung_lu_sets(n_nodes=w["n"], seed=seed)
    a, b = synth.minhash_coeffs(w["n_hashes"], seed=seed + 1)
    return objs, (a, b)


class Pipeline:
    """Device buffers and the library calls of one step."""

    def __init__(self, B, torch, w: dict, objs, hashp, device):
        self.B, self.torch, self.w, self.dev = B, torch, w, device
        t = torch
        self.ctx = B.Context(device.index or 0)
        self.kind = w["kind"]
        N = objs.n
        self.N = N
        B.blsh_ctx_reserve(self.ctx, N)          # the hot calls allocate nothing
        u32 = lambda a: t.from_numpy(np.ascontiguousarray(a).view(np.int32)).to(device)
        self.indptr = t.from_numpy(objs.indptr).to(device)
        self.indices = u32(objs.indices) if objs.indices.size else t.zeros(1, dtype=t.int32, device=device)
        self.values = None if objs.values is None else t.from_numpy(objs.values).to(device)
        self.dense = bool(w.get("dense"))
        if self.dense:
            # X [N][d] shares its storage with the CSR values Lite reads
            self.X = self.values.view(N, w["d"])
            self.dense_ws = t.zeros(max(1, B.blsh_srp_dense_workspace(N, w["d"], w["bits"])), dtype=t.uint8,
                                    device=device)
        if self.kind == 1:
            self.R = t.from_numpy(hashp).to(device)
            self.W = w["bits"] // 32
            if w.get("r_format") == "q16":
                self.Rq = B.blsh_quantize_gaussian(self.ctx, self.R)
                B.blsh_status(self.ctx)
                del self.R
        else:
            self.a, self.b = u32(hashp[0]), u32(hashp[1])
            self.W = w["n_hashes"]
        self.sig = t.zeros((N, self.W), dtype=t.int32, device=device)
        self.need = t.zeros(N, dtype=t.uint8, device=device)
        params = B.make_params(kind=self.kind, t=w["t"], k=w["k"], n_max=w["n_max"], h=w["h"])
        t0 = time.perf_counter()
        self.tab = B.blsh_tables_build(self.ctx, params)
        self.tables_ms = (time.perf_counter() - t0) * 1e3
        self.n_pairs = t.zeros(1, dtype=t.int64, device=device)
        self.allpairs = w.get("candidates") == "allpairs"
        self.dim = objs.dim
        self.nnz = int(objs.indptr[-1])
        self.hash()
        if self.allpairs:
            # candidates by prefix filtering: a count-only call sizes the key
            # buffer, a full one the pair count
            self.n_dups = t.zeros(1, dtype=t.int64, device=device)
            ws0 = t.zeros(B.blsh_allpairs_workspace(N, self.nnz, self.dim, 0), dtype=t.uint8, device=device)
            B.blsh_allpairs_candidates(self.ctx, self.indptr, self.indices, self.values, self.dim, w["t"], self.kind,
                                       None, self.n_pairs, ws0, 0, self.n_dups, nnz=self.nnz)
            B.blsh_status(self.ctx)
            self.max_dups = int(self.n_dups.item())
            del ws0
            self.ws = t.zeros(B.blsh_allpairs_workspace(N, self.nnz, self.dim, self.max_dups), dtype=t.uint8,
                              device=device)
            self.pairs = t.zeros((max(self.max_dups, 1), 2), dtype=t.int32, device=device)
            self.band()
            B.blsh_status(self.ctx)
        else:
            self.ws = t.zeros(B.blsh_lsh_candidates_workspace(N, self.kind, w["rows"], w["bands"]), dtype=t.uint8,
                              device=device)
            # size the candidate buffer with a count-only pass
            B.blsh_lsh_candidates(self.ctx, self.sig, self.kind, w["rows"], w["bands"], None, self.n_pairs, self.ws)
            B.blsh_status(self.ctx)
        self.P = int(self.n_pairs.item())
        cap = self.P + 1024
        if not self.allpairs:
            self.pairs = t.zeros((cap, 2), dtype=t.int32, device=device)
        self.status = t.zeros(cap, dtype=t.uint8, device=device)
        self.n_used = t.zeros(cap, dtype=t.int16, device=device)
        self.m = t.zeros(cap, dtype=t.int16, device=device)
        self.est = t.full((cap,), float("nan"), dtype=t.float32, device=device)   # pruned pairs' entries stay NaN
        self.hist = t.zeros(self.tab.levels, dtype=t.int64, device=device)
        self.lstatus = t.zeros(cap, dtype=t.uint8, device=device)
        self.sim = t.full((cap,), float("nan"), dtype=t.float64, device=device)
        self.out1 = t.zeros(cap, dtype=t.int64, device=device)
        self.out2 = t.zeros(cap, dtype=t.int64, device=device)
        self.n_out = t.zeros(2, dtype=t.int64, device=device)
        self.band()
        B.blsh_status(self.ctx)
        # autotune the verification plan on the real candidates (with the
        # chunk size k too, where the workload asks for it)
        self.k_ms = None
        if w.get("tune_k"):
            tab, self.plan, self.k_ms = B.blsh_autotune_k(self.ctx, params, w["tune_k"], self.pairs[: self.P],
                                                          self.sig, self.status[: self.P], self.n_used[: self.P],
                                                          self.m[: self.P], self.est[: self.P])
            self.tab.close()
            self.tab = tab
            w["k"], w["h"] = tab.params.k, tab.params.h
            self.hist = t.zeros(self.tab.levels, dtype=t.int64, device=device)
        else:
            self.plan = B.blsh_autotune(self.ctx, self.tab, self.pairs[: self.P], self.sig, self.status[: self.P],
                                        self.n_used[: self.P], self.m[: self.P], self.est[: self.P])
        B.blsh_status(self.ctx)
        self.est.fill_(float("nan"))   # autotune's estimates (from the lazily hashed prefix) are not outputs

    # the stages of a step, each one library call
    @property
    def lazy_bits(self):
        """Hashes computed for every object (the rest only for the objects of
        pairs still undecided after them: Section 3, lazy hashing); 0 = all."""
        lazy = self.kind == 1 and not self.dense and "r_format" not in self.w and self.with_lite
        L = self.w.get("lazy_bits", 0) if lazy else 0
        if 0 < L < self.w["rows"] * self.w["bands"]:
            raise ValueError(f"lazy_bits={L} leaves hashes that banding reads ({self.w['rows']} x {self.w['bands']})")
        return L if 0 < L < self.w["bits"] else 0

    def hash(self):
        B = self.B
        if self.lazy_bits:
            B.blsh_srp_sparse_cols(self.ctx, self.indptr, self.indices, self.values, self.R, self.sig, 0,
                                   self.lazy_bits)
        elif self.dense:
            B.blsh_srp_dense(self.ctx, self.X, self.R, self.sig, margin=self.w["margin"], workspace=self.dense_ws)
        elif self.kind == 1 and self.w.get("r_format") == "q16":
            B.blsh_srp_sparse_q16(self.ctx, self.indptr, self.indices, self.values, self.Rq, self.sig)
        elif self.kind == 1:
            B.blsh_srp_sparse(self.ctx, self.indptr, self.indices, self.values, self.R, self.sig)
        else:
            B.blsh_minhash(self.ctx, self.indptr, self.indices, self.W, self.a, self.b, self.sig)

    def band(self):
        w = self.w
        if self.allpairs:
            self.B.blsh_allpairs_candidates(self.ctx, self.indptr, self.indices, self.values, self.dim, w["t"],
                                            self.kind, self.pairs, self.n_pairs, self.ws, self.max_dups,
                                            nnz=self.nnz)
            return
        self.B.blsh_lsh_candidates(self.ctx, self.sig, self.kind, w["rows"], w["bands"], self.pairs, self.n_pairs,
                                   self.ws)

    def verify(self):
        if self.lazy_bits and self.with_lite:
            # the first lazy_bits hashes decide most pairs; the others mark
            # their objects in `need` and are finished by hash_rest + resume
            self.need.zero_()
            self.B.blsh_verify_both_capped(self.ctx, self.tab, self.lazy_bits, self.pairs, self.sig, self.status,
                                           self.n_used, self.m, self.est, self.hist, self.indptr, self.indices,
                                           self.values, self.lstatus, self.sim, self.need, P_dev=self.n_pairs)
        elif self.with_lite:   # Algorithms 1 and 2 in one pass over the candidates
            self.B.blsh_verify_both(self.ctx, self.tab, self.pairs, self.sig, self.status, self.n_used, self.m,
                                    self.est, self.hist, self.indptr, self.indices, self.values, self.lstatus,
                                    self.sim, P_dev=self.n_pairs)
        else:
            self.B.blsh_verify(self.ctx, self.tab, self.pairs, self.sig, self.status, self.n_used, self.m,
                               self.est, self.hist, P_dev=self.n_pairs)

    def hash_rest(self):
        """The remaining hashes of the objects marked in `need`."""
        L = self.lazy_bits
        self.B.blsh_srp_sparse_cols(self.ctx, self.indptr, self.indices, self.values, self.R, self.sig, L,
                                    self.w["bits"] - L, row_mask=self.need)

    def resume(self):
        """Algorithm 1 for the pairs the first lazy_bits hashes left open."""
        self.B.blsh_verify_resume(self.ctx, self.tab, self.pairs, self.sig, self.status, self.n_used, self.m,
                                  self.est, self.hist, P_dev=self.n_pairs)

    def lite(self):
        self.B.blsh_verify_lite(self.ctx, self.tab, self.pairs, self.sig, self.indptr, self.indices, self.values,
                                self.lstatus, self.sim, P_dev=self.n_pairs)

    def compact(self):
        B = self.B
        B.blsh_compact(self.ctx, self.status, (1 << B.ACCEPT) | (1 << B.ACCEPT_AT_MAX), self.out1, self.n_out[0:1],
                       P_dev=self.n_pairs)
        if self.with_lite:
            B.blsh_compact(self.ctx, self.lstatus, 1 << B.LITE_ACCEPT, self.out2, self.n_out[1:2],
                           P_dev=self.n_pairs)

    @property
    def with_lite(self):
        return "lite" in self.w.get("stages", ("lite",))

    @property
    def STAGES(self):
        """The stages of a step, each one library call ("verify" runs both
        algorithms when the workload has Lite; with lazy hashing it stops at
        lazy_bits hashes and hash_rest + resume finish the open pairs)."""
        if self.lazy_bits and self.with_lite:
            return ("hash", "band", "verify", "hash_rest", "resume", "compact")
        return ("hash", "band", "verify", "compact")

    def step(self):
        for s in self.STAGES:
            getattr(self, s)()


# ---------------------------------------------------------------------------
# measurement helpers
# ---------------------------------------------------------------------------

class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines: list[str] = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# DRAM bytes (read + write) of a kernel's launches in one step, from one ncu
# capture of the kernel as it stands (dram__bytes_read.sum +
# dram__bytes_write.sum of the bench step under --profile-step); reported as
# the roofline's traffic for the workload it was taken on (per step, like the
# algorithmic bytes), and to be taken again whenever the kernel changes.
NCU_TRAFFIC = {("large-mixed", "srp_sparse4_kernel (two-byte codes)"): (20874986240 + 163516160) + (6676972544 + 165890816)}


def load_tensor_peak():
    """Dense BF16 tensor peak: the sustained figure (a kernel inside a long
    step), else the burst figure, else the fallback."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(p))
        if "bf16_tflops_sustained" in d:
            return d["bf16_tflops_sustained"], "measured (sustained)"
        return d["bf16_tflops"], "measured"
    except (OSError, KeyError, ValueError):
        return 1900.0, "fallback"


def bind_numa(torch, dev) -> dict:
    """Restrict this process to the host CPUs of the GPU's own NUMA node, so
    that pinned host buffers allocated afterwards (first touch) sit in the
    memory next to the GPU's host link rather than behind the inter-socket
    link.  Reads the node from sysfs by the GPU's PCI address; leaves the
    affinity alone where sysfs gives no node.  Returns what it found."""
    info = {"node": None, "cpus": None, "bound": False}
    try:
        p = torch.cuda.get_device_properties(dev)
        addr = "%04x:%02x:%02x.0" % (p.pci_domain_id, p.pci_bus_id, p.pci_device_id)
        base = "/sys/bus/pci/devices/" + addr
        info["pci"] = addr
        with open(base + "/numa_node") as f:
            node = int(f.read().strip())
        info["node"] = node
        if node < 0:
            return info
        with open("/sys/devices/system/node/node%d/cpulist" % node) as f:
            text = f.read().strip()
        cpus = set()
        for part in text.split(","):
            if "-" in part:
                a, b = part.split("-")
                cpus.update(range(int(a), int(b) + 1))
            elif part:
                cpus.add(int(part))
        allowed = os.sched_getaffinity(0)
        use = cpus & allowed
        info["cpus"] = len(use)
        info["allowed"] = len(allowed)
        if use and use != allowed:
            os.sched_setaffinity(0, use)
            info["bound"] = True
    except (OSError, ValueError, AttributeError) as e:
        info["error"] = type(e).__name__
    return info


def measure_plain(B, torch, pipe, flush, stream, stage_ms, step_ms, reps: int = 2):
    """The plain GPU form of the same step: eager launches (no CUDA graph),
    every hash of every object computed up front (no lazy hashing), the
    plain verification launch (one thread per pair, no persistence or work
    stealing, no autotuning), Algorithms 1 and 2 as separate passes and, for
    dense rows, the FP32 CUDA-core projection instead of the BF16 tensor
    cores.  Same outputs (both forms
    are bit-exact to the oracle); returns the times and the speedups."""
    plain = B.blsh_plan(B.PLAN_PLAIN, 1, 256, 0, 0)
    times = {"hash": [], "verify": [], "step": []}
    for i in range(reps):
        flush.fill_(float(i))
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
        ev[0].record(stream)
        if pipe.dense:
            B.blsh_srp_dense(pipe.ctx, pipe.X, pipe.R, pipe.sig, margin=pipe.w["margin"], workspace=None)
        elif pipe.lazy_bits:   # every hash of every object
            B.blsh_srp_sparse(pipe.ctx, pipe.indptr, pipe.indices, pipe.values, pipe.R, pipe.sig)
        else:
            pipe.hash()
        ev[1].record(stream)
        pipe.band()
        ev[2].record(stream)
        B.blsh_verify(pipe.ctx, pipe.tab, pipe.pairs, pipe.sig, pipe.status, pipe.n_used, pipe.m, pipe.est,
                      pipe.hist, P_dev=pipe.n_pairs, plan=plain)
        if pipe.with_lite:   # Algorithm 2 as its own pass, under the same plain plan
            B.blsh_set_plan(pipe.ctx, pipe.tab, plain)
            pipe.lite()
            B.blsh_set_plan(pipe.ctx, pipe.tab, pipe.plan)
        ev[3].record(stream)
        pipe.compact()
        ev[4].record(stream)
        torch.cuda.synchronize()
        times["hash"].append(ev[0].elapsed_time(ev[1]))
        times["verify"].append(ev[2].elapsed_time(ev[3]))
        times["step"].append(ev[0].elapsed_time(ev[4]))
    if B.blsh_status(pipe.ctx) != 0:
        raise RuntimeError("plain-form step failed")
    t = {k: float(np.mean(v)) for k, v in times.items()}
    return {"form": "eager launches, all hashes up front, plain verify launches, Algorithms 1 and 2 as separate passes"
                    + (", FP32 CUDA-core projection" if pipe.dense else ""),
            "step_ms": round(t["step"], 4), "verify_ms": round(t["verify"], 4), "hash_ms": round(t["hash"], 4),
            "speedup_step": round(t["step"] / step_ms, 3),
            "speedup_verify": round(t["verify"] / (stage_ms["verify"] + stage_ms.get("resume", 0.0)), 3),
            "speedup_hash": round(t["hash"] / (stage_ms["hash"] + stage_ms.get("hash_rest", 0.0)), 3)}


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(p))
        return d["hbm_gbs"], "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def csr_rows_bytes(indptr, indices, rows, ncols, esize):
    """Sparse SRP over the objects `rows` (bool mask or None = all) and ncols
    hash columns: per object two indptr entries and ncols/8 signature bytes
    written, per nonzero its index and value, and each distinct row of R
    that those nonzeros touch once (ncols * esize bytes)."""
    if rows is None:
        nnz, n, idx = int(indptr[-1]), len(indptr) - 1, indices
    else:
        sel = np.flatnonzero(rows)
        lo, hi = indptr[sel], indptr[sel + 1]
        nnz, n = int((hi - lo).sum()), sel.size
        idx = indices[np.concatenate([np.arange(a, b) for a, b in zip(lo, hi)])] if n else indices[:0]
    return nnz * 8 + n * (16 + ncols // 8) + int(np.unique(idx).size) * ncols * esize


def verification_totals(work, timed):
    """The verification stage's algorithmic bytes and device time per step:
    every verification kernel that ran (the two-pass form in one kernel, or
    its first pass and verify_kernel, the lazy form's resume).  With two
    kernels the bytes are split between the passes for the per-kernel
    figures."""
    total = work["verify_kernel"][0]
    first = work.pop("verify_first_kernel", (0, "B"))[0]
    if "verify_first_kernel" in timed:
        work["verify_first_kernel"] = (first, "B")
        work["verify_kernel"] = (total - first, "B")
    if "verify_tile_kernel" in timed:     # both passes in one kernel
        work["verify_tile_kernel"] = (total, "B")
    names = [n for n in ("verify_tile_kernel", "verify_first_kernel", "verify_kernel", "verify_resume_kernel")
             if n in timed]
    vbytes = total + work.get("verify_resume_kernel", (0, "B"))[0]
    v_ms = sum(timed[n][1] for n in names)
    return vbytes, v_ms, " + ".join(names)


def kernel_work(B, pipe, w, objs, st, nu, lst, need):
    """Algorithmic work of one step per kernel name: {name: (amount, unit)}
    with unit "B" (bytes moved at least once) or "flop".  Counts what each
    launch must read and write; re-reads (L2 hits or not) are not counted."""
    P, N, k = pipe.P, pipe.N, w["k"]
    work = {}
    kept = (st == B.ACCEPT) | (st == B.ACCEPT_AT_MAX)
    per_chunk = 8 * k if w["kind"] == 0 else k // 4          # both rows' k hashes
    lazy = pipe.lazy_bits
    if lazy:
        capped = np.minimum(nu.astype(np.int64), lazy) // k
        resumed = nu.astype(np.int64) > lazy
        work["verify_kernel"] = (P * (8 + 5 + 1) + 4 * int((kept & ~resumed).sum())
                                 + int(capped.sum()) * per_chunk, "B")
        r = int(resumed.sum())
        work["verify_resume_kernel"] = (P + r * (8 + 5) + 4 * int((kept & resumed).sum())
                                        + int((nu[resumed].astype(np.int64) // k).sum()) * per_chunk, "B")
    else:
        work["verify_kernel"] = (P * (8 + 5 + (1 if pipe.with_lite else 0)) + 4 * int(kept.sum())
                                 + int((nu.astype(np.int64) // k).sum()) * per_chunk, "B")
    # the part of those bytes a first pass over every pair's first four
    # chunks moves (the two-pass form: verify_first_kernel, then
    # verify_kernel over the open pairs): the pair, its outputs, four chunks
    c4 = np.minimum(nu.astype(np.int64) // k, 4)
    work["verify_first_kernel"] = (P * (8 + 5 + (1 if pipe.with_lite else 0))
                                  + 4 * int((kept & (nu.astype(np.int64) <= 4 * k)).sum())
                                  + int(c4.sum()) * per_chunk, "B")
    if pipe.with_lite:
        surv = (lst == B.LITE_ACCEPT) | (lst == B.LITE_REJECT)
        pr = pipe.pairs[:P].cpu().numpy().astype(np.int64)[surv]
        row_nnz = np.diff(objs.indptr)
        vb = 8 if objs.values is not None else 4
        work["lite_collect_kernel"] = (P + 8 * int(surv.sum()), "B")
        work["lite_queue_kernel"] = (int(surv.sum()) * (8 + 32 + 9)
                                     + int((row_nnz[pr[:, 0]] + row_nnz[pr[:, 1]]).sum()) * vb, "B")
    if pipe.dense:
        work["srp_dense_tc_persistent"] = (3 * 2 * N * w["d"] * w["bits"], "flop")
    elif w["kind"] == 1:
        es = 2 if w.get("r_format") == "q16" else 4
        name = "srp_sparse4_kernel (two-byte codes)" if w.get("r_format") == "q16" else "srp_sparse4_kernel"
        b = csr_rows_bytes(objs.indptr, objs.indices, None, lazy or w["bits"], es)
        rows_nnz = np.diff(objs.indptr)
        gathered = int(rows_nnz.sum()) * (lazy or w["bits"]) * es
        if lazy:
            b += csr_rows_bytes(objs.indptr, objs.indices, need, w["bits"] - lazy, es)
            gathered += int(rows_nnz[need].sum()) * (w["bits"] - lazy) * es
        work[name] = (b, "B")
        # every nonzero reads its row of R (L2 hits for the rows other objects
        # brought in): the traffic between L2 and the SMs
        work[name + " gathered"] = (gathered, "B")
        work["srp_sparse_kernel"] = work[name]    # the generic form (other column counts)
    else:
        nnz = int(objs.indptr[-1])
        work["minhash_kernel"] = (nnz * 4 + N * (8 + 4 * w["n_hashes"]), "B")
    # banding: n = N * bands (object, band) entries
    n, rows, bands = N * w["bands"], w["rows"], w["bands"]
    if w["kind"] == 1:
        kb = 4 if max(1, (bands - 1).bit_length()) + rows <= 32 else 8
        obj_rows = N * bands * ((rows + 7) // 8)
    else:   # 32-bit class keys while a row of class ids fits the staging (32 words), else 64-bit band hashes
        kb = 4 if ((bands + 3) & ~3) <= 32 else 8
        obj_rows = N * bands * 4
    emit = "emit_warp_kernel"
    passes = (8 * kb + 7) // 8 if w["kind"] == 0 else (max(1, (bands - 1).bit_length()) + rows + 7) // 8
    sig_bytes = N * bands * rows // 8 if w["kind"] == 1 else N * bands * rows * 4   # the banded hashes
    work["band_keys_kernel"] = (sig_bytes + n * (kb + 4) + obj_rows, "B")
    work["digit_hist_kernel"] = (passes * n * kb, "B")
    work["digit_scatter_kernel"] = (passes * 2 * n * (kb + 4), "B")
    work[emit + " (count pass)"] = (n * (kb + 4) + obj_rows + n * 8, "B")
    work[emit + " (write pass)"] = (n * (kb + 4 + 8) + obj_rows + P * 8, "B")
    for ps in (" (count pass)", " (write pass)"):    # the unstaged form
        work["emit_kernel" + ps] = work[emit + ps]
    if getattr(pipe, "allpairs", False):
        # prefix filtering instead of banding: per nonzero its index and value
        # read by the statistics, the prefix pass (flag written) and the index
        # keys (8 B written); two stable radix sorts of (8 B key + 4 B value)
        # items, read and written once per 8-bit pass; the candidate keys
        # (8 B per key with duplicates) written once, then the distinct pairs
        nnz, dim, dups = pipe.nnz, pipe.dim, pipe.max_dups
        xb = max(1, int(N).bit_length())
        p_idx = (xb + max(1, int(dim).bit_length()) + 1 + 7) // 8
        p_key = (32 + xb + 1 + 7) // 8
        for name in list(work):
            if name.startswith(("band_keys", "digit_", "emit_", "class_id")):
                del work[name]
        work["ap_stats_kernel"] = (nnz * 8 + dim * 8, "B")
        work["ap_prefix_warp_kernel"] = (nnz * 9, "B")
        work["ap_prefix_cta_kernel"] = (nnz * 9, "B")
        work["ap_index_keys_kernel"] = (nnz * (5 + 8) + N * 16, "B")
        work["digit_hist_kernel"] = (p_idx * nnz * 8 + p_key * dups * 8, "B")
        work["digit_scatter_kernel"] = (p_idx * 2 * nnz * 12 + p_key * 2 * dups * 12, "B")
        work["ap_emit_kernel (count pass)"] = (nnz * 4 + N * 24, "B")
        work["ap_emit_kernel (write pass)"] = (nnz * 4 + N * 24 + dups * 16, "B")
        work["ap_mark_kernel"] = (dups * 12, "B")
        work["ap_write_kernel"] = (dups * 16 + P * 8, "B")
    n_keep = int(kept.sum())
    work["compact_count"] = ((2 if pipe.with_lite else 1) * P, "B")
    work["compact_write"] = ((2 if pipe.with_lite else 1) * P + 8 * n_keep, "B")
    return work


def combine_ranks(dist, step_ms: float, pairs: int, e2e_ms: float, device):
    """Whole-job numbers of a replicated run: the slowest rank's step and
    end-to-end times (max over ranks) and the pairs of all ranks (sum).
    Each rank verifies its own batch, so the units add up (weak scaling)."""
    if dist is None:
        return step_ms, pairs, e2e_ms
    import torch
    t = torch.tensor([step_ms, e2e_ms], dtype=torch.float64, device=device)
    p = torch.tensor([float(pairs)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(p, op=dist.ReduceOp.SUM)
    return float(t[0].item()), int(p[0].item()), float(t[1].item())


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

def run_ours(args, w):
    import torch

    import paper_1110_1328_gb300 as B

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    B.lib()

    objs, hashp = make_inputs(w, rank)
    pipe = Pipeline(B, torch, w, objs, hashp, device)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=device)

    for _ in range(args.warmup):
        pipe.step()
    rc = B.blsh_status(pipe.ctx)
    if rc != 0:
        raise RuntimeError(f"warm-up step failed with {rc}")
    launches0 = B.blsh_launch_count(pipe.ctx)
    pipe.step()
    launches_per_step = B.blsh_launch_count(pipe.ctx) - launches0
    torch.cuda.synchronize()

    # capture one step in a CUDA graph (all stages, no host sync inside)
    graph = None
    if not args.no_graph:
        try:
            g = torch.cuda.CUDAGraph()
            s = torch.cuda.Stream()
            s.wait_stream(stream)
            with torch.cuda.stream(s):
                pipe.step()          # warm on the capture stream
            stream.wait_stream(s)
            torch.cuda.synchronize()
            with torch.cuda.graph(g):
                pipe.step()
            torch.cuda.synchronize()
            g.replay()
            torch.cuda.synchronize()
            graph = g
        except Exception as e:   # capture is an optimisation; eager launches do the same work
            print(f"graph capture failed, timing eager launches: {e}", file=sys.stderr)
            graph = None
    B.blsh_status(pipe.ctx)

    def one_step():
        if graph is not None:
            graph.replay()
        else:
            pipe.step()

    # ---- device-timed steps ----
    clocks = ClockSampler(local)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    wall0 = time.perf_counter()
    for i in range(args.steps):
        flush.fill_(float(i))            # L2 flush between timed steps (256 MB write)
        starts[i].record(stream)
        one_step()
        ends[i].record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    if dist:
        dist.barrier()
    clk = clocks.stop()
    rc, ctr = B.blsh_status(pipe.ctx, counters=True)
    if rc != 0:
        raise RuntimeError(f"timed steps reported {rc}")
    # signs the FP32 bound left to the FP64 recheck, and exactly-zero dots
    rechecks = {"rechecked_per_step": ctr[2] / args.steps, "zero_dots_per_step": ctr[3] / args.steps}
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    my_ms = float(np.mean(step_ms))

    # ---- per-stage and per-kernel device times (eager steps: events around
    # each library call, and the library's own events around each launch) ----
    stage_ms = {s: [] for s in pipe.STAGES}
    reps = max(3, min(args.steps, 5))
    B.blsh_timing_begin(pipe.ctx)
    for i in range(reps):
        flush.fill_(float(i))
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(len(pipe.STAGES) + 1)]
        evs[0].record(stream)
        for j, s in enumerate(pipe.STAGES):
            getattr(pipe, s)()
            evs[j + 1].record(stream)
        torch.cuda.synchronize()
        for j, s in enumerate(pipe.STAGES):
            stage_ms[s].append(evs[j].elapsed_time(evs[j + 1]))
    records = B.blsh_timing_end(pipe.ctx)
    stage_ms = {s: float(np.mean(v)) for s, v in stage_ms.items()}
    kernel_ms = {}   # name -> [launches per step, device ms per step]
    for name, t_ms in records:
        k = kernel_ms.setdefault(name, [0, 0.0])
        k[0] += 1
        k[1] += t_ms
    kernel_ms = {n: [c / reps, t / reps] for n, (c, t) in kernel_ms.items()}

    vs_plain = measure_plain(B, torch, pipe, flush, stream, stage_ms, my_ms)

    # ---- end to end through the public API, host buffers ----
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    h_indptr = pin(objs.indptr)
    h_indices = pin(objs.indices.view(np.int32))
    h_values = None if objs.values is None else pin(objs.values)
    h_counts = torch.zeros(2, dtype=torch.int64).pin_memory()
    h_out1 = torch.zeros(pipe.P + 1024, dtype=torch.int64).pin_memory()
    h_out2 = torch.zeros(pipe.P + 1024, dtype=torch.int64).pin_memory()
    e2e_ms, h2d, d2h = [], 0, 0
    for i in range(args.steps):
        flush.fill_(float(i))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        if pipe.dense:
            # the step's input is X; Lite's row structure is fixed by the shape
            pipe.values.copy_(h_values, non_blocking=True)
            nb_in = h_values.numel() * 4
        else:
            pipe.indptr.copy_(h_indptr, non_blocking=True)
            pipe.indices[: h_indices.numel()].copy_(h_indices, non_blocking=True)
            nb_in = h_indptr.numel() * 8 + h_indices.numel() * 4
            if h_values is not None:
                pipe.values.copy_(h_values, non_blocking=True)
                nb_in += h_values.numel() * 4
        one_step()
        h_counts.copy_(pipe.n_out, non_blocking=True)
        torch.cuda.current_stream().synchronize()
        n1, n2 = int(h_counts[0]), int(h_counts[1])
        h_out1[:n1].copy_(pipe.out1[:n1], non_blocking=True)
        h_out2[:n2].copy_(pipe.out2[:n2], non_blocking=True)
        torch.cuda.current_stream().synchronize()
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
        h2d, d2h = nb_in, 16 + 8 * (n1 + n2)
    e2e_step = float(np.mean(e2e_ms))
    ms, P_total, e2e_max = combine_ranks(dist, my_ms, pipe.P, e2e_step, device)
    value = P_total / (ms / 1e3)
    e2e_val = P_total / (e2e_max / 1e3)

    # ---- outputs of the last step, for the record ----
    st = pipe.status[: pipe.P].cpu().numpy()
    nu = pipe.n_used[: pipe.P].cpu().numpy().view(np.uint16)
    hist = pipe.hist.cpu().numpy()
    n1, n2 = [int(x) for x in pipe.n_out.cpu()]

    peak, peak_kind = load_peaks()
    lst = pipe.lstatus[: pipe.P].cpu().numpy() if pipe.with_lite else None
    need = pipe.need.cpu().numpy().astype(bool) if pipe.lazy_bits else None
    kept = int(((st == B.ACCEPT) | (st == B.ACCEPT_AT_MAX)).sum())
    survivors = int(((lst == B.LITE_ACCEPT) | (lst == B.LITE_REJECT)).sum()) if pipe.with_lite else 0
    # hashes computed per step (with lazy hashing: the prefix for every
    # object, the rest for the objects of the pairs it left open)
    hash_ms = stage_ms["hash"] + stage_ms.get("hash_rest", 0.0)
    if w["kind"] == 1:
        lazy = pipe.lazy_bits
        hashes = pipe.N * (lazy or w["bits"]) + (int(need.sum()) * (w["bits"] - lazy) if lazy else 0)
    else:
        hashes = int(objs.indptr[-1]) * w["n_hashes"]
    hashes_per_s = hashes / (hash_ms / 1e3)
    work = kernel_work(B, pipe, w, objs, st, nu, lst, need)
    vbytes, v_ms, v_names = verification_totals(work, kernel_ms)
    # the dominant kernel: the most device time per step of the launches the
    # library timed (the exclusive scan helper is three small launches)
    timed = {n: v for n, v in kernel_ms.items() if not n.startswith("exclusive scan")}
    dom = max(timed, key=lambda n: timed[n][1])
    dom_launches, dom_ms = timed[dom]
    amount, unit = work.get(dom, (None, None))
    if unit == "flop":
        tf_peak, tf_kind = load_tensor_peak()
        ach = amount / (dom_ms / 1e3) / 1e12
        roofline = {"bound": "tensor", "kernel": dom, "achieved": round(ach, 1), "peak": tf_peak,
                    "unit": "TFLOP/s", "frac": round(ach / tf_peak, 4), "traffic": None, "peak_source": tf_kind,
                    "algorithmic_flops": int(amount)}
    else:
        ach = amount / (dom_ms / 1e3) / 1e9 if amount is not None else None
        roofline = {"bound": "hbm", "kernel": dom, "achieved": None if ach is None else round(ach, 1),
                    "peak": peak, "unit": "GB/s", "frac": None if ach is None else round(ach / peak, 4),
                    "traffic": NCU_TRAFFIC.get((args.workload, dom)), "peak_source": peak_kind,
                    "algorithmic_bytes": amount}
    if dom + " gathered" in work:
        gb = work[dom + " gathered"][0]
        roofline["gathered_bytes"] = int(gb)
        roofline["gathered_GBps"] = round(gb / (dom_ms / 1e3) / 1e9, 1)
    roofline.update({"launches_per_step": dom_launches, "ms_per_step": round(dom_ms, 4),
                     "timing": "library CUDA events around each launch on its stream, eager steps"})
    kernels = {n: {"launches": c, "ms": round(t, 4),
                   **({"GBps": round(work[n][0] / (t / 1e3) / 1e9, 1)} if n in work and work[n][1] == "B" else {}),
                   **({"TFLOPs": round(work[n][0] / (t / 1e3) / 1e12, 1)} if n in work and work[n][1] == "flop"
                      else {})}
               for n, (c, t) in sorted(kernel_ms.items(), key=lambda kv: -kv[1][1])}
    v_ach = vbytes / (v_ms / 1e3) / 1e9

    out = {
        "metric": METRIC,
        "value": round(value, 1),
        "unit": "pairs/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(ms, 4),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "u32",
        "data": "synthetic",
        "config": {"workload": args.workload + ": " + w["text"], "objects": pipe.N, "candidate_pairs": pipe.P,
                   "l2": "flushed between timed steps (256 MB write)", "cuda_graph": graph is not None,
                   "plan": dict(pipe.plan.as_dict(), k=w["k"],
                                **({"ms_per_call_by_k": pipe.k_ms} if pipe.k_ms else {})),
                   "tables_build_ms": round(pipe.tables_ms, 2),
                   "lazy_bits": pipe.lazy_bits,
                   "parallelism": f"replicas x{world}" if world > 1 else "1 GPU"},
        "e2e": {"value": round(e2e_val, 1), "unit": "pairs/s", "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h), "ms_per_step": round(e2e_step, 4)},
        "gpu_launches": int(launches_per_step * args.steps),
        "roofline": roofline,
        "verify_hbm": {"achieved": round(v_ach, 1), "peak": peak, "unit": "GB/s", "frac": round(v_ach / peak, 4),
                       "algorithmic_bytes": int(vbytes), "ms": round(v_ms, 4),
                       "kernels": v_names,
                       "counts": "per pair: its indices, its outputs and the chunks it compares; a row shared by several "
                                 "pairs is counted for each, so where pairs share rows (L2 re-reads) the figure can "
                                 "exceed the copy bandwidth"},
        "kernels": kernels,
        "hashes_per_s": round(hashes_per_s, 1),
        "hashes_per_step": int(hashes),
        "stage_ms": {k: round(v, 4) for k, v in stage_ms.items()},
        "outputs": {"bayeslsh_kept": n1, "lite_kept": n2, "pruned": int((st == B.PRUNED).sum()),
                    "stop_hist_first4": [int(x) for x in hist[:4]]},
        "clocks": clk,
        "wall_s_timed_loop": round(wall, 3),
        "vs_plain": vs_plain,
        "srp_signs": rechecks,
    }
    if args.profile_step:
        # one more eager step inside an NVTX range, for ncu --nvtx-include "blsh_step/"
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("blsh_step")
        pipe.step()
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
    if rank == 0 and not args.no_cpu_baseline and world == 1:
        out["cpu_baseline"] = cpu_baseline(w, objs, hashp, pipe.P)
    elif rank == 0 and world > 1:
        out["cpu_baseline"] = None
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def run_sweep(args, w):
    """The paper's parameter study (Section 5, "Effect of varying parameters"):
    gamma, delta and epsilon varied one at a time over 0.01 .. 0.09 with the
    other two at 0.05, Algorithm 1 on the cosine-small candidates at t = 0.7;
    per setting the verification time and the quality measure the study
    reports (fraction of output estimates off by more than 0.05, mean error,
    recall).  The exact similarity of every candidate comes from Algorithm 2's
    exact pass with a threshold that prunes nothing; the fixed-n estimator
    over all 2,048 hashes ("LSH Approx") is measured beside it."""
    import torch

    import paper_1110_1328_gb300 as B
    dev = torch.device("cuda", 0)
    base = WORKLOADS["cosine-small"]
    objs, R = make_inputs(base)
    pipe = Pipeline(B, torch, base, objs, R, dev)
    # every setting reads up to all 2,048 hashes: compute them all (the
    # pipeline's own hash stage computes only the lazy prefix)
    B.blsh_srp_sparse(pipe.ctx, pipe.indptr, pipe.indices, pipe.values, pipe.R, pipe.sig)
    pipe.band()
    assert B.blsh_status(pipe.ctx) == 0
    P = pipe.P
    pairs, sig = pipe.pairs[:P], pipe.sig

    def timed(fn, reps=3):
        ts = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return float(np.median(ts))

    # exact similarity of every candidate: Lite with t = 0.01 prunes nothing
    tab0 = B.blsh_tables_build(pipe.ctx, B.make_params(kind=1, t=0.01, k=32, n_max=2048, h=32))
    lst = torch.zeros(P, dtype=torch.uint8, device=dev)
    sim = torch.zeros(P, dtype=torch.float64, device=dev)
    exact_ms = timed(lambda: B.blsh_verify_lite(pipe.ctx, tab0, pairs, sig, pipe.indptr, pipe.indices, pipe.values,
                                                lst, sim))
    assert B.blsh_status(pipe.ctx) == 0
    s_exact = sim.cpu().numpy()
    assert not np.isnan(s_exact).any()
    t = 0.7
    truth = s_exact >= t
    n_true = int(truth.sum())
    st = torch.zeros(P, dtype=torch.uint8, device=dev)
    est = torch.zeros(P, dtype=torch.float32, device=dev)
    nu = torch.zeros(P, dtype=torch.int16, device=dev)
    rows = []
    for name in ("gamma", "delta", "eps"):
        for v in (0.01, 0.03, 0.05, 0.07, 0.09):
            kw = dict(gamma=0.05, delta=0.05, eps=0.05)
            kw[name] = v
            tab = B.blsh_tables_build(pipe.ctx, B.make_params(kind=1, t=t, k=32, n_max=2048, h=128, **kw))
            ms = timed(lambda: B.blsh_verify(pipe.ctx, tab, pairs, sig, st, nu, None, est))
            assert B.blsh_status(pipe.ctx) == 0
            out = np.isin(st.cpu().numpy(), (B.ACCEPT, B.ACCEPT_AT_MAX))
            err = np.abs(est.cpu().numpy()[out].astype(np.float64) - s_exact[out])
            rows.append({"vary": name, "value": v, "verify_ms": round(ms, 4), "output_pairs": int(out.sum()),
                         "frac_err_gt_0.05": round(float((err > 0.05).mean()), 5) if out.any() else None,
                         "mean_err": round(float(err.mean()), 5) if out.any() else None,
                         "recall": round(float((out & truth).sum() / max(n_true, 1)), 5),
                         "mean_hashes": round(float(nu.cpu().numpy().view(np.uint16).mean()), 1)})
    # the fixed-n estimator over all 2,048 hashes
    m = torch.zeros(P, dtype=torch.int16, device=dev)
    keep = torch.zeros(P, dtype=torch.uint8, device=dev)
    ms = timed(lambda: B.blsh_estimate_mle(pipe.ctx, 1, 2048, t, pairs, sig, m, est, keep))
    assert B.blsh_status(pipe.ctx) == 0
    out = keep.cpu().numpy() == 1
    err = np.abs(est.cpu().numpy()[out].astype(np.float64) - s_exact[out])
    approx = {"verify_ms": round(ms, 4), "output_pairs": int(out.sum()),
              "frac_err_gt_0.05": round(float((err > 0.05).mean()), 5), "mean_err": round(float(err.mean()), 5),
              "recall": round(float((out & truth).sum() / max(n_true, 1)), 5)}
    print(json.dumps({"metric": "parameter study (gamma, delta, epsilon) on cosine-small candidates, t = 0.7",
                      "candidate_pairs": P, "true_pairs": n_true, "exact_all_ms": round(exact_ms, 4),
                      "lsh_approx_2048": approx, "bayeslsh": rows,
                      "config": {"workload": "sweep: " + w["text"]}}), flush=True)


def run_verify_large(args, w):
    """Algorithm 1 alone over uniform random pairs of random signatures: every
    signature gather misses L2, so this measures verification at HBM scale."""
    import torch

    import paper_1110_1328_gb300 as B
    dev = torch.device("cuda", 0)
    ctx = B.Context(0)
    g = torch.Generator(device=dev)
    g.manual_seed(w["seed"])
    N, W, P = w["n"], w["bits"] // 32, w["pairs"]
    B.blsh_ctx_reserve(ctx, N)
    sig = torch.randint(-2 ** 31, 2 ** 31 - 1, (N, W), dtype=torch.int32, device=dev, generator=g)
    x = torch.randint(0, N, (P,), dtype=torch.int64, device=dev, generator=g)
    y = torch.randint(0, N, (P,), dtype=torch.int64, device=dev, generator=g)
    pairs = torch.stack([torch.minimum(x, y), torch.maximum(x, y)], 1).to(torch.int32)
    del x, y
    tab = B.blsh_tables_build(ctx, B.make_params(kind=1, t=w["t"], n_max=w["n_max"], k=w["k"], h=w["h"]))
    st = torch.zeros(P, dtype=torch.uint8, device=dev)
    nu = torch.zeros(P, dtype=torch.int16, device=dev)
    m = torch.zeros(P, dtype=torch.int16, device=dev)
    est = torch.zeros(P, dtype=torch.float32, device=dev)
    hist = torch.zeros(tab.levels, dtype=torch.int64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    plan = B.blsh_autotune(ctx, tab, pairs[:20_000_000], sig, st[:20_000_000])
    for _ in range(args.warmup):
        B.blsh_verify(ctx, tab, pairs, sig, st, nu, m, est, hist)
    torch.cuda.synchronize()
    ts = []
    clocks = ClockSampler(0)
    clocks.start()
    time.sleep(0.3)
    for i in range(args.steps):
        flush.fill_(float(i))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        B.blsh_verify(ctx, tab, pairs, sig, st, nu, m, est, hist)
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    clk = clocks.stop()
    assert B.blsh_status(ctx) == 0
    ms = float(np.mean(ts))
    # the call's launches one by one (the plane copy, then the kernel)
    B.blsh_timing_begin(ctx)
    for i in range(3):
        flush.fill_(float(i))
        B.blsh_verify(ctx, tab, pairs, sig, st, nu, m, est, hist)
    kern = {}
    for name, t_ms in B.blsh_timing_end(ctx):
        kern.setdefault(name, []).append(t_ms)
    kern = {n: round(float(np.mean(v)), 4) for n, v in kern.items()}
    if args.profile_step:
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("blsh_step")
        B.blsh_verify(ctx, tab, pairs, sig, st, nu, m, est, hist)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
    h = hist.cpu().numpy()
    chunks = float((h * np.arange(1, len(h) + 1)).sum())
    peak, peak_kind = load_peaks()
    stn = st.cpu().numpy()
    kept = int(((stn == B.ACCEPT) | (stn == B.ACCEPT_AT_MAX)).sum())
    alg = P * (8 + 5) + 4 * kept + chunks * (w["k"] // 4)
    sector = P * (8 + 9) + P * 2 * 32
    v_names = [n for n in ("verify_tile_kernel", "verify_first_kernel", "verify_kernel") if n in kern]
    vk = sum(kern[n] for n in v_names) or ms
    print(json.dumps({"metric": METRIC, "value": round(P / (ms / 1e3), 1), "unit": "pairs/s", "n_gpus": 1,
                      "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 4),
                      "higher_is_better": True, "dtype": "u32", "data": "synthetic",
                      "config": {"workload": args.workload + ": " + w["text"], "plan": plan.as_dict(),
                                 "l2": "flushed between timed steps (256 MB write)"},
                      "verify_hbm": {"algorithmic_bytes": int(alg), "achieved": round(alg / (vk / 1e3) / 1e9, 1),
                                     "frac": round(alg / (vk / 1e3) / 1e9 / peak, 4), "kernel": " + ".join(v_names),
                                     "kernel_ms": vk, "sector_floor_bytes": int(sector),
                                     "sector_floor_GBps": round(sector / (vk / 1e3) / 1e9, 1),
                                     "peak": peak, "peak_source": peak_kind, "unit": "GB/s"},
                      "kernels_ms": kern, "clocks": clk,
                      "stop_hist_first4": [int(v) for v in h[:4]], "mean_chunks": round(chunks / P, 4)}),
          flush=True)


class LargePipeline:
    """The 5e6-vector mixed workload: inputs drawn on the GPU, R generated on
    the device as two-byte codes (68.7 GB).  One step: the first lazy_bits
    hashes of every object, banding, then for every batch of candidates
    (sized by free HBM, or capped) Algorithms 1 and 2 over those hashes, the
    remaining hashes of the objects of the pairs still open, Algorithm 1
    finished for those pairs, and the compaction of both output sets into
    the batch's segment of the global output arrays (indices relative to the
    batch's first pair)."""

    def __init__(self, B, torch, w, device, batch_cap=None):
        import synth
        self.B, self.torch, self.w, self.dev = B, torch, w, device
        t = torch
        self.ctx = B.Context(device.index or 0)
        self.indptr, self.indices, self.values = synth.large_tfidf_device(
            n_docs=w["n"], dim=w["dim"], seed=w["seed"], n_groups=w.get("n_groups", 100_000), device=device)
        torch.cuda.synchronize()
        self.N, self.W, self.bits = w["n"], w["bits"] // 32, w["bits"]
        self.nnz = int(self.indptr[-1].item())
        B.blsh_ctx_reserve(self.ctx, self.N)           # the hot calls below allocate nothing
        self.Rq = B.blsh_gaussian_codes(self.ctx, w["r_seed"], w["dim"], w["bits"])
        self.sig = t.zeros((self.N, self.W), dtype=t.int32, device=device)
        self.need = t.zeros(self.N, dtype=t.uint8, device=device)
        self.tab = B.blsh_tables_build(self.ctx, B.make_params(kind=1, t=w["t"], k=w["k"], n_max=w["n_max"],
                                                               h=w["h"]))
        self.ws = t.zeros(B.blsh_lsh_candidates_workspace(self.N, 1, w["rows"], w["bands"]), dtype=t.uint8,
                          device=device)
        self.n_pairs = t.zeros(1, dtype=t.int64, device=device)
        self.hash()
        B.blsh_lsh_candidates(self.ctx, self.sig, 1, w["rows"], w["bands"], None, self.n_pairs, self.ws)
        if B.blsh_status(self.ctx) not in (B.OK, B.ETRUNC):     # a count-only pass (capacity 0) truncates
            raise RuntimeError("candidate count pass failed")
        self.P = int(self.n_pairs.item())
        if self.P > 4_000_000_000:
            raise RuntimeError(f"{self.P} candidates: more than this workload's pair buffer is sized for")
        self.pairs = t.zeros((self.P + 1024, 2), dtype=t.int32, device=device)
        # the output sets: each batch writes its kept indices into its own
        # segment [b0, b0 + n) of these
        self.out1 = t.zeros(max(self.P, 1), dtype=t.int64, device=device)
        self.out2 = t.zeros(max(self.P, 1), dtype=t.int64, device=device)
        self.set_batch(batch_cap)
        self.keep1 = (1 << B.ACCEPT) | (1 << B.ACCEPT_AT_MAX)
        self.keep2 = 1 << B.LITE_ACCEPT
        self.band()
        if B.blsh_status(self.ctx) != 0:
            raise RuntimeError("banding failed")
        # the verification plan, tuned on a prefix of the real candidates
        n_t = min(self.P, 20_000_000, self.batch)
        self.plan = B.blsh_autotune(self.ctx, self.tab, self.pairs[:n_t], self.sig, self.status[:n_t],
                                    self.n_used[:n_t], self.m[:n_t], self.est[:n_t])
        if B.blsh_status(self.ctx) != 0:
            raise RuntimeError("autotune failed")

    def set_batch(self, batch_cap=None):
        """Sizes the per-batch buffers: as many pairs per batch as free HBM
        allows (4 GB kept free), at most batch_cap."""
        from paper_1110_1328_gb300.batches import batch_ranges
        t, device = self.torch, self.dev
        for name in ("status", "n_used", "m", "est", "lstatus", "sim"):
            setattr(self, name, None)
        t.cuda.empty_cache()
        # per pair of a batch: status, n_used, m, est, Lite status, sim (18 B)
        free, _ = t.cuda.mem_get_info(device)
        per_pair = 1 + 2 + 2 + 4 + 1 + 8
        batch = int(max(1 << 20, (free - (4 << 30)) // per_pair))
        if batch_cap:
            batch = min(batch, int(batch_cap))
        self.batch = max(1, min(batch, self.P))
        self.ranges = batch_ranges(self.P, self.batch)
        bsz = self.batch
        self.status = t.zeros(bsz, dtype=t.uint8, device=device)
        self.n_used = t.zeros(bsz, dtype=t.int16, device=device)
        self.m = t.zeros(bsz, dtype=t.int16, device=device)
        self.est = t.zeros(bsz, dtype=t.float32, device=device)
        self.lstatus = t.zeros(bsz, dtype=t.uint8, device=device)
        self.sim = t.zeros(bsz, dtype=t.float64, device=device)
        self.hist = t.zeros((len(self.ranges), self.tab.levels), dtype=t.int64, device=device)
        self.n_out = t.zeros((len(self.ranges), 2), dtype=t.int64, device=device)

    @property
    def lazy_bits(self):
        """Hashes computed for every object before verification (Section 3:
        the rest only for the objects of the pairs still undecided); 0 = all."""
        L = self.w.get("lazy_bits", 0)
        if 0 < L < max(self.w["rows"] * self.w["bands"], self.w["h"]):
            raise ValueError(f"lazy_bits={L} leaves hashes that banding or Lite read")
        return L if 0 < L < self.bits else 0

    def hash(self):
        L = self.lazy_bits
        if L:
            self.B.blsh_srp_sparse_q16_cols(self.ctx, self.indptr, self.indices, self.values, self.Rq, self.sig, 0, L)
        else:
            self.B.blsh_srp_sparse_q16(self.ctx, self.indptr, self.indices, self.values, self.Rq, self.sig)

    def band(self):
        w = self.w
        self.B.blsh_lsh_candidates(self.ctx, self.sig, 1, w["rows"], w["bands"], self.pairs, self.n_pairs, self.ws)

    def verify_batch(self, b, b0, n, P_dev=None):
        """Algorithms 1 and 2 and the two compactions for pairs [b0, b0 + n)."""
        B, ctx, tab = self.B, self.ctx, self.tab
        pairs = self.pairs[b0:b0 + n]
        st, nu, m, est = self.status[:n], self.n_used[:n], self.m[:n], self.est[:n]
        lst, sim, hist = self.lstatus[:n], self.sim[:n], self.hist[b]
        L = self.lazy_bits
        if L:
            self.need.zero_()
            B.blsh_verify_both_capped(ctx, tab, L, pairs, self.sig, st, nu, m, est, hist, self.indptr, self.indices,
                                      self.values, lst, sim, self.need, P_dev=P_dev)
            B.blsh_srp_sparse_q16_cols(ctx, self.indptr, self.indices, self.values, self.Rq, self.sig, L,
                                       self.bits - L, row_mask=self.need)
            B.blsh_verify_resume(ctx, tab, pairs, self.sig, st, nu, m, est, hist, P_dev=P_dev)
        else:
            B.blsh_verify_both(ctx, tab, pairs, self.sig, st, nu, m, est, hist, self.indptr, self.indices,
                               self.values, lst, sim, P_dev=P_dev)
        B.blsh_compact(ctx, st, self.keep1, self.out1[b0:b0 + n], self.n_out[b, 0:1], P_dev=P_dev)
        B.blsh_compact(ctx, lst, self.keep2, self.out2[b0:b0 + n], self.n_out[b, 1:2], P_dev=P_dev)

    def verify(self):
        # one batch: the candidate count is read on the device (no host sync
        # between banding and verification); several: fixed host ranges
        single = len(self.ranges) == 1
        for b, (b0, n) in enumerate(self.ranges):
            self.verify_batch(b, b0, n, P_dev=self.n_pairs if single else None)

    def verify_streamed(self, checkpoint=None, on_batch=None):
        """The verification stage batch by batch, eagerly, with the host-side
        record of progress saved after every batch (an interrupted job
        resumes at its first unfinished batch).  on_batch(b, b0, n), if
        given, runs after batch b's calls (its outputs are then on the
        device)."""
        from paper_1110_1328_gb300.batches import stream_batches
        w = self.w
        job = {"workload": "large-mixed", "n": self.N, "seed": w["seed"], "r_seed": w["r_seed"], "P": self.P,
               "batch": self.batch, "lazy_bits": self.lazy_bits}

        def run(b, b0, n):
            self.verify_batch(b, b0, n)
            if on_batch is not None:
                on_batch(b, b0, n)
            rc = self.B.blsh_status(self.ctx)
            if rc != 0:
                raise RuntimeError(f"batch {b} failed with {rc}")
            return [int(x) for x in self.n_out[b].cpu()], [int(x) for x in self.hist[b].cpu()]

        return stream_batches(self.P, self.batch, run, job, checkpoint, 2, self.tab.levels)

    STAGES = ("hash", "band", "verify")

    def step(self):
        for s_ in self.STAGES:
            getattr(self, s_)()

    # The step's inputs (the CSR rows) and output sets, as a set of buffers
    # that can be swapped: a second set lets the inputs of one step be copied
    # in while another step runs.
    IO = ("indptr", "indices", "values", "out1", "out2", "n_out")

    def buffer_set(self):
        return {k: getattr(self, k) for k in self.IO}

    def new_buffer_set(self):
        return {k: self.torch.empty_like(getattr(self, k)) for k in self.IO}

    def use_buffer_set(self, bs):
        for k, v in bs.items():
            setattr(self, k, v)

    def kept_counts(self):
        return [int(x) for x in self.n_out.sum(0).cpu()]

    def kept_indices(self):
        """The two output sets as global pair indices (host arrays)."""
        counts = self.n_out.cpu().numpy()
        o1, o2 = [], []
        for (b0, n), (c1, c2) in zip(self.ranges, counts):
            o1.append(self.out1[b0:b0 + int(c1)].cpu().numpy() + b0)
            o2.append(self.out2[b0:b0 + int(c2)].cpu().numpy() + b0)
        return np.concatenate(o1) if o1 else np.zeros(0, np.int64), np.concatenate(o2) if o2 else np.zeros(0, np.int64)


def large_e2e(B, torch, pipe, stream, steps, use_graph, kept, depth=3):
    """The large workload end to end through the API with host buffers, as a
    batch pipeline runs it: every step's inputs (the CSR rows, 1.18 GB) are
    copied from pinned host memory and its two output sets (the counts, then
    the kept indices of every device batch) copied back, all inside the timed
    region.  The device buffers form a ring of `depth` sets (one CUDA graph
    per set; two if a third does not fit): the inputs of step i + depth - 1
    are copied while step i runs, so a host copy that runs slow for a while
    (the host link is shared) has depth - 1 steps to finish, and step i's
    outputs are read while step i + 1 runs.  Returns (ms per step, H2D bytes
    per step, D2H bytes per step, the steps' own device time per step, the
    device's wait for a step's inputs per step, the input copy's own rate in
    GB/s when timed alone, and per step the input copy's duration, its end
    relative to its step's start and the wait, with the ring's depth)."""
    pin = lambda x: x.cpu().pin_memory()
    h_in = {k: pin(getattr(pipe, k)) for k in ("indptr", "indices", "values")}
    sets = [pipe.buffer_set(), pipe.new_buffer_set()]
    while len(sets) < depth:
        try:
            sets.append(pipe.new_buffer_set())
        except torch.cuda.OutOfMemoryError:
            torch.cuda.empty_cache()
            break
    D = len(sets)
    graphs = []
    for bs in sets:
        pipe.use_buffer_set(bs)
        for k, v in h_in.items():
            bs[k].copy_(v)
        if use_graph:
            g = torch.cuda.CUDAGraph()
            s = torch.cuda.Stream()
            s.wait_stream(stream)
            with torch.cuda.stream(s):
                pipe.step()
            stream.wait_stream(s)
            torch.cuda.synchronize()
            with torch.cuda.graph(g):
                pipe.step()
            torch.cuda.synchronize()
            graphs.append(g)
    if B.blsh_status(pipe.ctx) != 0:
        raise RuntimeError("end-to-end set-up failed")
    nb = len(pipe.ranges)
    h_counts = [torch.zeros((nb, 2), dtype=torch.int64).pin_memory() for _ in range(D)]
    h_out1 = torch.zeros(kept[0] + 1024, dtype=torch.int64).pin_memory()
    h_out2 = torch.zeros(kept[1] + 1024, dtype=torch.int64).pin_memory()
    h2d = sum(v.numel() * v.element_size() for v in h_in.values())
    copy_in, copy_out = torch.cuda.Stream(), torch.cuda.Stream()
    ev_in = [torch.cuda.Event() for _ in range(D)]
    ev_cnt = [torch.cuda.Event() for _ in range(D)]
    ev_out = [None] * D
    d2h = [0]
    copy_ev = []      # (start, end) of every input copy on the copy-in stream

    def issue_inputs(b):
        # into set b once the step that last used it, and the copy of its
        # outputs, are done
        with torch.cuda.stream(copy_in):
            if ev_out[b] is not None:
                copy_in.wait_event(ev_out[b])
            c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            c0.record(copy_in)
            for k, v in h_in.items():
                sets[b][k].copy_(v, non_blocking=True)
            c1.record(copy_in)
            ev_in[b].record(copy_in)
            copy_ev.append((c0, c1))

    def finish(b):
        # the step that ran on set b: its counts on the host, then its output sets
        ev_cnt[b].synchronize()
        o1 = o2 = 0
        with torch.cuda.stream(copy_out):
            for (b0, _), (c1, c2) in zip(pipe.ranges, h_counts[b].tolist()):
                c1, c2 = min(int(c1), h_out1.numel() - o1), min(int(c2), h_out2.numel() - o2)
                if c1:
                    h_out1[o1:o1 + c1].copy_(sets[b]["out1"][b0:b0 + c1], non_blocking=True)
                if c2:
                    h_out2[o2:o2 + c2].copy_(sets[b]["out2"][b0:b0 + c2], non_blocking=True)
                o1, o2 = o1 + c1, o2 + c2
            ev_out[b] = torch.cuda.Event()
            ev_out[b].record(copy_out)
        d2h[0] = 16 * nb + 8 * (o1 + o2)

    # the link alone: the step's input copy timed by itself (twice)
    link = []
    for _ in range(2):
        a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(copy_in):
            a.record(copy_in)
            for k, v in h_in.items():
                sets[0][k].copy_(v, non_blocking=True)
            z.record(copy_in)
        z.synchronize()
        link.append(h2d / (a.elapsed_time(z) * 1e6))
    ev_w = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ev_s = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ev_e = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for j in range(min(D - 1, steps)):
        issue_inputs(j)
    for i in range(steps):
        b = i % D
        ev_w[i].record(stream)
        stream.wait_event(ev_in[b])
        ev_s[i].record(stream)
        if use_graph:
            graphs[b].replay()
        else:
            pipe.use_buffer_set(sets[b])
            pipe.step()
        ev_e[i].record(stream)
        done = torch.cuda.Event()
        done.record(stream)
        # step i is queued: the host now finishes step i-1 (its counts are on
        # the host once it completes; its output copies go on the copy-out
        # stream ahead of anything that waits for step i), then queues step
        # i's count copy and the inputs of step i + D - 1 into step i-1's set,
        # so the device always has the next step waiting and the input copies
        # overlap running steps
        if i >= 1:
            finish((i - 1) % D)
        with torch.cuda.stream(copy_out):
            copy_out.wait_event(done)
            h_counts[b].copy_(sets[b]["n_out"], non_blocking=True)
            ev_cnt[b].record(copy_out)
        if i + D - 1 < steps:
            issue_inputs((i + D - 1) % D)
    finish((steps - 1) % D)
    torch.cuda.synchronize()
    ms = (time.perf_counter() - t0) * 1e3 / steps
    if B.blsh_status(pipe.ctx) != 0:
        raise RuntimeError("end-to-end steps failed")
    pipe.use_buffer_set(sets[0])
    device_ms = float(np.mean([s_.elapsed_time(e_) for s_, e_ in zip(ev_s, ev_e)]))
    wait_ms = float(np.mean([w_.elapsed_time(s_) for w_, s_ in zip(ev_w, ev_s)]))
    # each input copy's duration, and how long before its step's start it ended
    copy_ms = [a.elapsed_time(z) for a, z in copy_ev]
    lead_ms = [z.elapsed_time(s_) for (a, z), s_ in zip(copy_ev, ev_s)]
    diag = {"depth": D, "input_copy_ms": [round(v, 3) for v in copy_ms],
            "copy_end_to_step_start_ms": [round(v, 3) for v in lead_ms],
            "input_wait_ms": [round(w_.elapsed_time(s_), 3) for w_, s_ in zip(ev_w, ev_s)]}
    del sets, graphs
    return ms, h2d, d2h[0], device_ms, wait_ms, max(link), diag


def large_kernel_work(pipe):
    """Algorithmic bytes of one large-mixed step per kernel name (each launch
    counted for what it must read and write at least once; L2 re-reads not
    counted), from the last step's outputs (exact with one batch; with
    several, the last batch's figures scaled to all pairs)."""
    torch, B, w = pipe.torch, pipe.B, pipe.w
    k, bits, L = w["k"], pipe.bits, pipe.lazy_bits
    P, N, nnz = pipe.P, pipe.N, pipe.nnz
    n_last = pipe.ranges[-1][1] if pipe.ranges else 0
    scale = P / max(n_last, 1)
    st = pipe.status[:n_last]
    nu = pipe.n_used[:n_last].to(torch.int64) & 0xFFFF
    lst = pipe.lstatus[:n_last]
    work = {}
    kept = (st == B.ACCEPT) | (st == B.ACCEPT_AT_MAX)
    chunks = nu // k
    per_chunk = k // 4
    if L:
        Lk = L // k
        resumed = nu > L
        capped = torch.clamp(chunks, max=Lk)
        work["verify_kernel"] = (scale * (n_last * 14 + 4 * int((kept & ~resumed).sum())
                                          + int(capped.sum()) * per_chunk), "B")
        r = int(resumed.sum())
        work["verify_resume_kernel"] = (scale * (n_last + r * 13 + 4 * int((kept & resumed).sum())
                                                 + int(chunks[resumed].sum()) * per_chunk), "B")
    else:
        work["verify_kernel"] = (scale * (n_last * 14 + 4 * int(kept.sum()) + int(chunks.sum()) * per_chunk), "B")
    # the first pass of the two-pass form: the pair, its outputs, four chunks
    work["verify_first_kernel"] = (scale * (n_last * 14 + 4 * int((kept & (nu <= 4 * k)).sum())
                                           + int(torch.clamp(chunks, max=4).sum()) * per_chunk), "B")
    # the projection: per nonzero its index and value, per row its indptr
    # pair and the signature bytes written, each distinct code row once
    row_len = pipe.indptr[1:] - pipe.indptr[:-1]
    distinct = int(torch.unique(pipe.indices).numel())
    cols = L or bits
    b_proj = nnz * 8 + N * (16 + cols // 8) + distinct * cols * 2
    gathered = nnz * cols * 2
    if L:
        sel = pipe.need.bool()
        n_sel = int(sel.sum())
        nnz_sel = int(row_len[sel].sum())
        rows_of = torch.repeat_interleave(sel, row_len)
        d_sel = int(torch.unique(pipe.indices[rows_of]).numel()) if n_sel else 0
        del rows_of
        b_proj += nnz_sel * 8 + n_sel * (16 + (bits - L) // 8) + d_sel * (bits - L) * 2
        gathered += nnz_sel * (bits - L) * 2
    name = "srp_sparse4_kernel (two-byte codes)"
    work[name] = (b_proj, "B")
    work[name + " gathered"] = (gathered, "B")
    # Lite's exact pass over the survivors
    surv = (lst == B.LITE_ACCEPT) | (lst == B.LITE_REJECT)
    ns = int(surv.sum())
    b0_last = pipe.ranges[-1][0] if pipe.ranges else 0
    pr = pipe.pairs[b0_last:b0_last + n_last][surv].to(torch.int64) if ns else None
    surv_nnz = int((row_len[pr[:, 0]] + row_len[pr[:, 1]]).sum()) if ns else 0
    work["lite_collect_kernel"] = (scale * (n_last + 8 * ns), "B")
    # per survivor: its pair, both rows' bounds, the two squared norms (when
    # formed), sim and status written, and both rows (index and value per
    # nonzero); the first 2^23 survivors go through the queue (8 B each), the
    # rest through the in-place pass, which also scans every status
    per_surv = (8 + 32 + 16 + 9) + (surv_nnz / ns * 8 if ns else 0)
    n_q = min(ns, 1 << 23)
    work["lite_queue_kernel"] = (scale * n_q * (per_surv + 8), "B")
    work["lite_exact_kernel"] = (scale * (n_last + (ns - n_q) * per_surv), "B")
    work["row_norm2_kernel"] = (nnz * 4 + N * 8, "B")
    # banding (cosine: packed band keys, LSD radix passes, emission)
    rows, bands = w["rows"], w["bands"]
    n = N * bands
    kb = 4 if max(1, (bands - 1).bit_length()) + rows <= 32 else 8
    obj_rows = N * bands * ((rows + 7) // 8)
    passes = (max(1, (bands - 1).bit_length()) + rows + 7) // 8
    work["band_keys_kernel"] = (N * bands * rows // 8 + n * (kb + 4) + obj_rows, "B")
    work["digit_hist_kernel"] = (passes * n * kb, "B")
    work["digit_scatter_kernel"] = (passes * 2 * n * (kb + 4), "B")
    work["emit_warp_kernel (count pass)"] = (n * (kb + 4) + obj_rows + n * 8, "B")
    work["emit_warp_kernel (write pass)"] = (n * (kb + 4 + 8) + obj_rows + P * 8, "B")
    n_keep = scale * int(kept.sum()) + scale * int((lst == B.LITE_ACCEPT).sum())
    work["compact_count"] = (2 * P, "B")
    work["compact_write"] = (2 * P + 8 * n_keep, "B")
    return {key: (int(v), u) for key, (v, u) in work.items()}


def run_large(args, w):
    """The 5e6-vector mixed workload (one GPU): K timed replays of one
    captured step (hash, band, batched verification and compaction), the
    per-kernel breakdown of eager steps, the end-to-end time through the
    API with host buffers, and the oracle's extrapolated throughput."""
    import torch

    import paper_1110_1328_gb300 as B
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    numa = bind_numa(torch, dev)
    B.lib()
    if world > 1:      # replicas: each rank its own batch of objects
        w = dict(w, seed=w["seed"] + 1000 * rank)
    t0 = time.perf_counter()
    pipe = LargePipeline(B, torch, w, dev, batch_cap=args.batch_pairs)
    setup_s = time.perf_counter() - t0
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        pipe.step()
    if B.blsh_status(pipe.ctx) != 0:
        raise RuntimeError("warm-up step failed")
    launches0 = B.blsh_launch_count(pipe.ctx)
    pipe.step()
    launches_per_step = B.blsh_launch_count(pipe.ctx) - launches0
    torch.cuda.synchronize()

    # one step captured in a CUDA graph (no host sync inside)
    graph = None
    if not args.no_graph:
        try:
            g = torch.cuda.CUDAGraph()
            s = torch.cuda.Stream()
            s.wait_stream(stream)
            with torch.cuda.stream(s):
                pipe.step()
            stream.wait_stream(s)
            torch.cuda.synchronize()
            with torch.cuda.graph(g):
                pipe.step()
            torch.cuda.synchronize()
            g.replay()
            torch.cuda.synchronize()
            graph = g
        except Exception as e:   # capture is an optimisation; eager launches do the same work
            print(f"graph capture failed, timing eager launches: {e}", file=sys.stderr)
            graph = None
    if B.blsh_status(pipe.ctx) != 0:
        raise RuntimeError("graph step failed")

    def one_step():
        if graph is not None:
            graph.replay()
        else:
            pipe.step()

    # ---- device-timed steps ----
    clocks = ClockSampler(local)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    wall0 = time.perf_counter()
    for i in range(args.steps):
        flush.fill_(float(i))            # L2 flush between timed steps (256 MB write)
        starts[i].record(stream)
        one_step()
        ends[i].record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    if dist:
        dist.barrier()
    clk = clocks.stop()
    rc, ctr = B.blsh_status(pipe.ctx, counters=True)
    if rc != 0:
        raise RuntimeError(f"timed steps reported {rc}")
    my_ms = float(np.mean([s_.elapsed_time(e_) for s_, e_ in zip(starts, ends)]))
    kept = pipe.kept_counts()
    hist = pipe.hist.sum(0).cpu().numpy()

    # ---- per-stage and per-kernel device times of eager steps ----
    reps = 2
    B.blsh_timing_begin(pipe.ctx, 8192)
    stage = {s_: 0.0 for s_ in pipe.STAGES}
    for i in range(reps):
        flush.fill_(float(i))
        for s_ in pipe.STAGES:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            getattr(pipe, s_)()
            e1.record(stream)
            torch.cuda.synchronize()
            stage[s_] += e0.elapsed_time(e1) / reps
    kern = {}
    for name, t_ms in B.blsh_timing_end(pipe.ctx, 8192):
        k_ = kern.setdefault(name, [0, 0.0])
        k_[0] += 1
        k_[1] += t_ms
    kern = {n: [c / reps, t_ / reps] for n, (c, t_) in kern.items()}
    if args.profile_step:
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("blsh_step")
        pipe.step()
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()

    # ---- end to end through the public API, host buffers ----
    e2e_step, h2d, d2h, e2e_dev, e2e_wait, e2e_link, e2e_diag = large_e2e(B, torch, pipe, stream, args.steps, graph is not None, kept)
    e2e_ms = [e2e_step]
    e2e_step = float(np.mean(e2e_ms))
    ms, P_total, e2e_max = combine_ranks(dist, my_ms, pipe.P, e2e_step, dev)
    value = P_total / (ms / 1e3)
    e2e_val = P_total / (e2e_max / 1e3)

    # ---- roofline of the dominant kernel ----
    peak, peak_kind = load_peaks()
    work = large_kernel_work(pipe)
    vbytes, v_ms, v_names = verification_totals(work, kern)
    timed = {n: v for n, v in kern.items() if not n.startswith("exclusive scan")}
    dom = max(timed, key=lambda n: timed[n][1])
    dom_launches, dom_ms = timed[dom]
    amount, unit = work.get(dom, (None, None))
    ach = amount / (dom_ms / 1e3) / 1e9 if amount is not None else None
    roofline = {"bound": "hbm", "kernel": dom, "achieved": None if ach is None else round(ach, 1), "peak": peak,
                "unit": "GB/s", "frac": None if ach is None else round(ach / peak, 4),
                "traffic": NCU_TRAFFIC.get((args.workload, dom)), "peak_source": peak_kind,
                "algorithmic_bytes": amount, "launches_per_step": dom_launches, "ms_per_step": round(dom_ms, 4),
                "timing": "library CUDA events around each launch on its stream, eager steps"}
    if dom + " gathered" in work:
        gb = work[dom + " gathered"][0]
        roofline["gathered_bytes"] = int(gb)
        roofline["gathered_GBps"] = round(gb / (dom_ms / 1e3) / 1e9, 1)
    kernels = {n: {"launches": c, "ms": round(t_, 4),
                   **({"GBps": round(work[n][0] / (t_ / 1e3) / 1e9, 1)} if n in work else {})}
               for n, (c, t_) in sorted(kern.items(), key=lambda kv: -kv[1][1])}
    v_ach = vbytes / (v_ms / 1e3) / 1e9 if v_ms else 0.0
    L = pipe.lazy_bits
    need_rows = int(pipe.need.sum().item()) if L else 0
    hashes = pipe.N * (L or pipe.bits) + need_rows * (pipe.bits - L if L else 0)
    hash_ms = kern.get("srp_sparse4_kernel (two-byte codes)", [0, 0.0])[1] + kern.get("srp_recheck_kernel", [0, 0.0])[1]
    out = {
        "metric": METRIC,
        "value": round(value, 1),
        "unit": "pairs/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(ms, 4),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "u32",
        "data": "synthetic",
        "config": {"workload": args.workload + ": " + w["text"], "objects": pipe.N, "nnz": pipe.nnz,
                   "candidate_pairs": pipe.P, "batch_pairs": pipe.batch, "batches": len(pipe.ranges),
                   "setup_s": round(setup_s, 1), "l2": "flushed between timed steps (256 MB write); the 68.7 GB "
                   "of codes and 1.3 GB of signatures exceed L2", "cuda_graph": graph is not None,
                   "plan": dict(pipe.plan.as_dict(), k=w["k"]), "lazy_bits": L,
                   "parallelism": f"replicas x{world}" if world > 1 else "1 GPU"},
        "e2e": {"value": round(e2e_val, 1), "unit": "pairs/s", "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h), "ms_per_step": round(e2e_step, 4),
                "device_ms_per_step": round(e2e_dev, 4), "input_wait_ms_per_step": round(e2e_wait, 4),
                "h2d_gbs_alone": round(e2e_link, 1), "host_numa": numa, "per_step": e2e_diag,
                "form": "inputs copied from pinned host memory and output sets copied back every step; a ring of "
                        "device buffer sets (per_step.depth), step i + depth - 1's inputs copied while step i runs, "
                        "step i's outputs read while step i+1 runs"},
        "gpu_launches": int(launches_per_step * args.steps),
        "roofline": roofline,
        "verify_hbm": {"achieved": round(v_ach, 1), "peak": peak, "unit": "GB/s", "frac": round(v_ach / peak, 4),
                       "algorithmic_bytes": int(vbytes), "ms": round(v_ms, 4),
                       "kernels": v_names,
                       "counts": "per pair: its indices, its outputs and the chunks it compares; a row shared by several "
                                 "pairs is counted for each, so where pairs share rows (L2 re-reads) the figure can "
                                 "exceed the copy bandwidth"},
        "kernels": kernels,
        "hashes_per_s": round(hashes / (hash_ms / 1e3), 1) if hash_ms else None,
        "hashes_per_step": int(hashes),
        "stage_ms": {k_: round(v, 4) for k_, v in stage.items()},
        "outputs": {"bayeslsh_kept": kept[0], "lite_kept": kept[1], "objects_hashed_in_full": need_rows,
                    "stop_hist_first4": [int(v) for v in hist[:4]]},
        "clocks": clk,
        "wall_s_timed_loop": round(wall, 3),
        "srp_signs": {"rechecked_per_step": ctr[2] / args.steps, "zero_dots_per_step": ctr[3] / args.steps},
    }
    if rank == 0 and not args.no_cpu_baseline and world == 1:
        out["cpu_baseline"] = large_cpu_baseline(pipe, w, seed=1)
    elif rank == 0 and world > 1:
        out["cpu_baseline"] = None
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def oracle_codes(O, seed, terms, bits, threads=1):
    """The oracle's own two-byte codes for the given rows of R (its generator,
    from the same counter definition as the library's)."""
    import concurrent.futures as cf
    out = np.zeros((len(terms), bits), np.uint16)

    def fill(lo, hi):
        for i in range(lo, hi):
            out[i] = O.gaussian_codes(seed, 1, bits, row0=int(terms[i]))[0]

    step = -(-len(terms) // max(threads, 1))
    with cf.ThreadPoolExecutor(max(threads, 1)) as ex:
        list(ex.map(lambda lo: fill(lo, min(lo + step, len(terms))), range(0, len(terms), step or 1)))
    return out


def large_oracle_inputs(pipe, w, seed, n_pairs=20_000, n_hash=2_000, threads=1):
    """The oracle's inputs for a seeded sample of the large workload:
      - n_hash objects drawn uniformly (their rows copied from the device,
        terms renumbered) with the oracle's own codes for their terms: the
        hashing and banding sample;
      - n_pairs candidate pairs drawn uniformly from the candidate list, their
        objects' rows and the oracle's own signatures of them (from its own
        codes, computed here, untimed): the verification sample."""
    import oracle as O
    import synth
    torch = pipe.torch
    rng = np.random.default_rng(seed)

    def rows_of(ids):
        ids_t = torch.from_numpy(ids.astype(np.int64)).to(pipe.dev)
        lo, hi = pipe.indptr[ids_t].cpu().numpy(), pipe.indptr[ids_t + 1].cpu().numpy()
        sel = np.concatenate([np.arange(a, b) for a, b in zip(lo, hi)]) if len(ids) else np.zeros(0, np.int64)
        sel_t = torch.from_numpy(sel).to(pipe.dev)
        terms = pipe.indices[sel_t].cpu().numpy().view(np.uint32)
        vals = pipe.values[sel_t].cpu().numpy()
        uterm, tinv = np.unique(terms, return_inverse=True)
        csr = synth.CSR(np.concatenate([[0], np.cumsum(hi - lo)]).astype(np.int64), tinv.astype(np.uint32), vals,
                        len(uterm))
        return csr, oracle_codes(O, w["r_seed"], uterm, w["bits"], threads)

    hash_ids = np.sort(rng.choice(pipe.N, min(n_hash, pipe.N), replace=False))
    hash_csr, hash_codes = rows_of(hash_ids)
    q = np.sort(rng.choice(pipe.P, min(n_pairs, pipe.P), replace=False))
    sp = pipe.pairs[torch.from_numpy(q).to(pipe.dev)].cpu().numpy().view(np.uint32)
    ids, inv = np.unique(sp.reshape(-1), return_inverse=True)
    pair_csr, pair_codes = rows_of(ids)
    sig = oracle_signatures(O, pair_csr, pair_codes, threads)
    del pair_codes
    return {"hash_csr": hash_csr, "hash_codes": hash_codes, "pair_csr": pair_csr, "pair_sig": sig,
            "pairs": inv.reshape(-1, 2).astype(np.uint32)}


def sub_csr(csr, lo, hi):
    import synth
    a, b = int(csr.indptr[lo]), int(csr.indptr[hi])
    return synth.CSR(csr.indptr[lo:hi + 1] - a, csr.indices[a:b], csr.values[a:b], csr.dim)


def oracle_signatures(O, csr, codes, threads=1):
    """The oracle's two-byte-code signatures of all bits of every row, the
    rows split over `threads` host threads."""
    import concurrent.futures as cf
    cuts = np.linspace(0, csr.n, threads + 1).astype(int)
    with cf.ThreadPoolExecutor(threads) as ex:
        parts = list(ex.map(lambda i: O.srp_sparse_q16(sub_csr(csr, cuts[i], cuts[i + 1]), codes), range(threads)))
    return np.concatenate(parts)


def large_oracle_times(O, w, inp, threads=1, min_verify_s=1.0):
    """Seconds the oracle takes on `threads` host threads for: the signatures
    (all bits) of the hashing sample, the banding of those signatures (one
    thread: the oracle's sort is sequential), and one pass of Algorithms 1
    and 2 with both compactions over the sampled pairs (repeated until
    min_verify_s, averaged).  Also counts the sampled pairs that do not
    collide in any band under the oracle's own signatures (0 expected)."""
    import concurrent.futures as cf
    p = O.Params(kind=1, t=w["t"], k=w["k"], n_max=w["n_max"], h=w["h"])
    tab = O.tables(p)
    t0 = time.perf_counter()
    hsig = oracle_signatures(O, inp["hash_csr"], inp["hash_codes"], threads)
    t_hash = time.perf_counter() - t0
    t0 = time.perf_counter()
    O.lsh_candidates(hsig, 1, w["rows"], w["bands"])
    t_band = time.perf_counter() - t0
    lp, sig, csr = inp["pairs"], inp["pair_sig"], inp["pair_csr"]
    r, bands = w["rows"], w["bands"]
    band = lambda s, b: (s[:, (b * r) // 32] >> np.uint32((b * r) % 32)) & np.uint32((1 << r) - 1)
    collide = np.zeros(len(lp), bool)
    for b in range(bands):
        collide |= band(sig[lp[:, 0]], b) == band(sig[lp[:, 1]], b)
    keep1 = (1 << O.ACCEPT) | (1 << O.ACCEPT_AT_MAX)
    cuts = np.linspace(0, len(lp), threads + 1).astype(int)

    def one(i):
        sl = lp[cuts[i]:cuts[i + 1]]
        res = O.verify(tab, sl, sig)
        O.compact(res.status, keep1)
        lres = O.verify_lite(tab, sl, sig, csr)
        O.compact(lres.status, 1 << O.LITE_ACCEPT)
        return res

    with cf.ThreadPoolExecutor(threads) as ex:
        reps, t0 = 0, time.perf_counter()
        while True:
            res = list(ex.map(one, range(threads)))
            reps += 1
            if time.perf_counter() - t0 >= min_verify_s:
                break
        t_verify = (time.perf_counter() - t0) / reps
    return {"hash_s": t_hash, "band_s": t_band, "verify_s": t_verify, "objects": inp["hash_csr"].n,
            "nnz": int(inp["hash_csr"].indptr[-1]), "pairs": len(lp), "not_colliding": int((~collide).sum())}


def extrapolate(t, N, nnz, P):
    """Seconds of one whole step over the full workload: hashing scaled by
    the nonzeros, banding by the objects, verification by the pairs."""
    return nnz * t["hash_s"] / max(t["nnz"], 1) + N * t["band_s"] / max(t["objects"], 1) + P * t["verify_s"] / max(
        t["pairs"], 1)


def large_cpu_baseline(pipe, w, seed=1):
    """The oracle timed on the host cores on a seeded sample of the large
    workload (its own signatures from its own codes), single-threaded and on
    all cores, extrapolated to the whole step: candidate pairs verified per
    second."""
    import oracle as O
    O.build()
    cores = len(os.sched_getaffinity(0))
    inp = large_oracle_inputs(pipe, w, seed, threads=cores)
    t1 = large_oracle_times(O, w, inp, threads=1)
    tc = large_oracle_times(O, w, inp, threads=cores)
    T1, TC = extrapolate(t1, pipe.N, pipe.nnz, pipe.P), extrapolate(tc, pipe.N, pipe.nnz, pipe.P)
    comp = lambda t: {"hash_s_per_1e6_nnz": round(t["hash_s"] / t["nnz"] * 1e6, 4),
                      "band_s_per_1e6_objects": round(t["band_s"] / t["objects"] * 1e6, 4),
                      "verify_pairs_per_s": round(t["pairs"] / t["verify_s"], 1)}
    return {"value": round(pipe.P / T1, 1), "unit": "pairs/s", "cores": 1, "kind": "oracle",
            "sample": f"seeded uniform samples of the workload: {t1['objects']} objects ({t1['nnz']} nonzeros) hashed "
                      f"over all {w['bits']} bits and banded, {t1['pairs']} of the {pipe.P} candidate pairs through "
                      f"Algorithms 1 and 2 and both compactions (the oracle's own signatures from its own codes); "
                      f"hashing scaled by nonzeros, banding by objects, verification by pairs to the full step "
                      f"({T1:.0f} s single-threaded); sampled pairs not colliding under the oracle's signatures: "
                      f"{t1['not_colliding']}",
            "components": comp(t1),
            "all_cores": {"value": round(pipe.P / TC, 1), "cores": cores, "step_s": round(TC, 1),
                          "components": comp(tc),
                          "form": "the same oracle calls over chunks of objects (hashing) and of pairs "
                                  "(verification) in host threads; banding single-threaded"}}


def run_reference_large(args, w):
    """The reference arm on the large workload: each step the single-threaded
    oracle over a bounded sample (hashing and banding of 2,000 objects,
    Algorithms 1 and 2 over 20,000 candidate pairs), extrapolated to the
    whole step as in the cpu_baseline leg.  The workload and its candidate
    list come from the GPU pipeline (inputs); the oracle checks that every
    sampled pair collides in a band under its own signatures."""
    import torch

    import oracle as O
    import paper_1110_1328_gb300 as B
    O.build()
    dev = torch.device("cuda", 0)
    B.lib()
    pipe = LargePipeline(B, torch, w, dev)
    pipe.step()
    if B.blsh_status(pipe.ctx) != 0:
        raise RuntimeError("workload step failed")
    cores = len(os.sched_getaffinity(0))
    inp = large_oracle_inputs(pipe, w, seed=1, threads=cores)
    for _ in range(args.warmup):
        large_oracle_times(O, w, inp, threads=1, min_verify_s=0.0)
    secs, ext = 0.0, 0.0
    nc = 0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        t = large_oracle_times(O, w, inp, threads=1, min_verify_s=0.0)
        secs += time.perf_counter() - t0
        ext += extrapolate(t, pipe.N, pipe.nnz, pipe.P)
        nc += t["not_colliding"]
    value = pipe.P * args.steps / ext
    sample = (f"each step: the single-threaded oracle over {inp['hash_csr'].n} objects (hashed over all {w['bits']} "
              f"bits, banded) and {len(inp['pairs'])} of the {pipe.P} candidate pairs (Algorithms 1 and 2, both "
              f"compactions), extrapolated to the whole step ({ext / args.steps:.0f} s); sampled pairs not colliding "
              f"under the oracle's signatures: {nc // max(args.steps, 1)}")
    out = {"impl": "reference", "metric": METRIC, "value": round(value, 1), "unit": "pairs/s", "n_gpus": 0,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(secs / args.steps * 1e3, 3),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": args.workload + ": " + w["text"], "extrapolated_step_s": round(ext / args.steps, 1)},
           "cpu_baseline": {"value": round(value, 1), "unit": "pairs/s", "cores": 1, "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": round(value, 1), "unit": "pairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# ---------------------------------------------------------------------------
# CPU oracle timings (the cpu_baseline leg and the reference arm)
# ---------------------------------------------------------------------------

def oracle_pass(O, w, objs, hashp):
    """One pass of the oracle over the given objects; returns (pairs, seconds)."""
    t0 = time.perf_counter()
    if getattr(objs, "X", None) is not None:
        sig = O.srp_dense(objs.X, hashp)
    elif w["kind"] == 1 and w.get("r_format") == "q16":
        sig = O.srp_sparse_q16(objs, O.quantize_gaussian(hashp)[0])
    elif w["kind"] == 1:
        sig = O.srp_sparse(objs, hashp)
    else:
        sig = O.minhash(objs, hashp[0], hashp[1])
    pairs = O.lsh_candidates(sig, w["kind"], w["rows"], w["bands"])
    p = O.Params(kind=w["kind"], t=w["t"], k=w["k"], n_max=w["n_max"], h=w["h"])
    tab = O.tables(p)
    t1 = time.perf_counter()
    r = O.verify(tab, pairs, sig)
    O.compact(r.status, (1 << O.ACCEPT) | (1 << O.ACCEPT_AT_MAX))
    if "lite" in w.get("stages", ("lite",)):
        lr = O.verify_lite(tab, pairs, sig, objs)
        O.compact(lr.status, 1 << O.LITE_ACCEPT)
    t2 = time.perf_counter()
    return len(pairs), t2 - t0, t1 - t0


def sample_objects(objs, n):
    """The first n objects of a workload (same generator, same distribution)."""
    e = int(objs.indptr[n])
    sub = synth.CSR(objs.indptr[: n + 1].copy(), objs.indices[:e], None if objs.values is None else objs.values[:e],
                    objs.dim)
    if getattr(objs, "X", None) is not None:
        sub.X = objs.X[:n]
    return sub


def cpu_baseline(w, objs, hashp, P_full):
    import oracle as O
    O.build()
    n = objs.n if objs.n <= 20000 else 20000
    sub = objs if n == objs.n else sample_objects(objs, n)
    P, secs, _ = oracle_pass(O, w, sub, hashp)
    return {"value": round(P / secs, 1), "unit": "pairs/s", "cores": 1, "kind": "oracle",
            "sample": f"one single-threaded oracle pass over the first {n} of {objs.n} objects "
                      f"({P} candidate pairs, {secs:.1f} s)"}


def run_reference(args, w):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    if args.workload == "large-mixed":
        run_reference_large(args, w)
        return
    if w.get("gpu_only"):
        print(json.dumps({"impl": "reference", "unavailable": "a GPU measurement workload; "
                                                               "the oracle arm runs on the pipeline workloads"}))
        return
    import oracle as O
    O.build()
    objs, hashp = make_inputs(w, 0)
    # each step: the oracle on a bounded slice of the same workload, sized for a
    # few seconds of CPU work per step
    n = min(objs.n, 4000 if w["kind"] == 1 else 20000)
    sub = sample_objects(objs, n)
    for _ in range(args.warmup):
        oracle_pass(O, w, sub, hashp)
    t0 = time.perf_counter()
    P = 0
    for _ in range(args.steps):
        p, _, _ = oracle_pass(O, w, sub, hashp)
        P += p
    secs = time.perf_counter() - t0
    value = P / secs
    out = {"impl": "reference", "metric": METRIC, "value": round(value, 1), "unit": "pairs/s", "n_gpus": 0,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(secs / args.steps * 1e3, 3),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": args.workload + ": " + w["text"]},
           "cpu_baseline": {"value": round(value, 1), "unit": "pairs/s", "cores": 1, "kind": "oracle",
                            "sample": f"each step: the oracle over the first {n} of {objs.n} objects "
                                      f"({P // args.steps} candidate pairs)"},
           "e2e": {"value": round(value, 1), "unit": "pairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="large-mixed", choices=sorted(WORKLOADS))
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-graph", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--profile-step", action="store_true",
                    help="run one extra eager step inside the NVTX range blsh_step (for ncu captures)")
    ap.add_argument("--lazy-bits", type=int, default=None,
                    help="sparse cosine: hashes computed for every object before verification (a multiple of 128; "
                         "0 = all up front); the workload's setting otherwise")
    ap.add_argument("--batch-pairs", type=int, default=None,
                    help="large-mixed: at most this many candidate pairs per device batch (default: sized by free HBM)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    w = dict(WORKLOADS[args.workload])
    if args.lazy_bits is not None:
        w["lazy_bits"] = args.lazy_bits
    if args.impl == "reference":
        run_reference(args, w)
    elif args.workload in ("verify-large", "verify-profile"):
        run_verify_large(args, w)
    elif args.workload in ("large-mixed", "large-profile"):
        run_large(args, w)
    elif args.workload == "sweep":
        run_sweep(args, w)
    else:
        run_ours(args, w)


if __name__ == "__main__":
    main()
