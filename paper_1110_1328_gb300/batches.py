"""Streaming candidate pairs through device-resident batches, with a resumable
record of progress.

Algorithms 1 and 2 treat every candidate pair on its own, so a candidate list
too large for the device's free memory is verified batch by batch: the pairs
[b0, b0 + n) of batch b go through the library's verification and compaction
calls with per-batch output buffers, and the kept indices of each batch (plus
b0) are the batch's part of the output set.  This module holds the host-side
part of that: the batch ranges, and a checkpoint file that records, after each
finished batch, the next unfinished one together with the kept counts and the
stop histogram accumulated so far, so that an interrupted job resumes at the
first batch it had not finished (the batch is the resumable unit) and never
counts a batch twice.  It runs no computation of the method: the calls made
for a batch are the caller's.
"""
from __future__ import annotations

import json
import os
from dataclasses import dataclass, field


def batch_ranges(P: int, batch: int) -> list[tuple[int, int]]:
    """(b0, n) of every batch of at most `batch` pairs covering [0, P)."""
    if P < 0 or batch <= 0:
        raise ValueError("P must be >= 0 and batch > 0")
    return [(b0, min(batch, P - b0)) for b0 in range(0, P, batch)]


@dataclass
class BatchRecord:
    """Progress of one streamed job: `job` identifies it (sizes, seeds, ...),
    `next_batch` is the first batch not yet finished, `kept` the kept counts
    per output set and `hist` the stop histogram summed over the finished
    batches."""
    job: dict
    next_batch: int = 0
    kept: list = field(default_factory=list)
    hist: list = field(default_factory=list)

    def to_json(self) -> str:
        return json.dumps({"job": self.job, "next_batch": self.next_batch, "kept": self.kept, "hist": self.hist})


class Checkpoint:
    """A BatchRecord kept in a file, replaced atomically after every batch."""

    def __init__(self, path: str):
        self.path = path

    def load(self, job: dict) -> BatchRecord:
        """The record of `job`, or a fresh one if the file is missing.  A file
        that records another job is an error (its counts must not be added to
        this one's)."""
        if not os.path.exists(self.path):
            return BatchRecord(job=job)
        with open(self.path) as f:
            d = json.load(f)
        if d.get("job") != job:
            raise ValueError(f"checkpoint {self.path} records another job: {d.get('job')}")
        return BatchRecord(job=d["job"], next_batch=int(d["next_batch"]), kept=list(d["kept"]), hist=list(d["hist"]))

    def save(self, rec: BatchRecord) -> None:
        tmp = f"{self.path}.tmp{os.getpid()}"
        with open(tmp, "w") as f:
            f.write(rec.to_json())
            f.flush()
            os.fsync(f.fileno())
        os.replace(tmp, self.path)

    def clear(self) -> None:
        if os.path.exists(self.path):
            os.remove(self.path)


def stream_batches(P: int, batch: int, run_batch, job: dict, checkpoint: Checkpoint | None = None,
                   n_kept: int = 2, levels: int = 0) -> BatchRecord:
    """Runs run_batch(b, b0, n) -> (kept counts, stop histogram) for every
    batch from the first unfinished one on, adding its results to the record
    and saving the record after each batch.  run_batch must leave nothing of
    a batch half-recorded: the record moves on only after it returns (it
    synchronises with the device before returning its counts).  Returns the
    final record."""
    ranges = batch_ranges(P, batch)
    rec = checkpoint.load(job) if checkpoint else BatchRecord(job=job)
    if not rec.kept:
        rec.kept = [0] * n_kept
    if not rec.hist:
        rec.hist = [0] * levels
    for b in range(rec.next_batch, len(ranges)):
        b0, n = ranges[b]
        kept, hist = run_batch(b, b0, n)
        rec.kept = [int(a) + int(c) for a, c in zip(rec.kept, kept)]
        if len(hist):
            rec.hist = [int(a) + int(c) for a, c in zip(rec.hist, hist)] if rec.hist else [int(c) for c in hist]
        rec.next_batch = b + 1
        if checkpoint:
            checkpoint.save(rec)
    return rec
