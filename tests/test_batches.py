"""Host-side batch streaming and its checkpoint record (the pair batch is the
resumable unit): an interrupted job resumes at its first unfinished batch,
every batch is counted once, and a record of another job is refused."""
import pytest

from paper_1110_1328_gb300.batches import BatchRecord, Checkpoint, batch_ranges, stream_batches


def test_batch_ranges_cover_every_pair_once():
    for P, b in ((0, 7), (1, 7), (7, 7), (8, 7), (1000, 333), (999_999_937, 123_456_789)):
        r = batch_ranges(P, b)
        assert sum(n for _, n in r) == P
        assert all(0 < n <= b for _, n in r)
        assert all(r[i][0] + r[i][1] == r[i + 1][0] for i in range(len(r) - 1))
        assert not r or r[0][0] == 0
    with pytest.raises(ValueError):
        batch_ranges(10, 0)


class Interrupt(Exception):
    pass


def fake_batch(seen, stop_at=None):
    """A batch's results as the device would give them: kept counts and a
    stop histogram that depend on the batch's pairs only."""
    def run(b, b0, n):
        if stop_at is not None and b == stop_at:
            raise Interrupt()
        seen.append(b)
        return [n // 3, n // 5], [n % 7, 1, b]
    return run


def test_interrupted_job_resumes_at_the_next_unfinished_batch(tmp_path):
    P, batch = 10_007, 1_000
    job = {"workload": "test", "P": P, "batch": batch}
    full = stream_batches(P, batch, fake_batch([]), job, None, levels=3)
    ck = Checkpoint(str(tmp_path / "ck.json"))
    seen = []
    with pytest.raises(Interrupt):
        stream_batches(P, batch, fake_batch(seen, stop_at=4), job, ck, levels=3)
    assert seen == [0, 1, 2, 3]
    rec = ck.load(job)
    assert rec.next_batch == 4
    # a second interruption later on, then completion
    with pytest.raises(Interrupt):
        stream_batches(P, batch, fake_batch(seen, stop_at=8), job, ck, levels=3)
    done = stream_batches(P, batch, fake_batch(seen), job, ck, levels=3)
    assert seen == list(range(len(batch_ranges(P, batch))))        # every batch exactly once
    assert done.next_batch == len(batch_ranges(P, batch))
    assert done.kept == full.kept and done.hist == full.hist
    # running again after completion does nothing more
    again = stream_batches(P, batch, fake_batch(seen), job, ck, levels=3)
    assert again.kept == full.kept and seen == list(range(11))


def test_checkpoint_of_another_job_is_refused(tmp_path):
    ck = Checkpoint(str(tmp_path / "ck.json"))
    ck.save(BatchRecord(job={"P": 5}, next_batch=1, kept=[1, 1], hist=[]))
    with pytest.raises(ValueError):
        ck.load({"P": 6})
    ck.clear()
    assert ck.load({"P": 6}).next_batch == 0
