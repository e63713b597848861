"""The word layout of the banding emission's keep record, checked on the CPU.

In a walk over partners [jmin, jmax) the count pass stores, for lane l, bit t
of word w at rec[32 w + l] for partner jmin + 32 w + t.  Its batches of at
most 32 partners do not start on word boundaries where the staged window
ends, so each batch's kept bits are spliced into the lane's words by a
register accumulator that stores a word once it is complete (and the last,
partial one at the end).  This file restates that accumulator and checks,
for every split of [jmin, jmax) into window and beyond-window batches, that
it writes each word exactly once with exactly the bits of direct placement,
and that the number of words is the one the count pass reserves."""
import random


def batches(jmin, jmax, win):
    """The walk's batches: inside the window, then past it, 32 at a time."""
    out = []
    wend = min(jmax, win)
    j0 = jmin
    while j0 < wend:
        n = min(wend - j0, 32)
        out.append((j0, n))
        j0 += n
    j0 = max(jmin, win)
    while j0 < jmax:
        n = min(jmax - j0, 32)
        out.append((j0, n))
        j0 += n
    return out


def spliced(jmin, jmax, win, keep_of):
    """The accumulator: returns {word index: word} as stored."""
    stored = {}
    ridx, racc = 0, 0

    def store(i, v):
        assert i not in stored, "a word stored twice"
        stored[i] = v

    for j0, n in batches(jmin, jmax, win):
        keep = keep_of(j0, n)
        g0 = j0 - jmin
        w, sh = g0 >> 5, g0 & 31
        if w != ridx:
            store(ridx, racc)
            racc, ridx = 0, w
        racc |= (keep << sh) & 0xFFFFFFFF
        if sh + n > 32:
            store(ridx, racc)
            ridx += 1
            racc = keep >> (32 - sh)
    if jmax > jmin:
        store(ridx, racc)
    return stored


def test_record_words_equal_direct_placement():
    rng = random.Random(3)
    for _ in range(4000):
        jmin = 1
        jmax = rng.choice([1, 2, 31, 32, 33, 64, 65, rng.randint(1, 400)])
        win = rng.choice([1, 2, 16, 32, 33, 100, rng.randint(1, 400)])
        kept = {j for j in range(jmin, jmax) if rng.random() < rng.choice([0.0, 0.1, 0.5, 1.0])}

        def keep_of(j0, n):
            return sum(1 << u for u in range(n) if j0 + u in kept)

        got = spliced(jmin, jmax, win, keep_of)
        words = (jmax - jmin + 31) // 32 if jmax > jmin else 0
        assert sorted(got) == list(range(words))          # every reserved word, once
        want = {}
        for j in kept:
            g = j - jmin
            want[g >> 5] = want.get(g >> 5, 0) | 1 << (g & 31)
        for w in range(words):
            assert got[w] == want.get(w, 0), (jmin, jmax, win, w)


def test_batches_cover_the_partner_range_in_order():
    for jmax in range(1, 140):
        for win in (1, 5, 32, 33, 64, 70, 200):
            js = [j for j0, n in batches(1, jmax, win) for j in range(j0, j0 + n)]
            assert js == list(range(1, jmax))
