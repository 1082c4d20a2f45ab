"""Pins of the oracle's evicting history model (Sec. 3.4.3), no GPU: a
hand-worked sequence, the no-pressure case against a plain set of seen keys,
and the rebase of priorities."""
import numpy as np

from oracle import pps_oracle as O


def _w(rank, f):
    return int(O.evict_word(rank, f))


def test_hand_worked_eviction_sequence():
    """T = 8, P = 3, every key homed at slot 0.

    Frame 1: A, B, C take slots 0, 1, 2 (fresh); D finds a full window whose
    entries are all from this frame and gets no history.
    Frame 2, order D, A, B, C: D evicts the smallest word (A, slot 0); A then
    evicts B (slot 1, the smallest of B(1), C(1), D(2)); B evicts C (slot 2);
    C meets D(2), A(2), B(2), all from this frame, and gets none."""
    table = np.zeros(8, dtype=np.uint32)
    A, B, C, D = 0x11, 0x22, 0x33, 0x44
    home = np.zeros(4, dtype=np.uint32)
    slot, fresh = O.history_evict_step(table, home, np.array([A, B, C, D], np.uint32), 1, 3)
    assert list(slot) == [0, 1, 2, -1] and list(fresh) == [True, True, True, False]
    assert [int(x) for x in table[:3]] == [_w(1, A), _w(1, B), _w(1, C)]
    slot, fresh = O.history_evict_step(table, home, np.array([D, A, B, C], np.uint32), 2, 3)
    assert list(slot) == [0, 1, 2, -1] and list(fresh) == [True, True, True, False]
    assert [int(x) for x in table[:3]] == [_w(2, D), _w(2, A), _w(2, B)]
    # frame 3: B finds its own entry (kept, priority refreshed, not fresh)
    slot, fresh = O.history_evict_step(table, home[:1], np.array([B], np.uint32), 3, 3)
    assert list(slot) == [2] and list(fresh) == [False]
    assert int(table[2]) == _w(3, B)


def test_without_pressure_nothing_is_evicted():
    """A table far larger than the keys: a cell is fresh exactly the first
    time its key is seen (checked against a plain set)."""
    rng = np.random.default_rng(0)
    keys = rng.integers(1, 2 ** 32, 3000, dtype=np.uint64).astype(np.uint32)
    homes = rng.integers(0, 1 << 16, 3000).astype(np.uint32)
    table = np.zeros(1 << 16, dtype=np.uint32)
    seen = set()
    for frame in range(1, 6):
        pick = rng.choice(3000, 1500, replace=False)
        slot, fresh = O.history_evict_step(table, homes[pick], keys[pick], frame, 16)
        assert np.all(slot >= 0)
        expect = np.array([int(k) & O.EVICT_FP_MASK not in seen for k in keys[pick]])
        # distinct keys may share 24 fingerprint bits only by chance; none do here
        assert np.array_equal(fresh, expect)
        seen.update(int(k) & O.EVICT_FP_MASK for k in keys[pick])
        assert np.all((table[table != 0] >> 24) <= frame)


def test_under_pressure_recent_entries_survive():
    """Region A's keys fill a small table in frames 1-2; region B's keys in
    frames 3-4 evict them: at frame 4 B's cells find their frame-3 entries,
    and A's cells at frame 5 start afresh."""
    rng = np.random.default_rng(1)
    T, P = 1 << 10, 16
    a = rng.integers(1, 2 ** 32, 700, dtype=np.uint64).astype(np.uint32)
    b = rng.integers(1, 2 ** 32, 700, dtype=np.uint64).astype(np.uint32)
    ha = rng.integers(0, T, 700).astype(np.uint32)
    hb = rng.integers(0, T, 700).astype(np.uint32)
    table = np.zeros(T, dtype=np.uint32)
    for frame in (1, 2):
        O.history_evict_step(table, ha, a, frame, P)
    s3, f3 = O.history_evict_step(table, hb, b, 3, P)
    assert f3[s3 >= 0].all() and (s3 >= 0).mean() > 0.9
    s4, f4 = O.history_evict_step(table, hb, b, 4, P)
    kept = s3 >= 0
    assert (~f4[kept]).mean() > 0.9  # B's entries from frame 3 are still there
    s5, f5 = O.history_evict_step(table, ha, a, 5, P)
    assert f5[s5 >= 0].mean() > 0.7  # most of A was evicted by B


def test_age_rebase_keeps_recent_order():
    f = np.arange(1, 7, dtype=np.uint32)
    ranks = [255, 200, 129, 128, 3, 1]
    table = np.array([int(O.evict_word(r, x)) for r, x in zip(ranks, f)] + [0], dtype=np.uint32)
    O.history_age(table, 128)
    got = [int(w) >> 24 for w in table[:6]]
    assert got == [127, 72, 1, 1, 1, 1]
    assert [int(w) & 0xFFFFFF for w in table[:6]] == list(range(1, 7))
    assert table[6] == 0
