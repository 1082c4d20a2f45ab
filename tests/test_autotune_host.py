"""The autotuner's choice among its trials (host logic, no GPU)."""
import pytest

from paper_1902_05942_gb300 import autotune


def _t(lg, P, ms, ovf):
    return {"log2_slots": lg, "max_probes": P, "ms": ms, "overflow": ovf}


def test_fastest_among_those_that_do_not_overflow():
    trials = [_t(21, 8, 0.20, 3e-4), _t(22, 16, 0.25, 0.0), _t(23, 16, 0.22, 5e-6),
              _t(24, 32, 0.30, 0.0)]
    assert autotune.choose(trials, 1e-5) == trials[2]
    # a stricter bar drops the 5e-6 candidate
    assert autotune.choose(trials, 0.0) == trials[1]


def test_least_overflow_when_none_qualifies():
    trials = [_t(21, 8, 0.10, 3e-3), _t(21, 16, 0.12, 1e-3), _t(22, 8, 0.09, 1e-3)]
    assert autotune.choose(trials, 1e-5) == trials[2]  # least overflow, then fastest


def test_no_trials_is_an_error():
    with pytest.raises(ValueError):
        autotune.choose([], 1e-5)


def test_near_ties_go_to_the_smaller_table_and_probe_limit():
    """Trials within 3 % of the fastest count as equally fast: the smaller
    table wins, then the smaller probe limit, so that two identical views
    timed with a little noise get the same choice."""
    a = [_t(24, 32, 0.200, 0.0), _t(22, 16, 0.205, 0.0), _t(22, 8, 0.204, 0.0),
         _t(21, 8, 0.30, 0.0)]
    b = [_t(24, 32, 0.206, 0.0), _t(22, 16, 0.201, 0.0), _t(22, 8, 0.203, 0.0),
         _t(21, 8, 0.31, 0.0)]
    assert autotune.choose(a, 1e-5) == a[2]
    assert autotune.choose(b, 1e-5) == b[2]
    # beyond the 3 % band the faster one wins
    c = [_t(24, 32, 0.200, 0.0), _t(22, 8, 0.210, 0.0)]
    assert autotune.choose(c, 1e-5) == c[0]


def test_batch_shape_choice():
    import torch  # noqa: F401  (the module imports torch)

    class FakeBatch:
        def __init__(self, ms):
            self.ms = ms

        def run(self, cams, frame):
            pass

        def close(self):
            pass

    times = {(2, 512): 1.00, (4, 512): 1.50, (2, 256): 0.99, (4, 256): 0.80}
    order = list(times)
    seen = []

    def make(w, blk):
        seen.append((w, blk))
        return FakeBatch(times[(w, blk)])

    # time with the fake batch's own number instead of CUDA events
    orig = autotune._time
    autotune._time = lambda fn, reps: seen and times[seen[-1]]
    try:
        shape, trials = autotune.tune_batch_shape(make, [], shapes=order)
    finally:
        autotune._time = orig
    assert shape == (4, 256)
    times[(4, 256)] = 0.995  # now within 3 % of (2, 256) and (2, 512): the first listed wins
    seen.clear()
    autotune._time = lambda fn, reps: seen and times[seen[-1]]
    try:
        shape, _ = autotune.tune_batch_shape(make, [], shapes=order)
    finally:
        autotune._time = orig
    assert shape == (2, 512)
