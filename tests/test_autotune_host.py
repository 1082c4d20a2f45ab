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
