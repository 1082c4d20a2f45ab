"""Failure detection without a GPU fault: every device wait of the library
has a time limit, after which the kernel records an error and returns.  Each
test makes one wait run out on a condition that nothing fulfils (a grid
barrier one CTA short, an mbarrier phase no operation completes), checks the
error word the host reads, and then runs a frame to show that the context is
still usable."""
import time

import numpy as np
import pytest
import torch

from oracle import pps_oracle as O
from paper_1902_05942_gb300 import configs, pps, scene

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1902_05942_gb300 import build
    build.build()
    torch.cuda.set_device(0)
    yield


@pytest.mark.parametrize("kind", [0, 1])
def test_a_stuck_wait_ends_with_an_error_status(kind):
    t0 = time.perf_counter()
    word = pps.pps_selftest_wait(kind, 20000)  # 20 ms
    elapsed = time.perf_counter() - t0
    assert word == 1
    assert elapsed < 10.0
    # the context is still usable: a small frame against the oracle
    w = configs.small()
    spec = configs.frame_spec(w, 0, 0)
    spec.view.width, spec.view.height = 64, 48
    cfg = w.filters[0]
    cfg.pixel_angle = spec.view.pixel_angle()
    v = scene.trace_stream(spec, 0, "cpu")
    tab = pps.Table(cfg)
    out = tab.filter({k: v[k].to("cuda") for k in scene.STREAMS}, spec.view.eye, 0)
    fr = O.filter_frame(O.KeyParams(**cfg.oracle_kwargs()), spec.view.eye, 0,
                        {k: v[k].numpy() for k in scene.STREAMS})
    assert np.array_equal(out["count"].cpu().numpy().astype(np.int64), fr.count)
    assert tab.stats()["device_error"] == 0
    tab.close()
