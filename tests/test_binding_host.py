"""The Python binding's argument checks (no GPU): every array passed to the
library must be a contiguous tensor of the right type, long enough, and on
the right side of the bus; the binding refuses anything else before calling
the library."""
import pytest
import torch

from paper_1902_05942_gb300 import pps


def _streams(n, dtype=torch.float32):
    return {k: torch.zeros(n, dtype=dtype) for k in pps.STREAM_NAMES}


def test_host_vertices_are_marshalled_for_host_calls():
    v = _streams(10)
    pv = pps.make_vertices(v, 10, device=False)
    assert pv.px == v["px"].data_ptr() and pv.b == v["b"].data_ptr()
    assert not pv.dist and not pv.extra


def test_device_calls_refuse_host_tensors():
    with pytest.raises(ValueError, match="CUDA"):
        pps.make_vertices(_streams(10), 10, device=True)


@pytest.mark.parametrize("bad", ["dtype", "short", "strided"])
def test_wrong_arrays_are_refused(bad):
    v = _streams(10)
    if bad == "dtype":
        v["pz"] = torch.zeros(10, dtype=torch.float64)
    elif bad == "short":
        v["nx"] = torch.zeros(9)
    else:
        v["r"] = torch.zeros(20)[::2]
    with pytest.raises(ValueError):
        pps.make_vertices(v, 10, device=False)


def test_optional_key_variant_arrays_are_checked_too():
    v = _streams(10)
    v["extra"] = torch.zeros(10, dtype=torch.float32)  # must be int32
    with pytest.raises(ValueError, match="extra"):
        pps.make_vertices(v, 10, device=False)
    v["extra"] = torch.zeros(10, dtype=torch.int32)
    v["dist"] = torch.ones(10)
    pv = pps.make_vertices(v, 10, device=False)
    assert pv.dist == v["dist"].data_ptr() and pv.extra == v["extra"].data_ptr()
