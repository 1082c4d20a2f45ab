"""GPU learned fallback against the MLP oracle (same BF16-rounded weights).

Every element of every result is held to a bound the oracle derives from its
own numbers (oracle/mlp_oracle.py: forward_bounds, backward_bounds,
adam_first_step_bounds): FP32 sums of exact BF16 products within (K + 1) 2^-23
of their absolute sums, FP32 bias additions within 2^-24, the encoder within
its stated error, and every BF16 rounding or ReLU mask that the GPU's
pre-rounding interval could push across a boundary allowed to land on either
side.  No GPU value enters a bound.  Two networks: random weights with biases
(the general case; the bounds widen where BF16 roundings straddle) and a
structured one whose hidden layers pass values through (the bounds shrink to
FP32 size, so layout, indexing, bias and rounding-point mistakes show).  And
a gain test: on low-count vertices the trained network beats the filter
alone against the noise-free field.
"""
import numpy as np
import pytest
import torch

from mlp_cases import random_weights, structured_weights
from oracle import mlp_oracle as M
from oracle import pps_oracle as O
from paper_1902_05942_gb300 import configs, pps, scene

pytestmark = pytest.mark.gpu

BOX = ((-100.0, -100.0, -100.0), (100.0, 100.0, 100.0))
WEIGHTS = {"random": random_weights, "structured": structured_weights,
           "structured_all": lambda s: structured_weights(s, "all")}


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1902_05942_gb300 import build
    build.build()
    torch.cuda.set_device(0)
    yield


def _verts(n, seed):
    rng = np.random.default_rng(seed)
    p = rng.uniform(-30, 30, (n, 3)).astype(np.float32)
    nn = rng.normal(size=(n, 3))
    nn = (nn / np.linalg.norm(nn, axis=1, keepdims=True)).astype(np.float32)
    rgb = rng.lognormal(-1, 1.0, (n, 3)).astype(np.float32)
    arrs = [p[:, 0], p[:, 1], p[:, 2], nn[:, 0], nn[:, 1], nn[:, 2], rgb[:, 0], rgb[:, 1], rgb[:, 2]]
    d = {k: torch.from_numpy(np.ascontiguousarray(a)).cuda() for k, a in zip(scene.STREAMS, arrs)}
    return d, p, nn, rgb


def _x(p, nn):
    return M.encode(p, nn, BOX[0], BOX[1])


def _within(got, ref, bound, what):
    err = np.abs(got - ref)
    bad = err > bound
    assert not bad.any(), (f"{what}: {bad.sum()} of {bad.size} elements outside their bounds; "
                           f"worst excess {np.max(err - bound):.3e}")


@pytest.mark.parametrize("kind", sorted(WEIGHTS))
def test_mlp_forward_matches_oracle(kind):
    w = WEIGHTS[kind](21)
    net = pps.MLP(pps.mlp_params(batch=256), init=w)
    d, p, nn, _ = _verts(1000, 1)
    out = net.forward(d)
    y = torch.stack([out[c] for c in "rgb"], 1).cpu().numpy().astype(np.float64)
    fb = M.forward_bounds(w.astype(np.float64), _x(p, nn), M.encoding_error())
    _within(y, fb.acts.y, fb.ey, f"forward ({kind})")
    net.close()


@pytest.mark.parametrize("kind", ["random", "structured"])
def test_mlp_gradient_matches_oracle(kind):
    """pps_mlp_gradient over a given sample list (three samples left out):
    every weight and bias gradient of every layer within its bound."""
    w = WEIGHTS[kind](22)
    net = pps.MLP(pps.mlp_params(batch=256), init=w)
    d, p, nn, rgb = _verts(300, 2)
    idx = np.arange(256, dtype=np.int32)
    idx[[3, 100, 255]] = -1  # left-out samples
    g = net.gradient(d, {c: d[c] for c in "rgb"}, torch.from_numpy(idx).cuda()).cpu().numpy()
    valid = (idx >= 0).astype(np.float64)
    sel = np.where(idx >= 0, idx, 0)
    w64 = w.astype(np.float64)
    fb = M.forward_bounds(w64, _x(p[sel], nn[sel]), M.encoding_error())
    ref, eg = M.backward_bounds(w64, fb, rgb[sel].astype(np.float64), valid, 256)
    _within(g.astype(np.float64), ref, eg, f"gradient ({kind})")
    net.close()


@pytest.mark.parametrize("kind", ["random", "structured"])
def test_mlp_training_step_matches_oracle(kind):
    """One pps_mlp_train step: the oracle's sample selection, gradient and
    first Adam step; all 13,699 FP32 master weights within their bounds."""
    w = WEIGHTS[kind](23)
    params = pps.mlp_params(batch=1024, steps=1, seed=99)
    net = pps.MLP(params, init=w)
    d, p, nn, rgb = _verts(5000, 3)
    count = np.random.default_rng(4).integers(1, 16, 5000).astype(np.int32)
    filt = {"r": d["r"], "g": d["g"], "b": d["b"], "count": torch.from_numpy(count).cuda()}
    net.train(d, filt, frame=5)
    got = net.get_weights().astype(np.float64)
    idx = M.select_samples(count, 99, 5, 0, 1024, 8)
    valid = (idx >= 0).astype(np.float64)
    sel = np.where(idx >= 0, idx, 0)
    w64 = w.astype(np.float64)
    fb = M.forward_bounds(w64, _x(p[sel], nn[sel]), M.encoding_error())
    g, eg = M.backward_bounds(w64, fb, rgb[sel].astype(np.float64), valid, 1024)
    ref, ew = M.adam_first_step_bounds(w64, g, eg)
    _within(got, ref, ew, f"Adam step ({kind})")
    net.close()


def test_mlp_training_step_with_several_tiles_per_cta():
    """A batch of 20,480 samples (160 tiles of 128) on a GPU with fewer
    multiprocessors: some CTAs of the training launch take two tiles.  All
    13,699 master weights after the first Adam step within their bounds."""
    w = WEIGHTS["random"](31)
    params = pps.mlp_params(batch=20480, steps=1, seed=7)
    net = pps.MLP(params, init=w)
    d, p, nn, rgb = _verts(60000, 8)
    count = np.random.default_rng(9).integers(1, 16, 60000).astype(np.int32)
    filt = {"r": d["r"], "g": d["g"], "b": d["b"], "count": torch.from_numpy(count).cuda()}
    net.train(d, filt, frame=2)
    got = net.get_weights().astype(np.float64)
    idx = M.select_samples(count, 7, 2, 0, 20480, 8)
    valid = (idx >= 0).astype(np.float64)
    sel = np.where(idx >= 0, idx, 0)
    w64 = w.astype(np.float64)
    fb = M.forward_bounds(w64, _x(p[sel], nn[sel]), M.encoding_error())
    g, eg = M.backward_bounds(w64, fb, rgb[sel].astype(np.float64), valid, 20480)
    ref, ew = M.adam_first_step_bounds(w64, g, eg)
    _within(got, ref, ew, "Adam step, several tiles per CTA")
    net.close()


def test_mlp_training_steps_across_launches():
    """Ten Adam steps per call run as two cooperative launches (at most eight
    steps each); three calls in a row.  The grid barriers' arrival counts
    carry over between launches: a wrong count would leave a barrier waiting
    until its time limit and raise the device error word, which get_weights
    reports.  The weights stay finite and move."""
    w = WEIGHTS["random"](33)
    net = pps.MLP(pps.mlp_params(batch=2048, steps=10, seed=3), init=w)
    d, _, _, _ = _verts(8000, 10)
    count = np.random.default_rng(11).integers(1, 16, 8000).astype(np.int32)
    filt = {"r": d["r"], "g": d["g"], "b": d["b"], "count": torch.from_numpy(count).cuda()}
    for f in range(3):
        net.train(d, filt, frame=f)
    got = net.get_weights()  # raises on a device error
    assert np.all(np.isfinite(got))
    assert np.abs(got - w).max() > 1e-3
    net.close()


def test_mlp_infer_replaces_only_low_count_vertices():
    w = M.he_init(24).astype(np.float32)
    net = pps.MLP(pps.mlp_params(batch=256, infer_max_count=4), init=w)
    d, _, _, rgb = _verts(3001, 5)
    rng = np.random.default_rng(6)
    count = rng.integers(0, 10, 3001).astype(np.int32)
    status = np.where(count < 4, 1, 0).astype(np.uint8)
    status[rng.choice(3001, 40, replace=False)] = 2  # overflowed vertices keep their value
    out = {"r": d["r"].clone(), "g": d["g"].clone(), "b": d["b"].clone(),
           "count": torch.from_numpy(count).cuda(), "status": torch.from_numpy(status).cuda()}
    net.infer(d, out)
    pred = net.forward(d)
    st = out["status"].cpu().numpy()
    hit = (count < 4) & (status != 2)
    assert np.array_equal(st[hit], np.full(hit.sum(), 3))
    assert np.array_equal(st[~hit], status[~hit])
    for c in "rgb":
        o = out[c].cpu().numpy()
        assert np.array_equal(o[hit], pred[c].cpu().numpy()[hit])
        assert np.array_equal(o[~hit], d[c].cpu().numpy()[~hit])
    net.close()


def test_trained_fallback_gains_over_filter_alone():
    """Radiance = smooth field x lognormal noise (with fireflies).  After
    online training over 12 frames (4 steps x 16,384 samples each, count >= 8),
    the network's answers for low-count vertices (count < 4) are closer to the
    noise-free field than the filter's own averages there."""
    w = configs.small()
    cfg = w.filters[0]
    net = pps.MLP(pps.mlp_params())
    tab = pps.Table(cfg)
    gain = None
    for f in range(12):
        spec = configs.frame_spec(w, 0, 0)
        spec.view = scene.View(480, 360, eye=(0.0, 3.0, -12.0), target=(0.0, 0.5, 0.0))
        cfg.pixel_angle = spec.view.pixel_angle()
        spec.bounces = 2
        spec.radiance = "field"
        v = scene.trace_stream(spec, f, "cuda")
        d = {k: v[k] for k in scene.STREAMS}
        out = tab.filter(d, spec.view.eye, f)
        net.train(d, out, f)
        filt = torch.stack([out[c] for c in "rgb"], 1).clone()
        net.infer(d, out)
        if f == 11:
            truth = torch.stack([v["truth_r"], v["truth_g"], v["truth_b"]], 1)
            low = out["status"] == pps.STATUS_MLP
            mlp = torch.stack([out[c] for c in "rgb"], 1)
            e_f = torch.sqrt(((filt[low] - truth[low]) ** 2).mean()).item()
            e_m = torch.sqrt(((mlp[low] - truth[low]) ** 2).mean()).item()
            gain = (e_f, e_m, int(low.sum().item()))
    e_f, e_m, nlow = gain
    print(f"low-count vertices {nlow}: RMSE filter {e_f:.4f}, filter + MLP {e_m:.4f}")
    assert nlow > 1000
    assert e_m < 0.8 * e_f
    tab.close()
    net.close()
