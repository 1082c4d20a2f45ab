"""Pins of the MLP oracle (no GPU): library BF16 rounding, libm encoding,
finite differences, the Adam closed form, a library network, sample selection."""
import math

import numpy as np
import pytest
import torch

from oracle import mlp_oracle as M


def test_parameter_layout():
    assert M.param_count() == 80 * 64 + 64 + 2 * (64 * 64 + 64) + 64 * 3 + 3 == 13699
    flat = np.arange(M.param_count(), dtype=np.float64)
    assert np.array_equal(M.pack(M.unpack(flat)), flat)


def test_bf16_round_matches_torch():
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.normal(0, 10, 20000), rng.normal(0, 1e-3, 2000),
                        # exact ties between two bfloat16 values
                        np.array([1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -(1.0 + 2 ** -8), 0.0, -0.0])])
    x = x.astype(np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(M.bf16_round(x), ref)


def test_encoding_matches_libm():
    pos = np.array([[0.3, -1.7, 12.5], [-20.0, 20.0, 0.0]], dtype=np.float32)
    nrm = np.array([[0.0, 1.0, 0.0], [0.6, 0.0, -0.8]], dtype=np.float32)
    lo, hi = (-20.0, -20.0, -20.0), (20.0, 20.0, 20.0)
    X = M.encode(pos, nrm, lo, hi)
    assert X.shape == (2, 80)
    for r in range(2):
        for a in range(3):
            # the normalized coordinate is an FP32 computation: (x - lo) * (1 / (hi - lo))
            inv = np.float32(np.float32(1.0) / np.float32(40.0))
            p = float(np.float32(np.float32(pos[r, a] - np.float32(-20.0)) * inv))
            p = min(max(p, 0.0), 1.0)
            for k in range(12):
                assert abs(X[r, a * 24 + 2 * k] - math.sin(math.pi * 2 ** k * p)) < 1e-9
                assert abs(X[r, a * 24 + 2 * k + 1] - math.cos(math.pi * 2 ** k * p)) < 1e-9
        assert np.array_equal(X[r, 72:75], nrm[r].astype(np.float64))
        assert not X[r, 75:].any()


def test_forward_matches_library_network():
    flat = M.he_init(3)
    rng = np.random.default_rng(4)
    X = rng.normal(size=(17, 80))
    net = torch.nn.Sequential(torch.nn.Linear(80, 64), torch.nn.ReLU(), torch.nn.Linear(64, 64),
                              torch.nn.ReLU(), torch.nn.Linear(64, 64), torch.nn.ReLU(),
                              torch.nn.Linear(64, 3)).double()
    with torch.no_grad():
        for lin, (W, b) in zip([net[0], net[2], net[4], net[6]], M.unpack(flat)):
            lin.weight.copy_(torch.from_numpy(W))
            lin.bias.copy_(torch.from_numpy(b))
        ref = net(torch.from_numpy(X)).numpy()
    assert np.allclose(M.forward(flat, X, bf16=False).y, ref, rtol=1e-12, atol=1e-12)


def test_backward_matches_finite_differences():
    flat = M.he_init(5)
    rng = np.random.default_rng(6)
    B = 8
    X = rng.normal(size=(B, 80))
    T = rng.normal(size=(B, 3))
    valid = np.array([1, 1, 0, 1, 1, 1, 0, 1], dtype=np.float64)

    def loss(p):
        return M.backward(p, M.forward(p, X, bf16=False), T, valid, B, bf16=False)[0]

    _, g = M.backward(flat, M.forward(flat, X, bf16=False), T, valid, B, bf16=False)
    idx = rng.choice(flat.size, 60, replace=False)
    idx = np.concatenate([idx, [M.param_count() - 1, 80 * 64 + 3]])  # an output and a layer-1 bias
    h = 1e-6
    for i in idx:
        e = np.zeros_like(flat)
        e[i] = h
        fd = (loss(flat + e) - loss(flat - e)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])), (i, fd, g[i])


def test_adam_closed_form():
    rng = np.random.default_rng(7)
    th = rng.normal(size=50)
    g = rng.normal(size=50)
    lr, b1, b2, eps = 1e-3, 0.9, 0.999, 1e-8
    th1, m, v = M.adam(th, g, np.zeros(50), np.zeros(50), 1, lr, b1, b2, eps)
    # first step: bias-corrected moments are g and g^2
    assert np.allclose(th1, th - lr * g / (np.abs(g) + eps), rtol=0, atol=1e-15)
    g2 = rng.normal(size=50)
    th2, _, _ = M.adam(th1, g2, m, v, 2, lr, b1, b2, eps)
    mh = (b1 * (1 - b1) * g + (1 - b1) * g2) / (1 - b1 ** 2)
    vh = (b2 * (1 - b2) * g ** 2 + (1 - b2) * g2 ** 2) / (1 - b2 ** 2)
    assert np.allclose(th2, th1 - lr * mh / (np.sqrt(vh) + eps), rtol=0, atol=1e-15)


def test_sample_selection_picks_eligible_vertices_uniformly():
    rng = np.random.default_rng(8)
    count = rng.integers(1, 20, 5000)
    idx = M.select_samples(count, 11, 3, 1, 20000, 8)
    ok = idx >= 0
    assert ok.mean() > 0.999
    assert np.all(count[idx[ok]] >= 8)
    elig = np.nonzero(count >= 8)[0]
    h = np.bincount(idx[ok], minlength=5000)[elig]
    e = ok.sum() / elig.size
    assert ((h - e) ** 2 / e).sum() < elig.size + 6 * np.sqrt(2 * elig.size)  # chi-square
    assert np.array_equal(idx, M.select_samples(count, 11, 3, 1, 20000, 8))
    assert not np.array_equal(idx, M.select_samples(count, 11, 3, 2, 20000, 8))


# ----------------------------------------------------------------------------
# The per-element error bounds (forward_bounds, backward_bounds,
# adam_first_step_bounds) against an independent FP32 evaluation of the same
# network: products of BF16 numbers summed in FP32 in random orders, FP32 bias
# additions, the encoding perturbed within its stated error before its BF16
# rounding.  Every such evaluation must land inside the bounds, element by
# element; planted mistakes must fall outside somewhere.
# ----------------------------------------------------------------------------
from mlp_cases import random_weights, structured_weights  # noqa: E402

F = np.float32


def _f32_sum(P, axis, rng):
    """Sum float32 products along `axis` in a random order, rounding to FP32
    after every addition."""
    P = np.moveaxis(P, axis, -1)
    P = P[..., rng.permutation(P.shape[-1])]
    return np.cumsum(P, axis=-1, dtype=F)[..., -1]


def _bf(x):
    return M.bf16_round(np.asarray(x, dtype=F)).astype(F)


def _emu_forward(flat, X, enc_err, rng, skip_bias=None, shift_col=False):
    layers = M.unpack(np.asarray(flat, dtype=np.float64))
    g = (X + rng.uniform(-1.0, 1.0, X.shape) * enc_err * 0.999).astype(F)
    h = _bf(g)
    xs = []
    y = None
    for li, (W, b) in enumerate(layers):
        xs.append(h)
        Wb = _bf(W)
        if shift_col and li == 0:
            Wb = np.roll(Wb, 1, axis=1)
        s = _f32_sum(h[:, None, :] * Wb[None, :, :], 2, rng)
        z = s if skip_bias == li else (s + F(b)).astype(F)
        if li < len(layers) - 1:
            h = _bf(np.maximum(z, F(0)))
        else:
            y = z
    return xs, y


def _emu_backward(flat, xs, y, T, valid, batch, rng, drop=None, flip=False):
    layers = M.unpack(np.asarray(flat, dtype=np.float64))
    diff = ((y - T.astype(F)).astype(F) * valid[:, None].astype(F)).astype(F)
    d = _bf((diff * F(1.0 / batch)).astype(F))
    if flip:
        d = -d
    if drop is not None:
        d = d.copy()
        d[drop] = 0
    grads = [None] * len(layers)
    for li in range(len(layers) - 1, -1, -1):
        W, _ = layers[li]
        x = xs[li]
        gW = _f32_sum(d[:, :, None] * x[:, None, :], 0, rng)
        gb = _f32_sum(d, 0, rng)
        grads[li] = (gW.astype(np.float64), gb.astype(np.float64))
        if li > 0:
            dh = _f32_sum(d[:, :, None] * _bf(W)[None, :, :], 1, rng)
            d = _bf(np.where(x > 0, dh, F(0)))
    return M.pack(grads)


def _emu_adam(flat, g, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    g = g.astype(F)
    m = (F(1 - b1) * g).astype(F)
    v = ((F(1 - b2) * g).astype(F) * g).astype(F)
    step = (F(lr) * ((m / F(1 - b1)).astype(F) / (np.sqrt((v / F(1 - b2)).astype(F)) + F(eps))
                     .astype(F)).astype(F)).astype(F)
    return (np.asarray(flat, F) - step).astype(np.float64)


def _case(n, seed):
    rng = np.random.default_rng(seed)
    p = rng.uniform(-30, 30, (n, 3)).astype(np.float32)
    nn = rng.normal(size=(n, 3))
    nn = (nn / np.linalg.norm(nn, axis=1, keepdims=True)).astype(np.float32)
    t = rng.lognormal(-1, 1.0, (n, 3))
    return M.encode(p, nn, (-100.0,) * 3, (100.0,) * 3), t


def _structured_all(seed):
    return structured_weights(seed, "all")


@pytest.mark.parametrize("weights", [random_weights, structured_weights, _structured_all])
@pytest.mark.parametrize("seed", [1, 2])
def test_bounds_hold_for_fp32_evaluations_in_random_orders(weights, seed):
    w = weights(10 + seed).astype(np.float64)
    X, T = _case(256, seed)
    valid = np.ones(256)
    valid[[3, 100, 255]] = 0
    enc = M.encoding_error()
    fb = M.forward_bounds(w, X, enc)
    g, eg = M.backward_bounds(w, fb, T, valid, 256)
    w1, ew = M.adam_first_step_bounds(w, g, eg)
    for trial in range(3):
        rng = np.random.default_rng(100 * seed + trial)
        xs, y = _emu_forward(w, X, enc, rng)
        assert np.all(np.abs(y - fb.acts.y) <= fb.ey)
        ge = _emu_backward(w, xs, y, T, valid, 256, rng)
        assert np.all(np.abs(ge - g) <= eg)
        assert np.all(np.abs(_emu_adam(w, ge) - w1) <= ew)


def test_structured_network_bounds_are_tight():
    """With pass-through hidden layers the bounds shrink to FP32 size almost
    everywhere: the output within 1e-4 of its scale, weight gradients within
    1e-3 of their magnitude (a sum over 256 samples), and the first Adam step
    (about lr times the gradient's sign) certain for almost every weight."""
    w = structured_weights(3).astype(np.float64)
    X, T = _case(256, 3)
    valid = np.ones(256)
    fb = M.forward_bounds(w, X, M.encoding_error())
    scale = np.sqrt((fb.acts.y ** 2).mean())
    assert np.median(fb.ey) <= 1e-4 * scale
    g, eg = M.backward_bounds(w, fb, T, valid, 256)
    nz = np.abs(g) > 1e-6
    assert np.median(eg[nz] / np.abs(g[nz])) <= 1e-3
    _, ew = M.adam_first_step_bounds(w, g, eg)
    assert np.mean(ew < 1e-5) > 0.95


def test_bounds_catch_planted_mistakes():
    """An FP32 evaluation with a mistake in it -- a sample left out of the
    gradient, a bias not added, the first layer reading the next input
    column, the output delta's sign flipped -- leaves the bounds somewhere."""
    w = structured_weights(4).astype(np.float64)
    X, T = _case(256, 4)
    valid = np.ones(256)
    enc = M.encoding_error()
    fb = M.forward_bounds(w, X, enc)
    g, eg = M.backward_bounds(w, fb, T, valid, 256)
    rng = np.random.default_rng(5)
    xs, y = _emu_forward(w, X, enc, rng, skip_bias=3)
    assert np.any(np.abs(y - fb.acts.y) > fb.ey)
    xs, y = _emu_forward(w, X, enc, rng, shift_col=True)
    assert np.any(np.abs(y - fb.acts.y) > fb.ey)
    xs, y = _emu_forward(w, X, enc, rng)
    for kw in (dict(drop=17), dict(flip=True)):
        ge = _emu_backward(w, xs, y, T, valid, 256, rng, **kw)
        assert np.any(np.abs(ge - g) > eg), kw
    # the random network catches them too
    w = random_weights(6).astype(np.float64)
    fb = M.forward_bounds(w, X, enc)
    g, eg = M.backward_bounds(w, fb, T, valid, 256)
    xs, y = _emu_forward(w, X, enc, rng)
    ge = _emu_backward(w, xs, y, T, valid, 256, rng, drop=17)
    assert np.any(np.abs(ge - g) > eg)
    for li in (0, 3):
        xs, y = _emu_forward(w, X, enc, rng, skip_bias=li)
        assert np.any(np.abs(y - fb.acts.y) > fb.ey), li
