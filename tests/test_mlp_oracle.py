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
