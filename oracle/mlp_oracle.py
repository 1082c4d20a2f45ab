"""CPU oracle of the learned fallback (test infrastructure only).

TEST INFRASTRUCTURE ONLY: imported by the tests and the benchmark's CPU
baseline, never by the CUDA library.  Written from the definition of the
network, independently of the GPU kernels.

The network (a fallback for cells with too few vertices, Sec. 3.3 motivates
such fallbacks; the network itself is the workload's addition to the method):

* input: the vertex position normalized to a box, p in [0, 1]^3, encoded per
  axis a and frequency k = 0..11 as (sin(pi 2^k p_a), cos(pi 2^k p_a)) -- 72
  values -- followed by the unit normal (3) and 5 zeros: 80 columns;
* three hidden layers of 64 with ReLU, a linear RGB output layer;
* BF16 weights and activations with FP32 accumulation: the encoded input and
  every hidden activation is rounded to BF16 (round to nearest even) before it
  enters the next product, and the weights used in products are the BF16
  copies of FP32 master weights; biases stay FP32;
* loss L = 1/(2B) sum_samples sum_channels (y - t)^2 over a batch of B
  samples (invalid samples contribute nothing), so dL/dy = (y - t) / B;
* backward: the output delta and every hidden delta are rounded to BF16
  before they enter products; ReLU passes the delta where the activation is
  positive; weight gradients are sums over the batch, bias gradients the
  column sums of the (rounded) deltas;
* Adam (Kingma & Ba 2015) on the FP32 master weights.

With `bf16=False` every rounding is skipped, which gives the plain FP64
network used to pin the backward pass with finite differences.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Dict, List, Tuple

import numpy as np

FREQS = 12
IN = 80  # 72 encoded position values, 3 normal values, 5 zero columns
HID = 64
OUT = 3
LAYERS = [(IN, HID), (HID, HID), (HID, HID), (HID, OUT)]


def param_count() -> int:
    return sum(i * o + o for i, o in LAYERS)


def unpack(flat: np.ndarray) -> List[Tuple[np.ndarray, np.ndarray]]:
    """Flat parameter vector -> [(W (out, in), b (out,)), ...] per layer."""
    out, o = [], 0
    for fi, fo in LAYERS:
        W = flat[o:o + fi * fo].reshape(fo, fi)
        o += fi * fo
        b = flat[o:o + fo]
        o += fo
        out.append((W, b))
    return out


def pack(layers) -> np.ndarray:
    return np.concatenate([np.concatenate([W.reshape(-1), b]) for W, b in layers])


def bf16_round(x: np.ndarray) -> np.ndarray:
    """Round to the nearest bfloat16 (ties to even), through float32."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def encode(pos: np.ndarray, nrm: np.ndarray, box_min, box_max) -> np.ndarray:
    """(N, 80) input rows: per axis, sin/cos of pi 2^k p for k = 0..11, then n."""
    pos = np.asarray(pos, dtype=np.float32)
    lo = np.asarray(box_min, dtype=np.float32)
    inv = (np.float32(1.0) / (np.asarray(box_max, dtype=np.float32) - lo)).astype(np.float32)
    p = np.clip((pos - lo) * inv, np.float32(0.0), np.float32(1.0)).astype(np.float64)
    N = p.shape[0]
    X = np.zeros((N, IN))
    for a in range(3):
        for k in range(FREQS):
            ang = np.pi * (2.0 ** k) * p[:, a]
            X[:, a * 2 * FREQS + 2 * k] = np.sin(ang)
            X[:, a * 2 * FREQS + 2 * k + 1] = np.cos(ang)
    X[:, 72:75] = np.asarray(nrm, dtype=np.float32)
    return X


@dataclass
class Acts:
    x: List[np.ndarray]  # inputs of each layer (as used in the products)
    z: List[np.ndarray]  # pre-activations of each layer
    y: np.ndarray


def forward(flat: np.ndarray, X: np.ndarray, bf16: bool = True) -> Acts:
    rnd = bf16_round if bf16 else (lambda a: a)
    layers = unpack(np.asarray(flat, dtype=np.float64))
    h = rnd(X)
    xs, zs = [], []
    for li, (W, b) in enumerate(layers):
        xs.append(h)
        z = h @ rnd(W).T + b
        zs.append(z)
        h = rnd(np.maximum(z, 0.0)) if li < len(layers) - 1 else z
    return Acts(xs, zs, h)


def backward(flat: np.ndarray, acts: Acts, T: np.ndarray, valid: np.ndarray, batch: int,
             bf16: bool = True) -> Tuple[float, np.ndarray]:
    """Loss and its gradient (flat, same layout as the parameters)."""
    rnd = bf16_round if bf16 else (lambda a: a)
    layers = unpack(np.asarray(flat, dtype=np.float64))
    diff = (acts.y - T) * valid[:, None]
    loss = 0.5 * float((diff ** 2).sum()) / batch
    d = rnd(diff / batch)
    grads = [None] * len(layers)
    for li in range(len(layers) - 1, -1, -1):
        W, _ = layers[li]
        x = acts.x[li]
        gW = d.T @ x
        gb = d.sum(axis=0)
        grads[li] = (gW, gb)
        if li > 0:
            dh = d @ rnd(W)
            d = rnd(dh * (acts.x[li] > 0))
    return loss, pack(grads)


def adam(flat, grad, m, v, step, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015), step counted from 1."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mh = m / (1.0 - beta1 ** step)
    vh = v / (1.0 - beta2 ** step)
    return flat - lr * mh / (np.sqrt(vh) + eps), m, v


def he_init(seed: int) -> np.ndarray:
    """He (Kaiming) normal initialisation, zero biases."""
    rng = np.random.default_rng(seed)
    return pack([(rng.normal(0.0, np.sqrt(2.0 / fi), (fo, fi)), np.zeros(fo)) for fi, fo in LAYERS])


def select_samples(count: np.ndarray, seed: int, frame: int, step: int, batch: int,
                   min_count: int, tries: int = 16):
    """Training samples: for sample i, the first of `tries` candidate vertices
    (Philox4x32-10, key (seed, frame), counter (i, step, try, 0); index =
    high 32 bits of x0 * n) whose cell count is >= min_count; -1 if none."""
    from .pps_oracle import philox4x32_10
    n = count.shape[0]
    idx = np.full(batch, -1, dtype=np.int64)
    i = np.arange(batch, dtype=np.uint32)
    for t in range(tries):
        x0, _, _, _ = philox4x32_10(i, np.full_like(i, step), np.full_like(i, t), 0,
                                    np.full_like(i, seed), np.full_like(i, frame))
        cand = ((x0.astype(np.uint64) * np.uint64(n)) >> np.uint64(32)).astype(np.int64)
        ok = (idx < 0) & (count[cand] >= min_count)
        idx[ok] = cand[ok]
    return idx
