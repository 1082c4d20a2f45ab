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


# ----------------------------------------------------------------------------
# Per-element error bounds of an FP32 / BF16 implementation against this
# oracle.
#
# A GPU evaluates the same network with the same BF16 weights, but sums its
# products in FP32 (in some order) and computes the encoding in FP32.  Its
# values therefore differ from the oracle's in two ways: (1) FP32 rounding of
# sums, bias additions and the encoding -- small, and bounded by the absolute
# values the oracle itself computes; (2) a BF16 rounding (or a ReLU mask) that
# falls the other way when the GPU's pre-rounding value and the oracle's lie
# on two sides of a rounding boundary.  Rounding is monotone, so when the
# GPU's pre-rounding value lies within e of the oracle's value a, its rounded
# value lies in [rnd(a - e), rnd(a + e)]: the bound on the rounded value is the
# distance from rnd(a) to the far end of that interval -- zero where the whole
# interval rounds to one BF16 number (the usual case), one BF16 step where it
# straddles a boundary.  Propagating these intervals layer by layer gives a
# bound for every element of every result, from the oracle's own numbers only.
#
# FP32 sums: K products summed in any order, each of the K - 1 additions off
# by less than one FP32 unit in the last place of its partial sum (2^-23 of it,
# whatever the rounding mode, truncation included) and every partial sum at
# most sum|products|, are within (K - 1) 2^-23 sum|products| of the exact sum
# (the products of two BF16 numbers are exact in FP32); the bounds below take
# (K + 1) 2^-23.  An FP32 addition of two numbers (a bias) is within 2^-24 of
# its exact value, relatively (round to nearest).
# ----------------------------------------------------------------------------
F32_EPS = 2.0 ** -24


def _sum_err(k: int) -> float:
    return (k + 1) * 2.0 ** -23


def rounding_bound(a: np.ndarray, e: np.ndarray, lo=None, hi=None) -> np.ndarray:
    """Largest |rnd(g) - rnd(a)| over GPU pre-rounding values g in [lo, hi]
    (default [a - e, a + e]), rnd = round to BF16."""
    lo = a - e if lo is None else lo
    hi = a + e if hi is None else hi
    r = bf16_round(a)
    return np.maximum(np.abs(bf16_round(hi) - r), np.abs(bf16_round(lo) - r))


def encoding_error(double_angle_steps: int = 3) -> np.ndarray:
    """Per input column, a bound on |GPU encoded value before BF16 rounding -
    oracle's value| for an encoder that evaluates sin/cos(pi 2^k p) of the
    FP32-normalized position with one library sincospi per group of
    frequencies and up to `double_angle_steps` double-angle steps after it
    (s' = 2 s c, c' = (c - s)(c + s)).  A library sincospi is taken within
    2^-23 (absolute) of the exact value; each step multiplies the error by at
    most 2 sqrt(2) (the partial derivatives of 2sc and c^2 - s^2 sum to
    2(|s| + |c|) <= 2 sqrt 2) and adds four roundings of values below 2 in
    magnitude (2^-23 each); the result is doubled for margin.  The normal
    columns and the padding are exact (0)."""
    e = np.zeros(IN)
    for a in range(3):
        for k in range(FREQS):
            q = min(k % 4, double_angle_steps)
            err = 2.0 ** -23
            for _ in range(q):
                err = 2.0 * np.sqrt(2.0) * err + 4 * 2.0 ** -23
            e[a * 2 * FREQS + 2 * k] = e[a * 2 * FREQS + 2 * k + 1] = 2.0 * err
    return e


@dataclass
class ActBounds:
    acts: Acts
    ex: List[np.ndarray]  # bound on |GPU - oracle| of each layer's input (as rounded)
    ez: List[np.ndarray]  # bound on each layer's FP32 pre-activation z (bias included)
    ey: np.ndarray        # bound on the output


def forward_bounds(flat: np.ndarray, X: np.ndarray, enc_err: np.ndarray) -> ActBounds:
    """The BF16 forward pass with a per-element bound on every quantity.
    `X` is the oracle's (unrounded) encoding, `enc_err` the bound per column
    on the GPU's encoding before its BF16 rounding (encoding_error)."""
    acts = forward(flat, X)
    layers = unpack(np.asarray(flat, dtype=np.float64))
    ex = rounding_bound(X, np.broadcast_to(enc_err, X.shape))
    exs, ezs = [], []
    ey = None
    for li, (W, _) in enumerate(layers):
        h = acts.x[li]
        aW = np.abs(bf16_round(W)).T
        z = acts.z[li]
        spread = ex @ aW
        absum = (np.abs(h) + ex) @ aW
        ez = spread + _sum_err(W.shape[1]) * absum
        ez = ez + F32_EPS * (np.abs(z) + ez)  # + bias in FP32
        exs.append(ex)
        ezs.append(ez)
        if li < len(layers) - 1:
            ex = rounding_bound(np.maximum(z, 0.0), None, lo=np.maximum(z - ez, 0.0),
                                hi=np.maximum(z + ez, 0.0))
        else:
            ey = ez
    return ActBounds(acts, exs, ezs, ey)


def backward_bounds(flat: np.ndarray, fb: ActBounds, T: np.ndarray, valid: np.ndarray,
                    batch: int) -> Tuple[np.ndarray, np.ndarray]:
    """The gradient (flat) and a per-element bound on |GPU - oracle| for an
    implementation that forms the output delta as rnd((fl32(y + b) - t) / B)
    (FP32 steps, B a power of two), sums each product over the batch in FP32,
    and rounds the deltas to BF16 after the ReLU mask of the BF16 activation.
    A mask is ambiguous where the activation's interval reaches zero: there
    the GPU's delta may be 0 or the product."""
    acts = fb.acts
    layers = unpack(np.asarray(flat, dtype=np.float64))
    _, g = backward(flat, acts, T, valid, batch)
    v = valid[:, None]
    diff = (acts.y - T) * v
    pre = diff / batch
    e_pre = (fb.ey + 2 * F32_EPS * (np.abs(acts.y) + np.abs(diff) + fb.ey)) * v / batch
    d = bf16_round(pre)
    ed = rounding_bound(pre, e_pre)
    bounds = [None] * len(layers)
    nb = batch + 64  # one MMA over the CTA's samples, then FP32 adds across CTAs
    for li in range(len(layers) - 1, -1, -1):
        W, _ = layers[li]
        x, exl = acts.x[li], fb.ex[li]
        ad, ax = np.abs(d) + ed, np.abs(x) + exl
        egW = np.abs(d).T @ exl + ed.T @ ax + _sum_err(nb) * (ad.T @ ax)
        egb = ed.sum(axis=0) + _sum_err(nb) * ad.sum(axis=0)
        bounds[li] = (egW, egb)
        if li > 0:
            aW = np.abs(bf16_round(W))
            dh = d @ bf16_round(W)
            edh = ed @ aW + _sum_err(W.shape[0]) * (ad @ aW)
            on = x > 0
            sure = x - exl > 0       # the GPU's activation is positive too
            amb = on != sure          # 0 < x <= its bound
            amb |= (~on) & (exl > 0)  # x = 0 but the GPU's may be positive
            m = dh * on
            lo = np.where(sure, dh - edh, np.where(amb, np.minimum(0.0, dh - edh), 0.0))
            hi = np.where(sure, dh + edh, np.where(amb, np.maximum(0.0, dh + edh), 0.0))
            ed = rounding_bound(m, None, lo=lo, hi=hi)
            d = bf16_round(m)
    return g, pack(bounds)


def adam_first_step_bounds(flat: np.ndarray, grad: np.ndarray, egrad: np.ndarray,
                           lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8) -> Tuple[np.ndarray, np.ndarray]:
    """The first Adam step from zero moments, w - lr g / (|g| + eps), and a
    per-element bound on |GPU - oracle| for an FP32 implementation whose
    gradient is within `egrad` of `grad`.  g / (|g| + eps) increases with g,
    so the GPU's step lies between its values at g - egrad and g + egrad; the
    FP32 evaluation of the moments, bias corrections, square root and division
    (about a dozen roundings, and fl32 of lr, beta1, beta2) moves the step by
    at most 32 2^-24 of itself; the final FP32 subtraction rounds once."""
    w_new, _, _ = adam(flat, grad, np.zeros_like(flat), np.zeros_like(flat), 1, lr, beta1,
                       beta2, eps)
    f = lambda g: g / (np.abs(g) + eps)
    step = lr * f(grad)
    span = lr * np.maximum(np.abs(f(grad + egrad) - f(grad)), np.abs(f(grad - egrad) - f(grad)))
    e = span + 32 * F32_EPS * (np.abs(step) + span) + F32_EPS * (np.abs(w_new) + lr)
    return w_new, e
