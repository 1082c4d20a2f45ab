"""Seeded weights for the learned-fallback tests (inputs only: no arithmetic
of the network lives here).

random_weights: He-normal weights with small random biases, the general case.
structured_weights: a network whose hidden layers pass values through
unchanged, so that an FP32 / BF16 implementation must reproduce the oracle
almost exactly: every row of layer 1 copies one input column scaled by a
power of two (no bias: a dyadic bias would put many sums exactly halfway
between two BF16 numbers); layers 2 and 3 are identities with zero biases (one
exact product per output, and x >= 0 after the ReLU, so x passes unchanged);
layer 4 is random, with a bias.  Every product there is exact and the only
roundings left are the encoding's, the output layer's FP32 sum and its bias
addition.  `columns` = "direct" copies only the encoded columns an encoder
computes with one library sincospi each (frequencies k = 0, 4, 8, whose error
is a single FP32 rounding) and the three normal columns; "all" picks among all
75 non-zero columns, double-angle ones included."""
import numpy as np

from oracle import mlp_oracle as M


def random_weights(seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    layers = [(rng.normal(0.0, np.sqrt(2.0 / fi), (fo, fi)), rng.normal(0.0, 0.1, fo))
              for fi, fo in M.LAYERS]
    return M.pack(layers).astype(np.float32)


def structured_weights(seed: int, columns: str = "direct") -> np.ndarray:
    rng = np.random.default_rng(seed)
    if columns == "direct":
        pool = [a * 24 + 2 * k + c for a in range(3) for k in (0, 4, 8) for c in (0, 1)]
    else:
        pool = list(range(72))
    pool = np.array(pool + [72, 73, 74])
    if pool.size >= 64:
        cols = np.concatenate([[72, 73, 74], rng.choice(pool[:72], 61, replace=False)])
    else:
        cols = np.concatenate([pool, rng.choice(pool, 64 - pool.size)])
    rng.shuffle(cols)
    W1 = np.zeros((64, 80))
    W1[np.arange(64), cols] = rng.choice([-2.0, -1.0, -0.5, 0.5, 1.0, 2.0], 64)
    b1 = np.zeros(64)
    eye = np.eye(64)
    W4 = rng.normal(0.0, np.sqrt(2.0 / 64), (3, 64))
    b4 = rng.normal(0.0, 0.1, 3)
    return M.pack([(W1, b1), (eye, np.zeros(64)), (eye, np.zeros(64)), (W4, b4)]).astype(np.float32)
