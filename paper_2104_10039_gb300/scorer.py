"""Host-side helpers of the learned correction's scorer (a per-vertex MLP
8 -> 64 -> 64 -> 1, beyond the paper): the parameter layout, deterministic
initial parameters, and a training loop over traces that calls the
library's training kernel. Every arithmetic step on the data runs in the
library (gg_mlp_score, gg_mlp_train); this module only arranges arguments."""
from __future__ import annotations

import numpy as np

N_IN, N_H = 8, 64
# FP32 parameter vector: W1[64][8], b1[64], W2[64][64], b2[64], w3[64], b3
OFF_W1, OFF_B1, OFF_W2, OFF_B2, OFF_W3, OFF_B3 = 0, 512, 576, 4672, 4736, 4800
N_PARAM = 4801
FEATURES = ("sqrt(in-degree)/64", "sqrt(out-degree)/64", "change(t-1)", "change(t-2)", "change(t-3)",
            "active in-edge fraction", "iteration/64", "app id")


def init_params(seed: int = 0) -> np.ndarray:
    """Uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights from numpy's PCG64
    with the given seed; zero biases."""
    rng = np.random.default_rng(seed)
    P = np.zeros(N_PARAM, np.float32)
    P[OFF_W1:OFF_B1] = rng.uniform(-1, 1, 512) / np.sqrt(8.0)
    P[OFF_W2:OFF_B2] = rng.uniform(-1, 1, 4096) / 8.0
    P[OFF_W3:OFF_B3] = rng.uniform(-1, 1, 64) / 8.0
    return P


def coprime_stride(rows: int, hint: int = 2654435761) -> int:
    """A stride coprime to rows: minibatch sample j of the data is row
    (j * stride) mod rows, a fixed permutation of the rows."""
    import math
    if rows <= 1:
        return 1
    s = hint % rows
    while s == 0 or math.gcd(s, rows) != 1:
        s = (s + 1) % rows
    return s
