"""Seeded initial parameters of the pivot-proposer network (not in the paper).

The network scores candidate rows and columns of a Pi block: F inputs, two hidden layers of h
ReLU units, one logit. Its flat FP32 parameter vector is W1 (h x F), b1 (h), W2 (h x h), b2 (h),
W3 (h), b3 (1). Initial weights are uniform in +-sqrt(6 / fan_in) (He et al., 2015), biases zero.
"""

from __future__ import annotations

import numpy as np


def proposer_init(seed: int, F: int, h: int = 128) -> np.ndarray:
    rng = np.random.default_rng(seed)
    out = np.zeros(h * F + h + h * h + h + h + 1, dtype=np.float32)
    o = 0
    for fan_in, count in ((F, h * F), (None, h), (h, h * h), (None, h), (h, h), (None, 1)):
        if fan_in is not None:
            out[o:o + count] = rng.uniform(-1.0, 1.0, count) * np.sqrt(6.0 / fan_in)
        o += count
    return out
