"""Seeded initial weights of the learned correction's network (3 x 3 x 3 convolutions,
1 -> 16 -> 16 -> 1 channels, no biases), flat in layer order with each layer laid out
[tap][out][in]: He-normal for the two ReLU layers, a ten times smaller normal for the
output layer so that the untrained stage starts close to the plain V-cycle."""
from __future__ import annotations

import numpy as np

LAYERS = ((1, 16), (16, 16), (16, 1))


def initial_weights(seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    out = []
    for l, (ci, co) in enumerate(LAYERS):
        std = np.sqrt(2.0 / (27 * ci)) if l < 2 else 0.1 * np.sqrt(1.0 / (27 * ci))
        out.append(rng.normal(0.0, std, 27 * co * ci))
    return np.concatenate(out).astype(np.float32).astype(np.float64)


def random_error(n: int, seed: int) -> np.ndarray:
    """Random starting errors of the training pairs (standard normal)."""
    return np.random.default_rng(seed).standard_normal(n)
