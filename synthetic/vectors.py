"""Seeded random grid vectors (standard normal, inactive entries zeroed by the caller)."""
from __future__ import annotations

import numpy as np


def random_grid_vector(n: int, seed: int, mask: np.ndarray | None = None) -> np.ndarray:
    rng = np.random.default_rng(seed)
    v = rng.standard_normal(n)
    if mask is not None:
        v = np.where(mask.astype(bool), v, 0.0)
    return v
