"""Seeded hole layouts for the box-minus-balls domains.

The physical domain is the box [lo, hi]^d with a set of disjoint balls (discs in 2-D,
spheres in 3-D) removed.  The layout is drawn with NumPy's PCG64 generator:

* one hole after another, radius r ~ U(r_lo, r_hi) first, then every centre
  coordinate ~ U(lo + r, hi - r), so every ball lies inside the box;
* a draw is rejected when it overlaps an earlier ball (|c_i - c_j| <= r_i + r_j) and
  is redrawn, up to 10^4 tries per hole.

Only random numbers are produced here; the level set built from them lives on each
side (oracle and library) separately.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass(frozen=True)
class HoleLayout:
    dim: int
    centers: np.ndarray   # (k, dim) float64
    radii: np.ndarray     # (k,) float64
    lo: float = 0.0
    hi: float = 1.0

    @property
    def n_holes(self) -> int:
        return int(self.radii.shape[0])


def random_holes(dim: int, count: int, r_lo: float, r_hi: float, seed: int,
                 lo: float = 0.0, hi: float = 1.0, max_tries: int = 10_000) -> HoleLayout:
    rng = np.random.default_rng(seed)
    centers: list[np.ndarray] = []
    radii: list[float] = []
    for _ in range(count):
        for _try in range(max_tries):
            r = float(rng.uniform(r_lo, r_hi))
            c = rng.uniform(lo + r, hi - r, size=dim)
            if all(np.linalg.norm(c - cj) > r + rj for cj, rj in zip(centers, radii)):
                centers.append(c)
                radii.append(r)
                break
        else:
            raise RuntimeError(f"could not place hole {len(radii)} without overlap")
    return HoleLayout(dim, np.asarray(centers, dtype=np.float64).reshape(count, dim),
                      np.asarray(radii, dtype=np.float64), lo, hi)


def config1_disc(seed: int) -> HoleLayout:
    """One disc of radius 0.3 whose centre is 0.5 + U(-0.05, 0.05) per coordinate."""
    rng = np.random.default_rng(seed)
    c = 0.5 + rng.uniform(-0.05, 0.05, size=2)
    return HoleLayout(2, c.reshape(1, 2).astype(np.float64), np.array([0.3]), 0.0, 1.0)


def config_layout(name: str, seed: int) -> HoleLayout:
    """Hole layout of a named workload (see synthetic.configs)."""
    if name == "disc1":
        return config1_disc(seed)
    if name == "discs10":
        return random_holes(2, 10, 0.03, 0.1, seed)
    if name == "spheres20":
        return random_holes(3, 20, 0.05, 0.15, seed)
    if name in ("none2", "none3"):
        d = int(name[-1])
        return HoleLayout(d, np.zeros((0, d)), np.zeros(0), 0.0, 1.0)
    if name.startswith("discs"):
        return random_holes(2, int(name[5:]), 0.03, 0.1, seed)
    if name.startswith("spheres"):
        return random_holes(3, int(name[7:]), 0.05, 0.15, seed)
    raise KeyError(name)
