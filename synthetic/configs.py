"""Named workload presets: the immersed Poisson problems the solver is exercised on.

Each preset fixes the background grid, basis, degree, number of multigrid levels,
quadrature depth, boundary-condition mode and hole layout.  basis 0 = B-spline,
1 = Lagrange; bc 0 = penalty (beta = 2/h), 1 = symmetric Nitsche.
"""
from __future__ import annotations

from dataclasses import dataclass


@dataclass(frozen=True)
class Preset:
    name: str
    dim: int
    n: int              # elements per direction on the finest grid
    basis: int          # 0 = B-spline, 1 = Lagrange
    degree: int
    levels: int
    depth: int          # cut-cell bisection depth
    bc: int             # 0 = penalty, 1 = Nitsche
    layout: str         # hole layout name understood by synthetic.geometry.config_layout


PRESETS = {
    # 2-D, 32x32, quadratic B-splines, one disc, depth 3, 3 levels
    "disc1_32_p2": Preset("disc1_32_p2", 2, 32, 0, 2, 3, 3, 1, "disc1"),
    # 2-D, 512x512, ten discs, depth 0, 6 levels
    "discs10_512_p1": Preset("discs10_512_p1", 2, 512, 1, 1, 6, 0, 1, "discs10"),
    "discs10_512_p2": Preset("discs10_512_p2", 2, 512, 0, 2, 6, 0, 1, "discs10"),
    "discs10_512_p3": Preset("discs10_512_p3", 2, 512, 0, 3, 6, 0, 1, "discs10"),
    # 3-D, 128^3, quadratic B-splines, twenty spheres, depth 2, 5 levels
    "spheres20_128_p2": Preset("spheres20_128_p2", 3, 128, 0, 2, 5, 2, 1, "spheres20"),
    # 3-D, 256^3 box without holes, quadratic B-splines, 6 levels: every vector is larger
    # than L2, so the V-cycle streams from HBM
    "box_256_p2": Preset("box_256_p2", 3, 256, 0, 2, 6, 0, 1, "none3"),
}


def preset(name: str, **overrides) -> Preset:
    p = PRESETS[name]
    if overrides:
        p = Preset(**{**p.__dict__, **overrides})
    return p
