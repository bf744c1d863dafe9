"""Implicit domains: Omega = {psi > 0} inside a box-shaped embedding domain (Sec. 2, Fig. 1).

Two kinds of level set are provided.

* ``Balls``: the box minus a union of disjoint balls, psi(x) = min_i (|x - c_i| - r_i).
  Cells are classified exactly with the ball-box distance test, so a hole that lies
  strictly inside a cell, or a ball that grazes a cell edge between two corners, is
  never missed.
* ``LevelSet``: any callable psi (the star of Fig. 1, a half plane, the tooth, apple and
  helix of Sec. 4.1).  Cells are classified by the signs of psi at their 2^d corners.

Reading of the silent points: points where psi == 0 exactly count as outside, and a
cell is ``full`` when psi > 0 on it up to measure zero, ``empty`` when psi <= 0 on all
of it, and ``cut`` otherwise.
"""
from __future__ import annotations

import itertools

import numpy as np

FULL, EMPTY, CUT = 0, 1, 2


def box_corners(lo: np.ndarray, hi: np.ndarray) -> np.ndarray:
    d = len(lo)
    return np.array([[hi[k] if (c >> k) & 1 else lo[k] for k in range(d)] for c in range(2 ** d)])


class Balls:
    """Box [lo, hi]^d minus disjoint closed balls; every box face is Dirichlet boundary."""

    box_dirichlet = True

    def __init__(self, centers, radii, lo: float = 0.0, hi: float = 1.0):
        self.centers = np.atleast_2d(np.asarray(centers, dtype=np.float64))
        self.radii = np.asarray(radii, dtype=np.float64).reshape(-1)
        self.dim = self.centers.shape[1]
        self.lo, self.hi = float(lo), float(hi)

    def psi(self, X: np.ndarray) -> np.ndarray:
        X = np.atleast_2d(X)
        if self.radii.size == 0:
            return np.full(X.shape[0], np.inf)
        dist = np.linalg.norm(X[:, None, :] - self.centers[None, :, :], axis=2) - self.radii[None, :]
        return dist.min(axis=1)

    def classify(self, lo: np.ndarray, hi: np.ndarray) -> int:
        """Exact classification of the closed box [lo, hi] against the balls."""
        cut = False
        for c, r in zip(self.centers, self.radii):
            nearest = np.clip(c, lo, hi)
            dmin = np.linalg.norm(nearest - c)
            far = np.where(np.abs(c - lo) > np.abs(c - hi), lo, hi)
            dmax = np.linalg.norm(far - c)
            if dmax <= r:
                return EMPTY          # the whole box lies in this ball
            if dmin < r:
                cut = True            # the ball reaches into the box
        return CUT if cut else FULL

    def classify_many(self, LO: np.ndarray, HI: np.ndarray) -> np.ndarray:
        """`classify` applied to every row of the box arrays LO, HI (same test, vectorised)."""
        out = np.full(LO.shape[0], FULL, dtype=np.int8)
        empty = np.zeros(LO.shape[0], dtype=bool)
        cut = np.zeros(LO.shape[0], dtype=bool)
        for c, r in zip(self.centers, self.radii):
            nearest = np.clip(c[None, :], LO, HI)
            dmin = np.linalg.norm(nearest - c[None, :], axis=1)
            far = np.where(np.abs(c[None, :] - LO) > np.abs(c[None, :] - HI), LO, HI)
            dmax = np.linalg.norm(far - c[None, :], axis=1)
            empty |= dmax <= r
            cut |= dmin < r
        out[cut] = CUT
        out[empty] = EMPTY
        return out


class LevelSet:
    """Generic level set psi; cells classified by corner signs.

    ``box_dirichlet`` says whether the box faces belong to the Dirichlet boundary (a
    domain cut out of the box) or not (a domain immersed in the box, whose boundary is
    {psi = 0} only).
    """

    def __init__(self, psi, dim: int, lo: float, hi: float, box_dirichlet: bool = False):
        self._psi, self.dim, self.lo, self.hi = psi, int(dim), float(lo), float(hi)
        self.box_dirichlet = bool(box_dirichlet)

    def psi(self, X: np.ndarray) -> np.ndarray:
        return self._psi(np.atleast_2d(X))

    def classify(self, lo: np.ndarray, hi: np.ndarray) -> int:
        v = self.psi(box_corners(lo, hi))
        if np.all(v > 0):
            return FULL
        if np.all(v <= 0):
            return EMPTY
        return CUT

    def classify_many(self, LO: np.ndarray, HI: np.ndarray) -> np.ndarray:
        d = LO.shape[1]
        vals = []
        for c in range(2 ** d):
            bits = np.array([(c >> k) & 1 for k in range(d)], dtype=bool)
            vals.append(self.psi(np.where(bits[None, :], HI, LO)))
        V = np.stack(vals, axis=1)
        out = np.full(LO.shape[0], CUT, dtype=np.int8)
        out[np.all(V > 0, axis=1)] = FULL
        out[np.all(V <= 0, axis=1)] = EMPTY
        return out


def star() -> LevelSet:
    """Fig. 1: psi = 0.5 + 0.1 sin(5 theta) - r on the embedding domain (-1, 1)^2."""
    def psi(X):
        r = np.hypot(X[:, 0], X[:, 1])
        th = np.arctan2(X[:, 1], X[:, 0])
        return 0.5 + 0.1 * np.sin(5.0 * th) - r
    return LevelSet(psi, 2, -1.0, 1.0)


def half_space(normal, offset, lo: float = 0.0, hi: float = 1.0) -> LevelSet:
    """psi = normal . x + offset (Omega_h is then exact: psi is linear)."""
    nrm = np.asarray(normal, dtype=np.float64)
    return LevelSet(lambda X: X @ nrm + offset, len(nrm), lo, hi, box_dirichlet=True)


def tooth() -> LevelSet:
    """Sec. 4.1.1: tooth on (-2, 2)^3: psi_1 = 16 (1 - sum_i exp(-rho_i)) - x^4 - y^4 - z^4,
    with the root tips below z = -1 trimmed by psi_2 = z + 1 (Omega = {psi_1 > 0, psi_2 > 0})."""
    def psi(X):
        x, y, z = X[:, 0], X[:, 1], X[:, 2]
        zz = (z + 2.0) / 2.0
        rho = [x ** 2 + y ** 2 + (z - 2.0) ** 2,
               (x - 2.0) ** 2 + (y - 2.0) ** 2 + zz ** 2,
               (x - 2.0) ** 2 + (y + 2.0) ** 2 + zz ** 2,
               (x + 2.0) ** 2 + (y + 2.0) ** 2 + zz ** 2,
               (x + 2.0) ** 2 + (y - 2.0) ** 2 + zz ** 2,
               x ** 2 + (y / 2.0) ** 2 + zz ** 2,
               (x / 2.0) ** 2 + y ** 2 + zz ** 2]
        s = sum(np.exp(-r) for r in rho)
        return np.minimum(16.0 * (1.0 - s) - x ** 4 - y ** 4 - z ** 4, z + 1.0)
    return LevelSet(psi, 3, -2.0, 2.0)


def apple() -> LevelSet:
    """Sec. 4.1.2: apple psi_1 with the bite psi_2 removed (Omega = {psi_1 > 0, psi_2 > 0})."""
    def psi(X):
        x, y, z = X[:, 0], X[:, 1], X[:, 2]
        r = np.hypot(x, y)
        p1 = 1.0 - (z / 1.7) ** 2 - (r / (1.0 + z / 17.0) - 0.7) ** 2
        p2 = (x - 2.0) ** 2 + y ** 2 + z ** 2 - 1.0
        return np.minimum(p1, p2)
    return LevelSet(psi, 3, -2.0, 2.0)


def helix() -> LevelSet:
    """Sec. 4.1.4: triple helix joined by rings at z = +-2 on (-2, 2)^3.

    Reading: Omega is the union of the three copies of psi_1 rotated by 0, 2 pi/3 and
    4 pi/3 about the z axis (arctan2 on its principal branch, as printed) and the two
    ring tubes psi_2^+-; the box cuts the rings in half.
    """
    r_in, R_out = 0.25, 1.5

    def psi(X):
        x, y, z = X[:, 0], X[:, 1], X[:, 2]
        r = np.hypot(x, y)
        out = np.full(X.shape[0], -np.inf)
        for k in range(3):
            rot = 2.0 * np.pi * k / 3.0
            xr = np.cos(rot) * x + np.sin(rot) * y
            yr = -np.sin(rot) * x + np.cos(rot) * y
            th = np.arctan2(yr, xr)
            out = np.maximum(out, r_in ** 2 - (r - R_out) ** 2 - (z - 2.0 * th / np.pi) ** 2)
        for s in (1.0, -1.0):
            out = np.maximum(out, r_in ** 2 - (r - R_out) ** 2 - (z + s * 2.0) ** 2)
        return out
    return LevelSet(psi, 3, -2.0, 2.0)


def leaf_boxes(lo: np.ndarray, hi: np.ndarray, depth: int):
    """The 2^(d*depth) leaves of `depth` uniform bisections of the box [lo, hi]."""
    d = len(lo)
    k = 2 ** depth
    step = (hi - lo) / k
    for idx in itertools.product(range(k), repeat=d):
        idx = np.array(idx[::-1])          # x index fastest
        a = lo + idx * step
        yield a, a + step


def active_elements_by_corners(geom: LevelSet, n: int, depth: int) -> np.ndarray:
    """Active elements (|K cap Omega_h| > 0) of a corner-classified level set, from psi on
    the lattice of leaf corners alone.

    With corner classification, a leaf is cut or full exactly when one of its corners
    has psi > 0, and then the clipped simplex at that corner keeps a positive volume;
    an element is therefore active exactly when psi > 0 at one of the corners of its
    2^(d*depth) leaves.  (Equal to ``Discretization.elem_active``; used where the
    full quadrature is too slow for this oracle, e.g. the DOF counts of Sec. 4.1.)
    Returns a boolean array of shape (n,)*d indexed [i_x, i_y, (i_z)].
    """
    d, k = geom.dim, 2 ** depth
    h = (geom.hi - geom.lo) / n
    x = geom.lo + np.arange(n * k + 1) * (h / k)
    act = np.zeros((n,) * d, dtype=bool)
    for s in range(n):                      # one slab of elements in the last direction
        last = x[s * k: s * k + k + 1]
        grids = np.meshgrid(*([x] * (d - 1) + [last]), indexing="ij")
        P = np.stack([g.ravel() for g in grids], axis=1)
        pos = (geom.psi(P) > 0).reshape(grids[0].shape)
        for off in itertools.product(range(k + 1), repeat=d - 1):
            sub = pos[tuple(slice(o, o + n * k, k) for o in off)]
            sub = sub[tuple(slice(0, n) for _ in range(d - 1))]
            act[(Ellipsis, s)] |= sub.any(axis=-1)
    return act
