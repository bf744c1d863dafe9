"""One-dimensional bases on a uniform background grid, and their tensor products.

Sec. 2 of the paper discretises on uniform grids with Lagrange functions and with
B-splines of degree p and maximal smoothness C^{p-1}.  The paper never writes the knot
vector down; the reading taken here is the open (clamped) uniform knot vector, which
gives n + p functions per direction on n elements.  Lagrange functions use equispaced
nodes, p n + 1 per direction.

Evaluation follows the textbook definitions: the Cox-de Boor recursion for B-splines
and the Lagrange interpolation polynomials for the nodal basis.  Points are always
given together with the element that contains them, so that the half-open-interval
convention of the recursion never has to be resolved at element boundaries.
"""
from __future__ import annotations

import numpy as np


class BSpline1D:
    """Open uniform B-splines of degree p on [lo, hi] with n elements (m = n + p functions)."""

    kind = "bspline"

    def __init__(self, n: int, p: int, lo: float = 0.0, hi: float = 1.0):
        self.n, self.p, self.lo, self.hi = int(n), int(p), float(lo), float(hi)
        self.h = (self.hi - self.lo) / self.n
        self.m = self.n + self.p
        inner = [self.lo + k * self.h for k in range(1, self.n)]
        self.knots = np.array([self.lo] * (p + 1) + inner + [self.hi] * (p + 1), dtype=np.float64)

    # global index of the local function a = 0 on element e: functions e .. e+p live there
    def first(self, e):
        return e

    def support(self, i: int) -> range:
        """Elements on which function i is non-zero: [i - p, i] clipped to the grid."""
        return range(max(0, i - self.p), min(self.n - 1, i) + 1)

    def is_nodal(self, i: int) -> bool:
        return True

    def _B(self, i, k, span, x):
        """Cox-de Boor: B_{i,k}(x) for x inside knot span `span` (so B_{i,0} = [i == span])."""
        t = self.knots
        if k == 0:
            return np.ones_like(x) if i == span else np.zeros_like(x)
        out = np.zeros_like(x)
        d1 = t[i + k] - t[i]
        if d1 > 0:
            out = out + (x - t[i]) / d1 * self._B(i, k - 1, span, x)
        d2 = t[i + k + 1] - t[i + 1]
        if d2 > 0:
            out = out + (t[i + k + 1] - x) / d2 * self._B(i + 1, k - 1, span, x)
        return out

    def eval(self, e: int, x: np.ndarray):
        """Values and first derivatives of the p+1 functions e..e+p at points x in element e.

        Returns two arrays of shape (p+1, len(x)).
        """
        x = np.asarray(x, dtype=np.float64)
        p, t = self.p, self.knots
        span = e + p
        vals = np.stack([self._B(e + a, p, span, x) for a in range(p + 1)])
        ders = np.zeros_like(vals)
        if p > 0:
            for a in range(p + 1):
                i = e + a
                d = np.zeros_like(x)
                d1 = t[i + p] - t[i]
                if d1 > 0:
                    d = d + p / d1 * self._B(i, p - 1, span, x)
                d2 = t[i + p + 1] - t[i + 1]
                if d2 > 0:
                    d = d - p / d2 * self._B(i + 1, p - 1, span, x)
                ders[a] = d
        return vals, ders

    def eval_global(self, i: int, x: np.ndarray) -> np.ndarray:
        """Value of global function i at arbitrary points x in [lo, hi] (0 outside its support)."""
        x = np.asarray(x, dtype=np.float64)
        e = np.clip(np.floor((x - self.lo) / self.h).astype(int), 0, self.n - 1)
        out = np.zeros_like(x)
        for el in np.unique(e):
            a = i - self.first(el)
            if 0 <= a <= self.p:
                sel = e == el
                out[sel] = self.eval(int(el), x[sel])[0][a]
        return out

    def greville(self) -> np.ndarray:
        """Greville abscissae (knot averages), one per function."""
        p, t = self.p, self.knots
        if p == 0:
            return 0.5 * (t[:-1] + t[1:])
        return np.array([t[i + 1:i + p + 1].mean() for i in range(self.m)])


class Lagrange1D:
    """C0 Lagrange functions of degree p on [lo, hi], equispaced nodes (m = p n + 1)."""

    kind = "lagrange"

    def __init__(self, n: int, p: int, lo: float = 0.0, hi: float = 1.0):
        self.n, self.p, self.lo, self.hi = int(n), int(p), float(lo), float(hi)
        self.h = (self.hi - self.lo) / self.n
        self.m = self.p * self.n + 1
        self.nodes = self.lo + np.arange(self.m) * (self.h / self.p)

    def first(self, e):
        return e * self.p

    def support(self, i: int) -> range:
        p = self.p
        if i % p == 0:   # vertex (nodal) function: the two elements sharing the vertex
            return range(max(0, i // p - 1), min(self.n - 1, i // p) + 1)
        return range(i // p, i // p + 1)

    def is_nodal(self, i: int) -> bool:
        """Functions that equal 1 at a grid vertex (the only ones that own Schwarz blocks)."""
        return i % self.p == 0

    def eval(self, e: int, x: np.ndarray):
        x = np.asarray(x, dtype=np.float64)
        p = self.p
        xn = self.lo + e * self.h + np.arange(p + 1) * (self.h / p)
        vals = np.ones((p + 1, x.size))
        ders = np.zeros((p + 1, x.size))
        for a in range(p + 1):
            for b in range(p + 1):
                if b != a:
                    vals[a] *= (x - xn[b]) / (xn[a] - xn[b])
            for c in range(p + 1):      # product rule: drop one factor at a time
                if c == a:
                    continue
                term = np.full(x.size, 1.0 / (xn[a] - xn[c]))
                for b in range(p + 1):
                    if b != a and b != c:
                        term *= (x - xn[b]) / (xn[a] - xn[b])
                ders[a] += term
        return vals, ders

    def eval_global(self, i: int, x: np.ndarray) -> np.ndarray:
        x = np.asarray(x, dtype=np.float64)
        e = np.clip(np.floor((x - self.lo) / self.h).astype(int), 0, self.n - 1)
        out = np.zeros_like(x)
        for el in np.unique(e):
            a = i - self.first(el)
            if 0 <= a <= self.p:
                sel = e == el
                out[sel] = self.eval(int(el), x[sel])[0][a]
        return out


def make_basis(kind: int, n: int, p: int, lo: float, hi: float):
    """kind 0 = B-spline, 1 = Lagrange."""
    return BSpline1D(n, p, lo, hi) if kind == 0 else Lagrange1D(n, p, lo, hi)


class TensorBasis:
    """Tensor product of one 1-D basis in each of d directions (x index fastest)."""

    def __init__(self, basis1d, dim: int):
        self.b, self.dim = basis1d, int(dim)
        self.n, self.p, self.m = basis1d.n, basis1d.p, basis1d.m
        self.h = basis1d.h
        self.n_elems = self.n ** dim
        self.n_funcs = self.m ** dim
        self.nloc = (self.p + 1) ** dim
        # local multi-indices a = (a0, a1, a2), a0 fastest
        self.local = np.array(np.unravel_index(np.arange(self.nloc), (self.p + 1,) * dim, order="F")).T

    def elem_multi(self, E: int):
        return np.unravel_index(E, (self.n,) * self.dim, order="F")

    def func_multi(self, I: int):
        return np.unravel_index(I, (self.m,) * self.dim, order="F")

    def func_flat(self, multi) -> int:
        return int(np.ravel_multi_index(tuple(multi), (self.m,) * self.dim, order="F"))

    def elem_box(self, E: int):
        e = np.array(self.elem_multi(E))
        lo = self.b.lo + e * self.h
        return lo, lo + self.h

    def elem_dofs(self, E: int) -> np.ndarray:
        """Global indices of the (p+1)^d functions that live on element E, local order."""
        e = self.elem_multi(E)
        first = np.array([self.b.first(int(ek)) for ek in e])
        g = first[None, :] + self.local
        return np.ravel_multi_index(tuple(g.T), (self.m,) * self.dim, order="F")

    def support_elems(self, I: int) -> list[int]:
        ranges = [self.b.support(int(ik)) for ik in self.func_multi(I)]
        grids = np.meshgrid(*ranges, indexing="ij")
        ems = np.stack([g.ravel() for g in grids])
        return sorted(np.ravel_multi_index(tuple(ems), (self.n,) * self.dim, order="F").tolist())

    def is_nodal(self, I: int) -> bool:
        """Nodal in every direction (Lagrange vertex function; every B-spline qualifies)."""
        return all(self.b.is_nodal(int(ik)) for ik in self.func_multi(I))

    def on_box_boundary(self, I: int) -> bool:
        """Non-zero somewhere on the boundary of the embedding box."""
        return any(ik == 0 or ik == self.m - 1 for ik in self.func_multi(I))

    def eval(self, E: int, X: np.ndarray):
        """Values (nloc, npts) and gradients (dim, nloc, npts) of the local functions of E at X."""
        X = np.atleast_2d(np.asarray(X, dtype=np.float64))
        e = self.elem_multi(E)
        per = [self.b.eval(int(e[k]), X[:, k]) for k in range(self.dim)]
        vals = np.ones((self.nloc, X.shape[0]))
        grads = np.ones((self.dim, self.nloc, X.shape[0]))
        for k in range(self.dim):
            v, d = per[k]
            vk = v[self.local[:, k]]
            dk = d[self.local[:, k]]
            vals *= vk
            for j in range(self.dim):
                grads[j] *= dk if j == k else vk
        return vals, grads
