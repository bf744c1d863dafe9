"""Pins of the oracle's bases and cut-cell quadrature against closed forms.

Nothing here compares the oracle with itself: every expected value comes from a
textbook formula (truncated-power B-splines, polygon areas, the divergence theorem,
Gauss exactness).
"""
import math

import numpy as np
import pytest

from oracle import geometry as G
from oracle.basis import BSpline1D, Lagrange1D, TensorBasis
from oracle.quadrature import (box_rule, clip_simplex, cut_element_rule, facet_rule,
                               gauss01, simplex_rule)


def cardinal_bspline(p, t):
    """Uniform cardinal B-spline of degree p on [0, p+1], truncated-power form."""
    t = np.asarray(t, dtype=float)
    s = np.zeros_like(t)
    for k in range(p + 2):
        s += (-1) ** k * math.comb(p + 1, k) * np.where(t > k, (t - k), 0.0) ** p
    return s / math.factorial(p)


@pytest.mark.parametrize("p", [1, 2, 3])
def test_bspline_interior_matches_cardinal(p):
    n = 12
    b = BSpline1D(n, p)
    rng = np.random.default_rng(0)
    for i in range(p, n):                 # functions whose knots are all simple
        x = rng.uniform(b.knots[i], b.knots[i + p + 1], 50)
        t = (x - b.knots[i]) / b.h
        np.testing.assert_allclose(b.eval_global(i, x), cardinal_bspline(p, t), atol=1e-13)


@pytest.mark.parametrize("p", [1, 2, 3])
def test_bspline_partition_of_unity_and_derivative(p):
    b = BSpline1D(7, p)
    rng = np.random.default_rng(1)
    for e in range(b.n):
        x = b.lo + (e + rng.uniform(0, 1, 20)) * b.h
        v, d = b.eval(e, x)
        np.testing.assert_allclose(v.sum(0), 1.0, atol=1e-14)
        np.testing.assert_allclose(d.sum(0), 0.0, atol=1e-11)
        eps = 1e-6
        vp, _ = b.eval(e, x + eps)
        vm, _ = b.eval(e, x - eps)
        np.testing.assert_allclose(d, (vp - vm) / (2 * eps), atol=1e-6 / b.h)


def test_linear_bspline_equals_linear_lagrange():
    b, l = BSpline1D(9, 1), Lagrange1D(9, 1)
    x = np.linspace(0, 1, 301)
    for i in range(b.m):
        np.testing.assert_allclose(b.eval_global(i, x), l.eval_global(i, x), atol=1e-14)


@pytest.mark.parametrize("p", [1, 2, 3])
def test_lagrange_kronecker_and_derivatives(p):
    l = Lagrange1D(5, p)
    for i in range(l.m):
        np.testing.assert_allclose(l.eval_global(i, l.nodes), (np.arange(l.m) == i).astype(float), atol=1e-13)
    x = 0.2 + 0.6 * np.random.default_rng(2).uniform(size=10) * l.h
    v, d = l.eval(1, x + l.h)
    eps = 1e-6
    vp, _ = l.eval(1, x + l.h + eps)
    vm, _ = l.eval(1, x + l.h - eps)
    np.testing.assert_allclose(d, (vp - vm) / (2 * eps), atol=1e-5 / l.h)


def test_gauss_exactness():
    for n in (2, 3, 4, 5):
        x, w = gauss01(n)
        for k in range(2 * n):
            assert abs(np.sum(w * x ** k) - 1.0 / (k + 1)) < 1e-14


@pytest.mark.parametrize("dim", [2, 3])
def test_simplex_rule_exact_to_degree(dim):
    n = 4                                   # p = 2: collapsed rule with p + 2 points
    rng = np.random.default_rng(3)
    V = rng.uniform(size=(dim + 1, dim))
    x, w = simplex_rule(V, n)
    vol = abs(np.linalg.det(V[1:] - V[0])) / math.factorial(dim)
    assert abs(w.sum() - vol) < 1e-14
    # barycentric monomial integrals: int lambda^alpha = d! alpha! / (d + |alpha|)! |T|
    lam = np.linalg.solve(np.vstack([np.ones(dim + 1), V.T]), np.vstack([np.ones(len(w)), x.T]))
    for alpha in [(2, 1, 0) + (0,) * (dim - 2), (1, 1, 1) + (0,) * (dim - 2), (0,) * dim + (3,)]:
        alpha = np.array(alpha[:dim + 1])
        if alpha.sum() > 2 * n - (dim + 1) + 1 - 1:
            continue
        val = np.sum(w * np.prod(lam ** alpha[:, None], axis=0))
        ex = math.factorial(dim) * np.prod([math.factorial(a) for a in alpha]) / math.factorial(dim + alpha.sum()) * vol
        assert abs(val - ex) < 1e-14 * max(1, abs(ex)) + 1e-16


def test_clip_halfplane_area_and_length():
    """A straight cut of a square: kept area and boundary length in closed form."""
    lo, hi = np.zeros(2), np.ones(2)
    geom = G.half_space([1.0, 0.5], -0.6)      # x + y/2 > 0.6
    vp, vw, bp, bw, bn = cut_element_rule(geom, lo, hi, 2, 0)
    # region x > 0.6 - y/2, y in [0, 1]: area = int_0^1 (1 - 0.6 + y/2) dy = 0.4 + 0.25
    assert abs(vw.sum() - 0.65) < 1e-14
    assert abs(bw.sum() - math.hypot(0.5, 1.0)) < 1e-14
    np.testing.assert_allclose(bn, np.tile(-np.array([1.0, 0.5]) / math.hypot(1, 0.5), (len(bw), 1)), atol=1e-15)
    # first moment: int x over the trapezoid
    ex = sum(0.5 * (1.0 - (0.6 - y / 2) ** 2) * wy for y, wy in zip(*gauss01(4)))
    assert abs(np.sum(vw * vp[:, 0]) - ex) < 1e-14


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("depth", [0, 2])
def test_divergence_theorem_on_immersed_ball(dim, depth):
    """int_{Omega_h} div F = int_{Gamma_h} F.n for a polynomial F on a ball inside the box.

    Omega_h is the polytope cut out by the linear interpolant, so the identity is exact
    when the rules integrate F.n and div F exactly; it pins facet weights and normals.
    """
    c = np.array([0.51, 0.47, 0.53][:dim])
    geom = G.LevelSet(lambda X: 0.3 - np.linalg.norm(X - c, axis=1), dim, 0.0, 1.0)
    n = 6 if dim == 2 else 4
    h = 1.0 / n
    F = lambda X: np.stack([X[:, 0] ** 2 * X[:, 1], X[:, 1] ** 2, X[:, -1] * X[:, 0]][:dim], axis=1)
    divF = lambda X: 2 * X[:, 0] * X[:, 1] + 2 * X[:, 1] + (X[:, 0] if dim == 3 else 0)
    vol = bnd = 0.0
    for idx in np.ndindex(*(n,) * dim):
        lo = np.array(idx[::-1], dtype=float) * h
        hi = lo + h
        cls = geom.classify(lo, hi)
        if cls == G.EMPTY:
            continue
        if cls == G.FULL:
            x, w = box_rule(lo, hi, 3)
            vol += np.sum(w * divF(x))
            continue
        vp, vw, bp, bw, bnorm = cut_element_rule(geom, lo, hi, 2, depth)
        vol += np.sum(vw * divF(vp))
        bnd += np.sum(bw * np.sum(F(bp) * bnorm, axis=1))
    assert abs(vol - bnd) < 1e-13


def test_disc_area_converges_quadratically():
    geom = lambda: G.Balls([[0.5, 0.5]], [0.3])
    errs = []
    for depth in (0, 1, 2, 3):
        g = geom()
        tot = 0.0
        n = 8
        for idx in np.ndindex(n, n):
            lo = np.array(idx[::-1], dtype=float) / n
            hi = lo + 1.0 / n
            cls = g.classify(lo, hi)
            if cls == G.FULL:
                tot += 1.0 / n ** 2
            elif cls == G.CUT:
                tot += cut_element_rule(g, lo, hi, 1, depth)[1].sum()
        errs.append(abs(tot - (1 - math.pi * 0.09)))
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(3)]
    assert min(rates) > 1.7, (errs, rates)


def test_ball_classification_catches_interior_hole():
    g = G.Balls([[0.55, 0.45]], [0.02])
    assert g.classify(np.array([0.5, 0.4]), np.array([0.6, 0.5])) == G.CUT   # hole strictly inside
    assert g.classify(np.array([0.7, 0.7]), np.array([0.8, 0.8])) == G.FULL
    assert g.classify(np.array([0.545, 0.445]), np.array([0.555, 0.455])) == G.EMPTY


def test_tensor_basis_products():
    tb = TensorBasis(BSpline1D(4, 2), 2)
    X = np.array([[0.3, 0.6], [0.26, 0.74]])
    E = 1 + 4 * 2
    vals, grads = tb.eval(E, X)
    dofs = tb.elem_dofs(E)
    for a, I in enumerate(dofs):
        ix, iy = tb.func_multi(int(I))
        ex = tb.b.eval_global(int(ix), X[:, 0]) * tb.b.eval_global(int(iy), X[:, 1])
        np.testing.assert_allclose(vals[a], ex, atol=1e-15)
