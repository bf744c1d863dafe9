"""Pins of the oracle's assembly (Sec. 2) against closed forms and exact solutions."""
import math

import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import geometry as G
from oracle.discretize import NITSCHE, PENALTY, Discretization, Manufactured, Polynomial, nitsche_beta
from test_oracle_basis_quadrature import cardinal_bspline


def toeplitz_1d(p, h):
    """Interior 1-D stiffness and mass stencils (offsets -p..p) from the cardinal B-spline."""
    x, w = np.polynomial.legendre.leggauss(8)
    K, M = np.zeros(2 * p + 1), np.zeros(2 * p + 1)
    eps = 1e-7
    for o in range(-p, p + 1):
        for a in range(p + 1):                       # unit intervals [a, a+1] of the support
            t = a + 0.5 * (x + 1)
            N0, N1 = cardinal_bspline(p, t), cardinal_bspline(p, t - o)
            d0 = (cardinal_bspline(p, t + eps) - cardinal_bspline(p, t - eps)) / (2 * eps)
            d1 = (cardinal_bspline(p, t - o + eps) - cardinal_bspline(p, t - o - eps)) / (2 * eps)
            M[o + p] += 0.5 * np.sum(w * N0 * N1) * h
            K[o + p] += 0.5 * np.sum(w * d0 * d1) / h
    return K, M


def test_known_quadratic_stencils():
    K, M = toeplitz_1d(2, 1.0)
    np.testing.assert_allclose(M, np.array([1, 26, 66, 26, 1]) / 120, atol=1e-9)
    np.testing.assert_allclose(K, np.array([-1, -2, 6, -2, -1]) / 6, atol=1e-6)


@pytest.mark.parametrize("p", [1, 2, 3])
def test_interior_rows_equal_tensor_stencil(p):
    """Rows whose support is all full equal (K (x) M + M (x) K) of the 1-D closed forms."""
    n = 24
    geom = G.Balls([[0.3, 0.35]], [0.1])
    d = Discretization(geom, 0, p, n, 0, NITSCHE)
    K, M = toeplitz_1d(p, 1.0 / n)
    A = d.A.tocsr()
    checked = 0
    for i in range(2 * p, n - p):
        for j in range(2 * p, n - p):
            I = d.tb.func_flat((i, j))
            if not all(d.elem_class[E] == G.FULL for E in d.tb.support_elems(I)):
                continue
            r = d.full_to_active[I]
            row = A.getrow(r)
            for ox in range(-p, p + 1):
                for oy in range(-p, p + 1):
                    J = d.tb.func_flat((i + ox, j + oy))
                    c = d.full_to_active[J]
                    ex = K[ox + p] * M[oy + p] + M[ox + p] * K[oy + p]
                    assert abs(row[0, c] - ex) < 1e-6 * abs(K).max()
            checked += 1
    assert checked > 20


@pytest.mark.parametrize("kind,p", [(0, 1), (0, 2), (0, 3), (1, 2)])
def test_box_without_holes_activity(kind, p):
    d = Discretization(G.Balls(np.zeros((0, 2)), np.zeros(0)), kind, p, 8, 0, NITSCHE)
    m = d.tb.m
    assert d.n_active == (m - 2) ** 2
    assert len(d.cut_elems) == 0


@pytest.mark.parametrize("bc", [PENALTY, NITSCHE])
def test_symmetric_positive_definite(bc):
    geom = G.Balls([[0.52, 0.47]], [0.3])
    d = Discretization(geom, 0, 2, 16, 2, bc)
    A = d.A.toarray()
    assert np.abs(A - A.T).max() < 1e-13 * np.abs(A).max()
    # SPD via Cholesky (eigenvalues of cut functions can sit at 1e-16 relative)
    np.linalg.cholesky(A)


@pytest.mark.parametrize("kind,p,dim", [(0, 1, 2), (0, 2, 2), (1, 2, 2), (0, 3, 2), (0, 2, 3)])
def test_nitsche_reproduces_polynomials(kind, p, dim):
    """u in V_h and exact quadrature => the Nitsche solution is u itself (consistency).

    2-D, p >= 2: u = x(1-x) y(1-y) vanishes on the box faces and lies in V_h; the rules
    integrate every term exactly.  Otherwise (p = 1, or 3-D where the collapsed rule is
    exact only to total degree 2p+1) u is affine plus a bilinear term in 2-D, on a ball
    immersed in the box, for which the rules are exact.
    """
    if p >= 2 and dim == 2:
        u = lambda X: np.prod(X * (1 - X), axis=1)
        def mlap(X):
            q = X * (1 - X)
            return sum(2.0 * np.prod(np.delete(q, k, axis=1), axis=1) for k in range(dim))
        geom = G.Balls([[0.5, 0.45, 0.55][:dim]], [0.23])
        n = 8 if dim == 2 else 4
    else:
        u = lambda X: 1.0 + X[:, 0] - 2.0 * X[:, 1] + (0.5 * X[:, 0] * X[:, 1] if dim == 2 else 0.7 * X[:, 2])
        mlap = lambda X: np.zeros(X.shape[0])
        c = np.array([0.5, 0.5, 0.5][:dim])
        geom = G.LevelSet(lambda X: 0.31 - np.linalg.norm(X - c, axis=1), dim, 0.0, 1.0)
        n = 8 if dim == 2 else 4
    d = Discretization(geom, kind, p, n, 1, NITSCHE, problem=Polynomial(u, mlap))
    x = spla.spsolve(d.A.tocsc(), d.b)
    rng = np.random.default_rng(4)
    P = rng.uniform(0.05, 0.95, size=(400, dim))
    P = P[geom.psi(P) > 0.02]
    np.testing.assert_allclose(d.evaluate(x, P), u(P), atol=1e-9)


@pytest.mark.slow
@pytest.mark.parametrize("p", [1, 2, 3])
def test_manufactured_convergence_rates_half_plane(p):
    """Straight immersed boundary (Omega_h exact): L2 rate p+1 and H1 rate p."""
    geom = G.half_space([1.0, 0.37], -0.41)
    u = Manufactured.u
    gu = lambda X: np.pi * np.stack([np.cos(np.pi * X[:, 0]) * np.sin(np.pi * X[:, 1]),
                                      np.sin(np.pi * X[:, 0]) * np.cos(np.pi * X[:, 1])], axis=1)
    e0, e1 = [], []
    for n in (8, 16, 32):
        d = Discretization(geom, 0, p, n, 0, NITSCHE)
        x = spla.spsolve(d.A.tocsc(), d.b)
        a, b = d.l2_h1_errors(x, u, gu)
        e0.append(a)
        e1.append(b)
    r0 = [math.log2(e0[i] / e0[i + 1]) for i in range(2)]
    r1 = [math.log2(e1[i] / e1[i + 1]) for i in range(2)]
    assert r0[-1] > p + 1 - 0.3, (e0, r0)
    assert r1[-1] > p - 0.3, (e1, r1)


def test_nitsche_beta_makes_element_form_coercive():
    """beta_K >= 2 C_K: x^T (S - C - C^T + beta B) x >= 1/2 x^T S x for all x on the element."""
    geom = G.Balls([[0.52, 0.47]], [0.3])
    d = Discretization(geom, 0, 2, 16, 2, NITSCHE, assemble=False)
    rng = np.random.default_rng(5)
    tested = 0
    for E in d.cut_elems[:20]:
        vp, vw, bp, bw, bn = d.cut_rule(int(E))
        if not len(bw):
            continue
        A, _, _, beta = d.element_system(int(E))
        vals, grads = d.tb.eval(int(E), vp)
        S = np.einsum("jaq,jbq,q->ab", grads, grads, vw)
        # A - S/2 must be positive semi-definite
        ev = np.linalg.eigvalsh(A - 0.5 * S)
        assert ev.min() > -1e-10 * np.abs(A).max()
        assert beta == 2.0 ** round(math.log2(beta))
        tested += 1
    assert tested > 5


def test_nitsche_beta_closed_form_1d_like():
    """A 2-function element where the eigenproblem is scalar: beta = 2^ceil(log2(2 b/s))."""
    S = np.array([[1.0, -1.0], [-1.0, 1.0]]) * 3.0
    B = np.array([[1.0, -1.0], [-1.0, 1.0]]) * 5.0
    assert nitsche_beta(S, B, 1.0) == 4.0          # lambda = 5/3 -> 2 lambda = 3.33 -> 4
    assert nitsche_beta(S, B, 1e-3) == 2048.0      # floor 1/h = 1000 -> 2000 -> 2048


def test_row_assembly_matches_global_assembly():
    """Rows of A and entries of b assembled one by one from the element systems of the
    support elements (the path the full-size parity tests take) equal the globally
    assembled system (batched tensor rule on full elements)."""
    from parity_utils import oracle_for
    pr, lay, d, H = oracle_for("disc1_32_p2")
    rng = np.random.default_rng(3)
    rows = np.unique(np.concatenate([rng.choice(d.active, 60, replace=False),
                                     [int(J) for E in d.cut_elems[:20] for J in d.tb.elem_dofs(int(E))
                                      if d.func_active_full[J]]]))
    got = d.assemble_rows(rows)
    pos = -np.ones(d.tb.n_funcs, dtype=np.int64)
    pos[d.active] = np.arange(d.n_active)
    Ad = d.A.tocsr()
    for I in rows:
        cols, vals, bI = got[int(I)]
        ref = Ad[pos[I]].toarray().ravel()
        row = np.zeros(d.n_active)
        row[pos[cols]] = vals
        scale = np.abs(ref).max()
        assert np.abs(row - ref).max() <= 1e-13 * scale
        assert abs(bI - d.b[pos[I]]) <= 1e-13 * np.abs(d.b).max()


@pytest.mark.parametrize("name,ov", [("disc1_32_p2", {}), ("spheres20_128_p2", dict(n=8, levels=2, depth=1))])
def test_local_rows_equal_global_assembly(name, ov):
    """LocalRows (cut elements integrated on demand, activity from each row's own support)
    gives exactly the rows and right-hand side entries of the global assembly, including
    inactive rows (empty) and box-face rows (excluded)."""
    from oracle.discretize import LocalRows
    from parity_utils import layout_for
    pr, lay = layout_for(name, **ov)
    geom = G.Balls(lay.centers, lay.radii, lay.lo, lay.hi)
    d = Discretization(geom, pr.basis, pr.degree, pr.n, pr.depth, pr.bc)
    loc = LocalRows(geom, pr.basis, pr.degree, pr.n, pr.depth, pr.bc)
    rng = np.random.default_rng(5)
    rows = np.unique(np.concatenate([rng.choice(d.tb.n_funcs, 60, replace=False),
                                     d.active[rng.choice(d.n_active, 60, replace=False)]]))
    got = loc.assemble_rows(rows)
    Af = d.A.tocsr()
    for I in rows:
        cols, vals, bI = got[int(I)]
        a = d.full_to_active[I]
        if a < 0:
            assert cols.size == 0 and bI == 0.0
            continue
        ref = Af[a]
        np.testing.assert_array_equal(cols, np.sort(d.active[ref.indices]))
        order = np.argsort(d.active[ref.indices])
        np.testing.assert_allclose(vals, ref.data[order], rtol=0, atol=1e-14 * np.abs(ref.data).max())
        assert abs(bI - d.b[a]) <= 1e-14 * np.abs(d.b).max()
