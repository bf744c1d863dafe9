"""Pins of the oracle's multigrid pieces (Sec. 3) against closed forms and invariants."""
import math

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse.linalg as spla

from oracle import geometry as G
from oracle.basis import BSpline1D, Lagrange1D, TensorBasis
from oracle.discretize import NITSCHE, PENALTY, Discretization
from oracle.multigrid import (Hierarchy, block_inverse, default_gamma, pcg, prune_block,
                              two_scale_1d)
from test_oracle_assembly import toeplitz_1d


@pytest.mark.parametrize("p", [1, 2, 3])
def test_two_scale_interior_binomial_and_identity(p):
    """Interior rows are binom(p+1, k) / 2^p (textbook subdivision); R Phi_f = Phi_c."""
    nc = 8
    bc, bf = BSpline1D(nc, p), BSpline1D(2 * nc, p)
    R1 = two_scale_1d(bc, bf)
    w = np.array([math.comb(p + 1, k) for k in range(p + 2)]) / 2 ** p
    for i in range(p, nc):                        # functions with simple knots only
        nz = np.flatnonzero(R1[i])
        np.testing.assert_allclose(R1[i, nz], w, atol=1e-14)
    x = np.random.default_rng(0).uniform(0, 1, 200)
    F = np.stack([bf.eval_global(a, x) for a in range(bf.m)])
    C = np.stack([bc.eval_global(i, x) for i in range(bc.m)])
    np.testing.assert_allclose(R1 @ F, C, atol=1e-14)
    np.testing.assert_allclose(R1.sum(0), 1.0, atol=1e-14)       # partition of unity


def test_two_scale_lagrange_identity():
    lc, lf = Lagrange1D(4, 2), Lagrange1D(8, 2)
    R1 = two_scale_1d(lc, lf)
    x = np.random.default_rng(1).uniform(0, 1, 100)
    F = np.stack([lf.eval_global(a, x) for a in range(lf.m)])
    C = np.stack([lc.eval_global(i, x) for i in range(lc.m)])
    np.testing.assert_allclose(R1 @ F, C, atol=1e-13)


@pytest.fixture(scope="module")
def disc_hier():
    geom = G.Balls([[0.52, 0.47]], [0.3])
    d = Discretization(geom, 0, 2, 32, 3, NITSCHE)
    return d, Hierarchy(d, 3)


def test_galerkin_interior_rows_equal_rediscretisation():
    """Coarse rows whose support holds only full elements equal the coarse tensor stencil."""
    d = Discretization(G.Balls([[0.3, 0.32]], [0.1]), 0, 2, 32, 1, NITSCHE)
    H = Hierarchy(d, 2)
    lev = H.lv[1]
    nc = lev.tb.n
    K, M = toeplitz_1d(2, 1.0 / nc)
    fine_full = (d.elem_class == G.FULL).reshape((d.n,) * 2, order="F")
    coarse_full = fine_full[0::2, 0::2] & fine_full[1::2, 0::2] & fine_full[0::2, 1::2] & fine_full[1::2, 1::2]
    coarse_full = coarse_full.ravel(order="F")
    pos = -np.ones(lev.tb.n_funcs, dtype=int)
    pos[lev.active] = np.arange(lev.active.size)
    A = lev.A.tocsr()
    checked = 0
    for i in range(4, nc - 2):
        for j in range(4, nc - 2):
            I = lev.tb.func_flat((i, j))
            if pos[I] < 0 or not all(coarse_full[E] for E in lev.tb.support_elems(I)):
                continue
            for ox in range(-2, 3):
                for oy in range(-2, 3):
                    J = lev.tb.func_flat((i + ox, j + oy))
                    ex = K[ox + 2] * M[oy + 2] + M[ox + 2] * K[oy + 2]
                    assert abs(A[pos[I], pos[J]] - ex) < 1e-6 * abs(K).max()
            checked += 1
    assert checked >= 40


def test_untrimmed_bspline_blocks_are_singletons(disc_hier):
    d, H = disc_hier
    lev = H.lv[3]
    sizes = {}
    for blk in lev.blocks:
        owner_full = lev.active[blk]
        sizes[len(blk)] = sizes.get(len(blk), 0) + 1
    # the deep interior has single-function blocks; every active function is in a block
    assert sizes[1] > 300
    covered = np.zeros(lev.active.size, dtype=bool)
    for blk in lev.blocks:
        covered[blk] = True
    assert covered.all() or lev.pruned > 0


def test_untrimmed_lagrange_blocks_have_size_2p_minus_1_to_d():
    """Sec. 3.4 (Remark on bases): untrimmed Lagrange blocks hold (2p-1)^d functions."""
    geom = G.Balls(np.zeros((0, 2)), np.zeros(0))
    d = Discretization(geom, 1, 2, 8, 0, NITSCHE)
    H = Hierarchy(d, 2)
    lev = H.lv[2]
    deep = [b for b in lev.blocks
            if all(2 <= k <= lev.tb.m - 3 for I in lev.active[b] for k in lev.tb.func_multi(int(I)))]
    assert deep and all(len(b) == 9 for b in deep)


def test_schwarz_relaxed_spectrum_bounded(disc_hier):
    """Eq. applyCS: lambda_max(gamma M^{-1} A) <= 1; M^{-1} SPD gives lambda_min > 0."""
    d, H = disc_hier
    for l in (3, 2):
        lev = H.lv[l]
        A = lev.A.toarray()
        Mi = lev.Minv.toarray()
        assert np.abs(Mi - Mi.T).max() <= 1e-12 * np.abs(Mi).max()
        L = np.linalg.cholesky(0.5 * (Mi + Mi.T))
        ev = np.linalg.eigvalsh(H.gamma * L.T @ A @ L)
        assert ev.max() <= 1.0 + 1e-8
        assert ev.min() > 0


def test_block_inverse_and_pruning():
    rng = np.random.default_rng(2)
    B = rng.standard_normal((5, 5))
    S = B @ B.T + 5 * np.eye(5)
    D = np.diag([1.0, 1e-9, 1.0, 1e-12, 3.0])
    A = D @ S @ D                                   # graded but S well conditioned
    Ai = block_inverse(A)
    # componentwise accuracy: D A^{-1} D is S^{-1} to working precision
    np.testing.assert_allclose((D @ Ai @ D) @ S, np.eye(5), atol=1e-13)
    _, idx, removed = prune_block(A, np.arange(5))
    # lambda ~ 1e-24 and then ~ 1e-18 (relative to the largest diagonal) go, in that order
    assert removed == 2 and list(idx) == [0, 2, 4]
    _, idx2, removed2 = prune_block(S, np.arange(5))
    assert removed2 == 0


def dense_vcycle(H, l=None):
    n = H.lv[H.L].A.shape[0]
    return np.stack([H.precondition(e) for e in np.eye(n)], axis=1)


@pytest.fixture(scope="module")
def small_hier():
    geom = G.Balls([[0.52, 0.47]], [0.3])
    d = Discretization(geom, 0, 2, 16, 2, NITSCHE)
    return d, Hierarchy(d, 2)


def test_vcycle_symmetric_and_error_propagation(small_hier):
    """B = B^T and I - B A = (I - g M^-T A)(I - R^T A_c^-1 R A)(I - g M^-1 A) (Eq. eigenMulti)."""
    d, H = small_hier
    B = dense_vcycle(H)
    assert np.abs(B - B.T).max() <= 1e-9 * np.abs(B).max()
    A = H.lv[2].A.toarray()
    Mi = H.gamma * H.lv[2].Minv.toarray()
    R = H.lv[2].R.toarray()
    Ac = H.lv[1].A.toarray()
    I = np.eye(A.shape[0])
    E = (I - Mi.T @ A) @ (I - R.T @ np.linalg.solve(Ac, R @ A)) @ (I - Mi @ A)
    # compare in the energy inner product (cut functions carry huge coefficients)
    Ah = sla.sqrtm(A).real
    lhs = Ah @ (I - B @ A) @ np.linalg.pinv(Ah)
    rhs = Ah @ E @ np.linalg.pinv(Ah)
    assert np.abs(lhs - rhs).max() < 1e-6


def test_vcycle_spectrum_in_unit_interval(small_hier):
    d, H = small_hier
    B = dense_vcycle(H)
    A = H.lv[2].A.toarray()
    L = np.linalg.cholesky(0.5 * (B + B.T))
    ev = np.linalg.eigvalsh(L.T @ A @ L)
    # B-splines need gamma = 1/(p+1)^d, which keeps lambda_min small (Sec. 3.4, end of
    # the additive Schwarz part); the invariant is 0 < lambda <= 1
    assert ev.min() > 0.0 and ev.max() <= 1.0 + 1e-8


def test_pcg_matches_direct_solve_in_energy_and_l2(disc_hier):
    d, H = disc_hier
    x, it, hist = pcg(d.A, d.b, H.precondition, 1e-10, 300)
    Ad = d.A.toarray()
    xd = sla.cho_solve(sla.cho_factor(Ad), d.b)
    e = x - xd
    assert math.sqrt(e @ Ad @ e / (xd @ Ad @ xd)) < 1e-8
    assert math.sqrt(e @ (d.M @ e) / (xd @ (d.M @ xd))) < 1e-8
    assert np.all(np.diff(np.log(hist)) < 1.0)


@pytest.mark.slow
def test_iterations_independent_of_mesh_size():
    """Sec. 4 / Sec. 5: iteration counts do not grow with the grid (same disc, 3 levels -> 5)."""
    its = []
    for n, L in ((32, 3), (64, 4), (128, 5)):
        geom = G.Balls([[0.52, 0.47]], [0.3])
        d = Discretization(geom, 0, 2, n, 0, NITSCHE)
        H = Hierarchy(d, L)
        _, it, _ = pcg(d.A, d.b, H.precondition, 1e-8, 400)
        its.append(it)
    assert max(its) - min(its) <= 0.25 * max(its), its


# ------------------------------------------------ coloured multiplicative Schwarz
@pytest.fixture(scope="module")
def mult_hier():
    geom = G.Balls([[0.52, 0.47]], [0.3])
    d = Discretization(geom, 0, 2, 16, 2, NITSCHE)
    return d, Hierarchy(d, 2, smoother="multiplicative")


def test_colour_classes_are_decoupled(mult_hier):
    """Blocks of one colour share no function and no matrix entry (Sec. 3.4: functions of
    blocks with equal colour have disjoint supports), so they do not see each other's
    residual updates; (p+1)^d = 9 colours for quadratic B-splines in 2-D."""
    d, H = mult_hier
    lev = H.lv[2]
    assert len(lev.colour_ops) == 9
    A = lev.A.tocsr()
    from oracle.multigrid import block_colour
    for col, C in enumerate(lev.colour_ops):
        # two different blocks of this colour: no common member, no coupling in A
        seen = np.zeros(C.shape[0], dtype=int)
        blocks_c = [b for b, o in zip(lev.blocks, lev.owners) if block_colour(lev.tb, o) == col]
        for k, b in enumerate(blocks_c):
            assert not seen[b].any()
            seen[b] = k + 1
        for k, b in enumerate(blocks_c):
            coupled = np.unique(A[b].indices)
            others = seen[coupled]
            assert np.all((others == 0) | (others == k + 1))


def sequential_multiplicative(A, blocks, inverses, r):
    """Eq. multiplicativeSchwarz1 taken literally: one block at a time, the residual
    updated after every block."""
    y = np.zeros_like(r)
    rt = r.copy()
    for idx, Ainv in zip(blocks, inverses):
        dy = np.zeros_like(r)
        dy[idx] = Ainv @ rt[idx]
        y += dy
        rt -= A @ dy
    return y


def test_coloured_sweep_equals_block_by_block_sweep(mult_hier):
    """The coloured sweep (residual updated once per colour) equals the block-by-block
    multiplicative Schwarz of Eq. multiplicativeSchwarz1 with the blocks in colour order,
    forward and reversed."""
    from oracle.multigrid import block_colour, block_inverse
    d, H = mult_hier
    lev = H.lv[2]
    A = lev.A.tocsr()
    colours = [block_colour(lev.tb, o) for o in lev.owners]
    order = sorted(range(len(lev.blocks)), key=lambda j: (colours[j], j))
    blocks = [lev.blocks[j] for j in order]
    invs = [block_inverse(A[b][:, b].toarray()) for b in blocks]
    r = np.random.default_rng(7).standard_normal(A.shape[0])
    fwd = sequential_multiplicative(A, blocks, invs, r)
    bwd = sequential_multiplicative(A, blocks[::-1], invs[::-1], r)
    got_f, got_b = H.smooth(2, r), H.smooth(2, r, adjoint=True)
    Ad = A.toarray()
    en = lambda v: math.sqrt(v @ Ad @ v)
    assert en(got_f - fwd) <= 1e-12 * en(fwd)
    assert en(got_b - bwd) <= 1e-12 * en(bwd)


def test_multiplicative_lagrange_p1_box_is_coloured_gauss_seidel():
    """Lagrange p = 1 without holes: every block is one function, so a forward sweep is
    point Gauss-Seidel with the unknowns ordered by colour, (D + L)^{-1} r, solved here
    by a library triangular solve."""
    geom = G.Balls(np.zeros((0, 2)), np.zeros(0))
    d = Discretization(geom, 1, 1, 8, 0, NITSCHE)
    H = Hierarchy(d, 2, smoother="multiplicative")
    lev = H.lv[2]
    assert all(b.size == 1 for b in lev.blocks) and len(lev.colour_ops) == 4
    from oracle.multigrid import block_colour
    col = np.empty(len(lev.blocks), dtype=int)
    for b, o in zip(lev.blocks, lev.owners):
        col[b[0]] = block_colour(lev.tb, o)
    perm = np.argsort(col, kind="stable")
    A = lev.A.tocsr()
    Ap = A[perm][:, perm]
    r = np.random.default_rng(3).standard_normal(A.shape[0])
    y = np.empty_like(r)
    y[perm] = spla.spsolve_triangular(sp_tril(Ap), r[perm], lower=True)
    np.testing.assert_allclose(H.smooth(2, r), y, rtol=1e-12, atol=1e-12 * np.abs(y).max())


def sp_tril(M):
    import scipy.sparse as sp
    return sp.tril(M, format="csr")


def test_multiplicative_vcycle_symmetric_error_propagation_and_spectrum(mult_hier):
    """With the reversed post-smoothing sweep the V-cycle is symmetric; its error
    propagation is E_post (I - R^T A_c^-1 R A) E_pre with E_pre = prod_c (I - B_c A) in
    colour order and E_post the reversed product (Eq. eigenMulti with M^-1 the
    multiplicative sweep); the spectrum of B A lies in (0, 1]."""
    d, H = mult_hier
    B = dense_vcycle(H)
    assert np.abs(B - B.T).max() <= 1e-9 * np.abs(B).max()
    lev = H.lv[2]
    A = lev.A.toarray()
    I = np.eye(A.shape[0])
    Epre, Epost = I.copy(), I.copy()
    for C in lev.colour_ops:
        Epre = (I - C.toarray() @ A) @ Epre
        Epost = Epost @ (I - C.toarray() @ A)
    R = lev.R.toarray()
    Ac = H.lv[1].A.toarray()
    E = Epost @ (I - R.T @ np.linalg.solve(Ac, R @ A)) @ Epre
    Ah = sla.sqrtm(A).real
    lhs = Ah @ (I - B @ A) @ np.linalg.pinv(Ah)
    rhs = Ah @ E @ np.linalg.pinv(Ah)
    assert np.abs(lhs - rhs).max() < 1e-6
    L = np.linalg.cholesky(0.5 * (B + B.T))
    ev = np.linalg.eigvalsh(L.T @ A @ L)
    assert ev.min() > 0.0 and ev.max() <= 1.0 + 1e-8


def test_multiplicative_better_conditioned_than_additive(small_hier, mult_hier):
    """Sec. 3.4: without the small relaxation parameter additive Schwarz needs, the
    multiplicative V-cycle gives a much smaller condition number of B A."""
    kappa = []
    for d, H in (small_hier, mult_hier):
        B = dense_vcycle(H)
        A = H.lv[2].A.toarray()
        L = np.linalg.cholesky(0.5 * (B + B.T))
        ev = np.linalg.eigvalsh(L.T @ A @ L)
        kappa.append(ev.max() / ev.min())
    assert kappa[1] < 0.5 * kappa[0], kappa
