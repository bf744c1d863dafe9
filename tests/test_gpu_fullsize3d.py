"""Parity at the full 3-D workload the benchmark times: 128^3 background grid, the unit cube
minus 20 seeded spheres, quadratic B-splines, depth-2 cut-cell quadrature, 5 levels
(1,965,303 active functions), FP64 and mixed-precision V-cycle, in the benchmark's launch
configuration (the solve graph; the CG's p^T A p apply draws its tiles from the dynamic
tile counter here, since the grid has 10,725 tiles).

The oracle cannot assemble this system at all (its cut-cell quadrature alone would take
hours), so its rows come from oracle.discretize.LocalRows, which integrates only the
elements in a sampled row's support:
* sampled rows of A x and entries of b, random rows and rows at cut elements;
* the residual b - A x of the GPU solution on those rows;
* properties that hold at any size: the V-cycle is symmetric and positive, the spectrum
  of B A lies in (0, 1] (Eq. eigenMulti), and u_h approximates the manufactured solution.
"""
import functools

import numpy as np
import pytest

torch = pytest.importorskip("torch")
lib = pytest.importorskip("paper_1903_10977_gb300")
from parity_utils import layout_for  # noqa: E402
from oracle import geometry as G  # noqa: E402
from oracle.discretize import LocalRows  # noqa: E402
from synthetic import random_grid_vector  # noqa: E402

pytestmark = pytest.mark.gpu
EPS = np.finfo(float).eps
NAME = "spheres20_128_p2"
N_RANDOM, N_CUT = 100, 30


def dev(v):
    return torch.as_tensor(np.ascontiguousarray(v), dtype=torch.float64, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


@functools.lru_cache(maxsize=1)
def oracle_rows():
    """Sampled full-grid rows (seeded: random grid rows and one function of each of a few
    cut elements) with the oracle's rows, right-hand side entries and activity."""
    pr, lay = layout_for(NAME)
    loc = LocalRows(G.Balls(lay.centers, lay.radii, lay.lo, lay.hi), pr.basis, pr.degree, pr.n, pr.depth, pr.bc)
    rng = np.random.default_rng(4321)
    rand = rng.choice(loc.tb.n_funcs, N_RANDOM, replace=False)
    cut = []
    for E in rng.choice(loc.cut_elems, N_CUT, replace=False):
        dofs = loc.tb.elem_dofs(int(E))
        cut.append(int(dofs[int(rng.integers(len(dofs)))]))
    rows = np.unique(np.concatenate([rand, np.array(cut, dtype=np.int64)]))
    A_rows = loc.assemble_rows(rows)
    active = np.array([A_rows[int(I)][0].size > 0 for I in rows])
    return pr, lay, loc, rows, A_rows, active


@pytest.fixture(scope="module", params=[0, 1], ids=["fp64", "mixed"])
def full(request):
    pr, lay, loc, rows, A_rows, active = oracle_rows()
    S = lib.Solver(pr.dim, lay.centers, lay.radii, pr.n, pr.degree, pr.levels, pr.depth, pr.bc, basis=pr.basis,
                   lo=lay.lo, hi=lay.hi, precision=request.param)
    yield request.param, loc, rows, A_rows, active, S
    S.close()


def row_dot(A_rows, I, x):
    cols, vals, _ = A_rows[int(I)]
    return float(vals @ x[cols]), float(np.abs(vals).sum() * (np.abs(x[cols]).max() if cols.size else 0.0)), cols.size


def test_full3d_activity_and_rhs_rows(full):
    precision, loc, rows, A_rows, active, S = full
    assert active.sum() > 0.7 * rows.size and (~active).sum() > 0      # both kinds sampled
    mask = S.active_mask().astype(bool)
    assert np.array_equal(mask[rows], active)
    b = host(S.rhs())
    ref = np.array([A_rows[int(I)][2] for I in rows])
    assert np.abs(b[rows] - ref).max() <= 1e-13 * np.abs(b).max()


def test_full3d_operator_rows(full):
    """Sampled rows of A x within (4 n eps + 1e-12) ||A_i||_1 max_j |x_j|, for two
    consecutive applies (the second after the tile counters re-armed themselves)."""
    precision, loc, rows, A_rows, active, S = full
    mask = S.active_mask().astype(float)
    x = random_grid_vector(mask.size, 93) * mask
    xd = dev(x)
    for _ in range(2):
        y = host(S.apply_operator(xd))
        worst = 0.0
        for I in rows:
            ref, scale, n = row_dot(A_rows, I, x)
            worst = max(worst, abs(y[I] - ref) / ((4 * n * EPS + 1e-12) * scale + 1e-300))
        assert worst <= 1.0, worst


def test_full3d_solve_residual_rows(full):
    """The benchmark's solve reaches 1e-8 with the true residual recomputed in FP64, and on
    the sampled rows the oracle's b_i - A_i x is no larger than the whole residual may be
    (plus the rounding of the row product)."""
    precision, loc, rows, A_rows, active, S = full
    b = S.rhs()
    x, res, _ = S.pcg_solve(b, rtol=1e-8, maxit=2000)
    assert res["status"] == lib.IMGM_OK and res["rel_residual"] <= 1e-8
    assert res["true_rel_residual"] <= 2e-8
    xh, bnorm = host(x), float(torch.linalg.vector_norm(b))
    for I in rows:
        ref, scale, n = row_dot(A_rows, I, xh)
        assert abs(A_rows[int(I)][2] - ref) <= 2e-8 * bnorm + 4 * n * EPS * scale
    assert not np.any(xh[rows[~active]])


def test_full3d_solution_approximates_manufactured(full):
    """u_h at random points well inside Omega against u = sin(pi x) sin(pi y) sin(pi z):
    at h = 1/128 the error is orders of magnitude below the 1e-3 bound, which any wrong
    term of the system or the solve would exceed."""
    precision, loc, rows, A_rows, active, S = full
    x, res, _ = S.pcg_solve(S.rhs(), rtol=1e-8, maxit=2000)
    coef = host(x)
    rng = np.random.default_rng(6)
    P = rng.uniform(0.0, 1.0, size=(3000, 3))
    P = P[loc.geom.psi(P) > 2.0 / loc.n][:300]
    e = np.clip(np.floor(P / loc.h).astype(int), 0, loc.n - 1)
    E = np.ravel_multi_index(tuple(e.T), (loc.n,) * 3, order="F")
    uh = np.empty(len(P))
    for k in range(len(P)):
        vals, _ = loc.tb.eval(int(E[k]), P[k:k + 1])
        uh[k] = coef[loc.tb.elem_dofs(int(E[k]))] @ vals[:, 0]
    u = np.prod(np.sin(np.pi * P), axis=1)
    assert np.abs(uh - u).max() < 1e-3


def test_full3d_vcycle_symmetric_positive_and_bounded(full):
    """<B u, v> = <u, B v>, <B u, u> > 0, and the largest eigenvalue of B A (power iteration
    in the A inner product) in (0.9, 1].  u and v are residuals A w of random w: the class
    of vectors the CG hands the V-cycle.  (The FP32 V-cycle works on Jacobi-scaled data,
    r / sqrt(A_ii); an O(1) entry on a function whose cut support makes A_ii tiny would
    leave the FP32 range there, while a residual's entry scales with its row.)"""
    precision, loc, rows, A_rows, active, S = full
    tol = 1e-11 if precision == 0 else 1e-5
    mask = S.active_mask().astype(float)
    u = S.apply_operator(dev(random_grid_vector(mask.size, 11) * mask))
    v = S.apply_operator(dev(random_grid_vector(mask.size, 12) * mask))
    Bu, Bv = S.apply_preconditioner(u), S.apply_preconditioner(v)
    buu, bvv = float(Bu @ u), float(Bv @ v)
    assert buu > 0 and bvv > 0
    assert abs(float(Bu @ v) - float(u @ Bv)) <= tol * np.sqrt(buu * bvv)
    w = u.clone()
    lam = 0.0
    for _ in range(30):
        Aw = S.apply_operator(w)
        BAw = S.apply_preconditioner(Aw)
        lam = float(Aw @ BAw) / float(Aw @ w)
        w = BAw / torch.sqrt(BAw @ S.apply_operator(BAw))
    assert 0.9 < lam <= 1.0 + (1e-10 if precision == 0 else 1e-4), lam
