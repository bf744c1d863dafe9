"""Parity at the full 512 x 512 workloads (10 discs, Lagrange p = 1 and B-splines p = 2, 3,
6 levels), in the configuration the benchmark times: the C-ABI solve from x0 = 0 to a
relative residual of 1e-8 through the captured solve graph, FP64 and mixed-precision
V-cycle, additive Schwarz (and, for p = 2, coloured multiplicative Schwarz).

The oracle cannot assemble and solve these systems in seconds, so the checks are of two
kinds:
* sampled outputs the oracle computes one by one: rows of A (assembled from the element
  systems of their support elements), entries of b, and the residual b - A x of the
  GPU solution on those rows;
* properties that hold at any size: the V-cycle B is symmetric and positive, and the
  spectrum of B A lies in (0, 1] (the error propagation of Eq. eigenMulti is a product
  S* (I - P) S with an A-orthogonal projector P, hence A-semidefinite), the FE solution
  approximates the manufactured solution, and the mixed-precision form reaches the
  residual of the FP64 form.
"""
import functools

import numpy as np
import pytest

torch = pytest.importorskip("torch")
lib = pytest.importorskip("paper_1903_10977_gb300")
from parity_utils import layout_for  # noqa: E402
from oracle import discretize as D  # noqa: E402
from oracle import geometry as G  # noqa: E402
from synthetic import random_grid_vector  # noqa: E402

pytestmark = pytest.mark.gpu
EPS = np.finfo(float).eps
NAMES = ["discs10_512_p1", "discs10_512_p2", "discs10_512_p3"]
N_RANDOM, N_CUT = 150, 150


def dev(v):
    return torch.as_tensor(np.ascontiguousarray(v), dtype=torch.float64, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


@functools.lru_cache(maxsize=2)
def oracle_rows(name: str):
    """Oracle discretisation (no global assembly) and sampled rows: random active rows
    and rows whose support holds a cut element (the assembled boundary band)."""
    pr, lay = layout_for(name)
    d = D.Discretization(G.Balls(lay.centers, lay.radii, lay.lo, lay.hi), pr.basis, pr.degree, pr.n, pr.depth, pr.bc,
                         assemble=False)
    rng = np.random.default_rng(1234)
    rand = rng.choice(d.active, N_RANDOM, replace=False)
    cut_rows = set()
    for E in rng.choice(d.cut_elems, min(N_CUT, d.cut_elems.size), replace=False):
        if d.elem_active[E]:
            dofs = [int(J) for J in d.tb.elem_dofs(int(E)) if d.func_active_full[J]]
            if dofs:
                cut_rows.add(dofs[int(rng.integers(len(dofs)))])
    rows = np.unique(np.concatenate([rand, np.array(sorted(cut_rows), dtype=np.int64)]))
    return pr, lay, d, rows, d.assemble_rows(rows)


FULL = [(n, p, 0) for n in NAMES for p in (0, 1)] + [("discs10_512_p2", p, 1) for p in (0, 1)]


@pytest.fixture(scope="module", params=FULL,
                ids=[f"{n}-{'fp64' if p == 0 else 'mixed'}{'-multiplicative' if m else ''}" for n, p, m in FULL])
def full(request):
    name, precision, smoother = request.param
    pr, lay, d, rows, A_rows = oracle_rows(name)
    S = lib.Solver(pr.dim, lay.centers, lay.radii, pr.n, pr.degree, pr.levels, pr.depth, pr.bc, basis=pr.basis,
                   lo=lay.lo, hi=lay.hi, precision=precision, smoother=smoother)
    yield precision, d, rows, A_rows, S
    S.close()


def row_dot(A_rows, I, x):
    cols, vals, _ = A_rows[int(I)]
    return float(vals @ x[cols]), float(np.abs(vals).sum() * (np.abs(x[cols]).max() if cols.size else 0.0)), cols.size


def test_full_active_set_and_rhs_rows(full):
    precision, d, rows, A_rows, S = full
    assert np.array_equal(np.flatnonzero(S.active_mask()), d.active)
    b = host(S.rhs())
    ref = np.array([A_rows[int(I)][2] for I in rows])
    scale = np.abs(b).max()
    assert np.abs(b[rows] - ref).max() <= 1e-13 * scale


def test_full_operator_rows(full):
    """Sampled rows of A x: within (4 n eps + 1e-12) ||A_i||_1 max_j |x_j| (the bound of
    the small-size parity tests)."""
    precision, d, rows, A_rows, S = full
    x = d.to_full(random_grid_vector(d.n_active, 91))
    y = host(S.apply_operator(dev(x)))
    worst = 0.0
    for I in rows:
        ref, scale, n = row_dot(A_rows, I, x)
        worst = max(worst, abs(y[I] - ref) / ((4 * n * EPS + 1e-12) * scale + 1e-300))
    assert worst <= 1.0, worst


def test_full_solve_residual_rows(full):
    """The benchmark's solve: converged to 1e-8 with the true residual recomputed in
    FP64, and on the sampled rows the oracle's b_i - A_i x is no larger than the whole
    residual may be."""
    precision, d, rows, A_rows, S = full
    b = S.rhs()
    x, res, _ = S.pcg_solve(b, rtol=1e-8, maxit=1000)
    assert res["status"] == lib.IMGM_OK and res["rel_residual"] <= 1e-8
    assert res["true_rel_residual"] <= 2e-8
    xh, bnorm = host(x), float(torch.linalg.vector_norm(b))
    r = np.array([A_rows[int(I)][2] - row_dot(A_rows, I, xh)[0] for I in rows])
    assert np.abs(r).max() <= 2e-8 * bnorm
    assert not np.any(np.delete(xh, d.active))


def test_full_solution_approximates_manufactured(full):
    """u_h at random points of Omega_h against u = sin(pi x) sin(pi y): the
    discretisation error at h = 1/512 (O(h^2) geometry, O(h^{p+1}) approximation) is
    orders of magnitude below the 1e-3 bound, which any wrong term of the system or the
    solve would exceed."""
    precision, d, rows, A_rows, S = full
    x, res, _ = S.pcg_solve(S.rhs(), rtol=1e-8, maxit=1000)
    coef = host(x)[d.active]
    rng = np.random.default_rng(5)
    P = rng.uniform(0.0, 1.0, size=(4000, 2))
    P = P[d.geom.psi(P) > 2.0 / d.n][:500]          # away from the piecewise-linear boundary
    uh = d.evaluate(coef, P)
    u = np.sin(np.pi * P[:, 0]) * np.sin(np.pi * P[:, 1])
    assert np.abs(uh - u).max() < 1e-3


def test_full_vcycle_symmetric_positive_and_bounded(full):
    """<B u, v> = <u, B v> and <B u, u> > 0 (to FP64 or FP32 rounding, measured in the
    B inner product), and the largest eigenvalue of B A, estimated by power iteration in
    the A inner product, does not exceed 1 (and is close to it: smooth modes)."""
    precision, d, rows, A_rows, S = full
    tol = 1e-11 if precision == 0 else 1e-5
    u = dev(d.to_full(random_grid_vector(d.n_active, 11)))
    v = dev(d.to_full(random_grid_vector(d.n_active, 12)))
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
