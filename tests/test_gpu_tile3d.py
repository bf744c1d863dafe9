"""The 3-D sum-factorised tile kernels (operator apply, residual modes, the CG's p^T A p),
forced onto the small 3-D parity grids with IMGM_TILE3D=1 (on the workloads they run on
levels with at least one tile per SM): parity with the oracle as for the row kernels."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
lib = pytest.importorskip("paper_1903_10977_gb300")
from parity_utils import energy_rel, mass_rel, oracle_for, solver_for  # noqa: E402
from oracle import multigrid as MG  # noqa: E402
from synthetic import random_grid_vector  # noqa: E402

pytestmark = pytest.mark.gpu
EPS = np.finfo(float).eps
CASES = [dict(n=16, levels=2, depth=1, degree=2), dict(n=8, levels=2, depth=1, degree=1),
         dict(n=8, levels=2, depth=1, degree=3)]


def dev(v):
    return torch.as_tensor(np.ascontiguousarray(v), dtype=torch.float64, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


@pytest.fixture(scope="module", params=CASES, ids=[f"p{c['degree']}-n{c['n']}" for c in CASES])
def case(request):
    mp = pytest.MonkeyPatch()
    mp.setenv("IMGM_TILE3D", "1")
    pr, lay, d, H = oracle_for("spheres20_128_p2", **request.param)
    S = solver_for(lib, pr, lay, precision=0)
    Sm = solver_for(lib, pr, lay, precision=1)
    yield d, H, S, Sm
    S.close()
    Sm.close()
    mp.undo()


def test_tile3d_apply_every_level(case):
    d, H, S, Sm = case
    for l in range(1, H.L + 1):
        lev = H.lv[l]
        x = random_grid_vector(lev.A.shape[0], 80 + l)
        full = np.zeros(lev.tb.n_funcs)
        full[lev.active] = x
        y = host(S.apply_operator(dev(full), level=l))
        ref = lev.A @ x
        absA = abs(lev.A).tocsr()
        xmax = absA.sign().multiply(np.abs(x)[None, :]).max(axis=1).toarray().ravel()
        n = np.diff(absA.indptr)
        bound = (4 * n * EPS + 1e-12) * np.asarray(absA.sum(axis=1)).ravel() * xmax + 1e-300
        assert np.max(np.abs(y[lev.active] - ref) / bound) <= 1.0
        assert not np.any(np.delete(y, lev.active))


def test_tile3d_vcycle_and_solve(case):
    d, H, S, Sm = case
    r = random_grid_vector(d.n_active, 90)
    ref = H.precondition(r)
    z = host(S.apply_preconditioner(dev(d.to_full(r))))
    assert energy_rel(z[d.active] - ref, ref, d.A) < 1e-10
    zm = host(Sm.apply_preconditioner(dev(d.to_full(r))))
    assert energy_rel(zm[d.active] - ref, ref, d.A) < 1e-4
    xr, it, _ = MG.pcg(d.A, d.b, H.precondition, rtol=1e-8, maxit=1000)
    for solver in (S, Sm):
        x, res, _ = solver.pcg_solve(dev(d.to_full(d.b)), rtol=1e-8, maxit=1000)
        assert res["status"] == lib.IMGM_OK and res["rel_residual"] <= 1e-8 and res["true_rel_residual"] <= 1e-7
        assert res["iterations"] <= 1.1 * it + 2
        assert mass_rel(host(x)[d.active] - xr, xr, d.M) < 1e-6
