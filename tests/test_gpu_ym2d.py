"""The 2-D sum-factorised y-marching kernel (operator apply, residual modes, the CG's
p^T A p, stored rows as tasks of 32), an option (IMGM_YM2D=1) beside the 2-D tile kernel,
which measures faster on the 512^2 levels: put onto every level of small 2-D parity grids,
parity with the oracle as for the row kernels.  With IMGM_ZM_BLOCKS=1 one block of 8 warps
draws every task from the level's counter, so each warp runs many tasks and the counter
re-arms itself between consecutive launches."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
lib = pytest.importorskip("paper_1903_10977_gb300")
from parity_utils import energy_rel, mass_rel, oracle_for, solver_for  # noqa: E402
from oracle import multigrid as MG  # noqa: E402
from synthetic import random_grid_vector  # noqa: E402

pytestmark = pytest.mark.gpu
EPS = np.finfo(float).eps
CASES = [dict(name="discs10_512_p2", n=64, levels=3, depth=1),
         dict(name="discs10_512_p2", n=32, levels=2, depth=1),
         dict(name="discs10_512_p1", n=32, levels=2, depth=1),
         dict(name="discs10_512_p3", n=32, levels=2, depth=1),
         dict(name="discs10_512_p2", n=64, levels=2, depth=1, blocks=1),
         dict(name="discs10_512_p3", n=32, levels=2, depth=1, blocks=1),
         dict(name="disc1_32_p2", n=32, levels=3, depth=3)]


def dev(v):
    return torch.as_tensor(np.ascontiguousarray(v), dtype=torch.float64, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def _id(c):
    return f"{c['name'].split('_')[0]}-p{c['name'][-1]}-n{c['n']}" + (f"-blocks{c['blocks']}" if "blocks" in c else "")


@pytest.fixture(scope="module", params=CASES, ids=[_id(c) for c in CASES])
def case(request):
    mp = pytest.MonkeyPatch()
    ov = dict(request.param)
    mp.setenv("IMGM_YM2D", "1")
    if "blocks" in ov:
        mp.setenv("IMGM_ZM_BLOCKS", str(ov.pop("blocks")))
    name = ov.pop("name")
    pr, lay, d, H = oracle_for(name, **ov)
    S = solver_for(lib, pr, lay, precision=0)
    Sm = solver_for(lib, pr, lay, precision=1)
    yield d, H, S, Sm
    S.close()
    Sm.close()
    mp.undo()


def test_ym2d_apply_every_level(case):
    """A x on every level, entry by entry within (4 n eps) sum_j |A_ij| max|x_j| over the
    row's n nonzeros; a second launch (the counter re-armed) gives the same bits."""
    d, H, S, Sm = case
    for l in range(1, H.L + 1):
        lev = H.lv[l]
        x = random_grid_vector(lev.A.shape[0], 80 + l)
        full = np.zeros(lev.tb.n_funcs)
        full[lev.active] = x
        y = host(S.apply_operator(dev(full), level=l))
        y2 = host(S.apply_operator(dev(full), level=l))
        assert np.array_equal(y, y2)
        ref = lev.A @ x
        absA = abs(lev.A).tocsr()
        xmax = absA.sign().multiply(np.abs(x)[None, :]).max(axis=1).toarray().ravel()
        n = np.diff(absA.indptr)
        bound = (4 * n * EPS + 1e-12) * np.asarray(absA.sum(axis=1)).ravel() * xmax + 1e-300
        assert np.max(np.abs(y[lev.active] - ref) / bound) <= 1.0
        assert not np.any(np.delete(y, lev.active))


def test_ym2d_vcycle_and_solve(case):
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


def test_ym2d_pcg_fixed_iterations(case):
    """Three CG steps from x0 = 0 (the finest apply with p^T A p in the same launch), twice in
    a row: the iterates equal the oracle's."""
    d, H, S, Sm = case
    ref, it, _ = MG.pcg(d.A, d.b, H.precondition, rtol=0.0, maxit=3)
    for _ in range(2):
        x, res, _ = S.pcg_solve(dev(d.to_full(d.b)), rtol=0.0, maxit=3)
        x = host(x)[d.active]
        assert res["iterations"] == 3 == it
        assert mass_rel(x - ref, ref, d.M) < 1e-10
        assert energy_rel(x - ref, ref, d.A) < 1e-10
