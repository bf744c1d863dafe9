"""The 3-D sum-factorised z-marching kernel (operator apply, residual modes, the CG's
p^T A p, stored rows as tasks of their own), forced onto the small 3-D parity grids with
IMGM_TILE3D=1 (on the workloads it runs on levels of 34^3 functions and more): parity with
the oracle as for the row kernels.  With IMGM_ZM_BLOCKS=1 one block of 8 warps draws every
task from the level's counter, so each warp runs many tasks and the counter re-arms
itself between consecutive launches (as on the full-size grids).  The 32^3 case has a
level of 34^3 functions, whose restriction and prolongation take the sum-factorised
three-pass kernels (the levels of the smaller cases take the direct ones).  IMGM_ZM_FORM
fixes the FP32 instances' form (planes in registers, staged per warp, or staged per CTA),
which the setup autotuner otherwise picks, so that every form meets the oracle."""
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
         dict(n=8, levels=2, depth=1, degree=3), dict(n=16, levels=2, depth=1, degree=2, blocks=1),
         dict(n=8, levels=2, depth=1, degree=3, blocks=1), dict(n=32, levels=3, depth=0, degree=2),
         dict(n=16, levels=2, depth=1, degree=2, form=1), dict(n=16, levels=2, depth=1, degree=2, form=2),
         dict(n=16, levels=2, depth=1, degree=3, form=2, blocks=1)]


def dev(v):
    return torch.as_tensor(np.ascontiguousarray(v), dtype=torch.float64, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


@pytest.fixture(scope="module", params=CASES,
                ids=[f"p{c['degree']}-n{c['n']}" + (f"-blocks{c['blocks']}" if "blocks" in c else "")
                     + (f"-form{c['form']}" if "form" in c else "") for c in CASES])
def case(request):
    mp = pytest.MonkeyPatch()
    mp.setenv("IMGM_TILE3D", "1")
    ov = dict(request.param)
    if "blocks" in ov:
        mp.setenv("IMGM_ZM_BLOCKS", str(ov.pop("blocks")))
    if "form" in ov:                      # the FP32 apply's form: 1 warp-staged, 2 CTA-staged
        mp.setenv("IMGM_ZM_FORM", str(ov.pop("form")))
    pr, lay, d, H = oracle_for("spheres20_128_p2", **ov)
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
        y2 = host(S.apply_operator(dev(full), level=l))     # the counter re-armed itself
        assert np.array_equal(y, y2)
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


def test_tile3d_pcg_fixed_iterations(case):
    """Three CG steps from x0 = 0 (the CG's apply with p^T A p, drawn from the counter, twice
    per solve step through two solves in a row): the iterates equal the oracle's."""
    d, H, S, Sm = case
    ref, it, _ = MG.pcg(d.A, d.b, H.precondition, rtol=0.0, maxit=3)
    for _ in range(2):
        x, res, _ = S.pcg_solve(dev(d.to_full(d.b)), rtol=0.0, maxit=3)
        x = host(x)[d.active]
        assert res["iterations"] == 3 == it
        assert mass_rel(x - ref, ref, d.M) < 1e-10
        assert energy_rel(x - ref, ref, d.A) < 1e-10


def test_tile3d_restrict_and_prolong(case):
    """R r and R^T x_c on every level, entry by entry within (4 n eps) ||R_i||_1 max|x| with
    n = (p + 2)^3 (the bound of the direct kernels; the three-pass sums are shorter)."""
    d, H, S, Sm = case
    for l in range(H.L, 1, -1):
        fine, coarse = H.lv[l], H.lv[l - 1]
        R = fine.R
        n_terms = (d.p + 2) ** 3
        r = random_grid_vector(fine.active.size, 20 + l)
        full = np.zeros(fine.tb.n_funcs)
        full[fine.active] = r
        rc = host(S.restrict(dev(full), level=l))
        ref = R @ r
        absR = abs(R).tocsr()
        bound = 4 * n_terms * EPS * np.asarray(absR.sum(axis=1)).ravel() * np.abs(r).max() + 1e-300
        assert np.max(np.abs(rc[coarse.active] - ref) / bound) <= 1.0, l
        assert not np.any(np.delete(rc, coarse.active))
        xc = random_grid_vector(coarse.active.size, 30 + l)
        fullc = np.zeros(coarse.tb.n_funcs)
        fullc[coarse.active] = xc
        e = host(S.prolong(dev(fullc), level=l))
        ref = R.T @ xc
        bound = 4 * n_terms * EPS * np.asarray(absR.T.sum(axis=1)).ravel() * np.abs(xc).max() + 1e-300
        assert np.max(np.abs(e[fine.active] - ref) / bound) <= 1.0, l
        assert not np.any(np.delete(e, fine.active))
