"""GPU parity of the coloured multiplicative Schwarz smoother (Sec. 3.4) and of the
V-cycle and CG solve built on it, against the FP64 CPU oracle, through the C-ABI.

Measures and tolerances as in the additive-smoother parity tests: the smoother and the
V-cycle in the energy norm (they invert block matrices), the converged solution in the
L2(Omega_h) norm of the FE function, iteration counts to 5 %."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
lib = pytest.importorskip("paper_1903_10977_gb300")
from parity_utils import energy_rel, mass_rel, oracle_for, solver_for  # noqa: E402
from oracle import multigrid as MG  # noqa: E402
from synthetic import random_grid_vector  # noqa: E402

pytestmark = pytest.mark.gpu

CASES = [
    ("disc1_32_p2", {}),
    ("discs10_512_p1", {"n": 64, "levels": 3}),
    ("discs10_512_p2", {"n": 128, "levels": 4}),
    ("discs10_512_p3", {"n": 64, "levels": 3}),
    ("spheres20_128_p2", {"n": 16, "levels": 2, "depth": 1}),
]
IDS = [f"{n}-{'-'.join(f'{k}{v}' for k, v in o.items())}" for n, o in CASES]


def dev(v):
    return torch.as_tensor(np.ascontiguousarray(v), dtype=torch.float64, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


@pytest.fixture(scope="module", params=CASES, ids=IDS)
def mult(request):
    name, ov = request.param
    pr, lay, d, H = oracle_for(name, smoother="multiplicative", **ov)
    S = solver_for(lib, pr, lay, smoother=1)
    yield pr, d, H, S
    S.close()


def test_multiplicative_smoother_every_level(mult):
    """One forward coloured sweep from zero on every level >= 2."""
    pr, d, H, S = mult
    for l in range(2, H.L + 1):
        lev = H.lv[l]
        r = random_grid_vector(lev.A.shape[0], 40 + l)
        full = np.zeros(lev.tb.n_funcs)
        full[lev.active] = r
        z = host(S.smooth(dev(full), level=l))
        ref = H.smooth(l, r)
        assert energy_rel(z[lev.active] - ref, ref, lev.A) < 1e-10
        assert not np.any(np.delete(z, lev.active))


def test_multiplicative_vcycle(mult):
    pr, d, H, S = mult
    r = random_grid_vector(d.n_active, 50)
    z = host(S.apply_preconditioner(dev(d.to_full(r))))
    ref = H.precondition(r)
    assert energy_rel(z[d.active] - ref, ref, d.A) < 1e-10


def test_multiplicative_pcg_converged(mult):
    pr, d, H, S = mult
    x, res, _ = S.pcg_solve(dev(d.to_full(d.b)), rtol=1e-8, maxit=1000)
    ref, it, _ = MG.pcg(d.A, d.b, H.precondition, rtol=1e-8, maxit=1000)
    x = host(x)[d.active]
    assert res["status"] == lib.IMGM_OK and abs(res["iterations"] - it) <= max(1, 0.05 * it)
    assert res["rel_residual"] <= 1e-8 and res["true_rel_residual"] <= 1e-7
    assert mass_rel(x - ref, ref, d.M) < (1e-10 if res["iterations"] == it else 1e-6)


@pytest.fixture(scope="module", params=CASES, ids=IDS)
def mult_mixed(request):
    name, ov = request.param
    pr, lay, d, H = oracle_for(name, smoother="multiplicative", **ov)
    S = solver_for(lib, pr, lay, smoother=1, precision=1)
    yield pr, d, H, S
    S.close()


def test_mixed_multiplicative_vcycle_and_solve(mult_mixed):
    """FP32 multiplicative V-cycle on Jacobi-scaled data: equal to the oracle's to FP32
    rounding, and the FP64 flexible CG reaches the same residual in at most 10 % more
    iterations."""
    pr, d, H, S = mult_mixed
    r = random_grid_vector(d.n_active, 51)
    z = host(S.apply_preconditioner(dev(d.to_full(r))))
    ref = H.precondition(r)
    assert energy_rel(z[d.active] - ref, ref, d.A) < 1e-4
    x, res, _ = S.pcg_solve(dev(d.to_full(d.b)), rtol=1e-8, maxit=1000)
    xr, it, _ = MG.pcg(d.A, d.b, H.precondition, rtol=1e-8, maxit=1000)
    assert res["status"] == lib.IMGM_OK and res["rel_residual"] <= 1e-8 and res["true_rel_residual"] <= 1e-7
    assert res["iterations"] <= 1.1 * it + 2
    assert mass_rel(host(x)[d.active] - xr, xr, d.M) < 1e-6
