"""The V-cycle with its finest level in FP64 and the levels below in FP32 (precision 2):
parity with the oracle's V-cycle (FP32 rounding enters only below the finest level) and
the FP64 flexible CG reaching the same residual in no more iterations than allowed for the
FP32 V-cycle."""
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
    ("spheres20_128_p2", {"n": 16, "levels": 2, "depth": 1}),
]


def dev(v):
    return torch.as_tensor(np.ascontiguousarray(v), dtype=torch.float64, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


@pytest.fixture(scope="module", params=CASES, ids=[f"{n}-{'-'.join(f'{k}{v}' for k, v in o.items())}" for n, o in CASES])
def hybrid(request):
    name, ov = request.param
    pr, lay, d, H = oracle_for(name, **ov)
    S = solver_for(lib, pr, lay, precision=2)
    yield d, H, S
    S.close()


def test_hybrid_vcycle_matches_oracle(hybrid):
    d, H, S = hybrid
    r = random_grid_vector(d.n_active, 71)
    ref = H.precondition(r)
    z = host(S.apply_preconditioner(dev(d.to_full(r))))
    assert energy_rel(z[d.active] - ref, ref, d.A) < 1e-4
    assert not np.any(np.delete(z, d.active))


def test_hybrid_solve(hybrid):
    d, H, S = hybrid
    x, res, _ = S.pcg_solve(dev(d.to_full(d.b)), rtol=1e-8, maxit=1000)
    ref, it, _ = MG.pcg(d.A, d.b, H.precondition, rtol=1e-8, maxit=1000)
    assert res["status"] == lib.IMGM_OK and res["rel_residual"] <= 1e-8 and res["true_rel_residual"] <= 1e-7
    assert res["iterations"] <= 1.1 * it + 2
    assert mass_rel(host(x)[d.active] - ref, ref, d.M) < 1e-6
