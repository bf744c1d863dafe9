"""Batched solves: several contexts (different problems, and clones of one problem for
more right-hand sides) solved concurrently by one graph launch.  Every solve of the batch
must match the oracle's CG on the same system (as in the single-solve parity tests) and
the same context's own single solve."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
lib = pytest.importorskip("paper_1903_10977_gb300")
from parity_utils import mass_rel, oracle_for, solver_for  # noqa: E402
from oracle import multigrid as MG  # noqa: E402

pytestmark = pytest.mark.gpu

PROBLEMS = [
    ("disc1_32_p2", {}, {"precision": 0}),
    ("discs10_512_p1", {"n": 64, "levels": 3}, {"precision": 1}),
    ("discs10_512_p2", {"n": 128, "levels": 4}, {"precision": 1}),
    ("discs10_512_p3", {"n": 64, "levels": 3}, {"precision": 0, "smoother": 1}),
    ("spheres20_128_p2", {"n": 16, "levels": 2, "depth": 1}, {"precision": 1}),
    ("spheres20_128_p2", {"n": 16, "levels": 3, "depth": 1, "degree": 1}, {"precision": 1}),
    ("spheres20_128_p2", {"n": 8, "levels": 2, "depth": 1, "degree": 3}, {"precision": 0}),
]
# 3-D members with up to eight right-hand sides (clones of one problem), 2-D ones with 1-3
RHS_PER_PROBLEM = [1, 3, 2, 1, 8, 4, 2]


def dev(v):
    return torch.as_tensor(np.ascontiguousarray(v), dtype=torch.float64, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


@pytest.fixture(scope="module")
def batch():
    entries = []          # (oracle disc, oracle hierarchy, context, right-hand side (active numbering))
    keep = []
    for (name, ov, kw), nrhs in zip(PROBLEMS, RHS_PER_PROBLEM):
        smoother = "multiplicative" if kw.get("smoother", 0) == 1 else "additive"
        pr, lay, d, H = oracle_for(name, smoother=smoother, **ov)
        S = solver_for(lib, pr, lay, **kw)
        keep.append(S)
        rng = np.random.default_rng(len(entries))
        for k in range(nrhs):
            ctx = S if k == 0 else S.clone()
            b = d.b if k == 0 else rng.standard_normal(d.n_active)      # random-normal right-hand sides
            entries.append((d, H, ctx, b))
    B = lib.Batch([e[2] for e in entries])
    bs = [dev(e[0].to_full(e[3])) for e in entries]
    xs, results = B.solve(bs, rtol=1e-8, maxit=1000)
    yield entries, bs, [host(x) for x in xs], results
    B.close()
    for _, _, ctx, _ in entries:
        ctx.close()


def test_batch_matches_oracle(batch):
    """Random-normal right-hand sides put O(1) weight on functions with tiny cut supports,
    whose solution coefficients are then of the size of 1/A_ii: the true residual of any
    FP64 iterate then stalls at eps ||A|| ||x|| above the recursively updated one, so it is
    compared with the oracle's own true residual for the same system."""
    entries, bs, xs, results = batch
    for (d, H, ctx, b), x, res in zip(entries, xs, results):
        ref, it, _ = MG.pcg(d.A, b, H.precondition, rtol=1e-8, maxit=1000)
        ref_true = np.linalg.norm(b - d.A @ ref) / np.linalg.norm(b)
        assert res["status"] == lib.IMGM_OK and res["rel_residual"] <= 1e-8
        assert res["true_rel_residual"] <= max(1e-7, 10 * ref_true), (res["true_rel_residual"], ref_true)
        assert res["iterations"] <= 1.1 * it + 2 and res["iterations"] >= 0.9 * it - 2
        assert mass_rel(x[d.active] - ref, ref, d.M) < 1e-6
        assert res["kernel_launches"] > 5 * res["iterations"]


def test_batch_matches_single_solves(batch):
    """The same context solved alone (its own graph) converges in the same number of
    iterations (to within one) to the same solution, to the accuracy of the stopping test:
    the Schwarz scatter's atomic adds and the 3-D apply's dynamic task order make the
    rounding of two runs differ, so the iterates are not bitwise equal (1e-7 in
    L2(Omega_h), as for converged solutions in the single-solve parity tests)."""
    entries, bs, xs, results = batch
    for (d, H, ctx, b), bd, x, res in zip(entries, bs, xs, results):
        xs1, r1, _ = ctx.pcg_solve(bd, rtol=1e-8, maxit=1000)
        assert abs(r1["iterations"] - res["iterations"]) <= 1
        assert mass_rel(host(xs1)[d.active] - x[d.active], x[d.active], d.M) < 1e-7


def test_clone_outlives_its_source():
    pr, lay, d, H = oracle_for("disc1_32_p2")
    S = solver_for(lib, pr, lay)
    C = S.clone()
    b = dev(d.to_full(d.b))
    x0, r0, _ = S.pcg_solve(b, rtol=1e-8, maxit=500)
    S.close()                             # the shared tables stay alive for the clone
    x1, r1, _ = C.pcg_solve(b, rtol=1e-8, maxit=500)
    assert r1["iterations"] == r0["iterations"]
    assert mass_rel(host(x1)[d.active] - host(x0)[d.active], host(x0)[d.active], d.M) < 1e-12
    C.close()


def test_batch_rejects_repeated_context():
    pr, lay, d, H = oracle_for("disc1_32_p2")
    S = solver_for(lib, pr, lay)
    with pytest.raises(lib.ImgmError):
        lib.Batch([S, S])
    with pytest.raises(lib.ImgmError):
        lib.Batch([])
    S.close()
