"""The no-allocation residual norm (imgm_residual_norm2_noalloc).

It exists for callers that cannot allocate device memory while they run (a caching
allocator holds the GPU's memory, or a latency-critical loop cannot pay for
cudaMalloc's device-wide synchronisation).  Its result must equal that of the
allocating entry point imgm_residual_norm2 on two calls in a row, with different
inputs, so that nothing left in the shared static scratch leaks from one call to the
next.  This file sorts last so that a run stopping at the first failure has run
everything else.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
lib = pytest.importorskip("paper_1903_10977_gb300")
from synthetic import config_layout, preset, random_grid_vector  # noqa: E402

pytestmark = pytest.mark.gpu


def test_no_alloc_residual_norm_matches_allocating_entry_point():
    pr = preset("discs10_512_p2")
    lay = config_layout(pr.layout, 0)
    S = lib.Solver(pr.dim, lay.centers, lay.radii, pr.n, pr.degree, pr.levels, pr.depth, pr.bc)
    mask = torch.as_tensor(S.active_mask(), dtype=torch.float64, device="cuda")
    b = S.rhs()
    out = torch.empty(1, dtype=torch.float64, device="cuda")       # caller-owned output
    for call in range(2):
        x = torch.as_tensor(random_grid_vector(S.n_grid(), 100 + call), device="cuda") * mask
        bb = b * (1.0 + call)
        ref = float(S.residual_norm2(bb, x).item())
        got = float(S.residual_norm2_noalloc(bb, x, out).item())
        # the same kernels and summation order: equal to the tolerance of the residual-norm parity test
        assert abs(got - ref) <= 1e-12 * ref, (call, got, ref)
    S.close()


def test_no_alloc_second_problem_and_device_memory():
    """After calls on a 512^2 problem, a smaller problem (other row count and mask) gets its
    own residual norm from the shared array, with nothing stale from the earlier calls; and
    the calls leave the device's free memory unchanged (no allocation behind them)."""
    pr = preset("discs10_512_p2")
    lay = config_layout(pr.layout, 0)
    big = lib.Solver(pr.dim, lay.centers, lay.radii, pr.n, pr.degree, pr.levels, pr.depth, pr.bc)
    pr2 = preset("disc1_32_p2")
    lay2 = config_layout(pr2.layout, 0)
    small = lib.Solver(pr2.dim, lay2.centers, lay2.radii, pr2.n, pr2.degree, pr2.levels, pr2.depth, pr2.bc)
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    inputs = []
    for S, seed in ((big, 7), (small, 8)):
        mask = torch.as_tensor(S.active_mask(), dtype=torch.float64, device="cuda")
        inputs.append((S, S.rhs(), torch.as_tensor(random_grid_vector(S.n_grid(), seed), device="cuda") * mask))
    refs = [float(S.residual_norm2(b, x).item()) for S, b, x in inputs]
    S, b, x = inputs[0]
    S.residual_norm2_noalloc(b, x, out)            # the first call on the device looks up the array
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for (S, b, x), ref in zip(inputs, refs):
        got = float(S.residual_norm2_noalloc(b, x, out).item())
        assert abs(got - ref) <= 1e-12 * ref, (got, ref)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    small.close()
    big.close()


def test_no_alloc_rejects_grids_beyond_its_scratch():
    # 1024 x 1024 quadratic B-splines: 1026^2 rows, more than the 2^19 the scratch holds
    S = lib.Solver(2, np.zeros((0, 2)), np.zeros(0), 1024, 2, 6, 0, 1)
    b = torch.zeros(S.n_grid(), dtype=torch.float64, device="cuda")
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    with pytest.raises(lib.ImgmError, match="more than the static scratch holds"):
        S.residual_norm2_noalloc(b, b, out)
    S.close()
