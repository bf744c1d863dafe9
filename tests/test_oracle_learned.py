"""Pins of the learned-correction oracle against library routines, closed forms and
invariants (no GPU).

* bfloat16 rounding: torch's float32 -> bfloat16 conversion (round to nearest even) and
  hand-checked ties;
* one convolution layer: scipy.ndimage.correlate with zero padding, per channel pair;
* the input gradient is the adjoint of the layer (<conv x, y> = <x, conv^T y>);
* the loss gradient: central finite differences of the loss in every layer;
* Adam's first step moves each weight by lr g / (|g| + eps) (closed form);
* the stage: exact error in, exact solution out (omega = 1); zero network, z unchanged;
  never a larger A-norm error than the V-cycle alone;
* flexible CG with a fixed SPD preconditioner takes the iterations of standard PCG
  (Polak-Ribiere = Fletcher-Reeves beta in exact arithmetic) and reaches the dense solve;
  FCG(m) for any m gives the PCG iterates then (the directions are A-conjugate already),
  and it converges with a preconditioner that varies from step to step;
* training pairs: e1 = (I - B A) e0 with B assembled column by column from the V-cycle.
"""
import numpy as np
import pytest
import scipy.ndimage as ndi
import scipy.sparse as sp

from oracle import learned as NL
from synthetic import initial_weights

torch = pytest.importorskip("torch")


def test_round_bf16_matches_torch_and_ties():
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.standard_normal(4000) * 10.0 ** rng.integers(-8, 8, 4000), [0.0, 1.0, -2.5]])
    x32 = x.astype(np.float32)
    ref = torch.from_numpy(x32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(NL.round_bf16(x32.astype(np.float64)), ref)
    # ties: 1 + 2^-8 lies halfway between 1 and 1 + 2^-7 (odd) -> 1; 1 + 3 2^-8 -> 1 + 2^-6
    assert NL.round_bf16(1.0 + 2.0 ** -8) == 1.0
    assert NL.round_bf16(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6
    assert NL.round_bf16(-(1.0 + 3 * 2.0 ** -8)) == -(1.0 + 2.0 ** -6)


def test_conv_layer_is_zero_padded_correlation():
    rng = np.random.default_rng(1)
    ci, co = 3, 2
    x = rng.standard_normal((ci, 5, 6, 7))
    W = rng.standard_normal((27, co, ci))
    y = NL.conv3d(x, W)
    for o in range(co):
        ref = np.zeros(x.shape[1:])
        for i in range(ci):
            k = W[:, o, i].reshape(3, 3, 3)            # [dz+1, dy+1, dx+1]
            ref += ndi.correlate(x[i], k, mode="constant", cval=0.0)
        assert np.allclose(y[o], ref, rtol=1e-13, atol=1e-13)


def test_conv_input_grad_is_adjoint():
    rng = np.random.default_rng(2)
    x = rng.standard_normal((4, 5, 4, 6))
    W = rng.standard_normal((27, 3, 4))
    dy = rng.standard_normal((3, 5, 4, 6))
    lhs = float(np.sum(NL.conv3d(x, W) * dy))
    rhs = float(np.sum(x * NL.conv3d_input_grad(dy, W)))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
    # the weight gradient is the derivative of the same bilinear form in W
    G = NL.conv3d_weight_grad(dy, x)
    assert abs(float(np.sum(G * W)) - lhs) <= 1e-12 * abs(lhs)


def test_loss_gradient_matches_finite_differences():
    rng = np.random.default_rng(3)
    shape = (5, 6, 7)
    mask = (rng.random(shape) < 0.8).astype(float)
    r = rng.standard_normal(shape) * mask
    e = rng.standard_normal(shape) * mask
    w = initial_weights(4) * 3.0
    scale = 1.0 / mask.sum()
    L0, g = NL.loss_and_grads(w, r, e, mask, scale, bf16=False)
    assert L0 > 0
    offsets = [0, 432, 432 + 6912]
    picks = np.concatenate([o + rng.choice(n, 12, replace=False) for o, n in zip(offsets, (432, 6912, 432))])
    h = 1e-6
    for k in picks:
        wp, wm = w.copy(), w.copy()
        wp[k] += h
        wm[k] -= h
        fd = (NL.loss_and_grads(wp, r, e, mask, scale, bf16=False)[0]
              - NL.loss_and_grads(wm, r, e, mask, scale, bf16=False)[0]) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(abs(g).max(), 1e-12), (k, fd, g[k])


def test_input_scale_is_homogeneous():
    """No biases and ReLU: N(a r) = a N(r) for a > 0 (exact forward), so the stage's step
    omega makes any input scale irrelevant."""
    rng = np.random.default_rng(12)
    shape = (4, 5, 6)
    mask = (rng.random(shape) < 0.7).astype(float)
    r = rng.standard_normal(shape)
    w = initial_weights(13)
    a, _ = NL.forward(w, r, mask, bf16=False, in_scale=8.0)
    b, _ = NL.forward(w, r, mask, bf16=False)
    assert np.allclose(a, 8.0 * b, rtol=1e-12, atol=1e-14)


def test_forward_bf16_rounds_only_where_stored():
    """With weights and data exactly representable in bfloat16 and small enough that no
    sum needs more than 8 bits, the bf16 and the exact forward agree exactly."""
    rng = np.random.default_rng(5)
    shape = (4, 5, 6)
    mask = np.ones(shape)
    r = rng.integers(-2, 3, shape) / 4.0
    w = np.zeros(NL.N_WEIGHTS)
    w[:432] = rng.integers(-1, 2, 432) / 8.0
    w[432:432 + 6912] = np.where(rng.random(6912) < 0.01, rng.integers(-1, 2, 6912) / 8.0, 0.0)
    w[432 + 6912:] = np.where(rng.random(432) < 0.05, 1.0 / 8.0, 0.0)
    a, _ = NL.forward(w, r, mask, bf16=True)
    b, _ = NL.forward(w, r, mask, bf16=False)
    assert np.array_equal(a, b)


def test_adam_first_step_closed_form():
    rng = np.random.default_rng(6)
    w = rng.standard_normal(50)
    g = rng.standard_normal(50)
    opt = NL.Adam(50, lr=1e-2, eps=1e-8)
    w1 = opt.step(w, g)
    assert np.allclose(w - w1, 1e-2 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=0)
    # and it minimises a separable quadratic
    target = rng.standard_normal(50)
    opt = NL.Adam(50, lr=0.05)
    x = np.zeros(50)
    for _ in range(2000):
        x = opt.step(x, 2 * (x - target))
    assert np.abs(x - target).max() < 1e-3


def _spd(n, seed):
    rng = np.random.default_rng(seed)
    M = rng.standard_normal((n, n))
    return sp.csr_matrix(M @ M.T + n * np.eye(n))


def test_stage_closed_forms():
    A = _spd(30, 7)
    Ad = A.toarray()
    rng = np.random.default_rng(8)
    r = rng.standard_normal(30)
    z = 0.3 * r
    exact = np.linalg.solve(Ad, r)
    zs, om = NL.stage(A, r, z, lambda r1: np.linalg.solve(Ad, r1))
    assert abs(om - 1.0) < 1e-12 and np.allclose(zs, exact, rtol=1e-12, atol=1e-12)
    zs, om = NL.stage(A, r, z, lambda r1: np.zeros_like(r1))
    assert om == 0.0 and np.array_equal(zs, z)
    # any proposal: the A-norm error of the correction equation does not grow
    for s in range(5):
        c = np.random.default_rng(s).standard_normal(30)
        zs, _ = NL.stage(A, r, z, lambda r1, c=c: c)
        ea, eb = zs - exact, z - exact
        assert ea @ Ad @ ea <= eb @ Ad @ eb * (1 + 1e-12)


def test_flexible_cg_reduces_to_pcg_for_fixed_preconditioner():
    from oracle.multigrid import pcg
    A = _spd(60, 9)
    D = sp.diags(1.0 / A.diagonal())
    b = np.random.default_rng(10).standard_normal(60)
    x1, k1, _ = NL.flexible_pcg(A, b, lambda r: D @ r, rtol=1e-10)
    x2, k2, _ = pcg(A, b, lambda r: D @ r, rtol=1e-10)
    assert k1 == k2
    ref = np.linalg.solve(A.toarray(), b)
    assert np.linalg.norm(x1 - ref) <= 1e-8 * np.linalg.norm(ref)


def test_training_pair_is_vcycle_error_propagation():
    from parity_utils import oracle_for
    pr, lay, d, H = oracle_for("disc1_32_p2", n=8, levels=2, depth=1)
    A = d.A
    n = A.shape[0]
    B = np.column_stack([H.precondition(np.eye(n)[:, j]) for j in range(n)])
    e0 = np.random.default_rng(11).standard_normal(n)
    r1, e1 = NL.training_pair(A, H.precondition, e0)
    e_ref = e0 - B @ (A @ e0)
    s = np.sqrt(np.mean(e_ref ** 2))
    assert np.allclose(e1, e_ref / s, rtol=1e-10, atol=1e-12)
    assert np.allclose(r1, (A @ e_ref) / s, rtol=1e-10, atol=1e-10)
    # the set's input scale is the reciprocal of the mean rms of its residuals
    assert abs(NL.input_scale([(r1, e1), (2 * r1, e1)]) - 1.0 / (1.5 * np.sqrt(np.mean(r1 ** 2)))) < 1e-12
    # the V-cycle is a contraction in the A-norm: the pair's error is smaller than e0's
    assert e_ref @ (A @ e_ref) < e0 @ (A @ e0)


def test_fcg_reduces_to_pcg_and_keeps_m_directions_conjugate():
    from oracle.multigrid import pcg
    A = _spd(60, 14)
    D = sp.diags(1.0 / A.diagonal())
    b = np.random.default_rng(15).standard_normal(60)
    x2, k2, h2 = pcg(A, b, lambda r: D @ r, rtol=1e-10)
    for m in (1, 3, 8):
        x1, k1, h1 = NL.fcg(A, b, lambda r: D @ r, m, rtol=1e-10)
        assert k1 == k2 and np.allclose(h1, h2, rtol=1e-6, atol=1e-14)
    x1, _, _ = NL.flexible_pcg(A, b, lambda r: D @ r, rtol=1e-10)
    assert np.allclose(NL.fcg(A, b, lambda r: D @ r, 1, rtol=1e-10)[0], x1, rtol=1e-8, atol=1e-12)
    # a preconditioner that changes every step: FCG(3) still converges
    rng = np.random.default_rng(16)

    def varying(r):
        return (1.0 + 0.5 * rng.random()) * (D @ r) + 0.1 * (D @ (D @ r))
    x, k, _ = NL.fcg(A, b, varying, 3, rtol=1e-10, maxit=500)
    assert np.linalg.norm(b - A @ x) <= 1e-9 * np.linalg.norm(b)
