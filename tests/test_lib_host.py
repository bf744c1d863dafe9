"""CPU tests of the library: it loads, exports the C-ABI, and its host-side setup
reproduces the oracle's discretisation and hierarchy (no GPU call is made here)."""
import os
import re

import numpy as np
import pytest

lib = pytest.importorskip("paper_1903_10977_gb300")
from parity_utils import coef_rows, minv_from_blocks, oracle_for, solver_for  # noqa: E402
from oracle import multigrid as MG  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_header_symbols_exported():
    hdr = open(os.path.join(ROOT, "include", "imgm.h")).read()
    declared = set(re.findall(r"\b(imgm_\w+)\s*\(", hdr))
    assert declared, "no declarations found"
    for name in declared:
        assert hasattr(lib._lib, name), name
    assert declared == set(lib.EXPORTED), declared ^ set(lib.EXPORTED)


CASES = [
    ("disc1_32_p2", {}),                                       # config 1 as printed
    ("disc1_32_p2", {"bc": 0}),                                # the paper's penalty form
    ("discs10_512_p1", {"n": 64, "levels": 3}),                # config 2 family, resized
    ("discs10_512_p2", {"n": 64, "levels": 4}),
    ("discs10_512_p3", {"n": 64, "levels": 3}),
    ("spheres20_128_p2", {"n": 16, "levels": 2, "depth": 1}),  # 3-D, resized
    ("spheres20_128_p2", {"n": 8, "levels": 2, "depth": 1, "degree": 1}),   # 3-D, linear
    ("spheres20_128_p2", {"n": 8, "levels": 2, "depth": 1, "degree": 3}),   # 3-D, cubic
]


@pytest.fixture(scope="module", params=CASES, ids=[f"{n}-{'-'.join(f'{k}{v}' for k, v in o.items())}" for n, o in CASES])
def pair(request):
    name, ov = request.param
    pr, lay, d, H = oracle_for(name, **ov)
    S = solver_for(lib, pr, lay, host_only=True)
    yield pr, d, H, S
    S.close()


def test_active_sets_bit_exact(pair):
    pr, d, H, S = pair
    for l in range(H.L, 0, -1):
        lev = H.lv[l]
        om = np.zeros(lev.tb.n_funcs, dtype=np.uint8)
        om[lev.active] = 1
        assert np.array_equal(S.active_mask(l), om), l


def test_operator_rows_all_levels(pair):
    pr, d, H, S = pair
    for l in range(H.L, 0, -1):
        lev = H.lv[l]
        ref = coef_rows(lev, pr.degree, pr.dim)
        got = S.host_operator_rows(lev.active, l)
        # every row to 1e-12 of its own largest entry (rows of sliver cut elements hold
        # Nitsche terms that cancel; elsewhere the agreement is a few eps)
        row_scale = np.abs(ref).max(axis=1)
        assert np.all(np.abs(got - ref).max(axis=1) <= 1e-12 * row_scale), l
        assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max(), l


def test_rhs(pair):
    pr, d, H, S = pair
    b = S.host_rhs()
    assert np.abs(b[d.active] - d.b).max() <= 1e-13 * np.abs(d.b).max()
    assert not np.any(np.delete(b, d.active))


def test_restriction_tables(pair):
    pr, d, H, S = pair
    for l in range(H.L, 1, -1):
        first, w = S.host_restriction(l)
        R1 = MG.two_scale_1d(H.lv[l - 1].tb.b, H.lv[l].tb.b)
        got = np.zeros_like(R1)
        for i in range(first.size):
            got[i, first[i]:first[i] + pr.degree + 2] = w[i]
        assert np.abs(got - R1).max() < 1e-14


def test_schwarz_operator(pair):
    """Same blocks (encapsulating supports), same Remark 3.3 removals, same inverses.

    Each block inverse is compared in the Jacobi-scaled form D A_j^{-1} D; two backward
    stable inversions of S_j = D^{-1} A_j D^{-1}, from blocks assembled independently (they
    agree to a few eps), agree to c n_j eps cond(S_j) relative to ||S_j^{-1}||; c = 64
    sets the tolerance block by block.
    """
    pr, d, H, S = pair
    eps = np.finfo(float).eps
    for l in range(H.L, 1, -1):
        lev = H.lv[l]
        ptr, idx, vptr, val, dinv = S.host_blocks(l)
        assert S.level_info(l)["pruned"] == lev.pruned
        A = lev.A.tocsr()
        pos = {int(I): k for k, I in enumerate(lev.active)}
        k = 0
        diag_ref = np.zeros(lev.tb.n_funcs)
        for blk in lev.blocks:
            Aj = A[blk][:, blk].toarray()
            inv = MG.block_inverse(Aj)
            if blk.size == 1:
                diag_ref[lev.active[blk[0]]] += inv[0, 0]
                continue
            got_idx = idx[ptr[k]:ptr[k + 1]]
            assert np.array_equal(got_idx, lev.active[blk]), (l, k)
            nj = blk.size
            got = val[vptr[k]:vptr[k + 1]].reshape(nj, nj).T
            dg = np.sqrt(np.diag(Aj))
            Sinv_ref = inv * dg[:, None] * dg[None, :]
            Sinv_got = got * dg[:, None] * dg[None, :]
            cond = np.linalg.cond(Aj / dg[:, None] / dg[None, :])
            tol = 64 * nj * eps * cond * np.abs(Sinv_ref).max()
            assert np.abs(Sinv_got - Sinv_ref).max() <= tol, (l, k, cond)
            k += 1
        assert k == len(ptr) - 1
        dA = np.zeros(lev.tb.n_funcs)
        dA[lev.active] = lev.A.diagonal()
        assert np.abs((dinv - diag_ref) * dA).max() < 1e-13


def test_coarse_inverse(pair):
    """Same kept rows; the inverse agrees in the scaled sense of test_schwarz_operator."""
    pr, d, H, S = pair
    rows, inv = S.host_coarse()
    assert np.array_equal(rows, H.lv[1].active[H.coarse_idx])
    A1 = H.lv[1].A.toarray()[np.ix_(H.coarse_idx, H.coarse_idx)]
    dg = np.sqrt(np.diag(A1))
    ref = H.coarse_inv * dg[:, None] * dg[None, :]
    got = inv * dg[:, None] * dg[None, :]
    cond = np.linalg.cond(A1 / dg[:, None] / dg[None, :])
    tol = 64 * A1.shape[0] * np.finfo(float).eps * cond * np.abs(ref).max()
    assert np.abs(got - ref).max() <= tol, cond


@pytest.mark.parametrize("kw,err", [
    (dict(n=30, levels=3), "multiple"),          # n not divisible by 2^(L-1)
    (dict(degree=4), "degree"),
    (dict(basis=1, degree=2), "Lagrange"),
    (dict(levels=1), "levels"),
    (dict(n=256, levels=2), "dense inverse allows at most"),   # coarsest level too large to invert densely
    (dict(precision=3), "precision"),
    (dict(precision=2, smoother=1), "additive smoother only"),
])
def test_invalid_configurations_are_rejected(kw, err):
    args = dict(dim=2, centers=[[0.5, 0.5]], radii=[0.2], n=32, degree=2, levels=3, depth=0, bc=1, host_only=True)
    args.update(kw)
    with pytest.raises(lib.ImgmError, match=err):
        lib.Solver(**args)


def test_box_without_holes():
    S = lib.Solver(2, np.zeros((0, 2)), np.zeros(0), 16, 2, 3, 0, 1, host_only=True)
    info = S.level_info(3)
    assert info["n_active"] == (16 + 2 - 2) ** 2 and info["n_band"] == 0


def test_learned_stage_arguments_checked_before_the_gpu():
    """The network and stage entry points reject bad arguments on the host, before any
    CUDA call (so these run without a GPU)."""
    import ctypes
    L = lib._lib
    out = ctypes.c_void_p()
    assert L.imgm_net_create(None, ctypes.byref(out)) == -1
    w = np.zeros(lib.NET_WEIGHTS, dtype=np.float32)
    assert L.imgm_net_create(w.ctypes.data_as(ctypes.c_void_p), None) == -1
    assert L.imgm_net_forward(None, 4, 4, 4, None, None, None, None) == -1
    assert L.imgm_net_accumulate(None, 4, 4, 4, None, None, None, 1.0, 1.0, None, None) == -1
    assert L.imgm_net_adam_step(None, 1e-3, 0.9, 0.999, 1e-8, None) == -1
    assert L.imgm_net_zero_grad(None, None) == -1
    assert L.imgm_net_get_weights(None, None) == -1
    pr, lay, _, _ = oracle_for("disc1_32_p2")
    S = solver_for(lib, pr, lay, host_only=True)
    assert L.imgm_set_fcg(None, 3) == -1
    for rc in (L.imgm_set_net(S._h, None), L.imgm_learned_stage(S._h, None, None, None, None),
               L.imgm_learned_pair(S._h, None, None, None, None, None), L.imgm_set_fcg(S._h, 3)):
        assert rc == -1                                  # a host-only handle has no device data
    S.close()


def test_train_net_schedule():
    """train_net: one zero_grad and one Adam step per step, `batch` accumulations taken in
    turn over the pairs, each pair's loss scaled by 1 / (batch * its active count), the set's
    input scale passed through."""
    torch = pytest.importorskip("torch")
    calls = []

    class FakeNet:
        def zero_grad(self, stream=None):
            calls.append(("zero",))

        def accumulate(self, x, target, shape, loss, mask=None, scale=1.0, in_scale=1.0, stream=None):
            calls.append(("acc", int(x[0].item()), scale, in_scale, shape))
            loss += 1.0

        def adam_step(self, lr, stream=None):
            calls.append(("adam", lr))

    pairs = [(torch.full((4,), float(k)), torch.zeros(4), torch.tensor([1, 1, 0, k % 2], dtype=torch.uint8))
             for k in range(3)]
    losses = lib.train_net(FakeNet(), pairs, (1, 2, 2), steps=2, lr=0.01, batch=2, in_scale=7.0)
    assert [c[0] for c in calls] == ["zero", "acc", "acc", "adam", "zero", "acc", "acc", "adam"]
    accs = [c for c in calls if c[0] == "acc"]
    assert [a[1] for a in accs] == [0, 1, 2, 0]
    assert [a[2] for a in accs] == [1 / (2 * 2), 1 / (2 * 3), 1 / (2 * 2), 1 / (2 * 2)]
    assert all(a[3] == 7.0 and a[4] == (1, 2, 2) for a in accs)
    assert losses.tolist() == [2.0, 2.0]
