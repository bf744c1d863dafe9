"""Geometric multigrid for the immersed system (Sec. 3) and multigrid-preconditioned CG.

* restriction R_l from the two-scale relation Phi_{l-1} = R_l Phi_l (Eq. coarsening);
  prolongation is R_l^T (Sec. 3.3);
* Galerkin coarse operators A_{l-1} = R_l A_l R_l^T, inheriting the fine weak form and
  its boundary parameters (Remark 3.1);
* additive Schwarz smoother M^{-1} = sum_j P_j (P_j^T A P_j)^{-1} P_j^T (Sec. 3.4) with
  one block per basis function made of the functions whose support in the physical
  domain lies inside its own (the encapsulating-support rule; for Lagrange bases only
  the nodal functions own blocks), the tiny-eigenvalue rule of Remark 3.3, and the
  relaxation gamma = 1 / max_K N_K (N_K = (p+1)^d for B-splines, 2^d for Lagrange);
* coloured multiplicative Schwarz (Sec. 3.4, the smoother of the paper's experiments):
  the blocks fall into classes of equal colour whose owners' supports are disjoint
  ((p+1)^d colours for B-splines, 2^d for Lagrange), the blocks of one colour act
  together on the current residual, and the residual is updated after each colour; the
  post-smoothing sweep takes the colours in reverse order, which makes it the adjoint of
  the pre-smoothing sweep, and no relaxation parameter is used;
* the V-cycle of Algorithm 1 with a direct solve on level 1, one pre- and one
  post-smoothing step, and the symmetric V-cycle as a CG preconditioner (Sec. 3.2).

Readings of the silent or ambiguous points:

* line 10 of Algorithm 1 subtracts A_l times the prolongated coarse correction only
  (the residual already accounts for the pre-smoothing step after line 5), so that the
  error propagation is (I - gamma M^{-T} A)(I - R^T B_{l-1} R A)(I - gamma M^{-1} A)
  as in Eq. eigenMulti;
* levels: the coarsest of L levels has n / 2^(L-1) elements per direction;
* the direct solve on level 1 inverts A_1 through its Jacobi-scaled Cholesky factor,
  after the Remark 3.3 rule has been applied to A_1 as a whole: cut functions can make
  the Galerkin coarse matrix numerically singular just like a Schwarz block, and the
  paper's treatment of such blocks is taken for it too (removed functions get no
  coarse correction);
* a coarse element is active when one of its fine children is; a coarse function is
  active when one of its support elements is (functions on a Dirichlet box face stay
  out, as on the finest level);
* the encapsulating-support test compares the sets of active support elements
  (B-splines and Lagrange functions are non-zero inside every element of their
  support, so this is the set inclusion of the supports within Omega_h);
* a Lagrange function that no nodal block contains gets a block of its own (additive
  smoother only: the paper's colouring covers the nodal blocks, so the multiplicative
  smoother rejects such levels);
* the colour of a block is that of its owner: the owner's index modulo p+1 in every
  direction for B-splines, its vertex index modulo 2 for Lagrange functions; colours are
  taken in increasing order of sum_k c_k (p+1)^k (2^k for Lagrange) in the
  pre-smoothing sweep;
* tiny-eigenvalue rule: while lambda_min(A_j) < 1e-16 max_i (A_j)_ii, the function
  with the largest |entry| of the eigenvector of lambda_min (lowest index on ties) leaves
  the block; lambda_min is taken as 1 / lambda_max(A_j^{-1}) with A_j^{-1} formed through
  the Cholesky factor of the Jacobi-scaled block, which fixes tiny eigenvalues of graded
  blocks to high relative accuracy (a plain eigh fixes them only to 1e-16 max|A_j|).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from .basis import BSpline1D, Lagrange1D, TensorBasis, make_basis

PRUNE_RATIO = 1e-16


def two_scale_1d(coarse, fine) -> np.ndarray:
    """Dense (m_c x m_f) matrix R1 with phi^c_i = sum_a R1[i, a] phi^f_a (Eq. coarsening).

    B-splines: both sides are evaluated at the fine Greville abscissae, where the fine
    collocation matrix is invertible (Schoenberg-Whitney), and R1^T = F^{-1} C.
    Lagrange: nodal interpolation, R1[i, a] = phi^c_i(x^f_a).
    """
    if isinstance(fine, Lagrange1D):
        return np.stack([coarse.eval_global(i, fine.nodes) for i in range(coarse.m)])
    X = fine.greville()
    F = np.stack([fine.eval_global(a, X) for a in range(fine.m)], axis=1)     # (q, a)
    C = np.stack([coarse.eval_global(i, X) for i in range(coarse.m)], axis=1)  # (q, i)
    R1 = np.linalg.solve(F, C).T
    R1[np.abs(R1) < 1e-13] = 0.0
    return R1


def kron_nd(mats_1d: list) -> sp.csr_matrix:
    """Tensor-product matrix for x-fastest flat indices: M_{d-1} (x) ... (x) M_0."""
    out = sp.csr_matrix(mats_1d[0])
    for M in mats_1d[1:]:
        out = sp.kron(sp.csr_matrix(M), out, format="csr")
    return out


class Level:
    """One level of the hierarchy: basis, activity, operator, smoother."""

    def __init__(self, tb: TensorBasis, elem_active: np.ndarray, A: sp.csr_matrix, active: np.ndarray):
        self.tb, self.elem_active, self.A, self.active = tb, elem_active, A, active
        self.R = None          # restriction to the next coarser level (active x active)
        self.Minv = None       # additive Schwarz operator sum_j P_j A_j^{-1} P_j^T
        self.blocks = []
        self.pruned = 0


def coarse_activity(tb_c: TensorBasis, fine_elem_active: np.ndarray, n_fine: int, dim: int,
                    box_dirichlet: bool = True):
    """Coarse elements active when one of their 2^d children is; coarse functions as on the fine level."""
    fa = fine_elem_active.reshape((n_fine,) * dim, order="F")
    sl = [fa[tuple(slice(o[k], None, 2) for k in range(dim))]
          for o in np.ndindex(*(2,) * dim)]
    ca = np.zeros_like(sl[0], dtype=bool)
    for s in sl:
        ca |= s
    elem_active = ca.ravel(order="F")
    func = np.zeros(tb_c.n_funcs, dtype=bool)
    for E in np.flatnonzero(elem_active):
        func[tb_c.elem_dofs(int(E))] = True
    if box_dirichlet:
        multi = np.array(np.unravel_index(np.arange(tb_c.n_funcs), (tb_c.m,) * dim, order="F"))
        func[np.any((multi == 0) | (multi == tb_c.m - 1), axis=0)] = False
    return elem_active, np.flatnonzero(func)


def schwarz_blocks(tb: TensorBasis, elem_active: np.ndarray, active: np.ndarray, with_owners: bool = False):
    """Index blocks by encapsulating supports (Sec. 3.4), in active numbering.

    with_owners: also return the owner of every block (full-grid index of the function
    whose support bounds it; -1 for the block of a function that no nodal block holds)."""
    pos = -np.ones(tb.n_funcs, dtype=np.int64)
    pos[active] = np.arange(active.size)
    act_el = {int(I): frozenset(E for E in tb.support_elems(int(I)) if elem_active[E]) for I in active}
    blocks, owners = [], []
    covered = np.zeros(active.size, dtype=bool)
    for I in active:
        I = int(I)
        if not tb.is_nodal(I):
            continue
        # candidates: the functions that live on one of I's support elements
        cand = set()
        for E in tb.support_elems(I):
            cand.update(int(J) for J in tb.elem_dofs(E) if pos[J] >= 0)
        blk = sorted(pos[J] for J in cand if act_el[J] <= act_el[I])
        blocks.append(np.array(blk, dtype=np.int64))
        owners.append(I)
        covered[blk] = True
    for k in np.flatnonzero(~covered):
        blocks.append(np.array([k], dtype=np.int64))
        owners.append(-1)
    return (blocks, owners) if with_owners else blocks


def block_colour(tb: TensorBasis, owner: int) -> int:
    """Colour of the block of `owner`: functions of equal colour have disjoint supports
    (Sec. 3.4): index mod (p+1) per direction for B-splines, vertex index mod 2 for
    Lagrange functions (vertex = node / p)."""
    multi = tb.func_multi(int(owner))
    if isinstance(tb.b, Lagrange1D):
        digits, base = [(int(i) // tb.b.p) % 2 for i in multi], 2
    else:
        digits, base = [int(i) % (tb.b.p + 1) for i in multi], tb.b.p + 1
    return int(sum(c * base ** k for k, c in enumerate(digits)))


def block_inverse(Aj: np.ndarray) -> np.ndarray:
    """A_j^{-1} through the Cholesky factor of the Jacobi-scaled block.

    A_j = D S D with D = diag(A_j)^{1/2}; A_j^{-1} = D^{-1} S^{-1} D^{-1}.  Blocks that
    hold functions with tiny cut supports are graded (diagonal entries spread over many
    orders of magnitude) while S stays well conditioned; inverting through S keeps every
    entry of the inverse accurate.  Raises LinAlgError when S is not positive definite.
    """
    dg = np.sqrt(np.diag(Aj))
    S = Aj / dg[:, None] / dg[None, :]
    Sinv = sla.cho_solve(sla.cho_factor(S, lower=True), np.eye(S.shape[0]))
    return Sinv / dg[:, None] / dg[None, :]


def smallest_eigenpair(Aj: np.ndarray):
    """lambda_min(A_j) and its eigenvector, as 1 / lambda_max(A_j^{-1}) when the scaled
    Cholesky factor exists (relative accuracy for graded blocks), else by a plain eigh."""
    try:
        Ainv = block_inverse(Aj)
        mu, V = np.linalg.eigh(0.5 * (Ainv + Ainv.T))
        return 1.0 / mu[-1], V[:, -1]
    except np.linalg.LinAlgError:
        lam, V = np.linalg.eigh(Aj)
        return lam[0], V[:, 0]


def prune_block(Aj: np.ndarray, idx: np.ndarray):
    """Remark 3.3: drop the dominant function of the eigenvector of a tiny eigenvalue."""
    removed = 0
    while idx.size > 1:
        lam, v = smallest_eigenpair(Aj)
        if lam >= PRUNE_RATIO * np.max(np.diag(Aj)):
            break
        k = int(np.argmax(np.abs(v)))                # argmax returns the lowest index on ties
        keep = np.arange(idx.size) != k
        idx, Aj = idx[keep], Aj[np.ix_(keep, keep)]
        removed += 1
    return Aj, idx, removed


def block_sum(n: int, blocks, inverses) -> sp.csr_matrix:
    """sum_j P_j A_j^{-1} P_j^T over the given blocks as a sparse n x n matrix."""
    if not blocks:
        return sp.csr_matrix((n, n))
    rows = [np.repeat(idx, idx.size) for idx in blocks]
    cols = [np.tile(idx, idx.size) for idx in blocks]
    vals = [inv.ravel() for inv in inverses]
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))


def schwarz_operator(A: sp.csr_matrix, blocks, with_inverses: bool = False):
    """sum_j P_j A_j^{-1} P_j^T as a sparse matrix, after the Remark 3.3 rule
    (with_inverses: also the kept blocks' inverses, in block order)."""
    kept, inverses, pruned = [], [], 0
    Ad = A.tocsr()
    for idx in blocks:
        Aj = Ad[idx][:, idx].toarray()
        Aj, idx, removed = prune_block(Aj, idx)
        pruned += removed
        inverses.append(block_inverse(Aj))
        kept.append(idx)
    Minv = block_sum(A.shape[0], kept, inverses)
    return (Minv, kept, pruned, inverses) if with_inverses else (Minv, kept, pruned)


def default_gamma(kind: int, p: int, dim: int) -> float:
    """gamma = 1 / max_K N_K (Eqs. applyASLemma-applyCS): (p+1)^-d B-splines, 2^-d Lagrange."""
    return 1.0 / ((p + 1) ** dim if kind == 0 else 2 ** dim)


class Hierarchy:
    """Levels L (finest) .. 1 (coarsest) built from a fine Discretization."""

    def __init__(self, disc, levels: int, gamma: float | None = None, smoother: str = "additive"):
        self.disc, self.L = disc, int(levels)
        if smoother not in ("additive", "multiplicative"):
            raise ValueError("smoother must be 'additive' or 'multiplicative'")
        self.smoother = smoother
        if smoother == "multiplicative":
            self.gamma = 1.0                              # no relaxation (Sec. 3.4)
        else:
            self.gamma = default_gamma(disc.kind, disc.p, disc.dim) if gamma is None else float(gamma)
        d, p, n = disc.dim, disc.p, disc.n
        if n % (2 ** (levels - 1)):
            raise ValueError("n must be divisible by 2^(levels-1)")
        self.lv = {levels: Level(disc.tb, disc.elem_active, disc.A, disc.active)}
        for l in range(levels, 1, -1):
            fine = self.lv[l]
            nc = fine.tb.n // 2
            b1c = make_basis(disc.kind, nc, p, disc.geom.lo, disc.geom.hi)
            tbc = TensorBasis(b1c, d)
            ea, act = coarse_activity(tbc, fine.elem_active, fine.tb.n, d, disc.geom.box_dirichlet)
            R1 = two_scale_1d(b1c, fine.tb.b)
            Rfull = kron_nd([R1] * d)
            R = Rfull[act][:, fine.active].tocsr()
            R.eliminate_zeros()
            fine.R = R
            Ac = (R @ fine.A @ R.T).tocsr()
            self.lv[l - 1] = Level(tbc, ea, Ac, act)
        for l in range(levels, 1, -1):
            lev = self.lv[l]
            blocks, owners = schwarz_blocks(lev.tb, lev.elem_active, lev.active, with_owners=True)
            lev.Minv, lev.blocks, lev.pruned, inverses = schwarz_operator(lev.A, blocks, with_inverses=True)
            lev.owners = owners
            if smoother == "multiplicative":
                if min(owners) < 0:
                    raise ValueError("multiplicative Schwarz: a function lies in no nodal block")
                colours = np.array([block_colour(lev.tb, o) for o in owners])
                n_col = (2 if isinstance(lev.tb.b, Lagrange1D) else p + 1) ** d
                lev.colour_ops = [block_sum(lev.A.shape[0], [lev.blocks[j] for j in np.flatnonzero(colours == c)],
                                            [inverses[j] for j in np.flatnonzero(colours == c)])
                                  for c in range(n_col)]
        A1 = self.lv[1].A.toarray()
        _, self.coarse_idx, self.coarse_pruned = prune_block(A1, np.arange(A1.shape[0]))
        self.coarse_inv = block_inverse(A1[np.ix_(self.coarse_idx, self.coarse_idx)])

    # -------------------------------------------------------------- Algorithm 1
    def smooth(self, l: int, r: np.ndarray, adjoint: bool = False) -> np.ndarray:
        """gamma M^{-1} r (adjoint: gamma M^{-T} r; M^{-1} is symmetric for additive Schwarz).

        Multiplicative: one coloured sweep from zero, colours in increasing order
        (adjoint: decreasing), the residual updated after every colour."""
        lev = self.lv[l]
        if self.smoother == "additive":
            return self.gamma * ((lev.Minv.T if adjoint else lev.Minv) @ r)
        order = range(len(lev.colour_ops))
        y = np.zeros_like(r)
        rt = r.copy()
        for c in (reversed(order) if adjoint else order):
            dy = lev.colour_ops[c] @ rt
            y = y + dy
            rt = rt - lev.A @ dy
        return y

    def vcycle(self, l: int, r: np.ndarray) -> np.ndarray:
        if l == 1:                                                      # line 14
            x = np.zeros_like(r)
            x[self.coarse_idx] = self.coarse_inv @ r[self.coarse_idx]
            return x
        lev = self.lv[l]
        x = np.zeros_like(r)                                            # line 2
        x = x + self.smooth(l, r)                                       # line 4
        r = r - lev.A @ x                                               # line 5
        rc = lev.R @ r                                                  # line 7
        xc = self.vcycle(l - 1, rc)                                     # line 8
        e = lev.R.T @ xc                                                # line 9
        x = x + e
        r = r - lev.A @ e                                               # line 10 (increment)
        x = x + self.smooth(l, r, adjoint=True)                         # line 12
        return x

    def precondition(self, r: np.ndarray) -> np.ndarray:
        return self.vcycle(self.L, r)


def pcg(A, b: np.ndarray, precond, rtol: float = 1e-8, maxit: int = 1000, x0=None):
    """Preconditioned conjugate gradients (Sec. 3.2: the V-cycle as SPD preconditioner).

    Stops when the recursively updated residual satisfies ||r|| <= rtol ||b||.
    Returns (x, iterations, history of ||r_k|| / ||b||).
    """
    x = np.zeros_like(b) if x0 is None else x0.copy()
    r = b - A @ x
    bnorm = np.linalg.norm(b)
    hist = [np.linalg.norm(r) / bnorm]
    if hist[-1] <= rtol:
        return x, 0, hist
    z = precond(r)
    p = z.copy()
    rz = r @ z
    for k in range(1, maxit + 1):
        q = A @ p
        alpha = rz / (p @ q)
        x = x + alpha * p
        r = r - alpha * q
        hist.append(np.linalg.norm(r) / bnorm)
        if hist[-1] <= rtol:
            return x, k, hist
        z = precond(r)
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, maxit, hist
