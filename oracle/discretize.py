"""Assembly of the immersed system A x = b (Sec. 2; Eqs. weakMulti, operatorsMulti, systemMulti).

Scalar model problem: -Laplace(u) = f in Omega, u = g on the immersed boundary
Gamma = {psi = 0}.  A_ij = a_h(phi_i, phi_j) and b_i = b_h(phi_i) with

* penalty (the paper's choice, Eq. operatorsMulti reduced to the scalar case, with
  beta = 2/h as in Sec. 3.1):
      a_h(v, u) = int_Omega grad v . grad u + beta int_Gamma v u
      b_h(v)    = int_Omega v f + beta int_Gamma v g
* symmetric Nitsche (Sec. 2 names it as the coercivity-preserving alternative and
  points to Embar et al. for the parameter):
      a_h(v, u) = int grad v . grad u - int_Gamma (d_n v u + v d_n u) + sum_K beta_K int_{Gamma cap K} v u
      b_h(v)    = int v f - int_Gamma d_n v g + sum_K beta_K int_{Gamma cap K} v g
  Reading for beta_K: twice the largest eigenvalue lambda_K of
  int_{Gamma cap K} d_n u d_n v = lambda int_{K cap Omega_h} grad u . grad v over the
  non-constant functions on K (so a_h is coercive), floored at 1/h and rounded up to a
  power of two, beta_K = 2^ceil(log2(2 max(lambda_K, 1/h))), so that the parameter does
  not depend on how the eigenvalue was rounded.

When the faces of the embedding box belong to the boundary of Omega (a domain cut out
of the box, ``geom.box_dirichlet``), they carry the homogeneous condition u = 0
strongly: every function that is non-zero on the box boundary is removed (reading; the
paper's own domains are immersed and never touch the box).

Activity (Sec. 2: the approximation space is spanned by the functions whose support
reaches into the physical domain): an element is active when |K cap Omega_h| > 0 and a
function is active when one of its support elements is active.  Vectors in this module are indexed by active function
(increasing full-grid index); ``Discretization.active`` maps them to the full grid.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from .basis import TensorBasis, make_basis
from .geometry import CUT, EMPTY, FULL
from .quadrature import box_rule, cut_element_rule, gauss01

PENALTY, NITSCHE = 0, 1


class Manufactured:
    """u = prod_k sin(pi x_k), f = d pi^2 u, g = u."""

    @staticmethod
    def u(X):
        return np.prod(np.sin(np.pi * X), axis=1)

    @staticmethod
    def f(X):
        return X.shape[1] * np.pi ** 2 * np.prod(np.sin(np.pi * X), axis=1)

    @staticmethod
    def g(X):
        return np.prod(np.sin(np.pi * X), axis=1)


class Polynomial:
    """u given as a callable polynomial with its negative Laplacian (reproduction tests)."""

    def __init__(self, u, minus_lap):
        self._u, self._f = u, minus_lap

    def u(self, X):
        return self._u(X)

    def f(self, X):
        return self._f(X)

    def g(self, X):
        return self._u(X)


def nitsche_beta(S: np.ndarray, Bn: np.ndarray, h: float) -> float:
    """beta_K = 2^ceil(log2(2 max(lambda_max, 1/h))), lambda_max of (Bn, S) on the non-constants."""
    nloc = S.shape[0]
    Q = sla.null_space(np.ones((1, nloc)))             # orthonormal basis of 1^perp
    Sh = Q.T @ S @ Q
    Bh = Q.T @ Bn @ Q
    mu, W = np.linalg.eigh(0.5 * (Sh + Sh.T))
    keep = mu > 1e-14 * mu.max()
    T = W[:, keep] / np.sqrt(mu[keep])
    lam = float(np.linalg.eigvalsh(T.T @ (0.5 * (Bh + Bh.T)) @ T).max())
    lam = max(lam, 1.0 / h)
    return 2.0 ** math.ceil(math.log2(2.0 * lam))


class Discretization:
    """Immersed discretization of one grid level (the finest level of the hierarchy)."""

    def __init__(self, geom, basis_kind: int, p: int, n: int, depth: int, bc: int = NITSCHE,
                 problem=Manufactured, assemble: bool = True, batch: int = 8192):
        self.geom, self.dim = geom, geom.dim
        self.kind, self.p, self.n, self.depth, self.bc = int(basis_kind), int(p), int(n), int(depth), int(bc)
        self.problem = problem
        self.tb = TensorBasis(make_basis(basis_kind, n, p, geom.lo, geom.hi), geom.dim)
        self.h = self.tb.h
        self.beta_penalty = 2.0 / self.h
        self._batch = batch
        self._classify()
        self._cut_cache: dict[int, tuple] = {}
        self._cut_volumes()
        self._activity()
        if assemble:
            self._assemble()

    # ----------------------------------------------------------------- geometry
    def _elem_boxes(self, Es: np.ndarray):
        multi = np.array(np.unravel_index(Es, (self.n,) * self.dim, order="F")).T
        lo = self.geom.lo + multi * self.h
        return lo, lo + self.h

    def _classify(self):
        Es = np.arange(self.tb.n_elems)
        LO, HI = self._elem_boxes(Es)
        self.elem_class = self.geom.classify_many(LO, HI)
        self.cut_elems = np.flatnonzero(self.elem_class == CUT)

    def cut_rule(self, E: int):
        if E not in self._cut_cache:
            lo, hi = self._elem_boxes(np.array([E]))
            self._cut_cache[E] = cut_element_rule(self.geom, lo[0], hi[0], self.p, self.depth)
        return self._cut_cache[E]

    def _cut_volumes(self):
        self.elem_volume = np.where(self.elem_class == FULL, self.h ** self.dim, 0.0)
        for E in self.cut_elems:
            self.elem_volume[E] = self.cut_rule(int(E))[1].sum()

    def _activity(self):
        self.elem_active = self.elem_volume > 0
        self.func_active_full = np.zeros(self.tb.n_funcs, dtype=bool)
        Es = np.flatnonzero(self.elem_active)
        if Es.size:
            self.func_active_full[self._elem_dofs_batch(Es).ravel()] = True
        if self.geom.box_dirichlet:
            multi = np.array(np.unravel_index(np.arange(self.tb.n_funcs), (self.tb.m,) * self.dim, order="F"))
            on_box = np.any((multi == 0) | (multi == self.tb.m - 1), axis=0)
            self.func_active_full[on_box] = False
        self.active = np.flatnonzero(self.func_active_full)
        self.n_active = int(self.active.size)
        self.full_to_active = -np.ones(self.tb.n_funcs, dtype=np.int64)
        self.full_to_active[self.active] = np.arange(self.n_active)

    # ---------------------------------------------------------- element systems
    def _local_system(self, E: int, vp, vw, bp, bw, bn):
        """Element matrix, element right-hand side and element mass matrix from a rule."""
        f, g = self.problem.f, self.problem.g
        vals, grads = self.tb.eval(E, vp) if len(vw) else (np.zeros((self.tb.nloc, 0)),) * 2
        S = np.einsum("jaq,jbq,q->ab", grads, grads, vw) if len(vw) else np.zeros((self.tb.nloc,) * 2)
        M = np.einsum("aq,bq,q->ab", vals, vals, vw) if len(vw) else np.zeros_like(S)
        rhs = vals @ (vw * f(vp)) if len(vw) else np.zeros(self.tb.nloc)
        A = S.copy()
        beta = None
        if len(bw):
            bv, bg = self.tb.eval(E, bp)
            dn = np.einsum("jaq,qj->aq", bg, bn)             # normal derivatives
            gq = g(bp)
            if self.bc == PENALTY:
                beta = self.beta_penalty
                A += beta * np.einsum("aq,bq,q->ab", bv, bv, bw)
                rhs += beta * bv @ (bw * gq)
            else:
                Bn = np.einsum("aq,bq,q->ab", dn, dn, bw)
                beta = nitsche_beta(S, Bn, self.h)
                C = np.einsum("aq,bq,q->ab", dn, bv, bw)
                A += -(C + C.T) + beta * np.einsum("aq,bq,q->ab", bv, bv, bw)
                rhs += -dn @ (bw * gq) + beta * bv @ (bw * gq)
        return A, rhs, M, beta

    def element_system(self, E: int):
        """(A_K, b_K, M_K, beta_K) of element E by its quadrature rule (full or cut)."""
        if self.elem_class[E] == FULL:
            lo, hi = self._elem_boxes(np.array([E]))
            vp, vw = box_rule(lo[0], hi[0], self.p + 1)
            return self._local_system(E, vp, vw, np.zeros((0, self.dim)), np.zeros(0),
                                      np.zeros((0, self.dim)))
        if self.elem_class[E] == EMPTY:
            z = np.zeros((self.tb.nloc, self.tb.nloc))
            return z, np.zeros(self.tb.nloc), z, None
        return self._local_system(E, *self.cut_rule(E))

    def _full_batch(self, Es: np.ndarray):
        """element_system for a batch of full elements: the same tensor Gauss rule, the
        basis values at the tensor points taken as products of 1-D values."""
        d, p, b1 = self.dim, self.p, self.tb.b
        x1, w1 = gauss01(p + 1)
        multi = np.array(np.unravel_index(Es, (self.n,) * d, order="F")).T     # (nB, d)
        LO, HI = self._elem_boxes(Es)
        nq1 = p + 1
        qidx = np.array(np.unravel_index(np.arange(nq1 ** d), (nq1,) * d, order="F")).T  # (nq, d)
        V = np.empty((len(Es), d, p + 1, nq1))
        D = np.empty_like(V)
        for k in range(d):
            for e in np.unique(multi[:, k]):
                sel = multi[:, k] == e
                xs = LO[sel, k][:, None] + (HI[sel, k] - LO[sel, k])[:, None] * x1[None, :]
                v, dv = b1.eval(int(e), xs[0])
                V[sel, k] = v
                D[sel, k] = dv
        loc = self.tb.local
        vals = np.ones((len(Es), self.tb.nloc, nq1 ** d))
        grads = np.ones((len(Es), d, self.tb.nloc, nq1 ** d))
        for k in range(d):
            vk = V[:, k][:, loc[:, k]][:, :, qidx[:, k]]
            dk = D[:, k][:, loc[:, k]][:, :, qidx[:, k]]
            vals *= vk
            for j in range(d):
                grads[:, j] *= dk if j == k else vk
        W = np.prod((HI - LO)[:, None, :] * w1[qidx][None, :, :], axis=2)           # (nB, nq)
        X = LO[:, None, :] + (HI - LO)[:, None, :] * x1[qidx][None, :, :]
        F = self.problem.f(X.reshape(-1, d)).reshape(W.shape)
        S = np.einsum("ejaq,ejbq,eq->eab", grads, grads, W)
        M = np.einsum("eaq,ebq,eq->eab", vals, vals, W)
        rhs = np.einsum("eaq,eq->ea", vals, W * F)
        return S, rhs, M

    # ----------------------------------------------------------------- assembly
    def _elem_dofs_batch(self, Es: np.ndarray) -> np.ndarray:
        multi = np.array(np.unravel_index(Es, (self.n,) * self.dim, order="F")).T
        first = np.stack([self.tb.b.first(multi[:, k]) for k in range(self.dim)], axis=1)
        g = first[:, None, :] + self.tb.local[None, :, :]
        return np.ravel_multi_index(tuple(np.moveaxis(g, 2, 0)), (self.tb.m,) * self.dim, order="F")

    def _assemble(self):
        N = self.tb.n_funcs
        rows, cols, av, mv = [], [], [], []
        bfull = np.zeros(N)
        self.beta = {}
        full = np.flatnonzero(self.elem_class == FULL)
        for s in range(0, full.size, self._batch):
            Es = full[s:s + self._batch]
            S, rhs, M = self._full_batch(Es)
            dofs = self._elem_dofs_batch(Es)
            rows.append(np.repeat(dofs, self.tb.nloc, axis=1).ravel())
            cols.append(np.tile(dofs, (1, self.tb.nloc)).ravel())
            av.append(S.ravel())
            mv.append(M.ravel())
            np.add.at(bfull, dofs.ravel(), rhs.ravel())
        for E in self.cut_elems:
            E = int(E)
            if not self.elem_active[E]:
                continue
            A, rhs, M, beta = self.element_system(E)
            if beta is not None:
                self.beta[E] = beta
            dofs = self.tb.elem_dofs(E)
            rows.append(np.repeat(dofs, self.tb.nloc))
            cols.append(np.tile(dofs, self.tb.nloc))
            av.append(A.ravel())
            mv.append(M.ravel())
            np.add.at(bfull, dofs, rhs)
        r = np.concatenate(rows)
        c = np.concatenate(cols)
        Afull = sp.csr_matrix((np.concatenate(av), (r, c)), shape=(N, N))
        Mfull = sp.csr_matrix((np.concatenate(mv), (r, c)), shape=(N, N))
        act = self.active
        self.A = Afull[act][:, act].tocsr()
        self.M = Mfull[act][:, act].tocsr()
        self.b = bfull[act]

    def assemble_rows(self, rows_full: np.ndarray):
        """Rows of A (in full-grid column indexing) and entries of b, assembled from the
        elements in their supports.

        Used where the whole matrix is too large for this oracle: returns a dict
        row -> (cols, vals, b_row) for the requested full-grid rows.
        """
        out = {}
        cache = {}
        for I in rows_full:
            I = int(I)
            acc: dict[int, float] = {}
            bI = 0.0
            if self.func_active_full[I]:
                for E in self.tb.support_elems(I):
                    if not self.elem_active[E]:
                        continue
                    if E not in cache:
                        cache[E] = self.element_system(E)[:2]
                    AK, bK = cache[E]
                    dofs = self.tb.elem_dofs(E)
                    a = int(np.flatnonzero(dofs == I)[0])
                    bI += bK[a]
                    for bi, J in enumerate(dofs):
                        if self.func_active_full[J]:
                            acc[int(J)] = acc.get(int(J), 0.0) + AK[a, bi]
            cols = np.array(sorted(acc), dtype=np.int64)
            out[I] = (cols, np.array([acc[j] for j in cols]), bI)
        return out

    # ------------------------------------------------------------------ helpers
    def to_full(self, v: np.ndarray) -> np.ndarray:
        out = np.zeros(self.tb.n_funcs)
        out[self.active] = v
        return out

    def to_active(self, v_full: np.ndarray) -> np.ndarray:
        return np.asarray(v_full)[self.active]

    def evaluate(self, coeffs_active: np.ndarray, X: np.ndarray) -> np.ndarray:
        """u_h at points X (each point is evaluated in the element that contains it)."""
        full = self.to_full(coeffs_active)
        X = np.atleast_2d(X)
        e = np.clip(np.floor((X - self.geom.lo) / self.h).astype(int), 0, self.n - 1)
        E = np.ravel_multi_index(tuple(e.T), (self.n,) * self.dim, order="F")
        out = np.zeros(X.shape[0])
        for el in np.unique(E):
            sel = E == el
            vals, _ = self.tb.eval(int(el), X[sel])
            out[sel] = full[self.tb.elem_dofs(int(el))] @ vals
        return out

    def l2_h1_errors(self, coeffs_active: np.ndarray, u, grad_u):
        """||u - u_h|| in L2(Omega_h) and the H1 seminorm error, by the element rules."""
        full = self.to_full(coeffs_active)
        e0 = e1 = 0.0
        for E in np.flatnonzero(self.elem_active):
            E = int(E)
            if self.elem_class[E] == FULL:
                lo, hi = self._elem_boxes(np.array([E]))
                vp, vw = box_rule(lo[0], hi[0], self.p + 1)
            else:
                vp, vw = self.cut_rule(E)[:2]
            if not len(vw):
                continue
            vals, grads = self.tb.eval(E, vp)
            c = full[self.tb.elem_dofs(E)]
            uh = c @ vals
            guh = np.einsum("a,jaq->qj", c, grads)
            e0 += np.sum(vw * (u(vp) - uh) ** 2)
            e1 += np.sum(vw * np.sum((grad_u(vp) - guh) ** 2, axis=1))
        return math.sqrt(e0), math.sqrt(e1)


class LocalRows(Discretization):
    """Rows of the immersed system assembled from their own support elements only, for
    grids too large for the global assembly above (test infrastructure, like the rest of
    this package).

    Same discretisation as Discretization (Sec. 2: the element systems, the activity rule
    and the box-face condition are those methods, unchanged); what differs is that cut
    elements are integrated on demand.  No global cut-volume pass is made, so a row's
    activity and its entries come from the elements of its own support:

    * row I is active iff it is not a box-face function (when the box faces carry u = 0)
      and some element of its support has positive measure in Omega_h;
    * a column J enters through an element K of supp(I) with positive measure; an
      inactive J (all of its support elements of zero measure) never meets such a K, so
      its entry is not formed at all, as in the global assembly, except for box-face
      functions, which are excluded explicitly.
    """

    def __init__(self, geom, basis_kind: int, p: int, n: int, depth: int, bc: int = NITSCHE,
                 problem=Manufactured):
        self.geom, self.dim = geom, geom.dim
        self.kind, self.p, self.n, self.depth, self.bc = int(basis_kind), int(p), int(n), int(depth), int(bc)
        self.problem = problem
        self.tb = TensorBasis(make_basis(basis_kind, n, p, geom.lo, geom.hi), geom.dim)
        self.h = self.tb.h
        self.beta_penalty = 2.0 / self.h
        self._batch = 8192
        self._classify()
        self._cut_cache = {}

    def on_box(self, J: int) -> bool:
        if not self.geom.box_dirichlet:
            return False
        multi = np.unravel_index(int(J), (self.tb.m,) * self.dim, order="F")
        return any(k == 0 or k == self.tb.m - 1 for k in multi)

    def element_active(self, E: int) -> bool:
        c = self.elem_class[E]
        if c == FULL:
            return True
        if c == EMPTY:
            return False
        return self.cut_rule(int(E))[1].sum() > 0

    def row_active(self, I: int) -> bool:
        return (not self.on_box(I)) and any(self.element_active(E) for E in self.tb.support_elems(int(I)))

    def assemble_rows(self, rows_full: np.ndarray):
        """Rows of A (full-grid column indexing) and entries of b: row -> (cols, vals, b_row);
        an inactive row comes back empty."""
        out = {}
        cache = {}
        for I in rows_full:
            I = int(I)
            acc: dict[int, float] = {}
            bI = 0.0
            if self.row_active(I):
                for E in self.tb.support_elems(I):
                    if not self.element_active(E):
                        continue
                    if E not in cache:
                        cache[E] = self.element_system(E)[:2]
                    AK, bK = cache[E]
                    dofs = self.tb.elem_dofs(E)
                    a = int(np.flatnonzero(dofs == I)[0])
                    bI += bK[a]
                    for bi, J in enumerate(dofs):
                        if not self.on_box(int(J)):
                            acc[int(J)] = acc.get(int(J), 0.0) + AK[a, bi]
            cols = np.array(sorted(acc), dtype=np.int64)
            out[I] = (cols, np.array([acc[j] for j in cols]), bI)
        return out
