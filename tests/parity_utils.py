"""Shared helpers of the parity tests: oracle construction and oracle <-> grid-vector maps.

Only the tests import this module; it calls the oracle and the library's Python binding
and holds none of the method's arithmetic.
"""
from __future__ import annotations

import functools

import numpy as np
import scipy.sparse as sp

from oracle import geometry as G
from oracle import discretize as D
from oracle import multigrid as MG
from synthetic import config_layout, preset


def layout_for(name: str, seed: int = 0, **overrides):
    pr = preset(name, **overrides)
    return pr, config_layout(pr.layout, seed)


@functools.lru_cache(maxsize=8)
def oracle_for(name: str, seed: int = 0, n: int | None = None, levels: int | None = None, depth: int | None = None,
               bc: int | None = None, smoother: str = "additive", degree: int | None = None):
    """(preset, layout, Discretization, Hierarchy) of the oracle for a workload (optionally resized)."""
    ov = {k: v for k, v in dict(n=n, levels=levels, depth=depth, bc=bc, degree=degree).items() if v is not None}
    pr, lay = layout_for(name, seed, **ov)
    d = _disc_for(name, seed, tuple(sorted(ov.items())))
    H = MG.Hierarchy(d, pr.levels, smoother=smoother)
    return pr, lay, d, H


@functools.lru_cache(maxsize=4)
def _disc_for(name: str, seed: int, ov: tuple):
    pr, lay = layout_for(name, seed, **dict(ov))
    geom = G.Balls(lay.centers, lay.radii, lay.lo, lay.hi)
    return D.Discretization(geom, pr.basis, pr.degree, pr.n, pr.depth, pr.bc)


def solver_for(lib, pr, lay, host_only=False, **kw):
    return lib.Solver(pr.dim, lay.centers, lay.radii, pr.n, pr.degree, pr.levels, pr.depth, pr.bc,
                      basis=pr.basis, lo=lay.lo, hi=lay.hi, host_only=host_only, **kw)


def coef_rows(lev, p: int, dim: int) -> np.ndarray:
    """Oracle operator rows of a level in the (2p+1)^d offset layout of the library."""
    W = 2 * p + 1
    m = lev.tb.m
    A = lev.A.tocsr()
    out = np.zeros((lev.active.size, W ** dim))
    act = lev.active
    for k in range(act.size):
        I = act[k]
        i = np.array(np.unravel_index(I, (m,) * dim, order="F"))
        lo, hi = A.indptr[k], A.indptr[k + 1]
        J = act[A.indices[lo:hi]]
        j = np.array(np.unravel_index(J, (m,) * dim, order="F"))
        o = j - i[:, None] + p
        ci = np.ravel_multi_index(tuple(o), (W,) * dim, order="F")
        np.add.at(out[k], ci, A.data[lo:hi])
    return out


def minv_from_blocks(ptr, idx, vptr, val, dinv, n_funcs: int, active: np.ndarray) -> sp.csr_matrix:
    """sum_j P_j A_j^{-1} P_j^T from the library's block arrays, in the oracle's active numbering."""
    rows, cols, vals = [], [], []
    for k in range(len(ptr) - 1):
        ids = idx[ptr[k]:ptr[k + 1]]
        nj = ids.size
        Ai = val[vptr[k]:vptr[k + 1]].reshape(nj, nj).T
        rows.append(np.repeat(ids, nj))
        cols.append(np.tile(ids, nj))
        vals.append(Ai.ravel())
    nz = np.flatnonzero(dinv)
    rows.append(nz)
    cols.append(nz)
    vals.append(dinv[nz])
    M = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n_funcs, n_funcs))
    return M[active][:, active].tocsr()


def energy_rel(e: np.ndarray, ref: np.ndarray, A) -> float:
    """||e||_A / ||ref||_A."""
    return float(np.sqrt(max(e @ (A @ e), 0.0) / max(ref @ (A @ ref), 1e-300)))


def mass_rel(e: np.ndarray, ref: np.ndarray, M) -> float:
    """Relative L2(Omega_h) error of FE coefficient vectors, via the mass matrix."""
    return float(np.sqrt(max(e @ (M @ e), 0.0) / max(ref @ (M @ ref), 1e-300)))
