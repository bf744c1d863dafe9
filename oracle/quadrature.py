"""Cut-cell quadrature (Sec. 2, Fig. 1): bisect, triangulate, clip, Gauss.

The paper integrates cut elements by recursively bisecting them up to an integration
depth, triangulating the leaves, and applying Gauss rules on the resulting sub-cells;
the boundary integrals use the sub-cell edges that approximate the boundary.  It gives
no rule orders and no triangulation.  The reading fixed here (both the oracle and the
library follow it, independently):

1. a cut element is bisected uniformly ``depth`` times; each leaf is classified like an
   element (``geometry.classify``);
2. a full leaf gets the tensor Gauss-Legendre rule with p+1 points per direction;
   an empty leaf is dropped;
3. a cut leaf is split into simplices along its main diagonal: 2 triangles
   (v00, v10, v11), (v00, v11, v01) in 2-D, the 6 Kuhn tetrahedra
   (v0, v0+e_a, v0+e_a+e_b, v111) for the permutations (a, b, c) in lexicographic order
   in 3-D;
4. psi is interpolated linearly from the simplex vertices and the simplex is clipped at
   psi_lin = 0.  A vertex is inside when psi > 0.  The crossing point on an edge from
   inside vertex a to outside vertex b is x_a + psi_a / (psi_a - psi_b) (x_b - x_a).
   With the inside vertices listed first in simplex order, the kept part is
     2-D  k=1: (a, x_ab, x_ac);   k=2: (a, b, x_bc), (a, x_bc, x_ac)
     3-D  k=1: (a, x_ab, x_ac, x_ad);
          k=2: prism (a, x_ac, x_ad | b, x_bc, x_bd);
          k=3: prism (a, b, c | x_ad, x_bd, x_cd);
     a prism (P0, P1, P2 | Q0, Q1, Q2) is split into (P0,P1,P2,Q2), (P0,P1,Q1,Q2), (P0,Q0,Q1,Q2);
   and the boundary facets are
     2-D  k=1: (x_ab, x_ac);  k=2: (x_ac, x_bc)
     3-D  k=1: (x_ab, x_ac, x_ad);  k=2: (x_ac, x_ad, x_bd), (x_ac, x_bd, x_bc);
          k=3: (x_ad, x_bd, x_cd);
   the outward normal is -grad(psi_lin) / |grad(psi_lin)|;
5. every kept simplex gets the collapsed (Duffy) Gauss-Legendre rule with p+2 points per
   direction, x = A + u (B - A) + u v (C - B) [+ u v w (D - C)], Jacobian u |det| (2-D) or
   u^2 v |det| (3-D); boundary segments get Gauss-Legendre with p+2 points, boundary
   triangles the collapsed rule with p+2 points per direction.
"""
from __future__ import annotations

import itertools

import numpy as np

from .geometry import CUT, EMPTY, FULL, leaf_boxes


def gauss01(n: int):
    """n-point Gauss-Legendre rule on [0, 1]."""
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (x + 1.0), 0.5 * w


def box_rule(lo: np.ndarray, hi: np.ndarray, n: int):
    """Tensor Gauss-Legendre rule with n points per direction on the box [lo, hi]."""
    d = len(lo)
    x1, w1 = gauss01(n)
    pts, wts = [], []
    for idx in itertools.product(range(n), repeat=d):
        idx = idx[::-1]
        pts.append([lo[k] + (hi[k] - lo[k]) * x1[idx[k]] for k in range(d)])
        wts.append(np.prod([(hi[k] - lo[k]) * w1[idx[k]] for k in range(d)]))
    return np.array(pts), np.array(wts)


def simplex_rule(V: np.ndarray, n: int):
    """Collapsed Gauss rule on the simplex with vertex rows V ((d+1) x d)."""
    x1, w1 = gauss01(n)
    d = V.shape[1]
    pts, wts = [], []
    if d == 2:
        A, B, C = V
        det = abs(np.linalg.det(np.stack([B - A, C - B])))
        for i in range(n):
            for j in range(n):
                u, v = x1[i], x1[j]
                pts.append(A + u * (B - A) + u * v * (C - B))
                wts.append(w1[i] * w1[j] * u * det)
    else:
        A, B, C, D = V
        det = abs(np.linalg.det(np.stack([B - A, C - B, D - C])))
        for i in range(n):
            for j in range(n):
                for k in range(n):
                    u, v, w = x1[i], x1[j], x1[k]
                    pts.append(A + u * (B - A) + u * v * (C - B) + u * v * w * (D - C))
                    wts.append(w1[i] * w1[j] * w1[k] * u * u * v * det)
    return np.array(pts), np.array(wts)


def facet_rule(F: np.ndarray, n: int):
    """Gauss rule on a boundary facet: a segment (2-D) or a triangle (3-D), rows = vertices."""
    x1, w1 = gauss01(n)
    if F.shape[1] == 2:
        P, Q = F
        L = np.linalg.norm(Q - P)
        return np.array([P + s * (Q - P) for s in x1]), w1 * L
    A, B, C = F
    area2 = np.linalg.norm(np.cross(B - A, C - B))
    pts, wts = [], []
    for i in range(n):
        for j in range(n):
            u, v = x1[i], x1[j]
            pts.append(A + u * (B - A) + u * v * (C - B))
            wts.append(w1[i] * w1[j] * u * area2)
    return np.array(pts), np.array(wts)


def kuhn_simplices(lo: np.ndarray, hi: np.ndarray):
    """Split the box [lo, hi] along its main diagonal (step 3 of the module docstring)."""
    d = len(lo)
    corner = lambda bits: np.array([hi[k] if bits[k] else lo[k] for k in range(d)])
    if d == 2:
        v00, v10, v01, v11 = corner((0, 0)), corner((1, 0)), corner((0, 1)), corner((1, 1))
        return [np.stack([v00, v10, v11]), np.stack([v00, v11, v01])]
    out = []
    for perm in itertools.permutations(range(3)):
        bits = [0, 0, 0]
        verts = [corner(bits)]
        for a in perm:
            bits[a] = 1
            verts.append(corner(bits))
        out.append(np.stack(verts))
    return out


def _cross(xa, xb, pa, pb):
    return xa + pa / (pa - pb) * (xb - xa)


def _prism(P, Q):
    return [np.stack([P[0], P[1], P[2], Q[2]]), np.stack([P[0], P[1], Q[1], Q[2]]),
            np.stack([P[0], Q[0], Q[1], Q[2]])]


def clip_simplex(V: np.ndarray, psi: np.ndarray):
    """Kept sub-simplices, boundary facets and outward normal of {psi_lin > 0} in simplex V."""
    d = V.shape[1]
    inside = [i for i in range(d + 1) if psi[i] > 0]
    outside = [i for i in range(d + 1) if psi[i] <= 0]
    k = len(inside)
    if k == d + 1:
        return [V], [], None
    if k == 0:
        return [], [], None
    # gradient of the linear interpolant: solve (V_i - V_0) . g = psi_i - psi_0
    g = np.linalg.solve(V[1:] - V[0], psi[1:] - psi[0])
    normal = -g / np.linalg.norm(g)
    X = lambda i, j: _cross(V[i], V[j], psi[i], psi[j])
    if d == 2:
        if k == 1:
            a, (b, c) = inside[0], outside
            return [np.stack([V[a], X(a, b), X(a, c)])], [np.stack([X(a, b), X(a, c)])], normal
        (a, b), c = inside, outside[0]
        return ([np.stack([V[a], V[b], X(b, c)]), np.stack([V[a], X(b, c), X(a, c)])],
                [np.stack([X(a, c), X(b, c)])], normal)
    if k == 1:
        a, (b, c, dd) = inside[0], outside
        return ([np.stack([V[a], X(a, b), X(a, c), X(a, dd)])],
                [np.stack([X(a, b), X(a, c), X(a, dd)])], normal)
    if k == 2:
        (a, b), (c, dd) = inside, outside
        P = [V[a], X(a, c), X(a, dd)]
        Q = [V[b], X(b, c), X(b, dd)]
        return (_prism(P, Q),
                [np.stack([X(a, c), X(a, dd), X(b, dd)]), np.stack([X(a, c), X(b, dd), X(b, c)])],
                normal)
    (a, b, c), dd = inside, outside[0]
    P = [V[a], V[b], V[c]]
    Q = [X(a, dd), X(b, dd), X(c, dd)]
    return _prism(P, Q), [np.stack([X(a, dd), X(b, dd), X(c, dd)])], normal


def cut_element_rule(geom, lo: np.ndarray, hi: np.ndarray, p: int, depth: int):
    """Volume and boundary quadrature of Omega_h inside the cut element [lo, hi].

    Returns (vol_pts, vol_wts, bnd_pts, bnd_wts, bnd_normals).
    """
    d = len(lo)
    vp, vw, bp, bw, bn = [], [], [], [], []
    for a, b in leaf_boxes(lo, hi, depth):
        cls = geom.classify(a, b)
        if cls == EMPTY:
            continue
        if cls == FULL:
            x, w = box_rule(a, b, p + 1)
            vp.append(x)
            vw.append(w)
            continue
        for S in kuhn_simplices(a, b):
            kept, facets, normal = clip_simplex(S, geom.psi(S))
            for T in kept:
                x, w = simplex_rule(T, p + 2)
                vp.append(x)
                vw.append(w)
            for F in facets:
                x, w = facet_rule(F, p + 2)
                bp.append(x)
                bw.append(w)
                bn.append(np.repeat(normal[None, :], len(w), axis=0))
    cat = lambda L, shape: np.concatenate(L) if L else np.zeros(shape)
    return (cat(vp, (0, d)), cat(vw, (0,)), cat(bp, (0, d)), cat(bw, (0,)), cat(bn, (0, d)))
