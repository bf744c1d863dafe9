"""Learned correction stage inside flexible CG: the plain FP64 definition.

TEST INFRASTRUCTURE ONLY (like the rest of ``oracle/``): only the tests, ``smoke()`` and
the CPU-baseline leg of ``bench.py`` import it.

The paper has no learned component: its preconditioner is the V-cycle of Algorithm 1
inside CG (Sec. 3.2).  This module defines the extension built beside it, in the terms
of the published methods it uses:

* the network N: three 3-D convolution layers on the background grid of the finest
  level's basis functions (1 -> 16 -> 16 -> 1 channels, 3 x 3 x 3 kernels, no biases,
  zero padding, ReLU after the first two layers), evaluated with its weights and its
  stored activations rounded to bfloat16 and its sums taken exactly (FP64 here);
  a layer is the cross-correlation y[v, o] = sum_t sum_i W[t, o, i] x[v + off_t, i],
  off_t = (dz, dy, dx) with t = 9 (dz + 1) + 3 (dy + 1) + (dx + 1);
* the stage: after the V-cycle z = B r, the residual left is r1 = r - A z, the network
  proposes c = N(r1) on the active functions, and z <- z + omega c with the step
  omega = (r1 . c) / (c . A c) that minimises the A-norm of the error left in the
  correction equation A e = r (omega = 0 when c . A c is not positive);
* training data: the V-cycle's own residual/error pairs, e1 = (I - B A) e0 and
  r1 = A e1 for random e0, both divided by the root mean square of e1 over the active
  functions, and every input multiplied by the set's scale 1 / mean(rms(r1)) (A scales
  with the mesh size; one factor for the whole set keeps the pairs one consistent map, and
  the stage's step omega makes the factor irrelevant when the network is used); the loss is the masked squared error sum_v m_v (N(r1)_v - e1_v)^2 times a
  caller-given scale (1 / number of active functions);
* gradients by the chain rule (reverse mode), Adam (Kingma and Ba, 2015, Algorithm 1)
  with bias correction on FP32 master weights;
* flexible CG with the Polak-Ribiere beta (z_{k+1} . (r_{k+1} - r_k)) / (z_k . r_k),
  as the stage makes the preconditioner vary from step to step (Notay, 2000), and its
  truncated form FCG(m), which A-orthogonalises each new direction against the last m
  directions instead of one (Notay, 2000): FCG(1) is the Polak-Ribiere form.
"""
from __future__ import annotations

import numpy as np

C = 16                                    # hidden channels
LAYERS = ((1, C), (C, C), (C, 1))         # (in, out) channels per layer
OFFSETS = [(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]
N_WEIGHTS = sum(27 * ci * co for ci, co in LAYERS)


def round_bf16(x):
    """Round to the nearest bfloat16 (8 significant bits, ties to even), from FP64."""
    x = np.asarray(x, dtype=np.float64)
    m, e = np.frexp(x)                    # x = m 2^e, 0.5 <= |m| < 1
    ulp = np.ldexp(1.0, e - 8)
    return np.where(x == 0.0, 0.0, np.rint(x / ulp) * ulp)


def to_input(r):
    """The network's input as stored: FP64 -> FP32 -> bfloat16 (each rounding to nearest even)."""
    return round_bf16(np.asarray(r, dtype=np.float64).astype(np.float32).astype(np.float64))


def split_weights(w):
    """Flat weight vector -> [W1, W2, W3], W_l[t, out, in]."""
    w = np.asarray(w, dtype=np.float64)
    out, k = [], 0
    for ci, co in LAYERS:
        out.append(w[k:k + 27 * co * ci].reshape(27, co, ci))
        k += 27 * co * ci
    return out


def join_weights(Ws):
    return np.concatenate([W.reshape(-1) for W in Ws])


def shift(x, off):
    """y[:, v] = x[:, v + off] with zero outside the grid; x has shape (channels, nz, ny, nx)."""
    y = np.zeros_like(x)
    src, dst = [slice(None)], [slice(None)]
    for o, n in zip(off, x.shape[1:]):
        src.append(slice(max(o, 0), n + min(o, 0)))
        dst.append(slice(max(-o, 0), n + min(-o, 0)))
    y[tuple(dst)] = x[tuple(src)]
    return y


def conv3d(x, W):
    """y[o, v] = sum_t sum_i W[t, o, i] x[i, v + off_t] (zero padding)."""
    y = np.zeros((W.shape[1],) + x.shape[1:])
    for t, off in enumerate(OFFSETS):
        y += np.einsum("oi,izyx->ozyx", W[t], shift(x, off))
    return y


def conv3d_input_grad(dy, W):
    """dL/dx of y = conv3d(x, W): dx[i, u] = sum_t sum_o W[t, o, i] dy[o, u - off_t]."""
    dx = np.zeros((W.shape[2],) + dy.shape[1:])
    for t, off in enumerate(OFFSETS):
        dx += np.einsum("oi,ozyx->izyx", W[t], shift(dy, tuple(-o for o in off)))
    return dx


def conv3d_weight_grad(dy, x):
    """dL/dW of y = conv3d(x, W): dW[t, o, i] = sum_v dy[o, v] x[i, v + off_t]."""
    return np.stack([np.einsum("ozyx,izyx->oi", dy, shift(x, off)) for off in OFFSETS])


def forward(w, r_grid, mask, bf16: bool = True, in_scale: float = 1.0):
    """N(r) on a grid (nz, ny, nx) with the active mask (same shape, 0/1).

    The network sees the input on the active functions only (zero elsewhere).
    Returns the output (masked, FP64) and the activations (input, a1, a2) as stored.
    With bf16, the weights, the input and the hidden activations are rounded to bfloat16
    where the kernels store them; the sums and the output stay exact.
    """
    Ws = split_weights(w)
    rnd = round_bf16 if bf16 else (lambda v: v)
    Ws = [rnd(W) for W in Ws]
    r_grid = np.asarray(r_grid, dtype=np.float64) * in_scale * mask
    x = (to_input(r_grid) if bf16 else r_grid)[None]
    a1 = rnd(np.maximum(conv3d(x, Ws[0]), 0.0))
    a2 = rnd(np.maximum(conv3d(a1, Ws[1]), 0.0))
    out = conv3d(a2, Ws[2])[0] * mask
    return out, (x, a1, a2)


def loss_and_grads(w, r_grid, e_grid, mask, scale: float, bf16: bool = True, in_scale: float = 1.0):
    """Loss scale * sum_v m_v (N(in_scale r)_v - e_v)^2 and its gradient with respect to
    the (FP32 master) weights, by reverse mode through the stored activations."""
    Ws = split_weights(w)
    rnd = round_bf16 if bf16 else (lambda v: v)
    Wq = [rnd(W) for W in Ws]
    out, (x, a1, a2) = forward(w, r_grid, mask, bf16, in_scale)
    diff = (out - e_grid) * mask
    loss = scale * float(np.sum(diff * diff))
    d3 = (2.0 * diff * scale)[None]
    g3 = conv3d_weight_grad(d3, a2)
    d2 = conv3d_input_grad(d3, Wq[2]) * (a2 > 0)
    g2 = conv3d_weight_grad(d2, a1)
    d1 = conv3d_input_grad(d2, Wq[1]) * (a1 > 0)
    g1 = conv3d_weight_grad(d1, x)
    return loss, join_weights([g1, g2, g3])


class Adam:
    """Adam with bias correction (Kingma and Ba, 2015, Algorithm 1)."""

    def __init__(self, n: int, lr: float, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8):
        self.m, self.v, self.t = np.zeros(n), np.zeros(n), 0
        self.lr, self.b1, self.b2, self.eps = lr, beta1, beta2, eps

    def step(self, w, g):
        self.t += 1
        self.m = self.b1 * self.m + (1.0 - self.b1) * g
        self.v = self.b2 * self.v + (1.0 - self.b2) * g * g
        mhat = self.m / (1.0 - self.b1 ** self.t)
        vhat = self.v / (1.0 - self.b2 ** self.t)
        return w - self.lr * mhat / (np.sqrt(vhat) + self.eps)


def training_pair(A, precondition, e0):
    """One V-cycle's residual/error pair from a random error e0 (active functions):
    e1 = e0 - B A e0, r1 = A e1, both divided by the root mean square of e1."""
    e1 = e0 - precondition(A @ e0)
    r1 = A @ e1
    s = np.sqrt(np.mean(e1 * e1))
    return r1 / s, e1 / s


def input_scale(pairs):
    """The training set's input scale: 1 / mean over its pairs of rms(r1)."""
    return 1.0 / float(np.mean([np.sqrt(np.mean(r * r)) for r, _ in pairs]))


def stage(A, r, z, net):
    """z + omega N(r - A z) with the energy-minimising omega (0 if c . A c <= 0)."""
    r1 = r - A @ z
    c = net(r1)
    Ac = A @ c
    den = float(c @ Ac)
    omega = float(r1 @ c) / den if den > 0.0 else 0.0
    return z + omega * c, omega


def flexible_pcg(A, b, precond, rtol: float = 1e-8, maxit: int = 1000):
    """CG with the Polak-Ribiere beta; returns (x, iterations, relative residual history)."""
    x = np.zeros_like(b)
    r = b.copy()
    bnorm = np.linalg.norm(b)
    hist = [np.linalg.norm(r) / bnorm]
    z = precond(r)
    p = z.copy()
    rz = float(r @ z)
    for k in range(1, maxit + 1):
        q = A @ p
        alpha = rz / float(p @ q)
        x = x + alpha * p
        r_new = r - alpha * q
        hist.append(np.linalg.norm(r_new) / bnorm)
        if hist[-1] <= rtol:
            return x, k, hist
        z = precond(r_new)
        beta = float(z @ (r_new - r)) / rz
        rz = float(z @ r_new)
        p = z + beta * p
        r = r_new
    return x, maxit, hist


def fcg(A, b, precond, m: int, rtol: float = 1e-8, maxit: int = 1000):
    """Truncated flexible CG, FCG(m): p_k = z_k minus its A-projections on the last m
    directions, alpha_k = (r_k . p_k) / (p_k . A p_k).  Returns (x, iterations, history)."""
    x = np.zeros_like(b)
    r = b.copy()
    bnorm = np.linalg.norm(b)
    hist = [np.linalg.norm(r) / bnorm]
    dirs = []                             # (p_j, A p_j, p_j . A p_j) of the last m steps
    for k in range(1, maxit + 1):
        z = precond(r)
        p = z.copy()
        for pj, qj, pqj in dirs:
            p = p - (float(z @ qj) / pqj) * pj
        q = A @ p
        pq = float(p @ q)
        alpha = float(r @ p) / pq
        x = x + alpha * p
        r = r - alpha * q
        hist.append(np.linalg.norm(r) / bnorm)
        if hist[-1] <= rtol:
            return x, k, hist
        dirs = (dirs + [(p, q, pq)])[-m:]
    return x, maxit, hist
