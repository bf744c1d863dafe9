"""GB300-native immersed-FE multigrid-preconditioned CG (de Prenter et al., arXiv 1903.10977).

Thin Python binding over the C-ABI library ``libimgm.so`` (declared in include/imgm.h):
argument marshalling only.  Every step of the solve runs in the library's CUDA kernels;
there is no Python or CPU implementation of any of them here.  Importing this package
fails loudly when the library has not been built (``python
paper_1903_10977_gb300/build.py``).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libimgm.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with `python paper_1903_10977_gb300/build.py`")

_lib = ctypes.CDLL(LIB_PATH)

IMGM_OK, IMGM_MAX_ITER = 0, 1
ERRORS = {-1: "invalid argument", -2: "unsupported", -3: "CUDA error", -4: "not SPD", -5: "CG breakdown"}


class Geometry(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n_holes", ctypes.c_int), ("centers", ctypes.POINTER(ctypes.c_double)),
                ("radii", ctypes.POINTER(ctypes.c_double)), ("lo", ctypes.c_double), ("hi", ctypes.c_double)]


class Config(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("basis", ctypes.c_int), ("degree", ctypes.c_int), ("levels", ctypes.c_int),
                ("depth", ctypes.c_int), ("bc", ctypes.c_int), ("gamma", ctypes.c_double),
                ("precision", ctypes.c_int), ("smoother", ctypes.c_int)]


class Result(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("status", ctypes.c_int), ("rel_residual", ctypes.c_double),
                ("true_rel_residual", ctypes.c_double), ("kernel_launches", ctypes.c_int64)]


class LevelInfo(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int64) for k in ("n_grid", "n_active", "m", "n_band", "n_blocks", "block_entries",
                                              "max_block", "pruned")]


_H = ctypes.c_void_p
_P = ctypes.c_void_p
_D = ctypes.c_double
_I = ctypes.c_int
_I64 = ctypes.c_int64

_SIGS = {
    "imgm_setup": (_I, [ctypes.POINTER(Geometry), ctypes.POINTER(Config), ctypes.POINTER(_H)]),
    "imgm_setup_host": (_I, [ctypes.POINTER(Geometry), ctypes.POINTER(Config), ctypes.POINTER(_H)]),
    "imgm_destroy": (None, [_H]),
    "imgm_last_error": (ctypes.c_char_p, [_H]),
    "imgm_levels": (_I, [_H]),
    "imgm_get_level_info": (_I, [_H, _I, ctypes.POINTER(LevelInfo)]),
    "imgm_active_mask": (_I, [_H, _I, _P]),
    "imgm_rhs": (_I, [_H, _P, _P]),
    "imgm_apply_operator": (_I, [_H, _I, _P, _P, _P]),
    "imgm_smooth": (_I, [_H, _I, _P, _P, _P]),
    "imgm_restrict": (_I, [_H, _I, _P, _P, _P]),
    "imgm_prolong": (_I, [_H, _I, _P, _P, _P]),
    "imgm_coarse_solve": (_I, [_H, _P, _P, _P]),
    "imgm_apply_preconditioner": (_I, [_H, _P, _P, _P]),
    "imgm_pcg_solve": (_I, [_H, _P, _P, _D, _I, ctypes.POINTER(Result), _P, _P]),
    "imgm_pcg_solve_host": (_I, [_H, _P, _P, _D, _I, ctypes.POINTER(Result), _P]),
    "imgm_residual_norm2": (_I, [_H, _P, _P, _P, _P]),
    "imgm_residual_norm2_noalloc": (_I, [_H, _P, _P, _P, _P]),
    "imgm_host_operator_rows": (_I, [_H, _I, _I64, _P, _P]),
    "imgm_host_rhs": (_I, [_H, _P]),
    "imgm_host_block_sizes": (_I, [_H, _I, ctypes.POINTER(_I64), ctypes.POINTER(_I64), ctypes.POINTER(_I64)]),
    "imgm_host_blocks": (_I, [_H, _I, _P, _P, _P, _P, _P]),
    "imgm_host_restriction": (_I, [_H, _I, _P, _P]),
    "imgm_host_coarse_size": (_I, [_H, ctypes.POINTER(_I64)]),
    "imgm_host_coarse": (_I, [_H, _P, _P]),
    "imgm_clone": (_I, [_H, ctypes.POINTER(_H)]),
    "imgm_batch_create": (_I, [ctypes.POINTER(_H), _I, ctypes.POINTER(_P)]),
    "imgm_batch_solve": (_I, [_P, ctypes.POINTER(_P), ctypes.POINTER(_P), _D, _I, ctypes.POINTER(Result), _P]),
    "imgm_batch_destroy": (None, [_P]),
    "imgm_net_create": (_I, [_P, ctypes.POINTER(_P)]),
    "imgm_net_destroy": (ctypes.c_int, [_P]),
    "imgm_set_fcg": (ctypes.c_int, [_H, ctypes.c_int]),
    "imgm_net_get_weights": (_I, [_P, _P]),
    "imgm_net_get_grads": (_I, [_P, _P]),
    "imgm_net_forward": (_I, [_P, _I, _I, _I, _P, _P, _P, _P]),
    "imgm_net_zero_grad": (_I, [_P, _P]),
    "imgm_net_accumulate": (_I, [_P, _I, _I, _I, _P, _P, _P, _D, _D, _P, _P]),
    "imgm_net_adam_step": (_I, [_P, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float, _P]),
    "imgm_set_net": (_I, [_H, _P]),
    "imgm_learned_stage": (_I, [_H, _P, _P, _P, _P]),
    "imgm_learned_pair": (_I, [_H, _P, _P, _P, _P, _P]),
}
NET_WEIGHTS = 7776
for _name, (_res, _args) in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args

EXPORTED = tuple(_SIGS)


class ImgmError(RuntimeError):
    pass


def _ptr(t):
    """Device pointer of a contiguous float64 CUDA tensor."""
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous():
        raise TypeError("expected a contiguous float64 CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


class Solver:
    """One immersed Poisson problem and its multigrid hierarchy on the current GPU.

    geometry: centers (k x dim) and radii (k) of the holes cut out of the box [lo, hi]^dim.
    host_only=True builds the hierarchy without the GPU (setup inspection only).
    """

    def __init__(self, dim, centers, radii, n, degree=2, levels=3, depth=0, bc=1, basis=0, gamma=0.0,
                 lo=0.0, hi=1.0, host_only=False, precision=0, smoother=0):
        self._c = np.ascontiguousarray(np.asarray(centers, dtype=np.float64).reshape(-1, dim))
        self._r = np.ascontiguousarray(np.asarray(radii, dtype=np.float64).reshape(-1))
        g = Geometry(dim, int(self._r.size), self._c.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                     self._r.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), lo, hi)
        cfg = Config(n, basis, degree, levels, depth, bc, gamma, precision, smoother)
        h = _H()
        fn = _lib.imgm_setup_host if host_only else _lib.imgm_setup
        rc = fn(ctypes.byref(g), ctypes.byref(cfg), ctypes.byref(h))
        if rc != IMGM_OK:
            raise ImgmError(f"setup failed ({ERRORS.get(rc, rc)}): {_lib.imgm_last_error(None).decode()}")
        self._h = h
        self.dim, self.p, self.host_only, self.precision = dim, degree, host_only, precision
        self.L = _lib.imgm_levels(h)
        self.ncoef = (2 * degree + 1) ** dim

    def _check(self, rc):
        if rc < 0:
            raise ImgmError(f"{ERRORS.get(rc, rc)}: {_lib.imgm_last_error(self._h).decode()}")
        return rc

    def close(self):
        if getattr(self, "_h", None):
            _lib.imgm_destroy(self._h)
            self._h = None

    def clone(self) -> "Solver":
        """Another solve context of the same problem (shared hierarchy, own vectors)."""
        h = _H()
        rc = _lib.imgm_clone(self._h, ctypes.byref(h))
        if rc != IMGM_OK:
            raise ImgmError(f"clone failed ({ERRORS.get(rc, rc)}): {_lib.imgm_last_error(None).decode()}")
        c = object.__new__(Solver)
        c.__dict__.update({k: v for k, v in self.__dict__.items() if k != "_h"})
        c._h = h
        c._parent = self              # keeps the Python object of the source alive as well
        return c

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---------------------------------------------------------------- sizes
    def level_info(self, level: int) -> dict:
        li = LevelInfo()
        self._check(_lib.imgm_get_level_info(self._h, level, ctypes.byref(li)))
        return {k: int(getattr(li, k)) for k, _ in LevelInfo._fields_}

    def n_grid(self, level: int | None = None) -> int:
        return self.level_info(self.L if level is None else level)["n_grid"]

    def active_mask(self, level: int | None = None) -> np.ndarray:
        level = self.L if level is None else level
        out = np.zeros(self.n_grid(level), dtype=np.uint8)
        self._check(_lib.imgm_active_mask(self._h, level, out.ctypes.data_as(ctypes.c_void_p)))
        return out

    # ----------------------------------------------------------- GPU calls
    def rhs(self, out=None, stream=None):
        import torch
        out = torch.empty(self.n_grid(), dtype=torch.float64, device="cuda") if out is None else out
        self._check(_lib.imgm_rhs(self._h, _ptr(out), _stream(stream)))
        return out

    def apply_operator(self, x, y=None, level=None, stream=None):
        import torch
        level = self.L if level is None else level
        y = torch.empty_like(x) if y is None else y
        self._check(_lib.imgm_apply_operator(self._h, level, _ptr(x), _ptr(y), _stream(stream)))
        return y

    def smooth(self, r, z=None, level=None, stream=None):
        import torch
        level = self.L if level is None else level
        z = torch.empty_like(r) if z is None else z
        self._check(_lib.imgm_smooth(self._h, level, _ptr(r), _ptr(z), _stream(stream)))
        return z

    def restrict(self, r, level=None, out=None, stream=None):
        import torch
        level = self.L if level is None else level
        out = torch.empty(self.n_grid(level - 1), dtype=torch.float64, device=r.device) if out is None else out
        self._check(_lib.imgm_restrict(self._h, level, _ptr(r), _ptr(out), _stream(stream)))
        return out

    def prolong(self, xc, level=None, out=None, stream=None):
        import torch
        level = self.L if level is None else level
        out = torch.empty(self.n_grid(level), dtype=torch.float64, device=xc.device) if out is None else out
        self._check(_lib.imgm_prolong(self._h, level, _ptr(xc), _ptr(out), _stream(stream)))
        return out

    def coarse_solve(self, r, out=None, stream=None):
        import torch
        out = torch.empty_like(r) if out is None else out
        self._check(_lib.imgm_coarse_solve(self._h, _ptr(r), _ptr(out), _stream(stream)))
        return out

    def apply_preconditioner(self, r, z=None, stream=None):
        import torch
        z = torch.empty_like(r) if z is None else z
        self._check(_lib.imgm_apply_preconditioner(self._h, _ptr(r), _ptr(z), _stream(stream)))
        return z

    def pcg_solve(self, b, x=None, rtol=1e-8, maxit=1000, hist=False, stream=None):
        """Solve A x = b from x (zeros when None); returns (x, result dict, history or None)."""
        import torch
        x = torch.zeros_like(b) if x is None else x
        hbuf = torch.zeros(maxit + 1, dtype=torch.float64, device=b.device) if hist else None
        res = Result()
        rc = _lib.imgm_pcg_solve(self._h, _ptr(b), _ptr(x), rtol, maxit, ctypes.byref(res),
                                 _ptr(hbuf) if hist else None, _stream(stream))
        self._check(rc)
        out = {"iterations": res.iterations, "status": res.status, "rel_residual": res.rel_residual,
               "true_rel_residual": res.true_rel_residual, "kernel_launches": res.kernel_launches}
        if hist:
            hbuf = hbuf[: res.iterations + 1]
        return x, out, hbuf

    # ------------------------------------------------------ learned stage
    def set_net(self, net: "Net | None"):
        """Attach a network to this context's solves (None detaches); see imgm_set_net."""
        self._check(_lib.imgm_set_net(self._h, net._n if net is not None else None))
        self._net = net               # keeps the network alive while attached

    def set_fcg(self, m: int):
        """Truncated flexible CG with m stored directions for the following solves (0: off)."""
        self._check(_lib.imgm_set_fcg(self._h, int(m)))

    def learned_stage(self, r, z, omega=None, stream=None):
        """z <- z + omega N(r - A z) in place with the attached network (z = B r on entry)."""
        self._check(_lib.imgm_learned_stage(self._h, _ptr(r), _ptr(z), _ptr(omega) if omega is not None else None,
                                            _stream(stream)))
        return z

    def learned_pair(self, e0, r1=None, e1=None, r_rms=None, stream=None):
        """Training pair of the V-cycle: e1 = e0 - B A e0, r1 = A e1, both divided by rms(e1);
        r_rms (optional one-element float64 CUDA tensor) receives rms(r1) afterwards."""
        import torch
        r1 = torch.empty_like(e0) if r1 is None else r1
        e1 = torch.empty_like(e0) if e1 is None else e1
        self._check(_lib.imgm_learned_pair(self._h, _ptr(e0), _ptr(r1), _ptr(e1),
                                           _ptr(r_rms) if r_rms is not None else None, _stream(stream)))
        return r1, e1

    def residual_norm2(self, b, x, out=None, stream=None):
        """||b - A x||^2 on the finest level, into a one-element CUDA tensor."""
        import torch
        out = torch.empty(1, dtype=torch.float64, device=b.device) if out is None else out
        self._check(_lib.imgm_residual_norm2(self._h, _ptr(b), _ptr(x), _ptr(out), _stream(stream)))
        return out

    def residual_norm2_noalloc(self, b, x, out, stream=None):
        """residual_norm2 without any device allocation by the library (out: a caller-owned
        one-element float64 CUDA tensor); see imgm_residual_norm2_noalloc in imgm.h."""
        self._check(_lib.imgm_residual_norm2_noalloc(self._h, _ptr(b), _ptr(x), _ptr(out), _stream(stream)))
        return out

    def pcg_solve_host(self, b_host: np.ndarray, x_host: np.ndarray | None = None, rtol=1e-8, maxit=1000,
                       stream=None):
        """Solve with host (ideally pinned) buffers: b -> device, solve, x -> host."""
        b_host = np.ascontiguousarray(b_host, dtype=np.float64)
        x_host = np.empty_like(b_host) if x_host is None else x_host
        res = Result()
        rc = _lib.imgm_pcg_solve_host(self._h, ctypes.c_void_p(b_host.ctypes.data),
                                      ctypes.c_void_p(x_host.ctypes.data), rtol, maxit, ctypes.byref(res),
                                      _stream(stream))
        self._check(rc)
        return x_host, {"iterations": res.iterations, "status": res.status, "rel_residual": res.rel_residual,
                        "true_rel_residual": res.true_rel_residual}

    def pcg_solve_host_ptr(self, b_ptr: int, x_ptr: int, rtol=1e-8, maxit=1000, stream=None):
        """pcg_solve_host on raw host addresses (e.g. pinned torch tensors' data_ptr())."""
        res = Result()
        rc = _lib.imgm_pcg_solve_host(self._h, ctypes.c_void_p(b_ptr), ctypes.c_void_p(x_ptr), rtol, maxit,
                                      ctypes.byref(res), _stream(stream))
        self._check(rc)
        return {"iterations": res.iterations, "status": res.status, "rel_residual": res.rel_residual,
                "true_rel_residual": res.true_rel_residual}

    # ------------------------------------------------------- setup inspection
    def host_operator_rows(self, rows, level=None) -> np.ndarray:
        level = self.L if level is None else level
        rows = np.ascontiguousarray(rows, dtype=np.int64)
        out = np.zeros((rows.size, self.ncoef))
        self._check(_lib.imgm_host_operator_rows(self._h, level, rows.size, rows.ctypes.data_as(ctypes.c_void_p),
                                                 out.ctypes.data_as(ctypes.c_void_p)))
        return out

    def host_rhs(self) -> np.ndarray:
        out = np.zeros(self.n_grid())
        self._check(_lib.imgm_host_rhs(self._h, out.ctypes.data_as(ctypes.c_void_p)))
        return out

    def host_block_sizes(self, level=None):
        """(stored blocks, sum of their sizes n_j, sum of n_j^2) of a level."""
        level = self.L if level is None else level
        nb, ni, nv = _I64(), _I64(), _I64()
        self._check(_lib.imgm_host_block_sizes(self._h, level, ctypes.byref(nb), ctypes.byref(ni), ctypes.byref(nv)))
        return nb.value, ni.value, nv.value

    def host_blocks(self, level=None):
        level = self.L if level is None else level
        nb, ni, nv = _I64(), _I64(), _I64()
        self._check(_lib.imgm_host_block_sizes(self._h, level, ctypes.byref(nb), ctypes.byref(ni), ctypes.byref(nv)))
        ptr = np.zeros(nb.value + 1, dtype=np.int64)
        idx = np.zeros(ni.value, dtype=np.int32)
        vptr = np.zeros(nb.value + 1, dtype=np.int64)
        val = np.zeros(nv.value)
        dinv = np.zeros(self.n_grid(level))
        self._check(_lib.imgm_host_blocks(self._h, level, *(a.ctypes.data_as(ctypes.c_void_p)
                                                             for a in (ptr, idx, vptr, val, dinv))))
        return ptr, idx, vptr, val, dinv

    def host_restriction(self, level=None):
        level = self.L if level is None else level
        mc = self.level_info(level - 1)["m"]
        first = np.zeros(mc, dtype=np.int32)
        w = np.zeros((mc, self.p + 2))
        self._check(_lib.imgm_host_restriction(self._h, level, first.ctypes.data_as(ctypes.c_void_p),
                                               w.ctypes.data_as(ctypes.c_void_p)))
        return first, w

    def host_coarse(self):
        nc = _I64()
        self._check(_lib.imgm_host_coarse_size(self._h, ctypes.byref(nc)))
        rows = np.zeros(nc.value, dtype=np.int32)
        inv = np.zeros((nc.value, nc.value))
        self._check(_lib.imgm_host_coarse(self._h, rows.ctypes.data_as(ctypes.c_void_p),
                                          inv.ctypes.data_as(ctypes.c_void_p)))
        return rows, inv


def _result_dict(res) -> dict:
    return {"iterations": res.iterations, "status": res.status, "rel_residual": res.rel_residual,
            "true_rel_residual": res.true_rel_residual, "kernel_launches": res.kernel_launches}


class Batch:
    """CG solves of several contexts (Solver objects, distinct; clones for more right-hand
    sides of one problem) run concurrently by one CUDA graph launch."""

    def __init__(self, solvers):
        self.solvers = list(solvers)
        arr = (_H * len(self.solvers))(*[s._h for s in self.solvers])
        b = _P()
        rc = _lib.imgm_batch_create(arr, len(self.solvers), ctypes.byref(b))
        if rc != IMGM_OK:
            raise ImgmError(f"batch failed ({ERRORS.get(rc, rc)}): {_lib.imgm_last_error(None).decode()}")
        self._b = b

    def solve(self, bs, xs=None, rtol=1e-8, maxit=1000, stream=None):
        """Solves solver[k] x_k = bs[k] for all k (xs: initial guesses, zeros when None);
        returns (xs, list of result dicts)."""
        import torch
        n = len(self.solvers)
        xs = [torch.zeros_like(b) for b in bs] if xs is None else xs
        pb = (_P * n)(*[_ptr(b).value for b in bs])
        px = (_P * n)(*[_ptr(x).value for x in xs])
        res = (Result * n)()
        rc = _lib.imgm_batch_solve(self._b, pb, px, rtol, maxit, res, _stream(stream))
        if rc < 0:
            raise ImgmError(f"{ERRORS.get(rc, rc)}: {_lib.imgm_last_error(None).decode()}")
        return xs, [_result_dict(r) for r in res]

    def close(self):
        if getattr(self, "_b", None):
            _lib.imgm_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _mask_ptr(mask):
    import torch
    if mask is None:
        return None
    if not isinstance(mask, torch.Tensor) or not mask.is_cuda or mask.dtype != torch.uint8 or not mask.is_contiguous():
        raise TypeError("expected a contiguous uint8 CUDA mask")
    return ctypes.c_void_p(mask.data_ptr())


class Net:
    """The learned stage's network (imgm_net): FP32 master weights, Adam state, bf16 copies.

    weights: IMGM_NET_WEIGHTS floats, layers 1 -> 16 -> 16 -> 1, each [tap][out][in]."""

    def __init__(self, weights):
        w = np.ascontiguousarray(np.asarray(weights, dtype=np.float32).reshape(-1))
        if w.size != NET_WEIGHTS:
            raise ValueError(f"expected {NET_WEIGHTS} weights, got {w.size}")
        n = _P()
        rc = _lib.imgm_net_create(w.ctypes.data_as(ctypes.c_void_p), ctypes.byref(n))
        if rc != IMGM_OK:
            raise ImgmError(f"network creation failed ({ERRORS.get(rc, rc)}): {_lib.imgm_last_error(None).decode()}")
        self._n = n

    def _check(self, rc):
        if rc < 0:
            raise ImgmError(f"{ERRORS.get(rc, rc)}: {_lib.imgm_last_error(None).decode()}")
        return rc

    def close(self):
        """Frees the network; raises ImgmError while a handle or a batch still holds it."""
        if getattr(self, "_n", None):
            self._check(_lib.imgm_net_destroy(self._n))
            self._n = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def weights(self) -> np.ndarray:
        out = np.zeros(NET_WEIGHTS, dtype=np.float32)
        self._check(_lib.imgm_net_get_weights(self._n, out.ctypes.data_as(ctypes.c_void_p)))
        return out

    def grads(self) -> np.ndarray:
        out = np.zeros(NET_WEIGHTS, dtype=np.float32)
        self._check(_lib.imgm_net_get_grads(self._n, out.ctypes.data_as(ctypes.c_void_p)))
        return out

    def forward(self, x, shape, mask=None, out=None, stream=None):
        """N(x) on a grid of shape (nz, ny, nx) (x: float64 CUDA vector, x fastest)."""
        import torch
        nz, ny, nx = shape
        out = torch.empty_like(x) if out is None else out
        self._check(_lib.imgm_net_forward(self._n, nx, ny, nz, _ptr(x), _mask_ptr(mask), _ptr(out), _stream(stream)))
        return out

    def zero_grad(self, stream=None):
        self._check(_lib.imgm_net_zero_grad(self._n, _stream(stream)))

    def accumulate(self, x, target, shape, loss, mask=None, scale=1.0, in_scale=1.0, stream=None):
        """Adds the gradient of scale * sum m (N(in_scale x) - target)^2; adds the loss to loss[0]."""
        nz, ny, nx = shape
        self._check(_lib.imgm_net_accumulate(self._n, nx, ny, nz, _ptr(x), _ptr(target), _mask_ptr(mask), in_scale,
                                             scale, _ptr(loss), _stream(stream)))

    def adam_step(self, lr, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
        self._check(_lib.imgm_net_adam_step(self._n, lr, beta1, beta2, eps, _stream(stream)))


def train_net(net: Net, pairs, shape, steps: int, lr: float = 1e-3, batch: int = 1, in_scale: float = 1.0,
              stream=None):
    """Adam on the V-cycle's residual/error pairs [(r1, e1, mask), ...] on grids of one
    shape (nz, ny, nx) (mask: uint8 CUDA vector of the pair's active functions): each step
    accumulates the gradient of `batch` pairs, taken in turn, and applies one update.  The
    loss of a pair is scaled by 1 / (batch * its number of active functions); every input
    is multiplied by in_scale (the set's 1 / mean rms(r1), see Solver.learned_pair).
    Returns the per-step losses (device tensor)."""
    import torch
    losses = torch.zeros(steps, dtype=torch.float64, device=pairs[0][0].device)
    scales = [1.0 / (batch * max(int(m.sum().item()), 1)) for _, _, m in pairs]
    k = 0
    for it in range(steps):
        net.zero_grad(stream)
        for _ in range(batch):
            r1, e1, mask = pairs[k % len(pairs)]
            net.accumulate(r1, e1, shape, losses[it:it + 1], mask=mask, scale=scales[k % len(pairs)],
                           in_scale=in_scale, stream=stream)
            k += 1
        net.adam_step(lr, stream=stream)
    return losses
