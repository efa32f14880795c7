"""Python binding of the md library: argument marshalling over the C ABI.

Every computation runs in the library's CUDA kernels; this module only
checks shapes/devices, passes pointers and streams, and raises on errors.
Tensors are torch CUDA tensors (torch provides device memory and streams).
"""
from __future__ import annotations

import ctypes as C
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import torch

from . import _lib as L


# Default damping of the Jacobi smoothing: the weighted Jacobi of the
# multigrid literature the paper's smoother follows (Trottenberg et al.),
# omega = 2/3.  For the Q1 stiffness stencil (centre 8/3, edges -1/6, corners
# -1/12, times h) the eigenvalues of D^{-1} K are
# 1 - (c1 c2 + c1 c3 + c2 c3)/4 - c1 c2 c3/4, c_i = cos(theta_i), which span
# [1/2, 3/2] on the high frequencies: omega = 2/3 damps those by at least 2/3.
# The library scales the rows the coupling makes heavy so that the spectrum
# of its D^{-1} C stays within (0, 2], where every omega < 1 contracts.
SMOOTH_OMEGA = 2.0 / 3.0


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _ptr(t: torch.Tensor | None, dtype=None, numel=None, name="tensor"):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name} must have {numel} entries, got {t.numel()}")
    return C.c_void_p(t.data_ptr())


class Operator:
    """One assembled instance: grid N, graph, radius, coupling beta (md_assemble)."""

    def __init__(self, N: int, graph: dict, beta: float, *, k_omega=1.0, sigma_omega=0.0, k_lambda=1.0,
                 dirichlet: bool = True, dirichlet_1d=None, u_d: float = 1.0):
        lib = L.load()
        xyz = np.ascontiguousarray(graph["xyz"], dtype=np.float64)
        edges = np.ascontiguousarray(graph["edges"], dtype=np.int32)
        g = L.MdGraph(len(xyz), xyz.ctypes.data_as(C.POINTER(C.c_double)), len(edges),
                      edges.ctypes.data_as(C.POINTER(C.c_int)), int(graph["elems"]))
        d1 = np.ascontiguousarray(dirichlet_1d if dirichlet_1d is not None else [], dtype=np.int32)
        prm = L.MdParams(k_omega, sigma_omega, k_lambda, 0 if dirichlet else 1, len(d1),
                         d1.ctypes.data_as(C.POINTER(C.c_int)) if len(d1) else None, float(u_d))
        h = C.c_void_p()
        torch.cuda.init()
        L.check(lib.md_assemble(int(N), C.byref(g), float(graph["radius"]), float(beta), C.byref(prm), C.byref(h)),
                "md_assemble")
        self._h = h
        info = L.MdOpInfo()
        L.check(lib.md_op_get_info(h, C.byref(info)), "md_op_get_info")
        self.N, self.n3, self.n1, self.nq, self.n_touch = info.N, info.n3, info.n1, info.nq, info.n_touch
        self.n, self.alpha, self.beta = info.n, info.alpha, info.beta

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            L.load().md_op_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def distance(self) -> torch.Tensor:
        d = torch.empty(self.n3, dtype=torch.float32, device="cuda")
        L.check(L.load().md_op_distance(self._h, _ptr(d), _stream()), "md_op_distance")
        return d

    def rhs(self, f: torch.Tensor | None, g: float = 1.0) -> torch.Tensor:
        b = torch.empty(self.n, dtype=torch.float64, device="cuda")
        L.check(L.load().md_rhs(self._h, _ptr(f, torch.float64, self.n3, "f"), float(g), _ptr(b), _stream()), "md_rhs")
        return b

    def apply(self, u: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        if u.dtype not in (torch.float32, torch.float64):
            raise ValueError("u must be float32 or float64")
        y = torch.empty_like(u) if out is None else out
        prec = L.MD_FP32 if u.dtype == torch.float32 else L.MD_FP64
        L.check(L.load().md_apply(self._h, prec, _ptr(u, u.dtype, self.n, "u"), _ptr(y, u.dtype, self.n, "y"),
                                  _stream()), "md_apply")
        return y

    def apply_noalloc(self, u: torch.Tensor, out: torch.Tensor) -> torch.Tensor:
        """y = A u without any device allocation (md_apply_noalloc): the
        scratch is a static array of the library, shared by all calls, so
        overlapping calls must be ordered; `out` must be given."""
        prec = L.MD_FP32 if u.dtype == torch.float32 else L.MD_FP64
        L.check(L.load().md_apply_noalloc(self._h, prec, _ptr(u, u.dtype, self.n, "u"),
                                          _ptr(out, u.dtype, self.n, "out"), _stream()), "md_apply_noalloc")
        return out

    def precondition(self, r: torch.Tensor, net: "Network | None" = None, out=None, order: str = "upper",
                     smooth: tuple[int, float] | None = None, inner: int | None = None) -> torch.Tensor:
        """z = Q r: block upper-triangular order (the paper's), or order='lower'
        (network first, then the 1D solve); net=None gives Jacobi.
        smooth=(nu, omega): nu damped Jacobi sweeps before and after the
        network (md_precondition_smoothed).  inner=m: the 3D solve as m
        inner FGMRES steps preconditioned by the network
        (md_precondition_inner)."""
        z = torch.empty_like(r) if out is None else out
        if order not in ("upper", "lower"):
            raise ValueError("order must be 'upper' or 'lower'")
        if inner is not None:
            if net is None or smooth is not None:
                raise ValueError("inner steps need a network and exclude smoothing")
            L.check(L.load().md_precondition_inner(self._h, net.handle, 1 if order == "lower" else 0, int(inner),
                                                   _ptr(r, torch.float32, self.n, "r"),
                                                   _ptr(z, torch.float32, self.n, "z"), _stream()),
                    "md_precondition_inner")
            return z
        if smooth is not None:
            if net is None:
                raise ValueError("smoothing wraps the network solve: give a network")
            L.check(L.load().md_precondition_smoothed(self._h, net.handle, 1 if order == "lower" else 0,
                                                      int(smooth[0]), float(smooth[1]),
                                                      _ptr(r, torch.float32, self.n, "r"),
                                                      _ptr(z, torch.float32, self.n, "z"), _stream()),
                    "md_precondition_smoothed")
            return z
        if order == "lower":
            if net is None:
                raise ValueError("the lower order needs a network")
            L.check(L.load().md_precondition_lower(self._h, net.handle, _ptr(r, torch.float32, self.n, "r"),
                                                   _ptr(z, torch.float32, self.n, "z"), _stream()),
                    "md_precondition_lower")
            return z
        L.check(L.load().md_precondition(self._h, net.handle if net is not None else None,
                                         _ptr(r, torch.float32, self.n, "r"), _ptr(z, torch.float32, self.n, "z"),
                                         _stream()), "md_precondition")
        return z

    def krylov_basis(self, b: torch.Tensor, m: int) -> torch.Tensor:
        """Orthonormal basis q_0 = b/||b||, ..., q_m of K_{m+1}(C, b), C the 3D
        block (md_krylov_basis); b float32 of length n3; returns (m+1, n3) float32."""
        Q = torch.empty((m + 1, self.n3), dtype=torch.float32, device="cuda")
        L.check(L.load().md_krylov_basis(self._h, _ptr(b, torch.float32, self.n3, "b"), int(m), _ptr(Q), _stream()),
                "md_krylov_basis")
        return Q

    def lift(self, r: torch.Tensor):
        """(l, z1): z1 = B11^{-1} r1 and its 3D forcing l = beta Pi^T W Psi z1
        (float32, n3 and n1) for a float32 vector r of length n."""
        l = torch.empty(self.n3, dtype=torch.float32, device="cuda")
        z1 = torch.empty(self.n1, dtype=torch.float32, device="cuda")
        L.check(L.load().md_lift(self._h, _ptr(r, torch.float32, self.n, "r"), _ptr(z1), _ptr(l), _stream()), "md_lift")
        return l, z1

    def solve(self, b: torch.Tensor, x0: torch.Tensor | None = None, net: "Network | None" = None,
              tol: float = 1e-8, restart: int = 30, maxit: int = 10000):
        """FGMRES with the network preconditioner (net given) or Jacobi-CG.
        Returns (x, iterations, true relative residual, converged)."""
        x = torch.zeros(self.n, dtype=torch.float64, device="cuda") if x0 is None else x0.clone()
        it = C.c_int()
        rr = C.c_double()
        s = L.check(L.load().md_solve(self._h, net.handle if net is not None else None,
                                      _ptr(b, torch.float64, self.n, "b"), _ptr(x), float(tol), int(restart),
                                      int(maxit), C.byref(it), C.byref(rr), _stream()),
                    "md_solve", allow=(L.MD_OK, L.MD_NOT_CONVERGED))
        return x, it.value, rr.value, s == L.MD_OK


def assemble(specs, threads: int | None = None) -> list[Operator]:
    """Operators of several independent instances, assembled on host threads.

    specs: one (N, graph, beta, keyword arguments of Operator) tuple per
    instance; the result is in the order of specs.  Each instance is one
    md_assemble call, whose FP64 geometry runs on the calling host thread (the
    call releases the interpreter lock) and whose uploads and distance-field
    kernel go to the current device of the caller, so instances are built
    side by side on up to `threads` host cores (default: the cores available)."""
    specs = list(specs)
    if not specs:
        return []
    torch.cuda.init()
    dev = torch.cuda.current_device()

    def one(spec):
        torch.cuda.set_device(dev)
        N, graph, beta, kw = spec
        return Operator(N, graph, beta, **kw)

    workers = min(len(specs), threads if threads else (len(os.sched_getaffinity(0)) or 1))
    if workers <= 1:
        return [one(sp) for sp in specs]
    with ThreadPoolExecutor(max_workers=workers) as pool:
        return list(pool.map(one, specs))


class Network:
    """The 6-layer convolutional preconditioner (weights on the device)."""

    def __init__(self, params: np.ndarray | None = None, *, handle=None):
        lib = L.load()
        if handle is not None:
            self._h = handle
            return
        p = np.ascontiguousarray(params, dtype=np.float32).ravel()
        h = C.c_void_p()
        L.check(lib.md_cnn_create(p.ctypes.data_as(C.POINTER(C.c_float)), p.size, C.byref(h)), "md_cnn_create")
        self._h = h

    @classmethod
    def load(cls, path: str) -> "Network":
        h = C.c_void_p()
        L.check(L.load().md_cnn_load(path.encode(), C.byref(h)), "md_cnn_load")
        return cls(handle=h)

    def save(self, path: str):
        L.check(L.load().md_cnn_save(self._h, path.encode()), "md_cnn_save")

    def params(self) -> np.ndarray:
        out = np.zeros(L.MD_CNN_NPARAMS, dtype=np.float32)
        L.check(L.load().md_cnn_get_params(self._h, out.ctypes.data_as(C.POINTER(C.c_float)), out.size),
                "md_cnn_get_params")
        return out

    @property
    def handle(self):
        return self._h

    def set_engine(self, engine: str):
        """'tensor' (tcgen05, default) or 'cuda_cores' (the cross-check path)."""
        code = {"tensor": 0, "cuda_cores": 1}[engine]
        L.check(L.load().md_cnn_set_engine(self._h, code), "md_cnn_set_engine")

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            L.load().md_cnn_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def forward(self, X: torch.Tensor) -> torch.Tensor:
        """X: (batch, 3, n, n, n) float32 CUDA -> (batch, 1, n, n, n)."""
        if X.dim() != 5 or X.shape[1] != 3 or not (X.shape[2] == X.shape[3] == X.shape[4]):
            raise ValueError("X must be (batch, 3, n, n, n)")
        X = X.contiguous()
        Y = torch.empty((X.shape[0], 1) + tuple(X.shape[2:]), dtype=torch.float32, device="cuda")
        L.check(L.load().md_cnn_forward(self._h, X.shape[2], X.shape[0], _ptr(X, torch.float32), _ptr(Y), _stream()),
                "md_cnn_forward")
        return Y


    def backward(self, X: torch.Tensor, dY: torch.Tensor, need_dx: bool = False):
        """Gradients of sum(dY * N(X)): (dparams (MD_CNN_NPARAMS,), dX or None)."""
        X = X.contiguous()
        dY = dY.contiguous()
        n = X.shape[2]
        dp = torch.empty(L.MD_CNN_NPARAMS, dtype=torch.float32, device="cuda")
        dX = torch.empty_like(X) if need_dx else None
        L.check(L.load().md_cnn_backward(self._h, n, X.shape[0], _ptr(X, torch.float32), _ptr(dY, torch.float32),
                                         _ptr(dp), _ptr(dX) if need_dx else None, _stream()), "md_cnn_backward")
        return dp, dX


class UNet:
    """The paper's U-net U3 (md_unet_*): 2 input channels, 1 output."""

    def __init__(self, params: np.ndarray):
        lib = L.load()
        p = np.ascontiguousarray(params, dtype=np.float32)
        h = C.c_void_p()
        L.check(lib.md_unet_create(p.ctypes.data_as(C.POINTER(C.c_float)), p.size, C.byref(h)), "md_unet_create")
        self._h = h

    @staticmethod
    def num_params() -> int:
        return int(L.load().md_unet_num_params())

    def forward(self, X: torch.Tensor) -> torch.Tensor:
        """X: (batch, 2, n, n, n) float32 CUDA -> (batch, 1, n, n, n)."""
        if X.dim() != 5 or X.shape[1] != 2 or not (X.shape[2] == X.shape[3] == X.shape[4]):
            raise ValueError("X must be (batch, 2, n, n, n)")
        X = X.contiguous()
        Y = torch.empty((X.shape[0], 1) + tuple(X.shape[2:]), dtype=torch.float32, device="cuda")
        L.check(L.load().md_unet_forward(self._h, X.shape[2], X.shape[0], _ptr(X, torch.float32), _ptr(Y), _stream()),
                "md_unet_forward")
        return Y

    def backward(self, X: torch.Tensor, dY: torch.Tensor, need_dx: bool = False):
        """Gradients of sum(dY * U(X)): (dparams (num_params,), dX or None)."""
        X = X.contiguous()
        dY = dY.contiguous()
        dp = torch.empty(self.num_params(), dtype=torch.float32, device="cuda")
        dX = torch.empty_like(X) if need_dx else None
        L.check(L.load().md_unet_backward(self._h, X.shape[2], X.shape[0], _ptr(X, torch.float32),
                                          _ptr(dY, torch.float32), _ptr(dp), _ptr(dX) if dX is not None else None,
                                          _stream()), "md_unet_backward")
        return dp, dX

    def train_loss(self, ops: list, residuals: list, with_grad: bool = True):
        """Mean training loss ||C z0 - b0||^2 / ||b0||^2 with the U-net as the
        3D block solve (md_unet_train_loss) and its parameter gradient."""
        loss = C.c_double()
        grad = torch.empty(self.num_params(), dtype=torch.float32, device="cuda") if with_grad else None
        rs = (C.c_void_p * len(residuals))(*[r.data_ptr() for r in residuals])
        L.check(L.load().md_unet_train_loss(self._h, len(ops), _op_array(ops), rs, C.byref(loss),
                                            _ptr(grad) if with_grad else None, _stream()), "md_unet_train_loss")
        return loss.value, grad

    def opt_step(self, grad: torch.Tensor, lr: float, betas=(0.9, 0.999), eps: float = 1e-8,
                 weight_decay: float = 1e-4):
        """One AdamW step on the parameters (md_unet_opt_step)."""
        L.check(L.load().md_unet_opt_step(self._h, _ptr(grad, torch.float32), float(lr), float(betas[0]),
                                          float(betas[1]), float(eps), float(weight_decay), _stream()),
                "md_unet_opt_step")

    def set_params(self, params: torch.Tensor):
        """Parameters from a float32 CUDA tensor (num_params,)."""
        L.check(L.load().md_unet_set_params(self._h, _ptr(params.contiguous(), torch.float32), 1, _stream()),
                "md_unet_set_params")

    def params(self) -> np.ndarray:
        out = np.empty(self.num_params(), dtype=np.float32)
        L.check(L.load().md_unet_get_params(self._h, out.ctypes.data_as(C.POINTER(C.c_float)), out.size),
                "md_unet_get_params")
        return out

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            L.load().md_unet_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class NetworkFunction(torch.autograd.Function):
    """Y = N(X) with the library's forward and backward kernels, for use
    inside torch autograd graphs.  The parameters are those held by `net`;
    their gradient is returned for a `params` tensor the caller passes
    (e.g. a flat FP32 copy of the weights it optimises)."""

    @staticmethod
    def forward(ctx, X, params, net):
        ctx.net = net
        ctx.save_for_backward(X)
        return net.forward(X)

    @staticmethod
    def backward(ctx, dY):
        (X,) = ctx.saved_tensors
        dp, dX = ctx.net.backward(X, dY, need_dx=ctx.needs_input_grad[0])
        return dX, dp, None


def _op_array(ops):
    return (C.c_void_p * len(ops))(*[o.handle.value for o in ops])


def train_loss(net: Network, ops: list, residuals: list, with_grad: bool = True):
    """Mean training loss ||C z0 - b0||^2 / ||b0||^2 over the samples
    (operator ops[i], residual residuals[i] float32 of length ops[i].n), and
    its gradient with respect to the flat parameters."""
    loss = C.c_double()
    grad = torch.empty(L.MD_CNN_NPARAMS, dtype=torch.float32, device="cuda") if with_grad else None
    rs = (C.c_void_p * len(residuals))(*[r.data_ptr() for r in residuals])
    L.check(L.load().md_train_loss(net.handle, len(ops), _op_array(ops), rs, C.byref(loss),
                                   _ptr(grad) if with_grad else None, _stream()), "md_train_loss")
    return loss.value, grad


def train(net: Network, ops: list, sample_op: list, residuals: list, *, epochs: int, batch: int = 32,
          lr: float = 1e-3, lr_min: float = 1e-5, betas=(0.9, 0.999), weight_decay: float = 1e-4,
          eps: float = 1e-8, seed: int = 0):
    """Unsupervised training (md_train) in place; returns the mean loss per epoch."""
    hist = (C.c_double * epochs)()
    so = (C.c_int * len(sample_op))(*sample_op)
    rs = (C.c_void_p * len(residuals))(*[r.data_ptr() for r in residuals])
    cfg = L.MdTrainCfg(len(ops), C.cast(_op_array(ops), C.POINTER(C.c_void_p)), len(sample_op),
                       C.cast(so, C.POINTER(C.c_int)), C.cast(rs, C.POINTER(C.c_void_p)), int(epochs), int(batch),
                       float(lr), float(lr_min), float(betas[0]), float(betas[1]), float(weight_decay), float(eps),
                       int(seed), C.cast(hist, C.POINTER(C.c_double)))
    L.check(L.load().md_train(net.handle, C.byref(cfg)), "md_train")
    return list(hist)


class Optimizer:
    """AdamW state for training loops the caller drives (md_opt_*): one step
    per call with a given gradient (device float32, MD_CNN_NPARAMS)."""

    def __init__(self, net: Network, *, betas=(0.9, 0.999), weight_decay: float = 1e-4, eps: float = 1e-8):
        h = C.c_void_p()
        L.check(L.load().md_opt_create(net.handle, C.byref(h)), "md_opt_create")
        self._h = h
        self.net = net
        self.betas, self.weight_decay, self.eps = betas, weight_decay, eps

    def step(self, grad: torch.Tensor, lr: float):
        L.check(L.load().md_opt_step(self._h, self.net.handle, _ptr(grad, torch.float32, L.MD_CNN_NPARAMS, "grad"),
                                     float(lr), float(self.betas[0]), float(self.betas[1]), float(self.eps),
                                     float(self.weight_decay), _stream()), "md_opt_step")

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            L.load().md_opt_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Many instances solved together (md_batch_*)."""

    SOLVERS = {"fgmres_cnn": L.MD_SOLVER_FGMRES_CNN, "fgmres_jacobi": L.MD_SOLVER_FGMRES_JACOBI,
               "cg_jacobi": L.MD_SOLVER_CG_JACOBI}

    def __init__(self, ops: list[Operator], solver: str = "fgmres_cnn", net: Network | None = None, restart: int = 30):
        lib = L.load()
        # the batch borrows the operators and the network: keep them alive
        self.ops = list(ops)
        self.net = net
        arr = (C.c_void_p * len(ops))(*[o.handle.value for o in ops])
        h = C.c_void_p()
        L.check(lib.md_batch_create(len(ops), arr, net.handle if net is not None else None, self.SOLVERS[solver],
                                    int(restart), C.byref(h)), "md_batch_create")
        self._h = h
        offs = (C.c_longlong * (len(ops) + 1))()
        L.check(lib.md_batch_offsets(h, offs), "md_batch_offsets")
        self.offsets = list(offs)
        self.total = self.offsets[-1]

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            L.load().md_batch_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def solve(self, b_all: torch.Tensor, x_all: torch.Tensor, tol: float = 1e-8, maxit: int = 10000):
        n = len(self.ops)
        it = (C.c_int * n)()
        rr = (C.c_double * n)()
        s = L.check(L.load().md_batch_solve(self._h, _ptr(b_all, torch.float64, self.total, "b"),
                                            _ptr(x_all, torch.float64, self.total, "x"), float(tol), int(maxit),
                                            it, rr, _stream()),
                    "md_batch_solve", allow=(L.MD_OK, L.MD_NOT_CONVERGED))
        return list(it), list(rr), s == L.MD_OK

    def set_prec_order(self, order: str):
        """'upper' (the paper's block order, default) or 'lower'."""
        if order not in ("upper", "lower"):
            raise ValueError("order must be 'upper' or 'lower'")
        L.check(L.load().md_batch_set_prec_order(self._h, 1 if order == "lower" else 0), "md_batch_set_prec_order")

    def set_smoothing(self, nu: int, omega: float | None = None):
        """nu damped Jacobi sweeps before and after the network (0: none);
        omega defaults to SMOOTH_OMEGA."""
        om = SMOOTH_OMEGA if omega is None else float(omega)
        L.check(L.load().md_batch_set_smoothing(self._h, int(nu), om), "md_batch_set_smoothing")

    def set_inner_iters(self, m: int):
        """The 3D block solve as m inner FGMRES steps (0: one network application)."""
        L.check(L.load().md_batch_set_inner_iters(self._h, int(m)), "md_batch_set_inner_iters")

    def set_profiling(self, enable: bool):
        L.check(L.load().md_batch_set_profiling(self._h, 1 if enable else 0), "md_batch_set_profiling")

    def set_unet(self, unet: "UNet | None"):
        """The U-net as the 3D block solve (None: the batch's network)."""
        L.check(L.load().md_batch_set_unet(self._h, unet._h if unet is not None else None), "md_batch_set_unet")
        self.unet = unet  # the batch borrows it

    def set_host_loop(self, enable: bool):
        """Host-driven restart cycles (for kernel profilers); default: one graph launch per solve."""
        L.check(L.load().md_batch_set_host_loop(self._h, int(bool(enable))), "md_batch_set_host_loop")

    def tuning(self) -> dict:
        t = L.MdTuning()
        L.check(L.load().md_batch_tuning(self._h, C.byref(t)), "md_batch_tuning")
        return {"tuned": bool(t.tuned), "vec_chunk": t.vec_chunk,
                "vec_us": {int(t.vec_candidates[i]): float(t.vec_us[i]) for i in range(t.n_vec)},
                "conv_tiles_per_step": t.conv_tps,
                "conv_us": {1: float(t.conv_us[0]), 2: float(t.conv_us[1])} if t.conv_tps else {}}

    def stats(self) -> dict:
        st = L.MdBatchStats()
        L.check(L.load().md_batch_stats(self._h, C.byref(st)), "md_batch_stats")
        return {k: getattr(st, k) for k, _ in L.MdBatchStats._fields_}

    def reset_stats(self):
        L.check(L.load().md_batch_reset_stats(self._h), "md_batch_reset_stats")

    def times(self):
        n = len(self.ops)
        t = (C.c_double * n)()
        L.check(L.load().md_batch_times(self._h, t), "md_batch_times")
        return list(t)
