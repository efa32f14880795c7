"""Solvers and the block preconditioner in FP64.

TEST INFRASTRUCTURE (oracle): see the package docstring.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import cnn as _cnn
from . import unet as _unet


def direct_solve(A: sp.spmatrix, b: np.ndarray) -> np.ndarray:
    """x = A^{-1} b by sparse LU (the plain definition of the solve every
    Krylov method of Section 4 converges to)."""
    return spla.spsolve(A.tocsc(), b)


def jacobi_cg(A: sp.spmatrix, b: np.ndarray, tol: float, maxit: int = 100000, x0=None):
    """Conjugate gradients preconditioned by diag(A)^{-1}.  A is SPD (remark
    after eq. setB).  Stops when the recursively updated ||r|| / ||b|| <= tol.
    Returns (x, iterations, true relative residual)."""
    dinv = 1.0 / A.diagonal()
    x = np.zeros_like(b) if x0 is None else x0.copy()
    r = b - A @ x
    nb = np.linalg.norm(b)
    if nb == 0.0:
        return x, 0, 0.0
    z = dinv * r
    p = z.copy()
    rho = r @ z
    it = 0
    while np.linalg.norm(r) / nb > tol and it < maxit:
        q = A @ p
        a = rho / (p @ q)
        x += a * p
        r -= a * q
        z = dinv * r
        rho_new = r @ z
        p = z + (rho_new / rho) * p
        rho = rho_new
        it += 1
    return x, it, float(np.linalg.norm(b - A @ x) / nb)


def fgmres(A, b: np.ndarray, precond, tol: float, restart: int = 30, maxit: int = 10000,
           history: list | None = None):
    """Right-preconditioned flexible GMRES(k) (Saad 1993; the solver of Section 4).

    Each cycle: r = b - A x, v_0 = r / ||r||; for j: z_j = P(v_j), w = A z_j,
    modified Gram-Schmidt against v_0..v_j into column j of the Hessenberg H,
    Givens rotations keep the least-squares residual estimate |g_{j+1}|;
    the cycle ends when the estimate <= tol ||b|| or after k steps, then
    x += Z y with H y = g.  Stops when the true ||b - A x|| / ||b|| <= tol.
    `precond` maps a vector to a vector (may be nonlinear); None is identity.
    Returns (x, iterations, true relative residual)."""
    n = len(b)
    x = np.zeros(n)
    nb = np.linalg.norm(b)
    if nb == 0.0:
        return x, 0, 0.0
    P = precond if precond is not None else (lambda v: v)
    it = 0
    while it < maxit:
        r = b - A @ x
        beta = np.linalg.norm(r)
        if beta / nb <= tol:
            break
        k = restart
        V = np.zeros((k + 1, n))
        Z = np.zeros((k, n))
        H = np.zeros((k + 1, k))
        cs = np.zeros(k)
        sn = np.zeros(k)
        g = np.zeros(k + 1)
        g[0] = beta
        V[0] = r / beta
        m = 0
        for j in range(k):
            Z[j] = P(V[j])
            w = A @ Z[j]
            for i in range(j + 1):
                H[i, j] = w @ V[i]
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] > 0:
                V[j + 1] = w / H[j + 1, j]
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = math.hypot(H[j, j], H[j + 1, j])
            cs[j] = H[j, j] / den
            sn[j] = H[j + 1, j] / den
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            it += 1
            m = j + 1
            if history is not None:
                history.append(abs(g[j + 1]) / nb)
            if abs(g[j + 1]) <= tol * nb or it >= maxit:
                break
        y = np.linalg.solve(np.triu(H[:m, :m]), g[:m])
        x = x + Z[:m].T @ y
    return x, it, float(np.linalg.norm(b - A @ x) / nb)


def smoothing_dinv(prob) -> np.ndarray:
    """The diagonal scaling of the Jacobi smoother of the 3D block C (the
    paper leaves the relaxation's damping open): rho_i / c_ii with
        rho_i = min(1, 2 c_ii / S_i),   S_i = sum_j |K00_ij| + beta sum_j (Pi^T W Pi)_ij,
    S_i bounding the absolute row sum of C (Gershgorin).  On rows of the
    Q1 stencil S_i <= 2 c_ii and rho_i = 1: plain Jacobi.  On rows the coupling
    makes heavy the scaling shrinks so that 2 diag(c_ii / rho_i) - C is
    diagonally dominant, and every sweep with damping omega < 1 contracts
    (without it, beta = 100 puts eigenvalues of D^{-1} C near 3).  Dirichlet
    rows: 1."""
    p = prob
    c = p.C.diagonal()
    S = np.asarray(abs(p.K00).sum(axis=1)).ravel() + p.beta * np.asarray(p.M00.sum(axis=1)).ravel()
    rho = np.minimum(1.0, 2.0 * c / S)
    rho[p.bd] = 1.0
    return rho / c


def jacobi_smooth(C: sp.spmatrix, b: np.ndarray, x0: np.ndarray, sweeps: int, omega: float,
                  dinv: np.ndarray | None = None) -> np.ndarray:
    """S_J(C, b, x0, maxit) of Section 5 ('Effect of pre- and post-smoothing'):
    `sweeps` damped Jacobi relaxations x <- x + omega D^{-1} (b - C x),
    started at x0; D^{-1} = dinv (default 1 / diag(C))."""
    if dinv is None:
        dinv = 1.0 / C.diagonal()
    x = x0.copy()
    for _ in range(sweeps):
        x = x + omega * dinv * (b - C @ x)
    return x


class BlockPreconditioner:
    """Q~: inverse of the block upper-triangular part of A, eq. (right-prec)
    and the two-step back substitution of eq. (twosteps):

        z1 = B11^{-1} r1                       (exact 1D solve)
        b0 = r0 - beta M01 z1 = r0 + l,  l = beta Pi^T W Psi z1   (eq. decoupled_3d_problem)
        z0 ~= C^{-1} b0                        (the 3D solve)

    The 3D solve is `mode`:
        'exact'  -- sparse direct solve with C;
        'cnn'    -- the network: s = ||b0||, X = [r0/s, l/s, d], z0 = (s/alpha) N(X)
                    on interior nodes (alpha as in the training loss of Section 5.1,
                    evaluated for this instance), z0 = r0 on Dirichlet nodes;
        'jacobi' -- z0 = b0 / diag(C);
        'unet'   -- the paper's U-net U3 (oracle/unet.py, FP64) on its two
                    input channels: s = ||b0||, X = [b0/s, d], z0 = (s/alpha) U(X)
                    on unknown nodes, z0 = r0 on Dirichlet nodes (params: its
                    flat parameter vector).

    order='lower' inverts the block lower-triangular part instead (the other
    reading of how the 1D unknowns follow from the network): the 3D block
    first with the 1D part absent from its right-hand side (l = 0, b0 = r0),
    then z1 = B11^{-1} (r1 - beta M10 z0) = B11^{-1} (r1 + beta Psi^T W Pi z0).

    inner=m > 0 replaces the single 3D solve by m steps of flexible GMRES on
    C z0 = b0 from z0 = 0, right-preconditioned by that solve (Section 6: the
    3D block of the coupled preconditioner is '3 steps of P-FGMRES'); in the
    'cnn' mode the first direction is the network on the block's own input
    [r0/s, l/s, d] and the later ones on [v_j, 0, d] (the unit Krylov
    vectors carry no separate lifted part).

    smooth=(nu, omega) wraps the 3D solve in Jacobi pre- and post-smoothing
    (Section 5, 'Effect of pre- and post-smoothing'), with the row scaling of
    smoothing_dinv:
        x = S_J(C, b0, 0, nu);  x += solve(b0 - C x);  z0 = S_J(C, b0, x, nu)
    where the correction solve sees the 3D residual b0 - C x with the lifted
    1D part l kept in its own network channel: [(b0 - C x - l)/s, l/s, d],
    s = ||b0 - C x|| (the split of b0 into r0 and l carried over to the
    residual).  nu = 0 is the plain preconditioner.
    """

    def __init__(self, prob, mode: str = "cnn", params=None, bf16: bool = True, order: str = "upper",
                 smooth: tuple[int, float] = (0, 1.0), inner: int = 0):
        if order not in ("upper", "lower"):
            raise ValueError("order must be 'upper' or 'lower'")
        if smooth[0] < 0:
            raise ValueError("smoothing sweeps must be >= 0")
        if inner < 0 or (inner > 0 and smooth[0] > 0):
            raise ValueError("inner steps must be >= 0 and are not combined with smoothing")
        self.inner = int(inner)
        self.p = prob
        self.mode = mode
        self.params = params
        self.bf16 = bf16
        self.order = order
        self.nu, self.omega = int(smooth[0]), float(smooth[1])
        self.sm_dinv = smoothing_dinv(prob) if self.nu > 0 else None
        self.B11_lu = spla.splu(prob.B11.tocsc())
        self.C_lu = spla.splu(prob.C.tocsc()) if mode == "exact" else None

    def lift(self, z1):
        return -self.p.beta * (self.p.M01 @ z1)

    def solve3(self, r0, l):
        """The 3D block solve for right-hand side r0 + l (l = the lifted 1D
        part), with Jacobi pre- and post-smoothing when nu > 0, or as m inner
        FGMRES steps when inner = m > 0."""
        if self.inner > 0:
            return self.inner_fgmres(r0, l)
        if self.nu == 0:
            return self.inner3(r0, l)
        C = self.p.C
        b0 = r0 + l
        x = jacobi_smooth(C, b0, np.zeros_like(b0), self.nu, self.omega, self.sm_dinv)
        x = x + self.inner3(b0 - C @ x - l, l)
        return jacobi_smooth(C, b0, x, self.nu, self.omega, self.sm_dinv)

    def inner_fgmres(self, r0, l):
        """m steps of right-preconditioned flexible GMRES on C z = r0 + l from
        z = 0 (the `fgmres` of this module, restart m, no early stop): its
        first basis vector is v0 = (r0 + l)/||r0 + l||, preconditioned with
        the split (r0, l) scaled alike; later ones as (v, 0)."""
        b0 = r0 + l
        nb = float(np.linalg.norm(b0))
        if nb == 0.0:
            return self.inner3(r0, l)
        calls = [0]

        def P(v):
            calls[0] += 1
            if calls[0] == 1:
                return self.inner3(r0 / nb, l / nb)
            return self.inner3(v, np.zeros_like(v))
        z, _, _ = fgmres(self.p.C, b0, P, 0.0, restart=self.inner, maxit=self.inner)
        return z

    def inner3(self, r0, l):
        """One application of the 3D solve of `mode` to r0 + l."""
        p = self.p
        b0 = r0 + l
        if self.mode == "exact":
            return self.C_lu.solve(b0)
        if self.mode == "jacobi":
            return b0 / p.C.diagonal()
        if self.mode == "unet":
            return unet_solve(p, r0, l, self.params)
        return network_solve(p, r0, l, self.params, self.bf16)

    def __call__(self, r):
        p = self.p
        r0, r1 = r[:p.n3], r[p.n3:]
        if self.order == "lower":
            z0 = self.solve3(r0, np.zeros_like(r0))
            z1 = self.B11_lu.solve(r1 - p.beta * (p.M01.T @ z0))
            return np.concatenate([z0, z1])
        z1 = self.B11_lu.solve(r1)
        z0 = self.solve3(r0, self.lift(z1))
        return np.concatenate([z0, z1])


def network_input(prob, r0, l):
    """X = [r0/s, l/s, d] on the grid (3, N+1, N+1, N+1), s = ||r0 + l||."""
    n = prob.N + 1
    s = float(np.linalg.norm(r0 + l))
    if s == 0.0:
        return None, 0.0
    X = np.stack([r0 / s, l / s, prob.dist]).reshape(3, n, n, n)
    return X, s


def network_solve(prob, r0, l, params, bf16=True):
    """z0 = (s/alpha) N([r0/s, l/s, d]) on interior nodes, r0 on Dirichlet nodes."""
    X, s = network_input(prob, r0, l)
    if X is None:
        return r0.copy()
    Y = _cnn.forward(X, params, bf16=bf16).reshape(-1)
    z0 = (s / prob.alpha) * Y
    z0[prob.bd] = r0[prob.bd]
    return z0


def unet_input(prob, r0, l):
    """The U-net's input X = [b0/s, d] (2, N+1, N+1, N+1), b0 = r0 + l, s = ||b0||."""
    n = prob.N + 1
    b0 = r0 + l
    s = float(np.linalg.norm(b0))
    if s == 0.0:
        return None, 0.0
    return np.stack([b0 / s, prob.dist]).reshape(2, n, n, n), s


def unet_solve(prob, r0, l, theta):
    """z0 = (s/alpha) U([b0/s, d]) on unknown nodes, r0 on Dirichlet nodes."""
    X, s = unet_input(prob, r0, l)
    if X is None:
        return r0.copy()
    z0 = (s / prob.alpha) * _unet.forward(X, theta).reshape(-1)
    z0[prob.bd] = r0[prob.bd]
    return z0


def training_loss_unet(prob, r0, l, theta, grad=False):
    """training_loss with the U-net as the 3D solve: L = ||C_II Y_I / alpha -
    b0_I / s||^2, Y = U([b0/s, d]); grad=True also returns the flat
    parameter gradient (oracle/unet.py backward)."""
    p = prob
    X, s = unet_input(p, r0, l)
    Y, cache = _unet.forward(X, theta, keep=True)
    y = Y.reshape(-1).copy()
    y[p.bd] = 0.0
    b_hat = (r0 + l) / s
    b_hat[p.bd] = 0.0
    Cy = p.C @ y
    Cy[p.bd] = 0.0
    res = Cy / p.alpha - b_hat
    L = float(res @ res)
    if not grad:
        return L
    dy = (2.0 / p.alpha) * (p.C.T @ res)
    dy[p.bd] = 0.0
    n = p.N + 1
    _, g = _unet.backward(dy.reshape(1, n, n, n), cache)
    return L, g


def training_loss(prob, r0, l, params, bf16=False, grad=False):
    """Unsupervised residual loss of one sample (Section 3.2 eq. risk with the
    squared norm of Section 5.1): with b0 = r0 + l, s = ||b0||,
        L = || C z0 - b0 ||^2 / ||b0||^2 = || C_II Y_I / alpha - b0_I / s ||^2,
    z0 = (s/alpha) Y restricted to interior nodes (Dirichlet rows excluded).
    grad=True also returns the parameter gradients (by hand, eq. of backward)."""
    p = prob
    X, s = network_input(p, r0, l)
    Y, saved = _cnn.forward(X, params, bf16=bf16, keep=True)
    y = Y.reshape(-1).copy()
    y[p.bd] = 0.0
    b_hat = (r0 + l) / s
    b_hat[p.bd] = 0.0
    Cy = p.C @ y
    Cy[p.bd] = 0.0
    res = Cy / p.alpha - b_hat
    L = float(res @ res)
    if not grad:
        return L
    dy = (2.0 / p.alpha) * (p.C.T @ res)
    dy[p.bd] = 0.0
    n = p.N + 1
    grads, _ = _cnn.backward(dy.reshape(1, n, n, n), params, saved)
    return L, grads
