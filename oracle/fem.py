"""Finite-element assembly of the 3D-1D coupled system, eq. (mainsys), in FP64 CSR.

TEST INFRASTRUCTURE (oracle): see the package docstring.

The discrete problem (Section 2.1): find u = [u0; u1] with
    A u = b,  A = K + beta * M,
    K = [[K00, 0], [0, kappa_L * K1]]           (bilinear forms a_Omega, a_Lambda, eq. aomega/alambda)
    M = [[Pi^T W Pi, -Pi^T W Psi], [-Psi^T W Pi, Psi^T W Psi]]
where u0 are Q1 nodal values on the uniform (N+1)^3 grid of the unit cube
(x fastest), u1 are P1 nodal values on the 1D mesh of the graph, Pi is the
cross-section average T_Lambda (trace on the cylinder surface averaged over
the circle, Section 2) evaluated at the 1D quadrature points, Psi evaluates
the 1D P1 field at the same points and W holds the quadrature weights, so that
(T u0 - u1, T v0 - v1)_Lambda is integrated by 2-point Gauss per 1D element.

Readings of points the paper leaves open:
  * boundary: homogeneous Dirichlet on every cube-boundary node, imposed by
    zeroing the node's row and column and putting 1 on the diagonal;
  * beta stands for the coupling factor 2*pi*eps and M uses unit line weight;
  * kappa_L = k_L * pi * R^2 (the |D| weight of a_Lambda) with k_L = 1;
  * 2 Gauss points per 1D element; 8 circle points theta_k = 2 pi k / 8 whose
    cosines/sines are taken exactly from {0, +-1, +-sqrt(1/2)}; the circle
    frame n1 = unit(t x e_a), e_a the axis of smallest |t . e_a| (lowest index
    on ties), n2 = t x n1;
  * a circle point is located in cell clamp(floor(x*N), 0, N-1) per axis and
    interpolated trilinearly; contributions of boundary nodes are dropped.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp

GAUSS_XI = ((1.0 - 1.0 / math.sqrt(3.0)) / 2.0, (1.0 + 1.0 / math.sqrt(3.0)) / 2.0)
_S = math.sqrt(0.5)
# cos/sin of theta_k = 2 pi k / 8, k = 0..7, written exactly
CIRCLE_COS = (1.0, _S, 0.0, -_S, -1.0, -_S, 0.0, _S)
CIRCLE_SIN = (0.0, _S, 1.0, _S, 0.0, -_S, -1.0, -_S)


def node_index(i, j, k, N):
    """Grid node (i, j, k) -> linear index, x fastest."""
    return i + (N + 1) * (j + (N + 1) * k)


def boundary_mask(N: int) -> np.ndarray:
    """True on the nodes of the cube boundary (the Dirichlet nodes)."""
    idx = np.arange(N + 1)
    b = (idx == 0) | (idx == N)
    m = b[:, None, None] | b[None, :, None] | b[None, None, :]  # [k, j, i]
    return m.ravel()


def grid_coords(N: int) -> np.ndarray:
    """(n3, 3) coordinates of the grid nodes, x fastest."""
    t = np.arange(N + 1) / N
    z, y, x = np.meshgrid(t, t, t, indexing="ij")
    return np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1)


def q1_element_matrices(h: float):
    """Element stiffness (grad phi_a, grad phi_b) and mass (phi_a, phi_b) of the
    trilinear brick [0, h]^3, by 2x2x2 Gauss quadrature (exact for both).
    Local node l = a + 2 b + 4 c for the corner at offset (a, b, c) h."""
    Ke = np.zeros((8, 8))
    Me = np.zeros((8, 8))
    wq = h ** 3 / 8.0
    for gx in GAUSS_XI:
        for gy in GAUSS_XI:
            for gz in GAUSS_XI:
                phi = np.zeros(8)
                grad = np.zeros((8, 3))
                for l in range(8):
                    a, b, c = l & 1, (l >> 1) & 1, (l >> 2) & 1
                    fx, dfx = (gx, 1.0 / h) if a else (1.0 - gx, -1.0 / h)
                    fy, dfy = (gy, 1.0 / h) if b else (1.0 - gy, -1.0 / h)
                    fz, dfz = (gz, 1.0 / h) if c else (1.0 - gz, -1.0 / h)
                    phi[l] = fx * fy * fz
                    grad[l] = (dfx * fy * fz, fx * dfy * fz, fx * fy * dfz)
                Ke += wq * grad @ grad.T
                Me += wq * np.outer(phi, phi)
    return Ke, Me


def assemble_q1(N: int, Ke: np.ndarray) -> sp.csr_matrix:
    """Element loop: scatter the 8x8 element matrix of every brick into the
    global (N+1)^3 matrix (a_Omega of eq. aomega on the uniform mesh)."""
    e = np.arange(N)
    ek, ej, ei = np.meshgrid(e, e, e, indexing="ij")
    base = node_index(ei.ravel(), ej.ravel(), ek.ravel(), N)
    offs = np.array([node_index(l & 1, (l >> 1) & 1, (l >> 2) & 1, N) for l in range(8)])
    nodes = base[:, None] + offs[None, :]
    rows = np.repeat(nodes[:, :, None], 8, axis=2)
    cols = np.repeat(nodes[:, None, :], 8, axis=1)
    vals = np.broadcast_to(Ke, rows.shape)
    n3 = (N + 1) ** 3
    return sp.coo_matrix((vals.ravel(), (rows.ravel(), cols.ravel())), shape=(n3, n3)).tocsr()


def mesh_1d(graph: dict):
    """P1 mesh of the graph: every edge split into `elems` equal elements.
    Node ids: the graph nodes first, then the interior points of edge e at
    V + e*(m-1) + (i-1), i = 1..m-1.  Returns (X1, elements (ne, 2))."""
    xyz = np.asarray(graph["xyz"], dtype=np.float64)
    edges = np.asarray(graph["edges"], dtype=np.int64)
    m = int(graph["elems"])
    V = len(xyz)
    pts = [xyz]
    elements = []
    for e, (p, q) in enumerate(edges):
        pa, pb = xyz[p], xyz[q]
        inner = [pa + (i / m) * (pb - pa) for i in range(1, m)]
        if inner:
            pts.append(np.array(inner))
        chain = [int(p)] + [V + e * (m - 1) + i for i in range(m - 1)] + [int(q)]
        elements += [(chain[i], chain[i + 1]) for i in range(m)]
    return np.concatenate(pts, axis=0), np.array(elements, dtype=np.int64)


def _norm3(v):
    return math.sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2])


def _cross(a, b):
    return np.array([a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]])


def circle_frame(t):
    """Unit normals (n1, n2) of the cross-section circle around tangent t."""
    ax = int(np.argmin(np.abs(t)))  # first index on ties
    ea = np.zeros(3)
    ea[ax] = 1.0
    v = _cross(t, ea)
    n1 = v / _norm3(v)
    n2 = _cross(t, n1)
    return n1, n2


def quadrature_1d(X1, elements, radius):
    """Gauss points of every 1D element with weight, P1 values and the 8
    circle points around each (the averaging of T_Lambda, Section 2).

    Returns dict with
        qa, qb   (nq,) element end nodes;  psa, psb (nq,) P1 values there
        w        (nq,) weights L_e / 2
        pts      (nq, 8, 3) circle points
    Point q = 2 * element + g, g = 0, 1."""
    ne = len(elements)
    qa = np.repeat(elements[:, 0], 2)
    qb = np.repeat(elements[:, 1], 2)
    psa = np.zeros(2 * ne)
    psb = np.zeros(2 * ne)
    w = np.zeros(2 * ne)
    pts = np.zeros((2 * ne, 8, 3))
    for el, (a, b) in enumerate(elements):
        d = X1[b] - X1[a]
        L = _norm3(d)
        t = d / L
        n1, n2 = circle_frame(t)
        for g, xi in enumerate(GAUSS_XI):
            q = 2 * el + g
            c = X1[a] + xi * d
            psa[q] = 1.0 - xi
            psb[q] = xi
            w[q] = L / 2.0
            for k in range(8):
                tmp = CIRCLE_COS[k] * n1 + CIRCLE_SIN[k] * n2
                pts[q, k] = c + radius * tmp
    return dict(qa=qa, qb=qb, psa=psa, psb=psb, w=w, pts=pts)


def averaging_operator(N: int, pts: np.ndarray, drop: np.ndarray | None) -> sp.csr_matrix:
    """Pi: row q = (1/8) sum_k u0^h(x_qk), u0^h the trilinear interpolant,
    i.e. the cross-section average of the trace (T_Lambda, Section 2).
    Columns of nodes flagged in `drop` are removed (Dirichlet nodes)."""
    nq = pts.shape[0]
    xs = pts * float(N)
    cell = np.clip(np.floor(xs), 0, N - 1).astype(np.int64)
    frac = xs - cell
    rows, cols, vals = [], [], []
    for corner in range(8):
        a, b, c = corner & 1, (corner >> 1) & 1, (corner >> 2) & 1
        wx = frac[..., 0] if a else 1.0 - frac[..., 0]
        wy = frac[..., 1] if b else 1.0 - frac[..., 1]
        wz = frac[..., 2] if c else 1.0 - frac[..., 2]
        node = node_index(cell[..., 0] + a, cell[..., 1] + b, cell[..., 2] + c, N)
        rows.append(np.repeat(np.arange(nq)[:, None], 8, axis=1).ravel())
        cols.append(node.ravel())
        vals.append((wx * wy * wz).ravel() / 8.0)
    rows = np.concatenate(rows)
    cols = np.concatenate(cols)
    vals = np.concatenate(vals)
    if drop is not None:
        keep = ~drop[cols]
        rows, cols, vals = rows[keep], cols[keep], vals[keep]
    n3 = (N + 1) ** 3
    P = sp.coo_matrix((vals, (rows, cols)), shape=(nq, n3)).tocsr()
    P.sum_duplicates()
    return P


def point_segment_distance(p: np.ndarray, a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Euclidean distance of the points p (n, 3) to the segment [a, b]."""
    d = b - a
    dd = float(d @ d)
    t = np.clip(((p - a) @ d) / dd, 0.0, 1.0)
    closest = a[None, :] + t[:, None] * d[None, :]
    return np.sqrt(np.sum((p - closest) ** 2, axis=1))


def distance_field(N: int, graph: dict) -> np.ndarray:
    """d_h: the distance d(Lambda) at every grid node (Section 2.1, the shape
    parameter mu), minimum over the graph's straight segments."""
    X = grid_coords(N)
    xyz = np.asarray(graph["xyz"], dtype=np.float64)
    d = np.full(len(X), np.inf)
    for p, q in np.asarray(graph["edges"]):
        d = np.minimum(d, point_segment_distance(X, xyz[p], xyz[q]))
    return d


class Problem:
    """All matrices of one instance (grid N, graph, beta) in FP64 CSR.

    Attributes
        A      full coupled matrix (n3 + n1 square), eq. (mainsys)
        C      3D block K00 + beta Pi^T W Pi (eq. matrixC), Dirichlet-masked
        B11    1D block kappa_L K1 + beta Psi^T W Psi
        M01    -Pi^T W Psi (so the 0-1 block of A is beta * M01)
        M00    Pi^T W Pi (so C = K00 + beta * M00)
        Pi, Psi, w, K1, kappa, Mass (unmasked Q1 mass), bd, dist, alpha
        d1     1D Dirichlet mask (n1), u_D its value

    dirichlet=False gives the natural (Neumann) condition on the cube faces of
    eq. (problem).  dirichlet_1d lists graph nodes carrying u_Lambda = u_D
    (the subset dLambda_D of eq. (problem)); those unknowns are eliminated
    symmetrically: their rows and columns of B11 become the identity, their
    columns of M01 zero, and their known value moves to the right-hand side
    (`rhs`).
    """

    def __init__(self, N: int, graph: dict, beta: float, *, k_omega: float = 1.0,
                 sigma_omega: float = 0.0, k_lambda: float = 1.0, dirichlet: bool = True,
                 dirichlet_1d=None, u_d: float = 1.0):
        self.N = N
        self.h = 1.0 / N
        self.n3 = (N + 1) ** 3
        self.beta = float(beta)
        self.graph = graph
        Ke, Me = q1_element_matrices(self.h)
        K00 = assemble_q1(N, k_omega * Ke + sigma_omega * Me)
        self.Mass = assemble_q1(N, Me)
        self.bd = boundary_mask(N) if dirichlet else np.zeros(self.n3, dtype=bool)
        X1, elements = mesh_1d(graph)
        self.X1, self.elements = X1, elements
        self.n1 = len(X1)
        quad = quadrature_1d(X1, elements, float(graph["radius"]))
        self.quad = quad
        self.nq = len(quad["w"])
        self.Pi = averaging_operator(N, quad["pts"], self.bd if dirichlet else None)
        nq, n1 = self.nq, self.n1
        self.Psi = sp.csr_matrix((np.concatenate([quad["psa"], quad["psb"]]),
                                  (np.concatenate([np.arange(nq), np.arange(nq)]),
                                   np.concatenate([quad["qa"], quad["qb"]]))), shape=(nq, n1))
        self.w = quad["w"]
        W = sp.diags(self.w)
        # 1D stiffness: element (a, b) of length L contributes (1/L)[[1,-1],[-1,1]]
        L = np.sqrt(np.sum((X1[elements[:, 1]] - X1[elements[:, 0]]) ** 2, axis=1))
        ea, eb = elements[:, 0], elements[:, 1]
        self.K1 = sp.coo_matrix((np.concatenate([1 / L, 1 / L, -1 / L, -1 / L]),
                                 (np.concatenate([ea, eb, ea, eb]), np.concatenate([ea, eb, eb, ea]))),
                                shape=(n1, n1)).tocsr()
        self.elem_len = L
        self.kappa = k_lambda * math.pi * float(graph["radius"]) ** 2
        M00 = (self.Pi.T @ W @ self.Pi).tocsr()
        self.M00 = M00
        M01_full = (-(self.Pi.T @ W @ self.Psi)).tocsr()
        M11 = (self.Psi.T @ W @ self.Psi).tocsr()
        # 1D Dirichlet nodes: eliminated (identity rows/columns), their value
        # enters the right-hand side through the columns kept here
        self.d1 = np.zeros(n1, dtype=bool)
        if dirichlet_1d is not None:
            self.d1[np.asarray(dirichlet_1d, dtype=np.int64)] = True
        self.u_d = float(u_d)
        keep1 = sp.diags((~self.d1).astype(np.float64))
        self.M01 = (M01_full @ keep1).tocsr()
        interior = sp.diags((~self.bd).astype(np.float64))
        K00m = (interior @ K00 @ interior + sp.diags(self.bd.astype(np.float64))).tocsr()
        self.K00 = K00m
        self.C = (K00m + self.beta * M00).tocsr()
        B11_full = (self.kappa * self.K1 + self.beta * M11).tocsr()
        self.B11 = (keep1 @ B11_full @ keep1 + sp.diags(self.d1.astype(np.float64))).tocsr()
        # what the fixed values contribute: b0 -= beta M01[:, D] u_D, b1[F] -= B11[F, D] u_D
        uD = self.u_d * self.d1.astype(np.float64)
        self._lift0 = -self.beta * (M01_full @ uD)
        self._lift1 = -(keep1 @ (B11_full @ uD)) + uD
        self.A = sp.bmat([[self.C, self.beta * self.M01],
                          [self.beta * self.M01.T, self.B11]], format="csr")
        self.n = self.n3 + self.n1
        self.diag = self.A.diagonal()
        dC = self.C.diagonal()[~self.bd]
        self.alpha = float(np.sqrt(np.mean(dC ** 2))) if dC.size else 1.0
        self.dist = distance_field(N, graph)
        self.load1 = np.zeros(n1)
        np.add.at(self.load1, ea, L / 2)
        np.add.at(self.load1, eb, L / 2)

    def rhs(self, f: np.ndarray | None, g: float) -> np.ndarray:
        """b = [M_Omega f ; g * int psi_i ds] with b0 = 0 on Dirichlet nodes,
        plus, with 1D Dirichlet nodes, the lifting of their value u_D
        (b1 = u_D on those nodes).  f: nodal source on the grid (None -> 0)."""
        b0 = np.zeros(self.n3) if f is None else self.Mass @ f
        b1 = g * self.load1
        b1[self.d1] = 0.0
        b0 = b0 + self._lift0
        b1 = b1 + self._lift1
        b0[self.bd] = 0.0
        return np.concatenate([b0, b1])

    def source(self, seed: int | None) -> np.ndarray | None:
        """Nodal f ~ N(0,1) on interior nodes, 0 on the boundary."""
        from mdgen import interior_source
        return interior_source(self.N, seed)

    def apply(self, u: np.ndarray) -> np.ndarray:
        return self.A @ u
