"""Pins of the oracle's assembly (oracle/fem.py) against facts fixed by the
paper and by the mathematics, not by the oracle itself."""
import json
import math
import os

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import mdgen
from oracle import fem

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def seg_graph(p0=(0.2, 0.5, 0.5), p1=(0.8, 0.5, 0.5), elems=32, R=0.02):
    return mdgen.straight_segment(p0, p1, elems, R)


def test_stencil_closed_form():
    """Interior rows of K00 and of the Q1 mass equal the closed-form stencils."""
    gold = json.load(open(os.path.join(GOLD, "q1_stencil.json")))
    N = 6
    h = 1.0 / N
    Ke, Me = fem.q1_element_matrices(h)
    K = fem.assemble_q1(N, Ke)
    M = fem.assemble_q1(N, Me)
    n = fem.node_index(3, 3, 3, N)
    for di in (-1, 0, 1):
        for dj in (-1, 0, 1):
            for dk in (-1, 0, 1):
                m = fem.node_index(3 + di, 3 + dj, 3 + dk, N)
                kind = ["centre", "face", "edge", "corner"][abs(di) + abs(dj) + abs(dk)]
                assert K[n, m] == pytest.approx(h * gold["stiffness_over_h"][kind], abs=1e-15)
                assert M[n, m] == pytest.approx(h ** 3 * gold["mass_over_h3"][kind], abs=1e-17)
    assert abs(K[n].sum()) < 1e-15  # constants are in the kernel of the Laplacian
    assert M[n].sum() == pytest.approx(h ** 3, rel=1e-14)  # int phi_n = h^3


def test_symmetric_positive_definite_dense():
    """A is SPD (remark after eq. setB): dense eigenvalues on a small mesh."""
    g = mdgen.random_tree(5, 0, depth=3, elems=4)
    p = fem.Problem(6, g, beta=3.0)
    A = p.A.toarray()
    assert np.max(np.abs(A - A.T)) <= 1e-14 * np.max(np.abs(A))
    ev = np.linalg.eigvalsh(A)
    assert ev.min() > 0


def test_symmetric_positive_definite_segment16():
    """Single-segment case, N = 16: symmetric, and positive Rayleigh quotients."""
    p = fem.Problem(16, seg_graph(), beta=1.0)
    D = (p.A - p.A.T)
    assert abs(D).max() <= 1e-14 * abs(p.A).max()
    rng = np.random.default_rng(0)
    for _ in range(20):
        v = rng.standard_normal(p.n)
        assert v @ (p.A @ v) > 0
    lam = spla.eigsh(p.A.tocsc(), k=1, sigma=0.0, which="LM", return_eigenvectors=False)
    assert lam[0] > 0


def test_coupling_vanishes_for_equal_constants():
    """T u0 - u1 = 0 when u0 = u1 = c (u-hat = u-bar): M u = 0 exactly."""
    g = mdgen.random_tree(11, 0, depth=3, elems=5)
    p = fem.Problem(16, g, beta=7.0)
    c = 2.5
    u = np.full(p.n, c)
    u[:p.n3][p.bd] = 0.0  # Dirichlet nodes carry no value; Pi never reads them
    t = p.Pi @ u[:p.n3] - p.Psi @ u[p.n3:]
    assert np.max(np.abs(t)) < 1e-13
    Mu = np.concatenate([p.Pi.T @ (p.w * t), -(p.Psi.T @ (p.w * t))])
    full = p.A @ u - np.concatenate([p.K00 @ u[:p.n3], p.kappa * (p.K1 @ u[p.n3:])])
    assert np.max(np.abs(full)) < 1e-12
    assert np.max(np.abs(Mu)) < 1e-13


def test_averaging_of_linear_field_is_centre_value():
    """The circle average of a linear field is its value on the centreline."""
    g = mdgen.random_tree(3, 0, depth=3, elems=4, radius_range=(0.03, 0.03))
    N = 12
    p = fem.Problem(N, g, beta=1.0, dirichlet=False)
    X = fem.grid_coords(N)
    coef = np.array([0.3, -1.1, 2.0])
    u0 = 0.7 + X @ coef
    centres = p.X1[p.quad["qa"]] * p.quad["psa"][:, None] + p.X1[p.quad["qb"]] * p.quad["psb"][:, None]
    exact = 0.7 + centres @ coef
    assert np.max(np.abs(p.Pi @ u0 - exact)) < 1e-13


def _hat(x, xn, h):
    return np.maximum(0.0, 1.0 - np.abs(x - xn) / h)


def test_averaging_matches_brute_force_basis_evaluation():
    """Pi u0 equals sum_n u_n phi_n(x) evaluated with every global basis
    function (no cell lookup), averaged over the 8 circle points."""
    g = mdgen.random_tree(4, 0, depth=2, elems=3)
    N = 5
    h = 1.0 / N
    p = fem.Problem(N, g, beta=1.0, dirichlet=False)
    X = fem.grid_coords(N)
    rng = np.random.default_rng(1)
    u0 = rng.standard_normal(p.n3)
    pts = p.quad["pts"].reshape(-1, 3)
    phi = (_hat(pts[:, None, 0], X[None, :, 0], h) * _hat(pts[:, None, 1], X[None, :, 1], h)
           * _hat(pts[:, None, 2], X[None, :, 2], h))
    brute = (phi @ u0).reshape(-1, 8).mean(axis=1)
    assert np.max(np.abs(p.Pi @ u0 - brute)) < 1e-13


def _dense_bruteforce_A(N, graph, beta, dirichlet):
    """Dense A by explicit integration with global basis functions:
    stiffness with a 4x4x4 Gauss rule per brick, coupling by evaluating every
    basis function at the circle points and every 1D hat at the Gauss points."""
    h = 1.0 / N
    X = fem.grid_coords(N)
    n3 = len(X)
    gx4, gw4 = np.polynomial.legendre.leggauss(4)
    gx4 = (gx4 + 1) / 2
    gw4 = gw4 / 2
    K = np.zeros((n3, n3))
    for k in range(N):
        for j in range(N):
            for i in range(N):
                corners = [fem.node_index(i + a, j + b, k + c, N)
                           for c in (0, 1) for b in (0, 1) for a in (0, 1)]
                for qx, wx in zip(gx4, gw4):
                    for qy, wy in zip(gx4, gw4):
                        for qz, wz in zip(gx4, gw4):
                            x = np.array([(i + qx) * h, (j + qy) * h, (k + qz) * h])
                            grads = []
                            for n in corners:
                                hx = _hat(x[0], X[n, 0], h)
                                hy = _hat(x[1], X[n, 1], h)
                                hz = _hat(x[2], X[n, 2], h)
                                d = [-np.sign(x[a] - X[n, a]) / h for a in range(3)]
                                grads.append([d[0] * hy * hz, hx * d[1] * hz, hx * hy * d[2]])
                            grads = np.array(grads)
                            K[np.ix_(corners, corners)] += wx * wy * wz * h ** 3 * grads @ grads.T
    X1, elements = fem.mesh_1d(graph)
    n1 = len(X1)
    R = graph["radius"]
    kappa = math.pi * R ** 2
    K1 = np.zeros((n1, n1))
    rows_T, rows_P, ws = [], [], []
    for a, b in elements:
        d = X1[b] - X1[a]
        L = np.linalg.norm(d)
        K1[np.ix_([a, b], [a, b])] += np.array([[1, -1], [-1, 1]]) / L
        t = d / L
        ax = int(np.argmin(np.abs(t)))
        e = np.zeros(3)
        e[ax] = 1
        n_1 = np.cross(t, e)
        n_1 /= np.linalg.norm(n_1)
        n_2 = np.cross(t, n_1)
        for xi in ((1 - 1 / np.sqrt(3)) / 2, (1 + 1 / np.sqrt(3)) / 2):
            c = X1[a] + xi * d
            th = 2 * np.pi * np.arange(8) / 8
            pts = c[None, :] + R * (np.cos(th)[:, None] * n_1 + np.sin(th)[:, None] * n_2)
            phi = (_hat(pts[:, None, 0], X[None, :, 0], h) * _hat(pts[:, None, 1], X[None, :, 1], h)
                   * _hat(pts[:, None, 2], X[None, :, 2], h))
            Trow = phi.mean(axis=0)
            Prow = np.zeros(n1)
            Prow[a] += 1 - xi
            Prow[b] += xi
            rows_T.append(Trow)
            rows_P.append(Prow)
            ws.append(L / 2)
    T = np.array(rows_T)
    P = np.array(rows_P)
    Wd = np.diag(ws)
    bd = fem.boundary_mask(N)
    if dirichlet:
        T[:, bd] = 0.0
        K[bd, :] = 0
        K[:, bd] = 0
        K[bd, bd] = 1.0
    A = np.block([[K + beta * T.T @ Wd @ T, -beta * T.T @ Wd @ P],
                  [-beta * P.T @ Wd @ T, kappa * K1 + beta * P.T @ Wd @ P]])
    return A


@pytest.mark.parametrize("dirichlet", [False, True])
def test_dense_bruteforce_equals_csr(dirichlet):
    """Tiny mesh (4^3 bricks, one segment of 2 elements): the CSR A equals a
    dense A built from the basis functions directly."""
    g = seg_graph(p0=(0.3, 0.45, 0.55), p1=(0.7, 0.6, 0.4), elems=2, R=0.05)
    N = 4
    p = fem.Problem(N, g, beta=2.0, dirichlet=dirichlet)
    Ad = _dense_bruteforce_A(N, g, 2.0, dirichlet)
    assert np.max(np.abs(p.A.toarray() - Ad)) <= 1e-13 * np.max(np.abs(Ad))


def test_manufactured_3d_second_order():
    """beta = 0, u = sin(pi x) sin(pi y) sin(pi z): the discrete L2 nodal error
    of the Q1 solution decays at rate 2 under refinement N = 8, 16, 32."""
    errs = []
    Ns = (8, 16, 32)
    for N in Ns:
        g = seg_graph()
        p = fem.Problem(N, g, beta=0.0)
        X = fem.grid_coords(N)
        u = np.sin(np.pi * X[:, 0]) * np.sin(np.pi * X[:, 1]) * np.sin(np.pi * X[:, 2])
        f = 3 * np.pi ** 2 * u
        b0 = p.Mass @ f
        b0[p.bd] = 0.0
        uh = spla.spsolve(p.C.tocsc(), b0)
        errs.append(math.sqrt(p.h ** 3 * np.sum((uh - u) ** 2)))
    rates = [math.log(errs[i] / errs[i + 1], 2) for i in range(len(Ns) - 1)]
    for r in rates:
        assert abs(r - 2.0) < 0.1, rates


def test_1d_p1_nodally_exact():
    """-kappa u'' = g on one segment with u = 0 at both ends: P1 nodal values
    equal the exact parabola g s (L - s) / (2 kappa)."""
    g = seg_graph(p0=(0.2, 0.3, 0.4), p1=(0.7, 0.6, 0.5), elems=9, R=0.02)
    p = fem.Problem(8, g, beta=0.0)
    s_nodes = np.linalg.norm(p.X1 - p.X1[0], axis=1)
    L = s_nodes[1]
    inner = np.arange(p.n1) > 1  # nodes 0 and 1 are the segment ends
    K = (p.kappa * p.K1).toarray()[np.ix_(inner, inner)]
    u = np.linalg.solve(K, 1.0 * p.load1[inner])
    exact = s_nodes[inner] * (L - s_nodes[inner]) / (2 * p.kappa)
    assert np.max(np.abs(u - exact)) <= 1e-11 * np.max(np.abs(exact))


def test_rhs_mass_source_constant():
    """b0 = M f: for f = 1 on all nodes an interior entry equals h^3."""
    p = fem.Problem(8, seg_graph(), beta=1.0)
    b = p.rhs(np.ones(p.n3), 1.0)
    n = fem.node_index(4, 4, 4, 8)
    assert b[n] == pytest.approx(p.h ** 3, rel=1e-14)
    assert np.all(b[:p.n3][p.bd] == 0)
    # int_Lambda psi_i ds sums to the graph length
    assert b[p.n3:].sum() == pytest.approx(0.6, rel=1e-14)


def test_distance_field_against_sampling():
    g = mdgen.random_tree(21, 0, depth=3)
    N = 8
    d = fem.distance_field(N, g)
    X = fem.grid_coords(N)
    xyz = g["xyz"]
    s = np.linspace(0, 1, 4001)
    pts = np.concatenate([xyz[a][None] + s[:, None] * (xyz[b] - xyz[a])[None] for a, b in g["edges"]])
    brute = np.min(np.linalg.norm(X[:, None, :] - pts[None, :, :], axis=2), axis=1)
    assert np.max(np.abs(d - brute)) < 2e-4
    assert np.all(d <= brute + 1e-15)
    # a grid node on the segment has distance 0
    p = fem.distance_field(16, seg_graph())
    assert p[fem.node_index(8, 8, 8, 16)] == 0.0
    assert p[fem.node_index(8, 10, 8, 16)] == pytest.approx(2 / 16, abs=1e-15)


def _tree_problem(**kw):
    g = mdgen.random_tree(303, 0, depth=3, elems=3)
    return fem.Problem(6, g, kw.pop("beta", 1.0), **kw)


def test_neumann_cube_with_1d_dirichlet_reproduces_constants():
    """Natural conditions on the cube faces, sigma = 0, no source, u_Lambda = 1
    on one graph end (eq. (problem)): the stiffness, the 1D stiffness and the
    coupling all annihilate constants (Pi and Psi are partitions of unity when
    no boundary weight is dropped), so the discrete solution is exactly 1 on
    every grid and graph node."""
    p = _tree_problem(beta=3.0, dirichlet=False, dirichlet_1d=[0], u_d=1.0)
    assert not p.bd.any() and p.d1.sum() == 1
    assert np.allclose(np.asarray(p.Pi.sum(axis=1)).ravel(), 1.0, atol=1e-14)
    b = p.rhs(None, 0.0)
    x = sp.linalg.spsolve(p.A.tocsc(), b)
    assert np.abs(x - 1.0).max() < 1e-10
    assert np.abs(p.A @ np.ones(p.n) - b).max() < 1e-12


def test_1d_dirichlet_without_coupling():
    """beta = 0: the graph problem alone with u = u_D on one end, natural
    conditions elsewhere and no load is u = u_D; the cube problem (sigma > 0,
    no source) is u = 0."""
    p = _tree_problem(beta=0.0, sigma_omega=0.5, dirichlet=False, dirichlet_1d=[0], u_d=2.5)
    x = sp.linalg.spsolve(p.A.tocsc(), p.rhs(None, 0.0))
    assert np.abs(x[p.n3:] - 2.5).max() < 1e-10
    assert np.abs(x[:p.n3]).max() < 1e-12


def test_neumann_1d_dirichlet_system_is_spd_and_matches_elimination():
    """The eliminated system is symmetric positive definite, and its solution
    restricted to the free unknowns equals the solution of the full system
    with the Dirichlet rows replaced by u = u_D (unsymmetric elimination)."""
    p = _tree_problem(beta=2.0, k_omega=1e-3, sigma_omega=1e-3, dirichlet=False, dirichlet_1d=[0, 2], u_d=1.0)
    A = p.A.toarray()
    assert np.abs(A - A.T).max() < 1e-14
    assert np.linalg.eigvalsh(A).min() > 0
    q = _tree_problem(beta=2.0, k_omega=1e-3, sigma_omega=1e-3, dirichlet=False)
    Af = q.A.toarray()
    rows = q.n3 + np.flatnonzero(p.d1)
    bf = q.rhs(None, 0.0)
    Af[rows, :] = 0.0
    Af[rows, rows] = 1.0
    bf[rows] = 1.0
    bf[q.n3:][~p.d1] = 0.0
    xf = np.linalg.solve(Af, bf)
    x = np.linalg.solve(A, p.rhs(None, 0.0))
    assert np.abs(x - xf).max() < 1e-10 * np.abs(xf).max()


@pytest.mark.parametrize("N,k_omega,sigma", [(4, 1.0, 0.0), (7, 2.5, 0.0), (10, 1.0, 3.0)])
def test_alpha_without_coupling_is_the_stencil_centre(N, k_omega, sigma):
    """alpha (Section 5.1: ||diag C|| / sqrt(N_h) over the unknown grid nodes)
    at beta = 0: every interior diagonal of C is the closed-form stencil centre
    k h 8/3 + sigma h^3 8/27, so alpha equals it whatever the graph."""
    gold = json.load(open(os.path.join(GOLD, "q1_stencil.json")))
    g = mdgen.random_tree(31, 0, depth=2, elems=3)
    p = fem.Problem(N, g, beta=0.0, k_omega=k_omega, sigma_omega=sigma)
    h = 1.0 / N
    centre = k_omega * h * gold["stiffness_over_h"]["centre"] + sigma * h ** 3 * gold["mass_over_h3"]["centre"]
    assert p.alpha == pytest.approx(centre, rel=1e-13)


def test_alpha_counts_interior_nodes_only():
    """With coupling, alpha^2 is the mean of c_ii^2 over the (N-1)^3 interior
    nodes: the Dirichlet rows (identity) do not enter.  Checked on N = 2,
    whose single interior node makes alpha its own diagonal, read off the
    operator by probing with the unit vector."""
    g = mdgen.straight_segment((0.3, 0.5, 0.5), (0.7, 0.5, 0.5), 4, 0.1)
    p = fem.Problem(2, g, beta=7.0)
    e = np.zeros(p.n)
    e[fem.node_index(1, 1, 1, 2)] = 1.0
    c = float(e @ (p.A @ e))
    assert c > 8.0 / 3.0 * 0.5  # the coupling adds to the stencil centre
    assert p.alpha == pytest.approx(c, rel=1e-14)
