"""Pins of the oracle solvers and block preconditioner (oracle/solvers.py)."""
import numpy as np
import pytest
import scipy.sparse as sp

import mdgen
from oracle import cnn, fem, solvers


@pytest.fixture(scope="module")
def seg16():
    w = mdgen.WORKLOADS["single_segment_16"]
    g = mdgen.straight_segment(w["p0"], w["p1"], w["elems"], w["radius"])
    return fem.Problem(16, g, beta=1.0)


@pytest.fixture(scope="module")
def tree8():
    return fem.Problem(8, mdgen.random_tree(77, 0, depth=3, elems=4), beta=10.0)


def test_direct_solve_manufactured(seg16):
    rng = np.random.default_rng(0)
    xm = rng.standard_normal(seg16.n)
    x = solvers.direct_solve(seg16.A, seg16.A @ xm)
    assert np.linalg.norm(x - xm) / np.linalg.norm(xm) < 1e-10


def test_jacobi_cg_single_segment(seg16):
    """Single segment, f = 0, g = 1: Jacobi-CG to 1e-10 agrees with the direct solve."""
    b = seg16.rhs(None, 1.0)
    x, it, rel = solvers.jacobi_cg(seg16.A, b, 1e-10)
    assert rel <= 2e-10
    xd = solvers.direct_solve(seg16.A, b)
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) < 1e-7
    assert 10 < it < 5000


def test_fgmres_exact_preconditioner_one_iteration(tree8):
    b = tree8.rhs(tree8.source(5), 1.0)
    lu = sp.linalg.splu(tree8.A.tocsc())
    x, it, rel = solvers.fgmres(tree8.A, b, lu.solve, 1e-10, restart=10)
    assert it == 1
    assert rel < 1e-12


def test_fgmres_identity_is_minimal_residual():
    """With P = I each iterate minimises ||b - A x|| over the Krylov space
    K_j(A, b): compare with least squares on an explicit orthonormal basis."""
    p = fem.Problem(4, mdgen.straight_segment((0.3, 0.4, 0.5), (0.7, 0.6, 0.5), 3, 0.05), beta=2.0)
    A = p.A.toarray()
    rng = np.random.default_rng(1)
    b = rng.standard_normal(p.n)
    hist = []
    solvers.fgmres(p.A, b, None, 1e-30, restart=12, maxit=12, history=hist)
    nb = np.linalg.norm(b)
    K = [b / nb]
    for j in range(1, 9):
        Q, _ = np.linalg.qr(np.array(K).T)
        y, *_ = np.linalg.lstsq(A @ Q, b, rcond=None)
        best = np.linalg.norm(b - A @ Q @ y) / nb
        # the power basis loses digits as j grows, hence the loose relative bound
        assert hist[j - 1] == pytest.approx(best, rel=1e-6, abs=1e-13)
        K.append(A @ K[-1])
        K[-1] /= np.linalg.norm(K[-1])


def test_fgmres_jacobi_reaches_tolerance(tree8):
    b = tree8.rhs(tree8.source(9), 1.0)
    dinv = 1.0 / tree8.A.diagonal()
    x, it, rel = solvers.fgmres(tree8.A, b, lambda v: dinv * v, 1e-8, restart=30)
    assert rel <= 1e-8
    xd = solvers.direct_solve(tree8.A, b)
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) < 1e-6


def test_block_preconditioner_inverts_upper_triangular_part(tree8):
    """Q~ with the exact 3D solve is the inverse of [[C, beta M01], [0, B11]]."""
    p = tree8
    U = sp.bmat([[p.C, p.beta * p.M01], [None, p.B11]], format="csr")
    Q = solvers.BlockPreconditioner(p, mode="exact")
    x = np.random.default_rng(2).standard_normal(p.n)
    assert np.linalg.norm(Q(U @ x) - x) / np.linalg.norm(x) < 1e-10
    # U differs from A only in the lower-left block
    L = p.A - U
    assert abs(L[:p.n3, :]).max() == 0
    assert abs(L[p.n3:, p.n3:]).max() == 0


def test_block_preconditioner_lower_order_inverts_lower_triangular_part(tree8):
    """order='lower' with the exact 3D solve is the inverse of [[C, 0], [A10, B11]],
    A10 the 1-0 block of A; its off-diagonal block is the one the upper order
    drops, and both orders give the same iterations on this instance (the
    reading that builds only the upper one on the GPU)."""
    p = tree8
    Lw = sp.bmat([[p.C, None], [p.A[p.n3:, :p.n3], p.B11]], format="csr")
    Q = solvers.BlockPreconditioner(p, mode="exact", order="lower")
    x = np.random.default_rng(3).standard_normal(p.n)
    assert np.linalg.norm(Q(Lw @ x) - x) / np.linalg.norm(x) < 1e-10
    assert abs((p.A - Lw)[p.n3:, :]).max() == 0
    b = p.rhs(p.source(7), 1.0)
    _, it_u, rel_u = solvers.fgmres(p.A, b, solvers.BlockPreconditioner(p, mode="exact"), 1e-8)
    _, it_l, rel_l = solvers.fgmres(p.A, b, Q, 1e-8)
    assert rel_u <= 1e-8 and rel_l <= 1e-8
    assert abs(it_u - it_l) <= 2


def test_cnn_preconditioner_homogeneous(tree8):
    """P(c v) = c P(v) for c > 0 (input normalisation by s = ||b0||)."""
    params = cnn.init_params(3)
    Q = solvers.BlockPreconditioner(tree8, mode="cnn", params=params, bf16=False)
    v = np.random.default_rng(3).standard_normal(tree8.n)
    v[:tree8.n3][tree8.bd] = 0
    z = Q(v)
    assert np.allclose(Q(3.5 * v), 3.5 * z, rtol=1e-12, atol=1e-14)
    # identity rows on Dirichlet nodes
    v2 = v.copy()
    v2[:tree8.n3][tree8.bd] = 1.25
    assert np.all(Q(v2)[:tree8.n3][tree8.bd] == 1.25)


def identity_params(offset=10.0):
    """A network whose output is channel 0 + channel 1 of its input: hidden
    channel 0 carries x + offset, where GELU(x + offset) = x + offset to FP64
    rounding for |x| << offset, and the next bias removes the offset."""
    chans = cnn.CHANNELS
    params = []
    for l, (ci, co) in enumerate(zip(chans[:-1], chans[1:])):
        W = np.zeros((co, ci, 3, 3, 3))
        b = np.zeros(co)
        if l == 0:
            W[0, 0, 1, 1, 1] = 1.0
            W[0, 1, 1, 1, 1] = 1.0
        else:
            W[0, 0, 1, 1, 1] = 1.0
            b[0] = -offset
        if l < len(chans) - 2:
            b[0] += offset
        params.append((W, b))
    return params


def test_cnn_preconditioner_with_identity_network(tree8):
    """Plumbing pin: with a network that returns r0/s + l/s, the CNN
    preconditioner equals z0 = b0 / alpha, z1 = B11^{-1} r1."""
    p = tree8
    Q = solvers.BlockPreconditioner(p, mode="cnn", params=identity_params(), bf16=False)
    v = np.random.default_rng(4).standard_normal(p.n)
    v[:p.n3][p.bd] = 0
    z = Q(v)
    z1 = solvers.direct_solve(p.B11, v[p.n3:])
    b0 = v[:p.n3] - p.beta * (p.M01 @ z1)
    assert np.allclose(z[p.n3:], z1, rtol=1e-12, atol=1e-14)
    assert np.max(np.abs(z[:p.n3] - b0 / p.alpha)) <= 1e-12 * np.max(np.abs(b0 / p.alpha))


def test_fgmres_cnn_preconditioner_converges(tree8):
    """FGMRES with the network preconditioner reaches the tolerance and the
    solution matches the direct solve (identity network, FP64)."""
    Q = solvers.BlockPreconditioner(tree8, mode="cnn", params=identity_params(), bf16=False)
    b = tree8.rhs(tree8.source(1), 1.0)
    x, it, rel = solvers.fgmres(tree8.A, b, Q, 1e-8, restart=30, maxit=3000)
    assert rel <= 1e-8
    xd = solvers.direct_solve(tree8.A, b)
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) < 1e-6


def _smoother(p, omega):
    """S = I - omega D_s^{-1} C as a function, D_s^{-1} the smoother's scaling."""
    dinv = solvers.smoothing_dinv(p)
    return lambda v: v - omega * dinv * (p.C @ v)


@pytest.mark.parametrize("beta", [1.0, 10.0, 100.0])
def test_smoothing_scaling_is_jacobi_on_stencil_rows_and_contracts(beta):
    """The smoother's scaling: 1/c_ii (plain Jacobi) on every row the
    coupling does not reach, including rows next to the boundary; at most
    that elsewhere; and with it the spectrum of D_s^{-1} C lies in (0, 2], so
    damped sweeps with omega <= 1 never amplify an error mode (the plain
    diagonal gives eigenvalues near 3 at beta = 100)."""
    p = fem.Problem(8, mdgen.random_tree(77, 0, depth=3, elems=4), beta=beta)
    ds = solvers.smoothing_dinv(p)
    d = p.C.diagonal()
    touched = np.asarray(p.M00.sum(axis=1)).ravel() > 0
    assert np.allclose(ds[~touched], 1.0 / d[~touched], rtol=1e-14, atol=0)
    assert np.all(ds <= 1.0 / d * (1 + 1e-14))
    sq = np.sqrt(ds)
    lam = np.linalg.eigvalsh((sp.diags(sq) @ p.C @ sp.diags(sq)).toarray())
    assert lam.min() > 0 and lam.max() <= 2.0 + 1e-12, (lam.min(), lam.max())
    plain = np.linalg.eigvalsh((sp.diags(1 / np.sqrt(d)) @ p.C @ sp.diags(1 / np.sqrt(d))).toarray())
    if beta == 100.0:
        assert plain.max() > 2.5


def test_jacobi_smooth_error_contracts_by_iteration_matrix(tree8):
    """Damped Jacobi on C x = b: the error after nu sweeps is
    (I - omega D^{-1} C)^nu times the initial error (textbook stationary
    iteration), and from x0 = 0 the first sweep is omega D^{-1} b."""
    p = tree8
    rng = np.random.default_rng(11)
    xs = rng.standard_normal(p.n3)
    b = p.C @ xs
    x0 = rng.standard_normal(p.n3)
    dinv = 1.0 / p.C.diagonal()
    S = lambda v: v - 0.8 * dinv * (p.C @ v)  # noqa: E731
    for nu in (1, 2, 3):
        e = x0 - xs
        for _ in range(nu):
            e = S(e)
        x = solvers.jacobi_smooth(p.C, b, x0, nu, 0.8)
        assert np.linalg.norm(x - xs - e) <= 1e-12 * np.linalg.norm(xs)
    x1 = solvers.jacobi_smooth(p.C, b, np.zeros(p.n3), 1, 0.8)
    assert np.allclose(x1, 0.8 * b / p.C.diagonal(), rtol=1e-14, atol=0)


@pytest.mark.parametrize("order", ["upper", "lower"])
@pytest.mark.parametrize("nu", [1, 2])
def test_smoothed_3d_solve_error_propagation(tree8, order, nu):
    """Pre- and post-smoothing around a linear 3D solve N: the error
    propagation of the smoothed solve is I - Q C = S^nu (I - N C) S^nu
    (symmetric two-level composition, S the Jacobi iteration matrix), with
    the lifted part l in its own channel, which must not change a linear
    solve: N = D^{-1} ('jacobi'), and N = I / alpha on interior rows, I on
    Dirichlet rows (the network returning channel 0 + channel 1)."""
    p = tree8
    omega = 0.7
    S = _smoother(p, omega)
    rng = np.random.default_rng(12 + nu)
    for mode, params, Nd in (("jacobi", None, 1.0 / p.C.diagonal()),
                             ("cnn", identity_params(), np.where(p.bd, 1.0, 1.0 / p.alpha))):
        Q = solvers.BlockPreconditioner(p, mode=mode, params=params, bf16=False, order=order,
                                        smooth=(nu, omega))
        for _ in range(2):
            x = rng.standard_normal(p.n3)
            x[p.bd] = rng.standard_normal(int(p.bd.sum()))
            l = rng.standard_normal(p.n3) if order == "upper" else np.zeros(p.n3)
            l[p.bd] = 0.0
            got = x - Q.solve3(p.C @ x - l, l)
            e = x.copy()
            for _ in range(nu):
                e = S(e)
            e = e - Nd * (p.C @ e)
            for _ in range(nu):
                e = S(e)
            assert np.linalg.norm(got - e) <= 1e-10 * np.linalg.norm(x), (mode, order, nu)


@pytest.mark.parametrize("order", ["upper", "lower"])
def test_smoothing_keeps_exact_block_inverse(tree8, order):
    """With the exact 3D solve the smoothed preconditioner still inverts the
    block triangular part (the correction removes the whole residual and
    post-smoothing leaves an exact solution unchanged)."""
    p = tree8
    if order == "upper":
        T = sp.bmat([[p.C, p.beta * p.M01], [None, p.B11]], format="csr")
    else:
        T = sp.bmat([[p.C, None], [p.A[p.n3:, :p.n3], p.B11]], format="csr")
    Q = solvers.BlockPreconditioner(p, mode="exact", order=order, smooth=(2, 0.8))
    x = np.random.default_rng(13).standard_normal(p.n)
    assert np.linalg.norm(Q(T @ x) - x) / np.linalg.norm(x) < 1e-10


@pytest.mark.parametrize("order", ["upper", "lower"])
def test_smoothed_cnn_preconditioner_homogeneous(tree8, order):
    """The smoothed network preconditioner stays positively homogeneous and
    reproduces r0 on Dirichlet nodes (identity rows of C, unit diagonal)."""
    p = tree8
    Q = solvers.BlockPreconditioner(p, mode="cnn", params=cnn.init_params(5), bf16=False, order=order,
                                    smooth=(1, 0.8))
    v = np.random.default_rng(14).standard_normal(p.n)
    v[:p.n3][p.bd] = 0
    z = Q(v)
    assert np.allclose(Q(2.5 * v), 2.5 * z, rtol=1e-12, atol=1e-14)
    v2 = v.copy()
    v2[:p.n3][p.bd] = 1.25
    assert np.allclose(Q(v2)[:p.n3][p.bd], 1.25, rtol=1e-14, atol=0)


@pytest.mark.parametrize("order", ["upper", "lower"])
def test_inner_fgmres_keeps_exact_block_inverse(tree8, order):
    """Inner FGMRES steps preconditioned by the exact 3D solve reach C^{-1} b0
    in the first step; the block preconditioner stays the inverse of the
    block triangular part."""
    p = tree8
    if order == "upper":
        T = sp.bmat([[p.C, p.beta * p.M01], [None, p.B11]], format="csr")
    else:
        T = sp.bmat([[p.C, None], [p.A[p.n3:, :p.n3], p.B11]], format="csr")
    Q = solvers.BlockPreconditioner(p, mode="exact", order=order, inner=3)
    x = np.random.default_rng(15).standard_normal(p.n)
    assert np.linalg.norm(Q(T @ x) - x) / np.linalg.norm(x) < 1e-9


@pytest.mark.parametrize("m", [1, 2, 3])
def test_inner_fgmres_with_jacobi_is_minimal_residual(tree8, m):
    """With the linear Jacobi 3D solve, m inner steps return the minimiser of
    ||b0 - C x|| over x in D^{-1} K_m(C D^{-1}, b0) (right-preconditioned
    GMRES): least squares on an explicit orthonormal basis of that space."""
    p = tree8
    rng = np.random.default_rng(16)
    r0 = rng.standard_normal(p.n3)
    l = rng.standard_normal(p.n3)
    l[p.bd] = 0.0
    b0 = r0 + l
    Q = solvers.BlockPreconditioner(p, mode="jacobi", inner=m)
    x = Q.solve3(r0, l)
    dinv = 1.0 / p.C.diagonal()
    K = [b0 / np.linalg.norm(b0)]
    for _ in range(m - 1):
        w = p.C @ (dinv * K[-1])
        K.append(w / np.linalg.norm(w))
    Qb, _ = np.linalg.qr(np.array(K).T)
    CB = p.C @ (dinv[:, None] * Qb)
    y, *_ = np.linalg.lstsq(CB, b0, rcond=None)
    ref = dinv * (Qb @ y)
    assert np.linalg.norm(x - ref) <= 1e-9 * np.linalg.norm(ref)


@pytest.mark.parametrize("order", ["upper", "lower"])
def test_one_inner_step_is_network_with_minimal_residual_scale(tree8, order):
    """One inner step with the network: z0 = c N(X) for the block's own
    input X = [r0/s, l/s, d] (the first direction keeps the split of b0),
    c = (C z, b0) / ||C z||^2 minimising ||b0 - c C z||; and the inner
    variant stays positively homogeneous."""
    p = tree8
    params = cnn.init_params(6)
    rng = np.random.default_rng(17)
    r0 = rng.standard_normal(p.n3)
    r0[p.bd] = 0.0
    l = rng.standard_normal(p.n3) if order == "upper" else np.zeros(p.n3)
    l[p.bd] = 0.0
    Q1 = solvers.BlockPreconditioner(p, mode="cnn", params=params, bf16=False, order=order, inner=1)
    Q0 = solvers.BlockPreconditioner(p, mode="cnn", params=params, bf16=False, order=order)
    z = Q0.solve3(r0, l)
    Cz = p.C @ z
    c = float(Cz @ (r0 + l)) / float(Cz @ Cz)
    assert np.allclose(Q1.solve3(r0, l), c * z, rtol=1e-10, atol=1e-12 * np.abs(z).max())
    Q3 = solvers.BlockPreconditioner(p, mode="cnn", params=params, bf16=False, order=order, inner=3)
    v = rng.standard_normal(p.n)
    v[:p.n3][p.bd] = 0.0
    zq = Q3(v)
    assert np.allclose(Q3(2.5 * v), 2.5 * zq, rtol=1e-9, atol=1e-12 * np.abs(zq).max())


def test_training_loss_is_the_coupled_residual_of_the_upper_preconditioner(tree8):
    """The training loss (Section 3.2 eq. (risk), the squared norm of Section
    5.1) against the coupled system itself: for the block upper-triangular
    preconditioner z = Q(r) (z1 = B11^{-1} r1, l = -beta M01 z1, z0 the
    network on b0 = r0 + l), the 3D rows of A z - r are
    C z0 + beta M01 z1 - r0 = C z0 - b0.  So the loss equals
    ||(A Q(r) - r)_0||^2 / ||b0||^2 over the interior grid rows, computed here
    from the full matrix A and the preconditioner, with no reference to the
    loss's own b0, s or alpha handling."""
    p = tree8
    rng = np.random.default_rng(42)
    params = cnn.init_params(5)
    r = rng.standard_normal(p.n)
    r[:p.n3][p.bd] = 0.0
    Q = solvers.BlockPreconditioner(p, mode="cnn", params=params, bf16=False, order="upper")
    z = Q(r)
    e = (p.A @ z - r)[:p.n3][~p.bd]
    z1 = z[p.n3:]
    b0 = r[:p.n3] - p.beta * (p.M01 @ z1)
    want = float(e @ e) / float(b0 @ b0)
    l = Q.lift(z1)
    got = solvers.training_loss(p, r[:p.n3], l, params)
    assert got == pytest.approx(want, rel=1e-10)
    # the lifted part matters at this coupling: the loss of r0 alone differs
    assert abs(solvers.training_loss(p, r[:p.n3], 0.0 * l, params) - want) > 1e-3 * want
