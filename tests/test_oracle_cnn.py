"""Pins of the oracle network (oracle/cnn.py)."""
import numpy as np
import pytest
import torch

import mdgen
from oracle import cnn, fem, solvers


def test_single_channel_hand_computation():
    """One 3x3x3 layer on a unit impulse: Y(p) = w(c - p) (cross-correlation),
    plus the bias everywhere."""
    rng = np.random.default_rng(0)
    W = rng.standard_normal((1, 1, 3, 3, 3))
    b = np.array([0.25])
    X = np.zeros((1, 5, 5, 5))
    X[0, 2, 2, 2] = 1.0
    Y = cnn.conv3d_same(X, W, b)
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                assert Y[0, 2 + dz, 2 + dy, 2 + dx] == pytest.approx(W[0, 0, 1 - dz, 1 - dy, 1 - dx] + 0.25, abs=1e-15)
    assert Y[0, 0, 0, 0] == 0.25


def test_centre_tap_is_identity_with_zero_padding():
    X = np.random.default_rng(1).standard_normal((2, 4, 5, 6))
    W = np.zeros((2, 2, 3, 3, 3))
    W[0, 0, 1, 1, 1] = 1.0
    W[1, 1, 1, 1, 1] = 1.0
    assert np.array_equal(cnn.conv3d_same(X, W, np.zeros(2)), X)


def test_shift_tap_reads_zero_padding():
    X = np.random.default_rng(2).standard_normal((1, 3, 3, 3))
    W = np.zeros((1, 1, 3, 3, 3))
    W[0, 0, 1, 1, 2] = 1.0  # reads x + 1
    Y = cnn.conv3d_same(X, W, np.zeros(1))
    assert np.array_equal(Y[0, :, :, :2], X[0, :, :, 1:])
    assert np.all(Y[0, :, :, 2] == 0)


def test_conv_matches_torch_conv3d():
    """Independent library routine: torch.nn.functional.conv3d (same
    cross-correlation orientation, zero padding 1) in float64 on the CPU."""
    rng = np.random.default_rng(3)
    X = rng.standard_normal((3, 6, 7, 5))
    W = rng.standard_normal((4, 3, 3, 3, 3))
    b = rng.standard_normal(4)
    ref = torch.nn.functional.conv3d(torch.from_numpy(X)[None], torch.from_numpy(W),
                                     torch.from_numpy(b), padding=1)[0].numpy()
    assert np.max(np.abs(cnn.conv3d_same(X, W, b) - ref)) < 1e-12


def test_gelu_values_and_derivative():
    x = np.linspace(-6, 6, 241)
    g = cnn.gelu(x)
    assert cnn.gelu(np.array([0.0]))[0] == 0.0
    assert abs(cnn.gelu(np.array([8.0]))[0] - 8.0) < 1e-12
    assert abs(cnn.gelu(np.array([-8.0]))[0]) < 1e-12
    ref = torch.nn.functional.gelu(torch.from_numpy(x), approximate="none").numpy()
    assert np.max(np.abs(g - ref)) < 1e-14
    e = 1e-6
    fd = (cnn.gelu(x + e) - cnn.gelu(x - e)) / (2 * e)
    assert np.max(np.abs(fd - cnn.gelu_grad(x))) < 1e-8


def test_round_bf16_against_torch():
    vals = np.concatenate([np.random.default_rng(4).standard_normal(10000) * 10,
                           [1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, -1.0 - 2 ** -8, 0.0, 1e-30]])
    ref = torch.from_numpy(vals.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(cnn.round_bf16(vals), ref)
    assert cnn.round_bf16(np.array([1.0 + 2 ** -8]))[0] == 1.0  # tie to even


def _toy_params(rng, channels):
    return [(rng.standard_normal((co, ci, 3, 3, 3)) * 0.4, rng.standard_normal(co) * 0.1)
            for ci, co in zip(channels[:-1], channels[1:])]


def test_backward_central_differences_toy():
    """4^3 grid, 4 channels, 6 layers: analytic gradients of <Y, G> equal FP64
    central differences (eps = 1e-6) to 1e-6 relative."""
    rng = np.random.default_rng(5)
    chans = (4, 4, 4, 4, 4, 4, 1)
    params = _toy_params(rng, chans)
    X = rng.standard_normal((4, 4, 4, 4))
    G = rng.standard_normal((1, 4, 4, 4))
    Y, saved = cnn.forward(X, params, keep=True)
    grads, dX = cnn.backward(G, params, saved)

    def f(ps, x=X):
        return float(np.sum(cnn.forward(x, ps) * G))

    eps = 1e-6
    for l in range(6):
        W, b = params[l]
        for idx in [tuple(rng.integers(0, s) for s in W.shape) for _ in range(4)]:
            Wp, Wm = W.copy(), W.copy()
            Wp[idx] += eps
            Wm[idx] -= eps
            pp = list(params); pp[l] = (Wp, b)
            pm = list(params); pm[l] = (Wm, b)
            fd = (f(pp) - f(pm)) / (2 * eps)
            assert abs(fd - grads[l][0][idx]) <= 1e-6 * max(1.0, abs(fd))
        j = int(rng.integers(0, len(b)))
        bp, bm = b.copy(), b.copy()
        bp[j] += eps
        bm[j] -= eps
        pp = list(params); pp[l] = (W, bp)
        pm = list(params); pm[l] = (W, bm)
        fd = (f(pp) - f(pm)) / (2 * eps)
        assert abs(fd - grads[l][1][j]) <= 1e-6 * max(1.0, abs(fd))
    idx = (1, 2, 0, 3)
    Xp, Xm = X.copy(), X.copy()
    Xp[idx] += eps
    Xm[idx] -= eps
    fd = (f(params, Xp) - f(params, Xm)) / (2 * eps)
    assert abs(fd - dX[idx]) <= 1e-6 * max(1.0, abs(fd))


def test_training_loss_gradient_central_differences():
    """The residual loss ||C z0 - b0||^2/||b0||^2 and its gradient (through C
    and the network) against central differences on a 4^3-node problem."""
    g = mdgen.straight_segment((0.3, 0.4, 0.5), (0.7, 0.6, 0.5), 4, 0.05)
    p = fem.Problem(3, g, beta=5.0)
    rng = np.random.default_rng(6)
    params = _toy_params(rng, (3, 4, 4, 4, 4, 4, 1))
    r0 = rng.standard_normal(p.n3)
    r0[p.bd] = 0
    l = solvers.BlockPreconditioner(p, mode="jacobi").lift(rng.standard_normal(p.n1))
    L, grads = solvers.training_loss(p, r0, l, params, grad=True)
    eps = 1e-6
    for lay in (0, 3, 5):
        W, b = params[lay]
        idx = tuple(rng.integers(0, s) for s in W.shape)
        Wp, Wm = W.copy(), W.copy()
        Wp[idx] += eps
        Wm[idx] -= eps
        pp = list(params); pp[lay] = (Wp, b)
        pm = list(params); pm[lay] = (Wm, b)
        fd = (solvers.training_loss(p, r0, l, pp) - solvers.training_loss(p, r0, l, pm)) / (2 * eps)
        assert abs(fd - grads[lay][0][idx]) <= 1e-6 * max(1.0, abs(fd))


def test_bf16_emulation_close_to_fp64():
    """BF16 storage of input and activations perturbs the output by a few BF16
    units (2^-8 relative) only."""
    rng = np.random.default_rng(7)
    params = cnn.init_params(11)
    X = rng.standard_normal((3, 9, 9, 9))
    y64 = cnn.forward(X, params)
    y16 = cnn.forward(X, params, bf16=True)
    rel = np.linalg.norm(y16 - y64) / np.linalg.norm(y64)
    assert rel < 3e-2
    assert rel > 0


def test_output_depends_on_radius_six_box_only():
    """Six 3x3x3 'same' layers: the output at a node is the network applied to
    the grid box of radius 6 around it, clipped at the grid faces (the
    property the full-size GPU parity samples rely on); a radius-5 box is not
    enough."""
    rng = np.random.default_rng(11)
    n = 15
    X = rng.standard_normal((3, n, n, n))
    params = cnn.init_params(5)
    full = cnn.forward(X, params)[0]
    for (z, y, x) in [(0, 0, 0), (7, 7, 7), (14, 3, 9), (2, 12, 6)]:
        for r, exact in ((6, True), (5, False)):
            lo = [max(0, c - r) for c in (z, y, x)]
            hi = [min(n, c + r + 1) for c in (z, y, x)]
            v = cnn.forward(X[:, lo[0]:hi[0], lo[1]:hi[1], lo[2]:hi[2]], params)[0][z - lo[0], y - lo[1], x - lo[2]]
            if exact:
                assert abs(v - full[z, y, x]) <= 1e-12 * (1 + abs(full[z, y, x]))
            elif (z, y, x) == (7, 7, 7):
                assert abs(v - full[z, y, x]) > 1e-9
