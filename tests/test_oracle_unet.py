"""Pins of the oracle's U-net (oracle/unet.py; Section 4.2 and the U3 table of
Section 5.1) against PyTorch's CPU implementations of the same operations
(conv3d, max_pool3d, conv_transpose3d) in FP64: each operation alone, the
whole network forward, and its gradients by autograd; the level sizes of a
21^3 input and the table's parameter counts."""
import numpy as np
import pytest
import torch
import torch.nn.functional as F

from oracle import unet



def t(a):
    return torch.from_numpy(np.ascontiguousarray(a))


def torch_unet(X, theta):
    """The same network composed from PyTorch's operations (batch of one)."""
    L = [(t(W), t(b)) for W, b in unet.unflatten(theta)]
    (W0, b0), (W1, b1), (W2, b2), (Wb, bb), (Wd1, bd1), (Wd0, bd0), (Wo, bo), (U1, c1), (U0, c0) = L
    g = lambda x: 0.5 * x * (1.0 + torch.erf(x / np.sqrt(2.0)))
    conv = lambda x, W, b: F.conv3d(x, W, b, padding=1)

    def up(x, U, c, like):
        y = F.conv_transpose3d(x, U, c, stride=2)
        pad = [0, like.shape[4] - y.shape[4], 0, like.shape[3] - y.shape[3], 0, like.shape[2] - y.shape[2]]
        return F.pad(y, pad)

    e0 = g(conv(X, W0, b0))
    e1 = g(conv(F.max_pool3d(e0, 2), W1, b1))
    e2 = g(conv(F.max_pool3d(e1, 2), W2, b2))
    eb = g(conv(e2, Wb, bb))
    d1 = g(conv(torch.cat([up(eb, U1, c1, e1), e1], 1), Wd1, bd1))
    d0 = g(conv(torch.cat([up(d1, U0, c0, e0), e0], 1), Wd0, bd0))
    return conv(d0, Wo, bo)


@pytest.mark.parametrize("n", [8, 9, 11])
def test_operations_match_torch(n):
    rng = np.random.default_rng(n)
    X = rng.standard_normal((3, n, n + 1, n + 2))
    assert np.allclose(unet.maxpool2(X), F.max_pool3d(t(X)[None], 2)[0].numpy(), rtol=0, atol=0)
    W = rng.standard_normal((3, 5, 2, 2, 2)); b = rng.standard_normal(5)
    size = (2 * (n // 2) + 1, 2 * ((n + 1) // 2), 2 * ((n + 2) // 2) + 1)
    P = unet.maxpool2(X)
    ref = F.conv_transpose3d(t(P)[None], t(W), t(b), stride=2)[0].numpy()
    got = unet.up2(P, W, b, size)
    z, y, x = ref.shape[1:]
    assert np.allclose(got[:, :z, :y, :x], ref, rtol=1e-13, atol=1e-13)
    assert np.all(got[:, z:] == 0) and np.all(got[:, :, y:] == 0) and np.all(got[:, :, :, x:] == 0)


def test_level_sizes_and_parameter_counts():
    """21^3 -> 10^3 -> 5^3 and back (the table's sizes); the middle rows'
    parameter counts of the table (conv weights, and for the first up level
    conv + transposed conv + its bias) are the network's."""
    Y, c = unet.forward(np.zeros((2, 21, 21, 21)), unet.random_params(0), keep=True)
    assert Y.shape == (1, 21, 21, 21)
    assert c["e1"].shape == (64, 10, 10, 10) and c["e2"].shape == (128, 5, 5, 5) and c["s1"].shape == (128, 10, 10, 10)
    shapes = unet.param_shapes()
    w = [int(np.prod(s)) for s, _ in shapes]
    assert w[1] == 55296 and w[2] == 221184 and w[3] == 442368
    assert w[4] + w[7] + shapes[7][1] == 286784
    assert 1.0e6 < unet.num_params() < 1.2e6


@pytest.mark.parametrize("n", [9, 12])
def test_forward_and_gradients_match_torch(n):
    rng = np.random.default_rng(100 + n)
    theta = unet.random_params(n)
    X = rng.standard_normal((2, n, n, n))
    Y, cache = unet.forward(X, theta, keep=True)
    Xt = t(X)[None].requires_grad_(True)
    th = t(theta).requires_grad_(True)
    # the torch composition takes its parameters from the same flat vector
    Yt = torch_unet_flat(Xt, th)
    assert np.max(np.abs(Y - Yt[0].detach().numpy())) <= 1e-12 * np.max(np.abs(Y))
    dY = rng.standard_normal(Y.shape)
    Yt.backward(t(dY)[None])
    dX, dth = unet.backward(dY, cache)
    assert np.linalg.norm(dX - Xt.grad[0].numpy()) <= 1e-11 * np.linalg.norm(dX)
    assert np.linalg.norm(dth - th.grad.numpy()) <= 1e-11 * np.linalg.norm(dth)


def torch_unet_flat(X, theta):
    """torch_unet with its parameters sliced from a flat torch vector (so
    autograd gives the flat gradient)."""
    layers, k = [], 0
    for wshape, nb in unet.param_shapes():
        nw = int(np.prod(wshape))
        layers.append((theta[k:k + nw].reshape(wshape), theta[k + nw:k + nw + nb]))
        k += nw + nb
    (W0, b0), (W1, b1), (W2, b2), (Wb, bb), (Wd1, bd1), (Wd0, bd0), (Wo, bo), (U1, c1), (U0, c0) = layers
    g = lambda x: 0.5 * x * (1.0 + torch.erf(x / np.sqrt(2.0)))
    conv = lambda x, W, b: F.conv3d(x, W, b, padding=1)

    def up(x, U, c, like):
        y = F.conv_transpose3d(x, U, c, stride=2)
        return F.pad(y, [0, like.shape[4] - y.shape[4], 0, like.shape[3] - y.shape[3], 0, like.shape[2] - y.shape[2]])

    e0 = g(conv(X, W0, b0))
    e1 = g(conv(F.max_pool3d(e0, 2), W1, b1))
    e2 = g(conv(F.max_pool3d(e1, 2), W2, b2))
    eb = g(conv(e2, Wb, bb))
    d1 = g(conv(torch.cat([up(eb, U1, c1, e1), e1], 1), Wd1, bd1))
    d0 = g(conv(torch.cat([up(d1, U0, c0, e0), e0], 1), Wd0, bd0))
    return conv(d0, Wo, bo)


def test_forward_matches_torch_composition_at_21():
    theta = unet.random_params(3)
    X = np.random.default_rng(5).standard_normal((2, 21, 21, 21))
    Y = unet.forward(X, theta)
    ref = torch_unet(t(X)[None], theta)[0].numpy()
    assert np.max(np.abs(Y - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_unet_training_loss_is_the_coupled_residual_and_its_gradient_is_consistent():
    """The U-net's training loss (Section 3.2 eq. (risk)) against the coupled
    system itself, as for the CNN: with the block upper-triangular
    preconditioner z = Q(r) whose 3D solve is the U-net, the 3D rows of
    A z - r are C z0 - b0, so the loss is ||(A Q(r) - r)_0||^2 / ||b0||^2 over
    the unknown rows.  Its parameter gradient against central differences
    along a random direction."""
    import mdgen
    from oracle import fem, solvers
    p = fem.Problem(8, mdgen.random_tree(77, 0, depth=3, elems=4), beta=10.0)
    rng = np.random.default_rng(3)
    theta = unet.random_params(11)
    r = rng.standard_normal(p.n)
    r[:p.n3][p.bd] = 0.0
    Q = solvers.BlockPreconditioner(p, mode="unet", params=theta, order="upper")
    z = Q(r)
    e = (p.A @ z - r)[:p.n3][~p.bd]
    z1 = z[p.n3:]
    b0 = r[:p.n3] - p.beta * (p.M01 @ z1)
    want = float(e @ e) / float(b0 @ b0)
    l = Q.lift(z1)
    L, g = solvers.training_loss_unet(p, r[:p.n3], l, theta, grad=True)
    assert L == np.float64(L) and abs(L - want) <= 1e-10 * want
    d = rng.standard_normal(theta.size)
    h = 1e-6
    fd = (solvers.training_loss_unet(p, r[:p.n3], l, theta + h * d) -
          solvers.training_loss_unet(p, r[:p.n3], l, theta - h * d)) / (2 * h)
    assert abs(fd - g @ d) <= 1e-5 * abs(fd)
