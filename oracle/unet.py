"""The paper's three-level U-net U3 in FP64, forward and backward.

TEST INFRASTRUCTURE (oracle): see the package docstring.

Section 4.2 defines the U-net recursively, U_j(X) = Psi_j([U_{j-1}(Phi_j(X)) | Phi_j(X)]),
with encoder layers Phi_j, decoder layers Psi_j and a channel-stacking skip
connection [a | b] at every level; the U3 table of Section 5.1 lists its layers
(input 2 channels at 21^3, 32 / 64 / 128 channels at 21^3 / 10^3 / 5^3, max
pooling on the way down, transposed convolutions and skips on the way up, one
output channel).  Reading of that table (its parameter counts reconcile for the
middle rows only: 55,296 = 32 x 64 x 27, 221,184 = 64 x 128 x 27, 442,368 =
128 x 128 x 27, 286,784 = 128 x 64 x 27 + 128 x 64 x 8 + 64):

  e0 = GELU(conv3(X; 2 -> 32))                         at n        (skip 0)
  e1 = GELU(conv3(maxpool2(e0); 32 -> 64))             at m1 = floor(n / 2)   (skip 1)
  e2 = GELU(conv3(maxpool2(e1); 64 -> 128))            at m2 = floor(m1 / 2)
  b  = GELU(conv3(e2; 128 -> 128))                     at m2
  d1 = GELU(conv3([up2(b; 128 -> 64) | e1]; 128 -> 64))  at m1
  d0 = GELU(conv3([up2(d1; 64 -> 32) | e0]; 64 -> 32))   at n
  Y  = conv3(d0; 32 -> 1)                              at n

conv3: 3x3x3, zero 'same' padding, bias (oracle/cnn.py conv3d_same);
maxpool2: 2x2x2 windows with stride 2, the last plane of an odd size dropped;
up2: transposed convolution with 2x2x2 kernels and stride 2, out[o, 2p + t] =
bias[o] + sum_c W[c, o, t] X[c, p] (t in {0, 1}^3), then zero planes appended
up to the skip's size (2 m <= size <= 2 m + 1); GELU(x) = x Phi(x).

Parameters, flat (the library's layout): for each of the seven conv3 layers in
the order above, then the two up2 layers (up2 of b, then of d1), the weights
then the biases; conv3 weights (c_out, c_in, 3, 3, 3) with kernel index =
offset + 1 in (z, y, x), up2 weights (c_in, c_out, 2, 2, 2) with index t.
"""
from __future__ import annotations

import numpy as np

from .cnn import conv3d_same, conv3d_same_input_grad, conv3d_same_weight_grad, gelu, gelu_grad

# (c_in, c_out) of the conv3 layers in order: e0, e1, e2, b, d1, d0, out
CONVS = ((2, 32), (32, 64), (64, 128), (128, 128), (128, 64), (64, 32), (32, 1))
# (c_in, c_out) of the up2 layers: after b, after d1
UPS = ((128, 64), (64, 32))


def param_shapes():
    """[(weight shape, bias length)] in the flat order."""
    out = [((co, ci, 3, 3, 3), co) for ci, co in CONVS]
    out += [((ci, co, 2, 2, 2), co) for ci, co in UPS]
    return out


def num_params() -> int:
    return sum(int(np.prod(w)) + b for w, b in param_shapes())


def unflatten(theta: np.ndarray):
    """Flat vector -> [(W, b)] for the conv3 layers then the up2 layers."""
    theta = np.asarray(theta, dtype=np.float64)
    if theta.size != num_params():
        raise ValueError(f"{theta.size} parameters, expected {num_params()}")
    layers, k = [], 0
    for wshape, nb in param_shapes():
        nw = int(np.prod(wshape))
        layers.append((theta[k:k + nw].reshape(wshape), theta[k + nw:k + nw + nb]))
        k += nw + nb
    return layers


def flatten(layers) -> np.ndarray:
    return np.concatenate([np.concatenate([np.ravel(W), np.ravel(b)]) for W, b in layers])


def random_params(seed: int = 0) -> np.ndarray:
    """He-normal weights (std sqrt(2 / fan_in); fan_in = 27 c_in for conv3,
    c_in for up2, whose outputs each see one input position), small biases."""
    rng = np.random.default_rng(seed)
    layers = []
    for wshape, nb in param_shapes():
        fan_in = wshape[1] * 27 if wshape[2] == 3 else wshape[0]
        layers.append((rng.normal(0.0, np.sqrt(2.0 / fan_in), wshape), rng.normal(0.0, 0.01, nb)))
    return flatten(layers)


def maxpool2(X: np.ndarray) -> np.ndarray:
    """Max over the 2x2x2 windows at even offsets; an odd size's last plane is dropped."""
    c, Z, Y, Xn = X.shape
    z, y, x = Z // 2, Y // 2, Xn // 2
    V = X[:, :2 * z, :2 * y, :2 * x].reshape(c, z, 2, y, 2, x, 2)
    return V.max(axis=(2, 4, 6))


def maxpool2_grad(dO: np.ndarray, X: np.ndarray) -> np.ndarray:
    """Adjoint: each output's gradient goes to its window's maximum (the first
    in (z, y, x) order among equal maxima)."""
    c, Z, Y, Xn = X.shape
    z, y, x = dO.shape[1:]
    dX = np.zeros_like(X)
    V = X[:, :2 * z, :2 * y, :2 * x].reshape(c, z, 2, y, 2, x, 2).transpose(0, 1, 3, 5, 2, 4, 6).reshape(c, z, y, x, 8)
    arg = V.argmax(axis=-1)
    for t in range(8):
        a, b2, d = t >> 2, (t >> 1) & 1, t & 1
        dX[:, a:2 * z:2, b2:2 * y:2, d:2 * x:2] += np.where(arg == t, dO, 0.0)
    return dX


def up2(X: np.ndarray, W: np.ndarray, b: np.ndarray, size) -> np.ndarray:
    """Transposed 2x2x2 convolution with stride 2, then zero planes up to size."""
    ci, z, y, x = X.shape
    co = W.shape[1]
    out = np.zeros((co,) + tuple(size))
    flat = X.reshape(ci, -1)
    for t in range(8):
        a, b2, d = t >> 2, (t >> 1) & 1, t & 1
        out[:, a:2 * z:2, b2:2 * y:2, d:2 * x:2] = (W[:, :, a, b2, d].T @ flat).reshape(co, z, y, x) + b[:, None, None, None]
    return out


def up2_grads(dO: np.ndarray, X: np.ndarray, W: np.ndarray):
    """(dX, dW, db) of up2 given the output gradient dO (the padding planes carry none)."""
    ci, z, y, x = X.shape
    dX = np.zeros_like(X)
    dW = np.zeros_like(W)
    db = np.zeros(W.shape[1])
    flat = X.reshape(ci, -1)
    for t in range(8):
        a, b2, d = t >> 2, (t >> 1) & 1, t & 1
        g = dO[:, a:2 * z:2, b2:2 * y:2, d:2 * x:2].reshape(W.shape[1], -1)
        dX += (W[:, :, a, b2, d] @ g).reshape(ci, z, y, x)
        dW[:, :, a, b2, d] = flat @ g.T
        db += g.sum(axis=1)
    return dX, dW, db


def forward(X: np.ndarray, theta: np.ndarray, keep: bool = False):
    """U3(X) for X of shape (2, n, n, n) (any spatial sizes >= 4); returns
    Y (1, ...) and, with keep, the intermediate tensors for backward."""
    L = unflatten(theta)
    (W0, b0), (W1, b1), (W2, b2), (Wb, bb), (Wd1, bd1), (Wd0, bd0), (Wo, bo), (U1, c1), (U0, c0) = L
    z0 = conv3d_same(X, W0, b0); e0 = gelu(z0)
    p0 = maxpool2(e0)
    z1 = conv3d_same(p0, W1, b1); e1 = gelu(z1)
    p1 = maxpool2(e1)
    z2 = conv3d_same(p1, W2, b2); e2 = gelu(z2)
    zb = conv3d_same(e2, Wb, bb); eb = gelu(zb)
    u1 = up2(eb, U1, c1, e1.shape[1:])
    s1 = np.concatenate([u1, e1])
    zd1 = conv3d_same(s1, Wd1, bd1); d1 = gelu(zd1)
    u0 = up2(d1, U0, c0, e0.shape[1:])
    s0 = np.concatenate([u0, e0])
    zd0 = conv3d_same(s0, Wd0, bd0); d0 = gelu(zd0)
    Y = conv3d_same(d0, Wo, bo)
    if not keep:
        return Y
    return Y, dict(X=X, z0=z0, e0=e0, p0=p0, z1=z1, e1=e1, p1=p1, z2=z2, e2=e2, zb=zb, eb=eb, s1=s1, zd1=zd1,
                   d1=d1, s0=s0, zd0=zd0, d0=d0, layers=L)


def backward(dY: np.ndarray, cache: dict):
    """(dX, dtheta) for the output gradient dY (1, ...)."""
    L = cache["layers"]
    (W0, _), (W1, _), (W2, _), (Wb, _), (Wd1, _), (Wd0, _), (Wo, _), (U1, _), (U0, _) = L
    g = [None] * len(L)
    g[6] = conv3d_same_weight_grad(dY, cache["d0"])
    dd0 = conv3d_same_input_grad(dY, Wo) * gelu_grad(cache["zd0"])
    g[5] = conv3d_same_weight_grad(dd0, cache["s0"])
    ds0 = conv3d_same_input_grad(dd0, Wd0)
    c_up0 = U0.shape[1]
    dd1, dU0, dc0 = up2_grads(ds0[:c_up0], cache["d1"], U0)
    g[8] = (dU0, dc0)
    de0 = ds0[c_up0:]
    dd1 = dd1 * gelu_grad(cache["zd1"])
    g[4] = conv3d_same_weight_grad(dd1, cache["s1"])
    ds1 = conv3d_same_input_grad(dd1, Wd1)
    c_up1 = U1.shape[1]
    deb, dU1, dc1 = up2_grads(ds1[:c_up1], cache["eb"], U1)
    g[7] = (dU1, dc1)
    de1 = ds1[c_up1:]
    dzb = deb * gelu_grad(cache["zb"])
    g[3] = conv3d_same_weight_grad(dzb, cache["e2"])
    de2 = conv3d_same_input_grad(dzb, Wb)
    dz2 = de2 * gelu_grad(cache["z2"])
    g[2] = conv3d_same_weight_grad(dz2, cache["p1"])
    de1 = de1 + maxpool2_grad(conv3d_same_input_grad(dz2, W2), cache["e1"])
    dz1 = de1 * gelu_grad(cache["z1"])
    g[1] = conv3d_same_weight_grad(dz1, cache["p0"])
    de0 = de0 + maxpool2_grad(conv3d_same_input_grad(dz1, W1), cache["e0"])
    dz0 = de0 * gelu_grad(cache["z0"])
    g[0] = conv3d_same_weight_grad(dz0, cache["X"])
    dX = conv3d_same_input_grad(dz0, W0)
    return dX, flatten(g)
