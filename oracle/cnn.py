"""The convolutional preconditioner network in FP64, forward and backward.

TEST INFRASTRUCTURE (oracle): see the package docstring.

Network (the fully convolutional hypothesis space of Section 4.2, with the
channel pattern this build uses): six 3x3x3 convolutions with zero 'same'
padding, channels 3 -> 32 -> 32 -> 32 -> 32 -> 32 -> 1, a bias on every
layer and GELU(x) = x * Phi(x) after layers 1-5.

Convolution (Section 4.2): Y_i = sum_j k_ij * X_j.  The paper writes the sum
over kernel offsets q with X(p - q); the code stores the kernel in the
cross-correlation orientation Y(p) = sum_q w(q) X(p + q), which is the same
operator with the kernel flipped (w(q) = k(-q)).

Tensors are (channels, z, y, x); weights (c_out, c_in, 3, 3, 3) indexed by
offset + 1 in (z, y, x).

Optional BF16 emulation (bf16=True) rounds the network input and every hidden
activation to bfloat16 (round to nearest even, through FP32), the precision
in which weights and activations are held; weights are expected to be
BF16-representable already.  Sums stay in FP64.
"""
from __future__ import annotations

import numpy as np
from scipy.special import erf

CHANNELS = (3, 32, 32, 32, 32, 32, 1)


def round_bf16(x: np.ndarray) -> np.ndarray:
    """Round to the nearest bfloat16 (ties to even), via FP32."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32).astype(np.float64)


def gelu(x):
    return 0.5 * x * (1.0 + erf(x / np.sqrt(2.0)))


def gelu_grad(x):
    return 0.5 * (1.0 + erf(x / np.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / np.sqrt(2.0 * np.pi)


def conv3d_same(X: np.ndarray, W: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Y[o, p] = b[o] + sum_{c, q in {-1,0,1}^3} W[o, c, q+1] X[c, p+q], zero outside."""
    cin, Z, Y, Xn = X.shape
    cout = W.shape[0]
    Xp = np.zeros((cin, Z + 2, Y + 2, Xn + 2))
    Xp[:, 1:-1, 1:-1, 1:-1] = X
    out = np.zeros((cout, Z, Y, Xn)) + b[:, None, None, None]
    for dz in range(3):
        for dy in range(3):
            for dx in range(3):
                sl = Xp[:, dz:dz + Z, dy:dy + Y, dx:dx + Xn].reshape(cin, -1)
                out += (W[:, :, dz, dy, dx] @ sl).reshape(cout, Z, Y, Xn)
    return out


def conv3d_same_input_grad(dY: np.ndarray, W: np.ndarray) -> np.ndarray:
    """Adjoint of conv3d_same in X: dX[c, p] = sum_{o, q} W[o, c, q+1] dY[o, p-q]."""
    cout, Z, Y, Xn = dY.shape
    cin = W.shape[1]
    dXp = np.zeros((cin, Z + 2, Y + 2, Xn + 2))
    flat = dY.reshape(cout, -1)
    for dz in range(3):
        for dy in range(3):
            for dx in range(3):
                dXp[:, dz:dz + Z, dy:dy + Y, dx:dx + Xn] += (W[:, :, dz, dy, dx].T @ flat).reshape(cin, Z, Y, Xn)
    return dXp[:, 1:-1, 1:-1, 1:-1]


def conv3d_same_weight_grad(dY: np.ndarray, X: np.ndarray):
    """dW[o, c, q+1] = sum_p dY[o, p] X[c, p+q];  db[o] = sum_p dY[o, p]."""
    cout, Z, Y, Xn = dY.shape
    cin = X.shape[0]
    Xp = np.zeros((cin, Z + 2, Y + 2, Xn + 2))
    Xp[:, 1:-1, 1:-1, 1:-1] = X
    flat = dY.reshape(cout, -1)
    dW = np.zeros((cout, cin, 3, 3, 3))
    for dz in range(3):
        for dy in range(3):
            for dx in range(3):
                sl = Xp[:, dz:dz + Z, dy:dy + Y, dx:dx + Xn].reshape(cin, -1)
                dW[:, :, dz, dy, dx] = flat @ sl.T
    return dW, flat.sum(axis=1)


def init_params(seed: int, channels=CHANNELS, bf16: bool = True):
    """He-style random weights (std sqrt(2 / fan_in)), small biases; BF16-representable if bf16."""
    rng = np.random.Generator(np.random.PCG64(seed))
    params = []
    for cin, cout in zip(channels[:-1], channels[1:]):
        W = rng.standard_normal((cout, cin, 3, 3, 3)) * np.sqrt(2.0 / (27 * cin))
        b = rng.standard_normal(cout) * 0.01
        if bf16:
            W = round_bf16(W)
            b = np.asarray(b, dtype=np.float32).astype(np.float64)
        params.append((W, b))
    return params


def forward(X: np.ndarray, params, bf16: bool = False, keep: bool = False):
    """Network output (1, z, y, x) for input X (3, z, y, x).
    keep=True also returns the list of (layer input, pre-activation)."""
    a = round_bf16(X) if bf16 else X
    saved = []
    L = len(params)
    for l, (W, b) in enumerate(params):
        z = conv3d_same(a, W, b)
        saved.append((a, z))
        if l < L - 1:
            a = gelu(z)
            if bf16:
                a = round_bf16(a)
        else:
            a = z
    return (a, saved) if keep else a


def backward(dY: np.ndarray, params, saved):
    """Gradients (dW, db) per layer and dX, for output gradient dY."""
    grads = [None] * len(params)
    g = dY
    for l in range(len(params) - 1, -1, -1):
        W, _ = params[l]
        a_in, z = saved[l]
        if l < len(params) - 1:
            g = g * gelu_grad(z)
        dW, db = conv3d_same_weight_grad(g, a_in)
        grads[l] = (dW, db)
        g = conv3d_same_input_grad(g, W)
    return grads, g
