"""Parameter vectors of the preconditioner network (flat FP32, md.h layout).

Layout: for each layer l (channels 3->32->32->32->32->32->1) the weights
W[c_out][c_in][kz][ky][kx] (offset q = k - 1, cross-correlation orientation)
followed by the biases b[c_out].
"""
from __future__ import annotations

import os

import numpy as np

CHANNELS = (3, 32, 32, 32, 32, 32, 1)
NPARAMS = sum(co * ci * 27 + co for ci, co in zip(CHANNELS[:-1], CHANNELS[1:]))
HERE = os.path.dirname(os.path.abspath(__file__))
TRAINED = os.path.join(HERE, "weights", "cnn_trained.bin")
# fine-tuned for the block lower-triangular order (1D parts of the training
# vectors zeroed: the network fitted to C z0 = r0)
TRAINED_LOWER = os.path.join(HERE, "weights", "cnn_trained_lower.bin")
# fine-tuned for the paper's own setting (natural conditions on the cube,
# k_Omega = sigma_Omega = 1e-3, eps = 1e-3, u_Lambda = 1 at the root: the
# train_paper_21 graphs), upper block order
TRAINED_PAPER = os.path.join(HERE, "weights", "cnn_paper21.bin")


def layers_to_flat(layers) -> np.ndarray:
    """[(W (co, ci, 3, 3, 3), b (co,)), ...] -> flat float32 vector."""
    parts = []
    for W, b in layers:
        parts.append(np.asarray(W, dtype=np.float64).ravel())
        parts.append(np.asarray(b, dtype=np.float64).ravel())
    flat = np.concatenate(parts).astype(np.float32)
    if flat.size != NPARAMS:
        raise ValueError(f"{flat.size} parameters, expected {NPARAMS}")
    return flat


def flat_to_layers(flat: np.ndarray):
    flat = np.asarray(flat, dtype=np.float64)
    out, o = [], 0
    for ci, co in zip(CHANNELS[:-1], CHANNELS[1:]):
        W = flat[o:o + co * ci * 27].reshape(co, ci, 3, 3, 3)
        o += co * ci * 27
        b = flat[o:o + co]
        o += co
        out.append((W, b))
    return out


def identity_pair_params() -> np.ndarray:
    """A network whose output is (channel 0 + channel 1) of its input, using
    GELU(u) - GELU(-u) = u: hidden channels 0/1 carry GELU(u), GELU(-u).
    All weights are +-1 (exact in BF16)."""
    layers = []
    for l, (ci, co) in enumerate(zip(CHANNELS[:-1], CHANNELS[1:])):
        W = np.zeros((co, ci, 3, 3, 3))
        b = np.zeros(co)
        if l == 0:
            W[0, 0, 1, 1, 1] = W[0, 1, 1, 1, 1] = 1.0
            W[1, 0, 1, 1, 1] = W[1, 1, 1, 1, 1] = -1.0
        elif l < len(CHANNELS) - 2:
            W[0, 0, 1, 1, 1], W[0, 1, 1, 1, 1] = 1.0, -1.0
            W[1, 0, 1, 1, 1], W[1, 1, 1, 1, 1] = -1.0, 1.0
        else:
            W[0, 0, 1, 1, 1], W[0, 1, 1, 1, 1] = 1.0, -1.0
        layers.append((W, b))
    return layers_to_flat(layers)


def random_params(seed: int) -> np.ndarray:
    """He-normal weights (std sqrt(2 / (27 c_in))), zero biases; the initial
    state of training."""
    rng = np.random.Generator(np.random.PCG64(seed))
    layers = []
    for ci, co in zip(CHANNELS[:-1], CHANNELS[1:]):
        layers.append((rng.standard_normal((co, ci, 3, 3, 3)) * np.sqrt(2.0 / (27 * ci)), np.zeros(co)))
    return layers_to_flat(layers)


def read_network_file(path: str) -> np.ndarray:
    """Parameters of a file written by md_cnn_save (magic MDCNN001, count,
    values, FNV-1a checksum)."""
    raw = open(path, "rb").read()
    if raw[:8] != b"MDCNN001":
        raise ValueError(f"{path}: not a network file")
    n = int(np.frombuffer(raw[8:16], dtype=np.int64)[0])
    vals = np.frombuffer(raw[16:16 + 4 * n], dtype=np.float32).copy()
    h = 1469598103934665603
    for byte in raw[16:16 + 4 * n]:
        h = ((h ^ byte) * 1099511628211) & 0xFFFFFFFFFFFFFFFF
    if int(np.frombuffer(raw[16 + 4 * n:24 + 4 * n], dtype=np.uint64)[0]) != h:
        raise ValueError(f"{path}: checksum mismatch")
    return vals


def paper_network_params() -> np.ndarray:
    """The network shipped for the paper's own setting (else the upper-order
    network)."""
    if os.path.exists(TRAINED_PAPER):
        return read_network_file(TRAINED_PAPER)
    return default_network_params("upper")


def default_network_params(order: str = "upper") -> np.ndarray:
    """The trained network shipped with the package for the block order
    ('upper', the paper's, or 'lower') if present, else the identity-pair
    network."""
    path = TRAINED_LOWER if order == "lower" and os.path.exists(TRAINED_LOWER) else TRAINED
    if os.path.exists(path):
        return read_network_file(path)
    return identity_pair_params()


# the U-net trained for the paper's own setting (train_paper_21), float32 .npy
TRAINED_UNET_PAPER = os.path.join(HERE, "weights", "unet_paper21.npy")


def paper_unet_params():
    """The shipped U-net for the paper's setting, or None."""
    return np.load(TRAINED_UNET_PAPER).astype(np.float32) if os.path.exists(TRAINED_UNET_PAPER) else None


# ---- the U-net U3 (md_unet_*): conv3 layers (c_in, c_out), then the up2 layers
UNET_CONVS = ((2, 32), (32, 64), (64, 128), (128, 128), (128, 64), (64, 32), (32, 1))
UNET_UPS = ((128, 64), (64, 32))


def unet_random_params(seed: int = 0) -> np.ndarray:
    """He-normal U-net weights (std sqrt(2 / fan_in); fan_in 27 c_in for a conv3,
    c_in for an up2), biases N(0, 0.01^2); the md_unet parameter layout."""
    rng = np.random.default_rng(seed)
    parts = []
    for ci, co in UNET_CONVS:
        parts += [rng.normal(0.0, np.sqrt(2.0 / (27 * ci)), co * ci * 27), rng.normal(0.0, 0.01, co)]
    for ci, co in UNET_UPS:
        parts += [rng.normal(0.0, np.sqrt(2.0 / ci), ci * co * 8), rng.normal(0.0, 0.01, co)]
    return np.concatenate(parts).astype(np.float32)
