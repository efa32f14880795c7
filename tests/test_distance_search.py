"""The distance field's two-stage search (CPU, no GPU).

The GPU kernel finds each grid node's distance to the 1D graph by searching all
segments with FP32 squared distances, then taking the FP64 minimum over the
segments whose FP32 value is within 1e-5 of the FP32 minimum.  That equals the
FP64 minimum over every segment as long as no FP32 squared distance is off by
more than half the margin.  These tests evaluate both precisions with the
kernel's formulas (FP32: p - a, t = clamp(((p - a) . d) / |d|^2), e = (p - a) - t d;
FP64: the formula of the plain search) at the grid nodes of workload graphs and
at random points close to the segments, and check that bound and that the FP64
minimiser is always among the candidates."""
import numpy as np
import pytest

import mdgen

MARGIN = 1e-5


def _segments(graph):
    xyz = np.asarray(graph["xyz"], dtype=np.float64)
    e = np.asarray(graph["edges"])
    return xyz[e[:, 0]], xyz[e[:, 1]]


def _q64(P, A, B):
    D = B - A
    dd = (D * D).sum(1)
    t = np.clip(((P[:, None, :] - A[None]) * D[None]).sum(-1) / dd[None], 0.0, 1.0)
    E = P[:, None, :] - (A[None] + t[..., None] * D[None])
    return (E * E).sum(-1)


def _q32(P32, A, B):
    D64 = B - A
    A32, D32 = A.astype(np.float32), D64.astype(np.float32)
    inv = (1.0 / (D64 * D64).sum(1)).astype(np.float32)
    U = (P32[:, None, :] - A32[None]).astype(np.float32)
    t = (U * D32[None]).sum(-1, dtype=np.float32) * inv[None]
    t = np.clip(t, np.float32(0), np.float32(1)).astype(np.float32)
    E = (U - t[..., None] * D32[None]).astype(np.float32)
    return (E * E).sum(-1, dtype=np.float32)


def _check(P64, P32, A, B):
    q64, q32 = _q64(P64, A, B), _q32(P32, A, B)
    assert np.max(np.abs(q32.astype(np.float64) - q64)) <= MARGIN / 2
    cand = q32 <= (q32.min(1) + np.float32(MARGIN))[:, None]
    assert cand[np.arange(len(P64)), q64.argmin(1)].all()
    return cand.sum(1)


@pytest.mark.parametrize("workload,index", [("batch256_mixed", 0), ("batch256_mixed", 3), ("paper_21", 1),
                                            ("transfer_64", 0)])
def test_grid_nodes_of_workload_graphs(workload, index):
    w = mdgen.workload_instance(workload, index)
    A, B = _segments(w["graph"])
    N = w["N"]
    step = max(1, (N + 1) // 20)
    ii = np.arange(0, N + 1, step)
    idx = np.stack(np.meshgrid(ii, ii, ii, indexing="ij"), -1).reshape(-1, 3)
    P64 = idx / N
    P32 = (idx.astype(np.float32) * np.float32(1.0 / N)).astype(np.float32)
    ncand = _check(P64, P32, A, B)
    assert ncand.max() <= 8


def test_points_near_the_segments():
    """Points within a few grid spacings of the graph, where the minimum is
    small and neighbouring segments compete."""
    w = mdgen.workload_instance("batch256_mixed", 5)
    A, B = _segments(w["graph"])
    rng = np.random.default_rng(11)
    k = rng.integers(0, len(A), 4000)
    t = rng.random(4000)
    P64 = A[k] + t[:, None] * (B[k] - A[k]) + rng.normal(0.0, 0.02, (4000, 3))
    P64 = np.clip(P64, 0.0, 1.0)
    P32 = P64.astype(np.float32)
    _check(P32.astype(np.float64), P32, A, B)
