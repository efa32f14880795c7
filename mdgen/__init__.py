"""Seeded synthetic inputs for the 3D-1D coupled problem.

This module is shared by the FP64 oracle (``oracle/``) and the CUDA path
(``paper_2505_08491_gb300``).  It holds no finite-element arithmetic: it only
draws graphs (the 1D network Lambda embedded in the unit cube, Section 2), the
scalar problem parameters of a workload, and random vectors.  Everything is a
deterministic function of integer seeds.

Graph format (a plain dict, consumed by both sides):
    xyz      float64 (n_nodes, 3)   node coordinates in [0, 1]^3
    edges    int32   (n_edges, 2)   node ids of each straight segment
    radius   float                  cylinder radius R (one per graph)
    elems    int                    P1 elements per segment
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "rng_for", "straight_segment", "random_tree", "normal_vector",
    "WORKLOADS", "workload_instance",
]

BOX_LO, BOX_HI = 0.1, 0.9


def rng_for(base_seed: int, instance: int = 0) -> np.random.Generator:
    """Independent stream for (base_seed, instance)."""
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([int(base_seed), int(instance)])))


def straight_segment(p0, p1, elems: int, radius: float) -> dict:
    """One straight segment from p0 to p1 (the single-vessel case)."""
    xyz = np.array([p0, p1], dtype=np.float64)
    return {"xyz": xyz, "edges": np.array([[0, 1]], dtype=np.int32),
            "radius": float(radius), "elems": int(elems)}


def _unit(v):
    return v / np.linalg.norm(v)


def _perp_frame(d):
    """Two unit vectors orthogonal to d and to each other."""
    a = np.zeros(3)
    a[int(np.argmin(np.abs(d)))] = 1.0
    u = _unit(np.cross(d, a))
    v = np.cross(d, u)
    return u, v


def _inside(p) -> bool:
    return bool(np.all(p >= BOX_LO) and np.all(p <= BOX_HI))


def _grow(rng, start, direction_fn, len_lo, len_hi):
    """Draw a segment end inside the box: up to 16 draws per length scale,
    halving the length scale up to 6 times, then head for the cube centre."""
    scale = 1.0
    for _ in range(7):
        for _ in range(16):
            d = direction_fn()
            length = scale * rng.uniform(len_lo, len_hi)
            end = start + length * d
            if _inside(end):
                return end, d
        scale *= 0.5
    d = _unit(np.array([0.5, 0.5, 0.5]) - start + 1e-12)
    length = min(len_lo, np.linalg.norm(np.array([0.5, 0.5, 0.5]) - start))
    return start + length * d, d


def random_tree(base_seed: int, instance: int, depth: int, *, elems: int = 8,
                radius_range=(0.01, 0.03), len_range=(0.08, 0.2),
                angle_deg=(20.0, 60.0)) -> dict:
    """Binary tree of ``depth`` generations (2**depth - 1 straight segments).

    Root at U[0.1,0.9]^3 with a direction uniform on the sphere; every segment
    end spawns two children, bent away from the parent direction by angles
    drawn from U(angle_deg) on opposite sides of a plane whose azimuth is
    uniform.  Every node stays in [0.1, 0.9]^3 (segments are straight, so the
    whole graph does).  Crossings of segments are not junctions.
    """
    rng = rng_for(base_seed, instance)
    radius = float(rng.uniform(*radius_range))
    lo, hi = len_range
    th_lo, th_hi = (math.radians(a) for a in angle_deg)
    root = rng.uniform(BOX_LO, BOX_HI, size=3)
    xyz = [root]
    edges = []

    def sphere_dir():
        return _unit(rng.standard_normal(3))

    end, d0 = _grow(rng, root, sphere_dir, lo, hi)
    xyz.append(end)
    edges.append((0, 1))
    frontier = [(1, d0)]
    for _gen in range(1, depth):
        nxt = []
        for node, d in frontier:
            u, v = _perp_frame(d)
            for side in (1.0, -1.0):
                def child_dir(d=d, u=u, v=v, side=side):
                    phi = rng.uniform(0.0, 2.0 * math.pi)
                    b = math.cos(phi) * u + math.sin(phi) * v
                    th = rng.uniform(th_lo, th_hi)
                    return _unit(math.cos(th) * d + side * math.sin(th) * b)
                end, dc = _grow(rng, xyz[node], child_dir, lo, hi)
                xyz.append(end)
                edges.append((node, len(xyz) - 1))
                nxt.append((len(xyz) - 1, dc))
        frontier = nxt
    return {"xyz": np.asarray(xyz, dtype=np.float64),
            "edges": np.asarray(edges, dtype=np.int32),
            "radius": radius, "elems": int(elems)}


def normal_vector(base_seed: int, instance: int, n: int, stream: int = 0) -> np.ndarray:
    """N(0, 1) float64 vector of length n for (seed, instance, stream)."""
    rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([int(base_seed), int(instance), 7919 + int(stream)])))
    return rng.standard_normal(n)


def interior_source(N: int, seed: int | None) -> np.ndarray | None:
    """Nodal source f ~ N(0, 1) on the interior nodes of the (N+1)^3 grid
    (x fastest), 0 on the cube boundary; None when seed is None (f = 0)."""
    if seed is None:
        return None
    f = normal_vector(seed, 0, (N + 1) ** 3)
    idx = np.arange(N + 1)
    b = (idx == 0) | (idx == N)
    f[(b[:, None, None] | b[None, :, None] | b[None, None, :]).ravel()] = 0.0
    return f


# Workload recipes.  Sizes are Q1 elements per cube edge (N); nodes (N+1)^3.
WORKLOADS = {
    # one straight segment, f = 0, g = 1, Jacobi-CG to 1e-10 in FP64
    "single_segment_16": dict(N=16, beta=1.0, kind="segment", elems=32, radius=0.02,
                              p0=(0.2, 0.5, 0.5), p1=(0.8, 0.5, 0.5), f="zero", g=1.0, tol=1e-10),
    # binary trees of depth 4 (15 segments), 8 elements per segment, f ~ N(0,1)
    "tree15_32": dict(N=32, beta=1.0, kind="tree", depth=(4, 4), elems=8, radius=(0.01, 0.03),
                      f="normal", g=1.0, tol=1e-8, restart=30, seed=1_000_000),
    # training graphs: depth 2-5, N in {16, 32}
    "train_trees": dict(N=(16, 32), beta=1.0, kind="tree", depth=(2, 5), elems=8, radius=(0.01, 0.03),
                        f="normal", g=1.0, seed=1),
    # resolution transfer: depth 5-7, 16 elements per segment, R ~ U(0.005, 0.02)
    # training over the deployment range: beta log-uniform [1, 100], 3-127 segments
    "train_trees_wide": dict(N=(16, 32), beta="loguniform", kind="tree", depth=(2, 7), elems=8,
                             radius=(0.005, 0.03), f="normal", g=1.0, seed=4_000_000),
    # training over the mixed batch's grid sizes: N in {32, 48, 64}, depth 2-7, beta log-uniform
    # [1, 100], R ~ U(0.01, 0.03); seeds disjoint from every evaluation workload
    "train_trees_mixed": dict(N=(32, 48, 64), beta="loguniform", kind="tree", depth=(2, 7), elems=8,
                              radius=(0.01, 0.03), f="normal", g=1.0, seed=6_000_000),
    # the mixed batch's grid sizes at beta = 1 (fine-tuning without the heavy-coupling rows)
    "train_trees_large": dict(N=(32, 48, 64), beta=1.0, kind="tree", depth=(2, 7), elems=8,
                              radius=(0.01, 0.03), f="normal", g=1.0, seed=9_000_000),
    "transfer_64": dict(N=64, beta=(1.0, 10.0, 100.0), kind="tree", depth=(5, 7), elems=16,
                        radius=(0.005, 0.02), f="normal", g=1.0, tol=1e-8, restart=50, seed=2_000_000),
    "transfer_128": dict(N=128, beta=(1.0, 10.0, 100.0), kind="tree", depth=(5, 7), elems=16,
                         radius=(0.005, 0.02), f="normal", g=1.0, tol=1e-8, restart=50, seed=2_000_000),
    # batched throughput: 256 instances, N in {32, 48, 64}, depth 3-8, beta log-uniform [1, 100]
    "batch256_mixed": dict(N=(32, 48, 64), beta="loguniform", kind="tree", depth=(3, 8), elems=8,
                           radius=(0.01, 0.03), f="normal", g=1.0, tol=1e-8, restart=30,
                           seed=3_000_000, count=256),
    # the paper's own setting (Section 2 eq. (problem), Section 5.1): 21^3 grid nodes, natural
    # conditions on the cube faces, k_Omega = sigma_Omega = 1e-3, eps = 1e-3 (coupling 2 pi eps,
    # vessel radius eps), u_Lambda = 1 at the tree's root, no source; trees of 1-127 segments;
    # FGMRES(20) to 1e-15 (Section 6)
    "paper_21": dict(N=20, beta=2.0 * np.pi * 1e-3, kind="tree", depth=(1, 7), elems=8, radius=(1e-3, 1e-3),
                     f="zero", g=0.0, tol=1e-15, restart=20, seed=5_000_000,
                     physics=dict(k_omega=1e-3, sigma_omega=1e-3, dirichlet=False, dirichlet_1d=(0,), u_d=1.0)),
    # training graphs of the paper's setting: the same physics and sizes as paper_21, seeds disjoint
    "train_paper_21": dict(N=20, beta=2.0 * np.pi * 1e-3, kind="tree", depth=(1, 7), elems=8, radius=(1e-3, 1e-3),
                           f="zero", g=0.0, seed=8_000_000,
                           physics=dict(k_omega=1e-3, sigma_omega=1e-3, dirichlet=False, dirichlet_1d=(0,), u_d=1.0)),
}


def workload_instance(name: str, i: int = 0) -> dict:
    """Problem instance i of a named workload: graph, N, beta, f-recipe.

    Returns dict(N, beta, graph, f_seed or None, g, instance, physics); physics
    holds the coefficients and boundary conditions of workloads that differ
    from the defaults (keyword arguments of the oracle's Problem), else {}.
    """
    w = WORKLOADS[name]
    if w["kind"] == "segment":
        g = straight_segment(w["p0"], w["p1"], w["elems"], w["radius"])
        return dict(N=w["N"], beta=w["beta"], graph=g, f_seed=None, g=w["g"], instance=i, physics={})
    seed = w["seed"] + i
    rng = rng_for(seed, 1)  # parameter stream, separate from the graph stream
    dlo, dhi = w["depth"]
    depth = int(rng.integers(dlo, dhi + 1))
    Ns = w["N"] if isinstance(w["N"], tuple) else (w["N"],)
    N = int(Ns[int(rng.integers(0, len(Ns)))])
    if w["beta"] == "loguniform":
        beta = float(10.0 ** rng.uniform(0.0, 2.0))
    elif isinstance(w["beta"], tuple):
        beta = float(w["beta"][int(rng.integers(0, len(w["beta"])))])
    else:
        beta = float(w["beta"])
    graph = random_tree(seed, 0, depth, elems=w["elems"], radius_range=w["radius"])
    f_seed = seed if w["f"] == "normal" else None
    return dict(N=N, beta=beta, graph=graph, f_seed=f_seed, g=w["g"], instance=i,
                physics=dict(w.get("physics", {})))
