"""Shared test helpers: instances for both sides, built only from mdgen."""
import numpy as np

import mdgen


def instance_cases():
    """(name, N, graph, beta, f_seed): small cases spanning several tiles and
    ragged tails, the single-segment case and a deep tree."""
    w = mdgen.WORKLOADS["single_segment_16"]
    seg = mdgen.straight_segment(w["p0"], w["p1"], w["elems"], w["radius"])
    return [
        ("segment16", 16, seg, 1.0, None),
        ("tree3_N9", 9, mdgen.random_tree(101, 0, depth=3, elems=5), 7.5, 3),
        ("tree4_N32", 32, mdgen.workload_instance("tree15_32", 0)["graph"], 1.0, 1_000_000),
        ("tree6_N21", 21, mdgen.random_tree(202, 0, depth=6, elems=3, radius_range=(0.01, 0.02)), 30.0, 11),
    ]


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
