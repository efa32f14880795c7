"""The seeded input generators (mdgen): determinism and the stated shapes."""
import math

import numpy as np

import mdgen


def test_tree_is_deterministic_and_sized():
    for depth in (1, 2, 4, 8):
        g1 = mdgen.random_tree(123, 4, depth)
        g2 = mdgen.random_tree(123, 4, depth)
        assert np.array_equal(g1["xyz"], g2["xyz"]) and np.array_equal(g1["edges"], g2["edges"])
        assert len(g1["edges"]) == 2 ** depth - 1
        assert len(g1["xyz"]) == 2 ** depth
        assert np.all(g1["xyz"] >= mdgen.BOX_LO) and np.all(g1["xyz"] <= mdgen.BOX_HI)
        assert 0.01 <= g1["radius"] <= 0.03
    assert not np.array_equal(mdgen.random_tree(123, 5, 4)["xyz"], mdgen.random_tree(123, 4, 4)["xyz"])


def test_tree_lengths_and_angles():
    g = mdgen.random_tree(9, 0, 5)
    xyz, edges = g["xyz"], g["edges"]
    L = np.linalg.norm(xyz[edges[:, 1]] - xyz[edges[:, 0]], axis=1)
    assert np.all(L <= 0.2 + 1e-12)
    assert np.all(L > 0)
    # most segments keep the drawn length (the rest were shortened to stay in the box)
    assert np.mean(L >= 0.08) > 0.5
    parent_of = {int(c): int(p) for p, c in edges}
    angles = []
    for p, c in edges:
        if int(p) in parent_of:
            gp = parent_of[int(p)]
            d1 = xyz[p] - xyz[gp]
            d2 = xyz[c] - xyz[p]
            angles.append(math.degrees(math.acos(np.clip(d1 @ d2 / np.linalg.norm(d1) / np.linalg.norm(d2), -1, 1))))
    angles = np.array(angles)
    assert np.mean((angles >= 20 - 1e-9) & (angles <= 60 + 1e-9)) > 0.5


def test_workload_instances():
    a = mdgen.workload_instance("tree15_32", 0)
    assert a["N"] == 32 and len(a["graph"]["edges"]) == 15 and a["beta"] == 1.0
    Ns = set()
    for i in range(40):
        w = mdgen.workload_instance("batch256_mixed", i)
        Ns.add(w["N"])
        assert 1.0 <= w["beta"] <= 100.0
        assert 7 <= len(w["graph"]["edges"]) <= 255
    assert Ns == {32, 48, 64}
    s = mdgen.workload_instance("single_segment_16")
    assert s["graph"]["elems"] == 32 and s["f_seed"] is None
    v1 = mdgen.normal_vector(5, 1, 100)
    assert np.array_equal(v1, mdgen.normal_vector(5, 1, 100))


def test_paper_workload_recipe():
    """The paper's setting (Section 2 eq. (problem), Section 5.1): 21^3 grid
    nodes, k = sigma = 1e-3, coupling 2 pi eps with eps = 1e-3 also the vessel
    radius, natural conditions on the cube, u_Lambda = 1 at the root; the
    oracle solves it and holds the root at exactly 1."""
    import numpy as np
    from oracle import fem, solvers
    w = mdgen.workload_instance("paper_21", 2)
    assert w["N"] == 20 and abs(w["beta"] - 2 * np.pi * 1e-3) < 1e-15
    assert w["graph"]["radius"] == 1e-3 and w["f_seed"] is None and w["g"] == 0.0
    ph = w["physics"]
    assert ph["dirichlet"] is False and tuple(ph["dirichlet_1d"]) == (0,)
    assert ph["k_omega"] == ph["sigma_omega"] == 1e-3
    assert mdgen.workload_instance("tree15_32", 0)["physics"] == {}
    p = fem.Problem(w["N"], w["graph"], w["beta"], **ph)
    b = p.rhs(None, w["g"])
    x, it, rel = solvers.fgmres(p.A, b, solvers.BlockPreconditioner(p, mode="exact"), 1e-13, restart=20)
    assert rel <= 1e-13
    assert x[p.n3 + 0] == 1.0 or abs(x[p.n3 + 0] - 1.0) < 1e-12
