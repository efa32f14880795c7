"""The paper's own setting on the GPU (Section 2 eq. (problem), Section 5.1):
natural conditions on the cube faces, k_Omega = sigma_Omega = 1e-3, the
vessel radius and the coupling's eps both 1e-3 (coupling 2 pi eps), u_Lambda
= 1 at the tree's root (graph node 0) and no source, on 21^3 grid nodes.  The
operator, the load vector (the known 1D value moved to the right-hand side),
alpha and the solves are checked against the oracle's assembly of the same
problem (its natural-condition and 1D-Dirichlet paths are pinned in
test_oracle_fem.py)."""
import numpy as np
import pytest
import torch

import mdgen
from helpers import rel_l2
from oracle import fem, solvers

pytestmark = pytest.mark.gpu

# paper_21 instances: 0 (127 segments), 2 (1 segment), 4 (7 segments)
CASES = (0, 2, 4)


def _pair(i):
    from paper_2505_08491_gb300 import Operator
    w = mdgen.workload_instance("paper_21", i)
    op = Operator(w["N"], w["graph"], w["beta"], **w["physics"])
    p = fem.Problem(w["N"], w["graph"], w["beta"], **w["physics"])
    return w, op, p


@pytest.mark.parametrize("i", CASES)
def test_paper_apply_rhs_alpha_match_oracle(i):
    w, op, p = _pair(i)
    assert (op.n3, op.n1) == (p.n3, p.n1)
    rng = np.random.default_rng(i)
    u = rng.standard_normal(p.n)
    ref = p.A @ u
    y64 = op.apply(torch.from_numpy(u).cuda()).cpu().numpy()
    assert rel_l2(y64, ref) <= 1e-12
    # every face, edge and corner row (natural conditions) to the same bound
    assert np.max(np.abs(y64 - ref)) <= 1e-12 * np.max(np.abs(ref))
    y32 = op.apply(torch.from_numpy(u.astype(np.float32)).cuda()).cpu().numpy()
    assert rel_l2(y32, ref) <= 1e-5
    b = p.rhs(p.source(w["f_seed"]), w["g"])
    bg = op.rhs(None, w["g"]).cpu().numpy()
    assert rel_l2(bg, b) <= 1e-13
    assert np.linalg.norm(b) > 0  # the 1D Dirichlet value drives the problem
    assert op.alpha == pytest.approx(p.alpha, rel=1e-12)


@pytest.mark.parametrize("i", CASES)
def test_paper_solves_match_oracle(i):
    """FGMRES(20) with the network (the paper's block order) and Jacobi-CG,
    to 1e-12 in the true FP64 residual, against the oracle's matrix and its
    sparse direct solution."""
    from paper_2505_08491_gb300 import Batch, Network
    from paper_2505_08491_gb300.weights import default_network_params
    w, op, p = _pair(i)
    b = p.rhs(p.source(w["f_seed"]), w["g"])
    xd = solvers.direct_solve(p.A, b)
    bt = op.rhs(None, w["g"])
    net = Network(default_network_params("upper"))
    for solver in ("fgmres_cnn", "cg_jacobi"):
        B = Batch([op], solver, net if solver == "fgmres_cnn" else None, restart=20)
        x = torch.zeros_like(bt)
        its, rels, ok = B.solve(bt, x, tol=1e-12, maxit=20000)
        assert ok and rels[0] <= 1e-12, (solver, its, rels)
        xn = x.cpu().numpy()
        assert np.linalg.norm(b - p.A @ xn) / np.linalg.norm(b) <= 1.01e-12
        assert rel_l2(xn, xd) <= 1e-6, solver
        B.close()
