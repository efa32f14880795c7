"""Solves through the C ABI against the oracle's direct solution."""
import numpy as np
import pytest
import torch

import mdgen
from helpers import instance_cases, rel_l2
from oracle import fem, solvers

pytestmark = pytest.mark.gpu


def test_jacobi_cg_single_segment():
    """Single segment, N = 16, f = 0, g = 1: Jacobi-CG (FP64) to 1e-10."""
    from paper_2505_08491_gb300 import Operator
    w = mdgen.WORKLOADS["single_segment_16"]
    g = mdgen.straight_segment(w["p0"], w["p1"], w["elems"], w["radius"])
    p = fem.Problem(16, g, 1.0)
    op = Operator(16, g, 1.0)
    b = op.rhs(None, 1.0)
    assert rel_l2(b.cpu().numpy(), p.rhs(None, 1.0)) <= 1e-14
    x, it, rel, ok = op.solve(b, tol=1e-10, maxit=5000)
    assert ok and rel <= 1e-10
    xd = solvers.direct_solve(p.A, p.rhs(None, 1.0))
    assert rel_l2(x.cpu().numpy(), xd) <= 1e-7
    xo, ito, relo = solvers.jacobi_cg(p.A, p.rhs(None, 1.0), 1e-10)
    assert abs(it - ito) <= max(2, 0.02 * ito)


@pytest.mark.parametrize("case", instance_cases(), ids=[c[0] for c in instance_cases()])
def test_fgmres_identity_pair_network(case):
    """FGMRES with the block preconditioner (identity-pair network) reaches
    1e-8 and matches the direct solution to 1e-6."""
    from paper_2505_08491_gb300 import Network, Operator
    from paper_2505_08491_gb300.weights import identity_pair_params
    name, N, g, beta, fseed = case
    p = fem.Problem(N, g, beta)
    op = Operator(N, g, beta)
    f = p.source(fseed)
    b = p.rhs(f, 1.0)
    x, it, rel, ok = op.solve(torch.from_numpy(b).cuda(), net=Network(identity_pair_params()), tol=1e-8,
                              restart=30, maxit=5000)
    assert ok and rel <= 1e-8
    xd = solvers.direct_solve(p.A, b)
    r = np.linalg.norm(b - p.A @ x.cpu().numpy()) / np.linalg.norm(b)
    assert r <= 1.01e-8
    assert rel_l2(x.cpu().numpy(), xd) <= 1e-6 * max(1.0, 1.0)


def test_batched_fgmres_jacobi_and_cg():
    """Several instances of different sizes in one batch: each converges and
    matches its own direct solve."""
    from paper_2505_08491_gb300 import Batch, Operator
    cases = instance_cases()
    probs = [fem.Problem(N, g, beta) for _, N, g, beta, _ in cases]
    ops = [Operator(N, g, beta) for _, N, g, beta, _ in cases]
    bs = [p.rhs(p.source(c[4]), 1.0) for p, c in zip(probs, cases)]
    for solver in ("fgmres_jacobi", "cg_jacobi"):
        B = Batch(ops, solver=solver, restart=30)
        b_all = torch.from_numpy(np.concatenate(bs)).cuda()
        x_all = torch.zeros_like(b_all)
        its, rels, ok = B.solve(b_all, x_all, tol=1e-8, maxit=20000)
        assert ok, (solver, its, rels)
        x = x_all.cpu().numpy()
        for i, p in enumerate(probs):
            xi = x[B.offsets[i]:B.offsets[i + 1]]
            true = np.linalg.norm(bs[i] - p.A @ xi) / np.linalg.norm(bs[i])
            assert true <= 1.01e-8, (solver, i, true)
            assert rels[i] == pytest.approx(true, rel=1e-3)
        B.close()


def test_solve_with_initial_guess_already_converged():
    from paper_2505_08491_gb300 import Operator
    name, N, g, beta, fseed = instance_cases()[1]
    p = fem.Problem(N, g, beta)
    op = Operator(N, g, beta)
    b = p.rhs(p.source(fseed), 1.0)
    xd = solvers.direct_solve(p.A, b)
    x, it, rel, ok = op.solve(torch.from_numpy(b).cuda(), x0=torch.from_numpy(xd).cuda(), tol=1e-8)
    assert ok and it == 0


def test_batched_solve_is_one_graph_launch():
    """A batched solve is one launch of its captured graph whatever the number
    of restart cycles (they run under a conditional WHILE node on the device),
    and the device-side counts and section times come back with it."""
    from paper_2505_08491_gb300 import Batch, Network, Operator
    from paper_2505_08491_gb300.weights import default_network_params
    insts = [mdgen.workload_instance("tree15_32", i) for i in range(3)]
    ops = [Operator(w["N"], w["graph"], w["beta"]) for w in insts]
    b = torch.cat([op.rhs(torch.from_numpy(mdgen.interior_source(w["N"], w["f_seed"])).cuda(), w["g"])
                   for w, op in zip(insts, ops)])
    net = Network(default_network_params())
    for solver, restart in (("fgmres_cnn", 8), ("cg_jacobi", 1)):
        B = Batch(ops, solver, net if solver == "fgmres_cnn" else None, restart=restart)
        B.set_profiling(True)
        x = torch.zeros_like(b)
        its, rels, ok = B.solve(b, x, tol=1e-8, maxit=20000)
        assert ok
        x.zero_()
        B.reset_stats()
        its, rels, ok = B.solve(b, x, tol=1e-8, maxit=20000)
        st = B.stats()
        assert ok and st["graph_launches"] == 1, st
        assert st["slot_gating"] == 2
        assert st["cycles"] >= (max(its) + restart - 1) // restart if solver == "fgmres_cnn" else st["cycles"] >= 1
        assert st["kernel_launches"] > 0
        if solver == "fgmres_cnn":
            # restart 8 and ~17 iterations: several cycles, every section timed
            assert st["cycles"] >= 3
            # four hidden convolutions per iteration slot that ran; at least one
            # slot per iteration of the slowest instance
            assert st["conv_hidden_launches"] % 4 == 0 and st["conv_hidden_launches"] >= 4 * max(its)
            for k in ("prec_ms", "conv_hidden_ms", "apply_ms", "arnoldi_ms", "restart_ms"):
                assert st[k] > 0, (k, st)
            assert st["conv_hidden_ms"] < st["prec_ms"]
        B.close()


def test_host_loop_gives_the_device_loop_result():
    """The host-driven loop (for kernel profilers) runs the same kernels as the
    one-launch solve: identical iterations and a bit-identical solution."""
    from paper_2505_08491_gb300 import Batch, Network, Operator
    from paper_2505_08491_gb300.weights import default_network_params
    insts = [mdgen.workload_instance("batch256_mixed", i) for i in (4, 13)]
    ops = [Operator(w["N"], w["graph"], w["beta"]) for w in insts]
    b = torch.cat([op.rhs(torch.from_numpy(mdgen.interior_source(w["N"], w["f_seed"])).cuda(), w["g"])
                   for w, op in zip(insts, ops)])
    net = Network(default_network_params("lower"))
    out = []
    for host in (False, True):
        B = Batch(ops, "fgmres_cnn", net, restart=30)
        B.set_prec_order("lower")
        B.set_host_loop(host)
        x = torch.zeros_like(b)
        its, rels, ok = B.solve(b, x, tol=1e-8)
        assert ok
        st = B.stats()
        assert (st["slot_gating"] == 3) == host
        assert st["graph_launches"] == (1 + st["cycles"] if host else 1)
        out.append((its, x.cpu().numpy()))
        B.close()
    assert out[0][0] == out[1][0]
    assert np.array_equal(out[0][1], out[1][1])
