"""What the trained network gains: FGMRES iterations to 1e-8 on unseen
15-segment trees at N = 32 with the trained network, against the same
solver without a learned 3D block (identity network, Jacobi) and against an
untrained network; plus parity of the solution and of the iteration count
with the FP64 oracle running the same weights."""
import os

import numpy as np
import pytest
import torch

import mdgen
from helpers import rel_l2
from oracle import cnn, fem, solvers

pytestmark = pytest.mark.gpu

COUNT = 8


@pytest.fixture(scope="module")
def setup():
    from paper_2505_08491_gb300 import Operator
    from paper_2505_08491_gb300.weights import TRAINED
    assert os.path.exists(TRAINED), "trained network file missing"
    insts = [mdgen.workload_instance("tree15_32", i) for i in range(COUNT)]
    ops = [Operator(w["N"], w["graph"], w["beta"]) for w in insts]
    bs = []
    for w, op in zip(insts, ops):
        f = mdgen.interior_source(w["N"], w["f_seed"])
        bs.append(op.rhs(torch.from_numpy(f).cuda(), w["g"]))
    return insts, ops, torch.cat(bs)


def mean_iters(ops, b_all, solver, params, stats=None):
    from paper_2505_08491_gb300 import Batch, Network
    net = Network(params) if params is not None else None
    B = Batch(ops, solver, net, restart=30)
    x = torch.zeros_like(b_all)
    its, rels, ok = B.solve(b_all, x, tol=1e-8, maxit=2000)
    if stats is not None:
        stats.update(B.stats())
    B.close()
    return float(np.mean(its)), ok, x


def test_trained_network_gain(setup):
    from paper_2505_08491_gb300.weights import default_network_params, identity_pair_params, random_params
    insts, ops, b_all = setup
    st = {}
    trained, ok_t, _ = mean_iters(ops, b_all, "fgmres_cnn", default_network_params(), st)
    # the stagnation safeguard stays off where the network works
    assert st["fallback_instances"] == 0
    identity, ok_i, _ = mean_iters(ops, b_all, "fgmres_cnn", identity_pair_params())
    jacobi, ok_j, _ = mean_iters(ops, b_all, "fgmres_jacobi", None)
    untrained, ok_u, _ = mean_iters(ops, b_all, "fgmres_cnn", random_params(0))
    assert ok_t and ok_i and ok_j
    assert trained < 0.5 * identity, (trained, identity)
    assert trained < 0.5 * jacobi, (trained, jacobi)
    assert trained < untrained, (trained, untrained)


def test_trained_solution_and_iterations_match_oracle(setup):
    from paper_2505_08491_gb300.weights import default_network_params, flat_to_layers
    insts, ops, b_all = setup
    w = insts[0]
    p = fem.Problem(w["N"], w["graph"], w["beta"])
    b = p.rhs(p.source(w["f_seed"]), w["g"])
    assert rel_l2(b_all[:p.n].cpu().numpy(), b) <= 1e-13
    its, ok, x_all = mean_iters(ops[:1], b_all[:p.n].contiguous(), "fgmres_cnn", default_network_params())
    x = x_all.cpu().numpy()
    assert ok
    assert np.linalg.norm(b - p.A @ x) / np.linalg.norm(b) <= 1.01e-8
    xd = solvers.direct_solve(p.A, b)
    assert rel_l2(x, xd) <= 1e-6
    layers = [(cnn.round_bf16(W), np.asarray(bb, np.float32).astype(np.float64))
              for W, bb in flat_to_layers(default_network_params())]
    Q = solvers.BlockPreconditioner(p, mode="cnn", params=layers, bf16=True)
    xo, it_o, rel_o = solvers.fgmres(p.A, b, Q, 1e-8, restart=30, maxit=500)
    assert rel_o <= 1e-8
    assert its <= 1.2 * it_o + 2 and it_o <= 1.2 * its + 2, (its, it_o)


def test_lower_block_order_solves_and_matches_oracle_iterations(setup):
    """The lower-triangular block order (network first, then the 1D solve)
    with the shipped network: converges on the benchmark instances, and its
    iteration count on instance 0 is the oracle's FP64 FGMRES with the same
    order and weights within 1.2x + 2."""
    from paper_2505_08491_gb300 import Batch, Network
    from paper_2505_08491_gb300.weights import default_network_params, flat_to_layers
    insts, ops, b_all = setup
    net = Network(default_network_params())
    B = Batch(ops, "fgmres_cnn", net, restart=30)
    B.set_prec_order("lower")
    x = torch.zeros_like(b_all)
    its, rels, ok = B.solve(b_all, x, tol=1e-8, maxit=2000)
    assert ok and max(rels) <= 1e-8
    w = insts[0]
    p = fem.Problem(w["N"], w["graph"], w["beta"])
    b = p.rhs(p.source(w["f_seed"]), w["g"])
    layers = [(cnn.round_bf16(W), np.asarray(bb, np.float32).astype(np.float64))
              for W, bb in flat_to_layers(default_network_params())]
    Q = solvers.BlockPreconditioner(p, mode="cnn", params=layers, bf16=True, order="lower")
    _, it_o, rel_o = solvers.fgmres(p.A, b, Q, 1e-8, restart=30, maxit=500)
    assert rel_o <= 1e-8
    assert its[0] <= 1.2 * it_o + 2 and it_o <= 1.2 * its[0] + 2, (its[0], it_o)


@pytest.mark.parametrize("order", ["upper", "lower"])
def test_smoothed_solve_matches_oracle_iterations(setup, order):
    """FGMRES(30) with one Jacobi sweep before and after the network
    (Section 5, pre- and post-smoothing) in the batched solve: converges on
    the benchmark instances to the true residual 1e-8, and on instance 0
    needs the oracle's FP64 FGMRES iterations with the same smoothing, order
    and weights within 1.2x + 2."""
    from paper_2505_08491_gb300 import SMOOTH_OMEGA, Batch, Network
    from paper_2505_08491_gb300.weights import default_network_params, flat_to_layers
    insts, ops, b_all = setup
    params = default_network_params(order)
    net = Network(params)
    B = Batch(ops, "fgmres_cnn", net, restart=30)
    B.set_prec_order(order)
    B.set_smoothing(1)
    x = torch.zeros_like(b_all)
    its, rels, ok = B.solve(b_all, x, tol=1e-8, maxit=2000)
    assert ok and max(rels) <= 1e-8
    assert B.stats()["fallback_instances"] == 0
    w = insts[0]
    p = fem.Problem(w["N"], w["graph"], w["beta"])
    b = p.rhs(p.source(w["f_seed"]), w["g"])
    xs = x[:p.n].cpu().numpy()
    assert np.linalg.norm(b - p.A @ xs) / np.linalg.norm(b) <= 1.01e-8
    layers = [(cnn.round_bf16(W), np.asarray(bb, np.float32).astype(np.float64)) for W, bb in flat_to_layers(params)]
    Q = solvers.BlockPreconditioner(p, mode="cnn", params=layers, bf16=True, order=order, smooth=(1, SMOOTH_OMEGA))
    _, it_o, rel_o = solvers.fgmres(p.A, b, Q, 1e-8, restart=30, maxit=500)
    assert rel_o <= 1e-8
    assert its[0] <= 1.2 * it_o + 2 and it_o <= 1.2 * its[0] + 2, (its[0], it_o)


@pytest.mark.parametrize("order", ["upper", "lower"])
def test_inner_fgmres_solve_matches_oracle_iterations(setup, order):
    """FGMRES(30) whose 3D block solve is three inner FGMRES steps with the
    network (Section 6) in the batched solve: converges on the benchmark
    instances to the true residual 1e-8, and on instance 0 needs the
    oracle's FP64 FGMRES iterations with the same inner steps, order and
    weights within 1.2x + 2."""
    from paper_2505_08491_gb300 import Batch, Network
    from paper_2505_08491_gb300.weights import default_network_params, flat_to_layers
    insts, ops, b_all = setup
    params = default_network_params(order)
    net = Network(params)
    B = Batch(ops, "fgmres_cnn", net, restart=30)
    B.set_prec_order(order)
    B.set_inner_iters(3)
    x = torch.zeros_like(b_all)
    its, rels, ok = B.solve(b_all, x, tol=1e-8, maxit=2000)
    assert ok and max(rels) <= 1e-8
    assert B.stats()["fallback_instances"] == 0
    w = insts[0]
    p = fem.Problem(w["N"], w["graph"], w["beta"])
    b = p.rhs(p.source(w["f_seed"]), w["g"])
    xs = x[:p.n].cpu().numpy()
    assert np.linalg.norm(b - p.A @ xs) / np.linalg.norm(b) <= 1.01e-8
    layers = [(cnn.round_bf16(W), np.asarray(bb, np.float32).astype(np.float64)) for W, bb in flat_to_layers(params)]
    Q = solvers.BlockPreconditioner(p, mode="cnn", params=layers, bf16=True, order=order, inner=3)
    _, it_o, rel_o = solvers.fgmres(p.A, b, Q, 1e-8, restart=30, maxit=500)
    assert rel_o <= 1e-8
    assert its[0] <= 1.2 * it_o + 2 and it_o <= 1.2 * its[0] + 2, (its[0], it_o)
