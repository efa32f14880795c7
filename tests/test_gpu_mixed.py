"""Parity on the mixed and the transfer workloads with the shipped networks.

* The mixed batch (grids of 32^3, 48^3 and 64^3 elements, trees of 7-255
  segments, beta log-uniform in [1, 100]): a batch of six of its instances,
  the heavy-coupling ones among them, solved together by FGMRES(30) with the
  network in both block orders.  Every instance is checked against the
  oracle: its right-hand side, its true residual through the oracle's matrix,
  and its solution against the oracle's FP64 Jacobi-CG solution to 1e-13.
  The upper order switches the instances its network does not precondition
  to Jacobi; those are checked the same way.
* Resolution transfer at 64^3 (network trained at N <= 32): one instance at
  each beta in {10, 100}, both orders.

The solution check follows from the residual only up to cond(A): with
||r|| / ||b|| <= tol the error is <= cond(A) tol.  At 64^3 the 3D block has
cond ~ 0.4 N^2 ~ 2e3, so the solves for the solution check run to tol 1e-10
(1e-10 x 2e3 = 2e-7 <= 1e-6), the residual check to the benchmark's 1e-8.
"""
import numpy as np
import pytest
import torch

import mdgen
from helpers import rel_l2
from oracle import fem, solvers

pytestmark = pytest.mark.gpu

# batch256_mixed instances: (index, N, beta, segments)
# 6: 64, 98.5, 127 | 9: 48, 46.8, 127 | 24: 32, 96.9, 63 | 36: 48, 51.9, 7
# 18: 64, 1.0, 15 | 35: 64, 44.0, 255
MIXED = (6, 9, 24, 36, 18, 35)


def _rhs(w, op):
    f = mdgen.interior_source(w["N"], w["f_seed"])
    return op.rhs(torch.from_numpy(f).cuda() if f is not None else None, w["g"])


def _oracle(w):
    p = fem.Problem(w["N"], w["graph"], w["beta"])
    return p, p.rhs(p.source(w["f_seed"]), w["g"])


def _solve(insts, order, restart, tol, maxit=20000):
    from paper_2505_08491_gb300 import Batch, Network, Operator
    from paper_2505_08491_gb300.weights import default_network_params
    ops = [Operator(w["N"], w["graph"], w["beta"]) for w in insts]
    b_all = torch.cat([_rhs(w, op) for w, op in zip(insts, ops)])
    net = Network(default_network_params(order))
    B = Batch(ops, "fgmres_cnn", net, restart=restart)
    B.set_prec_order(order)
    x_all = torch.zeros_like(b_all)
    its, rels, ok = B.solve(b_all, x_all, tol=tol, maxit=maxit)
    return B, b_all.cpu().numpy(), x_all.cpu().numpy(), its, rels, ok


@pytest.mark.parametrize("order", ["lower", "upper"])
def test_mixed_batch_network_solves_match_oracle(order):
    insts = [mdgen.workload_instance("batch256_mixed", i) for i in MIXED]
    B, bs, xs, its, rels, ok = _solve(insts, order, 30, 1e-8)
    assert ok and max(rels) <= 1e-8, (its, rels)
    fallback = B.stats()["fallback_instances"]
    print(f"order {order}: iterations {its}, Jacobi fallback instances {fallback}")
    for i, w in enumerate(insts):
        p, b = _oracle(w)
        sl = slice(B.offsets[i], B.offsets[i + 1])
        assert rel_l2(bs[sl], b) <= 1e-13
        assert np.linalg.norm(b - p.A @ xs[sl]) / np.linalg.norm(b) <= 1.01e-8, (MIXED[i], w["N"], w["beta"])


@pytest.mark.parametrize("order", ["lower", "upper"])
def test_mixed_batch_solutions_match_oracle_cg(order):
    """The two heaviest instances (64^3 at beta 98.5, 48^3 at beta 46.8) in one
    batch to tol 1e-10, against the oracle's FP64 Jacobi-CG solution to 1e-13."""
    insts = [mdgen.workload_instance("batch256_mixed", i) for i in MIXED[:2]]
    B, bs, xs, its, rels, ok = _solve(insts, order, 30, 1e-10)
    assert ok and max(rels) <= 1e-10, (its, rels)
    for i, w in enumerate(insts):
        p, b = _oracle(w)
        xc, _, relc = solvers.jacobi_cg(p.A, b, 1e-13)
        assert relc <= 1e-12
        sl = slice(B.offsets[i], B.offsets[i + 1])
        assert rel_l2(xs[sl], xc) <= 1e-6, (MIXED[i], w["N"], w["beta"])


@pytest.mark.parametrize("order", ["lower", "upper"])
@pytest.mark.parametrize("beta", [10.0, 100.0])
def test_transfer_64_solve_matches_oracle(order, beta):
    """One 64^3 resolution-transfer instance (FGMRES(50)) at beta = 10 and 100:
    the residual through the oracle's matrix at tol 1e-8, and the solution at
    tol 1e-10 against the oracle's Jacobi-CG."""
    w = next(mdgen.workload_instance("transfer_64", i) for i in range(30)
             if mdgen.workload_instance("transfer_64", i)["beta"] == beta)
    p, b = _oracle(w)
    B, bs, xs, its, rels, ok = _solve([w], order, 50, 1e-8)
    assert ok and rels[0] <= 1e-8, (its, rels)
    assert rel_l2(bs, b) <= 1e-13
    assert np.linalg.norm(b - p.A @ xs) / np.linalg.norm(b) <= 1.01e-8
    B, bs, xs, its, rels, ok = _solve([w], order, 50, 1e-10)
    assert ok and rels[0] <= 1e-10, (its, rels)
    xc, _, relc = solvers.jacobi_cg(p.A, b, 1e-13)
    assert relc <= 1e-12
    assert rel_l2(xs, xc) <= 1e-6
