"""Backward kernels and training against the FP64 oracle.

The GPU stores activations, weights and activation gradients in BF16 and
accumulates in FP32; gradients are compared with the oracle's FP64 analytic
gradients (taken on the same BF16-rounded forward) by cosine >= 0.999 and
relative L2 <= 2e-2 per layer."""
import numpy as np
import pytest
import torch

import mdgen
from helpers import instance_cases, rel_l2
from oracle import cnn, fem, solvers

pytestmark = pytest.mark.gpu


def flat_grads(grads):
    return np.concatenate([np.concatenate([dW.ravel(), db.ravel()]) for dW, db in grads])


def layer_slices():
    o, out = 0, []
    for ci, co in zip(cnn.CHANNELS[:-1], cnn.CHANNELS[1:]):
        out.append(slice(o, o + co * ci * 27 + co))
        o += co * ci * 27 + co
    return out


def cosine(a, b):
    return float(a @ b / (np.linalg.norm(a) * np.linalg.norm(b)))


@pytest.mark.parametrize("engine", ["tensor", "cuda_cores"])
@pytest.mark.parametrize("n", [5, 9])
def test_network_backward_matches_oracle(n, engine):
    from paper_2505_08491_gb300 import Network
    from paper_2505_08491_gb300.weights import flat_to_layers, random_params
    flat = random_params(31)
    layers = [(cnn.round_bf16(W), np.asarray(b, np.float32).astype(np.float64)) for W, b in flat_to_layers(flat)]
    net = Network(flat)
    net.set_engine(engine)
    rng = np.random.default_rng(n)
    X = rng.standard_normal((2, 3, n, n, n)).astype(np.float32)
    dY = rng.standard_normal((2, 1, n, n, n)).astype(np.float32)
    dp, dX = net.backward(torch.from_numpy(X).cuda(), torch.from_numpy(dY).cuda(), need_dx=True)
    dp = dp.cpu().numpy().astype(np.float64)
    dX = dX.cpu().numpy()
    ref = 0
    refX = []
    for s in range(2):
        _, saved = cnn.forward(X[s].astype(np.float64), layers, bf16=True, keep=True)
        grads, gx = cnn.backward(dY[s].astype(np.float64), layers, saved)
        ref = ref + flat_grads(grads)
        refX.append(gx)
    for sl in layer_slices():
        assert cosine(dp[sl], ref[sl]) >= 0.999
        assert rel_l2(dp[sl], ref[sl]) <= 2e-2
    assert cosine(dX.ravel().astype(np.float64), np.stack(refX).ravel()) >= 0.999


def test_network_function_autograd():
    """NetworkFunction inside torch autograd: gradients reach X and params."""
    from paper_2505_08491_gb300 import Network, NetworkFunction
    from paper_2505_08491_gb300.weights import random_params
    flat = random_params(4)
    net = Network(flat)
    X = torch.randn(1, 3, 7, 7, 7, device="cuda", requires_grad=True)
    P = torch.from_numpy(flat).cuda().requires_grad_(True)
    Y = NetworkFunction.apply(X, P, net)
    (Y * Y).sum().backward()
    dp, dX = net.backward(X.detach(), 2 * Y.detach(), need_dx=True)
    assert torch.allclose(P.grad, dp) and torch.allclose(X.grad, dX)


def _samples(N, count, seed):
    from paper_2505_08491_gb300 import Operator
    probs, ops, rs = [], [], []
    for i in range(count):
        g = mdgen.random_tree(seed + i, 0, depth=3, elems=4)
        p = fem.Problem(N, g, 3.0 + i)
        r = mdgen.normal_vector(seed, i, p.n).astype(np.float32)
        r[:p.n3][p.bd] = 0
        probs.append(p)
        ops.append(Operator(N, g, 3.0 + i))
        rs.append(r)
    return probs, ops, rs


def test_train_loss_and_gradient_match_oracle():
    from paper_2505_08491_gb300 import Network, train_loss
    from paper_2505_08491_gb300.weights import flat_to_layers, random_params
    probs, ops, rs = _samples(8, 3, 500)
    flat = random_params(6)
    layers = [(cnn.round_bf16(W), np.asarray(b, np.float32).astype(np.float64)) for W, b in flat_to_layers(flat)]
    net = Network(flat)
    loss, grad = train_loss(net, ops, [torch.from_numpy(r).cuda() for r in rs])
    grad = grad.cpu().numpy().astype(np.float64)
    ref_l, ref_g = 0.0, 0.0
    for p, r in zip(probs, rs):
        Q = solvers.BlockPreconditioner(p, mode="jacobi")
        z1 = solvers.direct_solve(p.B11, r[p.n3:].astype(np.float64))
        lift = Q.lift(z1)
        L, g = solvers.training_loss(p, r[:p.n3].astype(np.float64), lift, layers, bf16=True, grad=True)
        ref_l += L / len(rs)
        ref_g = ref_g + flat_grads(g) / len(rs)
    assert loss == pytest.approx(ref_l, rel=2e-2)
    assert cosine(grad, ref_g) >= 0.99


def test_training_reduces_loss():
    from paper_2505_08491_gb300 import Network, train, train_loss
    from paper_2505_08491_gb300.weights import random_params
    probs, ops, rs = _samples(8, 4, 900)
    samples, sop = [], []
    for i, (p, r) in enumerate(zip(probs, rs)):
        for k in range(4):
            v = mdgen.normal_vector(77 + k, i, p.n).astype(np.float32)
            v[:p.n3][p.bd] = 0
            samples.append(torch.from_numpy(v).cuda())
            sop.append(i)
    net = Network(random_params(1))
    l0, _ = train_loss(net, [ops[i] for i in sop], samples, with_grad=False)
    hist = train(net, ops, sop, samples, epochs=30, batch=4, lr=1e-3, lr_min=1e-4, seed=3)
    l1, _ = train_loss(net, [ops[i] for i in sop], samples, with_grad=False)
    assert np.all(np.isfinite(hist))
    assert l1 < 0.5 * l0, (l0, l1, hist[:3], hist[-3:])


def test_krylov_training_samples_match_oracle_basis():
    """The paper's training vectors for one graph (Section 4.1): b from the 1D
    load through md_lift, and q5..q8 of the Krylov basis of the 3D block
    started at b.  Against the oracle's own construction (B11 LU, M01, C, MGS in
    FP64): the Krylov vectors agree up to sign to 1e-5 (the GPU lift is FP32;
    perturbing b at that level moves q5..q8 of this instance by <= 4e-7 in the
    oracle), are orthonormal, and vanish on Dirichlet nodes."""
    from paper_2505_08491_gb300 import Operator
    from paper_2505_08491_gb300.train_net import krylov_samples
    name, N, g, beta, _ = instance_cases()[1]
    p = fem.Problem(N, g, beta)
    op = Operator(N, g, beta)
    samples = [v.double().cpu().numpy() for v in krylov_samples(op, 1.0)]
    assert len(samples) == 5
    b_r = samples[0]
    assert np.all(b_r[:p.n3] == 0.0)
    assert rel_l2(b_r[p.n3:], p.rhs(None, 1.0)[p.n3:]) <= 1e-6
    # oracle basis
    z1 = solvers.BlockPreconditioner(p, mode="jacobi").B11_lu.solve(p.rhs(None, 1.0)[p.n3:])
    q = [-beta * (p.M01 @ z1)]
    q[0] = q[0] / np.linalg.norm(q[0])
    for _ in range(8):
        w = p.C @ q[-1]
        for _ in range(2):
            for qi in q:
                w -= (qi @ w) * qi
        q.append(w / np.linalg.norm(w))
    Q = np.stack([s[:p.n3] for s in samples[1:]])
    for i, qg in enumerate(Q):
        ref = q[5 + i]
        assert min(np.linalg.norm(qg - ref), np.linalg.norm(qg + ref)) <= 1e-5, i
        assert np.all(qg[p.bd] == 0.0)
    assert np.allclose(Q @ Q.T, np.eye(4), atol=1e-6)
    assert all(np.all(s[p.n3:] == 0.0) for s in samples[1:])
