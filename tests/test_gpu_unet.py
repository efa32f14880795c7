"""The U-net U3 on the GPU (md_unet_forward) against the oracle's FP64 U-net
(oracle/unet.py, pinned against PyTorch's operations in test_oracle_unet.py),
on random He-initialised weights and N(0,1) inputs: even and odd sizes (the
odd sizes drop a plane in pooling and append one after up-sampling), the
paper's 21^3 and a batch.  FP32 storage and accumulation over at most
27 x 128 terms per output: the relative error stays within a few 1e-6; the
bound is 2e-5, node by node within 2e-5 of the output's maximum."""
import numpy as np
import pytest
import torch

from helpers import rel_l2
from oracle import unet

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,batch", [(8, 1), (9, 2), (21, 2), (22, 1)])
def test_unet_forward_matches_oracle(n, batch):
    from paper_2505_08491_gb300 import UNet
    theta = unet.random_params(7 + n)
    assert UNet.num_params() == unet.num_params()
    rng = np.random.default_rng(n)
    X = rng.standard_normal((batch, 2, n, n, n))
    net = UNet(theta.astype(np.float32))
    Y = net.forward(torch.from_numpy(X.astype(np.float32)).cuda()).cpu().numpy().astype(np.float64)
    for b in range(batch):
        ref = unet.forward(X[b].astype(np.float32).astype(np.float64), theta.astype(np.float32).astype(np.float64))
        assert rel_l2(Y[b].ravel(), ref.ravel()) <= 2e-5, (n, b)
        assert np.max(np.abs(Y[b] - ref)) <= 2e-5 * np.max(np.abs(ref)), (n, b)
    net.close()


def test_unet_rejects_bad_sizes():
    from paper_2505_08491_gb300 import UNet
    net = UNet(unet.random_params(0).astype(np.float32))
    with pytest.raises(RuntimeError):
        net.forward(torch.zeros((1, 2, 3, 3, 3), device="cuda"))
    net.close()


@pytest.mark.parametrize("n,batch", [(9, 2), (12, 1)])
def test_unet_backward_matches_oracle(n, batch):
    """Input and parameter gradients of sum(dY * U(X)) against the oracle's
    FP64 backward (pinned against autograd): FP32 sums of up to 27 x 128 x n^3
    products, in an order that varies (atomic additions), relative L2 2e-4,
    and per layer the weight gradients within 1e-3 of that layer's norm."""
    from paper_2505_08491_gb300 import UNet
    theta = unet.random_params(30 + n).astype(np.float32)
    rng = np.random.default_rng(n + 1)
    X = rng.standard_normal((batch, 2, n, n, n)).astype(np.float32)
    dY = rng.standard_normal((batch, 1, n, n, n)).astype(np.float32)
    net = UNet(theta)
    dp, dX = net.backward(torch.from_numpy(X).cuda(), torch.from_numpy(dY).cuda(), need_dx=True)
    dp = dp.cpu().numpy().astype(np.float64)
    dX = dX.cpu().numpy().astype(np.float64)
    ref_p = np.zeros(unet.num_params())
    for b in range(batch):
        _, cache = unet.forward(X[b].astype(np.float64), theta.astype(np.float64), keep=True)
        rdX, rdp = unet.backward(dY[b].astype(np.float64), cache)
        ref_p += rdp
        assert rel_l2(dX[b].ravel(), rdX.ravel()) <= 2e-4, b
    assert rel_l2(dp, ref_p) <= 2e-4
    k = 0
    for wshape, nb in unet.param_shapes():
        nw = int(np.prod(wshape)) + nb
        seg, ref = dp[k:k + nw], ref_p[k:k + nw]
        assert np.linalg.norm(seg - ref) <= 1e-3 * np.linalg.norm(ref), wshape
        k += nw
    net.close()


def test_unet_parameters_round_trip():
    from paper_2505_08491_gb300 import UNet
    theta = unet.random_params(2).astype(np.float32)
    net = UNet(theta)
    assert np.array_equal(net.params(), theta)
    other = unet.random_params(3).astype(np.float32)
    net.set_params(torch.from_numpy(other).cuda())
    torch.cuda.synchronize()
    assert np.array_equal(net.params(), other)
    net.close()


def test_unet_train_loss_and_gradient_match_oracle():
    """md_unet_train_loss against the oracle's U-net loss (pinned in
    test_oracle_unet.py against the coupled residual of the preconditioner)
    on three 9^3-node instances with 1D parts (the lift l enters b0): the
    mean loss to 1e-4 relative and the gradient to 1e-3 relative L2 (FP32
    network and operator; the oracle's l from an FP64 direct 1D solve, the
    library's from its FP32 tree sweeps)."""
    import mdgen
    from oracle import fem, solvers
    from paper_2505_08491_gb300 import Operator, UNet
    probs, ops, rs = [], [], []
    for i in range(3):
        g = mdgen.random_tree(600 + i, 0, depth=3, elems=4)
        p = fem.Problem(8, g, 3.0 + i)
        r = mdgen.normal_vector(600, i, p.n).astype(np.float32)
        r[:p.n3][p.bd] = 0
        probs.append(p)
        ops.append(Operator(8, g, 3.0 + i))
        rs.append(r)
    theta = unet.random_params(21).astype(np.float32)
    net = UNet(theta)
    loss, grad = net.train_loss(ops, [torch.from_numpy(r).cuda() for r in rs])
    grad = grad.cpu().numpy().astype(np.float64)
    ref_l, ref_g = 0.0, 0.0
    for p, r in zip(probs, rs):
        Q = solvers.BlockPreconditioner(p, mode="jacobi")
        lift = Q.lift(solvers.direct_solve(p.B11, r[p.n3:].astype(np.float64)))
        L, g = solvers.training_loss_unet(p, r[:p.n3].astype(np.float64), lift, theta.astype(np.float64), grad=True)
        ref_l += L / len(rs)
        ref_g = ref_g + g / len(rs)
    assert loss == pytest.approx(ref_l, rel=1e-4)
    assert rel_l2(grad, ref_g) <= 1e-3
    net.close()


def test_unet_training_reduces_loss():
    """A few AdamW steps (md_unet_opt_step) on md_unet_train_loss's gradient
    lower the loss of a fixed minibatch."""
    import mdgen
    from paper_2505_08491_gb300 import Operator, UNet
    ops, rs = [], []
    for i in range(4):
        g = mdgen.random_tree(700 + i, 0, depth=3, elems=4)
        op = Operator(8, g, 1.0)
        r = mdgen.normal_vector(700, i, op.n).astype(np.float32)
        r[op.n3:] = 0
        M = 9
        idx = np.arange(M)
        bd = ((idx == 0) | (idx == M - 1))
        mask = ~(bd[:, None, None] | bd[None, :, None] | bd[None, None, :]).ravel()
        r[:op.n3] *= mask
        ops.append(op)
        rs.append(torch.from_numpy(r).cuda())
    net = UNet(unet.random_params(5).astype(np.float32))
    l0, _ = net.train_loss(ops, rs, with_grad=False)
    for _ in range(40):
        _, gr = net.train_loss(ops, rs)
        net.opt_step(gr, lr=1e-3)
    l1, _ = net.train_loss(ops, rs, with_grad=False)
    assert np.isfinite(l1) and l1 < 0.5 * l0, (l0, l1)
    net.close()


def identity_pair_unet():
    """U-net parameters with U(X) = X[0]: e0 = [GELU(x0), GELU(-x0), 0, ...]
    (centre taps +-1), d0 = [GELU(e0_0 - e0_1), GELU(e0_1 - e0_0), 0, ...] =
    [GELU(x0), GELU(-x0), ...] (the skip half of its input), Y = d0_0 - d0_1
    = x0 (GELU(u) - GELU(-u) = u); every other weight and bias zero, so the
    coarser levels and the up-sampled halves carry zeros."""
    layers = [(np.zeros(w), np.zeros(b)) for w, b in unet.param_shapes()]
    W0 = layers[0][0]
    W0[0, 0, 1, 1, 1], W0[1, 0, 1, 1, 1] = 1.0, -1.0
    Wd0 = layers[5][0]             # conv 64 -> 32 on [up0 (32) | e0 (32)]
    Wd0[0, 32, 1, 1, 1], Wd0[0, 33, 1, 1, 1] = 1.0, -1.0
    Wd0[1, 32, 1, 1, 1], Wd0[1, 33, 1, 1, 1] = -1.0, 1.0
    Wo = layers[6][0]
    Wo[0, 0, 1, 1, 1], Wo[0, 1, 1, 1, 1] = 1.0, -1.0
    return unet.flatten(layers)


@pytest.mark.parametrize("order", ["upper", "lower"])
def test_batched_solve_with_unet_matches_oracle(order):
    """The batched FGMRES(30) with the U-net as the 3D block solve
    (md_batch_set_unet) against the oracle's FGMRES with the same block
    preconditioner (mode 'unet') on three 9^3-node tree instances: the
    identity-pair U-net makes the 3D solve z0 = b0 / alpha, a deterministic
    preconditioner both sides apply alike.  Iterations within 1.2x + 2 (the
    orthogonalisation and precision differ), the true residual to 1.01e-8
    and the solution against the sparse direct one to 1e-6."""
    import mdgen
    from oracle import fem, solvers
    from paper_2505_08491_gb300 import Batch, Network, Operator, UNet
    from paper_2505_08491_gb300.weights import default_network_params
    theta = identity_pair_unet()
    probs, ops, bs = [], [], []
    for i in range(3):
        g = mdgen.random_tree(800 + i, 0, depth=3, elems=4)
        p = fem.Problem(8, g, 1.0 + i)
        probs.append(p)
        ops.append(Operator(8, g, 1.0 + i))
        bs.append(p.rhs(p.source(800 + i), 1.0))
    net = Network(default_network_params(order))
    un = UNet(theta.astype(np.float32))
    B = Batch(ops, "fgmres_cnn", net, restart=30)
    B.set_prec_order(order)
    B.set_unet(un)
    b_all = torch.from_numpy(np.concatenate(bs)).cuda()
    x_all = torch.zeros_like(b_all)
    its, rels, ok = B.solve(b_all, x_all, tol=1e-8, maxit=3000)
    assert ok, (its, rels)
    assert B.stats()["fallback_instances"] == 0
    x = x_all.cpu().numpy()
    for i, p in enumerate(probs):
        xi = x[B.offsets[i]:B.offsets[i + 1]]
        assert np.linalg.norm(bs[i] - p.A @ xi) / np.linalg.norm(bs[i]) <= 1.01e-8
        assert rel_l2(xi, solvers.direct_solve(p.A, bs[i])) <= 1e-6
        Q = solvers.BlockPreconditioner(p, mode="unet", params=theta, order=order)
        _, it_ref, rel_ref = solvers.fgmres(p.A, bs[i], Q, 1e-8, restart=30, maxit=3000)
        assert rel_ref <= 1e-8 and its[i] <= 1.2 * it_ref + 2 and it_ref <= 1.2 * its[i] + 2, (i, its[i], it_ref)
    B.close()
    un.close()
