"""The multi-rank path of the benchmark on CPU (gloo, world size 2): ranks
solve disjoint instance blocks, and the whole-job throughput takes the
slowest rank's time and every rank's solves."""
import os
import socket
import sys

import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    insts = bench.instances("tree15_32", rank, 3)
    local_ms = 100.0 * (rank + 1)          # rank 1 is the slower one
    max_ms, total, value = bench.job_throughput(local_ms, len(insts) * 2, world, "cpu", dist)
    seeds = torch.tensor([float(w["instance"]) for w in insts])
    gathered = [torch.zeros_like(seeds) for _ in range(world)]
    dist.all_gather(gathered, seeds)
    out[rank] = (max_ms, total, value, sorted(float(v) for g in gathered for v in g.tolist()))
    dist.destroy_process_group()


def test_two_ranks_gloo():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        max_ms, total, value, seeds = res[r]
        assert max_ms == 200.0
        assert total == 12                      # 2 ranks x 3 instances x 2 steps
        assert abs(value - 12 / 0.2) < 1e-9
        assert seeds == [0.0, 1.0, 2.0, 3.0, 4.0, 5.0]   # disjoint blocks covering 0..5


# ---- every rank runs the CPU side of the path on its own block ----------------

BLOCK = 2


def _solve_block(insts):
    """The oracle's FP64 Jacobi-CG on each instance of a block: iterations,
    true relative residual and solution norm (what a rank reports back)."""
    from oracle import fem, solvers
    out = []
    for w in insts:
        p = fem.Problem(w["N"], w["graph"], w["beta"])
        b = p.rhs(p.source(w["f_seed"]), w["g"])
        x, it, rel = solvers.jacobi_cg(p.A, b, 1e-8)
        out.append((int(w["instance"]), it, rel, float(x @ x)))
    return out


def _rank_solve(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine = _solve_block(bench.instances("tree15_32", rank, BLOCK))
    got = [None] * world
    dist.all_gather_object(got, mine)
    out[rank] = got
    dist.destroy_process_group()


def test_ranks_solve_disjoint_blocks_and_gather():
    """Two gloo ranks each assemble and solve (oracle, CPU) their own block of
    the benchmark's instances; the gathered results are those of one process
    solving all of them."""
    sys.path.insert(0, ROOT)
    import bench
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_solve, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    ref = _solve_block(bench.instances("tree15_32", 0, world * BLOCK))
    for r in range(world):
        flat = [row for block in res[r] for row in block]
        assert [row[0] for row in flat] == list(range(world * BLOCK))
        for a, b in zip(flat, ref):
            assert a[1] == b[1] and a[2] <= 1e-8 and abs(a[3] - b[3]) <= 1e-12 * abs(b[3])


# ---- data-parallel training: the gradient all-reduce ---------------------------

def _toy_samples(n, seed):
    """n training samples of a 4^3-node problem and a toy 6-layer network
    (4 channels), for the FP64 oracle's loss and gradient."""
    import numpy as np

    import mdgen
    from oracle import fem, solvers
    g = mdgen.straight_segment((0.3, 0.4, 0.5), (0.7, 0.6, 0.5), 4, 0.05)
    p = fem.Problem(3, g, beta=5.0)
    rng = np.random.default_rng(seed)
    samples = []
    for _ in range(n):
        r0 = rng.standard_normal(p.n3)
        r0[p.bd] = 0.0
        l = solvers.BlockPreconditioner(p, mode="jacobi").lift(rng.standard_normal(p.n1))
        samples.append((r0, l))
    return p, samples


def _toy_params():
    import numpy as np
    rng = np.random.default_rng(99)
    ch = (3, 4, 4, 4, 4, 4, 1)
    return [(rng.standard_normal((co, ci, 3, 3, 3)) * np.sqrt(2.0 / (27 * ci)), 0.1 * rng.standard_normal(co))
            for ci, co in zip(ch[:-1], ch[1:])]


def _flat(grads):
    import numpy as np
    return np.concatenate([np.concatenate([dW.ravel(), db.ravel()]) for dW, db in grads])


def _unflat(v, like):
    out, k = [], 0
    for W, b in like:
        out.append((v[k:k + W.size].reshape(W.shape), v[k + W.size:k + W.size + b.size]))
        k += W.size + b.size
    return out


def _mean_grad(p, samples, params, idx):
    """Mean oracle loss and gradient over samples[idx] (what md_train_loss
    computes on a GPU)."""
    import numpy as np

    from oracle import solvers
    Ls, gs = [], []
    for i in idx:
        r0, l = samples[i]
        L, g = solvers.training_loss(p, r0, l, params, grad=True)
        Ls.append(L)
        gs.append(_flat(g))
    return float(np.mean(Ls)), torch.from_numpy(np.mean(gs, axis=0))


def _adam_step(state, grad, lr):
    """A plain AdamW step on the flat parameters (the update md_opt_step makes)."""
    import numpy as np
    b1, b2, eps, wd = 0.9, 0.999, 1e-8, 1e-4
    state["t"] += 1
    g = grad.numpy()
    state["m"] = b1 * state["m"] + (1 - b1) * g
    state["v"] = b2 * state["v"] + (1 - b2) * g * g
    mh = state["m"] / (1 - b1 ** state["t"])
    vh = state["v"] / (1 - b2 ** state["t"])
    w = state["w"] * (1 - lr * wd)
    state["w"] = w - lr * mh / (np.sqrt(vh) + eps)


def _rank_dp(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import numpy as np

    from paper_2505_08491_gb300.data_parallel import average_gradient, shard, train_data_parallel
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    p, samples = _toy_samples(6, 5)
    mine = list(shard(len(samples), rank, world))
    params = _toy_params()
    # one averaged gradient over the whole local block
    _, g = _mean_grad(p, samples, params, mine)
    avg = average_gradient(g, len(mine), dist)
    # two epochs of the loop, minibatches of 2, the update on the flat parameters
    w0 = _flat(params)
    state = {"w": w0.copy(), "m": np.zeros_like(w0), "v": np.zeros_like(w0), "t": 0}
    local = [samples[i] for i in mine]
    hist = train_data_parallel(len(local), lambda idx: _mean_grad(p, local, _unflat(state["w"], params), idx),
                               lambda grad, lr: _adam_step(state, grad, lr), epochs=2, batch=2, lr=1e-2,
                               lr_min=1e-3, seed=7, dist=dist)
    out[rank] = (mine, avg.numpy(), state["w"], hist)
    dist.destroy_process_group()


def test_data_parallel_gradient_average_and_training_loop():
    """Two gloo ranks holding disjoint halves of the samples: the averaged
    gradient equals the one-process gradient of the union, and two epochs of
    the data-parallel loop leave identical parameters on both ranks, equal to
    one process replaying the same union minibatches."""
    import numpy as np

    from paper_2505_08491_gb300.data_parallel import cosine_lr
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_dp, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    p, samples = _toy_samples(6, 5)
    params = _toy_params()
    blocks = [res[r][0] for r in range(world)]
    assert sorted(i for b in blocks for i in b) == list(range(6)) and not set(blocks[0]) & set(blocks[1])
    _, union = _mean_grad(p, samples, params, range(6))
    for r in range(world):
        assert np.allclose(res[r][1], union.numpy(), rtol=1e-12, atol=1e-15)
    assert np.array_equal(res[0][2], res[1][2])                 # identical copies
    # replay in one process: each step's minibatch is the union of the ranks'
    w0 = _flat(params)
    state = {"w": w0.copy(), "m": np.zeros_like(w0), "v": np.zeros_like(w0), "t": 0}
    rngs = [np.random.default_rng(7 + r) for r in range(world)]
    k = 0
    for _ in range(2):
        perms = [rng.permutation(3) for rng in rngs]
        for j in range(1):                                      # 3 local samples // batch 2
            idx = [blocks[r][i] for r in range(world) for i in perms[r][2 * j:2 * j + 2]]
            _, g = _mean_grad(p, samples, _unflat(state["w"], params), idx)
            _adam_step(state, g, cosine_lr(k, 2, 1e-2, 1e-3))
            k += 1
    assert np.allclose(res[0][2], state["w"], rtol=1e-12, atol=1e-14)
    assert not np.allclose(res[0][2], w0)                       # the loop did move the parameters
