"""Data-parallel training of the preconditioner network (one process per GPU).

Each process holds its own block of the training samples and its own copy of
the network.  Per step, every process computes the mean loss
||C z0 - b0||^2 / ||b0||^2 (Section 3.2 eq. (risk), Section 5.1) and its
gradient over its local minibatch on its GPU (``md_train_loss``); two
all-reduces (the count-weighted gradients, then the counts) give every
process the gradient of the mean loss over the union of the minibatches,
and every process applies the same AdamW step (``md_opt_step``) to its copy,
so the copies stay identical.  The only collective is that all-reduce of the
114,209 FP32 gradient values (plus two scalars) per step.

The gradient and the update are arguments, so that the collective logic can
be exercised on CPU processes with another gradient (the tests use the FP64
oracle's).
"""
from __future__ import annotations

import math

import numpy as np
import torch


def shard(n_items: int, rank: int, world: int) -> range:
    """Process `rank`'s contiguous block of n_items (the blocks of all ranks
    are disjoint and cover every item; sizes differ by at most one)."""
    return range(rank * n_items // world, (rank + 1) * n_items // world)


def average_gradient(grad: torch.Tensor, count: int, dist, group=None) -> torch.Tensor:
    """The mean-loss gradient over every process's samples, from each
    process's mean-loss gradient `grad` over its `count` samples:
    sum_r count_r grad_r / sum_r count_r."""
    weighted = grad * float(count)
    n = torch.tensor([float(count)], dtype=torch.float64, device=grad.device)
    dist.all_reduce(weighted, group=group)
    dist.all_reduce(n, group=group)
    if n.item() <= 0:
        raise ValueError("no samples on any process")
    return weighted / float(n.item())


def cosine_lr(step: int, total: int, lr: float, lr_min: float) -> float:
    """md_train's schedule: cosine decay from lr to lr_min over the steps."""
    frac = step / (total - 1) if total > 1 else 1.0
    return lr_min + 0.5 * (lr - lr_min) * (1.0 + math.cos(math.pi * frac))


def train_data_parallel(n_local: int, grad_fn, step_fn, *, epochs: int, batch: int, lr: float = 1e-3,
                        lr_min: float = 1e-5, seed: int = 0, dist=None, group=None):
    """Data-parallel training loop over this process's n_local samples.

    grad_fn(indices) -> (mean loss, mean-loss gradient tensor) over the local
    samples `indices`; step_fn(gradient, lr) applies one optimizer step.  Every
    process takes the same number of steps per epoch (the smallest local
    count over the processes, in minibatches of `batch`), shuffles its own
    samples (seed + rank), and steps with the averaged gradient.  Returns the
    mean loss over all processes' samples per epoch."""
    world = dist.get_world_size(group) if dist is not None else 1
    rank = dist.get_rank(group) if dist is not None else 0
    steps = torch.tensor([float(n_local // batch)], dtype=torch.float64)
    if dist is not None:
        dist.all_reduce(steps, op=dist.ReduceOp.MIN, group=group)
    steps = int(steps.item())
    if steps == 0:
        raise ValueError("fewer local samples than one minibatch on some process")
    rng = np.random.default_rng(seed + rank)
    total = steps * epochs
    history, k = [], 0
    for _ in range(epochs):
        perm = rng.permutation(n_local)
        loss_sum = 0.0
        for j in range(steps):
            idx = perm[j * batch:(j + 1) * batch]
            loss, grad = grad_fn(idx)
            if dist is not None and world > 1:
                grad = average_gradient(grad, len(idx), dist, group)
                lt = torch.tensor([float(loss)], dtype=torch.float64, device=grad.device)
                dist.all_reduce(lt, group=group)
                loss = float(lt.item()) / world
            step_fn(grad, cosine_lr(k, total, lr, lr_min))
            loss_sum += float(loss)
            k += 1
        history.append(loss_sum / steps)
    return history


def gpu_functions(net, ops: list, sample_op: list, residuals: list, *, betas=(0.9, 0.999),
                  weight_decay: float = 1e-4, eps: float = 1e-8):
    """grad_fn and step_fn of train_data_parallel on this process's GPU: the
    library's loss and gradient (md_train_loss) over local samples, and its
    AdamW step (md_opt_step) on `net`.  ops[sample_op[i]] and residuals[i]
    (float32 CUDA tensors of the operator's length) are the local samples.
    Samples of one minibatch must share a grid size."""
    from .api import Optimizer, train_loss
    opt = Optimizer(net, betas=betas, weight_decay=weight_decay, eps=eps)

    def grad_fn(idx):
        loss, grad = train_loss(net, [ops[sample_op[i]] for i in idx], [residuals[i] for i in idx])
        return loss, grad

    def step_fn(grad, lr):
        opt.step(grad, lr)

    return grad_fn, step_fn, opt
