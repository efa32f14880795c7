"""Train the preconditioner network and save it (weights/cnn_trained.bin).

Training set (the unsupervised residual set of Section 4.1, on seeded random
trees): workload train_trees = graphs of 3-31 segments (binary trees of depth
2-5) on grids N = 16 and 32, beta = 1; train_trees_wide = 3-127 segments,
radius U(0.005, 0.03), beta log-uniform in [1, 100].  Per graph 8 right-hand sides of the block preconditioner:
4 random vectors (N(0,1) on every unknown, zero on Dirichlet nodes; the
high-frequency augmentation of Section 4.1.2) and the residuals of the
Jacobi-preconditioned FGMRES(30) solve of the graph's own problem after 5,
10, 20 and 30 iterations (residuals the solver actually meets).  --set kry,
hf and all build the paper's sets instead or in addition: b, the 3D forcing
of the 1D problem (eq. (setB)), with the Krylov vectors q5..q8 of the 3D
block started at b (Section 4.1.1) or with random vectors (Section 4.1.2).
Loss, AdamW and the cosine schedule run in md_train.

Usage: python -m paper_2505_08491_gb300.train_net --graphs 1024 --epochs 20
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

import mdgen  # noqa: E402
from paper_2505_08491_gb300 import Batch, Network, Operator, train  # noqa: E402
from paper_2505_08491_gb300.weights import TRAINED, random_params  # noqa: E402

HARVEST = (5, 10, 20, 30)


def interior_mask(N):
    idx = np.arange(N + 1)
    b = (idx == 0) | (idx == N)
    return ~(b[:, None, None] | b[None, :, None] | b[None, None, :]).ravel()


def krylov_samples(op, g: float):
    """The paper's samples for one graph (Section 4.1, eq. (setB) and the
    Krylov augmentation of Section 4.1.1): b = the 3D forcing of the 1D
    problem (l = beta Pi^T W Psi B11^{-1} f1 for the 1D load f1), as the
    residual [0; f1] that produces it, and q5..q8 of an orthonormal basis
    q0 = b/||b||, q1, ..., q8 of the Krylov space of the 3D block C started
    at b (modified Gram-Schmidt, twice, in FP64), as residuals [q; 0]."""
    n3, n = op.n3, op.n
    f1 = op.rhs(None, g)[n3:].float()
    rb = torch.zeros(n, dtype=torch.float32, device="cuda")
    rb[n3:] = f1
    l, _ = op.lift(rb)
    out = [rb]
    Q = op.krylov_basis(l.contiguous(), 8)          # q0..q8 of K_9(C, b), FP64 two-pass MGS in the library
    for qi in Q[5:9]:
        r = torch.zeros(n, dtype=torch.float32, device="cuda")
        r[:n3] = qi
        out.append(r)
    return out


def build_set(n_graphs: int, first: int = 0, workload: str = "train_trees", kind: str = "residuals"):
    """kind: 'residuals' (4 random vectors + 4 harvested FGMRES residuals per
    graph), 'base' ({b} alone, the paper's set B of eq. (setB) without
    augmentation), 'kry' ({b} and q5..q8, the paper's Krylov-augmented set),
    'hf' ({b} and 4 random vectors, the paper's high-frequency set) or 'all'
    (residuals, b and q5..q8)."""
    insts = [mdgen.workload_instance(workload, first + i) for i in range(n_graphs)]
    ops = [Operator(w["N"], w["graph"], w["beta"], **w["physics"]) for w in insts]
    samples, sample_op = [], []
    by_N = {}
    for i, (w, op) in enumerate(zip(insts, ops)):
        by_N.setdefault(w["N"], []).append(i)
        if kind in ("base", "kry", "hf", "all"):
            ks = krylov_samples(op, w["g"])
            for r in (ks if kind in ("kry", "all") else ks[:1]):
                samples.append(r)
                sample_op.append(i)
        if kind in ("kry", "base"):
            continue
        # random vectors on the unknowns: with natural conditions on the cube
        # every grid node is one
        m3 = interior_mask(w["N"]) if w["physics"].get("dirichlet", True) else np.ones(op.n3, bool)
        mask = torch.from_numpy(np.concatenate([m3, np.ones(op.n1, bool)])).cuda()
        for k in range(4):
            v = torch.from_numpy(mdgen.normal_vector(w["f_seed"] or 0, first + i, op.n, stream=k).astype(np.float32)).cuda()
            samples.append(v * mask)
            sample_op.append(i)
    if kind in ("base", "kry", "hf"):
        return ops, samples, sample_op
    # harvested residuals, batched per grid size
    for N, idx in by_N.items():
        sub = [ops[i] for i in idx]
        bs = []
        for i in idx:
            w = insts[i]
            f = mdgen.interior_source(w["N"], w["f_seed"])
            bs.append(ops[i].rhs(torch.from_numpy(f).cuda() if f is not None else None, w["g"]))
        b_all = torch.cat(bs)
        B = Batch(sub, "fgmres_jacobi", restart=30)
        for k in HARVEST:
            x_all = torch.zeros_like(b_all)
            B.solve(b_all, x_all, tol=1e-14, maxit=k)
            for j, i in enumerate(idx):
                o0, o1 = B.offsets[j], B.offsets[j + 1]
                r = bs[j] - ops[i].apply(x_all[o0:o1].contiguous())
                samples.append(r.float())
                sample_op.append(i)
        B.close()
    return ops, samples, sample_op


def mean_iterations(net, count: int, order: str = "upper"):
    """Mean and max FGMRES(30) iterations to 1e-8 with `net` on the first
    `count` tree15_32 instances, solved as one batch."""
    insts = [mdgen.workload_instance("tree15_32", i) for i in range(count)]
    ops = [Operator(w["N"], w["graph"], w["beta"]) for w in insts]
    b = torch.cat([op.rhs(torch.from_numpy(mdgen.interior_source(w["N"], w["f_seed"])).cuda(), w["g"])
                   for w, op in zip(insts, ops)])
    B = Batch(ops, "fgmres_cnn", net, restart=30)
    B.set_prec_order(order)
    x = torch.zeros_like(b)
    its, rels, ok = B.solve(b, x, tol=1e-8, maxit=3000)
    fb = B.stats()["fallback_instances"]
    B.close()
    return float(np.mean(its)), int(np.max(its)), bool(ok), int(fb)


def evaluate(net, workload: str, count: int, order: str = "upper", tol: float | None = None,
             restart: int | None = None, inner: int = 0, maxit: int = 20000, unet=None) -> dict:
    """FGMRES iterations to `tol` (the workload's own tolerance by default)
    with `net` on the first `count` instances of `workload`, solved as one
    batch from x0 = 0, and Jacobi-CG on the same batch for comparison; every
    instance as [index, segments, iterations, final true residual]."""
    w0 = mdgen.WORKLOADS[workload]
    tol = float(w0.get("tol", 1e-8)) if tol is None else float(tol)
    restart = int(w0.get("restart", 30)) if restart is None else int(restart)
    insts = [mdgen.workload_instance(workload, i) for i in range(count)]
    ops = [Operator(w["N"], w["graph"], w["beta"], **w["physics"]) for w in insts]
    b = torch.cat([op.rhs(torch.from_numpy(f).cuda() if (f := mdgen.interior_source(w["N"], w["f_seed"])) is not None
                          else None, w["g"]) for w, op in zip(insts, ops)])
    out = {"workload": workload, "instances": count, "order": order, "inner": inner, "tol": tol, "restart": restart,
           "network": "unet" if unet is not None else "cnn"}
    for solver in ("fgmres_cnn", "cg_jacobi"):
        B = Batch(ops, solver, net if solver == "fgmres_cnn" else None, restart=restart)
        if solver == "fgmres_cnn":
            B.set_prec_order(order)
            if inner:
                B.set_inner_iters(inner)
            if unet is not None:
                B.set_unet(unet)
        x = torch.zeros_like(b)
        its, rels, _ = B.solve(b, x, tol=tol, maxit=maxit)
        fb = B.stats().get("fallback_instances", 0) if solver == "fgmres_cnn" else 0
        B.close()
        conv = [k for k in range(count) if rels[k] <= tol]
        out[solver] = {"converged": len(conv), "mean_iterations_converged": float(np.mean([its[k] for k in conv])) if conv else None,
                       "median_iterations": float(np.median(its)), "max_iterations": int(np.max(its)),
                       "jacobi_fallback_instances": int(fb),
                       "per_instance": [[k, len(insts[k]["graph"]["edges"]), int(its[k]), float(rels[k])]
                                        for k in range(count)]}
    return out


def train_unet(net, ops, sample_op, samples, *, epochs: int, batch: int, lr: float, lr_min: float, seed: int = 0):
    """The U-net's unsupervised training: AdamW (md_unet_opt_step) on the
    mean loss of minibatches of samples that share a grid size
    (md_unet_train_loss), cosine decay of the learning rate from lr to
    lr_min.  Returns the mean loss per epoch."""
    by_n = {}
    for i, k in enumerate(sample_op):
        by_n.setdefault(ops[k].N, []).append(i)
    rng = np.random.default_rng(seed)
    steps = sum(len(v) // batch for v in by_n.values())
    if steps == 0:
        raise ValueError("fewer samples than one minibatch")
    total, k, hist = steps * epochs, 0, []
    for _ in range(epochs):
        batches = []
        for idx in by_n.values():
            perm = rng.permutation(idx)
            batches += [perm[j * batch:(j + 1) * batch] for j in range(len(perm) // batch)]
        order = rng.permutation(len(batches))
        acc = 0.0
        for bi in order:
            mb = batches[bi]
            loss, grad = net.train_loss([ops[sample_op[i]] for i in mb], [samples[i] for i in mb])
            frac = k / (total - 1) if total > 1 else 1.0
            net.opt_step(grad, lr_min + 0.5 * (lr - lr_min) * (1.0 + np.cos(np.pi * frac)))
            acc += loss
            k += 1
        hist.append(acc / len(batches))
    return hist


def ablation(args):
    """One network per training set from the same initialisation, evaluated
    on the 32^3 tree workload (the analogue of the paper's Table 5)."""
    rows = {}
    for kind in ("base", "kry", "hf"):
        t0 = time.time()
        ops, samples, sample_op = build_set(args.graphs, workload=args.workload, kind=kind)
        torch.cuda.synchronize()
        t1 = time.time()
        net = Network(random_params(args.seed))
        hist = train(net, ops, sample_op, samples, epochs=args.epochs, batch=args.batch, lr=args.lr,
                     lr_min=args.lr_min, seed=args.seed)
        t2 = time.time()
        mean_it, max_it, ok, fb = mean_iterations(net, args.eval_count)
        rows[kind] = {"samples": len(samples), "final_loss": hist[-1], "set_seconds": t1 - t0,
                      "train_seconds": t2 - t1, "mean_iterations": mean_it, "max_iterations": max_it,
                      "converged": ok, "jacobi_fallback_instances": fb}
        net.close()
    print(json.dumps({"ablation": rows, "graphs": args.graphs, "epochs": args.epochs, "lr": args.lr,
                      "seed": args.seed, "eval": f"tree15_32, {args.eval_count} instances, FGMRES(30), tol 1e-8"}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--graphs", type=int, default=1024)
    ap.add_argument("--epochs", type=int, default=20)
    ap.add_argument("--batch", type=int, default=32)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--lr-min", type=float, default=1e-5)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--out", default=TRAINED)
    ap.add_argument("--init", default=None, help="start from this network file")
    ap.add_argument("--workload", default="train_trees",
                    choices=["train_trees", "train_trees_wide", "train_trees_mixed", "train_trees_large",
                             "train_paper_21"])
    ap.add_argument("--set", default="residuals", choices=["residuals", "base", "kry", "hf", "all"],
                    help="training vectors per graph (see build_set)")
    ap.add_argument("--ablation", action="store_true",
                    help="the training-set ablation of Section 4.1 (the paper's Table 5): one network per set "
                         "(base = {b} alone, kry = {b} + q5..q8, hf = {b} + 4 random vectors), the same seed, "
                         "epochs and learning rate, each evaluated by the mean FGMRES(30) iterations on "
                         "--eval-count tree15_32 instances (upper block order); prints one JSON line")
    ap.add_argument("--eval-count", type=int, default=100)
    ap.add_argument("--zero-1d", action="store_true",
                    help="train for the block lower-triangular order: the 1D part of every training vector is "
                         "zeroed, so the network sees [r0/s, 0, d] and is fitted to C z0 = r0")
    ap.add_argument("--eval-workload", default=None,
                    help="after training (or, with --eval-only, for the --init network) print the FGMRES and "
                         "Jacobi-CG iterations on the first --eval-count instances of this workload")
    ap.add_argument("--eval-only", action="store_true")
    ap.add_argument("--eval-tol", type=float, default=None, help="tolerance (default: the workload's)")
    ap.add_argument("--eval-inner", type=int, default=0, help="inner FGMRES steps of the 3D block solve")
    ap.add_argument("--eval-order", default="upper", choices=["upper", "lower"])
    ap.add_argument("--arch", default="cnn", choices=["cnn", "unet"],
                    help="the network: the six-layer CNN (md_cnn) or the paper's U-net U3 (md_unet; its parameters "
                         "saved as a float32 .npy, --init loads one)")
    args = ap.parse_args()
    if args.arch == "unet":
        return main_unet(args)
    if args.ablation:
        return ablation(args)
    if args.eval_only:
        net = Network.load(args.init) if args.init else Network(random_params(args.seed))
        print(json.dumps({"network": args.init, **evaluate(net, args.eval_workload or "tree15_32", args.eval_count,
                                                            args.eval_order, args.eval_tol, inner=args.eval_inner)}))
        return
    t0 = time.time()
    ops, samples, sample_op = build_set(args.graphs, workload=args.workload, kind=args.set)
    if args.zero_1d:
        kept, kept_op = [], []
        for r, i in zip(samples, sample_op):
            r = r.clone()
            r[ops[i].n3:] = 0.0
            if float(torch.linalg.vector_norm(r)) > 0.0:
                kept.append(r)
                kept_op.append(i)
        samples, sample_op = kept, kept_op
    torch.cuda.synchronize()
    t1 = time.time()
    net = Network.load(args.init) if args.init else Network(random_params(args.seed))
    hist = train(net, ops, sample_op, samples, epochs=args.epochs, batch=args.batch, lr=args.lr,
                 lr_min=args.lr_min, seed=args.seed)
    t2 = time.time()
    os.makedirs(os.path.dirname(args.out), exist_ok=True)
    net.save(args.out)
    rec = {"workload": args.workload, "set": args.set, "zero_1d": args.zero_1d, "graphs": args.graphs,
           "samples": len(samples), "epochs": args.epochs, "set_seconds": t1 - t0, "train_seconds": t2 - t1,
           "loss": hist}
    if args.eval_workload:
        rec["evaluation"] = evaluate(net, args.eval_workload, args.eval_count, args.eval_order, args.eval_tol,
                                     inner=args.eval_inner)
    print(json.dumps(rec))


def main_unet(args):
    """--arch unet: train (or, with --eval-only, evaluate) the U-net."""
    from paper_2505_08491_gb300 import Network, UNet
    from paper_2505_08491_gb300.weights import default_network_params, unet_random_params
    params = np.load(args.init).astype(np.float32) if args.init else unet_random_params(args.seed)
    net = UNet(params)
    rec = {"arch": "unet", "init": args.init}
    if not args.eval_only:
        t0 = time.time()
        ops, samples, sample_op = build_set(args.graphs, workload=args.workload, kind=args.set)
        if args.zero_1d:
            for i, r in enumerate(samples):
                samples[i] = r.clone()
                samples[i][ops[sample_op[i]].n3:] = 0.0
        torch.cuda.synchronize()
        t1 = time.time()
        hist = train_unet(net, ops, sample_op, samples, epochs=args.epochs, batch=args.batch, lr=args.lr,
                          lr_min=args.lr_min, seed=args.seed)
        t2 = time.time()
        out = os.path.join(os.path.dirname(TRAINED), "unet_trained.npy") if args.out == TRAINED else args.out
        out = out if out.endswith(".npy") else os.path.splitext(out)[0] + ".npy"
        os.makedirs(os.path.dirname(os.path.abspath(out)), exist_ok=True)
        np.save(out, net.params())
        rec.update({"workload": args.workload, "set": args.set, "zero_1d": args.zero_1d, "graphs": args.graphs,
                    "samples": len(samples), "epochs": args.epochs, "set_seconds": t1 - t0,
                    "train_seconds": t2 - t1, "loss": hist, "out": out})
    if args.eval_workload:
        cnn = Network(default_network_params(args.eval_order))
        rec["evaluation"] = evaluate(cnn, args.eval_workload, args.eval_count, args.eval_order, args.eval_tol,
                                     unet=net)
    print(json.dumps(rec))


if __name__ == "__main__":
    main()
