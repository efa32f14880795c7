"""Run the preconditioner network forward on a batch of grids, for profiling
(ncu) the convolution kernels in isolation.

Usage: python -m paper_2505_08491_gb300.profile_net --batch 16 --n 33 --passes 4
"""
from __future__ import annotations

import argparse
import os
import sys

import numpy as np
import torch

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

from paper_2505_08491_gb300 import Network  # noqa: E402
from paper_2505_08491_gb300.weights import random_params  # noqa: E402


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--batch", type=int, default=16)
    ap.add_argument("--n", type=int, default=33, help="grid nodes per edge")
    ap.add_argument("--passes", type=int, default=4)
    ap.add_argument("--engine", default="tensor", choices=["tensor", "cuda_cores"])
    args = ap.parse_args()
    net = Network(random_params(1))
    net.set_engine(args.engine)
    n = args.n
    X = torch.from_numpy(np.random.default_rng(0).standard_normal((args.batch, 3, n, n, n)).astype(np.float32)).cuda()
    times = []
    for _ in range(args.passes):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        Y = net.forward(X)
        e1.record()
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    nodes = args.batch * n ** 3
    flop = nodes * 2 * 27 * (3 * 32 + 4 * 32 * 32 + 32)
    best = min(times[1:]) if len(times) > 1 else times[0]
    print("ok", float(Y.abs().mean()), "ms per forward (incl. workspace setup):",
          [round(t, 3) for t in times], "network TFLOP/s (best):", round(flop / best / 1e9, 1))


if __name__ == "__main__":
    main()
