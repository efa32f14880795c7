"""Parity of the operator apply, load vector and distance field (CUDA path
through the C ABI) against the FP64 oracle."""
import numpy as np
import pytest
import torch

from helpers import instance_cases, rel_l2
from oracle import fem

pytestmark = pytest.mark.gpu

CASES = instance_cases()


@pytest.fixture(scope="module", params=CASES, ids=[c[0] for c in CASES])
def pair(request):
    from paper_2505_08491_gb300 import Operator
    name, N, g, beta, fseed = request.param
    return fem.Problem(N, g, beta), Operator(N, g, beta), fseed


def test_sizes_match(pair):
    p, op, _ = pair
    assert (op.n3, op.n1, op.nq, op.n) == (p.n3, p.n1, p.nq, p.n)
    assert op.alpha == pytest.approx(p.alpha, rel=1e-12)
    assert op.n_touch == len(np.unique(p.Pi.indices))


def test_apply_fp64(pair):
    p, op, _ = pair
    rng = np.random.default_rng(0)
    for _ in range(2):
        u = rng.standard_normal(p.n)
        y = op.apply(torch.from_numpy(u).cuda()).cpu().numpy()
        ref = p.A @ u
        assert rel_l2(y, ref) <= 1e-12
        assert np.max(np.abs(y - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_apply_fp32(pair):
    p, op, _ = pair
    u = np.random.default_rng(1).standard_normal(p.n).astype(np.float32)
    y = op.apply(torch.from_numpy(u).cuda()).cpu().numpy()
    ref = p.A @ u.astype(np.float64)
    assert rel_l2(y, ref) <= 1e-5


def test_apply_structured_inputs(pair):
    """Constant fields (coupling null) and a unit vector on a touched node."""
    p, op, _ = pair
    u = np.ones(p.n)
    y = op.apply(torch.from_numpy(u).cuda()).cpu().numpy()
    assert rel_l2(y, p.A @ u) <= 1e-12
    e = np.zeros(p.n)
    e[p.Pi.indices[0]] = 1.0
    y = op.apply(torch.from_numpy(e).cuda()).cpu().numpy()
    assert np.max(np.abs(y - p.A @ e)) <= 1e-13 * max(1.0, np.max(np.abs(p.A @ e)))


def test_rhs(pair):
    p, op, fseed = pair
    f = p.source(fseed)
    ft = torch.from_numpy(f).cuda() if f is not None else None
    b = op.rhs(ft, 1.0).cpu().numpy()
    ref = p.rhs(f, 1.0)
    assert rel_l2(b, ref) <= 1e-13


def test_distance(pair):
    p, op, _ = pair
    d = op.distance().cpu().numpy()
    assert np.max(np.abs(d - p.dist)) <= 1e-7 * max(1.0, p.dist.max())


def test_jacobi_precondition_is_diag_inverse(pair):
    p, op, _ = pair
    r = np.random.default_rng(2).standard_normal(p.n).astype(np.float32)
    z = op.precondition(torch.from_numpy(r).cuda()).cpu().numpy()
    assert rel_l2(z, r / p.diag) <= 1e-6
