"""md_apply_noalloc, the allocation-free variant of the operator apply for
callers that cannot allocate device memory (its scratch is a static device
array of the library).  It must give what md_apply gives, call after call:
two calls in a row on different operators check that the shared scratch
left by the first call does not leak into the second.  Runs last (file
name) so that a failure here comes after every other test."""
import numpy as np
import pytest
import torch

from helpers import instance_cases, rel_l2

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-12), (torch.float32, 1e-5)])
def test_noalloc_apply_matches_apply_twice(dtype, tol):
    from paper_2505_08491_gb300 import Operator
    cases = instance_cases()
    ops = [Operator(N, g, beta) for _, N, g, beta, _ in (cases[1], cases[2])]
    rng = np.random.default_rng(5)
    for op in ops:  # two calls in a row, different operators
        u = torch.from_numpy(rng.standard_normal(op.n)).to(dtype).cuda()
        ref = op.apply(u)
        out = torch.empty_like(u)
        op.apply_noalloc(u, out)
        torch.cuda.synchronize()
        assert rel_l2(out.cpu().numpy(), ref.cpu().numpy()) <= tol
    # and the same operator again, after the other one used the scratch
    u = torch.from_numpy(rng.standard_normal(ops[0].n)).to(dtype).cuda()
    out = torch.empty_like(u)
    ops[0].apply_noalloc(u, out)
    torch.cuda.synchronize()
    assert rel_l2(out.cpu().numpy(), ops[0].apply(u).cpu().numpy()) <= tol


def test_noalloc_rejects_oversized_operator():
    """An operator with more quadrature points than the static scratch holds
    is refused before any device work."""
    import mdgen
    from paper_2505_08491_gb300 import Operator
    from paper_2505_08491_gb300._lib import MdError
    g = mdgen.random_tree(3, 0, depth=5, elems=300)  # 31 segments x 300 elements x 2 points > 16384
    op = Operator(16, g, 1.0)
    assert op.nq > 16384
    u = torch.zeros(op.n, dtype=torch.float64, device="cuda")
    with pytest.raises(MdError, match="MD_ERR_ARG"):
        op.apply_noalloc(u, torch.empty_like(u))
