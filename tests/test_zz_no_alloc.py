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


def test_noalloc_allocates_nothing_and_runs_on_a_side_stream():
    """After the first call (the set-up), a burst of calls on a non-default
    stream, alternating FP32 and FP64 on the shared scratch, leaves the
    device's free memory unchanged and gives md_apply's results."""
    from paper_2505_08491_gb300 import Operator
    cases = instance_cases()
    op = Operator(*[cases[1][k] for k in (1, 2, 3)])
    rng = np.random.default_rng(9)
    u64 = torch.from_numpy(rng.standard_normal(op.n)).cuda()
    u32 = u64.float()
    ref64, ref32 = op.apply(u64), op.apply(u32)
    o64, o32 = torch.empty_like(u64), torch.empty_like(u32)
    side = torch.cuda.Stream()
    op.apply_noalloc(u64, o64)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    with torch.cuda.stream(side):
        for _ in range(10):
            op.apply_noalloc(u64, o64)
            op.apply_noalloc(u32, o32)
    side.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert rel_l2(o64.cpu().numpy(), ref64.cpu().numpy()) <= 1e-12
    assert rel_l2(o32.cpu().numpy(), ref32.cpu().numpy()) <= 1e-5
