"""pdr_adjacency_static: the entry point for callers that cannot allocate.

A caller whose device memory belongs to another allocator (a framework's
caching pool, or a service that reserves everything at start-up) cannot call
cudaMalloc and so cannot create a solver context.  pdr_adjacency_static takes
that caller's device arrays and works in a fixed scratch area compiled into
the library.  These checks call it through the C ABI and compare its output
with the context path's (pdr_create + pdr_adjacency): integer results, so
bit-exact, on two calls in a row (the scratch keeps the previous call's
contents, which must not leak into the next).  This file is collected last.
"""

import numpy as np
import pytest

from paper_2108_07549_gb300 import instances as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2108_07549_gb300 import build, pdr

    build.build()
    pdr.load()
    return torch, pdr


def _run_static(torch, pdr, inst):
    row_ptr = torch.from_numpy(inst.row_ptr.astype(np.int64)).cuda()
    col = torch.from_numpy(inst.col.astype(np.int32)).cuda()
    in_ptr = torch.full((inst.n + 1,), -7, dtype=torch.int64, device="cuda")
    in_eid = torch.full((max(inst.m, 1),), -7, dtype=torch.int32, device="cuda")
    deg = torch.full((inst.n,), -7, dtype=torch.int32, device="cuda")
    pdr.adjacency_static(inst.n, inst.m, row_ptr.data_ptr(), col.data_ptr(), in_ptr.data_ptr(), in_eid.data_ptr(),
                         deg.data_ptr(), stream=torch.cuda.current_stream().cuda_stream)
    return in_ptr.cpu().numpy(), in_eid.cpu().numpy()[: inst.m], deg.cpu().numpy()


def test_static_adjacency_matches_context_path_twice(dev):
    torch, pdr = dev
    rng = np.random.default_rng(11)
    big = I.knn2500_k500(1.2)
    small = I.make_instance("digraph40", I.random_digraph(40, 3, rng), 4, ("uniform_int", 1, 5), 1.1, rng)
    # the large graph first, then a smaller one: stale counts from the first
    # call would corrupt the second if the scratch were not cleared
    for inst in (big, small):
        got = _run_static(torch, pdr, inst)
        with pdr.Solver.from_instance(inst) as s:
            want = s.adjacency()
        for g, w in zip(got, want):
            np.testing.assert_array_equal(g, w)


def test_static_adjacency_rejects_oversize_and_malformed(dev):
    torch, pdr = dev
    with pytest.raises(pdr.PdrError, match="262144"):
        pdr.adjacency_static(1 << 19, 0, 16, 16, 16, 16, 16)
    row_ptr = torch.tensor([0, 1, 2], dtype=torch.int64, device="cuda")
    col = torch.tensor([1, 5], dtype=torch.int32, device="cuda")  # 5 is out of range
    out = torch.zeros(8, dtype=torch.int64, device="cuda")
    with pytest.raises(pdr.PdrError, match="malformed"):
        pdr.adjacency_static(2, 2, row_ptr.data_ptr(), col.data_ptr(), out.data_ptr(), out.data_ptr(),
                             out.data_ptr())
