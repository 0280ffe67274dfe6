"""Host-side failure injection: every device allocation that pdr_create and
pdr_batch_create make can fail (pdr_debug_fail_alloc), and each such call
returns PDR_ERR_OOM, releases what it had allocated and leaves the library
usable: a solve afterwards gives the same result as one that never saw a
failure.  Nothing fails on the GPU itself."""

import numpy as np
import pytest

from paper_2108_07549_gb300 import instances as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pdr():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2108_07549_gb300 import build, pdr as _pdr

    build.build()
    _pdr.load()
    return _pdr


def test_every_create_allocation_can_fail(pdr):
    lib = pdr.load()
    inst = I.grid5_k10(1.3)
    opts = dict(eps_obj=0.0, resid_tol=0.0, max_sweeps=200)
    with pdr.Solver.from_instance(inst, **opts) as s:
        want = s.solve()
        f_want = s.flows()
    failed = 0
    for nth in range(1, 500):
        lib.pdr_debug_fail_alloc(nth)
        try:
            with pdr.Solver.from_instance(inst, **opts):
                pass
        except pdr.PdrError as e:
            assert e.status == pdr.ERR_OOM and "injected" in str(e), (nth, e)
            failed += 1
            continue
        finally:
            lib.pdr_debug_fail_alloc(0)
        break
    assert failed >= 20, failed  # pdr_create makes dozens of device allocations
    with pdr.Solver.from_instance(inst, **opts) as s:
        r = s.solve()
        assert r["sweeps"] == want["sweeps"]
        np.testing.assert_array_equal(s.flows(), f_want)


def test_batch_create_allocation_failure(pdr):
    lib = pdr.load()
    insts = [I.grid5_k10(1.3), I.grid5_k10(0.6)]
    opts = dict(precision=pdr.PREC_FP32_FP64TAIL, eps_obj=0.0, resid_tol=1e-6, eps_rel=1e-13, max_sweeps=100000)
    for nth in (1, 7, 40):  # in the first context, deep in it, in the second
        lib.pdr_debug_fail_alloc(nth)
        try:
            with pytest.raises(pdr.PdrError) as e:
                pdr.Batch(insts, **opts)
            assert e.value.status == pdr.ERR_OOM
        finally:
            lib.pdr_debug_fail_alloc(0)
    with pdr.Batch(insts, **opts) as B:
        res = B.solve()
    for x, r in zip(insts, res):
        with pdr.Solver.from_instance(x, **opts) as s:
            assert s.solve()["verdict"] == r["verdict"] != pdr.VERDICT_UNKNOWN
