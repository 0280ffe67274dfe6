"""The batched form at full size: batch256 (256 random out-degree-4 digraphs, n
in [100, 5000], K in [10, 1000], one fifth at 0.7x capacity) in the launch
configuration `bench.py --workload batch256` times.

After 100 sweeps of every instance in one graph launch, sampled instances
are checked three ways: the batch's flows equal, bit for bit, a
single-instance solve that runs the edge-kernel variant the batch's
autotuner chose for that instance (the same kernels with the same
arguments); the single-instance form's next sweep from those flows matches
the FP64 oracle's to the FP32 tolerance of test_gpu_parity; and every
instance ran exactly the requested sweeps.
"""

import os

import numpy as np
import pytest

import oracle
from paper_2108_07549_gb300 import instances as I

pytestmark = [pytest.mark.gpu, pytest.mark.slow]
FP32_FLOOR = 1e-36


@pytest.fixture(scope="module")
def batch256():
    # a spawn pool: safe whatever CUDA state this process already has
    return I.batch256(seed=0, processes=min(16, os.cpu_count() or 1))


@pytest.fixture(scope="module")
def pdr():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2108_07549_gb300 import build, pdr as _pdr

    build.build()
    _pdr.load()
    return _pdr


def test_full_batch_matches_single_solves_and_oracle(pdr, batch256):
    insts = batch256
    S = 100
    opts = dict(precision=pdr.PREC_FP32, eps_obj=0.0, resid_tol=0.0, max_sweeps=S)
    work = np.array([x.m * x.K for x in insts])
    rng = np.random.default_rng(6)
    sample = sorted({int(work.argmax()), int(work.argmin()), *rng.choice(len(insts), 3, replace=False).tolist()})
    with pdr.Batch(insts, **opts) as B:
        res = B.solve()
        cfg, _ = B.tuning()
        flows = {i: B.solver(i).flows() for i in sample}
    assert all(r["sweeps"] == S for r in res)
    for i in sample:
        x = insts[i]
        with pdr.Solver.from_instance(x, edge_variant=int(cfg[i]), **opts) as s:
            s.solve()
            np.testing.assert_array_equal(s.flows(), flows[i], err_msg=f"instance {i}")
            # one more sweep from the batch's flows against the oracle
            if x.m * x.K <= 5_000_000:
                s.set_flows(flows[i])
                s.sweeps(1)
                got = s.flows()
                P = oracle.Problem.from_instance(x)
                f = flows[i]
                _, h = P.excess(f)
                want, _, _ = P.qp_all(h, f)
                sig = (np.abs(f) + np.abs(h[x.src]) + np.abs(h[x.col])).max(axis=1)[:, None]
                bad = np.abs(got - want) > 1e-5 * np.maximum(np.abs(want), sig) + FP32_FLOOR
                assert not bad.any(), (i, np.argwhere(bad)[:5])
