"""Time limits of the device-side waits.

The bulk-copy excess form waits on shared-memory barriers, each wait with a
time limit.  pdr_debug_wait shortens the limit to about a millisecond and
makes the producer withhold the end marker of its ring, a barrier phase that
nothing else completes.  Every block's consumers then wait out the limit
with no copy in flight, set the device fault flag and leave.  The call
returns PDR_ERR_TIMEOUT, and the same context then sweeps correctly again.

The persistent engine's grid barrier bounds each wait by elapsed time on the
GPU's global timer.  pdr_debug_barrier shortens that limit to a millisecond
and makes block 0 leave the kernel at its first barrier without arriving
(it has no copy in flight); the other blocks wait out the limit, raise the
barrier's failure flag and leave, and the solve returns PDR_ERR_TIMEOUT.
Nothing faults, traps or hangs the GPU.
"""

import time

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


def instance():
    rng = np.random.default_rng(77)
    return I.make_instance("grid6_k33", I.grid_graph(6), 33, ("lognormal", 1.0, 0.5), 1.2, rng)


@pytest.mark.parametrize("form", [1, 2, 3, 4, 5])
def test_wait_runs_out_and_the_context_recovers(pdr, form):
    inst = instance()
    rng = np.random.default_rng(2)
    f = rng.exponential(1.0, (inst.m, inst.K)) * (rng.random((inst.m, inst.K)) < 0.4)
    with pdr.Solver.from_instance(inst, excess_variant=form) as s:
        s.set_flows(f)
        s.sweeps(3)
        want = s.flows()
    with pdr.Solver.from_instance(inst, excess_variant=form, max_sweeps=100) as s:
        s.debug_wait(2_000_000, hold_end=True)
        s.set_flows(f)
        with pytest.raises(pdr.PdrError) as e:
            s.sweeps(1)
        assert e.value.status == pdr.ERR_TIMEOUT
        for eng in (0, 1):  # host loop and graph: the solve stops at the first sweep
            s.set_options(use_graph=eng)
            with pytest.raises(pdr.PdrError) as e:
                s.solve()
            assert e.value.status == pdr.ERR_TIMEOUT
        s.debug_wait(1 << 32, hold_end=False)
        s.set_flows(f)
        s.sweeps(3)
        np.testing.assert_array_equal(s.flows(), want)


def test_hook_rejects_bad_arguments(pdr):
    with pdr.Solver.from_instance(instance()) as s:
        for cycles, hold in ((999, 0), ((1 << 32) + 1, 0), (10_000, 2)):
            with pytest.raises(pdr.PdrError) as e:
                s._check(s._lib.pdr_debug_wait(s._h, cycles, hold))
            assert e.value.status == pdr.ERR_INVALID_ARG


def test_persistent_barrier_runs_out_and_the_context_recovers(pdr):
    inst = instance()
    opts = dict(use_graph=2, precision=pdr.PREC_FP32, eps_obj=0.0, resid_tol=0.0, max_sweeps=5)
    with pdr.Solver.from_instance(inst, **opts) as s:
        assert s.solve()["sweeps"] == 5
        want = s.flows()
    with pdr.Solver.from_instance(inst, **opts) as s:
        s.debug_barrier(1_000_000, withhold=True)
        for _ in range(2):  # the same context times out again: the barrier is cleared per launch
            t0 = time.perf_counter()
            with pytest.raises(pdr.PdrError) as e:
                s.solve()
            assert e.value.status == pdr.ERR_TIMEOUT
            assert time.perf_counter() - t0 < 1.5  # the 1 ms limit, not the 2 s default
            s.reset()
        s.debug_barrier(2_000_000_000, withhold=False)
        r = s.solve()
        assert r["sweeps"] == 5
        np.testing.assert_array_equal(s.flows(), want)


def test_barrier_hook_rejects_bad_arguments(pdr):
    with pdr.Solver.from_instance(instance()) as s:
        for ns, hold in ((99_999, 0), (2_000_000_001, 0), (1_000_000, 2)):
            with pytest.raises(pdr.PdrError) as e:
                s._check(s._lib.pdr_debug_barrier(s._h, ns, hold))
            assert e.value.status == pdr.ERR_INVALID_ARG
