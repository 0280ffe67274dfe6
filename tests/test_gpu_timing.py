"""The measurement entry points: pdr_time_sweeps runs the sweeps of
pdr_sweeps (same flows afterwards, bit for bit) and reports positive mean
kernel durations; pdr_time_kernel leaves the current flows and the next
sweep's warm starts as they were."""

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


@pytest.mark.parametrize("algo", ["eso", "gdm"])
def test_time_sweeps_runs_the_same_sweeps(pdr, algo):
    rng = np.random.default_rng(77)
    inst = I.make_instance("grid6_k33", I.grid_graph(6), 33, ("lognormal", 1.0, 0.5), 1.2, rng)
    a = pdr.ALGO_ESO if algo == "eso" else pdr.ALGO_GDM
    with pdr.Solver.from_instance(inst, algo=a) as s:
        s.sweeps(300)
        want = s.flows()
    with pdr.Solver.from_instance(inst, algo=a) as s:
        tx, tu = s.time_sweeps(300)
        assert tx > 0 and tu > 0
        np.testing.assert_array_equal(s.flows(), want)
        # timing the kernels alone changes neither the flows nor the next sweep
        s.time_kernel("qp", 5, 0)
        s.time_kernel("excess", 5, 1 << 20)
        np.testing.assert_array_equal(s.flows(), want)
        s.sweeps(7)
        got = s.flows()
    with pdr.Solver.from_instance(inst, algo=a) as s:
        s.sweeps(300)
        s.sweeps(7)
        np.testing.assert_array_equal(got, s.flows())
