"""The batched form: many uneven instances in one graph launch per solve.

Every instance of a batch runs the same kernels as a single-instance solve
(only the edge-kernel variant may differ: the batch's autotuner picks it by
timing), stops by its own rules, and must reach the verdict its capacity
recipe fixes.  Results are compared with single-instance solves of the same
instances; variants differ in summation order, so floating-point results are
compared to tolerances, integers and verdicts exactly.
"""

import numpy as np
import pytest

import oracle
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


def uneven_batch(seed=5, count=10):
    """Random out-degree-3 digraphs, n in [20, 120), K in [1, 40); every fourth at 0.6x capacity."""
    rng = np.random.default_rng(seed)
    out = []
    for b in range(count):
        n = int(rng.integers(20, 120))
        K = int(rng.integers(1, 40))
        g = I.random_digraph(n, 3, np.random.default_rng([seed, b]))
        factor = 0.6 if b % 4 == 3 else 1.2
        out.append(I.make_instance(f"b{b}", g, K, ("uniform_int", 1, 10), factor, np.random.default_rng([seed, b, 1])))
    return out


OPTS = dict(precision=1, eps_obj=0.0, resid_tol=1e-6, eps_rel=1e-13, max_sweeps=400000)


def test_batch_verdicts_and_single_solves_agree(pdr):
    insts = uneven_batch()
    with pdr.Batch(insts, **OPTS) as B:
        res = B.solve()
        flows = [B.solver(i).flows() for i in range(len(insts))]
    for inst, r, f in zip(insts, res, flows):
        want = inst.feasible_by_construction
        if want is not None:
            assert r["verdict"] == (pdr.VERDICT_FEASIBLE if want else pdr.VERDICT_INFEASIBLE), (inst.name, r)
        with pdr.Solver.from_instance(inst, **OPTS) as s:
            r1 = s.solve()
        assert r["verdict"] == r1["verdict"], (inst.name, r, r1)
        assert abs(r["sweeps"] - r1["sweeps"]) <= max(2, 0.01 * r1["sweeps"]), (inst.name, r["sweeps"], r1["sweeps"])
        # the batch's flows satisfy eq. (1) per the oracle when feasible
        if r["verdict"] == pdr.VERDICT_FEASIBLE:
            ref = oracle.Problem.from_instance(inst).residuals(f)
            assert ref["cap_rel"] <= 1e-6 and ref["cons_rel"] <= 1e-6


def test_batch_fixed_sweeps_match_single(pdr):
    insts = uneven_batch(seed=9, count=6)
    opts = dict(precision=0, eps_obj=0.0, resid_tol=0.0, max_sweeps=150)
    with pdr.Batch(insts, **opts) as B:
        res = B.solve()
        flows = [B.solver(i).flows() for i in range(len(insts))]
        cfg, us = B.tuning()
    for inst, r, f in zip(insts, res, flows):
        assert r["sweeps"] == 150 and r["stop_name"] == "max_sweeps"
        with pdr.Solver.from_instance(inst, **opts) as s:
            s.solve()
            f1 = s.flows()
        scale = max(1.0, np.abs(f1).max())
        assert np.abs(f - f1).max() <= 1e-4 * scale, inst.name
    assert np.all(cfg >= 0)


def test_batch_reset_and_resolve_is_deterministic(pdr):
    insts = uneven_batch(seed=13, count=5)
    with pdr.Batch(insts, precision=0, eps_obj=1e-6, max_sweeps=20000) as B:
        a = B.solve()
        fa = [B.solver(i).flows() for i in range(len(insts))]
        B.reset()
        b = B.solve()
        fb = [B.solver(i).flows() for i in range(len(insts))]
    for x, y in zip(a, b):
        assert x["sweeps"] == y["sweeps"] and x["z"] == y["z"]
    for x, y in zip(fa, fb):
        np.testing.assert_array_equal(x, y)


def test_batch_host_loop_matches_graph(pdr):
    insts = uneven_batch(seed=17, count=4)
    out = []
    for g in (1, 0):
        with pdr.Batch(insts, precision=1, eps_obj=1e-7, max_sweeps=50000, use_graph=g) as B:
            out.append(B.solve())
    for x, y in zip(*out):
        assert x["verdict"] == y["verdict"] and abs(x["sweeps"] - y["sweeps"]) <= 2


def test_batch_fp64_tail_matches_single_solves(pdr):
    """PDR_PREC_FP32_FP64TAIL in the batch: FP32 sweeps for every instance,
    then FP64 sweeps for the instances whose FP32 phase stopped on the
    objective rules, each from its own FP32 flows, exactly as pdr_solve."""
    insts = uneven_batch(seed=23, count=8)
    opts = dict(precision=pdr.PREC_FP32_FP64TAIL, eps_obj=0.0, resid_tol=1e-6, eps_rel=1e-13, max_sweeps=600000)
    with pdr.Batch(insts, **opts) as B:
        res = B.solve()
        flows = [B.solver(i).flows() for i in range(len(insts))]
        again = B.solve()  # resumes: FP64 instances stay in FP64
    for inst, r, f, r2 in zip(insts, res, flows, again):
        want = inst.feasible_by_construction
        if want is not None:
            assert r["verdict"] == (pdr.VERDICT_FEASIBLE if want else pdr.VERDICT_INFEASIBLE), (inst.name, r)
        with pdr.Solver.from_instance(inst, **opts) as s:
            r1 = s.solve()
        assert r["verdict"] == r1["verdict"], (inst.name, r, r1)
        assert (r["sweeps_fp64"] > 0) == (r1["sweeps_fp64"] > 0), (inst.name, r, r1)
        if r["verdict"] == pdr.VERDICT_FEASIBLE:
            ref = oracle.Problem.from_instance(inst).residuals(f)
            assert ref["cap_rel"] <= 1e-6 and ref["cons_rel"] <= 1e-6
        assert r2["verdict"] == r["verdict"]
