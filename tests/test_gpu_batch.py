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


def small_batch(seed=31, count=40):
    """Instances small enough for the one-block-per-instance engine (m * K_p <= 2^18):
    random out-degree-3 digraphs, n in [20, 300), K in [1, 120), every fifth at 0.6x capacity."""
    rng = np.random.default_rng(seed)
    out = []
    for b in range(count):
        n = int(rng.integers(20, 300))
        K = int(rng.integers(1, 120))
        g = I.random_digraph(n, 3, np.random.default_rng([seed, b]))
        factor = 0.6 if b % 5 == 4 else 1.2
        out.append(I.make_instance(f"s{b}", g, K, ("uniform_int", 1, 10), factor, np.random.default_rng([seed, b, 1])))
    return out


@pytest.mark.parametrize("prec", [0, 1])
def test_block_engine_equals_single_solves_bit_for_bit(pdr, prec):
    """The one-block-per-instance engine runs, per element, the standalone
    kernels' arithmetic in their order: after a fixed number of sweeps every
    instance's flows equal, bit for bit, a single-instance solve with the
    variant the batch chose; the next sweep from them matches the oracle."""
    insts = small_batch()
    S = 137  # odd, and more than one launch's worth is not needed to cover the parity swap
    opts = dict(precision=prec, eps_obj=0.0, resid_tol=0.0, max_sweeps=S)
    with pdr.Batch(insts, **opts) as B:
        res = B.solve()
        cfg, _ = B.tuning()
        flows = [B.solver(i).flows() for i in range(len(insts))]
    assert all(r["sweeps"] == S and r["stop_name"] == "max_sweeps" for r in res)
    for i, x in enumerate(insts):
        with pdr.Solver.from_instance(x, edge_variant=int(cfg[i]), **opts) as s:
            r1 = s.solve()
            np.testing.assert_array_equal(s.flows(), flows[i], err_msg=x.name)
        assert abs(r1["z"] - res[i]["z"]) <= 1e-12 * max(1.0, r1["z"])
    x, f = insts[3], flows[3]
    P = oracle.Problem.from_instance(x)
    _, h = P.excess(f)
    want, _, _ = P.qp_all(h, f)
    with pdr.Solver.from_instance(x, precision=prec) as s:
        s.set_flows(f)
        s.sweeps(1)
        got = s.flows()
    sig = (np.abs(f) + np.abs(h[x.src]) + np.abs(h[x.col])).max(axis=1)[:, None]
    tol = 1e-5 if prec == 0 else 1e-12
    assert np.all(np.abs(got - want) <= tol * np.maximum(np.abs(want), sig) + 1e-36)


def test_block_engine_verdicts_and_long_solves(pdr):
    """Solves longer than one launch of the engine (2048 sweeps), stopped per
    instance by their own rules, in the tail mode: verdicts as constructed and
    as the graph-free host loop finds them, residuals <= 1e-6 per the oracle."""
    insts = small_batch(seed=37, count=24)
    opts = dict(precision=pdr.PREC_FP32_FP64TAIL, eps_obj=0.0, resid_tol=1e-6, eps_rel=1e-13, max_sweeps=300000)
    with pdr.Batch(insts, **opts) as B:
        res = B.solve()
        flows = [B.solver(i).flows() for i in range(len(insts))]
    with pdr.Batch(insts, use_graph=0, **opts) as B0:
        res0 = B0.solve()
    assert max(r["sweeps"] for r in res) > 2048
    for x, r, r0, f in zip(insts, res, res0, flows):
        want = x.feasible_by_construction
        assert r["verdict"] == (pdr.VERDICT_FEASIBLE if want else pdr.VERDICT_INFEASIBLE), (x.name, r)
        assert r["verdict"] == r0["verdict"], (x.name, r, r0)
        if r["verdict"] == pdr.VERDICT_FEASIBLE:
            ref = oracle.Problem.from_instance(x).residuals(f)
            assert ref["cap_rel"] <= 1e-6 and ref["cons_rel"] <= 1e-6
