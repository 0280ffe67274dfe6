"""GPU parity for the capacity-kept form (PDR_ALGO_CK, Program (6)) against the
FP64 oracle's capacity-kept step and solve.

Tolerances as in test_gpu_parity: FP32 sweeps 1e-5 of the row scale plus a
1e-36 floor, FP64 1e-12; the FP64 stop sweep equals the oracle's and the z
trace agrees to 1e-9; verdicts are identical.
"""

import numpy as np
import pytest

import oracle
from paper_2108_07549_gb300 import instances as I

pytestmark = pytest.mark.gpu
FP32_FLOOR = 1e-36


@pytest.fixture(scope="module")
def pdr():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2108_07549_gb300 import build, pdr as _pdr

    build.build()
    _pdr.load()
    return _pdr


def small_instances():
    rng = np.random.default_rng(57)
    return [I.grid5_k10(1.3), I.grid5_k10(1.3).with_factor(0.6),
            I.make_instance("digraph30_k7", I.random_digraph(30, 3, rng), 7, ("uniform_int", 1, 9), 0.7, rng),
            I.make_instance("grid6_k33", I.grid_graph(6), 33, ("lognormal", 1.0, 0.5), 0.9, rng)]


def check_sweep(inst, f, got, tol, floor):
    P = oracle.Problem.from_instance(inst)
    _, h = P.excess(f)
    want, g, _ = P.ck_all(h, f)
    sig = (np.abs(f) + np.abs(h[inst.src]) + np.abs(h[inst.col])).max(axis=1)[:, None]
    bad = np.abs(got - want) > tol * np.maximum(np.abs(want), sig) + floor
    assert not bad.any(), (inst.name, np.argwhere(bad)[:5], np.abs(got - want).max())
    assert np.all(got.sum(1) <= inst.u + tol * np.maximum(inst.u, sig[:, 0] * inst.K))


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_one_sweep_matches_oracle_every_variant(pdr, prec):
    rng = np.random.default_rng(8)
    p = pdr.PREC_FP32 if prec == "fp32" else pdr.PREC_FP64
    tol, floor = (1e-5, FP32_FLOOR) if prec == "fp32" else (1e-12, 0.0)
    for inst in small_instances():
        f = rng.exponential(1.0, (inst.m, inst.K)) * (rng.random((inst.m, inst.K)) < 0.4)
        f = f.astype(np.float32).astype(np.float64)
        for v in [v for v, cap, _ in pdr.edge_variants(p) if cap >= inst.K][:6] + [-1]:
            with pdr.Solver.from_instance(inst, precision=p, algo=pdr.ALGO_CK, edge_variant=v) as s:
                s.set_flows(f)
                s.sweeps(1)
                check_sweep(inst, f, s.flows(), tol, floor)


def test_fp64_solve_matches_oracle_stop_and_trace(pdr):
    for inst in small_instances()[:3]:
        P = oracle.Problem.from_instance(inst)
        f_ref, rep, zt = P.solve_ck(max_sweeps=50000, eps_obj=1e-6, trace=True)
        with pdr.Solver.from_instance(inst, precision=pdr.PREC_FP64, algo=pdr.ALGO_CK, eps_obj=1e-6, resid_tol=0.0,
                                      trace_len=60000) as s:
            r = s.solve()
            tr = s.trace()
            f = s.flows()
        assert r["sweeps"] == rep["sweeps"] and r["stop_name"] == "objective", (inst.name, r, rep)
        np.testing.assert_allclose(tr, zt, rtol=1e-9)
        assert np.all(np.diff(tr) <= 1e-12 * tr[:-1])  # projected gradient: z never rises
        np.testing.assert_allclose(f, f_ref, rtol=1e-7, atol=1e-9 * inst.d.max())
        assert r["cap_abs"] <= 1e-12 * inst.u.max()


def test_verdicts_match_construction_and_oracle(pdr):
    for inst in small_instances():
        with pdr.Solver.from_instance(inst, precision=pdr.PREC_FP32_FP64TAIL, algo=pdr.ALGO_CK, eps_obj=0.0,
                                      resid_tol=1e-6, eps_rel=1e-13, max_sweeps=600000) as s:
            r = s.solve()
        want = inst.feasible_by_construction
        assert r["verdict"] != pdr.VERDICT_UNKNOWN, (inst.name, r)
        if want is not None:
            assert (r["verdict"] == pdr.VERDICT_FEASIBLE) == want, (inst.name, r)
        P = oracle.Problem.from_instance(inst)
        f, rep = P.solve_ck(max_sweeps=600000, eps_obj=0.0, resid_tol=1e-6)
        v = P.residuals(f)["verdict"]
        if v == oracle.VERDICT_UNKNOWN:
            f, _ = P.solve_ck(max_sweeps=600000, eps_obj=1e-15, f0=f)
            v = P.residuals(f)["verdict"]
        assert r["verdict"] == v, (inst.name, r, v)


def test_full_size_sweep_parity_knn2500(pdr, knn2500):
    inst = knn2500
    with pdr.Solver.from_instance(inst, precision=pdr.PREC_FP32, algo=pdr.ALGO_CK) as s:
        s.sweeps(60)
        f = s.flows()
        s.sweeps(1)
        got = s.flows()
    P = oracle.Problem.from_instance(inst)
    _, h = P.excess(f)
    want, _, _ = P.ck_all(h, f)
    sig = (np.abs(f) + np.abs(h[inst.src]) + np.abs(h[inst.col])).max(axis=1)[:, None]
    with np.errstate(divide="ignore"):  # all-zero rows: 0 error over a 0 scale
        err = (np.abs(got - want) - FP32_FLOOR) / np.maximum(np.abs(want), sig)
    assert err.max() <= 1e-5, err.max()


def test_engines_and_batch(pdr):
    """The persistent engine gives the graph engine's flows bit for bit; a batch
    reaches the single solves' verdicts; there are no learning rates."""
    inst = small_instances()[3]
    opts = dict(precision=pdr.PREC_FP32, algo=pdr.ALGO_CK, eps_obj=0.0, resid_tol=0.0, max_sweeps=1030)
    flows = []
    for eng in (1, 2):
        with pdr.Solver.from_instance(inst, use_graph=eng, **opts) as s:
            s.solve()
            flows.append(s.flows())
    np.testing.assert_array_equal(flows[0], flows[1])
    insts = small_instances()
    bopts = dict(precision=pdr.PREC_FP32_FP64TAIL, algo=pdr.ALGO_CK, eps_obj=0.0, resid_tol=1e-6, eps_rel=1e-13,
                 max_sweeps=600000)
    with pdr.Batch(insts, **bopts) as B:
        res = B.solve()
    for x, r in zip(insts, res):
        with pdr.Solver.from_instance(x, **bopts) as s:
            assert s.solve()["verdict"] == r["verdict"], x.name
    with pdr.Solver.from_instance(inst, algo=pdr.ALGO_CK) as s:
        with pytest.raises(pdr.PdrError):
            s.gd_state()
