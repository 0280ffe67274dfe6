"""The persistent sweep engine (use_graph = 2): one cooperative kernel runs the
excess pass and the edge QPs of every sweep, separated by grid barriers.

Per element it performs the same arithmetic as the standalone kernels in the
same order, so with the stop rules off the flows after any number of sweeps
are bit-identical to the CUDA-graph engine's (the launches restart every 1024
sweeps, which the full-size case crosses twice).  The objective is reduced
over a different number of blocks, so z and the stop sweep are compared to
rounding-level tolerances; against the FP64 oracle the stop sweep is equal.
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


def small_instances():
    rng = np.random.default_rng(41)
    return [I.grid5_k10(1.3), I.grid5_k10(1.3).with_factor(0.6),
            I.make_instance("digraph30_k7", I.random_digraph(30, 3, rng), 7, ("uniform_int", 1, 9), 1.1, rng),
            I.make_instance("grid6_k33", I.grid_graph(6), 33, ("lognormal", 1.0, 0.5), 1.2, rng)]


def run(pdr, inst, engine, **opts):
    with pdr.Solver.from_instance(inst, use_graph=engine, **opts) as s:
        r = s.solve()
        return r, s.flows(), (s.trace() if opts.get("trace_len") else None)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_fixed_sweeps_bit_identical_to_graph_engine(pdr, prec):
    p = pdr.PREC_FP32 if prec == "fp32" else pdr.PREC_FP64
    for inst in small_instances():
        for S in (1, 2, 7, 1030):
            opts = dict(precision=p, eps_obj=0.0, resid_tol=0.0, max_sweeps=S)
            r1, f1, _ = run(pdr, inst, 1, **opts)
            r2, f2, _ = run(pdr, inst, 2, **opts)
            assert r1["sweeps"] == r2["sweeps"] == S
            np.testing.assert_array_equal(f1, f2, err_msg=f"{inst.name} S={S}")
            assert abs(r1["z"] - r2["z"]) <= 1e-12 * r1["z"]


def test_fp64_stop_and_trace_match_oracle(pdr):
    for inst in small_instances()[:3]:
        P = oracle.Problem.from_instance(inst)
        f_ref, rep, zt = P.solve_eso(max_sweeps=50000, eps_obj=1e-6, trace=True)
        r, f, tr = run(pdr, inst, 2, precision=pdr.PREC_FP64, eps_obj=1e-6, resid_tol=0.0, trace_len=60000)
        assert r["sweeps"] == rep["sweeps"] and r["stop_name"] == "objective", (inst.name, r, rep)
        np.testing.assert_allclose(tr, zt, rtol=1e-9)
        np.testing.assert_allclose(f, f_ref, rtol=1e-7, atol=1e-9 * inst.d.max())


def test_stop_rules_and_verdicts_agree_with_graph_engine(pdr):
    """The paper's stop (eps_obj = 1e-6) in FP32 and with the FP64 tail, and
    the residual stop that decides the verdict (eps_obj off)."""
    for inst in small_instances():
        for p, eps in ((pdr.PREC_FP32, 1e-6), (pdr.PREC_FP32_FP64TAIL, 1e-6), (pdr.PREC_FP32_FP64TAIL, 0.0)):
            opts = dict(precision=p, eps_obj=eps, resid_tol=1e-6, eps_rel=1e-13, max_sweeps=600000)
            r1, f1, _ = run(pdr, inst, 1, **opts)
            r2, f2, _ = run(pdr, inst, 2, **opts)
            assert r1["verdict"] == r2["verdict"] and r1["stop_reason"] == r2["stop_reason"], (inst.name, r1, r2)
            assert abs(r1["sweeps"] - r2["sweeps"]) <= 2, (inst.name, r1["sweeps"], r2["sweeps"])
            want = inst.feasible_by_construction
            if want is not None and eps == 0.0:
                assert (r2["verdict"] == pdr.VERDICT_FEASIBLE) == want, (inst.name, r2)
                assert r2["verdict"] != pdr.VERDICT_UNKNOWN, (inst.name, r2)


def test_full_size_knn2500_bit_identical_across_launches(pdr, knn2500):
    """The bench workload over 2500 sweeps: three persistent launches (1024,
    1024 and 452 sweeps) against the graph engine."""
    opts = dict(precision=pdr.PREC_FP32, eps_obj=0.0, resid_tol=0.0, max_sweeps=2500)
    r1, f1, _ = run(pdr, knn2500, 1, **opts)
    r2, f2, _ = run(pdr, knn2500, 2, **opts)
    assert r1["sweeps"] == r2["sweeps"] == 2500
    np.testing.assert_array_equal(f1, f2)
    assert abs(r1["z"] - r2["z"]) <= 1e-12 * r1["z"]


def test_engines_that_do_not_apply_fall_back(pdr):
    rng = np.random.default_rng(3)
    inst = I.make_instance("grid11_k3001", I.grid_graph(11), 3001, ("uniform_int", 1, 5), 0.9, rng)
    opts = dict(precision=pdr.PREC_FP32, eps_obj=0.0, resid_tol=0.0, max_sweeps=5)
    r1, f1, _ = run(pdr, inst, 1, **opts)  # block-form variant: no persistent form
    r2, f2, _ = run(pdr, inst, 2, **opts)
    np.testing.assert_array_equal(f1, f2)
    inst = small_instances()[2]
    for algo in (pdr.ALGO_AGD, pdr.ALGO_GDM):  # Alg. 3 / Alg. 4 run in the graph engine
        r1, f1, _ = run(pdr, inst, 1, algo=algo, **opts)
        r2, f2, _ = run(pdr, inst, 2, algo=algo, **opts)
        np.testing.assert_array_equal(f1, f2)


def test_switching_engines_mid_solve(pdr):
    """The objective partials are kept in each engine's own layout: after a
    persistent solve the standalone kernels (objective(), sweeps()) see the
    z of the current flows, and a persistent solve started after sweeps()
    evaluates the z of its starting flows first (trace entry 0)."""
    inst = small_instances()[3]
    P = oracle.Problem.from_instance(inst)

    def z_of(f):
        _, h = P.excess(f)
        return P.objective(h, P.congestion(f))

    with pdr.Solver.from_instance(inst, use_graph=2, precision=pdr.PREC_FP64, eps_obj=0.0, resid_tol=0.0,
                                  max_sweeps=40, trace_len=100) as s:
        s.solve()
        z = z_of(s.flows())
        assert abs(s.objective() - z) <= 1e-12 * z
        s.sweeps(3)
        z = z_of(s.flows())
        assert abs(s.objective() - z) <= 1e-12 * z
        s.solve()
        tr = s.trace()
        assert tr.shape[0] == 41 and abs(tr[0] - z) <= 1e-12 * z
        z = z_of(s.flows())
        assert abs(s.objective() - z) <= 1e-12 * z


def test_option_validation(pdr):
    with pytest.raises(pdr.PdrError):
        pdr.Solver.from_instance(small_instances()[0], use_graph=4)  # engines are 0..3
