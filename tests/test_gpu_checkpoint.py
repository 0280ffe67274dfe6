"""Checkpoint and resume of a solve (pdr_get_state / pdr_set_state).

A sweep of Alg. 1 depends only on the flows (and the warm starts of its
root searches, which decide near-ties); Alg. 3 adds the learning rates and
the iteration counter, Alg. 4 the velocities.  A checkpoint holds all of
them, so a solve interrupted after N1 sweeps and resumed in a new context
gives the flows of the uninterrupted solve bit for bit, counts its sweeps
the same way, and continues its objective trace (to rounding: the
congestion partials are recomputed from the restored flows).  Cases: the
four algorithms in FP32 and FP64, interruption by pdr_sweeps and by a
stopped solve, the paper's stop rule across a resume, the FP64 tail, the
bench instance, and rejected checkpoints.
"""

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


def small():
    rng = np.random.default_rng(77)
    return [I.make_instance("grid6_k33", I.grid_graph(6), 33, ("lognormal", 1.0, 0.5), 1.2, rng),
            I.make_instance("digraph30_k7", I.random_digraph(30, 3, rng), 7, ("uniform_int", 1, 9), 0.8, rng)]


ALGOS = ["eso", "agd", "gdm", "ck"]


def algo_id(pdr, name):
    return {"eso": pdr.ALGO_ESO, "agd": pdr.ALGO_AGD, "gdm": pdr.ALGO_GDM, "ck": pdr.ALGO_CK}[name]


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("algo", ALGOS)
def test_resume_after_a_stopped_solve(pdr, algo, prec):
    p = pdr.PREC_FP32 if prec == "fp32" else pdr.PREC_FP64
    N1, N2 = 37, 41
    for inst in small():
        opts = dict(precision=p, algo=algo_id(pdr, algo), eps_obj=0.0, resid_tol=0.0, trace_len=200)
        with pdr.Solver.from_instance(inst, max_sweeps=N1 + N2, **opts) as s:
            r_ref = s.solve()
            f_ref, tr_ref = s.flows(), s.trace()
        with pdr.Solver.from_instance(inst, max_sweeps=N1, **opts) as s:
            r1 = s.solve()
            state = s.get_state()
        assert r1["sweeps"] == N1
        with pdr.Solver.from_instance(inst, max_sweeps=N1 + N2, **opts) as s:
            s.set_state(state)
            r = s.solve()
            f, tr = s.flows(), s.trace()
        assert r["sweeps"] == r_ref["sweeps"] == N1 + N2, (inst.name, r, r_ref)
        np.testing.assert_array_equal(f, f_ref, err_msg=inst.name)
        assert tr.shape == tr_ref.shape
        np.testing.assert_allclose(tr, tr_ref, rtol=1e-5 if prec == "fp32" else 1e-12, err_msg=inst.name)


@pytest.mark.parametrize("algo", ALGOS)
def test_resume_after_forced_sweeps(pdr, algo):
    inst = small()[0]
    opts = dict(algo=algo_id(pdr, algo))
    with pdr.Solver.from_instance(inst, **opts) as s:
        s.sweeps(50)
        f_ref = s.flows()
    with pdr.Solver.from_instance(inst, **opts) as s:
        s.sweeps(23)
        state = s.get_state()
    with pdr.Solver.from_instance(inst, **opts) as s:
        s.set_state(state)
        s.sweeps(27)
        np.testing.assert_array_equal(s.flows(), f_ref)


def test_paper_stop_rule_across_a_resume(pdr):
    """FP64, |z^(t) - z^(t-1)| < 1e-6: the resumed solve stops at the
    uninterrupted solve's sweep with its flows."""
    for inst in small():
        opts = dict(precision=pdr.PREC_FP64, eps_obj=1e-6, resid_tol=0.0, max_sweeps=100000)
        with pdr.Solver.from_instance(inst, **opts) as s:
            r_ref = s.solve()
            f_ref = s.flows()
        assert r_ref["stop_name"] == "objective" and r_ref["sweeps"] > 20
        with pdr.Solver.from_instance(inst, **dict(opts, max_sweeps=r_ref["sweeps"] // 2)) as s:
            s.solve()
            state = s.get_state()
        with pdr.Solver.from_instance(inst, **opts) as s:
            s.set_state(state)
            r = s.solve()
            assert r["sweeps"] == r_ref["sweeps"] and r["stop_name"] == "objective", (inst.name, r, r_ref)
            np.testing.assert_array_equal(s.flows(), f_ref)


def test_fp64_tail_checkpoint(pdr):
    """A checkpoint taken in the FP64 tail resumes in FP64 with the same
    split of FP32 and FP64 sweeps."""
    inst = small()[0]
    opts = dict(precision=pdr.PREC_FP32_FP64TAIL, eps_obj=0.0, resid_tol=1e-6, eps_rel=1e-13, max_sweeps=600000)
    with pdr.Solver.from_instance(inst, **opts) as s:
        r_ref = s.solve()
        f_ref = s.flows()
    n32 = r_ref["sweeps"] - r_ref["sweeps_fp64"]
    assert r_ref["sweeps_fp64"] >= 2, r_ref
    with pdr.Solver.from_instance(inst, **dict(opts, max_sweeps=n32 + r_ref["sweeps_fp64"] // 2)) as s:
        r1 = s.solve()
        assert r1["sweeps_fp64"] > 0
        state = s.get_state()
    with pdr.Solver.from_instance(inst, **opts) as s:
        s.set_state(state)
        r = s.solve()
        assert (r["sweeps"], r["sweeps_fp64"]) == (r_ref["sweeps"], r_ref["sweeps_fp64"]), (r, r_ref)
        np.testing.assert_array_equal(s.flows(), f_ref)


def test_full_size_knn2500(pdr, knn2500):
    opts = dict(eps_obj=0.0, resid_tol=0.0)
    with pdr.Solver.from_instance(knn2500, max_sweeps=300, **opts) as s:
        s.solve()
        f_ref = s.flows()
    with pdr.Solver.from_instance(knn2500, max_sweeps=130, **opts) as s:
        s.solve()
        state = s.get_state()
    assert len(state) > 4 * knn2500.m * knn2500.K
    with pdr.Solver.from_instance(knn2500, max_sweeps=300, **opts) as s:
        s.set_state(state)
        assert s.solve()["sweeps"] == 300
        np.testing.assert_array_equal(s.flows(), f_ref)


def test_rejected_checkpoints(pdr):
    a, b = small()
    with pdr.Solver.from_instance(a, max_sweeps=5) as s:
        s.solve()
        state = s.get_state()
        with pytest.raises(pdr.PdrError):
            s.set_state(state[:-8])  # truncated
        with pytest.raises(pdr.PdrError):
            s.set_state(b"XXXX" + state[4:])  # not a checkpoint
    with pdr.Solver.from_instance(b) as s, pytest.raises(pdr.PdrError):
        s.set_state(state)  # other sizes
    with pdr.Solver.from_instance(a, algo=pdr.ALGO_AGD) as s, pytest.raises(pdr.PdrError):
        s.set_state(state)  # other algorithm
    with pdr.Solver.from_instance(a, precision=pdr.PREC_FP64) as s, pytest.raises(pdr.PdrError):
        s.set_state(state)  # FP32 checkpoint in an FP64 context
    # a rejected checkpoint leaves the context usable, and a reset cancels a resume
    with pdr.Solver.from_instance(a, max_sweeps=5) as s:
        s.set_state(state)
        s.reset()
        assert s.solve()["sweeps"] == 5
