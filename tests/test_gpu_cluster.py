"""The cluster engine (pdr_options.use_graph = 3): one thread-block cluster
runs a small instance's whole solve (the batched form's engine, with one
instance).  Its sweeps, objective and flows equal the CUDA-graph engine's
bit for bit, across launches of 2048 sweeps and in every precision mode
(FP64 sweeps run on the graph engine, here and in the batched form); an
instance it does not take runs on the graph engine.  Small instances run the
kernel's shared-memory form, larger single-block ones its global-memory
form (dg60_k40 in FP32 is the former, dg80_k200 the latter)."""

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


def solve(pdr, inst, engine, **opts):
    with pdr.Solver.from_instance(inst, use_graph=engine, **opts) as s:
        r = s.solve()
        return r, s.flows()


@pytest.mark.parametrize("prec", ["fp32", "fp64", "tail"])
@pytest.mark.parametrize("algo", ["eso", "ck"])
def test_cluster_engine_equals_graph_engine(pdr, prec, algo):
    p = {"fp32": pdr.PREC_FP32, "fp64": pdr.PREC_FP64, "tail": pdr.PREC_FP32_FP64TAIL}[prec]
    a = pdr.ALGO_ESO if algo == "eso" else pdr.ALGO_CK
    rng = np.random.default_rng(5)
    insts = [I.grid5_k10(1.3), I.grid5_k10(0.6),
             I.make_instance("dg60_k40", I.random_digraph(60, 3, rng), 40, ("uniform_int", 1, 9), 1.0, rng),
             I.make_instance("dg80_k200", I.random_digraph(80, 3, rng), 200, ("uniform_int", 1, 9), 1.0, rng)]
    for inst in insts:
        opts = dict(precision=p, algo=a, eps_obj=0.0, resid_tol=1e-6, max_sweeps=5000)
        r1, f1 = solve(pdr, inst, 1, **opts)
        r3, f3 = solve(pdr, inst, 3, **opts)
        assert r3["sweeps"] == r1["sweeps"] and r3["sweeps_fp64"] == r1["sweeps_fp64"], inst.name
        assert r3["stop_reason"] == r1["stop_reason"] and r3["verdict"] == r1["verdict"], inst.name
        assert r3["z"] == r1["z"], inst.name
        np.testing.assert_array_equal(f3, f1, err_msg=inst.name)


def test_cluster_engine_runs_several_launches_and_resumes(pdr):
    """A solve longer than one launch (2048 sweeps), then a second solve call
    that continues from the returned flows: both as the graph engine's."""
    inst = I.grid5_k10(1.3)
    opts = dict(precision=pdr.PREC_FP32, eps_obj=0.0, resid_tol=0.0, max_sweeps=4500)
    out = {}
    for engine in (1, 3):
        with pdr.Solver.from_instance(inst, use_graph=engine, **opts) as s:
            r = s.solve()
            f = s.flows()
            r2 = s.solve()
            out[engine] = (r, f, r2, s.flows())
    (ra, fa, ra2, fa2), (rb, fb, rb2, fb2) = out[1], out[3]
    assert ra["sweeps"] == rb["sweeps"] == 4500 and ra["z"] == rb["z"]
    np.testing.assert_array_equal(fa, fb)
    assert ra2["sweeps"] == rb2["sweeps"] and ra2["z"] == rb2["z"]
    np.testing.assert_array_equal(fa2, fb2)


def test_instance_too_large_for_a_cluster_runs_on_the_graph(pdr):
    """knn2500_k500 (m x K = 7.5e6 > 2^18): use_graph = 3 falls back to the
    graph engine, with its results."""
    inst = I.knn2500_k500()
    opts = dict(precision=pdr.PREC_FP32, eps_obj=0.0, resid_tol=0.0, max_sweeps=40)
    r1, f1 = solve(pdr, inst, 1, **opts)
    r3, f3 = solve(pdr, inst, 3, **opts)
    assert r1["sweeps"] == r3["sweeps"] == 40 and r1["z"] == r3["z"]
    np.testing.assert_array_equal(f1, f3)


def test_use_graph_out_of_range_is_rejected(pdr):
    with pytest.raises(pdr.PdrError):
        pdr.Solver.from_instance(I.grid5_k10(1.3), use_graph=4)
