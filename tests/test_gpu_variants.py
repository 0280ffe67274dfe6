"""Every edge-kernel variant (pdr_options.edge_variant) computes the same
sweep: lane groups of 4..32 lanes, one block per edge, and the persistent
pipelined warp form.  Each is compared with the FP64 oracle on one sweep from
the same state (tolerances as in test_gpu_parity: FP32 1e-5 of the row scale
plus a 1e-36 floor, FP64 1e-12), in the decision block's objective, and over
a whole graph-loop solve (same stop sweep and verdict as the default variant).
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


def instances():
    rng = np.random.default_rng(91)
    return [I.make_instance("grid6_k33", I.grid_graph(6), 33, ("lognormal", 1.0, 0.5), 1.2, rng),
            I.make_instance("digraph60_k5", I.random_digraph(60, 3, rng), 5, ("uniform_int", 1, 9), 0.8, rng),
            I.make_instance("grid5_k130", I.grid_graph(5), 130, ("uniform_int", 1, 6), 1.0, rng)]


def fitting(pdr, K, prec):
    return [v for v, cap, _ in pdr.edge_variants(prec) if cap >= K]


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_every_variant_one_sweep_matches_oracle(pdr, prec):
    rng = np.random.default_rng(3)
    p = pdr.PREC_FP32 if prec == "fp32" else pdr.PREC_FP64
    tol, floor = (1e-5, FP32_FLOOR) if prec == "fp32" else (1e-12, 0.0)
    for inst in instances():
        P = oracle.Problem.from_instance(inst)
        f = rng.exponential(1.0, (inst.m, inst.K)) * (rng.random((inst.m, inst.K)) < 0.4)
        f = f.astype(np.float32).astype(np.float64)
        _, h = P.excess(f)
        want, _, _ = P.qp_all(h, f)
        sig = (np.abs(f) + np.abs(h[inst.src]) + np.abs(h[inst.col])).max(axis=1)[:, None]
        vs = fitting(pdr, inst.K, p)
        assert any(pipe for v, _, pipe in pdr.edge_variants(p) if v in vs) or inst.K > 512
        for v in vs:
            with pdr.Solver.from_instance(inst, precision=p, edge_variant=v) as s:
                s.set_flows(f)
                s.sweeps(1)
                got = s.flows()
                z = s.objective()
            bad = np.abs(got - want) > tol * np.maximum(np.abs(want), sig) + floor
            assert not bad.any(), (inst.name, v, np.argwhere(bad)[:5])
            _, h2 = P.excess(got)
            z_want = P.objective(h2, P.congestion(got))
            assert abs(z - z_want) <= (1e-5 if prec == "fp32" else 1e-12) * z_want, (inst.name, v, z, z_want)


def test_variant_solves_agree(pdr):
    inst = instances()[0]
    base = None
    for v in fitting(pdr, inst.K, pdr.PREC_FP64):
        with pdr.Solver.from_instance(inst, precision=pdr.PREC_FP64, eps_obj=1e-6, resid_tol=0.0,
                                      edge_variant=v) as s:
            r = s.solve()
        if base is None:
            base = r
        assert r["sweeps"] == base["sweeps"] and r["verdict"] == base["verdict"], (v, r, base)
        assert abs(r["z"] - base["z"]) <= 1e-10 * base["z"]


def test_variant_switch_and_rejection(pdr):
    inst = instances()[2]  # K = 130: too long for the 4..16-lane groups and 32 x 1 vectors
    small = [v for v, cap, _ in pdr.edge_variants(pdr.PREC_FP32) if cap < inst.K]
    assert small
    with pytest.raises(pdr.PdrError):
        pdr.Solver.from_instance(inst, edge_variant=small[-1])
    rng = np.random.default_rng(5)
    f = rng.exponential(1.0, (inst.m, inst.K)).astype(np.float32).astype(np.float64)
    pipes = [v for v, cap, pipe in pdr.edge_variants(pdr.PREC_FP32) if pipe and cap >= inst.K]
    with pdr.Solver.from_instance(inst, precision=pdr.PREC_FP32) as s:
        s.set_flows(f)
        s.sweeps(3)
        ref = s.flows()
        s.set_flows(f)
        s.set_options(edge_variant=pipes[0])  # switching mid-state keeps the flows
        s.sweeps(3)
        got = s.flows()
        with pytest.raises(pdr.PdrError):
            s.set_options(edge_variant=small[-1])
        s.sweeps(1)  # the failed switch left the context usable
    assert np.abs(got - ref).max() <= 1e-5 * max(1.0, np.abs(ref).max())


def test_pipelined_variant_full_size_knn2500(pdr, knn2500):
    """The bench workload (m = 15,000 edges over 2 x 152 resident blocks, so
    every warp walks several edges and prefetches across them): 60 FP32 sweeps
    then one sweep compared with the oracle."""
    inst = knn2500
    P = oracle.Problem.from_instance(inst)
    pipe = [v for v, cap, p in pdr.edge_variants(pdr.PREC_FP32) if p and cap >= inst.K][0]
    with pdr.Solver.from_instance(inst, precision=pdr.PREC_FP32, edge_variant=pipe) as s:
        s.sweeps(60)
        f = s.flows()
        s.sweeps(1)
        got = s.flows()
    _, h = P.excess(f)
    want, _, _ = P.qp_all(h, f)
    sig = (np.abs(f) + np.abs(h[inst.src]) + np.abs(h[inst.col])).max(axis=1)[:, None]
    # an edge with zero flows and equal zero heights has scale 0: there the
    # error must stay within the floor (-inf after the division), else +inf
    with np.errstate(divide="ignore"):
        err = (np.abs(got - want) - FP32_FLOOR) / np.maximum(np.abs(want), sig)
    assert err.max() <= 1e-5, err.max()
