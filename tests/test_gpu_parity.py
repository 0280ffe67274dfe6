"""GPU parity: the CUDA path through the C ABI against the FP64 CPU oracle.

Tolerances (derived from the arithmetic, stated per check):
  * integer work (adjacency, degrees, sweep counts, verdicts): bit-exact;
  * FP64 kernels: 1e-12 relative to the row scale (only summation order and
    fused multiply-adds differ from the oracle);
  * FP32 kernels on the same FP32-representable input: 1e-5 relative to the
    row scale sigma_e = max_k (|f_e,k| + |h_ik| + |h_jk|) of the edge (every
    FP32 operand of c_k = f_k + (h_ik - h_jk)/2 is bounded by sigma_e, and the
    few dozen roundings on the way to f' stay below 1e-5 * sigma_e); heights
    relative to (sum_edges |f| + |hat-Delta|) / delta_i.  FP32 comparisons
    add an absolute floor of 1e-36: below the smallest normal FP32 number
    (1.2e-38) the spacing of representable values is fixed at 2^-149, so a
    relative bound cannot hold for flows that have decayed to that range.
"""

import numpy as np
import pytest

FP32_FLOOR = 1e-36

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


def random_state(inst, rng, density=0.3, scale=1.0, fp32=True):
    f = rng.exponential(scale, (inst.m, inst.K)) * (rng.random((inst.m, inst.K)) < density)
    return f.astype(np.float32).astype(np.float64) if fp32 else f


def height_scale(P, f, inst):
    """(sum over incident edges of |f| + |hat-Delta|) / delta_i, per (i, k)."""
    tot = np.zeros((inst.n, inst.K))
    np.add.at(tot, inst.src, np.abs(f))
    np.add.at(tot, inst.col, np.abs(f))
    tot[inst.s, np.arange(inst.K)] += inst.d
    tot[inst.t, np.arange(inst.K)] += inst.d
    return tot / np.maximum(P.deg, 1)[:, None]


def edge_scale(inst, f, h):
    return (np.abs(f) + np.abs(h[inst.src]) + np.abs(h[inst.col])).max(axis=1)


def tiny_instances():
    rng = np.random.default_rng(77)
    out = [I.grid5_k10(1.3), I.grid5_k10(1.3).with_factor(0.6)]
    # ragged K (not a multiple of 4), parallel arcs, vertices of degree 0
    g = I.random_digraph(30, 3, rng)
    out.append(I.make_instance("digraph30_k7", g, 7, ("uniform_int", 1, 9), 1.1, rng))
    out.append(I.make_instance("grid4_k1", I.grid_graph(4), 1, ("uniform_int", 3, 3), 0.8, rng))
    out.append(I.make_instance("grid6_k33", I.grid_graph(6), 33, ("lognormal", 1.0, 0.5), 1.2, rng))
    return out


# --------------------------------------------------------------------------- a0: adjacency


@pytest.mark.parametrize("which", ["grid5", "knn2500", "digraph_isolated"])
def test_adjacency_bit_exact(pdr, which, knn2500):
    if which == "grid5":
        inst = I.grid5_k10()
    elif which == "knn2500":
        inst = knn2500
    else:
        # vertices 6..9 have no edges at all
        rng = np.random.default_rng(3)
        n, rp, col = I.random_digraph(6, 2, rng)
        rp = np.concatenate([rp, np.full(4, rp[-1])])
        inst = I.Instance("iso", 10, rp, col, np.ones(col.shape[0]), np.array([0], np.int32),
                          np.array([1], np.int32), np.array([1.0]), 1.0, np.ones(col.shape[0]), np.array([1]))
    P = oracle.Problem.from_instance(inst)
    with pdr.Solver.from_instance(inst) as s:
        in_ptr, in_eid, deg = s.adjacency()
    np.testing.assert_array_equal(in_ptr, P.in_ptr)
    np.testing.assert_array_equal(in_eid, P.in_eid)
    np.testing.assert_array_equal(deg, P.deg)


# --------------------------------------------------------------------------- a1-a3: heights, congestion, objective


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_heights_congestion_objective(pdr, prec):
    rng = np.random.default_rng(1)
    for inst in tiny_instances() + [I.knn2500_k500()]:
        P = oracle.Problem.from_instance(inst)
        f = random_state(inst, rng)
        p = pdr.PREC_FP32 if prec == "fp32" else pdr.PREC_FP64
        with pdr.Solver.from_instance(inst, precision=p) as s:
            s.set_flows(f)
            h = s.heights()
            psi = s.congestion()
            z = s.objective()
        _, h_ref = P.excess(f)
        psi_ref = P.congestion(f)
        z_ref = P.objective(h_ref, psi_ref)
        tol = 1e-5 if prec == "fp32" else 1e-12
        floor = FP32_FLOOR if prec == "fp32" else 0.0
        hs = height_scale(P, f, inst)
        assert np.all(np.abs(h - h_ref) <= tol * hs + floor), inst.name
        ps = np.abs(f).sum(1) + inst.u
        assert np.all(np.abs(psi - psi_ref) <= tol * ps), inst.name
        assert abs(z - z_ref) <= (1e-5 if prec == "fp32" else 1e-11) * z_ref, inst.name


# --------------------------------------------------------------------------- a4: one sweep from identical state


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_one_sweep_matches_oracle(pdr, prec):
    rng = np.random.default_rng(2)
    for inst in tiny_instances():
        P = oracle.Problem.from_instance(inst)
        for trial in range(3):
            f = random_state(inst, rng, density=0.2 + 0.3 * trial, scale=0.5 + trial)
            p = pdr.PREC_FP32 if prec == "fp32" else pdr.PREC_FP64
            with pdr.Solver.from_instance(inst, precision=p) as s:
                s.set_flows(f)
                s.sweeps(1)
                got = s.flows()
            _, h = P.excess(f)
            want, _, _ = P.qp_all(h, f)
            sig = edge_scale(inst, f, h)[:, None]
            tol = 1e-5 if prec == "fp32" else 1e-12
            floor = FP32_FLOOR if prec == "fp32" else 0.0
            bad = np.abs(got - want) > tol * np.maximum(np.abs(want), sig) + floor
            assert not bad.any(), (inst.name, trial, np.argwhere(bad)[:5], np.abs(got - want).max())
            assert got.min() >= 0.0


def test_large_k_block_kernel_sweep(pdr):
    """K beyond the lane-group kernels (K > 2048) runs the one-edge-per-block form."""
    rng = np.random.default_rng(4)
    for K in (3001, 10000):
        inst = I.make_instance(f"grid11_k{K}", I.grid_graph(11), K, ("uniform_int", 1, 5), 0.9, rng)
        P = oracle.Problem.from_instance(inst)
        f = random_state(inst, rng, density=0.5)
        for prec, tol in ((pdr.PREC_FP32, 1e-5), (pdr.PREC_FP64, 1e-12)):
            with pdr.Solver.from_instance(inst, precision=prec) as s:
                s.set_flows(f)
                s.sweeps(1)
                got = s.flows()
            _, h = P.excess(f)
            want, _, _ = P.qp_all(h, f)
            sig = edge_scale(inst, f, h)[:, None]
            floor = FP32_FLOOR if prec == pdr.PREC_FP32 else 0.0
            assert np.all(np.abs(got - want) <= tol * np.maximum(np.abs(want), sig) + floor), (K, prec)


def test_full_size_sweep_parity_knn2500(pdr, knn2500):
    """The bench workload (n=2500, m=15000, K=500) in the bench's launch configuration:
    100 FP32 sweeps from f = 0 on the GPU, then one more sweep compared element by
    element with the oracle's sweep from the same (FP32) state."""
    inst = knn2500
    P = oracle.Problem.from_instance(inst)
    with pdr.Solver.from_instance(inst, precision=pdr.PREC_FP32) as s:
        s.sweeps(100)
        f = s.flows()
        h_gpu = s.heights()
        s.sweeps(1)
        got = s.flows()
    _, h = P.excess(f)
    hs = height_scale(P, f, inst)
    herr = np.abs(h_gpu - h) - 1e-5 * hs - FP32_FLOOR
    assert herr.max() <= 0.0, (np.unravel_index(herr.argmax(), herr.shape), h_gpu.flat[herr.argmax()],
                               h.flat[herr.argmax()], hs.flat[herr.argmax()])
    want, _, _ = P.qp_all(h, f)
    sig = edge_scale(inst, f, h)[:, None]
    err = np.maximum(np.abs(got - want) - FP32_FLOOR, 0.0) / np.maximum(np.maximum(np.abs(want), sig), 1e-300)
    assert err.max() <= 1e-5, err.max()
    # element by element, relative to the element itself, on every entry that
    # carries flow (|f'| > 1e-3 of the mean demand).  f' = c - theta is formed
    # in FP32 from c and theta of the row's scale sigma_e, so an entry far below
    # sigma_e carries the rounding of sigma_e: up to ~1e-4 of itself for an
    # entry 1e-3 of sigma_e.  The distribution must stay at a few FP32 ulps.
    big = np.abs(want) > 1e-3 * inst.d.mean()
    rel = np.abs(got - want)[big] / np.abs(want[big])
    q999 = np.quantile(rel, 0.999)
    assert rel.shape[0] > 1000
    assert rel.max() <= 1e-4 and q999 <= 5e-6, ("max", rel.max(), "p99.9", q999, "entries", rel.shape[0])


# --------------------------------------------------------------------------- Alg. 1 loop: stop rule, trace


def test_fp64_solve_matches_oracle_trace_and_stop(pdr):
    """FP64 on the device: the paper's stop rule fires at the same sweep as the oracle,
    and the objective trace agrees to 1e-9 relative at every sweep."""
    for inst in tiny_instances()[:3]:
        P = oracle.Problem.from_instance(inst)
        f_ref, rep, zt = P.solve_eso(max_sweeps=50000, eps_obj=1e-6, trace=True)
        with pdr.Solver.from_instance(inst, precision=pdr.PREC_FP64, eps_obj=1e-6, resid_tol=0.0,
                                      trace_len=60000) as s:
            r = s.solve()
            tr = s.trace()
            f = s.flows()
        assert r["sweeps"] == rep["sweeps"] and r["stop_name"] == "objective", (inst.name, r, rep)
        assert tr.shape[0] == rep["sweeps"] + 1
        np.testing.assert_allclose(tr, zt, rtol=1e-9)
        assert np.all(np.diff(tr) <= 1e-12 * tr[:-1])  # Section 4 theorem: non-increasing
        np.testing.assert_allclose(f, f_ref, rtol=1e-7, atol=1e-9 * inst.d.max())


def test_fp32_trace_tracks_fp64_oracle(pdr):
    """FP32 bulk: z^(t) stays within 1e-4 relative of the FP64 oracle for the first sweeps."""
    inst = I.grid5_k10()
    P = oracle.Problem.from_instance(inst)
    _, _, zt = P.solve_eso(max_sweeps=500, eps_obj=0.0, trace=True)
    with pdr.Solver.from_instance(inst, precision=pdr.PREC_FP32, eps_obj=0.0, resid_tol=0.0, max_sweeps=500,
                                  trace_len=1000) as s:
        r = s.solve()
        tr = s.trace()
    assert r["sweeps"] == 500 and r["stop_name"] == "max_sweeps"
    np.testing.assert_allclose(tr, zt, rtol=1e-4)


def test_max_sweeps_zero_and_paper_stop_returns_ft(pdr):
    inst = I.grid5_k10()
    P = oracle.Problem.from_instance(inst)
    with pdr.Solver.from_instance(inst, precision=pdr.PREC_FP64, max_sweeps=0) as s:
        r = s.solve()
        assert r["sweeps"] == 0 and r["stop_name"] == "max_sweeps"
        assert np.all(s.flows() == 0.0)
        _, h = P.excess(np.zeros((inst.m, inst.K)))
        assert abs(r["z"] - P.objective(h, np.zeros(inst.m))) <= 1e-12 * r["z"]


# --------------------------------------------------------------------------- a5: residuals, certificate, verdicts


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_residuals_match_oracle(pdr, prec):
    rng = np.random.default_rng(9)
    for inst in tiny_instances():
        P = oracle.Problem.from_instance(inst)
        f = random_state(inst, rng)
        p = pdr.PREC_FP32 if prec == "fp32" else pdr.PREC_FP64
        with pdr.Solver.from_instance(inst, precision=p) as s:
            s.set_flows(f)
            r = s.residuals()
        ref = P.residuals(f)
        for key in ("z", "cap_abs", "cap_rel", "cons_abs", "cons_rel", "margin"):
            assert abs(r[key] - ref[key]) <= 1e-12 * max(1.0, abs(ref[key]), ref["margin_scale"]), (inst.name, key)
        assert r["f_min"] == ref["f_min"]
        assert r["verdict"] == ref["verdict"]


@pytest.mark.parametrize("prec", ["fp64", "tail"])
def test_verdicts_tiny(pdr, prec):
    """Verdicts equal the oracle's on the tiny instances (FP64 or FP32 with FP64 tail)."""
    for inst in tiny_instances():
        P = oracle.Problem.from_instance(inst)
        f_ref, rep = P.solve_eso(max_sweeps=300000, eps_obj=0.0, resid_tol=1e-6)
        if rep["stop_reason"] != 2:
            f_ref, rep = P.solve_eso(max_sweeps=300000, eps_obj=1e-15, f0=f_ref)
        want = P.residuals(f_ref)["verdict"]
        p = pdr.PREC_FP64 if prec == "fp64" else pdr.PREC_FP32_FP64TAIL
        with pdr.Solver.from_instance(inst, precision=p, eps_obj=0.0, resid_tol=1e-6, eps_rel=1e-13,
                                      max_sweeps=600000) as s:
            r = s.solve()
            f = s.flows()
        assert r["verdict"] == want, (inst.name, r, rep)
        if prec == "tail":  # the rule that ended the FP32 phase is reported
            assert r["stop_name_fp32"] in ("stall", "plateau", "objective", "relative", "residual"), r
            assert (r["sweeps_fp64"] > 0) == (r["stop_name_fp32"] != "residual"), r
        else:
            assert r["stop_name_fp32"] == "-", r
        if want == pdr.VERDICT_FEASIBLE:
            ref = P.residuals(f)
            assert ref["cap_rel"] <= 1e-6 and ref["cons_rel"] <= 1e-6
        if inst.feasible_by_construction is not None:
            assert (r["verdict"] == pdr.VERDICT_FEASIBLE) == inst.feasible_by_construction


def test_isolated_endpoint_and_no_edges(pdr):
    # commodity 0 -> 2 where vertex 2 has no edges
    with pdr.Solver(3, [0, 1, 2, 2], [1, 0], [5.0, 5.0], [0], [2], [1.0]) as s:
        r = s.solve()
        assert r["verdict"] == pdr.VERDICT_INFEASIBLE
    with pdr.Solver(2, [0, 0, 0], [], [], [0], [1], [2.0], max_sweeps=10) as s:
        r = s.solve()
        assert r["verdict"] == pdr.VERDICT_INFEASIBLE and r["sweeps"] <= 10


def test_zero_capacity_edges_carry_no_flow_at_feasibility(pdr):
    inst = I.grid5_k10(1.3)
    assert (inst.u == 0).sum() > 0
    with pdr.Solver.from_instance(inst, precision=pdr.PREC_FP64, eps_obj=0.0, resid_tol=1e-6) as s:
        r = s.solve()
        f = s.flows()
    assert r["verdict"] == pdr.VERDICT_FEASIBLE
    ubar = inst.u[inst.u > 0].mean()
    assert f[inst.u == 0].sum(1).max() <= 1e-6 * ubar


def test_repeat_solves_are_deterministic(pdr, knn2500):
    with pdr.Solver.from_instance(knn2500, precision=pdr.PREC_FP32, eps_obj=0.0, resid_tol=0.0,
                                  max_sweeps=300) as s:
        s.solve()
        a = s.flows()
        s.reset()
        s.solve()
        b = s.flows()
    np.testing.assert_array_equal(a, b)


def test_host_loop_matches_graph_loop(pdr, knn2500):
    """use_graph = 0 launches the same kernels from a host loop: same sweeps, same flows."""
    out = []
    for g in (1, 0):
        with pdr.Solver.from_instance(knn2500, precision=pdr.PREC_FP32, eps_obj=1e-2, resid_tol=0.0,
                                      max_sweeps=5000, use_graph=g) as s:
            r = s.solve()
            out.append((r["sweeps"], r["stop_name"], s.flows()))
    assert out[0][0] == out[1][0] and out[0][1] == out[1][1] == "objective"
    np.testing.assert_array_equal(out[0][2], out[1][2])


def test_padding_stays_zero_at_the_capacity_boundary(pdr):
    """Near convergence many edges sit at s = sum max(0, c) ~ u, where FP32
    rounding can make a Case 2 root come out just below 0; the root search
    takes Case 1 there (root 0), so the zero padding of the rows (K = 33 is
    padded to 36) stays exactly 0 and the residuals equal the oracle's."""
    import struct

    rng = np.random.default_rng(77)
    inst = I.make_instance("grid6_k33", I.grid_graph(6), 33, ("lognormal", 1.0, 0.5), 1.2, rng)
    with pdr.Solver.from_instance(inst, precision=pdr.PREC_FP32, eps_obj=0.0, resid_tol=0.0, max_sweeps=12000) as s:
        r = s.solve()
        f = s.flows()
        st = s.get_state()
        Kp = s.Kp
    hdr = 112  # the checkpoint header: magic, version, 6 ints, 5 int64, 2 doubles, int64, 2 doubles
    assert struct.unpack_from("<I", st, 0)[0] == 0x53524450
    raw = np.frombuffer(st[hdr:hdr + inst.m * Kp * 4], dtype=np.float32).reshape(inst.m, Kp)
    np.testing.assert_array_equal(raw[:, :inst.K], f.astype(np.float32))
    assert np.all(raw[:, inst.K:] == 0.0)
    ref = oracle.Problem.from_instance(inst).residuals(f)
    for key in ("cap_rel", "cons_rel", "z"):
        assert abs(r[key] - ref[key]) <= 1e-12 * max(1.0, abs(ref[key]), ref["margin_scale"]), key


def test_flows_into_pinned_and_device_buffers(pdr):
    """pdr_flows writes the same doubles into pageable host memory (staging
    copy), pinned host memory and device memory (a widening kernel)."""
    import ctypes

    import torch

    inst = tiny_instances()[4]  # K = 33: rows padded to 36
    for prec in (pdr.PREC_FP32, pdr.PREC_FP64):
        with pdr.Solver.from_instance(inst, precision=prec, eps_obj=0.0, resid_tol=0.0, max_sweeps=25) as s:
            s.solve()
            want = s.flows()
            pinned = torch.empty((inst.m, inst.K), dtype=torch.float64).pin_memory()
            dev = torch.full((inst.m, inst.K), -1.0, dtype=torch.float64, device="cuda")
            for buf in (pinned, dev):
                s._check(s._lib.pdr_flows(s._h, ctypes.c_void_p(buf.data_ptr())))
                np.testing.assert_array_equal(buf.cpu().numpy(), want)
