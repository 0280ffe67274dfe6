"""Pins for the oracle's capacity-kept variant (Program (6), Section "Further
Discussion on Optimality Condition").

The paper gives Program (6) and its KKT conditions but no algorithm; the
oracle reads Alg. 1 with the capacity kept in the local step: every edge
projects c_k = f_k + (h_ik - h_jk)/2 onto {f' >= 0, sum_k f'_k <= u}.
Pinned here against things other than the oracle itself: the K = 1 clamp,
exact enumeration of the faces for K = 2 and 3, the projection's
variational inequality, Alg. 2's Case 1 for uncapacitated edges, the descent
lemma for projected gradient steps (the step is one with step 1/2, and
1/2 <= 1/L for L <= 2 by Gershgorin on B D^-1 B^T), the paper's KKT
conditions (i)-(iii) at the limit, and an LP on tiny instances.
"""

from __future__ import annotations

import itertools

import numpy as np
import pytest

import oracle
from paper_2108_07549_gb300 import instances as I


def _c(hi, hj, f):
    return np.asarray(f) + 0.5 * (np.asarray(hi) - np.asarray(hj))


def brute_force_projection(c, u):
    """Minimiser of sum (x - c)^2 over {x >= 0, sum x <= u} by enumerating the
    faces: a set Z of coordinates fixed at 0, with or without sum x = u."""
    K = len(c)
    best = None
    for mask in itertools.product([0, 1], repeat=K):
        free = [k for k in range(K) if mask[k]]
        for tight in (False, True):
            x = np.zeros(K)
            if tight:
                if not free:
                    continue
                g = (sum(c[k] for k in free) - u) / len(free)
                for k in free:
                    x[k] = c[k] - g
            else:
                for k in free:
                    x[k] = c[k]
            if x.min() < -1e-12 or x.sum() > u + 1e-12:
                continue
            val = float(((x - c) ** 2).sum())
            if best is None or val < best[0] - 1e-15:
                best = (val, x)
    return best[1]


def test_k1_is_a_clamp():
    rng = np.random.default_rng(1)
    for _ in range(200):
        hi, hj, f = rng.normal(0, 2, 3)
        u = float(rng.choice([0.0, rng.uniform(0, 3)]))
        out, g, fb = oracle.edge_ck([hi], [hj], [abs(f)], u)
        c = abs(f) + 0.5 * (hi - hj)
        assert out[0] == pytest.approx(min(max(c, 0.0), u), abs=1e-14)
        assert not fb


@pytest.mark.parametrize("K", [2, 3])
def test_small_k_matches_face_enumeration(K):
    rng = np.random.default_rng(10 + K)
    for _ in range(300):
        hi, hj = rng.normal(0, 2, K), rng.normal(0, 2, K)
        f = rng.exponential(1.0, K) * (rng.random(K) < 0.7)
        u = float(rng.choice([0.0, rng.uniform(0, 4)]))
        out, g, _ = oracle.edge_ck(hi, hj, f, u)
        want = brute_force_projection(_c(hi, hj, f), u)
        np.testing.assert_allclose(out, want, atol=1e-12)


def test_projection_variational_inequality_and_threshold_form():
    """x = P(c) iff (c - x) . (y - x) <= 0 for every feasible y; and x = max(0, c - g)
    with g >= 0, g (sum x - u) = 0."""
    rng = np.random.default_rng(3)
    for K in (5, 17, 64):
        for _ in range(40):
            hi, hj = rng.normal(0, 3, K), rng.normal(0, 3, K)
            f = rng.exponential(1.0, K) * (rng.random(K) < 0.5)
            u = float(rng.uniform(0, 2 * K))
            x, g, _ = oracle.edge_ck(hi, hj, f, u)
            c = _c(hi, hj, f)
            assert x.min() >= 0 and x.sum() <= u * (1 + 1e-12) + 1e-12
            assert g >= 0 and abs(g * (x.sum() - u)) <= 1e-9 * max(1.0, u)
            np.testing.assert_allclose(x, np.maximum(0.0, c - g), atol=1e-12)
            for _ in range(20):  # random feasible points
                y = rng.exponential(1.0, K) * (rng.random(K) < 0.6)
                if y.sum() > u:
                    y *= u / y.sum() * rng.uniform(0, 1)
                assert np.dot(c - x, y - x) <= 1e-9 * (1 + np.abs(c).sum() * max(1.0, u))


def test_uncapacitated_edges_take_alg2_case1(grid5):
    """With capacities no flow can reach, both steps are f' = max(0, c)."""
    inst = grid5
    P = oracle.Problem(inst.n, inst.row_ptr, inst.col, np.full(inst.m, 1e12), inst.s, inst.t, inst.d)
    rng = np.random.default_rng(4)
    f = rng.exponential(1.0, (inst.m, inst.K)) * (rng.random((inst.m, inst.K)) < 0.4)
    _, h = P.excess(f)
    a, _, _ = P.qp_all(h, f)
    b, g, _ = P.ck_all(h, f)
    np.testing.assert_array_equal(a, b)
    assert np.all(g == 0.0)


def test_descent_lemma_and_capacity_kept(grid5, grid5_bad):
    """z_6 = 1/2 sum delta h^2 is non-increasing along the iteration (projected
    gradient with step 1/2 <= 1/L), and every iterate keeps the capacities."""
    for inst in (grid5, grid5_bad):
        P = oracle.Problem.from_instance(inst)
        f, rep, zt = P.solve_ck(max_sweeps=3000, eps_obj=0.0, trace=True)
        assert np.all(np.diff(zt) <= 1e-12 * zt[:-1])
        assert np.all(f.sum(1) <= inst.u * (1 + 1e-12) + 1e-12) and f.min() >= 0.0
        # the projected-gradient step: grad_f z_6 = h_j - h_i, so c = f - 1/2 grad
        _, h = P.excess(f)
        c = f + 0.5 * (h[inst.src] - h[inst.col])
        nxt = P.ck_sweep(f)
        for e in range(inst.m):
            # near-degenerate faces differ in x by O(sqrt(rounding)): compare the
            # projection's objective, which is what the brute force minimises
            want = brute_force_projection(c[e], inst.u[e])
            x = nxt[e]
            assert x.min() >= 0 and x.sum() <= inst.u[e] * (1 + 1e-12) + 1e-12
            assert ((x - c[e]) ** 2).sum() <= ((want - c[e]) ** 2).sum() + 1e-12 * (1 + (c[e] ** 2).sum())


def test_feasible_instance_reaches_zero_objective(grid5):
    """Program (6) has minimum 0 iff eq. (1) is feasible: the residuals vanish."""
    P = oracle.Problem.from_instance(grid5)
    f, rep = P.solve_ck(max_sweeps=200000, eps_obj=0.0, resid_tol=1e-6)
    assert rep["stop_reason"] == 2
    res = P.residuals(f)
    assert res["verdict"] == oracle.VERDICT_FEASIBLE and res["cap_abs"] <= 1e-12


def test_infeasible_limit_satisfies_the_papers_kkt_conditions(grid5_bad):
    """At the limit: (i) used commodities on unsaturated edges have h_i = h_j;
    (ii) on a saturated edge all used commodities share one height
    difference, the pipe pressure; (iii) unused ones are at or below it; and
    the heights certify infeasibility (Farkas margin > 0)."""
    inst = grid5_bad
    P = oracle.Problem.from_instance(inst)
    f, rep = P.solve_ck(max_sweeps=200000, eps_obj=1e-15)
    _, h = P.excess(f)
    dh = h[inst.src] - h[inst.col]
    used = f > 1e-9 * inst.d[None, :]
    sat = f.sum(1) >= inst.u * (1 - 1e-9)
    scale = np.abs(h).max()
    for e in range(inst.m):
        if not used[e].any():
            continue
        if not sat[e]:
            assert np.abs(dh[e, used[e]]).max() <= 1e-6 * scale
        else:
            pressure = dh[e, used[e]]
            assert pressure.max() - pressure.min() <= 1e-6 * scale
            assert pressure.min() >= -1e-6 * scale
            assert dh[e, ~used[e]].max(initial=-np.inf) <= pressure.max() + 1e-6 * scale
    res = P.residuals(f)
    assert res["verdict"] == oracle.VERDICT_INFEASIBLE and res["margin"] > 0


@pytest.mark.slow
def test_verdicts_agree_with_lp():
    """Capacity-kept verdicts on small random instances match an LP away from the boundary."""
    from test_oracle import _lp_max_concurrent

    checked = 0
    for seed in range(6):
        rng = np.random.default_rng(1000 + seed)
        g = I.grid_graph(3) if seed % 2 == 0 else I.random_digraph(8, 3, rng)
        base = I.make_instance(f"lp{seed}", g, 3, ("uniform_int", 1, 5), 1.0, rng)
        for factor in (0.5, 0.75, 1.0, 1.3):
            inst = base.with_factor(factor)
            lam = _lp_max_concurrent(inst)
            if 0.97 < lam < 1.03:
                continue
            P = oracle.Problem.from_instance(inst)
            f, rep = P.solve_ck(max_sweeps=400000, eps_obj=0.0, resid_tol=1e-6)
            v = P.residuals(f)["verdict"]
            if v == oracle.VERDICT_UNKNOWN:
                f, rep = P.solve_ck(max_sweeps=400000, eps_obj=1e-15, f0=f)
                v = P.residuals(f)["verdict"]
            expect = oracle.VERDICT_FEASIBLE if lam >= 1.0 else oracle.VERDICT_INFEASIBLE
            assert v == expect, (seed, factor, lam, rep)
            checked += 1
    assert checked >= 12
