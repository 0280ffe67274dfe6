"""Pins for the FP64 oracle: every check compares it with something other than itself.

Brute force over faces of the edge QP in exact rational arithmetic, a generic
bound-constrained minimiser, the K = 1 closed form, KKT conditions, a
hand-derived worked example, invariants of eq. (3)/(8), the gradient identity
(eq. "cpgrad"), the monotonicity theorem of Section 4, an LP feasibility
solver and max-flow for one commodity.
"""

from __future__ import annotations

import itertools
import os
from fractions import Fraction as Fr

import numpy as np
import pytest

import oracle
from paper_2108_07549_gb300 import instances as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------- helpers


def eq10_objective(hi, hj, f, u, f_new, r):
    """The edge subproblem objective of eq. (10), evaluated term by term."""
    tot = sum(f_new) + r - u
    a = sum((hi[k] + f[k] - f_new[k]) ** 2 for k in range(len(f)))
    b = sum((hj[k] - f[k] + f_new[k]) ** 2 for k in range(len(f)))
    return (tot * tot + a + b) / 2


def _solve_linear(A, b):
    """Exact Gaussian elimination over Fractions."""
    n = len(b)
    M = [row[:] + [b[i]] for i, row in enumerate(A)]
    for col in range(n):
        piv = next(r for r in range(col, n) if M[r][col] != 0)
        M[col], M[piv] = M[piv], M[col]
        for r in range(n):
            if r != col and M[r][col] != 0:
                fac = M[r][col] / M[col][col]
                M[r] = [x - fac * y for x, y in zip(M[r], M[col])]
    return [M[i][n] / M[i][i] for i in range(n)]


def brute_force_qp(hi, hj, f, u):
    """Exact minimiser of eq. (10) by enumerating faces of {f' >= 0, r >= 0}.

    On each face the free variables satisfy grad = 0, a linear system solved
    exactly; the minimiser of the strictly convex QP is the primal-feasible
    face stationary point of least objective.  Works on Fractions.
    """
    K = len(f)
    best = None
    for mask in itertools.product([0, 1], repeat=K):
        A = [k for k in range(K) if mask[k]]
        for r_free in (False, True):
            nv = len(A) + (1 if r_free else 0)
            # unknowns: f'_A (and r); gradient of eq. (10):
            #   d/df'_k = (S + r - u) - (hi_k + f_k - f'_k) + (hj_k - f_k + f'_k)
            #   d/dr    = (S + r - u)
            rows, rhs = [], []
            for a_idx, k in enumerate(A):
                row = [Fr(1)] * len(A) + ([Fr(1)] if r_free else [])
                row[a_idx] += 2
                rows.append(row)
                rhs.append(u + hi[k] + f[k] - hj[k] + f[k])
            if r_free:
                rows.append([Fr(1)] * nv)
                rhs.append(u)
            sol = _solve_linear(rows, rhs) if nv else []
            fn = [Fr(0)] * K
            for a_idx, k in enumerate(A):
                fn[k] = sol[a_idx]
            r = sol[-1] if r_free else Fr(0)
            if any(x < 0 for x in fn) or r < 0:
                continue
            val = eq10_objective(hi, hj, f, u, fn, r)
            if best is None or val < best[0]:
                best = (val, fn, r)
    return best


def rand_dyadic(rng, size, lo, hi, denom=64):
    return [Fr(int(x), denom) for x in rng.integers(lo * denom, hi * denom + 1, size=size)]


def load_golden(name):
    out = {}
    for line in open(os.path.join(GOLDEN, name)):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        key, val = line.split(":", 1)
        out[key.strip()] = [Fr(x) for x in val.split()]
    return out


# --------------------------------------------------------------------------- edge QP (Alg. 2)


@pytest.mark.parametrize("K", [1, 2, 3, 4, 5])
def test_edge_qp_matches_exact_face_enumeration(K):
    """Alg. 2 equals the exact minimiser of eq. (10) for small K (rational inputs)."""
    rng = np.random.default_rng(100 + K)
    cases = 120 if K <= 3 else 40
    for case in range(cases):
        hi = rand_dyadic(rng, K, -3, 3)
        hj = rand_dyadic(rng, K, -3, 3)
        f = rand_dyadic(rng, K, 0, 2)
        if case % 7 == 0:
            f = [Fr(0)] * K
        u = rand_dyadic(rng, 1, 0, 4)[0] if case % 5 else Fr(0)
        val, fn, r = brute_force_qp(hi, hj, f, u)
        got, r_got, psi_got, _ = oracle.edge_qp([float(x) for x in hi], [float(x) for x in hj],
                                                [float(x) for x in f], float(u))
        np.testing.assert_allclose(got, [float(x) for x in fn], rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(r_got, float(r), rtol=1e-12, atol=1e-12)
        psi_exact = max(Fr(0), sum(fn) + r - u)
        np.testing.assert_allclose(psi_got, float(psi_exact), rtol=1e-12, atol=1e-12)


def test_edge_qp_k1_closed_form():
    """K = 1: f' = max(0, c) when c <= u, else (2c + u)/3 (from stationarity with r = 0)."""
    rng = np.random.default_rng(7)
    for _ in range(500):
        hi, hj = rng.uniform(-5, 5, 2)
        f = rng.uniform(0, 3)
        u = rng.uniform(0, 4) if rng.random() < 0.8 else 0.0
        c = f + (hi - hj) / 2
        expect = max(0.0, c) if c <= u else (2 * c + u) / 3
        got = oracle.edge_qp([hi], [hj], [f], u)[0][0]
        assert abs(got - expect) <= 1e-12 * max(1.0, abs(expect))


def test_edge_qp_hand_example_k2():
    """c = (3, 1), u = 2: Case 2 with p = 2, psi = 1, f' = (5/2, 1/2) (Alg. 2 by hand)."""
    # c_k = f_k + (h_ik - h_jk)/2 with f = 0, h_i = 2c, h_j = 0
    got, r, psi, fb = oracle.edge_qp([6.0, 2.0], [0.0, 0.0], [0.0, 0.0], 2.0)
    assert not fb
    np.testing.assert_allclose(got, [2.5, 0.5], rtol=0, atol=1e-15)
    assert r == 0.0 and abs(psi - 1.0) < 1e-15


def test_edge_qp_special_cases():
    """All c <= 0 gives zero flow; s == u takes Case 1; u = 0 with positive c congests."""
    got, r, psi, _ = oracle.edge_qp([-1.0, -2.0], [1.0, 0.0], [0.5, 0.5], 1.0)
    np.testing.assert_array_equal(got, [0.0, 0.0])
    assert psi == 0.0 and r == 1.0
    # s == u: c = (1, 1), u = 2
    got, r, psi, _ = oracle.edge_qp([2.0, 2.0], [0.0, 0.0], [0.0, 0.0], 2.0)
    np.testing.assert_array_equal(got, [1.0, 1.0])
    assert psi == 0.0 and r == 0.0
    # u = 0, c = (1, 1): psi = (2 - 0)/(1 + 1) = 1, f' = 1/2 each
    got, r, psi, _ = oracle.edge_qp([2.0, 2.0], [0.0, 0.0], [0.0, 0.0], 0.0)
    np.testing.assert_allclose(got, [0.5, 0.5], atol=1e-15)
    assert abs(psi - 1.0) < 1e-15
    # ties among the sorted potentials do not change the root
    got, r, psi, fb = oracle.edge_qp([4.0, 4.0, 4.0, 1.0], [0.0] * 4, [0.0] * 4, 1.0)
    val, fn, rr = brute_force_qp([Fr(4), Fr(4), Fr(4), Fr(1)], [Fr(0)] * 4, [Fr(0)] * 4, Fr(1))
    np.testing.assert_allclose(got, [float(x) for x in fn], atol=1e-14)


@pytest.mark.parametrize("K", [64, 500])
def test_edge_qp_kkt_and_generic_minimiser(K):
    """Large K: KKT conditions of eq. (10) hold, and L-BFGS-B on eq. (10) finds the same point."""
    from scipy.optimize import minimize

    rng = np.random.default_rng(K)
    for case in range(6):
        hi = rng.normal(0, 1, K)
        hj = rng.normal(0, 1, K)
        f = np.abs(rng.normal(0, 0.5, K)) * (rng.random(K) < 0.6)
        u = float(rng.uniform(0, 0.3 * K)) if case else 0.0
        fn, r, psi, _ = oracle.edge_qp(hi, hj, f, u)
        c = (hi - hj + 2 * f) / 2  # the "driving potential" of Section 4.4.1
        assert fn.min() >= 0 and r >= 0
        assert abs(psi - max(0.0, fn.sum() - u)) <= 1e-10 * max(1.0, u)
        assert psi * r == 0.0
        act = fn > 0
        np.testing.assert_allclose(2 * (fn[act] - c[act]) + psi, 0.0, atol=1e-10)
        assert np.all(c[~act] <= psi / 2 + 1e-10)

        def obj(x):
            fp, rr = x[:K], x[K]
            tot = fp.sum() + rr - u
            g_f = tot - (hi + f - fp) + (hj - f + fp)
            val = 0.5 * (tot ** 2 + ((hi + f - fp) ** 2).sum() + ((hj - f + fp) ** 2).sum())
            return val, np.concatenate([g_f, [tot]])

        x0 = np.concatenate([f, [0.0]])
        res = minimize(obj, x0, jac=True, method="L-BFGS-B", bounds=[(0, None)] * (K + 1),
                       options={"ftol": 1e-15, "gtol": 1e-11, "maxiter": 20000})
        np.testing.assert_allclose(fn, res.x[:K], atol=2e-5)  # L-BFGS-B converges to ~1e-6
        ref_val = obj(np.concatenate([fn, [r]]))[0]
        assert ref_val <= res.fun + 1e-9 * max(1.0, abs(res.fun))


# --------------------------------------------------------------------------- graph notation


def test_adjacency_matches_sorted_construction(knn2500):
    inst = knn2500
    P = oracle.Problem.from_instance(inst)
    order = np.argsort(inst.col, kind="stable")  # in-edges grouped by head, ascending edge id
    np.testing.assert_array_equal(P.in_eid, order)
    counts = np.bincount(inst.col, minlength=inst.n)
    np.testing.assert_array_equal(np.diff(P.in_ptr), counts)
    np.testing.assert_array_equal(P.src, inst.src)
    np.testing.assert_array_equal(P.deg, np.diff(inst.row_ptr) + counts)
    assert int(P.deg.sum()) == 2 * inst.m


def test_adjacency_rejects_bad_csr():
    with pytest.raises(ValueError):
        oracle.Problem(3, [0, 1, 2, 3], [1, 2, 3], [1.0] * 3, [0], [1], [1.0])
    with pytest.raises(ValueError):
        oracle.Problem(3, [0, 2, 1, 3], [1, 2, 0], [1.0] * 3, [0], [1], [1.0])


# --------------------------------------------------------------------------- excess, height, objective


def test_zero_flow_excess_and_objective_closed_form(grid5):
    """At f = 0: Delta = hat-Delta (eq. (3h)), h = Delta/delta, z = 1/2 sum_k d_k^2 (1/delta_s + 1/delta_t)."""
    P = oracle.Problem.from_instance(grid5)
    f = np.zeros((grid5.m, grid5.K))
    Delta, h = P.excess(f)
    expect = np.zeros((grid5.n, grid5.K))
    for k in range(grid5.K):
        expect[grid5.s[k], k] += grid5.d[k]
        expect[grid5.t[k], k] -= grid5.d[k]
    np.testing.assert_array_equal(Delta, expect)
    np.testing.assert_allclose(h, expect / P.deg[:, None], rtol=1e-15)
    z = P.objective(h, P.congestion(f))
    z0 = 0.5 * sum(grid5.d[k] ** 2 * (1 / P.deg[grid5.s[k]] + 1 / P.deg[grid5.t[k]]) for k in range(grid5.K))
    assert abs(z - z0) <= 1e-13 * z0


def test_excess_sums_to_zero_and_objective_forms_agree(knn2500):
    """sum_i Delta_ik = 0 for every k; vertex form of z equals the edge form of eq. (8)."""
    inst = knn2500
    P = oracle.Problem.from_instance(inst)
    rng = np.random.default_rng(3)
    f = rng.exponential(0.3, (inst.m, inst.K)) * (rng.random((inst.m, inst.K)) < 0.2)
    Delta, h = P.excess(f)
    scale = np.abs(f).sum() + inst.d.sum()
    assert np.abs(Delta.sum(axis=0)).max() <= 1e-12 * scale
    psi = P.congestion(f)
    z_v = P.objective(h, psi)
    # edge form, summed here from the oracle's h and psi
    z_e = 0.5 * ((psi ** 2).sum() + (h[inst.src] ** 2).sum() + (h[inst.col] ** 2).sum())
    assert abs(z_v - z_e) <= 1e-12 * z_v
    assert abs(P.objective_edges(h, psi) - z_v) <= 1e-12 * z_v
    # eq. (41) directly
    np.testing.assert_allclose(psi, np.maximum(0.0, f.sum(1) - inst.u), rtol=1e-13, atol=1e-13)


def test_gradient_identity_cpgrad(grid5):
    """dz/df_ij,k = psi_ij + h_jk - h_ik (eq. "cpgrad"), by central differences of the oracle's z."""
    inst = grid5
    P = oracle.Problem.from_instance(inst)
    rng = np.random.default_rng(11)
    f = rng.uniform(0.1, 2.0, (inst.m, inst.K))
    # push some edges over capacity so psi > 0 there
    f[: inst.m // 3] *= 3.0

    def z_of(ff):
        _, hh = P.excess(ff)
        return P.objective(hh, P.congestion(ff))

    _, h = P.excess(f)
    psi = P.congestion(f)
    eps = 1e-6
    for _ in range(60):
        e = int(rng.integers(inst.m))
        k = int(rng.integers(inst.K))
        fp, fm = f.copy(), f.copy()
        fp[e, k] += eps
        fm[e, k] -= eps
        fd = (z_of(fp) - z_of(fm)) / (2 * eps)
        grad = psi[e] + h[inst.col[e], k] - h[inst.src[e], k]
        assert abs(fd - grad) <= 1e-6 * max(1.0, abs(grad)), (e, k, fd, grad)


# --------------------------------------------------------------------------- Alg. 1


def test_two_vertex_golden():
    """The hand-derived example in tests/golden/two_vertex_k1.txt (eq. (2), (3), (41), Alg. 1, Alg. 2)."""
    g = load_golden("two_vertex_k1.txt")
    P = oracle.Problem(2, [int(x) for x in g["row_ptr"]], [int(x) for x in g["col"]],
                       [float(x) for x in g["u"]], [int(x) for x in g["s"]], [int(x) for x in g["t"]],
                       [float(x) for x in g["d"]])
    f = np.zeros((2, 1))
    _, h = P.excess(f)
    assert P.objective(h, P.congestion(f)) == float(g["z0"][0])
    f1 = P.sweep(f)
    np.testing.assert_allclose(f1[:, 0], [float(x) for x in g["f1"]], atol=1e-15)
    _, h1 = P.excess(f1)
    assert abs(P.objective(h1, P.congestion(f1)) - float(g["z1"][0])) < 1e-15
    f2 = P.sweep(f1)
    np.testing.assert_allclose(f2[:, 0], [float(x) for x in g["f2"]], atol=1e-15)
    _, h2 = P.excess(f2)
    np.testing.assert_allclose(h2[:, 0], [float(x) for x in g["h2"]], atol=1e-15)
    np.testing.assert_allclose(P.congestion(f2), [float(x) for x in g["psi2"]], atol=1e-15)
    assert abs(P.objective(h2, P.congestion(f2)) - float(g["z2"][0])) < 1e-15
    f_lim, rep = P.solve_eso(max_sweeps=2000, eps_obj=0.0)
    np.testing.assert_allclose(f_lim[:, 0], [float(x) for x in g["f_limit"]], atol=1e-12)
    assert abs(rep["z"] - float(g["z_limit"][0])) < 1e-12
    res = P.residuals(f_lim)
    assert abs(res["margin"] - float(g["margin_limit"][0])) < 1e-10
    assert res["verdict"] == oracle.VERDICT_INFEASIBLE


def test_objective_monotone_and_surrogate_bound(grid5, grid5_bad):
    """Section 4 theorem: z(f^(t+1)) <= Q(f^(t+1), f^(t)) <= z(f^(t))."""
    for inst in (grid5, grid5_bad):
        P = oracle.Problem.from_instance(inst)
        f = np.zeros((inst.m, inst.K))
        for _ in range(150):
            _, h = P.excess(f)
            z = P.objective(h, P.congestion(f))
            f_next = P.sweep(f)
            dF = f_next - f
            psi_next = P.congestion(f_next)
            Q = 0.5 * ((psi_next ** 2).sum() + ((h[inst.src] - dF) ** 2).sum() + ((h[inst.col] + dF) ** 2).sum())
            _, h_next = P.excess(f_next)
            z_next = P.objective(h_next, psi_next)
            assert z_next <= Q * (1 + 1e-12) + 1e-15
            assert Q <= z * (1 + 1e-12) + 1e-15
            f = f_next


def _independent_residuals(inst, f):
    """eq. (1) constraint violations computed directly from the flows."""
    cap = np.maximum(0.0, f.sum(1) - inst.u)
    net = np.zeros((inst.n, inst.K))
    np.add.at(net, inst.src, f)
    np.add.at(net, inst.col, -f)  # out - in
    rhs = np.zeros((inst.n, inst.K))
    rhs[inst.s, np.arange(inst.K)] += inst.d
    rhs[inst.t, np.arange(inst.K)] -= inst.d
    cons = np.abs(net - rhs) / inst.d[None, :]
    return cap, cons


def test_solve_feasible_grid_reaches_residual_target(grid5):
    P = oracle.Problem.from_instance(grid5)
    f, rep = P.solve_eso(max_sweeps=100000, eps_obj=0.0, resid_tol=1e-6)
    assert rep["stop_reason"] == 2
    cap, cons = _independent_residuals(grid5, f)
    ubar = grid5.u[grid5.u > 0].mean()
    assert (cap / np.maximum(grid5.u, ubar)).max() <= 1e-6
    assert cons.max() <= 1e-6
    assert f.min() >= 0.0
    assert P.residuals(f)["verdict"] == oracle.VERDICT_FEASIBLE


def test_solve_paper_stop_rule(grid5):
    """The stop rule |z^(t) - z^(t-1)| < 1e-6 of Alg. 1 fires, and returns f^(t)."""
    P = oracle.Problem.from_instance(grid5)
    f, rep, zt = P.solve_eso(max_sweeps=100000, eps_obj=1e-6, trace=True)
    assert rep["stop_reason"] == 1
    t = rep["sweeps"]
    assert abs(zt[t] - zt[t - 1]) < 1e-6 and np.all(np.abs(np.diff(zt[:t])) >= 1e-6)
    _, h = P.excess(f)
    assert P.objective(h, P.congestion(f)) == rep["z"]


def test_infeasible_twin_certificate_and_stability(grid5_bad):
    """0.6x capacities: infeasible by construction; the Farkas margin is positive and
    the limit is a nonzero-stable pseudo-flow (Def. 1 and Theorem 2)."""
    inst = grid5_bad
    assert inst.feasible_by_construction is False
    P = oracle.Problem.from_instance(inst)
    f, rep = P.solve_eso(max_sweeps=30000, eps_obj=1e-14)
    res = P.residuals(f)
    assert res["verdict"] == oracle.VERDICT_INFEASIBLE and res["margin"] > 0
    # the margin tends to 2 z* at the optimum
    assert abs(res["margin"] - 2 * res["z"]) <= 1e-3 * res["z"]
    # independent check of the certificate: (pi = h, l) is dual feasible and margin > 0
    _, h = P.excess(f)
    l = np.maximum(0.0, (h[inst.src] - h[inst.col]).max(1))
    assert np.all(h[inst.src] - h[inst.col] <= l[:, None])
    gain = (inst.d * (h[inst.s, np.arange(inst.K)] - h[inst.t, np.arange(inst.K)])).sum()
    assert gain - (inst.u * l).sum() > 0
    # stable pseudo-flow: phi = 0 on used edges, phi <= 0 on unused ones
    psi = P.congestion(f)
    phi = h[inst.src] - h[inst.col] - psi[:, None]
    used = f > 1e-9 * inst.d[None, :]
    assert np.abs(phi[used]).max() <= 1e-5
    assert phi[~used].max() <= 1e-5


# --------------------------------------------------------------------------- verdicts vs independent solvers


def _lp_max_concurrent(inst):
    """Largest lambda with lambda*d routable within u (eq. (1) as an LP, scipy HiGHS)."""
    from scipy.optimize import linprog
    from scipy.sparse import coo_matrix, vstack, hstack

    m, K, n = inst.m, inst.K, inst.n
    nv = m * K + 1  # flows f[e, k] at e*K + k, then lambda
    # conservation: out - in - lambda * hat(d) = 0 for every (i, k)
    rows, cols, vals = [], [], []
    for e in range(m):
        for k in range(K):
            rows += [inst.src[e] * K + k, inst.col[e] * K + k]
            cols += [e * K + k, e * K + k]
            vals += [1.0, -1.0]
    for k in range(K):
        rows += [inst.s[k] * K + k, inst.t[k] * K + k]
        cols += [m * K, m * K]
        vals += [-inst.d[k], inst.d[k]]
    A_eq = coo_matrix((vals, (rows, cols)), shape=(n * K, nv))
    cap = coo_matrix((np.ones(m * K), (np.repeat(np.arange(m), K), np.arange(m * K))), shape=(m, nv))
    c = np.zeros(nv)
    c[-1] = -1.0
    res = linprog(c, A_ub=cap, b_ub=inst.u, A_eq=A_eq, b_eq=np.zeros(n * K),
                  bounds=[(0, None)] * (m * K) + [(0, 10.0)], method="highs")
    assert res.status == 0
    return -res.fun


@pytest.mark.slow
def test_verdicts_agree_with_lp():
    """Oracle verdicts on small random instances match an LP (scipy HiGHS) away from the boundary."""
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
            f, rep = P.solve_eso(max_sweeps=400000, eps_obj=0.0, resid_tol=1e-6)
            v = P.residuals(f)["verdict"]
            if v == oracle.VERDICT_UNKNOWN:
                f, rep = P.solve_eso(max_sweeps=400000, eps_obj=1e-15, f0=f)
                v = P.residuals(f)["verdict"]
            expect = oracle.VERDICT_FEASIBLE if lam >= 1.0 else oracle.VERDICT_INFEASIBLE
            assert v == expect, (seed, factor, lam, rep)
            checked += 1
    assert checked >= 12


def test_single_commodity_verdict_matches_max_flow():
    """K = 1: eq. (1) is feasible iff max-flow(s, t) >= d (integer capacities, scipy)."""
    from scipy.sparse import csr_matrix
    from scipy.sparse.csgraph import maximum_flow

    for seed in range(6):
        rng = np.random.default_rng(2000 + seed)
        n, row_ptr, col = I.random_digraph(7, 3, rng)
        m = col.shape[0]
        u = rng.integers(0, 4, size=m).astype(np.float64)
        src = np.repeat(np.arange(n), np.diff(row_ptr))
        cap = csr_matrix((u.astype(np.int32), (src, col)), shape=(n, n))  # parallel arcs summed
        s, t = 0, n - 1
        mf = maximum_flow(cap, s, t).flow_value
        for d in (max(1, mf - 1), mf + 1):
            if d == mf:
                continue
            P = oracle.Problem(n, row_ptr, col, u, [s], [t], [float(d)])
            f, rep = P.solve_eso(max_sweeps=400000, eps_obj=0.0, resid_tol=1e-6)
            v = P.residuals(f)["verdict"]
            if v == oracle.VERDICT_UNKNOWN:
                f, rep = P.solve_eso(max_sweeps=400000, eps_obj=1e-15, f0=f)
                v = P.residuals(f)["verdict"]
            expect = oracle.VERDICT_FEASIBLE if d <= mf else oracle.VERDICT_INFEASIBLE
            assert v == expect, (seed, d, mf, rep)


def test_isolated_endpoint_is_infeasible():
    # vertex 2 has no edges; commodity 0 -> 2
    P = oracle.Problem(3, [0, 1, 2, 2], [1, 0], [5.0, 5.0], [0], [2], [1.0])
    res = P.residuals(np.zeros((2, 1)))
    assert res["isolated"] == 1 and res["verdict"] == oracle.VERDICT_INFEASIBLE


def test_results_do_not_depend_on_thread_count(knn2500):
    P = oracle.Problem.from_instance(knn2500)
    rng = np.random.default_rng(5)
    f = rng.exponential(0.2, (knn2500.m, knn2500.K)) * (rng.random((knn2500.m, knn2500.K)) < 0.1)
    prev = oracle.set_threads(1)
    a = P.sweep(f)
    oracle.set_threads(4)
    b = P.sweep(f)
    oracle.set_threads(prev)
    np.testing.assert_array_equal(a, b)


# --------------------------------------------------------------------------- per-vertex / per-edge helpers


def test_excess_vertex_and_congestion_edge_equal_full_passes(knn2500):
    """The per-vertex excess (eq. (3), (3h), (2)) and per-edge congestion (eq. (41))
    helpers, which check the sampled full-size GPU sweeps, equal the rows of the
    full passes bit for bit on knn2500_k500 with random flows (same summation
    order), read through a compact row store with the rows shuffled."""
    inst = knn2500
    P = oracle.Problem.from_instance(inst)
    rng = np.random.default_rng(11)
    f = rng.exponential(1.0, (inst.m, inst.K)) * (rng.random((inst.m, inst.K)) < 0.3)
    Delta, h = P.excess(f)
    psi = P.congestion(f)
    perm = rng.permutation(inst.m)
    row_of_edge = np.empty(inst.m, dtype=np.int64)
    row_of_edge[perm] = np.arange(inst.m)
    rows = f[perm]
    for i in range(inst.n):
        D_i, h_i = P.excess_vertex(i, row_of_edge, rows)
        np.testing.assert_array_equal(D_i, Delta[i])
        np.testing.assert_array_equal(h_i, h[i])
    for e in range(inst.m):
        assert oracle.congestion_edge(f[e], inst.u[e]) == psi[e]
    # a missing incident row is reported, not read
    row_of_edge[int(inst.row_ptr[7])] = -1
    with pytest.raises(ValueError):
        P.excess_vertex(7, row_of_edge, rows)
