"""Pins for the oracle's Alg. 3 (PDR-AGD) and Alg. 4 (PDR-GDM).

Hand-derived single steps, the local objective change against a direct
evaluation of eq. (9), the Section 4 majorise-minimise argument (every
accepted edge step lowers the surrogate, so AGD's z never rises), GDM with
gamma = 0 reducing exactly to AGD, and verdicts on the capacity twins.
"""

import os

import numpy as np
import pytest

import oracle
from paper_2108_07549_gb300 import instances as I


def eq9_value(hi, hj, f, df, u):
    """eq. (9) with the slack r chosen optimally (r = max(0, u - sum(f + df)))."""
    tot = float(np.sum(f + df))
    over = max(0.0, tot - u)
    return 0.5 * (over ** 2 + np.sum((hi - df) ** 2) + np.sum((hj + df) ** 2))


def test_agd_hand_step_accept():
    """K = 1, h = (1, -1), psi = 0, f = 0, u = 10, beta = .25: phi = 2, step .5,
    dz = .25 - 2 * .5 = -.75 <= 0, accepted; t = 0 doubles beta to .5 (= beta_max)."""
    prm = oracle.gd_params(False, 1)
    f, v, b, acc, dz = oracle.gd_edge(prm, [1.0], [-1.0], 0.0, 10.0, [0.0], None, 0.25, 0)
    assert acc and f[0] == 0.5 and dz == -0.75 and b == 0.5


def test_agd_hand_step_reject():
    """K = 2, h_i = (2, -2), h_j = 0, f = 0, beta = 2: steps (4, 0) (the second is
    projected to -f = 0), dz = 16 - 8 = 8 > 0, rejected; beta halves to 1 (t = 1)."""
    prm = oracle.gd_params(False, 2, beta_max=4.0)
    f, v, b, acc, dz = oracle.gd_edge(prm, [2.0, -2.0], [0.0, 0.0], 0.0, 100.0, [0.0, 0.0], None, 2.0, 1)
    assert not acc and dz == 8.0 and b == 1.0
    np.testing.assert_array_equal(f, [0.0, 0.0])


def test_beta_floor_and_ceiling():
    prm = oracle.gd_params(False, 4)  # beta_min = .25
    _, _, b, acc, _ = oracle.gd_edge(prm, [2.0, -2.0, 0, 0], [0.0] * 4, 0.0, 100.0, [0.0] * 4, None, 0.3, 3)
    # a rejected step at beta .3 would give .15; the floor is 1/K = .25
    if not acc:
        assert b == 0.25
    _, _, b, _, _ = oracle.gd_edge(prm, [0.1] * 4, [0.0] * 4, 0.0, 100.0, [0.0] * 4, None, 0.4, 20)
    assert b == 0.5  # t = 20: 0.4 * 2 clamped to beta_max


@pytest.mark.parametrize("momentum", [False, True])
def test_local_objective_change_matches_eq9(momentum):
    """dz reported by the edge step equals eq. (9) at the step minus eq. (9) at zero."""
    rng = np.random.default_rng(5)
    prm = oracle.gd_params(momentum, 8, beta_max=2.0)
    for _ in range(300):
        K = 8
        hi, hj = rng.normal(0, 1, K), rng.normal(0, 1, K)
        f = np.abs(rng.normal(0, 1, K)) * (rng.random(K) < 0.7)
        u = float(rng.uniform(0, 6))
        psi = max(0.0, f.sum() - u)
        beta = float(rng.uniform(0.05, 1.5))
        df = np.maximum(-f, beta * (hi - hj - psi))
        _, _, _, acc, dz = oracle.gd_edge(prm, hi, hj, psi, u, f, None, beta, 3)
        direct = eq9_value(hi, hj, f, df, u) - eq9_value(hi, hj, f, np.zeros(K), u)
        assert abs(dz - direct) <= 1e-12 * max(1.0, abs(direct))
        assert acc == (dz <= 0.0)


def test_agd_objective_never_rises(grid5, grid5_bad):
    """Each accepted edge step lowers the edge surrogate of Section 4's proof, so
    z(f^(t+1)) <= Q <= z(f^(t)) holds for Alg. 3 as for Alg. 1."""
    for inst in (grid5, grid5_bad):
        P = oracle.Problem.from_instance(inst)
        _, _, _, rep, zt = P.solve_gd(oracle.gd_params(False, inst.K), max_sweeps=3000, eps_obj=0.0, trace=True)
        assert np.all(np.diff(zt) <= 1e-12 * zt[:-1])


def test_gdm_with_zero_momentum_is_agd(grid5):
    """Alg. 4 with gamma = 0: v = Delta f and max(0, f + Delta f) = f + Delta f, i.e. Alg. 3."""
    P = oracle.Problem.from_instance(grid5)
    base = oracle.gd_params(False, grid5.K)
    agd = P.solve_gd(base, max_sweeps=700, eps_obj=0.0)
    gdm = P.solve_gd(dict(base, momentum=1, gamma=0.0), max_sweeps=700, eps_obj=0.0)
    np.testing.assert_array_equal(agd[0], gdm[0])
    np.testing.assert_array_equal(agd[2], gdm[2])


def test_gd_sweep_matches_solve(grid5):
    """The one-sweep helper and the solve loop take the same steps."""
    P = oracle.Problem.from_instance(grid5)
    prm = oracle.gd_params(True, grid5.K)
    f = np.zeros((grid5.m, grid5.K))
    v = np.zeros_like(f)
    b = np.full(grid5.m, prm["beta_init"])
    for t in range(25):
        f, v, b = P.gd_sweep(prm, f, v, b, t)
    f2, v2, b2, rep = P.solve_gd(prm, max_sweeps=25, eps_obj=0.0)
    np.testing.assert_allclose(f, f2, rtol=0, atol=1e-15)
    np.testing.assert_allclose(v, v2, rtol=0, atol=1e-15)
    np.testing.assert_array_equal(b, b2)


@pytest.mark.parametrize("momentum", [False, True])
def test_gd_verdicts_on_twins(grid5, grid5_bad, momentum):
    """Both heuristics reach the same verdicts as Alg. 1 on the capacity twins."""
    prm_ok = oracle.gd_params(momentum, grid5.K)
    P = oracle.Problem.from_instance(grid5)
    f, v, b, rep = P.solve_gd(prm_ok, max_sweeps=200000, eps_obj=0.0, resid_tol=1e-6)
    assert rep["stop_reason"] == 2 and P.residuals(f)["verdict"] == oracle.VERDICT_FEASIBLE
    Q = oracle.Problem.from_instance(grid5_bad)
    f, v, b, rep = Q.solve_gd(prm_ok, max_sweeps=200000, eps_obj=1e-12)
    res = Q.residuals(f)
    assert res["verdict"] == oracle.VERDICT_INFEASIBLE and abs(res["margin"] - 2 * res["z"]) <= 1e-3 * res["z"]


# --------------------------------------------------------------------------- Alg. 4 momentum step by hand


def test_gdm_hand_step_accept_with_clamp():
    """Alg. 4, K = 2, gamma = .9, v = (-2, .3), f = (1, .5), h_i = (1, .2), h_j = 0,
    psi = 0, u = 10, beta = .5, t = 3 (no periodic increase):
      phi = (1, .2), df = (.5, .1), psi' = 0, dz = (.25 - .5) + (.01 - .02) = -.26 -> accepted;
      v' = (.9 * -2 + .5, .9 * .3 + .1) = (-1.3, .37);
      f' = (max(0, 1 - 1.3), max(0, .5 + .37)) = (0, .87).
    The velocity keeps its negative entry (only f is projected).  Wrong readings fail:
    max(0, f + df) + gamma v gives f'_0 = -.3; no projection gives -.3;
    v' = gamma (v + df) gives f'_1 = .86."""
    prm = oracle.gd_params(True, 2, gamma=0.9, beta_min=0.05, beta_max=1.0)
    f, v, b, acc, dz = oracle.gd_edge(prm, [1.0, 0.2], [0.0, 0.0], 0.0, 10.0, [1.0, 0.5], [-2.0, 0.3], 0.5, 3)
    assert acc and abs(dz - (-0.26)) < 1e-15 and b == 0.5
    np.testing.assert_allclose(v, [-1.3, 0.37], rtol=0, atol=1e-15)
    np.testing.assert_allclose(f, [0.0, 0.87], rtol=0, atol=1e-15)
    assert f[0] == 0.0


def test_gdm_hand_step_reject_keeps_velocity():
    """Alg. 4, K = 2, rejected step: f = (1, .5), v = (-2, .3), h_i = (2, -2), h_j = 0,
    psi = 0, u = 100, beta = 2, t = 1: phi = (2, -2), df = (max(-1, 4), max(-.5, -4)) = (4, -.5),
    dz = (16 - 8) + (.25 - 1) = 7.25 > 0 -> f and v unchanged, beta = max(beta_min, 2 * .5) = 1."""
    prm = oracle.gd_params(True, 2, gamma=0.9, beta_min=0.05, beta_max=4.0)
    f, v, b, acc, dz = oracle.gd_edge(prm, [2.0, -2.0], [0.0, 0.0], 0.0, 100.0, [1.0, 0.5], [-2.0, 0.3], 2.0, 1)
    assert not acc and dz == 7.25 and b == 1.0
    np.testing.assert_array_equal(f, [1.0, 0.5])
    np.testing.assert_array_equal(v, [-2.0, 0.3])


def test_gdm_golden_trace():
    """tests/golden/two_vertex_k1_gdm.txt: three iterations of Alg. 4 derived by hand in
    exact dyadic rationals (so the FP64 oracle must reproduce them exactly), including
    the momentum overshoot that makes z rise."""
    from fractions import Fraction as Fr

    g = {}
    path = os.path.join(os.path.dirname(__file__), "golden", "two_vertex_k1_gdm.txt")
    for line in open(path):
        line = line.strip()
        if line and not line.startswith("#"):
            key, val = line.split(":", 1)
            g[key.strip()] = [float(Fr(x)) for x in val.split()]
    P = oracle.Problem(2, [int(x) for x in g["row_ptr"]], [int(x) for x in g["col"]], g["u"],
                       [int(x) for x in g["s"]], [int(x) for x in g["t"]], g["d"])
    b0, bmin, bmax, ainc, adec, gamma = g["params"]
    prm = dict(momentum=1, beta_init=b0, beta_min=bmin, beta_max=bmax, alpha_inc=ainc, alpha_dec=adec, gamma=gamma)
    f = np.zeros((2, 1))
    v = np.zeros((2, 1))
    beta = np.full(2, b0)
    for t in range(3):
        f, v, beta = P.gd_sweep(prm, f, v, beta, t)
        np.testing.assert_array_equal(f[:, 0], g[f"f{t + 1}"])
        np.testing.assert_array_equal(v[:, 0], g[f"v{t + 1}"])
    np.testing.assert_array_equal(beta, g["beta3"])
    f3, v3, beta3, rep, zt = P.solve_gd(prm, max_sweeps=3, eps_obj=0.0, trace=True)
    np.testing.assert_array_equal(zt, g["z"])
    np.testing.assert_array_equal(f3[:, 0], g["f3"])
    np.testing.assert_array_equal(v3[:, 0], g["v3"])
    np.testing.assert_array_equal(beta3, g["beta3"])
