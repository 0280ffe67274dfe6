"""Pins for the oracle's reverse mode through T unrolled sweeps of Alg. 1.

L(u, d) = z(f^(T)) with f^(0) = 0.  Pinned by FP64 central finite differences
of the oracle's own forward (a different computation from the reverse pass),
by the closed form at T = 0, and by Euler's identity: every step of Alg. 1
(the linear excess and heights, max(0, .), the root of Alg. 2) is positively
homogeneous of degree 1 in (f, u, d), so f^(T) is, and z is homogeneous of
degree 2: u . dL/du + d . dL/dd = 2 L.
"""

import numpy as np
import pytest

import oracle
from paper_2108_07549_gb300 import instances as I


def problem(inst, u=None, d=None):
    return oracle.Problem(inst.n, inst.row_ptr, inst.col, inst.u if u is None else u, inst.s, inst.t,
                          inst.d if d is None else d)


def cases():
    rng = np.random.default_rng(21)
    return [I.grid5_k10(1.0), I.grid5_k10(1.0).with_factor(0.6),
            I.make_instance("dg25_k7", I.random_digraph(25, 3, rng), 7, ("uniform_int", 1, 9), 0.9, rng)]


def objective_at(inst, T, which, idx, delta, ck=False):
    if which == "u":
        u = inst.u.copy()
        u[idx] += delta
        P = problem(inst, u=u)
    else:
        d = inst.d.copy()
        d[idx] += delta
        P = problem(inst, d=d)
    return P.unrolled_objective_ck(T) if ck else P.unrolled_objective(T)


def check_derivative(inst, T, which, idx, g, ck=False):
    """At a smooth point g must equal the central difference; where L has a
    kink exactly at the point (max(0, .) or an active-set boundary of Alg. 2
    hit exactly, which integer data make common), the one-sided derivatives
    differ and g must equal one of them.  Returns 1 if checked."""
    h = 1e-5
    L = [objective_at(inst, T, which, idx, q * h, ck) for q in (-2, -1, 0, 1, 2)]
    # second-order one-sided differences: exact for quadratics, O(h^2) otherwise
    right = (-3 * L[2] + 4 * L[3] - L[4]) / (2 * h)
    left = (3 * L[2] - 4 * L[1] + L[0]) / (2 * h)
    scale = max(1.0, abs(left), abs(right))
    if abs(right - left) <= 1e-8 * scale:
        central = (L[3] - L[1]) / (2 * h)
        assert abs(g - central) <= 1e-7 * scale, (inst.name, T, which, idx, g, central)
    else:
        assert min(abs(g - left), abs(g - right)) <= 1e-7 * scale, (inst.name, T, which, idx, g, left, right)
    return 1


@pytest.mark.parametrize("T", [1, 5, 20])
def test_adjoint_matches_finite_differences(T):
    checked = 0
    for inst in cases():
        L, gu, gd = problem(inst).adjoint_eso(T)
        for k in range(inst.K):
            checked += check_derivative(inst, T, "d", k, gd[k])
        for e in np.nonzero(inst.u > 0)[0][:12]:
            checked += check_derivative(inst, T, "u", e, gu[e])
    assert checked >= 40


def test_adjoint_at_zero_sweeps_closed_form():
    """T = 0: L = 1/2 sum_k d_k^2 (1/delta_s + 1/delta_t), dL/dd_k = d_k (1/delta_s + 1/delta_t), dL/du = 0."""
    inst = cases()[2]
    P = problem(inst)
    L, gu, gd = P.adjoint_eso(0)
    w = 1.0 / P.deg[inst.s] + 1.0 / P.deg[inst.t]
    assert abs(L - 0.5 * np.sum(inst.d ** 2 * w)) <= 1e-13 * L
    np.testing.assert_allclose(gd, inst.d * w, rtol=1e-14)
    assert np.all(gu == 0.0)


@pytest.mark.parametrize("T", [3, 30])
def test_euler_identity_degree_two(T):
    for inst in cases():
        L, gu, gd = problem(inst).adjoint_eso(T)
        lhs = float(np.dot(inst.u, gu) + np.dot(inst.d, gd))
        assert abs(lhs - 2 * L) <= 1e-10 * max(1.0, L), (inst.name, T, lhs, 2 * L)


def test_forward_of_adjoint_is_the_solver():
    """The L of the reverse pass equals z after T sweeps of the ordinary solve."""
    inst = cases()[0]
    P = problem(inst)
    L, _, _ = P.adjoint_eso(25)
    f, rep = P.solve_eso(max_sweeps=25, eps_obj=0.0)
    assert rep["sweeps"] == 25 and abs(rep["z"] - L) <= 1e-14 * L
    assert abs(P.unrolled_objective(25) - L) <= 1e-14 * L


@pytest.mark.parametrize("T", [1, 6, 20])
def test_capacity_kept_adjoint_matches_finite_differences(T):
    """The same checks through T sweeps of the capacity-kept step (Program (6))."""
    checked = 0
    for inst in cases():
        L, gu, gd = problem(inst).adjoint_ck(T)
        assert abs(L - problem(inst).unrolled_objective_ck(T)) <= 1e-14 * L
        for k in range(inst.K):
            checked += check_derivative(inst, T, "d", k, gd[k], ck=True)
        for e in np.nonzero(inst.u > 0)[0][:12]:
            checked += check_derivative(inst, T, "u", e, gu[e], ck=True)
    assert checked >= 40


def test_capacity_kept_adjoint_euler_identity():
    """The capacity-kept step is positively homogeneous of degree 1 in (f, u, d)
    as well, so u . dL/du + d . dL/dd = 2 L."""
    for inst in cases():
        L, gu, gd = problem(inst).adjoint_ck(25)
        assert abs(np.dot(inst.u, gu) + np.dot(inst.d, gd) - 2 * L) <= 1e-10 * max(1.0, L)
