"""GPU reverse mode (pdr_backward) against the oracle's reverse mode and FP64
finite differences.

The instances get non-integer capacities and demands so that exact ties (the
kinks of max(0, .) and of Alg. 2's active sets, which integer data make
common) are unlikely.  The FP32 gradients are compared element by element,
at 1e-4 relative to the element, with an absolute floor of 1e-6 of the
largest entry (entries that small are sums of rounding-size terms in FP32).
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


def jittered(inst, seed):
    rng = np.random.default_rng(seed)
    return I.Instance(inst.name + "~", inst.n, inst.row_ptr, inst.col, inst.u * rng.uniform(0.9, 1.1, inst.m),
                      inst.s, inst.t, inst.d * rng.uniform(0.9, 1.1, inst.K), inst.factor, inst.load, inst.hops)


def cases():
    rng = np.random.default_rng(21)
    return [jittered(I.grid5_k10(1.0), 1), jittered(I.grid5_k10(0.6), 2),
            jittered(I.make_instance("dg40_k9", I.random_digraph(40, 3, rng), 9, ("uniform_int", 1, 9), 0.9, rng), 3),
            jittered(I.make_instance("grid6_k33", I.grid_graph(6), 33, ("lognormal", 1.0, 0.5), 1.1, rng), 4)]


@pytest.mark.parametrize("T,ckpt", [(0, 1), (1, 1), (7, 3), (20, 10), (25, 25)])
def test_fp64_reverse_mode_matches_oracle(pdr, T, ckpt):
    for inst in cases():
        Lr, gur, gdr = oracle.Problem.from_instance(inst).adjoint_eso(T)
        with pdr.Solver.from_instance(inst, precision=pdr.PREC_FP64) as s:
            L, gu, gd = s.backward(T, ckpt)
        assert abs(L - Lr) <= 1e-12 * Lr
        np.testing.assert_allclose(gd, gdr, rtol=1e-9, atol=1e-12 * np.abs(gdr).max())
        np.testing.assert_allclose(gu, gur, rtol=1e-9, atol=1e-12 * max(1.0, np.abs(gur).max()))


def elementwise_close(g, gr, rel=1e-4, floor=1e-6):
    """|g - gr| <= rel |gr| + floor max |gr|, element by element; returns the worst ratio."""
    bound = rel * np.abs(gr) + floor * np.abs(gr).max()
    return float((np.abs(g - gr) / bound).max())


def test_fp32_reverse_mode_matches_fp64_oracle(pdr):
    for inst in cases():
        for T in (10, 30):
            Lr, gur, gdr = oracle.Problem.from_instance(inst).adjoint_eso(T)
            with pdr.Solver.from_instance(inst, precision=pdr.PREC_FP32) as s:
                L, gu, gd = s.backward(T, 10)
            assert abs(L - Lr) <= 1e-5 * Lr
            worst = elementwise_close(np.concatenate([gu, gd]), np.concatenate([gur, gdr]))
            assert worst <= 1.0, (inst.name, T, worst)


def test_euler_identity_on_gpu(pdr):
    """z(f^(T)) is homogeneous of degree 2 in (u, d): u . dL/du + d . dL/dd = 2 L."""
    for inst in cases():
        for prec, tol in ((pdr.PREC_FP64, 1e-10), (pdr.PREC_FP32, 1e-5)):
            with pdr.Solver.from_instance(inst, precision=prec) as s:
                L, gu, gd = s.backward(15, 4)
            assert abs(np.dot(inst.u, gu) + np.dot(inst.d, gd) - 2 * L) <= tol * max(1.0, L)


def test_backward_leaves_final_flows_and_matches_solve(pdr):
    inst = cases()[0]
    with pdr.Solver.from_instance(inst, precision=pdr.PREC_FP64, eps_obj=0.0, resid_tol=0.0, max_sweeps=12) as s:
        L, _, _ = s.backward(12, 5)
        f_back = s.flows()
        s.reset()
        r = s.solve()
        assert r["sweeps"] == 12 and abs(r["z"] - L) <= 1e-12 * L
        np.testing.assert_array_equal(s.flows(), f_back)


def test_set_data_and_errors(pdr):
    inst = cases()[2]
    with pdr.Solver.from_instance(inst, precision=pdr.PREC_FP64) as s:
        L0, _, _ = s.backward(5, 2, grads=False)
        s.set_data(u=inst.u * 2.0, d=inst.d * 2.0)
        L1, _, _ = s.backward(5, 2, grads=False)
        assert abs(L1 - 4.0 * L0) <= 1e-11 * L1  # degree-2 homogeneity again
        with pytest.raises(pdr.PdrError):
            s.set_data(u=-inst.u)
        with pytest.raises(pdr.PdrError):
            s.backward(-1, 2)
    with pdr.Solver.from_instance(inst, algo=pdr.ALGO_AGD) as s:
        with pytest.raises(pdr.PdrError):
            s.backward(3, 1)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_capacity_kept_reverse_mode_matches_oracle(pdr, prec):
    """pdr_backward through capacity-kept sweeps (Program (6)) against the
    oracle's reverse mode: FP64 to 1e-9, FP32 to 1e-4 element by element."""
    p = pdr.PREC_FP64 if prec == "fp64" else pdr.PREC_FP32
    for inst in cases():
        Lr, gur, gdr = oracle.Problem.from_instance(inst).adjoint_ck(20)
        with pdr.Solver.from_instance(inst, precision=p, algo=pdr.ALGO_CK) as s:
            L, gu, gd = s.backward(20, 6)
        if prec == "fp64":
            assert abs(L - Lr) <= 1e-12 * Lr
            np.testing.assert_allclose(gd, gdr, rtol=1e-9, atol=1e-12 * np.abs(gdr).max())
            np.testing.assert_allclose(gu, gur, rtol=1e-9, atol=1e-12 * max(1.0, np.abs(gur).max()))
        else:
            assert abs(L - Lr) <= 1e-5 * Lr
            worst = elementwise_close(np.concatenate([gu, gd]), np.concatenate([gur, gdr]))
            assert worst <= 1.0, (inst.name, worst)


def test_kept_workspace_gives_the_same_gradients(pdr):
    """The context keeps the reverse-mode workspace between calls: a second
    call reuses it, a call with another T and checkpoint interval reuses
    what fits and grows the rest, and each gives the gradients of a fresh
    context bit for bit."""
    inst = block_cases()[0]
    with pdr.Solver.from_instance(inst, precision=pdr.PREC_FP32) as s:
        first = s.backward(9, 4)
        again = s.backward(9, 4)
        other = s.backward(13, 3)
    with pdr.Solver.from_instance(inst, precision=pdr.PREC_FP32) as s:
        fresh = s.backward(13, 3)
    for a, b in ((first, again), (other, fresh)):
        assert a[0] == b[0]
        np.testing.assert_array_equal(a[1], b[1])
        np.testing.assert_array_equal(a[2], b[2])


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("algo", ["eso", "ck"])
def test_keep_every_sweep_equals_checkpointed(pdr, prec, algo):
    """ckpt_every = 1 keeps every sweep of the forward pass instead of
    recomputing segments; the gradients are the checkpointed ones bit for
    bit (the recomputation is deterministic), also for T = 0 and T = 1, for
    Alg. 2 and for the capacity-kept step of Program (6)."""
    p = pdr.PREC_FP64 if prec == "fp64" else pdr.PREC_FP32
    alg = pdr.ALGO_ESO if algo == "eso" else pdr.ALGO_CK
    for inst in (cases()[2], block_cases()[1]):
        for T, C in ((0, 3), (1, 3), (11, 4)):
            with pdr.Solver.from_instance(inst, precision=p, algo=alg) as s:
                a = s.backward(T, C)
                fa = s.flows()
                b = s.backward(T, 1)
                fb = s.flows()
            assert a[0] == b[0], (inst.name, T)
            np.testing.assert_array_equal(a[1], b[1])
            np.testing.assert_array_equal(a[2], b[2])
            np.testing.assert_array_equal(fa, fb)


def block_cases():
    """Rows long enough for the block form of the backward edge step (more
    than 64 vectors of the row): K = 601 (ragged: padded to 604) takes the
    128 x 2 form in FP32 and 128 x 4 in FP64; K = 1500 takes 128 x 4 and
    256 x 4."""
    rng = np.random.default_rng(23)
    return [jittered(I.make_instance("grid6_k601", I.grid_graph(6), 601, ("lognormal", 1.0, 0.5), 1.1, rng), 5),
            jittered(I.make_instance("dg60_k1500", I.random_digraph(60, 3, rng), 1500, ("uniform_int", 1, 9), 0.9,
                                     rng), 6)]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("algo", ["eso", "ck"])
def test_block_form_reverse_mode_matches_oracle(pdr, prec, algo):
    """The block form against the oracle's reverse mode (Alg. 2 and Program
    (6)): FP64 to 1e-9, FP32 to 1e-4 element by element."""
    p = pdr.PREC_FP64 if prec == "fp64" else pdr.PREC_FP32
    for inst in block_cases():
        ref = oracle.Problem.from_instance(inst)
        Lr, gur, gdr = ref.adjoint_eso(12) if algo == "eso" else ref.adjoint_ck(12)
        with pdr.Solver.from_instance(inst, precision=p, algo=pdr.ALGO_ESO if algo == "eso" else pdr.ALGO_CK) as s:
            L, gu, gd = s.backward(12, 5)
        if prec == "fp64":
            assert abs(L - Lr) <= 1e-12 * Lr
            np.testing.assert_allclose(gd, gdr, rtol=1e-9, atol=1e-12 * np.abs(gdr).max())
            np.testing.assert_allclose(gu, gur, rtol=1e-9, atol=1e-12 * max(1.0, np.abs(gur).max()))
        else:
            assert abs(L - Lr) <= 1e-5 * Lr
            worst = elementwise_close(np.concatenate([gu, gd]), np.concatenate([gur, gdr]))
            assert worst <= 1.0, (inst.name, worst)


def test_torch_autograd_function(pdr):
    import torch

    from paper_2108_07549_gb300.autograd import unrolled_objective

    inst = cases()[3]
    Lr, gur, gdr = oracle.Problem.from_instance(inst).adjoint_eso(10)
    with pdr.Solver.from_instance(inst, precision=pdr.PREC_FP64) as s:
        u = torch.tensor(inst.u, dtype=torch.float64, requires_grad=True)
        d = torch.tensor(inst.d, dtype=torch.float64, requires_grad=True)
        L = unrolled_objective(s, u, d, T=10, ckpt_every=3)
        (3.0 * L).backward()
    assert abs(float(L.detach()) - Lr) <= 1e-12 * Lr
    np.testing.assert_allclose(u.grad.numpy(), 3.0 * gur, rtol=1e-9, atol=1e-12 * max(1.0, np.abs(gur).max()))
    np.testing.assert_allclose(d.grad.numpy(), 3.0 * gdr, rtol=1e-9, atol=1e-12 * np.abs(gdr).max())


def test_torch_autograd_on_the_device(pdr):
    """CUDA tensors: u and d enter as device pointers (pdr_set_data on the
    device) and the gradients come back as device tensors, equal to the FP64
    oracle's reverse mode; the device and host set_data paths give the same
    objective bit for bit; out-of-domain device data is rejected."""
    import torch

    from paper_2108_07549_gb300.autograd import unrolled_objective

    inst = cases()[3]
    Lr, gur, gdr = oracle.Problem.from_instance(inst).adjoint_eso(10)
    with pdr.Solver.from_instance(inst, precision=pdr.PREC_FP64) as s:
        u = torch.tensor(inst.u, dtype=torch.float64, device="cuda", requires_grad=True)
        d = torch.tensor(inst.d, dtype=torch.float64, device="cuda", requires_grad=True)
        L = unrolled_objective(s, u, d, T=10, ckpt_every=3)
        (2.0 * L).backward()
        assert u.grad.is_cuda and d.grad.is_cuda
        assert abs(float(L.detach()) - Lr) <= 1e-12 * Lr
        np.testing.assert_allclose(u.grad.cpu().numpy(), 2.0 * gur, rtol=1e-9,
                                   atol=1e-12 * max(1.0, np.abs(gur).max()))
        np.testing.assert_allclose(d.grad.cpu().numpy(), 2.0 * gdr, rtol=1e-9, atol=1e-12 * np.abs(gdr).max())
        # device and host paths of pdr_set_data agree bit for bit
        u2 = inst.u * 1.25
        s.set_data_device(torch.tensor(u2, dtype=torch.float64, device="cuda").data_ptr(), 0)
        torch.cuda.synchronize()
        L_dev = s.backward(7, 3, grads=False)[0]
        s.set_data(u=u2)
        L_host = s.backward(7, 3, grads=False)[0]
        assert L_dev == L_host
        bad = torch.tensor(-inst.u, dtype=torch.float64, device="cuda")
        with pytest.raises(pdr.PdrError) as e:
            s.set_data_device(bad.data_ptr(), 0)
        assert e.value.status == pdr.ERR_INVALID_ARG
        assert s.backward(7, 3, grads=False)[0] == L_host  # nothing changed


@pytest.mark.slow
def test_full_size_fp32_gradient_vs_fp64_finite_differences(pdr):
    """digraph20k_k2000 (n=20,000, m=100,000, K=2,000), T = 50 sweeps with
    checkpoints every 10: the FP32 reverse mode against FP64 central
    differences of the GPU's FP64 forward on 64 sampled capacities and 8
    sampled demands (1e-3 relative)."""
    inst = I.digraph20k_k2000(1.05, seed=0)
    T = 50
    with pdr.Solver.from_instance(inst, precision=pdr.PREC_FP32) as s32:
        L32, gu, gd = s32.backward(T, 10)
    rng = np.random.default_rng(0)
    edges = rng.choice(np.nonzero(inst.u > 0)[0], 64, replace=False)
    comms = rng.choice(inst.K, 8, replace=False)
    checked = 0
    with pdr.Solver.from_instance(inst, precision=pdr.PREC_FP64) as s64:
        L64, _, _ = s64.backward(T, 10, grads=False)
        assert abs(L32 - L64) <= 1e-5 * L64

        def L_at(u, d):
            s64.set_data(u=u, d=d)
            return s64.backward(T, 10, grads=False)[0]

        for which, idx, g in [("u", e, gu[e]) for e in edges] + [("d", k, gd[k]) for k in comms]:
            base = inst.u if which == "u" else inst.d
            h = 1e-4 * base[idx]
            vals = []
            for q in (-1, 0, 1):
                if q == 0:
                    vals.append(L64)  # the unperturbed objective
                    continue
                x = base.copy()
                x[idx] += q * h
                vals.append(L_at(x, inst.d) if which == "u" else L_at(inst.u, x))
            left, right = (vals[1] - vals[0]) / h, (vals[2] - vals[1]) / h
            central = (vals[2] - vals[0]) / (2 * h)
            scale = max(abs(central), 1e-3 * abs(L64) / base[idx])
            if abs(right - left) > 1e-3 * max(abs(left), abs(right), 1e-12):
                continue  # a kink inside the stencil
            assert abs(g - central) <= 1e-3 * scale, (which, idx, g, central)
            checked += 1
        s64.set_data(u=inst.u, d=inst.d)
    assert checked >= 56
