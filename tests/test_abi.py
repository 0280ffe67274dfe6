"""CPU-side checks of the C ABI: the library loads, exports every declared entry
point, and rejects invalid instances before touching the GPU."""

import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2108_07549_gb300 import build, pdr

    build.build()
    return pdr.load()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "pdr.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pdr_[a-z_0-9]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(lib):
    from paper_2108_07549_gb300 import pdr

    names = declared_functions()
    assert len(names) >= 18
    for name in names:
        assert hasattr(lib, name), name
    assert sorted(pdr.EXPORTS) == names


def test_default_options(lib):
    from paper_2108_07549_gb300 import pdr

    o = pdr.default_options()
    assert o.precision == pdr.PREC_FP32 and o.use_graph == 1
    assert o.eps_obj == 1e-6 and o.resid_tol == 1e-6 and o.eps_rel == 0.0
    assert o.max_sweeps == 1000000 and o.trace_len == 0
    assert o.algo == pdr.ALGO_ESO and o.beta_init == 0.0 and o.gamma == -1.0
    assert o.edge_variant == -1
    assert lib.pdr_default_options(None) == 1


def _create(lib, n, row_ptr, col, u, s, t, d, opt=None):
    a = [np.ascontiguousarray(x, dt) for x, dt in ((row_ptr, np.int64), (col, np.int32), (u, np.float64),
                                                    (s, np.int32), (t, np.int32), (d, np.float64))]
    p = [x.ctypes.data_as(C.c_void_p) for x in a]
    h = C.c_void_p()
    st = lib.pdr_create(n, len(a[1]), p[0], p[1], p[2], len(a[3]), p[3], p[4], p[5], opt, None, C.byref(h))
    return st, lib.pdr_last_error(None).decode(), h


BASE = dict(n=3, row_ptr=[0, 1, 2, 3], col=[1, 2, 0], u=[1.0, 1.0, 1.0], s=[0], t=[2], d=[1.0])


@pytest.mark.parametrize("change, needle", [
    (dict(n=0, row_ptr=[0]), "n must be"),
    (dict(row_ptr=[1, 1, 2, 3]), "row_ptr[0]"),
    (dict(row_ptr=[0, 2, 1, 3]), "non-decreasing"),
    (dict(row_ptr=[0, 1, 2, 2]), "row_ptr[n]"),
    (dict(col=[1, 3, 0]), "col out of range"),
    (dict(col=[1, 1, 0]), "self-loop"),
    (dict(u=[1.0, -1.0, 1.0]), "capacity"),
    (dict(u=[1.0, float("nan"), 1.0]), "capacity"),
    (dict(s=[0], t=[0]), "s_k == t_k"),
    (dict(s=[5]), "out of range"),
    (dict(d=[0.0]), "demand"),
    (dict(d=[float("inf")]), "demand"),
    (dict(s=[], t=[], d=[]), "K must be"),
])
def test_create_rejects_invalid_instances(lib, change, needle):
    """eq. (1) domain: u >= 0, s_k != t_k, d_k > 0, a well-formed CSR without self-loops."""
    args = dict(BASE)
    args.update(change)
    st, msg, h = _create(lib, **args)
    assert st == 1 and needle in msg, (st, msg)
    assert not h.value


def test_create_rejects_bad_options(lib):
    from paper_2108_07549_gb300 import pdr

    o = pdr.default_options(precision=7)
    st, msg, _ = _create(lib, **BASE, opt=C.byref(o))
    assert st == 1 and "precision" in msg
    o = pdr.default_options(max_sweeps=-1)
    st, msg, _ = _create(lib, **BASE, opt=C.byref(o))
    assert st == 1 and "max_sweeps" in msg
    o = pdr.default_options(algo=4)
    st, msg, _ = _create(lib, **BASE, opt=C.byref(o))
    assert st == 1 and "algo" in msg
    o = pdr.default_options(algo=2, gamma=1.5)
    st, msg, _ = _create(lib, **BASE, opt=C.byref(o))
    assert st == 1 and "gamma" in msg
    for v in (-2, lib.pdr_num_edge_variants()):
        o = pdr.default_options(edge_variant=v)
        st, msg, _ = _create(lib, **BASE, opt=C.byref(o))
        assert st == 1 and "edge_variant" in msg
    for v in (-2, 6):
        o = pdr.default_options(excess_variant=v)
        st, msg, _ = _create(lib, **BASE, opt=C.byref(o))
        assert st == 1 and "excess_variant" in msg
    assert pdr.default_options().excess_variant == -1


def test_edge_variant_table(lib):
    """Every variant holds a whole number of vectors per lane (4 floats or 2
    doubles), the plain forms come in ascending capacity, and each pipelined
    form has a plain form of the same capacity."""
    from paper_2108_07549_gb300 import pdr

    t32, t64 = pdr.edge_variants(pdr.PREC_FP32), pdr.edge_variants(pdr.PREC_FP64)
    assert len(t32) == lib.pdr_num_edge_variants() >= 14
    plain = [c for _, c, p in t32 if not p]
    assert plain == sorted(plain) and plain[0] == 16 and plain[-1] == 32768
    for (v, c32, p32), (_, c64, p64) in zip(t32, t64):
        assert c32 == 2 * c64 and c32 % 16 == 0 and p32 == p64
        if p32:
            assert c32 in plain
    pipe = C.c_int32(7)
    assert lib.pdr_edge_variant_capacity(-1, 0, C.byref(pipe)) == -1 and pipe.value == 7
    assert lib.pdr_edge_variant_capacity(0, 2, None) == -1


def test_null_context_calls_fail_cleanly(lib):
    assert lib.pdr_solve(None, None) == 1
    assert lib.pdr_sweeps(None, 1) == 1
    assert lib.pdr_reset(None) == 1
    assert lib.pdr_state_size(None, None) == 1
    assert lib.pdr_get_state(None, None, 0) == 1
    assert lib.pdr_set_state(None, None, 0) == 1
    assert lib.pdr_debug_wait(None, 10_000, 0) == 1
    assert lib.pdr_debug_barrier(None, 1_000_000, 0) == 1
    assert lib.pdr_time_sweeps(None, 1, None, None) == 1
    assert lib.pdr_debug_fail_alloc(-1) == 1
    assert lib.pdr_debug_fail_alloc(0) == 0
    lib.pdr_destroy(None)


def test_batch_create_rejects_invalid_instances(lib):
    from paper_2108_07549_gb300 import pdr

    good = pdr.InstanceC(3, 1, 3, *(x.ctypes.data_as(C.c_void_p) for x in _BASE_ARRAYS))
    bad = pdr.InstanceC(3, 1, 3, *(x.ctypes.data_as(C.c_void_p) for x in _BAD_ARRAYS))
    arr = (pdr.InstanceC * 2)(good, bad)
    h = C.c_void_p()
    assert lib.pdr_batch_create(0, arr, None, None, C.byref(h)) == 1
    assert lib.pdr_batch_create(2, arr, None, None, C.byref(h)) == 1
    assert "instance 1" in lib.pdr_last_error(None).decode() and "self-loop" in lib.pdr_last_error(None).decode()
    o = pdr.default_options(precision=7)
    assert lib.pdr_batch_create(1, arr, C.byref(o), None, C.byref(h)) == 1
    assert "precision" in lib.pdr_last_error(None).decode()
    assert not h.value


_BASE_ARRAYS = [np.array([0, 1, 2, 3], np.int64), np.array([1, 2, 0], np.int32), np.ones(3),
                np.array([0], np.int32), np.array([2], np.int32), np.ones(1)]
_BAD_ARRAYS = [np.array([0, 1, 2, 3], np.int64), np.array([1, 2, 2], np.int32), np.ones(3),
               np.array([0], np.int32), np.array([2], np.int32), np.ones(1)]
