"""FP64 CPU oracle for PDR -- test infrastructure only.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline /
reference arm may import this package.  It is independent of the CUDA path:
it shares no code with ``paper_2108_07549_gb300`` and imports nothing from it.

``pdr_oracle.c`` holds the arithmetic (plain C, double precision, no FMA
contraction); this module compiles it with gcc on first use and wraps it with
ctypes.  Every wrapper names the passage of the paper (arXiv 2108.07549) that
its C function follows.

Parity status: every function here is pinned by ``tests/test_oracle.py``
against brute force, closed forms, invariants, an LP and a max-flow solver;
none is "parity unpinned".
"""

from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pdr_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

VERDICT_UNKNOWN, VERDICT_FEASIBLE, VERDICT_INFEASIBLE = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile ``pdr_oracle.c`` into ``liboracle.so`` (gcc, -O2, no FMA contraction, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared",
               "-std=c11", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class _Problem(C.Structure):
    _fields_ = [
        ("n", C.c_int32), ("m", C.c_int64), ("K", C.c_int32),
        ("row_ptr", C.c_void_p), ("col", C.c_void_p), ("u", C.c_void_p),
        ("s", C.c_void_p), ("t", C.c_void_p), ("d", C.c_void_p),
        ("in_ptr", C.c_void_p), ("in_eid", C.c_void_p), ("src", C.c_void_p), ("deg", C.c_void_p),
    ]


class _Residuals(C.Structure):
    _fields_ = [
        ("z", C.c_double), ("cap_abs", C.c_double), ("cap_rel", C.c_double),
        ("cons_abs", C.c_double), ("cons_rel", C.c_double), ("f_min", C.c_double),
        ("margin", C.c_double), ("margin_scale", C.c_double),
        ("verdict", C.c_int32), ("isolated", C.c_int32),
    ]


class _Options(C.Structure):
    _fields_ = [("max_sweeps", C.c_int64), ("eps_obj", C.c_double), ("resid_tol", C.c_double)]


class _GDParams(C.Structure):
    _fields_ = [("momentum", C.c_int32), ("pad", C.c_int32), ("beta_init", C.c_double), ("beta_min", C.c_double),
                ("beta_max", C.c_double), ("alpha_inc", C.c_double), ("alpha_dec", C.c_double),
                ("gamma", C.c_double)]


def gd_params(momentum: bool, K: int, **overrides) -> dict:
    """Section 7 parameters: AGD (Alg. 3) beta_init .25, beta_max .5; GDM (Alg. 4)
    beta_init .1, beta_max .2, gamma .9; both beta_min 1/K, alpha_inc 2, alpha_dec .5."""
    if momentum:
        p = dict(momentum=1, beta_init=0.1, beta_min=1.0 / K, beta_max=0.2, alpha_inc=2.0, alpha_dec=0.5, gamma=0.9)
    else:
        p = dict(momentum=0, beta_init=0.25, beta_min=1.0 / K, beta_max=0.5, alpha_inc=2.0, alpha_dec=0.5, gamma=0.0)
    p.update(overrides)
    return p


def _gd_struct(p: dict) -> _GDParams:
    return _GDParams(int(p["momentum"]), 0, p["beta_init"], p["beta_min"], p["beta_max"], p["alpha_inc"],
                     p["alpha_dec"], p["gamma"])


class _Report(C.Structure):
    _fields_ = [("sweeps", C.c_int64), ("z", C.c_double), ("z_prev", C.c_double),
                ("stop_reason", C.c_int32), ("qp_fallbacks", C.c_int64)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            P = C.POINTER(_Problem)
            vp = C.c_void_p
            lib.orc_adjacency.argtypes = [P]
            lib.orc_adjacency.restype = C.c_int32
            lib.orc_excess.argtypes = [P, vp, vp, vp]
            lib.orc_excess.restype = None
            lib.orc_excess_vertex.argtypes = [P, vp, vp, C.c_int32, vp, vp]
            lib.orc_excess_vertex.restype = C.c_int32
            lib.orc_congestion_edge.argtypes = [C.c_int32, vp, C.c_double]
            lib.orc_congestion_edge.restype = C.c_double
            lib.orc_congestion.argtypes = [P, vp, vp]
            lib.orc_congestion.restype = None
            lib.orc_objective.argtypes = [P, vp, vp]
            lib.orc_objective.restype = C.c_double
            lib.orc_objective_edges.argtypes = [P, vp, vp]
            lib.orc_objective_edges.restype = C.c_double
            lib.orc_edge_qp.argtypes = [C.c_int32, vp, vp, vp, C.c_double, vp,
                                        C.POINTER(C.c_double), C.POINTER(C.c_double), vp, vp]
            lib.orc_edge_qp.restype = C.c_int32
            lib.orc_qp_all.argtypes = [P, vp, vp, vp, vp]
            lib.orc_qp_all.restype = C.c_int64
            lib.orc_residuals_at.argtypes = [P, vp, C.c_double, C.POINTER(_Residuals)]
            lib.orc_residuals_at.restype = None
            lib.orc_solve_eso.argtypes = [P, C.POINTER(_Options), vp, C.POINTER(_Report), vp, C.c_int64]
            lib.orc_solve_eso.restype = C.c_int32
            lib.orc_edge_ck.argtypes = [C.c_int32, vp, vp, vp, C.c_double, vp, C.POINTER(C.c_double), vp, vp]
            lib.orc_edge_ck.restype = C.c_int32
            lib.orc_ck_all.argtypes = [P, vp, vp, vp, vp]
            lib.orc_ck_all.restype = C.c_int64
            lib.orc_solve_ck.argtypes = [P, C.POINTER(_Options), vp, C.POINTER(_Report), vp, C.c_int64]
            lib.orc_solve_ck.restype = C.c_int32
            G = C.POINTER(_GDParams)
            lib.orc_gd_edge.argtypes = [G, C.c_int32, vp, vp, C.c_double, C.c_double, vp, vp,
                                        C.POINTER(C.c_double), C.c_int64, vp, C.POINTER(C.c_double)]
            lib.orc_gd_edge.restype = C.c_int32
            lib.orc_solve_gd.argtypes = [P, C.POINTER(_Options), G, vp, vp, vp, C.POINTER(_Report), vp, C.c_int64]
            lib.orc_solve_gd.restype = C.c_int32
            lib.orc_adjoint_eso.argtypes = [P, C.c_int64, C.POINTER(C.c_double), vp, vp]
            lib.orc_adjoint_eso.restype = C.c_int32
            lib.orc_unrolled_objective.argtypes = [P, C.c_int64]
            lib.orc_unrolled_objective.restype = C.c_double
            lib.orc_adjoint_ck.argtypes = [P, C.c_int64, C.POINTER(C.c_double), vp, vp]
            lib.orc_adjoint_ck.restype = C.c_int32
            lib.orc_unrolled_objective_ck.argtypes = [P, C.c_int64]
            lib.orc_unrolled_objective_ck.restype = C.c_double
            lib.orc_set_threads.argtypes = [C.c_int32]
            lib.orc_set_threads.restype = None
            lib.orc_max_threads.argtypes = []
            lib.orc_max_threads.restype = C.c_int32
            # one thread unless a caller asks for more (set_threads): the
            # per-sweep parallel regions cost more than they save on small cases
            lib.orc_set_threads(1)
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def set_threads(threads: int) -> int:
    """Set the OpenMP thread count for the per-edge / per-vertex loops; returns the count in use."""
    lib = _load()
    lib.orc_set_threads(int(threads))
    return int(lib.orc_max_threads())


class Problem:
    """An instance of eq. (1) held in the oracle's own arrays.

    ``row_ptr, col`` give the out-adjacency (edge id = CSR position), ``u``
    the capacities and ``(s, t, d)`` the commodities.  Construction builds the
    in-adjacency, edge tails and degrees (Table "Notation").
    """

    def __init__(self, n, row_ptr, col, u, s, t, d):
        self.n = int(n)
        self.row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
        self.col = np.ascontiguousarray(col, dtype=np.int32)
        self.u = np.ascontiguousarray(u, dtype=np.float64)
        self.s = np.ascontiguousarray(s, dtype=np.int32)
        self.t = np.ascontiguousarray(t, dtype=np.int32)
        self.d = np.ascontiguousarray(d, dtype=np.float64)
        self.m = int(self.col.shape[0])
        self.K = int(self.s.shape[0])
        self.in_ptr = np.zeros(self.n + 1, dtype=np.int64)
        self.in_eid = np.zeros(self.m, dtype=np.int64)
        self.src = np.zeros(self.m, dtype=np.int32)
        self.deg = np.zeros(self.n, dtype=np.int32)
        self._c = _Problem(self.n, self.m, self.K, _ptr(self.row_ptr), _ptr(self.col), _ptr(self.u),
                           _ptr(self.s), _ptr(self.t), _ptr(self.d), _ptr(self.in_ptr), _ptr(self.in_eid),
                           _ptr(self.src), _ptr(self.deg))
        if _load().orc_adjacency(C.byref(self._c)) != 0:
            raise ValueError("malformed CSR")

    @classmethod
    def from_instance(cls, inst):
        return cls(inst.n, inst.row_ptr, inst.col, inst.u, inst.s, inst.t, inst.d)

    def _f(self, f):
        f = np.ascontiguousarray(f, dtype=np.float64)
        if f.shape != (self.m, self.K):
            raise ValueError(f"flows must have shape {(self.m, self.K)}")
        return f

    def excess(self, f):
        """(Delta, h), both [n, K]: eq. (3) with eq. (3h), then eq. (2)."""
        f = self._f(f)
        Delta = np.empty((self.n, self.K))
        h = np.empty((self.n, self.K))
        _load().orc_excess(C.byref(self._c), _ptr(f), _ptr(Delta), _ptr(h))
        return Delta, h

    def excess_vertex(self, i, row_of_edge, rows):
        """(Delta_i, h_i) at one vertex from a compact row store: rows[row_of_edge[e]] is
        f[e, :] for every edge incident to i (row_of_edge[e] = -1 where absent)."""
        row_of_edge = np.ascontiguousarray(row_of_edge, dtype=np.int64)
        rows = np.ascontiguousarray(rows, dtype=np.float64)
        D = np.empty(self.K)
        h = np.empty(self.K)
        if _load().orc_excess_vertex(C.byref(self._c), _ptr(row_of_edge), _ptr(rows), int(i), _ptr(D), _ptr(h)):
            raise ValueError("a row incident to the vertex is missing")
        return D, h

    def congestion(self, f):
        """psi [m]: eq. (41)."""
        f = self._f(f)
        psi = np.empty(self.m)
        _load().orc_congestion(C.byref(self._c), _ptr(f), _ptr(psi))
        return psi

    def objective(self, h, psi):
        """z of Alg. 1: 1/2 sum psi^2 + 1/2 sum delta_i h^2."""
        h = np.ascontiguousarray(h, dtype=np.float64)
        psi = np.ascontiguousarray(psi, dtype=np.float64)
        return float(_load().orc_objective(C.byref(self._c), _ptr(h), _ptr(psi)))

    def objective_edges(self, h, psi):
        """z in the edge-separable form of eq. (8)."""
        h = np.ascontiguousarray(h, dtype=np.float64)
        psi = np.ascontiguousarray(psi, dtype=np.float64)
        return float(_load().orc_objective_edges(C.byref(self._c), _ptr(h), _ptr(psi)))

    def qp_all(self, h, f):
        """(f_next, psi_next, fallbacks): Alg. 2 on every edge from heights h (Jacobi step of Alg. 1)."""
        f = self._f(f)
        h = np.ascontiguousarray(h, dtype=np.float64)
        f_next = np.empty_like(f)
        psi = np.empty(self.m)
        fb = _load().orc_qp_all(C.byref(self._c), _ptr(h), _ptr(f), _ptr(f_next), _ptr(psi))
        return f_next, psi, int(fb)

    def sweep(self, f):
        """One iteration of Alg. 1 without the stop test: f^(t) -> f^(t+1)."""
        _, h = self.excess(f)
        return self.qp_all(h, f)[0]

    def ck_all(self, h, f):
        """(f_next, g, fallbacks): the capacity-kept step of Program (6) on every edge from heights h."""
        f = self._f(f)
        h = np.ascontiguousarray(h, dtype=np.float64)
        f_next = np.empty_like(f)
        g = np.empty(self.m)
        fb = _load().orc_ck_all(C.byref(self._c), _ptr(h), _ptr(f), _ptr(f_next), _ptr(g))
        return f_next, g, int(fb)

    def ck_sweep(self, f):
        """One capacity-kept iteration without the stop test: f^(t) -> f^(t+1)."""
        _, h = self.excess(f)
        return self.ck_all(h, f)[0]

    def solve_ck(self, max_sweeps=100000, eps_obj=1e-6, resid_tol=0.0, f0=None, trace=False):
        """Alg. 1 with the capacity-kept step (Program (6)) from f0 (default 0).
        Returns (f, report dict[, ztrace])."""
        f = np.zeros((self.m, self.K)) if f0 is None else self._f(f0).copy()
        opt = _Options(int(max_sweeps), float(eps_obj), float(resid_tol))
        rep = _Report()
        zt = np.full(int(max_sweeps) + 1, np.nan) if trace else None
        rc = _load().orc_solve_ck(C.byref(self._c), C.byref(opt), _ptr(f), C.byref(rep),
                                  _ptr(zt) if trace else None, int(max_sweeps) + 1 if trace else 0)
        if rc != 0:
            raise MemoryError("oracle solve failed to allocate")
        out = {k: getattr(rep, k) for k, _ in _Report._fields_}
        if trace:
            return f, out, zt[: out["sweeps"] + 1]
        return f, out

    def residuals(self, f, tol=1e-6):
        """eq. (1) residuals, Farkas margin and verdict at flows f (dict)."""
        f = self._f(f)
        R = _Residuals()
        _load().orc_residuals_at(C.byref(self._c), _ptr(f), float(tol), C.byref(R))
        return {k: getattr(R, k) for k, _ in _Residuals._fields_}

    def solve_gd(self, params: dict, max_sweeps=100000, eps_obj=1e-6, resid_tol=0.0, f0=None, v0=None, beta0=None,
                 trace=False):
        """Alg. 3 (params["momentum"] = 0) or Alg. 4 (= 1) from (f0, v0, beta0)
        (default 0, 0, beta_init).  Returns (f, v, beta, report dict[, ztrace])."""
        f = np.zeros((self.m, self.K)) if f0 is None else self._f(f0).copy()
        v = np.zeros((self.m, self.K)) if v0 is None else self._f(v0).copy()
        beta = (np.full(self.m, float(params["beta_init"])) if beta0 is None
                else np.ascontiguousarray(beta0, dtype=np.float64).copy())
        opt = _Options(int(max_sweeps), float(eps_obj), float(resid_tol))
        rep = _Report()
        g = _gd_struct(params)
        zt = np.full(int(max_sweeps) + 1, np.nan) if trace else None
        rc = _load().orc_solve_gd(C.byref(self._c), C.byref(opt), C.byref(g), _ptr(f), _ptr(v), _ptr(beta),
                                  C.byref(rep), _ptr(zt) if trace else None, int(max_sweeps) + 1 if trace else 0)
        if rc != 0:
            raise MemoryError("oracle solve failed to allocate")
        out = {k: getattr(rep, k) for k, _ in _Report._fields_}
        if trace:
            return f, v, beta, out, zt[: out["sweeps"] + 1]
        return f, v, beta, out

    def gd_sweep(self, params: dict, f, v, beta, t):
        """One iteration of Alg. 3 / Alg. 4 without the stop test, at iteration t:
        returns (f, v, beta) of iteration t + 1."""
        f = self._f(f).copy()
        v = self._f(v).copy()
        beta = np.ascontiguousarray(beta, dtype=np.float64).copy()
        _, h = self.excess(f)
        psi = self.congestion(f)
        for e in range(self.m):
            fe, ve, be, _, _ = gd_edge(params, h[self.src[e]], h[self.col[e]], psi[e], self.u[e], f[e], v[e],
                                       beta[e], t)
            f[e], v[e], beta[e] = fe, ve, be
        return f, v, beta

    def adjoint_eso(self, T: int):
        """(L, dL/du [m], dL/dd [K]) for L(u, d) = z(f^(T)) after T sweeps of Alg. 1 from f = 0."""
        L = C.c_double()
        gu = np.empty(self.m)
        gd = np.empty(self.K)
        if _load().orc_adjoint_eso(C.byref(self._c), int(T), C.byref(L), _ptr(gu), _ptr(gd)) != 0:
            raise MemoryError("oracle adjoint failed to allocate")
        return L.value, gu, gd

    def unrolled_objective(self, T: int) -> float:
        """z(f^(T)) after T sweeps of Alg. 1 from f = 0 (with this problem's u and d)."""
        return float(_load().orc_unrolled_objective(C.byref(self._c), int(T)))

    def adjoint_ck(self, T: int):
        """(L, dL/du, dL/dd) for L = z(f^(T)) after T capacity-kept sweeps (Program (6)) from f = 0."""
        L = C.c_double()
        gu = np.empty(self.m)
        gd = np.empty(self.K)
        if _load().orc_adjoint_ck(C.byref(self._c), int(T), C.byref(L), _ptr(gu), _ptr(gd)) != 0:
            raise MemoryError("oracle adjoint failed to allocate")
        return L.value, gu, gd

    def unrolled_objective_ck(self, T: int) -> float:
        """z(f^(T)) after T capacity-kept sweeps from f = 0."""
        return float(_load().orc_unrolled_objective_ck(C.byref(self._c), int(T)))

    def solve_eso(self, max_sweeps=100000, eps_obj=1e-6, resid_tol=0.0, f0=None, trace=False):
        """Alg. 1 with Alg. 2 from f0 (default 0).  Returns (f, report dict[, ztrace])."""
        f = np.zeros((self.m, self.K)) if f0 is None else self._f(f0).copy()
        opt = _Options(int(max_sweeps), float(eps_obj), float(resid_tol))
        rep = _Report()
        zt = np.full(int(max_sweeps) + 1, np.nan) if trace else None
        rc = _load().orc_solve_eso(C.byref(self._c), C.byref(opt), _ptr(f), C.byref(rep),
                                   _ptr(zt) if trace else None, int(max_sweeps) + 1 if trace else 0)
        if rc != 0:
            raise MemoryError("oracle solve failed to allocate")
        out = {k: getattr(rep, k) for k, _ in _Report._fields_}
        if trace:
            return f, out, zt[: out["sweeps"] + 1]
        return f, out


def congestion_edge(f_row, u) -> float:
    """eq. (41) for one edge from its row of flows."""
    f_row = np.ascontiguousarray(f_row, dtype=np.float64)
    return float(_load().orc_congestion_edge(int(f_row.shape[0]), _ptr(f_row), float(u)))


def gd_edge(params: dict, hi, hj, psi, u, f, v, beta, t):
    """One edge step of Alg. 3 / Alg. 4 at iteration t.
    Returns (f_new, v_new, beta_new, accepted, dz)."""
    hi = np.ascontiguousarray(hi, dtype=np.float64)
    hj = np.ascontiguousarray(hj, dtype=np.float64)
    f = np.array(f, dtype=np.float64)
    v = np.array(v if v is not None else np.zeros_like(f), dtype=np.float64)
    K = int(f.shape[0])
    b = C.c_double(float(beta))
    dz = C.c_double()
    df = np.empty(max(K, 1))
    g = _gd_struct(params)
    acc = _load().orc_gd_edge(C.byref(g), K, _ptr(hi), _ptr(hj), float(psi), float(u), _ptr(f), _ptr(v),
                              C.byref(b), int(t), _ptr(df), C.byref(dz))
    return f, v, b.value, bool(acc), dz.value


def edge_ck(hi, hj, f, u):
    """The capacity-kept step of Program (6) on one edge: returns (f_new, g, used_fallback)."""
    hi = np.ascontiguousarray(hi, dtype=np.float64)
    hj = np.ascontiguousarray(hj, dtype=np.float64)
    f = np.ascontiguousarray(f, dtype=np.float64)
    K = int(f.shape[0])
    out = np.empty(K)
    c = np.empty(max(K, 1))
    pos = np.empty(max(K, 1))
    g = C.c_double()
    fb = _load().orc_edge_ck(K, _ptr(hi), _ptr(hj), _ptr(f), float(u), _ptr(out), C.byref(g), _ptr(c), _ptr(pos))
    return out, g.value, bool(fb)


def edge_qp(hi, hj, f, u):
    """Alg. 2 on one edge: returns (f_new, r, psi, used_active_set_rule)."""
    hi = np.ascontiguousarray(hi, dtype=np.float64)
    hj = np.ascontiguousarray(hj, dtype=np.float64)
    f = np.ascontiguousarray(f, dtype=np.float64)
    K = int(f.shape[0])
    out = np.empty(K)
    c = np.empty(max(K, 1))
    pos = np.empty(max(K, 1))
    r = C.c_double()
    psi = C.c_double()
    fb = _load().orc_edge_qp(K, _ptr(hi), _ptr(hj), _ptr(f), float(u), _ptr(out), C.byref(r), C.byref(psi),
                             _ptr(c), _ptr(pos))
    return out, r.value, psi.value, bool(fb)
