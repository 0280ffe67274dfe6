"""Thin ctypes binding of libpdr (the C ABI declared in include/pdr.h).

Argument marshalling only: every step of the method runs in the library's
CUDA kernels.  The library must have been built for sm_103a
(``__graft_entry__.build()`` or ``python -m paper_2108_07549_gb300.build``);
there is no CPU fallback, and loading fails loudly if ``libpdr.so`` is
missing.

``Solver`` wraps one ``pdr_ctx``: an instance of eq. (1) held on the GPU and
solved by Alg. 1 (Potential Difference Reduction with the exact edge solver of
Alg. 2) of arXiv 2108.07549.
"""

from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpdr.so")

PREC_FP32, PREC_FP64, PREC_FP32_FP64TAIL = 0, 1, 2
ALGO_ESO, ALGO_AGD, ALGO_GDM, ALGO_CK = 0, 1, 2, 3
VERDICT_UNKNOWN, VERDICT_FEASIBLE, VERDICT_INFEASIBLE = 0, 1, 2
(OK, ERR_INVALID_ARG, ERR_OOM, ERR_CUDA, ERR_NUMERIC, ERR_NOT_SOLVED, ERR_UNSUPPORTED,
 ERR_TIMEOUT) = range(8)  # pdr_status
STOP_NAMES = {0: "max_sweeps", 1: "objective", 2: "residual", 3: "relative", 4: "numeric", 5: "stall",
              6: "plateau"}
VERDICT_NAMES = {0: "unknown", 1: "feasible", 2: "infeasible"}

#: every entry point declared in include/pdr.h
EXPORTS = (
    "pdr_default_options", "pdr_create", "pdr_set_options", "pdr_solve", "pdr_sweeps", "pdr_reset",
    "pdr_set_flows", "pdr_flows", "pdr_heights", "pdr_congestion", "pdr_objective", "pdr_adjacency",
    "pdr_residuals", "pdr_trace", "pdr_sizes", "pdr_time_kernel", "pdr_last_error", "pdr_destroy",
    "pdr_adjacency_static", "pdr_gd_state", "pdr_set_gd_state", "pdr_flow_rows",
    "pdr_batch_create", "pdr_batch_solve", "pdr_batch_reset", "pdr_batch_context", "pdr_batch_tuning",
    "pdr_batch_destroy", "pdr_set_data", "pdr_backward", "pdr_num_edge_variants", "pdr_edge_variant_capacity",
    "pdr_state_size", "pdr_get_state", "pdr_set_state", "pdr_debug_wait", "pdr_time_sweeps",
    "pdr_debug_fail_alloc", "pdr_debug_barrier",
)


class PdrError(RuntimeError):
    """A libpdr call returned a status other than PDR_OK."""

    def __init__(self, status: int, message: str):
        super().__init__(f"libpdr status {status}: {message}")
        self.status = status


class Options(C.Structure):
    _fields_ = [
        ("precision", C.c_int32), ("use_graph", C.c_int32), ("eps_obj", C.c_double), ("resid_tol", C.c_double),
        ("eps_rel", C.c_double), ("max_sweeps", C.c_int64), ("trace_len", C.c_int32), ("algo", C.c_int32),
        ("beta_init", C.c_double), ("beta_min", C.c_double), ("beta_max", C.c_double), ("alpha_inc", C.c_double),
        ("alpha_dec", C.c_double), ("gamma", C.c_double), ("edge_variant", C.c_int32),
        ("excess_variant", C.c_int32),
    ]


class Result(C.Structure):
    _fields_ = [
        ("sweeps", C.c_int64), ("sweeps_fp64", C.c_int64), ("z", C.c_double), ("dz", C.c_double),
        ("cap_abs", C.c_double), ("cap_rel", C.c_double), ("cons_abs", C.c_double), ("cons_rel", C.c_double),
        ("f_min", C.c_double), ("margin", C.c_double), ("margin_scale", C.c_double), ("ms_total", C.c_double),
        ("verdict", C.c_int32), ("stop_reason", C.c_int32), ("stop_reason_fp32", C.c_int32), ("pad", C.c_int32),
    ]

    def as_dict(self) -> dict:
        out = {k: getattr(self, k) for k, _ in self._fields_}
        out["verdict_name"] = VERDICT_NAMES.get(self.verdict, "?")
        out["stop_name"] = STOP_NAMES.get(self.stop_reason, "?")
        out["stop_name_fp32"] = STOP_NAMES.get(self.stop_reason_fp32, "-")
        return out


class InstanceC(C.Structure):
    _fields_ = [("n", C.c_int32), ("K", C.c_int32), ("m", C.c_int64), ("row_ptr", C.c_void_p), ("col", C.c_void_p),
                ("u", C.c_void_p), ("s", C.c_void_p), ("t", C.c_void_p), ("d", C.c_void_p)]


_lib = None


def load(path: str = LIB_PATH):
    """Opens libpdr.so and declares every entry point's signature."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with __graft_entry__.build() "
                           "(there is no CPU fallback)")
    lib = C.CDLL(path)
    vp, i32, i64, dbl = C.c_void_p, C.c_int32, C.c_int64, C.c_double
    P = C.POINTER
    sig = {
        "pdr_default_options": ([P(Options)], i32),
        "pdr_create": ([i32, i64, vp, vp, vp, i32, vp, vp, vp, P(Options), vp, P(vp)], i32),
        "pdr_set_options": ([vp, P(Options)], i32),
        "pdr_solve": ([vp, P(Result)], i32),
        "pdr_sweeps": ([vp, i64], i32),
        "pdr_reset": ([vp], i32),
        "pdr_set_flows": ([vp, vp], i32),
        "pdr_flows": ([vp, vp], i32),
        "pdr_state_size": ([vp, P(i64)], i32),
        "pdr_get_state": ([vp, vp, i64], i32),
        "pdr_set_state": ([vp, vp, i64], i32),
        "pdr_debug_wait": ([vp, i64, i32], i32),
        "pdr_debug_barrier": ([vp, i64, i32], i32),
        "pdr_time_sweeps": ([vp, i64, P(dbl), P(dbl)], i32),
        "pdr_debug_fail_alloc": ([i64], i32),
        "pdr_heights": ([vp, vp], i32),
        "pdr_congestion": ([vp, vp], i32),
        "pdr_objective": ([vp, P(dbl)], i32),
        "pdr_adjacency": ([vp, vp, vp, vp], i32),
        "pdr_residuals": ([vp, P(Result)], i32),
        "pdr_trace": ([vp, vp, i64, P(i64)], i32),
        "pdr_sizes": ([vp, P(i32), P(i64), P(i32), P(i32)], i32),
        "pdr_time_kernel": ([vp, i32, i32, i64, P(dbl)], i32),
        "pdr_num_edge_variants": ([], i32),
        "pdr_edge_variant_capacity": ([i32, i32, P(i32)], i32),
        "pdr_last_error": ([vp], C.c_char_p),
        "pdr_destroy": ([vp], None),
        "pdr_adjacency_static": ([i32, i64, vp, vp, vp, vp, vp, vp], i32),
        "pdr_gd_state": ([vp, vp, vp], i32),
        "pdr_flow_rows": ([vp, i32, vp, i64, vp], i32),
        "pdr_batch_create": ([i32, P(InstanceC), P(Options), vp, P(vp)], i32),
        "pdr_batch_solve": ([vp, P(Result)], i32),
        "pdr_batch_reset": ([vp], i32),
        "pdr_batch_context": ([vp, i32, P(vp)], i32),
        "pdr_batch_tuning": ([vp, vp, vp], i32),
        "pdr_batch_destroy": ([vp], None),
        "pdr_set_data": ([vp, vp, vp], i32),
        "pdr_backward": ([vp, i64, i32, P(dbl), vp, vp], i32),
        "pdr_set_gd_state": ([vp, vp, vp], i32),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def default_options(**overrides) -> Options:
    o = Options()
    load().pdr_default_options(C.byref(o))
    for k, v in overrides.items():
        if not hasattr(o, k):
            raise KeyError(f"unknown option {k!r}")
        setattr(o, k, v)
    return o


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _current_stream():
    """The CUDA stream torch is using on the current device (None if torch has no CUDA)."""
    try:
        import torch

        if torch.cuda.is_available():
            return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    except ImportError:
        pass
    return None


def edge_variants(precision: int = 0) -> list:
    """The edge-kernel variant table: (index, row capacity in `precision`, form) per entry; form is 0 for
    the plain forms, 1 for the pipelined warp forms, 2 for the staged block forms."""
    lib = load()
    out = []
    for v in range(lib.pdr_num_edge_variants()):
        pipe = C.c_int32(0)
        cap = lib.pdr_edge_variant_capacity(v, precision, C.byref(pipe))
        out.append((v, cap, int(pipe.value)))
    return out


def adjacency_static(n, m, row_ptr, col, in_ptr, in_eid, deg, stream=None):
    """In-adjacency and degrees of a device-resident graph with no allocation
    (pdr_adjacency_static).  Every array argument is a device address (an
    int, e.g. ``tensor.data_ptr()``): row_ptr int64 [n+1] and col int32 [m]
    in, in_ptr int64 [n+1], in_eid int32 [m] and deg int32 [n] out.  For
    callers that may not allocate device memory; see include/pdr.h."""
    lib = load()
    if stream is None:
        stream = _current_stream()
    elif not isinstance(stream, C.c_void_p):
        stream = C.c_void_p(int(stream))
    st = lib.pdr_adjacency_static(int(n), int(m), C.c_void_p(row_ptr), C.c_void_p(col), C.c_void_p(in_ptr),
                                  C.c_void_p(in_eid), C.c_void_p(deg), stream)
    if st != 0:
        raise PdrError(st, lib.pdr_last_error(None).decode())


class Solver:
    """One instance of eq. (1) on the GPU, solved by Alg. 1 / Alg. 2.

    ``row_ptr, col`` are the out-adjacency (edge id = CSR position), ``u`` the
    capacities, ``(s, t, d)`` the commodities.  Keyword options are the fields
    of ``pdr_options``.  ``stream`` is a ``cudaStream_t`` value (default: the
    current torch stream).
    """

    def __init__(self, n, row_ptr, col, u, s, t, d, stream=None, **options):
        lib = load()
        self._lib = lib
        self.n = int(n)
        row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
        col = np.ascontiguousarray(col, dtype=np.int32)
        u = np.ascontiguousarray(u, dtype=np.float64)
        s = np.ascontiguousarray(s, dtype=np.int32)
        t = np.ascontiguousarray(t, dtype=np.int32)
        d = np.ascontiguousarray(d, dtype=np.float64)
        self.m = int(col.shape[0])
        self.K = int(s.shape[0])
        if t.shape[0] != self.K or d.shape[0] != self.K or u.shape[0] != self.m or row_ptr.shape[0] != self.n + 1:
            raise ValueError("array lengths do not match n, m, K")
        self.options = default_options(**options)
        if stream is None:
            stream = _current_stream()
        elif not isinstance(stream, C.c_void_p):
            stream = C.c_void_p(int(stream))
        self._stream = stream
        h = C.c_void_p()
        st = lib.pdr_create(self.n, self.m, _ptr(row_ptr), _ptr(col), _ptr(u), self.K, _ptr(s), _ptr(t), _ptr(d),
                            C.byref(self.options), stream, C.byref(h))
        if st != 0:
            raise PdrError(st, lib.pdr_last_error(None).decode())
        self._h = h
        self.Kp = self.sizes()[3]

    @classmethod
    def from_instance(cls, inst, stream=None, **options):
        return cls(inst.n, inst.row_ptr, inst.col, inst.u, inst.s, inst.t, inst.d, stream=stream, **options)

    # ------------------------------------------------------------------ plumbing
    def _check(self, status):
        if status != 0:
            raise PdrError(status, self._lib.pdr_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            self._lib.pdr_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # ------------------------------------------------------------------ API
    def set_options(self, **options):
        o = default_options()
        for k, _ in Options._fields_:
            setattr(o, k, getattr(self.options, k))
        for k, v in options.items():
            if not hasattr(o, k):
                raise KeyError(f"unknown option {k!r}")
            setattr(o, k, v)
        self._check(self._lib.pdr_set_options(self._h, C.byref(o)))
        self.options = o

    def solve(self) -> dict:
        r = Result()
        self._check(self._lib.pdr_solve(self._h, C.byref(r)))
        return r.as_dict()

    def sweeps(self, count: int):
        self._check(self._lib.pdr_sweeps(self._h, int(count)))

    def reset(self):
        self._check(self._lib.pdr_reset(self._h))

    def set_flows(self, f):
        f = np.ascontiguousarray(f, dtype=np.float64)
        if f.shape != (self.m, self.K):
            raise ValueError(f"flows must have shape {(self.m, self.K)}")
        self._check(self._lib.pdr_set_flows(self._h, _ptr(f)))

    def flows(self) -> np.ndarray:
        f = np.empty((self.m, self.K), dtype=np.float64)
        self._check(self._lib.pdr_flows(self._h, _ptr(f)))
        return f

    def get_state(self) -> bytes:
        """Checkpoint of the solve (pdr_get_state) as bytes."""
        n = C.c_int64()
        self._check(self._lib.pdr_state_size(self._h, C.byref(n)))
        buf = C.create_string_buffer(max(n.value, 1))
        self._check(self._lib.pdr_get_state(self._h, buf, n.value))
        return buf.raw[: n.value]

    def set_state(self, state: bytes):
        """Restores a checkpoint (pdr_set_state); the next solve continues it."""
        buf = C.create_string_buffer(bytes(state), len(state))
        self._check(self._lib.pdr_set_state(self._h, buf, len(state)))

    def debug_wait(self, cycles: int = 1 << 32, hold_end: bool = False):
        """Test hook (pdr_debug_wait): the device wait limit and the end-marker hold."""
        self._check(self._lib.pdr_debug_wait(self._h, int(cycles), int(bool(hold_end))))

    def debug_barrier(self, limit_ns: int = 2_000_000_000, withhold: bool = False):
        """pdr_debug_barrier (test hook): time limit of the persistent engine's grid
        barrier, and whether block 0 withholds its arrival."""
        self._check(self._lib.pdr_debug_barrier(self._h, int(limit_ns), int(bool(withhold))))

    def flow_rows(self, edges, velocities: bool = False) -> np.ndarray:
        """Rows f[e, :] (or the Alg. 4 velocities v[e, :]) for the given edge ids ([len(edges), K])."""
        edges = np.ascontiguousarray(edges, dtype=np.int64)
        out = np.empty((edges.shape[0], self.K), dtype=np.float64)
        self._check(self._lib.pdr_flow_rows(self._h, 1 if velocities else 0, _ptr(edges), int(edges.shape[0]),
                                            _ptr(out)))
        return out

    def gd_state(self, with_velocities: bool = True):
        """(beta [m], v [m, K] or None) of Alg. 3 / Alg. 4 at the current iteration."""
        beta = np.empty(self.m, dtype=np.float64)
        v = np.empty((self.m, self.K), dtype=np.float64) if with_velocities else None
        self._check(self._lib.pdr_gd_state(self._h, _ptr(beta), None if v is None else _ptr(v)))
        return beta, v

    def set_gd_state(self, beta, v=None):
        beta = np.ascontiguousarray(beta, dtype=np.float64)
        vv = None if v is None else np.ascontiguousarray(v, dtype=np.float64)
        self._check(self._lib.pdr_set_gd_state(self._h, _ptr(beta), None if vv is None else _ptr(vv)))

    def set_data(self, u=None, d=None):
        """Replace the capacities and/or demands (the flows are kept)."""
        uu = None if u is None else np.ascontiguousarray(u, dtype=np.float64)
        dd = None if d is None else np.ascontiguousarray(d, dtype=np.float64)
        if uu is not None and uu.shape != (self.m,):
            raise ValueError("u must have shape (m,)")
        if dd is not None and dd.shape != (self.K,):
            raise ValueError("d must have shape (K,)")
        self._check(self._lib.pdr_set_data(self._h, None if uu is None else _ptr(uu), None if dd is None else _ptr(dd)))

    def set_data_device(self, u_ptr: int = 0, d_ptr: int = 0):
        """pdr_set_data from device arrays (device addresses as ints, e.g.
        ``tensor.data_ptr()`` of contiguous float64 CUDA tensors; 0 keeps the
        current values).  Checked and converted on the device."""
        self._check(self._lib.pdr_set_data(self._h, C.c_void_p(u_ptr) if u_ptr else None,
                                           C.c_void_p(d_ptr) if d_ptr else None))

    def backward_into(self, T: int, ckpt_every: int, gu_ptr: int = 0, gd_ptr: int = 0) -> float:
        """pdr_backward writing dL/du and dL/dd to device arrays (float64 [m] and
        [K], device addresses as ints; 0 skips that gradient); returns L."""
        L = C.c_double()
        self._check(self._lib.pdr_backward(self._h, int(T), int(ckpt_every), C.byref(L),
                                           C.c_void_p(gu_ptr) if gu_ptr else None,
                                           C.c_void_p(gd_ptr) if gd_ptr else None))
        return L.value

    def backward(self, T: int, ckpt_every: int = 10, grads: bool = True):
        """(L, dL/du, dL/dd) for L = z(f^(T)) after T sweeps of Alg. 1 from f = 0
        (gradients None if grads is False)."""
        L = C.c_double()
        gu = np.empty(self.m) if grads else None
        gd = np.empty(self.K) if grads else None
        self._check(self._lib.pdr_backward(self._h, int(T), int(ckpt_every), C.byref(L),
                                           None if gu is None else _ptr(gu), None if gd is None else _ptr(gd)))
        return L.value, gu, gd

    def heights(self) -> np.ndarray:
        h = np.empty((self.n, self.K), dtype=np.float64)
        self._check(self._lib.pdr_heights(self._h, _ptr(h)))
        return h

    def congestion(self) -> np.ndarray:
        psi = np.empty(self.m, dtype=np.float64)
        self._check(self._lib.pdr_congestion(self._h, _ptr(psi)))
        return psi

    def objective(self) -> float:
        z = C.c_double()
        self._check(self._lib.pdr_objective(self._h, C.byref(z)))
        return z.value

    def adjacency(self):
        in_ptr = np.empty(self.n + 1, dtype=np.int64)
        in_eid = np.empty(self.m, dtype=np.int32)
        deg = np.empty(self.n, dtype=np.int32)
        self._check(self._lib.pdr_adjacency(self._h, _ptr(in_ptr), _ptr(in_eid), _ptr(deg)))
        return in_ptr, in_eid, deg

    def residuals(self) -> dict:
        r = Result()
        self._check(self._lib.pdr_residuals(self._h, C.byref(r)))
        return r.as_dict()

    def trace(self) -> np.ndarray:
        cap = int(self.options.trace_len)
        z = np.empty(max(cap, 1), dtype=np.float64)
        cnt = C.c_int64()
        self._check(self._lib.pdr_trace(self._h, _ptr(z), cap, C.byref(cnt)))
        return z[: cnt.value].copy()

    def sizes(self):
        n, m, K, Kp = C.c_int32(), C.c_int64(), C.c_int32(), C.c_int32()
        self._check(self._lib.pdr_sizes(self._h, C.byref(n), C.byref(m), C.byref(K), C.byref(Kp)))
        return n.value, m.value, K.value, Kp.value

    def time_sweeps(self, count: int):
        """pdr_time_sweeps: mean ms of the excess and update kernels over `count` sweeps."""
        mx, mu = C.c_double(), C.c_double()
        self._check(self._lib.pdr_time_sweeps(self._h, int(count), C.byref(mx), C.byref(mu)))
        return mx.value, mu.value

    def time_kernel(self, which: str = "qp", launches: int = 20, flush_bytes: int = 0) -> float:
        """Mean duration (ms) of one launch of the edge QP ("qp") or excess ("excess") kernel."""
        ms = C.c_double()
        w = {"qp": 0, "excess": 1}[which]
        self._check(self._lib.pdr_time_kernel(self._h, w, int(launches), int(flush_bytes), C.byref(ms)))
        return ms.value


class _BorrowedSolver(Solver):
    """A Solver view of a context owned by a Batch (never destroyed by Python)."""

    def __init__(self, lib, handle, inst_sizes, options):
        self._lib = lib
        self._h = handle
        self.n, self.m, self.K = inst_sizes
        self.options = options
        self.Kp = self.sizes()[3]

    def close(self):
        self._h = None


class Batch:
    """Many independent instances solved together (the batched form).

    ``instances`` is a sequence of objects with ``n, row_ptr, col, u, s, t, d``
    (e.g. ``instances.Instance``).  One CUDA graph launch per ``solve()``
    runs every instance to its own stop rule.
    """

    def __init__(self, instances, stream=None, **options):
        lib = load()
        self._lib = lib
        self._keep = []
        arr = (InstanceC * len(instances))()
        for i, inst in enumerate(instances):
            a = [np.ascontiguousarray(x, dt) for x, dt in ((inst.row_ptr, np.int64), (inst.col, np.int32),
                                                            (inst.u, np.float64), (inst.s, np.int32),
                                                            (inst.t, np.int32), (inst.d, np.float64))]
            self._keep.append(a)
            arr[i] = InstanceC(int(inst.n), int(a[3].shape[0]), int(a[1].shape[0]), *(_ptr(x) for x in a))
        self.options = default_options(**options)
        if stream is None:
            stream = _current_stream()
        elif not isinstance(stream, C.c_void_p):
            stream = C.c_void_p(int(stream))
        h = C.c_void_p()
        st = lib.pdr_batch_create(len(instances), arr, C.byref(self.options), stream, C.byref(h))
        if st != 0:
            raise PdrError(st, lib.pdr_last_error(None).decode())
        self._h = h
        self.count = len(instances)
        self._sizes = [(int(x.n), int(x.col.shape[0]), int(x.s.shape[0])) for x in instances]

    def _check(self, status):
        if status != 0:
            raise PdrError(status, self._lib.pdr_last_error(None).decode())

    def solve(self):
        res = (Result * self.count)()
        self._check(self._lib.pdr_batch_solve(self._h, res))
        return [r.as_dict() for r in res]

    def reset(self):
        self._check(self._lib.pdr_batch_reset(self._h))

    def solver(self, index: int) -> Solver:
        """A read-out view of instance ``index`` (flows, residuals, adjacency...)."""
        h = C.c_void_p()
        self._check(self._lib.pdr_batch_context(self._h, int(index), C.byref(h)))
        return _BorrowedSolver(self._lib, h, self._sizes[index], self.options)

    def tuning(self):
        cfg = np.empty(self.count, dtype=np.int32)
        us = np.empty(self.count, dtype=np.float64)
        self._check(self._lib.pdr_batch_tuning(self._h, _ptr(cfg), _ptr(us)))
        return cfg, us

    def close(self):
        if getattr(self, "_h", None):
            self._lib.pdr_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
