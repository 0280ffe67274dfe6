"""Seeded synthetic multicommodity-flow instances.

This module builds inputs only: directed graphs, origin-destination pairs,
demands and capacities.  It holds none of the PDR method's arithmetic, so both
the CUDA path and the CPU oracle may take their inputs from here.

The shapes stand in for the paper's benchmark families (Section 7, "Test
Problems"): grid networks (a x a bidirectional grids, most vertices of degree
four), planar networks (random points in the plane joined to neighbouring
points) and sparse random networks.  The benchmark files themselves are not
used.

Capacities follow one recipe throughout: route every commodity along a
hop-shortest path chosen with seeded random tie-breaking, accumulate the
resulting edge load, and scale it by ``factor``.  With ``factor >= 1`` that
routing is itself a feasible flow for eq. (1).  With ``factor < 1`` the total
capacity is below sum_k d_k * dist(s_k, t_k), the least total edge flow any
feasible routing needs, so the instance is infeasible by construction.

Every array is produced by numpy's PCG64 generator from an integer seed, so an
instance is reproducible from (recipe, seed) on any host.
"""

from __future__ import annotations

from dataclasses import dataclass, replace

import numpy as np

__all__ = [
    "Instance",
    "grid_graph",
    "knn_graph",
    "random_digraph",
    "make_instance",
    "grid5_k10",
    "knn2500_k500",
    "grid100_k10000",
    "digraph20k_k2000",
    "batch256",
]


@dataclass(frozen=True)
class Instance:
    """A multicommodity-flow feasibility instance (eq. (1)).

    Edge ``e`` of the graph is CSR position ``e``: its tail is the vertex ``i``
    with ``row_ptr[i] <= e < row_ptr[i+1]`` and its head is ``col[e]``.
    """

    name: str
    n: int
    row_ptr: np.ndarray  # int64 [n+1]
    col: np.ndarray  # int32 [m]
    u: np.ndarray  # float64 [m] capacities
    s: np.ndarray  # int32 [K] origins
    t: np.ndarray  # int32 [K] destinations
    d: np.ndarray  # float64 [K] demands
    factor: float  # capacity = factor * witness routing load
    load: np.ndarray  # float64 [m] witness routing load
    hops: np.ndarray  # int64 [K] hop distance s_k -> t_k

    @property
    def m(self) -> int:
        return int(self.col.shape[0])

    @property
    def K(self) -> int:
        return int(self.s.shape[0])

    @property
    def src(self) -> np.ndarray:
        """Tail vertex of every edge (int32 [m])."""
        return np.repeat(np.arange(self.n, dtype=np.int32), np.diff(self.row_ptr)).astype(np.int32)

    @property
    def feasible_by_construction(self):
        """True/False when the capacity recipe decides feasibility, else None."""
        if self.factor >= 1.0:
            return True
        if float(self.u.sum()) < float(np.dot(self.d, self.hops)):
            return False
        return None

    def with_factor(self, factor: float, name: str | None = None) -> "Instance":
        """The same graph and commodities with capacities ``factor * load``."""
        return replace(self, name=name or f"{self.name}@{factor:g}", factor=float(factor),
                       u=self.load * float(factor))


# --------------------------------------------------------------------------- graphs


def _csr(n: int, src: np.ndarray, dst: np.ndarray):
    """CSR of an edge list, edges kept in list order within each tail vertex."""
    order = np.argsort(src, kind="stable")
    col = dst[order].astype(np.int32)
    counts = np.bincount(src, minlength=n).astype(np.int64)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    return row_ptr, col


def grid_graph(a: int):
    """a x a bidirectional grid: n = a^2, m = 4a(a-1); vertex (r, c) is r*a + c."""
    src, dst = [], []
    for r in range(a):
        for c in range(a):
            v = r * a + c
            for dr, dc in ((0, 1), (0, -1), (1, 0), (-1, 0)):
                rr, cc = r + dr, c + dc
                if 0 <= rr < a and 0 <= cc < a:
                    src.append(v)
                    dst.append(rr * a + cc)
    n = a * a
    return (n,) + _csr(n, np.asarray(src, np.int64), np.asarray(dst, np.int64))


def knn_graph(n: int, k: int, rng: np.random.Generator):
    """Random points in the unit square, each joined both ways to its k nearest.

    Every (vertex, neighbour) link gives two arcs, so m = 2 * k * n exactly.
    Mutual nearest neighbours therefore get two parallel arcs in each
    direction; parallel arcs are ordinary edges of the multigraph, each with
    its own capacity.
    """
    pts = rng.random((n, 2))
    d2 = ((pts[:, None, :] - pts[None, :, :]) ** 2).sum(-1)
    np.fill_diagonal(d2, np.inf)
    nearest = np.argsort(d2, axis=1, kind="stable")[:, :k]
    a = np.repeat(np.arange(n, dtype=np.int64), k)
    b = nearest.reshape(-1).astype(np.int64)
    src = np.concatenate([a, b])
    dst = np.concatenate([b, a])
    return (n,) + _csr(n, src, dst)


def random_digraph(n: int, outdeg: int, rng: np.random.Generator):
    """Each vertex gets ``outdeg`` distinct random heads other than itself."""
    src = np.repeat(np.arange(n, dtype=np.int64), outdeg)
    dst = np.empty(n * outdeg, dtype=np.int64)
    for v in range(n):
        pick = rng.choice(n - 1, size=outdeg, replace=False)
        pick = np.sort(pick)
        pick[pick >= v] += 1
        dst[v * outdeg:(v + 1) * outdeg] = pick
    return (n,) + _csr(n, src, dst)


# --------------------------------------------------------------------------- routing


def _hop_dist_to(n, row_ptr, col, targets):
    """dist[b, v] = hop distance v -> targets[b] (inf if unreachable)."""
    from scipy.sparse import csr_matrix
    from scipy.sparse.csgraph import shortest_path

    m = col.shape[0]
    src = np.repeat(np.arange(n), np.diff(row_ptr))
    # reversed graph: an edge (i, j) becomes (j, i)
    rev = csr_matrix((np.ones(m), (col.astype(np.int64), src)), shape=(n, n))
    return shortest_path(rev, method="D", directed=True, unweighted=True, indices=targets)


def _sample_pairs(n, K, rng, row_ptr, col, chunk=512):
    """K distinct (s, t) pairs, s != t, t reachable from s; with hop distances."""
    if K > n * (n - 1):
        raise ValueError(f"{K} distinct pairs do not exist on {n} vertices")
    seen = set()
    rounds = 0
    s_out, t_out, h_out = [], [], []
    while len(s_out) < K:
        rounds += 1
        if rounds > 10000:
            raise ValueError(f"could not draw {K} distinct reachable pairs")
        need = K - len(s_out)
        cand_s = rng.integers(0, n, size=max(need, 8))
        cand_t = rng.integers(0, n, size=max(need, 8))
        keep = cand_s != cand_t
        cand_s, cand_t = cand_s[keep], cand_t[keep]
        for lo in range(0, cand_t.shape[0], chunk):
            ts = cand_t[lo:lo + chunk]
            ss = cand_s[lo:lo + chunk]
            dist = _hop_dist_to(n, row_ptr, col, ts)
            hop = dist[np.arange(ts.shape[0]), ss]
            for a, b, h in zip(ss.tolist(), ts.tolist(), hop.tolist()):
                if len(s_out) >= K:
                    break
                if not np.isfinite(h) or (a, b) in seen:
                    continue
                seen.add((a, b))
                s_out.append(a)
                t_out.append(b)
                h_out.append(int(h))
            if len(s_out) >= K:
                break
    return (np.asarray(s_out, np.int32), np.asarray(t_out, np.int32), np.asarray(h_out, np.int64))


def _route_load(n, row_ptr, col, s, t, d, rng, chunk=512):
    """Load of routing every commodity on a random hop-shortest path."""
    m = col.shape[0]
    deg = np.diff(row_ptr)
    D = int(deg.max()) if n else 0
    # padded out-edge table [n, D], -1 where a vertex has fewer out-edges
    nbr = np.full((n, max(D, 1)), -1, dtype=np.int64)
    for j in range(D):
        has = deg > j
        nbr[has, j] = row_ptr[:-1][has] + j
    load = np.zeros(m, dtype=np.float64)
    K = s.shape[0]
    for lo in range(0, K, chunk):
        ss = s[lo:lo + chunk].astype(np.int64)
        ts = t[lo:lo + chunk].astype(np.int64)
        dd = d[lo:lo + chunk]
        B = ss.shape[0]
        dist = _hop_dist_to(n, row_ptr, col, ts)
        rows = np.arange(B)
        cur = ss.copy()
        active = cur != ts
        while active.any():
            E = nbr[cur]  # [B, D]
            valid = E >= 0
            V = np.where(valid, col[np.where(valid, E, 0)], 0)
            ok = valid & (dist[rows[:, None], V] == (dist[rows, cur] - 1)[:, None])
            keys = rng.random(E.shape)
            keys[~ok] = -1.0
            pick = np.argmax(keys, axis=1)
            e = E[rows, pick]
            np.add.at(load, e[active], dd[active])
            cur = np.where(active, col[np.where(active, e, 0)].astype(np.int64), cur)
            active = cur != ts
    return load


# --------------------------------------------------------------------------- instances


def make_instance(name, graph, K, demand, factor, rng) -> Instance:
    """Commodities, demands and capacities on ``graph = (n, row_ptr, col)``.

    ``demand`` is ("uniform_int", lo, hi) for integers in [lo, hi] or
    ("lognormal", mu, sigma).
    """
    n, row_ptr, col = graph
    s, t, hops = _sample_pairs(n, K, rng, row_ptr, col)
    kind = demand[0]
    if kind == "uniform_int":
        d = rng.integers(demand[1], demand[2] + 1, size=K).astype(np.float64)
    elif kind == "lognormal":
        d = rng.lognormal(demand[1], demand[2], size=K)
    else:
        raise ValueError(f"unknown demand distribution {kind!r}")
    load = _route_load(n, row_ptr, col, s, t, d, rng)
    return Instance(name=name, n=int(n), row_ptr=row_ptr.astype(np.int64), col=col.astype(np.int32),
                    u=load * float(factor), s=s, t=t, d=d, factor=float(factor), load=load, hops=hops)


def grid5_k10(factor: float = 1.3, seed: int = 0) -> Instance:
    """5x5 bidirectional grid (n=25, m=80), K=10, integer demands in [1, 10]."""
    rng = np.random.default_rng(seed)
    return make_instance(f"grid5_k10@{factor:g}", grid_graph(5), 10, ("uniform_int", 1, 10), factor, rng)


def knn2500_k500(factor: float = 1.2, seed: int = 0) -> Instance:
    """n=2500 random points, 3-nearest-neighbour links both ways, K=500, demands in [1, 20]."""
    rng = np.random.default_rng(seed)
    g = knn_graph(2500, 3, rng)
    return make_instance(f"knn2500_k500@{factor:g}", g, 500, ("uniform_int", 1, 20), factor, rng)


def grid100_k10000(factor: float = 1.1, seed: int = 0) -> Instance:
    """100x100 bidirectional grid (n=10,000, m=39,600), K=10,000, lognormal(1, 0.5) demands."""
    rng = np.random.default_rng(seed)
    return make_instance(f"grid100_k10000@{factor:g}", grid_graph(100), 10000, ("lognormal", 1.0, 0.5),
                         factor, rng)


def digraph20k_k2000(factor: float = 1.05, seed: int = 0) -> Instance:
    """Random digraph n=20,000 with out-degree 5 (m=100,000), K=2000, demands in [1, 10]."""
    rng = np.random.default_rng(seed)
    g = random_digraph(20000, 5, rng)
    return make_instance(f"digraph20k_k2000@{factor:g}", g, 2000, ("uniform_int", 1, 10), factor, rng)


def _batch_member(args):
    seed, b, n, K, factor = args
    sub = np.random.default_rng([seed, b])
    g = random_digraph(n, 4, sub)
    return make_instance(f"batch{b}@{factor:g}", g, K, ("uniform_int", 1, 10), factor, sub)


def batch256(seed: int = 0, count: int = 256, n_range=(100, 5000), k_range=(10, 1000),
             infeasible_share: float = 0.2, processes: int = 0):
    """Independent instances of uneven size: random out-degree-4 digraphs.

    n and K are uniform in their ranges, demands integers in [1, 10],
    capacities 1.2x the routing load, and ``infeasible_share`` of the
    instances scaled to 0.7x instead (infeasible by construction).  Instance
    b draws from its own generator seeded by (seed, b), so ``processes > 1``
    (a spawn-context pool; call it before any CUDA work) gives the same
    instances faster.
    """
    rng = np.random.default_rng(seed)
    n_bad = int(round(infeasible_share * count))
    bad = set(rng.choice(count, size=n_bad, replace=False).tolist())
    jobs = []
    for b in range(count):
        n = int(rng.integers(n_range[0], n_range[1] + 1))
        K = int(rng.integers(k_range[0], k_range[1] + 1))
        jobs.append((seed, b, n, K, 0.7 if b in bad else 1.2))
    if processes and processes > 1:
        import concurrent.futures as cf
        import multiprocessing as mp

        with cf.ProcessPoolExecutor(max_workers=processes, mp_context=mp.get_context("spawn")) as ex:
            return list(ex.map(_batch_member, jobs, chunksize=4))
    return [_batch_member(j) for j in jobs]
