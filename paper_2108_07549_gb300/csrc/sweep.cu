// sweep.cu -- the two kernels of one PDR sweep (Alg. 1 loop body).
//
//  excess_kernel  eq. (3) + eq. (3h): Delta_ik = sum_in f - sum_out f + hat-Delta_ik,
//                 eq. (2): h_ik = Delta_ik / delta_i, and per-block partials
//                 of the objective of Alg. 1.
//  edge_kernel    Alg. 2 on every edge: the exact minimiser of eq. (10),
//                 f' = max(0, c - psi'/2) with c_k = f_k + (h_ik - h_jk)/2,
//                 written to the other flow buffer, followed by the
//                 congestion psi = max(0, sum_k f' - u) (eq. (41)) of the
//                 stored new flows.  One extra block of the same launch
//                 reduces the objective partials in FP64 (fixed order, no
//                 floating-point atomics) and takes the stop decision while
//                 the other blocks solve the edge QPs; if it stops, f^(t) in
//                 the input buffer is the result and f^(t+1) is discarded,
//                 exactly as Alg. 1 returns f^(t).
//
// Alg. 2 sorts the positive potentials to find the congested root.  Here the
// same root is found without a sort: with theta = psi'/2 and the active set
// A = {k : c_k > theta}, the root satisfies theta = (sum_A c - u)/(2 + |A|)
// (Section 4.4.3, Case 2).  Starting from A = {c > 0}, theta(A) never exceeds
// the root, so every element with c_k <= theta(A) is inactive at the root;
// dropping them and recomputing theta increases theta monotonically and
// stops, after at most |A| rounds, at the active set of the root (the
// active-set iteration of Michelot 1986 for projections onto a simplex,
// applied to this problem).  Each round is one group-wide sum and count held
// in registers, so no row is sorted or re-read.
#include "sweep_common.cuh"

namespace pdr {
namespace {

template <typename T>
__global__ void __launch_bounds__(kThreads) finalize_kernel(SweepArgs<T> a)
{
    reduce_and_finalize(a);
}

// ------------------------------------------------------------------ excess and heights

template <typename T, bool SH = false>
__device__ __forceinline__ void excess_tail(const SweepArgs<T>& a, int block, int nblocks,
                                            typename Acc<T>::V zacc, T cons);

// Body of one excess pass run by block `block` of `nblocks` (the standalone
// kernel passes its own grid; the persistent kernel its whole grid).  SH:
// the objective partials live in shared memory (the one-block engine).
template <typename T, bool SH = false>
__device__ __forceinline__ void excess_body(const SweepArgs<T>& a, int block, int nblocks)
{
    using VT = typename VecOf<T>::type;
    using A = Acc<T>;
    constexpr int N = VecOf<T>::N;
    volatile DevState* vst = a.st;
    if (block == 0 && threadIdx.x == 0) a.st->t_sweep = vst->t;
    const uint32_t vpr = (uint32_t)(a.Kp / N);
    const uint64_t total = (uint64_t)a.n * vpr;
    const uint64_t stride = (uint64_t)nblocks * blockDim.x;
    typename A::V zacc = A::zero();
    T cons = T(0);
    for (uint64_t idx = (uint64_t)block * blockDim.x + threadIdx.x; idx < total; idx += stride) {
        uint32_t i, v;
        if (total <= 0xffffffffull) {
            i = (uint32_t)idx / vpr;
            v = (uint32_t)idx - i * vpr;
        } else {
            i = (uint32_t)(idx / vpr);
            v = (uint32_t)(idx - (uint64_t)i * vpr);
        }
        T acc[N];
#pragma unroll
        for (int j = 0; j < N; ++j) acc[j] = T(0);
        // incidence list: in-edges e (added), then out-edges ~e (subtracted),
        // up to eight rows in flight; the additions keep list order
        const int64_t q0 = a.inc_ptr[i], q1 = a.inc_ptr[i + 1];
        int64_t q = q0;
        for (; q + 8 <= q1; q += 8) {
            int32_t ev[8];
            T x[8][N];
#pragma unroll
            for (int u = 0; u < 8; ++u) ev[u] = a.inc[q + u];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int64_t e = ev[u] >= 0 ? ev[u] : ~ev[u];
                unpack(reinterpret_cast<const VT*>(a.f + e * a.Kp)[v], x[u]);
            }
#pragma unroll
            for (int u = 0; u < 8; ++u)
#pragma unroll
                for (int j = 0; j < N; ++j) acc[j] = ev[u] >= 0 ? acc[j] + x[u][j] : acc[j] - x[u][j];
        }
        if (q + 4 <= q1) {
            int32_t ev[4];
            T x[4][N];
#pragma unroll
            for (int u = 0; u < 4; ++u) ev[u] = a.inc[q + u];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int64_t e = ev[u] >= 0 ? ev[u] : ~ev[u];
                unpack(reinterpret_cast<const VT*>(a.f + e * a.Kp)[v], x[u]);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int j = 0; j < N; ++j) acc[j] = ev[u] >= 0 ? acc[j] + x[u][j] : acc[j] - x[u][j];
            q += 4;
        }
        for (; q < q1; ++q) {
            const int32_t ev = a.inc[q];
            const int64_t e = ev >= 0 ? ev : ~ev;
            T x[N];
            unpack(reinterpret_cast<const VT*>(a.f + e * a.Kp)[v], x);
#pragma unroll
            for (int j = 0; j < N; ++j) acc[j] = ev >= 0 ? acc[j] + x[j] : acc[j] - x[j];
        }
        const int k0 = (int)v * N;
#pragma unroll
        for (int j = 0; j < N; ++j) {
            const int k = k0 + j;
            if (a.s[k] == (int)i) acc[j] += a.dem[k];
            else if (a.t[k] == (int)i) acc[j] -= a.dem[k];
        }
        const T dgt = T((int)(q1 - q0));  // delta_i < 2^31: a 32-bit conversion
        const T idg = a.inv_deg[i];
        T hv[N];
#pragma unroll
        for (int j = 0; j < N; ++j) hv[j] = acc[j] * idg;
        reinterpret_cast<VT*>(a.h + (int64_t)i * a.Kp)[v] = pack4(hv);
        // delta_i h^2 and |Delta|/d; pad entries have h = 0 and 1/d = 0
        T zt = T(0);
#pragma unroll
        for (int j = 0; j < N; ++j) {
            zt += dgt * hv[j] * hv[j];
            const T r = fabs(acc[j]) * a.inv_dem[k0 + j];
            cons = r > cons ? r : cons;
        }
        zacc = A::add(zacc, zt);
    }
    excess_tail<T, SH>(a, block, nblocks, zacc, cons);
}

// End of an excess pass in every block: add this block's fixed slice of the
// edge kernel's psi partials and write the block's three partials.  Every
// thread of the block calls it.
template <typename T, bool SH>
__device__ __forceinline__ void excess_tail(const SweepArgs<T>& a, int block, int nblocks,
                                            typename Acc<T>::V zacc, T cons)
{
    using A = Acc<T>;
    T capb = T(0);
    {
        // the block's slice [lo, hi) of the edge partials (SH: the one block takes all)
        const int64_t lo = SH ? 0 : (int64_t)block * a.n_psi / nblocks;
        const int64_t hi = SH ? a.n_psi : (int64_t)(block + 1) * a.n_psi / nblocks;
        const typename A::S* pp = reinterpret_cast<const typename A::S*>(a.part_psi);
        for (int64_t b = lo + threadIdx.x; b < hi; b += blockDim.x) {
            zacc = A::add(zacc, A::unstore(ld_part<SH>(pp + b)));
            const T c = ld_part<SH>(a.part_cap + b);
            capb = c > capb ? c : capb;
        }
    }
    block_acc_max2<T>(zacc, cons, capb);
    if (threadIdx.x == 0) {
        a.part_h[block] = A::to_double(zacc);
        a.part_cons[block] = cons;
        a.part_capb[block] = capb;
    }
}

template <typename T>
__global__ void __launch_bounds__(kThreads) excess_kernel(SweepArgs<T> a)
{
    pdl_wait();     // the previous sweep's edge kernel has finished (no-op without PDL)
    pdl_trigger();  // one wave: the edge kernel's blocks may queue behind this one's
    volatile DevState* vst = a.st;
    if (sweep_stopped(a)) return;  // an earlier sweep of this solve stopped
    excess_body<T>(a, blockIdx.x, gridDim.x);
}

// ------------------------------------------------------------------ excess by bulk copies
//
// The same pass as excess_body, with the incident flow rows brought into
// shared memory by cp.async.bulk instead of per-thread gathers: the sums
// run in the same order, so the heights are bit-identical.  Block b owns
// the vertices xv_start[b] .. xv_start[b+1]-1 (contiguous, about equal
// incidence count).  A vertex row is cut into 2 KB segments (512 FP32 or 256
// FP64 values); a unit is one (vertex, segment) and a batch is up to R
// incident rows of a unit.  One producer warp walks the units segment by
// segment (all of the block's vertices for segment 0, then segment 1, ...),
// reads inc_ptr and 1/delta 32 vertices at a time and the incidence list
// through a window of 64 entries held in its lanes (the lists of a block's
// vertices are contiguous), and issues one bulk copy per row into a ring of
// S stages; four consumer warps (one 16-byte vector per thread) add the
// rows in list order and write the unit's heights after its last batch,
// with the commodity data of their values (s, t, d, 1/d) held in registers
// for the whole segment.  Full and empty mbarriers order the ring.  Every wait has
// a time limit; a block whose wait runs out sets DevState::fault and stop,
// waits (with the same limit) for the copies it issued, and leaves.

// C consumer threads (one 16-byte vector each) per block, plus the producer
// warp; a row segment is C x 16 bytes (2 KB for C = 128, 512 B for C = 32).
// Smaller segments keep every block's pass over one segment of all its rows
// smaller, so that a row's second visit (from its other endpoint, in another
// block) finds it in L2 when the two endpoints are far apart in vertex order.
template <int C>
__host__ __device__ constexpr int xseg_bytes()
{
    return C * 16;
}
constexpr int kXFirst = 1, kXLast = 2, kXEnd = 4;

struct XDesc {
    int32_t i, c, nrows, flags;
    uint32_t sign;  // bit r: row r of the batch is an in-edge (added), else an out-edge
    int32_t deg;    // delta_i
    double idg;     // 1/delta_i in the working precision (exact in double)
};

template <int S, int R, int C>
constexpr size_t excess_bulk_smem()
{
    return (size_t)S * R * xseg_bytes<C>() + (size_t)S * (2 * sizeof(uint64_t) + sizeof(XDesc));
}

// S stages of R row segments of C x 16 bytes
template <typename T, int S, int R, int C>
__global__ void __launch_bounds__(C + 32) excess_bulk_kernel(SweepArgs<T> a)
{
    using VT = typename VecOf<T>::type;
    using A = Acc<T>;
    constexpr int N = VecOf<T>::N;
    constexpr int kXCons = C;
    constexpr int kXSegBytes = xseg_bytes<C>();
    constexpr int W = kXSegBytes / (int)sizeof(T);  // values per segment
    extern __shared__ __align__(128) unsigned char xsm[];
    unsigned char* ring = xsm;
    uint64_t* full = reinterpret_cast<uint64_t*>(xsm + (size_t)S * R * kXSegBytes);
    uint64_t* empty = full + S;
    XDesc* desc = reinterpret_cast<XDesc*>(empty + S);

    const int block = blockIdx.x;
    const int lane = threadIdx.x & 31;
    const bool producer = threadIdx.x >= kXCons;
    if (threadIdx.x == 0) {
        for (int q = 0; q < S; ++q) {
            mbar_init(&full[q], 1);
            mbar_init(&empty[q], kXCons / 32);
        }
        mbar_init_fence();
    }
    // The adjacency and the commodity data do not change during a solve:
    // read the first of them before waiting for the previous kernel.
    // Producer lane l: inc_ptr and 1/delta of vertex vlo + l (and of
    // vlo + 32 + l), incidence entries wb0 + l and wb0 + 32 + l.
    // Consumer: the commodity data of its values in segment 0.
    const int32_t vlo = a.xv_start[block], vhi = a.xv_start[block + 1];
    const int nseg = (a.Kp + W - 1) / W;
    const int64_t ninc = 2 * a.m;
    const int64_t vlim = (int64_t)a.n;
    int64_t ip0 = 0, ipn0 = 0, wb0 = 0;
    T dg0 = T(0), dgn0 = T(0);
    int32_t cur0 = 0, nxt0 = 0;
    T dk[N], idk[N];
    int32_t sk[N], tk[N];
    const int tid = threadIdx.x;
    bool mine = tid * N < a.Kp;  // consumer: this thread's values exist in segment 0
    if (producer) {
        ip0 = vlo + lane <= vlim ? a.inc_ptr[vlo + lane] : 0;
        ipn0 = vlo + 32 + lane <= vlim ? a.inc_ptr[vlo + 32 + lane] : 0;
        dg0 = vlo + lane < vlim ? a.inv_deg[vlo + lane] : T(0);
        dgn0 = vlo + 32 + lane < vlim ? a.inv_deg[vlo + 32 + lane] : T(0);
        wb0 = __shfl_sync(kFull, ip0, 0);
        cur0 = wb0 + lane < ninc ? a.inc[wb0 + lane] : 0;
        nxt0 = wb0 + 32 + lane < ninc ? a.inc[wb0 + 32 + lane] : 0;
    } else if (mine) {
#pragma unroll
        for (int q = 0; q < N; ++q) {
            sk[q] = a.s[tid * N + q];
            tk[q] = a.t[tid * N + q];
            dk[q] = a.dem[tid * N + q];
            idk[q] = a.inv_dem[tid * N + q];
        }
    }

    pdl_wait();
    pdl_trigger();  // one wave
    volatile DevState* vst = a.st;
    if (sweep_stopped(a)) return;  // an earlier sweep of this solve stopped
    if (block == 0 && threadIdx.x == 0) a.st->t_sweep = vst->t;

    typename A::V zacc = A::zero();
    T cons = T(0);
    bool ok = true;
    if (producer) {
        // producer warp; every branch below is warp-uniform
        uint32_t j = 0;
        // units in segment-major order: every vertex of the range for segment 0, then 1, ...
        for (int c = 0; c < nseg && ok; ++c) {
            const int width = min(W, a.Kp - c * W);
            const uint32_t bytes = (uint32_t)width * (uint32_t)sizeof(T);
            int64_t ip = ip0, ipn = ipn0, wb = wb0;
            T dg = dg0, dgn = dgn0;
            int32_t cur = cur0, nxt = nxt0;
            int32_t vb = vlo;
            for (int32_t i = vlo; i < vhi && ok; ++i) {
                if (i - vb == 32) {  // next 32 vertices
                    vb += 32;
                    ip = ipn;
                    dg = dgn;
                    ipn = (int64_t)vb + 32 + lane <= vlim ? a.inc_ptr[vb + 32 + lane] : 0;
                    dgn = (int64_t)vb + 32 + lane < vlim ? a.inv_deg[vb + 32 + lane] : T(0);
                }
                const int o = i - vb;
                const int64_t q0 = __shfl_sync(kFull, ip, o);
                const int64_t q1a = __shfl_sync(kFull, ip, (o + 1) & 31), q1b = __shfl_sync(kFull, ipn, 0);
                const int64_t q1 = o < 31 ? q1a : q1b;
                const T idg = __shfl_sync(kFull, dg, o);
                if (q0 >= wb + 64) {  // keep wb <= q0 < wb + 32
                    wb = q0;
                    cur = wb + lane < ninc ? a.inc[wb + lane] : 0;
                    nxt = wb + 32 + lane < ninc ? a.inc[wb + 32 + lane] : 0;
                } else if (q0 >= wb + 32) {
                    cur = nxt;
                    wb += 32;
                    nxt = wb + 32 + lane < ninc ? a.inc[wb + 32 + lane] : 0;
                }
                for (int64_t r0 = q0;; r0 += R) {
                    const int nr = (int)(q1 - r0 < R ? q1 - r0 : R);  // 0: isolated vertex
                    const int slot = (int)(j % S);
                    const uint32_t ph = (j / S) & 1u;
                    if (j >= (uint32_t)S && !__all_sync(kFull, mbar_wait(&empty[slot], ph ^ 1u, a.wait_cycles))) {
                        ok = false;
                        break;
                    }
                    const int64_t r = r0 + lane, off = r - wb;  // off >= 0
                    const int32_t from_cur = __shfl_sync(kFull, cur, (int)(off & 31));
                    const int32_t from_nxt = __shfl_sync(kFull, nxt, (int)(off & 31));
                    int32_t ev = 0;
                    if (lane < nr) ev = off < 32 ? from_cur : (off < 64 ? from_nxt : a.inc[r]);
                    const uint32_t sign = __ballot_sync(kFull, lane < nr && ev >= 0);
                    if (lane == 0) {
                        XDesc& d = desc[slot];
                        d.i = i;
                        d.c = c;
                        d.nrows = nr;
                        d.sign = sign;
                        d.deg = (int32_t)(q1 - q0);
                        d.flags = (r0 == q0 ? kXFirst : 0) | (r0 + R >= q1 ? kXLast : 0);
                        d.idg = (double)idg;
                        mbar_arrive_expect_tx(&full[slot], (uint32_t)nr * bytes);
                    }
                    __syncwarp();
                    if (lane < nr) {
                        const int64_t e = ev >= 0 ? ev : ~ev;
                        bulk_g2s(ring + ((size_t)slot * R + lane) * kXSegBytes, a.f + e * a.Kp + (int64_t)c * W,
                                 bytes, &full[slot]);
                    }
                    ++j;
                    if (r0 + R >= q1) break;
                }
            }
        }
        if (ok) {  // end marker
            const int slot = (int)(j % S);
            const uint32_t ph = (j / S) & 1u;
            if (j >= (uint32_t)S && !__all_sync(kFull, mbar_wait(&empty[slot], ph ^ 1u, a.wait_cycles))) {
                ok = false;
            } else if (lane == 0 && !a.hold_end) {  // hold_end: a test of the consumers' time limit
                desc[slot].flags = kXEnd;
                desc[slot].nrows = 0;
                mbar_arrive(&full[slot]);
            }
        }
        if (!ok) {
            // wait (limited) for the copies of the last S batches, then leave
            for (uint32_t q = j > (uint32_t)S ? j - S : 0; q < j; ++q) mbar_wait(&full[q % S], (q / S) & 1u, a.wait_cycles);
        }
    } else {
        // consumers: thread tid holds values tid*N .. tid*N+N-1 of the segment;
        // the commodity data of those values is reloaded when the segment changes
        T acc[N];
        int cs = 0;
#pragma unroll
        for (int q = 0; q < N; ++q) acc[q] = T(0);
        for (uint32_t j = 0;; ++j) {
            const int slot = (int)(j % S);
            const uint32_t ph = (j / S) & 1u;
            if (!__all_sync(kFull, mbar_wait(&full[slot], ph, a.wait_cycles))) {
                ok = false;
                break;
            }
            const XDesc d = desc[slot];
            if (d.flags & kXEnd) break;
            if (d.c != cs) {
                cs = d.c;
                const int k0 = cs * W + tid * N;
                mine = k0 < a.Kp && tid * N < W;
                if (mine) {
#pragma unroll
                    for (int q = 0; q < N; ++q) {
                        sk[q] = a.s[k0 + q];
                        tk[q] = a.t[k0 + q];
                        dk[q] = a.dem[k0 + q];
                        idk[q] = a.inv_dem[k0 + q];
                    }
                }
            }
            if (d.flags & kXFirst) {
#pragma unroll
                for (int q = 0; q < N; ++q) acc[q] = T(0);
            }
            if (mine) {
                const VT* rows = reinterpret_cast<const VT*>(ring + (size_t)slot * R * kXSegBytes) + tid;
                for (int r = 0; r < d.nrows; ++r) {
                    T x[N];
                    unpack(rows[r * (kXSegBytes / 16)], x);
                    const bool add = (d.sign >> r) & 1u;
#pragma unroll
                    for (int q = 0; q < N; ++q) acc[q] = add ? acc[q] + x[q] : acc[q] - x[q];
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[slot]);
            if ((d.flags & kXLast) && mine) {
                const int32_t i = d.i;
#pragma unroll
                for (int q = 0; q < N; ++q) {
                    if (sk[q] == i) acc[q] += dk[q];
                    else if (tk[q] == i) acc[q] -= dk[q];
                }
                const T dgt = T(d.deg);
                const T idg = (T)d.idg;
                T hv[N];
#pragma unroll
                for (int q = 0; q < N; ++q) hv[q] = acc[q] * idg;
                reinterpret_cast<VT*>(a.h + (int64_t)i * a.Kp + cs * W + tid * N)[0] = pack4(hv);
                T zt = T(0);
#pragma unroll
                for (int q = 0; q < N; ++q) {
                    zt += dgt * hv[q] * hv[q];
                    const T rr = fabs(acc[q]) * idk[q];
                    cons = rr > cons ? rr : cons;
                }
                zacc = A::add(zacc, zt);
            }
        }
    }
    if (!__syncthreads_and(ok)) {
        if (threadIdx.x == 0) {
            a.st->fault = 1;
            stop_from_kernel(a);
        }
    }
    excess_tail<T>(a, block, gridDim.x, zacc, cons);
}

// xv_start[b] = the first vertex i with inc_ptr[i] + 2 i >= b * (inc_ptr[n] + 2 n) / grid
__global__ void excess_split_kernel(const int64_t* inc_ptr, int32_t n, int grid, int32_t* xv_start)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b > grid) return;
    const int64_t total = inc_ptr[n] + 2 * (int64_t)n;
    const int64_t target = total / grid * b + total % grid * b / grid;  // floor(total * b / grid)
    int32_t lo = 0, hi = n;  // the answer lies in [lo, hi]
    while (lo < hi) {
        const int32_t mid = lo + (hi - lo) / 2;
        if (inc_ptr[mid] + 2 * (int64_t)mid >= target) hi = mid;
        else lo = mid + 1;
    }
    xv_start[b] = lo;
}

// ------------------------------------------------------------------ the root search of Alg. 2
//
// Every pass over a row returns three group-wide values for a threshold w:
// S(w) = sum of the c_k > w, n(w) = their number and m(w) = the smallest of
// them.  theta = (S(w) - u)/(2 + n(w)) is the root of the active set
// A = {c > w}; if m(w) > theta, no element of A falls at or below theta, so A
// is the active set of its own root and the search ends without another
// pass.  Otherwise the elements c <= theta leave (Michelot's step) and the
// next pass starts at theta.  In a converged solve the warm start w lies just
// below the root with no element in between, so one pass decides the edge.

template <int G, typename X>
__device__ __forceinline__ X group_min(X x)
{
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) {
        const X y = __shfl_xor_sync(kFull, x, o);
        x = y < x ? y : x;
    }
    return x;
}

template <typename T, int G, int V, int N>
__device__ __forceinline__ void above(const T (&c)[V][N], T w, T& S, int& n, T& mn)
{
    T sl = T(0), ml = T(INFINITY);
    int nl = 0;
#pragma unroll
    for (int q = 0; q < V; ++q)
#pragma unroll
        for (int j = 0; j < N; ++j) {
            const T x = c[q][j];
            if (x > w) {
                sl += x;
                ++nl;
                ml = x < ml ? x : ml;
            }
        }
    S = group_sum<G>(sl);
    if constexpr (G == 32 && sizeof(T) == 4) {
        // whole-warp groups: one redux each for the count and the minimum
        // (every counted x exceeds w >= 0, so ml is positive or +inf and its
        // bit pattern orders as an unsigned integer)
        n = (int)__reduce_add_sync(kFull, (unsigned)nl);
        mn = __uint_as_float(__reduce_min_sync(kFull, __float_as_uint(ml)));
    } else {
        n = group_sum<G>(nl);
        mn = group_min<G>(ml);
    }
}

// Case decision and root from the sums above a threshold w >= 0 that is known
// to lie at or below the root (w = 0, or g(w) >= 0 certified).  den = 2 for
// Alg. 2 (the congestion term of eq. (10) gives theta = (S_A - u)/(2 + |A|));
// den = 0 with the capacity kept (Program (6): sum_A (c - theta) = u).
template <typename T>
__device__ __forceinline__ void start_root(T S, int n, T mn, T ue, int den, T& theta, int& nA, bool& done)
{
    if (S <= ue) {  // Case 1 of Alg. 2: nothing to shed
        theta = T(0);
        done = true;
    } else {  // Case 2 (S > u >= 0, so n >= 1)
        theta = (S - ue) / T(den + n);
        nA = n;
        done = mn > theta;
    }
}

// theta = psi'/2 for the row c (all lanes of the warp call it; `valid` is
// uniform over the lane group).  w0 is the warm start (>= 0).
template <typename T, int G, int V, int N>
__device__ __forceinline__ T qp_root_group(const T (&c)[V][N], T ue, T w0, bool valid, int Kp, int den)
{
    T S, mn, theta = T(0);
    int n, nA = 0;
    bool done = !valid, cold = false;
    above<T, G, V, N>(c, w0, S, n, mn);
    if (valid) {
        if (w0 <= T(0)) start_root(S, n, mn, ue, den, theta, nA, done);
        else if (n > 0 && S - T(n) * w0 - ue - T(den) * w0 >= T(0)) {
            // g(w0) = sum max(0, c - w0) - u - den w0 >= 0: w0 <= root, Case 2
            theta = (S - ue) / T(den + n);
            nA = n;
            done = mn > theta;
        } else {
            cold = true;  // the root dropped below the warm start
        }
    }
    if (__any_sync(kFull, cold)) {
        T S0, m0;
        int n0;
        above<T, G, V, N>(c, T(0), S0, n0, m0);
        if (cold) start_root(S0, n0, m0, ue, den, theta, nA, done);
    }
    for (int it = 0; __any_sync(kFull, !done); ++it) {
        T S2, m2;
        int n2;
        above<T, G, V, N>(c, theta, S2, n2, m2);
        if (!done) {
            if (n2 >= nA || n2 == 0) done = true;  // no element left: keep theta
            else {
                nA = n2;
                theta = (S2 - ue) / T(den + n2);
                done = m2 > theta;
            }
        }
        if (it > Kp + 2) break;  // unreachable: nA drops every round
    }
    // A Case 2 root below 0 can only come from rounding in sums that put
    // s = sum max(0, c) within rounding of u: that edge is in Case 1 (root 0).
    // Without the clamp, f' = max(0, c - theta) would lift every c <= 0 --
    // the zero padding included -- to -theta.
    return theta > T(0) ? theta : T(0);
}

// Warm start of the next sweep's root search from this sweep's root theta
// and the previous one, prev.  A root that rose is expected to stay at or
// above theta; one that fell is expected to fall by about as much again.
// Starting the search at the previous root itself leaves out the many
// entries whose flows have decayed to zero, which sit just above it (c_k =
// theta + f'_k): one pass decides almost every edge.  A start above the
// new root is detected by its certificate g(w) < 0 and costs a cold pass.
template <typename T>
__device__ __forceinline__ T next_warm_start(T theta, T prev)
{
    if (theta > prev) return theta;
    const T w = T(0.999) * theta + T(2) * (theta - prev);
    return w > T(0) ? w : T(0);
}

// ------------------------------------------------------------------ edge QP, lane-group form

// One aligned group of G lanes per edge; each lane keeps V vectors of the
// edge's row in registers (vector q of lane l is row vector l + q*G, so a
// group reads contiguous memory).  K <= G * V * N.
// Loads of data written by an earlier kernel of the same sweep: through the
// read-only path in a standalone kernel; plain (coherent) loads inside the
// persistent kernel, where the data changes between its grid barriers.
template <bool P, typename X>
__device__ __forceinline__ X ld_row(const X* p)
{
    if constexpr (P) return *p;
    else return __ldg(p);
}

// Body of one edge-QP pass of the lane-group form, run by edge block `block`
// of `nblocks` (the decision block is not counted).
template <typename T, int G, int V, bool P>
__device__ __forceinline__ void edge_group_body(const SweepArgs<T>& a, int block, int nblocks)
{
    using VT = typename VecOf<T>::type;
    constexpr int N = VecOf<T>::N;
    constexpr int GPW = 32 / G;  // groups per warp
    using A = Acc<T>;
    const int lane = threadIdx.x & 31;
    const int gl = lane & (G - 1);
    const int gw = lane / G;
    const int64_t warp = ((int64_t)block * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)nblocks * blockDim.x) >> 5;
    const int vpr = a.Kp / N;
    const bool psi_only = (a.mode == MODE_PSI);
    typename A::V zpsi = A::zero();
    T capmax = T(0);
    for (int64_t base = warp * GPW; base < a.m; base += nwarps * GPW) {
        const int64_t e = base + gw;
        const bool valid = e < a.m;
        if (a.pf_edges > 0 && valid && e + a.pf_edges < a.m)  // the flow row a later wave reads
            prefetch_l2(a.f + (e + a.pf_edges) * a.Kp, (int64_t)a.Kp * sizeof(T), gl, G);
        const T ue = valid ? a.u[e] : T(0);
        T c[V][N];
        const T* frow = a.f + (valid ? e : 0) * a.Kp;
        T* orow = a.f_out + (valid ? e : 0) * a.Kp;
        if (psi_only) {
#pragma unroll
            for (int q = 0; q < V; ++q) {
                const int v = gl + q * G;
                if (valid && v < vpr) unpack(reinterpret_cast<const VT*>(frow)[v], c[q]);
                else
#pragma unroll
                    for (int j = 0; j < N; ++j) c[q][j] = T(0);
            }
        } else {
            const int i = valid ? a.src[e] : 0;
            const int jv = valid ? a.col[e] : 0;
            const VT* hi = reinterpret_cast<const VT*>(a.h + (int64_t)i * a.Kp);
            const VT* hj = reinterpret_cast<const VT*>(a.h + (int64_t)jv * a.Kp);
#pragma unroll
            for (int q = 0; q < V; ++q) {
                const int v = gl + q * G;
                if (valid && v < vpr) {
                    T fx[N], ax[N], bx[N];
                    unpack(reinterpret_cast<const VT*>(frow)[v], fx);
                    unpack(ld_row<P>(hi + v), ax);
                    unpack(ld_row<P>(hj + v), bx);
                    // c_k = 1/2 ((h_ik + f_k) - (h_jk - f_k)) = f_k + (h_ik - h_jk)/2
#pragma unroll
                    for (int j = 0; j < N; ++j) c[q][j] = fma(T(0.5), ax[j] - bx[j], fx[j]);
                } else {
#pragma unroll
                    for (int j = 0; j < N; ++j) c[q][j] = T(0);
                }
            }
        }
        T psi;
        if (!psi_only) {
            // warm start left by the previous sweep (roots in [0, m), starts in [m, 2m))
            const T w = valid ? a.theta_in[a.m + e] : T(0);
            const int den = a.ck ? 0 : 2;
            const T theta = qp_root_group<T, G, V, N>(c, ue, w, valid, a.Kp, den);
            if (valid && gl == 0) {
                a.theta[a.m + e] = next_warm_start(theta, a.theta_in[e]);
                a.theta[e] = theta;
            }
            // f' = max(0, c - theta); at the root sum f' - u = den theta, so the
            // congestion of the new flows is psi' = 2 theta for Alg. 2 and 0 with
            // the capacity kept (and 0 in Case 1)
#pragma unroll
            for (int q = 0; q < V; ++q) {
                const int v = gl + q * G;
                T o[N];
#pragma unroll
                for (int j = 0; j < N; ++j) {
                    const T x = c[q][j] - theta;
                    o[j] = x > T(0) ? x : T(0);
                }
                if (valid && v < vpr) reinterpret_cast<VT*>(orow)[v] = pack4(o);
            }
            psi = T(den) * theta;
        } else {
            // congestion of the stored flows
            T rs = T(0);
#pragma unroll
            for (int q = 0; q < V; ++q)
#pragma unroll
                for (int j = 0; j < N; ++j) rs += c[q][j];
            rs = group_sum<G>(rs);
            psi = rs - ue > T(0) ? rs - ue : T(0);
        }
        if (valid && gl == 0) {
            zpsi = A::add(zpsi, psi * psi);
            const T c = psi * a.inv_scale_t[e];
            capmax = c > capmax ? c : capmax;
            if (a.psi_out) a.psi_out[e] = psi;
        }
    }
    // one partial per warp, no block barrier
    warp_acc_max<T>(zpsi, capmax);
    if (lane == 0) {
        reinterpret_cast<typename A::S*>(a.part_psi)[warp] = A::store(zpsi);
        a.part_cap[warp] = capmax;
    }
}

template <typename T, int G, int V>
__global__ void __launch_bounds__(kThreads) edge_group_kernel(SweepArgs<T> a)
{
    pdl_wait();  // the excess kernel has finished (no-op without PDL)
    volatile DevState* vst = a.st;
    if (sweep_stopped(a)) return;  // an earlier sweep of this solve stopped
    if (blockIdx.x == gridDim.x - 1) {               // the decision block
        if (a.mode != MODE_PSI) reduce_and_finalize(a);
        return;
    }
    if (final_evaluation(a)) return;  // the sweep cap stops this sweep: its output is not used
    edge_group_body<T, G, V, false>(a, blockIdx.x, gridDim.x - 1);
}

// ------------------------------------------------------------------ edge QP, pipelined lane-group form

// Persistent form of edge_group_kernel for one 32-lane group per edge: each
// warp walks a fixed stride of edges and loads the next edge's three rows
// into registers before it solves the current one, so the loads of edge
// e + stride are in flight during the active-set search of edge e.
template <typename T, int V>
__device__ __forceinline__ void pipe_load(const SweepArgs<T>& a, int64_t e, int gl, int vpr,
                                          typename VecOf<T>::type (&fv)[V], typename VecOf<T>::type (&av)[V],
                                          typename VecOf<T>::type (&bv)[V])
{
    using VT = typename VecOf<T>::type;
    const bool valid = e < a.m;
    const VT* frow = reinterpret_cast<const VT*>(a.f + (valid ? e : 0) * a.Kp);
    const VT* hi = reinterpret_cast<const VT*>(a.h + (int64_t)(valid ? a.src[e] : 0) * a.Kp);
    const VT* hj = reinterpret_cast<const VT*>(a.h + (int64_t)(valid ? a.col[e] : 0) * a.Kp);
#pragma unroll
    for (int q = 0; q < V; ++q) {
        const int v = gl + q * 32;
        if (valid && v < vpr) {
            fv[q] = frow[v];
            av[q] = __ldg(hi + v);
            bv[q] = __ldg(hj + v);
        }
    }
}

template <typename T, int V>
__global__ void __launch_bounds__(kThreads, 2) edge_pipe_kernel(SweepArgs<T> a)
{
    pdl_wait();  // the excess kernel has finished (no-op without PDL)
    using VT = typename VecOf<T>::type;
    using A = Acc<T>;
    constexpr int N = VecOf<T>::N;
    volatile DevState* vst = a.st;
    if (sweep_stopped(a)) return;  // an earlier sweep of this solve stopped
    if (blockIdx.x == gridDim.x - 1) {
        if (a.mode != MODE_PSI) reduce_and_finalize(a);
        return;
    }
    if (final_evaluation(a)) return;  // the sweep cap stops this sweep: its output is not used
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)(gridDim.x - 1) * blockDim.x) >> 5;
    const int vpr = a.Kp / N;
    const bool psi_only = (a.mode == MODE_PSI);
    typename A::V zpsi = A::zero();
    T capmax = T(0);
    VT fv[V], av[V], bv[V];
#pragma unroll
    for (int q = 0; q < V; ++q) fv[q] = av[q] = bv[q] = VT{};
    pipe_load<T, V>(a, warp, lane, vpr, fv, av, bv);
    for (int64_t e = warp; e < a.m; e += nwarps) {
        // rows of this edge into c, then start the next edge's loads
        T c[V][N];
#pragma unroll
        for (int q = 0; q < V; ++q) {
            T fx[N], ax[N], bx[N];
            unpack(fv[q], fx);
            unpack(av[q], ax);
            unpack(bv[q], bx);
#pragma unroll
            for (int j = 0; j < N; ++j) c[q][j] = psi_only ? fx[j] : fma(T(0.5), ax[j] - bx[j], fx[j]);
        }
        const T ue = a.u[e];
        const int64_t en = e + nwarps;
#pragma unroll
        for (int q = 0; q < V; ++q) fv[q] = av[q] = bv[q] = VT{};
        if (en < a.m) pipe_load<T, V>(a, en, lane, vpr, fv, av, bv);
        T psi;
        if (!psi_only) {
            const int den = a.ck ? 0 : 2;
            const T theta = qp_root_group<T, 32, V, N>(c, ue, a.theta_in[a.m + e], true, a.Kp, den);
            if (lane == 0) {
                a.theta[a.m + e] = next_warm_start(theta, a.theta_in[e]);
                a.theta[e] = theta;
            }
            T* orow = a.f_out + e * a.Kp;
#pragma unroll
            for (int q = 0; q < V; ++q) {
                const int v = lane + q * 32;
                T o[N];
#pragma unroll
                for (int j = 0; j < N; ++j) {
                    const T x = c[q][j] - theta;
                    o[j] = x > T(0) ? x : T(0);
                }
                if (v < vpr) reinterpret_cast<VT*>(orow)[v] = pack4(o);
            }
            psi = T(den) * theta;  // sum f' - u at the root
        } else {
            T rs = T(0);
#pragma unroll
            for (int q = 0; q < V; ++q)
#pragma unroll
                for (int j = 0; j < N; ++j) rs += c[q][j];
            rs = group_sum<32>(rs);
            psi = rs - ue > T(0) ? rs - ue : T(0);
        }
        if (lane == 0) {
            zpsi = A::add(zpsi, psi * psi);
            const T cc = psi * a.inv_scale_t[e];
            capmax = cc > capmax ? cc : capmax;
            if (a.psi_out) a.psi_out[e] = psi;
        }
    }
    warp_acc_max<T>(zpsi, capmax);
    if (lane == 0) {
        reinterpret_cast<typename A::S*>(a.part_psi)[warp] = A::store(zpsi);
        a.part_cap[warp] = capmax;
    }
}

// ------------------------------------------------------------------ edge QP, block form (large K)

// Block-wide S(w), n(w), m(w) of a row held by the whole block (thread l keeps
// vectors l + q*B); the same value in every thread.  The warp partials go to
// slots 0..31 of sa/sb/sm (33 entries each); warp 0 combines them lane-parallel
// and leaves the totals in slot 32, which every thread reads after the second
// barrier.  A serial walk over the partials by every thread would put one
// dependent shared-memory load per warp on the critical path of every pass.
template <typename T, int V, int N>
__device__ __forceinline__ void block_above(const T (&c)[V][N], T w, T& S, int& n, T& mn, T* sa, int* sb, T* sm)
{
    T sl = T(0), ml = T(INFINITY);
    int nl = 0;
#pragma unroll
    for (int q = 0; q < V; ++q)
#pragma unroll
        for (int j = 0; j < N; ++j) {
            const T x = c[q][j];
            if (x > w) {
                sl += x;
                ++nl;
                ml = x < ml ? x : ml;
            }
        }
    warp_sum_count_min(sl, nl, ml);
    const int wi = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) {
        sa[wi] = sl;
        sb[wi] = nl;
        sm[wi] = ml;
    }
    __syncthreads();
    if (wi == 0) {
        const int nw = blockDim.x >> 5;
        T ts = l < nw ? sa[l] : T(0), tm = l < nw ? sm[l] : T(INFINITY);
        int tn = l < nw ? sb[l] : 0;
        warp_sum_count_min(ts, tn, tm);
        if (l == 0) {
            sa[32] = ts;
            sb[32] = tn;
            sm[32] = tm;
        }
    }
    __syncthreads();
    S = sa[32];
    n = sb[32];
    mn = sm[32];
}

// One block of B threads per edge; thread l keeps row vectors l + q*B.
template <typename T, int B, int V>
__global__ void __launch_bounds__(B, block_min_blocks(B, V)) edge_block_kernel(SweepArgs<T> a)
{
    pdl_wait();  // the excess kernel has finished (no-op without PDL)
    using VT = typename VecOf<T>::type;
    constexpr int N = VecOf<T>::N;
    using A = Acc<T>;
    __shared__ T sa_buf[33];
    __shared__ int sb_buf[33];
    __shared__ T sm_buf[33];
    volatile DevState* vst = a.st;
    if (sweep_stopped(a)) return;  // an earlier sweep of this solve stopped
    if (blockIdx.x == gridDim.x - 1) {               // the decision block
        if (a.mode != MODE_PSI) reduce_and_finalize(a);
        return;
    }
    if (final_evaluation(a)) return;  // the sweep cap stops this sweep: its output is not used
    const int vpr = a.Kp / N;
    const bool psi_only = (a.mode == MODE_PSI);
    const bool hint = a.l2_hints != 0;
    const uint64_t pol_first = l2_evict_first();
    typename A::V zpsi = A::zero();
    T capmax = T(0);
    for (int64_t e = blockIdx.x; e < a.m; e += gridDim.x - 1) {
        const int64_t ep = e + a.pf_edges;  // an edge of a later wave
        const bool pf = a.pf_edges > 0 && ep < a.m;
        int32_t ps = 0, pc = 0;
        if (pf) {
            ps = a.src[ep];
            pc = a.col[ep];
            prefetch_l2(a.f + ep * a.Kp, (int64_t)a.Kp * sizeof(T), threadIdx.x, B);
        }
        const T ue = a.u[e];
        T c[V][N];
        const T* frow = a.f + e * a.Kp;
        T* orow = a.f_out + e * a.Kp;
        const VT* hi = reinterpret_cast<const VT*>(a.h + (int64_t)a.src[e] * a.Kp);
        const VT* hj = reinterpret_cast<const VT*>(a.h + (int64_t)a.col[e] * a.Kp);
#pragma unroll
        for (int q = 0; q < V; ++q) {
            const int v = threadIdx.x + q * B;
            if (v < vpr) {
                T fx[N];
                if (hint) unpack(ld_hint(reinterpret_cast<const VT*>(frow) + v, pol_first), fx);
                else unpack(reinterpret_cast<const VT*>(frow)[v], fx);
                if (psi_only) {
#pragma unroll
                    for (int j = 0; j < N; ++j) c[q][j] = fx[j];
                } else {
                    T ax[N], bx[N];
                    unpack(__ldg(hi + v), ax);
                    unpack(__ldg(hj + v), bx);
#pragma unroll
                    for (int j = 0; j < N; ++j) c[q][j] = fma(T(0.5), ax[j] - bx[j], fx[j]);
                }
            } else {
#pragma unroll
                for (int j = 0; j < N; ++j) c[q][j] = T(0);
            }
        }
        T psi;
        if (!psi_only) {
            // the lane-group search with block-wide sums, counts and minima
            const T w0 = a.theta_in[a.m + e];
            const int den = a.ck ? 0 : 2;
            T S, mn, theta = T(0);
            int n, nA = 0;
            bool done = false;
            block_above<T, V, N>(c, w0, S, n, mn, sa_buf, sb_buf, sm_buf);
            if (w0 <= T(0)) start_root(S, n, mn, ue, den, theta, nA, done);
            else if (n > 0 && S - T(n) * w0 - ue - T(den) * w0 >= T(0)) {
                theta = (S - ue) / T(den + n);
                nA = n;
                done = mn > theta;
            } else {
                block_above<T, V, N>(c, T(0), S, n, mn, sa_buf, sb_buf, sm_buf);
                start_root(S, n, mn, ue, den, theta, nA, done);
            }
            for (int it = 0; !done && it <= a.Kp + 2; ++it) {  // block-uniform
                block_above<T, V, N>(c, theta, S, n, mn, sa_buf, sb_buf, sm_buf);
                if (n >= nA || n == 0) break;
                nA = n;
                theta = (S - ue) / T(den + n);
                done = mn > theta;
            }
            if (theta < T(0)) theta = T(0);  // a root below 0 is rounding at s = u: Case 1 (as qp_root_group)
            if (threadIdx.x == 0) {
                a.theta[a.m + e] = next_warm_start(theta, a.theta_in[e]);
                a.theta[e] = theta;
            }
            if (pf) {  // its height rows, now that its endpoints have arrived
                prefetch_l2(a.h + (int64_t)ps * a.Kp, (int64_t)a.Kp * sizeof(T), threadIdx.x, B);
                prefetch_l2(a.h + (int64_t)pc * a.Kp, (int64_t)a.Kp * sizeof(T), threadIdx.x, B);
            }
#pragma unroll
            for (int q = 0; q < V; ++q) {
                const int v = threadIdx.x + q * B;
                T o[N];
#pragma unroll
                for (int j = 0; j < N; ++j) {
                    const T x = c[q][j] - theta;
                    o[j] = x > T(0) ? x : T(0);
                }
                if (v < vpr) {
                    if (hint) st_hint(reinterpret_cast<VT*>(orow) + v, pack4(o), pol_first);
                    else reinterpret_cast<VT*>(orow)[v] = pack4(o);
                }
            }
            psi = T(den) * theta;  // sum f' - u at the root
        } else {
            T rs = T(0);
            int dummy = 0;
#pragma unroll
            for (int q = 0; q < V; ++q)
#pragma unroll
                for (int j = 0; j < N; ++j) rs += c[q][j];
            block_sum2(rs, dummy, sa_buf, sb_buf);
            psi = rs - ue > T(0) ? rs - ue : T(0);
        }
        if (threadIdx.x == 0) {
            zpsi = A::add(zpsi, psi * psi);
            const T c = psi * a.inv_scale_t[e];
            capmax = c > capmax ? c : capmax;
            if (a.psi_out) a.psi_out[e] = psi;
        }
    }
    // one partial per block, held by thread 0
    if (threadIdx.x == 0) {
        reinterpret_cast<typename A::S*>(a.part_psi)[blockIdx.x] = A::store(zpsi);
        a.part_cap[blockIdx.x] = capmax;
    }
}

// ------------------------------------------------------------------ persistent sweep kernel
//
// For instances whose two sweep kernels last only a few microseconds each,
// the fixed cost of a kernel boundary (launch, ramp-up, drain) is a large
// share of the sweep.  This kernel keeps one cooperative grid resident for
// many sweeps: the excess pass over all blocks, a grid barrier, the edge QPs
// over all blocks but the last, which reduces the objective and takes the stop
// decision meanwhile (as the decision block of the standalone edge kernel),
// and a second barrier after which every block reads the same stop flag.

__device__ __forceinline__ unsigned int ld_acquire_u32(const unsigned int* p)
{
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_u32(unsigned int* p, unsigned int v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Nanoseconds of the GPU's global timer (the same clock in every SM).
__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Sense-by-generation barrier over the whole (co-resident) grid.  A wait
// gives up after limit_ns nanoseconds of the global timer (elapsed time, not
// a poll count) and raises bar->failed, which ends every other block's wait
// too.  Returns false in every thread of a block whose wait timed out or saw
// another block's timeout.  withhold (test hook, uniform per block): the
// block leaves without arriving, so the others' waits run out.
__device__ __forceinline__ bool grid_sync(GridBarrier* bar, long long limit_ns, bool withhold)
{
    __shared__ int ok;
    if (withhold) return false;
    __syncthreads();
    if (threadIdx.x == 0) {
        // the generation is read before arriving, so the last arrival's
        // increment is always seen as a change
        const unsigned int gen = ld_acquire_u32(&bar->gen);
        __threadfence();
        const unsigned int arrived = atomicAdd(&bar->count, 1u) + 1u;
        int good = 1;
        if (arrived == gridDim.x) {
            atomicExch(&bar->count, 0u);
            __threadfence();
            st_release_u32(&bar->gen, gen + 1u);
        } else {
            const unsigned long long t0 = global_ns();
            while (ld_acquire_u32(&bar->gen) == gen) {
                if (ld_acquire_u32(&bar->failed) != 0u || (long long)(global_ns() - t0) > limit_ns) {
                    atomicExch(&bar->failed, 1u);
                    good = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        ok = good;
    }
    __syncthreads();
    return ok != 0;
}

template <typename T, int G, int V>
__global__ void __launch_bounds__(kThreads, (V <= 4 ? 4 : 3))
    persistent_kernel(SweepArgs<T> a, int64_t sweeps, GridBarrier* bar, int psi_prologue)
{
    volatile DevState* vst = a.st;
    const int nb = gridDim.x - 1;  // edge blocks; block nb decides
    const bool hold = a.hold_barrier != 0 && blockIdx.x == 0;  // test hook: block 0 never arrives
    // congestion partials of the current flows in this grid's layout (a
    // later launch of the same solve finds them written by its predecessor)
    if (psi_prologue) {
        SweepArgs<T> b = a;
        b.mode = MODE_PSI;
        if ((int)blockIdx.x < nb) edge_group_body<T, G, V, true>(b, blockIdx.x, nb);
        if (!grid_sync(bar, a.barrier_ns, hold)) return;
    }
    for (int64_t q = 0; q < sweeps; ++q) {
        if (vst->stop) break;  // the same value in every block (read after a barrier)
        SweepArgs<T> b = a;
        if (q & 1) {
            b.f = a.f_out;
            b.f_out = a.f;
            b.theta_in = a.theta;
            b.theta = const_cast<T*>(a.theta_in);
        }
        excess_body<T>(b, blockIdx.x, gridDim.x);
        if (!grid_sync(bar, a.barrier_ns, hold)) return;
        if ((int)blockIdx.x == nb) reduce_and_finalize(b);
        else edge_group_body<T, G, V, true>(b, blockIdx.x, nb);
        if (!grid_sync(bar, a.barrier_ns, hold)) return;
    }
}

// ------------------------------------------------------------------ edge QP, staged block form
//
// Persistent form of edge_block_kernel for long rows: one block per SM walks
// a stride of edges and keeps the next edge's three rows (f, h_i, h_j) in
// flight as cp.async.bulk copies into shared memory while it solves the
// current edge from registers.  Thread 0 issues the next edge's copies as
// soon as every thread has moved the current rows into registers, so each
// SM always has one edge's rows on the way from memory, through the root
// search and the stores of the current edge, with no L2 prefetch
// guesswork.  The flow rows stream with an L2 evict-first hint.  Per element
// the arithmetic and its order are edge_block_kernel's, so the flows are
// bit-identical to it.  Each wait on the copies is limited (a.wait_cycles);
// one that runs out records the fault, ends the solve, waits (limited) for
// the copy in flight and leaves.
template <typename T, int B, int V>
__global__ void __launch_bounds__(B, 1) edge_staged_kernel(SweepArgs<T> a)
{
    pdl_wait();  // the excess kernel has finished (no-op without PDL)
    using VT = typename VecOf<T>::type;
    constexpr int N = VecOf<T>::N;
    using A = Acc<T>;
    extern __shared__ __align__(128) unsigned char esm[];
    __shared__ __align__(8) uint64_t full;
    __shared__ T sa_buf[33];
    __shared__ int sb_buf[33];
    __shared__ T sm_buf[33];
    volatile DevState* vst = a.st;
    if (sweep_stopped(a)) return;  // an earlier sweep of this solve stopped
    if (blockIdx.x == gridDim.x - 1) {  // the decision block
        if (a.mode != MODE_PSI) reduce_and_finalize(a);
        return;
    }
    if (final_evaluation(a)) return;  // the sweep cap stops this sweep: its output is not used
    const int nb = gridDim.x - 1;
    const int vpr = a.Kp / N;
    const uint32_t row_bytes = (uint32_t)a.Kp * (uint32_t)sizeof(T);
    const bool psi_only = (a.mode == MODE_PSI);
    const VT* sf = reinterpret_cast<const VT*>(esm);
    const VT* shi = sf + vpr;
    const VT* shj = shi + vpr;
    const uint64_t pol_first = l2_evict_first();
    auto stage = [&](int64_t e) {  // thread 0: the rows of edge e into shared memory
        mbar_arrive_expect_tx(&full, psi_only ? row_bytes : 3u * row_bytes);
        bulk_g2s_hint(esm, a.f + e * a.Kp, row_bytes, &full, pol_first);
        if (!psi_only) {
            bulk_g2s(esm + row_bytes, a.h + (int64_t)a.src[e] * a.Kp, row_bytes, &full);
            bulk_g2s(esm + 2 * (size_t)row_bytes, a.h + (int64_t)a.col[e] * a.Kp, row_bytes, &full);
        }
    };
    if (threadIdx.x == 0) {
        mbar_init(&full, 1);
        mbar_init_fence();
        if ((int64_t)blockIdx.x < a.m) stage(blockIdx.x);
    }
    __syncthreads();
    typename A::V zpsi = A::zero();
    T capmax = T(0);
    uint32_t phase = 0;
    for (int64_t e = blockIdx.x; e < a.m; e += nb) {
        const bool landed = mbar_wait(&full, phase, a.wait_cycles);
        if (__syncthreads_or(!landed)) {
            if (threadIdx.x == 0) {
                a.st->fault = 1;
                stop_from_kernel(a);
            }
            mbar_wait(&full, phase, a.wait_cycles);  // the copy in flight, then leave
            return;
        }
        phase ^= 1u;
        const T ue = a.u[e];
        T c[V][N];
#pragma unroll
        for (int q = 0; q < V; ++q) {
            const int v = threadIdx.x + q * B;
            if (v < vpr) {
                T fx[N];
                unpack(sf[v], fx);
                if (psi_only) {
#pragma unroll
                    for (int j = 0; j < N; ++j) c[q][j] = fx[j];
                } else {
                    T ax[N], bx[N];
                    unpack(shi[v], ax);
                    unpack(shj[v], bx);
#pragma unroll
                    for (int j = 0; j < N; ++j) c[q][j] = fma(T(0.5), ax[j] - bx[j], fx[j]);
                }
            } else {
#pragma unroll
                for (int j = 0; j < N; ++j) c[q][j] = T(0);
            }
        }
        __syncthreads();  // every row is in registers: the staging buffer is free
        if (threadIdx.x == 0 && e + nb < a.m) stage(e + nb);
        T* orow = a.f_out + e * a.Kp;
        T psi;
        if (!psi_only) {
            const T w0 = a.theta_in[a.m + e];
            const int den = a.ck ? 0 : 2;
            T S, mn, theta = T(0);
            int n, nA = 0;
            bool done = false;
            block_above<T, V, N>(c, w0, S, n, mn, sa_buf, sb_buf, sm_buf);
            if (w0 <= T(0)) start_root(S, n, mn, ue, den, theta, nA, done);
            else if (n > 0 && S - T(n) * w0 - ue - T(den) * w0 >= T(0)) {
                theta = (S - ue) / T(den + n);
                nA = n;
                done = mn > theta;
            } else {
                block_above<T, V, N>(c, T(0), S, n, mn, sa_buf, sb_buf, sm_buf);
                start_root(S, n, mn, ue, den, theta, nA, done);
            }
            for (int it = 0; !done && it <= a.Kp + 2; ++it) {  // block-uniform
                block_above<T, V, N>(c, theta, S, n, mn, sa_buf, sb_buf, sm_buf);
                if (n >= nA || n == 0) break;
                nA = n;
                theta = (S - ue) / T(den + n);
                done = mn > theta;
            }
            if (theta < T(0)) theta = T(0);  // a root below 0 is rounding at s = u: Case 1
            if (threadIdx.x == 0) {
                a.theta[a.m + e] = next_warm_start(theta, a.theta_in[e]);
                a.theta[e] = theta;
            }
#pragma unroll
            for (int q = 0; q < V; ++q) {
                const int v = threadIdx.x + q * B;
                T o[N];
#pragma unroll
                for (int j = 0; j < N; ++j) {
                    const T x = c[q][j] - theta;
                    o[j] = x > T(0) ? x : T(0);
                }
                if (v < vpr) st_hint(reinterpret_cast<VT*>(orow) + v, pack4(o), pol_first);
            }
            psi = T(den) * theta;  // sum f' - u at the root
        } else {
            T rs = T(0);
            int dummy = 0;
#pragma unroll
            for (int q = 0; q < V; ++q)
#pragma unroll
                for (int j = 0; j < N; ++j) rs += c[q][j];
            block_sum2(rs, dummy, sa_buf, sb_buf);
            psi = rs - ue > T(0) ? rs - ue : T(0);
        }
        if (threadIdx.x == 0) {
            zpsi = A::add(zpsi, psi * psi);
            const T cp = psi * a.inv_scale_t[e];
            capmax = cp > capmax ? cp : capmax;
            if (a.psi_out) a.psi_out[e] = psi;
        }
    }
    // one partial per block, held by thread 0
    if (threadIdx.x == 0) {
        reinterpret_cast<typename A::S*>(a.part_psi)[blockIdx.x] = A::store(zpsi);
        a.part_cap[blockIdx.x] = capmax;
    }
}

// ------------------------------------------------------------------ batched form: one cluster per instance
//
// For a batch of small instances one launch runs every instance's solve: the
// csize consecutive blocks of a thread-block cluster own instance
// ids[blockIdx.x / csize] and run Alg. 1 sweep after sweep -- the excess
// pass, the objective and stop test, then (unless it stopped) the edge QPs --
// separated only by cluster barriers (block barriers for csize = 1), until
// its own stop rule fires or `sweeps` sweeps are done.  A finished instance's
// blocks leave and free their SM slots, which is the per-instance
// convergence mask.  Per element the arithmetic and its order are those of
// the standalone kernels with the same lane-group variant, so the flows equal
// theirs bit for bit; the objective's partials are grouped per block (z
// agrees to rounding).  The flows start in the buffer args[i] names and every
// applied sweep swaps the buffers.

// All threads of the cluster; release/acquire at cluster scope orders the
// global-memory writes of one phase before the reads of the next.
__device__ __forceinline__ void cluster_sync_all()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// Shared-memory form (SM, one block per instance): the block copies the
// instance's mutable arrays -- both flow buffers, the heights, both root
// buffers, the objective partials -- and its solver state into shared
// memory, with the read-only arrays the sweep reads (incidence lists,
// commodities, capacities, endpoints, scales), runs its sweeps there, and
// copies the mutable ones back before it returns.  The phases then pass
// their data through shared memory instead of L2, whose latency is what a
// sweep of a small instance waits on.  The arithmetic and the order of
// every reduction are unchanged, so flows, roots, z and the stop sweep
// equal the global-memory form's bit for bit.  Layout (each part 16-byte
// aligned): f buffer 0 and 1 [m][Kp], h [n][Kp], roots 0 and 1 [2m], psi
// partials [n_psi] (stored pairs) and [n_psi], excess partials (one each),
// then inc_ptr [n+1], inc [2m], s, t, dem, 1/d [Kp], u, src, col,
// 1/scale [m], 1/delta [n].
template <typename T>
struct BlockSmem {
    int64_t f0, f1, h, th0, th1, ppsi, pcap, ph, pcons, pcapb;
    int64_t incp, inc, s, t, dem, idem, u, src, col, isc, ideg, bytes;
};

template <typename T>
__host__ __device__ inline BlockSmem<T> block_smem_layout(int64_t n, int64_t m, int64_t Kp, int64_t n_psi)
{
    auto up = [](int64_t x) { return (x + 15) & ~int64_t(15); };
    BlockSmem<T> L{};
    int64_t o = 0;
    L.f0 = o;    o = up(o + m * Kp * (int64_t)sizeof(T));
    L.f1 = o;    o = up(o + m * Kp * (int64_t)sizeof(T));
    L.h = o;     o = up(o + n * Kp * (int64_t)sizeof(T));
    L.th0 = o;   o = up(o + 2 * m * (int64_t)sizeof(T));
    L.th1 = o;   o = up(o + 2 * m * (int64_t)sizeof(T));
    L.ppsi = o;  o = up(o + n_psi * (int64_t)sizeof(typename Acc<T>::S));
    L.pcap = o;  o = up(o + n_psi * (int64_t)sizeof(T));
    L.ph = o;    o = up(o + (int64_t)sizeof(double));
    L.pcons = o; o = up(o + (int64_t)sizeof(T));
    L.pcapb = o; o = up(o + (int64_t)sizeof(T));
    L.incp = o;  o = up(o + (n + 1) * (int64_t)sizeof(int64_t));
    L.inc = o;   o = up(o + 2 * m * (int64_t)sizeof(int32_t));
    L.s = o;     o = up(o + Kp * (int64_t)sizeof(int32_t));
    L.t = o;     o = up(o + Kp * (int64_t)sizeof(int32_t));
    L.dem = o;   o = up(o + Kp * (int64_t)sizeof(T));
    L.idem = o;  o = up(o + Kp * (int64_t)sizeof(T));
    L.u = o;     o = up(o + m * (int64_t)sizeof(T));
    L.src = o;   o = up(o + m * (int64_t)sizeof(int32_t));
    L.col = o;   o = up(o + m * (int64_t)sizeof(int32_t));
    L.isc = o;   o = up(o + m * (int64_t)sizeof(T));
    L.ideg = o;  o = up(o + n * (int64_t)sizeof(T));
    L.bytes = o;
    return L;
}

// count elements of X from src to dst by the whole block
template <typename X>
__device__ __forceinline__ void block_copy(X* __restrict__ dst, const X* __restrict__ src, int64_t count)
{
    for (int64_t q = threadIdx.x; q < count; q += blockDim.x) dst[q] = src[q];
}

template <typename T, int G, int V, bool SM>
__global__ void __launch_bounds__(kBatchThreads, 2)
    batch_block_kernel(const SweepArgs<T>* __restrict__ args, const int* __restrict__ ids, int csize,
                       int64_t sweeps, int psi_prologue)
{
    using VT = typename VecOf<T>::type;
    using S = typename Acc<T>::S;
    // the instance's arguments live in shared memory (not in every thread's
    // registers); thread 0 of every block swaps its buffers between sweeps
    __shared__ SweepArgs<T> sa;
    __shared__ int stop;
    __shared__ DevState sst;  // SM: the solver state while the block runs
    extern __shared__ __align__(16) unsigned char smem[];
    const int rank = (int)(blockIdx.x % (unsigned)csize);
    auto sync = [csize]() {
        if (csize > 1) cluster_sync_all();
        else __syncthreads();
    };
    if (threadIdx.x == 0) {
        sa = args[ids[blockIdx.x / (unsigned)csize]];
        stop = reinterpret_cast<volatile DevState*>(sa.st)->stop;
        if (psi_prologue) sa.mode = MODE_PSI;
    }
    __syncthreads();
    if (stop) return;  // the same value in every block of the cluster (no block of it has run yet)
    // SM: the global buffers, to which the shared copies return at the end
    T* const gf0 = sa.f;
    T* const gf1 = sa.f_out;
    T* const gh = sa.h;
    T* const gth0 = const_cast<T*>(sa.theta_in);
    T* const gth1 = sa.theta;
    S* const gpsi = reinterpret_cast<S*>(sa.part_psi);
    T* const gcap = sa.part_cap;
    DevState* const gst = sa.st;
    const BlockSmem<T> L = block_smem_layout<T>(sa.n, sa.m, sa.Kp, sa.n_psi);
    if constexpr (SM) {
        const int64_t rowv = sa.m * sa.Kp / VecOf<T>::N;
        block_copy(reinterpret_cast<VT*>(smem + L.f0), reinterpret_cast<const VT*>(gf0), rowv);
        block_copy(reinterpret_cast<VT*>(smem + L.f1), reinterpret_cast<const VT*>(gf1), rowv);
        block_copy(reinterpret_cast<VT*>(smem + L.h), reinterpret_cast<const VT*>(gh),
                   (int64_t)sa.n * sa.Kp / VecOf<T>::N);
        block_copy(reinterpret_cast<T*>(smem + L.th0), gth0, 2 * sa.m);
        block_copy(reinterpret_cast<T*>(smem + L.th1), gth1, 2 * sa.m);
        block_copy(reinterpret_cast<S*>(smem + L.ppsi), gpsi, sa.n_psi);
        block_copy(reinterpret_cast<T*>(smem + L.pcap), gcap, sa.n_psi);
        block_copy(reinterpret_cast<int64_t*>(smem + L.incp), sa.inc_ptr, (int64_t)sa.n + 1);
        block_copy(reinterpret_cast<int32_t*>(smem + L.inc), sa.inc, 2 * sa.m);
        block_copy(reinterpret_cast<int32_t*>(smem + L.s), sa.s, (int64_t)sa.Kp);
        block_copy(reinterpret_cast<int32_t*>(smem + L.t), sa.t, (int64_t)sa.Kp);
        block_copy(reinterpret_cast<T*>(smem + L.dem), sa.dem, (int64_t)sa.Kp);
        block_copy(reinterpret_cast<T*>(smem + L.idem), sa.inv_dem, (int64_t)sa.Kp);
        block_copy(reinterpret_cast<T*>(smem + L.u), sa.u, sa.m);
        block_copy(reinterpret_cast<int32_t*>(smem + L.src), sa.src, sa.m);
        block_copy(reinterpret_cast<int32_t*>(smem + L.col), sa.col, sa.m);
        block_copy(reinterpret_cast<T*>(smem + L.isc), sa.inv_scale_t, sa.m);
        block_copy(reinterpret_cast<T*>(smem + L.ideg), sa.inv_deg, (int64_t)sa.n);
        __syncthreads();  // every thread has read sa's global pointers
        if (threadIdx.x == 0) {
            sst = *gst;
            sa.f = reinterpret_cast<T*>(smem + L.f0);
            sa.f_out = reinterpret_cast<T*>(smem + L.f1);
            sa.h = reinterpret_cast<T*>(smem + L.h);
            sa.theta_in = reinterpret_cast<const T*>(smem + L.th0);
            sa.theta = reinterpret_cast<T*>(smem + L.th1);
            sa.part_psi = smem + L.ppsi;
            sa.part_cap = reinterpret_cast<T*>(smem + L.pcap);
            sa.part_h = reinterpret_cast<double*>(smem + L.ph);
            sa.part_cons = reinterpret_cast<T*>(smem + L.pcons);
            sa.part_capb = reinterpret_cast<T*>(smem + L.pcapb);
            sa.inc_ptr = reinterpret_cast<const int64_t*>(smem + L.incp);
            sa.inc = reinterpret_cast<const int32_t*>(smem + L.inc);
            sa.s = reinterpret_cast<const int32_t*>(smem + L.s);
            sa.t = reinterpret_cast<const int32_t*>(smem + L.t);
            sa.dem = reinterpret_cast<const T*>(smem + L.dem);
            sa.inv_dem = reinterpret_cast<const T*>(smem + L.idem);
            sa.u = reinterpret_cast<const T*>(smem + L.u);
            sa.src = reinterpret_cast<const int32_t*>(smem + L.src);
            sa.col = reinterpret_cast<const int32_t*>(smem + L.col);
            sa.inv_scale_t = reinterpret_cast<const T*>(smem + L.isc);
            sa.inv_deg = reinterpret_cast<const T*>(smem + L.ideg);
            sa.st = &sst;
        }
        __syncthreads();
    }
    if (psi_prologue) {  // congestion partials of the starting flows, in this kernel's layout
        edge_group_body<T, G, V, true>(sa, rank, csize);
        sync();
        if (threadIdx.x == 0) sa.mode = MODE_SOLVE;
        __syncthreads();
    }
    for (int64_t q = 0; q < sweeps; ++q) {
        excess_body<T, SM>(sa, rank, csize);
        sync();
        if (rank == 0) reduce_and_finalize<T, SM>(sa);
        sync();
        if (threadIdx.x == 0) stop = reinterpret_cast<volatile DevState*>(sa.st)->stop;
        __syncthreads();
        if (stop) break;  // f^(t) stays in sa.f
        edge_group_body<T, G, V, true>(sa, rank, csize);
        sync();
        if (threadIdx.x == 0) {  // f^(t+1) becomes the current flows
            T* f = sa.f;
            sa.f = sa.f_out;
            sa.f_out = f;
            const T* th = sa.theta_in;
            sa.theta_in = sa.theta;
            sa.theta = const_cast<T*>(th);
        }
        __syncthreads();
    }
    if constexpr (SM) {  // every buffer back to its global counterpart
        const int64_t rowv = sa.m * sa.Kp / VecOf<T>::N;
        block_copy(reinterpret_cast<VT*>(gf0), reinterpret_cast<const VT*>(smem + L.f0), rowv);
        block_copy(reinterpret_cast<VT*>(gf1), reinterpret_cast<const VT*>(smem + L.f1), rowv);
        block_copy(reinterpret_cast<VT*>(gh), reinterpret_cast<const VT*>(smem + L.h),
                   (int64_t)sa.n * sa.Kp / VecOf<T>::N);
        block_copy(gth0, reinterpret_cast<const T*>(smem + L.th0), 2 * sa.m);
        block_copy(gth1, reinterpret_cast<const T*>(smem + L.th1), 2 * sa.m);
        block_copy(gpsi, reinterpret_cast<const S*>(smem + L.ppsi), sa.n_psi);
        block_copy(gcap, reinterpret_cast<const T*>(smem + L.pcap), sa.n_psi);
        if (threadIdx.x == 0) *gst = sst;
    }
}

template <typename T, int G, int V>
cudaError_t persistent_occupancy(int* blocks)
{
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, persistent_kernel<T, G, V>, kThreads, 0);
}

// dst[r*K + k] = src[r*Kp + k] as double: the padded rows of a flow array
// packed and widened into a caller's buffer that the GPU can write.
template <typename T>
__global__ void widen_rows_kernel(const T* __restrict__ src, int64_t rows, int K, int Kp, double* __restrict__ dst)
{
    const int64_t total = rows * (int64_t)K;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = q / K;
        dst[q] = (double)src[r * Kp + (q - r * K)];
    }
}

__global__ void convert_kernel(const float* __restrict__ a, double* __restrict__ b, int64_t count)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
        b[i] = (double)a[i];
}

// Variant table: capacity (elements per row) of each configuration.
struct EdgeCfg {
    int G;        // lanes per edge (0 = block form)
    int B;        // block size of the block form
    int V;        // vectors per lane
    int P;        // 1 = pipelined persistent warp form (Alg. 2 only)
};
constexpr EdgeCfg kCfg[] = {
    // 0..15 ordered by capacity (elements per row); of equal capacities the
    // first is the default (measured fastest for Alg. 2: 128 x 4 on
    // digraph20k_k2000, 512 x 5 on grid100_k10000); the block forms keep
    // 2-12 edges in flight per SM (block_min_blocks)
    {4, 0, 1, 0},   {8, 0, 1, 0},   {16, 0, 1, 0},  {32, 0, 1, 0},   {32, 0, 2, 0},
    {32, 0, 4, 0},  {32, 0, 8, 0},  {0, 128, 4, 0}, {0, 256, 2, 0},  {0, 512, 2, 0},
    {0, 512, 3, 0}, {0, 512, 4, 0}, {0, 512, 5, 0}, {0, 256, 10, 0}, {0, 512, 8, 0},
    {0, 1024, 8, 0},
    // 16..18: the pipelined forms of 3..5 (the gradient kernels of Alg. 3/4
    // run the plain form of the same capacity); at 8 vectors per lane the
    // prefetched rows no longer fit in registers
    {32, 0, 1, 1},  {32, 0, 2, 1},  {32, 0, 4, 1},
    // 19..20: the staged forms of 12 and 14 (bulk copies of the next edge's
    // rows into shared memory: 3 rows of up to 40 / 64 KB)
    {0, 512, 5, 2}, {0, 512, 8, 2},
};
constexpr int kFirstPipelined = 16;
constexpr int kFirstStaged = 19;
constexpr int kNumCfg = sizeof(kCfg) / sizeof(kCfg[0]);

template <typename T>
int capacity(int cfg)
{
    const EdgeCfg& c = kCfg[cfg];
    return (c.G ? c.G : c.B) * c.V * VecOf<T>::N;
}

}  // namespace

template <typename T>
int edge_config(int Kp)
{
    for (int i = 0; i < kNumCfg; ++i)
        if (!kCfg[i].P && capacity<T>(i) >= Kp) return i;
    return -1;
}

template <typename T, int V>
int pipe_resident()
{
    int blocks = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, edge_pipe_kernel<T, V>, kThreads, 0) != cudaSuccess ||
        blocks < 1) {
        cudaGetLastError();
        return 2;
    }
    return blocks;
}

template <typename T>
size_t staged_smem(int Kp)
{
    return 3 * (size_t)Kp * sizeof(T);
}

// The staged forms take their three rows in dynamic shared memory (above the
// 48 KB default): allowed once, at create time, for the largest rows.
template <typename T>
void staged_setup(int cfg)
{
    const int cap = capacity<T>(cfg);
    const int bytes = (int)staged_smem<T>(cap);
    if (cfg == kFirstStaged)
        cudaFuncSetAttribute(edge_staged_kernel<T, 512, 5>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    else
        cudaFuncSetAttribute(edge_staged_kernel<T, 512, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    cudaGetLastError();
}

template <typename T>
int edge_grid(int cfg, int64_t m, int num_sms)
{
    const EdgeCfg& c = kCfg[cfg];
    int64_t want, cap;
    if (c.P == 2) {
        // one block per SM, each walking a stride of edges
        staged_setup<T>(cfg);
        const int64_t g = m < num_sms ? m : num_sms;
        return (int)(g < 1 ? 1 : g);
    }
    if (c.P) {
        // one wave of resident warps, each walking a stride of edges
        const int per_sm = c.V == 1 ? pipe_resident<T, 1>() : c.V == 2 ? pipe_resident<T, 2>() : pipe_resident<T, 4>();
        const int64_t per_block = kThreads / 32;
        want = (m + per_block - 1) / per_block;
        cap = (int64_t)num_sms * per_sm;
        const int64_t g = want < cap ? want : cap;
        return (int)(g < 1 ? 1 : g);
    }
    if (c.G) {
        const int64_t per_block = kThreads / c.G;
        want = (m + per_block - 1) / per_block;
    } else {
        want = m;
    }
    cap = 1 << 20;  // beyond this the kernels loop over edges
    int64_t g = want < cap ? want : cap;
    return (int)(g < 1 ? 1 : g);
}

template <typename T>
int edge_capacity(int cfg)
{
    return (cfg >= 0 && cfg < kNumCfg) ? capacity<T>(cfg) : -1;
}

int num_edge_configs() { return kNumCfg; }

template <typename T>
int64_t edge_parts(int cfg, int grid)
{
    return kCfg[cfg].G ? (int64_t)grid * (kThreads / 32) : (int64_t)grid;
}

// One wave of resident blocks (or fewer if the rows are fewer): the grid-
// stride loop then spreads the rows evenly and leaves no partial last wave.
int excess_grid(int32_t n, int Kp, int vec, int num_sms, int resident_blocks)
{
    const int64_t total = (int64_t)n * (Kp / vec);
    int64_t want = (total + kThreads - 1) / kThreads;
    const int64_t cap = (int64_t)num_sms * (resident_blocks > 0 ? resident_blocks : 4);
    int64_t g = want < cap ? want : cap;
    return (int)(g < 1 ? 1 : g);
}

template <typename T>
int excess_resident_blocks()
{
    int blocks = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, excess_kernel<T>, kThreads, 0) != cudaSuccess) {
        cudaGetLastError();
        return 4;
    }
    return blocks;
}
template int excess_resident_blocks<float>();
template int excess_resident_blocks<double>();

// A launch with or without programmatic dependent launch (PDL): with it,
// the kernel may be scheduled while the previous kernel on the stream (or
// in the graph) is still running; its griddepcontrol.wait then holds it
// until that kernel has finished and its writes are visible.
template <typename T>
cudaError_t launch_one(void (*kernel)(SweepArgs<T>), int grid, int block, cudaStream_t stream, bool pdl,
                       const SweepArgs<T>& a, size_t smem = 0)
{
    if (!pdl) {
        kernel<<<grid, block, smem, stream>>>(a);
        return cudaGetLastError();
    }
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr{};
    attr.id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr.val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, a);
}

template <typename T, int S, int R, int C>
cudaError_t launch_bulk(const SweepArgs<T>& a, cudaStream_t stream, bool pdl)
{
    return launch_one<T>(excess_bulk_kernel<T, S, R, C>, a.grid_v, C + 32, stream, pdl, a, excess_bulk_smem<S, R, C>());
}

// Excess forms: 0 the per-thread gathers; bulk copies 1: 4 x 8 segments of
// 2 KB, 2: 2 x 8 of 2 KB, 3: 4 x 4 of 2 KB, 4: 2 x 8 of 512 B, 5: 4 x 8 of 512 B.
template <typename T>
cudaError_t launch_excess(const SweepArgs<T>& a, cudaStream_t stream, bool pdl)
{
    switch (a.excess_form) {
    case 1: return launch_bulk<T, 4, 8, 128>(a, stream, pdl);
    case 2: return launch_bulk<T, 2, 8, 128>(a, stream, pdl);
    case 3: return launch_bulk<T, 4, 4, 128>(a, stream, pdl);
    case 4: return launch_bulk<T, 2, 8, 32>(a, stream, pdl);
    case 5: return launch_bulk<T, 4, 8, 32>(a, stream, pdl);
    default: return launch_one<T>(excess_kernel<T>, a.grid_v, kThreads, stream, pdl, a);
    }
}

template <typename T, int S, int R, int C>
int bulk_resident()
{
    const size_t smem = excess_bulk_smem<S, R, C>();
    int blocks = 0;
    if (cudaFuncSetAttribute(excess_bulk_kernel<T, S, R, C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, excess_bulk_kernel<T, S, R, C>, C + 32, smem) !=
            cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return blocks;
}

template <typename T>
int excess_bulk_resident_blocks(int form)
{
    switch (form) {
    case 1: return bulk_resident<T, 4, 8, 128>();
    case 2: return bulk_resident<T, 2, 8, 128>();
    case 3: return bulk_resident<T, 4, 4, 128>();
    case 4: return bulk_resident<T, 2, 8, 32>();
    case 5: return bulk_resident<T, 4, 8, 32>();
    default: return 0;
    }
}
template int excess_bulk_resident_blocks<float>(int);
template int excess_bulk_resident_blocks<double>(int);

cudaError_t launch_excess_split(const int64_t* inc_ptr, int32_t n, int grid, int32_t* xv_start, cudaStream_t stream)
{
    excess_split_kernel<<<(grid + 1 + 255) / 256, 256, 0, stream>>>(inc_ptr, n, grid, xv_start);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_finalize(const SweepArgs<T>& a, cudaStream_t stream)
{
    finalize_kernel<T><<<1, kThreads, 0, stream>>>(a);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_edge(const SweepArgs<T>& a, int cfg, cudaStream_t stream, bool pdl)
{
    const int g = a.grid_e + 1;  // edge blocks plus the decision block
    switch (cfg) {
    case 0: return launch_one<T>(edge_group_kernel<T, 4, 1>, g, kThreads, stream, pdl, a);
    case 1: return launch_one<T>(edge_group_kernel<T, 8, 1>, g, kThreads, stream, pdl, a);
    case 2: return launch_one<T>(edge_group_kernel<T, 16, 1>, g, kThreads, stream, pdl, a);
    case 3: return launch_one<T>(edge_group_kernel<T, 32, 1>, g, kThreads, stream, pdl, a);
    case 4: return launch_one<T>(edge_group_kernel<T, 32, 2>, g, kThreads, stream, pdl, a);
    case 5: return launch_one<T>(edge_group_kernel<T, 32, 4>, g, kThreads, stream, pdl, a);
    case 6: return launch_one<T>(edge_group_kernel<T, 32, 8>, g, kThreads, stream, pdl, a);
    case 7: return launch_one<T>(edge_block_kernel<T, 128, 4>, g, 128, stream, pdl, a);
    case 8: return launch_one<T>(edge_block_kernel<T, 256, 2>, g, 256, stream, pdl, a);
    case 9: return launch_one<T>(edge_block_kernel<T, 512, 2>, g, 512, stream, pdl, a);
    case 10: return launch_one<T>(edge_block_kernel<T, 512, 3>, g, 512, stream, pdl, a);
    case 11: return launch_one<T>(edge_block_kernel<T, 512, 4>, g, 512, stream, pdl, a);
    case 12: return launch_one<T>(edge_block_kernel<T, 512, 5>, g, 512, stream, pdl, a);
    case 13: return launch_one<T>(edge_block_kernel<T, 256, 10>, g, 256, stream, pdl, a);
    case 14: return launch_one<T>(edge_block_kernel<T, 512, 8>, g, 512, stream, pdl, a);
    case 15: return launch_one<T>(edge_block_kernel<T, 1024, 8>, g, 1024, stream, pdl, a);
    case 16: return launch_one<T>(edge_pipe_kernel<T, 1>, g, kThreads, stream, pdl, a);
    case 17: return launch_one<T>(edge_pipe_kernel<T, 2>, g, kThreads, stream, pdl, a);
    case 18: return launch_one<T>(edge_pipe_kernel<T, 4>, g, kThreads, stream, pdl, a);
    case 19: return launch_one<T>(edge_staged_kernel<T, 512, 5>, g, 512, stream, pdl, a, staged_smem<T>(a.Kp));
    case 20: return launch_one<T>(edge_staged_kernel<T, 512, 8>, g, 512, stream, pdl, a, staged_smem<T>(a.Kp));
    default: return cudaErrorInvalidValue;
    }
}

template <typename T>
int persistent_grid(int cfg, int64_t m, int32_t n, int Kp, int num_sms)
{
    cfg = edge_plain_config(cfg);
    if (cfg < 0 || cfg >= kNumCfg || !kCfg[cfg].G || m <= 0) return 0;
    int per_sm = 0;
    cudaError_t e;
    switch (cfg) {
    case 0: e = persistent_occupancy<T, 4, 1>(&per_sm); break;
    case 1: e = persistent_occupancy<T, 8, 1>(&per_sm); break;
    case 2: e = persistent_occupancy<T, 16, 1>(&per_sm); break;
    case 3: e = persistent_occupancy<T, 32, 1>(&per_sm); break;
    case 4: e = persistent_occupancy<T, 32, 2>(&per_sm); break;
    case 5: e = persistent_occupancy<T, 32, 4>(&per_sm); break;
    case 6: e = persistent_occupancy<T, 32, 8>(&per_sm); break;
    default: return 0;
    }
    if (e != cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        return 0;
    }
    // no more blocks than either pass has work for (each costs an arrival at
    // every barrier), at least one edge block and the decision block
    const int64_t groups_per_block = kThreads / kCfg[cfg].G;
    const int64_t want_e = (m + groups_per_block - 1) / groups_per_block + 1;
    const int64_t want_v = ((int64_t)n * (Kp / VecOf<T>::N) + kThreads - 1) / kThreads;
    int64_t g = want_e > want_v ? want_e : want_v;
    const int64_t cap = (int64_t)num_sms * per_sm;
    if (g > cap) g = cap;
    return g < 2 ? 2 : (int)g;
}

template <typename T, int G, int V>
cudaError_t launch_batch_block_gv(const SweepArgs<T>* args, const int* ids, int count, int csize, int64_t sweeps,
                                  int psi_prologue, cudaStream_t stream, int64_t smem)
{
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)(count * csize));
    cfg.blockDim = dim3(kBatchThreads);
    cfg.stream = stream;
    cudaLaunchAttribute attr{};
    attr.id = cudaLaunchAttributeClusterDimension;
    attr.val.clusterDim.x = (unsigned)csize;
    attr.val.clusterDim.y = 1;
    attr.val.clusterDim.z = 1;
    cfg.attrs = &attr;
    cfg.numAttrs = csize > 1 ? 1 : 0;
    if (smem > 0) {
        const cudaError_t e = cudaFuncSetAttribute(batch_block_kernel<T, G, V, true>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        cfg.dynamicSmemBytes = (size_t)smem;
        return cudaLaunchKernelEx(&cfg, batch_block_kernel<T, G, V, true>, args, ids, csize, sweeps, psi_prologue);
    }
    return cudaLaunchKernelEx(&cfg, batch_block_kernel<T, G, V, false>, args, ids, csize, sweeps, psi_prologue);
}

template <typename T>
cudaError_t launch_batch_block(int cfg, const SweepArgs<T>* args, const int* ids, int count, int csize, int64_t sweeps,
                               int psi_prologue, cudaStream_t stream, int64_t smem)
{
    if (count <= 0) return cudaSuccess;
    if (csize < 1 || csize > 8 || (csize & (csize - 1))) return cudaErrorInvalidValue;
    if (smem < 0 || smem > kBlockSmemMax || (smem > 0 && csize != 1)) return cudaErrorInvalidValue;
    switch (edge_plain_config(cfg)) {
    case 0: return launch_batch_block_gv<T, 4, 1>(args, ids, count, csize, sweeps, psi_prologue, stream, smem);
    case 1: return launch_batch_block_gv<T, 8, 1>(args, ids, count, csize, sweeps, psi_prologue, stream, smem);
    case 2: return launch_batch_block_gv<T, 16, 1>(args, ids, count, csize, sweeps, psi_prologue, stream, smem);
    case 3: return launch_batch_block_gv<T, 32, 1>(args, ids, count, csize, sweeps, psi_prologue, stream, smem);
    case 4: return launch_batch_block_gv<T, 32, 2>(args, ids, count, csize, sweeps, psi_prologue, stream, smem);
    case 5: return launch_batch_block_gv<T, 32, 4>(args, ids, count, csize, sweeps, psi_prologue, stream, smem);
    default: return cudaErrorInvalidValue;
    }
}
template cudaError_t launch_batch_block<float>(int, const SweepArgs<float>*, const int*, int, int, int64_t, int,
                                               cudaStream_t, int64_t);
template cudaError_t launch_batch_block<double>(int, const SweepArgs<double>*, const int*, int, int, int64_t, int,
                                                cudaStream_t, int64_t);

template <typename T>
int64_t block_smem_bytes(int64_t n, int64_t m, int64_t Kp, int64_t n_psi)
{
    return block_smem_layout<T>(n, m, Kp, n_psi).bytes;
}
template int64_t block_smem_bytes<float>(int64_t, int64_t, int64_t, int64_t);
template int64_t block_smem_bytes<double>(int64_t, int64_t, int64_t, int64_t);

bool batch_block_config(int cfg)
{
    const int c = edge_plain_config(cfg);
    return c >= 0 && c < kNumCfg && kCfg[c].G > 0;
}

template <typename T>
cudaError_t launch_widen_rows(const T* src, int64_t rows, int K, int Kp, double* dst, cudaStream_t stream)
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t want = (rows * (int64_t)K + 255) / 256;
    const int64_t cap = (int64_t)(sms > 0 ? sms : 1) * 8;
    const int grid = (int)(want < 1 ? 1 : (want < cap ? want : cap));
    widen_rows_kernel<T><<<grid, 256, 0, stream>>>(src, rows, K, Kp, dst);
    return cudaGetLastError();
}
template cudaError_t launch_widen_rows<float>(const float*, int64_t, int, int, double*, cudaStream_t);
template cudaError_t launch_widen_rows<double>(const double*, int64_t, int, int, double*, cudaStream_t);

template <typename T>
cudaError_t launch_persistent(const SweepArgs<T>& a, int cfg, int grid, int64_t sweeps, GridBarrier* bar,
                              int psi_prologue, cudaStream_t stream)
{
    SweepArgs<T> args = a;
    void* params[] = {&args, &sweeps, &bar, &psi_prologue};
    void* fn = nullptr;
    switch (edge_plain_config(cfg)) {
    case 0: fn = (void*)persistent_kernel<T, 4, 1>; break;
    case 1: fn = (void*)persistent_kernel<T, 8, 1>; break;
    case 2: fn = (void*)persistent_kernel<T, 16, 1>; break;
    case 3: fn = (void*)persistent_kernel<T, 32, 1>; break;
    case 4: fn = (void*)persistent_kernel<T, 32, 2>; break;
    case 5: fn = (void*)persistent_kernel<T, 32, 4>; break;
    case 6: fn = (void*)persistent_kernel<T, 32, 8>; break;
    default: return cudaErrorInvalidValue;
    }
    return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(kThreads), params, 0, stream);
}

template int persistent_grid<float>(int, int64_t, int32_t, int, int);
template int persistent_grid<double>(int, int64_t, int32_t, int, int);
template cudaError_t launch_persistent<float>(const SweepArgs<float>&, int, int, int64_t, GridBarrier*, int,
                                              cudaStream_t);
template cudaError_t launch_persistent<double>(const SweepArgs<double>&, int, int, int64_t, GridBarrier*, int,
                                               cudaStream_t);

template <typename T>
int64_t edge_prefetch_distance(int cfg, int num_sms)
{
    if (cfg < 0 || cfg >= kNumCfg || kCfg[cfg].P) return 0;
    const EdgeCfg& c = kCfg[cfg];
    int per_sm = 0;
    cudaError_t e = cudaSuccess;
    switch (cfg) {
    case 0: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, edge_group_kernel<T, 4, 1>, kThreads, 0); break;
    case 1: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, edge_group_kernel<T, 8, 1>, kThreads, 0); break;
    case 2: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, edge_group_kernel<T, 16, 1>, kThreads, 0); break;
    case 3: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, edge_group_kernel<T, 32, 1>, kThreads, 0); break;
    case 4: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, edge_group_kernel<T, 32, 2>, kThreads, 0); break;
    case 5: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, edge_group_kernel<T, 32, 4>, kThreads, 0); break;
    case 6: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, edge_group_kernel<T, 32, 8>, kThreads, 0); break;
    case 7: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, edge_block_kernel<T, 128, 4>, 128, 0); break;
    case 8: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, edge_block_kernel<T, 256, 2>, 256, 0); break;
    case 9: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, edge_block_kernel<T, 512, 2>, 512, 0); break;
    case 10: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, edge_block_kernel<T, 512, 3>, 512, 0); break;
    case 11: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, edge_block_kernel<T, 512, 4>, 512, 0); break;
    case 12: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, edge_block_kernel<T, 512, 5>, 512, 0); break;
    case 13: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, edge_block_kernel<T, 256, 10>, 256, 0); break;
    case 14: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, edge_block_kernel<T, 512, 8>, 512, 0); break;
    case 15: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, edge_block_kernel<T, 1024, 8>, 1024, 0); break;
    default: return 0;
    }
    if (e != cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        return 0;
    }
    const int64_t per_block = c.G ? kThreads / c.G : 1;
    return (int64_t)num_sms * per_sm * per_block;
}

template int64_t edge_prefetch_distance<float>(int, int);
template int64_t edge_prefetch_distance<double>(int, int);

int edge_group_lanes(int cfg)
{
    cfg = edge_plain_config(cfg);
    return (cfg >= 0 && cfg < kNumCfg && kCfg[cfg].G) ? kCfg[cfg].G : 32;
}

int edge_plain_config(int cfg)
{
    if (cfg < 0 || cfg >= kNumCfg || !kCfg[cfg].P) return cfg;
    if (kCfg[cfg].P == 1) return 3 + (cfg - kFirstPipelined);
    return cfg == kFirstStaged ? 12 : 14;  // the block form of the same shape
}

bool edge_config_pipelined(int cfg) { return cfg >= 0 && cfg < kNumCfg && kCfg[cfg].P == 1; }
bool edge_config_staged(int cfg) { return cfg >= 0 && cfg < kNumCfg && kCfg[cfg].P == 2; }

cudaError_t launch_convert_f32_to_f64(const float* a, double* b, int64_t count, cudaStream_t stream)
{
    if (count <= 0) return cudaSuccess;
    int64_t blocks = (count + kThreads - 1) / kThreads;
    if (blocks > 4096) blocks = 4096;
    convert_kernel<<<(int)blocks, kThreads, 0, stream>>>(a, b, count);
    return cudaGetLastError();
}

template int edge_config<float>(int);
template int edge_config<double>(int);
template int edge_grid<float>(int, int64_t, int);
template int64_t edge_parts<float>(int, int);
template int edge_capacity<float>(int);
template int edge_capacity<double>(int);
template int64_t edge_parts<double>(int, int);
template int edge_grid<double>(int, int64_t, int);
template cudaError_t launch_excess<float>(const SweepArgs<float>&, cudaStream_t, bool);
template cudaError_t launch_excess<double>(const SweepArgs<double>&, cudaStream_t, bool);
template cudaError_t launch_edge<float>(const SweepArgs<float>&, int, cudaStream_t, bool);
template cudaError_t launch_finalize<float>(const SweepArgs<float>&, cudaStream_t);
template cudaError_t launch_finalize<double>(const SweepArgs<double>&, cudaStream_t);
template cudaError_t launch_edge<double>(const SweepArgs<double>&, int, cudaStream_t, bool);

}  // namespace pdr
