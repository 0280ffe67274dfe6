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

template <typename T>
__global__ void __launch_bounds__(kThreads) excess_kernel(SweepArgs<T> a)
{
    using VT = typename VecOf<T>::type;
    using A = Acc<T>;
    constexpr int N = VecOf<T>::N;
    volatile DevState* vst = a.st;
    if (a.mode == MODE_SOLVE && vst->stop) return;  // an earlier sweep of this launch stopped
    if (blockIdx.x == 0 && threadIdx.x == 0) a.st->t_sweep = vst->t;
    const uint32_t vpr = (uint32_t)(a.Kp / N);
    const uint64_t total = (uint64_t)a.n * vpr;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    typename A::V zacc = A::zero();
    T cons = T(0);
    for (uint64_t idx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += stride) {
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
        const T dgt = T(q1 - q0);
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
    // this block's fixed slice of the edge kernel's psi partials
    T capb = T(0);
    {
        const int64_t lo = (int64_t)blockIdx.x * a.n_psi / gridDim.x;
        const int64_t hi = (int64_t)(blockIdx.x + 1) * a.n_psi / gridDim.x;
        const typename A::S* pp = reinterpret_cast<const typename A::S*>(a.part_psi);
        for (int64_t b = lo + threadIdx.x; b < hi; b += blockDim.x) {
            zacc = A::add(zacc, A::load(pp + b));
            const T c = __ldcg(a.part_cap + b);
            capb = c > capb ? c : capb;
        }
    }
    block_acc_max2<T>(zacc, cons, capb);
    if (threadIdx.x == 0) {
        a.part_h[blockIdx.x] = A::to_double(zacc);
        a.part_cons[blockIdx.x] = cons;
        a.part_capb[blockIdx.x] = capb;
    }
}

// ------------------------------------------------------------------ edge QP, lane-group form

// One aligned group of G lanes per edge; each lane keeps V vectors of the
// edge's row in registers (vector q of lane l is row vector l + q*G, so a
// group reads contiguous memory).  K <= G * V * N.
template <typename T, int G, int V>
__global__ void __launch_bounds__(kThreads) edge_group_kernel(SweepArgs<T> a)
{
    using VT = typename VecOf<T>::type;
    constexpr int N = VecOf<T>::N;
    constexpr int GPW = 32 / G;  // groups per warp
    using A = Acc<T>;
    volatile DevState* vst = a.st;
    if (a.mode == MODE_SOLVE && vst->stop) return;  // an earlier sweep of this launch stopped
    if (blockIdx.x == gridDim.x - 1) {               // the decision block
        if (a.mode != MODE_PSI) reduce_and_finalize(a);
        return;
    }
    const int lane = threadIdx.x & 31;
    const int gl = lane & (G - 1);
    const int gw = lane / G;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)(gridDim.x - 1) * blockDim.x) >> 5;
    const int vpr = a.Kp / N;
    const bool psi_only = (a.mode == MODE_PSI);
    typename A::V zpsi = A::zero();
    T capmax = T(0);
    for (int64_t base = warp * GPW; base < a.m; base += nwarps * GPW) {
        const int64_t e = base + gw;
        const bool valid = e < a.m;
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
                    unpack(__ldg(hi + v), ax);
                    unpack(__ldg(hj + v), bx);
                    // c_k = 1/2 ((h_ik + f_k) - (h_jk - f_k)) = f_k + (h_ik - h_jk)/2
#pragma unroll
                    for (int j = 0; j < N; ++j) c[q][j] = fma(T(0.5), ax[j] - bx[j], fx[j]);
                } else {
#pragma unroll
                    for (int j = 0; j < N; ++j) c[q][j] = T(0);
                }
            }
        }
        T theta = T(0);
        if (!psi_only) {
            // One pass gives s = sum_k max(0, c_k), |{c_k > 0}|, and the same
            // two sums above a warm start w slightly below the previous
            // sweep's root.  g(theta) = sum_k max(0, c_k - theta) - u - 2 theta
            // decreases in theta and vanishes at the root, so g(w) >= 0
            // certifies w <= root and the active set lies inside {c > w}.
            const T w = valid ? a.theta[e] * T(0.999) : T(0);
            T sp = T(0), sw = T(0);
            int np = 0, nw = 0;
#pragma unroll
            for (int q = 0; q < V; ++q)
#pragma unroll
                for (int j = 0; j < N; ++j) {
                    const T x = c[q][j];
                    if (x > T(0)) {
                        sp += x;
                        ++np;
                    }
                    if (x > w) {
                        sw += x;
                        ++nw;
                    }
                }
            const T s = group_sum<G>(sp);
            const int n0 = group_sum<G>(np);
            const T S_w = group_sum<G>(sw);
            const int n_w = group_sum<G>(nw);
            const bool congested = valid && s > ue;  // Case 2 of Alg. 2 (s <= u is Case 1)
            bool done = !congested;
            int nA = n0;
            if (congested) {
                if (w > T(0) && S_w - T(n_w) * w - ue - T(2) * w >= T(0)) {
                    nA = n_w;
                    theta = (S_w - ue) / T(2 + n_w);
                } else {
                    theta = (s - ue) / T(2 + n0);
                }
            }
            for (int it = 0; __any_sync(kFull, !done); ++it) {
                T sa = T(0);
                int na = 0;
#pragma unroll
                for (int q = 0; q < V; ++q)
#pragma unroll
                    for (int j = 0; j < N; ++j)
                        if (c[q][j] > theta) {
                            sa += c[q][j];
                            ++na;
                        }
                const T S2 = group_sum<G>(sa);
                const int n2 = group_sum<G>(na);
                if (!done) {
                    if (n2 >= nA) done = true;
                    else {
                        nA = n2;
                        theta = (S2 - ue) / T(2 + n2);
                    }
                }
                if (it > a.Kp + 2) break;  // unreachable: nA drops every round
            }
            if (valid && gl == 0) a.theta[e] = theta;
        }
        // f' = max(0, c - psi'/2); psi of the stored flows
        T rs = T(0);
#pragma unroll
        for (int q = 0; q < V; ++q) {
            const int v = gl + q * G;
            T o[N];
#pragma unroll
            for (int j = 0; j < N; ++j) {
                const T x = c[q][j] - theta;
                o[j] = x > T(0) ? x : T(0);
                rs += o[j];
            }
            if (!psi_only && valid && v < vpr) reinterpret_cast<VT*>(orow)[v] = pack4(o);
        }
        rs = group_sum<G>(rs);
        if (valid && gl == 0) {
            const T over = rs - ue;
            const T psi = over > T(0) ? over : T(0);
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
    using VT = typename VecOf<T>::type;
    using A = Acc<T>;
    constexpr int N = VecOf<T>::N;
    volatile DevState* vst = a.st;
    if (a.mode == MODE_SOLVE && vst->stop) return;
    if (blockIdx.x == gridDim.x - 1) {
        if (a.mode != MODE_PSI) reduce_and_finalize(a);
        return;
    }
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
        T theta = T(0);
        if (!psi_only) {
            const T w = a.theta[e] * T(0.999);
            T sp = T(0), sw = T(0);
            int np = 0, nw = 0;
#pragma unroll
            for (int q = 0; q < V; ++q)
#pragma unroll
                for (int j = 0; j < N; ++j) {
                    const T x = c[q][j];
                    if (x > T(0)) {
                        sp += x;
                        ++np;
                    }
                    if (x > w) {
                        sw += x;
                        ++nw;
                    }
                }
            const T s = group_sum<32>(sp);
            const int n0 = group_sum<32>(np);
            const T S_w = group_sum<32>(sw);
            const int n_w = group_sum<32>(nw);
            if (s > ue) {  // warp-uniform
                int nA = n0;
                if (w > T(0) && S_w - T(n_w) * w - ue - T(2) * w >= T(0)) {
                    nA = n_w;
                    theta = (S_w - ue) / T(2 + n_w);
                } else {
                    theta = (s - ue) / T(2 + n0);
                }
                for (int it = 0; it <= a.Kp + 2; ++it) {
                    T sa = T(0);
                    int na = 0;
#pragma unroll
                    for (int q = 0; q < V; ++q)
#pragma unroll
                        for (int j = 0; j < N; ++j)
                            if (c[q][j] > theta) {
                                sa += c[q][j];
                                ++na;
                            }
                    const T S2 = group_sum<32>(sa);
                    const int n2 = group_sum<32>(na);
                    if (n2 >= nA) break;
                    nA = n2;
                    theta = (S2 - ue) / T(2 + n2);
                }
            }
            if (lane == 0) a.theta[e] = theta;
        }
        T rs = T(0);
        T* orow = a.f_out + e * a.Kp;
#pragma unroll
        for (int q = 0; q < V; ++q) {
            const int v = lane + q * 32;
            T o[N];
#pragma unroll
            for (int j = 0; j < N; ++j) {
                const T x = c[q][j] - theta;
                o[j] = x > T(0) ? x : T(0);
                rs += o[j];
            }
            if (!psi_only && v < vpr) reinterpret_cast<VT*>(orow)[v] = pack4(o);
        }
        rs = group_sum<32>(rs);
        if (lane == 0) {
            const T over = rs - ue;
            const T psi = over > T(0) ? over : T(0);
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

// One block of B threads per edge; thread l keeps row vectors l + q*B.
template <typename T, int B, int V>
__global__ void __launch_bounds__(B, (B <= 512 ? 2 : 1)) edge_block_kernel(SweepArgs<T> a)
{
    using VT = typename VecOf<T>::type;
    constexpr int N = VecOf<T>::N;
    using A = Acc<T>;
    __shared__ T sa_buf[32];
    __shared__ int sb_buf[32];
    volatile DevState* vst = a.st;
    if (a.mode == MODE_SOLVE && vst->stop) return;  // an earlier sweep of this launch stopped
    if (blockIdx.x == gridDim.x - 1) {               // the decision block
        if (a.mode != MODE_PSI) reduce_and_finalize(a);
        return;
    }
    const int vpr = a.Kp / N;
    const bool psi_only = (a.mode == MODE_PSI);
    typename A::V zpsi = A::zero();
    T capmax = T(0);
    for (int64_t e = blockIdx.x; e < a.m; e += gridDim.x - 1) {
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
                unpack(reinterpret_cast<const VT*>(frow)[v], fx);
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
        T theta = T(0);
        if (!psi_only) {
            // same warm-started active-set search as the lane-group form
            const T w = a.theta[e] * T(0.999);
            T s = T(0), S_w = T(0);
            int n0 = 0, n_w = 0;
#pragma unroll
            for (int q = 0; q < V; ++q)
#pragma unroll
                for (int j = 0; j < N; ++j) {
                    const T x = c[q][j];
                    if (x > T(0)) {
                        s += x;
                        ++n0;
                    }
                    if (x > w) {
                        S_w += x;
                        ++n_w;
                    }
                }
            block_sum2(s, n0, sa_buf, sb_buf);
            block_sum2(S_w, n_w, sa_buf, sb_buf);
            if (s > ue) {  // block-uniform
                int nA = n0;
                if (w > T(0) && S_w - T(n_w) * w - ue - T(2) * w >= T(0)) {
                    nA = n_w;
                    theta = (S_w - ue) / T(2 + n_w);
                } else {
                    theta = (s - ue) / T(2 + n0);
                }
                for (int it = 0; it <= a.Kp + 2; ++it) {
                    T S2 = T(0);
                    int n2 = 0;
#pragma unroll
                    for (int q = 0; q < V; ++q)
#pragma unroll
                        for (int j = 0; j < N; ++j)
                            if (c[q][j] > theta) {
                                S2 += c[q][j];
                                ++n2;
                            }
                    block_sum2(S2, n2, sa_buf, sb_buf);
                    if (n2 >= nA) break;
                    nA = n2;
                    theta = (S2 - ue) / T(2 + n2);
                }
            }
            if (threadIdx.x == 0) a.theta[e] = theta;
        }
        T rs = T(0);
#pragma unroll
        for (int q = 0; q < V; ++q) {
            const int v = threadIdx.x + q * B;
            T o[N];
#pragma unroll
            for (int j = 0; j < N; ++j) {
                const T x = c[q][j] - theta;
                o[j] = x > T(0) ? x : T(0);
                rs += o[j];
            }
            if (!psi_only && v < vpr) reinterpret_cast<VT*>(orow)[v] = pack4(o);
        }
        int dummy = 0;
        block_sum2(rs, dummy, sa_buf, sb_buf);
        if (threadIdx.x == 0) {
            const T over = rs - ue;
            const T psi = over > T(0) ? over : T(0);
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
    // 0..13 ordered by capacity (elements per row); two 512-thread blocks fit
    // on an SM, so the block forms keep two edges in flight per SM up to 16,384
    {4, 0, 1, 0},   {8, 0, 1, 0},   {16, 0, 1, 0},  {32, 0, 1, 0},  {32, 0, 2, 0},
    {32, 0, 4, 0},  {32, 0, 8, 0},  {0, 256, 2, 0}, {0, 512, 2, 0}, {0, 512, 3, 0},
    {0, 512, 4, 0}, {0, 512, 5, 0}, {0, 512, 8, 0}, {0, 1024, 8, 0},
    // 14..16: the pipelined forms of 3..5 (the gradient kernels of Alg. 3/4
    // run the plain form of the same capacity); at 8 vectors per lane the
    // prefetched rows no longer fit in registers
    {32, 0, 1, 1},  {32, 0, 2, 1},  {32, 0, 4, 1},
};
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
int edge_grid(int cfg, int64_t m, int num_sms)
{
    const EdgeCfg& c = kCfg[cfg];
    int64_t want, cap;
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

template <typename T>
cudaError_t launch_excess(const SweepArgs<T>& a, cudaStream_t stream)
{
    excess_kernel<T><<<a.grid_v, kThreads, 0, stream>>>(a);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_finalize(const SweepArgs<T>& a, cudaStream_t stream)
{
    finalize_kernel<T><<<1, kThreads, 0, stream>>>(a);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_edge(const SweepArgs<T>& a, int cfg, cudaStream_t stream)
{
    const int g = a.grid_e + 1;  // edge blocks plus the decision block
    switch (cfg) {
    case 0: edge_group_kernel<T, 4, 1><<<g, kThreads, 0, stream>>>(a); break;
    case 1: edge_group_kernel<T, 8, 1><<<g, kThreads, 0, stream>>>(a); break;
    case 2: edge_group_kernel<T, 16, 1><<<g, kThreads, 0, stream>>>(a); break;
    case 3: edge_group_kernel<T, 32, 1><<<g, kThreads, 0, stream>>>(a); break;
    case 4: edge_group_kernel<T, 32, 2><<<g, kThreads, 0, stream>>>(a); break;
    case 5: edge_group_kernel<T, 32, 4><<<g, kThreads, 0, stream>>>(a); break;
    case 6: edge_group_kernel<T, 32, 8><<<g, kThreads, 0, stream>>>(a); break;
    case 7: edge_block_kernel<T, 256, 2><<<g, 256, 0, stream>>>(a); break;
    case 8: edge_block_kernel<T, 512, 2><<<g, 512, 0, stream>>>(a); break;
    case 9: edge_block_kernel<T, 512, 3><<<g, 512, 0, stream>>>(a); break;
    case 10: edge_block_kernel<T, 512, 4><<<g, 512, 0, stream>>>(a); break;
    case 11: edge_block_kernel<T, 512, 5><<<g, 512, 0, stream>>>(a); break;
    case 12: edge_block_kernel<T, 512, 8><<<g, 512, 0, stream>>>(a); break;
    case 13: edge_block_kernel<T, 1024, 8><<<g, 1024, 0, stream>>>(a); break;
    case 14: edge_pipe_kernel<T, 1><<<g, kThreads, 0, stream>>>(a); break;
    case 15: edge_pipe_kernel<T, 2><<<g, kThreads, 0, stream>>>(a); break;
    case 16: edge_pipe_kernel<T, 4><<<g, kThreads, 0, stream>>>(a); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

int edge_plain_config(int cfg) { return (cfg >= 0 && cfg < kNumCfg && kCfg[cfg].P) ? 3 + (cfg - 14) : cfg; }

bool edge_config_pipelined(int cfg) { return cfg >= 0 && cfg < kNumCfg && kCfg[cfg].P; }

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
template cudaError_t launch_excess<float>(const SweepArgs<float>&, cudaStream_t);
template cudaError_t launch_excess<double>(const SweepArgs<double>&, cudaStream_t);
template cudaError_t launch_edge<float>(const SweepArgs<float>&, int, cudaStream_t);
template cudaError_t launch_finalize<float>(const SweepArgs<float>&, cudaStream_t);
template cudaError_t launch_finalize<double>(const SweepArgs<double>&, cudaStream_t);
template cudaError_t launch_edge<double>(const SweepArgs<double>&, int, cudaStream_t);

}  // namespace pdr
