// adjoint.cu -- reverse mode through T unrolled sweeps of Alg. 1 (with
// Alg. 2's step, or the capacity-kept step of Program (6), where the
// Jacobian is the same with 2 + |A| replaced by |A|).
//
// L(u, d) = z(f^(T)) with f^(0) = 0 and f^(t+1) = one sweep (eq. (3), (2),
// then Alg. 2 on every edge).  With fbar = dL/df^(t+1) the backward step of
// sweep t is:
//   edge     c_k = f_k + (h_ik - h_jk)/2 and the stored root theta_e of the
//            sweep give the active set (A = {c_k > theta} if theta > 0, else
//            {c_k > 0}); Alg. 2's Jacobian gives
//            cbar_k = [k in A] (fbar_k - [theta > 0] Sbar / (2 + |A|)),
//            Sbar = sum_{k in A} fbar_k, and ubar_e += [theta > 0] Sbar/(2 + |A|);
//   vertex   Dbar_ik = (sum_{e out of i} cbar_e,k - sum_{e into i} cbar_e,k) / (2 delta_i)
//            (h = Delta/delta, and c takes +h_i/2 and -h_j/2);
//   demand   dbar_k += Dbar_{s_k,k} - Dbar_{t_k,k} (eq. (3h));
//   flows    dL/df^(t)_e,k = cbar_e,k + Dbar_{j,k} - Dbar_{i,k} (eq. (3)), formed
//            on the fly by the next (earlier) sweep's edge step.
// The seeds at T are dz/df = psi + h_j - h_i (eq. "cpgrad"), dz/du = -psi
// and dz/dd_k = h_{s_k,k} - h_{t_k,k}.  One warp per edge row, two passes
// over the row (the second from L1/L2), so any K works.
#include "sweep_common.cuh"

namespace pdr {
namespace {

// All row accesses are vectors of 16 bytes (float4 / double2): rows are
// padded to Kp, a multiple of the vector width, and the padding stays 0.

// Warp per edge: seeds dL/df = psi + h_j - h_i and dL/du = -psi at f^(T).
template <typename T>
__global__ void __launch_bounds__(kThreads) seed_edge_kernel(SweepArgs<T> a, T* __restrict__ fbar,
                                                             double* __restrict__ ubar)
{
    using VT = typename VecOf<T>::type;
    constexpr int N = VecOf<T>::N;
    const int lane = threadIdx.x & 31;
    const int vpr = a.Kp / N;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t e = w0; e < a.m; e += nw) {
        const VT* fr = reinterpret_cast<const VT*>(a.f + e * a.Kp);
        T s = T(0);
        for (int v = lane; v < vpr; v += 32) {
            T x[N];
            unpack(fr[v], x);
#pragma unroll
            for (int j = 0; j < N; ++j) s += x[j];
        }
        s = group_sum<32>(s);
        const T over = s - a.u[e];
        const T psi = over > T(0) ? over : T(0);
        const VT* hi = reinterpret_cast<const VT*>(a.h + (int64_t)a.src[e] * a.Kp);
        const VT* hj = reinterpret_cast<const VT*>(a.h + (int64_t)a.col[e] * a.Kp);
        VT* out = reinterpret_cast<VT*>(fbar + e * a.Kp);
        for (int v = lane; v < vpr; v += 32) {
            T x[N], y[N], o[N];
            unpack(hi[v], x);
            unpack(hj[v], y);
#pragma unroll
            for (int j = 0; j < N; ++j) o[j] = v * N + j < a.K ? psi + y[j] - x[j] : T(0);
            out[v] = pack4(o);
        }
        if (lane == 0) ubar[e] = -(double)psi;
    }
}

// dL/dd_k = h_{s_k,k} - h_{t_k,k} (seed) or += Dbar_{s_k,k} - Dbar_{t_k,k} (per sweep).
template <typename T>
__global__ void demand_kernel(SweepArgs<T> a, const T* __restrict__ x, double* __restrict__ dbar, int accumulate)
{
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < a.K; k += gridDim.x * blockDim.x) {
        const double v = (double)x[(int64_t)a.s[k] * a.Kp + k] - (double)x[(int64_t)a.t[k] * a.Kp + k];
        dbar[k] = accumulate ? dbar[k] + v : v;
    }
}

// Warp per edge: Alg. 2's Jacobian applied to fbar = dL/df^(t+1) (see the
// file comment).  fbar is either read (the seed, at t + 1 = T) or formed on
// the fly from the previous backward step's results, fbar = cbar^(t+1) +
// Dbar^(t+1)_j - Dbar^(t+1)_i (`fused`), which saves writing and reading it.
// cbar is updated in place: each element is read (as part of fbar) and then
// written by the same lane.  Pass 1 decides every element's membership of the
// active set (c > cut) from f and both height rows and records it as warp
// ballots in `mask` (N words per 32 vectors of the row); pass 2 re-reads only
// fbar's rows.
template <typename T, bool FUSED>
__device__ __forceinline__ void fbar_vec(const typename VecOf<T>::type* fb, const typename VecOf<T>::type* cb,
                                         const typename VecOf<T>::type* di, const typename VecOf<T>::type* dj, int v,
                                         T (&g)[VecOf<T>::N])
{
    constexpr int N = VecOf<T>::N;
    if constexpr (FUSED) {
        T c[N], x[N], y[N];
        unpack(cb[v], c);
        unpack(di[v], x);
        unpack(dj[v], y);
#pragma unroll
        for (int j = 0; j < N; ++j) g[j] = c[j] + y[j] - x[j];
    } else {
        unpack(fb[v], g);
    }
}

template <typename T, bool FUSED>
__global__ void __launch_bounds__(kThreads) edge_backward_kernel(SweepArgs<T> a, const T* __restrict__ theta,
                                                                 const T* __restrict__ fbar, T* cbar,
                                                                 const T* __restrict__ Dbar, double* __restrict__ ubar,
                                                                 uint32_t* __restrict__ mask)
{
    using VT = typename VecOf<T>::type;
    constexpr int N = VecOf<T>::N;
    const int lane = threadIdx.x & 31;
    const int vpr = a.Kp / N;
    const int nq = (vpr + 31) / 32;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t e = w0; e < a.m; e += nw) {
        const T th = theta[e];
        const bool congested = th > T(0);
        const T cut = congested ? th : T(0);
        const int32_t ti = a.src[e], tj = a.col[e];
        const VT* fr = reinterpret_cast<const VT*>(a.f + e * a.Kp);
        const VT* hi = reinterpret_cast<const VT*>(a.h + (int64_t)ti * a.Kp);
        const VT* hj = reinterpret_cast<const VT*>(a.h + (int64_t)tj * a.Kp);
        const VT* fb = FUSED ? nullptr : reinterpret_cast<const VT*>(fbar + e * a.Kp);
        VT* cb = reinterpret_cast<VT*>(cbar + e * a.Kp);
        const VT* di = FUSED ? reinterpret_cast<const VT*>(Dbar + (int64_t)ti * a.Kp) : nullptr;
        const VT* dj = FUSED ? reinterpret_cast<const VT*>(Dbar + (int64_t)tj * a.Kp) : nullptr;
        uint32_t* me = mask + e * (int64_t)nq * N;
        T sb = T(0);
        int na = 0;
        for (int q = 0; q < nq; ++q) {  // every lane takes every round: the ballots need the whole warp
            const int v = q * 32 + lane;
            const bool live = v < vpr;
            T f[N] = {}, x[N] = {}, y[N] = {}, g[N] = {};
            if (live) {
                unpack(fr[v], f);
                unpack(hi[v], x);
                unpack(hj[v], y);
                fbar_vec<T, FUSED>(fb, cb, di, dj, v, g);
            }
#pragma unroll
            for (int j = 0; j < N; ++j) {
                const bool act = live && fma(T(0.5), x[j] - y[j], f[j]) > cut;  // the edge-QP kernel's c
                if (act) {
                    sb += g[j];
                    ++na;
                }
                const uint32_t b = __ballot_sync(kFull, act);
                if (lane == j) me[q * N + j] = b;
            }
        }
        __syncwarp();  // the ballots written above are read by every lane below
        sb = group_sum<32>(sb);
        na = group_sum<32>(na);
        // Alg. 2: theta = (S_A - u)/(2 + |A|); capacity kept: (S_A - u)/|A|.  With
        // the capacity kept and u = 0 no element is active and nothing flows back.
        const T corr = (congested && na > 0) ? sb / T((a.ck ? 0 : 2) + na) : T(0);
        for (int q = 0; q < nq; ++q) {
            const int v = q * 32 + lane;
            if (v >= vpr) continue;
            T g[N], o[N];
            fbar_vec<T, FUSED>(fb, cb, di, dj, v, g);
#pragma unroll
            for (int j = 0; j < N; ++j) o[j] = ((me[q * N + j] >> lane) & 1u) ? g[j] - corr : T(0);
            cb[v] = pack4(o);
        }
        if (lane == 0) ubar[e] += (double)corr;
    }
}

// Block of B threads per edge for long rows (thread l holds row vectors l +
// q*B): the same step as edge_backward_kernel, but the row's cotangent and
// its active-set bits stay in registers between the block-wide sum and the
// write, so every input row is read once (the warp form reads fbar, or cbar
// and both Dbar rows, a second time).
template <typename T, int B, int V, bool FUSED>
__global__ void __launch_bounds__(B, (1024 / B > 1 ? 1024 / B : 1))
    edge_backward_block_kernel(SweepArgs<T> a, const T* __restrict__ theta, const T* __restrict__ fbar, T* cbar,
                               const T* __restrict__ Dbar, double* __restrict__ ubar)
{
    using VT = typename VecOf<T>::type;
    constexpr int N = VecOf<T>::N;
    static_assert(V * N <= 32, "one bit per held value");
    __shared__ T sa_buf[33];
    __shared__ int sb_buf[33];
    const int vpr = a.Kp / N;
    for (int64_t e = blockIdx.x; e < a.m; e += gridDim.x) {
        const T th = theta[e];
        const bool congested = th > T(0);
        const T cut = congested ? th : T(0);
        const int32_t ti = a.src[e], tj = a.col[e];
        const VT* fr = reinterpret_cast<const VT*>(a.f + e * a.Kp);
        const VT* hi = reinterpret_cast<const VT*>(a.h + (int64_t)ti * a.Kp);
        const VT* hj = reinterpret_cast<const VT*>(a.h + (int64_t)tj * a.Kp);
        const VT* fb = FUSED ? nullptr : reinterpret_cast<const VT*>(fbar + e * a.Kp);
        VT* cb = reinterpret_cast<VT*>(cbar + e * a.Kp);
        const VT* di = FUSED ? reinterpret_cast<const VT*>(Dbar + (int64_t)ti * a.Kp) : nullptr;
        const VT* dj = FUSED ? reinterpret_cast<const VT*>(Dbar + (int64_t)tj * a.Kp) : nullptr;
        T g[V][N];
        uint32_t act = 0;  // bit q*N + j: value j of vector q is in the active set
        T sb = T(0);
        int na = 0;
#pragma unroll
        for (int q = 0; q < V; ++q) {
            const int v = threadIdx.x + q * B;
            if (v < vpr) {
                T f[N], x[N], y[N];
                unpack(fr[v], f);
                unpack(hi[v], x);
                unpack(hj[v], y);
                fbar_vec<T, FUSED>(fb, cb, di, dj, v, g[q]);
#pragma unroll
                for (int j = 0; j < N; ++j)
                    if (fma(T(0.5), x[j] - y[j], f[j]) > cut) {  // the edge-QP kernel's c
                        act |= 1u << (q * N + j);
                        sb += g[q][j];
                        ++na;
                    }
            } else {
#pragma unroll
                for (int j = 0; j < N; ++j) g[q][j] = T(0);
            }
        }
        block_sum2(sb, na, sa_buf, sb_buf);
        const T corr = (congested && na > 0) ? sb / T((a.ck ? 0 : 2) + na) : T(0);
#pragma unroll
        for (int q = 0; q < V; ++q) {
            const int v = threadIdx.x + q * B;
            if (v < vpr) {
                T o[N];
#pragma unroll
                for (int j = 0; j < N; ++j) o[j] = ((act >> (q * N + j)) & 1u) ? g[q][j] - corr : T(0);
                cb[v] = pack4(o);
            }
        }
        if (threadIdx.x == 0) ubar[e] += (double)corr;
    }
}

// Thread per (vertex, vector): Dbar = (sum_out cbar - sum_in cbar) / (2 delta),
// the incidence list traversed in its stored order as by the excess kernel.
template <typename T>
__global__ void __launch_bounds__(kThreads) vertex_backward_kernel(SweepArgs<T> a, const T* __restrict__ cbar,
                                                                   T* __restrict__ Dbar)
{
    using VT = typename VecOf<T>::type;
    constexpr int N = VecOf<T>::N;
    const int64_t vpr = a.Kp / N;
    const int64_t total = (int64_t)a.n * vpr;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int32_t i = (int32_t)(idx / vpr);
        const int64_t v = idx - (int64_t)i * vpr;
        T acc[N];
#pragma unroll
        for (int j = 0; j < N; ++j) acc[j] = T(0);
        const int64_t q1 = a.inc_ptr[i + 1];
        int64_t q = a.inc_ptr[i];
        for (; q + 4 <= q1; q += 4) {  // four rows in flight
            int32_t ev[4];
            T x[4][N];
#pragma unroll
            for (int u = 0; u < 4; ++u) ev[u] = a.inc[q + u];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int64_t e = ev[u] >= 0 ? ev[u] : ~ev[u];
                unpack(reinterpret_cast<const VT*>(cbar + e * a.Kp)[v], x[u]);
            }
            // in-edges (ev >= 0) took -h_j/2, out-edges (~e) took +h_i/2
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int j = 0; j < N; ++j) acc[j] = ev[u] >= 0 ? acc[j] - x[u][j] : acc[j] + x[u][j];
        }
        for (; q < q1; ++q) {
            const int32_t ev = a.inc[q];
            const int64_t e = ev >= 0 ? ev : ~ev;
            T x[N];
            unpack(reinterpret_cast<const VT*>(cbar + e * a.Kp)[v], x);
#pragma unroll
            for (int j = 0; j < N; ++j) acc[j] = ev >= 0 ? acc[j] - x[j] : acc[j] + x[j];
        }
        const T s = T(0.5) * a.inv_deg[i];
        T o[N];
#pragma unroll
        for (int j = 0; j < N; ++j) o[j] = acc[j] * s;
        reinterpret_cast<VT*>(Dbar + (int64_t)i * a.Kp)[v] = pack4(o);
    }
}

int blocks(int64_t work, int per_block, int num_sms)
{
    int64_t b = (work + per_block - 1) / per_block;
    const int64_t cap = (int64_t)num_sms * 16;
    if (b > cap) b = cap;
    return (int)(b < 1 ? 1 : b);
}

}  // namespace

template <typename T>
cudaError_t launch_seed(const SweepArgs<T>& a, T* fbar, double* ubar, double* dbar, int num_sms, cudaStream_t s)
{
    seed_edge_kernel<T><<<blocks(a.m * 32, kThreads, num_sms), kThreads, 0, s>>>(a, fbar, ubar);
    demand_kernel<T><<<blocks(a.K, kThreads, num_sms), kThreads, 0, s>>>(a, a.h, dbar, 0);
    return cudaGetLastError();
}

template <typename T, int B, int V>
void launch_backward_block(const SweepArgs<T>& a, const T* theta, const T* fbar, T* cbar, T* Dbar, double* ubar,
                           int fused, int num_sms, cudaStream_t s)
{
    const int64_t per_sm = 1024 / B > 1 ? 1024 / B : 1;  // resident under the kernel's launch bounds
    const int g = (int)(a.m < per_sm * num_sms ? a.m : per_sm * num_sms);
    if (fused) edge_backward_block_kernel<T, B, V, true><<<g, B, 0, s>>>(a, theta, fbar, cbar, Dbar, ubar);
    else edge_backward_block_kernel<T, B, V, false><<<g, B, 0, s>>>(a, theta, fbar, cbar, Dbar, ubar);
}

// The edge step's form: the block form with the smallest row capacity that
// holds Kp, for rows longer than two vectors per lane of a warp; else (and
// beyond the largest block capacity) the warp form.
template <typename T>
int backward_block_form(int Kp)
{
    const int vpr = Kp / VecOf<T>::N;
    if (vpr <= 64) return -1;
    const int cap[] = {128 * 2, 128 * 4, 256 * 4, 512 * 4, 512 * 5, 512 * 8, 1024 * 8};  // vectors, B x V
    for (int i = 0; i < 7; ++i)
        if (vpr <= cap[i]) return i;
    return -1;
}

template <typename T>
cudaError_t launch_backward_sweep(const SweepArgs<T>& a, const T* theta, const T* fbar, T* cbar, T* Dbar,
                                  double* ubar, double* dbar, uint32_t* mask, int fused, int num_sms, cudaStream_t s)
{
    const int ge = blocks(a.m * 32, kThreads, num_sms);
    switch (a.m > 0 ? backward_block_form<T>(a.Kp) : -1) {
    case 0: launch_backward_block<T, 128, 2>(a, theta, fbar, cbar, Dbar, ubar, fused, num_sms, s); break;
    case 1: launch_backward_block<T, 128, 4>(a, theta, fbar, cbar, Dbar, ubar, fused, num_sms, s); break;
    case 2: launch_backward_block<T, 256, 4>(a, theta, fbar, cbar, Dbar, ubar, fused, num_sms, s); break;
    case 3: launch_backward_block<T, 512, 4>(a, theta, fbar, cbar, Dbar, ubar, fused, num_sms, s); break;
    case 4: launch_backward_block<T, 512, 5>(a, theta, fbar, cbar, Dbar, ubar, fused, num_sms, s); break;
    case 5: launch_backward_block<T, 512, 8>(a, theta, fbar, cbar, Dbar, ubar, fused, num_sms, s); break;
    case 6: launch_backward_block<T, 1024, 8>(a, theta, fbar, cbar, Dbar, ubar, fused, num_sms, s); break;
    default:
        if (fused) edge_backward_kernel<T, true><<<ge, kThreads, 0, s>>>(a, theta, fbar, cbar, Dbar, ubar, mask);
        else edge_backward_kernel<T, false><<<ge, kThreads, 0, s>>>(a, theta, fbar, cbar, Dbar, ubar, mask);
    }
    vertex_backward_kernel<T><<<blocks((int64_t)a.n * (a.Kp / VecOf<T>::N), kThreads, num_sms), kThreads, 0, s>>>(
        a, cbar, Dbar);
    demand_kernel<T><<<blocks(a.K, kThreads, num_sms), kThreads, 0, s>>>(a, Dbar, dbar, 1);
    return cudaGetLastError();
}

template cudaError_t launch_seed<float>(const SweepArgs<float>&, float*, double*, double*, int, cudaStream_t);
template cudaError_t launch_seed<double>(const SweepArgs<double>&, double*, double*, double*, int, cudaStream_t);
template cudaError_t launch_backward_sweep<float>(const SweepArgs<float>&, const float*, const float*, float*, float*,
                                                  double*, double*, uint32_t*, int, int, cudaStream_t);
template cudaError_t launch_backward_sweep<double>(const SweepArgs<double>&, const double*, const double*, double*,
                                                   double*, double*, double*, uint32_t*, int, int, cudaStream_t);

}  // namespace pdr
