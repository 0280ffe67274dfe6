// adjoint.cu -- reverse mode through T unrolled sweeps of Alg. 1.
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
//   flows    dL/df^(t)_e,k = cbar_e,k + Dbar_{j,k} - Dbar_{i,k} (eq. (3)).
// The seeds at T are dz/df = psi + h_j - h_i (eq. "cpgrad"), dz/du = -psi
// and dz/dd_k = h_{s_k,k} - h_{t_k,k}.  One warp per edge row, two passes
// over the row (the second from L1/L2), so any K works.
#include "sweep_common.cuh"

namespace pdr {
namespace {

// Warp per edge: seeds dL/df = psi + h_j - h_i and dL/du = -psi at f^(T).
template <typename T>
__global__ void __launch_bounds__(kThreads) seed_edge_kernel(SweepArgs<T> a, T* __restrict__ fbar,
                                                             double* __restrict__ ubar)
{
    const int lane = threadIdx.x & 31;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t e = w0; e < a.m; e += nw) {
        const T* fr = a.f + e * a.Kp;
        T s = T(0);
        for (int k = lane; k < a.K; k += 32) s += fr[k];
        s = group_sum<32>(s);
        const T over = s - a.u[e];
        const T psi = over > T(0) ? over : T(0);
        const T* hi = a.h + (int64_t)a.src[e] * a.Kp;
        const T* hj = a.h + (int64_t)a.col[e] * a.Kp;
        for (int k = lane; k < a.Kp; k += 32) fbar[e * a.Kp + k] = k < a.K ? psi + hj[k] - hi[k] : T(0);
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

// Warp per edge: Alg. 2's Jacobian applied to fbar (see the file comment).
template <typename T>
__global__ void __launch_bounds__(kThreads) edge_backward_kernel(SweepArgs<T> a, const T* __restrict__ theta,
                                                                 const T* __restrict__ fbar, T* __restrict__ cbar,
                                                                 double* __restrict__ ubar)
{
    const int lane = threadIdx.x & 31;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t e = w0; e < a.m; e += nw) {
        const T th = theta[e];
        const bool congested = th > T(0);
        const T cut = congested ? th : T(0);
        const T* fr = a.f + e * a.Kp;
        const T* hi = a.h + (int64_t)a.src[e] * a.Kp;
        const T* hj = a.h + (int64_t)a.col[e] * a.Kp;
        const T* fb = fbar + e * a.Kp;
        T sb = T(0);
        int na = 0;
        for (int k = lane; k < a.K; k += 32) {
            const T c = fma(T(0.5), hi[k] - hj[k], fr[k]);  // the same c as the edge-QP kernel
            if (c > cut) {
                sb += fb[k];
                ++na;
            }
        }
        sb = group_sum<32>(sb);
        na = group_sum<32>(na);
        const T corr = congested ? sb / T(2 + na) : T(0);
        for (int k = lane; k < a.Kp; k += 32) {
            T out = T(0);
            if (k < a.K) {
                const T c = fma(T(0.5), hi[k] - hj[k], fr[k]);
                out = c > cut ? fb[k] - corr : T(0);
            }
            cbar[e * a.Kp + k] = out;
        }
        if (lane == 0) ubar[e] += (double)corr;
    }
}

// Thread per (vertex, k): Dbar = (sum_out cbar - sum_in cbar) / (2 delta).
template <typename T>
__global__ void __launch_bounds__(kThreads) vertex_backward_kernel(SweepArgs<T> a, const T* __restrict__ cbar,
                                                                   T* __restrict__ Dbar)
{
    const int64_t total = (int64_t)a.n * a.Kp;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int32_t i = (int32_t)(idx / a.Kp);
        const int32_t k = (int32_t)(idx - (int64_t)i * a.Kp);
        T acc = T(0);
        for (int64_t q = a.inc_ptr[i]; q < a.inc_ptr[i + 1]; ++q) {
            const int32_t ev = a.inc[q];
            // in-edges (ev >= 0) took -h_j/2, out-edges (~e) took +h_i/2
            if (ev >= 0) acc -= cbar[(int64_t)ev * a.Kp + k];
            else acc += cbar[(int64_t)(~ev) * a.Kp + k];
        }
        Dbar[idx] = T(0.5) * acc * a.inv_deg[i];
    }
}

// Thread per (edge, k): dL/df^(t) = cbar + Dbar_j - Dbar_i.
template <typename T>
__global__ void __launch_bounds__(kThreads) edge_adjoint_kernel(SweepArgs<T> a, const T* __restrict__ cbar,
                                                                const T* __restrict__ Dbar, T* __restrict__ fbar)
{
    const int64_t total = a.m * a.Kp;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = idx / a.Kp;
        const int32_t k = (int32_t)(idx - e * a.Kp);
        fbar[idx] = cbar[idx] + Dbar[(int64_t)a.col[e] * a.Kp + k] - Dbar[(int64_t)a.src[e] * a.Kp + k];
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

template <typename T>
cudaError_t launch_backward_sweep(const SweepArgs<T>& a, const T* theta, T* fbar, T* cbar, T* Dbar, double* ubar,
                                  double* dbar, int num_sms, cudaStream_t s)
{
    edge_backward_kernel<T><<<blocks(a.m * 32, kThreads, num_sms), kThreads, 0, s>>>(a, theta, fbar, cbar, ubar);
    vertex_backward_kernel<T><<<blocks((int64_t)a.n * a.Kp, kThreads, num_sms), kThreads, 0, s>>>(a, cbar, Dbar);
    demand_kernel<T><<<blocks(a.K, kThreads, num_sms), kThreads, 0, s>>>(a, Dbar, dbar, 1);
    edge_adjoint_kernel<T><<<blocks(a.m * a.Kp, kThreads, num_sms), kThreads, 0, s>>>(a, cbar, Dbar, fbar);
    return cudaGetLastError();
}

template cudaError_t launch_seed<float>(const SweepArgs<float>&, float*, double*, double*, int, cudaStream_t);
template cudaError_t launch_seed<double>(const SweepArgs<double>&, double*, double*, double*, int, cudaStream_t);
template cudaError_t launch_backward_sweep<float>(const SweepArgs<float>&, const float*, float*, float*, float*,
                                                  double*, double*, int, cudaStream_t);
template cudaError_t launch_backward_sweep<double>(const SweepArgs<double>&, const double*, double*, double*,
                                                   double*, double*, double*, int, cudaStream_t);

}  // namespace pdr
