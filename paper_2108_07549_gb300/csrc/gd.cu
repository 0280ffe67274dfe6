// gd.cu -- the flow update of Alg. 3 (PDR via adaptive gradient descent) and
// Alg. 4 (PDR via gradient descent with momentum).
//
// Per edge (i, j), with h and psi of iteration t:
//   phi_k   = h_ik - h_jk - psi_ij                       (potential difference, eq. (4))
//   df_k    = max(-f_k, beta_ij * phi_k)                 (projected step)
//   dz      = 1/2 (psi'^2 - psi^2) + sum_k (df_k^2 - (h_ik - h_jk) df_k)
//             with psi' = max(0, sum_k (f_k + df_k) - u)  (eq. (9) at the step minus at 0)
//   dz <= 0: accept  (Alg. 3: f += df;  Alg. 4: v = gamma v + df, f = max(0, f + v))
//   else   : reject, beta = max(beta_min, beta * alpha_dec)
//   t mod 10 = 0: beta = min(beta_max, beta * alpha_inc) (after the decision)
// The new flows, velocities and rates go to the other buffers; psi of the
// stored new flows feeds the objective exactly as in the edge-QP kernel, and
// the launch's extra block takes the stop decision.
#include "sweep_common.cuh"

namespace pdr {
namespace {

template <typename T>
__device__ __forceinline__ T new_beta(const SweepArgs<T>& a, T beta, bool accept, bool grow)
{
    if (!accept) {
        const T b = beta * a.alpha_dec;
        beta = b > a.beta_min ? b : a.beta_min;
    }
    if (grow) {
        const T b = beta * a.alpha_inc;
        beta = b < a.beta_max ? b : a.beta_max;
    }
    return beta;
}

// One aligned group of G lanes per edge; lane l holds row vectors l + q*G.
template <typename T, int G, int V, bool M>
__global__ void __launch_bounds__(kThreads) gd_group_kernel(SweepArgs<T> a)
{
    using VT = typename VecOf<T>::type;
    using A = Acc<T>;
    constexpr int N = VecOf<T>::N;
    constexpr int GPW = 32 / G;
    volatile DevState* vst = a.st;
    if (sweep_stopped(a)) return;  // an earlier sweep of this solve stopped
    if (blockIdx.x == gridDim.x - 1) {               // the decision block
        if (a.mode != MODE_PSI) reduce_and_finalize(a);
        return;
    }
    if (final_evaluation(a)) return;  // the sweep cap stops this sweep: its output is not used
    const bool grow = (vst->t_sweep % 10) == 0;
    const int lane = threadIdx.x & 31;
    const int gl = lane & (G - 1);
    const int gw = lane / G;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)(gridDim.x - 1) * blockDim.x) >> 5;
    const int vpr = a.Kp / N;
    typename A::V zpsi = A::zero();
    T capmax = T(0);
    for (int64_t base = warp * GPW; base < a.m; base += nwarps * GPW) {
        const int64_t e = base + gw;
        const bool valid = e < a.m;
        const T ue = valid ? a.u[e] : T(0);
        const T beta = valid ? a.beta_in[e] : T(0);
        const int64_t row = (valid ? e : 0) * a.Kp;
        const VT* hi = reinterpret_cast<const VT*>(a.h + (int64_t)(valid ? a.src[e] : 0) * a.Kp);
        const VT* hj = reinterpret_cast<const VT*>(a.h + (int64_t)(valid ? a.col[e] : 0) * a.Kp);
        // h_ik - h_jk stays in registers; the flow row (read-only in this
        // sweep: the new flows go to the other buffer) is re-read from L1
        const VT* frow = reinterpret_cast<const VT*>(a.f + row);
        T d[V][N];
        T fs = T(0);
#pragma unroll
        for (int q = 0; q < V; ++q) {
            const int v = gl + q * G;
            if (valid && v < vpr) {
                T fx[N], ax[N], bx[N];
                unpack(__ldg(frow + v), fx);
                unpack(__ldg(hi + v), ax);
                unpack(__ldg(hj + v), bx);
#pragma unroll
                for (int j = 0; j < N; ++j) {
                    d[q][j] = ax[j] - bx[j];
                    fs += fx[j];
                }
            } else {
#pragma unroll
                for (int j = 0; j < N; ++j) d[q][j] = T(0);
            }
        }
        fs = group_sum<G>(fs);
        const T over0 = fs - ue;
        const T psi = over0 > T(0) ? over0 : T(0);  // psi^(t), eq. (41)
        T s2 = T(0), D = T(0);
#pragma unroll
        for (int q = 0; q < V; ++q) {
            const int v = gl + q * G;
            T fx[N];
            if (valid && v < vpr) unpack(__ldg(frow + v), fx);
            else
#pragma unroll
                for (int j = 0; j < N; ++j) fx[j] = T(0);
#pragma unroll
            for (int j = 0; j < N; ++j) {
                const T st = beta * (d[q][j] - psi);
                const T df = st > -fx[j] ? st : -fx[j];
                s2 += fx[j] + df;
                D += df * (df - d[q][j]);
            }
        }
        s2 = group_sum<G>(s2);
        D = group_sum<G>(D);
        const T over1 = s2 - ue;
        const T psin = over1 > T(0) ? over1 : T(0);
        const T dz = T(0.5) * (psin * psin - psi * psi) + D;
        const bool accept = dz <= T(0);  // identical in every lane of the group
        T rs = T(0);
#pragma unroll
        for (int q = 0; q < V; ++q) {
            const int v = gl + q * G;
            const bool live = valid && v < vpr;
            T fx[N], vin[N], o[N], vo[N];
            if (live) unpack(__ldg(frow + v), fx);
            else
#pragma unroll
                for (int j = 0; j < N; ++j) fx[j] = T(0);
            if (M && live) unpack(__ldg(reinterpret_cast<const VT*>(a.v_in + row) + v), vin);
#pragma unroll
            for (int j = 0; j < N; ++j) {
                const T st = beta * (d[q][j] - psi);
                const T df = st > -fx[j] ? st : -fx[j];
                if constexpr (M) {
                    const T vv = live ? vin[j] : T(0);
                    vo[j] = accept ? a.gamma * vv + df : vv;
                    const T x = fx[j] + vo[j];
                    o[j] = accept ? (x > T(0) ? x : T(0)) : fx[j];
                } else {
                    o[j] = accept ? fx[j] + df : fx[j];
                }
                rs += o[j];
            }
            if (live) {
                reinterpret_cast<VT*>(a.f_out + row)[v] = pack4(o);
                if (M) reinterpret_cast<VT*>(a.v_out + row)[v] = pack4(vo);
            }
        }
        rs = group_sum<G>(rs);
        if (valid && gl == 0) {
            a.beta_out[e] = new_beta(a, beta, accept, grow);
            const T over = rs - ue;
            const T p = over > T(0) ? over : T(0);
            zpsi = A::add(zpsi, p * p);
            const T c = p * a.inv_scale_t[e];
            capmax = c > capmax ? c : capmax;
        }
    }
    warp_acc_max<T>(zpsi, capmax);
    if (lane == 0) {
        reinterpret_cast<typename A::S*>(a.part_psi)[warp] = A::store(zpsi);
        a.part_cap[warp] = capmax;
    }
}

// One block of B threads per edge (large K); thread l holds row vectors l + q*B.
template <typename T, int B, int V, bool M>
__global__ void __launch_bounds__(B, gd_min_blocks(B, V)) gd_block_kernel(SweepArgs<T> a)
{
    using VT = typename VecOf<T>::type;
    using A = Acc<T>;
    constexpr int N = VecOf<T>::N;
    __shared__ T sa_buf[33];
    __shared__ int sb_buf[33];
    __shared__ T sc_buf[33];
    volatile DevState* vst = a.st;
    if (sweep_stopped(a)) return;  // an earlier sweep of this solve stopped
    if (blockIdx.x == gridDim.x - 1) {
        if (a.mode != MODE_PSI) reduce_and_finalize(a);
        return;
    }
    if (final_evaluation(a)) return;  // the sweep cap stops this sweep: its output is not used
    const bool grow = (vst->t_sweep % 10) == 0;
    const int vpr = a.Kp / N;
    typename A::V zpsi = A::zero();
    T capmax = T(0);
    int dummy = 0;
    for (int64_t e = blockIdx.x; e < a.m; e += gridDim.x - 1) {
        const T ue = a.u[e];
        const T beta = a.beta_in[e];
        const int64_t row = e * a.Kp;
        const VT* hi = reinterpret_cast<const VT*>(a.h + (int64_t)a.src[e] * a.Kp);
        const VT* hj = reinterpret_cast<const VT*>(a.h + (int64_t)a.col[e] * a.Kp);
        const VT* frow = reinterpret_cast<const VT*>(a.f + row);
        T d[V][N];
        T fs = T(0);
#pragma unroll
        for (int q = 0; q < V; ++q) {
            const int v = threadIdx.x + q * B;
            if (v < vpr) {
                T fx[N], ax[N], bx[N];
                unpack(__ldg(frow + v), fx);
                unpack(__ldg(hi + v), ax);
                unpack(__ldg(hj + v), bx);
#pragma unroll
                for (int j = 0; j < N; ++j) {
                    d[q][j] = ax[j] - bx[j];
                    fs += fx[j];
                }
            } else {
#pragma unroll
                for (int j = 0; j < N; ++j) d[q][j] = T(0);
            }
        }
        block_sum2(fs, dummy, sa_buf, sb_buf);
        const T over0 = fs - ue;
        const T psi = over0 > T(0) ? over0 : T(0);
        T s2 = T(0), D = T(0);
#pragma unroll
        for (int q = 0; q < V; ++q) {
            const int v = threadIdx.x + q * B;
            T fx[N];
            if (v < vpr) unpack(__ldg(frow + v), fx);
            else
#pragma unroll
                for (int j = 0; j < N; ++j) fx[j] = T(0);
#pragma unroll
            for (int j = 0; j < N; ++j) {
                const T st = beta * (d[q][j] - psi);
                const T df = st > -fx[j] ? st : -fx[j];
                s2 += fx[j] + df;
                D += df * (df - d[q][j]);
            }
        }
        block_sum_pair(s2, D, sa_buf, sc_buf);
        const T over1 = s2 - ue;
        const T psin = over1 > T(0) ? over1 : T(0);
        const T dz = T(0.5) * (psin * psin - psi * psi) + D;
        const bool accept = dz <= T(0);  // block-uniform
        T rs = T(0);
#pragma unroll
        for (int q = 0; q < V; ++q) {
            const int v = threadIdx.x + q * B;
            const bool live = v < vpr;
            T fx[N], vin[N], o[N], vo[N];
            if (live) unpack(__ldg(frow + v), fx);
            else
#pragma unroll
                for (int j = 0; j < N; ++j) fx[j] = T(0);
            if (M && live) unpack(__ldg(reinterpret_cast<const VT*>(a.v_in + row) + v), vin);
#pragma unroll
            for (int j = 0; j < N; ++j) {
                const T st = beta * (d[q][j] - psi);
                const T df = st > -fx[j] ? st : -fx[j];
                if constexpr (M) {
                    const T vv = live ? vin[j] : T(0);
                    vo[j] = accept ? a.gamma * vv + df : vv;
                    const T x = fx[j] + vo[j];
                    o[j] = accept ? (x > T(0) ? x : T(0)) : fx[j];
                } else {
                    o[j] = accept ? fx[j] + df : fx[j];
                }
                rs += o[j];
            }
            if (live) {
                reinterpret_cast<VT*>(a.f_out + row)[v] = pack4(o);
                if (M) reinterpret_cast<VT*>(a.v_out + row)[v] = pack4(vo);
            }
        }
        // Alg. 3 stores f + df (accepted) or f (rejected), whose sums s2 and
        // fs were formed above in this very order; Alg. 4 re-sums its row
        if constexpr (M) block_sum2(rs, dummy, sa_buf, sb_buf);
        else rs = accept ? s2 : fs;
        if (threadIdx.x == 0) {
            a.beta_out[e] = new_beta(a, beta, accept, grow);
            const T over = rs - ue;
            const T p = over > T(0) ? over : T(0);
            zpsi = A::add(zpsi, p * p);
            const T c = p * a.inv_scale_t[e];
            capmax = c > capmax ? c : capmax;
        }
    }
    if (threadIdx.x == 0) {
        reinterpret_cast<typename A::S*>(a.part_psi)[blockIdx.x] = A::store(zpsi);
        a.part_cap[blockIdx.x] = capmax;
    }
}

}  // namespace

// Same variant table as the edge-QP kernels (sweep.cu: kCfg); a pipelined
// variant runs the plain form of the same capacity (the kernels stride over
// the edges, so any grid works).
template <typename T, bool M>
cudaError_t launch_gd_m(const SweepArgs<T>& a, int cfg, cudaStream_t stream)
{
    const int g = a.grid_e + 1;
    switch (edge_plain_config(cfg)) {
    case 0: gd_group_kernel<T, 4, 1, M><<<g, kThreads, 0, stream>>>(a); break;
    case 1: gd_group_kernel<T, 8, 1, M><<<g, kThreads, 0, stream>>>(a); break;
    case 2: gd_group_kernel<T, 16, 1, M><<<g, kThreads, 0, stream>>>(a); break;
    case 3: gd_group_kernel<T, 32, 1, M><<<g, kThreads, 0, stream>>>(a); break;
    case 4: gd_group_kernel<T, 32, 2, M><<<g, kThreads, 0, stream>>>(a); break;
    case 5: gd_group_kernel<T, 32, 4, M><<<g, kThreads, 0, stream>>>(a); break;
    case 6: gd_group_kernel<T, 32, 8, M><<<g, kThreads, 0, stream>>>(a); break;
    case 7: gd_block_kernel<T, 128, 4, M><<<g, 128, 0, stream>>>(a); break;
    case 8: gd_block_kernel<T, 256, 2, M><<<g, 256, 0, stream>>>(a); break;
    case 9: gd_block_kernel<T, 512, 2, M><<<g, 512, 0, stream>>>(a); break;
    case 10: gd_block_kernel<T, 512, 3, M><<<g, 512, 0, stream>>>(a); break;
    case 11: gd_block_kernel<T, 512, 4, M><<<g, 512, 0, stream>>>(a); break;
    case 12: gd_block_kernel<T, 512, 5, M><<<g, 512, 0, stream>>>(a); break;
    case 13: gd_block_kernel<T, 256, 10, M><<<g, 256, 0, stream>>>(a); break;
    case 14: gd_block_kernel<T, 512, 8, M><<<g, 512, 0, stream>>>(a); break;
    case 15: gd_block_kernel<T, 1024, 8, M><<<g, 1024, 0, stream>>>(a); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// Same variant table as the edge-QP kernels (sweep.cu: kCfg); a pipelined
// variant runs the plain form of the same capacity (the kernels stride over
// the edges, so any grid works).  Alg. 3 and Alg. 4 are compiled apart, so
// that Alg. 3 carries no velocity registers.
template <typename T>
cudaError_t launch_gd(const SweepArgs<T>& a, int cfg, cudaStream_t stream)
{
    return a.momentum ? launch_gd_m<T, true>(a, cfg, stream) : launch_gd_m<T, false>(a, cfg, stream);
}

template cudaError_t launch_gd<float>(const SweepArgs<float>&, int, cudaStream_t);
template cudaError_t launch_gd<double>(const SweepArgs<double>&, int, cudaStream_t);

}  // namespace pdr
