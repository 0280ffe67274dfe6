// residuals.cu -- eq. (1) residuals, objective and infeasibility certificate
// of the stored flows, all accumulated in FP64 whatever the working
// precision of the flows.
//
//  vertex pass  Delta_ik (eq. (3), (3h)) and h_ik = Delta_ik / delta_i
//               (eq. (2)) in FP64; per block: sum delta h^2, max |Delta|,
//               max |Delta| / d_k.
//  edge pass    sum_k f_e,k, psi_e (eq. (41)), the certificate length
//               l_e = max(0, max_k (h_ik - h_jk)) and min_k f_e,k; per block:
//               sum psi^2, max psi, max psi/scale, sum u_e l_e, min f.
//  final pass   one block: gain = sum_k d_k (h_{s_k,k} - h_{t_k,k}), the
//               reduction of every partial in a fixed order, and
//               margin = gain - sum_e u_e l_e.
//
// Certificate (Theorems 1 and 2, made explicit by Farkas' lemma): with
// potentials pi = h and lengths l >= 0 with pi_ik - pi_jk <= l_e on every
// edge, any feasible flow satisfies
//   sum_k d_k (pi_{s_k,k} - pi_{t_k,k}) = sum_{e,k} f_e,k (pi_ik - pi_jk)
//                                      <= sum_e l_e sum_k f_e,k <= sum_e u_e l_e,
// so margin > 0 proves that eq. (1) has no solution.
#include "pdr_internal.cuh"

#include <math.h>

namespace pdr {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kVParts = 3;  // per vertex block: zsum, cons_abs, cons_rel
constexpr int kEParts = 5;  // per edge block: psi2, cap_abs, cap_rel, cost, fmin

__device__ __forceinline__ double wsum(double x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
    return x;
}
__device__ __forceinline__ double wmax(double x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x = fmax(x, __shfl_xor_sync(kFull, x, o));
    return x;
}
__device__ __forceinline__ double wmin(double x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x = fmin(x, __shfl_xor_sync(kFull, x, o));
    return x;
}

// Block reduction of up to 5 values with per-slot operations (0 sum, 1 max,
// 2 min); the results are valid in thread 0.
template <int NV>
__device__ void block_reduce(double* v, const int* op, double (*smem)[32])
{
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        v[q] = op[q] == 0 ? wsum(v[q]) : op[q] == 1 ? wmax(v[q]) : wmin(v[q]);
        if (l == 0) smem[q][w] = v[q];
    }
    __syncthreads();
    if (w == 0) {
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            const double idn = op[q] == 2 ? INFINITY : 0.0;
            double x = l < nw ? smem[q][l] : idn;
            v[q] = op[q] == 0 ? wsum(x) : op[q] == 1 ? wmax(x) : wmin(x);
        }
    }
    __syncthreads();
}

template <typename T>
__global__ void __launch_bounds__(256) resid_vertex_kernel(SweepArgs<T> a, const double* __restrict__ dem_d,
                                                           double* __restrict__ h64, double* __restrict__ part)
{
    __shared__ double smem[5][32];
    double zsum = 0.0, cabs = 0.0, crel = 0.0;
    const int64_t total = (int64_t)a.n * a.K;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int32_t i = (int32_t)(idx / a.K);
        const int32_t k = (int32_t)(idx - (int64_t)i * a.K);
        double acc = 0.0;
        for (int64_t q = a.in_ptr[i]; q < a.in_ptr[i + 1]; ++q) acc += (double)a.f[(int64_t)a.in_eid[q] * a.Kp + k];
        for (int64_t e = a.row_ptr[i]; e < a.row_ptr[i + 1]; ++e) acc -= (double)a.f[e * a.Kp + k];
        if (a.s[k] == i) acc += dem_d[k];
        else if (a.t[k] == i) acc -= dem_d[k];
        const int dg = a.deg[i];
        const double h = dg > 0 ? acc / (double)dg : 0.0;
        h64[(int64_t)i * a.Kp + k] = h;
        zsum += (double)dg * h * h;
        cabs = fmax(cabs, fabs(acc));
        crel = fmax(crel, fabs(acc) / dem_d[k]);
    }
    double v[3] = {zsum, cabs, crel};
    const int op[3] = {0, 1, 1};
    block_reduce<3>(v, op, smem);
    if (threadIdx.x == 0)
        for (int q = 0; q < kVParts; ++q) part[(int64_t)blockIdx.x * kVParts + q] = v[q];
}

// One warp per edge.
template <typename T>
__global__ void __launch_bounds__(256) resid_edge_kernel(SweepArgs<T> a, const double* __restrict__ u_d,
                                                         const double* __restrict__ h64, double* __restrict__ part)
{
    __shared__ double smem[5][32];
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    double psi2 = 0.0, capa = 0.0, capr = 0.0, cost = 0.0, fmn = INFINITY;
    for (int64_t e = warp; e < a.m; e += nwarps) {
        const T* fr = a.f + e * a.Kp;
        const double* hi = h64 + (int64_t)a.src[e] * a.Kp;
        const double* hj = h64 + (int64_t)a.col[e] * a.Kp;
        double tot = 0.0, l = 0.0, mn = INFINITY;
        for (int k = lane; k < a.K; k += 32) {
            const double x = (double)fr[k];
            tot += x;
            mn = fmin(mn, x);
            l = fmax(l, hi[k] - hj[k]);
        }
        tot = wsum(tot);
        l = wmax(l);
        mn = wmin(mn);
        if (lane == 0) {
            const double over = tot - u_d[e];
            const double psi = over > 0.0 ? over : 0.0;
            psi2 += psi * psi;
            capa = fmax(capa, psi);
            capr = fmax(capr, psi * a.inv_scale[e]);
            cost += u_d[e] * l;
            fmn = fmin(fmn, mn);
        }
    }
    double v[5] = {psi2, capa, capr, cost, fmn};
    const int op[5] = {0, 1, 1, 0, 2};
    block_reduce<5>(v, op, smem);
    if (threadIdx.x == 0)
        for (int q = 0; q < kEParts; ++q) part[(int64_t)blockIdx.x * kEParts + q] = v[q];
}

template <typename T>
__global__ void __launch_bounds__(256) resid_final_kernel(SweepArgs<T> a, const double* __restrict__ dem_d,
                                                          const double* __restrict__ h64,
                                                          const double* __restrict__ part, int32_t grid_v,
                                                          int32_t grid_e, ResidOut* __restrict__ out)
{
    __shared__ double smem[5][32];
    double gain = 0.0, gabs = 0.0;
    for (int k = threadIdx.x; k < a.K; k += blockDim.x) {
        const double diff = h64[(int64_t)a.s[k] * a.Kp + k] - h64[(int64_t)a.t[k] * a.Kp + k];
        gain += dem_d[k] * diff;
        gabs += dem_d[k] * fabs(diff);
    }
    double zv = 0.0, cabs = 0.0, crel = 0.0;
    for (int b = threadIdx.x; b < grid_v; b += blockDim.x) {
        zv += part[(int64_t)b * kVParts + 0];
        cabs = fmax(cabs, part[(int64_t)b * kVParts + 1]);
        crel = fmax(crel, part[(int64_t)b * kVParts + 2]);
    }
    const double* pe = part + (int64_t)grid_v * kVParts;
    double psi2 = 0.0, capa = 0.0, capr = 0.0, cost = 0.0, fmn = INFINITY;
    for (int b = threadIdx.x; b < grid_e; b += blockDim.x) {
        psi2 += pe[(int64_t)b * kEParts + 0];
        capa = fmax(capa, pe[(int64_t)b * kEParts + 1]);
        capr = fmax(capr, pe[(int64_t)b * kEParts + 2]);
        cost += pe[(int64_t)b * kEParts + 3];
        fmn = fmin(fmn, pe[(int64_t)b * kEParts + 4]);
    }
    double v1[5] = {gain, gabs, zv, cabs, crel};
    const int op1[5] = {0, 0, 0, 1, 1};
    block_reduce<5>(v1, op1, smem);
    double v2[5] = {psi2, capa, capr, cost, fmn};
    const int op2[5] = {0, 1, 1, 0, 2};
    block_reduce<5>(v2, op2, smem);
    if (threadIdx.x == 0) {
        out->z = 0.5 * (v2[0] + v1[2]);
        out->cap_abs = v2[1];
        out->cap_rel = v2[2];
        out->cons_abs = v1[3];
        out->cons_rel = v1[4];
        out->f_min = a.m > 0 ? v2[4] : 0.0;
        out->margin = v1[0] - v2[3];
        out->margin_scale = v1[1] + v2[3];
    }
}

}  // namespace

int resid_part_count(int32_t grid_v, int32_t grid_e) { return grid_v * kVParts + grid_e * kEParts; }

template <typename T>
cudaError_t launch_residuals(const SweepArgs<T>& a, const double* u_d, const double* dem_d, double* h64,
                             double* part, int32_t grid_v, int32_t grid_e, ResidOut* out, cudaStream_t stream)
{
    resid_vertex_kernel<T><<<grid_v, 256, 0, stream>>>(a, dem_d, h64, part);
    resid_edge_kernel<T><<<grid_e, 256, 0, stream>>>(a, u_d, h64, part + (int64_t)grid_v * kVParts);
    resid_final_kernel<T><<<1, 256, 0, stream>>>(a, dem_d, h64, part, grid_v, grid_e, out);
    return cudaGetLastError();
}

template cudaError_t launch_residuals<float>(const SweepArgs<float>&, const double*, const double*, double*,
                                             double*, int32_t, int32_t, ResidOut*, cudaStream_t);
template cudaError_t launch_residuals<double>(const SweepArgs<double>&, const double*, const double*, double*,
                                              double*, int32_t, int32_t, ResidOut*, cudaStream_t);

}  // namespace pdr
