// residuals.cu -- eq. (1) residuals, objective and infeasibility certificate
// of the stored flows, all accumulated in FP64 whatever the working
// precision of the flows.
//
//  vertex pass  Delta_ik (eq. (3), (3h)) and h_ik = Delta_ik / delta_i
//               (eq. (2)) in FP64 (FP32 flows summed error-free in FP32
//               pairs first); per block: sum delta h^2, max |Delta|,
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

// Exact error of one addition (Knuth's TwoSum): a + b = s + e exactly.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// Running sum of FP32 terms kept as an unevaluated pair (hi + lo): every
// addition is error-free (TwoSum) and only the small error terms are added
// in FP32, so hi + lo is the exact sum to about 2^-45 of the largest partial
// sum, well inside FP64 rounding of the quantities formed from it.
struct PairSum {
    float hi = 0.f, lo = 0.f;
    __device__ __forceinline__ void add(float x)
    {
        float e;
        two_sum(hi, x, hi, e);
        lo = __fadd_rn(lo, e);
    }
    __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

// Four consecutive elements of a padded row as doubles.
__device__ __forceinline__ void load4(const double* p, double* x)
{
    const double2 a = __ldg(reinterpret_cast<const double2*>(p));
    const double2 b = __ldg(reinterpret_cast<const double2*>(p) + 1);
    x[0] = a.x, x[1] = a.y, x[2] = b.x, x[3] = b.y;
}

// The largest |Delta_ik| and |Delta_ik| / d_k are found in FP64 without an
// FP64 division per element: an element goes through the exact FP64 path
// only when its FP32 estimate (relative error below 2^-21) comes within
// 2^-18 of the FP32 estimate of the best exact value so far, so no element
// that could be the maximum is skipped.
constexpr float kSlack = 0.99999619f;  // 1 - 2^-18

// Vertex pass: one warp per vertex, each lane four commodities at a time.
// Delta_ik = sum over in-edges (ascending id) - sum over out-edges
// (ascending) + the source/sink term (eq. (3), (3h)); h = Delta / delta_i
// (eq. (2)).  FP32 flows are summed error-free (PairSum), FP64 flows in FP64.
template <typename T>
__global__ void __launch_bounds__(256) resid_vertex_kernel(SweepArgs<T> a, ResidIn r, double* __restrict__ h64,
                                                           double* __restrict__ part)
{
    __shared__ double smem[5][32];
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int nvec = a.Kp / 4;
    double zsum = 0.0, cabs = 0.0, crel = 0.0;
    float cabs32 = 0.f, crel32 = 0.f;  // FP32 estimates of the elements behind cabs, crel
    for (int64_t i = warp; i < a.n; i += nwarps) {
        const int64_t i0 = a.in_ptr[i], i1 = a.in_ptr[i + 1], o0 = a.row_ptr[i], o1 = a.row_ptr[i + 1];
        const double invdeg = r.inv_deg_d[i];
        for (int v = lane; v < nvec; v += 32) {
            const int k0 = 4 * v;
            double D[4];
            float D32[4];
            if constexpr (sizeof(T) == 4) {
                PairSum acc[4];
                for (int64_t q = i0; q < i1; ++q) {
                    const float4 x = __ldg(reinterpret_cast<const float4*>(a.f + (int64_t)a.in_eid[q] * a.Kp + k0));
                    acc[0].add(x.x), acc[1].add(x.y), acc[2].add(x.z), acc[3].add(x.w);
                }
                for (int64_t e = o0; e < o1; ++e) {
                    const float4 x = __ldg(reinterpret_cast<const float4*>(a.f + e * a.Kp + k0));
                    acc[0].add(-x.x), acc[1].add(-x.y), acc[2].add(-x.z), acc[3].add(-x.w);
                }
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    D[j] = acc[j].value();
                    D32[j] = __fadd_rn(acc[j].hi, acc[j].lo);
                }
            } else {
#pragma unroll
                for (int j = 0; j < 4; ++j) D[j] = 0.0;
                double x[4];
                for (int64_t q = i0; q < i1; ++q) {
                    load4(reinterpret_cast<const double*>(a.f) + (int64_t)a.in_eid[q] * a.Kp + k0, x);
#pragma unroll
                    for (int j = 0; j < 4; ++j) D[j] += x[j];
                }
                for (int64_t e = o0; e < o1; ++e) {
                    load4(reinterpret_cast<const double*>(a.f) + e * a.Kp + k0, x);
#pragma unroll
                    for (int j = 0; j < 4; ++j) D[j] -= x[j];
                }
#pragma unroll
                for (int j = 0; j < 4; ++j) D32[j] = (float)D[j];
            }
            const int4 sv = __ldg(reinterpret_cast<const int4*>(a.s + k0));
            const int4 tv = __ldg(reinterpret_cast<const int4*>(a.t + k0));
            const int ss[4] = {sv.x, sv.y, sv.z, sv.w}, tt[4] = {tv.x, tv.y, tv.z, tv.w};
            double h[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int k = k0 + j;
                if (k >= a.K) D[j] = 0.0;  // the padding carries no commodity
                if (ss[j] == (int)i || tt[j] == (int)i) {  // padding has s = t = -1
                    D[j] += ss[j] == (int)i ? r.dem_d[k] : -r.dem_d[k];
                    D32[j] = (float)D[j];
                }
                h[j] = D[j] * invdeg;
                zsum = fma(D[j], h[j], zsum);  // delta_i h^2 = Delta h
                if (D[j] != 0.0) {
                    const float ad = fabsf(D32[j]);
                    if (ad >= cabs32 * kSlack) {
                        cabs = fmax(cabs, fabs(D[j]));
                        cabs32 = fmaxf(cabs32, ad);
                    }
                    const float rel = ad * r.inv_dem_f[k];
                    if (rel >= crel32 * kSlack) {
                        crel = fmax(crel, fabs(D[j]) / r.dem_d[k]);
                        crel32 = fmaxf(crel32, rel);
                    }
                }
            }
            double2* hp = reinterpret_cast<double2*>(h64 + i * a.Kp + k0);
            hp[0] = make_double2(h[0], h[1]);
            hp[1] = make_double2(h[2], h[3]);
        }
    }
    double v[3] = {zsum, cabs, crel};
    const int op[3] = {0, 1, 1};
    block_reduce<3>(v, op, smem);
    if (threadIdx.x == 0)
        for (int q = 0; q < kVParts; ++q) part[(int64_t)blockIdx.x * kVParts + q] = v[q];
}

// Edge pass: one warp per edge, each lane four commodities at a time:
// sum_k f_e,k (error-free pairs for FP32 flows), psi_e (eq. (41)), min_k f_e,k
// and the certificate length l_e = max(0, max_k (h_ik - h_jk)) in FP64 (only
// where u_e > 0: an edge without capacity adds nothing to sum_e u_e l_e).
template <typename T>
__global__ void __launch_bounds__(256) resid_edge_kernel(SweepArgs<T> a, ResidIn r, const double* __restrict__ h64,
                                                         double* __restrict__ part)
{
    __shared__ double smem[5][32];
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int nvec = a.Kp / 4;
    double psi2 = 0.0, capa = 0.0, capr = 0.0, cost = 0.0, fmn = INFINITY;
    for (int64_t e = warp; e < a.m; e += nwarps) {
        const double ue = r.u_d[e];
        const bool need_l = ue > 0.0;
        const double* hi = h64 + (int64_t)a.src[e] * a.Kp;
        const double* hj = h64 + (int64_t)a.col[e] * a.Kp;
        double tot = 0.0, l = 0.0, mn = INFINITY;
        if constexpr (sizeof(T) == 4) {
            PairSum acc;
            float mn32 = INFINITY;
            for (int v = lane; v < nvec; v += 32) {
                const int k0 = 4 * v;
                const float4 x = __ldg(reinterpret_cast<const float4*>(a.f + e * a.Kp + k0));
                const float xs[4] = {x.x, x.y, x.z, x.w};
                const int nk = a.K - k0 < 4 ? a.K - k0 : 4;  // the padding carries no commodity
                for (int j = 0; j < nk; ++j) {
                    acc.add(xs[j]);
                    mn32 = fminf(mn32, xs[j]);
                }
                if (need_l) {
                    double p[4], q[4];
                    load4(hi + k0, p);
                    load4(hj + k0, q);
                    for (int j = 0; j < nk; ++j) l = fmax(l, p[j] - q[j]);
                }
            }
            tot = (double)acc.hi + (double)acc.lo;
            mn = (double)mn32;
        } else {
            for (int v = lane; v < nvec; v += 32) {
                const int k0 = 4 * v;
                double x[4];
                load4(reinterpret_cast<const double*>(a.f) + e * a.Kp + k0, x);
                const int nk = a.K - k0 < 4 ? a.K - k0 : 4;  // the padding carries no commodity
                for (int j = 0; j < nk; ++j) {
                    tot += x[j];
                    mn = fmin(mn, x[j]);
                }
                if (need_l) {
                    double p[4], q[4];
                    load4(hi + k0, p);
                    load4(hj + k0, q);
                    for (int j = 0; j < nk; ++j) l = fmax(l, p[j] - q[j]);
                }
            }
        }
        tot = wsum(tot);
        l = wmax(l);
        mn = wmin(mn);
        if (lane == 0) {
            const double over = tot - ue;
            const double psi = over > 0.0 ? over : 0.0;
            psi2 += psi * psi;
            capa = fmax(capa, psi);
            capr = fmax(capr, psi * a.inv_scale[e]);
            cost += ue * l;
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
cudaError_t launch_residuals(const SweepArgs<T>& a, const ResidIn& r, double* h64, double* part, int32_t grid_v,
                             int32_t grid_e, ResidOut* out, cudaStream_t stream)
{
    resid_vertex_kernel<T><<<grid_v, 256, 0, stream>>>(a, r, h64, part);
    resid_edge_kernel<T><<<grid_e, 256, 0, stream>>>(a, r, h64, part + (int64_t)grid_v * kVParts);
    resid_final_kernel<T><<<1, 256, 0, stream>>>(a, r.dem_d, h64, part, grid_v, grid_e, out);
    return cudaGetLastError();
}

template cudaError_t launch_residuals<float>(const SweepArgs<float>&, const ResidIn&, double*, double*, int32_t,
                                             int32_t, ResidOut*, cudaStream_t);
template cudaError_t launch_residuals<double>(const SweepArgs<double>&, const ResidIn&, double*, double*, int32_t,
                                              int32_t, ResidOut*, cudaStream_t);

}  // namespace pdr
