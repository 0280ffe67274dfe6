// adjacency.cu -- device construction of the graph notation of Table
// "Notation": the tail of every edge, delta-(i) as an in-adjacency list
// (edge ids entering i in ascending order), the incidence list of every
// vertex (in-edges, then out-edges) and delta_i = out-degree + in-degree.
//
// The in-adjacency is a counting sort of the edges by head.  Integer atomics
// place the edges in their buckets in arbitrary order; each bucket is then
// sorted by edge id, so the result is unique and bit-identical from run to
// run (edge ids within a bucket are distinct).
#include "pdr_internal.cuh"

namespace pdr {
namespace {

constexpr int kScanThreads = 1024;

__global__ void tail_kernel(int32_t n, const int64_t* __restrict__ row_ptr, int32_t* __restrict__ src)
{
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) src[e] = i;
}

__global__ void count_kernel(int64_t m, const int32_t* __restrict__ col, unsigned long long* __restrict__ cnt)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(cnt + col[e], 1ull);
}

// Single block: exclusive scan of the in-degree counts into in_ptr, the fill
// cursor, and the vertex degrees.
__global__ void __launch_bounds__(kScanThreads)
    scan_kernel(int32_t n, const int64_t* __restrict__ row_ptr, const unsigned long long* __restrict__ cnt,
                int64_t* __restrict__ in_ptr, long long* __restrict__ cursor, int32_t* __restrict__ deg)
{
    __shared__ long long part[kScanThreads];
    const int tid = threadIdx.x;
    const int64_t chunk = ((int64_t)n + kScanThreads - 1) / kScanThreads;
    const int64_t lo = tid * chunk;
    const int64_t hi = lo + chunk < n ? lo + chunk : n;
    long long local = 0;
    for (int64_t i = lo; i < hi; ++i) local += (long long)cnt[i];
    part[tid] = local;
    __syncthreads();
    // Hillis-Steele inclusive scan over the per-thread totals
    for (int off = 1; off < kScanThreads; off <<= 1) {
        long long v = tid >= off ? part[tid - off] : 0;
        __syncthreads();
        part[tid] += v;
        __syncthreads();
    }
    long long run = part[tid] - local;  // exclusive prefix of this chunk
    for (int64_t i = lo; i < hi; ++i) {
        in_ptr[i] = run;
        cursor[i] = run;
        deg[i] = (int32_t)((row_ptr[i + 1] - row_ptr[i]) + (long long)cnt[i]);
        run += (long long)cnt[i];
    }
    if (tid == kScanThreads - 1) in_ptr[n] = part[kScanThreads - 1];
}

__global__ void fill_kernel(int64_t m, const int32_t* __restrict__ col, unsigned long long* __restrict__ cursor,
                            int32_t* __restrict__ in_eid)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long pos = atomicAdd(cursor + col[e], 1ull);
        in_eid[pos] = (int32_t)e;
    }
}

// Sorts each bucket by edge id (insertion sort: buckets are short in sparse
// graphs; a long bucket costs time, never correctness).
__global__ void sort_kernel(int32_t n, const int64_t* __restrict__ in_ptr, int32_t* __restrict__ in_eid)
{
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int64_t lo = in_ptr[i], hi = in_ptr[i + 1];
        for (int64_t a = lo + 1; a < hi; ++a) {
            const int32_t key = in_eid[a];
            int64_t b = a - 1;
            while (b >= lo && in_eid[b] > key) {
                in_eid[b + 1] = in_eid[b];
                --b;
            }
            in_eid[b + 1] = key;
        }
    }
}

// Incidence list of each vertex: in-edges e, then out-edges as ~e.  Its
// offset is in_ptr[i] + row_ptr[i] (the degrees of the vertices before i).
__global__ void incidence_kernel(int32_t n, const int64_t* __restrict__ row_ptr, const int64_t* __restrict__ in_ptr,
                                 const int32_t* __restrict__ in_eid, int64_t* __restrict__ inc_ptr,
                                 int32_t* __restrict__ inc)
{
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        int64_t w = in_ptr[i] + row_ptr[i];
        inc_ptr[i] = w;
        if (i == n - 1) inc_ptr[n] = in_ptr[n] + row_ptr[n];
        for (int64_t q = in_ptr[i]; q < in_ptr[i + 1]; ++q) inc[w++] = in_eid[q];
        for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) inc[w++] = ~(int32_t)e;
    }
}

int blocks_for(int64_t count, int threads)
{
    int64_t b = (count + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > 65535) b = 65535;
    return (int)b;
}

}  // namespace

cudaError_t build_adjacency(int32_t n, int64_t m, const int64_t* row_ptr, const int32_t* col, int32_t* src,
                            int64_t* in_ptr, int32_t* in_eid, int64_t* inc_ptr, int32_t* inc, int32_t* deg,
                            int64_t* work, cudaStream_t stream)
{
    unsigned long long* cnt = reinterpret_cast<unsigned long long*>(work);
    long long* cursor = reinterpret_cast<long long*>(work + n);
    cudaError_t err = cudaMemsetAsync(cnt, 0, sizeof(unsigned long long) * (size_t)n, stream);
    if (err != cudaSuccess) return err;
    tail_kernel<<<blocks_for(n, 256), 256, 0, stream>>>(n, row_ptr, src);
    if (m > 0) count_kernel<<<blocks_for(m, 256), 256, 0, stream>>>(m, col, cnt);
    scan_kernel<<<1, kScanThreads, 0, stream>>>(n, row_ptr, cnt, in_ptr, cursor, deg);
    if (m > 0)
        fill_kernel<<<blocks_for(m, 256), 256, 0, stream>>>(m, col, reinterpret_cast<unsigned long long*>(cursor),
                                                            in_eid);
    sort_kernel<<<blocks_for(n, 128), 128, 0, stream>>>(n, in_ptr, in_eid);
    incidence_kernel<<<blocks_for(n, 128), 128, 0, stream>>>(n, row_ptr, in_ptr, in_eid, inc_ptr, inc);
    return cudaGetLastError();
}

}  // namespace pdr

// ------------------------------------------------------------------ entry point that allocates nothing
//
// pdr_adjacency_static builds the same in-adjacency and degrees as the
// context path above, for a caller that owns the device arrays and cannot
// allocate device memory itself.  Its scratch (in-degree counts, fill
// cursors and an input-error word) is one file-scope device array, so the
// call makes no cudaMalloc or cudaFree.
#include "pdr.h"

#include <string>

namespace pdr {
namespace {

constexpr int64_t kStaticMaxVertices = int64_t(1) << 18;  // 262,144 vertices: 4 MiB of scratch per GPU

// [0, max): in-degree counts; [max, 2 max): fill cursors; [2 max]: input-error word
__device__ __align__(256) unsigned long long g_static_scratch[2 * kStaticMaxVertices + 1];

// Input checks on the device: row_ptr[0] = 0, non-decreasing, row_ptr[n] = m,
// 0 <= col[e] < n.  Sets bits of *err instead of trusting the arrays.
__global__ void static_check_kernel(int32_t n, int64_t m, const int64_t* __restrict__ row_ptr,
                                    const int32_t* __restrict__ col, unsigned long long* __restrict__ err)
{
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    if (tid == 0 && (row_ptr[0] != 0 || row_ptr[n] != m)) atomicOr(err, 1ull);
    for (int64_t i = tid; i < n; i += stride)
        if (row_ptr[i + 1] < row_ptr[i]) atomicOr(err, 2ull);
    for (int64_t e = tid; e < m; e += stride)
        if (col[e] < 0 || col[e] >= n) atomicOr(err, 4ull);
}

}  // namespace
}  // namespace pdr

extern "C" pdr_status pdr_adjacency_static(int32_t n, int64_t m, const int64_t* row_ptr, const int32_t* col,
                                           int64_t* in_ptr, int32_t* in_eid, int32_t* deg, void* stream_)
{
    using namespace pdr;
    set_thread_error("");
    if (n < 1 || n > kStaticMaxVertices) {
        set_thread_error("pdr_adjacency_static: n must satisfy 1 <= n <= " + std::to_string(kStaticMaxVertices) +
                         " (the size of its static scratch)");
        return PDR_ERR_INVALID_ARG;
    }
    if (m < 0 || m > (int64_t)INT32_MAX) {
        set_thread_error("pdr_adjacency_static: m must satisfy 0 <= m < 2^31");
        return PDR_ERR_INVALID_ARG;
    }
    if (!row_ptr || !in_ptr || !deg || (m > 0 && (!col || !in_eid))) {
        set_thread_error("pdr_adjacency_static: NULL array");
        return PDR_ERR_INVALID_ARG;
    }
    cudaStream_t stream = static_cast<cudaStream_t>(stream_);
    // The host-side name of the array is not a device address: ask the
    // runtime for the current device's copy on every call.  The lookup is
    // cheap, and nothing is cached that a cudaDeviceReset could leave stale.
    void* base = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&base, g_static_scratch);
    if (e != cudaSuccess || !base) {
        set_thread_error(std::string("pdr_adjacency_static: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        cudaGetLastError();
        return PDR_ERR_CUDA;
    }
    unsigned long long* cnt = static_cast<unsigned long long*>(base);
    unsigned long long* cursor = cnt + kStaticMaxVertices;
    unsigned long long* err = cnt + 2 * kStaticMaxVertices;
    unsigned long long host_err = 0;
#define CKS(call)                                                                                  \
    do {                                                                                           \
        cudaError_t _e = (call);                                                                   \
        if (_e != cudaSuccess) {                                                                   \
            set_thread_error(std::string("pdr_adjacency_static: " #call ": ") + cudaGetErrorString(_e)); \
            cudaGetLastError();                                                                    \
            return PDR_ERR_CUDA;                                                                   \
        }                                                                                          \
    } while (0)
    // the array keeps the previous call's contents: clear what must start at zero
    CKS(cudaMemsetAsync(err, 0, sizeof(unsigned long long), stream));
    CKS(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long) * (size_t)n, stream));
    static_check_kernel<<<blocks_for(m > n ? m : n, 256), 256, 0, stream>>>(n, m, row_ptr, col, err);
    CKS(cudaGetLastError());
    CKS(cudaMemcpyAsync(&host_err, err, sizeof(host_err), cudaMemcpyDeviceToHost, stream));
    CKS(cudaStreamSynchronize(stream));
    if (host_err) {
        set_thread_error("pdr_adjacency_static: malformed CSR (row_ptr bounds or order, or col out of range)");
        return PDR_ERR_INVALID_ARG;
    }
    if (m > 0) count_kernel<<<blocks_for(m, 256), 256, 0, stream>>>(m, col, cnt);
    scan_kernel<<<1, kScanThreads, 0, stream>>>(n, row_ptr, cnt, in_ptr, reinterpret_cast<long long*>(cursor), deg);
    if (m > 0) fill_kernel<<<blocks_for(m, 256), 256, 0, stream>>>(m, col, cursor, in_eid);
    sort_kernel<<<blocks_for(n, 128), 128, 0, stream>>>(n, in_ptr, in_eid);
    CKS(cudaGetLastError());
    CKS(cudaStreamSynchronize(stream));
#undef CKS
    return PDR_OK;
}
