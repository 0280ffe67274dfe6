// sweep_common.cuh -- device helpers shared by the sweep kernels (sweep.cu)
// and the gradient-step kernels (gd.cu): vector access, lane-group and block
// reductions, the objective accumulators, and the objective reduction / stop
// decision of Alg. 1 (also used unchanged by Alg. 3 and Alg. 4).
#pragma once

#include "pdr_internal.cuh"

#include <math.h>

namespace pdr {
namespace {

constexpr unsigned kFull = 0xffffffffu;

template <typename T>
struct VecOf;
template <>
struct VecOf<float> {
    using type = float4;
    static constexpr int N = 4;
};
template <>
struct VecOf<double> {
    using type = double2;
    static constexpr int N = 2;
};

__device__ __forceinline__ void unpack(const float4& v, float* x)
{
    x[0] = v.x;
    x[1] = v.y;
    x[2] = v.z;
    x[3] = v.w;
}
__device__ __forceinline__ void unpack(const double2& v, double* x)
{
    x[0] = v.x;
    x[1] = v.y;
}
__device__ __forceinline__ float4 pack4(const float* x) { return make_float4(x[0], x[1], x[2], x[3]); }
__device__ __forceinline__ double2 pack4(const double* x) { return make_double2(x[0], x[1]); }

// Programmatic dependent launch: wait until the kernels this grid depends on
// have completed and their writes are visible, and allow the dependent grid
// to be scheduled.  Both are no-ops for a grid launched without PDL.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// L2 prefetch of the `bytes` bytes at p, one 128-byte line per thread and
// round (thread `tid` of `nthreads`).  Only addresses inside the array are
// passed; a prefetch never blocks the thread.
__device__ __forceinline__ void prefetch_l2(const void* p, int64_t bytes, int tid, int nthreads)
{
    const char* c = static_cast<const char*>(p);
    for (int64_t off = (int64_t)tid * 128; off < bytes; off += (int64_t)nthreads * 128)
        asm volatile("prefetch.global.L2 [%0];" ::"l"(c + off));
}

// L2 eviction priority for working sets larger than L2: the flow rows stream
// through the edge kernel once (evict first), so that they do not push out
// the height rows, which every edge at a vertex gathers.  The policy comes
// from createpolicy; loads go through the read-only path.  (Marking the
// heights evict-last instead left such lines behind after a solve and slowed
// the kernels that ran next.)
__device__ __forceinline__ uint64_t l2_evict_first()
{
    uint64_t p;
    asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ float4 ld_hint(const float4* p, uint64_t pol)
{
    float4 v;
    asm("ld.global.nc.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
        : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
        : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ double2 ld_hint(const double2* p, uint64_t pol)
{
    double2 v;
    asm("ld.global.nc.L2::cache_hint.v2.f64 {%0, %1}, [%2], %3;" : "=d"(v.x), "=d"(v.y) : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ void st_hint(float4* p, float4 v, uint64_t pol)
{
    asm volatile("st.global.L2::cache_hint.v4.f32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(p), "f"(v.x), "f"(v.y),
                 "f"(v.z), "f"(v.w), "l"(pol)
                 : "memory");
}
__device__ __forceinline__ void st_hint(double2* p, double2 v, uint64_t pol)
{
    asm volatile("st.global.L2::cache_hint.v2.f64 [%0], {%1, %2}, %3;" ::"l"(p), "d"(v.x), "d"(v.y), "l"(pol)
                 : "memory");
}

// Shared-memory barriers (mbarrier) and bulk global -> shared copies
// (cp.async.bulk, completed on an mbarrier by byte count).  A CTA launched
// without clusters is its own cluster of one, so its shared::cta addresses
// are valid shared::cluster destinations.
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
// makes the initialised barriers visible to the other threads and the async proxy
__device__ __forceinline__ void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_arrive(uint64_t* bar)
{
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_u32(bar))
                 : "memory");
}
// arrival that also announces `bytes` of bulk copies completing on this phase
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(
                     smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Waits for the completion of the phase with the given parity, for at most
// about `limit` clock cycles; false if it ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, long long limit)
{
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > limit) return false;
    return true;
}
// bytes (a multiple of 16) from global src to shared dst, both 16-byte aligned
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

// The same copy with an L2 cache-policy hint (createpolicy) for the source.
__device__ __forceinline__ void bulk_g2s_hint(void* dst, const void* src, uint32_t bytes, uint64_t* bar, uint64_t pol)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(pol)
        : "memory");
}

// Sum over the G lanes of an aligned lane group (xor offsets below G stay
// inside the group).  Every lane of the warp must call it.  IEEE addition is
// commutative, so every lane of the group ends with the same value.
template <int G, typename X>
__device__ __forceinline__ X group_sum(X x)
{
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
    return x;
}

template <typename X>
__device__ __forceinline__ X warp_max(X x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const X y = __shfl_xor_sync(kFull, x, o);
        x = y > x ? y : x;
    }
    return x;
}

// Warp-wide sum, count and minimum, in every lane.  For float the count and
// the minimum take one redux each: the values combined are positive or +inf
// (sums above a threshold w >= 0), so their bit patterns order as unsigned
// integers.
template <typename T>
__device__ __forceinline__ void warp_sum_count_min(T& s, int& n, T& mn)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(kFull, s, o);
    if constexpr (sizeof(T) == 4) {
        n = (int)__reduce_add_sync(kFull, (unsigned)n);
        mn = __uint_as_float(__reduce_min_sync(kFull, __float_as_uint(mn)));
    } else {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            n += __shfl_xor_sync(kFull, n, o);
            const T y = __shfl_xor_sync(kFull, mn, o);
            mn = y < mn ? y : mn;
        }
    }
}

// Block-wide reductions broadcast to every thread.  The warp partials go to
// slots 0..31 of the caller's buffers (33 entries each); warp 0 combines them
// lane-parallel and leaves the totals in slot 32, read by every thread after
// the second barrier.  (The next call writes slots 0..31 before its first
// barrier and slot 32 only after it, so no trailing barrier is needed.)

// Sum of a value and a count.
template <typename T>
__device__ __forceinline__ void block_sum2(T& a, int& b, T* sa, int* sb)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(kFull, a, o);
        b += __shfl_xor_sync(kFull, b, o);
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) {
        sa[w] = a;
        sb[w] = b;
    }
    __syncthreads();
    if (w == 0) {
        const int nw = blockDim.x >> 5;
        T ta = l < nw ? sa[l] : T(0);
        int tb = l < nw ? sb[l] : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            ta += __shfl_xor_sync(kFull, ta, o);
            tb += __shfl_xor_sync(kFull, tb, o);
        }
        if (l == 0) {
            sa[32] = ta;
            sb[32] = tb;
        }
    }
    __syncthreads();
    a = sa[32];
    b = sb[32];
}

// Sums of two values.
template <typename T>
__device__ __forceinline__ void block_sum_pair(T& a, T& b, T* sa, T* sb)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(kFull, a, o);
        b += __shfl_xor_sync(kFull, b, o);
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) {
        sa[w] = a;
        sb[w] = b;
    }
    __syncthreads();
    if (w == 0) {
        const int nw = blockDim.x >> 5;
        T ta = l < nw ? sa[l] : T(0), tb = l < nw ? sb[l] : T(0);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            ta += __shfl_xor_sync(kFull, ta, o);
            tb += __shfl_xor_sync(kFull, tb, o);
        }
        if (l == 0) {
            sa[32] = ta;
            sb[32] = tb;
        }
    }
    __syncthreads();
    a = sa[32];
    b = sb[32];
}

// ------------------------------------------------------------------ objective accumulators
//
// GB300 issues FP64 at a small fraction of its FP32 rate, so the per-element
// sums behind the objective stay off the FP64 pipe in FP32 mode: terms are
// formed in FP32 and summed as an unevaluated pair hi + lo with the
// error-free TwoSum transformation (Knuth; Dekker 1971), which keeps about 44
// significant bits.  Only the cross-block reduction and the stop decision
// run in FP64.  In FP64 mode the accumulator is a plain double.
template <typename T>
struct Acc;

template <>
struct Acc<float> {
    struct V {
        float hi, lo;
    };
    using S = float2;  // stored form
    static __device__ __forceinline__ V zero() { return {0.f, 0.f}; }
    static __device__ __forceinline__ V add(V a, V b)
    {
        const float s = a.hi + b.hi;
        const float bb = s - a.hi;
        const float e = ((a.hi - (s - bb)) + (b.hi - bb)) + (a.lo + b.lo);
        const float hi = s + e;
        return {hi, e - (hi - s)};
    }
    static __device__ __forceinline__ V add(V a, float b) { return add(a, V{b, 0.f}); }
    static __device__ __forceinline__ V shfl(V a, int o)
    {
        return {__shfl_xor_sync(kFull, a.hi, o), __shfl_xor_sync(kFull, a.lo, o)};
    }
    static __device__ __forceinline__ S store(V a) { return make_float2(a.hi, a.lo); }
    static __device__ __forceinline__ V load(const S* p) { const float2 x = __ldcg(p); return {x.x, x.y}; }
    static __device__ __forceinline__ V unstore(S x) { return {x.x, x.y}; }
    static __device__ __forceinline__ bool nonzero(V a) { return a.hi != 0.f || a.lo != 0.f; }
    static __device__ __forceinline__ double to_double(V a) { return (double)a.hi + (double)a.lo; }
};

template <>
struct Acc<double> {
    using V = double;
    using S = double;
    static __device__ __forceinline__ V zero() { return 0.0; }
    static __device__ __forceinline__ V add(V a, V b) { return a + b; }
    static __device__ __forceinline__ V shfl(V a, int o) { return __shfl_xor_sync(kFull, a, o); }
    static __device__ __forceinline__ S store(V a) { return a; }
    static __device__ __forceinline__ V load(const S* p) { return __ldcg(p); }
    static __device__ __forceinline__ V unstore(S x) { return x; }
    static __device__ __forceinline__ bool nonzero(V a) { return a != 0.0; }
    static __device__ __forceinline__ double to_double(V a) { return a; }
};

// Zero sums and maxima.  The terms reduced below are sums of squares and
// maxima of non-negative values, and an accumulator pair is normalised
// (hi = hi + lo rounded), so adding a zero pair, or taking the maximum with
// zero, returns the other operand unchanged: a warp whose values are all
// zero skips its reduction, and the block reduction skips such warps,
// without changing any finite result.  (NaN counts as nonzero; an
// accumulator that overflowed stops the solve as non-finite either way.)
template <typename T>
__device__ __forceinline__ bool acc_max_nonzero(typename Acc<T>::V z, T m)
{
    return Acc<T>::nonzero(z) || m != T(0);
}

// Warp reduction of (sum, max): the result is valid in lane 0 (lane 0 always
// combines in the same order, so it is deterministic).
template <typename T>
__device__ __forceinline__ void warp_acc_max(typename Acc<T>::V& z, T& mx)
{
    if (!__any_sync(kFull, acc_max_nonzero<T>(z, mx))) return;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) z = Acc<T>::add(z, Acc<T>::shfl(z, o));
    mx = warp_max(mx);
}

// Block reduction of (sum, max, max); the result is valid in thread 0, which
// adds the warps' results in warp order (the all-zero warps left out).
template <typename T>
__device__ void block_acc_max2(typename Acc<T>::V& z, T& m1, T& m2)
{
    using V = typename Acc<T>::V;
    __shared__ V sz[32];
    __shared__ T s1[32], s2[32];
    if (__any_sync(kFull, acc_max_nonzero<T>(z, m1) || m2 != T(0))) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) z = Acc<T>::add(z, Acc<T>::shfl(z, o));
        m1 = warp_max(m1);
        m2 = warp_max(m2);
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) {
        sz[w] = z;
        s1[w] = m1;
        s2[w] = m2;
    }
    __syncthreads();
    if (w == 0) {
        const int nw = blockDim.x >> 5;
        const bool nz = l < nw && (acc_max_nonzero<T>(sz[l], s1[l]) || s2[l] != T(0));
        const unsigned live = __ballot_sync(kFull, nz);
        if (l == 0)
            for (unsigned b = live & ~1u; b; b &= b - 1) {
                const int q = __ffs(b) - 1;
                z = Acc<T>::add(z, sz[q]);
                m1 = s1[q] > m1 ? s1[q] : m1;
                m2 = s2[q] > m2 ? s2[q] : m2;
            }
    }
}

// ------------------------------------------------------------------ objective and stop rules

// True if an earlier sweep of this solve has stopped; the kernel then does
// nothing.  Thread 0 reads the flag once for the whole block, so every
// thread takes the same branch even while the decision block of the same
// launch raises the flag.  In a one-instance graph, block 0 of such a kernel
// also clears the while loop's condition.  The call is idempotent, so no
// path that raises the flag can leave the loop running.
template <typename T>
__device__ __forceinline__ bool sweep_stopped(const SweepArgs<T>& a)
{
    __shared__ int stopped;
    if (threadIdx.x == 0) {
        stopped = a.mode == MODE_SOLVE && reinterpret_cast<volatile DevState*>(a.st)->stop;
        if (stopped && a.use_cond && !a.active && blockIdx.x == 0) cudaGraphSetConditional(a.cond, 0);
    }
    __syncthreads();
    return stopped != 0;
}

// True in an edge kernel's update blocks during a solve's evaluation at
// t = max_sweeps: that sweep stops by the sweep cap whatever its objective,
// so its new flows would be discarded and the updates are skipped.  The
// congestion partials of the returned flows f^(t), written by the previous
// sweep's edge kernel, then stay in place.  t_sweep is the t of the sweep in
// flight (written by the excess kernel before this launch may start), so the
// decision block advancing t in the same launch does not affect the test.
template <typename T>
__device__ __forceinline__ bool final_evaluation(const SweepArgs<T>& a)
{
    __shared__ int fin;
    if (threadIdx.x == 0) {
        const volatile DevState* v = a.st;
        fin = a.mode == MODE_SOLVE && v->t_sweep >= v->max_sweeps;
    }
    __syncthreads();
    return fin != 0;
}

// Ends this instance's solve from a kernel other than the decision block
// (a wait that ran out), exactly once.  It raises the stop flag and, in a
// graph, ends the while loop.  A batch's loop ends with its last running
// instance.
template <typename T>
__device__ void stop_from_kernel(const SweepArgs<T>& a)
{
    if (atomicExch(&a.st->stop, 1) != 0) return;
    const bool last = a.active ? atomicSub(a.active, 1u) == 1u : true;
    if (a.use_cond && last) cudaGraphSetConditional(a.cond, 0);
}

// Alg. 1: z = 1/2 sum psi^2 + 1/2 sum delta h^2 and the stop test, run by one
// thread after every partial of this sweep is final.
template <typename T>
__device__ void finalize(const SweepArgs<T>& a, double zsum, double cons, double cap)
{
    DevState* st = a.st;
    const double z = 0.5 * zsum;
    st->z = z;
    st->cap_rel = cap;
    st->cons_rel = cons;
    if (a.mode == MODE_EVAL) return;
    const double dz = z - st->z_prev;
    st->dz = dz;
    if (a.trace && st->evals < st->trace_len) a.trace[st->evals] = z;
    st->evals += 1;
    int stop = 0, reason = STOP_MAX_SWEEPS;
    if (a.mode == MODE_SOLVE) {
        if (!isfinite(z)) {
            stop = 1;
            reason = STOP_NUMERIC;
        } else if (st->t >= st->max_sweeps) {
            stop = 1;
            reason = STOP_MAX_SWEEPS;
        } else if (st->eps_obj > 0.0 && fabs(dz) < st->eps_obj) {
            stop = 1;
            reason = STOP_OBJECTIVE;
        } else if (st->resid_tol > 0.0 && cap <= st->resid_tol && cons <= st->resid_tol) {
            stop = 1;
            reason = STOP_RESIDUAL;
        } else if (st->eps_rel > 0.0 && fabs(dz) <= st->eps_rel * z) {
            stop = 1;
            reason = STOP_RELATIVE;
        } else if (st->stop_on_rise && dz >= 0.0) {
            // the Section 4 theorem makes z non-increasing in exact arithmetic,
            // so a rise means rounding now dominates the progress
            stop = 1;
            reason = STOP_STALL;
        } else if (st->plat_window > 0) {
            // residual plateau: the best r = max(cap_rel, cons_rel) of a window of
            // sweeps improves on the previous window's best by less than
            // kPlateauGain -- the FP32 rounding floor, not a slow descent (which
            // still improves every window)
            const double r = fmax(cap, cons);
            if (r < st->plat_cur) st->plat_cur = r;
            if (st->t - st->plat_t0 + 1 >= st->plat_window) {
                // only near the target, where FP32 rounding can be the limit: a
                // stall far above it is the method's own slow phase
                const double ceiling = kPlateauCeiling * (st->resid_tol > 0.0 ? st->resid_tol : 1e-6);
                if (st->plat_cur <= ceiling && st->plat_cur > (1.0 - kPlateauGain) * st->plat_prev) {
                    stop = 1;
                    reason = STOP_PLATEAU;
                }
                st->plat_prev = st->plat_cur;
                st->plat_cur = INFINITY;
                st->plat_t0 = st->t + 1;
            }
        }
    }
    if (stop) {
        st->stop = 1;
        st->reason = reason;
        // one instance: its stop ends the loop; a batch ends with its last instance
        const bool last = a.active ? atomicSub(a.active, 1u) == 1u : true;
        if (a.use_cond && last) cudaGraphSetConditional(a.cond, 0);
    } else {
        st->z_prev = z;
        st->t += 1;
    }
}

// Load of an objective partial that another block of the same launch may
// have written: at L2 (coherent) from global memory; SH = true when the
// partials live in the block's shared memory (the one-block engine), where
// a plain load is the coherent one.
template <bool SH, typename X>
__device__ __forceinline__ X ld_part(const X* p)
{
    if constexpr (SH) return *p;
    else return __ldcg(p);
}

// FP64 reduction of the excess blocks' partials in a fixed order, then the
// objective and the stop test.  Run by one whole block.
template <typename T, bool SH = false>
__device__ void reduce_and_finalize(const SweepArgs<T>& a)
{
    if (SH && a.grid_v == 1) {
        // one partial of each kind: the block reduction below would add and
        // compare only zeros to thread 0's values, so thread 0 forms the
        // same result directly
        if (threadIdx.x == 0) {
            const double zs = 0.0 + ld_part<SH>(a.part_h);
            const T c1 = ld_part<SH>(a.part_cons), c2 = ld_part<SH>(a.part_capb);
            finalize(a, zs, (double)(c1 > T(0) ? c1 : T(0)), (double)(c2 > T(0) ? c2 : T(0)));
        }
        return;
    }
    __shared__ double sz[32];
    __shared__ T sm1[32], sm2[32];
    double zs = 0.0;
    T cm = T(0), cp = T(0);
    for (int b = threadIdx.x; b < a.grid_v; b += blockDim.x) {
        zs += ld_part<SH>(a.part_h + b);
        const T c1 = ld_part<SH>(a.part_cons + b);
        const T c2 = ld_part<SH>(a.part_capb + b);
        cm = c1 > cm ? c1 : cm;
        cp = c2 > cp ? c2 : cp;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) zs += __shfl_xor_sync(kFull, zs, o);
    cm = warp_max(cm);
    cp = warp_max(cp);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) {
        sz[w] = zs;
        sm1[w] = cm;
        sm2[w] = cp;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const int nw = blockDim.x >> 5;
        for (int q = 1; q < nw; ++q) {
            zs += sz[q];
            cm = sm1[q] > cm ? sm1[q] : cm;
            cp = sm2[q] > cp ? sm2[q] : cp;
        }
        finalize(a, zs, (double)cm, (double)cp);
    }
}

}  // namespace
}  // namespace pdr
