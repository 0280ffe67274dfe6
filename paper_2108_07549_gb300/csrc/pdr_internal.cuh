// pdr_internal.cuh -- shared declarations of libpdr's CUDA translation units.
//
// Device layout (all arrays owned by one pdr_ctx):
//   f[e*Kp + k]   flows, edge-major, rows padded to Kp = round_up(K, 4) so
//                 every row starts on a 16-byte boundary; pad entries stay 0
//   h[i*Kp + k]   heights, vertex-major, same padding
//   s, t [Kp]     commodity endpoints, padded with -1 (never a vertex)
//   dem [Kp]      demands, padded with 0
//   row_ptr/col   out-adjacency (edge id = CSR position), src = edge tails
//   in_ptr/in_eid in-adjacency, edge ids ascending within each vertex
//   inc_ptr/inc   incidence list of each vertex: its in-edges e (ascending),
//                 then its out-edges stored as ~e (ascending); delta_i is
//                 inc_ptr[i+1] - inc_ptr[i]
//   deg           delta_i = out-degree + in-degree
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

namespace pdr {

constexpr int kThreads = 256;  // block size of every sweep kernel
constexpr int kBatchThreads = 512;  // block size of the one-block-per-instance batch kernel
constexpr int kExcessForms = 6;     // excess kernel forms: 0 gathers, 1..5 bulk copies
// Resident blocks per SM that the block forms of the edge kernels are
// compiled for (the register cap that follows from it: 65,536 / (B x that)).
constexpr int block_min_blocks(int B, int V)
{
    return B <= 128 ? 12 : B <= 256 ? (V <= 2 ? 6 : 4) : B <= 512 ? (V <= 5 ? 3 : 2) : (V <= 3 ? 2 : 1);
}
// The same for the Alg. 3 / Alg. 4 block forms (more live values per element).
constexpr int gd_min_blocks(int B, int V)
{
    return B <= 128 ? 10 : B <= 256 ? (V <= 2 ? 5 : 3) : B <= 512 ? 2 : 1;
}
constexpr long long kWaitCycles = 4ll << 30;  // default limit of a device-side wait: ~2 s at the SM clock
constexpr long long kBarrierNs = 2000000000ll;  // default limit of a grid-barrier wait: 2 s of the global timer

// Kernel modes.
enum : int {
    MODE_SOLVE = 0,   // honour and apply the stop rules
    MODE_EVAL = 1,    // compute h and z only; no stop decision, no counter change
    MODE_FORCED = 2,  // one sweep with the stop rules disabled
    MODE_PSI = 3      // edge kernel: congestion of the stored flows only (no QP)
};

enum : int {
    STOP_MAX_SWEEPS = 0,
    STOP_OBJECTIVE = 1,
    STOP_RESIDUAL = 2,
    STOP_RELATIVE = 3,
    STOP_NUMERIC = 4,
    STOP_STALL = 5,
    STOP_PLATEAU = 6
};

// Solver state that lives on the device and is updated by the decision block
// of the edge kernel, so the sweep loop never returns to the host.
struct DevState {
    double z;          // objective z^(t) of the current flows
    double z_prev;     // objective of the previous sweep (+inf at the start)
    double dz;         // z - z_prev at the last evaluation
    double cap_rel;    // max_e psi_e / max(u_e, mean positive u) at the last evaluation
    double cons_rel;   // max_{i,k} |Delta_ik| / d_k at the last evaluation
    double eps_obj;    // |dz| < eps_obj stops (<= 0: off)
    double resid_tol;  // cap_rel, cons_rel <= resid_tol stops (<= 0: off)
    double eps_rel;    // |dz| <= eps_rel * z stops (<= 0: off)
    long long t;          // QP updates applied
    long long max_sweeps; // t >= max_sweeps stops
    long long trace_len;  // capacity of the z trace
    long long evals;      // objective evaluations written to the trace
    int stop;             // 1 once a stop rule fired
    int reason;           // STOP_* code
    int stop_on_rise;     // 1: z^(t) >= z^(t-1) stops (the FP32 rounding floor)
    int fault;            // 1: a kernel's wait on a shared-memory barrier ran out of its
                          // limit (the sweep is invalid; the solve stops with an error)
    long long t_sweep;    // t of the sweep in flight (written by the excess kernel, read by
                          // the gradient-step kernels while the decision block advances t)
    // residual plateau (FP32 phase of the tail mode): r = max(cap_rel, cons_rel)
    long long plat_window;  // sweeps per window (0: off)
    long long plat_t0;      // t at which the current window began
    double plat_cur;        // smallest r in the current window
    double plat_prev;       // smallest r in the previous window (+inf before the first)
};
constexpr long long kPlateauWindow = 1024;  // sweeps per window of the plateau rule
constexpr double kPlateauGain = 1e-4;       // a window must lower the best residual by this fraction
constexpr double kPlateauCeiling = 1e3;     // ... once it is below this multiple of resid_tol

// Grid barrier of the persistent sweep kernel (device memory, zeroed before
// each launch).  `failed` is set when a wait ran out of its time limit;
// every block then leaves the kernel and the host reports the error.
struct GridBarrier {
    unsigned int count;   // blocks arrived at the current barrier
    unsigned int gen;     // barrier generation, advanced by the last arrival
    unsigned int failed;  // 1: a wait timed out
    unsigned int pad;
};

template <typename T>
struct SweepArgs {
    int32_t n;
    int64_t m;
    int32_t K, Kp;
    const int64_t* row_ptr;
    const int32_t* col;
    const int32_t* src;
    const int64_t* in_ptr;
    const int32_t* in_eid;
    const int64_t* inc_ptr;
    const int32_t* inc;
    const int32_t* deg;
    const int32_t* s;
    const int32_t* t;
    const T* dem;
    const T* inv_dem;  // [Kp] 1/d_k, 0 in the padding
    const T* u;
    const double* inv_scale;  // [m] 1 / max(u_e, mean positive u)
    const T* inv_scale_t;     // the same in the working precision
    const T* inv_deg;   // [n] 1/delta_i (0 for isolated vertices)
    T* f;               // flows read by this sweep, f^(t)
    T* f_out;           // flows written by the edge QP, f^(t+1) (the other buffer)
    T* h;
    const T* theta_in;  // [2m] of the sweep that made f: [0, m) the root psi'/2 of each edge QP
                        // (0 = none), [m, 2m) the warm start of this sweep's root search
    T* theta;           // [2m] this sweep's roots and the next sweep's warm starts (the other
                        // buffer, like f_out)
    // Objective partials.  Edge kernels write one partial per warp (lane-group
    // form) or per block (block form): the sum of psi^2 as an accumulator
    // pair and the largest psi/scale.  Each excess block adds a fixed slice
    // of those to its own sum of delta h^2 and writes one FP64 value; the
    // last excess block reduces those in FP64.
    double* part_h;     // [grid_v] per excess block: slice of psi^2 + delta h^2
    T* part_cons;       // [grid_v] per excess block: max |Delta|/d
    T* part_capb;       // [grid_v] per excess block: max psi/scale of its slice
    void* part_psi;     // [n_psi] per edge warp/block: sum psi^2 (float2 pair or double)
    T* part_cap;        // [n_psi] per edge warp/block: max psi/scale
    int32_t grid_v, grid_e;
    int excess_form;    // excess kernel: 0 = per-thread gathers, 1..3 = bulk-copy pipeline
                        // (stages x row segments per block: 4 x 8, 2 x 8, 4 x 4)
    const int32_t* xv_start;  // [grid_v + 1] bulk-copy form: first vertex of each block
    long long wait_cycles;    // bulk-copy form: time limit of a barrier wait, in SM clock cycles
    int hold_end;             // bulk-copy form, tests only: the producer never posts its end
                              // marker, so the consumers' last wait runs out (no copy in flight)
    long long barrier_ns;     // persistent engine: time limit of a grid-barrier wait, in ns
    int hold_barrier;         // persistent engine, tests only: block 0 leaves without arriving
                              // at its first grid barrier, so the other blocks' waits run out
    int64_t n_psi;      // number of edge partials
    int64_t pf_edges;   // edge QP: L2 prefetch of the rows of edge e + pf_edges while
                        // edge e is solved (about one wave of resident edges ahead; 0: off)
    int l2_hints;       // 1: the working set exceeds L2; the edge QP streams flow rows evict-first
    // Alg. 3 / Alg. 4 state (double-buffered like the flows) and parameters
    const T* beta_in;   // [m] learning rates beta_ij of iteration t
    T* beta_out;        // [m] learning rates of iteration t+1
    const T* v_in;      // [m][Kp] velocities of iteration t (Alg. 4)
    T* v_out;           // [m][Kp] velocities of iteration t+1 (Alg. 4)
    int momentum;       // 0: Alg. 3, 1: Alg. 4
    int ck;             // edge QP: 1 = capacity kept (Program (6)): f' = P(c) onto {f >= 0, sum f <= u}
    T beta_min, beta_max, alpha_inc, alpha_dec, gamma;
    T* psi_out;         // optional [m] congestion output of the edge kernel
    DevState* st;
    double* trace;
    unsigned int* active;  // batched solves: instances still running (NULL for one instance)
    cudaGraphConditionalHandle cond;
    int use_cond;
    int mode;
};

// Launchers (sweep.cu).  Each returns the launch error.
// pdl: programmatic dependent launch (the kernel waits in griddepcontrol.wait
// for the previous kernel), used in the captured sweep loop.
template <typename T>
cudaError_t launch_excess(const SweepArgs<T>& a, cudaStream_t stream, bool pdl = false);
// Objective reduction and stop decision on their own (one block); the edge
// kernel does the same work in its extra block during a sweep.
template <typename T>
cudaError_t launch_finalize(const SweepArgs<T>& a, cudaStream_t stream);
template <typename T>
cudaError_t launch_edge(const SweepArgs<T>& a, int cfg, cudaStream_t stream, bool pdl = false);
template <typename T>
int edge_config(int Kp);  // picks the edge-kernel variant for a row length
template <typename T>
int edge_grid(int cfg, int64_t m, int num_sms);  // grid size of that variant
template <typename T>
int64_t edge_parts(int cfg, int grid);  // number of partials that grid writes
template <typename T>
int edge_capacity(int cfg);             // elements per row a variant holds (-1 if none)
int num_edge_configs();
int edge_plain_config(int cfg);          // the non-pipelined variant of the same capacity
int edge_group_lanes(int cfg);           // lanes per edge of a lane-group variant
template <typename T>
int64_t edge_prefetch_distance(int cfg, int num_sms);  // edges solved by one wave of resident blocks
bool edge_config_pipelined(int cfg);
bool edge_config_staged(int cfg);       // the bulk-copy staged block forms
int excess_grid(int32_t n, int Kp, int vec, int num_sms, int resident_blocks);
// Persistent sweep kernel (sweep.cu): excess and edge QP of every sweep in one
// cooperative launch, separated by grid barriers; runs up to `sweeps` sweeps
// of Alg. 1 or until the stop rules fire.  Only the lane-group variants.
template <typename T>
int persistent_grid(int cfg, int64_t m, int32_t n, int Kp, int num_sms);  // 0: not available
// Batched form, one thread-block cluster of csize blocks (1, 2, 4 or 8) per
// instance: instances ids[0..count) of args run up to `sweeps` sweeps each
// with the lane-group variant cfg (true for batch_block_config);
// psi_prologue: first launch of a solve.  smem > 0 (csize = 1 only, at most
// kBlockSmemMax): the shared-memory form, each block holding its instance's
// flows, heights, roots, partials and state in smem bytes of shared memory
// (the largest block_smem_bytes of the instances launched).
template <typename T>
cudaError_t launch_batch_block(int cfg, const SweepArgs<T>* args, const int* ids, int count, int csize, int64_t sweeps,
                               int psi_prologue, cudaStream_t stream, int64_t smem = 0);
bool batch_block_config(int cfg);
// Shared memory of the one-block form for an instance of n vertices, m edges,
// rows of Kp values and n_psi edge partials, in bytes.
template <typename T>
int64_t block_smem_bytes(int64_t n, int64_t m, int64_t Kp, int64_t n_psi);
// Largest shared-memory form: two blocks of it fit on one SM.
constexpr int64_t kBlockSmemMax = 100 * 1024;

// Packs and widens m padded rows into dst[rows*K] (double), dst writable by the GPU.
template <typename T>
cudaError_t launch_widen_rows(const T* src, int64_t rows, int K, int Kp, double* dst, cudaStream_t stream);

template <typename T>
cudaError_t launch_persistent(const SweepArgs<T>& a, int cfg, int grid, int64_t sweeps, GridBarrier* bar,
                              int psi_prologue, cudaStream_t stream);
template <typename T>
int excess_resident_blocks();  // excess blocks resident per SM (occupancy)
// Bulk-copy excess form (1..3): blocks resident per SM (0 if it cannot run);
// sets the kernel's shared-memory limit on first use.
template <typename T>
int excess_bulk_resident_blocks(int form);
// Splits vertices 0..n-1 into `grid` contiguous ranges of about equal
// incidence count (plus a per-vertex term): xv_start[b] = first vertex of block b,
// xv_start[grid] = n.
cudaError_t launch_excess_split(const int64_t* inc_ptr, int32_t n, int grid, int32_t* xv_start,
                                cudaStream_t stream);
cudaError_t launch_convert_f32_to_f64(const float* a, double* b, int64_t count, cudaStream_t stream);

// Gradient-step kernels of Alg. 3 / Alg. 4 (gd.cu); same grid, partials and
// decision block as launch_edge.
template <typename T>
cudaError_t launch_gd(const SweepArgs<T>& a, int cfg, cudaStream_t stream);

// Adjacency builder (adjacency.cu): in-adjacency, incidence lists, edge
// tails and degrees.  work must hold 2*n + 1 int64 entries.
cudaError_t build_adjacency(int32_t n, int64_t m, const int64_t* row_ptr, const int32_t* col, int32_t* src,
                            int64_t* in_ptr, int32_t* in_eid, int64_t* inc_ptr, int32_t* inc, int32_t* deg,
                            int64_t* work, cudaStream_t stream);

// Reverse mode through unrolled sweeps (adjoint.cu).
template <typename T>
cudaError_t launch_seed(const SweepArgs<T>& a, T* fbar, double* ubar, double* dbar, int num_sms, cudaStream_t s);
template <typename T>
cudaError_t launch_backward_sweep(const SweepArgs<T>& a, const T* theta, const T* fbar, T* cbar, T* Dbar, double* ubar,
                                  double* dbar, uint32_t* mask, int fused, int num_sms, cudaStream_t s);
// words of the active-set ballots launch_backward_sweep keeps per edge
inline int64_t backward_mask_words(int Kp, int vec) { return (int64_t)((Kp / vec + 31) / 32) * vec; }

// Residuals and certificate (residuals.cu).
struct ResidOut {
    double z, cap_abs, cap_rel, cons_abs, cons_rel, f_min, margin, margin_scale;
};
// Instance data of the residual pass, all in FP64 except the FP32 copy of
// 1/d used to screen candidates for the largest relative imbalance.
struct ResidIn {
    const double* u_d;        // [m] capacities
    const double* dem_d;      // [Kp] demands (0 in the padding)
    const double* inv_deg_d;  // [n] 1/delta_i (0 for isolated vertices)
    const float* inv_dem_f;   // [Kp] 1/d_k rounded to FP32 (0 in the padding)
};

template <typename T>
cudaError_t launch_residuals(const SweepArgs<T>& a, const ResidIn& r, double* h64, double* part, int32_t grid_v,
                             int32_t grid_e, ResidOut* out, cudaStream_t stream);
int resid_part_count(int32_t grid_v, int32_t grid_e);

// Message returned by pdr_last_error(NULL) on the calling thread (api.cu).
void set_thread_error(const std::string& msg);

}  // namespace pdr
