// api.cu -- the C ABI declared in include/pdr.h.
//
// A context holds one instance of eq. (1) on the device and runs Alg. 1 on
// it.  Flows live in two buffers: a sweep reads f^(t) from one and the edge
// QP writes f^(t+1) to the other, so the stop decision (taken by an extra
// block of the edge kernel, concurrently with the QPs) can still return
// f^(t).  pdr_solve launches one CUDA graph whose only node is a conditional
// "while" loop over a body of kUnroll sweeps; the decision block clears the
// loop condition, so a whole solve is one launch and one host
// synchronisation.  If the runtime cannot build that graph, the same kernels
// are launched from a host loop that reads the stop flag back between
// chunks of sweeps.
#include "pdr.h"
#include "pdr_internal.cuh"

#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

using namespace pdr;

namespace {

thread_local std::string g_create_error;

int round_up4(int k) { return (k + 3) / 4 * 4; }

constexpr int kUnroll = 32;     // sweeps per iteration of the graph's while loop (even)
constexpr int kHostChunk = 256; // sweeps between stop-flag reads of the host loop (even)
// Working sets above this stream from HBM every sweep (GB300: 129 MB of L2;
// measured L2-resident streaming holds up to ~90 MB and collapses by 120 MB).
constexpr double kL2Bytes = 96.0 * 1024 * 1024;

void fill_defaults(pdr_options* o)
{
    std::memset(o, 0, sizeof(*o));
    o->precision = PDR_PREC_FP32;
    o->use_graph = 1;
    o->eps_obj = 1e-6;
    o->resid_tol = 1e-6;
    o->eps_rel = 0.0;
    o->max_sweeps = 1000000;
    o->trace_len = 0;
    o->algo = PDR_ALGO_ESO;
    o->beta_init = o->beta_min = o->beta_max = o->alpha_inc = o->alpha_dec = 0.0;
    o->gamma = -1.0;
    o->edge_variant = -1;
    o->excess_variant = -1;
}

// Alg. 3 / Alg. 4: the gradient-step kernels with learning rates; Alg. 1
// and its capacity-kept form run the edge-QP kernels.
bool is_gd(const pdr_options& o) { return o.algo == PDR_ALGO_AGD || o.algo == PDR_ALGO_GDM; }

bool options_ok(const pdr_options* o, std::string* why)
{
    if (o->precision < PDR_PREC_FP32 || o->precision > PDR_PREC_FP32_FP64TAIL) {
        *why = "precision must be 0 (FP32), 1 (FP64) or 2 (FP32 with FP64 tail)";
        return false;
    }
    if (!std::isfinite(o->eps_obj) || !std::isfinite(o->resid_tol) || !std::isfinite(o->eps_rel)) {
        *why = "eps_obj, resid_tol and eps_rel must be finite";
        return false;
    }
    if (o->use_graph < 0 || o->use_graph > 3) {
        *why = "use_graph must be 0 (host loop), 1 (CUDA graph), 2 (persistent kernel) or 3 (cluster kernel)";
        return false;
    }
    if (o->max_sweeps < 0) {
        *why = "max_sweeps must be >= 0";
        return false;
    }
    if (o->trace_len < 0) {
        *why = "trace_len must be >= 0";
        return false;
    }
    if (o->algo < PDR_ALGO_ESO || o->algo > PDR_ALGO_CK) {
        *why = "algo must be 0 (ESO), 1 (AGD), 2 (GDM) or 3 (capacity kept)";
        return false;
    }
    if (o->excess_variant < -1 || o->excess_variant > kExcessForms - 1) {
        *why = "excess_variant must be -1 (default), 0 (gathers) or 1..5 (bulk copies)";
        return false;
    }
    const double g[] = {o->beta_init, o->beta_min, o->beta_max, o->alpha_inc, o->alpha_dec, o->gamma};
    for (double x : g)
        if (!std::isfinite(x)) {
            *why = "learning-rate parameters must be finite";
            return false;
        }
    if (o->gamma >= 1.0) {
        *why = "gamma must be < 1";
        return false;
    }
    if (o->edge_variant < -1 || o->edge_variant >= num_edge_configs()) {
        *why = "edge_variant must be -1 or an index of the variant table";
        return false;
    }
    return true;
}

}  // namespace

void pdr::set_thread_error(const std::string& msg) { g_create_error = msg; }

struct pdr_ctx {
    int32_t n = 0;
    int64_t m = 0;
    int32_t K = 0, Kp = 0;
    pdr_options opt{};
    cudaStream_t stream = nullptr;
    cudaStream_t cap_stream = nullptr;
    int num_sms = 0;
    bool isolated = false;

    // instance
    int64_t *row_ptr = nullptr, *in_ptr = nullptr, *inc_ptr = nullptr, *work = nullptr;
    int32_t *col = nullptr, *src = nullptr, *in_eid = nullptr, *inc = nullptr, *deg = nullptr, *s = nullptr,
            *t = nullptr;
    double *u_d = nullptr, *dem_d = nullptr, *inv_scale = nullptr;
    float *u_f = nullptr, *dem_f = nullptr, *inv_dem_f = nullptr, *inv_scale_f = nullptr;
    double* inv_dem_d = nullptr;
    // state
    float *f32[2] = {nullptr, nullptr}, *h32 = nullptr, *inv_deg_f = nullptr;
    double *f64[2] = {nullptr, nullptr}, *h64 = nullptr, *inv_deg_d = nullptr;
    int cur = 0;  // buffer holding the current flows
    // [2m] roots of the edge QPs and warm starts of the next sweep,
    // double-buffered like the flows: theta[b] holds the roots ([0, m)) of
    // the sweep that produced the flows in buffer b and the warm starts
    // ([m, 2m)) of the sweep that reads them; 16 bytes per edge covers both
    // precisions
    double* theta[2] = {nullptr, nullptr};
    // Alg. 3 / Alg. 4 state, double-buffered like the flows
    double* beta_buf[2] = {nullptr, nullptr};  // [m], 8 bytes per edge covers both precisions
    float* v32[2] = {nullptr, nullptr};
    double* v64[2] = {nullptr, nullptr};
    // effective Alg. 3 / Alg. 4 parameters
    double g_beta_init = 0, g_beta_min = 0, g_beta_max = 0, g_alpha_inc = 0, g_alpha_dec = 0, g_gamma = 0;
    int cur_prec = 0;  // precision of the current flows: 0 FP32, 1 FP64
    double* part_h = nullptr;
    // partials typed by the working precision: 8 bytes per entry covers both
    double *part_cons = nullptr, *part_capb = nullptr, *part_psi = nullptr, *part_cap = nullptr;
    int grid_v[2] = {1, 1}, grid_e[2] = {1, 1}, cfg[2] = {-1, -1};
    // excess kernel form (0: gathers, 1..3: bulk copies); grid and vertex split of each bulk form
    int xform = 0;
    int xgrid[kExcessForms] = {};
    int32_t* xv_start[kExcessForms] = {};
    int64_t n_psi[2] = {1, 1};
    int pgrid[2] = {0, 0};         // persistent kernel grid per precision (0: not available)
    int64_t pf[2] = {0, 0};        // edge-kernel L2 prefetch distance per precision (edges)
    GridBarrier* bar = nullptr;    // its grid barrier
    DevState* st = nullptr;
    DevState* hst = nullptr;  // pinned mirror
    double* trace = nullptr;
    int64_t trace_cap = 0;
    // residuals
    double *r_h64 = nullptr, *r_part = nullptr;
    int* data_err = nullptr;  // error bits of a device-side pdr_set_data
    int reason_fp32 = -1;     // tail mode: the stop reason of the last FP32 phase
    ResidOut* r_out = nullptr;
    ResidOut* hr_out = nullptr;  // pinned
    int r_grid_v = 1, r_grid_e = 1;
    void* psi_tmp = nullptr;
    // graphs
    cudaGraph_t graph[2] = {nullptr, nullptr};
    cudaGraphExec_t exec[2] = {nullptr, nullptr};
    cudaGraphConditionalHandle cond[2] = {0, 0};
    bool graph_tried[2] = {false, false};
    bool graph_ok[2] = {false, false};
    bool graph_pdl[2] = {false, false};  // the graph's kernels use programmatic dependent launch

    pdr_result last{};
    std::string err;
    // checkpoint / resume: the next pdr_solve continues the restored sweep
    // counter and objective instead of starting afresh
    bool resume_pending = false;
    // device-side wait limit (cycles) and the end-marker hold of the bulk-copy
    // excess form; changed only by pdr_debug_wait (tests of the time limit)
    long long wait_cycles = kWaitCycles;
    int hold_end = 0;
    // persistent engine's grid barrier; changed only by pdr_debug_barrier
    long long barrier_ns = kBarrierNs;
    int hold_barrier = 0;
    int64_t t_widen = -1;  // t at which the FP64 tail of the last solve began (-1: none)
    unsigned char* cl_args = nullptr;  // the cluster engine's arguments and instance id (device)
    // reverse-mode workspace (pdr_backward: checkpoints, segment states,
    // cotangents), kept for later calls: the i-th buffer a call asks for is
    // reused when it is large enough, so calls with the same T, checkpoint
    // interval and precision allocate nothing.  Freed by pdr_destroy, and
    // after a failed pdr_backward.
    std::vector<std::pair<void*, size_t>> adj_ws;

    pdr_status fail(pdr_status code, const std::string& msg)
    {
        err = msg;
        return code;
    }
    pdr_status cuda_fail(const char* what, cudaError_t e)
    {
        err = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
        return PDR_ERR_CUDA;
    }
};

#define CK(call)                                              \
    do {                                                      \
        cudaError_t _e = (call);                              \
        if (_e != cudaSuccess) return ctx->cuda_fail(#call, _e); \
    } while (0)

namespace {

// Host-side failure injection (pdr_debug_fail_alloc): when positive, the
// device allocation that brings it to 0 fails as if the device were full.
std::atomic<int64_t> g_fail_alloc{0};

bool injected_alloc_failure()
{
    int64_t k = g_fail_alloc.load();
    while (k > 0)
        if (g_fail_alloc.compare_exchange_weak(k, k - 1)) return k == 1;
    return false;
}

template <typename T>
T* dalloc(pdr_ctx* ctx, size_t count, pdr_status* st)
{
    void* p = nullptr;
    if (count == 0) count = 1;
    if (injected_alloc_failure()) {
        *st = PDR_ERR_OOM;
        ctx->err = "cudaMalloc: injected allocation failure";
        return nullptr;
    }
    cudaError_t e = cudaMalloc(&p, sizeof(T) * count);
    if (e != cudaSuccess) {
        *st = (e == cudaErrorMemoryAllocation) ? PDR_ERR_OOM : PDR_ERR_CUDA;
        ctx->err = std::string("cudaMalloc: ") + cudaGetErrorString(e);
        cudaGetLastError();
        return nullptr;
    }
    return static_cast<T*>(p);
}

template <typename T>
struct Prec;
template <>
struct Prec<float> {
    static constexpr int id = 0;
    static float* f(pdr_ctx* c, int b) { return c->f32[b]; }
    static float* h(pdr_ctx* c) { return c->h32; }
    static const float* u(pdr_ctx* c) { return c->u_f; }
    static const float* dem(pdr_ctx* c) { return c->dem_f; }
    static const float* inv_dem(pdr_ctx* c) { return c->inv_dem_f; }
    static const float* inv_scale(pdr_ctx* c) { return c->inv_scale_f; }
    static const float* inv_deg(pdr_ctx* c) { return c->inv_deg_f; }
    static float* v(pdr_ctx* c, int b) { return c->v32[b]; }
};
template <>
struct Prec<double> {
    static constexpr int id = 1;
    static double* f(pdr_ctx* c, int b) { return c->f64[b]; }
    static double* h(pdr_ctx* c) { return c->h64; }
    static const double* u(pdr_ctx* c) { return c->u_d; }
    static const double* dem(pdr_ctx* c) { return c->dem_d; }
    static const double* inv_dem(pdr_ctx* c) { return c->inv_dem_d; }
    static const double* inv_scale(pdr_ctx* c) { return c->inv_scale; }
    static const double* inv_deg(pdr_ctx* c) { return c->inv_deg_d; }
    static double* v(pdr_ctx* c, int b) { return c->v64[b]; }
};

// Kernel arguments for a sweep that reads buffer (base ^ par) and writes the
// other one.  base defaults to the buffer of the current flows.
template <typename T>
SweepArgs<T> make_args(pdr_ctx* ctx, int mode, int use_cond = 0, cudaGraphConditionalHandle cond = 0, int par = 0,
                       int base = -1)
{
    SweepArgs<T> a{};
    const int p = Prec<T>::id;
    a.n = ctx->n;
    a.m = ctx->m;
    a.K = ctx->K;
    a.Kp = ctx->Kp;
    a.row_ptr = ctx->row_ptr;
    a.col = ctx->col;
    a.src = ctx->src;
    a.in_ptr = ctx->in_ptr;
    a.in_eid = ctx->in_eid;
    a.inc_ptr = ctx->inc_ptr;
    a.inc = ctx->inc;
    a.deg = ctx->deg;
    a.s = ctx->s;
    a.t = ctx->t;
    a.dem = Prec<T>::dem(ctx);
    a.inv_dem = Prec<T>::inv_dem(ctx);
    a.u = Prec<T>::u(ctx);
    a.inv_scale = ctx->inv_scale;
    a.inv_scale_t = Prec<T>::inv_scale(ctx);
    a.inv_deg = Prec<T>::inv_deg(ctx);
    const int b = ((base < 0 ? ctx->cur : base) ^ par) & 1;
    a.theta_in = reinterpret_cast<const T*>(ctx->theta[b]);
    a.theta = reinterpret_cast<T*>(ctx->theta[b ^ 1]);
    a.f = Prec<T>::f(ctx, b);
    a.f_out = Prec<T>::f(ctx, b ^ 1);
    a.beta_in = reinterpret_cast<const T*>(ctx->beta_buf[b]);
    a.beta_out = reinterpret_cast<T*>(ctx->beta_buf[b ^ 1]);
    a.v_in = Prec<T>::v(ctx, b);
    a.v_out = Prec<T>::v(ctx, b ^ 1);
    a.momentum = ctx->opt.algo == PDR_ALGO_GDM ? 1 : 0;
    a.ck = ctx->opt.algo == PDR_ALGO_CK ? 1 : 0;
    a.beta_min = (T)ctx->g_beta_min;
    a.beta_max = (T)ctx->g_beta_max;
    a.alpha_inc = (T)ctx->g_alpha_inc;
    a.alpha_dec = (T)ctx->g_alpha_dec;
    a.gamma = (T)ctx->g_gamma;
    a.h = Prec<T>::h(ctx);
    a.part_h = ctx->part_h;
    a.part_cons = reinterpret_cast<T*>(ctx->part_cons);
    a.part_capb = reinterpret_cast<T*>(ctx->part_capb);
    a.part_psi = ctx->part_psi;
    a.part_cap = reinterpret_cast<T*>(ctx->part_cap);
    a.excess_form = ctx->xform;
    a.xv_start = ctx->xv_start[ctx->xform];
    a.wait_cycles = ctx->wait_cycles;
    a.hold_end = ctx->hold_end;
    a.barrier_ns = ctx->barrier_ns;
    a.hold_barrier = ctx->hold_barrier;
    a.grid_v = ctx->xform ? ctx->xgrid[ctx->xform] : ctx->grid_v[p];
    a.grid_e = ctx->grid_e[p];
    a.n_psi = ctx->n_psi[p];
    a.pf_edges = ctx->pf[p];
    a.l2_hints = ctx->pf[p] > 0 ? 1 : 0;
    a.psi_out = nullptr;
    a.st = ctx->st;
    a.trace = ctx->trace;
    a.active = nullptr;
    a.cond = cond;
    a.use_cond = use_cond;
    a.mode = mode;
    return a;
}

// Allocates the FP64 state on first use.
pdr_status ensure_fp64(pdr_ctx* ctx)
{
    if (ctx->f64[0]) return PDR_OK;
    pdr_status st = PDR_OK;
    const size_t fm = (size_t)ctx->m * ctx->Kp, hn = (size_t)ctx->n * ctx->Kp;
    for (int b = 0; b < 2; ++b) {
        ctx->f64[b] = dalloc<double>(ctx, fm, &st);
        if (!ctx->f64[b]) return st;
        CK(cudaMemsetAsync(ctx->f64[b], 0, sizeof(double) * (fm ? fm : 1), ctx->stream));
    }
    ctx->h64 = dalloc<double>(ctx, hn, &st);
    if (!ctx->h64) return st;
    CK(cudaMemsetAsync(ctx->h64, 0, sizeof(double) * (hn ? hn : 1), ctx->stream));
    return PDR_OK;
}

pdr_status ensure_fp32(pdr_ctx* ctx)
{
    if (ctx->f32[0]) return PDR_OK;
    pdr_status st = PDR_OK;
    const size_t fm = (size_t)ctx->m * ctx->Kp, hn = (size_t)ctx->n * ctx->Kp;
    for (int b = 0; b < 2; ++b) {
        ctx->f32[b] = dalloc<float>(ctx, fm, &st);
        if (!ctx->f32[b]) return st;
        CK(cudaMemsetAsync(ctx->f32[b], 0, sizeof(float) * (fm ? fm : 1), ctx->stream));
    }
    ctx->h32 = dalloc<float>(ctx, hn, &st);
    if (!ctx->h32) return st;
    CK(cudaMemsetAsync(ctx->h32, 0, sizeof(float) * (hn ? hn : 1), ctx->stream));
    return PDR_OK;
}

// Effective Alg. 3 / Alg. 4 parameters: the caller's, or Section 7's.
void resolve_gd_params(pdr_ctx* ctx)
{
    const pdr_options& o = ctx->opt;
    const bool gdm = o.algo == PDR_ALGO_GDM;
    ctx->g_beta_init = o.beta_init > 0 ? o.beta_init : (gdm ? 0.1 : 0.25);
    ctx->g_beta_min = o.beta_min > 0 ? o.beta_min : 1.0 / ctx->K;
    ctx->g_beta_max = o.beta_max > 0 ? o.beta_max : (gdm ? 0.2 : 0.5);
    ctx->g_alpha_inc = o.alpha_inc > 0 ? o.alpha_inc : 2.0;
    ctx->g_alpha_dec = o.alpha_dec > 0 ? o.alpha_dec : 0.5;
    ctx->g_gamma = o.gamma >= 0 ? o.gamma : (gdm ? 0.9 : 0.0);
}

// The flow update of one sweep: the edge QP (Alg. 2) or the gradient step.
template <typename T>
cudaError_t launch_update(pdr_ctx* ctx, const SweepArgs<T>& a, cudaStream_t stream, bool pdl = false)
{
    const int cfg = ctx->cfg[Prec<T>::id];
    return is_gd(ctx->opt) ? launch_gd<T>(a, cfg, stream) : launch_edge<T>(a, cfg, stream, pdl);
}

// Velocity buffers of the working precision (Alg. 4 only).
template <typename T>
pdr_status ensure_velocity(pdr_ctx* ctx)
{
    if (ctx->opt.algo != PDR_ALGO_GDM) return PDR_OK;
    const size_t fm = (size_t)ctx->m * ctx->Kp;
    for (int b = 0; b < 2; ++b) {
        T*& buf = Prec<T>::id ? reinterpret_cast<T*&>(ctx->v64[b]) : reinterpret_cast<T*&>(ctx->v32[b]);
        if (buf) continue;
        pdr_status st = PDR_OK;
        buf = dalloc<T>(ctx, fm, &st);
        if (!buf) return st;
        CK(cudaMemsetAsync(buf, 0, sizeof(T) * (fm ? fm : 1), ctx->stream));
    }
    return PDR_OK;
}

// Learning rates = beta_init and velocities = 0 in buffer 0 (precision T).
template <typename T>
pdr_status init_gd_state(pdr_ctx* ctx)
{
    if (ctx->m == 0) return PDR_OK;
    std::vector<T> b(ctx->m, (T)ctx->g_beta_init);
    CK(cudaMemcpyAsync(ctx->beta_buf[0], b.data(), sizeof(T) * ctx->m, cudaMemcpyHostToDevice, ctx->stream));
    if (ctx->opt.algo == PDR_ALGO_GDM) {
        pdr_status s = ensure_velocity<T>(ctx);
        if (s != PDR_OK) return s;
        CK(cudaMemsetAsync(Prec<T>::v(ctx, 0), 0, sizeof(T) * (size_t)ctx->m * ctx->Kp, ctx->stream));
    }
    CK(cudaStreamSynchronize(ctx->stream));
    return PDR_OK;
}

pdr_status init_gd_state_current(pdr_ctx* ctx)
{
    return ctx->cur_prec ? init_gd_state<double>(ctx) : init_gd_state<float>(ctx);
}

// Moves the current flows into buffer 0 (the graphs are captured for it).
template <typename T>
pdr_status flows_to_buffer0(pdr_ctx* ctx)
{
    if (ctx->cur == 0) return PDR_OK;
    const size_t bytes = sizeof(T) * (size_t)ctx->m * ctx->Kp;
    if (bytes) CK(cudaMemcpyAsync(Prec<T>::f(ctx, 0), Prec<T>::f(ctx, 1), bytes, cudaMemcpyDeviceToDevice, ctx->stream));
    if (ctx->m > 0)
        CK(cudaMemcpyAsync(ctx->beta_buf[0], ctx->beta_buf[1], sizeof(T) * ctx->m, cudaMemcpyDeviceToDevice,
                           ctx->stream));
    if (ctx->opt.algo == PDR_ALGO_GDM && bytes && Prec<T>::v(ctx, 1))
        CK(cudaMemcpyAsync(Prec<T>::v(ctx, 0), Prec<T>::v(ctx, 1), bytes, cudaMemcpyDeviceToDevice, ctx->stream));
    if (ctx->m > 0)
        CK(cudaMemcpyAsync(ctx->theta[0], ctx->theta[1], sizeof(T) * 2 * ctx->m, cudaMemcpyDeviceToDevice,
                           ctx->stream));
    ctx->cur = 0;
    return PDR_OK;
}

pdr_status flows_to_buffer0_current(pdr_ctx* ctx)
{
    return ctx->cur_prec ? flows_to_buffer0<double>(ctx) : flows_to_buffer0<float>(ctx);
}

int start_prec(const pdr_options& o) { return o.precision == PDR_PREC_FP64 ? 1 : 0; }

// Recomputes the congestion partials of the current flows.
template <typename T>
pdr_status refresh_psi(pdr_ctx* ctx, T* psi_out = nullptr, bool keep_theta = false)
{
    if (!psi_out && !keep_theta) {
        // new flows: the edge QPs start their root search cold
        for (int b = 0; b < 2; ++b)
            CK(cudaMemsetAsync(ctx->theta[b], 0, sizeof(double) * 2 * (ctx->m > 0 ? ctx->m : 1), ctx->stream));
    }
    SweepArgs<T> a = make_args<T>(ctx, MODE_PSI);
    a.psi_out = psi_out;
    if (ctx->m > 0) {
        CK(launch_edge<T>(a, ctx->cfg[Prec<T>::id], ctx->stream));
    } else {
        CK(cudaMemsetAsync(ctx->part_psi, 0, sizeof(double) * ctx->n_psi[Prec<T>::id], ctx->stream));
        CK(cudaMemsetAsync(ctx->part_cap, 0, sizeof(double) * ctx->n_psi[Prec<T>::id], ctx->stream));
    }
    return PDR_OK;
}

pdr_status refresh_psi_current(pdr_ctx* ctx)
{
    return ctx->cur_prec ? refresh_psi<double>(ctx) : refresh_psi<float>(ctx);
}

template <typename T>
int64_t prefetch_policy(const pdr_ctx* ctx, int cfg)
{
    const double rows = (2.0 * (double)ctx->m + (double)ctx->n) * (double)ctx->Kp;
    return rows * sizeof(T) > kL2Bytes ? edge_prefetch_distance<T>(cfg, ctx->num_sms) : 0;
}

// The edge-kernel variant of each precision: the caller's (it must hold the
// rows in every precision the solve uses) or the library's choice.  Sets
// cfg, grid_e and n_psi; cfg = -1 for a precision whose rows no variant holds.
pdr_status select_edge_variants(pdr_ctx* ctx, const pdr_options& o)
{
    const int Kp = ctx->Kp;
    int c32, c64;
    if (o.edge_variant >= 0) {
        c32 = c64 = o.edge_variant;
        const bool need32 = o.precision != PDR_PREC_FP64, need64 = o.precision != PDR_PREC_FP32;
        if ((need32 && edge_capacity<float>(c32) < Kp) || (need64 && edge_capacity<double>(c64) < Kp))
            return ctx->fail(PDR_ERR_INVALID_ARG, "edge_variant " + std::to_string(o.edge_variant) +
                                                      " does not hold rows of K = " + std::to_string(ctx->K));
        if (edge_capacity<float>(c32) < Kp) c32 = edge_config<float>(Kp);
        if (edge_capacity<double>(c64) < Kp) c64 = edge_config<double>(Kp);
    } else {
        c32 = edge_config<float>(Kp);
        c64 = edge_config<double>(Kp);
    }
    if (c32 < 0 || (o.precision != PDR_PREC_FP32 && c64 < 0))
        return ctx->fail(PDR_ERR_UNSUPPORTED,
                         "K = " + std::to_string(ctx->K) + " exceeds the largest edge-kernel row supported by this build");
    ctx->cfg[0] = c32;
    ctx->cfg[1] = c64;
    ctx->grid_e[0] = edge_grid<float>(c32, ctx->m, ctx->num_sms);
    ctx->grid_e[1] = c64 >= 0 ? edge_grid<double>(c64, ctx->m, ctx->num_sms) : 1;
    ctx->n_psi[0] = edge_parts<float>(c32, ctx->grid_e[0]);
    ctx->n_psi[1] = c64 >= 0 ? edge_parts<double>(c64, ctx->grid_e[1]) : 1;
    // L2 prefetch of later waves' rows pays only when the rows come from HBM:
    // when both flow buffers and the heights fit in L2 (as they stay across
    // sweeps) the prefetches are pure overhead
    ctx->pf[0] = prefetch_policy<float>(ctx, c32);
    ctx->pf[1] = c64 >= 0 ? prefetch_policy<double>(ctx, c64) : 0;
    ctx->pgrid[0] = persistent_grid<float>(c32, ctx->m, ctx->n, Kp, ctx->num_sms);
    ctx->pgrid[1] = c64 >= 0 ? persistent_grid<double>(c64, ctx->m, ctx->n, Kp, ctx->num_sms) : 0;
    return PDR_OK;
}

__global__ void set_state_kernel(DevState* st, DevState v) { *st = v; }

// pdr_set_data from device arrays, the same arithmetic as the host path.
// Block 0 thread 0 checks the domain and sums the positive capacities in
// edge order (the mean positive capacity scales cap_rel, as at create time);
// nothing is written when a value is out of its domain.
__global__ void set_data_check_kernel(int64_t m, int K, const double* __restrict__ u, const double* __restrict__ d,
                                      double* __restrict__ ubar, int* __restrict__ err)
{
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    int bad = 0;
    double usum = 0.0;
    int64_t upos = 0;
    if (u)
        for (int64_t e = 0; e < m; ++e) {
            const double x = u[e];
            if (!isfinite(x) || x < 0.0) bad |= 1;
            if (x > 0.0) {
                usum += x;
                ++upos;
            }
        }
    if (d)
        for (int k = 0; k < K; ++k)
            if (!isfinite(d[k]) || !(d[k] > 0.0)) bad |= 2;
    *ubar = upos ? usum / (double)upos : 1.0;
    *err = bad;
}

__global__ void set_data_fill_kernel(int64_t m, int K, int Kp, const double* __restrict__ u,
                                     const double* __restrict__ d, const double* __restrict__ ubar,
                                     const int* __restrict__ err, double* u_d, float* u_f, double* inv_scale,
                                     float* inv_scale_f, double* dem_d, float* dem_f, double* inv_dem_d,
                                     float* inv_dem_f)
{
    if (*err) return;
    const double ub = *ubar;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u && e < m; e += stride) {
        const double x = u[e];
        const double inv = 1.0 / (x > ub ? x : ub);
        u_d[e] = x;
        u_f[e] = (float)x;
        inv_scale[e] = inv;
        inv_scale_f[e] = (float)inv;
    }
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; d && k < Kp; k += stride) {
        const double x = k < K ? d[k] : 0.0;
        dem_d[k] = x;
        dem_f[k] = (float)x;
        inv_dem_d[k] = k < K ? 1.0 / x : 0.0;
        inv_dem_f[k] = k < K ? (float)(1.0 / x) : 0.0f;
    }
}

cudaError_t launch_set_data(int64_t m, int K, int Kp, const double* u, const double* d, double* u_d, float* u_f,
                            double* inv_scale, float* inv_scale_f, double* dem_d, float* dem_f, double* inv_dem_d,
                            float* inv_dem_f, int* err, cudaStream_t stream)
{
    // the mean positive capacity sits in the slot after the error word
    double* ubar = reinterpret_cast<double*>(err) + 1;
    set_data_check_kernel<<<1, 32, 0, stream>>>(m, K, u, d, ubar, err);
    const int64_t want = ((m > Kp ? m : Kp) + 255) / 256;
    const int grid = (int)(want < 1 ? 1 : (want < 1024 ? want : 1024));
    set_data_fill_kernel<<<grid, 256, 0, stream>>>(m, K, Kp, u, d, ubar, err, u_d, u_f, inv_scale, inv_scale_f,
                                                   dem_d, dem_f, inv_dem_d, inv_dem_f);
    return cudaGetLastError();
}

pdr_status init_state(pdr_ctx* ctx, bool fresh, int stop_on_rise, bool keep_zprev = false)
{
    if (fresh) ctx->resume_pending = false;
    DevState v{};
    v.z = 0.0;
    v.z_prev = keep_zprev ? ctx->hst->z_prev : INFINITY;
    v.dz = 0.0;
    v.eps_obj = ctx->opt.eps_obj;
    v.resid_tol = ctx->opt.resid_tol;
    v.eps_rel = ctx->opt.eps_rel;
    v.t = fresh ? 0 : ctx->hst->t;
    v.max_sweeps = ctx->opt.max_sweeps;
    v.trace_len = ctx->trace_cap;
    v.evals = fresh ? 0 : ctx->hst->evals;
    v.stop = 0;
    v.reason = 0;
    v.stop_on_rise = stop_on_rise;
    // the residual-plateau rule runs with the stall rule, in the FP32 phase of
    // the tail mode, and starts its windows at this phase's first sweep
    v.plat_window = stop_on_rise ? kPlateauWindow : 0;
    v.plat_t0 = keep_zprev ? ctx->hst->plat_t0 : v.t;  // a resumed solve keeps its windows
    v.plat_cur = keep_zprev ? ctx->hst->plat_cur : INFINITY;
    v.plat_prev = keep_zprev ? ctx->hst->plat_prev : INFINITY;
    set_state_kernel<<<1, 1, 0, ctx->stream>>>(ctx->st, v);
    CK(cudaGetLastError());
    return PDR_OK;
}

pdr_status read_state(pdr_ctx* ctx)
{
    CK(cudaMemcpyAsync(ctx->hst, ctx->st, sizeof(DevState), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if (ctx->hst->fault)
        return ctx->fail(PDR_ERR_TIMEOUT, "excess kernel: a shared-memory barrier wait ran out of its time limit");
    return PDR_OK;
}

// The sweep loop as one graph: a conditional WHILE node whose body holds
// kUnroll sweeps (excess kernel, then update kernel).  For Alg. 1 the body's
// kernels are captured with programmatic dependent launch (each may be
// scheduled while its predecessor drains); if the runtime refuses that, the
// body is captured again with plain launches.
template <typename T>
bool try_build_graph(pdr_ctx* ctx, bool pdl)
{
    const int p = Prec<T>::id;
    cudaGraph_t g = nullptr;
    cudaGraphConditionalHandle h;
    cudaGraphNode_t node;
    cudaGraphNodeParams np{};
    cudaGraph_t body, captured;
    cudaGraphExec_t exec = nullptr;
    if (cudaGraphCreate(&g, 0) != cudaSuccess) goto fail;
    if (cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault) != cudaSuccess) goto fail;
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    if (cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np) != cudaSuccess) goto fail;
    body = np.conditional.phGraph_out[0];
    if (cudaStreamBeginCaptureToGraph(ctx->cap_stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) !=
        cudaSuccess)
        goto fail;
    {
        cudaError_t e1 = cudaSuccess;
        for (int q = 0; q < kUnroll && e1 == cudaSuccess; ++q) {
            SweepArgs<T> a = make_args<T>(ctx, MODE_SOLVE, 1, h, q & 1, 0);
            // the first kernel of the body follows the conditional node: plain
            e1 = launch_excess<T>(a, ctx->cap_stream, pdl && q > 0);
            if (e1 == cudaSuccess) e1 = launch_update<T>(ctx, a, ctx->cap_stream, pdl);
        }
        cudaError_t e3 = cudaStreamEndCapture(ctx->cap_stream, &captured);
        if (e1 != cudaSuccess || e3 != cudaSuccess) goto fail;
    }
    if (cudaGraphInstantiate(&exec, g, 0) != cudaSuccess) goto fail;
    ctx->graph[p] = g;
    ctx->exec[p] = exec;
    ctx->cond[p] = h;
    ctx->graph_ok[p] = true;
    ctx->graph_pdl[p] = pdl;
    return true;
fail:
    cudaGetLastError();
    if (g) cudaGraphDestroy(g);
    return false;
}

template <typename T>
pdr_status build_graph(pdr_ctx* ctx)
{
    const int p = Prec<T>::id;
    ctx->graph_tried[p] = true;
    ctx->graph_ok[p] = false;
    if (!is_gd(ctx->opt) && try_build_graph<T>(ctx, true)) return PDR_OK;
    try_build_graph<T>(ctx, false);
    return PDR_OK;  // if both failed, the host loop takes over
}

// The FP32 phase of PDR_PREC_FP32_FP64TAIL hands over to FP64 when it stopped
// on the objective rules or stalled (not on the residual rule, the sweep
// limit or a non-finite z).
bool needs_fp64_tail(int reason)
{
    return reason == STOP_OBJECTIVE || reason == STOP_RELATIVE || reason == STOP_STALL || reason == STOP_PLATEAU;
}

// Moves the current FP32 state (flows; Alg. 3/4 rates and velocities) into
// FP64 buffer 0 and makes FP64 the working precision.
pdr_status widen_to_fp64(pdr_ctx* ctx)
{
    pdr_status s = ensure_fp64(ctx);
    if (s != PDR_OK) return s;
    CK(launch_convert_f32_to_f64(ctx->f32[ctx->cur], ctx->f64[0], (int64_t)ctx->m * ctx->Kp, ctx->stream));
    if (is_gd(ctx->opt) && ctx->m > 0) {
        // learning rates (and velocities) follow the flows into FP64
        // (through a root buffer as scratch: the FP64 phase starts its root searches cold)
        CK(launch_convert_f32_to_f64(reinterpret_cast<const float*>(ctx->beta_buf[ctx->cur]), ctx->theta[0], ctx->m,
                                     ctx->stream));
        CK(cudaMemcpyAsync(ctx->beta_buf[0], ctx->theta[0], sizeof(double) * ctx->m, cudaMemcpyDeviceToDevice,
                           ctx->stream));
        if (ctx->opt.algo == PDR_ALGO_GDM) {
            s = ensure_velocity<double>(ctx);
            if (s != PDR_OK) return s;
            CK(launch_convert_f32_to_f64(ctx->v32[ctx->cur], ctx->v64[0], (int64_t)ctx->m * ctx->Kp, ctx->stream));
        }
    }
    ctx->cur = 0;
    ctx->cur_prec = 1;
    return refresh_psi<double>(ctx);
}

constexpr int64_t kPersistChunk = 1024;  // sweeps per persistent launch (even)
constexpr int64_t kBlockElems = int64_t(1) << 18;  // m x Kp up to which one cluster solves an instance
constexpr int64_t kBlockChunk = 2048;              // sweeps per launch of the cluster kernel

// Blocks of the thread-block cluster that runs an instance's whole solve:
// enough that each lane group handles at most 16 edges per sweep (1..8).
int batch_cluster_size(const pdr_ctx* c, int p);

// Shared memory of the one-block engine's shared-memory form for instance c
// in precision p, or 0 where it does not apply (a cluster of several blocks,
// or more than kBlockSmemMax bytes).
int64_t block_smem(const pdr_ctx* c, int p)
{
    if (batch_cluster_size(c, p) != 1) return 0;
    const int64_t n_psi = kBatchThreads / 32;
    const int64_t b = p == Prec<double>::id ? block_smem_bytes<double>(c->n, c->m, c->Kp, n_psi)
                                         : block_smem_bytes<float>(c->n, c->m, c->Kp, n_psi);
    return b <= kBlockSmemMax ? b : 0;
}

// The cluster engine (use_graph = 3, and the batched form's small
// instances) applies to Alg. 1 and Program (6) on a small instance whose
// edge variant is a lane-group form of at most 4 vectors per lane.
bool cluster_eligible(const pdr_ctx* ctx, int p)
{
    const int cfg = ctx->cfg[p];
    return !is_gd(ctx->opt) && ctx->m > 0 && ctx->m * (int64_t)ctx->Kp <= kBlockElems && batch_block_config(cfg) &&
           edge_plain_config(cfg) <= 5;
}

// Alg. 1 by the cluster kernel (use_graph = 3): one thread-block cluster runs
// the excess pass, the objective and stop test and the edge QPs of every
// sweep, separated by cluster barriers, for kBlockChunk sweeps per launch
// until the stop rules fire; the flows start in buffer 0.  The per-element
// arithmetic is the standalone kernels' (the batched form's engine, with one
// instance).
template <typename T>
pdr_status run_cluster(pdr_ctx* ctx, int64_t t_start)
{
    const int p = Prec<T>::id;
    if (!ctx->cl_args) {
        pdr_status st = PDR_OK;
        ctx->cl_args = dalloc<unsigned char>(ctx, sizeof(SweepArgs<double>) + 64, &st);
        if (!ctx->cl_args) return st;
    }
    SweepArgs<T>* dargs = reinterpret_cast<SweepArgs<T>*>(ctx->cl_args);
    int* dids = reinterpret_cast<int*>(ctx->cl_args + sizeof(SweepArgs<double>) + 32);
    CK(cudaMemsetAsync(dids, 0, sizeof(int), ctx->stream));  // the instance id: 0, its arguments at dargs[0]
    const int csize = batch_cluster_size(ctx, p);
    for (bool first = true;; first = false) {
        const int par = first ? 0 : (int)((ctx->hst->t - t_start) & 1);
        SweepArgs<T> a = make_args<T>(ctx, MODE_SOLVE, 0, 0, par, 0);
        a.excess_form = 0;  // the gather form, run by the cluster's blocks
        a.grid_v = csize;
        a.grid_e = csize;
        a.n_psi = csize * (kBatchThreads / 32);
        a.pf_edges = 0;
        a.l2_hints = 0;
        a.active = nullptr;
        CK(cudaMemcpyAsync(dargs, &a, sizeof(a), cudaMemcpyHostToDevice, ctx->stream));
        CK(launch_batch_block<T>(edge_plain_config(ctx->cfg[p]), dargs, dids, 1, csize, kBlockChunk, first ? 1 : 0,
                                 ctx->stream, block_smem(ctx, p)));
        const pdr_status s = read_state(ctx);  // synchronises the stream
        if (s != PDR_OK) return s;
        if (ctx->hst->stop) break;
    }
    ctx->cur = (int)((ctx->hst->t - t_start) & 1);
    // the current flows' congestion partials in the standalone kernels' layout
    return refresh_psi<T>(ctx, nullptr, true);
}

// The persistent engine applies to Alg. 1 with a lane-group variant.
bool persistent_ok(const pdr_ctx* ctx, int p)
{
    return ctx->opt.use_graph == 2 && !is_gd(ctx->opt) && ctx->pgrid[p] >= 2;
}

// Excess kernel form from the options: -1 takes the default, 0..3 that
// form; a bulk-copy form that cannot be resident on this device is refused.
// The default is bulk-copy form 2 (two stages of eight row segments, six
// blocks per SM on GB300), the fastest form measured on the grid, k-NN and
// random-digraph workloads; the gathers where it cannot be resident.
constexpr int kDefaultExcessForm = 2;
pdr_status select_excess_form(pdr_ctx* ctx, const pdr_options& o)
{
    const int v = o.excess_variant >= 0 ? o.excess_variant : (ctx->xgrid[kDefaultExcessForm] > 0 ? kDefaultExcessForm : 0);
    if (v > 0 && ctx->xgrid[v] <= 0)
        return ctx->fail(PDR_ERR_INVALID_ARG, "excess_variant " + std::to_string(v) + " cannot run on this device");
    ctx->xform = v;
    return PDR_OK;
}

// Alg. 1 by the persistent kernel: launches of kPersistChunk sweeps until the
// stop rules fire; the flows start in buffer 0.  *ran = false if the first
// cooperative launch was refused (the caller then uses the graph engine).
template <typename T>
pdr_status run_persistent(pdr_ctx* ctx, bool* ran)
{
    const int p = Prec<T>::id;
    const int grid = ctx->pgrid[p];
    SweepArgs<T> a = make_args<T>(ctx, MODE_SOLVE, 0, 0, 0, 0);
    a.excess_form = 0;  // the persistent kernel runs the gather form of the excess pass
    a.grid_v = grid;
    a.grid_e = grid - 1;
    a.n_psi = (int64_t)(grid - 1) * (kThreads / 32);
    // each warp's next edge: one round of the whole grid ahead
    a.pf_edges = (int64_t)(grid - 1) * (kThreads / edge_group_lanes(ctx->cfg[p]));
    pdr_status s = PDR_OK;
    *ran = false;
    for (int launch = 0;; ++launch) {
        CK(cudaMemsetAsync(ctx->bar, 0, sizeof(GridBarrier), ctx->stream));
        const cudaError_t le = launch_persistent<T>(a, ctx->cfg[p], grid, kPersistChunk, ctx->bar,
                                                    launch == 0 ? 1 : 0, ctx->stream);
        if (le != cudaSuccess) {
            if (launch > 0) return ctx->cuda_fail("launch_persistent", le);
            cudaGetLastError();  // e.g. too large for co-residency here: never try again
            ctx->pgrid[0] = ctx->pgrid[1] = 0;
            return PDR_OK;
        }
        *ran = true;
        GridBarrier hb{};
        CK(cudaMemcpyAsync(&hb, ctx->bar, sizeof(GridBarrier), cudaMemcpyDeviceToHost, ctx->stream));
        s = read_state(ctx);  // synchronises the stream
        if (s != PDR_OK) return s;
        if (hb.failed) return ctx->fail(PDR_ERR_TIMEOUT, "persistent sweep kernel: a grid barrier timed out");
        if (ctx->hst->stop) break;
    }
    // the other engines read the congestion partials in the standalone layout
    return refresh_psi<T>(ctx, nullptr, true);
}

// One phase of Alg. 1 in precision T, from the state set by init_state
// (whose t is t_start).  Afterwards the current flows f^(t) sit in buffer
// (t - t_start) mod 2: every sweep that does not stop swaps the buffers.
template <typename T>
pdr_status run_phase(pdr_ctx* ctx, int64_t t_start)
{
    const int p = Prec<T>::id;
    pdr_status s = ensure_velocity<T>(ctx);
    if (s != PDR_OK) return s;
    s = flows_to_buffer0<T>(ctx);
    if (s != PDR_OK) return s;
    // one instance's FP64 sweeps stay on the graph engine: one block is held
    // to one SM's FP64 rate, a small fraction of its FP32 rate on this GPU,
    // and loses to the kernels that spread a sweep over several SMs
    if (ctx->opt.use_graph == 3 && p == Prec<float>::id && cluster_eligible(ctx, p)) return run_cluster<T>(ctx, t_start);
    if (persistent_ok(ctx, p)) {
        bool ran = false;
        s = run_persistent<T>(ctx, &ran);
        if (s != PDR_OK) return s;
        if (ran) {
            ctx->cur = (int)((ctx->hst->t - t_start) & 1);
            return PDR_OK;
        }
    }
    if (ctx->opt.use_graph && !ctx->graph_tried[p]) {
        s = build_graph<T>(ctx);
        if (s != PDR_OK) return s;
    }
    if (ctx->opt.use_graph && ctx->graph_ok[p]) {
        CK(cudaGraphLaunch(ctx->exec[p], ctx->stream));
        s = read_state(ctx);
    } else {
        // host loop fallback: chunks of an even number of sweeps, then a look
        // at the stop flag (a chunk that does not stop leaves f in buffer 0)
        for (;;) {
            for (int q = 0; q < kHostChunk; ++q) {
                SweepArgs<T> a = make_args<T>(ctx, MODE_SOLVE, 0, 0, q & 1, 0);
                CK(launch_excess<T>(a, ctx->stream));
                CK(launch_update<T>(ctx, a, ctx->stream));
            }
            s = read_state(ctx);
            if (s != PDR_OK || ctx->hst->stop) break;
        }
    }
    if (s != PDR_OK) return s;
    ctx->cur = (int)((ctx->hst->t - t_start) & 1);
    // The sweep that stopped also ran its edge QPs (their output is
    // discarded) and wrote their congestion partials: recompute those of the
    // returned flows f^(t), keeping the warm starts.  A stop by the sweep cap
    // skipped those updates (final_evaluation), so its partials are still
    // the returned flows'.
    if (ctx->hst->stop && ctx->hst->reason != STOP_MAX_SWEEPS) return refresh_psi<T>(ctx, nullptr, true);
    return PDR_OK;
}

template <typename T>
pdr_status residuals_T(pdr_ctx* ctx)
{
    SweepArgs<T> a = make_args<T>(ctx, MODE_EVAL);
    const ResidIn r{ctx->u_d, ctx->dem_d, ctx->inv_deg_d, ctx->inv_dem_f};
    CK(launch_residuals<T>(a, r, ctx->r_h64, ctx->r_part, ctx->r_grid_v, ctx->r_grid_e, ctx->r_out, ctx->stream));
    CK(cudaMemcpyAsync(ctx->hr_out, ctx->r_out, sizeof(ResidOut), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return PDR_OK;
}

pdr_status residuals_into(pdr_ctx* ctx, pdr_result* r)
{
    pdr_status s = ctx->cur_prec ? residuals_T<double>(ctx) : residuals_T<float>(ctx);
    if (s != PDR_OK) return s;
    const ResidOut& o = *ctx->hr_out;
    r->z = o.z;
    r->cap_abs = o.cap_abs;
    r->cap_rel = o.cap_rel;
    r->cons_abs = o.cons_abs;
    r->cons_rel = o.cons_rel;
    r->f_min = o.f_min;
    r->margin = o.margin;
    r->margin_scale = o.margin_scale;
    const double tol = ctx->opt.resid_tol > 0.0 ? ctx->opt.resid_tol : 1e-6;
    if (ctx->isolated || o.margin > 1e-9 * o.margin_scale) r->verdict = PDR_VERDICT_INFEASIBLE;
    else if (o.cap_rel <= tol && o.cons_rel <= tol) r->verdict = PDR_VERDICT_FEASIBLE;
    else r->verdict = PDR_VERDICT_UNKNOWN;
    return PDR_OK;
}

// True for memory that only the device may dereference (device or managed
// allocations); host memory, pinned or not, is read by the host directly.
bool is_device_memory(const void* p)
{
    if (!p) return false;
    cudaPointerAttributes attr{};
    if (cudaPointerGetAttributes(&attr, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged;
}

// Copies a padded device array [rows x Kp] of T into host double [rows x K].
template <typename T>
pdr_status copy_rows_out(pdr_ctx* ctx, const T* dsrc, int64_t rows, double* out)
{
    if (rows == 0) return PDR_OK;
    std::vector<T> tmp((size_t)rows * ctx->K);
    CK(cudaMemcpy2DAsync(tmp.data(), sizeof(T) * ctx->K, dsrc, sizeof(T) * ctx->Kp, sizeof(T) * ctx->K, (size_t)rows,
                         cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    for (size_t q = 0; q < tmp.size(); ++q) out[q] = (double)tmp[q];
    return PDR_OK;
}

template <typename T>
pdr_status copy_rows_in(pdr_ctx* ctx, const double* in, int64_t rows, T* ddst)
{
    if (rows == 0) return PDR_OK;
    std::vector<T> tmp((size_t)rows * ctx->K);
    for (size_t q = 0; q < tmp.size(); ++q) tmp[q] = (T)in[q];
    CK(cudaMemcpy2DAsync(ddst, sizeof(T) * ctx->Kp, tmp.data(), sizeof(T) * ctx->K, sizeof(T) * ctx->K, (size_t)rows,
                         cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return PDR_OK;
}

pdr_status destroy_graphs(pdr_ctx* ctx)
{
    for (int p = 0; p < 2; ++p) {
        if (ctx->exec[p]) cudaGraphExecDestroy(ctx->exec[p]);
        if (ctx->graph[p]) cudaGraphDestroy(ctx->graph[p]);
        ctx->exec[p] = nullptr;
        ctx->graph[p] = nullptr;
        ctx->graph_tried[p] = false;
        ctx->graph_ok[p] = false;
    }
    return PDR_OK;
}

// Host-side checks of an instance (the domain stated in include/pdr.h);
// returns an empty string if it is valid.
std::string validate_instance(int32_t n, int64_t m, const int64_t* row_ptr, const int32_t* col, const double* u,
                              int32_t K, const int32_t* s, const int32_t* t, const double* d)
{
    if (n < 1) return "n must be >= 1";
    if (m < 0 || m > (int64_t)INT32_MAX) return "m must satisfy 0 <= m < 2^31";
    if (K < 1) return "K must be >= 1";
    if (!row_ptr || (m > 0 && (!col || !u)) || !s || !t || !d) return "NULL input array";
    if (row_ptr[0] != 0) return "row_ptr[0] must be 0";
    if (row_ptr[n] != m) return "row_ptr[n] must equal m";
    for (int32_t i = 0; i < n; ++i) {
        if (row_ptr[i + 1] < row_ptr[i]) return "row_ptr must be non-decreasing (vertex " + std::to_string(i) + ")";
        for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
            if (col[e] < 0 || col[e] >= n) return "col out of range at edge " + std::to_string(e);
            if (col[e] == i) return "self-loop at edge " + std::to_string(e);
        }
    }
    for (int64_t e = 0; e < m; ++e)
        if (!std::isfinite(u[e]) || u[e] < 0.0) return "capacity must be finite and >= 0 at edge " + std::to_string(e);
    for (int32_t k = 0; k < K; ++k) {
        if (s[k] < 0 || s[k] >= n || t[k] < 0 || t[k] >= n)
            return "commodity endpoint out of range at k = " + std::to_string(k);
        if (s[k] == t[k]) return "s_k == t_k at k = " + std::to_string(k);
        if (!std::isfinite(d[k]) || !(d[k] > 0.0)) return "demand must be finite and > 0 at k = " + std::to_string(k);
    }
    return "";
}


void release_adjoint_workspace(pdr_ctx* ctx)
{
    for (auto& w : ctx->adj_ws)
        if (w.first) cudaFree(w.first);
    ctx->adj_ws.clear();
}

// Reverse mode through T sweeps (pdr_backward), precision T.
template <typename T>
pdr_status backward_T(pdr_ctx* ctx, int64_t Tn, int32_t C, double* L, double* grad_u, double* grad_d)
{
    const size_t fm = (size_t)ctx->m * ctx->Kp, hn = (size_t)ctx->n * ctx->Kp;
    const size_t mm = (size_t)(ctx->m > 0 ? ctx->m : 1);
    const int64_t nseg = Tn > 0 ? (Tn + C - 1) / C : 0;
    const bool grads = grad_u || grad_d;
    // ckpt_every = 1: the forward pass keeps every sweep's flows f^(0..T),
    // heights h^(0..T-1) and roots (with the warm starts they leave), each
    // sweep writing its own buffers, so the backward pass recomputes nothing
    const bool keep_all = grads && C == 1;
    pdr_status st = PDR_OK;
    auto cleanup = [&]() { release_adjoint_workspace(ctx); };  // failure paths only
    size_t slot = 0;
    auto grab = [&](size_t bytes) -> void* {  // the next buffer of the kept workspace
        if (bytes == 0) bytes = 1;
        if (slot == ctx->adj_ws.size()) ctx->adj_ws.push_back({nullptr, 0});
        auto& w = ctx->adj_ws[slot];
        if (w.second < bytes) {
            if (w.first) cudaFree(w.first);
            w = {nullptr, 0};
            void* q = nullptr;
            if (cudaMalloc(&q, bytes) != cudaSuccess) {
                cudaGetLastError();
                return nullptr;
            }
            w = {q, bytes};
        }
        ++slot;
        return w.first;
    };
#define CKB(call)                                        \
    do {                                                 \
        cudaError_t _e = (call);                         \
        if (_e != cudaSuccess) {                         \
            st = ctx->cuda_fail(#call, _e);              \
            cleanup();                                   \
            return st;                                   \
        }                                                \
    } while (0)
    std::vector<T*> fs(keep_all ? Tn + 1 : 0), hs(keep_all ? Tn : 0), ths(keep_all ? Tn : 0);
    for (auto& q : fs)
        if (!(q = (T*)grab(sizeof(T) * fm))) return cleanup(), ctx->fail(PDR_ERR_OOM, "sweep-state allocation failed");
    for (auto& q : hs)
        if (!(q = (T*)grab(sizeof(T) * hn))) return cleanup(), ctx->fail(PDR_ERR_OOM, "sweep-state allocation failed");
    for (auto& q : ths)
        if (!(q = (T*)grab(sizeof(T) * 2 * mm))) return cleanup(), ctx->fail(PDR_ERR_OOM, "sweep-state allocation failed");
    // otherwise checkpoints of the flows and of the roots and warm starts at t = 0, C, 2C, ...
    const bool ckpt = grads && !keep_all;
    std::vector<T*> ck(ckpt ? nseg : 0), thck(ckpt ? nseg : 0), seg, th, hseg;
    for (auto& q : ck)
        if (!(q = (T*)grab(sizeof(T) * fm))) return cleanup(), ctx->fail(PDR_ERR_OOM, "checkpoint allocation failed");
    for (auto& q : thck)
        if (!(q = (T*)grab(sizeof(T) * 2 * mm))) return cleanup(), ctx->fail(PDR_ERR_OOM, "checkpoint allocation failed");
    T *fbar = nullptr, *cbar = nullptr, *Dbar = nullptr;
    double *ubar = nullptr, *dbar = nullptr;
    uint32_t* mask = nullptr;
    if (ckpt) {
        seg.resize(C + 1);
        th.resize(C);
        for (auto& q : seg)
            if (!(q = (T*)grab(sizeof(T) * fm))) return cleanup(), ctx->fail(PDR_ERR_OOM, "segment allocation failed");
        for (auto& q : th)
            if (!(q = (T*)grab(sizeof(T) * mm))) return cleanup(), ctx->fail(PDR_ERR_OOM, "segment allocation failed");
        hseg.resize(C);  // the heights of every sweep of a segment, kept from its recomputation
        for (auto& q : hseg)
            if (!(q = (T*)grab(sizeof(T) * hn))) return cleanup(), ctx->fail(PDR_ERR_OOM, "segment allocation failed");
    }
    if (grads) {
        fbar = (T*)grab(sizeof(T) * fm);
        cbar = (T*)grab(sizeof(T) * fm);
        Dbar = (T*)grab(sizeof(T) * hn);
        ubar = (double*)grab(sizeof(double) * mm);
        dbar = (double*)grab(sizeof(double) * ctx->K);
        mask = (uint32_t*)grab(sizeof(uint32_t) * mm * backward_mask_words(ctx->Kp, 16 / sizeof(T)));
        if (!fbar || !cbar || !Dbar || !ubar || !dbar || !mask)
            return cleanup(), ctx->fail(PDR_ERR_OOM, "adjoint allocation failed");
    }
    // forward from f = 0 (pdr_backward reset the flows), cold roots
    if (keep_all) {
        CKB(cudaMemcpyAsync(fs[0], Prec<T>::f(ctx, ctx->cur), sizeof(T) * fm, cudaMemcpyDeviceToDevice, ctx->stream));
        for (int64_t t = 0; t < Tn; ++t) {
            SweepArgs<T> a = make_args<T>(ctx, MODE_FORCED);
            a.f = fs[t];
            a.f_out = fs[t + 1];
            a.h = hs[t];
            if (t > 0) a.theta_in = ths[t - 1];
            a.theta = ths[t];
            CKB(launch_excess<T>(a, ctx->stream));
            CKB(launch_edge<T>(a, ctx->cfg[Prec<T>::id], ctx->stream));
        }
        if (Tn > 0) {  // f^(T) and the last roots become the current state
            CKB(cudaMemcpyAsync(Prec<T>::f(ctx, ctx->cur), fs[Tn], sizeof(T) * fm, cudaMemcpyDeviceToDevice,
                                ctx->stream));
            CKB(cudaMemcpyAsync(ctx->theta[ctx->cur], ths[Tn - 1], sizeof(T) * 2 * ctx->m, cudaMemcpyDeviceToDevice,
                                ctx->stream));
        }
    }
    for (int64_t t = 0; !keep_all && t < Tn; ++t) {
        if (grads && t % C == 0) {  // the flows and the warm starts sweep t reads
            CKB(cudaMemcpyAsync(ck[t / C], Prec<T>::f(ctx, ctx->cur), sizeof(T) * fm, cudaMemcpyDeviceToDevice, ctx->stream));
            CKB(cudaMemcpyAsync(thck[t / C], ctx->theta[ctx->cur], sizeof(T) * 2 * ctx->m, cudaMemcpyDeviceToDevice,
                                ctx->stream));
        }
        SweepArgs<T> a = make_args<T>(ctx, MODE_FORCED);
        CKB(launch_excess<T>(a, ctx->stream));
        CKB(launch_edge<T>(a, ctx->cfg[Prec<T>::id], ctx->stream));
        ctx->cur ^= 1;
    }
    // L = z(f^(T)) and the seeds
    {
        SweepArgs<T> a = make_args<T>(ctx, MODE_EVAL);
        CKB(launch_excess<T>(a, ctx->stream));
        CKB(launch_finalize<T>(a, ctx->stream));
        if (grads) CKB(launch_seed<T>(a, fbar, ubar, dbar, ctx->num_sms, ctx->stream));
    }
    st = read_state(ctx);
    if (st != PDR_OK) return cleanup(), st;
    if (L) *L = ctx->hst->z;
    // backward from the kept sweeps
    for (int64_t t = Tn - 1; keep_all && t >= 0; --t) {
        SweepArgs<T> a = make_args<T>(ctx, MODE_EVAL);
        a.f = fs[t];
        a.h = hs[t];
        CKB(launch_backward_sweep<T>(a, ths[t], fbar, cbar, Dbar, ubar, dbar, mask, t == Tn - 1 ? 0 : 1,
                                     ctx->num_sms, ctx->stream));
    }
    // or segment by segment from the last
    for (int64_t sgi = nseg - 1; ckpt && sgi >= 0; --sgi) {
        const int64_t t0 = sgi * C, t1 = (t0 + C < Tn) ? t0 + C : Tn;
        CKB(cudaMemcpyAsync(seg[0], ck[sgi], sizeof(T) * fm, cudaMemcpyDeviceToDevice, ctx->stream));
        CKB(cudaMemcpyAsync(ctx->theta[0], thck[sgi], sizeof(T) * 2 * ctx->m, cudaMemcpyDeviceToDevice, ctx->stream));
        for (int64_t t = t0; t < t1; ++t) {  // recompute f^(t0+1..t1-1); keep each sweep's heights and roots
            const int rb = (int)((t - t0) & 1);
            SweepArgs<T> a = make_args<T>(ctx, MODE_FORCED);
            a.f = seg[t - t0];
            a.f_out = seg[t - t0 + 1];
            a.h = hseg[t - t0];
            a.theta_in = reinterpret_cast<const T*>(ctx->theta[rb]);
            a.theta = reinterpret_cast<T*>(ctx->theta[rb ^ 1]);
            CKB(launch_excess<T>(a, ctx->stream));
            CKB(launch_edge<T>(a, ctx->cfg[Prec<T>::id], ctx->stream));
            CKB(cudaMemcpyAsync(th[t - t0], ctx->theta[rb ^ 1], sizeof(T) * ctx->m, cudaMemcpyDeviceToDevice,
                                ctx->stream));
        }
        for (int64_t t = t1 - 1; t >= t0; --t) {
            SweepArgs<T> a = make_args<T>(ctx, MODE_EVAL);
            a.f = seg[t - t0];
            a.h = hseg[t - t0];  // h^(t), from the recomputation above
            // the first step reads the seed; later ones form dL/df^(t+1) from cbar and Dbar
            CKB(launch_backward_sweep<T>(a, th[t - t0], fbar, cbar, Dbar, ubar, dbar, mask, t == Tn - 1 ? 0 : 1,
                                         ctx->num_sms, ctx->stream));
        }
    }
    // the gradients go to host or device memory alike (unified addressing)
    if (grad_u && ctx->m > 0)
        CKB(cudaMemcpyAsync(grad_u, ubar, sizeof(double) * ctx->m, cudaMemcpyDefault, ctx->stream));
    if (grad_d) CKB(cudaMemcpyAsync(grad_d, dbar, sizeof(double) * ctx->K, cudaMemcpyDefault, ctx->stream));
    CKB(cudaStreamSynchronize(ctx->stream));
#undef CKB
    // a time limit that ran out in a kernel of the recomputed segments or of
    // the backward pass
    st = read_state(ctx);
    if (st != PDR_OK) return cleanup(), st;
    // f^(T) stays the current flows; partials and state follow it
    st = refresh_psi<T>(ctx);
    if (st != PDR_OK) return st;
    return init_state(ctx, true, 0);
}

}  // namespace

extern "C" {

pdr_status pdr_default_options(pdr_options* opt)
{
    if (!opt) return PDR_ERR_INVALID_ARG;
    fill_defaults(opt);
    return PDR_OK;
}

const char* pdr_last_error(const pdr_ctx* ctx) { return ctx ? ctx->err.c_str() : g_create_error.c_str(); }

void pdr_destroy(pdr_ctx* ctx)
{
    if (!ctx) return;
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    destroy_graphs(ctx);
    void* dev[] = {ctx->row_ptr, ctx->in_ptr, ctx->inc_ptr, ctx->inc, ctx->work, ctx->col, ctx->src, ctx->in_eid,
                   ctx->deg, ctx->s, ctx->t,
                   ctx->u_d, ctx->dem_d, ctx->inv_scale, ctx->u_f, ctx->dem_f, ctx->inv_dem_f, ctx->inv_dem_d,
                   ctx->f32[0], ctx->f32[1], ctx->h32, ctx->f64[0], ctx->f64[1], ctx->h64, ctx->part_h, ctx->part_cons, ctx->part_capb, ctx->part_psi, ctx->part_cap, ctx->st,
                   ctx->trace, ctx->inv_scale_f, ctx->inv_deg_f, ctx->inv_deg_d, ctx->theta[0], ctx->theta[1],
                   ctx->beta_buf[0], ctx->beta_buf[1], ctx->v32[0], ctx->v32[1], ctx->v64[0], ctx->v64[1],
                   ctx->r_h64, ctx->r_part, ctx->r_out, ctx->psi_tmp, ctx->bar, ctx->xv_start[1], ctx->xv_start[2], ctx->xv_start[3],
                   ctx->xv_start[4], ctx->xv_start[5],
                   ctx->data_err, ctx->cl_args};
    for (void* p : dev)
        if (p) cudaFree(p);
    release_adjoint_workspace(ctx);
    if (ctx->hst) cudaFreeHost(ctx->hst);
    if (ctx->hr_out) cudaFreeHost(ctx->hr_out);
    if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
    cudaGetLastError();
    delete ctx;
}

pdr_status pdr_create(int32_t n, int64_t m, const int64_t* row_ptr, const int32_t* col, const double* u, int32_t K,
                      const int32_t* s, const int32_t* t, const double* d, const pdr_options* opt, void* stream,
                      pdr_ctx** out)
{
    g_create_error.clear();
    auto bad = [](const std::string& msg) {
        g_create_error = msg;
        return PDR_ERR_INVALID_ARG;
    };
    if (!out) return bad("out is NULL");
    *out = nullptr;
    {
        const std::string why = validate_instance(n, m, row_ptr, col, u, K, s, t, d);
        if (!why.empty()) return bad(why);
    }
    pdr_options o;
    fill_defaults(&o);
    if (opt) o = *opt;
    std::string why;
    if (!options_ok(&o, &why)) return bad(why);

    pdr_ctx* ctx = new pdr_ctx();
    ctx->n = n;
    ctx->m = m;
    ctx->K = K;
    ctx->Kp = round_up4(K);
    ctx->opt = o;
    ctx->stream = static_cast<cudaStream_t>(stream);
    auto give_up = [&](pdr_status code) {
        g_create_error = ctx->err;
        pdr_destroy(ctx);
        return code;
    };
#define CKC(call)                                                    \
    do {                                                             \
        cudaError_t _e = (call);                                     \
        if (_e != cudaSuccess) return give_up(ctx->cuda_fail(#call, _e)); \
    } while (0)
    int dev = 0;
    CKC(cudaGetDevice(&dev));
    CKC(cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, dev));
    CKC(cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));

    const int Kp = ctx->Kp;
    {
        const pdr_status vs = select_edge_variants(ctx, o);
        if (vs != PDR_OK) return give_up(vs);
    }
    ctx->grid_v[0] = excess_grid(n, Kp, 4, ctx->num_sms, excess_resident_blocks<float>());
    ctx->grid_v[1] = excess_grid(n, Kp, 2, ctx->num_sms, excess_resident_blocks<double>());
    ctx->r_grid_v = excess_grid(n, Kp, 1, ctx->num_sms, 8);
    for (int f = 1; f < kExcessForms; ++f) {
        const int r32 = excess_bulk_resident_blocks<float>(f), r64 = excess_bulk_resident_blocks<double>(f);
        const int64_t r = r32 < r64 ? r32 : r64;
        const int64_t g = r * ctx->num_sms < n ? r * ctx->num_sms : n;
        ctx->xgrid[f] = r > 0 ? (int)(g < 1 ? 1 : g) : 0;
    }
    {
        const pdr_status xs = select_excess_form(ctx, o);
        if (xs != PDR_OK) return give_up(xs);
    }
    {
        int64_t we = (m * 32 + 255) / 256;
        int64_t cap = (int64_t)ctx->num_sms * 8;
        ctx->r_grid_e = (int)(we < 1 ? 1 : (we < cap ? we : cap));
    }

    pdr_status st = PDR_OK;
#define ALLOC(ptr, T, count)                            \
    do {                                                \
        ptr = dalloc<T>(ctx, (size_t)(count), &st);     \
        if (!ptr) return give_up(st);                   \
    } while (0)
    ALLOC(ctx->row_ptr, int64_t, n + 1);
    ALLOC(ctx->in_ptr, int64_t, n + 1);
    ALLOC(ctx->work, int64_t, 2 * (int64_t)n + 1);
    ALLOC(ctx->col, int32_t, m);
    ALLOC(ctx->src, int32_t, m);
    ALLOC(ctx->in_eid, int32_t, m);
    ALLOC(ctx->inc_ptr, int64_t, n + 1);
    ALLOC(ctx->inc, int32_t, 2 * m);
    ALLOC(ctx->deg, int32_t, n);
    ALLOC(ctx->s, int32_t, Kp);
    ALLOC(ctx->t, int32_t, Kp);
    ALLOC(ctx->u_d, double, m);
    ALLOC(ctx->u_f, float, m);
    ALLOC(ctx->inv_scale, double, m);
    ALLOC(ctx->inv_scale_f, float, m);
    ALLOC(ctx->inv_deg_f, float, n);
    ALLOC(ctx->inv_deg_d, double, n);
    ALLOC(ctx->theta[0], double, 2 * (m > 0 ? m : 1));
    ALLOC(ctx->theta[1], double, 2 * (m > 0 ? m : 1));
    ALLOC(ctx->beta_buf[0], double, m);
    ALLOC(ctx->beta_buf[1], double, m);
    ALLOC(ctx->dem_d, double, Kp);
    ALLOC(ctx->dem_f, float, Kp);
    ALLOC(ctx->inv_dem_d, double, Kp);
    ALLOC(ctx->inv_dem_f, float, Kp);
    int gv = ctx->grid_v[0] > ctx->grid_v[1] ? ctx->grid_v[0] : ctx->grid_v[1];
    for (int f = 1; f < kExcessForms; ++f) {
        if (ctx->xgrid[f] > gv) gv = ctx->xgrid[f];
        if (ctx->xgrid[f] > 0) ALLOC(ctx->xv_start[f], int32_t, ctx->xgrid[f] + 1);
    }
    int64_t np = ctx->n_psi[0] > ctx->n_psi[1] ? ctx->n_psi[0] : ctx->n_psi[1];
    if (np < m + 8) np = m + 8;  // any standalone variant writes at most m + 8 edge partials
    // the persistent kernel: at most 8 blocks of 256 threads per SM, one
    // partial per block and per warp
    if (gv < 8 * ctx->num_sms) gv = 8 * ctx->num_sms;
    if (np < 64 * (int64_t)ctx->num_sms) np = 64 * (int64_t)ctx->num_sms;
    ALLOC(ctx->part_h, double, gv);
    ALLOC(ctx->part_cons, double, gv);
    ALLOC(ctx->part_capb, double, gv);
    ALLOC(ctx->part_psi, double, np);
    ALLOC(ctx->part_cap, double, np);
    ALLOC(ctx->st, DevState, 1);
    ALLOC(ctx->bar, GridBarrier, 1);
    ctx->trace_cap = o.trace_len;
    ALLOC(ctx->trace, double, ctx->trace_cap > 0 ? ctx->trace_cap : 1);
    ALLOC(ctx->r_h64, double, (size_t)n * Kp);
    ALLOC(ctx->r_part, double, resid_part_count(ctx->r_grid_v, ctx->r_grid_e));
    ALLOC(ctx->r_out, ResidOut, 1);
    ALLOC(ctx->psi_tmp, double, m);
    ALLOC(ctx->data_err, int, 4);  // error word, then the mean positive capacity (8-byte aligned)
    CKC(cudaMallocHost(&ctx->hst, sizeof(DevState)));
    CKC(cudaMallocHost(&ctx->hr_out, sizeof(ResidOut)));
    std::memset(ctx->hst, 0, sizeof(DevState));

    // host-side staging of the instance
    std::vector<int32_t> sp(Kp, -1), tp(Kp, -1);
    std::vector<double> dp(Kp, 0.0);
    std::vector<float> dpf(Kp, 0.0f), idf(Kp, 0.0f);
    std::vector<double> idd(Kp, 0.0);
    for (int k = 0; k < K; ++k) {
        sp[k] = s[k];
        tp[k] = t[k];
        dp[k] = d[k];
        dpf[k] = (float)d[k];
        idd[k] = 1.0 / d[k];
        idf[k] = (float)(1.0 / d[k]);
    }
    double usum = 0.0;
    int64_t upos = 0;
    for (int64_t e = 0; e < m; ++e)
        if (u[e] > 0.0) {
            usum += u[e];
            ++upos;
        }
    const double ubar = upos ? usum / (double)upos : 1.0;
    std::vector<double> inv(m > 0 ? m : 1);
    std::vector<float> uf(m > 0 ? m : 1), invf(m > 0 ? m : 1);
    for (int64_t e = 0; e < m; ++e) {
        inv[e] = 1.0 / (u[e] > ubar ? u[e] : ubar);
        invf[e] = (float)inv[e];
        uf[e] = (float)u[e];
    }
    CKC(cudaMemcpyAsync(ctx->row_ptr, row_ptr, sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice, ctx->stream));
    if (m > 0) {
        CKC(cudaMemcpyAsync(ctx->col, col, sizeof(int32_t) * m, cudaMemcpyHostToDevice, ctx->stream));
        CKC(cudaMemcpyAsync(ctx->u_d, u, sizeof(double) * m, cudaMemcpyHostToDevice, ctx->stream));
        CKC(cudaMemcpyAsync(ctx->u_f, uf.data(), sizeof(float) * m, cudaMemcpyHostToDevice, ctx->stream));
        CKC(cudaMemcpyAsync(ctx->inv_scale, inv.data(), sizeof(double) * m, cudaMemcpyHostToDevice, ctx->stream));
        CKC(cudaMemcpyAsync(ctx->inv_scale_f, invf.data(), sizeof(float) * m, cudaMemcpyHostToDevice, ctx->stream));
    }
    CKC(cudaMemcpyAsync(ctx->s, sp.data(), sizeof(int32_t) * Kp, cudaMemcpyHostToDevice, ctx->stream));
    CKC(cudaMemcpyAsync(ctx->t, tp.data(), sizeof(int32_t) * Kp, cudaMemcpyHostToDevice, ctx->stream));
    CKC(cudaMemcpyAsync(ctx->dem_d, dp.data(), sizeof(double) * Kp, cudaMemcpyHostToDevice, ctx->stream));
    CKC(cudaMemcpyAsync(ctx->dem_f, dpf.data(), sizeof(float) * Kp, cudaMemcpyHostToDevice, ctx->stream));
    CKC(cudaMemcpyAsync(ctx->inv_dem_d, idd.data(), sizeof(double) * Kp, cudaMemcpyHostToDevice, ctx->stream));
    CKC(cudaMemcpyAsync(ctx->inv_dem_f, idf.data(), sizeof(float) * Kp, cudaMemcpyHostToDevice, ctx->stream));
    CKC(build_adjacency(n, m, ctx->row_ptr, ctx->col, ctx->src, ctx->in_ptr, ctx->in_eid, ctx->inc_ptr, ctx->inc,
                        ctx->deg, ctx->work, ctx->stream));
    for (int f = 1; f < kExcessForms; ++f)
        if (ctx->xgrid[f] > 0) CKC(launch_excess_split(ctx->inc_ptr, n, ctx->xgrid[f], ctx->xv_start[f], ctx->stream));
    // degree-0 commodity endpoints make the instance infeasible outright
    {
        std::vector<int32_t> hdeg(n);
        CKC(cudaMemcpyAsync(hdeg.data(), ctx->deg, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, ctx->stream));
        CKC(cudaStreamSynchronize(ctx->stream));
        for (int k = 0; k < K; ++k)
            if (hdeg[s[k]] == 0 || hdeg[t[k]] == 0) ctx->isolated = true;
        std::vector<double> idd_v(n);
        std::vector<float> idf_v(n);
        for (int32_t i = 0; i < n; ++i) {
            idd_v[i] = hdeg[i] > 0 ? 1.0 / (double)hdeg[i] : 0.0;
            idf_v[i] = hdeg[i] > 0 ? 1.0f / (float)hdeg[i] : 0.0f;
        }
        CKC(cudaMemcpyAsync(ctx->inv_deg_d, idd_v.data(), sizeof(double) * n, cudaMemcpyHostToDevice, ctx->stream));
        CKC(cudaMemcpyAsync(ctx->inv_deg_f, idf_v.data(), sizeof(float) * n, cudaMemcpyHostToDevice, ctx->stream));
        CKC(cudaStreamSynchronize(ctx->stream));
    }
    ctx->cur_prec = start_prec(o);
    resolve_gd_params(ctx);
    st = ctx->cur_prec ? ensure_fp64(ctx) : ensure_fp32(ctx);
    if (st != PDR_OK) return give_up(st);
    st = init_gd_state_current(ctx);
    if (st != PDR_OK) return give_up(st);
    st = refresh_psi_current(ctx);
    if (st != PDR_OK) return give_up(st);
    st = init_state(ctx, true, 0);
    if (st != PDR_OK) return give_up(st);
    CKC(cudaStreamSynchronize(ctx->stream));
#undef ALLOC
#undef CKC
    *out = ctx;
    return PDR_OK;
}

pdr_status pdr_set_options(pdr_ctx* ctx, const pdr_options* opt)
{
    if (!ctx) return PDR_ERR_INVALID_ARG;
    pdr_options o;
    fill_defaults(&o);
    if (opt) o = *opt;
    std::string why;
    if (!options_ok(&o, &why)) return ctx->fail(PDR_ERR_INVALID_ARG, why);
    const bool variant_changed = o.edge_variant != ctx->opt.edge_variant ||
                                 (o.precision != PDR_PREC_FP32 && ctx->cfg[1] < 0);
    if (variant_changed) {
        const pdr_status vs = select_edge_variants(ctx, o);  // writes nothing on failure
        if (vs != PDR_OK) return vs;
        destroy_graphs(ctx);  // the graphs captured the old launch shapes
    }
    if (o.trace_len != ctx->trace_cap) {
        if (ctx->trace) cudaFree(ctx->trace);
        pdr_status st = PDR_OK;
        ctx->trace = dalloc<double>(ctx, o.trace_len > 0 ? o.trace_len : 1, &st);
        if (!ctx->trace) return st;
        ctx->trace_cap = o.trace_len;
        destroy_graphs(ctx);  // the graphs captured the old trace pointer
    }
    const bool gd_changed = o.algo != ctx->opt.algo || o.beta_init != ctx->opt.beta_init ||
                            o.beta_min != ctx->opt.beta_min || o.beta_max != ctx->opt.beta_max ||
                            o.alpha_inc != ctx->opt.alpha_inc || o.alpha_dec != ctx->opt.alpha_dec ||
                            o.gamma != ctx->opt.gamma;
    if (o.excess_variant != ctx->opt.excess_variant) {
        const pdr_status xs = select_excess_form(ctx, o);
        if (xs != PDR_OK) return xs;
        destroy_graphs(ctx);
    }
    if (gd_changed || o.use_graph != ctx->opt.use_graph) destroy_graphs(ctx);  // captured arguments change
    const int want = start_prec(o);
    if (want != ctx->cur_prec && o.precision != PDR_PREC_FP32_FP64TAIL) {
        // move the current flows into the new working precision
        std::vector<double> f((size_t)ctx->m * ctx->K);
        pdr_status s = pdr_flows(ctx, f.data());
        if (s != PDR_OK) return s;
        ctx->opt = o;
        resolve_gd_params(ctx);
        s = want ? ensure_fp64(ctx) : ensure_fp32(ctx);
        if (s != PDR_OK) return s;
        ctx->cur_prec = want;
        return pdr_set_flows(ctx, f.data());
    }
    ctx->opt = o;
    resolve_gd_params(ctx);
    if (gd_changed) {
        // a new algorithm or new rates: learning rates and velocities restart, the flows stay
        pdr_status s = flows_to_buffer0_current(ctx);
        if (s != PDR_OK) return s;
        s = init_gd_state_current(ctx);
        if (s != PDR_OK) return s;
    }
    // a new variant writes its congestion partials in another layout
    if (variant_changed) return refresh_psi_current(ctx);
    return PDR_OK;
}

pdr_status pdr_reset(pdr_ctx* ctx)
{
    if (!ctx) return PDR_ERR_INVALID_ARG;
    ctx->cur_prec = start_prec(ctx->opt);
    pdr_status s = ctx->cur_prec ? ensure_fp64(ctx) : ensure_fp32(ctx);
    if (s != PDR_OK) return s;
    const size_t fm = (size_t)ctx->m * ctx->Kp;
    ctx->cur = 0;
    if (ctx->cur_prec) CK(cudaMemsetAsync(ctx->f64[0], 0, sizeof(double) * (fm ? fm : 1), ctx->stream));
    else CK(cudaMemsetAsync(ctx->f32[0], 0, sizeof(float) * (fm ? fm : 1), ctx->stream));
    s = init_gd_state_current(ctx);
    if (s != PDR_OK) return s;
    s = refresh_psi_current(ctx);
    if (s != PDR_OK) return s;
    s = init_state(ctx, true, 0);
    if (s != PDR_OK) return s;
    return read_state(ctx);
}

pdr_status pdr_set_flows(pdr_ctx* ctx, const double* f)
{
    if (!ctx || (!f && ctx->m > 0)) return ctx ? ctx->fail(PDR_ERR_INVALID_ARG, "f is NULL") : PDR_ERR_INVALID_ARG;
    if (ctx->opt.precision != PDR_PREC_FP32_FP64TAIL) ctx->cur_prec = start_prec(ctx->opt);
    pdr_status s = ctx->cur_prec ? ensure_fp64(ctx) : ensure_fp32(ctx);
    if (s != PDR_OK) return s;
    ctx->cur = 0;
    s = ctx->cur_prec ? copy_rows_in<double>(ctx, f, ctx->m, ctx->f64[0])
                      : copy_rows_in<float>(ctx, f, ctx->m, ctx->f32[0]);
    if (s != PDR_OK) return s;
    s = init_gd_state_current(ctx);
    if (s != PDR_OK) return s;
    s = refresh_psi_current(ctx);
    if (s != PDR_OK) return s;
    s = init_state(ctx, true, 0);
    if (s != PDR_OK) return s;
    return read_state(ctx);
}

pdr_status pdr_flows(pdr_ctx* ctx, double* f)
{
    if (!ctx || (!f && ctx->m > 0)) return ctx ? ctx->fail(PDR_ERR_INVALID_ARG, "f is NULL") : PDR_ERR_INVALID_ARG;
    if (ctx->m == 0) return PDR_OK;
    // A destination the GPU can write (pinned host memory, device or managed
    // memory) receives the widened rows straight from a kernel; pageable
    // host memory goes through a host-side staging copy.
    cudaPointerAttributes attr{};
    const cudaError_t ae = cudaPointerGetAttributes(&attr, f);
    if (ae != cudaSuccess) cudaGetLastError();
    if (ae == cudaSuccess && attr.type != cudaMemoryTypeUnregistered && attr.devicePointer) {
        double* dst = static_cast<double*>(attr.devicePointer);
        if (ctx->cur_prec) CK(launch_widen_rows<double>(ctx->f64[ctx->cur], ctx->m, ctx->K, ctx->Kp, dst, ctx->stream));
        else CK(launch_widen_rows<float>(ctx->f32[ctx->cur], ctx->m, ctx->K, ctx->Kp, dst, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        return PDR_OK;
    }
    return ctx->cur_prec ? copy_rows_out<double>(ctx, ctx->f64[ctx->cur], ctx->m, f)
                         : copy_rows_out<float>(ctx, ctx->f32[ctx->cur], ctx->m, f);
}

// ------------------------------------------------------------------ checkpoint / resume
//
// A checkpoint holds, in the working precision and in this order: a header,
// the flows (m x Kp), the warm starts (m), the Alg. 3/4 rates (m, Alg. 3/4
// only), the Alg. 4 velocities (m x Kp, Alg. 4 only) and the objective
// trace so far.  Restoring it and solving on gives the flows of the
// uninterrupted solve bit for bit (a sweep depends only on these).

namespace {
constexpr uint32_t kStateMagic = 0x53524450u;  // "PDRS"
constexpr uint32_t kStateVersion = 2;

struct StateHeader {
    uint32_t magic, version;
    int32_t n, K, Kp, algo, prec, stopped;
    int64_t m, t, evals, t_widen, ntrace;
    double z_prev, z;
    int64_t plat_t0;            // residual-plateau window of the tail mode's FP32 phase
    double plat_cur, plat_prev;
};

struct StateLayout {
    int64_t f, theta, beta, v, trace, total;  // byte counts (total includes the header)
};

StateLayout state_layout(const pdr_ctx* ctx, int prec, int64_t ntrace)
{
    const int64_t sz = prec ? 8 : 4, fm = (int64_t)ctx->m * ctx->Kp;
    StateLayout L{};
    L.f = sz * fm;
    L.theta = 2 * sz * ctx->m;  // roots and warm starts
    L.beta = is_gd(ctx->opt) ? sz * ctx->m : 0;
    L.v = ctx->opt.algo == PDR_ALGO_GDM ? sz * fm : 0;
    L.trace = 8 * ntrace;
    L.total = (int64_t)sizeof(StateHeader) + L.f + L.theta + L.beta + L.v + L.trace;
    return L;
}

int64_t trace_kept(const pdr_ctx* ctx)
{
    const int64_t e = ctx->hst->evals;
    return e < ctx->trace_cap ? e : ctx->trace_cap;
}

void* dev_v(pdr_ctx* ctx, int prec, int b) { return prec ? (void*)ctx->v64[b] : (void*)ctx->v32[b]; }
void* dev_f(pdr_ctx* ctx, int prec, int b) { return prec ? (void*)ctx->f64[b] : (void*)ctx->f32[b]; }
}  // namespace

pdr_status pdr_state_size(pdr_ctx* ctx, int64_t* bytes)
{
    if (!ctx || !bytes) return ctx ? ctx->fail(PDR_ERR_INVALID_ARG, "bytes is NULL") : PDR_ERR_INVALID_ARG;
    pdr_status s = read_state(ctx);
    if (s != PDR_OK) return s;
    *bytes = state_layout(ctx, ctx->cur_prec, trace_kept(ctx)).total;
    return PDR_OK;
}

pdr_status pdr_get_state(pdr_ctx* ctx, void* buf, int64_t bytes)
{
    if (!ctx || !buf) return ctx ? ctx->fail(PDR_ERR_INVALID_ARG, "buf is NULL") : PDR_ERR_INVALID_ARG;
    pdr_status s = read_state(ctx);
    if (s != PDR_OK) return s;
    const int prec = ctx->cur_prec;
    const int64_t ntrace = trace_kept(ctx);
    const StateLayout L = state_layout(ctx, prec, ntrace);
    if (bytes < L.total) return ctx->fail(PDR_ERR_INVALID_ARG, "buffer smaller than pdr_state_size");
    StateHeader h{};
    h.magic = kStateMagic;
    h.version = kStateVersion;
    h.n = ctx->n;
    h.K = ctx->K;
    h.Kp = ctx->Kp;
    h.algo = ctx->opt.algo;
    h.prec = prec;
    h.stopped = ctx->hst->stop;
    h.m = ctx->m;
    h.t = ctx->hst->t;
    h.evals = ctx->hst->evals;
    h.t_widen = ctx->t_widen;
    h.ntrace = ntrace;
    h.z_prev = ctx->hst->z_prev;
    h.z = ctx->hst->z;
    h.plat_t0 = ctx->hst->plat_t0;
    h.plat_cur = ctx->hst->plat_cur;
    h.plat_prev = ctx->hst->plat_prev;
    char* out = static_cast<char*>(buf);
    std::memcpy(out, &h, sizeof h);
    char* q = out + sizeof h;
    if (L.f) CK(cudaMemcpyAsync(q, dev_f(ctx, prec, ctx->cur), L.f, cudaMemcpyDeviceToHost, ctx->stream));
    q += L.f;
    if (L.theta) CK(cudaMemcpyAsync(q, ctx->theta[ctx->cur], L.theta, cudaMemcpyDeviceToHost, ctx->stream));
    q += L.theta;
    if (L.beta) CK(cudaMemcpyAsync(q, ctx->beta_buf[ctx->cur], L.beta, cudaMemcpyDeviceToHost, ctx->stream));
    q += L.beta;
    if (L.v) {
        const void* v = dev_v(ctx, prec, ctx->cur);
        if (v) CK(cudaMemcpyAsync(q, v, L.v, cudaMemcpyDeviceToHost, ctx->stream));
        else std::memset(q, 0, (size_t)L.v);  // no Alg. 4 sweep has run: v = 0
    }
    q += L.v;
    if (L.trace) CK(cudaMemcpyAsync(q, ctx->trace, L.trace, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return PDR_OK;
}

pdr_status pdr_set_state(pdr_ctx* ctx, const void* buf, int64_t bytes)
{
    if (!ctx || !buf) return ctx ? ctx->fail(PDR_ERR_INVALID_ARG, "buf is NULL") : PDR_ERR_INVALID_ARG;
    if (bytes < (int64_t)sizeof(StateHeader)) return ctx->fail(PDR_ERR_INVALID_ARG, "buffer too small");
    StateHeader h;
    std::memcpy(&h, buf, sizeof h);
    if (h.magic != kStateMagic || h.version != kStateVersion)
        return ctx->fail(PDR_ERR_INVALID_ARG, "not a checkpoint of this library version");
    if (h.n != ctx->n || h.m != ctx->m || h.K != ctx->K || h.Kp != ctx->Kp)
        return ctx->fail(PDR_ERR_INVALID_ARG, "checkpoint of an instance of other sizes");
    if (h.algo != ctx->opt.algo) return ctx->fail(PDR_ERR_INVALID_ARG, "checkpoint of another algorithm");
    if (h.prec != 0 && h.prec != 1) return ctx->fail(PDR_ERR_INVALID_ARG, "bad precision in checkpoint");
    if (h.prec == 1 && ctx->opt.precision == PDR_PREC_FP32)
        return ctx->fail(PDR_ERR_INVALID_ARG, "an FP64 checkpoint needs precision FP64 or FP32 with FP64 tail");
    if (h.prec == 0 && ctx->opt.precision == PDR_PREC_FP64)
        return ctx->fail(PDR_ERR_INVALID_ARG, "an FP32 checkpoint needs precision FP32 or FP32 with FP64 tail");
    if (h.t < 0 || h.evals < 0 || h.ntrace < 0 || h.ntrace > h.evals)
        return ctx->fail(PDR_ERR_INVALID_ARG, "bad counters in checkpoint");
    const StateLayout L = state_layout(ctx, h.prec, h.ntrace);
    if (bytes < L.total) return ctx->fail(PDR_ERR_INVALID_ARG, "checkpoint truncated");
    ctx->cur_prec = h.prec;
    pdr_status s = h.prec ? ensure_fp64(ctx) : ensure_fp32(ctx);
    if (s != PDR_OK) return s;
    if (L.v) {
        s = h.prec ? ensure_velocity<double>(ctx) : ensure_velocity<float>(ctx);
        if (s != PDR_OK) return s;
    }
    ctx->cur = 0;
    const char* q = static_cast<const char*>(buf) + sizeof h;
    if (L.f) CK(cudaMemcpyAsync(dev_f(ctx, h.prec, 0), q, L.f, cudaMemcpyHostToDevice, ctx->stream));
    q += L.f;
    if (L.theta) CK(cudaMemcpyAsync(ctx->theta[0], q, L.theta, cudaMemcpyHostToDevice, ctx->stream));
    q += L.theta;
    if (L.beta) CK(cudaMemcpyAsync(ctx->beta_buf[0], q, L.beta, cudaMemcpyHostToDevice, ctx->stream));
    q += L.beta;
    if (L.v) CK(cudaMemcpyAsync(dev_v(ctx, h.prec, 0), q, L.v, cudaMemcpyHostToDevice, ctx->stream));
    q += L.v;
    const int64_t nt = h.ntrace < ctx->trace_cap ? h.ntrace : ctx->trace_cap;
    if (nt > 0) CK(cudaMemcpyAsync(ctx->trace, q, 8 * nt, cudaMemcpyHostToDevice, ctx->stream));
    s = h.prec ? refresh_psi<double>(ctx, nullptr, true) : refresh_psi<float>(ctx, nullptr, true);
    if (s != PDR_OK) return s;
    // The device state between sweeps t-1 and t.  A checkpoint taken after a
    // stop holds f^(t) with sweep t evaluated but not applied: the resumed
    // solve evaluates it again, in the same trace slot.
    DevState v{};
    v.z = h.z;
    v.z_prev = h.z_prev;
    v.eps_obj = ctx->opt.eps_obj;
    v.resid_tol = ctx->opt.resid_tol;
    v.eps_rel = ctx->opt.eps_rel;
    v.t = h.t;
    v.max_sweeps = ctx->opt.max_sweeps;
    v.trace_len = ctx->trace_cap;
    v.evals = h.stopped && h.evals > 0 ? h.evals - 1 : h.evals;
    v.plat_t0 = h.plat_t0;
    v.plat_cur = h.plat_cur;
    v.plat_prev = h.plat_prev;
    set_state_kernel<<<1, 1, 0, ctx->stream>>>(ctx->st, v);
    CK(cudaGetLastError());
    s = read_state(ctx);
    if (s != PDR_OK) return s;
    ctx->t_widen = h.t_widen;
    ctx->resume_pending = true;
    return PDR_OK;
}

pdr_status pdr_debug_fail_alloc(int64_t nth)
{
    if (nth < 0) return PDR_ERR_INVALID_ARG;
    g_fail_alloc.store(nth);
    return PDR_OK;
}

pdr_status pdr_debug_wait(pdr_ctx* ctx, int64_t cycles, int32_t hold_end)
{
    if (!ctx) return PDR_ERR_INVALID_ARG;
    if (cycles < 1000 || cycles > kWaitCycles)
        return ctx->fail(PDR_ERR_INVALID_ARG, "cycles must lie in [1000, 2^32]");
    if (hold_end != 0 && hold_end != 1) return ctx->fail(PDR_ERR_INVALID_ARG, "hold_end must be 0 or 1");
    ctx->wait_cycles = cycles;
    ctx->hold_end = hold_end;
    destroy_graphs(ctx);  // the graphs captured the old launch arguments
    return PDR_OK;
}

pdr_status pdr_debug_barrier(pdr_ctx* ctx, int64_t limit_ns, int32_t withhold)
{
    if (!ctx) return PDR_ERR_INVALID_ARG;
    if (limit_ns < 100000 || limit_ns > kBarrierNs)
        return ctx->fail(PDR_ERR_INVALID_ARG, "limit_ns must lie in [1e5, 2e9]");
    if (withhold != 0 && withhold != 1) return ctx->fail(PDR_ERR_INVALID_ARG, "withhold must be 0 or 1");
    ctx->barrier_ns = limit_ns;
    ctx->hold_barrier = withhold;
    return PDR_OK;
}

pdr_status pdr_backward(pdr_ctx* ctx, int64_t T, int32_t ckpt_every, double* L, double* grad_u, double* grad_d)
{
    if (!ctx) return PDR_ERR_INVALID_ARG;
    if (T < 0 || ckpt_every < 1) return ctx->fail(PDR_ERR_INVALID_ARG, "T must be >= 0 and ckpt_every >= 1");
    if (is_gd(ctx->opt))
        return ctx->fail(PDR_ERR_INVALID_ARG,
                         "the differentiated form runs Alg. 1 (algo = PDR_ALGO_ESO or PDR_ALGO_CK)");
    pdr_status s = pdr_reset(ctx);  // f = 0 in the starting precision
    if (s != PDR_OK) return s;
    return ctx->cur_prec ? backward_T<double>(ctx, T, ckpt_every, L, grad_u, grad_d)
                         : backward_T<float>(ctx, T, ckpt_every, L, grad_u, grad_d);
}

pdr_status pdr_set_data(pdr_ctx* ctx, const double* u, const double* d)
{
    if (!ctx) return PDR_ERR_INVALID_ARG;
    // arrays the host cannot read directly (device or managed memory) are
    // checked and converted on the device
    if (is_device_memory(u) || is_device_memory(d)) {
        if ((u && !is_device_memory(u)) || (d && !is_device_memory(d)))
            return ctx->fail(PDR_ERR_INVALID_ARG, "u and d must both be host or both be device memory");
        int bad = 0;
        CK(launch_set_data(ctx->m, ctx->K, ctx->Kp, u, d, ctx->u_d, ctx->u_f, ctx->inv_scale, ctx->inv_scale_f,
                           ctx->dem_d, ctx->dem_f, ctx->inv_dem_d, ctx->inv_dem_f, ctx->data_err, ctx->stream));
        CK(cudaMemcpyAsync(&bad, ctx->data_err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        if (bad & 1) return ctx->fail(PDR_ERR_INVALID_ARG, "capacities must be finite and >= 0 (nothing changed)");
        if (bad & 2) return ctx->fail(PDR_ERR_INVALID_ARG, "demands must be finite and > 0 (nothing changed)");
        return refresh_psi_current(ctx);
    }
    if (u)
        for (int64_t e = 0; e < ctx->m; ++e)
            if (!std::isfinite(u[e]) || u[e] < 0.0)
                return ctx->fail(PDR_ERR_INVALID_ARG, "capacity must be finite and >= 0 at edge " + std::to_string(e));
    if (d)
        for (int32_t k = 0; k < ctx->K; ++k)
            if (!std::isfinite(d[k]) || !(d[k] > 0.0))
                return ctx->fail(PDR_ERR_INVALID_ARG, "demand must be finite and > 0 at k = " + std::to_string(k));
    if (u && ctx->m > 0) {
        double usum = 0.0;
        int64_t upos = 0;
        for (int64_t e = 0; e < ctx->m; ++e)
            if (u[e] > 0.0) {
                usum += u[e];
                ++upos;
            }
        const double ubar = upos ? usum / (double)upos : 1.0;
        std::vector<double> inv(ctx->m);
        std::vector<float> uf(ctx->m), invf(ctx->m);
        for (int64_t e = 0; e < ctx->m; ++e) {
            inv[e] = 1.0 / (u[e] > ubar ? u[e] : ubar);
            invf[e] = (float)inv[e];
            uf[e] = (float)u[e];
        }
        CK(cudaMemcpyAsync(ctx->u_d, u, sizeof(double) * ctx->m, cudaMemcpyHostToDevice, ctx->stream));
        CK(cudaMemcpyAsync(ctx->u_f, uf.data(), sizeof(float) * ctx->m, cudaMemcpyHostToDevice, ctx->stream));
        CK(cudaMemcpyAsync(ctx->inv_scale, inv.data(), sizeof(double) * ctx->m, cudaMemcpyHostToDevice, ctx->stream));
        CK(cudaMemcpyAsync(ctx->inv_scale_f, invf.data(), sizeof(float) * ctx->m, cudaMemcpyHostToDevice,
                           ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
    }
    if (d) {
        const int Kp = ctx->Kp;
        std::vector<double> dp(Kp, 0.0), idd(Kp, 0.0);
        std::vector<float> dpf(Kp, 0.0f), idf(Kp, 0.0f);
        for (int k = 0; k < ctx->K; ++k) {
            dp[k] = d[k];
            dpf[k] = (float)d[k];
            idd[k] = 1.0 / d[k];
            idf[k] = (float)(1.0 / d[k]);
        }
        CK(cudaMemcpyAsync(ctx->dem_d, dp.data(), sizeof(double) * Kp, cudaMemcpyHostToDevice, ctx->stream));
        CK(cudaMemcpyAsync(ctx->dem_f, dpf.data(), sizeof(float) * Kp, cudaMemcpyHostToDevice, ctx->stream));
        CK(cudaMemcpyAsync(ctx->inv_dem_d, idd.data(), sizeof(double) * Kp, cudaMemcpyHostToDevice, ctx->stream));
        CK(cudaMemcpyAsync(ctx->inv_dem_f, idf.data(), sizeof(float) * Kp, cudaMemcpyHostToDevice, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
    }
    return refresh_psi_current(ctx);
}

pdr_status pdr_flow_rows(pdr_ctx* ctx, int32_t which, const int64_t* edges, int64_t count, double* out)
{
    if (!ctx || count < 0 || (count > 0 && (!edges || !out)) || (which != 0 && which != 1))
        return ctx ? ctx->fail(PDR_ERR_INVALID_ARG, "bad row request") : PDR_ERR_INVALID_ARG;
    if (which == 1 && ctx->opt.algo != PDR_ALGO_GDM)
        return ctx->fail(PDR_ERR_INVALID_ARG, "velocities exist only for Alg. 4");
    for (int64_t q = 0; q < count; ++q)
        if (edges[q] < 0 || edges[q] >= ctx->m)
            return ctx->fail(PDR_ERR_INVALID_ARG, "edge id out of range at " + std::to_string(q));
    if (which == 1) {
        pdr_status s = ctx->cur_prec ? ensure_velocity<double>(ctx) : ensure_velocity<float>(ctx);
        if (s != PDR_OK) return s;
    }
    const int K = ctx->K;
    if (ctx->cur_prec) {
        const double* base = which ? ctx->v64[ctx->cur] : ctx->f64[ctx->cur];
        for (int64_t q = 0; q < count; ++q)
            CK(cudaMemcpyAsync(out + q * K, base + edges[q] * ctx->Kp, sizeof(double) * K, cudaMemcpyDeviceToHost,
                               ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        return PDR_OK;
    }
    const float* base = which ? ctx->v32[ctx->cur] : ctx->f32[ctx->cur];
    std::vector<float> tmp((size_t)count * K);
    for (int64_t q = 0; q < count; ++q)
        CK(cudaMemcpyAsync(tmp.data() + q * K, base + edges[q] * ctx->Kp, sizeof(float) * K, cudaMemcpyDeviceToHost,
                           ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    for (size_t q = 0; q < tmp.size(); ++q) out[q] = tmp[q];
    return PDR_OK;
}

pdr_status pdr_gd_state(pdr_ctx* ctx, double* beta, double* v)
{
    if (!ctx) return PDR_ERR_INVALID_ARG;
    if (!is_gd(ctx->opt))
        return ctx->fail(PDR_ERR_INVALID_ARG, "the context runs Alg. 1 or its capacity-kept form (no learning rates)");
    const int b = ctx->cur;
    if (beta && ctx->m > 0) {
        if (ctx->cur_prec) {
            CK(cudaMemcpyAsync(beta, ctx->beta_buf[b], sizeof(double) * ctx->m, cudaMemcpyDeviceToHost, ctx->stream));
            CK(cudaStreamSynchronize(ctx->stream));
        } else {
            std::vector<float> tmp(ctx->m);
            CK(cudaMemcpyAsync(tmp.data(), ctx->beta_buf[b], sizeof(float) * ctx->m, cudaMemcpyDeviceToHost,
                               ctx->stream));
            CK(cudaStreamSynchronize(ctx->stream));
            for (int64_t e = 0; e < ctx->m; ++e) beta[e] = tmp[e];
        }
    }
    if (v) {
        if (ctx->opt.algo != PDR_ALGO_GDM) {
            std::memset(v, 0, sizeof(double) * (size_t)ctx->m * ctx->K);
        } else {
            pdr_status s = ctx->cur_prec ? ensure_velocity<double>(ctx) : ensure_velocity<float>(ctx);
            if (s != PDR_OK) return s;
            s = ctx->cur_prec ? copy_rows_out<double>(ctx, ctx->v64[b], ctx->m, v)
                              : copy_rows_out<float>(ctx, ctx->v32[b], ctx->m, v);
            if (s != PDR_OK) return s;
        }
    }
    return PDR_OK;
}

pdr_status pdr_set_gd_state(pdr_ctx* ctx, const double* beta, const double* v)
{
    if (!ctx || (!beta && ctx->m > 0)) return ctx ? ctx->fail(PDR_ERR_INVALID_ARG, "beta is NULL") : PDR_ERR_INVALID_ARG;
    if (!is_gd(ctx->opt))
        return ctx->fail(PDR_ERR_INVALID_ARG, "the context runs Alg. 1 or its capacity-kept form (no learning rates)");
    for (int64_t e = 0; e < ctx->m; ++e)
        if (!(beta[e] > 0.0) || !std::isfinite(beta[e]))
            return ctx->fail(PDR_ERR_INVALID_ARG, "beta must be finite and > 0 at edge " + std::to_string(e));
    pdr_status s = flows_to_buffer0_current(ctx);
    if (s != PDR_OK) return s;
    if (ctx->m > 0) {
        if (ctx->cur_prec) {
            CK(cudaMemcpyAsync(ctx->beta_buf[0], beta, sizeof(double) * ctx->m, cudaMemcpyHostToDevice, ctx->stream));
        } else {
            std::vector<float> tmp(beta, beta + ctx->m);
            CK(cudaMemcpyAsync(ctx->beta_buf[0], tmp.data(), sizeof(float) * ctx->m, cudaMemcpyHostToDevice,
                               ctx->stream));
        }
        CK(cudaStreamSynchronize(ctx->stream));
    }
    if (ctx->opt.algo == PDR_ALGO_GDM) {
        s = ctx->cur_prec ? ensure_velocity<double>(ctx) : ensure_velocity<float>(ctx);
        if (s != PDR_OK) return s;
        const size_t fm = (size_t)ctx->m * ctx->Kp;
        if (!v) {
            if (ctx->cur_prec) CK(cudaMemsetAsync(ctx->v64[0], 0, sizeof(double) * (fm ? fm : 1), ctx->stream));
            else CK(cudaMemsetAsync(ctx->v32[0], 0, sizeof(float) * (fm ? fm : 1), ctx->stream));
        } else {
            s = ctx->cur_prec ? copy_rows_in<double>(ctx, v, ctx->m, ctx->v64[0])
                              : copy_rows_in<float>(ctx, v, ctx->m, ctx->v32[0]);
            if (s != PDR_OK) return s;
        }
    }
    CK(cudaStreamSynchronize(ctx->stream));
    return PDR_OK;
}

pdr_status pdr_heights(pdr_ctx* ctx, double* h)
{
    if (!ctx || !h) return ctx ? ctx->fail(PDR_ERR_INVALID_ARG, "h is NULL") : PDR_ERR_INVALID_ARG;
    if (ctx->cur_prec) {
        CK(launch_excess<double>(make_args<double>(ctx, MODE_EVAL), ctx->stream));
        return copy_rows_out<double>(ctx, ctx->h64, ctx->n, h);
    }
    CK(launch_excess<float>(make_args<float>(ctx, MODE_EVAL), ctx->stream));
    return copy_rows_out<float>(ctx, ctx->h32, ctx->n, h);
}

pdr_status pdr_congestion(pdr_ctx* ctx, double* psi)
{
    if (!ctx || (!psi && ctx->m > 0)) return ctx ? ctx->fail(PDR_ERR_INVALID_ARG, "psi is NULL") : PDR_ERR_INVALID_ARG;
    if (ctx->m == 0) return PDR_OK;
    pdr_status s;
    if (ctx->cur_prec) {
        double* tmp = static_cast<double*>(ctx->psi_tmp);
        s = refresh_psi<double>(ctx, tmp);
        if (s != PDR_OK) return s;
        CK(cudaMemcpyAsync(psi, tmp, sizeof(double) * ctx->m, cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        return PDR_OK;
    }
    float* tmp = static_cast<float*>(ctx->psi_tmp);
    s = refresh_psi<float>(ctx, tmp);
    if (s != PDR_OK) return s;
    std::vector<float> hv(ctx->m);
    CK(cudaMemcpyAsync(hv.data(), tmp, sizeof(float) * ctx->m, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    for (int64_t e = 0; e < ctx->m; ++e) psi[e] = (double)hv[e];
    return PDR_OK;
}

pdr_status pdr_objective(pdr_ctx* ctx, double* z)
{
    if (!ctx || !z) return ctx ? ctx->fail(PDR_ERR_INVALID_ARG, "z is NULL") : PDR_ERR_INVALID_ARG;
    if (ctx->cur_prec) {
        CK(launch_excess<double>(make_args<double>(ctx, MODE_EVAL), ctx->stream));
        CK(launch_finalize<double>(make_args<double>(ctx, MODE_EVAL), ctx->stream));
    } else {
        CK(launch_excess<float>(make_args<float>(ctx, MODE_EVAL), ctx->stream));
        CK(launch_finalize<float>(make_args<float>(ctx, MODE_EVAL), ctx->stream));
    }
    pdr_status s = read_state(ctx);
    if (s != PDR_OK) return s;
    *z = ctx->hst->z;
    return PDR_OK;
}

pdr_status pdr_adjacency(pdr_ctx* ctx, int64_t* in_ptr, int32_t* in_eid, int32_t* deg)
{
    if (!ctx) return PDR_ERR_INVALID_ARG;
    if (in_ptr) CK(cudaMemcpyAsync(in_ptr, ctx->in_ptr, sizeof(int64_t) * (ctx->n + 1), cudaMemcpyDeviceToHost, ctx->stream));
    if (in_eid && ctx->m > 0)
        CK(cudaMemcpyAsync(in_eid, ctx->in_eid, sizeof(int32_t) * ctx->m, cudaMemcpyDeviceToHost, ctx->stream));
    if (deg) CK(cudaMemcpyAsync(deg, ctx->deg, sizeof(int32_t) * ctx->n, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return PDR_OK;
}

pdr_status pdr_sweeps(pdr_ctx* ctx, int64_t count)
{
    if (!ctx) return PDR_ERR_INVALID_ARG;
    if (count < 0) return ctx->fail(PDR_ERR_INVALID_ARG, "count must be >= 0");
    pdr_status s = read_state(ctx);
    if (s != PDR_OK) return s;
    s = init_state(ctx, false, 0);  // t continues (it drives the Alg. 3 / Alg. 4 schedule)
    if (s != PDR_OK) return s;
    s = ctx->cur_prec ? ensure_velocity<double>(ctx) : ensure_velocity<float>(ctx);
    if (s != PDR_OK) return s;
    for (int64_t q = 0; q < count; ++q) {
        const int par = (int)(q & 1);
        if (ctx->cur_prec) {
            SweepArgs<double> a = make_args<double>(ctx, MODE_FORCED, 0, 0, par);
            CK(launch_excess<double>(a, ctx->stream));
            CK(launch_update<double>(ctx, a, ctx->stream));
        } else {
            SweepArgs<float> a = make_args<float>(ctx, MODE_FORCED, 0, 0, par);
            CK(launch_excess<float>(a, ctx->stream));
            CK(launch_update<float>(ctx, a, ctx->stream));
        }
    }
    ctx->cur ^= (int)(count & 1);
    return read_state(ctx);
}

// pdr_sweeps with CUDA events around every kernel launch, in chunks of up
// to kTimeChunk sweeps (one stream synchronisation per chunk).
pdr_status pdr_time_sweeps(pdr_ctx* ctx, int64_t count, double* ms_excess, double* ms_update)
{
    if (!ctx || !ms_excess || !ms_update) return PDR_ERR_INVALID_ARG;
    if (count < 1) return ctx->fail(PDR_ERR_INVALID_ARG, "count must be >= 1");
    constexpr int kTimeChunk = 256;
    pdr_status s = read_state(ctx);
    if (s != PDR_OK) return s;
    s = init_state(ctx, false, 0);
    if (s != PDR_OK) return s;
    s = ctx->cur_prec ? ensure_velocity<double>(ctx) : ensure_velocity<float>(ctx);
    if (s != PDR_OK) return s;
    std::vector<cudaEvent_t> ev(3 * kTimeChunk, nullptr);
    auto cleanup = [&]() {
        for (cudaEvent_t e : ev)
            if (e) cudaEventDestroy(e);
    };
    double tx = 0.0, tu = 0.0;
    for (cudaEvent_t& e : ev)
        if (cudaEventCreate(&e) != cudaSuccess) return cleanup(), ctx->fail(PDR_ERR_CUDA, "cudaEventCreate failed");
    for (int64_t q0 = 0; q0 < count; q0 += kTimeChunk) {
        const int64_t nq = count - q0 < kTimeChunk ? count - q0 : kTimeChunk;
        for (int64_t j = 0; j < nq; ++j) {
            const int par = (int)((q0 + j) & 1);
            cudaError_t e = cudaEventRecord(ev[3 * j], ctx->stream);
            if (ctx->cur_prec) {
                SweepArgs<double> a = make_args<double>(ctx, MODE_FORCED, 0, 0, par);
                if (e == cudaSuccess) e = launch_excess<double>(a, ctx->stream);
                if (e == cudaSuccess) e = cudaEventRecord(ev[3 * j + 1], ctx->stream);
                if (e == cudaSuccess) e = launch_update<double>(ctx, a, ctx->stream);
            } else {
                SweepArgs<float> a = make_args<float>(ctx, MODE_FORCED, 0, 0, par);
                if (e == cudaSuccess) e = launch_excess<float>(a, ctx->stream);
                if (e == cudaSuccess) e = cudaEventRecord(ev[3 * j + 1], ctx->stream);
                if (e == cudaSuccess) e = launch_update<float>(ctx, a, ctx->stream);
            }
            if (e == cudaSuccess) e = cudaEventRecord(ev[3 * j + 2], ctx->stream);
            if (e != cudaSuccess) return cleanup(), ctx->cuda_fail("timed sweep", e);
        }
        cudaError_t e = cudaStreamSynchronize(ctx->stream);
        for (int64_t j = 0; j < nq && e == cudaSuccess; ++j) {
            float a = 0.f, b = 0.f;
            e = cudaEventElapsedTime(&a, ev[3 * j], ev[3 * j + 1]);
            if (e == cudaSuccess) e = cudaEventElapsedTime(&b, ev[3 * j + 1], ev[3 * j + 2]);
            tx += a;
            tu += b;
        }
        if (e != cudaSuccess) return cleanup(), ctx->cuda_fail("timed sweep events", e);
    }
    cleanup();
    ctx->cur ^= (int)(count & 1);
    *ms_excess = tx / (double)count;
    *ms_update = tu / (double)count;
    return read_state(ctx);
}

pdr_status pdr_solve(pdr_ctx* ctx, pdr_result* out)
{
    if (!ctx) return PDR_ERR_INVALID_ARG;
    const auto t0 = std::chrono::steady_clock::now();
    const bool tail = ctx->opt.precision == PDR_PREC_FP32_FP64TAIL;
    const bool resume = ctx->resume_pending;  // continue a restored checkpoint
    ctx->resume_pending = false;
    pdr_status s = init_state(ctx, !resume, (tail && ctx->cur_prec == 0) ? 1 : 0, resume);
    if (s != PDR_OK) return s;
    if (!resume) ctx->t_widen = -1;
    const int64_t t_start = resume ? ctx->hst->t : 0;
    s = ctx->cur_prec ? run_phase<double>(ctx, t_start) : run_phase<float>(ctx, t_start);
    if (s != PDR_OK) return s;
    const int r = ctx->hst->reason;
    const int reason32 = (tail && ctx->cur_prec == 0) ? r : (tail ? ctx->reason_fp32 : -1);
    if (tail && ctx->cur_prec == 0 && needs_fp64_tail(r)) {
        ctx->t_widen = ctx->hst->t;
        s = widen_to_fp64(ctx);
        if (s != PDR_OK) return s;
        s = init_state(ctx, false, 0);
        if (s != PDR_OK) return s;
        s = run_phase<double>(ctx, ctx->hst->t);
        if (s != PDR_OK) return s;
    }
    pdr_result res{};
    res.sweeps = ctx->hst->t;
    res.sweeps_fp64 = ctx->cur_prec ? ctx->hst->t - (ctx->t_widen >= 0 ? ctx->t_widen : 0) : 0;
    res.dz = ctx->hst->dz;
    res.stop_reason = ctx->hst->reason;
    res.stop_reason_fp32 = reason32;
    ctx->reason_fp32 = reason32;
    s = residuals_into(ctx, &res);
    if (s != PDR_OK) return s;
    res.ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    ctx->last = res;
    if (out) *out = res;
    if (res.stop_reason == STOP_NUMERIC) return ctx->fail(PDR_ERR_NUMERIC, "the objective became non-finite");
    return PDR_OK;
}

pdr_status pdr_residuals(pdr_ctx* ctx, pdr_result* out)
{
    if (!ctx || !out) return ctx ? ctx->fail(PDR_ERR_INVALID_ARG, "out is NULL") : PDR_ERR_INVALID_ARG;
    pdr_result res = ctx->last;
    pdr_status s = residuals_into(ctx, &res);
    if (s != PDR_OK) return s;
    *out = res;
    return PDR_OK;
}

pdr_status pdr_trace(pdr_ctx* ctx, double* z, int64_t len, int64_t* count)
{
    if (!ctx || !count || (len > 0 && !z)) return ctx ? ctx->fail(PDR_ERR_INVALID_ARG, "bad trace arguments")
                                                      : PDR_ERR_INVALID_ARG;
    pdr_status s = read_state(ctx);
    if (s != PDR_OK) return s;
    int64_t have = ctx->hst->evals < ctx->trace_cap ? ctx->hst->evals : ctx->trace_cap;
    if (have > len) have = len;
    if (have > 0) {
        CK(cudaMemcpyAsync(z, ctx->trace, sizeof(double) * have, cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
    }
    *count = have;
    return PDR_OK;
}

pdr_status pdr_sizes(const pdr_ctx* ctx, int32_t* n, int64_t* m, int32_t* K, int32_t* Kp)
{
    if (!ctx) return PDR_ERR_INVALID_ARG;
    if (n) *n = ctx->n;
    if (m) *m = ctx->m;
    if (K) *K = ctx->K;
    if (Kp) *Kp = ctx->Kp;
    return PDR_OK;
}

int32_t pdr_num_edge_variants(void) { return num_edge_configs(); }

int32_t pdr_edge_variant_capacity(int32_t v, int32_t precision, int32_t* pipelined)
{
    if (v < 0 || v >= num_edge_configs() || (precision != PDR_PREC_FP32 && precision != PDR_PREC_FP64)) return -1;
    if (pipelined) *pipelined = edge_config_pipelined(v) ? 1 : edge_config_staged(v) ? 2 : 0;
    return precision == PDR_PREC_FP32 ? edge_capacity<float>(v) : edge_capacity<double>(v);
}

pdr_status pdr_time_kernel(pdr_ctx* ctx, int32_t which, int32_t launches, int64_t flush_bytes, double* ms)
{
    if (!ctx || !ms) return PDR_ERR_INVALID_ARG;
    if ((which != 0 && which != 1) || launches < 1 || flush_bytes < 0)
        return ctx->fail(PDR_ERR_INVALID_ARG, "which must be 0 or 1, launches >= 1, flush_bytes >= 0");
    if (which == 0 && ctx->m == 0) return ctx->fail(PDR_ERR_INVALID_ARG, "no edges");
    const bool f64 = ctx->cur_prec == 1;
    void* flush = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    double total = 0.0;
    pdr_status status = PDR_OK;
    auto cleanup = [&]() {
        if (flush) cudaFree(flush);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
    };
#define CKT(call)                                     \
    do {                                              \
        cudaError_t _e = (call);                      \
        if (_e != cudaSuccess) {                      \
            status = ctx->cuda_fail(#call, _e);       \
            cleanup();                                \
            return status;                            \
        }                                             \
    } while (0)
    CKT(cudaEventCreate(&e0));
    CKT(cudaEventCreate(&e1));
    if (flush_bytes > 0) CKT(cudaMalloc(&flush, (size_t)flush_bytes));
    // the QP launches run the decision block, which advances the counter:
    // the device state is put back afterwards
    {
        const pdr_status s = read_state(ctx);
        if (s != PDR_OK) return cleanup(), s;
    }
    const DevState saved = *ctx->hst;
    // heights of the current flows for the QP launches
    if (f64) CKT(launch_excess<double>(make_args<double>(ctx, MODE_EVAL), ctx->stream));
    else CKT(launch_excess<float>(make_args<float>(ctx, MODE_EVAL), ctx->stream));
    for (int q = 0; q < launches; ++q) {
        if (flush) CKT(cudaMemsetAsync(flush, q & 0xff, (size_t)flush_bytes, ctx->stream));
        CKT(cudaEventRecord(e0, ctx->stream));
        if (which == 0) {
            // reads the current flows and the roots of the sweep that made
            // them (the warm starts of the solve's next sweep), writes the
            // other buffers: every launch repeats that next sweep
            if (f64) CKT(launch_update<double>(ctx, make_args<double>(ctx, MODE_FORCED), ctx->stream));
            else CKT(launch_update<float>(ctx, make_args<float>(ctx, MODE_FORCED), ctx->stream));
        } else {
            if (f64) CKT(launch_excess<double>(make_args<double>(ctx, MODE_EVAL), ctx->stream));
            else CKT(launch_excess<float>(make_args<float>(ctx, MODE_EVAL), ctx->stream));
        }
        CKT(cudaEventRecord(e1, ctx->stream));
        CKT(cudaEventSynchronize(e1));
        float el = 0.f;
        CKT(cudaEventElapsedTime(&el, e0, e1));
        total += el;
    }
    {
        // restore the congestion partials of the current flows; the roots
        // that warm-start the next sweep (theta[cur]) were only read
        pdr_status s = f64 ? refresh_psi<double>(ctx, nullptr, true) : refresh_psi<float>(ctx, nullptr, true);
        if (s != PDR_OK) {
            cleanup();
            return s;
        }
    }
    set_state_kernel<<<1, 1, 0, ctx->stream>>>(ctx->st, saved);
    CKT(cudaGetLastError());
    CKT(cudaStreamSynchronize(ctx->stream));
#undef CKT
    cleanup();
    *ms = total / launches;
    return read_state(ctx);
}

}  // extern "C"

// ------------------------------------------------------------------ batched form

struct pdr_batch {
    int32_t count = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t cap_stream = nullptr;
    std::vector<cudaStream_t> pool;  // capture streams: one branch per instance
    std::vector<pdr_ctx*> ctx;
    std::vector<int32_t> tuned_cfg;
    std::vector<double> tuned_us;
    unsigned int* active = nullptr;  // device counter of running instances
    // one graph per precision, over the instances it was captured for
    cudaGraph_t graph[2] = {nullptr, nullptr};
    cudaGraphExec_t exec[2] = {nullptr, nullptr};
    std::vector<char> graph_mask[2];
    bool graph_tried[2] = {false, false}, graph_ok[2] = {false, false};
    // one-block-per-instance engine: the instances one block solves at speed
    void* bargs[2] = {nullptr, nullptr};  // device SweepArgs<float> / <double> [count]
    int* bids = nullptr;                  // device instance ids [count], grouped by variant
    void* hstage = nullptr;               // pinned staging of the arguments and ids
};

namespace {

constexpr int kBatchUnroll = 2;  // sweeps per instance per iteration of the batch's while loop
constexpr int kBatchPool = 32;   // capture streams

pdr_status batch_fail(pdr_status code, const std::string& msg)
{
    pdr::set_thread_error(msg);
    return code;
}

// Times the edge-kernel variants that hold this instance's rows (the
// smallest three plain forms by capacity and, for Alg. 2, the smallest
// pipelined form) and keeps the fastest.  Launches read the
// current flows and write the other buffer, so the state is unchanged.
template <typename T>
pdr_status autotune(pdr_ctx* ctx, int32_t* best_cfg, double* best_us)
{
    const int p = Prec<T>::id;
    std::vector<int> cand;
    bool pipe = false;
    for (int c = 0; c < num_edge_configs(); ++c) {
        if (edge_capacity<T>(c) < ctx->Kp) continue;
        if (edge_config_pipelined(c)) {
            if (!pipe && !is_gd(ctx->opt)) cand.push_back(c);
            pipe = true;
        } else if ((int)cand.size() < 3) {
            cand.push_back(c);
        }
    }
    *best_cfg = ctx->cfg[p];
    *best_us = -1.0;
    if (ctx->m == 0 || cand.size() <= 1) return PDR_OK;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    CK(launch_excess<T>(make_args<T>(ctx, MODE_EVAL), ctx->stream));
    double best = 1e30;
    for (int c : cand) {
        ctx->cfg[p] = c;
        ctx->grid_e[p] = edge_grid<T>(c, ctx->m, ctx->num_sms);
        ctx->n_psi[p] = edge_parts<T>(c, ctx->grid_e[p]);
        ctx->pf[p] = prefetch_policy<T>(ctx, c);
        double tot = 0.0;
        for (int r = 0; r < 4; ++r) {
            cudaEventRecord(e0, ctx->stream);
            launch_update<T>(ctx, make_args<T>(ctx, MODE_FORCED), ctx->stream);
            cudaEventRecord(e1, ctx->stream);
            cudaError_t err = cudaEventSynchronize(e1);
            if (err != cudaSuccess) {
                cudaEventDestroy(e0);
                cudaEventDestroy(e1);
                return ctx->cuda_fail("autotune", err);
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (r > 0) tot += ms;  // the first launch warms up
        }
        const double us = tot / 3.0 * 1e3;
        if (us < best) {
            best = us;
            *best_cfg = c;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ctx->cfg[p] = *best_cfg;
    ctx->grid_e[p] = edge_grid<T>(*best_cfg, ctx->m, ctx->num_sms);
    ctx->n_psi[p] = edge_parts<T>(*best_cfg, ctx->grid_e[p]);
    ctx->pf[p] = prefetch_policy<T>(ctx, *best_cfg);
    ctx->pgrid[p] = persistent_grid<T>(*best_cfg, ctx->m, ctx->n, ctx->Kp, ctx->num_sms);
    *best_us = best;
    destroy_graphs(ctx);
    pdr_status s = refresh_psi<T>(ctx);
    if (s != PDR_OK) return s;
    return init_state(ctx, true, 0);
}

void batch_destroy_graph(pdr_batch* b, int p)
{
    if (b->exec[p]) cudaGraphExecDestroy(b->exec[p]);
    if (b->graph[p]) cudaGraphDestroy(b->graph[p]);
    b->exec[p] = nullptr;
    b->graph[p] = nullptr;
    b->graph_tried[p] = b->graph_ok[p] = false;
    b->graph_mask[p].clear();
}

template <typename T>
SweepArgs<T> batch_args(pdr_batch* b, pdr_ctx* ctx, int use_cond, cudaGraphConditionalHandle h, int par)
{
    SweepArgs<T> a = make_args<T>(ctx, MODE_SOLVE, use_cond, h, par, 0);
    a.active = b->active;
    return a;
}

// One graph: a conditional while node whose body forks one branch per
// running instance (kBatchUnroll sweeps each) and joins them.
template <typename T>
void batch_build_graph(pdr_batch* b, const std::vector<char>& run)
{
    const int p = Prec<T>::id;
    b->graph_tried[p] = true;
    b->graph_mask[p] = run;
    cudaGraph_t g = nullptr;
    cudaGraphConditionalHandle h;
    cudaGraphNode_t node;
    cudaGraphNodeParams np{};
    cudaGraph_t body, captured;
    cudaGraphExec_t exec = nullptr;
    std::vector<cudaEvent_t> ev;
    bool ok = true;
    if (cudaGraphCreate(&g, 0) != cudaSuccess) goto fail;
    if (cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault) != cudaSuccess) goto fail;
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    if (cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np) != cudaSuccess) goto fail;
    body = np.conditional.phGraph_out[0];
    ev.resize(b->pool.size() + 1);
    for (auto& e : ev)
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) ok = false;
    if (!ok) goto fail;
    if (cudaStreamBeginCaptureToGraph(b->cap_stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) !=
        cudaSuccess)
        goto fail;
    {
        cudaError_t e = cudaEventRecord(ev[0], b->cap_stream);
        for (size_t p = 0; p < b->pool.size() && e == cudaSuccess; ++p) e = cudaStreamWaitEvent(b->pool[p], ev[0], 0);
        for (int32_t i = 0, r = 0; i < b->count && e == cudaSuccess; ++i) {
            if (!run[i]) continue;
            cudaStream_t s = b->pool[(r++) % b->pool.size()];
            for (int q = 0; q < kBatchUnroll && e == cudaSuccess; ++q) {
                SweepArgs<T> a = batch_args<T>(b, b->ctx[i], 1, h, q & 1);
                e = launch_excess<T>(a, s);
                if (e == cudaSuccess) e = launch_update<T>(b->ctx[i], a, s);
            }
        }
        for (size_t p = 0; p < b->pool.size() && e == cudaSuccess; ++p) {
            e = cudaEventRecord(ev[p + 1], b->pool[p]);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(b->cap_stream, ev[p + 1], 0);
        }
        cudaError_t e3 = cudaStreamEndCapture(b->cap_stream, &captured);
        if (e != cudaSuccess || e3 != cudaSuccess) goto fail;
    }
    if (cudaGraphInstantiate(&exec, g, 0) != cudaSuccess) goto fail;
    for (auto& e : ev) cudaEventDestroy(e);
    b->graph[p] = g;
    b->exec[p] = exec;
    b->graph_ok[p] = true;
    return;
fail:
    cudaGetLastError();
    for (auto& e : ev)
        if (e) cudaEventDestroy(e);
    if (g) cudaGraphDestroy(g);
    b->graph_ok[p] = false;
}

__global__ void set_counter_kernel(unsigned int* c, unsigned int v) { *c = v; }

// Alg. 1 in precision T for the instances with run[i] set, from the states
// their callers initialised (instance i's sweep counter starting at
// t_start[i]); the others keep their stopped state.
// Blocks of the cluster that solves an instance on the one-cluster-per-
// instance engine: enough that each lane group of the cluster handles at
// most about 16 edges per sweep (the edges of a group run one after the
// other), a power of two up to 8.
int batch_cluster_size(const pdr_ctx* c, int p)
{
    const int G = edge_group_lanes(c->cfg[p]);
    const int64_t groups = (int64_t)(kBatchThreads / 32) * (32 / G);
    const int64_t want = (c->m + groups * 16 - 1) / (groups * 16);
    int cs = 1;
    while (cs < want && cs < 8) cs <<= 1;
    return cs;
}

// True if instance i runs on the one-cluster-per-instance engine in
// precision p (cluster_eligible: a small instance with a lane-group variant
// of at most 4 vectors per lane; the larger ones spill at the block's
// register budget).  FP64 sweeps run on the graph: one block has one SM's
// FP64 rate, and the graph's kernels spread each instance over several SMs.
bool batch_resident(const pdr_batch* b, int32_t i, int p)
{
    return p == Prec<float>::id && cluster_eligible(b->ctx[i], p);
}

// The instances of `blk` (set up by batch_run) on the one-block-per-instance
// engine: launches of kBlockChunk sweeps, one per edge-kernel variant on its
// own stream so that they run side by side, until every instance stopped.
template <typename T>
pdr_status batch_block_run(pdr_batch* b, const std::vector<char>& blk, const std::vector<int64_t>& t_start)
{
    const int p = Prec<T>::id;
    std::vector<int32_t> live;
    for (int32_t i = 0; i < b->count; ++i)
        if (blk[i]) live.push_back(i);
    SweepArgs<T>* hargs = static_cast<SweepArgs<T>*>(b->hstage);
    int* hids = reinterpret_cast<int*>(hargs + b->count);
    SweepArgs<T>* dargs = static_cast<SweepArgs<T>*>(b->bargs[p]);
    std::vector<cudaEvent_t> ev;
    auto done = [&](pdr_status st) {
        for (cudaEvent_t e : ev) cudaEventDestroy(e);
        return st;
    };
    auto cuda_err = [&](const char* what, cudaError_t e) {
        return done(batch_fail(PDR_ERR_CUDA, std::string("batch: ") + what + ": " + cudaGetErrorString(e)));
    };
    for (int q = 0; q < 7; ++q) {  // the fork event and one per launch group (more on demand)
        cudaEvent_t e;
        const cudaError_t er = cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
        if (er != cudaSuccess) return cuda_err("event", er);
        ev.push_back(e);
    }
    bool first = true;
    while (!live.empty()) {
        // arguments with the buffer parity of each instance's current flows
        for (int32_t i : live) {
            pdr_ctx* c = b->ctx[i];
            const int par = first ? 0 : (int)((c->hst->t - t_start[i]) & 1);
            const int csize = batch_cluster_size(c, p);
            SweepArgs<T> a = make_args<T>(c, MODE_SOLVE, 0, 0, par, 0);
            a.excess_form = 0;  // the gather form, run by the cluster's blocks
            a.grid_v = csize;
            a.grid_e = csize;
            a.n_psi = csize * (kBatchThreads / 32);
            a.pf_edges = 0;
            a.l2_hints = 0;
            a.active = nullptr;
            hargs[i] = a;
        }
        // one launch per (lane-group variant, cluster size, form), largest
        // clusters first; single blocks whose instance fits in shared memory
        // run the shared-memory form, with the largest of their sizes
        struct Group {
            int cfg, csize, off, count;
            int64_t smem;
        };
        std::vector<Group> groups;
        int pos = 0;
        for (int csize = 8; csize >= 1; csize >>= 1)
            for (int cfg = 0; cfg <= 5; ++cfg)
                for (int sm = 0; sm < (csize == 1 ? 2 : 1); ++sm) {
                    const int off = pos;
                    int64_t smem = 0;
                    for (int32_t i : live) {
                        const pdr_ctx* c = b->ctx[i];
                        if (edge_plain_config(c->cfg[p]) != cfg || batch_cluster_size(c, p) != csize) continue;
                        const int64_t need = csize == 1 ? block_smem(c, p) : 0;
                        if ((need > 0) != (sm == 1)) continue;
                        hids[pos++] = i;
                        smem = need > smem ? need : smem;
                    }
                    if (pos > off) groups.push_back({cfg, csize, off, pos - off, smem});
                }
        cudaError_t e = cudaMemcpyAsync(dargs, hargs, sizeof(SweepArgs<T>) * b->count, cudaMemcpyHostToDevice,
                                        b->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(b->bids, hids, sizeof(int) * pos, cudaMemcpyHostToDevice, b->stream);
        if (e == cudaSuccess) e = cudaEventRecord(ev[0], b->stream);
        for (size_t g = 0; g < groups.size() && e == cudaSuccess; ++g) {
            while (ev.size() < g + 2) {
                cudaEvent_t x;
                e = cudaEventCreateWithFlags(&x, cudaEventDisableTiming);
                if (e != cudaSuccess) break;
                ev.push_back(x);
            }
            if (e != cudaSuccess) break;
            cudaStream_t sg = b->pool[g % b->pool.size()];
            e = cudaStreamWaitEvent(sg, ev[0], 0);
            if (e == cudaSuccess)
                e = launch_batch_block<T>(groups[g].cfg, dargs, b->bids + groups[g].off, groups[g].count, groups[g].csize,
                                          kBlockChunk, first ? 1 : 0, sg, groups[g].smem);
            if (e == cudaSuccess) e = cudaEventRecord(ev[1 + g], sg);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, ev[1 + g], 0);
        }
        for (size_t q = 0; q < live.size() && e == cudaSuccess; ++q) {
            pdr_ctx* c = b->ctx[live[q]];
            e = cudaMemcpyAsync(c->hst, c->st, sizeof(DevState), cudaMemcpyDeviceToHost, b->stream);
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
        if (e != cudaSuccess) return cuda_err("one-block-per-instance engine", e);
        std::vector<int32_t> next;
        for (int32_t i : live) {
            if (b->ctx[i]->hst->fault)
                return done(batch_fail(PDR_ERR_TIMEOUT, "instance " + std::to_string(i) + ": a device wait timed out"));
            if (!b->ctx[i]->hst->stop) next.push_back(i);
        }
        live.swap(next);
        first = false;
    }
    // current flows, and the congestion partials in the standalone kernels' layout
    for (int32_t i = 0; i < b->count; ++i) {
        if (!blk[i]) continue;
        pdr_ctx* c = b->ctx[i];
        c->cur = (int)((c->hst->t - t_start[i]) & 1);
        const pdr_status st = refresh_psi<T>(c, nullptr, true);
        if (st != PDR_OK) return done(st);
    }
    return done(PDR_OK);
}

template <typename T>
pdr_status batch_run(pdr_batch* b, const std::vector<char>& run_all, const std::vector<int64_t>& t_start)
{
    const int p = Prec<T>::id;
    // small instances go to the one-block-per-instance engine, the others to the graph
    std::vector<char> blk(b->count, 0), run(run_all);
    bool any_blk = false;
    const bool use_graph = b->ctx[0]->opt.use_graph != 0;
    for (int32_t i = 0; i < b->count; ++i)
        if (run_all[i] && use_graph && batch_resident(b, i, p)) {
            blk[i] = 1;
            run[i] = 0;
            any_blk = true;
        }
    unsigned int running = 0;
    for (int32_t i = 0; i < b->count; ++i) {
        if (!run_all[i]) continue;
        pdr_ctx* c = b->ctx[i];
        pdr_status s = ensure_velocity<T>(c);
        if (s != PDR_OK) return s;
        s = flows_to_buffer0<T>(c);
        if (s != PDR_OK) return s;
        if (run[i]) ++running;
    }
    if (any_blk) {
        const pdr_status s = batch_block_run<T>(b, blk, t_start);
        if (s != PDR_OK) return s;
    }
    if (running == 0) return PDR_OK;
    set_counter_kernel<<<1, 1, 0, b->stream>>>(b->active, running);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return batch_fail(PDR_ERR_CUDA, std::string("batch: ") + cudaGetErrorString(e));
    if (use_graph && (!b->graph_tried[p] || b->graph_mask[p] != run)) {
        batch_destroy_graph(b, p);
        batch_build_graph<T>(b, run);
    }
    if (use_graph && b->graph_ok[p]) {
        e = cudaGraphLaunch(b->exec[p], b->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
        if (e != cudaSuccess) return batch_fail(PDR_ERR_CUDA, std::string("batch graph: ") + cudaGetErrorString(e));
    } else {
        // host loop: chunks of an even number of sweeps for every running instance
        for (;;) {
            for (int q = 0; q < 64; ++q)
                for (int32_t i = 0; i < b->count; ++i) {
                    if (!run[i]) continue;
                    SweepArgs<T> a = batch_args<T>(b, b->ctx[i], 0, 0, q & 1);
                    launch_excess<T>(a, b->stream);
                    launch_update<T>(b->ctx[i], a, b->stream);
                }
            unsigned int left = 0;
            e = cudaMemcpyAsync(&left, b->active, sizeof(left), cudaMemcpyDeviceToHost, b->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
            if (e != cudaSuccess) return batch_fail(PDR_ERR_CUDA, std::string("batch: ") + cudaGetErrorString(e));
            if (left == 0) break;
        }
    }
    for (int32_t i = 0; i < b->count; ++i) {
        if (!run[i]) continue;
        pdr_ctx* c = b->ctx[i];
        pdr_status s = read_state(c);
        if (s != PDR_OK) return s;
        c->cur = (int)((c->hst->t - t_start[i]) & 1);
    }
    return PDR_OK;
}

}  // namespace

extern "C" {

pdr_status pdr_batch_create(int32_t count, const pdr_instance* inst, const pdr_options* opt, void* stream,
                            pdr_batch** out)
{
    pdr::set_thread_error("");
    if (!out) return batch_fail(PDR_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (count < 1 || !inst) return batch_fail(PDR_ERR_INVALID_ARG, "count must be >= 1 and inst non-NULL");
    pdr_options o;
    fill_defaults(&o);
    if (opt) o = *opt;
    {
        std::string why;
        if (!options_ok(&o, &why)) return batch_fail(PDR_ERR_INVALID_ARG, why);
    }
    for (int32_t i = 0; i < count; ++i) {
        const pdr_instance& q = inst[i];
        const std::string why = validate_instance(q.n, q.m, q.row_ptr, q.col, q.u, q.K, q.s, q.t, q.d);
        if (!why.empty()) return batch_fail(PDR_ERR_INVALID_ARG, "instance " + std::to_string(i) + ": " + why);
    }
    pdr_batch* b = new pdr_batch();
    b->count = count;
    b->stream = static_cast<cudaStream_t>(stream);
    auto give_up = [&](pdr_status code, const std::string& msg) {
        pdr_batch_destroy(b);
        return batch_fail(code, msg);
    };
    if (cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
        return give_up(PDR_ERR_CUDA, "batch: stream creation failed");
    const int np = count < kBatchPool ? count : kBatchPool;
    for (int p = 0; p < np; ++p) {
        cudaStream_t s;
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess)
            return give_up(PDR_ERR_CUDA, "batch: stream creation failed");
        b->pool.push_back(s);
    }
    if (cudaMalloc(&b->active, sizeof(unsigned int)) != cudaSuccess) {
        cudaGetLastError();
        return give_up(PDR_ERR_OOM, "batch: counter allocation failed");
    }
    for (int32_t i = 0; i < count; ++i) {
        const pdr_instance& q = inst[i];
        pdr_ctx* c = nullptr;
        pdr_status s = pdr_create(q.n, q.m, q.row_ptr, q.col, q.u, q.K, q.s, q.t, q.d, &o, stream, &c);
        if (s != PDR_OK) {
            const std::string why = pdr_last_error(nullptr);
            return give_up(s, "instance " + std::to_string(i) + ": " + why);
        }
        b->ctx.push_back(c);
    }
    b->tuned_cfg.assign(count, -1);
    b->tuned_us.assign(count, -1.0);
    for (int p = 0; p < 2; ++p)
        if (cudaMalloc(&b->bargs[p], sizeof(SweepArgs<double>) * count) != cudaSuccess) {
            cudaGetLastError();
            return give_up(PDR_ERR_OOM, "batch: argument table allocation failed");
        }
    if (cudaMalloc(&b->bids, sizeof(int) * count) != cudaSuccess ||
        cudaMallocHost(&b->hstage, (sizeof(SweepArgs<double>) + sizeof(int)) * count) != cudaSuccess) {
        cudaGetLastError();
        return give_up(PDR_ERR_OOM, "batch: argument table allocation failed");
    }
    for (int32_t i = 0; i < count; ++i) {
        pdr_ctx* c = b->ctx[i];
        if (o.edge_variant >= 0) {  // the caller's variant: no tuning
            b->tuned_cfg[i] = c->cfg[c->cur_prec];
            continue;
        }
        pdr_status s = c->cur_prec ? autotune<double>(c, &b->tuned_cfg[i], &b->tuned_us[i])
                                   : autotune<float>(c, &b->tuned_cfg[i], &b->tuned_us[i]);
        if (s != PDR_OK) return give_up(s, "instance " + std::to_string(i) + ": " + c->err);
    }
    *out = b;
    return PDR_OK;
}

pdr_status pdr_batch_solve(pdr_batch* b, pdr_result* results)
{
    if (!b) return PDR_ERR_INVALID_ARG;
    const auto t0 = std::chrono::steady_clock::now();
    const int32_t B = b->count;
    const bool tail = b->ctx[0]->opt.precision == PDR_PREC_FP32_FP64TAIL;
    std::vector<char> run32(B, 0), run64(B, 0);
    std::vector<int64_t> t_start(B, 0), sweeps32(B, 0);
    std::vector<int32_t> reason32(B, -1);
    pdr_status s = PDR_OK;
    // every instance starts a fresh solve from its current flows, as pdr_solve
    for (int32_t i = 0; i < B; ++i) {
        pdr_ctx* c = b->ctx[i];
        s = init_state(c, true, (tail && c->cur_prec == 0) ? 1 : 0);
        if (s != PDR_OK) return s;
        (c->cur_prec ? run64 : run32)[i] = 1;
    }
    s = batch_run<float>(b, run32, t_start);
    if (s != PDR_OK) return s;
    if (tail) {
        // instances whose FP32 phase stopped on the objective rules continue in FP64
        bool any = false;
        for (int32_t i = 0; i < B; ++i) {
            pdr_ctx* c = b->ctx[i];
            if (!run32[i]) continue;
            s = read_state(c);
            if (s != PDR_OK) return s;
            sweeps32[i] = c->hst->t;
            reason32[i] = c->hst->reason;
            if (needs_fp64_tail(c->hst->reason)) {
                s = widen_to_fp64(c);
                if (s != PDR_OK) return s;
                s = init_state(c, false, 0);
                if (s != PDR_OK) return s;
                t_start[i] = c->hst->t;
                run64[i] = 1;
            }
            any = any || run64[i];
        }
        for (int32_t i = 0; i < B && !any; ++i) any = run64[i];
        if (any)
            for (pdr_ctx* c : b->ctx) {  // stable device pointers for the FP64 graph
                s = ensure_fp64(c);
                if (s != PDR_OK) return s;
            }
    }
    s = batch_run<double>(b, run64, t_start);
    if (s != PDR_OK) return s;
    const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    bool numeric = false;
    for (int32_t i = 0; i < b->count; ++i) {
        pdr_ctx* c = b->ctx[i];
        s = read_state(c);
        if (s != PDR_OK) return s;
        pdr_result r{};
        r.sweeps = c->hst->t;
        r.sweeps_fp64 = c->cur_prec ? c->hst->t - sweeps32[i] : 0;
        r.dz = c->hst->dz;
        r.stop_reason = c->hst->reason;
        r.stop_reason_fp32 = tail ? reason32[i] : -1;
        s = residuals_into(c, &r);
        if (s != PDR_OK) return batch_fail(s, "instance " + std::to_string(i) + ": " + c->err);
        r.ms_total = ms;
        c->last = r;
        if (results) results[i] = r;
        if (r.stop_reason == STOP_NUMERIC) numeric = true;
    }
    if (numeric) return batch_fail(PDR_ERR_NUMERIC, "an instance's objective became non-finite");
    return PDR_OK;
}

pdr_status pdr_batch_reset(pdr_batch* b)
{
    if (!b) return PDR_ERR_INVALID_ARG;
    for (pdr_ctx* c : b->ctx) {
        pdr_status s = pdr_reset(c);
        if (s != PDR_OK) return s;
    }
    return PDR_OK;
}

pdr_status pdr_batch_context(pdr_batch* b, int32_t index, pdr_ctx** ctx)
{
    if (!b || !ctx || index < 0 || index >= b->count) return PDR_ERR_INVALID_ARG;
    *ctx = b->ctx[index];
    return PDR_OK;
}

pdr_status pdr_batch_tuning(const pdr_batch* b, int32_t* cfg, double* us)
{
    if (!b) return PDR_ERR_INVALID_ARG;
    for (int32_t i = 0; i < b->count; ++i) {
        if (cfg) cfg[i] = b->tuned_cfg[i];
        if (us) us[i] = b->tuned_us[i];
    }
    return PDR_OK;
}

void pdr_batch_destroy(pdr_batch* b)
{
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    batch_destroy_graph(b, 0);
    batch_destroy_graph(b, 1);
    for (pdr_ctx* c : b->ctx) pdr_destroy(c);
    for (cudaStream_t s : b->pool) cudaStreamDestroy(s);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    if (b->active) cudaFree(b->active);
    for (void* q : b->bargs)
        if (q) cudaFree(q);
    if (b->bids) cudaFree(b->bids);
    if (b->hstage) cudaFreeHost(b->hstage);
    cudaGetLastError();
    delete b;
}

}  // extern "C"
