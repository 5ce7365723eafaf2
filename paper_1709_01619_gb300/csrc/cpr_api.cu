// cpr_api.cu -- the C ABI of libcpr.so (declared in include/cpr.h).
//
// A context owns the operator tables, two stage buffers (q1, q2 of the SSP-RK3
// scheme, Sec. 4), the element-average buffer of the limiter, the limiter
// marks, the device control block (simulated time, step size, the running
// maximum speed of the CFL reduction) and the CUDA graphs of the RK loop.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdint>
#include <cstring>
#include <new>
#include <string>

#include "../../include/cpr.h"
#include "cpr_internal.h"
#include "cpr_aux.cuh"
#include "cpr_launch.h"

using cpr::Ctrl;
using cpr::LaunchCfg;

struct cpr_ctx {
    cpr_config cfg{};
    cudaStream_t stream = nullptr;
    cudaStream_t cap = nullptr;  // capture stream for the step graphs
    int device = 0;
    int V = 1, n = 2;
    long long ne = 0, npts = 0, nstate = 0;
    size_t esize = 8;
    LaunchCfg lc{};
    void* q1 = nullptr;
    void* q2 = nullptr;
    void* avg = nullptr;
    int* marks = nullptr;
    Ctrl* ctrl = nullptr;
    double* partials = nullptr;
    double* h_partials = nullptr;  // pinned
    Ctrl* h_ctrl = nullptr;        // pinned
    int norm_blocks = 1;
    void* host_state = nullptr;    // device copy for cpr_step_host
    void* lo = nullptr;            // low part of the state (FP32 increment form)
    void* adj1 = nullptr;          // adjoint scratch (allocated on first use)
    void* adj2 = nullptr;
    bool use_inc = false;          // FP32 without limiter: increment form of SSP-RK3
    const void* graph_q = nullptr;
    cudaGraphExec_t g1 = nullptr, g2 = nullptr, gK = nullptr;
    std::string err;
};

static thread_local std::string g_init_err;
static const int kStepsPerGraph = 32;

#define CPR_CUDA(ctx, call)                                                                   \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess) {                                                              \
            (ctx)->err = std::string(#call) + ": " + cudaGetErrorString(e_);                  \
            return CPR_ECUDA;                                                                 \
        }                                                                                     \
    } while (0)

static cpr_status fail(cpr_ctx* ctx, cpr_status st, const char* msg)
{
    if (ctx) ctx->err = msg;
    return st;
}

// Device state arrays are read with 16-byte vector loads.
static bool aligned(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// ---------------------------------------------------------------------------
// small device kernels of the time control
// ---------------------------------------------------------------------------
__global__ void ctrl_configure_kernel(Ctrl* c, double dt_fixed, double t_end, double cfl_h)
{
    c->dt_fixed = dt_fixed;
    c->t_end = t_end;
    c->cfl_h = cfl_h;
    c->done = 0;
    c->counter = 0;
    c->parity = 0;
    if (dt_fixed > 0.0) cpr::ctrl_next_dt(c, c->max_wave);
}

// Increment form: after an odd number of completed steps the state sits in
// the context's second buffer; copy it back to the caller's array.
__global__ void parity_copy_kernel(const Ctrl* c, float* dst, const float* src, long long n)
{
    if (!c->parity) return;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        dst[i] = src[i];
}

__global__ void ctrl_set_time_kernel(Ctrl* c, double t, long long steps)
{
    c->t = t;
    c->steps = steps;
    c->done = 0;
    c->last = 0;
}

// ---------------------------------------------------------------------------
// dtype dispatch
// ---------------------------------------------------------------------------
static cudaError_t stage_inc(cpr_ctx* c, int mode, const void* qs, const void* qb, void* out, bool wave,
                             cudaStream_t s)
{
    cpr::StagePtrs b{qs, qb, nullptr, out, c->lo, nullptr};
    return cpr::launch_stage<float>(c->lc, mode, b, wave, s);
}
static cudaError_t stage(cpr_ctx* c, int mode, const void* qs, const void* qn, void* out, void* avg, bool wave,
                         cudaStream_t s)
{
    return c->cfg.dtype == CPR_F32 ? cpr::launch_stage<float>(c->lc, mode, qs, qn, out, avg, wave, s)
                                   : cpr::launch_stage<double>(c->lc, mode, qs, qn, out, avg, wave, s);
}
static cudaError_t averages(cpr_ctx* c, const void* q, void* avg, cudaStream_t s)
{
    return c->cfg.dtype == CPR_F32 ? cpr::launch_averages<float>(c->lc, q, avg, s)
                                   : cpr::launch_averages<double>(c->lc, q, avg, s);
}
static cudaError_t limit(cpr_ctx* c, void* q, const void* avg, int role, cudaStream_t s)
{
    return c->cfg.dtype == CPR_F32 ? cpr::launch_limit<float>(c->lc, q, avg, role, s)
                                   : cpr::launch_limit<double>(c->lc, q, avg, role, s);
}
static cudaError_t wave(cpr_ctx* c, const void* q, cudaStream_t s)
{
    return c->cfg.dtype == CPR_F32 ? cpr::launch_wave<float>(c->lc, q, s) : cpr::launch_wave<double>(c->lc, q, s);
}
static cudaError_t norms(cpr_ctx* c, const void* q, const void* ref, cudaStream_t s)
{
    return c->cfg.dtype == CPR_F32 ? cpr::launch_norms<float>(c->lc, q, ref, c->norm_blocks, s)
                                   : cpr::launch_norms<double>(c->lc, q, ref, c->norm_blocks, s);
}

// ---------------------------------------------------------------------------
// configuration
// ---------------------------------------------------------------------------
bool cpr_fill_launch_cfg(const cpr_config* cfg, LaunchCfg* out)
{
    LaunchCfg lc{};
    lc.eqn = cfg->eqn;
    lc.p = cfg->p;
    lc.div = cfg->div;
    // Roe's flux for advection is the upwind flux
    lc.flux = cfg->flux == CPR_FLUX_UPWIND ? cpr::FLUX_UPWIND
              : cfg->flux == CPR_FLUX_ROE   ? (cfg->eqn == CPR_EULER ? cpr::FLUX_ROE : cpr::FLUX_UPWIND)
                                            : cpr::FLUX_RUSANOV;
    lc.nx = cfg->nx;
    lc.ny = cfg->ny;
    lc.bcx = cfg->bc_x == CPR_BC_TRANSMISSIVE;
    lc.bcy = cfg->bc_y == CPR_BC_TRANSMISSIVE;
    lc.ne = (long long)cfg->nx * cfg->ny;
    lc.npts = lc.ne * (cfg->p + 1) * (cfg->p + 1);
    lc.hx = (cfg->x1 - cfg->x0) / cfg->nx;
    lc.hy = (cfg->y1 - cfg->y0) / cfg->ny;
    lc.gamma = cfg->gamma;
    lc.ax = cfg->ax;
    lc.ay = cfg->ay;
    lc.tvb_M = cfg->tvb_M;
    lc.lim_eps = cfg->lim_eps;
    lc.fv_order = cfg->scheme == CPR_SCHEME_FV_MUSCL3 ? 3 : 2;
    lc.l2_bytes = cpr::current_l2_bytes();
    lc.sms = cpr::current_sm_count();
    if (cpr::build_tables(cfg->p, cfg->pts, cfg->corr, &lc.tab) != 0) return false;
    *out = lc;
    return true;
}

const char* cpr_validate_config(const cpr_config* c)
{
    if (!c) return "cfg is NULL";
    if (c->eqn != CPR_ADVECTION && c->eqn != CPR_EULER) return "eqn must be CPR_ADVECTION or CPR_EULER";
    if (c->nx < 1 || c->ny < 1) return "nx and ny must be >= 1";
    if (c->nx > (1 << 20) || c->ny > (1 << 20)) return "nx and ny must be <= 2^20";
    if (!(c->x1 > c->x0) || !(c->y1 > c->y0)) return "domain needs x1 > x0 and y1 > y0";
    if (!std::isfinite(c->x0) || !std::isfinite(c->x1) || !std::isfinite(c->y0) || !std::isfinite(c->y1))
        return "domain bounds must be finite";
    if (c->scheme != CPR_SCHEME_CPR && c->scheme != CPR_SCHEME_FV_MUSCL && c->scheme != CPR_SCHEME_FV_MUSCL3)
        return "scheme must be CPR_SCHEME_CPR, CPR_SCHEME_FV_MUSCL or CPR_SCHEME_FV_MUSCL3";
    if (c->scheme != CPR_SCHEME_CPR) {
        if (c->p != 0) return "the FV schemes need p = 0 (one average per element)";
        if (c->limiter != 0) return "the FV schemes limit their slopes themselves: limiter must be 0";
    } else if (c->p < 1 || c->p > 4) {
        return "p must be in [1, 4]";
    }
    if (c->pts != CPR_PTS_GAUSS && c->pts != CPR_PTS_LOBATTO) return "pts must be CPR_PTS_GAUSS or CPR_PTS_LOBATTO";
    if (c->corr != CPR_CORR_GDG && c->corr != CPR_CORR_NDG && c->corr != CPR_CORR_NDG_LUMPED)
        return "corr must be CPR_CORR_GDG, CPR_CORR_NDG or CPR_CORR_NDG_LUMPED";
    if (c->flux != CPR_FLUX_RUSANOV && c->flux != CPR_FLUX_UPWIND && c->flux != CPR_FLUX_ROE)
        return "flux must be CPR_FLUX_RUSANOV, CPR_FLUX_UPWIND or CPR_FLUX_ROE";
    if (c->flux == CPR_FLUX_UPWIND && c->eqn != CPR_ADVECTION) return "CPR_FLUX_UPWIND needs CPR_ADVECTION";
    if (c->div != CPR_DIV_LP && c->div != CPR_DIV_CHAIN) return "div must be CPR_DIV_LP or CPR_DIV_CHAIN";
    if ((c->bc_x != CPR_BC_PERIODIC && c->bc_x != CPR_BC_TRANSMISSIVE) ||
        (c->bc_y != CPR_BC_PERIODIC && c->bc_y != CPR_BC_TRANSMISSIVE))
        return "bc_x and bc_y must be CPR_BC_PERIODIC or CPR_BC_TRANSMISSIVE";
    if (c->eqn == CPR_EULER && !(c->gamma > 1.0)) return "gamma must be > 1";
    if (c->eqn == CPR_ADVECTION && (!std::isfinite(c->ax) || !std::isfinite(c->ay))) return "ax, ay must be finite";
    if (c->limiter != 0 && c->limiter != 1) return "limiter must be 0 or 1";
    if (!(c->tvb_M >= 0.0) || !(c->lim_eps >= 0.0)) return "tvb_M and lim_eps must be >= 0";
    if (c->dtype != CPR_F64 && c->dtype != CPR_F32) return "dtype must be CPR_F64 or CPR_F32";
    if (!(c->cfl >= 0.0)) return "cfl must be >= 0";
    return nullptr;
}

static void free_all(cpr_ctx* c)
{
    if (c->g1) cudaGraphExecDestroy(c->g1);
    if (c->g2) cudaGraphExecDestroy(c->g2);
    if (c->gK) cudaGraphExecDestroy(c->gK);
    cudaFree(c->lo);
    cudaFree(c->adj1);
    cudaFree(c->adj2);
    cudaFree(c->q1);
    cudaFree(c->q2);
    cudaFree(c->avg);
    cudaFree(c->marks);
    cudaFree(c->ctrl);
    cudaFree(c->partials);
    cudaFree(c->host_state);
    if (c->h_partials) cudaFreeHost(c->h_partials);
    if (c->h_ctrl) cudaFreeHost(c->h_ctrl);
    if (c->cap) cudaStreamDestroy(c->cap);
}

extern "C" cpr_status cpr_init(const cpr_config* cfg, void* stream, cpr_ctx** out)
{
    if (!out) {
        g_init_err = "out is NULL";
        return CPR_EINVAL;
    }
    *out = nullptr;
    if (const char* msg = cpr_validate_config(cfg)) {
        g_init_err = msg;
        return CPR_EINVAL;
    }
    cpr_ctx* c = new (std::nothrow) cpr_ctx();
    if (!c) {
        g_init_err = "host allocation failed";
        return CPR_ENOMEM;
    }
    c->cfg = *cfg;
    c->stream = static_cast<cudaStream_t>(stream);
    cudaGetDevice(&c->device);
    c->V = cfg->eqn == CPR_EULER ? 4 : 1;
    c->n = cfg->p + 1;
    c->ne = (long long)cfg->nx * cfg->ny;
    c->npts = c->ne * c->n * c->n;
    c->nstate = c->npts * c->V;
    c->esize = cfg->dtype == CPR_F32 ? 4 : 8;

    if (!cpr_fill_launch_cfg(cfg, &c->lc)) {
        delete c;
        g_init_err = "table construction failed";
        return CPR_EINVAL;
    }
    LaunchCfg& lc = c->lc;

    c->norm_blocks = (int)std::min<long long>(1024, std::max<long long>(1, (c->ne + 255) / 256));
    const size_t sbytes = (size_t)c->nstate * c->esize;
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = cudaMalloc(&c->q1, sbytes);
    if (e == cudaSuccess) e = cudaMalloc(&c->q2, sbytes);
    c->use_inc = cfg->dtype == CPR_F32 && !cfg->limiter;
    if (e == cudaSuccess && c->use_inc) e = cudaMalloc(&c->lo, sbytes);
    if (e == cudaSuccess) e = cudaMalloc(&c->avg, (size_t)c->V * c->ne * c->esize);
    if (e == cudaSuccess) e = cudaMalloc((void**)&c->marks, (size_t)c->ne * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc((void**)&c->ctrl, sizeof(Ctrl));
    if (e == cudaSuccess) e = cudaMalloc((void**)&c->partials, (size_t)c->norm_blocks * cpr::kNormVals * 8);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&c->h_partials, (size_t)c->norm_blocks * cpr::kNormVals * 8);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&c->h_ctrl, sizeof(Ctrl));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->ctrl, 0, sizeof(Ctrl), c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->marks, 0, (size_t)c->ne * sizeof(int), c->stream);
    lc.ctrl = c->ctrl;
    lc.marks = c->marks;
    lc.partials = c->partials;
    if (e == cudaSuccess)
        e = cfg->dtype == CPR_F32 ? cpr::prepare_stage<float>(lc) : cpr::prepare_stage<double>(lc);
    if (e != cudaSuccess) {
        g_init_err = std::string("CUDA: ") + cudaGetErrorString(e);
        const cpr_status st = (e == cudaErrorMemoryAllocation) ? CPR_ENOMEM : CPR_ECUDA;
        free_all(c);
        delete c;
        return st;
    }
    *out = c;
    return CPR_OK;
}

extern "C" void cpr_destroy(cpr_ctx* c)
{
    if (!c) return;
    cudaStreamSynchronize(c->stream);
    free_all(c);
    delete c;
}

extern "C" size_t cpr_state_elems(const cpr_ctx* c) { return c ? (size_t)c->nstate : 0; }

extern "C" const char* cpr_last_error(const cpr_ctx* c) { return c ? c->err.c_str() : g_init_err.c_str(); }

extern "C" cpr_status cpr_point_coords(const cpr_ctx* c, double* x, double* y)
{
    if (!c || !x || !y) return CPR_EINVAL;
    const int n = c->n;
    const cpr::HostTab& t = c->lc.tab;
    for (long long e = 0; e < c->ne; ++e) {
        const int i = (int)(e % c->cfg.nx), j = (int)(e / c->cfg.nx);
        for (int b = 0; b < n; ++b)
            for (int a = 0; a < n; ++a) {
                x[e * n * n + b * n + a] = c->cfg.x0 + c->lc.hx * (i + 0.5 * (t.xi[a] + 1.0));
                y[e * n * n + b * n + a] = c->cfg.y0 + c->lc.hy * (j + 0.5 * (t.xi[b] + 1.0));
            }
    }
    return CPR_OK;
}

// ---------------------------------------------------------------------------
// residual, step, limiter
// ---------------------------------------------------------------------------
extern "C" cpr_status cpr_residual(cpr_ctx* c, const void* q, void* r)
{
    if (!c) return CPR_EINVAL;
    if (!q || !r) return fail(c, CPR_EINVAL, "q_dev and r_dev must be non-NULL");
    if (q == r) return fail(c, CPR_EINVAL, "q_dev and r_dev must not alias");
    if (!aligned(q) || !aligned(r)) return fail(c, CPR_EINVAL, "state arrays must be 16-byte aligned");
    CPR_CUDA(c, stage(c, 0, q, nullptr, r, nullptr, false, c->stream));
    return CPR_OK;
}

// Enqueue one SSP-RK3 step on stream s (Sec. 4):
//   q1 = q + dt R(q); q2 = 3/4 q + 1/4 (q1 + dt R(q1)); q = 1/3 q + 2/3 (q2 + dt R(q2)),
// each stage result limited when the limiter is on.
// The stage kernel of a limited run (the one that writes the averages)
// clears the marked-element count for the limiter pass that follows it, and
// skips that once t_end is reached, so the count survives the idle steps of
// a run asked for more steps than it needs.
static cudaError_t enqueue_step(cpr_ctx* c, void* q, cudaStream_t s)
{
    const bool lim = c->cfg.limiter != 0;
    void* avg = lim ? c->avg : nullptr;
    cudaError_t e;
    if ((e = stage(c, 1, q, nullptr, c->q1, avg, false, s)) != cudaSuccess) return e;
    if (lim && (e = limit(c, c->q1, c->avg, 1, s)) != cudaSuccess) return e;
    if ((e = stage(c, 2, c->q1, q, c->q2, avg, false, s)) != cudaSuccess) return e;
    if (lim && (e = limit(c, c->q2, c->avg, 1, s)) != cudaSuccess) return e;
    if ((e = stage(c, 3, c->q2, q, q, avg, !lim, s)) != cudaSuccess) return e;
    if (lim && (e = limit(c, q, c->avg, 2, s)) != cudaSuccess) return e;
    return cudaSuccess;
}

// Increment form (FP32, no limiter), one step with the state's high part in
// x: B1 -> y, B2 -> z, new high part -> y (B1 is dead by then).  The next
// step runs with x and y swapped, so two steps bring the state back to x.
static cudaError_t enqueue_inc_step(cpr_ctx* c, void* x, void* y, cudaStream_t s)
{
    cudaError_t e;
    if ((e = stage_inc(c, cpr::MODE_INC1, x, nullptr, y, false, s)) != cudaSuccess) return e;
    if ((e = stage_inc(c, cpr::MODE_INC2, x, y, c->q2, false, s)) != cudaSuccess) return e;
    return stage_inc(c, cpr::MODE_INC3, x, c->q2, y, true, s);
}

// steps: 1 (one step from q), or an even count of alternating steps.
static cudaError_t capture(cpr_ctx* c, void* q, int steps, cudaGraphExec_t* exec)
{
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    cudaError_t ee = cudaSuccess;
    for (int k = 0; k < steps && ee == cudaSuccess; ++k) {
        if (c->use_inc) ee = (k % 2 == 0) ? enqueue_inc_step(c, q, c->q1, c->cap) : enqueue_inc_step(c, c->q1, q, c->cap);
        else ee = enqueue_step(c, q, c->cap);
    }
    e = cudaStreamEndCapture(c->cap, &g);
    if (ee != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return ee;
    }
    if (e != cudaSuccess) return e;
    e = cudaGraphInstantiate(exec, g, 0);
    cudaGraphDestroy(g);
    return e;
}

static cudaError_t ensure_graphs(cpr_ctx* c, void* q)
{
    if (c->graph_q == q && c->g1 && c->g2 && c->gK) return cudaSuccess;
    if (c->g1) cudaGraphExecDestroy(c->g1);
    if (c->g2) cudaGraphExecDestroy(c->g2);
    if (c->gK) cudaGraphExecDestroy(c->gK);
    c->g1 = c->g2 = c->gK = nullptr;
    c->graph_q = nullptr;
    cudaError_t e = capture(c, q, 1, &c->g1);
    if (e == cudaSuccess) e = capture(c, q, 2, &c->g2);
    if (e == cudaSuccess) e = capture(c, q, kStepsPerGraph, &c->gK);
    if (e == cudaSuccess) c->graph_q = q;
    return e;
}

extern "C" cpr_status cpr_step(cpr_ctx* c, void* q, int nsteps, double dt_fixed, double t_end)
{
    if (!c) return CPR_EINVAL;
    if (!q) return fail(c, CPR_EINVAL, "q_dev must be non-NULL");
    if (!aligned(q)) return fail(c, CPR_EINVAL, "state arrays must be 16-byte aligned");
    if (nsteps < 0) return fail(c, CPR_EINVAL, "nsteps must be >= 0");
    if (!std::isfinite(dt_fixed) || !std::isfinite(t_end)) return fail(c, CPR_EINVAL, "dt_fixed, t_end must be finite");
    if (dt_fixed <= 0.0 && !(c->cfg.cfl > 0.0)) return fail(c, CPR_EINVAL, "CFL steps need cfg.cfl > 0");
    if (nsteps == 0) return CPR_OK;
    const double cfl_h = c->cfg.cfl * std::min(c->lc.hx, c->lc.hy);
    ctrl_configure_kernel<<<1, 1, 0, c->stream>>>(c->ctrl, dt_fixed, t_end, cfl_h);
    CPR_CUDA(c, cudaGetLastError());
    if (dt_fixed <= 0.0) CPR_CUDA(c, wave(c, q, c->stream));
    CPR_CUDA(c, ensure_graphs(c, q));
    if (c->use_inc) CPR_CUDA(c, cudaMemsetAsync(c->lo, 0, (size_t)c->nstate * c->esize, c->stream));
    for (int k = 0; k < nsteps / kStepsPerGraph; ++k) CPR_CUDA(c, cudaGraphLaunch(c->gK, c->stream));
    const int rest = nsteps % kStepsPerGraph;
    if (c->use_inc) {
        for (int k = 0; k < rest / 2; ++k) CPR_CUDA(c, cudaGraphLaunch(c->g2, c->stream));
        if (rest % 2) CPR_CUDA(c, cudaGraphLaunch(c->g1, c->stream));
        parity_copy_kernel<<<1024, 256, 0, c->stream>>>(c->ctrl, static_cast<float*>(q),
                                                        static_cast<const float*>(c->q1), c->nstate);
        CPR_CUDA(c, cudaGetLastError());
    } else {
        for (int k = 0; k < rest; ++k) CPR_CUDA(c, cudaGraphLaunch(c->g1, c->stream));
    }
    return CPR_OK;
}

extern "C" cpr_status cpr_step_host(cpr_ctx* c, const void* qin, void* qout, int nsteps, double dt_fixed,
                                    double t_end)
{
    if (!c) return CPR_EINVAL;
    if (!qin || !qout) return fail(c, CPR_EINVAL, "host buffers must be non-NULL");
    const size_t bytes = (size_t)c->nstate * c->esize;
    if (!c->host_state) CPR_CUDA(c, cudaMalloc(&c->host_state, bytes));
    CPR_CUDA(c, cudaMemcpyAsync(c->host_state, qin, bytes, cudaMemcpyHostToDevice, c->stream));
    cpr_status st = cpr_step(c, c->host_state, nsteps, dt_fixed, t_end);
    if (st != CPR_OK) return st;
    CPR_CUDA(c, cudaMemcpyAsync(qout, c->host_state, bytes, cudaMemcpyDeviceToHost, c->stream));
    CPR_CUDA(c, cudaStreamSynchronize(c->stream));
    return CPR_OK;
}

extern "C" cpr_status cpr_limit(cpr_ctx* c, void* q)
{
    if (!c) return CPR_EINVAL;
    if (c->cfg.scheme != CPR_SCHEME_CPR)
        return fail(c, CPR_EINVAL, "the FV schemes limit their slopes themselves: no troubled-cell limiter");
    if (!q) return fail(c, CPR_EINVAL, "q_dev must be non-NULL");
    if (!aligned(q)) return fail(c, CPR_EINVAL, "state arrays must be 16-byte aligned");
    CPR_CUDA(c, averages(c, q, c->avg, c->stream));
    CPR_CUDA(c, cudaMemsetAsync(&c->ctrl->marked, 0, sizeof(long long), c->stream));
    CPR_CUDA(c, limit(c, q, c->avg, 0, c->stream));
    return CPR_OK;
}

extern "C" cpr_status cpr_get_marks(cpr_ctx* c, int* marks)
{
    if (!c) return CPR_EINVAL;
    if (!marks) return fail(c, CPR_EINVAL, "marks_host must be non-NULL");
    CPR_CUDA(c, cudaMemcpyAsync(marks, c->marks, (size_t)c->ne * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CPR_CUDA(c, cudaStreamSynchronize(c->stream));
    return CPR_OK;
}

extern "C" cpr_status cpr_averages(cpr_ctx* c, const void* q, void* avg)
{
    if (!c) return CPR_EINVAL;
    if (!q || !avg) return fail(c, CPR_EINVAL, "q_dev and avg_dev must be non-NULL");
    CPR_CUDA(c, averages(c, q, avg, c->stream));
    return CPR_OK;
}

extern "C" cpr_status cpr_norms(cpr_ctx* c, const void* q, const void* ref, cpr_norms_out* out)
{
    if (!c) return CPR_EINVAL;
    if (!q || !out) return fail(c, CPR_EINVAL, "q_dev and out must be non-NULL");
    CPR_CUDA(c, norms(c, q, ref, c->stream));
    const size_t pb = (size_t)c->norm_blocks * cpr::kNormVals * sizeof(double);
    CPR_CUDA(c, cudaMemcpyAsync(c->h_partials, c->partials, pb, cudaMemcpyDeviceToHost, c->stream));
    CPR_CUDA(c, cudaMemcpyAsync(c->h_ctrl, c->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, c->stream));
    CPR_CUDA(c, cudaStreamSynchronize(c->stream));
    double acc[cpr::kNormVals] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int b = 0; b < c->norm_blocks; ++b)
        for (int k = 0; k < cpr::kNormVals; ++k) {
            const double v = c->h_partials[(size_t)b * cpr::kNormVals + k];
            if (k == 6) acc[k] = v > acc[k] ? v : acc[k];
            else acc[k] += v;
        }
    std::memset(out, 0, sizeof(*out));
    for (int v = 0; v < c->V; ++v) out->sum_avg[v] = acc[v];
    if (ref) {
        out->l2_abs = std::sqrt(acc[4]);
        out->l2_rel = acc[5] > 0.0 ? std::sqrt(acc[4] / acc[5]) : std::sqrt(acc[4]);
    }
    out->max_wave = acc[6];
    out->n_nonphys = (long long)acc[7];
    out->n_marked = c->h_ctrl->marked;
    out->t = c->h_ctrl->t;
    out->steps = c->h_ctrl->steps;
    return out->n_nonphys > 0 ? CPR_ENONPHYS : CPR_OK;
}

extern "C" cpr_status cpr_set_time(cpr_ctx* c, double t, long long steps)
{
    if (!c) return CPR_EINVAL;
    if (!std::isfinite(t) || steps < 0) return fail(c, CPR_EINVAL, "t must be finite and steps >= 0");
    ctrl_set_time_kernel<<<1, 1, 0, c->stream>>>(c->ctrl, t, steps);
    CPR_CUDA(c, cudaGetLastError());
    return CPR_OK;
}

extern "C" cpr_status cpr_get_time(cpr_ctx* c, double* t, long long* steps)
{
    if (!c) return CPR_EINVAL;
    CPR_CUDA(c, cudaMemcpyAsync(c->h_ctrl, c->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, c->stream));
    CPR_CUDA(c, cudaStreamSynchronize(c->stream));
    if (t) *t = c->h_ctrl->t;
    if (steps) *steps = c->h_ctrl->steps;
    return CPR_OK;
}

static cudaError_t vjp(cpr_ctx* c, const cpr::VjpPtrs& b, cudaStream_t s)
{
    return c->cfg.dtype == CPR_F32 ? cpr::launch_vjp<float>(c->lc, b, s, false)
                                   : cpr::launch_vjp<double>(c->lc, b, s, false);
}

static cpr_status vjp_check(cpr_ctx* c)
{
    if (c->cfg.div != CPR_DIV_LP) return fail(c, CPR_EINVAL, "the adjoint needs the LP divergence");
    if (c->cfg.limiter) return fail(c, CPR_EINVAL, "the adjoint covers unlimited runs only");
    CPR_CUDA(c, c->cfg.dtype == CPR_F32 ? cpr::launch_vjp<float>(c->lc, cpr::VjpPtrs{}, c->stream, true)
                                        : cpr::launch_vjp<double>(c->lc, cpr::VjpPtrs{}, c->stream, true));
    return CPR_OK;
}

extern "C" cpr_status cpr_residual_vjp(cpr_ctx* c, const void* q, const void* rbar, void* qbar)
{
    if (!c) return CPR_EINVAL;
    if (c->cfg.scheme != CPR_SCHEME_CPR) return fail(c, CPR_EINVAL, "no adjoint for the FV schemes");
    if (c->cfg.flux == CPR_FLUX_ROE) return fail(c, CPR_EINVAL, "no adjoint for the Roe flux");
    if (!q || !rbar || !qbar) return fail(c, CPR_EINVAL, "q_dev, rbar_dev and qbar_dev must be non-NULL");
    if (qbar == q || qbar == rbar) return fail(c, CPR_EINVAL, "qbar_dev must not alias q_dev or rbar_dev");
    if (!aligned(q) || !aligned(rbar) || !aligned(qbar)) return fail(c, CPR_EINVAL, "state arrays must be 16-byte aligned");
    cpr_status st = vjp_check(c);
    if (st != CPR_OK) return st;
    cpr::VjpPtrs b{q, rbar, qbar, nullptr, nullptr, nullptr, 0.0, 0.0, 0.0, 1.0};
    CPR_CUDA(c, vjp(c, b, c->stream));
    return CPR_OK;
}

// Checks shared by the step adjoint entry points.
static cpr_status step_adjoint_check(cpr_ctx* c, double dt)
{
    if (c->cfg.scheme != CPR_SCHEME_CPR) return fail(c, CPR_EINVAL, "no adjoint for the FV schemes");
    if (c->cfg.flux == CPR_FLUX_ROE) return fail(c, CPR_EINVAL, "no adjoint for the Roe flux");
    if (!(dt > 0.0) || !std::isfinite(dt)) return fail(c, CPR_EINVAL, "dt must be finite and > 0");
    return vjp_check(c);
}

// Transpose of one SSP-RK3 step from q with step dt around its stage states
// q1, q2:
//   b2 = 2/3 (qbar_out + dt J(q2)^T qbar_out)
//   b1 = 1/4 (b2 + dt J(q1)^T b2)
//   qbar_in = 1/3 qbar_out + 3/4 b2 + b1 + dt J(q)^T b1
static cpr_status step_vjp_chain(cpr_ctx* c, const void* q, const void* q1, const void* q2, const void* qbar_out,
                                 void* qbar_in, double dt)
{
    const size_t bytes = (size_t)c->nstate * c->esize;
    if (!c->adj1) CPR_CUDA(c, cudaMalloc(&c->adj1, bytes));
    if (!c->adj2) CPR_CUDA(c, cudaMalloc(&c->adj2, bytes));
    cpr::VjpPtrs b2{q2, qbar_out, c->adj1, qbar_out, nullptr, nullptr, 2.0 / 3.0, 0.0, 0.0, 2.0 / 3.0 * dt};
    CPR_CUDA(c, vjp(c, b2, c->stream));
    cpr::VjpPtrs b1{q1, c->adj1, c->adj2, c->adj1, nullptr, nullptr, 0.25, 0.0, 0.0, 0.25 * dt};
    CPR_CUDA(c, vjp(c, b1, c->stream));
    cpr::VjpPtrs b0{q, c->adj2, qbar_in, qbar_out, c->adj1, c->adj2, 1.0 / 3.0, 0.75, 1.0, dt};
    CPR_CUDA(c, vjp(c, b0, c->stream));
    return CPR_OK;
}

// Stage states of one Shu-Osher step of size dt (out = q_next).
static cpr_status so_stages(cpr_ctx* c, const void* q, void* q1, void* q2, void* q_next, double dt)
{
    ctrl_configure_kernel<<<1, 1, 0, c->stream>>>(c->ctrl, dt, 0.0, 0.0);
    CPR_CUDA(c, cudaGetLastError());
    CPR_CUDA(c, stage(c, cpr::MODE_SO1, q, nullptr, q1, nullptr, false, c->stream));
    CPR_CUDA(c, stage(c, cpr::MODE_SO2, q1, q, q2, nullptr, false, c->stream));
    if (q_next) CPR_CUDA(c, stage(c, cpr::MODE_SO3, q2, q, q_next, nullptr, false, c->stream));
    return CPR_OK;
}

// Transpose of one SSP-RK3 step from q with step dt, stages recomputed (in
// the context's stage buffers).
extern "C" cpr_status cpr_step_vjp(cpr_ctx* c, const void* q, const void* qbar_out, void* qbar_in, double dt)
{
    if (!c) return CPR_EINVAL;
    if (!q || !qbar_out || !qbar_in) return fail(c, CPR_EINVAL, "q_dev, qbar_out_dev and qbar_in_dev must be non-NULL");
    if (q == qbar_out || q == qbar_in) return fail(c, CPR_EINVAL, "q_dev must not alias the cotangents");
    if (!aligned(q) || !aligned(qbar_out) || !aligned(qbar_in))
        return fail(c, CPR_EINVAL, "state arrays must be 16-byte aligned");
    cpr_status st = step_adjoint_check(c, dt);
    if (st != CPR_OK) return st;
    if ((st = so_stages(c, q, c->q1, c->q2, nullptr, dt)) != CPR_OK) return st;
    return step_vjp_chain(c, q, c->q1, c->q2, qbar_out, qbar_in, dt);
}

extern "C" cpr_status cpr_step_stages(cpr_ctx* c, const void* q, void* q1, void* q2, void* q_next, double dt)
{
    if (!c) return CPR_EINVAL;
    if (!q || !q1 || !q2 || !q_next) return fail(c, CPR_EINVAL, "q_dev, q1_dev, q2_dev and q_next_dev must be non-NULL");
    if (q1 == q || q2 == q || q1 == q2 || q_next == q1 || q_next == q2)
        return fail(c, CPR_EINVAL, "q1_dev, q2_dev and q_next_dev must not alias q_dev or each other");
    if (!aligned(q) || !aligned(q1) || !aligned(q2) || !aligned(q_next))
        return fail(c, CPR_EINVAL, "state arrays must be 16-byte aligned");
    if (c->cfg.limiter) return fail(c, CPR_EINVAL, "the stage states of an unlimited step only");
    cpr_status st = step_adjoint_check(c, dt);
    if (st != CPR_OK) return st;
    return so_stages(c, q, q1, q2, q_next, dt);
}

extern "C" cpr_status cpr_step_vjp_stages(cpr_ctx* c, const void* q, const void* q1, const void* q2,
                                          const void* qbar_out, void* qbar_in, double dt)
{
    if (!c) return CPR_EINVAL;
    if (!q || !q1 || !q2 || !qbar_out || !qbar_in)
        return fail(c, CPR_EINVAL, "q_dev, q1_dev, q2_dev, qbar_out_dev and qbar_in_dev must be non-NULL");
    for (const void* x : {q, q1, q2})
        if (x == qbar_out || x == qbar_in) return fail(c, CPR_EINVAL, "the states must not alias the cotangents");
    if (!aligned(q) || !aligned(q1) || !aligned(q2) || !aligned(qbar_out) || !aligned(qbar_in))
        return fail(c, CPR_EINVAL, "state arrays must be 16-byte aligned");
    cpr_status st = step_adjoint_check(c, dt);
    if (st != CPR_OK) return st;
    return step_vjp_chain(c, q, q1, q2, qbar_out, qbar_in, dt);
}
