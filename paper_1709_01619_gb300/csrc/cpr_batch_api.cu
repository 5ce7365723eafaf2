// cpr_batch_api.cu -- C ABI of the batched solver (include/cpr.h, cpr_batch_*).
//
// A batch owns, per instance, two stage buffers, the low part of the state
// (FP32) and a time-control block; per order group, the device work-list
// tables of both tile families; and the CUDA graphs of the RK loop (one
// launch per order group and stage, or per-instance launch chains).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "cpr_batch.cuh"
#include "cpr_tabconv.cuh"
#include "cpr_internal.h"
#include "cpr_reduce.cuh"

using cpr::BatchArgs;
using cpr::BatchInst;
using cpr::Ctrl;
using cpr::LaunchCfg;
using cpr::StagePtrs;

namespace {

const int kBatchStepsPerGraph = 8;

struct Group {
    int p = 0;
    std::vector<int> members;                // instance indices
    int total[cpr::kBatchFamilies] = {0, 0};  // work items per family
    void* d_inst[cpr::kBatchFamilies] = {nullptr, nullptr};
    void* h_inst[cpr::kBatchFamilies] = {nullptr, nullptr};  // pinned mirrors
    int* d_map[cpr::kBatchFamilies] = {nullptr, nullptr};     // work item -> instance (member index)
    int fam = 0;                              // chosen tile family
    int grid = 0;                             // chosen grid (= total: one CTA per tile)
    int occ[cpr::kBatchFamilies] = {0, 0};    // resident CTAs per SM
};

thread_local std::string g_batch_init_err;

}  // namespace

struct cpr_batch {
    int n = 0;
    int V = 1;
    int dtype = CPR_F32;
    bool use_inc = false;
    cudaStream_t stream = nullptr;
    cudaStream_t cap = nullptr;
    int sms = 1;
    std::vector<cpr_config> cfgs;
    std::vector<LaunchCfg> lcs;
    std::vector<long long> nstate;
    std::vector<void*> Y, Z, lo;
    std::vector<void*> host_state;  // device copies for cpr_batch_step_host (first use)
    // cpr_batch_step_host in the per-instance form: a head graph whose chain
    // of instance i starts with the copy of its state in, and a tail graph
    // whose chain ends with the copy out, so that the copies of some
    // instances overlap the steps of others; bound to the host buffers (and
    // the run kind and tail length) they were captured for
    cudaGraphExec_t gh_head = nullptr, gh_tail = nullptr;
    std::vector<const void*> gh_in;
    std::vector<void*> gh_out;
    int gh_tail_steps = -1;
    int gh_cfl = -1;
    std::vector<int> order;  // instances by decreasing state size (copies of the largest first)
    // cpr_batch_step in the per-instance form: the same head and tail graphs
    // without the copies (the first CFL step sizes and cleared low parts of
    // every instance in its own chain instead of one stream)
    cudaGraphExec_t gd_head = nullptr, gd_tail = nullptr;
    int gd_tail_steps = -1;
    int gd_cfl = -1;
    Ctrl* ctrls = nullptr;
    Ctrl* h_ctrls = nullptr;      // pinned
    Ctrl* ctrl_backup = nullptr;  // device, for the autotuner
    std::vector<Group> groups;
    std::vector<const void*> x_cached;
    cudaGraphExec_t g1 = nullptr, g2 = nullptr, gK = nullptr;
    bool graphs_valid = false;
    // per-instance form (chosen by the autotuner): every instance runs the
    // single-problem stage kernel on a stream of its own inside the graphs,
    // its arguments in the kernel parameters; the chains join only at the
    // end of a graph
    bool per_inst = false;
    std::vector<cudaStream_t> ist;
    std::vector<cudaEvent_t> iev;
    cudaEvent_t fork_ev = nullptr;
    std::string err;
};

#define BATCH_CUDA(b, call)                                                                  \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess) {                                                             \
            (b)->err = std::string(#call) + ": " + cudaGetErrorString(e_);                   \
            return CPR_ECUDA;                                                                \
        }                                                                                    \
    } while (0)

namespace {

__global__ void batch_configure_kernel(Ctrl* c, int n, double dt_fixed, double t_end, const double* cfl_h)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    Ctrl* k = c + i;
    k->dt_fixed = dt_fixed;
    k->t_end = t_end;
    k->cfl_h = cfl_h[i];
    k->done = 0;
    k->counter = 0;
    k->parity = 0;
    if (dt_fixed > 0.0) cpr::ctrl_next_dt(k, k->max_wave);
}

// Increment form: instances whose state ended in Y after an odd number of
// steps are copied back to the caller's array.
template <class T>
__global__ void batch_parity_copy_kernel(const BatchInst<T>* inst, int V)
{
    const BatchInst<T>& I = inst[blockIdx.y];
    if (!I.ctrl->parity) return;
    const long long n = I.npts * V;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        I.X[i] = I.Y[i];
}

template <class T>
cudaError_t batch_launch(cpr_batch* b, Group& g, int fam, int grid, int mode, int swap, cudaStream_t s)
{
    BatchArgs<T> B;
    B.inst = static_cast<const BatchInst<T>*>(g.d_inst[fam]);
    B.tile_inst = g.d_map[fam];
    B.ninst = (int)g.members.size();
    B.total = g.total[fam];
    B.mode = mode;
    B.swap = swap;
    B.tab = cpr::host_tab<T>(b->lcs[g.members[0]].tab);
    B.tp = cpr::host_tabpr<T>(b->lcs[g.members[0]].tab);
    const LaunchCfg& lc = b->lcs[g.members[0]];
    return fam == 0 ? cpr::batch_fam<T, 0>(g.p, lc.eqn, lc.flux, B, grid, s, 0, nullptr)
                    : cpr::batch_fam<T, 1>(g.p, lc.eqn, lc.flux, B, grid, s, 0, nullptr);
}

cudaError_t batch_stage(cpr_batch* b, int mode, int swap, cudaStream_t s)
{
    for (Group& g : b->groups) {
        cudaError_t e = b->dtype == CPR_F32 ? batch_launch<float>(b, g, g.fam, g.grid, mode, swap, s)
                                            : batch_launch<double>(b, g, g.fam, g.grid, mode, swap, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// One RK3 step of every instance: increment form (FP32, high part in X when
// swap == 0, else in Y) or Shu-Osher stages (FP64).
cudaError_t batch_enqueue_step(cpr_batch* b, int swap, cudaStream_t s)
{
    cudaError_t e;
    if (b->use_inc) {
        if ((e = batch_stage(b, cpr::MODE_INC1, swap, s)) != cudaSuccess) return e;
        if ((e = batch_stage(b, cpr::MODE_INC2, swap, s)) != cudaSuccess) return e;
        return batch_stage(b, cpr::MODE_INC3, swap, s);
    }
    if ((e = batch_stage(b, cpr::MODE_SO1, 0, s)) != cudaSuccess) return e;
    if ((e = batch_stage(b, cpr::MODE_SO2, 0, s)) != cudaSuccess) return e;
    return batch_stage(b, cpr::MODE_SO3, 0, s);
}

// One stage of instance i with the single-problem kernel (buffers as in
// batch_item).
cudaError_t inst_stage(cpr_batch* b, int i, int mode, int swap, cudaStream_t s)
{
    void* X = const_cast<void*>(b->x_cached[i]);
    void* Y = b->Y[i];
    void* Z = b->Z[i];
    void* hiq = swap ? Y : X;
    void* other = swap ? X : Y;
    StagePtrs p{};
    p.lo = b->lo[i];
    switch (mode) {
    case cpr::MODE_SO1: p.qs = X; p.out = Y; break;
    case cpr::MODE_SO2: p.qs = Y; p.qn = X; p.out = Z; break;
    case cpr::MODE_SO3: p.qs = Z; p.qn = X; p.out = X; break;
    case cpr::MODE_INC1: p.qs = hiq; p.out = other; break;
    case cpr::MODE_INC2: p.qs = hiq; p.qb = other; p.out = Z; break;
    default: p.qs = hiq; p.qb = Z; p.out = other; break;
    }
    const bool wave = mode == cpr::MODE_SO3 || mode == cpr::MODE_INC3;
    return b->dtype == CPR_F32 ? cpr::launch_stage<float>(b->lcs[i], mode, p, wave, s)
                               : cpr::launch_stage<double>(b->lcs[i], mode, p, wave, s);
}

cudaError_t ensure_inst_streams(cpr_batch* b)
{
    if (!b->ist.empty()) return cudaSuccess;
    cudaError_t e = cudaEventCreateWithFlags(&b->fork_ev, cudaEventDisableTiming);
    for (int i = 0; i < b->n && e == cudaSuccess; ++i) {
        cudaStream_t st = nullptr;
        cudaEvent_t ev = nullptr;
        e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        b->ist.push_back(st);
        b->iev.push_back(ev);
    }
    for (int i = 0; i < b->n && e == cudaSuccess; ++i) {
        const LaunchCfg& lc = b->lcs[i];
        e = b->dtype == CPR_F32 ? cpr::prepare_stage<float>(lc) : cpr::prepare_stage<double>(lc);
    }
    return e;
}

// `steps` RK3 steps of instance i on stream si (the increment form's high
// part alternating between the caller's array and Y, starting in the
// caller's); timing: stages 1 and 2 only, as below.
cudaError_t enqueue_inst_steps(cpr_batch* b, int i, int steps, cudaStream_t si, bool timing)
{
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < steps && e == cudaSuccess; ++k) {
        if (timing) {
            e = inst_stage(b, i, b->use_inc ? cpr::MODE_INC1 : cpr::MODE_SO1, 0, si);
            if (e == cudaSuccess) e = inst_stage(b, i, b->use_inc ? cpr::MODE_INC2 : cpr::MODE_SO2, 0, si);
        } else if (b->use_inc) {
            const int sw = k % 2;
            e = inst_stage(b, i, cpr::MODE_INC1, sw, si);
            if (e == cudaSuccess) e = inst_stage(b, i, cpr::MODE_INC2, sw, si);
            if (e == cudaSuccess) e = inst_stage(b, i, cpr::MODE_INC3, sw, si);
        } else {
            e = inst_stage(b, i, cpr::MODE_SO1, 0, si);
            if (e == cudaSuccess) e = inst_stage(b, i, cpr::MODE_SO2, 0, si);
            if (e == cudaSuccess) e = inst_stage(b, i, cpr::MODE_SO3, 0, si);
        }
    }
    return e;
}

// Enqueue on s (which must be capturing) `steps` RK3 steps of every instance
// as independent chains: fork from s, one stream per instance, join back.
// timing != 0: only stages 1 and 2 with swap 0 (they leave the caller's
// states, the low parts and the time control untouched), for the autotuner.
cudaError_t enqueue_inst_chains(cpr_batch* b, int steps, cudaStream_t s, bool timing)
{
    cudaError_t e = cudaEventRecord(b->fork_ev, s);
    for (int i = 0; i < b->n && e == cudaSuccess; ++i) {
        cudaStream_t si = b->ist[i];
        e = cudaStreamWaitEvent(si, b->fork_ev, 0);
        if (e == cudaSuccess) e = enqueue_inst_steps(b, i, steps, si, timing);
        if (e == cudaSuccess) e = cudaEventRecord(b->iev[i], si);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, b->iev[i], 0);
    }
    return e;
}

cudaError_t batch_capture(cpr_batch* b, int steps, cudaGraphExec_t* exec)
{
    if (b->per_inst) {
        cudaGraph_t g = nullptr;
        cudaError_t e = ensure_inst_streams(b);
        if (e != cudaSuccess) return e;
        e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return e;
        const cudaError_t ee = enqueue_inst_chains(b, steps, b->cap, false);
        e = cudaStreamEndCapture(b->cap, &g);
        if (ee != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return ee;
        }
        if (e != cudaSuccess) return e;
        e = cudaGraphInstantiate(exec, g, 0);
        cudaGraphDestroy(g);
        return e;
    }
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    cudaError_t ee = cudaSuccess;
    for (int k = 0; k < steps && ee == cudaSuccess; ++k) ee = batch_enqueue_step(b, k % 2, b->cap);
    e = cudaStreamEndCapture(b->cap, &g);
    if (ee != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return ee;
    }
    if (e != cudaSuccess) return e;
    e = cudaGraphInstantiate(exec, g, 0);
    cudaGraphDestroy(g);
    return e;
}

void drop_graphs(cpr_batch* b)
{
    if (b->g1) cudaGraphExecDestroy(b->g1);
    if (b->g2) cudaGraphExecDestroy(b->g2);
    if (b->gK) cudaGraphExecDestroy(b->gK);
    if (b->gh_head) cudaGraphExecDestroy(b->gh_head);
    if (b->gh_tail) cudaGraphExecDestroy(b->gh_tail);
    if (b->gd_head) cudaGraphExecDestroy(b->gd_head);
    if (b->gd_tail) cudaGraphExecDestroy(b->gd_tail);
    b->g1 = b->g2 = b->gK = b->gh_head = b->gh_tail = b->gd_head = b->gd_tail = nullptr;
    b->gd_tail_steps = b->gd_cfl = -1;
    b->gh_in.clear();
    b->gh_out.clear();
    b->gh_tail_steps = b->gh_cfl = -1;
    b->graphs_valid = false;
}

cudaError_t ensure_batch_graphs(cpr_batch* b)
{
    if (b->graphs_valid) return cudaSuccess;
    drop_graphs(b);
    cudaError_t e = batch_capture(b, 1, &b->g1);
    if (e == cudaSuccess) e = batch_capture(b, 2, &b->g2);
    if (e == cudaSuccess) e = batch_capture(b, kBatchStepsPerGraph, &b->gK);
    b->graphs_valid = e == cudaSuccess;
    return e;
}

// Work-list tables of one dtype (host mirrors in pinned memory, device copy).
template <class T>
void fill_tables(cpr_batch* b, Group& g, const void* const* x)
{
    for (int fam = 0; fam < cpr::kBatchFamilies; ++fam) {
        int tx, ty;
        cpr::batch_tile(fam, &tx, &ty);
        BatchInst<T>* h = static_cast<BatchInst<T>*>(g.h_inst[fam]);
        int tile0 = 0;
        for (size_t m = 0; m < g.members.size(); ++m) {
            const int i = g.members[m];
            const LaunchCfg& lc = b->lcs[i];
            BatchInst<T>& I = h[m];
            I.X = static_cast<T*>(const_cast<void*>(x ? x[i] : nullptr));
            I.Y = static_cast<T*>(b->Y[i]);
            I.Z = static_cast<T*>(b->Z[i]);
            I.lo = static_cast<T*>(b->lo[i]);
            I.ctrl = b->ctrls + i;
            I.npts = lc.npts;
            I.nx = lc.nx;
            I.ny = lc.ny;
            I.bcx = lc.bcx;
            I.bcy = lc.bcy;
            I.tiles_x = (lc.nx + tx - 1) / tx;
            I.ntiles = I.tiles_x * ((lc.ny + ty - 1) / ty);
            I.tile0 = tile0;
            tile0 += I.ntiles;
            I.rhx2 = T(2.0 / lc.hx);
            I.rhy2 = T(2.0 / lc.hy);
            I.ph.gamma = T(lc.gamma);
            I.ph.ax = T(lc.ax);
            I.ph.ay = T(lc.ay);
        }
        g.total[fam] = tile0;
    }
}

template <class T>
cudaError_t upload_tables(cpr_batch* b, Group& g, cudaStream_t s)
{
    for (int fam = 0; fam < cpr::kBatchFamilies; ++fam) {
        cudaError_t e = cudaMemcpyAsync(g.d_inst[fam], g.h_inst[fam], sizeof(BatchInst<T>) * g.members.size(),
                                        cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Work item -> instance maps of both tile families (fixed for the batch's
// lifetime: they depend on the grids only).
cudaError_t build_tile_maps(cpr_batch* b, Group& g)
{
    for (int fam = 0; fam < cpr::kBatchFamilies; ++fam) {
        int tx, ty;
        cpr::batch_tile(fam, &tx, &ty);
        std::vector<int> map;
        map.reserve(g.total[fam]);
        for (size_t m = 0; m < g.members.size(); ++m) {
            const LaunchCfg& lc = b->lcs[g.members[m]];
            const int nt = ((lc.nx + tx - 1) / tx) * ((lc.ny + ty - 1) / ty);
            map.insert(map.end(), nt, (int)m);
        }
        if ((int)map.size() != g.total[fam]) return cudaErrorInvalidValue;
        cudaError_t e = cudaMalloc(&g.d_map[fam], sizeof(int) * map.size());
        if (e == cudaSuccess) e = cudaMemcpy(g.d_map[fam], map.data(), sizeof(int) * map.size(), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

template <class T>
cudaError_t group_occupancy(cpr_batch* b, Group& g)
{
    const LaunchCfg& lc = b->lcs[g.members[0]];
    BatchArgs<T> B{};
    for (int fam = 0; fam < cpr::kBatchFamilies; ++fam) {
        cudaError_t e = fam == 0 ? cpr::batch_fam<T, 0>(g.p, lc.eqn, lc.flux, B, 0, 0, 1, nullptr)
                                 : cpr::batch_fam<T, 1>(g.p, lc.eqn, lc.flux, B, 0, 0, 1, nullptr);
        if (e != cudaSuccess) return e;
        e = fam == 0 ? cpr::batch_fam<T, 0>(g.p, lc.eqn, lc.flux, B, 0, 0, 2, &g.occ[0])
                     : cpr::batch_fam<T, 1>(g.p, lc.eqn, lc.flux, B, 0, 0, 2, &g.occ[1]);
        if (e != cudaSuccess) return e;
        g.occ[fam] = std::max(1, g.occ[fam]);
    }
    g.fam = 0;
    g.grid = g.total[0];  // untuned: one CTA per tile
    return cudaSuccess;
}

void free_batch(cpr_batch* b)
{
    drop_graphs(b);
    for (void* p : b->Y) cudaFree(p);
    for (void* p : b->Z) cudaFree(p);
    for (void* p : b->lo) cudaFree(p);
    for (void* p : b->host_state) cudaFree(p);
    for (Group& g : b->groups)
        for (int f = 0; f < cpr::kBatchFamilies; ++f) {
            cudaFree(g.d_inst[f]);
            cudaFree(g.d_map[f]);
            if (g.h_inst[f]) cudaFreeHost(g.h_inst[f]);
        }
    cudaFree(b->ctrls);
    cudaFree(b->ctrl_backup);
    if (b->h_ctrls) cudaFreeHost(b->h_ctrls);
    if (b->cap) cudaStreamDestroy(b->cap);
    for (cudaStream_t st : b->ist)
        if (st) cudaStreamDestroy(st);
    for (cudaEvent_t ev : b->iev)
        if (ev) cudaEventDestroy(ev);
    if (b->fork_ev) cudaEventDestroy(b->fork_ev);
}

}  // namespace

extern "C" cpr_status cpr_batch_init(const cpr_config* cfgs, int n, void* stream, cpr_batch** out)
{
    if (!out) {
        g_batch_init_err = "out is NULL";
        return CPR_EINVAL;
    }
    *out = nullptr;
    if (!cfgs || n < 1) {
        g_batch_init_err = "cfgs must hold n >= 1 configurations";
        return CPR_EINVAL;
    }
    for (int i = 0; i < n; ++i) {
        if (const char* msg = cpr_validate_config(&cfgs[i])) {
            g_batch_init_err = std::string("instance ") + std::to_string(i) + ": " + msg;
            return CPR_EINVAL;
        }
        const cpr_config& a = cfgs[0];
        const cpr_config& c = cfgs[i];
        if (c.eqn != a.eqn || c.dtype != a.dtype || c.flux != a.flux) {
            g_batch_init_err = "all instances need the same eqn, dtype and flux";
            return CPR_EINVAL;
        }
        if (c.scheme != CPR_SCHEME_CPR || c.div != CPR_DIV_LP || c.pts != CPR_PTS_GAUSS || c.limiter ||
            c.flux == CPR_FLUX_ROE) {
            g_batch_init_err = "batches run CPR with Gauss points, LP divergence, no limiter, Rusanov or upwind flux";
            return CPR_EINVAL;
        }
    }
    cpr_batch* b = new (std::nothrow) cpr_batch();
    if (!b) {
        g_batch_init_err = "host allocation failed";
        return CPR_ENOMEM;
    }
    b->n = n;
    b->V = cfgs[0].eqn == CPR_EULER ? 4 : 1;
    b->dtype = cfgs[0].dtype;
    b->use_inc = b->dtype == CPR_F32;
    b->stream = static_cast<cudaStream_t>(stream);
    b->cfgs.assign(cfgs, cfgs + n);
    b->lcs.resize(n);
    b->nstate.resize(n);
    b->Y.assign(n, nullptr);
    b->Z.assign(n, nullptr);
    b->lo.assign(n, nullptr);
    const size_t esize = b->dtype == CPR_F32 ? 4 : 8;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev);
    for (int i = 0; i < n && e == cudaSuccess; ++i) {
        if (!cpr_fill_launch_cfg(&cfgs[i], &b->lcs[i])) {
            free_batch(b);
            delete b;
            g_batch_init_err = "table construction failed";
            return CPR_EINVAL;
        }
        LaunchCfg& lc = b->lcs[i];
        // instances share the SMs: keep the stage kernel that four CTAs of
        // any instances can share (the two-CTA instantiation in per-instance
        // chains measured slower on 64 ragged instances)
        lc.sms = 0;
        b->nstate[i] = lc.npts * b->V;
        const size_t bytes = (size_t)b->nstate[i] * esize;
        e = cudaMalloc(&b->Y[i], bytes);
        if (e == cudaSuccess) e = cudaMalloc(&b->Z[i], bytes);
        if (e == cudaSuccess && b->use_inc) e = cudaMalloc(&b->lo[i], bytes);
    }
    if (e == cudaSuccess) e = cudaMalloc((void**)&b->ctrls, sizeof(Ctrl) * n);
    if (e == cudaSuccess) e = cudaMalloc((void**)&b->ctrl_backup, sizeof(Ctrl) * n);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&b->h_ctrls, sizeof(Ctrl) * n);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->ctrls, 0, sizeof(Ctrl) * n, b->stream);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
    for (int i = 0; i < n && e == cudaSuccess; ++i) {
        b->lcs[i].ctrl = b->ctrls + i;
    }
    // order groups
    for (int p = 1; p <= 4 && e == cudaSuccess; ++p) {
        Group g;
        g.p = p;
        for (int i = 0; i < n; ++i)
            if (cfgs[i].p == p) g.members.push_back(i);
        if (g.members.empty()) continue;
        const size_t isz = (b->dtype == CPR_F32 ? sizeof(BatchInst<float>) : sizeof(BatchInst<double>)) *
                           g.members.size();
        for (int fam = 0; fam < cpr::kBatchFamilies && e == cudaSuccess; ++fam) {
            e = cudaMalloc(&g.d_inst[fam], isz);
            if (e == cudaSuccess) e = cudaMallocHost(&g.h_inst[fam], isz);
        }
        if (e != cudaSuccess) break;
        if (b->dtype == CPR_F32) {
            fill_tables<float>(b, g, nullptr);
            e = group_occupancy<float>(b, g);
        } else {
            fill_tables<double>(b, g, nullptr);
            e = group_occupancy<double>(b, g);
        }
        if (e == cudaSuccess) e = build_tile_maps(b, g);
        b->groups.push_back(g);
    }
    if (e != cudaSuccess) {
        g_batch_init_err = std::string("CUDA: ") + cudaGetErrorString(e);
        const cpr_status st = e == cudaErrorMemoryAllocation ? CPR_ENOMEM : CPR_ECUDA;
        free_batch(b);
        delete b;
        return st;
    }
    b->x_cached.assign(n, nullptr);
    *out = b;
    return CPR_OK;
}

extern "C" void cpr_batch_destroy(cpr_batch* b)
{
    if (!b) return;
    cudaStreamSynchronize(b->stream);
    free_batch(b);
    delete b;
}

extern "C" const char* cpr_batch_last_error(const cpr_batch* b)
{
    return b ? b->err.c_str() : g_batch_init_err.c_str();
}

static cpr_status batch_bind(cpr_batch* b, void* const* q)
{
    if (!q) {
        b->err = "q_devs must be non-NULL";
        return CPR_EINVAL;
    }
    bool changed = false;
    for (int i = 0; i < b->n; ++i) {
        if (!q[i] || (reinterpret_cast<uintptr_t>(q[i]) & 15u)) {
            b->err = "every q_devs[i] must be a non-NULL 16-byte aligned device array";
            return CPR_EINVAL;
        }
        changed = changed || q[i] != b->x_cached[i];
    }
    if (!changed) return CPR_OK;
    // the device tables are read by graphs in flight: wait before rewriting
    BATCH_CUDA(b, cudaStreamSynchronize(b->stream));
    for (Group& g : b->groups) {
        if (b->dtype == CPR_F32) {
            fill_tables<float>(b, g, q);
            BATCH_CUDA(b, upload_tables<float>(b, g, b->stream));
        } else {
            fill_tables<double>(b, g, q);
            BATCH_CUDA(b, upload_tables<double>(b, g, b->stream));
        }
    }
    for (int i = 0; i < b->n; ++i) b->x_cached[i] = q[i];
    if (b->per_inst) drop_graphs(b);  // their kernel parameters hold the pointers
    return CPR_OK;
}

// The step size and end time of every instance's control block; then, unless
// the caller's graphs do it per instance (in_graph), the first CFL step size
// of every instance and the cleared low parts.
static cpr_status batch_prelude(cpr_batch* b, void* const* q, double dt_fixed, double t_end, double* cfl_h_dev,
                                bool in_graph)
{
    batch_configure_kernel<<<(b->n + 127) / 128, 128, 0, b->stream>>>(b->ctrls, b->n, dt_fixed, t_end, cfl_h_dev);
    BATCH_CUDA(b, cudaGetLastError());
    if (in_graph) return CPR_OK;
    if (dt_fixed <= 0.0)
        for (int i = 0; i < b->n; ++i)
            BATCH_CUDA(b, b->dtype == CPR_F32 ? cpr::launch_wave<float>(b->lcs[i], q[i], b->stream)
                                              : cpr::launch_wave<double>(b->lcs[i], q[i], b->stream));
    if (b->use_inc)
        for (int i = 0; i < b->n; ++i)
            BATCH_CUDA(b, cudaMemsetAsync(b->lo[i], 0, (size_t)b->nstate[i] * 4, b->stream));
    return CPR_OK;
}

// Argument checks, binding and the prelude shared by the device and host
// entry points; *run is false when there is nothing to step.
static cpr_status batch_begin(cpr_batch* b, void* const* q, int nsteps, double dt_fixed, double t_end,
                              bool in_graph, bool* run)
{
    *run = false;
    if (nsteps < 0 || !std::isfinite(dt_fixed) || !std::isfinite(t_end)) {
        b->err = "nsteps must be >= 0, dt_fixed and t_end finite";
        return CPR_EINVAL;
    }
    if (dt_fixed <= 0.0)
        for (const cpr_config& c : b->cfgs)
            if (!(c.cfl > 0.0)) {
                b->err = "CFL steps need cfg.cfl > 0 for every instance";
                return CPR_EINVAL;
            }
    cpr_status st = batch_bind(b, q);
    if (st != CPR_OK || nsteps == 0) return st;
    // per-instance cfl * h, staged through the pinned control mirror
    double* cflh = reinterpret_cast<double*>(b->h_ctrls);
    static_assert(sizeof(Ctrl) >= sizeof(double), "control block too small");
    BATCH_CUDA(b, cudaStreamSynchronize(b->stream));
    for (int i = 0; i < b->n; ++i) cflh[i] = b->cfgs[i].cfl * std::min(b->lcs[i].hx, b->lcs[i].hy);
    double* cflh_dev = reinterpret_cast<double*>(b->ctrl_backup);
    BATCH_CUDA(b, cudaMemcpyAsync(cflh_dev, cflh, sizeof(double) * b->n, cudaMemcpyHostToDevice, b->stream));
    if ((st = batch_prelude(b, q, dt_fixed, t_end, cflh_dev, in_graph)) != CPR_OK) return st;
    *run = true;
    return CPR_OK;
}

// Head (head = true) or tail graph of a run in the per-instance form: per
// instance, on its own stream, largest first, the copy of its state in (host
// entry point: q_in), its first CFL step size (cfl) and cleared low part,
// then `steps` steps (head); or `steps` steps, the copy back of a state left
// in Y and the copy of the state out (q_out) (tail).  The instance states are
// the bound arrays (x_cached).
static cudaError_t capture_chain_graph(cpr_batch* b, bool head, const void* const* q_in, void* const* q_out,
                                      int steps, bool cfl, cudaGraphExec_t* exec)
{
    const size_t esize = b->dtype == CPR_F32 ? 4 : 8;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    cudaError_t ee = cudaEventRecord(b->fork_ev, b->cap);
    for (int r = 0; r < b->n && ee == cudaSuccess; ++r) {
        const int i = b->order[r];
        cudaStream_t si = b->ist[i];
        const size_t bytes = (size_t)b->nstate[i] * esize;
        ee = cudaStreamWaitEvent(si, b->fork_ev, 0);
        void* X = const_cast<void*>(b->x_cached[i]);
        if (head) {
            if (ee == cudaSuccess && q_in)
                ee = cudaMemcpyAsync(X, q_in[i], bytes, cudaMemcpyHostToDevice, si);
            if (ee == cudaSuccess && cfl)
                ee = b->dtype == CPR_F32 ? cpr::launch_wave<float>(b->lcs[i], X, si)
                                         : cpr::launch_wave<double>(b->lcs[i], X, si);
            if (ee == cudaSuccess && b->use_inc) ee = cudaMemsetAsync(b->lo[i], 0, (size_t)b->nstate[i] * 4, si);
        }
        if (ee == cudaSuccess) ee = enqueue_inst_steps(b, i, steps, si, false);
        if (!head) {
            if (ee == cudaSuccess && b->use_inc) {
                // this instance's entry in its order group's table
                for (Group& gr : b->groups)
                    for (size_t m = 0; m < gr.members.size(); ++m)
                        if (gr.members[m] == i) {
                            batch_parity_copy_kernel<float><<<dim3(64, 1), 256, 0, si>>>(
                                static_cast<const BatchInst<float>*>(gr.d_inst[0]) + m, b->V);
                            ee = cudaGetLastError();
                        }
            }
            if (ee == cudaSuccess && q_out)
                ee = cudaMemcpyAsync(q_out[i], X, bytes, cudaMemcpyDeviceToHost, si);
        }
        if (ee == cudaSuccess) ee = cudaEventRecord(b->iev[i], si);
        if (ee == cudaSuccess) ee = cudaStreamWaitEvent(b->cap, b->iev[i], 0);
    }
    e = cudaStreamEndCapture(b->cap, &g);
    if (ee != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return ee;
    }
    if (e != cudaSuccess) return e;
    e = cudaGraphInstantiate(exec, g, 0);
    cudaGraphDestroy(g);
    return e;
}

// Every host buffer page-locked (a copy from pageable memory cannot be
// captured in a graph).
static bool all_pinned(int n, const void* const* a)
{
    for (int i = 0; i < n; ++i) {
        cudaPointerAttributes at{};
        if (cudaPointerGetAttributes(&at, a[i]) != cudaSuccess) {
            (void)cudaGetLastError();
            return false;
        }
        if (at.type != cudaMemoryTypeHost) return false;
    }
    return true;
}

// A run of nsteps >= 2K steps in the per-instance form: the head graph (K
// steps), K-step graphs, the tail graph (K..2K-1 steps); q_in / q_out: the
// host buffers of the host entry point (null: the device one).
static cpr_status run_chains(cpr_batch* b, int nsteps, double dt_fixed, const void* const* q_in, void* const* q_out)
{
    const int K = kBatchStepsPerGraph;
    BATCH_CUDA(b, ensure_inst_streams(b));
    if ((int)b->order.size() != b->n) {
        b->order.resize(b->n);
        for (int i = 0; i < b->n; ++i) b->order[i] = i;
        std::stable_sort(b->order.begin(), b->order.end(),
                         [b](int x, int y) { return b->nstate[x] > b->nstate[y]; });
    }
    BATCH_CUDA(b, ensure_batch_graphs(b));
    const int tail = K + nsteps % K, mid = (nsteps - K - tail) / K;
    const int cfl = dt_fixed <= 0.0 ? 1 : 0;
    cudaGraphExec_t* head = &b->gd_head;
    cudaGraphExec_t* tailg = &b->gd_tail;
    if (q_in) {
        head = &b->gh_head;
        tailg = &b->gh_tail;
        const bool same_in = (int)b->gh_in.size() == b->n && std::equal(b->gh_in.begin(), b->gh_in.end(), q_in);
        const bool same_out =
            (int)b->gh_out.size() == b->n && std::equal(b->gh_out.begin(), b->gh_out.end(), q_out);
        if (!b->gh_head || !same_in || b->gh_cfl != cfl) {
            if (b->gh_head) cudaGraphExecDestroy(b->gh_head);
            b->gh_head = nullptr;
            b->gh_in.clear();
            BATCH_CUDA(b, capture_chain_graph(b, true, q_in, q_out, K, cfl != 0, &b->gh_head));
            b->gh_in.assign(q_in, q_in + b->n);
            b->gh_cfl = cfl;
        }
        if (!b->gh_tail || !same_out || b->gh_tail_steps != tail) {
            if (b->gh_tail) cudaGraphExecDestroy(b->gh_tail);
            b->gh_tail = nullptr;
            b->gh_out.clear();
            BATCH_CUDA(b, capture_chain_graph(b, false, q_in, q_out, tail, cfl != 0, &b->gh_tail));
            b->gh_out.assign(q_out, q_out + b->n);
            b->gh_tail_steps = tail;
        }
    } else {
        if (!b->gd_head || b->gd_cfl != cfl) {
            if (b->gd_head) cudaGraphExecDestroy(b->gd_head);
            b->gd_head = nullptr;
            BATCH_CUDA(b, capture_chain_graph(b, true, nullptr, nullptr, K, cfl != 0, &b->gd_head));
            b->gd_cfl = cfl;
        }
        if (!b->gd_tail || b->gd_tail_steps != tail) {
            if (b->gd_tail) cudaGraphExecDestroy(b->gd_tail);
            b->gd_tail = nullptr;
            BATCH_CUDA(b, capture_chain_graph(b, false, nullptr, nullptr, tail, cfl != 0, &b->gd_tail));
            b->gd_tail_steps = tail;
        }
    }
    BATCH_CUDA(b, cudaGraphLaunch(*head, b->stream));
    for (int k = 0; k < mid; ++k) BATCH_CUDA(b, cudaGraphLaunch(b->gK, b->stream));
    BATCH_CUDA(b, cudaGraphLaunch(*tailg, b->stream));
    return CPR_OK;
}

extern "C" cpr_status cpr_batch_step(cpr_batch* b, void* const* q, int nsteps, double dt_fixed, double t_end)
{
    if (!b) return CPR_EINVAL;
    // per-instance form: the first CFL step sizes, the cleared low parts and
    // the copies back of states left in Y inside the instances' own chains
    const bool chains = b->per_inst && nsteps >= 2 * kBatchStepsPerGraph;
    bool run = false;
    cpr_status st = batch_begin(b, q, nsteps, dt_fixed, t_end, chains, &run);
    if (st != CPR_OK || !run) return st;
    if (chains) return run_chains(b, nsteps, dt_fixed, nullptr, nullptr);
    BATCH_CUDA(b, ensure_batch_graphs(b));
    for (int k = 0; k < nsteps / kBatchStepsPerGraph; ++k) BATCH_CUDA(b, cudaGraphLaunch(b->gK, b->stream));
    const int rest = nsteps % kBatchStepsPerGraph;
    if (b->use_inc) {
        for (int k = 0; k < rest / 2; ++k) BATCH_CUDA(b, cudaGraphLaunch(b->g2, b->stream));
        if (rest % 2) BATCH_CUDA(b, cudaGraphLaunch(b->g1, b->stream));
        for (Group& g : b->groups) {
            batch_parity_copy_kernel<float><<<dim3(64, (unsigned)g.members.size()), 256, 0, b->stream>>>(
                static_cast<const BatchInst<float>*>(g.d_inst[0]), b->V);
            BATCH_CUDA(b, cudaGetLastError());
        }
    } else {
        for (int k = 0; k < rest; ++k) BATCH_CUDA(b, cudaGraphLaunch(b->g1, b->stream));
    }
    return CPR_OK;
}

extern "C" cpr_status cpr_batch_step_host(cpr_batch* b, const void* const* q_in, void* const* q_out, int nsteps,
                                          double dt_fixed, double t_end)
{
    if (!b) return CPR_EINVAL;
    if (!q_in || !q_out) {
        b->err = "q_in_host and q_out_host must be non-NULL";
        return CPR_EINVAL;
    }
    for (int i = 0; i < b->n; ++i)
        if (!q_in[i] || !q_out[i]) {
            b->err = "every host buffer must be non-NULL";
            return CPR_EINVAL;
        }
    const size_t esize = b->dtype == CPR_F32 ? 4 : 8;
    if (b->host_state.empty()) {
        b->host_state.assign(b->n, nullptr);
        for (int i = 0; i < b->n; ++i) {
            const cudaError_t e = cudaMalloc(&b->host_state[i], (size_t)b->nstate[i] * esize);
            if (e != cudaSuccess) {
                for (void* p : b->host_state) cudaFree(p);
                b->host_state.clear();
                b->err = std::string("cudaMalloc: ") + cudaGetErrorString(e);
                return e == cudaErrorMemoryAllocation ? CPR_ENOMEM : CPR_ECUDA;
            }
        }
    }
    const int K = kBatchStepsPerGraph;
    const bool overlap = b->per_inst && nsteps >= 2 * K && all_pinned(b->n, q_in) &&
                         all_pinned(b->n, const_cast<const void* const*>(q_out));
    if (!overlap) {
        // grouped form, short runs or pageable buffers: copies in, the steps,
        // copies out, one after the other
        for (int i = 0; i < b->n; ++i)
            BATCH_CUDA(b, cudaMemcpyAsync(b->host_state[i], q_in[i], (size_t)b->nstate[i] * esize,
                                          cudaMemcpyHostToDevice, b->stream));
        const cpr_status st = cpr_batch_step(b, b->host_state.data(), nsteps, dt_fixed, t_end);
        if (st != CPR_OK) return st;
        for (int i = 0; i < b->n; ++i)
            BATCH_CUDA(b, cudaMemcpyAsync(q_out[i], b->host_state[i], (size_t)b->nstate[i] * esize,
                                          cudaMemcpyDeviceToHost, b->stream));
        BATCH_CUDA(b, cudaStreamSynchronize(b->stream));
        return CPR_OK;
    }
    // Per-instance form: the head graph copies each instance in and runs its
    // first K steps on its own stream (largest instances first), so later
    // copies overlap earlier instances' steps; the middle runs the usual
    // K-step graphs; the tail graph runs each instance's last K..2K-1 steps
    // and copies it out, overlapping the copies of the instances that finish
    // first with the steps of the others.  The same kernels in the same
    // order per instance: the results equal the device entry point's.
    bool run = false;
    cpr_status st = batch_begin(b, b->host_state.data(), nsteps, dt_fixed, t_end, true, &run);
    if (st != CPR_OK || !run) return st;
    if ((st = run_chains(b, nsteps, dt_fixed, q_in, q_out)) != CPR_OK) return st;
    BATCH_CUDA(b, cudaStreamSynchronize(b->stream));
    return CPR_OK;
}

extern "C" cpr_status cpr_batch_set_form(cpr_batch* b, int per_instance)
{
    if (!b) return CPR_EINVAL;
    if (per_instance != 0 && per_instance != 1) {
        b->err = "per_instance must be 0 or 1";
        return CPR_EINVAL;
    }
    BATCH_CUDA(b, cudaStreamSynchronize(b->stream));
    b->per_inst = per_instance != 0;
    drop_graphs(b);
    return CPR_OK;
}

extern "C" cpr_status cpr_batch_get_time(cpr_batch* b, int i, double* t, long long* steps)
{
    if (!b) return CPR_EINVAL;
    if (i < 0 || i >= b->n) {
        b->err = "instance index out of range";
        return CPR_EINVAL;
    }
    BATCH_CUDA(b, cudaMemcpyAsync(b->h_ctrls + i, b->ctrls + i, sizeof(Ctrl), cudaMemcpyDeviceToHost, b->stream));
    BATCH_CUDA(b, cudaStreamSynchronize(b->stream));
    if (t) *t = b->h_ctrls[i].t;
    if (steps) *steps = b->h_ctrls[i].steps;
    return CPR_OK;
}

extern "C" cpr_status cpr_batch_set_time(cpr_batch* b, double t, long long steps)
{
    if (!b) return CPR_EINVAL;
    if (!std::isfinite(t) || steps < 0) {
        b->err = "t must be finite and steps >= 0";
        return CPR_EINVAL;
    }
    BATCH_CUDA(b, cudaStreamSynchronize(b->stream));
    BATCH_CUDA(b, cudaMemcpy(b->h_ctrls, b->ctrls, sizeof(Ctrl) * b->n, cudaMemcpyDeviceToHost));
    for (int i = 0; i < b->n; ++i) {
        b->h_ctrls[i].t = t;
        b->h_ctrls[i].steps = steps;
        b->h_ctrls[i].done = 0;
        b->h_ctrls[i].last = 0;
    }
    BATCH_CUDA(b, cudaMemcpy(b->ctrls, b->h_ctrls, sizeof(Ctrl) * b->n, cudaMemcpyHostToDevice));
    return CPR_OK;
}

// Autotuner: for every order group, time one RK3 step of that group (the
// stages that leave the caller's arrays untouched) for every tile family,
// with one CTA per tile and with every persistent grid of 1..occupancy CTAs
// per SM that is smaller than that, and keep the fastest.  The time-control blocks are saved and restored around the runs.
extern "C" cpr_status cpr_batch_tune(cpr_batch* b, void* const* q, int* choices, int* ngroups)
{
    if (!b) return CPR_EINVAL;
    cpr_status st = batch_bind(b, q);
    if (st != CPR_OK) return st;
    BATCH_CUDA(b, cudaMemcpyAsync(b->ctrl_backup, b->ctrls, sizeof(Ctrl) * b->n, cudaMemcpyDeviceToDevice,
                                  b->stream));
    // a small fixed step, no end time, for the timing runs
    batch_configure_kernel<<<(b->n + 127) / 128, 128, 0, b->stream>>>(b->ctrls, b->n, 1e-6, 0.0,
                                                                       reinterpret_cast<double*>(b->ctrl_backup));
    BATCH_CUDA(b, cudaGetLastError());
    cudaEvent_t e0, e1;
    BATCH_CUDA(b, cudaEventCreate(&e0));
    BATCH_CUDA(b, cudaEventCreate(&e1));
    const int modes_inc[3] = {cpr::MODE_INC1, cpr::MODE_INC2, cpr::MODE_INC3};
    const int modes_so[2] = {cpr::MODE_SO1, cpr::MODE_SO2};  // SO3 writes the state
    for (Group& g : b->groups) {
        float best = 1e30f;
        int best_fam = g.fam, best_grid = g.grid;
        for (int fam = 0; fam < cpr::kBatchFamilies; ++fam)
            for (int c = 0; c <= g.occ[fam]; ++c) {
                // c = 0: one CTA per tile; c >= 1: persistent grid of c CTAs per SM
                if (c > 0 && b->sms * c >= g.total[fam]) break;
                const int grid = c == 0 ? g.total[fam] : b->sms * c;
                auto run = [&]() -> cudaError_t {
                    const int nm = b->use_inc ? 3 : 2;
                    for (int m = 0; m < nm; ++m) {
                        const int mode = b->use_inc ? modes_inc[m] : modes_so[m];
                        cudaError_t e = b->dtype == CPR_F32 ? batch_launch<float>(b, g, fam, grid, mode, 0, b->stream)
                                                            : batch_launch<double>(b, g, fam, grid, mode, 0, b->stream);
                        if (e != cudaSuccess) return e;
                    }
                    return cudaSuccess;
                };
                BATCH_CUDA(b, run());
                BATCH_CUDA(b, cudaEventRecord(e0, b->stream));
                for (int r = 0; r < 3; ++r) BATCH_CUDA(b, run());
                BATCH_CUDA(b, cudaEventRecord(e1, b->stream));
                BATCH_CUDA(b, cudaEventSynchronize(e1));
                float ms = 0.f;
                BATCH_CUDA(b, cudaEventElapsedTime(&ms, e0, e1));
                if (ms < best) {
                    best = ms;
                    best_fam = fam;
                    best_grid = grid;
                }
            }
        g.fam = best_fam;
        g.grid = best_grid;
    }
    // The grouped launches just chosen against per-instance chains (stages 1
    // and 2 of every instance, each form captured in a graph and timed over
    // three replays).
    {
        auto timed = [&](bool inst, float* ms) -> cudaError_t {
            cudaGraph_t gr = nullptr;
            cudaGraphExec_t ex = nullptr;
            cudaError_t e = inst ? ensure_inst_streams(b) : cudaSuccess;
            if (e != cudaSuccess) return e;
            e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
            if (e != cudaSuccess) return e;
            cudaError_t ee = cudaSuccess;
            if (inst) {
                ee = enqueue_inst_chains(b, 1, b->cap, true);
            } else {
                for (int m = 0; m < 2 && ee == cudaSuccess; ++m) {
                    const int mode = b->use_inc ? modes_inc[m] : modes_so[m];
                    for (Group& g : b->groups) {
                        ee = b->dtype == CPR_F32 ? batch_launch<float>(b, g, g.fam, g.grid, mode, 0, b->cap)
                                                 : batch_launch<double>(b, g, g.fam, g.grid, mode, 0, b->cap);
                        if (ee != cudaSuccess) break;
                    }
                }
            }
            e = cudaStreamEndCapture(b->cap, &gr);
            if (ee == cudaSuccess && e == cudaSuccess) e = cudaGraphInstantiate(&ex, gr, 0);
            if (gr) cudaGraphDestroy(gr);
            if (ee != cudaSuccess) e = ee;
            if (e == cudaSuccess) e = cudaGraphLaunch(ex, b->stream);
            if (e == cudaSuccess) e = cudaEventRecord(e0, b->stream);
            for (int r = 0; r < 3 && e == cudaSuccess; ++r) e = cudaGraphLaunch(ex, b->stream);
            if (e == cudaSuccess) e = cudaEventRecord(e1, b->stream);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
            if (ex) cudaGraphExecDestroy(ex);
            return e;
        };
        float t_grouped = 0.f, t_inst = 0.f;
        BATCH_CUDA(b, timed(false, &t_grouped));
        BATCH_CUDA(b, timed(true, &t_inst));
        b->per_inst = t_inst < t_grouped;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    BATCH_CUDA(b, cudaMemcpyAsync(b->ctrls, b->ctrl_backup, sizeof(Ctrl) * b->n, cudaMemcpyDeviceToDevice,
                                  b->stream));
    BATCH_CUDA(b, cudaStreamSynchronize(b->stream));
    drop_graphs(b);
    if (ngroups) *ngroups = (int)b->groups.size();
    if (choices)
        for (size_t k = 0; k < b->groups.size(); ++k) {
            choices[3 * k] = b->groups[k].p;
            choices[3 * k + 1] = b->per_inst ? 2 : b->groups[k].fam;
            choices[3 * k + 2] = b->per_inst ? 0 : b->groups[k].grid;
        }
    return CPR_OK;
}
