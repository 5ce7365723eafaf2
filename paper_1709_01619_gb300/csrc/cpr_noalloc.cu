// cpr_noalloc.cu -- cpr_step_noalloc: fixed-step SSP-RK3 steps without any
// device allocation.
//
// Some callers cannot let a library allocate device memory: a host framework
// that owns the whole device through its own pool allocator (a cudaMalloc
// behind its back can fail or break its accounting), or a latency-critical
// loop where cudaMalloc/cudaFree, which may synchronise the device, are not
// allowed.  For them this entry point runs the same stage kernels as
// cpr_step, with the two stage buffers and the small control block in one
// file-scope device array instead of context-owned allocations.
//
// The array is kNoAllocStateBytes * 2 + kNoAllocCtrlBytes bytes; every GPU
// that loads libcpr.so holds it until the process exits.  All calls share
// it and it keeps the previous call's contents, so the control block is
// rewritten at the start of every call, and calls that overlap on the GPU
// (different streams, or threads without ordering between them) race on it.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <mutex>

#include "../../include/cpr.h"
#include "cpr_launch.h"

namespace {

constexpr size_t kNoAllocCtrlBytes = 256;
constexpr size_t kNoAllocStateBytes = CPR_NOALLOC_MAX_STATE_BYTES;
constexpr size_t kNoAllocBytes = kNoAllocCtrlBytes + 2 * kNoAllocStateBytes;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

std::mutex g_mutex;
void* g_scratch_addr[kMaxDevices] = {};

__global__ void noalloc_ctrl_init(cpr::Ctrl* c, double dt)
{
    c->t = 0.0;
    c->dt = dt;
    c->t_end = 0.0;
    c->dt_fixed = dt;
    c->cfl_h = 0.0;
    c->max_wave = 0.0;
    c->steps = 0;
    c->marked = 0;
    c->counter = 0;
    c->done = 0;
    c->last = 0;
    c->wmax = 0ull;
}

// Device address of the scratch array on the current device.  In host code
// the array's name is only a host-side stand-in, so the address comes from
// cudaGetSymbolAddress, once per device, with that device current.
cudaError_t scratch_address(void** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" cpr_status cpr_step_noalloc(const cpr_config* cfg, void* q_dev, int nsteps, double dt, void* stream)
{
    using cpr::LaunchCfg;
    if (!cfg || !q_dev) return CPR_EINVAL;
    if ((reinterpret_cast<uintptr_t>(q_dev) & 15u) != 0) return CPR_EINVAL;
    if (nsteps < 0 || !(dt > 0.0) || !std::isfinite(dt)) return CPR_EINVAL;
    if (cfg->eqn != CPR_ADVECTION && cfg->eqn != CPR_EULER) return CPR_EINVAL;
    if (cfg->nx < 1 || cfg->ny < 1 || cfg->nx > (1 << 20) || cfg->ny > (1 << 20) || cfg->p < 1 || cfg->p > 4 || !(cfg->x1 > cfg->x0) ||
        !(cfg->y1 > cfg->y0) || (cfg->pts != CPR_PTS_GAUSS && cfg->pts != CPR_PTS_LOBATTO) ||
        (cfg->corr != CPR_CORR_GDG && cfg->corr != CPR_CORR_NDG && cfg->corr != CPR_CORR_NDG_LUMPED) || (cfg->div != CPR_DIV_LP && cfg->div != CPR_DIV_CHAIN) ||
        (cfg->flux != CPR_FLUX_RUSANOV && !(cfg->flux == CPR_FLUX_UPWIND && cfg->eqn == CPR_ADVECTION)) ||
        (cfg->bc_x != CPR_BC_PERIODIC && cfg->bc_x != CPR_BC_TRANSMISSIVE) ||
        (cfg->bc_y != CPR_BC_PERIODIC && cfg->bc_y != CPR_BC_TRANSMISSIVE) ||
        (cfg->dtype != CPR_F64 && cfg->dtype != CPR_F32) || (cfg->eqn == CPR_EULER && !(cfg->gamma > 1.0)))
        return CPR_EINVAL;
    if (cfg->limiter) return CPR_EINVAL;
    const int V = cfg->eqn == CPR_EULER ? 4 : 1;
    const long long n = cfg->p + 1;
    const long long ne = (long long)cfg->nx * cfg->ny;
    const size_t esize = cfg->dtype == CPR_F32 ? 4 : 8;
    const size_t state_bytes = (size_t)(V * ne * n * n) * esize;
    if (state_bytes > kNoAllocStateBytes) return CPR_EINVAL;  // beyond the fixed scratch
    if (nsteps == 0) return CPR_OK;

    void* base = nullptr;
    cudaError_t e = scratch_address(&base);
    if (e != cudaSuccess) return CPR_ECUDA;
    unsigned char* b = static_cast<unsigned char*>(base);
    cpr::Ctrl* ctrl = reinterpret_cast<cpr::Ctrl*>(b);
    void* q1 = b + kNoAllocCtrlBytes;
    void* q2 = b + kNoAllocCtrlBytes + kNoAllocStateBytes;

    LaunchCfg lc{};
    lc.eqn = cfg->eqn;
    lc.p = cfg->p;
    lc.div = cfg->div;
    lc.flux = cfg->flux == CPR_FLUX_UPWIND ? cpr::FLUX_UPWIND : cpr::FLUX_RUSANOV;
    lc.nx = cfg->nx;
    lc.ny = cfg->ny;
    lc.bcx = cfg->bc_x == CPR_BC_TRANSMISSIVE;
    lc.bcy = cfg->bc_y == CPR_BC_TRANSMISSIVE;
    lc.ne = ne;
    lc.npts = ne * n * n;
    lc.hx = (cfg->x1 - cfg->x0) / cfg->nx;
    lc.hy = (cfg->y1 - cfg->y0) / cfg->ny;
    lc.gamma = cfg->gamma;
    lc.ax = cfg->ax;
    lc.ay = cfg->ay;
    lc.tvb_M = cfg->tvb_M;
    lc.lim_eps = cfg->lim_eps;
    lc.ctrl = ctrl;
    lc.l2_bytes = cpr::current_l2_bytes();
    lc.sms = cpr::current_sm_count();
    if (cpr::build_tables(cfg->p, cfg->pts, cfg->corr, &lc.tab) != 0) return CPR_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const bool f32 = cfg->dtype == CPR_F32;
    e = f32 ? cpr::prepare_stage<float>(lc) : cpr::prepare_stage<double>(lc);
    if (e == cudaSuccess) {
        noalloc_ctrl_init<<<1, 1, 0, s>>>(ctrl, dt);
        e = cudaGetLastError();
    }
    for (int k = 0; k < nsteps && e == cudaSuccess; ++k) {
        auto st = [&](int mode, const void* qs, const void* qn, void* out) {
            return f32 ? cpr::launch_stage<float>(lc, mode, qs, qn, out, nullptr, false, s)
                       : cpr::launch_stage<double>(lc, mode, qs, qn, out, nullptr, false, s);
        };
        e = st(1, q_dev, nullptr, q1);
        if (e == cudaSuccess) e = st(2, q1, q_dev, q2);
        if (e == cudaSuccess) e = st(3, q2, q_dev, q_dev);
    }
    return e == cudaSuccess ? CPR_OK : CPR_ECUDA;
}
