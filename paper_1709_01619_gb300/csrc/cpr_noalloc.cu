// cpr_noalloc.cu -- cpr_step_noalloc: fixed-step SSP-RK3 steps without any
// device allocation.
//
// Some callers cannot let a library allocate device memory: a host framework
// that owns the whole device through its own pool allocator (a cudaMalloc
// behind its back can fail or break its accounting), or a latency-critical
// loop where cudaMalloc/cudaFree, which may synchronise the device, are not
// allowed.  For them this entry point runs the same stage kernels as
// cpr_step, with the stage buffers, the low part of the FP32 state and the
// small control block in one file-scope device array instead of
// context-owned allocations.
//
// The array is kNoAllocCtrlBytes + 3 * kNoAllocStateBytes bytes; every GPU
// that loads libcpr.so holds it until the process exits.  All calls share
// it and it keeps the previous call's contents, so the control block is
// rewritten and the low part cleared at the start of every call, and calls
// that overlap on the GPU (different streams, or threads without ordering
// between them) race on it.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "../../include/cpr.h"
#include "cpr_internal.h"
#include "cpr_launch.h"

namespace {

constexpr size_t kNoAllocCtrlBytes = 256;
constexpr size_t kNoAllocStateBytes = CPR_NOALLOC_MAX_STATE_BYTES;
// control block | stage buffer 1 | stage buffer 2 | low part (FP32)
constexpr size_t kNoAllocBytes = kNoAllocCtrlBytes + 3 * kNoAllocStateBytes;
static_assert(sizeof(cpr::Ctrl) <= kNoAllocCtrlBytes, "the control block must fit its slot");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

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
    c->parity = 0;
    c->wmax = 0ull;
}

// Device address of the scratch array on the current device.  In host code
// the array's name is only a host-side stand-in, so the address comes from
// cudaGetSymbolAddress with the device current.  It is looked up on every
// call (a cheap query once the module is loaded), so a reset of the device
// between calls leaves no stale address behind.
cudaError_t scratch_address(void** out)
{
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    *out = p;
    return cudaSuccess;
}

}  // namespace

extern "C" cpr_status cpr_step_noalloc(const cpr_config* cfg, void* q_dev, int nsteps, double dt, void* stream)
{
    using cpr::LaunchCfg;
    using cpr::StagePtrs;
    // the configuration rules of cpr_init, then this entry point's own
    if (!cfg || !q_dev || cpr_validate_config(cfg)) return CPR_EINVAL;
    if (cfg->limiter || cfg->scheme != CPR_SCHEME_CPR) return CPR_EINVAL;
    if ((reinterpret_cast<uintptr_t>(q_dev) & 15u) != 0) return CPR_EINVAL;
    if (nsteps < 0 || !(dt > 0.0) || !std::isfinite(dt)) return CPR_EINVAL;
    const int V = cfg->eqn == CPR_EULER ? 4 : 1;
    const long long n = cfg->p + 1;
    const long long ne = (long long)cfg->nx * cfg->ny;
    const bool f32 = cfg->dtype == CPR_F32;
    const size_t state_bytes = (size_t)(V * ne * n * n) * (f32 ? 4 : 8);
    if (state_bytes > kNoAllocStateBytes) return CPR_EINVAL;  // beyond the fixed scratch
    if (nsteps == 0) return CPR_OK;

    LaunchCfg lc{};
    if (!cpr_fill_launch_cfg(cfg, &lc)) return CPR_EINVAL;
    void* base = nullptr;
    cudaError_t e = scratch_address(&base);
    if (e != cudaSuccess) return CPR_ECUDA;
    unsigned char* b = static_cast<unsigned char*>(base);
    cpr::Ctrl* ctrl = reinterpret_cast<cpr::Ctrl*>(b);
    void* q1 = b + kNoAllocCtrlBytes;
    void* q2 = b + kNoAllocCtrlBytes + kNoAllocStateBytes;
    void* lo = b + kNoAllocCtrlBytes + 2 * kNoAllocStateBytes;
    lc.ctrl = ctrl;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    e = f32 ? cpr::prepare_stage<float>(lc) : cpr::prepare_stage<double>(lc);
    if (e == cudaSuccess) {
        noalloc_ctrl_init<<<1, 1, 0, s>>>(ctrl, dt);
        e = cudaGetLastError();
    }
    if (f32) {
        // The compensated increment form of cpr_step (FP32):
        //   B1 = dt R(q); B2 = (B1 + dt R(q + B1)) / 4; q' = q + 2/3 (B2 + dt R(q + B2)),
        // with q' kept as a high part and a low part (the low part starts
        // at zero).  The high part alternates between q_dev and stage
        // buffer 1, so after an odd step count it is copied back.
        if (e == cudaSuccess) e = cudaMemsetAsync(lo, 0, state_bytes, s);
        void* x = q_dev;
        void* y = q1;
        for (int k = 0; k < nsteps && e == cudaSuccess; ++k) {
            e = cpr::launch_stage<float>(lc, cpr::MODE_INC1, StagePtrs{x, nullptr, nullptr, y, lo, nullptr}, false, s);
            if (e == cudaSuccess)
                e = cpr::launch_stage<float>(lc, cpr::MODE_INC2, StagePtrs{x, y, nullptr, q2, lo, nullptr}, false, s);
            if (e == cudaSuccess)
                e = cpr::launch_stage<float>(lc, cpr::MODE_INC3, StagePtrs{x, q2, nullptr, y, lo, nullptr}, false, s);
            void* t = x;
            x = y;
            y = t;
        }
        if (e == cudaSuccess && x != q_dev) e = cudaMemcpyAsync(q_dev, x, state_bytes, cudaMemcpyDeviceToDevice, s);
    } else {
        // FP64: the Shu-Osher stages of cpr_step
        for (int k = 0; k < nsteps && e == cudaSuccess; ++k) {
            e = cpr::launch_stage<double>(lc, cpr::MODE_SO1, q_dev, nullptr, q1, nullptr, false, s);
            if (e == cudaSuccess) e = cpr::launch_stage<double>(lc, cpr::MODE_SO2, q1, q_dev, q2, nullptr, false, s);
            if (e == cudaSuccess) e = cpr::launch_stage<double>(lc, cpr::MODE_SO3, q2, q_dev, q_dev, nullptr, false, s);
        }
    }
    return e == cudaSuccess ? CPR_OK : CPR_ECUDA;
}
