// cpr_launch.h -- host-side interface between the C ABI and the per-dtype,
// per-order kernel translation units.
#pragma once

#include <cuda_runtime.h>

#include "cpr_common.cuh"

namespace cpr {

// FP64 operator tables built on the host (see cpr_tables.cpp).
struct HostTab {
    int n;
    double xi[kMaxN], w[kMaxN];
    double D[kMaxN][kMaxN];  // D[a][l] = l_l'(xi_a)
    double lm[kMaxN], lp[kMaxN];
    double dgl[kMaxN], dgr[kMaxN];
};

// Fill *t for order p, point family pts (0 Gauss-Legendre, 1
// Gauss-Lobatto) and edge correction corr (0 Radau g_DG, 1 nodal-DG lift
// with the exact mass matrix, 2 with the lumped one).  Returns 0 on success.
int build_tables(int p, int pts, int corr, HostTab* t);

// Everything a launch needs, independent of the state dtype.
struct LaunchCfg {
    int eqn, p, div, flux;  // flux: FLUX_RUSANOV, FLUX_UPWIND or FLUX_ROE
    int fv_order;           // FV schemes (p = 0): MUSCL order, 2 or 3
    long long l2_bytes;     // L2 size of the device (0: unknown)
    int sms;                // SMs of the device: a stage launch of at most two CTAs per SM takes
                            // the instantiation compiled for two resident CTAs (0: never)
    int nx, ny, bcx, bcy;
    long long ne, npts;
    double hx, hy, gamma, ax, ay, tvb_M, lim_eps;
    HostTab tab;
    Ctrl* ctrl;
    int* marks;        // limiter marks
    double* partials;  // norms partials
};

// SM count of the current device (0 when it cannot be queried).
inline int current_sm_count()
{
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess)
        return n;
    (void)cudaGetLastError();
    return 0;
}

// L2 size of the current device in bytes (0 when it cannot be queried).
inline long long current_l2_bytes()
{
    int dev = 0, l2 = 0;
    if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev) == cudaSuccess)
        return l2;
    (void)cudaGetLastError();
    return 0;
}

// Element tile of one stage-kernel CTA per order (compile-time; overridable
// for tuning sweeps with -DCPR_TILE_X=.., -DCPR_TILE_Y=.., -DCPR_TILE_X_P4=..,
// -DCPR_TILE_Y_P4=..):
// 8 x 8 elements, and 8 x 4 for p = 4, whose 160-thread CTAs keep the
// threads per SM of 320-thread ones (the register budget scales with the
// tile) while twice as many CTAs per SM hide each other's barriers (820^2
// p = 4: 328 -> 306 us per stage launch; 8 x 4 tiles for p = 2 and 3 were
// slower, 308 -> 339 and 216 -> 230 us).
#ifndef CPR_TILE_X
#define CPR_TILE_X 8
#endif
#ifndef CPR_TILE_Y
#define CPR_TILE_Y 8
#endif
#ifndef CPR_TILE_X_P4
#define CPR_TILE_X_P4 CPR_TILE_X
#endif
#ifndef CPR_TILE_Y_P4
#define CPR_TILE_Y_P4 4
#endif
constexpr int stage_tile_x(int p) { return p == 4 ? CPR_TILE_X_P4 : CPR_TILE_X; }
constexpr int stage_tile_y(int p) { return p == 4 ? CPR_TILE_Y_P4 : CPR_TILE_Y; }

inline int stage_ctas(const LaunchCfg& c)
{
    const int tx = stage_tile_x(c.p), ty = stage_tile_y(c.p);
    return ((c.nx + tx - 1) / tx) * ((c.ny + ty - 1) / ty);
}

// Buffers of one stage launch (see the modes of cpr_stage.cuh): qs the stage
// input (hi of q^n in the increment modes), qb the increment added to it
// (modes 5, 6), qn q^n (modes 2, 3), out the result, lo the low part of q^n
// (mode 6, in place), avg the fused element averages of out (nullable).
struct StagePtrs {
    const void* qs;
    const void* qb;
    const void* qn;
    void* out;
    void* lo;
    void* avg;
};

// Stage kernel for one (dtype, order).  do_wave closes the step on the
// device (stage 3).
template <class T, int P>
cudaError_t launch_stage_p(const LaunchCfg& c, int mode, const StagePtrs& b, bool do_wave, cudaStream_t s);
template <class T, int P>
cudaError_t prepare_stage_p(const LaunchCfg& c);

// FV stage kernel (p = 0; cpr_fv.cuh), same modes and buffers as the CPR one.
template <class T>
cudaError_t launch_fv(const LaunchCfg& c, int mode, const StagePtrs& b, bool do_wave, cudaStream_t s);

template <class T>
cudaError_t launch_stage(const LaunchCfg& c, int mode, const StagePtrs& b, bool do_wave, cudaStream_t s);
// Shu-Osher / residual form: modes 0..3.
template <class T>
cudaError_t launch_stage(const LaunchCfg& c, int mode, const void* qs, const void* qn, void* out, void* avg,
                         bool do_wave, cudaStream_t s);
template <class T>
cudaError_t prepare_stage(const LaunchCfg& c);
template <class T>
cudaError_t launch_averages(const LaunchCfg& c, const void* q, void* avg, cudaStream_t s);
// role 0: stand-alone pass; 1: after stage 1 or 2 of a step (does nothing
// once t_end is reached); 2: after stage 3 (also closes the step: the last
// CTA advances the simulated time and sets the next step size).
template <class T>
cudaError_t launch_limit(const LaunchCfg& c, void* q, const void* avg, int role, cudaStream_t s);
template <class T>
cudaError_t launch_wave(const LaunchCfg& c, const void* q, cudaStream_t s);
template <class T>
cudaError_t launch_norms(const LaunchCfg& c, const void* q, const void* ref, int nblocks, cudaStream_t s);

// ---- discrete adjoint (cpr_adjoint.cuh) -----------------------------------
// out = c0 X0 + c1 X1 + c2 X2 + cv (dR/dq)^T(q) rbar; the X are nullable.
struct VjpPtrs {
    const void* q;
    const void* rbar;
    void* out;
    const void* X0;
    const void* X1;
    const void* X2;
    double c0, c1, c2, cv;
};
template <class T, int P>
cudaError_t launch_vjp_p(const LaunchCfg& c, const VjpPtrs& b, cudaStream_t s, bool prepare);
template <class T>
cudaError_t launch_vjp(const LaunchCfg& c, const VjpPtrs& b, cudaStream_t s, bool prepare);

// ---- batched launches (cpr_batch.cuh) ------------------------------------
template <class T>
struct BatchArgs;

// Elements per tile of tile family fam of the batched kernels.
inline void batch_tile(int fam, int* tx, int* ty)
{
    *tx = fam == 0 ? 8 : 16;
    *ty = fam == 0 ? 8 : 4;
}
constexpr int kBatchFamilies = 2;

// One launch of the batched stage kernel of order p.  what 0: launch;
// 1: set the kernel's shared-memory limit; 2: *occ = resident CTAs per SM.
template <class T, int FAM>
cudaError_t batch_fam(int p, int eqn, int flux, const BatchArgs<T>& B, int grid, cudaStream_t s, int what,
                      int* occ);

}  // namespace cpr
