// cpr_reduce.cuh -- block reductions and the device-side time control.
//
// The CFL step of Sec. 4 (Eq. 36) needs the maximum signal speed of the whole
// state.  Every CTA of the kernel that produces the state writes its partial
// maximum; the last CTA to finish (ticket from an atomic counter, no waiting)
// reduces the partials in a fixed order and updates the control block: it
// advances the simulated time by the step just completed and sets the next
// step size, so the RK loop never synchronises with the host.
#pragma once

#include "cpr_common.cuh"

namespace cpr {

template <class T>
__device__ __forceinline__ T warp_max(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        T w = __shfl_xor_sync(0xffffffffu, v, o);
        v = w > v ? w : v;
    }
    return v;
}

// Maximum over the CTA; every thread receives the result.
template <class T>
__device__ __forceinline__ T block_max(T v)
{
    __shared__ T red[32];
    v = warp_max(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    T r = red[0];
    for (int i = 1; i < nw; ++i) r = red[i] > r ? red[i] : r;
    return r;
}

// Next step size: the fixed step, or cfl * h / max_speed; shortened so that
// the step ends exactly at t_end; done once t_end is reached.
__device__ __forceinline__ void ctrl_next_dt(Ctrl* c, double max_speed)
{
    double dt = c->dt_fixed > 0.0 ? c->dt_fixed : c->cfl_h / max_speed;
    c->last = 0;
    if (c->t_end > 0.0) {
        if (c->t >= c->t_end) {
            c->done = 1;
            dt = 0.0;
        } else if (c->t + dt >= c->t_end) {
            dt = c->t_end - c->t;
            c->last = 1;
        }
    }
    c->dt = dt;
    c->max_wave = max_speed;
}

// Close the step in flight: t += dt (or t = t_end for the shortened last
// step), count it, and set the next step size.
__device__ __forceinline__ void ctrl_advance(Ctrl* c, double max_speed)
{
    c->t = c->last ? c->t_end : c->t + c->dt;
    c->steps += 1;
    c->parity ^= 1;
    ctrl_next_dt(c, max_speed);
}

// Last-CTA reduction of the per-CTA maxima (call with the CTA maximum in m,
// from all threads of the CTA).  Every CTA folds its maximum into one word
// of the control block with an integer atomic maximum (non-negative doubles
// order as their bit patterns, so the result is the exact maximum in any
// order; a NaN is left out, as a comparison-based maximum leaves it out);
// the CTA that arrives last reads and clears it and closes the step.
// advance: close the step (stage 3) or only set the next step size (start
// of a run).  nslots: the CTAs (or tiles) that report.
template <class T>
__device__ __forceinline__ void last_cta_time_update(T m, Ctrl* ctrl, bool advance, int nslots)
{
    __shared__ int s_last;
    if (threadIdx.x == 0) {
        const double md = (double)m;
        if (md > 0.0) atomicMax(&ctrl->wmax, (unsigned long long)__double_as_longlong(md));
        __threadfence();
        const unsigned int ticket = atomicAdd(&ctrl->counter, 1u);
        s_last = ticket == (unsigned int)nslots - 1;
    }
    __syncthreads();
    if (s_last && threadIdx.x == 0) {
        __threadfence();
        const double r = __longlong_as_double((long long)atomicExch(&ctrl->wmax, 0ull));
        ctrl->counter = 0;
        if (advance) ctrl_advance(ctrl, r);
        else ctrl_next_dt(ctrl, r);
    }
}

}  // namespace cpr
