// cpr_reduce.cuh -- the CTA reduction of the maximum speed and the device-side
// time control.
//
// The CFL step of Sec. 4 (Eq. 36) needs the maximum signal speed of the whole
// state.  Every CTA of the kernel that produces the state folds its maximum
// into one word of the control block (an exact atomic maximum); the last CTA
// to finish (ticket from an atomic counter, no waiting) reads it and updates
// the control block: it advances the simulated time by the step just
// completed and sets the next step size, so the RK loop never synchronises
// with the host.
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

// Last-CTA reduction of the per-CTA maxima, called once per CTA (or once per
// tile, with a barrier between tiles) by all its threads, each with its own
// value m.  One barrier gathers the warps' maxima; thread 0 alone then folds
// the CTA's maximum into one word of the control block with an integer
// atomic maximum (non-negative doubles order as their bit patterns, so the
// result is the exact maximum in any order; a NaN is left out, as a
// comparison-based maximum leaves it out) and takes a ticket; the CTA that
// takes the last of nslots tickets reads and clears the word and closes the
// step.  The other threads are done after the barrier (a barrier after the
// ticket, to tell every thread which CTA was last, measured slower on the
// 64-instance batch).  advance: close the step (stage 3) or only set the
// next step size (start of a run).  with_max = false (a run of fixed steps,
// uniform over the grid): the ticket alone.
template <class T>
__device__ __forceinline__ void block_time_update(T m, Ctrl* ctrl, bool advance, int nslots, bool with_max = true)
{
    __shared__ T red[32];
    if (with_max) {
        m = warp_max(m);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        T r = T(0);
        for (int i = 0; with_max && i < nw; ++i) r = red[i] > r ? red[i] : r;
        const double md = (double)r;
        if (md > 0.0) atomicMax(&ctrl->wmax, (unsigned long long)__double_as_longlong(md));
        __threadfence();
        const unsigned int ticket = atomicAdd(&ctrl->counter, 1u);
        if (ticket == (unsigned int)nslots - 1) {
            __threadfence();
            const double w = __longlong_as_double((long long)atomicExch(&ctrl->wmax, 0ull));
            ctrl->counter = 0;
            if (advance) ctrl_advance(ctrl, w);
            else ctrl_next_dt(ctrl, w);
        }
    }
}

}  // namespace cpr
