// cpr_aux.cuh -- the passes around the stage kernel: element averages
// (Algorithm 9), the troubled-cell limiter (Sec. 2.6 Eq. 35, Algorithms
// 10-11), the initial max-speed pass of a CFL run (Eq. 36) and the FP64
// norms.
#pragma once

#include "cpr_common.cuh"
#include "cpr_reduce.cuh"

namespace cpr {

template <class T>
struct AuxArgs {
    T* q;             // state (limited in place by the limiter)
    const T* ref;     // norms: reference state (nullable)
    const T* avg_in;  // limiter: element averages of q
    T* avg_out;       // averages kernel output
    int* marks;       // limiter: marks[e]
    Ctrl* ctrl;
    double* partials; // norms: per-CTA FP64 partial results
    long long ne, npts;
    int nx, ny, bcx, bcy;
    unsigned int nx_magic;  // e / nx = div_invariant(e, nx, nx_magic, nx_shift) for e < 2^32
    int nx_shift;
    int do_wave;
    int check_done;   // limiter inside a step: do nothing once t_end is reached
    T hx, hy, tvb_M, lim_eps;
    Phys<T> ph;
    Tab<T> tab;
    Tab<double> tab64;  // FP64 weights for the norms
    double gamma64, ax64, ay64;
};

// Unsigned division by an invariant divisor d (Granlund & Montgomery,
// "Division by Invariant Integers using Multiplication", 1994): with
// l = ceil(log2 d) and m = floor(2^32 (2^l - d) / d) + 1, n / d is
// (t + ((n - t) >> 1)) >> (l - 1), t the high word of m n, for every 32-bit
// n; d = 1 is n itself.  div_magic runs on the host.
inline void div_magic(unsigned int d, unsigned int* m, int* l)
{
    int s = 0;
    while (s < 32 && (1ull << s) < d) ++s;
    *l = s;
    *m = (unsigned int)((((1ull << 32) * ((1ull << s) - d)) / d + 1) & 0xffffffffull);
}
__device__ __forceinline__ unsigned int div_invariant(unsigned int n, unsigned int d, unsigned int m, int l)
{
    if (d == 1u) return n;
    const unsigned int t = __umulhi(m, n);
    return (t + ((n - t) >> 1)) >> (l - 1);
}

// Element average with the same operation order as the stage kernel: row sums
// with the per-row weights, then the sum over rows.
template <int N, int V, class T>
__device__ __forceinline__ void element_average(const T* vals /* [V][N*N] */, const Tab<T>& tb, T* avg)
{
#pragma unroll
    for (int v = 0; v < V; ++v) {
        T s = T(0);
#pragma unroll
        for (int b = 0; b < N; ++b) {
            T r = tb.cavg[b][0] * vals[v * N * N + b * N];
#pragma unroll
            for (int a = 1; a < N; ++a) r = fma(tb.cavg[b][a], vals[v * N * N + b * N + a], r);
            s = b == 0 ? r : s + r;
        }
        avg[v] = s;
    }
}

// Elements per CTA of the element-wise passes: 64, or 32 where the staged
// elements would not fit the 48 KB of static shared memory.
template <class T, int P, int EQ>
struct AuxShape {
    static constexpr int N = P + 1, NN = N * N, V = NVars<EQ>::value;
    static constexpr int EB = (V * kAuxElems * (NN + 1) * (int)sizeof(T) <= 48 * 1024) ? kAuxElems : kAuxElems / 2;
};

// Coalesced copy of EB consecutive elements into shared memory,
// sm[(v * EB + le) * (NN + 1) + pt] (one pad word against bank conflicts
// when each thread walks its own element).
template <int N, int V, int EB, class T>
__device__ __forceinline__ void load_elements(const T* __restrict__ q, long long npts, long long e0, int cnt,
                                              T* sm)
{
    constexpr int NN = N * N;
    for (int v = 0; v < V; ++v) {
        const T* src = q + v * npts + e0 * NN;
        for (int idx = threadIdx.x; idx < cnt * NN; idx += blockDim.x)
            sm[(v * EB + idx / NN) * (NN + 1) + idx % NN] = src[idx];
    }
}

template <class T, int P, int EQ>
__global__ void __launch_bounds__(AuxShape<T, P, EQ>::EB) cpr_averages_kernel(const AuxArgs<T> A)
{
    constexpr int N = P + 1, NN = N * N, V = NVars<EQ>::value, EB = AuxShape<T, P, EQ>::EB;
    __shared__ T sm[V * EB * (NN + 1)];
    const long long e0 = (long long)blockIdx.x * EB;
    const int cnt = (int)min((long long)EB, A.ne - e0);
    load_elements<N, V, EB>(A.q, A.npts, e0, cnt, sm);
    __syncthreads();
    const int le = threadIdx.x;
    if (le < cnt) {
        T vals[V * NN], avg[V];
#pragma unroll
        for (int v = 0; v < V; ++v)
#pragma unroll
            for (int pt = 0; pt < NN; ++pt) vals[v * NN + pt] = sm[(v * EB + le) * (NN + 1) + pt];
        element_average<N, V>(vals, A.tab, avg);
#pragma unroll
        for (int v = 0; v < V; ++v) A.avg_out[v * A.ne + e0 + le] = avg[v];
    }
}

// Staging of EB consecutive elements by all NT threads of the CTA:
// sm[(v * EB + le) * ES + pt] with the element stride ES = NN rounded up to
// an odd number (a thread walking its own element meets no bank conflict).
// For odd NN the block is a plain copy; a full block issues all of a
// thread's loads before its first shared-memory store.
template <int N>
struct LimStride {
    static constexpr int NN = N * N, ES = NN | 1;
};

template <int N, int V, int EB, int NT, class T>
__device__ __forceinline__ void load_elements_all(const T* __restrict__ q, long long npts, long long e0, int cnt,
                                                  T* sm)
{
    constexpr int NN = N * N, ES = LimStride<N>::ES, PER = EB * NN, K = (PER + NT - 1) / NT;
    if (cnt == EB) {
        T r[V][K];
#pragma unroll
        for (int v = 0; v < V; ++v)
#pragma unroll
            for (int k = 0; k < K; ++k) {
                const int w = (int)threadIdx.x + k * NT;
                if (PER % NT == 0 || w < PER) r[v][k] = q[v * npts + e0 * NN + w];
            }
#pragma unroll
        for (int v = 0; v < V; ++v)
#pragma unroll
            for (int k = 0; k < K; ++k) {
                const int w = (int)threadIdx.x + k * NT;
                if (PER % NT == 0 || w < PER) sm[v * EB * ES + (ES == NN ? w : (w / NN) * ES + w % NN)] = r[v][k];
            }
    } else {
        for (int v = 0; v < V; ++v) {
            const T* src = q + v * npts + e0 * NN;
            for (int w = threadIdx.x; w < cnt * NN; w += NT) sm[v * EB * ES + (w / NN) * ES + w % NN] = src[w];
        }
    }
}

// Bounds of the marking test along one direction.  With A = M h^2, c the
// minmod of the two neighbour-average differences across the edge (zero
// unless they share a sign) and the outward edge deviation d, a point is
// troubled when |d| > A and |d - minmod(d, D+, D-)| > eps, where the
// three-argument minmod is min(d, c) for d, c > 0, max(d, c) for d, c < 0,
// else 0 (the TVB minmod keeps d itself when |d| <= A, where the point is
// not troubled either way).  On each side of zero that test is monotone in
// d, so it is the same as d > hi or d < lo with
//   c > 0:  hi = max(A, c + eps),  lo = -max(A, eps)
//   c < 0:  hi = max(A, eps),      lo = min(-A, c - eps)
//   c = 0:  hi = max(A, eps),      lo = -max(A, eps)
// and an edge is troubled exactly when its largest deviation exceeds hi or
// its smallest is below lo: two comparisons per edge instead of a minmod
// test per edge point.
template <class T>
__device__ __forceinline__ void tvb_bounds(T c, T mh2, T eps, T& lo, T& hi)
{
    const T a = ::fmax(mh2, eps);
    hi = c > T(0) ? ::fmax(mh2, c + eps) : a;
    lo = c < T(0) ? ::fmin(-mh2, c - eps) : -a;
}

// Troubled-cell limiter.  One thread per (element, variable), variable-major
// in the CTA (thread v * EB + le), so that the loads of the neighbour
// averages are coalesced and each thread holds one variable's N^2 values.
// Marking (Algorithm 10): for every variable and every edge point, the
// outward edge deviation delta = s (q_edge - qbar) (s = +1 on right/top edges,
// -1 on left/bottom) is compared with the TVB minmod of delta and the
// differences of the neighbouring averages across that edge; the element is
// marked when |delta - mt| > eps anywhere (the OR over edge points and
// variables of Algorithm 11, taken in shared memory), tested through the
// extreme deviations of each edge against the bounds of tvb_bounds.  Limiting (Eq. 35, per
// direction): q_ab = qbar + (xi_a hx / 2) mm(Dx+ / hx, Dx- / hx)
// + (eta_b hy / 2) mm(Dy+ / hy, Dy- / hy).  A transmissive boundary
// contributes a ghost average equal to the element's own average.  The fused
// max signal speed splits an element's points over its V threads.
template <class T, int P, int EQ>
struct LimShape {
    static constexpr int V = NVars<EQ>::value, EB = AuxShape<T, P, EQ>::EB, NT = V * EB;
};

template <class T, int P, int EQ>
__global__ void __launch_bounds__(LimShape<T, P, EQ>::NT) cpr_limit_kernel(const AuxArgs<T> A)
{
    constexpr int N = P + 1, NN = N * N, V = NVars<EQ>::value, EB = AuxShape<T, P, EQ>::EB;
    constexpr int NT = LimShape<T, P, EQ>::NT;
    constexpr int ES = LimStride<N>::ES;
    __shared__ T sm[V * EB * ES];
    __shared__ int s_mark[EB];
    static_assert(EB % 32 == 0, "one variable per warp");
    if (A.check_done && A.ctrl->done) return;  // uniform exit
    const long long e0 = (long long)blockIdx.x * EB;
    const int cnt = (int)min((long long)EB, A.ne - e0);
    const int v = (int)threadIdx.x / EB, le = (int)threadIdx.x - v * EB;
    const Tab<T>& tb = A.tab;
    // own and neighbour averages first: their loads overlap the staging of
    // the element values below
    const long long e = e0 + min(le, max(cnt - 1, 0));
    // element (i, j): a multiplication by the divisor's magic number while
    // the element index fits 32 bits (a division by a runtime value costs
    // tens of instructions, a 64-bit one over a hundred)
    int i, j;
    if (A.ne <= 0xffffffffll) {
        const unsigned int eu = (unsigned int)e;
        j = (int)div_invariant(eu, (unsigned int)A.nx, A.nx_magic, A.nx_shift);
        i = (int)(eu - (unsigned int)j * (unsigned int)A.nx);
    } else {
        j = (int)(e / A.nx);
        i = (int)(e - (long long)j * A.nx);
    }
    const long long eL = i > 0 ? e - 1 : (A.bcx ? -1 : e + A.nx - 1);
    const long long eR = i < A.nx - 1 ? e + 1 : (A.bcx ? -1 : e - (A.nx - 1));
    const long long eB = j > 0 ? e - A.nx : (A.bcy ? -1 : e + (long long)A.nx * (A.ny - 1));
    const long long eT = j < A.ny - 1 ? e + A.nx : (A.bcy ? -1 : e - (long long)A.nx * (A.ny - 1));
    const T* av = A.avg_in + v * A.ne;
    const T qk = av[e];
    const T aL = eL >= 0 ? av[eL] : qk, aR = eR >= 0 ? av[eR] : qk;
    const T aB = eB >= 0 ? av[eB] : qk, aT = eT >= 0 ? av[eT] : qk;
    load_elements_all<N, V, EB, NT>(A.q, A.npts, e0, cnt, sm);
    if (threadIdx.x < EB) s_mark[threadIdx.x] = 0;
    __syncthreads();
    T* mine = &sm[(v * EB + le) * ES];
    if (le < cnt) {
        T vals[NN];
#pragma unroll
        for (int pt = 0; pt < NN; ++pt) vals[pt] = mine[pt];
        // minmod of the neighbour differences per direction (zero unless
        // both share a sign), M h^2 per direction, and the bounds of the
        // outward deviation (tvb_bounds)
        const T cx = minmod2(aR - qk, qk - aL), cy = minmod2(aT - qk, qk - aB);
        T lox, hix, loy, hiy;
        tvb_bounds(cx, A.tvb_M * A.hx * A.hx, A.lim_eps, lox, hix);
        tvb_bounds(cy, A.tvb_M * A.hy * A.hy, A.lim_eps, loy, hiy);
        // extreme edge values per edge: the outward deviation is q_edge - qbar
        // on the right / top edges and qbar - q_edge on the left / bottom ones
        T mnL = T(0), mxL = T(0), mnR = T(0), mxR = T(0), mnB = T(0), mxB = T(0), mnT = T(0), mxT = T(0);
#pragma unroll
        for (int kk = 0; kk < N; ++kk) {
            T row[N], col[N];
#pragma unroll
            for (int l = 0; l < N; ++l) {
                row[l] = vals[kk * N + l];
                col[l] = vals[l * N + kk];
            }
            T sL = tb.lm[0] * row[0], sR = tb.lp[0] * row[0];
            T sB = tb.lm[0] * col[0], sT = tb.lp[0] * col[0];
#pragma unroll
            for (int l = 1; l < N; ++l) {
                sL = fma(tb.lm[l], row[l], sL);
                sR = fma(tb.lp[l], row[l], sR);
                sB = fma(tb.lm[l], col[l], sB);
                sT = fma(tb.lp[l], col[l], sT);
            }
            mnL = kk ? ::fmin(mnL, sL) : sL;
            mxL = kk ? ::fmax(mxL, sL) : sL;
            mnR = kk ? ::fmin(mnR, sR) : sR;
            mxR = kk ? ::fmax(mxR, sR) : sR;
            mnB = kk ? ::fmin(mnB, sB) : sB;
            mxB = kk ? ::fmax(mxB, sB) : sB;
            mnT = kk ? ::fmin(mnT, sT) : sT;
            mxT = kk ? ::fmax(mxT, sT) : sT;
        }
        const bool troubled = (qk - mnL > hix) | (qk - mxL < lox) | (mxR - qk > hix) | (mnR - qk < lox) |
                              (qk - mnB > hiy) | (qk - mxB < loy) | (mxT - qk > hiy) | (mnT - qk < loy);
        if (troubled) s_mark[le] = 1;  // every writer stores 1
    }
    __syncthreads();
    const int marked = le < cnt ? s_mark[le] : 0;
    if (marked) {
        // mm(D+ / h, D- / h) = mm(D+, D-) / h bit for bit (division by a
        // positive h keeps the order and signs of the rounded quotients)
        const T sx = minmod2(aR - qk, qk - aL) / A.hx;
        const T sy = minmod2(aT - qk, qk - aB) / A.hy;
        T* dst = A.q + v * A.npts + e * NN;
#pragma unroll
        for (int b = 0; b < N; ++b)
#pragma unroll
            for (int a = 0; a < N; ++a) {
                const T x = (T(0.5) * A.hx * tb.xi[a]) * sx;
                const T y = (T(0.5) * A.hy * tb.xi[b]) * sy;
                const T val = (qk + x) + y;
                mine[b * N + a] = val;
                dst[b * N + a] = val;
            }
    }
    if (v == 0) {
        // the marks, and their count per warp (a ballot; EB is a multiple of
        // 32, so v is uniform over a warp) added to the run's integer count
        if (le < cnt) A.marks[e] = marked;
        const unsigned int bal = __ballot_sync(0xffffffffu, le < cnt && marked);
        if ((threadIdx.x & 31) == 0 && bal)
            atomicAdd(reinterpret_cast<unsigned long long*>(&A.ctrl->marked), (unsigned long long)__popc(bal));
    }
    if (A.do_wave) {
        __syncthreads();  // the limited values of the element's other variables
        T m = T(0);
        if (le < cnt) {
#pragma unroll
            for (int k = 0; k < (NN + V - 1) / V; ++k) {
                const int pt = v + k * V;
                if (pt < NN) {
                    T qp[V];
#pragma unroll
                    for (int w = 0; w < V; ++w) qp[w] = sm[(w * EB + le) * ES + pt];
                    const T s = point_speed<EQ>(qp, A.ph);
                    m = s > m ? s : m;
                }
            }
        }
        block_time_update<T>(m, A.ctrl, /*advance=*/true, gridDim.x);
    }
}

// Max signal speed of a state and the first step size of a CFL run.
template <class T, int P, int EQ>
__global__ void __launch_bounds__(256) cpr_wave_kernel(const AuxArgs<T> A)
{
    constexpr int V = NVars<EQ>::value;
    T m = T(0);
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < A.npts;
         k += (long long)gridDim.x * blockDim.x) {
        T qp[V];
#pragma unroll
        for (int v = 0; v < V; ++v) qp[v] = A.q[v * A.npts + k];
        const T s = point_speed<EQ>(qp, A.ph);
        m = s > m ? s : m;
    }
    block_time_update<T>(m, A.ctrl, /*advance=*/false, gridDim.x);
}

// FP64 norms, pass 1: each CTA reduces a contiguous element range in a fixed
// order and writes 8 partial values:
//   [0..3] sum of element averages per variable, [4] sum (q - ref)^2,
//   [5] sum ref^2, [6] max speed, [7] count of non-physical points.
// The element average uses the FP64 weights w_a w_b / 4 in point order.
constexpr int kNormThreads = 256;
constexpr int kNormVals = 8;

template <class T, int P, int EQ>
__global__ void __launch_bounds__(kNormThreads) cpr_norms_kernel(const AuxArgs<T> A)
{
    constexpr int N = P + 1, NN = N * N, V = NVars<EQ>::value;
    const long long chunk = (A.ne + gridDim.x - 1) / gridDim.x;
    const long long eb = (long long)blockIdx.x * chunk;
    const long long ee = min(A.ne, eb + chunk);
    double acc[kNormVals] = {0, 0, 0, 0, 0, 0, 0, 0};
    Phys<double> ph64;
    ph64.gamma = A.gamma64;
    ph64.ax = A.ax64;
    ph64.ay = A.ay64;
    for (long long e = eb + threadIdx.x; e < ee; e += blockDim.x) {
        for (int v = 0; v < V; ++v) {
            double s = 0.0;
            for (int b = 0; b < N; ++b)
                for (int a = 0; a < N; ++a)
                    s = __dadd_rn(s, __dmul_rn(__dmul_rn(__dmul_rn(A.tab64.w[a], A.tab64.w[b]), 0.25),
                                               (double)A.q[v * A.npts + e * NN + b * N + a]));
            acc[v] += s;
        }
        for (int pt = 0; pt < NN; ++pt) {
            double qp[4] = {0, 0, 0, 0};
            for (int v = 0; v < V; ++v) {
                const double x = (double)A.q[v * A.npts + e * NN + pt];
                qp[v] = x;
                if (A.ref) {
                    const double r = (double)A.ref[v * A.npts + e * NN + pt];
                    acc[4] += (x - r) * (x - r);
                    acc[5] += r * r;
                }
            }
            if (point_ok<EQ>(qp, ph64)) {
                const double s = point_speed<EQ>(qp, ph64);
                acc[6] = s > acc[6] ? s : acc[6];
            } else {
                acc[7] += 1.0;
            }
        }
    }
    __shared__ double red[kNormThreads][kNormVals];
    for (int k = 0; k < kNormVals; ++k) red[threadIdx.x][k] = acc[k];
    __syncthreads();
    for (int s = kNormThreads / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s)
            for (int k = 0; k < kNormVals; ++k) {
                if (k == 6) red[threadIdx.x][k] = fmax(red[threadIdx.x][k], red[threadIdx.x + s][k]);
                else red[threadIdx.x][k] += red[threadIdx.x + s][k];
            }
        __syncthreads();
    }
    if (threadIdx.x < kNormVals) A.partials[(long long)blockIdx.x * kNormVals + threadIdx.x] = red[0][threadIdx.x];
}

}  // namespace cpr
