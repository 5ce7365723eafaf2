// cpr_adjoint.cuh -- transpose of the CPR residual (discrete adjoint).
//
// qbar = (dR/dq)^T rbar for the LP divergence (Sec. 2.2, Eq. 16-17 with the
// flux interpolant differentiated), written as a gather: every element
// collects the contributions to its own points, so no two CTAs write the
// same value and no atomics are needed.
//
// With xb = -(2/hx) rbar along a row (and yb = -(2/hy) rbar along a column):
//   volume and edge-flux terms:  fbar_l = sum_a xb_a M_al,
//       M_al = D_al - l_l(-1) g_L'(xi_a) - l_l(+1) g_R'(xi_a),
//       qbar_l += A_x(q_l)^T fbar_l                       (A_x = df/dq)
//   common flux on a face: its cotangent is the sum of the two sides'
//       W = sum_a xb_a g_L'(xi_a) (element above / right of the face)
//         + sum_a xb_a g_R'(xi_a) (element below / left),
//       and the transpose of the Rusanov flux maps W to the cotangents of
//       the two edge states, which the edge interpolation spreads back to
//       the points (qbar_l += l_l(+-1) qbar_edge).
// Each element applies the face transpose of its four faces to its own side
// only: a face shared by two CTAs is transposed by both, from the same bits.
//
// Epilogue: out = c0 X0 + c1 X1 + c2 X2 + cv qbar (the X optional), so that
// the transpose of one SSP-RK3 step is three launches.
#pragma once

#include "cpr_common.cuh"
#include "cpr_stage.cuh"

namespace cpr {

template <class T>
struct VjpArgs {
    const T* q;
    const T* rbar;
    T* out;
    const T* X0;
    const T* X1;
    const T* X2;
    T c0, c1, c2, cv;
    long long npts;
    int nx, ny, bcx, bcy, tiles_x;
    T rhx2, rhy2;
    Phys<T> ph;
    Tab<T> tab;
    T M[kMaxN][kMaxN];
};

template <int N, int V, int TX, int TY>
struct VjpLayout {
    static constexpr int NN = N * N;
    static constexpr int ES = (NN % 4 == 0) ? NN + 4 : ((NN + 3) / 4) * 4;
    static constexpr int E = TX * TY;
    static constexpr int SQ = V * E * ES;
    static constexpr int XR = V * TY * (TX + 1) * N;  // right-edge values, elements -1..TX-1
    static constexpr int XH = V * TY * N;             // left-edge values of the right halo
    static constexpr int XQ = V * TY * TX * N;        // face results for the left element
    static constexpr int YT = V * (TY + 1) * TX * N;
    static constexpr int YH = V * TX * N;
    static constexpr int YQ = V * TY * TX * N;
    // q and rbar (the column accumulator later reuses the tile of q); edge
    // states and edge cotangents of both directions; face results
    static constexpr int TOTAL = 2 * SQ + 2 * (XR + XH + YT + YH) + XQ + YQ;
    __device__ static int sq(int v, int el, int pt) { return (v * E + el) * ES + pt; }
    __device__ static int xr(int v, int ty, int f, int k) { return ((v * TY + ty) * (TX + 1) + f) * N + k; }
    __device__ static int xh(int v, int ty, int k) { return (v * TY + ty) * N + k; }
    __device__ static int xq(int v, int ty, int tx, int k) { return ((v * TY + ty) * TX + tx) * N + k; }
    __device__ static int yt(int v, int g, int tx, int k) { return ((v * (TY + 1) + g) * TX + tx) * N + k; }
    __device__ static int yh(int v, int tx, int k) { return (v * TX + tx) * N + k; }
    __device__ static int yq(int v, int ty, int tx, int k) { return ((v * TY + ty) * TX + tx) * N + k; }
};

// Resident CTAs per SM the register budget is sized for (0: no bound): in
// FP32, for tiles of 32 elements, as many as the shared memory holds
// (p = 2: 8, p = 3: 6 with 16 bytes of spills, p = 4: 4; unbounded, the
// registers allowed 7, 5 and 3; 1024^2 p = 3: 0.364 -> 0.351 ms per
// launch), scaled for other tile sizes; FP64 unbounded.
template <class T, int P, int ELEMS>
constexpr int vjp_min_blocks()
{
    return sizeof(T) == 8 ? 0 : (P == 2 ? 8 : (P == 3 ? 6 : (P == 4 ? 4 : 0))) * 32 / ELEMS;
}

template <class T, int P, int EQ, int FLUX, int TX, int TY>
__global__ void __launch_bounds__(TX * TY * (P + 1), (vjp_min_blocks<T, P, TX * TY>()))
cpr_residual_vjp_kernel(const VjpArgs<T> A)
{
    constexpr int N = P + 1, NN = N * N, V = NVars<EQ>::value;
    constexpr int NT = TX * TY * N;
    using L = VjpLayout<N, V, TX, TY>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sq = reinterpret_cast<T*>(smem_raw);
    T* sr = sq + L::SQ;
    // column contributions to qbar, over the tile of q: thread (el, k) writes
    // only the column k of element el that it has read itself, after the
    // barrier that ends every thread's row reads
    T* qb = sq;
    T* xRq = sr + L::SQ;         // right edge states
    T* xRw = xRq + L::XR;        // right-edge flux cotangents  sum xb g_R'
    T* xHq = xRw + L::XR;        // left edge state of the right halo
    T* xHw = xHq + L::XH;        // its left-edge cotangent     sum xb g_L'
    T* yTq = xHw + L::XH;
    T* yTw = yTq + L::YT;
    T* yHq = yTw + L::YT;
    T* yHw = yHq + L::YH;
    T* xQ = yHw + L::YH;         // lower-state cotangent of a face, for the left element
    T* yQ = xQ + L::XQ;

    const int tid = threadIdx.x;
    const int i0 = (blockIdx.x % A.tiles_x) * TX;
    const int j0 = (blockIdx.x / A.tiles_x) * TY;
    const int TXe = min(TX, A.nx - i0), TYe = min(TY, A.ny - j0);
    const int el = tid / N, k = tid % N;
    const int tx = el % TX, ty = el / TX;
    const bool valid = tx < TXe && ty < TYe;
    const long long e = (long long)(j0 + ty) * A.nx + (i0 + tx);
    const Tab<T>& tb = A.tab;

    // ---- phase 1: tile rows of q and rbar; halo lines ----------------------
    if (valid) {
#pragma unroll
        for (int v = 0; v < V; ++v) {
            T row[N];
            gload_row<N>(A.q + v * A.npts + e * NN + k * N, row);
            sm_store_row<N>(sq + L::sq(v, el, k * N), row);
            gload_row<N>(A.rbar + v * A.npts + e * NN + k * N, row);
            sm_store_row<N>(sr + L::sq(v, el, k * N), row);
        }
    }
    {
        constexpr int NXH = 2 * TY * N, NYH = 2 * TX * N;
        for (int t = tid; t < NXH + NYH; t += NT) {
            const bool xdir = t < NXH;
            const int r0 = xdir ? t : t - NXH;
            const int side = xdir ? r0 / (TY * N) : r0 / (TX * N);
            const int r = xdir ? r0 % (TY * N) : r0 % (TX * N);
            const int pos = r / N, kk = r % N;
            if (pos >= (xdir ? TYe : TXe)) continue;
            int gi, gj;
            if (xdir) {
                gi = side ? i0 + TXe : i0 - 1;
                gj = j0 + pos;
                if (gi < 0 || gi >= A.nx) {
                    if (A.bcx) continue;
                    gi = gi < 0 ? gi + A.nx : gi - A.nx;
                }
            } else {
                gi = i0 + pos;
                gj = side ? j0 + TYe : j0 - 1;
                if (gj < 0 || gj >= A.ny) {
                    if (A.bcy) continue;
                    gj = gj < 0 ? gj + A.ny : gj - A.ny;
                }
            }
            const long long eh = (long long)gj * A.nx + gi;
            // the edge facing the tile: right/top edge of the lower halo,
            // left/bottom edge of the upper halo
            const T* ce = side ? tb.lm : tb.lp;
            const T* cg = side ? tb.dgl : tb.dgr;
            const T sc = xdir ? -A.rhx2 : -A.rhy2;
#pragma unroll
            for (int v = 0; v < V; ++v) {
                const T* sq_ = A.q + v * A.npts + eh * NN;
                const T* sr_ = A.rbar + v * A.npts + eh * NN;
                T lq[N], lr[N];
#pragma unroll
                for (int l = 0; l < N; ++l) {
                    const int pt = xdir ? kk * N + l : l * N + kk;
                    lq[l] = sq_[pt];
                    lr[l] = sc * sr_[pt];
                }
                const T dq = line_dot<N>(ce, lq), dw = line_dot<N>(cg, lr);
                if (xdir) {
                    if (side) { xHq[L::xh(v, pos, kk)] = dq; xHw[L::xh(v, pos, kk)] = dw; }
                    else { xRq[L::xr(v, pos, 0, kk)] = dq; xRw[L::xr(v, pos, 0, kk)] = dw; }
                } else {
                    if (side) { yHq[L::yh(v, pos, kk)] = dq; yHw[L::yh(v, pos, kk)] = dw; }
                    else { yTq[L::yt(v, 0, pos, kk)] = dq; yTw[L::yt(v, 0, pos, kk)] = dw; }
                }
            }
        }
    }
    __syncthreads();

    const bool lwall = A.bcx && i0 + tx == 0, bwall = A.bcy && j0 + ty == 0;
    const bool redge = tx == TXe - 1, tedge = ty == TYe - 1;
    const bool rwall = A.bcx && i0 + TXe == A.nx, twall = A.bcy && j0 + TYe == A.ny;

    // ---- phase 2: volume terms, edge states and edge cotangents -------------
    T qrow[N][V];                 // this row's qbar
    T eL[V], eR[V], wL[V], wR[V];  // left/right edge states and cotangents (row k)
    T eB[V], eT[V], wB[V], wT[V];  // bottom/top (column k)
    if (valid) {
        T q[N][V], xb[N][V], col[N];
#pragma unroll
        for (int v = 0; v < V; ++v) {
            T row[N], rr[N];
            sm_load_row<N>(sq + L::sq(v, el, k * N), row);
            sm_load_row<N>(sr + L::sq(v, el, k * N), rr);
#pragma unroll
            for (int a = 0; a < N; ++a) {
                q[a][v] = row[a];
                xb[a][v] = -A.rhx2 * rr[a];
            }
        }
#pragma unroll
        for (int l = 0; l < N; ++l) {
            T fb[V];
#pragma unroll
            for (int v = 0; v < V; ++v) {
                T s = xb[0][v] * A.M[0][l];
#pragma unroll
                for (int a = 1; a < N; ++a) s = fma(xb[a][v], A.M[a][l], s);
                fb[v] = s;
                qrow[l][v] = T(0);
            }
            flux_vjp<EQ, 0>(q[l], fb, A.ph, qrow[l]);
        }
#pragma unroll
        for (int v = 0; v < V; ++v) {
#pragma unroll
            for (int l = 0; l < N; ++l) col[l] = q[l][v];
            eL[v] = line_dot<N>(tb.lm, col);
            eR[v] = line_dot<N>(tb.lp, col);
#pragma unroll
            for (int l = 0; l < N; ++l) col[l] = xb[l][v];
            wL[v] = line_dot<N>(tb.dgl, col);
            wR[v] = line_dot<N>(tb.dgr, col);
            xRq[L::xr(v, ty, tx + 1, k)] = eR[v];
            xRw[L::xr(v, ty, tx + 1, k)] = wR[v];
        }
    }
    __syncthreads();  // the rows of the tile of q are read: it becomes the column accumulator
    if (valid) {
        T q[N][V], xb[N][V], col[N];
        // column k
#pragma unroll
        for (int b = 0; b < N; ++b)
#pragma unroll
            for (int v = 0; v < V; ++v) {
                q[b][v] = sq[L::sq(v, el, b * N + k)];
                xb[b][v] = -A.rhy2 * sr[L::sq(v, el, b * N + k)];
            }
#pragma unroll
        for (int l = 0; l < N; ++l) {
            T gb[V], c[V];
#pragma unroll
            for (int v = 0; v < V; ++v) {
                T s = xb[0][v] * A.M[0][l];
#pragma unroll
                for (int b = 1; b < N; ++b) s = fma(xb[b][v], A.M[b][l], s);
                gb[v] = s;
                c[v] = T(0);
            }
            flux_vjp<EQ, 1>(q[l], gb, A.ph, c);
#pragma unroll
            for (int v = 0; v < V; ++v) qb[L::sq(v, el, l * N + k)] = c[v];
        }
#pragma unroll
        for (int v = 0; v < V; ++v) {
#pragma unroll
            for (int l = 0; l < N; ++l) col[l] = q[l][v];
            eB[v] = line_dot<N>(tb.lm, col);
            eT[v] = line_dot<N>(tb.lp, col);
#pragma unroll
            for (int l = 0; l < N; ++l) col[l] = xb[l][v];
            wB[v] = line_dot<N>(tb.dgl, col);
            wT[v] = line_dot<N>(tb.dgr, col);
            yTq[L::yt(v, ty + 1, tx, k)] = eT[v];
            yTw[L::yt(v, ty + 1, tx, k)] = wT[v];
        }
    }
    __syncthreads();

    // ---- phase 3: face transposes on the own faces --------------------------
    if (valid) {
        T qm[V], W[V], bm[V], bp[V];
        // left face: lower state = right edge of the left element
#pragma unroll
        for (int v = 0; v < V; ++v) {
            qm[v] = lwall ? eL[v] : xRq[L::xr(v, ty, tx, k)];
            W[v] = wL[v] + (lwall ? T(0) : xRw[L::xr(v, ty, tx, k)]);
        }
        common_flux_vjp<EQ, FLUX, 0>(qm, eL, W, A.ph, bm, bp);
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const T own = bp[v] + (lwall ? bm[v] : T(0));
#pragma unroll
            for (int l = 0; l < N; ++l) qrow[l][v] += tb.lm[l] * own;
            if (!lwall && tx > 0) xQ[L::xq(v, ty, tx, k)] = bm[v];
        }
        if (redge) {
            T qp[V];
#pragma unroll
            for (int v = 0; v < V; ++v) {
                qp[v] = rwall ? eR[v] : xHq[L::xh(v, ty, k)];
                W[v] = wR[v] + (rwall ? T(0) : xHw[L::xh(v, ty, k)]);
            }
            common_flux_vjp<EQ, FLUX, 0>(eR, qp, W, A.ph, bm, bp);
#pragma unroll
            for (int v = 0; v < V; ++v) {
                const T own = bm[v] + (rwall ? bp[v] : T(0));
#pragma unroll
                for (int l = 0; l < N; ++l) qrow[l][v] += tb.lp[l] * own;
            }
        }
        // bottom face (column k)
#pragma unroll
        for (int v = 0; v < V; ++v) {
            qm[v] = bwall ? eB[v] : yTq[L::yt(v, ty, tx, k)];
            W[v] = wB[v] + (bwall ? T(0) : yTw[L::yt(v, ty, tx, k)]);
        }
        common_flux_vjp<EQ, FLUX, 1>(qm, eB, W, A.ph, bm, bp);
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const T own = bp[v] + (bwall ? bm[v] : T(0));
#pragma unroll
            for (int l = 0; l < N; ++l) qb[L::sq(v, el, l * N + k)] += tb.lm[l] * own;
            if (!bwall && ty > 0) yQ[L::yq(v, ty, tx, k)] = bm[v];
        }
        if (tedge) {
            T qp[V];
#pragma unroll
            for (int v = 0; v < V; ++v) {
                qp[v] = twall ? eT[v] : yHq[L::yh(v, tx, k)];
                W[v] = wT[v] + (twall ? T(0) : yHw[L::yh(v, tx, k)]);
            }
            common_flux_vjp<EQ, FLUX, 1>(eT, qp, W, A.ph, bm, bp);
#pragma unroll
            for (int v = 0; v < V; ++v) {
                const T own = bm[v] + (twall ? bp[v] : T(0));
#pragma unroll
                for (int l = 0; l < N; ++l) qb[L::sq(v, el, l * N + k)] += tb.lp[l] * own;
            }
        }
    }
    __syncthreads();

    // ---- phase 4: faces transposed by the right / upper neighbour ---------
    if (valid) {
#pragma unroll
        for (int v = 0; v < V; ++v) {
            if (!redge) {
                const T own = xQ[L::xq(v, ty, tx + 1, k)];
#pragma unroll
                for (int l = 0; l < N; ++l) qrow[l][v] += tb.lp[l] * own;
            }
            if (!tedge) {
                const T own = yQ[L::yq(v, ty + 1, tx, k)];
#pragma unroll
                for (int l = 0; l < N; ++l) qb[L::sq(v, el, l * N + k)] += tb.lp[l] * own;
            }
        }
    }
    __syncthreads();

    // ---- phase 5: row total and epilogue -------------------------------------
    if (valid) {
        const long long off = e * NN + k * N;
#pragma unroll
        for (int v = 0; v < V; ++v) {
            T acc[N], o[N];
            sm_load_row<N>(qb + L::sq(v, el, k * N), acc);
#pragma unroll
            for (int a = 0; a < N; ++a) o[a] = A.cv * (qrow[a][v] + acc[a]);
            if (A.X0) {
                T x[N];
                gload_row<N>(A.X0 + v * A.npts + off, x);
#pragma unroll
                for (int a = 0; a < N; ++a) o[a] += A.c0 * x[a];
            }
            if (A.X1) {
                T x[N];
                gload_row<N>(A.X1 + v * A.npts + off, x);
#pragma unroll
                for (int a = 0; a < N; ++a) o[a] += A.c1 * x[a];
            }
            if (A.X2) {
                T x[N];
                gload_row<N>(A.X2 + v * A.npts + off, x);
#pragma unroll
                for (int a = 0; a < N; ++a) o[a] += A.c2 * x[a];
            }
            gstore_row<N>(A.out + v * A.npts + off, o);
        }
    }
}

}  // namespace cpr
