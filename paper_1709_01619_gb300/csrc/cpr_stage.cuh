// cpr_stage.cuh -- fused CPR residual + SSP-RK3 stage kernel.
//
// One CTA owns a tile of TX x TY elements and computes, for every solution
// point of the tile, the CPR right-hand side of Sec. 2.2 (Eq. 16-17)
//   R_ab = -(2/hx) [ sum_l D_al f_lb + (F*_L,b - f_L,b) g_L'(xi_a) + (F*_R,b - f_R,b) g_R'(xi_a) ]
//          -(2/hy) [ sum_l D_bl g_al + (G*_B,a - g_B,a) g_L'(eta_b) + (G*_T,a - g_T,a) g_R'(eta_b) ]
// and then the stage update of the three-stage SSP Runge-Kutta scheme of
// Sec. 4, out = cA q^n + cB (q_s + dt R), in one pass over HBM.
//
// Thread roles (N = p+1 points per direction, NT = TX*TY*N threads):
//   thread (el, k) is the x-line "row k of element el" and the y-line
//   "column k of element el".  Its row stays in registers from load to store;
//   its column is read from the shared-memory copy of the tile.
// Phases (barriers between them):
//   1 load q_s rows (registers + shared), halo elements (shared)
//   2 x-lines: flux, d/dxi (LP: of the flux; CR: chain rule), edge states;
//     y-lines: same along eta; halo lines: edge states only
//   3 common flux on every face point of the tile (one evaluation per face)
//   4 y-lines: correction along eta, y-part of R into shared memory
//   5 x-lines: correction along xi, add y-part, stage update, store row;
//     optional fused element averages (Algorithm 9) and max signal speed.
// Element coupling (the only non-local data, Fig. 2) comes through the halo
// ring of neighbour elements, which neighbouring CTAs read from L2.
#pragma once

#include "cpr_common.cuh"
#include "cpr_reduce.cuh"

namespace cpr {

template <class T>
struct StageArgs {
    const T* qs;      // stage input state
    const T* qn;      // q^n (read when mode >= 2)
    T* out;           // stage output (mode >= 1) or residual (mode 0)
    T* avg;           // element averages of out (do_avg)
    T* wave;          // per-CTA partial max speed (do_wave)
    Ctrl* ctrl;       // time control (mode >= 1)
    long long npts;   // points per variable, ne * N * N
    int nx, ny;
    int bcx, bcy;     // 1: transmissive
    int tiles_x;
    int mode;         // 0: residual, 1..3: SSP-RK3 stage
    int do_avg, do_wave;
    T rhx2, rhy2;     // 2/hx, 2/hy
    Phys<T> ph;
    Tab<T> tab;
};

template <int N, int V, int TX, int TY>
struct StageLayout {
    static constexpr int NN = N * N;
    static constexpr int SQ = V * (TY + 2) * (TX + 2) * NN;  // tile + halo ring
    static constexpr int XS = V * TY * (TX + 1) * N;         // one x-face array
    static constexpr int YS = V * (TY + 1) * TX * N;         // one y-face array
    static constexpr int TOTAL = SQ + 3 * XS + 3 * YS;
    __device__ static int sq(int v, int ly, int lx, int pt) {
        return ((v * (TY + 2) + ly) * (TX + 2) + lx) * NN + pt;
    }
    __device__ static int xs(int v, int ty, int f, int k) { return ((v * TY + ty) * (TX + 1) + f) * N + k; }
    __device__ static int ys(int v, int g, int tx, int k) { return ((v * (TY + 1) + g) * TX + tx) * N + k; }
};

// Edge value of a line of N values: sum_l c_l x_l, in one fixed fma order so
// that every CTA computing the same trace gets the same bits.
template <int N, class T>
__device__ __forceinline__ T line_dot(const T* c, const T* x)
{
    T s = c[0] * x[0];
#pragma unroll
    for (int l = 1; l < N; ++l) s = fma(c[l], x[l], s);
    return s;
}

template <int N, int V, class T>
__device__ __forceinline__ void load_row(const T* __restrict__ src, long long npts, T (&q)[N][V])
{
#pragma unroll
    for (int v = 0; v < V; ++v) {
        const T* s = src + v * npts;
        if constexpr (sizeof(T) == 4 && N == 4) {
            float4 t = *reinterpret_cast<const float4*>(s);
            q[0][v] = t.x; q[1][v] = t.y; q[2][v] = t.z; q[3][v] = t.w;
        } else if constexpr (sizeof(T) == 4 && N == 2) {
            float2 t = *reinterpret_cast<const float2*>(s);
            q[0][v] = t.x; q[1][v] = t.y;
        } else if constexpr (sizeof(T) == 8 && N % 2 == 0) {
#pragma unroll
            for (int a = 0; a < N; a += 2) {
                double2 t = *reinterpret_cast<const double2*>(s + a);
                q[a][v] = t.x; q[a + 1][v] = t.y;
            }
        } else {
#pragma unroll
            for (int a = 0; a < N; ++a) q[a][v] = s[a];
        }
    }
}

template <int N, int V, class T>
__device__ __forceinline__ void store_row(T* __restrict__ dst, long long npts, const T (&o)[N][V])
{
#pragma unroll
    for (int v = 0; v < V; ++v) {
        T* d = dst + v * npts;
        if constexpr (sizeof(T) == 4 && N == 4) {
            *reinterpret_cast<float4*>(d) = make_float4(o[0][v], o[1][v], o[2][v], o[3][v]);
        } else if constexpr (sizeof(T) == 4 && N == 2) {
            *reinterpret_cast<float2*>(d) = make_float2(o[0][v], o[1][v]);
        } else if constexpr (sizeof(T) == 8 && N % 2 == 0) {
#pragma unroll
            for (int a = 0; a < N; a += 2) *reinterpret_cast<double2*>(d + a) = make_double2(o[a][v], o[a + 1][v]);
        } else {
#pragma unroll
            for (int a = 0; a < N; ++a) d[a] = o[a][v];
        }
    }
}

template <class T, int P, int EQ, int DIV, int FLUX, int TX, int TY>
__global__ void __launch_bounds__(TX * TY * (P + 1))
cpr_stage_kernel(const StageArgs<T> A)
{
    constexpr int N = P + 1, NN = N * N, V = NVars<EQ>::value;
    constexpr int NT = TX * TY * N;
    using L = StageLayout<N, V, TX, TY>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sq = reinterpret_cast<T*>(smem_raw);
    T* xL = sq + L::SQ;  // left edge state of elements 0..TXe (index = element)
    T* xR = xL + L::XS;  // right edge state of elements -1..TXe-1 (index = element + 1)
    T* xF = xR + L::XS;  // common flux on x-faces 0..TXe (face f between elements f-1, f)
    T* yB = xF + L::XS;
    T* yT = yB + L::YS;
    T* yG = yT + L::YS;
    T* ryS = sq;         // y-part of R, reuses the tile copy once it is dead
    T* avS = xL;         // row partial sums of the averages, reuses xL

    if (A.mode > 0 && A.ctrl->done) return;  // t_end reached: uniform exit

    const int tid = threadIdx.x;
    const int i0 = (blockIdx.x % A.tiles_x) * TX;
    const int j0 = (blockIdx.x / A.tiles_x) * TY;
    const int TXe = min(TX, A.nx - i0), TYe = min(TY, A.ny - j0);
    const int el = tid / N, k = tid % N;
    const int tx = el % TX, ty = el / TX;
    const bool valid = tx < TXe && ty < TYe;
    const long long e = (long long)(j0 + ty) * A.nx + (i0 + tx);
    const Tab<T>& tb = A.tab;

    // ---- phase 1: load ----------------------------------------------------
    T q[N][V];
    if (valid) {
        load_row<N, V>(A.qs + e * NN + k * N, A.npts, q);
#pragma unroll
        for (int v = 0; v < V; ++v)
#pragma unroll
            for (int a = 0; a < N; ++a) sq[L::sq(v, ty + 1, tx + 1, k * N + a)] = q[a][v];
    }
    {
        const int nh = 2 * TYe + 2 * TXe;
        for (int idx = tid; idx < nh * NN; idx += NT) {
            const int h = idx / NN, pt = idx % NN;
            int lx, ly;
            if (h < TYe) { lx = -1; ly = h; }
            else if (h < 2 * TYe) { lx = TXe; ly = h - TYe; }
            else if (h < 2 * TYe + TXe) { lx = h - 2 * TYe; ly = -1; }
            else { lx = h - 2 * TYe - TXe; ly = TYe; }
            int gi = i0 + lx, gj = j0 + ly;
            if (gi < 0 || gi >= A.nx) {
                if (A.bcx) continue;
                gi = (gi + A.nx) % A.nx;
            }
            if (gj < 0 || gj >= A.ny) {
                if (A.bcy) continue;
                gj = (gj + A.ny) % A.ny;
            }
            const long long eh = (long long)gj * A.nx + gi;
#pragma unroll
            for (int v = 0; v < V; ++v) sq[L::sq(v, ly + 1, lx + 1, pt)] = A.qs[v * A.npts + eh * NN + pt];
        }
    }
    __syncthreads();

    // ---- phase 2: line operators ----------------------------------------
    T rx[N][V], ry[N][V];
    T fL[V], fR[V], gB[V], gT[V];
    if (valid) {
        // x-line: row k of element el, held in registers
        T f[N][V];
#pragma unroll
        for (int a = 0; a < N; ++a) flux_x<EQ>(q[a], A.ph, f[a]);
        T col[N];
        T qL[V], qR[V];
#pragma unroll
        for (int v = 0; v < V; ++v) {
#pragma unroll
            for (int l = 0; l < N; ++l) col[l] = q[l][v];
            qL[v] = line_dot<N>(tb.lm, col);
            qR[v] = line_dot<N>(tb.lp, col);
        }
        if constexpr (DIV == DIV_LP) {
#pragma unroll
            for (int v = 0; v < V; ++v) {
#pragma unroll
                for (int l = 0; l < N; ++l) col[l] = f[l][v];
#pragma unroll
                for (int a = 0; a < N; ++a) rx[a][v] = line_dot<N>(tb.D[a], col);
                fL[v] = line_dot<N>(tb.lm, col);
                fR[v] = line_dot<N>(tb.lp, col);
            }
        } else {
#pragma unroll
            for (int a = 0; a < N; ++a) {
                T dq[V];
#pragma unroll
                for (int v = 0; v < V; ++v) {
#pragma unroll
                    for (int l = 0; l < N; ++l) col[l] = q[l][v];
                    dq[v] = line_dot<N>(tb.D[a], col);
                }
                flux_jvp<EQ, 0>(q[a], dq, A.ph, rx[a]);
            }
            flux_x<EQ>(qL, A.ph, fL);
            flux_x<EQ>(qR, A.ph, fR);
        }
#pragma unroll
        for (int v = 0; v < V; ++v) {
            xL[L::xs(v, ty, tx, k)] = qL[v];
            xR[L::xs(v, ty, tx + 1, k)] = qR[v];
        }
        // y-line: column k of element el, from shared memory
        T c[N][V], g[N][V];
#pragma unroll
        for (int b = 0; b < N; ++b)
#pragma unroll
            for (int v = 0; v < V; ++v) c[b][v] = sq[L::sq(v, ty + 1, tx + 1, b * N + k)];
#pragma unroll
        for (int b = 0; b < N; ++b) flux_y<EQ>(c[b], A.ph, g[b]);
        T qB[V], qT[V];
#pragma unroll
        for (int v = 0; v < V; ++v) {
#pragma unroll
            for (int l = 0; l < N; ++l) col[l] = c[l][v];
            qB[v] = line_dot<N>(tb.lm, col);
            qT[v] = line_dot<N>(tb.lp, col);
        }
        if constexpr (DIV == DIV_LP) {
#pragma unroll
            for (int v = 0; v < V; ++v) {
#pragma unroll
                for (int l = 0; l < N; ++l) col[l] = g[l][v];
#pragma unroll
                for (int b = 0; b < N; ++b) ry[b][v] = line_dot<N>(tb.D[b], col);
                gB[v] = line_dot<N>(tb.lm, col);
                gT[v] = line_dot<N>(tb.lp, col);
            }
        } else {
#pragma unroll
            for (int b = 0; b < N; ++b) {
                T dq[V];
#pragma unroll
                for (int v = 0; v < V; ++v) {
#pragma unroll
                    for (int l = 0; l < N; ++l) col[l] = c[l][v];
                    dq[v] = line_dot<N>(tb.D[b], col);
                }
                flux_jvp<EQ, 1>(c[b], dq, A.ph, ry[b]);
            }
            flux_y<EQ>(qB, A.ph, gB);
            flux_y<EQ>(qT, A.ph, gT);
        }
#pragma unroll
        for (int v = 0; v < V; ++v) {
            yB[L::ys(v, ty, tx, k)] = qB[v];
            yT[L::ys(v, ty + 1, tx, k)] = qT[v];
        }
    }
    {
        // edge states of the halo elements facing the tile
        const int nxh = 2 * TYe * N, nyh = 2 * TXe * N;
        for (int task = tid; task < nxh + nyh; task += NT) {
            T col[N];
            if (task < nxh) {
                const int side = task / (TYe * N), r = task % (TYe * N);
                const int ly = r / N, kk = r % N;
                const int lx = side ? TXe : -1;
                const int gi = i0 + lx;
                if (A.bcx && (gi < 0 || gi >= A.nx)) continue;
#pragma unroll
                for (int v = 0; v < V; ++v) {
#pragma unroll
                    for (int l = 0; l < N; ++l) col[l] = sq[L::sq(v, ly + 1, lx + 1, kk * N + l)];
                    if (side) xL[L::xs(v, ly, TXe, kk)] = line_dot<N>(tb.lm, col);
                    else xR[L::xs(v, ly, 0, kk)] = line_dot<N>(tb.lp, col);
                }
            } else {
                const int r0 = task - nxh;
                const int side = r0 / (TXe * N), r = r0 % (TXe * N);
                const int lx = r / N, kk = r % N;
                const int ly = side ? TYe : -1;
                const int gj = j0 + ly;
                if (A.bcy && (gj < 0 || gj >= A.ny)) continue;
#pragma unroll
                for (int v = 0; v < V; ++v) {
#pragma unroll
                    for (int l = 0; l < N; ++l) col[l] = sq[L::sq(v, ly + 1, lx + 1, l * N + kk)];
                    if (side) yB[L::ys(v, TYe, lx, kk)] = line_dot<N>(tb.lm, col);
                    else yT[L::ys(v, 0, lx, kk)] = line_dot<N>(tb.lp, col);
                }
            }
        }
    }
    __syncthreads();

    // ---- phase 3: common flux, one evaluation per face point --------------
    {
        const int nxf = TYe * (TXe + 1) * N, nyf = TXe * (TYe + 1) * N;
        for (int task = tid; task < nxf + nyf; task += NT) {
            T qm[V], qp[V], F[V];
            if (task < nxf) {
                const int ly = task / ((TXe + 1) * N), r = task % ((TXe + 1) * N);
                const int f = r / N, kk = r % N;
                const int gf = i0 + f;  // global face: between elements gf-1 and gf
                const bool left_wall = A.bcx && gf == 0, right_wall = A.bcx && gf == A.nx;
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    T a = left_wall ? T(0) : xR[L::xs(v, ly, f, kk)];
                    T b = right_wall ? T(0) : xL[L::xs(v, ly, f, kk)];
                    qm[v] = left_wall ? b : a;
                    qp[v] = right_wall ? a : b;
                }
                common_flux<EQ, FLUX, 0>(qm, qp, A.ph, F);
#pragma unroll
                for (int v = 0; v < V; ++v) xF[L::xs(v, ly, f, kk)] = F[v];
            } else {
                const int r0 = task - nxf;
                const int lx = r0 / ((TYe + 1) * N), r = r0 % ((TYe + 1) * N);
                const int gl = r / N, kk = r % N;
                const int gg = j0 + gl;
                const bool bot_wall = A.bcy && gg == 0, top_wall = A.bcy && gg == A.ny;
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    T a = bot_wall ? T(0) : yT[L::ys(v, gl, lx, kk)];
                    T b = top_wall ? T(0) : yB[L::ys(v, gl, lx, kk)];
                    qm[v] = bot_wall ? b : a;
                    qp[v] = top_wall ? a : b;
                }
                common_flux<EQ, FLUX, 1>(qm, qp, A.ph, F);
#pragma unroll
                for (int v = 0; v < V; ++v) yG[L::ys(v, gl, lx, kk)] = F[v];
            }
        }
    }
    __syncthreads();

    // ---- phase 4: correction along eta, y-part of R -----------------------
    if (valid) {
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const T JB = yG[L::ys(v, ty, tx, k)] - gB[v];
            const T JT = yG[L::ys(v, ty + 1, tx, k)] - gT[v];
#pragma unroll
            for (int b = 0; b < N; ++b) {
                T ys = ry[b][v] + JB * tb.dgl[b];
                ys = ys + JT * tb.dgr[b];
                ryS[(v * TX * TY + el) * NN + b * N + k] = -A.rhy2 * ys;
            }
        }
    }
    __syncthreads();

    // ---- phase 5: correction along xi, stage update, store ------------------
    T o[N][V];
    if (valid) {
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const T JL = xF[L::xs(v, ty, tx, k)] - fL[v];
            const T JR = xF[L::xs(v, ty, tx + 1, k)] - fR[v];
#pragma unroll
            for (int a = 0; a < N; ++a) {
                T xs = rx[a][v] + JL * tb.dgl[a];
                xs = xs + JR * tb.dgr[a];
                o[a][v] = -A.rhx2 * xs + ryS[(v * TX * TY + el) * NN + k * N + a];
            }
        }
        if (A.mode >= 1) {
            const T dt = T(A.ctrl->dt);
            if (A.mode == 1) {
#pragma unroll
                for (int a = 0; a < N; ++a)
#pragma unroll
                    for (int v = 0; v < V; ++v) o[a][v] = q[a][v] + dt * o[a][v];
            } else {
                T qn[N][V];
                load_row<N, V>(A.qn + e * NN + k * N, A.npts, qn);
                const T cA = A.mode == 2 ? T(0.75) : T(1.0 / 3.0);
                const T cB = A.mode == 2 ? T(0.25) : T(2.0 / 3.0);
#pragma unroll
                for (int a = 0; a < N; ++a)
#pragma unroll
                    for (int v = 0; v < V; ++v) o[a][v] = cA * qn[a][v] + cB * (q[a][v] + dt * o[a][v]);
            }
        }
        store_row<N, V>(A.out + e * NN + k * N, A.npts, o);
    }

    // ---- fused element averages (Algorithm 9) -----------------------------
    if (A.do_avg) {
        if (valid) {
#pragma unroll
            for (int v = 0; v < V; ++v) {
                T col[N];
#pragma unroll
                for (int a = 0; a < N; ++a) col[a] = o[a][v];
                avS[(v * TX * TY + el) * N + k] = line_dot<N>(tb.cavg[k], col);
            }
        }
        __syncthreads();
        if (valid && k == 0) {
#pragma unroll
            for (int v = 0; v < V; ++v) {
                T s = avS[(v * TX * TY + el) * N];
#pragma unroll
                for (int b = 1; b < N; ++b) s = s + avS[(v * TX * TY + el) * N + b];
                A.avg[(long long)v * (A.npts / NN) + e] = s;
            }
        }
    }

    // ---- fused max signal speed for the next CFL step ---------------------
    if (A.do_wave) {
        T m = T(0);
        if (valid) {
#pragma unroll
            for (int a = 0; a < N; ++a) {
                T s = point_speed<EQ>(o[a], A.ph);
                m = s > m ? s : m;
            }
        }
        m = block_max<T>(m);
        last_cta_time_update<T>(m, A.wave, A.ctrl, /*advance=*/true);
    }
}

}  // namespace cpr
