/*
 * oracle.h -- FP64 CPU oracle of the CPR (Correction Procedure via
 * Reconstruction) hot path of Zimmerman, Regele & Wie, "A Comparative Study of
 * 2D Numerical Methods with GPU Computing" (arXiv 1709.01619).
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the plain, slow, obviously
 * correct reference that the CUDA path is checked against.  Only the test
 * suite, the smoke check and the CPU-baseline leg of the benchmark may load
 * it.  It shares no code, header, table or constant with the CUDA path.
 *
 * Everything is double precision.  Build with -ffp-contract=off so that the
 * results do not depend on whether the host compiler fuses multiply-adds.
 *
 * State layout (same convention as the product, restated here on purpose):
 *   q[v][e][b*n + a],  v = variable, e = j*nx + i (element (i, j), x fastest),
 *   a = solution-point index in xi (x), b = solution-point index in eta (y),
 *   n = p + 1 points per direction.
 * Euler variables: (rho, rho*u, rho*v, e) -- Sec. 2, Eq. 3.
 * Linear advection: one variable.
 *
 * Parity status of each function is recorded next to it:
 *   "pinned by ..."   names the independent checks in tests/test_oracle_*.py
 *   "parity unpinned" marks a function whose only check is invariants.
 */
#ifndef CPR_ORACLE_H
#define CPR_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

#define ORACLE_PMAX 6 /* highest supported order p (n = p + 1 <= 7) */
#define ORACLE_NMAX (ORACLE_PMAX + 1)

enum { OR_ADVECTION = 0, OR_EULER = 1 };
enum { OR_GAUSS = 0, OR_LOBATTO = 1 };
enum { OR_DIV_LP = 0, OR_DIV_CHAIN = 1 };
enum { OR_RUSANOV = 0, OR_UPWIND = 1, OR_ROE = 2 };
enum { OR_PERIODIC = 0, OR_TRANSMISSIVE = 1 };
enum { OR_CPR = 0, OR_FV_MUSCL = 1, OR_FV_MUSCL3 = 2 };
enum { OR_CORR_GDG = 0, OR_CORR_NDG = 1, OR_CORR_NDG_LUMPED = 2 };

typedef struct {
    int eqn;                 /* OR_ADVECTION or OR_EULER                     */
    int nx, ny;              /* elements in x and y                          */
    int p;                   /* polynomial order, 1..ORACLE_PMAX              */
    double x0, x1, y0, y1;   /* domain                                        */
    int pts;                 /* OR_GAUSS or OR_LOBATTO solution points        */
    int div;                 /* OR_DIV_LP (differentiate interpolated flux)   */
                             /* or OR_DIV_CHAIN (paper's chain rule, Sec 2.2) */
    int flux;                /* OR_RUSANOV, OR_UPWIND (advection only) or     */
                             /* OR_ROE (Roe's linearised Riemann solver)      */
    double ax, ay;           /* advection velocity                            */
    double gamma;            /* ratio of specific heats (Euler)               */
    int bc_x, bc_y;          /* OR_PERIODIC or OR_TRANSMISSIVE                */
    int limiter;             /* 1: troubled-cell limiter after every stage    */
    double tvb_M;            /* TVB constant M (0: plain minmod)              */
    double lim_eps;          /* marking threshold epsilon (Sec. 2.6)          */
    double cfl;              /* CFL number for oracle_dt                      */
    int scheme;              /* OR_CPR, or OR_FV_MUSCL: one average per       */
                             /* element (p = 0), second-order MUSCL with      */
                             /* minmod slopes (Sec. 2.1, 2.6, Algorithm 1),   */
                             /* or OR_FV_MUSCL3: third-order MUSCL (Sec. 2.6) */
    int corr;                /* CPR edge correction: OR_CORR_GDG (Radau       */
                             /* g_DG, Sec. 2.2), OR_CORR_NDG (the lifting     */
                             /* operator M^-1 M^A of nodal DG, Sec. 2.3, with */
                             /* the exact mass matrix) or OR_CORR_NDG_LUMPED  */
                             /* (the same with the mass matrices integrated   */
                             /* by the solution-point quadrature)             */
} oracle_cfg;

/* 1D operator tables for n = p + 1 points. */
typedef struct {
    int n;
    double xi[ORACLE_NMAX];           /* solution points on [-1, 1], ascending */
    double w[ORACLE_NMAX];            /* quadrature weights                    */
    double D[ORACLE_NMAX][ORACLE_NMAX]; /* D[a][l] = l_l'(xi_a)               */
    double lm[ORACLE_NMAX];           /* l_l(-1)                               */
    double lp[ORACLE_NMAX];           /* l_l(+1)                               */
    double dgl[ORACLE_NMAX];          /* g_L'(xi_a), left Radau correction     */
    double dgr[ORACLE_NMAX];          /* g_R'(xi_a), right Radau correction    */
} oracle_tab;

/* Legendre polynomial P_k(x) and its derivative (Bonnet recurrence). */
double oracle_legendre(int k, double x);
double oracle_legendre_d(int k, double x);

/* Fill the tables; returns 0 on success, -1 on bad arguments.
 * Pinned by: numpy leggauss nodes/weights, exactness of D on monomials,
 * g_L(-1)=1, g_L(1)=0, sum_a w_a g_L'(xi_a) = -1 (tests/test_oracle_tables.py). */
int oracle_tables(int p, int pts, oracle_tab* T);

/* The same tables with dgl, dgr replaced by the edge-correction
 * coefficients of corr:
 *   OR_CORR_GDG         the Radau derivatives of oracle_tables;
 *   OR_CORR_NDG         nodal DG in strong form (Sec. 2.3): the lifting
 *                       matrix L = M^-1 M^A; on a tensor-product element it
 *                       acts along each line with dgr = M^-1 l(+1),
 *                       dgl = -M^-1 l(-1), M_ij = int l_i l_j over [-1, 1]
 *                       (exact: Gauss rule of n + 1 points);
 *   OR_CORR_NDG_LUMPED  the same with M integrated by the solution points'
 *                       own quadrature (M = diag(w)).
 * Pinned by: NDG equals the Radau derivatives (the equivalence of FR with
 * g_DG and DG), lumped equals exact on Gauss points (the n-point rule is
 * exact for degree 2p), the lumped Lobatto lift is +-p(p+1)/2 at the end
 * node and zero elsewhere (end weight 2/(p(p+1))), and each lift integrates
 * to +-1 (tests/test_oracle_ndg.py). */
int oracle_tables_corr(int p, int pts, int corr, oracle_tab* T);

/* Number of doubles in one state vector: V * nx * ny * (p+1)^2. */
long oracle_state_size(const oracle_cfg* c);
int oracle_nvars(const oracle_cfg* c);

/* Physical coordinates of every solution point, layout x[e][b*n+a]. */
int oracle_point_coords(const oracle_cfg* c, double* x, double* y);

/* Common (Riemann) flux through a face with unit normal (nx, ny) between the
 * state qm on the minus side and qp on the plus side (Sec. 4, Rusanov).
 * Pinned by consistency F(q,q) = f_n(q) and the swap symmetry.
 * OR_ROE: Roe's approximate Riemann solver (Roe-averaged states, the four
 * characteristic fields of the 2D Euler equations along the normal) with
 * the Harten-Hyman entropy fix on the two acoustic fields; for
 * advection it is the upwind flux.  Pinned by consistency, swap symmetry, a
 * stationary contact and a stationary normal shock resolved exactly, and
 * pure upwinding of supersonic states. */
void oracle_common_flux(const oracle_cfg* c, const double* qm, const double* qp,
                        double nx, double ny, double* F);

/* CPR semi-discrete right-hand side R(q) = dq/dt (Sec. 2.2, Eq. 16).
 * Pinned by: equality with an independent modal DG for linear advection,
 * order p+1 convergence, freestream preservation, conservation.
 * scheme == OR_FV_MUSCL: the FV semi-discretisation of Sec. 2.1,
 * dq_ij/dt = -(f_{i+1/2,j} - f_{i-1/2,j})/dx - (g_{i,j+1/2} - g_{i,j-1/2})/dy,
 * with face states reconstructed by second-order MUSCL with minmod-limited
 * slopes (Sec. 2.6) and the common flux of oracle_common_flux.  Pinned by:
 * freestream, conservation, exactness on linear data, reduction to
 * first-order upwind when every slope is limited to zero, total variation
 * diminishing in 1D, second-order convergence, x-y symmetry. */
int oracle_residual(const oracle_cfg* c, const double* q, double* R);

/* Element averages, Algorithm 9: avg[v][e] = sum_l (w_a w_b / 4) q[v][e][l]. */
int oracle_averages(const oracle_cfg* c, const double* q, double* avg);

/* Troubled-cell limiter, Sec. 2.6 Eq. 35 with Algorithms 10-11 (in place).
 * marks[e] (nullable) receives 1 for limited elements; margin[e] (nullable)
 * receives max over edges/variables of |delta - mt(delta, D+, D-)| - eps, the
 * signed distance of the marking decision from its threshold.
 * Returns the number of marked elements.
 * Pinned by: mean preservation, linear fields are fixed points, no marks under a large TVB constant, monotone 1D step. */
long oracle_limit(const oracle_cfg* c, double* q, int* marks, double* margin);

/* Largest signal speed over all solution points: sqrt(u^2+v^2)+c (Euler) or
 * |a| (advection). */
double oracle_max_wave(const oracle_cfg* c, const double* q);

/* CFL time step of Sec. 4, Eq. 36: dt = cfl * min(hx, hy) / max_wave. */
double oracle_dt(const oracle_cfg* c, const double* q);

/* One three-stage SSP Runge-Kutta step (Sec. 4; Shu-Osher form), limiter
 * applied after every stage when c->limiter != 0.  q is updated in place.
 * Pinned by: y' = lambda y gives 1 + z + z^2/2 + z^3/6. */
int oracle_rk3_step(const oracle_cfg* c, double* q, double dt);

/* Up to nsteps SSP-RK3 steps of fixed size dt (dt > 0) or CFL size (dt <= 0).
 * With t_end > 0 the step that would pass t_end is shortened to land on it
 * (time set to t_end exactly) and no step is taken once t_end is reached.
 * *t (nullable) is the start time and receives the end time.  Returns the
 * number of steps taken. */
long oracle_run(const oracle_cfg* c, double* q, long nsteps, double dt,
                double t_end, double* t);

/* Norms of Sec. 4: sum_avg[v] = sum_e avg[v][e]; l2_rel = ||q - ref||_2 /
 * ||ref||_2 over all values (ref nullable); n_nonphys = points with
 * rho <= 0, p <= 0 or a non-finite value. */
typedef struct {
    double sum_avg[4];
    double l2_abs, l2_rel;
    double max_wave;
    long long n_nonphys;
} oracle_norms_out;
int oracle_norms(const oracle_cfg* c, const double* q, const double* ref,
                 oracle_norms_out* out);

/* Exact-solution element averages by a 10x10 Gauss rule per element
 * (Sec. 4: errors compare averaged solution with averaged exact solution).
 * kind 0: advection sin(2 pi (x - ax t)) sin(2 pi (y - ay t)) (1 value/elem)
 * kind 1: isentropic vortex of Sec. 4.1 convected by (uinf, vinf) on the
 *         periodic box, nearest image; writes all 4 conserved averages.
 * par (vortex): {eps, xc, yc, uinf, vinf}. */
int oracle_exact_averages(const oracle_cfg* c, int kind, const double* par,
                          double t, double* avg);

/* RMS over elements of the density-average error (Sec. 4, Tables 6-7). */
double oracle_rho_avg_error(const oracle_cfg* c, const double* q,
                            const double* exact_avg);

/* Discrete adjoint (transpose Jacobian-vector products) on small grids.
 * oracle_residual_jvp: dR = (dR/dq) dq.  oracle_residual_vjp: qbar =
 * (dR/dq)^T rbar.  oracle_rk3_vjp: qbar_in = (dq_{n+1}/dq_n)^T qbar_out for
 * one unlimited SSP-RK3 step at fixed dt from state q.
 * Pinned by: central differences of oracle_residual / oracle_rk3_step and the
 * dot-product identity <J v, w> = <v, J^T w> (tests/test_oracle_adjoint.py). */
int oracle_residual_jvp(const oracle_cfg* c, const double* q, const double* dq,
                        double* dR);
int oracle_residual_vjp(const oracle_cfg* c, const double* q,
                        const double* rbar, double* qbar);
int oracle_rk3_vjp(const oracle_cfg* c, const double* q, double dt,
                   const double* qbar_out, double* qbar_in);

/* Threads used by the element loops (OpenMP), 1 when built without it. */
int oracle_threads(void);
void oracle_set_threads(int n);

#ifdef __cplusplus
}
#endif
#endif
