/*
 * cpr.h -- C ABI of libcpr.so, the GB300 (sm_103a) CUDA implementation of the
 * Correction Procedure via Reconstruction (CPR) hot path of Zimmerman, Regele
 * & Wie, "A Comparative Study of 2D Numerical Methods with GPU Computing"
 * (arXiv 1709.01619): the CPR semi-discrete residual for 2D linear advection
 * and the compressible Euler equations on structured quadrilateral elements
 * (Sec. 2.2, Eq. 16-17), advanced by three-stage SSP Runge-Kutta with a CFL
 * time step (Sec. 4, Eq. 36), with the troubled-cell minmod/TVB limiter for
 * discontinuous flows (Sec. 2.6, Eq. 35, Algorithms 10-11).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * State layout ("element-major structure of arrays"): a contiguous array of
 * V * nx * ny * (p+1)^2 values of the configured dtype,
 *     q[v][e][b*(p+1) + a],   e = j*nx + i,
 * v the variable (V = 1 for advection; V = 4 for Euler with the conserved
 * variables (rho, rho u, rho v, e) of Sec. 2 Eq. 3), (i, j) the element, a the
 * solution point along x and b along y.  Solution points on the reference
 * element [-1,1]^2 are the tensor product of Gauss-Legendre (default) or
 * Gauss-Lobatto (the paper's choice, Sec. 2.2 and Fig. 1b) points.
 *
 * Ownership: the caller owns every state buffer it passes (device memory of
 * the context's device, at least 16-byte aligned -- cudaMalloc and the
 * PyTorch caching allocator give 256 -- never aliasing one another unless
 * stated; a misaligned array is rejected with CPR_EINVAL).  The
 * context owns its operator tables, stage scratch buffers, reduction buffers,
 * CUDA graphs and the simulated time.
 *
 * Streams: all device work of a context is issued on the stream given to
 * cpr_init (NULL = the legacy default stream), in call order.  Calls return
 * once the work is enqueued, except cpr_norms, cpr_get_marks, cpr_get_time
 * and cpr_step_host, which synchronise that stream.  Asynchronous CUDA errors
 * surface as CPR_ECUDA at the next synchronising call.
 *
 * Errors: every call returns a cpr_status; nothing is thrown across the ABI.
 * Invalid arguments (NULL pointers, sizes, unsupported option combinations)
 * return CPR_EINVAL before any launch.  cpr_last_error gives a message.
 */
#ifndef CPR_H
#define CPR_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    CPR_OK = 0,
    CPR_EINVAL = 1,    /* bad argument or unsupported option combination */
    CPR_ENOMEM = 2,    /* device or host allocation failed                */
    CPR_ECUDA = 3,     /* a CUDA runtime call or a kernel failed          */
    CPR_ENONPHYS = 4,  /* state holds rho <= 0, p <= 0 or a non-finite value */
    CPR_ETIMEOUT = 5,  /* a bounded device wait gave up                   */
    CPR_ENOTIMPL = 6   /* option recognised but not built                 */
} cpr_status;

enum { CPR_ADVECTION = 0, CPR_EULER = 1 };                       /* cpr_config.eqn  */
enum { CPR_PTS_GAUSS = 0, CPR_PTS_LOBATTO = 1 };                 /* .pts            */
enum { CPR_CORR_GDG = 0, CPR_CORR_NDG = 1, CPR_CORR_NDG_LUMPED = 2 }; /* .corr      */
enum { CPR_FLUX_RUSANOV = 0, CPR_FLUX_UPWIND = 1, CPR_FLUX_ROE = 2 }; /* .flux      */
enum { CPR_DIV_LP = 0, CPR_DIV_CHAIN = 1 };                      /* .div            */
enum { CPR_BC_PERIODIC = 0, CPR_BC_TRANSMISSIVE = 1 };           /* .bc_x, .bc_y    */
enum { CPR_F64 = 0, CPR_F32 = 1 };                               /* .dtype          */
enum { CPR_SCHEME_CPR = 0, CPR_SCHEME_FV_MUSCL = 1, CPR_SCHEME_FV_MUSCL3 = 2 }; /* .scheme */

/* Problem and scheme description.
 *   eqn      CPR_ADVECTION (u_t + ax u_x + ay u_y = 0) or CPR_EULER (Sec. 2).
 *   nx, ny   elements in x and y, each >= 1.
 *   x0..y1   rectangular domain, x1 > x0, y1 > y0; uniform elements.
 *   p        polynomial order, 1 <= p <= 4 (p+1 points per direction).
 *   pts      solution points: Gauss-Legendre or Gauss-Lobatto.
 *   corr     edge correction: CPR_CORR_GDG, the derivatives of the Radau
 *            correction polynomials g_DG (Sec. 2.2); CPR_CORR_NDG, the
 *            lifting operator M^-1 M^A of the nodal DG strong form (Sec.
 *            2.3) with the exact mass matrix, which acts along each line
 *            of the tensor-product element (the same scheme as g_DG, the
 *            equivalence of DG and FR, with tables formed by a mass-matrix
 *            solve); CPR_CORR_NDG_LUMPED, the same with the mass matrices
 *            integrated by the solution points' own quadrature (equal to
 *            the exact one on Gauss points; on Gauss-Lobatto points the
 *            lift acts on the end points only, 'DG spectral element').
 *   flux     common flux: Rusanov (Sec. 4) for both equations, exact upwind
 *            for advection, or Roe's approximate Riemann solver with the
 *            Harten-Hyman entropy fix (the upwind flux for advection); the
 *            adjoint entry points and batches do not take CPR_FLUX_ROE.
 *   div      flux divergence: CPR_DIV_LP differentiates the Lagrange
 *            interpolant of the flux; CPR_DIV_CHAIN is the paper's chain rule
 *            A(q) dq/dxi (Sec. 2.2).
 *   ax, ay   advection velocity; gamma ratio of specific heats (Euler).
 *   bc_x/y   periodic or transmissive (ghost state = interior edge state).
 *   limiter  1: troubled-cell limiter on every stage result and in
 *            cpr_limit; tvb_M is the TVB constant M (0: plain minmod) and
 *            lim_eps the marking threshold (the paper uses 1e-3).
 *   dtype    arithmetic and storage type of the state: CPR_F64 or CPR_F32.
 *            Reductions and simulated time are FP64 in both.
 *   cfl      CFL number of the time step dt = cfl * min(hx, hy) / max_speed
 *            (Sec. 4, Eq. 36), max_speed = max over points of |u| + c.
 *   scheme   CPR_SCHEME_CPR, or CPR_SCHEME_FV_MUSCL: the finite-volume
 *            comparison scheme of the paper (Sec. 2.1), one average per
 *            element, face states by second-order MUSCL reconstruction with
 *            minmod-limited slopes (Sec. 2.6, Algorithm 1), the same common
 *            flux, boundary conditions, time stepping and CFL rule; or
 *            CPR_SCHEME_FV_MUSCL3, the same with the third-order MUSCL
 *            reconstruction of Sec. 2.6 (van Leer's kappa = 1/3 face values,
 *            each one-sided difference limited by minmod against four times
 *            the other, so that a face state never leaves the range of the
 *            two averages beside it).  FV needs
 *            p = 0 and limiter = 0 (pts, corr and div are ignored); its state
 *            is q[v][e] (one value per element, the element centre stands
 *            for the element in cpr_point_coords); cpr_limit, the adjoint
 *            entry points and batches return CPR_EINVAL for it. */
typedef struct {
    int eqn;
    int nx, ny;
    double x0, x1, y0, y1;
    int p;
    int pts;
    int corr;
    int flux;
    int div;
    double ax, ay, gamma;
    int bc_x, bc_y;
    int limiter;
    double tvb_M, lim_eps;
    int dtype;
    double cfl;
    int scheme;
} cpr_config;

/* Results of cpr_norms (all FP64).
 *   sum_avg[v]  sum over elements of the element average of variable v
 *               (Algorithm 9; conserved to round-off on periodic grids);
 *   l2_abs/rel  ||q - q_ref||_2 and ||q - q_ref||_2 / ||q_ref||_2 over all
 *               values (0 when no reference is given);
 *   max_wave    max over points of |u| + c (|a| for advection);
 *   n_nonphys   points with rho <= 0, p <= 0 or a non-finite value;
 *   n_marked    elements marked by the most recent limiter pass;
 *   t, steps    simulated time and RK3 steps taken by this context. */
typedef struct {
    double sum_avg[4];
    double l2_abs, l2_rel;
    double max_wave;
    long long n_nonphys;
    long long n_marked;
    double t;
    long long steps;
} cpr_norms_out;

typedef struct cpr_ctx cpr_ctx;

/* Create a context on the current CUDA device.  Validates *cfg (CPR_EINVAL),
 * builds the operator tables on the host in FP64, allocates the stage
 * scratch (two state-sized buffers), reduction buffers and the control
 * block, and sets the simulated time to 0.  stream is a cudaStream_t (may be
 * NULL).  On failure *out is NULL. */
cpr_status cpr_init(const cpr_config* cfg, void* stream, cpr_ctx** out);

/* Release everything the context owns (NULL is accepted). */
void cpr_destroy(cpr_ctx* ctx);

/* Number of values in one state array: V * nx * ny * (p+1)^2. */
size_t cpr_state_elems(const cpr_ctx* ctx);

/* Message of the last failed call on ctx (or of the last failed cpr_init when
 * ctx is NULL).  Valid until the next call on the same context. */
const char* cpr_last_error(const cpr_ctx* ctx);

/* Physical coordinates of every solution point, host arrays of
 * nx*ny*(p+1)^2 doubles each, layout x[e][b*(p+1) + a] (the affine map of
 * the standard element, Sec. 2). */
cpr_status cpr_point_coords(const cpr_ctx* ctx, double* x_host, double* y_host);

/* r = R(q), the CPR right-hand side dq/dt = -(Pi[div F] + delta) at every
 * solution point (Sec. 2.2, Eq. 16-17), with the common flux of cfg.flux on
 * every face.  q_dev and r_dev: device state arrays; must not alias. */
cpr_status cpr_residual(cpr_ctx* ctx, const void* q_dev, void* r_dev);

/* Advance q_dev in place by up to nsteps SSP-RK3 steps (Sec. 4):
 *   q1 = q + dt R(q);  q2 = 3/4 q + 1/4 (q1 + dt R(q1));
 *   q  = 1/3 q + 2/3 (q2 + dt R(q2)),
 * applying the limiter to q1, q2 and q when cfg.limiter is set.
 * dt_fixed > 0: every step uses dt_fixed.  dt_fixed <= 0: each step uses the
 * CFL step of the state at its start, computed on the device.
 * t_end > 0: no step goes past simulated time t_end; the step that reaches
 * it is shortened to land on t_end and the remaining steps do no work.
 * The simulated time and step count advance on the device, so consecutive
 * steps need no host synchronisation; the RK loop runs as CUDA graph
 * replays. */
cpr_status cpr_step(cpr_ctx* ctx, void* q_dev, int nsteps, double dt_fixed, double t_end);

/* Same as cpr_step for a state held in HOST memory: copies q_in_host to the
 * device, steps, copies the result to q_out_host (may equal q_in_host) and
 * synchronises.  Pinned host memory gives the fastest copies.  The device
 * state lives in a context-owned buffer allocated on first use. */
cpr_status cpr_step_host(cpr_ctx* ctx, const void* q_in_host, void* q_out_host, int nsteps,
                         double dt_fixed, double t_end);

/* Apply the troubled-cell limiter once to q_dev in place (Sec. 2.6 Eq. 35,
 * Algorithms 10-11): an element is marked when, at any edge point and for
 * any variable, |delta - mt(delta, D+, D-)| > lim_eps, where delta is the
 * outward deviation of the edge value from the element average, D+/D- the
 * differences of neighbouring averages across that edge, and mt the TVB
 * minmod; marked elements become qbar + (x - x0) mm(Dx+/hx, Dx-/hx)
 * + (y - y0) mm(Dy+/hy, Dy-/hy).  Works whether or not cfg.limiter is set. */
cpr_status cpr_limit(cpr_ctx* ctx, void* q_dev);

/* Marks of the most recent limiter pass: marks_host[e] = 1 for limited
 * elements (nx*ny ints).  Synchronises. */
cpr_status cpr_get_marks(cpr_ctx* ctx, int* marks_host);

/* Element averages of q_dev (Algorithm 9): avg_dev[v][e] = sum over points of
 * (w_a w_b / 4) q[v][e][b*n+a], V*nx*ny values of the state dtype. */
cpr_status cpr_averages(cpr_ctx* ctx, const void* q_dev, void* avg_dev);

/* FP64 norms of q_dev (q_ref_dev nullable), see cpr_norms_out; deterministic
 * (fixed reduction order).  Synchronises.  Returns CPR_ENONPHYS (with *out
 * filled) when n_nonphys > 0. */
cpr_status cpr_norms(cpr_ctx* ctx, const void* q_dev, const void* q_ref_dev, cpr_norms_out* out);

/* Simulated time and step counter of the context. */
cpr_status cpr_set_time(cpr_ctx* ctx, double t, long long steps);
cpr_status cpr_get_time(cpr_ctx* ctx, double* t, long long* steps);

/* Discrete adjoint (smooth, unlimited, LP divergence):
 * cpr_residual_vjp: qbar = (dR/dq)^T rbar at state q.
 * cpr_step_vjp: qbar_in = (dq_{n+1}/dq_n)^T qbar_out for one SSP-RK3 step of
 * size dt from state q_dev (stages recomputed internally).
 * All arguments are device state arrays that must not alias. */
cpr_status cpr_residual_vjp(cpr_ctx* ctx, const void* q_dev, const void* rbar_dev, void* qbar_dev);
cpr_status cpr_step_vjp(cpr_ctx* ctx, const void* q_dev, const void* qbar_out_dev, void* qbar_in_dev,
                        double dt);

/* The two halves of cpr_step_vjp for a reverse sweep over stored steps:
 * cpr_step_stages runs one SSP-RK3 step of size dt from q_dev in the
 * Shu-Osher form of Sec. 4, keeping its stage states:
 *   q1 = q + dt R(q),  q2 = 3/4 q + 1/4 (q1 + dt R(q1)),
 *   q_next = 1/3 q + 2/3 (q2 + dt R(q2))
 * (the arithmetic of cpr_step's FP64 path; the context's simulated time is
 * not advanced); cpr_step_vjp_stages is cpr_step_vjp with those stage states
 * given instead of recomputed, so a reverse sweep costs the three transposed
 * residuals per step.  Same conditions as cpr_step_vjp (CPR scheme, LP
 * divergence, no limiter, dt finite and > 0); q1, q2 and q_next must not
 * alias q or each other (q_next may be q for cpr_step_stages, which then
 * overwrites it), the cotangents must not alias any state. */
cpr_status cpr_step_stages(cpr_ctx* ctx, const void* q_dev, void* q1_dev, void* q2_dev, void* q_next_dev,
                           double dt);
cpr_status cpr_step_vjp_stages(cpr_ctx* ctx, const void* q_dev, const void* q1_dev, const void* q2_dev,
                               const void* qbar_out_dev, void* qbar_in_dev, double dt);

/* ---- batches ------------------------------------------------------------
 * Many independent problems of uneven size and order advanced together (no
 * counterpart in the paper's single-grid runs).  For every SSP-RK3 stage
 * there is one launch per polynomial order present in the batch; it covers
 * the tiles of all instances of that order, either one CTA per tile or a
 * persistent grid whose CTAs walk the tile list (the autotuner picks).  Each
 * instance keeps its own simulated time and CFL step.  All instances share
 * eqn, dtype and flux; batches run Gauss points, the LP divergence and no
 * limiter (CPR_EINVAL otherwise).  FP32 batches use the compensated
 * increment form of the RK stages like cpr_step. */
typedef struct cpr_batch cpr_batch;

/* Create a batch of n instances (cfgs[0..n-1]) on the current device; the
 * batch owns two stage buffers, the low part of the state (FP32) and a
 * control block per instance. */
cpr_status cpr_batch_init(const cpr_config* cfgs, int n, void* stream, cpr_batch** out);
void cpr_batch_destroy(cpr_batch* b);
const char* cpr_batch_last_error(const cpr_batch* b);

/* Advance every instance i, state q_devs[i] (layout of cfgs[i], in place),
 * by up to nsteps SSP-RK3 steps with the semantics of cpr_step (dt_fixed,
 * t_end apply to every instance; CFL steps are per instance).  Changing the
 * set of q_devs pointers between calls synchronises the stream once. */
cpr_status cpr_batch_step(cpr_batch* b, void* const* q_devs, int nsteps, double dt_fixed, double t_end);

/* Same as cpr_batch_step for states held in HOST memory: copies every
 * q_in_host[i] (layout of cfgs[i]) to a batch-owned device array (allocated
 * on first use), steps, copies the results to q_out_host[i] (may equal
 * q_in_host[i]) and synchronises; the results equal cpr_batch_step's bit for
 * bit.  In the per-instance form (cpr_batch_set_form / cpr_batch_tune), with
 * nsteps >= 16 and every buffer page-locked (cudaHostAlloc or registered),
 * each instance's copies run in its own chain of steps, so that they
 * overlap the steps of other instances; the graphs that do this are bound
 * to the host buffers and captured again when the buffers change.  Other
 * calls copy in, step and copy out one after the other. */
cpr_status cpr_batch_step_host(cpr_batch* b, const void* const* q_in_host, void* const* q_out_host, int nsteps,
                               double dt_fixed, double t_end);

/* Autotuner: for each order group, times one RK3 step for each tile family
 * (8x8 and 16x4 elements per CTA) with one CTA per tile and with each
 * persistent grid of 1..max resident CTAs per SM smaller than that, and
 * keeps the fastest; then times the whole batch in that grouped form against
 * the per-instance form (see cpr_batch_set_form) and keeps the faster.  The
 * states q_devs are not modified and the simulated times are kept.  choices
 * (nullable) receives 3 ints per group: p, family, grid size (equal to the
 * group's tile count for one CTA per tile; family 2 and grid 0 when the
 * per-instance form won); *ngroups (nullable) the group count (at most 4).
 * Synchronises. */
cpr_status cpr_batch_tune(cpr_batch* b, void* const* q_devs, int* choices, int* ngroups);

/* Form of the batched step.  0 (the default): one launch per order group
 * and stage over the work list of all tiles of that order.  1: every
 * instance runs the single-problem stage kernel on a stream of its own
 * inside the step graphs (independent chains, joined at the end of a graph;
 * the state pointers are baked into the graphs, which are re-captured when
 * they change).  Results are the same to rounding.  Synchronises;
 * CPR_EINVAL for another value. */
cpr_status cpr_batch_set_form(cpr_batch* b, int per_instance);

/* Simulated time and steps of instance i (synchronises); set the time of
 * every instance (synchronises). */
cpr_status cpr_batch_get_time(cpr_batch* b, int i, double* t, long long* steps);
cpr_status cpr_batch_set_time(cpr_batch* b, double t, long long steps);

/* Largest state, in bytes, that cpr_step_noalloc accepts (16 MiB). */
#define CPR_NOALLOC_MAX_STATE_BYTES (16u << 20)

/* cpr_step_noalloc -- nsteps SSP-RK3 steps of fixed size dt on q_dev, in
 * place, with no context and no device allocation.  The paper has no
 * counterpart: this entry point exists for callers that cannot let a library
 * allocate device memory, such as a host framework whose own pool allocator
 * owns the device memory (an allocation behind its back can fail or break
 * its accounting) or a latency-critical loop where cudaMalloc/cudaFree, which
 * may synchronise the device, are not allowed.
 *   cfg     problem description, validated as by cpr_init; in addition the
 *           limiter must be off and the scheme CPR_SCHEME_CPR (CPR_EINVAL
 *           otherwise); cfl is ignored.
 *   q_dev   device state array (layout and alignment as above), the only
 *           memory the caller provides; it holds the result.
 *   dt      step size (> 0); stream: cudaStream_t or NULL.
 * Arithmetic: the stages of cpr_step with a fixed step -- FP64 the
 * Shu-Osher stages, FP32 the compensated increment form (the new state kept
 * as a high and a low part, the low part cleared at the start of each call),
 * so results equal those of cpr_step called with the same steps.
 * The two stage buffers, the FP32 low part and the control block live in one
 * file-scope device array of 3 * CPR_NOALLOC_MAX_STATE_BYTES + 256 bytes
 * that every GPU loading libcpr.so holds until the process exits.  A state
 * larger than CPR_NOALLOC_MAX_STATE_BYTES returns CPR_EINVAL before any
 * work.  Every call looks up the array's device address on the current
 * device (cudaGetSymbolAddress); the first call on a device also loads the
 * kernels there, so make that first call before any stream capture.  All
 * calls share the array and it keeps the previous call's contents: each call
 * rewrites the control block and clears the low part first, and calls that
 * overlap on the GPU (different streams, or host threads without ordering
 * between them) race on it.  Returns CPR_ECUDA if the symbol lookup or a
 * launch fails.  Simulated time is not tracked. */
cpr_status cpr_step_noalloc(const cpr_config* cfg, void* q_dev, int nsteps, double dt, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* CPR_H */
