/*
 * kbl.h -- C ABI of libkbl, a GB300 (sm_103a) implementation of the kinetic
 * bounds and limiting of Dzanic & Martinelli, "High-order limiting methods
 * using maximum principle bounds derived from the Boltzmann equation I: Euler
 * equations" (arXiv 2407.20966), inside an explicit Gauss-Legendre flux
 * reconstruction (nodal DG) Euler SSP-RK3 stage.
 *
 * Every compute call runs hand-written CUDA kernels on the context's stream;
 * there is no CPU fallback.  Calls are asynchronous unless stated otherwise.
 *
 * Conventions
 *   d      dimension, 1 or 2; nv = d + 2 components (rho, m_x[, m_y], E).
 *   p      order 1..5; Ns = (p+1)^d Gauss-Legendre solution points per
 *          element, x index fastest (node j*(p+1) + i).
 *   faces  1D: 0 = -x, 1 = +x, one point each.  2D: 0 = -x, 1 = +x, 2 = -y,
 *          3 = +y, p+1 Gauss-Legendre points each, ordered by increasing
 *          coordinate along the face; face point f*(p+1) + k.  Nfp = 2 (1D)
 *          or 4(p+1) (2D).
 *   stencil (Sec. 5 of the paper): S = the Ns solution points, the Nfp own
 *          face points, then the exterior values at the same Nfp points;
 *          |S| = Ns + 2 Nfp.  The limiting set V is the first Ns + Nfp.
 *   layouts (all FP64, C order, device memory unless a name says host):
 *          solution  w  [nv][E][Ns]
 *          traces    wf [nv][E][Nfp]   interior value at each face point
 *          residual  R  [nv][E][Ns]    R = -div F (FR with g_DG correction)
 *          bounds    bnd[2][nv][E]     bnd[0] lower, bnd[1] upper
 *          alpha     [2][E]            alpha_min (Eq. 39), alpha_P (Eq. 49)
 *   mesh   axis-aligned Cartesian elements.  nbr[E][2d] >= 0 is the element
 *          across face f, matched to its face f^1 with the same point order;
 *          nbr < 0 marks a boundary face with exterior state bc[-(nbr+1)].
 *
 * Ownership: the caller owns every array passed in; the library owns its
 * context, its copy of the mesh and its scratch space (allocated by
 * kbl_mesh_upload, freed by kbl_destroy).
 *
 * Errors: every call returns kbl_status and never aborts or traps.
 * KBL_EINVAL for bad arguments (nothing is launched); KBL_ECUDA when a CUDA
 * call fails; a device-side check that meets a non-physical stencil state
 * (rho <= 0 or P <= 0) writes NaN bounds for that element and raises a flag
 * that kbl_check / kbl_read_counters report as KBL_ENONPHYSICAL.
 * kbl_last_error gives a message for the last failure of a context.
 */
#ifndef KBL_H
#define KBL_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    KBL_OK = 0,
    KBL_EINVAL = 1,
    KBL_ENONPHYSICAL = 2,
    KBL_ECUDA = 3,
    KBL_ENOMEM = 4,
    KBL_ETIMEOUT = 5,
    KBL_ESTATE = 6
} kbl_status;

/* Arithmetic of the path.
 * KBL_FP64: everything in FP64.
 * KBL_FP32_MIXED: Maxwellians, envelopes and velocity sums in FP32 (2D: each thread sums its
 *   16 velocity nodes, the threads' sums meet in a pairwise tree, at most 25 roundings of the sum
 *   of magnitudes, which for these single-signed sums is the sum itself: <= 1.5e-6 relative;
 *   1D: compensated block sums); the residual and the time step in FP32 arithmetic on FP64
 *   storage; FP64 for rho E - |m|^2/2 and its positivity test in the bounds, the state, the
 *   face traces and the limiter (whose FP32 screen only certifies alpha = 1 exactly). */
typedef enum { KBL_FP64 = 0, KBL_FP32_MIXED = 1 } kbl_precision;

typedef struct {
    int dim;          /* 1 or 2 */
    int p;            /* polynomial order, 1..5 */
    int nu[2];        /* velocity points per axis (Sec. 3.7); 2D: nu[0] == nu[1], 2..64 (8, 16,
                         32 and 64 fill the kernels' tiles; other counts run on the next
                         tile up with zero-weight padding); 1D: 2..4096 */
    double gamma;     /* ratio of specific heats */
    double k;         /* box half-width in thermal units, Eq. 45 (4 in Sec. 5) */
    double r_fac;     /* relaxation of the envelopes, Eq. 40 (1e-3; 0 = strict) */
    double eps;       /* threshold of the alpha rule stated under Eq. 37 (1e-13) */
    double rho_floor; /* density floor on rho_min, Sec. 3.8 (1e-12) */
    double p_floor;   /* pressure floor of Eq. 47-49 (1e-12) */
    int eps_rule;     /* 0: alpha_i = 0 when |min_V - mean| or |max_V - mean| < eps
                         (as printed); 1: such a component is skipped */
    int precision;    /* kbl_precision */
    int uncoupled;    /* 0: every component takes alpha_min = min_i alpha_i (Eq. 38-39, the
                         paper's choice); 1: each component its own alpha_i (the independent
                         limiting stated after Eq. 39).  The pressure step of Eq. 47-49
                         follows in both cases; alpha[0][e] reports alpha_min. */
    int flux;         /* common flux of the residual: 0 Rusanov with the Davis wavespeed
                         (assumption (iv) of Sec. 4), 1 HLLC (Toro, Spruce & Speares 1994,
                         the flux of the experiments, Sec. 5), 2 HLL (Harten, Lax & van
                         Leer 1983, the flux of the Sedov run, Sec. 6.6), both with Davis
                         wave-speed estimates.  Other values: KBL_EINVAL.  The residual
                         adjoint covers flux 0. */
    int quadrature;   /* velocity quadrature on the equispaced grid: 0 the trapezoidal rule
                         (Sec. 3.7, Sec. 5), 1 Romberg (the alternative Sec. 5 names): with
                         nu - 1 = 2^L m, m odd, Richardson extrapolation of the L + 1 nested
                         trapezoidal sums of steps 2^L h .. h; needs nu - 1 even (KBL_EINVAL
                         otherwise).  Its weights are positive, so every envelope argument
                         of Sec. 4 holds unchanged.  The bounds adjoint covers 0. */
    int stencil;      /* 0: the numerical stencil of Sec. 5 (the |S| = Ns + 2 Nfp rows above);
                         1 (1D only, else KBL_EINVAL): the element's own solution points and all
                         solution points of both face neighbours, |S| = 3 Ns (a boundary face
                         contributes its boundary state Ns times); V, the limiting set, is
                         unchanged.  Bounds, gather and step follow it. */
} kbl_config;

typedef struct kbl_ctx kbl_ctx;

/* Counters of the limiter since the last read (kbl_read_counters clears them). */
typedef struct {
    int32_t nonphysical;      /* a stencil state with rho <= 0 or P <= 0 was met */
    int32_t timeout;          /* a bounded device wait gave up: an mbarrier wait of the
                                 tensor-core residual (KBL_TUNE_RHS_TC) that ran out */
    int64_t limited_elements; /* element-stages with alpha_min < 1 (Eq. 39) */
    int64_t pressure_relimits;/* element-stages where the step of Eq. 48 was taken */
    int64_t eps_rule_activations; /* (element, component) pairs where the epsilon rule stated
                                 under Eq. 37 decided alpha_i (|min_V - mean| or
                                 |max_V - mean| below eps) */
    int64_t mean_outside_bounds;  /* (element, component) pairs whose element mean lay outside
                                 [w_min, w_max] (the case the absolute values of Eq. 37 cover) */
    int64_t alpha_hist[10];   /* limited element-stages by alpha_min: bin k counts
                                 k/10 <= alpha_min < (k+1)/10 (their sum is limited_elements) */
} kbl_counters;

/* Fill cfg with the paper's defaults for dimension d and order p: gamma 1.4,
 * k = 4, nu = 32 per axis in 2D and 64 in 1D, r_fac = 1e-3, eps = 1e-13,
 * floors 1e-12, eps_rule 0, FP64, coupled limiting, Rusanov flux, trapezoidal rule, the
 * stencil of Sec. 5. */
kbl_status kbl_config_default(kbl_config* cfg, int dim, int p);

/* Create a context bound to `cuda_stream` (a cudaStream_t, NULL = legacy
 * default stream).  Synchronous.  *out is NULL on failure. */
kbl_status kbl_create(kbl_ctx** out, const kbl_config* cfg, void* cuda_stream);
/* Free the context and everything it allocated (mesh copy, scratch, adjoint
 * storage).  KBL_EINVAL for NULL.  The caller's arrays are untouched. */
kbl_status kbl_destroy(kbl_ctx* ctx);
/* Bind later launches (the step graph's included) to another stream. */
kbl_status kbl_set_stream(kbl_ctx* ctx, void* cuda_stream);
/* Message of the context's last failure (owned by the context; valid until the
 * next call on it); "null context" for NULL. */
const char* kbl_last_error(const kbl_ctx* ctx);
/* Layout sizes: conserved variables nv = d + 2, solution points Ns = (p+1)^d,
 * face points Nfp (2 in 1D, 4 (p+1) in 2D), stencil states Ns + 2 Nfp (Sec. 5);
 * -1 for NULL. */
int kbl_nv(const kbl_ctx* ctx);
int kbl_ns(const kbl_ctx* ctx);
int kbl_nfp(const kbl_ctx* ctx);
int kbl_nstencil(const kbl_ctx* ctx);

/* Upload a mesh (HOST arrays, copied; synchronous) and size the scratch
 * space: nbr[E][2d], h[E][d] element widths (> 0), bc[n_bc][nv] boundary
 * states.  Every negative nbr must name a valid boundary id.  n_elem may be 0. */
kbl_status kbl_mesh_upload(kbl_ctx* ctx, int n_elem, const int32_t* nbr_host,
                           const double* h_host, int n_bc, const double* bc_host);

/* Copy one of the library's FR operators to a HOST buffer of n doubles:
 * 0 nodes x[p+1], 1 weights[p+1], 2 l_i(-1)[p+1], 3 l_i(+1)[p+1],
 * 4 D[p+1][p+1] with D[i][m] = l_m'(x_i), 5 g_L'(x_i)[p+1], 6 g_R'(x_i)[p+1]. */
kbl_status kbl_get_operator(const kbl_ctx* ctx, int which, double* host_out, int n);

/* The 2D FR residual of Sec. 2.3 (g_DG correction, Sec. 5) as one matrix per order p: with
 * Ns = (p+1)^2 and K = 2 Ns + 4 (p+1), the residual of an element is R[v][n] = sum_k X[v][k]
 * B[k][n], X[v] = [(2/h_x) Fx_v at the Ns solution points, (2/h_y) Fy_v at them, (2/h_x) F*_v at
 * the 2(p+1) face points of faces 0 and 1, (2/h_y) F*_v at those of faces 2 and 3] (F* the common
 * flux, face-point order of this header).  The interpolated discontinuous flux is folded into the
 * derivative: B holds -(D[i][m] - g_L'(x_i) l_m(-1) - g_R'(x_i) l_m(+1)) along each axis and the
 * lifting -g_L', -g_R'.  The tensor-core residual (KBL_TUNE_RHS_TC) multiplies by it.  Host only,
 * no context, no device call: for checking.  host_out[K][Ns] row-major, n >= K Ns; KBL_EINVAL
 * for p outside 1..5 or a short buffer. */
kbl_status kbl_residual_operator(int p, double* host_out, int n);

/* The velocity quadrature weights the kernels apply on one axis of nu points, in
 * units of the grid spacing (Sec. 3.7, Sec. 5): quadrature 0 the trapezoidal rule,
 * 1 Romberg (see kbl_config.quadrature).  Host only, no context, no device call:
 * for checking.  host_out[nu]; KBL_EINVAL for nu < 2, an unknown rule or, with
 * Romberg, nu - 1 odd. */
kbl_status kbl_velocity_weights(int nu, int quadrature, double* host_out);

/* Interior values at the face points: wf = interpolation of w (Sec. 2.3). */
kbl_status kbl_traces(kbl_ctx* ctx, const double* w, double* wf);

/* Gather the stencil of elements e0 .. e0+n-1 into S[n][|S|][nv] (a plain
 * copy of values of w, wf and the boundary states: bit-exact). */
kbl_status kbl_gather_stencil(kbl_ctx* ctx, const double* w, const double* wf,
                              int e0, int n, double* S);

/* Kinetic bounds of every element (Sec. 3.3-3.8): Maxwellians of the stencil
 * states (Eq. 8), their pointwise envelopes (Eq. 32) relaxed by r_fac (Eq. 40)
 * with separate envelopes for the translational and internal-energy parts
 * (Eq. 44), trapezoidal sums on the per-element box of Eq. 45 (Eq. 33-36, 46),
 * then rho_min <- max(rho_min, rho_floor). */
kbl_status kbl_bounds(kbl_ctx* ctx, const double* w, const double* wf, double* bnd);

/* The same bounds for stencils the caller assembles (Eq. 29-46 take any set of
 * states): for element families whose traces live outside this library --
 * triangles with their own solution and face points, unstructured meshes.
 * S: DEVICE, conservative states S[n_elem][n_states][4] (element e's stencil is
 * S[e][0..n_states-1]); bnd: DEVICE, bnd[2][4][n_elem] as kbl_bounds writes it.
 * Uses the context's configuration (velocity grid, k, r_fac, floors, quadrature,
 * precision); needs no mesh.  2D only, 1 <= n_states <= 64, else KBL_EINVAL.
 * Asynchronous on the context's stream; a non-physical state gives NaN bounds
 * for its element and raises the non-physical flag. */
kbl_status kbl_bounds_stencil(kbl_ctx* ctx, int n_elem, int n_states, const double* S, double* bnd);

/* Limiting of node sets the caller assembles (Eq. 37-39, then Eq. 47-49), for element
 * families whose operators live outside this library.  Per element e: ns solution values
 * U[e][ns][nv] (DEVICE, limited in place) whose mean is sum W U / sum W with the positive
 * weights W[ns] (HOST, copied), nf face values F[e][nf][nv] (DEVICE, read only: they
 * enter the extremes over V and the pressure minimum; recompute them from the limited U,
 * which for an interpolation with weights summing to one equals limiting them), bounds
 * bnd[2][nv][n_elem] (DEVICE).  alpha (DEVICE, may be NULL) receives alpha_min and
 * alpha_P as alpha[2][n_elem].  Uses the context's eps, eps reading, coupled or uncoupled
 * form, gamma and p_floor; FP64 whatever the precision; needs no mesh.  1 <= ns <= 64,
 * 0 <= nf <= 64, else KBL_EINVAL.  Asynchronous; the limited and re-limited counts add to
 * the context's counters. */
kbl_status kbl_limit_nodes(kbl_ctx* ctx, int n_elem, int ns, int nf, const double* W, double* U,
                           const double* F, const double* bnd, double* alpha);

/* FR residual R = -div F with the configured interface flux (Rusanov,
 * assumption (iv) of Sec. 4, or HLLC) and the g_DG correction; wf must hold the
 * traces of w. */
kbl_status kbl_rhs(kbl_ctx* ctx, const double* w, const double* wf, double* R);

/* Limit w in place against bnd (Eq. 37-39, then Eq. 47-49); alpha may be NULL. */
kbl_status kbl_limit(kbl_ctx* ctx, double* w, const double* bnd, double* alpha);

/* One SSP-RK3 stage s in {0,1,2} (Shu-Osher form) fused with the limiter:
 * wout = limit(a_s wn + b_s (ws + dt R), bnd), dt read from the device scalar
 * dt_dev.  wout may alias wn.  alpha may be NULL. */
kbl_status kbl_stage(kbl_ctx* ctx, int s, const double* wn, const double* ws,
                     const double* R, const double* bnd, const double* dt_dev,
                     double* wout, double* alpha);

/* dt_dev (device scalar) = cfl * min over elements, solution points and axes
 * of h / (|U_axis| + c). */
kbl_status kbl_dt(kbl_ctx* ctx, const double* w, double cfl, double* dt_dev);

/* One full time step on device data: dt from w (clipped so the context's
 * time does not pass its end time), then three stages, each computing traces,
 * bounds and residual of its input and applying kbl_stage.  w is replaced by
 * the new solution.  Uses the context's scratch; launched as a CUDA graph
 * after the first call with a given w. */
kbl_status kbl_step(kbl_ctx* ctx, double* w, double cfl);

/* Time of the context (device scalars): set t and the end time (INFINITY for
 * none); kbl_time_sync reads t back (synchronous). */
kbl_status kbl_set_time(kbl_ctx* ctx, double t, double t_end);
kbl_status kbl_time_sync(kbl_ctx* ctx, double* t_host);

/* End-to-end run on HOST buffers: copy w_host_in to the device, take n_steps
 * steps of kbl_step, copy the result to w_host_out (may alias w_host_in).
 * Synchronous.  Device buffers are the context's own. */
kbl_status kbl_run_host(kbl_ctx* ctx, const double* w_host_in, double* w_host_out,
                        int n_steps, double cfl);

/* End-to-end runs of an ensemble of independent states on the context's mesh, from HOST
 * buffers (pinned for the copies to overlap): member k's state w_host_in + k * nv * E * Ns
 * takes n_steps steps of kbl_step, each member from the context's time at the call (with the
 * end-time clip of kbl_step), and lands in w_host_out + k * nv * E * Ns (the output may alias the
 * input).  Two device copies of the state alternate: member k+1's host-to-device copy and member
 * k-1's device-to-host copy run while member k steps (one cudaMemcpyAsync per member and
 * direction, on two copy streams of the context).  The first call allocates the second device
 * copy.  Afterwards the context's time is the last member's end time.  Synchronous. */
kbl_status kbl_run_host_ensemble(kbl_ctx* ctx, int n_members, const double* w_host_in, double* w_host_out,
                                 int n_steps, double cfl);

/* Wait for the context's stream and report device-side flags (then clear
 * them): KBL_ENONPHYSICAL if a non-physical state was met. */
kbl_status kbl_check(kbl_ctx* ctx);
/* The same wait, with the flags and the limiting counters copied to *out (HOST)
 * before they are cleared; returns what kbl_check would. */
kbl_status kbl_read_counters(kbl_ctx* ctx, kbl_counters* out);

/* Number of kernel launches the context has issued (graph launches count
 * the kernels inside them). */
int64_t kbl_launch_count(const kbl_ctx* ctx);

/* Launch-shape knobs (not part of the method; results do not depend on them
 * beyond FP32 rounding order).  KBL_TUNE_BOUNDS_TILE selects the FP32 2D
 * bounds thread tile for grids of 32 or 64 points per axis: 0 = 4 x 4 velocity
 * nodes per thread, 1 = 4 x 2, 2 = 2 x 4.  Setting a knob drops the captured
 * step graph. */
typedef enum { KBL_TUNE_BOUNDS_TILE = 0, KBL_TUNE_RHS_TC = 1, KBL_TUNE_RHS_OVERLAP = 2 } kbl_tune_key;
/* KBL_TUNE_RHS_TC: 1 runs the FP32-mixed 2D residual of orders 2 and 3 with its operator
 * product (operator 7 of kbl_get_operator) on the tensor cores (tcgen05, TF32 split into
 * hi + lo pairs, FP32 accumulation; element tiles staged by TMA), 0 on the CUDA cores.  Other
 * orders, 1D and FP64 always use the CUDA cores.  Default 0 (CUDA cores: measured faster on the
 * benchmark workloads).  Setting it drops the captured step graph. */
/* KBL_TUNE_RHS_OVERLAP: 1 (default) the step graph overlaps its kernels: the time step runs on a
 * branch of its own beside the traces, and the main chain (traces, then per stage residual,
 * bounds, stage + limiter) launches each kernel as a programmatic dependent of the one before,
 * so that its blocks start as the previous kernel's last blocks finish; the stage kernel forms
 * the stage combination and the bound-free part of its screen before the bounds kernel has
 * finished, and waits for it before it reads the bounds.  0: one ordinary launch after the
 * other.  The same arithmetic runs either way: results are identical.  Setting it drops the
 * captured step graph. */
kbl_status kbl_set_tuning(kbl_ctx* ctx, int key, int value);   /* KBL_EINVAL for an unknown key or value */
kbl_status kbl_get_tuning(const kbl_ctx* ctx, int key, int* value);

/* ---- Batched form -----------------------------------------------------------
 * Many independent 2D problems (axis-aligned quad meshes) with uneven element
 * counts and orders p = 1..4, advanced together: each phase of a step is ONE
 * persistent launch over all problems (blocks pull cost-sorted work items from a
 * device counter), or the whole step one launch (kbl_batch_set_form), captured
 * once as a CUDA graph.  Each
 * problem keeps its own time step.  Precision is KBL_FP32_MIXED.
 * Problem i's data are concatenated in problem order: nbr (E_i x 4, element
 * indices local to the problem, negative = local boundary id), h (E_i x 2),
 * bc (n_bc_i x 4).  Its state lives at state_offsets[i] (in doubles) of one
 * buffer, with the single-mesh layout w_i[4][E_i][(p_i+1)^2]. */
typedef struct kbl_batch kbl_batch;

/* cfg supplies dim (must be 2), nu (must be 32 x 32), gamma, k, r_fac, eps,
 * floors, the eps reading, the limiting form and the flux; cfg->p is ignored,
 * cfg->precision must be KBL_FP32_MIXED and cfg->quadrature 0 (KBL_EINVAL
 * otherwise).  HOST arrays, copied.  Synchronous; allocates the batch's device
 * memory. */
kbl_status kbl_batch_create(kbl_batch** out, const kbl_config* cfg, int n_problems,
                            const int32_t* p, const int32_t* n_elem, const int32_t* nbr,
                            const double* h, const int32_t* n_bc, const double* bc,
                            void* cuda_stream);
/* Free the batch and its device memory; KBL_EINVAL for NULL. */
kbl_status kbl_batch_destroy(kbl_batch* b);
/* Message of the batch's last failure (owned by the batch). */
const char* kbl_batch_last_error(const kbl_batch* b);
/* state_offsets[n_problems+1] (doubles) and elem_offsets[n_problems+1] (HOST). */
kbl_status kbl_batch_layout(const kbl_batch* b, int64_t* state_offsets, int64_t* elem_offsets);
/* FR nodes of order p (HOST, p+1 values), for building initial states. */
kbl_status kbl_batch_nodes(const kbl_batch* b, int p, double* host_out, int n);
/* One SSP-RK3 step of every problem, each with dt = cfl * its own CFL limit. */
kbl_status kbl_batch_step(kbl_batch* b, double* w, double cfl);
/* The phases of one batched stage as separate calls, running the persistent kernels of
 * kbl_batch_step: for checking a stage of every problem against kbl_traces + kbl_bounds,
 * kbl_rhs and kbl_stage on identical inputs.  All arrays DEVICE, in the concatenated
 * layout: w, ws, wn, R, wout like the state (problem i at state_offsets[i]); bnd with
 * problem i's bounds [2][4][E_i] at 8 * elem_offsets[i]; dt_dev[n_problems].
 * kbl_batch_bounds: face traces (batch scratch) then the kinetic bounds of Sec. 3.3-3.8.
 * kbl_batch_rhs: face traces then the FR residual of Sec. 2.3 with the configured flux.
 * kbl_batch_stage: wout = limit(a_s wn + b_s (ws + dt R), bnd) (Sec. 5 SSP-RK3, Eq. 37-39,
 * Eq. 47-49) for stage st in {0,1,2}; wout may alias wn.  Asynchronous on the batch's
 * stream; KBL_EINVAL for a null array or a bad stage. */
kbl_status kbl_batch_bounds(kbl_batch* b, const double* w, double* bnd);
kbl_status kbl_batch_rhs(kbl_batch* b, const double* w, double* R);
kbl_status kbl_batch_stage(kbl_batch* b, int st, const double* wn, const double* ws, const double* R,
                           const double* bnd, const double* dt_dev, double* wout);
/* End-to-end run on HOST buffers (pinned for the copies to overlap): the batch state
 * w_host_in (concatenated layout) is copied to the batch's own device copy, every problem takes
 * n_steps steps of kbl_batch_step, and the result is copied to w_host_out (may alias
 * w_host_in).  The problems are cut into up to 8 groups of consecutive problems of similar state
 * size, each with its own work items and step graph: group g's host-to-device copy, group
 * g-1's steps and group g-2's device-to-host copy run at the same time on three streams (one
 * cudaMemcpyAsync per group and direction).  The first call allocates the device copy (one state)
 * and the groups.  Synchronous; the batch's scratch, per-problem time steps and clocks are those
 * of kbl_batch_step. */
kbl_status kbl_batch_run_host(kbl_batch* b, const double* w_host_in, double* w_host_out, int n_steps, double cfl);
/* Device time of the bounds launch of the last kbl_batch_bounds call (CUDA events on the batch's
 * stream around that launch alone; synchronous): for measuring the dominant phase in the
 * launch shape the step graph uses.  KBL_ESTATE before any kbl_batch_bounds call. */
kbl_status kbl_batch_bounds_ms(kbl_batch* b, double* ms);
/* Form of kbl_batch_step: 1 ONE persistent launch for the whole step, whose blocks pull the
 * work items of all 13 phases (time step; per stage traces, bounds, residual, stage + limiter)
 * in phase order and wait, per problem, only for the earlier phases that problem's item depends
 * on (bounded waits: a wait that runs out raises the timeout flag, which kbl_batch_check
 * reports as KBL_ETIMEOUT, and ends the launch); 0 (default) one persistent launch per phase
 * (14 launches), each in the launch shape the autotuner picks for its phase -- measured about
 * 6% faster on the batched benchmark workload, as the one-launch kernel is compiled for the
 * register budget of its most demanding phase.  Both run the same device code per element:
 * results are identical.  Drops the captured graphs.  KBL_EINVAL for other values. */
kbl_status kbl_batch_set_form(kbl_batch* b, int fused);
/* For testing the timeout path of the fused form without a fault: with on != 0 the first bounds
 * item of the next steps waits for a completion count that no item reaches, so that wait runs
 * out after wait_polls polls of about a microsecond (a second by default) and the step ends
 * with KBL_ETIMEOUT (its state is then undefined); on = 0 restores normal steps.  wait_polls
 * also bounds every other wait of the fused form.  Drops the captured graphs. */
kbl_status kbl_batch_stall_test(kbl_batch* b, int on, int wait_polls);
/* Per-problem time step of the last step (HOST, n_problems values; synchronous). */
kbl_status kbl_batch_dt(kbl_batch* b, double* dt_host);
/* Time the bounds phase on state w for every combination of thread tile
 * (velocity nodes per thread: 4x4, 4x2, 2x4; the fused form takes the 128-thread 4x2 and 2x4),
 * elements per work item and resident blocks per SM, on a fixed sample of the work items
 * (every eighth), and keep the fastest.  Synchronous.  out_ms (may be NULL) receives the best time of
 * the sample, out_cmp (may be NULL) the envelope comparisons the sample needs
 * (4 |S| N_u per element). */
kbl_status kbl_batch_autotune(kbl_batch* b, const double* w, double* out_ms, double* out_cmp);
/* Current launch shape: [tile, elements per item, blocks per SM, items]. */
kbl_status kbl_batch_tuning(const kbl_batch* b, int32_t* out4);
/* Wait for the batch's stream and report (then clear) its device flags, as kbl_check. */
kbl_status kbl_batch_check(kbl_batch* b);
/* Kernel launches the batch has issued (graph launches count their kernels). */
int64_t kbl_batch_launch_count(const kbl_batch* b);

/* ---- Reverse mode (adjoint) --------------------------------------------------
 * Hand-written vector-Jacobian products of the 2D path (FP64, any precision of
 * the context for the *_vjp calls; the step adjoints need a KBL_FP64 context).
 * Each *_vjp call takes the forward inputs and the cotangent of the forward
 * output and ADDS the cotangents of the inputs into caller-owned device arrays
 * (exceptions are stated).  Where the method takes a min or a max (the envelopes
 * of Eq. 32, the box of Eq. 45, the extrema over V and P_min of Eq. 47, the
 * Davis wavespeed of the Rusanov flux) the first element of the set in its
 * natural order wins ties and receives the whole cotangent (stencil order of
 * this header; V order = solution points then face points; components in
 * order).  In Eq. 37 the 1 wins ties over the upper ratio, which wins over the
 * lower one; in Eq. 39 the lowest component wins.  The epsilon rule under
 * Eq. 37, the density floor of Sec. 3.8 (ties included), alpha_P = 0 and the
 * sign split of the momentum sums (Eq. 35-36) contribute no derivative.
 *
 * Trace cotangents come in two arrays of the traces' layout: wfb[v][e][fp]
 * for the use of e's own trace, wfb_ext[v][e][fp] for its use as the exterior
 * value of the neighbour across that face.  The cotangent of wf is their sum;
 * boundary states get none. */

/* wb += cotangent of w through wf = traces(w): transposed interpolation of
 * wfb (+ wfb_ext, which may be NULL). */
kbl_status kbl_traces_vjp(kbl_ctx* ctx, const double* wfb, const double* wfb_ext, double* wb);

/* Residual R = rhs(w, wf) of kbl_rhs: given Rb, wb += (dR/dw)^T Rb,
 * wfb / wfb_ext += (dR/dwf)^T Rb.  Ties of the Rusanov wavespeed (s_L = s_R)
 * take the minus-side state; |u| at u = 0 takes the + branch. */
kbl_status kbl_rhs_vjp(kbl_ctx* ctx, const double* w, const double* wf, const double* Rb,
                       double* wb, double* wfb, double* wfb_ext);

/* Bounds bnd = bounds(w, wf) of kbl_bounds (FP64 arithmetic whatever the
 * context's precision): given bndb[2][nv][E], adds the cotangents of the
 * stencil states.  bnd must hold the forward result (it decides the density
 * floor).  Elements with a non-physical stencil raise the flag and add
 * nothing. */
kbl_status kbl_bounds_vjp(kbl_ctx* ctx, const double* w, const double* wf, const double* bnd,
                          const double* bndb, double* wb, double* wfb, double* wfb_ext);

/* Stage s of kbl_stage with dt given on the host: out = limit(a_s wn + b_s (ws
 * + dt R), bnd).  Given ob (cotangent of out): wnb = a_s g (or wnb += a_s g when
 * accumulate_wn != 0), wsb = b_s g, Rb = b_s dt g, where g is the cotangent of
 * the combined state; bndb[2][nv][E] = cotangent of bnd.  wsb, Rb, bndb are
 * overwritten; ob must not alias any output.  dt itself is held fixed. */
kbl_status kbl_stage_vjp(kbl_ctx* ctx, int s, double dt, const double* wn, const double* ws,
                         const double* R, const double* bnd, const double* ob, int accumulate_wn,
                         double* wnb, double* wsb, double* Rb, double* bndb);

/* Integrated entropy of w: J = sum_e |J_e| sum_n W_n rho ln(P rho^-gamma), the
 * density-weighted log of the physical entropy s = P rho^-gamma of Sec. 6, with the
 * Gauss-Legendre weights; written to the device scalar J_dev (fixed summation
 * order: deterministic).  kbl_entropy_vjp: wb = Jb dJ/dw (overwritten). */
kbl_status kbl_entropy(kbl_ctx* ctx, const double* w, double* J_dev);
kbl_status kbl_entropy_vjp(kbl_ctx* ctx, const double* w, double Jb, double* wb);

/* One time step with a given dt (no CFL rule, no end-time clip; the context's
 * time is not advanced): the three stages of kbl_step. */
kbl_status kbl_step_fixed(kbl_ctx* ctx, double* w, double dt);

/* n steps of kbl_step_fixed in place (dts: host array of n).  With bnd_out
 * (device, [n][3][2][nv][E]) the bounds of every stage are kept there, for
 * kbl_adjoint_segment to reuse; may be NULL. */
kbl_status kbl_forward_segment(kbl_ctx* ctx, double* w, const double* dts, int n, double* bnd_out);

/* Reverse of kbl_step_fixed(w, dt): on entry wbar is the cotangent of the
 * step's output, on exit the cotangent of w (w itself is not changed).  Same as
 * kbl_adjoint_segment with n = 1. */
kbl_status kbl_adjoint_step(kbl_ctx* ctx, const double* w, double dt, double* wbar);

/* Reverse of n fixed-dt steps from w0 (dts: host array of n).  A forward pass
 * over the segment keeps, for every step, its input, its stage inputs and each
 * stage's traces, bounds and residual; the reverse pass then runs the stage,
 * residual, bounds and trace VJPs backwards through all 3n stages without
 * recomputing anything.  bnd_in: the stage bounds kept by kbl_forward_segment
 * over the same steps from the same w0 ([n][3][2][nv][E], device), which the
 * forward pass then takes instead of recomputing them (the bounds are the
 * costly part of a stage); NULL to recompute.  wbar: cotangent of the final
 * state in, of w0 out.  Scratch (context-owned, grown on first use): (6 n + 4)
 * solution-sized arrays, (3 n + 2) trace-sized and (3 n + 1) bound-sized ones.
 * The unit of checkpointed reverse mode: a caller that keeps every K-th state of
 * a long run calls this once per segment of K steps. */
kbl_status kbl_adjoint_segment(kbl_ctx* ctx, const double* w0, const double* dts, int n,
                               const double* bnd_in, double* wbar);

/* Element bounds without any device allocation.  The paper has no
 * counterpart to this call; it exists for callers that cannot call
 * cudaMalloc: applications that hand all device memory to their own pool at
 * start-up and forbid side allocations, and time-critical loops that cannot
 * afford the implicit device synchronisation of cudaMalloc / cudaFree.  A
 * context (kbl_create, kbl_mesh_upload) allocates, so this call takes no
 * context: the caller passes the configuration (host struct) and every array
 * on the device -- nbr_dev[E][2d] (int32, the layout of kbl_mesh_upload, which
 * this call does not validate: out-of-range entries are undefined behaviour),
 * bc_dev[n_bc][nv], the solution w_dev[nv][E][Ns] and the output
 * bnd_dev[2][nv][E] -- and the stream.  The result equals kbl_traces followed by
 * kbl_bounds of a context with the same configuration and mesh (the same
 * kernels run).  The face traces needed as scratch live in one file-scope
 * device array of 2^20 doubles (8 MiB) that every GPU loading the library
 * keeps until the process exits, so n_elem * (d+2) * Nfp must not exceed
 * 1048576 (16384 two-dimensional P3 elements); larger meshes, like bad
 * configurations, return KBL_EINVAL before anything is launched.  The
 * trapezoidal rule only (quadrature 0): a weight table would need an
 * allocation.  No
 * cudaMalloc, cudaFree or other allocating routine is called.  Asynchronous;
 * a non-physical stencil state gives NaN bounds for its element.  The first
 * call on each device looks up the device address of the scratch array
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  All calls share the one scratch array, which
 * keeps the last call's contents: calls that overlap on the GPU (different
 * streams, or host threads on the same device) race on it and must be
 * serialised by the caller. */
kbl_status kbl_bounds_noalloc(const kbl_config* cfg, int n_elem, const int32_t* nbr_dev,
                              int n_bc, const double* bc_dev, const double* w_dev,
                              double* bnd_dev, void* cuda_stream);

/* ---- triangles (Sec. 5) ----------------------------------------------------
 * Affine triangles with the Williams-Shunn solution points of order p in {1, 2}
 * (3 and 6 points: the interior symmetric rules of degree 2 and 4, which are
 * also the mean weights of the limiter) and p + 1 Gauss-Legendre flux points per
 * edge; the residual is flux reconstruction with the DG correction (a strong-form
 * nodal DG residual with the exact diagonal mass matrix), and a step is SSP-RK3
 * with the kinetic bounds of every element's stencil (its solution points, its
 * flux points and their exterior values, Sec. 5) and the node-set limiter after
 * every stage.  KBL_FP64: everything in FP64; KBL_FP32_MIXED: the bounds and the
 * residual as in that mode for quads (FP32 arithmetic on FP64 storage), the
 * traces, the state and the limiter FP64.
 * Reference triangle (0,0), (1,0), (0,1); edge f runs from vertex f to vertex
 * (f + 1) % 3, its flux points in that direction; the element across the edge
 * runs it the other way.  All arrays are element-major: solution
 * w[E][ns][4] (ns = (p+1)(p+2)/2), traces wf[E][nfp][4] (nfp = 3 (p+1), edge by
 * edge), stencils S[E][ns + 2 nfp][4] (solution points, flux points, exterior
 * values).  Device arrays unless marked HOST; calls are asynchronous on the
 * stream given at creation unless stated. */
typedef struct kbl_tri kbl_tri;

/* Solution points rs[ns][2] and weights w[ns] (HOST, sum 1/2) of order p on the
 * reference triangle; KBL_EINVAL for p outside {1, 2}. */
kbl_status kbl_tri_points(int p, double* rs, double* w);

/* A triangle mesh: xy[E][3][2] (HOST) vertices counterclockwise; nbr[E][3] (HOST)
 * the element across edge f, or -(b+1) for boundary state b; nbr_edge[E][3]
 * (HOST) that element's edge matched to f; bc[n_bc][4] (HOST) boundary states.
 * cfg: dim 2, p in {1, 2}, gamma, flux, bounds and limiter settings as for
 * kbl_create.  Copies everything; allocates a context for the bounds and the
 * limiter and the step's scratch ((12 ns + 4 nfp + 8) E doubles).
 * KBL_EINVAL for a bad configuration, an out-of-range neighbour or a clockwise or
 * degenerate element; KBL_ENOMEM / KBL_ECUDA on allocation failure. */
kbl_status kbl_tri_create(kbl_tri** out, const kbl_config* cfg, int n_elem, const double* xy,
                          const int32_t* nbr, const int32_t* nbr_edge, int n_bc, const double* bc,
                          void* cuda_stream);
/* Curved (quadratic) triangles, as the paper's triangle run uses: xy6[E][6][2] (HOST), the three
 * corners counterclockwise, then the points of edges 0, 1, 2 at mid-parameter; the element is the
 * image of the reference triangle under the quadratic Lagrange map of these six points.  The
 * residual takes the transformed-flux form: with adj J = |J| J^-1 at each solution point and the
 * edge's stretch sigma = |dx/dt| / |dxi/dt| and physical unit normal at each flux point,
 *   R_i = -(1/|J_i|) [ sum_j (Dr_ij (adj J F)_r,j + Ds_ij (adj J F)_s,j)
 *                      + sum_q phi_i(x_q) gw_q L_f / (2 w_i) (sigma_q F*_n,q - ((adj J F)_h . nh)(x_q)) ],
 * the solution points carrying the lumped mass w_i |J_i|, which the limiter's mean then uses;
 * h of the time step comes from the corners.  Neighbours must share their edges' three points.
 * Otherwise as kbl_tri_create; KBL_EINVAL also for a map that folds (|J| <= 0 at a solution
 * point). */
kbl_status kbl_tri_create_curved(kbl_tri** out, const kbl_config* cfg, int n_elem, const double* xy6,
                                 const int32_t* nbr, const int32_t* nbr_edge, int n_bc, const double* bc,
                                 void* cuda_stream);
kbl_status kbl_tri_destroy(kbl_tri* t);
const char* kbl_tri_last_error(const kbl_tri* t);

/* Interior values at the flux points: wf = interpolation of w (Eq. 2 on triangles). */
kbl_status kbl_tri_traces(kbl_tri* t, const double* w, double* wf);

/* Stencils of Sec. 5 for every element, from w and its traces wf. */
kbl_status kbl_tri_gather_stencil(kbl_tri* t, const double* w, const double* wf, double* S);

/* Kinetic bounds bnd[2][4][E] (the layout of kbl_bounds) of every element's stencil, gathered
 * inside the bounds kernel from w and its traces wf: equal bit for bit to
 * kbl_tri_gather_stencil followed by kbl_bounds_stencil with the mesh's configuration, without
 * the stencil array.  The bounds of kbl_tri_step. */
kbl_status kbl_tri_bounds(kbl_tri* t, const double* w, const double* wf, double* bnd);

/* Residual R[E][ns][4] = -div F_h - sum_q lift (F*_n - F_h . n): the
 * interpolated flux's divergence and the DG lifting of the flux-point jumps, with
 * the configured common flux of the states rotated into each edge's normal frame.
 * FP64, or FP32 arithmetic on FP64 storage in KBL_FP32_MIXED. */
kbl_status kbl_tri_residual(kbl_tri* t, const double* w, const double* wf, double* R);

/* Time step (synchronous): cfl * min over elements and solution points of
 * h / (|U| + c), h = 2 area / longest edge; *dt_host = 0 for an empty mesh. */
kbl_status kbl_tri_dt(kbl_tri* t, const double* w, double cfl, double* dt_host);

/* One SSP-RK3 step of w (in place) with the given dt: per stage the kinetic
 * bounds of the stencils of the stage input (kbl_tri_bounds), the residual (on a
 * second stream, beside the bounds), the Shu-Osher combination, the traces of
 * the combined state and the node-set limiter (kbl_limit_nodes with the solution
 * points' weights), whose limited face values are the next stage's traces.
 * Non-physical states raise the flag kbl_tri_check reports. */
kbl_status kbl_tri_step(kbl_tri* t, double* w, double dt);

/* Wait for the stream and report (then clear) the device flags, as kbl_check. */
kbl_status kbl_tri_check(kbl_tri* t);

#ifdef __cplusplus
}
#endif
#endif
