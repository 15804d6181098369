/*
 * st.h -- C ABI of the GB300 space-time sparse-grid wave solver.
 *
 * The library solves the linear wave equation of Eq. (1),
 *     d_t^2 u - div(c^2 grad u) = f in Omega x (0,T),  u = 0 on dOmega,
 *     u(.,0) = u0, d_t u(.,0) = v0,
 * on a box Omega in R^d (d = 1, 2, 3) with the conforming space-time Galerkin
 * method of Section 2.2 (Eq. (9)): Q1 finite elements in space, C^1 quadratic
 * splines in time with w(0) = 0, the exponentially weighted form of Eq. (6);
 * and combines the anisotropic full-grid solutions with the +-1 coefficients of
 * the combination formula, Eq. (19).
 *
 * Levels: level j means 2^j uniform cells per direction on the box (space) or
 * 2^j uniform intervals on (0,T) (time).  The component set of Eq. (19) is
 *   (mx + a, mt + J - a, +1), a = 0..J,   (mx + a - 1, mt + J - a, -1), a = 1..J,
 * ordered as listed (all +1 terms by increasing spatial level, then all -1 terms).
 *
 * Data discretisation (the same reading as the reference oracle): c^2 is
 * sampled at cell centres and held constant per cell; u0, v0 and the spatial
 * factors of f are replaced by their Q1 nodal interpolants at each
 * component's spatial level; time integrals use 8-point Gauss-Legendre per
 * time interval.
 *
 * Memory: the handle owns every device buffer it uses.  Callbacks are called
 * only inside st_setup and their data is copied.  Output buffers passed to
 * st_combine / st_component_coeffs are owned by the caller.  All GPU work is
 * enqueued on the stream given in st_options (0 = legacy default stream).
 * A handle is not thread safe; use one handle per host thread and stream.
 *
 * Errors: every call returns an st_status; st_last_error(h) returns a static
 * or handle-owned message for the last failure on that handle (or on handle
 * creation when h is NULL).  No call aborts the process.
 */
#ifndef ST_H_
#define ST_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  ST_OK = 0,
  ST_ERR_ARG = 1,            /* invalid argument or unsupported size */
  ST_ERR_CUDA = 2,           /* a CUDA runtime call failed */
  ST_ERR_OOM = 3,            /* device allocation failed */
  ST_ERR_NOT_CONVERGED = 4,  /* an iterative solve hit its iteration limit */
  ST_ERR_STATE = 5,          /* call out of order (e.g. combine before solve) */
  ST_ERR_CALLBACK = 6,       /* a user callback returned non-zero */
  ST_ERR_NUMERIC = 7,        /* NaN/Inf or a breakdown in a factorisation */
  ST_ERR_TIMEOUT = 8         /* a bounded wait inside a kernel gave up */
} st_status;

typedef enum { ST_FP64 = 0, ST_FP32_IR = 1 } st_precision;

/* Vectorised data callbacks.  pts is n x d, point-major (x0 y0 z0 x1 y1 ...).
 * They write n values to out and return 0 on success. */
typedef int (*st_space_fn)(int64_t n, const double* pts, double* out, void* user);
typedef int (*st_time_fn)(int64_t n, const double* t, double* out, void* user);
typedef int (*st_spacetime_fn)(int64_t n, const double* pts, double t, double* out, void* user);

typedef struct {
  st_space_fn fn;  /* NULL = the zero function */
  void* user;
} st_field;

/* One separable source term g(x) s(t) of f. */
typedef struct {
  st_space_fn g;
  void* g_user;
  st_time_fn s;
  void* s_user;
} st_source_term;

/* The problem of Eq. (1) with the combination levels of Eq. (19). */
typedef struct {
  int d;                    /* space dimension, 1..3 */
  double lo[3], hi[3];      /* box Omega = prod (lo_k, hi_k) */
  double T;                 /* final time, > 0 */
  st_field c2;              /* c^2(x) > 0, sampled at cell centres (required) */
  int n_terms;              /* number of separable source terms */
  const st_source_term* terms;
  st_spacetime_fn f_general; /* optional non-separable part f(x,t); NULL = 0 */
  void* f_user;
  st_field u0, v0;          /* initial displacement and velocity (NULL = 0) */
  int J;                    /* combination level J >= 0 */
  int mx, mt;               /* coarsest spatial / temporal levels */
  /* Optional nodal parametrisation (the parameters of st_misfit_gradient):
   * c2_nodal, if not NULL, holds (2^param_level+1)^d values of c^2 at the
   * nodes of the uniform grid of level param_level of the box (boundary
   * included, x fastest), and c^2(x) is their multilinear interpolant (the c2
   * callback is then not used); g_nodal likewise replaces the spatial factor g
   * of the first source term (n_terms >= 1).  The values are copied during
   * st_setup.  The gradient's transposed map uses the same interpolation. */
  const double* c2_nodal;
  const double* g_nodal;
  int param_level;          /* 0..12; used only with c2_nodal or g_nodal */
} st_problem;

typedef struct {
  int precision;    /* st_precision */
  double tol;       /* target normwise backward error of each component,
                       ||F - S U|| / (||S|| ||U|| + ||F||) (0 = default 1e-14) */
  int max_iter;     /* inner Krylov iteration limit per mode (0 = default) */
  int max_sweeps;   /* refinement sweeps per component (0 = default) */
  void* stream;     /* cudaStream_t */
  double inner_tol; /* relative residual at which a mode's inner Krylov solve
                       stops within one refinement sweep (0 = default: 1e-12
                       for FP64 inner solves, 1e-4 for FP32) */
  int max_direct_rows;  /* spatial grids with at most this many unknowns
                           (and a band of at most 1024) are solved by the
                           banded direct method, larger ones by multigrid-
                           preconditioned COCG (0 = default 32768) */
  int autotune;         /* stencil launch shapes (time modes per thread, CTA
                           size) timed per grid size and mode count at setup,
                           before the COCG graphs are captured, and kept for the
                           process: 0 or 1 = on (default), -1 = the built-in rule */
  int64_t mem_cap_bytes; /* device memory this handle may allocate in total
                            (0 = no cap); an allocation beyond it fails with
                            ST_ERR_OOM, as a real allocation failure would */
  int64_t wait_cycles;  /* cycle budget of each bounded copy wait in the
                           single-warp banded solves (grids with a half
                           bandwidth above 128 that are not power-of-two
                           bands): 0 = 2^31, about one second; a wait that runs
                           out makes the solve return ST_ERR_TIMEOUT */
  int inject_stall;     /* fault injection for failure tests: 1 = the first
                           factor-row copy of every single-warp banded solve is
                           never issued, so its bounded wait runs out after
                           wait_cycles and the solve returns ST_ERR_TIMEOUT;
                           0 = off (default) */
  int device_loop;      /* 0 = host-driven solves (default): the refinement
                           sweeps and, for multigrid components, graph launches
                           of 4 COCG iterations with a host check of
                           convergence after each; k = 4, 8 or 16 = every
                           forward solve is one CUDA graph launch: the sweeps
                           run in a conditional WHILE node whose stopping test
                           (the backward error, the sweep limit, status words)
                           is taken on the device, and each sweep's COCG loop
                           in a nested WHILE node of k iterations per test.
                           st_solve_component, st_solve_batch and
                           st_solve_combine then enqueue every component from
                           the calling thread and synchronise once per call to
                           read the solves' records (st_solve_combine: before
                           its last combination levels end) */
} st_options;

typedef struct {
  int jx, jt, coef;         /* levels and combination coefficient */
  int64_t n_space, n_time;  /* dim V_jx, dim V_jt */
  int method;               /* 0 = time eigenbasis, 1 = space eigenbasis */
  int n_modes;              /* spatial problems solved per sweep */
} st_component_info;

typedef struct {
  int sweeps;               /* refinement sweeps taken */
  int max_inner_iters;      /* largest inner Krylov count over modes and sweeps */
  double rel_residual;      /* final ||F - S U|| / ||F|| (FP64, 2-norms) */
  double backward_error;    /* final ||F - S U|| / (||S|| ||U|| + ||F||), ||S|| bounded above */
  int status;               /* st_status of this component */
} st_solve_info;

typedef struct st_handle st_handle;

/* Build everything that depends only on the problem (levels, c^2, data):
 * time matrices and their FP64 eigenbasis, spatial level hierarchy, sampled
 * data, factorisations of the coarsest multigrid operators.  Reads the
 * problem and its callbacks; copies what it needs. */
st_status st_setup(const st_problem* problem, const st_options* options, st_handle** out);

/* Number of components (2J+1) and their description, in component order. */
st_status st_num_components(const st_handle* h, int* n);
st_status st_component(const st_handle* h, int k, st_component_info* info);

/* Solve component k (0 <= k < n), or all components when k == -1, Eq. (9).
 * Asynchronous on the handle's stream unless info != NULL, in which case it
 * synchronises and fills info (for k == -1, the worst component). */
st_status st_solve_component(st_handle* h, int k, st_solve_info* info);

/* Solve every component of n independent handles (instances) together: the
 * (handle, component) pairs, largest first, are taken by a pool of at most
 * max_threads host threads (0 = 32), each component on its own stream, so
 * components of different instances overlap on the GPU.  Each handle's
 * stream waits for its components.  info (nullable): the worst component
 * over all handles; with info the call synchronises every handle's stream.
 * A handle listed twice is refused (ST_ERR_ARG). */
st_status st_solve_batch(st_handle* const* hs, int n, int max_threads, st_solve_info* info);

/* Evaluate u^CF of Eq. (19) on the nodal target grid of spatial level jx_star
 * and temporal level jt_star: (2^jx*+1)^d nodes (boundary included,
 * lexicographic, x fastest) times 2^jt*+1 uniform times of [0,T] (time
 * slowest).  out_dev: caller-owned device array of that many doubles.
 * Requires every component to be solved (ST_ERR_STATE otherwise). */
st_status st_combine(st_handle* h, int jx_star, int jt_star, double* out_dev);

/* st_solve_component(h, -1) followed by st_combine(h, jx*, jt*, out_dev), with
 * the combination overlapped with the solves: each level of the hierarchical
 * combination is enqueued on the handle's stream as soon as the components it
 * adds have finished, so the coarse levels run while the largest components
 * are still being solved.  Same result, layout and errors as the two calls;
 * info (nullable) as for st_solve_component (the call then synchronises). */
st_status st_solve_combine(st_handle* h, int jx_star, int jt_star, double* out_dev, st_solve_info* info);

/* The part of the sum of Eq. (19) contributed by the listed components
 * comps[0..ncomp-1] (distinct indices, each solved), on the same target grid
 * and layout as st_combine.  Eq. (19) is linear in the components, so the
 * parts of disjoint sets that cover all components add up to st_combine's
 * result: the combination step of a run that shards components over GPUs
 * (each rank combines its own, then one sum-reduction of the target array).
 * Handles with more than 64 components are refused (ST_ERR_ARG); so are
 * repeated or out-of-range indices; an unsolved listed component gives
 * ST_ERR_STATE.  Partial-sum buffers are cached per (target, set). */
st_status st_combine_subset(st_handle* h, int jx_star, int jt_star, const int* comps, int ncomp, double* out_dev);

/* ---------------------------------------------------------------------
 * Receiver misfit and its gradient (adjoint of Eq. (9); an extension: the
 * paper states the forward problem only).
 *
 * Receivers: x_rec (host, n_rec x d, inside the closed domain).  Target
 * times: t_s = s T / 2^jt* (s = 0 .. 2^jt*).
 *
 * st_receiver_values: out_dev (device, (2^jt*+1) x n_rec, time slowest) =
 * u^CF(x_r, t_s) of Eq. (19), evaluated from the components directly (the
 * same values as st_combine's target grid interpolated multilinearly).
 * Requires every component solved (ST_ERR_STATE).
 *
 * st_misfit_gradient: J = 1/2 sum_s w_s sum_r (u^CF(x_r, t_s) - d[s][r])^2
 * with trapezoid weights w_s on [0, T] and observations d_obs_dev (device,
 * same layout as out_dev above); its gradient with respect to
 *   - the nodal values of c^2 (st_problem.c2_nodal, required: ST_ERR_STATE
 *     otherwise) on the uniform grid of level jp = st_problem.param_level
 *     (ST_ERR_ARG for another jp), sampled at cell centres by multilinear
 *     interpolation, into dc2_dev (device, (2^jp+1)^d doubles);
 *   - the nodal values of the spatial factor g of the first separable source
 *     term (st_problem.g_nodal, required when there is a source term),
 *     interpolated multilinearly to the nodes of every component level, into
 *     dg_dev (zero if there is no source term).
 * For each component k it solves the adjoint system S_k^T L_k = G_k
 * (G_k = coef_k E_k^T (w * misfit), E_k the evaluation at the receivers) with
 * the forward machinery (transposed time factors, same spatial modes, the
 * same precision and refinement as the handle), then reduces
 * dJ/dc2_e = -L_k^T (B (x) K_e) U_k per cell and dJ/dg = M_load^T sum_i b[i] L_k[i]
 * onto the parameter grid, by the transpose of the same interpolation that
 * st_setup used to sample the nodal fields.  u0 must be zero (ST_ERR_ARG
 * otherwise).  J_out is written on the
 * host; info (nullable) reports the adjoint solves like st_solve_component.
 * Synchronises the handle's stream before returning. */
st_status st_receiver_values(st_handle* h, int jt_star, const double* x_rec, int n_rec, double* out_dev);
st_status st_misfit_gradient(st_handle* h, int jt_star, const double* x_rec, int n_rec, const double* d_obs_dev,
                             int jp, double* J_out, double* dc2_dev, double* dg_dev, st_solve_info* info);

/* Energy of the combined solution, Section 6.3:
 *   E(t_i; u^CF) = 1/2 ( ||d_t u^CF(., t_i)||^2_{L^2} + ||c grad u^CF(., t_i)||^2_{L^2} )
 * at the ntimes times t_i in [0, T] (host array), written to energy_out (host,
 * ntimes doubles).  u^CF and d_t u^CF are formed on all nodes of the uniform
 * grid of spatial level jx_eval (0 = the finest component level, the only
 * other value accepted), where the combined solution is Q1 in space, and the
 * integrals are taken exactly per cell with c^2 cellwise at that level's cell
 * centres.  Requires every component solved (ST_ERR_STATE); ST_ERR_ARG for
 * times outside [0, T] or another jx_eval; device memory for the levels and
 * tables is taken with cudaMallocAsync on the handle's stream (ST_ERR_OOM if
 * that fails).  Synchronises the handle's stream. */
st_status st_energy(st_handle* h, const double* times, int ntimes, int jx_eval, double* energy_out);

/* Copy the FP64 coefficient array U_k (n_time x n_space, time-major) of a
 * solved component to caller-owned host memory. */
st_status st_component_coeffs(st_handle* h, int k, double* host_out);

/* Total space-time degrees of freedom of all components (N^sparse_DoFs). */
st_status st_total_dofs(const st_handle* h, int64_t* dofs);

/* Bytes this handle has copied host->device and device->host since creation
 * (setup uploads, convergence flags and norms read back, component copies). */
st_status st_transfer_bytes(const st_handle* h, int64_t* h2d, int64_t* d2h);

/* Number of kernels this handle has launched since creation. */
st_status st_kernel_launches(const st_handle* h, int64_t* count);

/* Per-kernel-class timing.  st_profile(h, 1) clears the record and starts
 * recording a CUDA event pair on the handle's stream around every kernel
 * launch (extra launch overhead: use it for a separate measurement pass);
 * st_profile(h, 0) stops.  st_profile_read synchronises and writes one
 * entry per kernel class and grid size seen since the last st_profile call,
 * named "<class>@<unknowns of the grid>" (at most max_out; *n_out receives
 * the count): launches, summed event time, and the algorithmic bytes and
 * flops of those launches. */
typedef struct {
  char name[32];
  int64_t launches;
  double ms;
  double bytes;
  double flops;
} st_kernel_stat;
st_status st_profile(st_handle* h, int enable);
st_status st_profile_read(st_handle* h, st_kernel_stat* out, int max_out, int* n_out);

/* Launch shapes chosen by the stencil autotuner so far in this process:
 * 7 ints per entry (operation 0 apply / 1 residual / 2 Jacobi / 3 first
 * Jacobi sweep, dimension, element size in bytes, grid nodes, time modes,
 * modes per thread (1, 2 or 4; 3 with the column-streaming kernel only),
 * threads per CTA, or 0 for the 2D shared-memory tile kernel, or 64 for the
 * 2D column-streaming kernel), at most max_entries written to out
 * (may be NULL); *n_out = the number of entries. */
st_status st_tuned_shapes(int* out, int max_entries, int* n_out);
/* Pin the launch shape of one (operation, dimension, element size, grid
 * nodes, modes) key, same 7-int layout; later launches with that key use it
 * whatever the autotune option.  ST_ERR_ARG for a shape that is not one of the
 * tuner's candidates. */
st_status st_set_tuned_shape(const int* entry);

st_status st_destroy(st_handle* h);
const char* st_last_error(const st_handle* h);

/* Allocation-free combination.  The paper has no counterpart: this entry
 * point exists for callers that cannot let the library allocate device memory
 * at call time (for instance when another allocator has reserved the device
 * memory, or inside a time-critical loop where cudaMalloc would synchronise
 * the device).  It computes the same target-grid values as st_combine from
 * caller-owned component arrays and writes them to caller-owned out_dev
 * ((2^jx*+1)^d x (2^jt*+1) doubles, layout as in st_combine).
 *
 * comps[k]: U = device array of component k's coefficients, (2^jt+1) x
 * (2^jx-1)^d doubles (time-major, interior nodes x fastest: the layout of
 * st_component_coeffs), lift = device array of u0 on all (2^jx+1)^d nodes of
 * level jx, boundary included, x fastest (NULL if u0 = 0), the levels jx, jt
 * and the combination coefficient (+1 or -1).  At most 64 components.  d must
 * be the space dimension of the problem the arrays came from: the call cannot
 * check the arrays' sizes against d, jx and jt, and the caller is responsible
 * for it (a mismatch makes the kernels read outside the arrays).
 *
 * Scratch: a fixed 32 MiB array in device global memory, part of the library
 * image, so every GPU that loads the library holds it until the process exits.
 * Requests whose tables and partial sums do not fit are rejected with
 * ST_ERR_ARG (so are bad arguments, and a current device ordinal of 64 or
 * more, beyond the call's per-device cache of the scratch address); a failed
 * CUDA call or launch gives ST_ERR_CUDA.  A CUDA error already pending on the
 * calling thread when the call starts is reported as ST_ERR_CUDA before any
 * work is enqueued and is left pending (not cleared).
 * The call allocates nothing: no cudaMalloc, cudaFree or allocating library
 * routine.  Its first call on a device looks up the device address of the
 * scratch array (with that device current); make that first call before any
 * stream capture.  Every call reuses the same scratch and overwrites all of
 * it that it reads, so calls that overlap on the GPU (different streams, or
 * different host threads on one device) race and must be serialised by the
 * caller.  Work is enqueued on `stream`; the call does not synchronise. */
typedef struct {
  const double* U;
  const double* lift;
  int jx, jt, coef;
} st_comb_input;
st_status st_combine_noalloc(const st_comb_input* comps, int ncomp, int d, double T, int jx_star, int jt_star,
                             double* out_dev, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* ST_H_ */
