/*
 * dg.h — C ABI of the GB300 (sm_103a) Runge–Kutta discontinuous Galerkin solver with the jump
 * filter of Wei, Zhou & Xia, arXiv 2407.19169.
 *
 * What one step computes (the paper's method, Sections 2-3):
 *   - modal DG on a uniform Cartesian mesh, Legendre basis on the reference cell
 *     (Eq. GLbasisequation; 2D tensor product Q^k or total degree P^k, Section 2.2);
 *   - volume integral (f(u_h), v_x) and local Lax–Friedrichs face fluxes (Eq. scheme:DG, Section 3);
 *   - third-order SSP Runge–Kutta in Shu–Osher form (Eq. rkdg1 / err_rk1);
 *   - after every stage the jump filter u^l <- exp(-sigma^l dt) u^l, with sigma^l from the jumps of
 *     the solution and its derivatives at the cell's own faces (Eqs. para:damp2-para:damp21 in 1D,
 *     para:damp22d-para:damp22d1 in 2D, max over components for systems, Eq. para:dampsystems1d;
 *     Euler parameters of Sections 3.1 and 3.2);
 *   - dt = CFL / max over cells of the wave-speed rate at cell averages, clipped to land on T
 *     (the CFL condition of Theorem 2.1).
 *
 * Conventions shared by every entry point:
 *   - Canonical state layout: u[(v * NM + m) * ncell + c], FP64, standard Legendre P_l(1) = 1.
 *     1D: c = i, m = l. 2D: c = i + nx * j (x fastest); m enumerates (p, q) with q outer and p inner
 *     (Q^k: m = p + (k+1) q; P^k: the same order with the modes p + q > k left out).
 *     Variables: scalar laws u; 1D Euler (rho, m, E); 2D Euler (rho, m_x, m_y, E).
 *   - Ownership: the library owns all device memory of a solver (or borrows the caller's workspace
 *     when dg_filter_params.workspace is set); the caller owns every host or device buffer passed
 *     in. cuda_stream is borrowed and must outlive the solver; NULL = a private stream the solver
 *     creates and destroys (the legacy default stream cannot hold a captured CUDA graph).
 *   - Errors: every call returns a dg_status; nothing throws or exits. A step that produces a
 *     non-physical or non-finite cell average returns DG_ERR_NONPHYSICAL and leaves the state at
 *     the last good step; afterwards only dg_read_state*, dg_write_state* (which clears the error)
 *     and dg_destroy are valid.
 *   - Threads: one solver per host thread, or external serialisation.
 *   - No CPU fallback: on a machine without a usable sm_103a GPU, dg_create fails with DG_ERR_CUDA.
 */
#ifndef DG_H
#define DG_H
#include <stddef.h>
#ifndef DG_API
#define DG_API __attribute__((visibility("default")))
#endif
#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  DG_OK = 0,
  DG_ERR_ARG = -1,          /* invalid argument (NULL pointer, size mismatch, bad enum)       */
  DG_ERR_OOM = -2,          /* device allocation failed                                        */
  DG_ERR_BUDGET = -3,       /* workspace too small / admission budget exceeded                 */
  DG_ERR_NONPHYSICAL = -4,  /* a cell average became non-finite, rho <= 0 or p <= 0            */
  DG_ERR_TIMEOUT = -5,      /* advance_to hit max_steps before reaching T; a bounded device wait
                               of dg_batch_run_persistent gave up                                  */
  DG_ERR_CUDA = -6,         /* a CUDA runtime call failed (message: dg_last_error)             */
  DG_ERR_STATE = -7,        /* call not valid in the solver's current state                    */
  DG_ERR_UNSUPPORTED = -8   /* configuration outside the compiled kernels (see dg_create)      */
} dg_status;

typedef enum { DG_EQ_ADVECTION = 0, DG_EQ_BURGERS = 1, DG_EQ_EULER = 2 } dg_equation;
typedef enum { DG_FLUX_LLF = 0 } dg_flux;
typedef enum { DG_BC_PERIODIC = 0, DG_BC_OUTFLOW = 1 } dg_bc;
typedef enum { DG_PREC_FP64 = 0, DG_PREC_FP32_MIXED = 1 } dg_precision;
typedef enum { DG_BASIS_Q = 0, DG_BASIS_P = 1 } dg_basis;
/* Damping coefficients of the filter (Section 2.1):
 *   DG_FILTER_JUMP    the paper's mode-dependent jump filter: the coefficient of a mode of total degree
 *                     l takes the jumps of the derivatives up to order l (Eqs. para:damp2-para:damp21,
 *                     2D: para:damp22d-para:damp22d1)
 *   DG_FILTER_GLOBAL  one coefficient for all modes, from the jumps of every derivative order the space
 *                     holds (Eq. para:damp; 2D: eq:2dalljumpvis1, orders up to 2k for Q^k), with the same
 *                     c_f factors as the jump filter
 *   DG_FILTER_OEDG    the OEDG damping as Section 2.1 restates it: sigma^l = max_v c_v (h ||[u_v]|| +
 *                     sum_{m<=l} (2m+1)/m! h^{m+1} ||[d^m u_v]||) / h^2, c_v = beta / (2 (2k-1)
 *                     ||u_v - avg(u_v)||_inf), the norm over the volume Gauss points of the whole mesh
 *                     (c_v = 0 for a constant variable); 2D: each direction with its own beta, h and
 *                     edges. Burgers and Euler, not with the positivity or hybrid limiter, not in
 *                     dg_batch_run or dg_step_noalloc (DG_ERR_UNSUPPORTED). Each stage then runs one more
 *                     kernel, because the coefficient needs the stage solution of the whole mesh */
typedef enum { DG_FILTER_JUMP = 0, DG_FILTER_GLOBAL = 1, DG_FILTER_OEDG = 2 } dg_filter_kind;

/* Initial conditions projected on the device (L2 projection, Gauss rule with nq_init points). */
typedef enum {
  DG_IC_SINE = 0,        /* scalar: a + b sin(w (x [+ y]) + phi); params a, b, w, phi              */
  DG_IC_RIEMANN1D = 1,   /* 1D Euler: rhoL,uL,pL, rhoR,uR,pR, x_split (primitive)                  */
  DG_IC_ENTROPY1D = 2,   /* 1D Euler: rho = r0 + A sin(w x), u = u0, p = p0; params r0,A,w,u0,p0   */
  DG_IC_QUADRANT2D = 3,  /* 2D Euler: (rho,u,v,p) for Q1..Q4, then x_split, y_split (18 params)     */
  DG_IC_VORTEX2D = 4     /* 2D Euler: isentropic vortex of Example 3.4(a); x0, y0, beta, t          */
} dg_ic;

/* Uniform Cartesian mesh (Section 2.1: K_j = [x_{j-1/2}, x_{j+1/2}]; Section 2.2: K_ij).
 * dim 1 uses nx, x0, x1, bc[0..1]; dim 2 also ny, y0, y1, bc[2..3]. bc: x-low, x-high, y-low,
 * y-high. Periodic sides must come in pairs (both sides of an axis alike). Outflow (the paper uses it
 * without defining it; the reading taken here): the ghost cell beyond a boundary face holds the
 * constant state equal to the adjacent interior cell's average. The LLF flux at that face is formed
 * from the interior trace and this constant ghost state (the average of the stage input), and the
 * filter's jumps there compare the interior cell's u~ and its derivatives with the ghost's constant
 * u~ average (all derivative jumps are then the interior derivatives themselves). */
typedef struct {
  int dim, nx, ny;
  double x0, x1, y0, y1;
  int bc[4];
} dg_mesh;

/* Filter and scheme parameters.
 *   enabled   1 = jump filter after every stage (the paper's scheme), 0 = plain RKDG
 *   cfl       CFL number (dt = cfl / max rate)
 *   gamma     ratio of specific heats (Euler)
 *   adv_speed linear-advection velocity
 *   basis     DG_BASIS_Q (tensor product, default) or DG_BASIS_P (total degree), 2D only
 *   nq        Gauss points per direction for volume and edge integrals; 0 or degree+1 only
 *   precision DG_PREC_FP64, or DG_PREC_FP32_MIXED (FP32 stage arithmetic, cell averages kept in
 *             double-float with compensated error-free updates)
 *   workspace optional caller-owned device buffer of at least dg_workspace_size bytes, aligned to
 *             256 bytes; NULL = the library allocates
 *   tile_rows rows per warp in the 2D stage kernel, 0 = default (the height that minimises the
 *             waves of resident warps times the rows a warp sweeps)
 *   tile_warps warps per thread block of the 2D stage kernel, 0 = default (the block size with the
 *             most resident warps per SM); both are tile-shape knobs for the autotuner, results do
 *             not depend on them
 *   positivity Euler only: 1 = the positivity-preserving limiter of Zhang and Shu after the filter in
 *             every stage (the paper applies it this way in Section 3.2), 0 = off (default): density
 *             is kept >= 1e-3 rho_bar and pressure >= min(1e-3 (rho_bar + |E_bar|), rho_bar, p_bar)
 *             (both precisions; the paper gives no margin) at the volume and edge Gauss points and,
 *             at degree 3, the Gauss-Lobatto mid-lines, by scaling the modes l >= 1; cell averages
 *             are untouched; the CFL rate then includes the wave speeds at those points
 *   hybrid    1 = the hybrid limiter of Algorithm 1 (Section 2.4) after every stage instead of the
 *             plain filter: cells whose jump indicator eta_j = ||[rho]||_{dK_j} / (2h) exceeds 1 are
 *             blended with their jump-filtered version by omega_j = (max eta - eta_j)/(max eta - 1),
 *             the others keep the unfiltered DG solution. Needs enabled = 1 and positivity = 0
 *             (DG_ERR_UNSUPPORTED otherwise); not available in dg_batch_run or dg_step_noalloc.
 *             0 = off (default)
 *   filter_kind DG_FILTER_JUMP (default), DG_FILTER_GLOBAL or DG_FILTER_OEDG (dg_filter_kind) */
typedef struct {
  int enabled;
  double cfl;
  double gamma;
  double adv_speed[2];
  int basis;
  int nq;
  int precision;
  void* workspace;
  size_t workspace_bytes;
  int tile_rows;
  int tile_warps;
  int positivity;
  int hybrid;
  int filter_kind;
} dg_filter_params;

typedef struct dg_solver dg_solver; /* opaque, library-owned */

/* Text for a status code; never NULL; static storage. */
DG_API const char* dg_status_string(int status);
/* Last CUDA error text seen by this library on the calling thread (static storage). */
DG_API const char* dg_last_error(void);
/* Fill *p with defaults: enabled 1, cfl 0.1, gamma 1.4, adv (1,0), Q^k, nq 0, FP64, no workspace. */
DG_API dg_status dg_params_default(dg_filter_params* p);

/* Bytes of device memory a solver with this configuration needs (state buffers + scalars). */
DG_API dg_status dg_workspace_size(const dg_mesh* mesh, int degree, int equation,
                            const dg_filter_params* params, size_t* bytes);

/* Create a solver. degree k in 1..3; equation: 1D advection/Burgers/Euler, 2D advection/Burgers/Euler.
 * The state starts at zero with t = 0 and must be set by dg_set_initial or dg_write_state*.
 * Errors: DG_ERR_ARG (NULL, nx < 1, bad enums, x1 <= x0, unpaired periodic sides),
 * DG_ERR_UNSUPPORTED (k > 3, nq not in {0, k+1}), DG_ERR_OOM, DG_ERR_BUDGET (workspace too small),
 * DG_ERR_CUDA (no device or no sm_103a image). */
DG_API dg_status dg_create(const dg_mesh* mesh, int degree, int equation, int flux,
                    const dg_filter_params* params, void* cuda_stream, dg_solver** out);

/* L2 projection of an analytic initial condition on the device (Gauss rule with nq_init points per
 * direction, 0 = k+3), then t = 0, steps = 0. Errors: DG_ERR_ARG (kind/params/equation mismatch). */
DG_API dg_status dg_set_initial(dg_solver* s, int ic_kind, const double* ic_params, int n_params, int nq_init);

/* Number of doubles of the canonical state: nvars * nmodes * ncells. */
DG_API dg_status dg_state_size(const dg_solver* s, size_t* n);

/* Copy a canonical FP64 state in (host or device pointer) and set the time; clears any error and
 * resets the step counter. n must equal dg_state_size. In the FP32 form, modes >= 1 are rounded to
 * FP32 and each cell average is split into a double-float pair. */
DG_API dg_status dg_write_state(dg_solver* s, const double* host_coeffs, size_t n, double t);
DG_API dg_status dg_write_state_device(dg_solver* s, const double* dev_coeffs, size_t n, double t);

/* Copy the canonical FP64 state out (host or device pointer) with its time. Synchronises the
 * solver's stream; the solve itself is not changed (the library refreshes its host copy of the
 * device step-control scalars and, in the FP32 form, uses its own conversion buffer). n must equal
 * dg_state_size. */
DG_API dg_status dg_read_state(const dg_solver* s, double* host_coeffs, size_t n, double* t);
DG_API dg_status dg_read_state_device(const dg_solver* s, double* dev_coeffs, size_t n, double* t);

/* One SSP-RK3 step with the filter after each stage; dt from the CFL condition (no clipping).
 * Synchronises; *dt_taken (may be NULL) receives the step size. */
DG_API dg_status dg_step(dg_solver* s, double* dt_taken);

/* Advance until t = T exactly (the last step is clipped) or max_steps steps have been taken,
 * whichever comes first. Synchronises. Returns DG_ERR_TIMEOUT if max_steps ran out first. */
DG_API dg_status dg_advance_to(dg_solver* s, double T, long long max_steps, long long* steps_taken);

/* Enqueue nsteps unclipped steps on the solver's stream without synchronising (for timing and for
 * overlapping several solvers). Replaces any stop condition set by dg_set_target (T_end = +inf).
 * Use dg_sync to wait and collect the status. */
DG_API dg_status dg_advance_steps(dg_solver* s, long long nsteps);

/* Set the device stop condition: stepping stops (further steps are no-ops) once t reaches T_end
 * (the last step is clipped to land on it) or after max_steps more steps. Synchronises. */
DG_API dg_status dg_set_target(dg_solver* s, double T_end, long long max_steps);

/* Batched stepping (many uneven solves at once): advance every solver in solvers[0..n-1] by up to
 * `steps` SSP-RK3 steps. Solvers of the same (dimension, degree) class share one work-list kernel
 * per stage whose warps take tile items from all instances of the class; the classes run as
 * parallel branches of one CUDA graph that holds a whole step and is replayed `steps` times on the
 * first solver's stream. Each solver keeps its own dt (its own CFL max) and stop condition
 * (dg_set_target): a solver that reaches its T_end or step limit idles. Results equal those of the
 * same solver stepped alone. Supported: Euler, FP32 form, 1D or 2D Q^k; all on one device.
 * Synchronises; returns DG_ERR_NONPHYSICAL if any solver failed (check each with dg_sync). */
DG_API dg_status dg_batch_run(dg_solver* const* solvers, int n, long long steps);

/* Batched stepping as dg_batch_run, with the same arguments, classes and results, in one persistent
 * launch per class instead of a replayed per-step graph: each class's kernel runs all `steps` steps of
 * its solvers. Its warps take tile items from a queue ordered by (step, stage, solver, item); before
 * an item a warp waits until every item of that solver's earlier stages has finished (a per-solver
 * counter on the device), and the last item of a solver's step advances its t and step count and
 * sets its next dt. Solvers therefore move through their stages independently: a small solver does
 * not wait for a large one. The launches are cooperative (all blocks resident). Every wait polls a
 * bounded number of times (about a second); if one gives up, all warps leave and the call returns
 * DG_ERR_TIMEOUT with the solvers' states undefined (a wait that is not broken lasts at most one
 * stage of its solver). Allocates a small device scratch block (16 bytes per solver) per call.
 * A class's launch runs until its whole queue (steps x 3 x its items) is taken, even after all its
 * solvers have reached their T_end: their items are then skipped, at about a microsecond of a warp
 * each, so pass a step count near the one needed (dg_batch_run idles the same way, per step).
 * steps above 2^30 are rejected with DG_ERR_ARG (the per-solver stage counters are 32-bit).
 * Synchronises; DG_ERR_NONPHYSICAL as dg_batch_run. Not while a stream is captured. */
DG_API dg_status dg_batch_run_persistent(dg_solver* const* solvers, int n, long long steps);

/* Wait for the solver's stream; report the time, the completed step count and any error. */
DG_API dg_status dg_sync(dg_solver* s, double* t, long long* steps);

/* Per-variable mass sum_cells |K| * u_bar (the conserved quantities, Section 2.4). Synchronises. */
DG_API dg_status dg_mass(dg_solver* s, double* mass_per_var);

/* Solver geometry: nvars, nmodes, ncells (any pointer may be NULL). */
DG_API dg_status dg_dims(const dg_solver* s, int* nvars, int* nmodes, long long* ncells);

/* Number of kernels this solver has launched (stage kernels, projections, reductions, copies). */
DG_API dg_status dg_kernel_launches(const dg_solver* s, long long* launches);

/* One FP64 SSP-RK3 step (jump filter after each stage) from u_in to u_out that allocates no device
 * memory. The paper has no counterpart to this entry point; it is for callers that cannot call
 * cudaMalloc where they want a step: code running while a stream is being captured into a CUDA graph,
 * frameworks that own every byte of device memory through a pre-planned arena, and latency-critical
 * loops that must not allocate or synchronise. They pass the input and output states; the two
 * intermediate stage states and the step-control scalars live in one static device array of
 * 32 MiB + 256 B, which every GPU that loads this library holds until the process exits. Meshes whose
 * two FP64 stage states do not fit in 32 MiB are rejected with DG_ERR_BUDGET before anything runs.
 *   mesh, degree, equation, params: as for dg_create; params->precision must be DG_PREC_FP64.
 *   u_in, u_out: device pointers to canonical FP64 states (dg_state_size doubles); must not overlap.
 *   dt_taken: host pointer or NULL. If non-NULL the call synchronises the stream, stores the step size
 *     and returns DG_ERR_NONPHYSICAL if a cell average became non-physical; if NULL nothing is read
 *     back and the call returns as soon as the kernels are enqueued. Pass NULL while the stream is
 *     being captured (a capture cannot synchronise). With NULL a non-physical step is not reported:
 *     u_out then holds the step's last stage output, and the next call's reset of the shared
 *     scalars erases the error record.
 *   cuda_stream: the stream the kernels run on (NULL = the legacy default stream).
 *   Arguments are checked as by dg_create (same status codes); also DG_ERR_UNSUPPORTED for the FP32
 *   form or the hybrid limiter; params->workspace, tile_rows and tile_warps are ignored.
 * The first call on a device (with that device current) sets the device up once: it checks for an
 * sm_103 GPU, copies the Gauss rules of the CFL-rate kernel to constant memory and looks up the
 * array's device address; make that first call before any stream capture. The cached address
 * belongs to the device's context of that moment: after cudaDeviceReset in the same process it is
 * stale and no further call may be made on that device. All calls share the array, which keeps the
 * last call's contents (each call resets the scalars it uses): calls that overlap on the GPU race. */
DG_API dg_status dg_step_noalloc(const dg_mesh* mesh, int degree, int equation,
                                 const dg_filter_params* params, const double* u_in, double* u_out,
                                 double* dt_taken, void* cuda_stream);

/* Release all device memory the library allocated for this solver. NULL is accepted. */
DG_API dg_status dg_destroy(dg_solver* s);

#ifdef __cplusplus
}
#endif
#endif /* DG_H */
