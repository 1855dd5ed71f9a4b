/* abd.h -- C ABI of the GB300 affine-body time-step library (libabd.so).
 *
 * The library computes one implicit time step of Affine Body Dynamics
 * (Lan, Kaufman, Li, Jiang, Yang, "Affine Body Dynamics: Fast, Stable and
 * Intersection-free Simulation of Stiff Materials", ACM TOG 2022):
 * given the state (q^t, qdot^t) of affine bodies q_b = (p, a1, a2, a3)
 * (Sec. 3, Eq. kinematic), it returns the minimiser of the incremental
 * potential
 *     E(q) = sum_b [ 1/2 |q_b - qtilde_b|_M^2 + dt^2 V_perp(q_b) ] + V_C(q) + V_F(q)
 * (Sec. 4; V_perp Sec. 3.2 Eq. orthogonality; V_C Eq. barrier with the
 * clamped log barrier Eq. clamped-b; V_F the friction potential of Sec. 4),
 * reached by Newton iterations whose steps are filtered by additive CCD
 * along linear vertex trajectories (Sec. 4.1) so the result is
 * intersection-free, with contact pairs culled by d-hat-dilated boxes
 * (Sec. 4.2) and the Hessian assembled as 12x12 body blocks (Sec. 4.3).
 *
 * Conventions shared by every call
 *   Layout   q and qdot are 12 doubles per body, body-major:
 *            q[12b+0..2] = p, q[12b+3+3i+c] = A[i][c] (rows of A, Sec. 3).
 *            Static bodies keep their q and have no degrees of freedom.
 *   Memory   *_dev pointers are device memory owned by the caller, borrowed
 *            for the duration of the call; *_host pointers are host memory.
 *            Descriptor arrays passed to abd_create_scene are copied; the
 *            caller may free them when the call returns.
 *   Streams  all device work is ordered on the CUDA stream given at
 *            creation.  Calls that return host values synchronise it.
 *   Errors   every call returns an abd_status; abd_last_error() gives a
 *            message.  Kernels never trap: they record failures in a device
 *            status word that the host reads.  A failed abd_step leaves the
 *            scene state as it was before the call.
 *   Numbers  the FP64 path decides pair membership and CCD step sizes with a
 *            fixed operation order and reduces sums in a fixed order, so two
 *            runs give bit-identical results.
 */
#ifndef ABD_H
#define ABD_H

#include <stddef.h>

#if defined(__GNUC__)
#define ABD_API __attribute__((visibility("default")))
#else
#define ABD_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct abd_scene abd_scene;

typedef enum {
  ABD_OK = 0,
  ABD_ERR_INVALID_ARG = 1,
  ABD_ERR_CUDA = 2,
  ABD_ERR_OOM = 3,
  ABD_ERR_CAPACITY = 4,             /* internal buffer too small (the step retries with larger ones) */
  ABD_ERR_INITIAL_INTERSECTION = 5, /* a contact pair at zero distance */
  ABD_ERR_NONFINITE = 6,            /* NaN / Inf in the state or the system */
  ABD_ERR_NEWTON_MAXITER = 7,
  ABD_ERR_LINESEARCH = 8,
  ABD_ERR_PCG_BREAKDOWN = 9,
  ABD_ERR_PCG_MAXITER = 10,
  ABD_ERR_CCD_MAXITER = 11
} abd_status;

/* Device allocator.  alloc returns device memory of `bytes` bytes usable on
 * `stream` (NULL on failure); free releases it.  Passing NULL to
 * abd_create_scene makes the library use cudaMalloc / cudaFree. */
typedef struct {
  void* (*alloc)(size_t bytes, void* stream, void* ctx);
  void (*free)(void* ptr, void* stream, void* ctx);
  void* ctx;
} abd_allocator;

/* Physical and solver parameters (Sec. 4 and Sec. 5.5 for d-hat). */
typedef struct {
  double dt;            /* time step (s) */
  double dhat;          /* barrier activation distance d-hat (m) */
  double kappa;         /* barrier stiffness of V_C */
  double gravity[3];    /* m/s^2 */
  double mu;            /* friction coefficient; 0 disables V_F */
  double eps_v;         /* friction mollifier velocity (m/s); eps = eps_v * dt */
  double newton_tol;    /* stop when max vertex |J dq| <= newton_tol (m); <= 0: 1e-5 x dynamic bbox diagonal x dt */
  double pcg_rel_tol;   /* PCG relative residual */
  double ls_slack_rel;  /* line search accepts E <= E0 + ls_slack_rel (|E0| + 1) */
  double ccd_s;         /* ACCD gap fraction s (the step keeps >= s of each pair's distance) */
  int newton_max, pcg_max, ls_max, ccd_max;
  int precision;        /* 0: FP64 throughout.  1: mixed - the PSD projection of the
                           6- and 9-dimensional barrier Hessians is taken from an
                           FP32 eigenbasis without FP64 refinement (distances,
                           barrier values and logs, energies, gradients, CCD, the
                           Newton test and the line search stay FP64); when a
                           step passes the Newton test, the test is repeated at
                           the same iterate with the FP64-refined projection, so
                           both modes stop on the same criterion */
  int dense_max_dofs;   /* 0: the linear solves use block-Jacobi PCG.  > 0: scenes with
                           12 x bodies <= dense_max_dofs (at most 3072 after padding to a
                           multiple of 32) solve by a dense Cholesky factorisation on the
                           device instead (Newton steps, abd_solve, abd_adjoint_step);
                           abd_solve_stats then reports 0 iterations and residual 0 */
} abd_params;

/* Scene description (host arrays, copied).  Vertices, triangles and edges
 * must be grouped by body in body order; tri / edge hold global vertex ids;
 * each dynamic body's triangles form a closed, outward-oriented surface
 * (its mass matrix comes from them by the divergence theorem, Sec. 3.1). */
typedef struct {
  int nb, nv, nt, ne;
  const double* xbar;             /* nv*3 rest-frame positions */
  const int* tri;                 /* nt*3 */
  const int* edge;                /* ne*2 */
  const int* vbody;               /* nv */
  const double* q0;               /* nb*12 */
  const double* qdot0;            /* nb*12 */
  const double* density;          /* nb, kg/m^3 */
  const double* kappa_body;       /* nb, orthogonality stiffness of V_perp */
  const unsigned char* is_static; /* nb */
} abd_scene_desc;

typedef struct {
  long n_candidates;   /* primitive pairs passing the box test (Sec. 4.2) */
  long n_active;       /* pairs with d < d-hat (terms of V_C) */
  long n_friction;     /* lagged friction pairs (terms of V_F) */
  long n_body_pairs;   /* body pairs carrying an off-diagonal Hessian slot */
} abd_pair_counts;

typedef struct {
  int iterations;
  double rel_residual;
} abd_solve_stats;

typedef struct {
  int newton_iters, pcg_iters;
  int ls_halvings;     /* line-search rounds after the first trial of each Newton iteration */
  long n_candidates, n_active, n_swept;
  double toi_min;      /* smallest CCD step bound seen in the step */
  double last_step;    /* max vertex |J dq| of the last Newton step */
  long kernel_launches;       /* kernels the library launched for the step(s) */
  long candidates_tested;     /* candidate pairs distance-tested in the step(s) */
  long active_evaluated;      /* barrier terms (E, gradient, Hessian) evaluated */
  int ccd_limited;     /* Newton iterations whose smallest island CCD bound was < 1 */
  int toi_hist[6];     /* Newton iterations by that bound: 1, [0.1,1), [0.01,0.1),
                          [1e-3,0.01), [1e-4,1e-3), below 1e-4 */
  int n_islands;       /* contact islands of the last Newton iteration */
  int ls_island_halvings_max;  /* most halvings any island needed in one Newton iteration */
} abd_step_stats;

/* Per-kernel timing of one kernel class, accumulated while profiling is on. */
typedef struct {
  const char* name;
  long launches;
  double total_ms;     /* sum of per-launch durations (CUDA events on the scene's stream) */
  double bytes;        /* algorithmic bytes of those launches (0 if not defined) */
  double flops;        /* algorithmic FP64 operations of those launches (0 if not defined) */
} abd_kernel_profile;

/* Fill *p with the defaults used by the benchmarks: dt 0.01, d-hat 1e-3,
 * kappa 1e8, gravity (0,0,-9.8), mu 0, eps_v 1e-3, newton_tol 0 (relative),
 * pcg_rel_tol 1e-4 (inexact Newton), ls_slack_rel 1e-12, ccd_s 0.1, caps 500/20000/30/10000. */
ABD_API void abd_default_params(abd_params* p);

/* Create a scene on the current CUDA device.  stream: a cudaStream_t (NULL =
 * legacy default stream).  Validates the description (grouping, indices,
 * closed meshes) and checks that no contact pair starts at zero distance
 * (ABD_ERR_INITIAL_INTERSECTION).  *out receives the scene on success. */
ABD_API abd_status abd_create_scene(const abd_scene_desc* desc, const abd_params* params, const abd_allocator* alloc,
                            void* stream, abd_scene** out);

/* Release every resource of the scene (NULL is accepted). */
ABD_API void abd_destroy(abd_scene* s);

/* Copy the state in (set) or out (get).  on_device != 0: q, qdot are device
 * pointers; else host.  Setting the state recomputes qtilde (Sec. 4) and the
 * lagged friction set.  Either pointer may be NULL on get. */
ABD_API abd_status abd_set_state(abd_scene* s, const double* q, const double* qdot, int on_device);
ABD_API abd_status abd_get_state(abd_scene* s, double* q, double* qdot, int on_device);

/* Energy, gradient and projected Hessian of the incremental potential at q
 * (Sec. 4 and Sec. 4.3), with qtilde and the friction set of the current
 * state.  E_host[5] = {total, inertia, orthogonality, barrier, friction};
 * g_dev: 12*nb doubles (zero rows for static bodies); counts may be NULL.
 * The Hessian and the pair sets stay in the scene for abd_get_hessian,
 * abd_get_pairs and abd_solve until the next call on the scene. */
ABD_API abd_status abd_energy_grad_hess(abd_scene* s, const double* q_dev, double* E_host, double* g_dev,
                                abd_pair_counts* counts);

/* Copy the Hessian of the last abd_energy_grad_hess to the host:
 * diag: nb*144 (row-major 12x12 per body; identity for static bodies);
 * bi, bj, blocks: the off-diagonal blocks H[bi][bj] (bi < bj, row-major,
 * rows = DOFs of bi), at most cap of them; *nblocks receives the count.
 * Blocks may be zero (body pairs whose boxes are near but no pair is active). */
ABD_API abd_status abd_get_hessian(abd_scene* s, double* diag, int* bi, int* bj, double* blocks, long cap, long* nblocks);

/* Copy a pair set of the last abd_energy_grad_hess to the host: which = 0
 * candidates, 1 active, 2 lagged friction.  kind 0 point-triangle (i vertex,
 * j triangle), 1 edge-edge (i, j edges of bodies a < b); type: distance
 * type (active and friction sets), d2: squared distance (active set).
 * Arrays may be NULL to query the count only. */
ABD_API abd_status abd_get_pairs(abd_scene* s, int which, int* kind, int* i, int* j, int* type, double* d2, long cap,
                         long* n);

/* Copy the lagged friction records of the current step start (Sec. 4,
 * friction potential V_F with lambda, the closest points and the normal
 * frozen at q^t), in the order of abd_get_pairs(which = 2): gamma (4 per
 * pair: the closest-point weights, so that sum_v gamma_v x_v is the point on
 * the first primitive minus the point on the second), normal (3 per pair,
 * unit) and offset (3 per pair, sum_v gamma_v x_v at q^t).  Host arrays, at
 * most cap records each; any may be NULL; *n receives the count. */
ABD_API abd_status abd_get_friction(abd_scene* s, double* gamma, double* normal, double* offset, long cap, long* n);

/* Solve H dq = rhs with block-Jacobi PCG on the Hessian of the last
 * abd_energy_grad_hess (the linear solve of each Newton iteration), or by the
 * dense Cholesky when dense_max_dofs covers the scene (stats: 0 iterations,
 * residual 0).  Static bodies' rows of dq are zero. */
ABD_API abd_status abd_solve(abd_scene* s, const double* rhs_dev, double* dq_dev, abd_solve_stats* stats);

/* Largest step alpha in (0, 1] such that the linear vertex trajectories from
 * x(q) to x(q + alpha dq) are intersection-free by additive CCD (Sec. 4.1). */
ABD_API abd_status abd_ccd_toi(abd_scene* s, const double* q_dev, const double* dq_dev, double* toi_host);

/* Advance nsteps implicit-Euler time steps (Sec. 4); stats (may be NULL)
 * receives the statistics of the last step. */
ABD_API abd_status abd_step(abd_scene* s, int nsteps, abd_step_stats* stats);

/* Launch shape of a scene's kernels and the size of its preconditioner's
 * clusters.  grid_div divides the grids that are sized by the device rather
 * than by a host-known count (kernels that grid-stride over a count held on
 * the device: barrier terms, assembly blocks, friction records,
 * incoming-pair lists); 1 = one full wave per kernel class (the default),
 * larger values leave SMs to the kernels of other scenes stepped
 * concurrently.  Results do not depend on it (every such kernel writes
 * per-item outputs or exact integer reductions).  Values outside 1..64
 * return ABD_ERR_INVALID_ARG.  The scene's captured launch sequences are
 * re-captured on its next step.
 *
 * cluster_max: the PCG's cluster block-Jacobi preconditioner cuts every
 * contact island (in breadth-first order) into runs of at most cluster_max
 * bodies and factors each run densely (one SM per run, (12 n)^3 / 3 flop);
 * 1 = plain block-Jacobi; 0 = the default, 12; at most 16.  Larger runs
 * cost more per factorisation and usually fewer PCG iterations; the Newton
 * directions differ only within the PCG tolerance.  Values outside 0..16
 * return ABD_ERR_INVALID_ARG. */
typedef struct {
  int grid_div;
  int cluster_max;
  int reserved[6];   /* zero */
} abd_tuning;
ABD_API abd_status abd_set_tuning(abd_scene* s, const abd_tuning* t);
ABD_API abd_status abd_get_tuning(const abd_scene* s, abd_tuning* t);

/* Step a batch of independent scenes nsteps each (the many-scene form of
 * Sec. 4's time step: every scene keeps its own Newton loop, line search
 * and convergence, so each result is bit-identical to abd_step on that scene
 * alone).  nworkers host threads (1..256) take scenes, largest body count
 * first, and drive each on its own stream; scenes must have distinct streams
 * for their work to overlap on the GPU, and must be created on the same
 * device.  status (n entries, may be NULL) receives each scene's result;
 * stats (n entries, may be NULL) each scene's abd_step_stats.  Returns
 * ABD_OK if every scene succeeded, else the first failing scene's status in
 * batch order (the other scenes still run; a failed scene is left at its
 * state before the failing step, as abd_step leaves it).  No other call may
 * use these scenes until it returns. */
ABD_API abd_status abd_step_batch(abd_scene* const* scenes, int n, int nsteps, int nworkers, abd_status* status,
                                  abd_step_stats* stats);

/* Profiling (the step's tracing facility): on != 0 starts recording CUDA
 * events around each launch of the timed kernel classes and clears the
 * accumulators; 0 stops.  abd_get_profile synchronises the stream and fills
 * up to cap entries (one per kernel class), *n the number of classes. */
ABD_API abd_status abd_set_profiling(abd_scene* s, int on);
ABD_API abd_status abd_get_profile(abd_scene* s, abd_kernel_profile* out, int cap, int* n);

/* Adjoint of one time step by the implicit function theorem (differentiating
 * through the step's minimisation of the IP, Sec. 4).  The step started at
 * (q_t, qdot_t) and ended at q_next; with H the UNPROJECTED Hessian of its IP
 * at q_next (body blocks M + dt^2 hess V_ortho, barrier terms without the PSD
 * clamp, friction with its lagged quantities held fixed) and
 *   rhs = dL/dq_next + dL/dqdot_next / dt   (qdot_next = (q_next - q_t)/dt),
 * it solves H lam = rhs by the block-Jacobi PCG to rel_tol (or by the dense
 * Cholesky when the scene was created with dense_max_dofs covering it; a
 * non-positive pivot is ABD_ERR_PCG_BREAKDOWN) and, since
 * dL/dq~ = M lam (q~ = q_t + dt qdot_t + dt^2 g):
 *   gq    <- M lam - dL/dqdot_next / dt          (dL/dq_t)
 *   gqdot <- dt M lam                            (dL/dqdot_t)
 *   gkappa += -dt^2 lam_b . grad V_b / kappa_b   (per body)
 * gq_dev / gqdot_dev (12 nb, device) hold dL/dq_next, dL/dqdot_next on entry
 * and are overwritten; gkappa_dev (nb, device) is accumulated; static rows are
 * zero.  Leaves the scene's state at (q_t, qdot_t).  Errors as abd_solve
 * (ABD_ERR_PCG_BREAKDOWN if H is not positive definite along the iterates). */
ABD_API abd_status abd_adjoint_step(abd_scene* s, const double* q_t_dev, const double* qdot_t_dev,
                                    const double* q_next_dev, double* gq_dev, double* gqdot_dev, double* gkappa_dev,
                                    double rel_tol, abd_solve_stats* stats);

/* Work counters of the barrier-term kernel, cumulative since the scene was
 * created (diagnostics of the eigen-projection's cost; no effect on
 * results).  Synchronises the scene's stream. */
typedef struct {
  unsigned long long barrier_terms[4]; /* terms evaluated, by reduced dimension m = 1, 2, 3 (index m) */
  unsigned long long sweeps_fp32;      /* FP32 Jacobi sweeps over all 6- and 9-dimensional terms */
  unsigned long long sweeps_fp64;      /* FP64 refinement sweeps over the same terms */
  unsigned long long capped_fp64;      /* terms whose FP64 sweeps reached the sweep cap */
  /* culling of the candidate enumeration (Sec. 4.2), summed over every
   * enumeration pass: all primitive pairs (point-triangle both ways,
   * edge-edge) of the body pairs whose d-hat-dilated boxes overlap; the pairs
   * left after restricting each body's primitives to the other body's box
   * (the i-AABB intersection test); the candidates passing the exact
   * primitive box test */
  unsigned long long prim_pairs_body;
  unsigned long long prim_pairs_iaabb;
  unsigned long long prim_pairs_cand;
} abd_counters;
ABD_API abd_status abd_get_counters(abd_scene* s, abd_counters* out);

/* Minimum additive-CCD time of impact over a caller-given list of pairs,
 * allocating nothing.  The paper has no counterpart: this serves callers
 * that cannot allocate device memory when they need a step bound (a fixed
 * memory pool owned elsewhere, allocation-free real-time loops).
 *   x_dev, dx_dev  nv*3 doubles (device): start positions and the linear
 *                  displacement of each vertex over the step
 *   verts_dev      npairs*4 ints (device): the pair's vertices, ordered as in
 *                  abd_get_pairs (point then triangle, or edge then edge)
 *   kind_dev       npairs bytes (device): 0 point-triangle, 1 edge-edge
 *   ccd_s, ccd_max ACCD gap fraction and iteration cap (as abd_params)
 *   toi_host       receives min over pairs of the time of impact in [0, 1]
 *                  (0: a pair starts at zero distance); when a pair reaches
 *                  ccd_max the call returns ABD_ERR_CCD_MAXITER and toi_host
 *                  still receives the minimum, in which such a pair counts
 *                  with the time it had advanced to (a conservative lower
 *                  bound: its trajectory is intersection-free up to there)
 * Scratch is a file-scope device array of 262,144 pair slots (2 MiB) that
 * every GPU loading the library holds until exit; npairs beyond that returns
 * ABD_ERR_CAPACITY, an out-of-range vertex or kind ABD_ERR_INVALID_ARG (the
 * kernel checks each index before it loads through it).
 * The first call in each CUDA context (per device: the primary context, or
 * a driver-API context current on the calling thread; again after
 * cudaDeviceReset) looks up the array's device address and caches it under
 * the context's id; make that first call before any stream capture.  All
 * calls share the one array, so calls that overlap on the GPU (other
 * streams, other threads) race.  The call synchronises `stream` (a
 * cudaStream_t, NULL = legacy default) and reports only errors of its own
 * launches and copies. */
ABD_API abd_status abd_ccd_toi_pairs_noalloc(const double* x_dev, const double* dx_dev, int nv, const int* verts_dev,
                                             const unsigned char* kind_dev, long npairs, double ccd_s, int ccd_max,
                                             void* stream, double* toi_host);

/* Message of the last error on the scene (empty string if none). */
ABD_API const char* abd_last_error(const abd_scene* s);

#ifdef __cplusplus
}
#endif
#endif
