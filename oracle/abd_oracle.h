/* CPU oracle for the affine-body implicit time step (Lan et al., "Affine Body
 * Dynamics", ACM TOG 2022).
 *
 * TEST INFRASTRUCTURE ONLY.  This is a plain, slow, single-threaded FP64
 * implementation written from the paper, used to check the CUDA library.
 * Only the tests, the smoke check and the benchmark's CPU-baseline leg may
 * load or run it; the CUDA library shares no code with it and never calls it.
 *
 * Conventions
 *   q for body b: q[12b+0..2] = p, q[12b+3+3i+c] = A[i][c] (rows of A,
 *   Sec. 3).  Vertices, triangles and edges are grouped by body in body order.
 *   A pair is (kind, i, j): kind 0 = point-triangle (i vertex, j triangle of
 *   another body), kind 1 = edge-edge (i edge of body a, j edge of body b,
 *   a < b).  Pairs whose two bodies are both static are never formed.
 */
#ifndef ABD_ORACLE_H
#define ABD_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_PT = 0, ORC_EE = 1 };

enum {
  ORC_OK = 0,
  ORC_ERR_NEWTON = 1,     /* Newton iteration cap reached */
  ORC_ERR_LINESEARCH = 2, /* backtracking cap reached */
  ORC_ERR_CCD = 3,        /* ACCD iteration cap reached */
  ORC_ERR_SOLVE = 4,      /* linear solve failed */
  ORC_ERR_INTERSECT = 5,  /* a pair at zero distance */
  ORC_ERR_ARG = 6
};

typedef struct {
  int nb, nv, nt, ne;
  const double* xbar;             /* nv*3 rest-frame positions */
  const int* tri;                 /* nt*3 vertex indices */
  const int* edge;                /* ne*2 vertex indices */
  const int* vbody;               /* nv body of each vertex */
  const double* density;          /* nb */
  const double* kappa_body;       /* nb orthogonality stiffness */
  const unsigned char* is_static; /* nb */
  double dt, dhat, kappa, gravity[3], mu, eps_v;
  double newton_tol;   /* vertex-space Newton step bound (m) */
  double ls_slack_rel; /* line search accepts E <= E0 + slack_rel*(|E0|+1) */
  double cg_tol;       /* relative residual of the iterative solve */
  double ccd_s;        /* ACCD gap fraction */
  int newton_max, ls_max, ccd_max, cg_max, dense_max_dof;
} orc_scene;

typedef struct {
  int newton_iters, ls_halvings, solve_iters, n_candidates, n_active, n_swept, n_friction;
  double toi_min, last_step;
} orc_stats;

typedef struct orc_ctx orc_ctx;

/* --- scene ---------------------------------------------------------------- */
orc_ctx* orc_create(const orc_scene* sc);
void orc_destroy(orc_ctx* c);
int orc_set_state(orc_ctx* c, const double* q, const double* qdot); /* also lags friction at q */
void orc_get_state(const orc_ctx* c, double* q, double* qdot);
void orc_get_qtilde(const orc_ctx* c, double* qtilde);

/* --- Sec. 3 / 3.1 ---------------------------------------------------------- */
void orc_body_moments(const orc_ctx* c, int body, double* vol, double m1[3], double S[9]);
void orc_mass_matrix(const orc_ctx* c, int body, double M[144]);
void orc_vertices(const orc_ctx* c, const double* q, double* x);     /* x: nv*3 */
void orc_displacements(const orc_ctx* c, const double* dq, double* dx);

/* --- Sec. 3.2: orthogonality potential of one body (jets) ------------------ */
double orc_ortho(const double q[12], double kappa, double vol, double g[12], double H[144]);

/* --- geometry ---------------------------------------------------------------- */
double orc_d2_pp(const double p[3], const double q[3]);
double orc_d2_pe(const double p[3], const double a[3], const double b[3]);
double orc_d2_pt_plane(const double p[3], const double a[3], const double b[3], const double c[3]);
double orc_d2_ee_line(const double a[3], const double b[3], const double c[3], const double d[3]);
double orc_pt_dist2(const double x0[3], const double x1[3], const double x2[3], const double x3[3], int* type);
double orc_ee_dist2(const double x0[3], const double x1[3], const double x2[3], const double x3[3], int* type);
double orc_pair_dist2(int kind, const double x[12], int* type);
double orc_barrier(double d, double dhat);
double orc_ee_cross2(const double x[12]); /* |(x1 - x0) x (x3 - x2)|^2, canonical order */
double orc_ee_mollifier(double c, double eps_x, double* dm, double* d2m);
int orc_pair_barrier(int kind, const double x[12], double dhat, double kappa, double eps_x, int project,
                     double* E, double g[12], double H[144]);
void orc_sym_eig(int n, const double* A, double* w, double* V);
void orc_project_psd(int n, double* A);
int orc_accd(int kind, const double x[12], const double dx[12], double s, double tmax, int max_iter, double* toi);
double orc_friction_pair(const double x[12], const double gamma[4], const double nrm[3], const double r[3],
                         double mu_lambda, double eps, double g[12], double H[144]);
/* friction closest-point weights (Sec. 4 lagged friction): returns d^2 and the
 * type; gamma such that sum_v gamma_v x_v = point on the first primitive minus
 * point on the second */
double orc_closest_weights(int kind, const double x[12], double gamma[4], int* type);

/* --- candidate sets ------------------------------------------------------------ */
/* x1 == NULL: proximity set at x0; otherwise swept set over segments x0 -> x1.
 * brute != 0 tests every primitive pair (no body-level culling).
 * Returns the number of pairs (may exceed cap; only cap are written). */
long orc_candidates(const orc_ctx* c, const double* x0, const double* x1, int brute, int* kind, int* pi,
                    int* pj, long cap);

/* --- IP energy, gradient, Hessian (Sec. 4) ---------------------------------- */
/* E[0] total, E[1] inertia, E[2] orthogonality, E[3] barrier, E[4] friction.
 * g: 12*nb (zero rows for static bodies).  Stores the projected Hessian and
 * the candidate / active pair lists in the context for the getters below. */
int orc_energy_grad_hess(orc_ctx* c, const double* q, double* E, double* g, int project);
double orc_energy(orc_ctx* c, const double* q);
long orc_active_pairs(orc_ctx* c, const double* q, int* kind, int* pi, int* pj, int* type, double* d2, long cap);
int orc_grad_rows(orc_ctx* c, const double* q, int nsel, const int* sel, double* grows);
long orc_hess_nblocks(const orc_ctx* c);
void orc_hess_copy(const orc_ctx* c, double* diag, int* bpairs, double* blocks);
long orc_pairs_count(const orc_ctx* c, int which); /* 0 candidates, 1 active, 2 friction */
void orc_pairs_copy(const orc_ctx* c, int which, int* kind, int* pi, int* pj, int* type, double* d2);
/* lagged friction records in the order of orc_pairs_copy(which = 2): closest-
 * point weights (4 per pair), unit normal and lagged offset (3 each) */
void orc_friction_copy(const orc_ctx* c, double* gamma, double* nrm, double* r);

/* --- solve, CCD, step ------------------------------------------------------ */
int orc_solve(orc_ctx* c, const double* rhs, double* dq, int* iters); /* H dq = rhs, last H */
/* x = A^-1 b for a symmetric A (n x n, row-major) by A = L D L^T without
 * pivoting (the adjoint's dense solve); -1 on a zero pivot */
int orc_ldl_solve(int n, const double* A, const double* b, double* x);
int orc_ccd_toi(orc_ctx* c, const double* q, const double* dq, double* toi);
int orc_step(orc_ctx* c, int nsteps, orc_stats* st);

/* --- adjoint (implicit function theorem) ----------------------------------- */
/* One step backwards: H(q_next) lam = rhs with the unprojected Hessian of the
 * step that started at (q_t, qdot_t); returns M lam (12 nb) and dL/dkappa (nb).
 * Leaves the context at state (q_t, qdot_t). */
int orc_adjoint_step(orc_ctx* c, const double* q_t, const double* qdot_t, const double* q_next, const double* rhs,
                     double* Mlam, double* gkappa);

#ifdef __cplusplus
}
#endif
#endif
