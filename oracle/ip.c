/* Oracle for the incremental potential of affine bodies and its Newton solve.
 *
 * TEST INFRASTRUCTURE ONLY: a plain, slow FP64 CPU implementation written
 * from the paper.  Only tests, the smoke check and the benchmark's CPU
 * baseline may load it; the CUDA library never does.
 *
 * Paper passages followed (Lan et al., Affine Body Dynamics, 2022):
 *   Sec. 3, Eq. kinematic       x = A xbar + p = J(xbar) q
 *   Sec. 3.1, Eq. mass          M = int rho J^T J
 *   Sec. 3.1, Eq. EL            f = sum_k J(xbar_k)^T f_k (gravity as a body force)
 *   Sec. 3.2, Eq. orthogonality V = kappa nu |A A^T - I|_F^2
 *   Sec. 4                      E_b = 1/2 |q - qtilde|_M^2 + dt^2 V,
 *                               qtilde = q^t + dt qdot^t + dt^2 M^-1 f
 *   Sec. 4, Eq. barrier/clamped-b  V_C = kappa sum B(d_i)
 *   Sec. 4 (friction)           V_F = sum mu lambda_j m_j(q)
 *   Sec. 4.1                    linear trajectories from the previous iterate, ACCD
 *   Sec. 4.2                    culling by d-hat-dilated body boxes
 *   Sec. 4.3                    12x12 diagonal blocks + off-diagonal body-pair blocks
 * Readings where the paper is silent are listed beside each function.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "abd_oracle.h"
#include "jet.h"

void orc_jet_pair_d2(jet* r, int kind, int type, const double x[12]);

/* ------------------------------------------------------------------------ */
/* growable pair list                                                       */
/* ------------------------------------------------------------------------ */

typedef struct {
  int *kind, *i, *j, *type;
  double* d2;
  long n, cap;
} plist;

static void pl_push(plist* L, int kind, int i, int j, int type, double d2) {
  if (L->n == L->cap) {
    long nc = L->cap ? 2 * L->cap : 1024;
    L->kind = (int*)realloc(L->kind, nc * sizeof(int));
    L->i = (int*)realloc(L->i, nc * sizeof(int));
    L->j = (int*)realloc(L->j, nc * sizeof(int));
    L->type = (int*)realloc(L->type, nc * sizeof(int));
    L->d2 = (double*)realloc(L->d2, nc * sizeof(double));
    L->cap = nc;
  }
  L->kind[L->n] = kind;
  L->i[L->n] = i;
  L->j[L->n] = j;
  L->type[L->n] = type;
  L->d2[L->n] = d2;
  L->n++;
}

static void pl_free(plist* L) {
  free(L->kind);
  free(L->i);
  free(L->j);
  free(L->type);
  free(L->d2);
  memset(L, 0, sizeof(*L));
}

/* lagged friction pair: closest-point weights gamma on the 4 pair vertices,
 * contact normal, lagged closest-point offset r and mu*lambda */
typedef struct {
  int kind, i, j, type;
  double gamma[4], n[3], r[3], mu_lambda;
} fpair;

struct orc_ctx {
  orc_scene sc;
  double *xbar, *density, *kappa_body;
  int *tri, *edge, *vbody;
  unsigned char* is_static;
  int *vbeg, *vend, *tbeg, *tend, *ebeg, *eend;
  double *vol, *m1, *S, *M; /* per body */
  double* l2e;               /* squared rest length of every edge */
  double *qt, *qdot, *qtilde;
  fpair* fr;
  long nfr;
  /* last energy evaluation */
  plist cand, act;
  double* diag;       /* nb*144 */
  int* bpairs;        /* 2*nblk */
  double* blocks;     /* 144*nblk */
  long nblk, blk_cap;
  orc_stats st;
};

/* ------------------------------------------------------------------------ */
/* small dense helpers                                                      */
/* ------------------------------------------------------------------------ */

/* in-place Cholesky of an n x n SPD matrix (lower factor); 0 on success */
static int chol(int n, double* A) {
  for (int j = 0; j < n; ++j) {
    double s = A[j * n + j];
    for (int k = 0; k < j; ++k) s -= A[j * n + k] * A[j * n + k];
    if (!(s > 0.0)) return -1;
    double l = sqrt(s);
    A[j * n + j] = l;
    for (int i = j + 1; i < n; ++i) {
      double t = A[i * n + j];
      for (int k = 0; k < j; ++k) t -= A[i * n + k] * A[j * n + k];
      A[i * n + j] = t / l;
    }
  }
  return 0;
}

static void chol_solve(int n, const double* L, double* x) {
  for (int i = 0; i < n; ++i) {
    double s = x[i];
    for (int k = 0; k < i; ++k) s -= L[i * n + k] * x[k];
    x[i] = s / L[i * n + i];
  }
  for (int i = n - 1; i >= 0; --i) {
    double s = x[i];
    for (int k = i + 1; k < n; ++k) s -= L[k * n + i] * x[k];
    x[i] = s / L[i * n + i];
  }
}

/* Symmetric indefinite factorisation A = L D L^T, L unit lower triangular,
 * D diagonal, without pivoting (exists when every leading principal minor is
 * nonzero; Golub & Van Loan, Matrix Computations, Sec. 4.1, the LDL^T
 * form).  Column j: v_k = L_jk d_k (k < j), d_j = a_jj - sum_k L_jk v_k,
 * L_ij = (a_ij - sum_k L_ik v_k) / d_j.  L below the diagonal and D on it,
 * in place.  Returns -1 on a zero or non-finite pivot. */
static int ldl(int n, double* A) {
  double* v = (double*)malloc(sizeof(double) * (n + 1));
  int bad = 0;
  for (int j = 0; j < n && !bad; ++j) {
    double d = A[(size_t)j * n + j];
    for (int k = 0; k < j; ++k) {
      v[k] = A[(size_t)j * n + k] * A[(size_t)k * n + k];
      d -= A[(size_t)j * n + k] * v[k];
    }
    if (!(fabs(d) > 0.0) || !isfinite(d)) {
      bad = 1;
      break;
    }
    A[(size_t)j * n + j] = d;
    for (int i = j + 1; i < n; ++i) {
      double t = A[(size_t)i * n + j];
      for (int k = 0; k < j; ++k) t -= A[(size_t)i * n + k] * v[k];
      A[(size_t)i * n + j] = t / d;
    }
  }
  free(v);
  return bad ? -1 : 0;
}

/* L z = b, w = D^-1 z, L^T x = w, in place */
static void ldl_solve(int n, const double* F, double* x) {
  for (int i = 0; i < n; ++i) {
    double s = x[i];
    for (int k = 0; k < i; ++k) s -= F[(size_t)i * n + k] * x[k];
    x[i] = s;
  }
  for (int i = 0; i < n; ++i) x[i] /= F[(size_t)i * n + i];
  for (int i = n - 1; i >= 0; --i) {
    double s = x[i];
    for (int k = i + 1; k < n; ++k) s -= F[(size_t)k * n + i] * x[k];
    x[i] = s;
  }
}

/* exported for the tests: x = A^-1 b by ldl(); A is not modified */
int orc_ldl_solve(int n, const double* A, const double* b, double* x) {
  double* F = (double*)malloc(sizeof(double) * ((size_t)n * n + 1));
  memcpy(F, A, sizeof(double) * (size_t)n * n);
  memcpy(x, b, sizeof(double) * n);
  int r = ldl(n, F);
  if (r == 0) ldl_solve(n, F, x);
  free(F);
  return r;
}

/* ------------------------------------------------------------------------ */
/* scene                                                                    */
/* ------------------------------------------------------------------------ */

static int ranges(int n, const int* owner, int nb, int* beg, int* end) {
  for (int b = 0; b < nb; ++b) beg[b] = end[b] = 0;
  int prev = -1;
  for (int k = 0; k < n; ++k) {
    int b = owner[k];
    if (b < 0 || b >= nb || b < prev) return -1; /* must be grouped in body order */
    if (b != prev) beg[b] = k;
    end[b] = k + 1;
    prev = b;
  }
  return 0;
}

#define DUP(dst, src, T, n)                 \
  do {                                      \
    dst = (T*)malloc(sizeof(T) * (size_t)((n) > 0 ? (n) : 1)); \
    memcpy(dst, src, sizeof(T) * (size_t)(n)); \
  } while (0)

orc_ctx* orc_create(const orc_scene* s) {
  orc_ctx* c = (orc_ctx*)calloc(1, sizeof(orc_ctx));
  c->sc = *s;
  int nb = s->nb;
  DUP(c->xbar, s->xbar, double, 3 * s->nv);
  DUP(c->tri, s->tri, int, 3 * s->nt);
  DUP(c->edge, s->edge, int, 2 * s->ne);
  DUP(c->vbody, s->vbody, int, s->nv);
  DUP(c->density, s->density, double, nb);
  DUP(c->kappa_body, s->kappa_body, double, nb);
  DUP(c->is_static, s->is_static, unsigned char, nb);
  c->sc.xbar = c->xbar;
  c->sc.tri = c->tri;
  c->sc.edge = c->edge;
  c->sc.vbody = c->vbody;
  c->sc.density = c->density;
  c->sc.kappa_body = c->kappa_body;
  c->sc.is_static = c->is_static;
  c->vbeg = (int*)calloc(nb, sizeof(int));
  c->vend = (int*)calloc(nb, sizeof(int));
  c->tbeg = (int*)calloc(nb, sizeof(int));
  c->tend = (int*)calloc(nb, sizeof(int));
  c->ebeg = (int*)calloc(nb, sizeof(int));
  c->eend = (int*)calloc(nb, sizeof(int));
  int* towner = (int*)malloc(sizeof(int) * (s->nt + 1));
  int* eowner = (int*)malloc(sizeof(int) * (s->ne + 1));
  for (int t = 0; t < s->nt; ++t) towner[t] = s->vbody[s->tri[3 * t]];
  for (int e = 0; e < s->ne; ++e) eowner[e] = s->vbody[s->edge[2 * e]];
  int bad = ranges(s->nv, s->vbody, nb, c->vbeg, c->vend) || ranges(s->nt, towner, nb, c->tbeg, c->tend) ||
            ranges(s->ne, eowner, nb, c->ebeg, c->eend);
  free(towner);
  free(eowner);
  if (bad) {
    orc_destroy(c);
    return NULL;
  }
  c->vol = (double*)calloc(nb, sizeof(double));
  c->m1 = (double*)calloc(3 * nb, sizeof(double));
  c->S = (double*)calloc(9 * nb, sizeof(double));
  c->M = (double*)calloc(144 * nb, sizeof(double));
  for (int b = 0; b < nb; ++b) {
    if (c->is_static[b]) continue;
    orc_body_moments(c, b, &c->vol[b], &c->m1[3 * b], &c->S[9 * b]);
    orc_mass_matrix(c, b, &c->M[144 * b]);
  }
  c->l2e = (double*)calloc(s->ne ? s->ne : 1, sizeof(double));
  for (int e = 0; e < s->ne; ++e) {
    const double* a = c->xbar + 3 * c->edge[2 * e];
    const double* b = c->xbar + 3 * c->edge[2 * e + 1];
    double d0 = b[0] - a[0], d1 = b[1] - a[1], d2 = b[2] - a[2];
    c->l2e[e] = fma(d2, d2, fma(d1, d1, d0 * d0));
  }
  c->qt = (double*)calloc(12 * nb, sizeof(double));
  c->qdot = (double*)calloc(12 * nb, sizeof(double));
  c->qtilde = (double*)calloc(12 * nb, sizeof(double));
  c->diag = (double*)calloc(144 * nb, sizeof(double));
  return c;
}

void orc_destroy(orc_ctx* c) {
  if (!c) return;
  free(c->xbar);
  free(c->l2e);
  free(c->tri);
  free(c->edge);
  free(c->vbody);
  free(c->density);
  free(c->kappa_body);
  free(c->is_static);
  free(c->vbeg);
  free(c->vend);
  free(c->tbeg);
  free(c->tend);
  free(c->ebeg);
  free(c->eend);
  free(c->vol);
  free(c->m1);
  free(c->S);
  free(c->M);
  free(c->qt);
  free(c->qdot);
  free(c->qtilde);
  free(c->fr);
  free(c->diag);
  free(c->bpairs);
  free(c->blocks);
  pl_free(&c->cand);
  pl_free(&c->act);
  free(c);
}

/* ------------------------------------------------------------------------ */
/* Sec. 3: x = A xbar + p.  Canonical order:                                 */
/* x_c = fma(A[c][2], xbar2, fma(A[c][1], xbar1, fma(A[c][0], xbar0, p_c))) */
/* ------------------------------------------------------------------------ */

static void affine_apply(const double* q, const double* xb, double* x) {
  for (int c = 0; c < 3; ++c) {
    const double* a = q + 3 + 3 * c;
    x[c] = fma(a[2], xb[2], fma(a[1], xb[1], fma(a[0], xb[0], q[c])));
  }
}

void orc_vertices(const orc_ctx* c, const double* q, double* x) {
  for (int k = 0; k < c->sc.nv; ++k) affine_apply(q + 12 * c->vbody[k], c->xbar + 3 * k, x + 3 * k);
}

/* J(xbar) dq: the same map applied to a search direction (Sec. 4.1) */
void orc_displacements(const orc_ctx* c, const double* dq, double* dx) { orc_vertices(c, dq, dx); }

/* ------------------------------------------------------------------------ */
/* Sec. 3.1: volume, first and second moments by the divergence theorem:    */
/* the closed, outward-oriented surface is a sum of signed tetrahedra       */
/* (0, v0, v1, v2) with volume det[v0 v1 v2]/6, centroid sum(v)/4 and       */
/* second moment V/20 (sum_i v_i v_i^T + s s^T), s = v0+v1+v2.               */
/* ------------------------------------------------------------------------ */

void orc_body_moments(const orc_ctx* c, int b, double* vol, double m1[3], double S[9]) {
  double V = 0.0, m[3] = {0, 0, 0}, s2[9] = {0};
  for (int t = c->tbeg[b]; t < c->tend[b]; ++t) {
    const double* v0 = c->xbar + 3 * c->tri[3 * t];
    const double* v1 = c->xbar + 3 * c->tri[3 * t + 1];
    const double* v2 = c->xbar + 3 * c->tri[3 * t + 2];
    double det = v0[0] * (v1[1] * v2[2] - v1[2] * v2[1]) - v0[1] * (v1[0] * v2[2] - v1[2] * v2[0]) +
                 v0[2] * (v1[0] * v2[1] - v1[1] * v2[0]);
    double Vt = det / 6.0;
    V += Vt;
    double s[3];
    for (int k = 0; k < 3; ++k) {
      s[k] = v0[k] + v1[k] + v2[k];
      m[k] += Vt * s[k] / 4.0;
    }
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j)
        s2[3 * i + j] += Vt / 20.0 * (v0[i] * v0[j] + v1[i] * v1[j] + v2[i] * v2[j] + s[i] * s[j]);
  }
  *vol = V;
  for (int k = 0; k < 3; ++k) m1[k] = m[k];
  for (int k = 0; k < 9; ++k) S[k] = s2[k];
}

/* DOF index of the coefficient multiplying w_u = (1, xbar)_u in x_c */
static int dof(int u, int cc) { return u == 0 ? cc : 3 + 3 * cc + (u - 1); }

/* M = rho int J^T J: with w = (1, xbar), J[c][dof(u,c)] = w_u, so
 * M[dof(u,c)][dof(v,d)] = rho delta_cd int w_u w_v. */
void orc_mass_matrix(const orc_ctx* c, int b, double M[144]) {
  double W[16];
  const double vol = c->vol[b];
  const double* m1 = c->m1 + 3 * b;
  const double* S = c->S + 9 * b;
  W[0] = vol;
  for (int k = 0; k < 3; ++k) W[1 + k] = W[4 * (1 + k)] = m1[k];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) W[4 * (1 + i) + 1 + j] = S[3 * i + j];
  memset(M, 0, 144 * sizeof(double));
  double rho = c->density[b];
  for (int cc = 0; cc < 3; ++cc)
    for (int u = 0; u < 4; ++u)
      for (int v = 0; v < 4; ++v) M[12 * dof(u, cc) + dof(v, cc)] = rho * W[4 * u + v];
}

/* ------------------------------------------------------------------------ */
/* Sec. 4: qtilde = q^t + dt qdot^t + dt^2 M^-1 f, f = int rho J^T g         */
/* ------------------------------------------------------------------------ */

static void predictor(orc_ctx* c) {
  const orc_scene* s = &c->sc;
  double dt = s->dt;
  for (int b = 0; b < s->nb; ++b) {
    double* qt = c->qtilde + 12 * b;
    const double* q = c->qt + 12 * b;
    const double* v = c->qdot + 12 * b;
    if (c->is_static[b]) {
      for (int k = 0; k < 12; ++k) qt[k] = q[k];
      continue;
    }
    /* f[dof(u,c)] = rho g_c int w_u */
    double W0[4] = {c->vol[b], c->m1[3 * b], c->m1[3 * b + 1], c->m1[3 * b + 2]};
    double f[12], L[144];
    for (int cc = 0; cc < 3; ++cc)
      for (int u = 0; u < 4; ++u) f[dof(u, cc)] = c->density[b] * s->gravity[cc] * W0[u];
    memcpy(L, c->M + 144 * b, sizeof(L));
    chol(12, L);
    chol_solve(12, L, f);
    for (int k = 0; k < 12; ++k) qt[k] = q[k] + dt * v[k] + dt * dt * f[k];
  }
}

/* ------------------------------------------------------------------------ */
/* Sec. 3.2: V = kappa nu |A A^T - I|_F^2 by jets over the 12 coordinates    */
/* ------------------------------------------------------------------------ */

double orc_ortho(const double q[12], double kappa, double vol, double g[12], double H[144]) {
  static jet a[9], acc, t, p, r;
  for (int k = 0; k < 9; ++k) jet_var(&a[k], q[3 + k], 3 + k);
  jet_const(&acc, 0.0);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      /* (A A^T)_ij - delta_ij, rows a_i . a_j */
      jet_mul(&t, &a[3 * i], &a[3 * j]);
      jet_mul(&p, &a[3 * i + 1], &a[3 * j + 1]);
      jet_add(&t, &t, &p);
      jet_mul(&p, &a[3 * i + 2], &a[3 * j + 2]);
      jet_add(&t, &t, &p);
      if (i == j) jet_add_const(&t, &t, -1.0);
      jet_sq(&r, &t);
      jet_add(&acc, &acc, &r);
    }
  jet_scale(&acc, &acc, kappa * vol);
  if (g) memcpy(g, acc.g, 12 * sizeof(double));
  if (H) memcpy(H, acc.h, 144 * sizeof(double));
  return acc.v;
}

/* Per-body IP term E_b = 1/2 (q-qt)^T M (q-qt) + dt^2 V.  Hessian reading:
 * the block M + dt^2 Hess V, used as it is when a Cholesky factorisation
 * succeeds (the block is positive definite).  When it fails, Hess V is
 * replaced by a positive semidefinite surrogate: V = kappa nu |C|_F^2 with
 * C = A A^T - I is a sum of squares, so its Hessian is the Gauss-Newton part
 * (positive semidefinite) plus the residual-curvature part 4 kappa nu C (x) I
 * (over the rows a_k of A); the surrogate keeps the first and clamps the
 * eigenvalues of the 3x3 C in the second, giving
 *   d2/da_k da_l = 4 kappa nu [C+_kl I + delta_kl A^T A + a_l a_k^T],
 * and the block M + dt^2 (surrogate) is positive definite because M is.  It
 * equals the true Hessian whenever C is positive semidefinite. */
static void ortho_hess_psd(const double q[12], double kappa, double vol, double H[144]) {
  double A[3][3], C[9], w[3], V[9], Cp[3][3];
  for (int i = 0; i < 3; ++i)
    for (int c = 0; c < 3; ++c) A[i][c] = q[3 + 3 * i + c];
  for (int k = 0; k < 3; ++k)
    for (int l = 0; l < 3; ++l)
      C[3 * k + l] = A[k][0] * A[l][0] + A[k][1] * A[l][1] + A[k][2] * A[l][2] - (k == l ? 1.0 : 0.0);
  orc_sym_eig(3, C, w, V);
  for (int k = 0; k < 3; ++k)
    for (int l = 0; l < 3; ++l) {
      double t = 0.0;
      for (int c = 0; c < 3; ++c)
        if (w[c] > 0.0) t += V[3 * k + c] * w[c] * V[3 * l + c];
      Cp[k][l] = t;
    }
  const double s4 = 4.0 * kappa * vol;
  for (int i = 0; i < 144; ++i) H[i] = 0.0;
  for (int k = 0; k < 3; ++k)
    for (int l = 0; l < 3; ++l)
      for (int ck = 0; ck < 3; ++ck)
        for (int cl = 0; cl < 3; ++cl) {
          double h = A[l][ck] * A[k][cl];            /* a_l a_k^T */
          if (ck == cl) h += Cp[k][l];               /* C+_kl I */
          if (k == l) h += A[0][ck] * A[0][cl] + A[1][ck] * A[1][cl] + A[2][ck] * A[2][cl];  /* A^T A */
          H[12 * (3 + 3 * k + ck) + 3 + 3 * l + cl] = s4 * h;
        }
}
static double body_terms(orc_ctx* c, int b, const double* q, double* g, double* H, int project, double* Eo) {
  const double* M = c->M + 144 * b;
  const double* qt = c->qtilde + 12 * b;
  double dq[12], Mdq[12];
  for (int k = 0; k < 12; ++k) dq[k] = q[k] - qt[k];
  double Ei = 0.0;
  for (int i = 0; i < 12; ++i) {
    double s = 0.0;
    for (int j = 0; j < 12; ++j) s += M[12 * i + j] * dq[j];
    Mdq[i] = s;
    Ei += 0.5 * dq[i] * s;
  }
  double dt2 = c->sc.dt * c->sc.dt;
  double gv[12], Hv[144];
  double V = orc_ortho(q, c->kappa_body[b], c->vol[b], gv, Hv);
  if (g)
    for (int k = 0; k < 12; ++k) g[k] = Mdq[k] + dt2 * gv[k];
  if (H) {
    /* the body block M + dt^2 hess V; when it is not positive definite
     * (Cholesky fails), M + dt^2 (the surrogate above) */
    for (int k = 0; k < 144; ++k) H[k] = M[k] + dt2 * Hv[k];
    if (project) {
      double L[144];
      memcpy(L, H, sizeof(L));
      if (chol(12, L)) {
        double P[144];
        ortho_hess_psd(q, c->kappa_body[b], c->vol[b], P);
        for (int k = 0; k < 144; ++k) H[k] = M[k] + dt2 * P[k];
      }
    }
  }
  *Eo = dt2 * V;
  return Ei;
}

/* ------------------------------------------------------------------------ */
/* Sec. 4.2: candidate pairs.  A primitive's box is the min/max of its      */
/* vertex positions (over both trajectory ends when swept).  Two boxes P, Q */
/* are a candidate when, on every axis, lo_P - hi_Q <= dhat and             */
/* lo_Q - hi_P <= dhat (each difference rounded once).  Body boxes use the  */
/* same test; since a body box contains its primitives' boxes and rounding   */
/* is monotone, body culling never removes a primitive candidate.           */
/* ------------------------------------------------------------------------ */

typedef struct {
  double lo[3], hi[3];
} box;

static void box_empty(box* b) {
  for (int k = 0; k < 3; ++k) {
    b->lo[k] = INFINITY;
    b->hi[k] = -INFINITY;
  }
}

static void box_add(box* b, const double* p) {
  for (int k = 0; k < 3; ++k) {
    if (p[k] < b->lo[k]) b->lo[k] = p[k];
    if (p[k] > b->hi[k]) b->hi[k] = p[k];
  }
}

static void box_vert(box* b, const double* x0, const double* x1, int v) {
  box_empty(b);
  box_add(b, x0 + 3 * v);
  if (x1) box_add(b, x1 + 3 * v);
}

static int box_near(const box* P, const box* Q, double dhat) {
  for (int k = 0; k < 3; ++k) {
    if (!(P->lo[k] - Q->hi[k] <= dhat)) return 0;
    if (!(Q->lo[k] - P->hi[k] <= dhat)) return 0;
  }
  return 1;
}

typedef struct {
  box* vb;
  box* tb;
  box* eb;
  box* bb;
} boxes;

static void make_boxes(const orc_ctx* c, const double* x0, const double* x1, boxes* B) {
  const orc_scene* s = &c->sc;
  B->vb = (box*)malloc(sizeof(box) * (s->nv + 1));
  B->tb = (box*)malloc(sizeof(box) * (s->nt + 1));
  B->eb = (box*)malloc(sizeof(box) * (s->ne + 1));
  B->bb = (box*)malloc(sizeof(box) * (s->nb + 1));
  for (int v = 0; v < s->nv; ++v) box_vert(&B->vb[v], x0, x1, v);
  for (int t = 0; t < s->nt; ++t) {
    box_empty(&B->tb[t]);
    for (int k = 0; k < 3; ++k) {
      int v = c->tri[3 * t + k];
      box_add(&B->tb[t], x0 + 3 * v);
      if (x1) box_add(&B->tb[t], x1 + 3 * v);
    }
  }
  for (int e = 0; e < s->ne; ++e) {
    box_empty(&B->eb[e]);
    for (int k = 0; k < 2; ++k) {
      int v = c->edge[2 * e + k];
      box_add(&B->eb[e], x0 + 3 * v);
      if (x1) box_add(&B->eb[e], x1 + 3 * v);
    }
  }
  for (int b = 0; b < s->nb; ++b) {
    box_empty(&B->bb[b]);
    for (int v = c->vbeg[b]; v < c->vend[b]; ++v) {
      box_add(&B->bb[b], x0 + 3 * v);
      if (x1) box_add(&B->bb[b], x1 + 3 * v);
    }
  }
}

static void free_boxes(boxes* B) {
  free(B->vb);
  free(B->tb);
  free(B->eb);
  free(B->bb);
}

static void body_pair_candidates(const orc_ctx* c, const boxes* B, int a, int b, plist* out) {
  double dh = c->sc.dhat;
  for (int v = c->vbeg[a]; v < c->vend[a]; ++v)
    for (int t = c->tbeg[b]; t < c->tend[b]; ++t)
      if (box_near(&B->vb[v], &B->tb[t], dh)) pl_push(out, ORC_PT, v, t, -1, 0.0);
  for (int v = c->vbeg[b]; v < c->vend[b]; ++v)
    for (int t = c->tbeg[a]; t < c->tend[a]; ++t)
      if (box_near(&B->vb[v], &B->tb[t], dh)) pl_push(out, ORC_PT, v, t, -1, 0.0);
  for (int e = c->ebeg[a]; e < c->eend[a]; ++e)
    for (int f = c->ebeg[b]; f < c->eend[b]; ++f)
      if (box_near(&B->eb[e], &B->eb[f], dh)) pl_push(out, ORC_EE, e, f, -1, 0.0);
}

static void collect(const orc_ctx* c, const double* x0, const double* x1, int brute, plist* out) {
  const orc_scene* s = &c->sc;
  boxes B;
  make_boxes(c, x0, x1, &B);
  out->n = 0;
  if (brute) {
    double dh = s->dhat;
    for (int v = 0; v < s->nv; ++v)
      for (int t = 0; t < s->nt; ++t) {
        int a = c->vbody[v], b = c->vbody[c->tri[3 * t]];
        if (a == b || (c->is_static[a] && c->is_static[b])) continue;
        if (box_near(&B.vb[v], &B.tb[t], dh)) pl_push(out, ORC_PT, v, t, -1, 0.0);
      }
    for (int e = 0; e < s->ne; ++e)
      for (int f = 0; f < s->ne; ++f) {
        int a = c->vbody[c->edge[2 * e]], b = c->vbody[c->edge[2 * f]];
        if (!(a < b) || (c->is_static[a] && c->is_static[b])) continue;
        if (box_near(&B.eb[e], &B.eb[f], dh)) pl_push(out, ORC_EE, e, f, -1, 0.0);
      }
  } else {
    for (int a = 0; a < s->nb; ++a)
      for (int b = a + 1; b < s->nb; ++b) {
        if (c->is_static[a] && c->is_static[b]) continue;
        if (!box_near(&B.bb[a], &B.bb[b], s->dhat)) continue;
        body_pair_candidates(c, &B, a, b, out);
      }
  }
  free_boxes(&B);
}

long orc_candidates(const orc_ctx* c, const double* x0, const double* x1, int brute, int* kind, int* pi, int* pj,
                    long cap) {
  plist L = {0};
  collect(c, x0, x1, brute, &L);
  for (long k = 0; k < L.n && k < cap; ++k) {
    kind[k] = L.kind[k];
    pi[k] = L.i[k];
    pj[k] = L.j[k];
  }
  long n = L.n;
  pl_free(&L);
  return n;
}

/* the four vertex indices of a pair */
static void pair_verts(const orc_ctx* c, int kind, int i, int j, int v[4]) {
  if (kind == ORC_PT) {
    v[0] = i;
    v[1] = c->tri[3 * j];
    v[2] = c->tri[3 * j + 1];
    v[3] = c->tri[3 * j + 2];
  } else {
    v[0] = c->edge[2 * i];
    v[1] = c->edge[2 * i + 1];
    v[2] = c->edge[2 * j];
    v[3] = c->edge[2 * j + 1];
  }
}

/* mollifier threshold of an edge-edge pair from the rest lengths (0 for a
 * point-triangle pair): eps_x = 1e-3 |rest e_i|^2 |rest e_j|^2 */
static double pair_eps_x(const orc_ctx* c, int kind, int i, int j) {
  if (kind != ORC_EE) return 0.0;
  return (1e-3 * c->l2e[i]) * c->l2e[j];
}

/* mollifier value of a pair at its vertex positions (1 unless a mollified
 * edge-edge pair) */
static double pair_mollifier(const orc_ctx* c, int kind, int i, int j, const double xx[12]) {
  if (kind != ORC_EE) return 1.0;
  return orc_ee_mollifier(orc_ee_cross2(xx), pair_eps_x(c, kind, i, j), NULL, NULL);
}

static void gather12(const double* x, const int v[4], double out[12]) {
  for (int k = 0; k < 4; ++k)
    for (int cc = 0; cc < 3; ++cc) out[3 * k + cc] = x[3 * v[k] + cc];
}

/* ------------------------------------------------------------------------ */
/* Sec. 4 friction: lagged at q^t.  For each pair with d < dhat at q^t:      */
/* lambda = -kappa B'(d) (the contact force magnitude; the paper's           */
/* "-kappa grad B" read as a scalar), closest-point weights gamma (point on  */
/* the first primitive minus point on the second), unit normal n, lagged     */
/* offset r = sum gamma_v x_v^t.  m_j = f0(|P (sum gamma_v x_v - r)|) with   */
/* P = I - n n^T and IPC's C1 mollifier f0 (eps = eps_v dt).                 */
/* ------------------------------------------------------------------------ */

static double seg_param(const double* p, const double* a, const double* b) {
  double e[3], w[3];
  for (int k = 0; k < 3; ++k) {
    e[k] = b[k] - a[k];
    w[k] = p[k] - a[k];
  }
  return (w[0] * e[0] + w[1] * e[1] + w[2] * e[2]) / (e[0] * e[0] + e[1] * e[1] + e[2] * e[2]);
}

static void closest_weights(int kind, int type, const double x[12], double gam[4]) {
  const double *x0 = x, *x1 = x + 3, *x2 = x + 6, *x3 = x + 9;
  for (int k = 0; k < 4; ++k) gam[k] = 0.0;
  if (kind == ORC_PT) {
    double b1 = 0, b2 = 0, b3 = 0, a;
    switch (type) {
      case 0: b1 = 1; break;
      case 1: b2 = 1; break;
      case 2: b3 = 1; break;
      case 3: a = seg_param(x0, x1, x2); b1 = 1 - a; b2 = a; break;
      case 4: a = seg_param(x0, x2, x3); b2 = 1 - a; b3 = a; break;
      case 5: a = seg_param(x0, x3, x1); b3 = 1 - a; b1 = a; break;
      default: {
        double e1[3], e2[3], w[3];
        for (int k = 0; k < 3; ++k) {
          e1[k] = x2[k] - x1[k];
          e2[k] = x3[k] - x1[k];
          w[k] = x0[k] - x1[k];
        }
        double a11 = e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2];
        double a12 = e1[0] * e2[0] + e1[1] * e2[1] + e1[2] * e2[2];
        double a22 = e2[0] * e2[0] + e2[1] * e2[1] + e2[2] * e2[2];
        double r1 = e1[0] * w[0] + e1[1] * w[1] + e1[2] * w[2];
        double r2 = e2[0] * w[0] + e2[1] * w[1] + e2[2] * w[2];
        double det = a11 * a22 - a12 * a12;
        b2 = (r1 * a22 - r2 * a12) / det;
        b3 = (a11 * r2 - a12 * r1) / det;
        b1 = 1 - b2 - b3;
      } break;
    }
    gam[0] = 1.0;
    gam[1] = -b1;
    gam[2] = -b2;
    gam[3] = -b3;
  } else {
    double s = 0, t = 0;
    switch (type) {
      case 0: s = 0; t = 0; break;
      case 1: s = 0; t = 1; break;
      case 2: s = 1; t = 0; break;
      case 3: s = 1; t = 1; break;
      case 4: s = 0; t = seg_param(x0, x2, x3); break;
      case 5: s = 1; t = seg_param(x1, x2, x3); break;
      case 6: t = 0; s = seg_param(x2, x0, x1); break;
      case 7: t = 1; s = seg_param(x3, x0, x1); break;
      default: {
        double e0[3], e1[3], w0[3];
        for (int k = 0; k < 3; ++k) {
          e0[k] = x1[k] - x0[k];
          e1[k] = x3[k] - x2[k];
          w0[k] = x0[k] - x2[k];
        }
        double A = e0[0] * e0[0] + e0[1] * e0[1] + e0[2] * e0[2];
        double B = e0[0] * e1[0] + e0[1] * e1[1] + e0[2] * e1[2];
        double C = e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2];
        double D = e0[0] * w0[0] + e0[1] * w0[1] + e0[2] * w0[2];
        double E = e1[0] * w0[0] + e1[1] * w0[1] + e1[2] * w0[2];
        double den = A * C - B * B;
        s = (B * E - C * D) / den;
        t = (A * E - B * D) / den;
      } break;
    }
    gam[0] = 1 - s;
    gam[1] = s;
    gam[2] = -(1 - t);
    gam[3] = -t;
  }
}

/* closest-point weights of a pair (test hook): the distance type from the
 * canonical classification, then gamma with sum_v gamma_v x_v = (closest
 * point on the first primitive) - (closest point on the second) */
double orc_closest_weights(int kind, const double x[12], double gamma[4], int* type) {
  int t = 0;
  double d2 = orc_pair_dist2(kind, x, &t);
  closest_weights(kind, t, x, gamma);
  if (type) *type = t;
  return d2;
}

/* derivative of the clamped barrier in d */
static double barrier_d1(double d, double dhat) {
  if (d >= dhat) return 0.0;
  double t = d - dhat;
  return -2.0 * t * log(d / dhat) - t * t / d;
}

static void lag_friction(orc_ctx* c) {
  free(c->fr);
  c->fr = NULL;
  c->nfr = 0;
  const orc_scene* s = &c->sc;
  if (!(s->mu > 0.0)) return;
  double* x = (double*)malloc(sizeof(double) * 3 * (s->nv + 1));
  orc_vertices(c, c->qt, x);
  plist L = {0};
  collect(c, x, NULL, 0, &L);
  long cap = L.n ? L.n : 1;
  c->fr = (fpair*)malloc(sizeof(fpair) * cap);
  for (long k = 0; k < L.n; ++k) {
    int v[4], type;
    double xx[12];
    pair_verts(c, L.kind[k], L.i[k], L.j[k], v);
    gather12(x, v, xx);
    double d2 = orc_pair_dist2(L.kind[k], xx, &type);
    if (!(d2 < s->dhat * s->dhat)) continue;
    double d = sqrt(d2);
    /* normal force magnitude; a mollified edge-edge pair carries m(c) */
    double lam = -s->kappa * barrier_d1(d, s->dhat) * pair_mollifier(c, L.kind[k], L.i[k], L.j[k], xx);
    if (!(lam > 0.0)) continue;
    fpair* F = &c->fr[c->nfr++];
    F->kind = L.kind[k];
    F->i = L.i[k];
    F->j = L.j[k];
    F->type = type;
    closest_weights(F->kind, type, xx, F->gamma);
    double dv[3] = {0, 0, 0};
    for (int m = 0; m < 4; ++m)
      for (int cc = 0; cc < 3; ++cc) dv[cc] += F->gamma[m] * xx[3 * m + cc];
    double nn = sqrt(dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2]);
    for (int cc = 0; cc < 3; ++cc) {
      F->n[cc] = dv[cc] / nn;
      F->r[cc] = dv[cc];
    }
    F->mu_lambda = s->mu * lam;
  }
  pl_free(&L);
  free(x);
}

/* mu lambda f0(|P (sum gamma_v x_v - r)|) and its derivatives (jets) */
double orc_friction_pair(const double x[12], const double gamma[4], const double nrm[3], const double r[3],
                         double mu_lambda, double eps, double g[12], double H[144]) {
  static jet u[3], w, t, s, f;
  /* w_c = sum_m gamma_m x_{m,c} - r_c */
  for (int cc = 0; cc < 3; ++cc) {
    jet_const(&u[cc], -r[cc]);
    for (int m = 0; m < 4; ++m) {
      jet_var(&w, x[3 * m + cc], 3 * m + cc);
      jet_scale(&w, &w, gamma[m]);
      jet_add(&u[cc], &u[cc], &w);
    }
  }
  /* tangential part: u - n (n.u) */
  jet_scale(&t, &u[0], nrm[0]);
  jet_scale(&w, &u[1], nrm[1]);
  jet_add(&t, &t, &w);
  jet_scale(&w, &u[2], nrm[2]);
  jet_add(&t, &t, &w);
  jet_const(&s, 0.0);
  for (int cc = 0; cc < 3; ++cc) {
    jet_scale(&w, &t, nrm[cc]);
    jet_sub(&w, &u[cc], &w);
    jet_sq(&w, &w);
    jet_add(&s, &s, &w);
  }
  /* f0 as a function of y^2 = s */
  double sv = s.v;
  if (sv >= eps * eps) {
    double y = sqrt(sv);
    jet_chain(&f, &s, y, 0.5 / y, -0.25 / (y * sv));
  } else {
    double y = sqrt(sv);
    double f0 = -sv * y / (3.0 * eps * eps) + sv / eps + eps / 3.0;
    double f1 = -y / (2.0 * eps * eps) + 1.0 / eps;
    double f2 = sv > 0.0 ? -1.0 / (4.0 * eps * eps * y) : 0.0;
    jet_chain(&f, &s, f0, f1, f2);
  }
  jet_scale(&f, &f, mu_lambda);
  if (g) memcpy(g, f.g, 12 * sizeof(double));
  if (H) memcpy(H, f.h, 144 * sizeof(double));
  return f.v;
}

/* ------------------------------------------------------------------------ */
/* Sec. 4.3: assembly.  For a vertex k of body b, J_k = [I3, I3 (x) xbar_k^T] */
/* (3x12).  Pair blocks J_k^T H_kl J_l go to (b_k, b_l): diagonal blocks per  */
/* body and one off-diagonal block per contacting dynamic body pair (a < b). */
/* Static bodies are fixed: their rows are identity with zero gradient.     */
/* ------------------------------------------------------------------------ */

static void jac(const double* xb, double J[36]) {
  memset(J, 0, 36 * sizeof(double));
  for (int cc = 0; cc < 3; ++cc) {
    J[12 * cc + cc] = 1.0;
    for (int m = 0; m < 3; ++m) J[12 * cc + 3 + 3 * cc + m] = xb[m];
  }
}

static int cmp_pair(const void* A, const void* B) {
  const int* a = (const int*)A;
  const int* b = (const int*)B;
  if (a[0] != b[0]) return a[0] < b[0] ? -1 : 1;
  if (a[1] != b[1]) return a[1] < b[1] ? -1 : 1;
  return 0;
}

static long find_block(const orc_ctx* c, int a, int b) {
  long lo = 0, hi = c->nblk - 1;
  while (lo <= hi) {
    long mid = (lo + hi) / 2;
    int* p = c->bpairs + 2 * mid;
    if (p[0] == a && p[1] == b) return mid;
    if (p[0] < a || (p[0] == a && p[1] < b)) lo = mid + 1;
    else hi = mid - 1;
  }
  return -1;
}

static void add_pair_blocks(orc_ctx* c, const int v[4], const double gx[12], const double Hx[144], double* g,
                            int hess) {
  double J[4][36];
  int bd[4];
  for (int k = 0; k < 4; ++k) {
    bd[k] = c->vbody[v[k]];
    jac(c->xbar + 3 * v[k], J[k]);
  }
  for (int k = 0; k < 4 && g; ++k) {
    if (c->is_static[bd[k]]) continue;
    double* gb = g + 12 * bd[k];
    for (int i = 0; i < 12; ++i) {
      double s = 0.0;
      for (int cc = 0; cc < 3; ++cc) s += J[k][12 * cc + i] * gx[3 * k + cc];
      gb[i] += s;
    }
  }
  for (int k = 0; k < 4 && hess; ++k)
    for (int l = 0; l < 4; ++l) {
      int a = bd[k], b = bd[l];
      if (c->is_static[a] || c->is_static[b] || a > b) continue;
      double* dst = (a == b) ? c->diag + 144 * a : c->blocks + 144 * find_block(c, a, b);
      /* J_k^T H_kl J_l */
      double T[36]; /* H_kl J_l : 3x12 */
      for (int cc = 0; cc < 3; ++cc)
        for (int j = 0; j < 12; ++j) {
          double s = 0.0;
          for (int dd = 0; dd < 3; ++dd) s += Hx[12 * (3 * k + cc) + 3 * l + dd] * J[l][12 * dd + j];
          T[12 * cc + j] = s;
        }
      for (int i = 0; i < 12; ++i)
        for (int j = 0; j < 12; ++j) {
          double s = 0.0;
          for (int cc = 0; cc < 3; ++cc) s += J[k][12 * cc + i] * T[12 * cc + j];
          dst[12 * i + j] += s;
        }
    }
}

/* body pairs (a<b, both dynamic) touched by the active and friction pairs */
static void build_pattern(orc_ctx* c, const plist* act) {
  long cap = 6 * (act->n + c->nfr) + 1;
  int* bp = (int*)malloc(sizeof(int) * 2 * cap);
  long n = 0;
  for (long k = 0; k < act->n + c->nfr; ++k) {
    int v[4];
    if (k < act->n) pair_verts(c, act->kind[k], act->i[k], act->j[k], v);
    else {
      const fpair* F = &c->fr[k - act->n];
      pair_verts(c, F->kind, F->i, F->j, v);
    }
    for (int a = 0; a < 4; ++a)
      for (int b = 0; b < 4; ++b) {
        int ba = c->vbody[v[a]], bb = c->vbody[v[b]];
        if (ba < bb && !c->is_static[ba] && !c->is_static[bb]) {
          if (n == cap) {
            cap *= 2;
            bp = (int*)realloc(bp, sizeof(int) * 2 * cap);
          }
          bp[2 * n] = ba;
          bp[2 * n + 1] = bb;
          n++;
        }
      }
  }
  qsort(bp, n, 2 * sizeof(int), cmp_pair);
  long u = 0;
  for (long k = 0; k < n; ++k)
    if (u == 0 || bp[2 * k] != bp[2 * (u - 1)] || bp[2 * k + 1] != bp[2 * (u - 1) + 1]) {
      bp[2 * u] = bp[2 * k];
      bp[2 * u + 1] = bp[2 * k + 1];
      u++;
    }
  free(c->bpairs);
  free(c->blocks);
  c->bpairs = bp;
  c->nblk = u;
  c->blocks = (double*)calloc(144 * (u ? u : 1), sizeof(double));
}

/* mu lambda f0(|P (sum gamma_v x_v - r)|), value only */
static double friction_value(const double x[12], const fpair* F, double eps) {
  double u[3], t = 0.0;
  for (int cc = 0; cc < 3; ++cc) {
    u[cc] = -F->r[cc];
    for (int m = 0; m < 4; ++m) u[cc] += F->gamma[m] * x[3 * m + cc];
    t += F->n[cc] * u[cc];
  }
  double y2 = 0.0;
  for (int cc = 0; cc < 3; ++cc) {
    double w = u[cc] - t * F->n[cc];
    y2 += w * w;
  }
  double y = sqrt(y2);
  double f0 = y >= eps ? y : -y * y2 / (3.0 * eps * eps) + y2 / eps + eps / 3.0;
  return F->mu_lambda * f0;
}

/* energy (and optionally gradient / Hessian) over the pairs of `cand` */
static int evaluate(orc_ctx* c, const double* q, const plist* cand, double* E, double* g, int hess, int project,
                    plist* act_out) {
  const orc_scene* s = &c->sc;
  double Ein = 0, Eo = 0, Eb = 0, Ef = 0;
  double* x = (double*)malloc(sizeof(double) * 3 * (s->nv + 1));
  orc_vertices(c, q, x);
  plist act = {0};
  for (long k = 0; k < cand->n; ++k) {
    int v[4], type;
    double xx[12];
    pair_verts(c, cand->kind[k], cand->i[k], cand->j[k], v);
    gather12(x, v, xx);
    double d2 = orc_pair_dist2(cand->kind[k], xx, &type);
    if (d2 < s->dhat * s->dhat) pl_push(&act, cand->kind[k], cand->i[k], cand->j[k], type, d2);
  }
  if (g) memset(g, 0, sizeof(double) * 12 * s->nb);
  if (hess) {
    build_pattern(c, &act);
    memset(c->diag, 0, sizeof(double) * 144 * s->nb);
  }
  for (int b = 0; b < s->nb; ++b) {
    if (s->is_static[b]) {
      if (hess)
        for (int i = 0; i < 12; ++i) c->diag[144 * b + 13 * i] = 1.0;
      continue;
    }
    double eo;
    Ein += body_terms(c, b, q + 12 * b, g ? g + 12 * b : NULL, hess ? c->diag + 144 * b : NULL, project, &eo);
    Eo += eo;
  }
  int status = ORC_OK;
  double gx[12], Hx[144];
  for (long k = 0; k < act.n; ++k) {
    int v[4];
    double xx[12], e;
    if (act.d2[k] == 0.0) status = ORC_ERR_INTERSECT;
    pair_verts(c, act.kind[k], act.i[k], act.j[k], v);
    gather12(x, v, xx);
    if (!g && !hess) { /* value only: kappa B(d) m(c) */
      Eb += s->kappa * orc_barrier(sqrt(act.d2[k]), s->dhat) * pair_mollifier(c, act.kind[k], act.i[k], act.j[k], xx);
      continue;
    }
    orc_pair_barrier(act.kind[k], xx, s->dhat, s->kappa, pair_eps_x(c, act.kind[k], act.i[k], act.j[k]), project, &e,
                     gx, Hx);
    Eb += e;
    add_pair_blocks(c, v, gx, Hx, g, hess);
  }
  double eps = s->eps_v * s->dt;
  for (long k = 0; k < c->nfr; ++k) {
    const fpair* F = &c->fr[k];
    int v[4];
    double xx[12];
    pair_verts(c, F->kind, F->i, F->j, v);
    gather12(x, v, xx);
    if (!g && !hess) {
      Ef += friction_value(xx, F, eps);
      continue;
    }
    Ef += orc_friction_pair(xx, F->gamma, F->n, F->r, F->mu_lambda, eps, gx, Hx);
    add_pair_blocks(c, v, gx, Hx, g, hess);
  }
  E[1] = Ein;
  E[2] = Eo;
  E[3] = Eb;
  E[4] = Ef;
  E[0] = ((Ein + Eo) + Eb) + Ef;
  if (act_out) {
    pl_free(act_out);
    *act_out = act;
  } else
    pl_free(&act);
  free(x);
  return status;
}

int orc_energy_grad_hess(orc_ctx* c, const double* q, double* E, double* g, int project) {
  const orc_scene* s = &c->sc;
  double* x = (double*)malloc(sizeof(double) * 3 * (s->nv + 1));
  orc_vertices(c, q, x);
  collect(c, x, NULL, 0, &c->cand);
  free(x);
  double* gs = g ? g : (double*)calloc(12 * s->nb, sizeof(double));
  int st = evaluate(c, q, &c->cand, E, gs, 1, project, &c->act);
  if (!g) free(gs);
  return st;
}

double orc_energy(orc_ctx* c, const double* q) {
  const orc_scene* s = &c->sc;
  double* x = (double*)malloc(sizeof(double) * 3 * (s->nv + 1));
  orc_vertices(c, q, x);
  plist L = {0};
  collect(c, x, NULL, 0, &L);
  free(x);
  double E[5];
  evaluate(c, q, &L, E, NULL, 0, 0, NULL);
  pl_free(&L);
  return E[0];
}

/* active pairs (canonical d^2 < dhat^2) at q, no derivatives */
long orc_active_pairs(orc_ctx* c, const double* q, int* kind, int* pi, int* pj, int* type, double* d2, long cap) {
  const orc_scene* s = &c->sc;
  double* x = (double*)malloc(sizeof(double) * 3 * (s->nv + 1));
  orc_vertices(c, q, x);
  plist L = {0};
  collect(c, x, NULL, 0, &L);
  long n = 0;
  for (long k = 0; k < L.n; ++k) {
    int v[4], ty;
    double xx[12];
    pair_verts(c, L.kind[k], L.i[k], L.j[k], v);
    gather12(x, v, xx);
    double dd = orc_pair_dist2(L.kind[k], xx, &ty);
    if (!(dd < s->dhat * s->dhat)) continue;
    if (n < cap) {
      kind[n] = L.kind[k];
      pi[n] = L.i[k];
      pj[n] = L.j[k];
      type[n] = ty;
      d2[n] = dd;
    }
    ++n;
  }
  pl_free(&L);
  free(x);
  return n;
}

/* gradient rows (12 each) of the selected bodies at q: body terms, every
 * active barrier term and every friction term touching them */
int orc_grad_rows(orc_ctx* c, const double* q, int nsel, const int* sel, double* grows) {
  const orc_scene* s = &c->sc;
  double* g = (double*)calloc(12 * (size_t)s->nb, sizeof(double));
  unsigned char* want = (unsigned char*)calloc(s->nb, 1);
  for (int k = 0; k < nsel; ++k) want[sel[k]] = 1;
  double* x = (double*)malloc(sizeof(double) * 3 * (s->nv + 1));
  orc_vertices(c, q, x);
  for (int k = 0; k < nsel; ++k) {
    int b = sel[k];
    if (s->is_static[b]) continue;
    double eo;
    body_terms(c, b, q + 12 * b, g + 12 * b, NULL, 0, &eo);
  }
  plist L = {0};
  collect(c, x, NULL, 0, &L);
  double gx[12], Hx[144], e;
  int status = ORC_OK;
  for (long k = 0; k < L.n; ++k) {
    int v[4], ty;
    double xx[12];
    pair_verts(c, L.kind[k], L.i[k], L.j[k], v);
    if (!(want[c->vbody[v[0]]] || want[c->vbody[v[3]]])) continue;
    gather12(x, v, xx);
    double dd = orc_pair_dist2(L.kind[k], xx, &ty);
    if (!(dd < s->dhat * s->dhat)) continue;
    if (dd == 0.0) status = ORC_ERR_INTERSECT;
    orc_pair_barrier(L.kind[k], xx, s->dhat, s->kappa, pair_eps_x(c, L.kind[k], L.i[k], L.j[k]), 0, &e, gx, Hx);
    add_pair_blocks(c, v, gx, Hx, g, 0);
  }
  double eps = s->eps_v * s->dt;
  for (long k = 0; k < c->nfr; ++k) {
    const fpair* F = &c->fr[k];
    int v[4];
    double xx[12];
    pair_verts(c, F->kind, F->i, F->j, v);
    if (!(want[c->vbody[v[0]]] || want[c->vbody[v[3]]])) continue;
    gather12(x, v, xx);
    orc_friction_pair(xx, F->gamma, F->n, F->r, F->mu_lambda, eps, gx, Hx);
    add_pair_blocks(c, v, gx, Hx, g, 0);
  }
  for (int k = 0; k < nsel; ++k) memcpy(grows + 12 * k, g + 12 * sel[k], 12 * sizeof(double));
  pl_free(&L);
  free(x);
  free(g);
  free(want);
  return status;
}

long orc_hess_nblocks(const orc_ctx* c) { return c->nblk; }

void orc_hess_copy(const orc_ctx* c, double* diag, int* bpairs, double* blocks) {
  memcpy(diag, c->diag, sizeof(double) * 144 * c->sc.nb);
  memcpy(bpairs, c->bpairs, sizeof(int) * 2 * c->nblk);
  memcpy(blocks, c->blocks, sizeof(double) * 144 * c->nblk);
}

long orc_pairs_count(const orc_ctx* c, int which) {
  if (which == 0) return c->cand.n;
  if (which == 1) return c->act.n;
  return c->nfr;
}

void orc_pairs_copy(const orc_ctx* c, int which, int* kind, int* pi, int* pj, int* type, double* d2) {
  if (which == 2) {
    for (long k = 0; k < c->nfr; ++k) {
      kind[k] = c->fr[k].kind;
      pi[k] = c->fr[k].i;
      pj[k] = c->fr[k].j;
      if (type) type[k] = c->fr[k].type;
      if (d2) d2[k] = c->fr[k].mu_lambda;
    }
    return;
  }
  const plist* L = which == 0 ? &c->cand : &c->act;
  for (long k = 0; k < L->n; ++k) {
    kind[k] = L->kind[k];
    pi[k] = L->i[k];
    pj[k] = L->j[k];
    if (type) type[k] = L->type[k];
    if (d2) d2[k] = L->d2[k];
  }
}

void orc_friction_copy(const orc_ctx* c, double* gamma, double* nrm, double* r) {
  for (long k = 0; k < c->nfr; ++k) {
    for (int m = 0; m < 4; ++m) gamma[4 * k + m] = c->fr[k].gamma[m];
    for (int m = 0; m < 3; ++m) {
      nrm[3 * k + m] = c->fr[k].n[m];
      r[3 * k + m] = c->fr[k].r[m];
    }
  }
}

/* ------------------------------------------------------------------------ */
/* linear solve of the last Hessian: dense Cholesky (the paper's direct LLT) */
/* for small systems, block-Jacobi preconditioned CG otherwise.             */
/* ------------------------------------------------------------------------ */

static void spmv(const orc_ctx* c, const double* v, double* y) {
  int nb = c->sc.nb;
  for (int b = 0; b < nb; ++b)
    for (int i = 0; i < 12; ++i) {
      double s = 0.0;
      for (int j = 0; j < 12; ++j) s += c->diag[144 * b + 12 * i + j] * v[12 * b + j];
      y[12 * b + i] = s;
    }
  for (long k = 0; k < c->nblk; ++k) {
    int a = c->bpairs[2 * k], b = c->bpairs[2 * k + 1];
    const double* B = c->blocks + 144 * k;
    for (int i = 0; i < 12; ++i)
      for (int j = 0; j < 12; ++j) {
        y[12 * a + i] += B[12 * i + j] * v[12 * b + j];
        y[12 * b + j] += B[12 * i + j] * v[12 * a + i];
      }
  }
}

/* indefinite != 0: the dense branch factors by ldl() instead of chol() (the
 * adjoint's unprojected Hessian, which may be indefinite at a converged
 * state; the implicit function theorem needs it nonsingular only) */
static int solve_system(orc_ctx* c, const double* rhs, double* dq, int* iters, int indefinite) {
  const orc_scene* s = &c->sc;
  int nb = s->nb;
  int* idx = (int*)malloc(sizeof(int) * nb);
  int nd = 0;
  for (int b = 0; b < nb; ++b) idx[b] = s->is_static[b] ? -1 : nd++;
  int n = 12 * nd;
  int status = ORC_OK;
  memset(dq, 0, sizeof(double) * 12 * nb);
  *iters = 0;
  if (n <= s->dense_max_dof) {
    double* A = (double*)calloc((size_t)n * n + 1, sizeof(double));
    double* x = (double*)malloc(sizeof(double) * (n + 1));
    for (int b = 0; b < nb; ++b) {
      if (idx[b] < 0) continue;
      for (int i = 0; i < 12; ++i) {
        x[12 * idx[b] + i] = rhs[12 * b + i];
        for (int j = 0; j < 12; ++j) A[(size_t)(12 * idx[b] + i) * n + 12 * idx[b] + j] = c->diag[144 * b + 12 * i + j];
      }
    }
    for (long k = 0; k < c->nblk; ++k) {
      int a = idx[c->bpairs[2 * k]], b = idx[c->bpairs[2 * k + 1]];
      for (int i = 0; i < 12; ++i)
        for (int j = 0; j < 12; ++j) {
          double v = c->blocks[144 * k + 12 * i + j];
          A[(size_t)(12 * a + i) * n + 12 * b + j] = v;
          A[(size_t)(12 * b + j) * n + 12 * a + i] = v;
        }
    }
    if ((indefinite ? ldl(n, A) : chol(n, A)) != 0) status = ORC_ERR_SOLVE;
    else {
      if (indefinite) ldl_solve(n, A, x);
      else chol_solve(n, A, x);
      for (int b = 0; b < nb; ++b)
        if (idx[b] >= 0)
          for (int i = 0; i < 12; ++i) dq[12 * b + i] = x[12 * idx[b] + i];
    }
    free(A);
    free(x);
    free(idx);
    return status;
  }
  /* block-Jacobi PCG */
  size_t N = 12 * (size_t)nb;
  double* L = (double*)malloc(sizeof(double) * 144 * nb);
  double *r = (double*)calloc(N, sizeof(double)), *z = (double*)calloc(N, sizeof(double));
  double *p = (double*)calloc(N, sizeof(double)), *Ap = (double*)calloc(N, sizeof(double));
  for (int b = 0; b < nb; ++b) {
    memcpy(L + 144 * b, c->diag + 144 * b, 144 * sizeof(double));
    if (chol(12, L + 144 * b) != 0) status = ORC_ERR_SOLVE;
  }
  double rr0 = 0.0;
  for (int b = 0; b < nb; ++b)
    for (int i = 0; i < 12; ++i) {
      r[12 * b + i] = idx[b] >= 0 ? rhs[12 * b + i] : 0.0;
      rr0 += r[12 * b + i] * r[12 * b + i];
    }
  double tol2 = s->cg_tol * s->cg_tol * rr0;
  double rz = 0.0;
  for (int b = 0; b < nb; ++b) {
    memcpy(z + 12 * b, r + 12 * b, 12 * sizeof(double));
    if (idx[b] >= 0) chol_solve(12, L + 144 * b, z + 12 * b);
    else memset(z + 12 * b, 0, 12 * sizeof(double));
  }
  for (size_t k = 0; k < N; ++k) {
    p[k] = z[k];
    rz += r[k] * z[k];
  }
  int it = 0;
  double rr = rr0;
  while (rr > tol2 && it < s->cg_max && status == ORC_OK) {
    spmv(c, p, Ap);
    for (int b = 0; b < nb; ++b)
      if (idx[b] < 0) memset(Ap + 12 * b, 0, 12 * sizeof(double));
    double pAp = 0.0;
    for (size_t k = 0; k < N; ++k) pAp += p[k] * Ap[k];
    if (!(pAp > 0.0)) {
      status = ORC_ERR_SOLVE;
      break;
    }
    double alpha = rz / pAp;
    rr = 0.0;
    for (size_t k = 0; k < N; ++k) {
      dq[k] += alpha * p[k];
      r[k] -= alpha * Ap[k];
      rr += r[k] * r[k];
    }
    double rz1 = 0.0;
    for (int b = 0; b < nb; ++b) {
      memcpy(z + 12 * b, r + 12 * b, 12 * sizeof(double));
      if (idx[b] >= 0) chol_solve(12, L + 144 * b, z + 12 * b);
      else memset(z + 12 * b, 0, 12 * sizeof(double));
    }
    for (size_t k = 0; k < N; ++k) rz1 += r[k] * z[k];
    double beta = rz1 / rz;
    rz = rz1;
    for (size_t k = 0; k < N; ++k) p[k] = z[k] + beta * p[k];
    ++it;
  }
  *iters = it;
  free(L);
  free(r);
  free(z);
  free(p);
  free(Ap);
  free(idx);
  return status;
}

int orc_solve(orc_ctx* c, const double* rhs, double* dq, int* iters) { return solve_system(c, rhs, dq, iters, 0); }

/* ------------------------------------------------------------------------ */
/* Sec. 4.1: step-size filter.  Swept candidates over x(q) -> x(q) + J dq,   */
/* ACCD per pair, alpha_max = min time of impact.                           */
/* ------------------------------------------------------------------------ */

static int ccd_over(orc_ctx* c, const double* x, const double* dx, const plist* sw, double* toi) {
  const orc_scene* s = &c->sc;
  double tmin = 1.0;
  int st = ORC_OK;
  for (long k = 0; k < sw->n; ++k) {
    int v[4];
    double xx[12], dd[12], t;
    pair_verts(c, sw->kind[k], sw->i[k], sw->j[k], v);
    gather12(x, v, xx);
    gather12(dx, v, dd);
    int r = orc_accd(sw->kind[k], xx, dd, s->ccd_s, 1.0, s->ccd_max, &t);
    if (r) st = r;
    if (t < tmin) tmin = t;
  }
  *toi = tmin;
  return st;
}

static void swept(orc_ctx* c, const double* q, const double* dq, double* x, double* dx, double* x1, plist* sw) {
  const orc_scene* s = &c->sc;
  orc_vertices(c, q, x);
  orc_displacements(c, dq, dx);
  for (long k = 0; k < 3L * s->nv; ++k) x1[k] = x[k] + dx[k];
  collect(c, x, x1, 0, sw);
}

int orc_ccd_toi(orc_ctx* c, const double* q, const double* dq, double* toi) {
  const orc_scene* s = &c->sc;
  size_t n3 = 3 * (size_t)s->nv + 1;
  double *x = (double*)malloc(sizeof(double) * n3), *dx = (double*)malloc(sizeof(double) * n3);
  double* x1 = (double*)malloc(sizeof(double) * n3);
  plist sw = {0};
  swept(c, q, dq, x, dx, x1, &sw);
  c->st.n_swept = (int)sw.n;
  int st = ccd_over(c, x, dx, &sw, toi);
  pl_free(&sw);
  free(x);
  free(dx);
  free(x1);
  return st;
}

/* ------------------------------------------------------------------------ */
/* state and the time step                                                  */
/* ------------------------------------------------------------------------ */

int orc_set_state(orc_ctx* c, const double* q, const double* qdot) {
  int nb = c->sc.nb;
  memcpy(c->qt, q, sizeof(double) * 12 * nb);
  memcpy(c->qdot, qdot, sizeof(double) * 12 * nb);
  predictor(c);
  lag_friction(c);
  return ORC_OK;
}

void orc_get_state(const orc_ctx* c, double* q, double* qdot) {
  int nb = c->sc.nb;
  if (q) memcpy(q, c->qt, sizeof(double) * 12 * nb);
  if (qdot) memcpy(qdot, c->qdot, sizeof(double) * 12 * nb);
}

void orc_get_qtilde(const orc_ctx* c, double* qtilde) { memcpy(qtilde, c->qtilde, sizeof(double) * 12 * c->sc.nb); }

/* One implicit-Euler step (Sec. 4; integrator reading: implicit Euler):
 * minimise E from q = q^t by Newton with the projected Hessian; stop when
 * the largest vertex displacement of the Newton step is <= newton_tol
 * (tested before the line search); otherwise alpha = CCD bound, halved until
 * E(q + alpha dq) <= E(q) + slack; finally qdot = (q - q^t) / dt. */
static int one_step(orc_ctx* c, orc_stats* st) {
  const orc_scene* s = &c->sc;
  int nb = s->nb;
  size_t N = 12 * (size_t)nb, n3 = 3 * (size_t)s->nv + 1;
  double* q = (double*)malloc(sizeof(double) * N);
  double* qn = (double*)malloc(sizeof(double) * N);
  double* g = (double*)malloc(sizeof(double) * N);
  double* dq = (double*)malloc(sizeof(double) * N);
  double* rhs = (double*)malloc(sizeof(double) * N);
  double *x = (double*)malloc(sizeof(double) * n3), *dx = (double*)malloc(sizeof(double) * n3);
  double* x1 = (double*)malloc(sizeof(double) * n3);
  memcpy(q, c->qt, sizeof(double) * N);
  memset(st, 0, sizeof(*st));
  st->toi_min = 1.0;
  int status = ORC_ERR_NEWTON;
  plist sw = {0};
  for (int it = 0; it < s->newton_max; ++it) {
    double E[5];
    int r = orc_energy_grad_hess(c, q, E, g, 1);
    if (r) {
      status = r;
      break;
    }
    st->n_candidates = (int)c->cand.n;
    st->n_active = (int)c->act.n;
    for (size_t k = 0; k < N; ++k) rhs[k] = -g[k];
    int its;
    r = orc_solve(c, rhs, dq, &its);
    st->solve_iters += its;
    if (r) {
      status = r;
      break;
    }
    orc_displacements(c, dq, dx);
    double m = 0.0;
    for (int v = 0; v < s->nv; ++v) {
      if (s->is_static[c->vbody[v]]) continue;
      double n2 = sqrt(dx[3 * v] * dx[3 * v] + dx[3 * v + 1] * dx[3 * v + 1] + dx[3 * v + 2] * dx[3 * v + 2]);
      if (n2 > m) m = n2;
    }
    st->last_step = m;
    if (m <= s->newton_tol) {
      status = ORC_OK;
      break;
    }
    st->newton_iters++;
    swept(c, q, dq, x, dx, x1, &sw);
    st->n_swept = (int)sw.n;
    double alpha;
    r = ccd_over(c, x, dx, &sw, &alpha);
    if (r) {
      status = r;
      break;
    }
    if (alpha < st->toi_min) st->toi_min = alpha;
    double E0[5], En[5];
    evaluate(c, q, &sw, E0, NULL, 0, 0, NULL);
    double slack = s->ls_slack_rel * (fabs(E0[0]) + 1.0);
    int ok = 0;
    for (int ls = 0; ls <= s->ls_max; ++ls) {
      for (size_t k = 0; k < N; ++k) qn[k] = q[k] + alpha * dq[k];
      evaluate(c, qn, &sw, En, NULL, 0, 0, NULL);
      if (En[0] <= E0[0] + slack) {
        ok = 1;
        break;
      }
      alpha *= 0.5;
      st->ls_halvings++;
    }
    if (!ok) {
      status = ORC_ERR_LINESEARCH;
      break;
    }
    memcpy(q, qn, sizeof(double) * N);
  }
  pl_free(&sw);
  if (status == ORC_OK) {
    for (size_t k = 0; k < N; ++k) {
      double v = (q[k] - c->qt[k]) / s->dt;
      c->qdot[k] = v;
      c->qt[k] = q[k];
    }
    for (int b = 0; b < nb; ++b)
      if (s->is_static[b])
        for (int k = 0; k < 12; ++k) c->qdot[12 * b + k] = 0.0;
    predictor(c);
    lag_friction(c);
    st->n_friction = (int)c->nfr;
  }
  free(q);
  free(qn);
  free(g);
  free(dq);
  free(rhs);
  free(x);
  free(dx);
  free(x1);
  return status;
}

int orc_step(orc_ctx* c, int nsteps, orc_stats* st) {
  orc_stats tmp;
  for (int k = 0; k < nsteps; ++k) {
    int r = one_step(c, st ? st : &tmp);
    if (r) return r;
  }
  return ORC_OK;
}


/* ------------------------------------------------------------------------ */
/* Adjoint of one step by the implicit function theorem.  The step's q^{t+1} */
/* minimises E(q; q~) with q~ = q^t + dt qdot^t + dt^2 g, so grad E(q^{t+1}) */
/* = 0 and, with H the unprojected Hessian there and H lam = dL/dq^{t+1},    */
/* dL/dq~ = M lam and dL/dkappa_b = -dt^2 lam_b . grad V_b / kappa_b.  The   */
/* lagged friction quantities are held fixed (their dependence on q^t is     */
/* not differentiated).  Returns M lam per body (zero rows for static        */
/* bodies) and dL/dkappa per body.  q^{t+1} is a stationary point of E,    */
/* not always a minimiser (H can have a small negative eigenvalue there);    */
/* the theorem needs H nonsingular only, so the dense solve is LDL^T.        */
/* ------------------------------------------------------------------------ */
int orc_adjoint_step(orc_ctx* c, const double* q_t, const double* qdot_t, const double* q_next, const double* rhs,
                     double* Mlam, double* gkappa) {
  const orc_scene* s = &c->sc;
  const int nb = s->nb;
  int st = orc_set_state(c, q_t, qdot_t);
  if (st != ORC_OK) return st;
  double E[5];
  double* g = (double*)calloc(12 * (size_t)nb, sizeof(double));
  double* lam = (double*)calloc(12 * (size_t)nb, sizeof(double));
  st = orc_energy_grad_hess(c, q_next, E, g, 0);
  int iters = 0;
  if (st == ORC_OK) st = solve_system(c, rhs, lam, &iters, 1);
  const double dt2 = s->dt * s->dt;
  for (int b = 0; b < nb; ++b) {
    double* o = Mlam + 12 * b;
    gkappa[b] = 0.0;
    if (s->is_static[b] || st != ORC_OK) {
      memset(o, 0, 12 * sizeof(double));
      continue;
    }
    const double* M = c->M + 144 * b;
    const double* l = lam + 12 * b;
    for (int i = 0; i < 12; ++i) {
      double t = 0.0;
      for (int j = 0; j < 12; ++j) t += M[12 * i + j] * l[j];
      o[i] = t;
    }
    double gv[12], Hv[144];
    orc_ortho(q_next + 12 * b, c->kappa_body[b], c->vol[b], gv, Hv);
    double t = 0.0;
    for (int i = 0; i < 12; ++i) t += l[i] * gv[i];
    gkappa[b] = -dt2 * t / c->kappa_body[b];
  }
  free(g);
  free(lam);
  return st;
}

