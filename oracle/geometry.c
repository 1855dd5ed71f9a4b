/* Oracle geometry: primitive distances, distance-type classification, the
 * clamped log barrier and its derivatives, PSD projection, additive CCD.
 *
 * TEST INFRASTRUCTURE ONLY: part of the CPU oracle.  Only tests, the smoke
 * check and the benchmark's CPU baseline may load it.
 *
 * Canonical floating point.  Every quantity that decides a set membership or a
 * step size (squared distances, distance types, ACCD) is evaluated with the
 * operation order written here, with contraction disabled at compile time
 * (-ffp-contract=off) and fused multiply-adds only where fma() is called:
 *   sub(a,b)   = (a0-b0, a1-b1, a2-b2)
 *   dot(a,b)   = fma(a2,b2, fma(a1,b1, a0*b0))
 *   cross(a,b) = (a1*b2 - a2*b1, a2*b0 - a0*b2, a0*b1 - a1*b0)
 * The same order is specified for the CUDA path, so the pair sets and
 * time-of-impact values of both sides can be compared bit for bit.
 */
#include <math.h>
#include <string.h>

#include "abd_oracle.h"
#include "jet.h"

/* ------------------------------------------------------------------------ */
/* canonical vector helpers                                                 */
/* ------------------------------------------------------------------------ */

static void vsub(double r[3], const double a[3], const double b[3]) {
  r[0] = a[0] - b[0];
  r[1] = a[1] - b[1];
  r[2] = a[2] - b[2];
}

static double vdot(const double a[3], const double b[3]) { return fma(a[2], b[2], fma(a[1], b[1], a[0] * b[0])); }

static void vcross(double r[3], const double a[3], const double b[3]) {
  double t0 = a[1] * b[2] - a[2] * b[1];
  double t1 = a[2] * b[0] - a[0] * b[2];
  double t2 = a[0] * b[1] - a[1] * b[0];
  r[0] = t0;
  r[1] = t1;
  r[2] = t2;
}

/* ------------------------------------------------------------------------ */
/* squared distances of the elementary types                                */
/* ------------------------------------------------------------------------ */

double orc_d2_pp(const double p[3], const double q[3]) {
  double e[3];
  vsub(e, p, q);
  return vdot(e, e);
}

/* distance from p to the line through a and b: |(a-p) x (b-p)|^2 / |b-a|^2 */
double orc_d2_pe(const double p[3], const double a[3], const double b[3]) {
  double u[3], v[3], c[3], e[3];
  vsub(u, a, p);
  vsub(v, b, p);
  vcross(c, u, v);
  vsub(e, b, a);
  return vdot(c, c) / vdot(e, e);
}

/* distance from p to the plane through a, b, c: ((p-a).n)^2 / |n|^2 */
double orc_d2_pt_plane(const double p[3], const double a[3], const double b[3], const double c[3]) {
  double ab[3], ac[3], n[3], ap[3];
  vsub(ab, b, a);
  vsub(ac, c, a);
  vcross(n, ab, ac);
  vsub(ap, p, a);
  double t = vdot(ap, n);
  return (t * t) / vdot(n, n);
}

/* distance between the lines through (a,b) and (c,d): ((c-a).n)^2/|n|^2 */
double orc_d2_ee_line(const double a[3], const double b[3], const double c[3], const double d[3]) {
  double e0[3], e1[3], n[3], w[3];
  vsub(e0, b, a);
  vsub(e1, d, c);
  vcross(n, e0, e1);
  vsub(w, c, a);
  double t = vdot(w, n);
  return (t * t) / vdot(n, n);
}

/* point p against the segment [a,b]: 0 -> closest is a, 1 -> b, 2 -> interior */
static double point_segment(const double p[3], const double a[3], const double b[3], int* branch) {
  double e[3], w[3];
  vsub(e, b, a);
  vsub(w, p, a);
  double t = vdot(w, e);
  if (t <= 0.0) {
    *branch = 0;
    return orc_d2_pp(p, a);
  }
  if (t >= vdot(e, e)) {
    *branch = 1;
    return orc_d2_pp(p, b);
  }
  *branch = 2;
  return orc_d2_pe(p, a, b);
}

/* Point x0 against triangle (x1, x2, x3).  Types:
 *   0,1,2: point-point with x1, x2, x3;  3,4,5: point-edge with (x1,x2),
 *   (x2,x3), (x3,x1);  6: point-plane (projection inside the triangle). */
double orc_pt_dist2(const double x0[3], const double x1[3], const double x2[3], const double x3[3], int* type) {
  double e01[3], e12[3], e20[3], n[3], w[3], c[3];
  vsub(e01, x2, x1);
  vsub(e12, x3, x2);
  vsub(e20, x1, x3);
  double ac[3];
  vsub(ac, x3, x1);
  vcross(n, e01, ac);
  int inside = 1;
  vsub(w, x0, x1);
  vcross(c, e01, w);
  if (vdot(c, n) < 0.0) inside = 0;
  vsub(w, x0, x2);
  vcross(c, e12, w);
  if (vdot(c, n) < 0.0) inside = 0;
  vsub(w, x0, x3);
  vcross(c, e20, w);
  if (vdot(c, n) < 0.0) inside = 0;
  if (inside) {
    *type = 6;
    return orc_d2_pt_plane(x0, x1, x2, x3);
  }
  static const int map[3][3] = {{0, 1, 3}, {1, 2, 4}, {2, 0, 5}};
  const double* ea[3] = {x1, x2, x3};
  const double* eb[3] = {x2, x3, x1};
  double best = 0.0;
  int bt = -1;
  for (int k = 0; k < 3; ++k) {
    int br;
    double d2 = point_segment(x0, ea[k], eb[k], &br);
    if (bt < 0 || d2 < best) {
      best = d2;
      bt = map[k][br];
    }
  }
  *type = bt;
  return best;
}

/* Edge (x0,x1) against edge (x2,x3).  Types:
 *   0: x0-x2, 1: x0-x3, 2: x1-x2, 3: x1-x3 (point-point);
 *   4: x0-(x2,x3), 5: x1-(x2,x3), 6: x2-(x0,x1), 7: x3-(x0,x1) (point-edge);
 *   8: line-line (both closest points interior). */
double orc_ee_dist2(const double x0[3], const double x1[3], const double x2[3], const double x3[3], int* type) {
  double e0[3], e1[3], n[3], w0[3];
  vsub(e0, x1, x0);
  vsub(e1, x3, x2);
  vcross(n, e0, e1);
  double nn = vdot(n, n);
  double A = vdot(e0, e0), C = vdot(e1, e1);
  int parallel = nn <= (1e-20 * A) * C;
  if (!parallel) {
    vsub(w0, x0, x2);
    double B = vdot(e0, e1), D = vdot(e0, w0), E = vdot(e1, w0);
    double den = A * C - B * B;
    double sn = B * E - C * D;
    double tn = A * E - B * D;
    if (sn > 0.0 && sn < den && tn > 0.0 && tn < den) {
      *type = 8;
      return orc_d2_ee_line(x0, x1, x2, x3);
    }
  }
  static const int map[4][3] = {{0, 1, 4}, {2, 3, 5}, {0, 2, 6}, {1, 3, 7}};
  const double* pp[4] = {x0, x1, x2, x3};
  const double* sa[4] = {x2, x2, x0, x0};
  const double* sb[4] = {x3, x3, x1, x1};
  double best = 0.0;
  int bt = -1;
  for (int k = 0; k < 4; ++k) {
    int br;
    double d2 = point_segment(pp[k], sa[k], sb[k], &br);
    if (bt < 0 || d2 < best) {
      best = d2;
      bt = map[k][br];
    }
  }
  *type = bt;
  return best;
}

double orc_pair_dist2(int kind, const double x[12], int* type) {
  if (kind == ORC_PT) return orc_pt_dist2(x, x + 3, x + 6, x + 9, type);
  return orc_ee_dist2(x, x + 3, x + 6, x + 9, type);
}

/* ------------------------------------------------------------------------ */
/* squared distance of a given type as a jet over the 12 pair coordinates   */
/* ------------------------------------------------------------------------ */

static void jet_d2_pp(jet* r, const jet3* p, const jet3* q) {
  jet3 e;
  jet3_sub(&e, p, q);
  jet3_dot(r, &e, &e);
}

static void jet_d2_pe(jet* r, const jet3* p, const jet3* a, const jet3* b) {
  jet3 u, v, c, e;
  jet n2, e2;
  jet3_sub(&u, a, p);
  jet3_sub(&v, b, p);
  jet3_cross(&c, &u, &v);
  jet3_sub(&e, b, a);
  jet3_dot(&n2, &c, &c);
  jet3_dot(&e2, &e, &e);
  jet_div(r, &n2, &e2);
}

static void jet_d2_plane(jet* r, const jet3* p, const jet3* a, const jet3* b, const jet3* c) {
  jet3 ab, ac, n, ap;
  jet t, t2, nn;
  jet3_sub(&ab, b, a);
  jet3_sub(&ac, c, a);
  jet3_cross(&n, &ab, &ac);
  jet3_sub(&ap, p, a);
  jet3_dot(&t, &ap, &n);
  jet_sq(&t2, &t);
  jet3_dot(&nn, &n, &n);
  jet_div(r, &t2, &nn);
}

/* r = squared distance of the given type, as a jet over x (12 coordinates) */
void orc_jet_pair_d2(jet* r, int kind, int type, const double x[12]) {
  jet3 v[4];
  for (int k = 0; k < 4; ++k) jet3_var(&v[k], x + 3 * k, 3 * k);
  if (kind == ORC_PT) {
    switch (type) {
      case 0: jet_d2_pp(r, &v[0], &v[1]); break;
      case 1: jet_d2_pp(r, &v[0], &v[2]); break;
      case 2: jet_d2_pp(r, &v[0], &v[3]); break;
      case 3: jet_d2_pe(r, &v[0], &v[1], &v[2]); break;
      case 4: jet_d2_pe(r, &v[0], &v[2], &v[3]); break;
      case 5: jet_d2_pe(r, &v[0], &v[3], &v[1]); break;
      default: jet_d2_plane(r, &v[0], &v[1], &v[2], &v[3]); break;
    }
  } else {
    switch (type) {
      case 0: jet_d2_pp(r, &v[0], &v[2]); break;
      case 1: jet_d2_pp(r, &v[0], &v[3]); break;
      case 2: jet_d2_pp(r, &v[1], &v[2]); break;
      case 3: jet_d2_pp(r, &v[1], &v[3]); break;
      case 4: jet_d2_pe(r, &v[0], &v[2], &v[3]); break;
      case 5: jet_d2_pe(r, &v[1], &v[2], &v[3]); break;
      case 6: jet_d2_pe(r, &v[2], &v[0], &v[1]); break;
      case 7: jet_d2_pe(r, &v[3], &v[0], &v[1]); break;
      default: {
        /* line-line: ((x2-x0).n)^2/|n|^2 with n = (x1-x0) x (x3-x2) */
        jet3 e0, e1, n, w;
        jet t, t2, nn;
        jet3_sub(&e0, &v[1], &v[0]);
        jet3_sub(&e1, &v[3], &v[2]);
        jet3_cross(&n, &e0, &e1);
        jet3_sub(&w, &v[2], &v[0]);
        jet3_dot(&t, &w, &n);
        jet_sq(&t2, &t);
        jet3_dot(&nn, &n, &n);
        jet_div(r, &t2, &nn);
      } break;
    }
  }
}

/* ------------------------------------------------------------------------ */
/* clamped log barrier, Eq. clamped-b: B(d) = -(d - dhat)^2 ln(d / dhat)     */
/* ------------------------------------------------------------------------ */

double orc_barrier(double d, double dhat) {
  if (d >= dhat) return 0.0;
  double t = d - dhat;
  return -(t * t) * log(d / dhat);
}

/* ------------------------------------------------------------------------ */
/* near-parallel edge-edge mollifier (IPC, Li et al. 2020): with              */
/* c = |e0 x e1|^2 and eps_x = 1e-3 |rest e0|^2 |rest e1|^2, the edge-edge    */
/* barrier is multiplied by m(c) = -c^2/eps_x^2 + 2c/eps_x for c < eps_x and  */
/* by 1 otherwise, so that it fades out (C1) as the two edges turn parallel,  */
/* where the line-line distance loses its conditioning.                       */
/* ------------------------------------------------------------------------ */

double orc_ee_cross2(const double x[12]) {
  double e0[3], e1[3], n[3];
  vsub(e0, x + 3, x);
  vsub(e1, x + 9, x + 6);
  vcross(n, e0, e1);
  return vdot(n, n);
}

double orc_ee_mollifier(double c, double eps_x, double* dm, double* d2m) {
  if (!(c < eps_x)) {
    if (dm) *dm = 0.0;
    if (d2m) *d2m = 0.0;
    return 1.0;
  }
  double r = c / eps_x;
  if (dm) *dm = (2.0 - 2.0 * r) / eps_x;
  if (d2m) *d2m = -2.0 / (eps_x * eps_x);
  return (2.0 - r) * r;
}

/* kappa * B(d(x)) with gradient and Hessian over the 12 coordinates, taken
 * by jets through d = sqrt(d^2) of the pair's distance type; the Hessian is
 * projected to the PSD cone when project != 0.  An edge-edge pair with
 * eps_x > 0 and |e0 x e1|^2 < eps_x carries the mollifier factor m above.
 * Returns 0 for an inactive pair (d^2 >= dhat^2), 1 otherwise. */
int orc_pair_barrier(int kind, const double x[12], double dhat, double kappa, double eps_x, int project,
                     double* E, double g[12], double H[144]) {
  int type;
  double d2 = orc_pair_dist2(kind, x, &type);
  *E = 0.0;
  memset(g, 0, 12 * sizeof(double));
  memset(H, 0, 144 * sizeof(double));
  if (!(d2 < dhat * dhat)) return 0;
  static jet s, d, t, t2, l, b;  /* large structs: static to keep the stack small */
  orc_jet_pair_d2(&s, kind, type, x);
  /* the barrier is a function of the distance; its value is the canonical
   * d^2 (the one that decides membership), its derivatives those of the
   * type's formula (near d-hat, B ~ (d - dhat)^2 amplifies any difference in
   * d by dhat / (dhat - d)) */
  s.v = d2;
  jet_sqrt(&d, &s);
  jet_add_const(&t, &d, -dhat);
  jet_sq(&t2, &t);
  jet_scale(&l, &d, 1.0 / dhat);
  jet_log(&l, &l);
  jet_mul(&b, &t2, &l);
  jet_scale(&b, &b, -kappa);
  if (kind == ORC_EE && eps_x > 0.0) {
    double c = orc_ee_cross2(x);
    if (c < eps_x) {
      /* m(c(x)) as a jet: c = |(x1 - x0) x (x3 - x2)|^2 */
      static jet3 v[4], e0, e1, n;
      static jet cj, mj, bm;
      for (int k = 0; k < 4; ++k) jet3_var(&v[k], x + 3 * k, 3 * k);
      jet3_sub(&e0, &v[1], &v[0]);
      jet3_sub(&e1, &v[3], &v[2]);
      jet3_cross(&n, &e0, &e1);
      jet3_dot(&cj, &n, &n);
      cj.v = c; /* canonical value, as for d^2 */
      double dm, d2m;
      double mv = orc_ee_mollifier(cj.v, eps_x, &dm, &d2m);
      jet_chain(&mj, &cj, mv, dm, d2m);
      jet_mul(&bm, &b, &mj);
      b = bm;
    }
  }
  *E = b.v;
  memcpy(g, b.g, 12 * sizeof(double));
  memcpy(H, b.h, 144 * sizeof(double));
  if (project) orc_project_psd(12, H);
  return 1;
}

/* ------------------------------------------------------------------------ */
/* PSD projection: symmetric eigen-decomposition by cyclic Jacobi rotations, */
/* negative eigenvalues clamped to zero, matrix rebuilt from the eigenpairs. */
/* ------------------------------------------------------------------------ */

void orc_sym_eig(int n, const double* A, double* w, double* V) {
  double W[144];
  for (int i = 0; i < n * n; ++i) W[i] = A[i];
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) V[i * n + j] = (i == j) ? 1.0 : 0.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        double a2 = W[i * n + j] * W[i * n + j];
        tot += a2;
        if (i != j) off += a2;
      }
    if (off <= 1e-36 * tot || off == 0.0) break;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        double apq = W[p * n + q];
        if (apq == 0.0) continue;
        double theta = (W[q * n + q] - W[p * n + p]) / (2.0 * apq);
        double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
        double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < n; ++k) { /* columns p, q */
          double wkp = W[k * n + p], wkq = W[k * n + q];
          W[k * n + p] = c * wkp - s * wkq;
          W[k * n + q] = s * wkp + c * wkq;
        }
        for (int k = 0; k < n; ++k) { /* rows p, q */
          double wpk = W[p * n + k], wqk = W[q * n + k];
          W[p * n + k] = c * wpk - s * wqk;
          W[q * n + k] = s * wpk + c * wqk;
        }
        for (int k = 0; k < n; ++k) {
          double vkp = V[k * n + p], vkq = V[k * n + q];
          V[k * n + p] = c * vkp - s * vkq;
          V[k * n + q] = s * vkp + c * vkq;
        }
      }
  }
  for (int i = 0; i < n; ++i) w[i] = W[i * n + i];
}

void orc_project_psd(int n, double* A) {
  double w[12], V[144];
  orc_sym_eig(n, A, w, V);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      double s = 0.0;
      for (int k = 0; k < n; ++k)
        if (w[k] > 0.0) s += V[i * n + k] * w[k] * V[j * n + k];
      A[i * n + j] = s;
    }
}

/* ------------------------------------------------------------------------ */
/* Additive CCD (Sec. 4.1 uses ACCD of Li et al., Codimensional IPC):       */
/* conservative advancement of the linear trajectory x + t dx, t in [0, 1]. */
/* ------------------------------------------------------------------------ */

int orc_accd(int kind, const double x_in[12], const double dx[12], double s, double tmax, int max_iter,
             double* toi) {
  double x[12], p[12];
  double mean[3];
  for (int c = 0; c < 3; ++c) mean[c] = ((dx[c] + dx[3 + c]) + (dx[6 + c] + dx[9 + c])) * 0.25;
  for (int k = 0; k < 4; ++k)
    for (int c = 0; c < 3; ++c) {
      p[3 * k + c] = dx[3 * k + c] - mean[c];
      x[3 * k + c] = x_in[3 * k + c];
    }
  double n0 = sqrt(vdot(p, p)), n1 = sqrt(vdot(p + 3, p + 3));
  double n2 = sqrt(vdot(p + 6, p + 6)), n3 = sqrt(vdot(p + 9, p + 9));
  double lp;
  if (kind == ORC_PT) {
    double m = n1 > n2 ? n1 : n2;
    m = m > n3 ? m : n3;
    lp = n0 + m;
  } else {
    double ma = n0 > n1 ? n0 : n1;
    double mb = n2 > n3 ? n2 : n3;
    lp = ma + mb;
  }
  if (lp == 0.0) {
    *toi = tmax;
    return 0;
  }
  int type;
  double d = sqrt(orc_pair_dist2(kind, x, &type));
  if (d == 0.0) {
    *toi = 0.0;
    return 0;
  }
  double g = s * d;
  double t = 0.0;
  double tl = ((1.0 - s) * d) / lp;
  for (int it = 0; it < max_iter; ++it) {
    for (int k = 0; k < 12; ++k) x[k] = x[k] + tl * p[k];
    d = sqrt(orc_pair_dist2(kind, x, &type));
    if (t > 0.0 && d < g) {
      *toi = t;
      return 0;
    }
    t = t + tl;
    if (t > tmax) {
      *toi = tmax;
      return 0;
    }
    tl = (0.9 * d) / lp;
  }
  *toi = t;
  return ORC_ERR_CCD;
}
