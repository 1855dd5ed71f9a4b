// Gradient and PSD-projected Hessian of one contact term in vertex space
// (12 coordinates: 4 vertices x 3).
//
// Barrier (Sec. 4, Eq. barrier and Eq. clamped-b): kappa * B(d), d = sqrt(s)
// with s the squared distance of the pair's distance type.  Every type's s is
// a function of a few difference vectors r = C x (C a 4 x m matrix with
// entries in {-1, 0, 1}, m = 1 point-point, 2 point-edge, 3 point-plane and
// line-line), so the Hessian has the form T H_r T^T with T = C (x) I3.  The
// PSD projection is taken in that m*3-dimensional space: with C = Q R
// (Q orthonormal columns), Proj(T H_r T^T) = T R^-1 Proj(R H_r R^T) R^-T T^T,
// which is exactly the eigenvalue clamp of the full 12x12 matrix at a
// fraction of the cost (a 9x9 instead of a 12x12 symmetric eigenproblem).
//
// Friction (Sec. 4, V_F = sum mu lambda_j m_j): m_j = f0(|P (sum gamma_v x_v
// - r)|), lagged normal n, P = I - n n^T, IPC's C1 mollifier f0 with
// eps = eps_v dt.  Its Hessian is PSD by construction.
#pragma once
#include <math.h>

#include "geom.cuh"

#ifndef ABD_HD
#define ABD_HD __host__ __device__ __forceinline__
#endif

namespace abd {

// packed upper triangle of a symmetric 12x12 matrix
ABD_HD int up12(int i, int j) { return i <= j ? i * 12 - (i * (i - 1)) / 2 + (j - i) : j * 12 - (j * (j - 1)) / 2 + (i - j); }

// ---------------------------------------------------------------------------
// symmetric eigen-decomposition by cyclic Jacobi rotations (n <= 9)
// A (n x n, row-major) is destroyed: its diagonal holds the eigenvalues;
// V receives the eigenvectors as columns.
// ---------------------------------------------------------------------------
template <int N, typename T>
ABD_HD void jacobi_eig(T* A, T* V) {
  for (int i = 0; i < N; ++i)
    for (int j = 0; j < N; ++j) V[i * N + j] = (i == j) ? T(1) : T(0);
  for (int sweep = 0; sweep < 16; ++sweep) {
    T off = 0, tot = 0;
    for (int i = 0; i < N; ++i)
      for (int j = 0; j < N; ++j) {
        T a2 = A[i * N + j] * A[i * N + j];
        tot += a2;
        if (i != j) off += a2;
      }
    if (!(off > tot * T(sizeof(T) == 8 ? 1e-32 : 1e-14))) break;
    for (int p = 0; p < N - 1; ++p)
      for (int q = p + 1; q < N; ++q) {
        T apq = A[p * N + q];
        if (apq == T(0)) continue;
        T theta = (A[q * N + q] - A[p * N + p]) / (T(2) * apq);
        T t = (theta >= T(0) ? T(1) : T(-1)) / (fabs(theta) + sqrt(theta * theta + T(1)));
        T c = T(1) / sqrt(t * t + T(1)), s = t * c;
        for (int k = 0; k < N; ++k) {
          T akp = A[k * N + p], akq = A[k * N + q];
          A[k * N + p] = c * akp - s * akq;
          A[k * N + q] = s * akp + c * akq;
        }
        for (int k = 0; k < N; ++k) {
          T apk = A[p * N + k], aqk = A[q * N + k];
          A[p * N + k] = c * apk - s * aqk;
          A[q * N + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < N; ++k) {
          T vkp = V[k * N + p], vkq = V[k * N + q];
          V[k * N + p] = c * vkp - s * vkq;
          V[k * N + q] = s * vkp + c * vkq;
        }
      }
  }
}

// ---------------------------------------------------------------------------
// reduced coordinates of each distance type
// ---------------------------------------------------------------------------
struct Reduced {
  int m;          // number of difference vectors (1, 2, 3)
  int form;       // 0: |e|^2, 1: point-line, 2: triple product over |e1 x e2|^2
  double C[4][3]; // x-vertex k -> coefficient on difference vector v
  v3 r[3];
};

ABD_HD void set_pp(Reduced& R, const v3* x, int i, int j) {
  R.m = 1;
  R.form = 0;
  for (int k = 0; k < 4; ++k) R.C[k][0] = R.C[k][1] = R.C[k][2] = 0.0;
  R.C[i][0] = 1.0;
  R.C[j][0] = -1.0;
  R.r[0] = x[i] - x[j];
}
// point p against the line through a, b: u = a - p, v = b - p
ABD_HD void set_pe(Reduced& R, const v3* x, int p, int a, int b) {
  R.m = 2;
  R.form = 1;
  for (int k = 0; k < 4; ++k) R.C[k][0] = R.C[k][1] = R.C[k][2] = 0.0;
  R.C[p][0] = -1.0;
  R.C[p][1] = -1.0;
  R.C[a][0] = 1.0;
  R.C[b][1] = 1.0;
  R.r[0] = x[a] - x[p];
  R.r[1] = x[b] - x[p];
}

ABD_HD void reduce(int kind, int type, const v3* x, Reduced& R) {
  for (int k = 0; k < 4; ++k) R.C[k][0] = R.C[k][1] = R.C[k][2] = 0.0;
  if (kind == 0) {
    switch (type) {
      case 0: set_pp(R, x, 0, 1); break;
      case 1: set_pp(R, x, 0, 2); break;
      case 2: set_pp(R, x, 0, 3); break;
      case 3: set_pe(R, x, 0, 1, 2); break;
      case 4: set_pe(R, x, 0, 2, 3); break;
      case 5: set_pe(R, x, 0, 3, 1); break;
      default:  // plane: w = x0 - x1, e1 = x2 - x1, e2 = x3 - x1
        R.m = 3;
        R.form = 2;
        R.C[0][0] = 1.0;
        R.C[1][0] = -1.0; R.C[1][1] = -1.0; R.C[1][2] = -1.0;
        R.C[2][1] = 1.0;
        R.C[3][2] = 1.0;
        R.r[0] = x[0] - x[1];
        R.r[1] = x[2] - x[1];
        R.r[2] = x[3] - x[1];
        break;
    }
  } else {
    switch (type) {
      case 0: set_pp(R, x, 0, 2); break;
      case 1: set_pp(R, x, 0, 3); break;
      case 2: set_pp(R, x, 1, 2); break;
      case 3: set_pp(R, x, 1, 3); break;
      case 4: set_pe(R, x, 0, 2, 3); break;
      case 5: set_pe(R, x, 1, 2, 3); break;
      case 6: set_pe(R, x, 2, 0, 1); break;
      case 7: set_pe(R, x, 3, 0, 1); break;
      default:  // line-line: w = x2 - x0, e0 = x1 - x0, e1 = x3 - x2
        R.m = 3;
        R.form = 2;
        R.C[0][0] = -1.0; R.C[0][1] = -1.0;
        R.C[1][1] = 1.0;
        R.C[2][0] = 1.0; R.C[2][2] = -1.0;
        R.C[3][2] = 1.0;
        R.r[0] = x[2] - x[0];
        R.r[1] = x[1] - x[0];
        R.r[2] = x[3] - x[2];
        break;
    }
  }
}

// H (n3 x n3 row-major, n3 = 3m): add s * a b^T into block (I, J)
ABD_HD void blk_outer(double* H, int n3, int I, int J, double s, v3 a, v3 b) {
  double av[3] = {a.x, a.y, a.z}, bv[3] = {b.x, b.y, b.z};
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) H[(3 * I + i) * n3 + 3 * J + j] += s * av[i] * bv[j];
}
ABD_HD void blk_ident(double* H, int n3, int I, int J, double s) {
  for (int i = 0; i < 3; ++i) H[(3 * I + i) * n3 + 3 * J + i] += s;
}
// add s * [v]x (cross-product matrix) into block (I, J)
ABD_HD void blk_skew(double* H, int n3, int I, int J, double s, v3 v) {
  H[(3 * I + 0) * n3 + 3 * J + 1] += -s * v.z;
  H[(3 * I + 0) * n3 + 3 * J + 2] += s * v.y;
  H[(3 * I + 1) * n3 + 3 * J + 0] += s * v.z;
  H[(3 * I + 1) * n3 + 3 * J + 2] += -s * v.x;
  H[(3 * I + 2) * n3 + 3 * J + 0] += -s * v.y;
  H[(3 * I + 2) * n3 + 3 * J + 1] += s * v.x;
}

// Lagrange identity L(u, v) = |u|^2 |v|^2 - (u.v)^2 = |u x v|^2: gradient
// into slots (I, J) of g and Hessian into blocks of H (scaled by s)
ABD_HD void lagrange_derivs(v3 u, v3 v, int I, int J, int n3, double sg, double sh, double* g, double* H) {
  double uu = dot(u, u), vv = dot(v, v), uv = dot(u, v);
  if (g) {
    v3 gu = (2.0 * vv) * u - (2.0 * uv) * v;
    v3 gv = (2.0 * uu) * v - (2.0 * uv) * u;
    g[3 * I] += sg * gu.x; g[3 * I + 1] += sg * gu.y; g[3 * I + 2] += sg * gu.z;
    g[3 * J] += sg * gv.x; g[3 * J + 1] += sg * gv.y; g[3 * J + 2] += sg * gv.z;
  }
  if (H) {
    blk_ident(H, n3, I, I, sh * 2.0 * vv);
    blk_outer(H, n3, I, I, -2.0 * sh, v, v);
    blk_ident(H, n3, J, J, sh * 2.0 * uu);
    blk_outer(H, n3, J, J, -2.0 * sh, u, u);
    // d2/du dv = 4 u v^T - 2 v u^T - 2 (u.v) I, and its transpose
    blk_outer(H, n3, I, J, 4.0 * sh, u, v);
    blk_outer(H, n3, I, J, -2.0 * sh, v, u);
    blk_ident(H, n3, I, J, -2.0 * sh * uv);
    blk_outer(H, n3, J, I, 4.0 * sh, v, u);
    blk_outer(H, n3, J, I, -2.0 * sh, u, v);
    blk_ident(H, n3, J, I, -2.0 * sh * uv);
  }
}

// s and its gradient / Hessian in the reduced coordinates (n3 = 3m)
ABD_HD double reduced_dist2(const Reduced& R, double* gs, double* Hs) {
  const int n3 = 3 * R.m;
  for (int i = 0; i < n3; ++i) gs[i] = 0.0;
  for (int i = 0; i < n3 * n3; ++i) Hs[i] = 0.0;
  if (R.form == 0) {
    v3 e = R.r[0];
    gs[0] = 2.0 * e.x; gs[1] = 2.0 * e.y; gs[2] = 2.0 * e.z;
    blk_ident(Hs, 3, 0, 0, 2.0);
    return dot(e, e);
  }
  // numerator N and denominator D with s = N / D
  double gN[9], gD[9], HN[81], HD[81];
  for (int i = 0; i < 9; ++i) gN[i] = gD[i] = 0.0;
  for (int i = 0; i < 81; ++i) HN[i] = HD[i] = 0.0;
  double N, D;
  if (R.form == 1) {
    v3 u = R.r[0], v = R.r[1];
    N = dot(u, u) * dot(v, v) - dot(u, v) * dot(u, v);
    lagrange_derivs(u, v, 0, 1, 6, 1.0, 1.0, gN, HN);
    v3 e = v - u;
    D = dot(e, e);
    // D = |v - u|^2: grad (-2e, 2e); Hessian [[2I, -2I], [-2I, 2I]]
    gD[0] = -2.0 * e.x; gD[1] = -2.0 * e.y; gD[2] = -2.0 * e.z;
    gD[3] = 2.0 * e.x; gD[4] = 2.0 * e.y; gD[5] = 2.0 * e.z;
    blk_ident(HD, 6, 0, 0, 2.0);
    blk_ident(HD, 6, 1, 1, 2.0);
    blk_ident(HD, 6, 0, 1, -2.0);
    blk_ident(HD, 6, 1, 0, -2.0);
  } else {
    // t = w . (e1 x e2); N = t^2; D = |e1 x e2|^2
    v3 w = R.r[0], e1 = R.r[1], e2 = R.r[2];
    v3 n = cross(e1, e2);
    double t = dot(w, n);
    v3 gw = n, g1 = cross(e2, w), g2 = cross(w, e1);
    double gt[9] = {gw.x, gw.y, gw.z, g1.x, g1.y, g1.z, g2.x, g2.y, g2.z};
    N = t * t;
    for (int i = 0; i < 9; ++i) gN[i] = 2.0 * t * gt[i];
    for (int i = 0; i < 9; ++i)
      for (int j = 0; j < 9; ++j) HN[i * 9 + j] = 2.0 * gt[i] * gt[j];
    // Hessian of the triple product: d2t/dw de1 = -[e2]x, d2t/dw de2 = [e1]x,
    // d2t/de1 de2 = -[w]x (and transposes)
    blk_skew(HN, 9, 0, 1, -2.0 * t, e2);
    blk_skew(HN, 9, 1, 0, 2.0 * t, e2);
    blk_skew(HN, 9, 0, 2, 2.0 * t, e1);
    blk_skew(HN, 9, 2, 0, -2.0 * t, e1);
    blk_skew(HN, 9, 1, 2, -2.0 * t, w);
    blk_skew(HN, 9, 2, 1, 2.0 * t, w);
    D = dot(n, n);
    lagrange_derivs(e1, e2, 1, 2, 9, 1.0, 1.0, gD, HD);
  }
  double s = N / D;
  double iD = 1.0 / D;
  for (int i = 0; i < n3; ++i) gs[i] = (gN[i] - s * gD[i]) * iD;
  for (int i = 0; i < n3; ++i)
    for (int j = 0; j < n3; ++j)
      Hs[i * n3 + j] = (HN[i * n3 + j] - s * HD[i * n3 + j] - gs[i] * gD[j] - gD[i] * gs[j]) * iD;
  return s;
}

// ---------------------------------------------------------------------------
// mollified edge-edge barrier kappa B(d) m(c) in the line-line coordinates
// y = (w, e0, e1) = (x2 - x0, x1 - x0, x3 - x2), the reduced coordinates of
// edge-edge type 8 whatever the pair's distance type: every type's difference
// vectors are integer combinations of y (a column c of C gives coefficients
// (c2 + c3, c1, c3)), and c = |e0 x e1|^2 depends on e0 and e1 only.
// Writes the gradient g9 and the (unprojected) Hessian H9 (9x9 row-major) of
// the product and returns its value.
// ---------------------------------------------------------------------------
ABD_HD double mollified_ee_term(int type, const v3* x, double dhat, double kappa, double c, double eps, double* g9,
                                double* H9) {
  Reduced Rt;
  reduce(1, type, x, Rt);
  const int mt = Rt.m, nt = 3 * mt;
  double gs[9], Hs[81];
  const double s = reduced_dist2(Rt, gs, Hs);
  const double d = sqrt(s);
  double B, B1, B2;
  barrier_derivs(d, dhat, B, B1, B2);
  const double cg = kappa * B1 / (2.0 * d);
  const double ca = kappa * (B2 / (4.0 * s) - B1 / (4.0 * d * s));
  double A[3][3];
  for (int w = 0; w < mt; ++w) {
    A[w][0] = Rt.C[2][w] + Rt.C[3][w];
    A[w][1] = Rt.C[1][w];
    A[w][2] = Rt.C[3][w];
  }
  // kappa B and its derivatives pulled back to y
  double gb[9];
  for (int J = 0; J < 3; ++J)
    for (int i = 0; i < 3; ++i) {
      double t = 0.0;
      for (int w = 0; w < mt; ++w) t += A[w][J] * gs[3 * w + i];
      gb[3 * J + i] = cg * t;
    }
  for (int J = 0; J < 3; ++J)
    for (int L = 0; L < 3; ++L)
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
          double t = 0.0;
          for (int w = 0; w < mt; ++w) {
            if (A[w][J] == 0.0) continue;
            for (int v = 0; v < mt; ++v)
              t += A[w][J] * A[v][L] * (ca * gs[3 * w + i] * gs[3 * v + j] + cg * Hs[(3 * w + i) * nt + 3 * v + j]);
          }
          H9[(3 * J + i) * 9 + 3 * L + j] = t;
        }
  // c = |e0 x e1|^2 (Lagrange identity) in slots e0 = 1, e1 = 2
  double gc[9], Hc[81];
  for (int i = 0; i < 9; ++i) gc[i] = 0.0;
  for (int i = 0; i < 81; ++i) Hc[i] = 0.0;
  lagrange_derivs(x[1] - x[0], x[3] - x[2], 1, 2, 9, 1.0, 1.0, gc, Hc);
  double dm, d2m;
  const double mv = ee_mollifier(c, eps, dm, d2m);
  const double Eb = kappa * B;
  // product rule: H = m Hb + Eb (m'' gc gc^T + m' Hc) + m' (gc gb^T + gb gc^T)
  for (int a = 0; a < 9; ++a)
    for (int b = 0; b < 9; ++b)
      H9[a * 9 + b] = mv * H9[a * 9 + b] + Eb * (d2m * gc[a] * gc[b] + dm * Hc[a * 9 + b]) +
                      dm * (gc[a] * gb[b] + gb[a] * gc[b]);
  for (int a = 0; a < 9; ++a) g9[a] = mv * gb[a] + Eb * dm * gc[a];
  return Eb * mv;
}

// ---------------------------------------------------------------------------
// lagged friction term
// ---------------------------------------------------------------------------
ABD_HD double friction_term(const v3* x, const double* gam, v3 n, v3 r, double mu_lambda, double eps, double* g12,
                            double* H78) {
  v3 w = (gam[0] * x[0] + gam[1] * x[1]) + (gam[2] * x[2] + gam[3] * x[3]) - r;
  v3 u = w - dot(n, w) * n;
  double y = sqrt(dot(u, u));
  double f0, f1, f1_over_y, df1;
  if (y >= eps) {
    f0 = y;
    f1 = 1.0;
    f1_over_y = 1.0 / y;
    df1 = 0.0;
  } else {
    f0 = -y * y * y / (3.0 * eps * eps) + y * y / eps + eps / 3.0;
    f1 = -y * y / (eps * eps) + 2.0 * y / eps;
    f1_over_y = -y / (eps * eps) + 2.0 / eps;
    df1 = -2.0 * y / (eps * eps) + 2.0 / eps;
  }
  v3 uh = y > 0.0 ? (1.0 / y) * u : v3{0.0, 0.0, 0.0};
  // Hu = df1 uh uh^T + (f1/y)(P - uh uh^T), P = I - n n^T
  double Hu[3][3];
  double nv[3] = {n.x, n.y, n.z}, uv[3] = {uh.x, uh.y, uh.z};
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double P = (i == j ? 1.0 : 0.0) - nv[i] * nv[j];
      Hu[i][j] = mu_lambda * (df1 * uv[i] * uv[j] + f1_over_y * (P - uv[i] * uv[j]));
    }
  for (int k = 0; k < 4; ++k) {
    g12[3 * k] = mu_lambda * gam[k] * f1 * uh.x;
    g12[3 * k + 1] = mu_lambda * gam[k] * f1 * uh.y;
    g12[3 * k + 2] = mu_lambda * gam[k] * f1 * uh.z;
  }
  for (int k = 0; k < 4; ++k)
    for (int l = k; l < 4; ++l)
      for (int i = 0; i < 3; ++i)
        for (int j = (k == l ? i : 0); j < 3; ++j) H78[up12(3 * k + i, 3 * l + j)] = gam[k] * gam[l] * Hu[i][j];
  return mu_lambda * f0;
}

}  // namespace abd
