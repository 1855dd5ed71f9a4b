// Small dense helpers shared by the contact kernels: symmetric eigen-
// decomposition by cyclic Jacobi (for rare fall-backs), the reduced
// coordinates of each distance type (Sec. 4) and the lagged friction term.
//
// Barrier (Sec. 4, Eq. barrier and Eq. clamped-b): every type's squared
// distance s is a function of a few difference vectors r = C x (C a 4 x m
// matrix with entries in {-1, 0, 1}, m = 1 point-point, 2 point-edge, 3
// point-plane and line-line); the barrier kernel works in those coordinates.
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
