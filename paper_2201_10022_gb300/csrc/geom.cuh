// Device geometry for the affine-body contact path: canonical squared
// distances and distance types of point-triangle and edge-edge pairs, the
// additive-CCD step (Sec. 4.1), and the derivatives of the clamped log
// barrier (Sec. 4, Eq. clamped-b).
//
// Canonical floating point.  Set membership (candidate / active pairs) and
// CCD step sizes are decided by the operation order below, written with
// round-to-nearest intrinsics so the compiler cannot contract or reorder:
//   sub(a,b)   = (a0-b0, a1-b1, a2-b2)
//   dot(a,b)   = fma(a2,b2, fma(a1,b1, a0*b0))
//   cross(a,b) = (a1*b2 - a2*b1, a2*b0 - a0*b2, a0*b1 - a1*b0)
// with divisions and square roots correctly rounded.  The CPU reference
// follows the same written order, so pair sets and times of impact can be
// compared bit for bit.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#ifndef ABD_HD
#define ABD_HD __host__ __device__ __forceinline__
#endif

namespace abd {

struct v3 {
  double x, y, z;
};

ABD_HD v3 mk(double x, double y, double z) { return v3{x, y, z}; }
ABD_HD v3 mk(const double4& a) { return v3{a.x, a.y, a.z}; }

// ---- canonical (non-contracted) vector operations -------------------------
__device__ __forceinline__ v3 csub(v3 a, v3 b) {
  return v3{__dsub_rn(a.x, b.x), __dsub_rn(a.y, b.y), __dsub_rn(a.z, b.z)};
}
__device__ __forceinline__ double cdot(v3 a, v3 b) {
  return __fma_rn(a.z, b.z, __fma_rn(a.y, b.y, __dmul_rn(a.x, b.x)));
}
__device__ __forceinline__ v3 ccross(v3 a, v3 b) {
  return v3{__dsub_rn(__dmul_rn(a.y, b.z), __dmul_rn(a.z, b.y)), __dsub_rn(__dmul_rn(a.z, b.x), __dmul_rn(a.x, b.z)),
            __dsub_rn(__dmul_rn(a.x, b.y), __dmul_rn(a.y, b.x))};
}

// ---- plain vector helpers for derivative code (contraction allowed) -------
ABD_HD v3 operator+(v3 a, v3 b) { return v3{a.x + b.x, a.y + b.y, a.z + b.z}; }
ABD_HD v3 operator-(v3 a, v3 b) { return v3{a.x - b.x, a.y - b.y, a.z - b.z}; }
ABD_HD v3 operator*(double s, v3 a) { return v3{s * a.x, s * a.y, s * a.z}; }
ABD_HD double dot(v3 a, v3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
ABD_HD v3 cross(v3 a, v3 b) {
  return v3{a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
ABD_HD double comp(v3 a, int i) { return i == 0 ? a.x : (i == 1 ? a.y : a.z); }

// ---------------------------------------------------------------------------
// canonical squared distances of the elementary types
// ---------------------------------------------------------------------------
__device__ __forceinline__ double d2_pp(v3 p, v3 q) {
  v3 e = csub(p, q);
  return cdot(e, e);
}
// point p to the line through a, b: |(a-p) x (b-p)|^2 / |b-a|^2
__device__ __forceinline__ double d2_pe(v3 p, v3 a, v3 b) {
  v3 u = csub(a, p), v = csub(b, p);
  v3 c = ccross(u, v);
  v3 e = csub(b, a);
  return __ddiv_rn(cdot(c, c), cdot(e, e));
}
// point p to the plane of (a, b, c): ((p-a).n)^2 / |n|^2, n = (b-a) x (c-a)
__device__ __forceinline__ double d2_plane(v3 p, v3 a, v3 b, v3 c) {
  v3 n = ccross(csub(b, a), csub(c, a));
  double t = cdot(csub(p, a), n);
  return __ddiv_rn(__dmul_rn(t, t), cdot(n, n));
}
// lines (a,b) and (c,d): ((c-a).n)^2 / |n|^2, n = (b-a) x (d-c)
__device__ __forceinline__ double d2_line(v3 a, v3 b, v3 c, v3 d) {
  v3 n = ccross(csub(b, a), csub(d, c));
  double t = cdot(csub(c, a), n);
  return __ddiv_rn(__dmul_rn(t, t), cdot(n, n));
}

// p against segment [a,b]; branch 0: endpoint a, 1: endpoint b, 2: interior
__device__ __forceinline__ double point_segment(v3 p, v3 a, v3 b, int& branch) {
  v3 e = csub(b, a);
  double t = cdot(csub(p, a), e);
  if (t <= 0.0) {
    branch = 0;
    return d2_pp(p, a);
  }
  if (t >= cdot(e, e)) {
    branch = 1;
    return d2_pp(p, b);
  }
  branch = 2;
  return d2_pe(p, a, b);
}

// Point x0 against triangle (x1,x2,x3).  Types 0..2: nearest vertex x1..x3;
// 3..5: nearest point inside edge (x1,x2), (x2,x3), (x3,x1); 6: plane.
__device__ __forceinline__ double pt_dist2(v3 x0, v3 x1, v3 x2, v3 x3, int& type) {
  v3 e01 = csub(x2, x1), e12 = csub(x3, x2), e20 = csub(x1, x3);
  v3 n = ccross(e01, csub(x3, x1));
  bool inside = true;
  if (cdot(ccross(e01, csub(x0, x1)), n) < 0.0) inside = false;
  if (cdot(ccross(e12, csub(x0, x2)), n) < 0.0) inside = false;
  if (cdot(ccross(e20, csub(x0, x3)), n) < 0.0) inside = false;
  if (inside) {
    type = 6;
    return d2_plane(x0, x1, x2, x3);
  }
  int br;
  double best = point_segment(x0, x1, x2, br);
  type = br == 0 ? 0 : (br == 1 ? 1 : 3);
  double d = point_segment(x0, x2, x3, br);
  if (d < best) {
    best = d;
    type = br == 0 ? 1 : (br == 1 ? 2 : 4);
  }
  d = point_segment(x0, x3, x1, br);
  if (d < best) {
    best = d;
    type = br == 0 ? 2 : (br == 1 ? 0 : 5);
  }
  return best;
}

// Edge (x0,x1) against edge (x2,x3).  Types 0..3: point-point x0x2, x0x3,
// x1x2, x1x3; 4..7: point-edge x0-(x2x3), x1-(x2x3), x2-(x0x1), x3-(x0x1);
// 8: line-line with both closest points interior.
__device__ __forceinline__ double ee_dist2(v3 x0, v3 x1, v3 x2, v3 x3, int& type) {
  v3 e0 = csub(x1, x0), e1 = csub(x3, x2);
  v3 n = ccross(e0, e1);
  double nn = cdot(n, n);
  double A = cdot(e0, e0), C = cdot(e1, e1);
  bool parallel = nn <= __dmul_rn(__dmul_rn(1e-20, A), C);
  if (!parallel) {
    v3 w0 = csub(x0, x2);
    double B = cdot(e0, e1), D = cdot(e0, w0), E = cdot(e1, w0);
    double den = __dsub_rn(__dmul_rn(A, C), __dmul_rn(B, B));
    double sn = __dsub_rn(__dmul_rn(B, E), __dmul_rn(C, D));
    double tn = __dsub_rn(__dmul_rn(A, E), __dmul_rn(B, D));
    if (sn > 0.0 && sn < den && tn > 0.0 && tn < den) {
      type = 8;
      return d2_line(x0, x1, x2, x3);
    }
  }
  int br;
  double best = point_segment(x0, x2, x3, br);
  type = br == 0 ? 0 : (br == 1 ? 1 : 4);
  double d = point_segment(x1, x2, x3, br);
  if (d < best) {
    best = d;
    type = br == 0 ? 2 : (br == 1 ? 3 : 5);
  }
  d = point_segment(x2, x0, x1, br);
  if (d < best) {
    best = d;
    type = br == 0 ? 0 : (br == 1 ? 2 : 6);
  }
  d = point_segment(x3, x0, x1, br);
  if (d < best) {
    best = d;
    type = br == 0 ? 1 : (br == 1 ? 3 : 7);
  }
  return best;
}

__device__ __forceinline__ double pair_dist2(int kind, const v3* x, int& type) {
  return kind == 0 ? pt_dist2(x[0], x[1], x[2], x[3], type) : ee_dist2(x[0], x[1], x[2], x[3], type);
}

// ---------------------------------------------------------------------------
// Additive CCD (ACCD, cited by Sec. 4.1): conservative advancement along the
// linear trajectory x + t dx, t in [0, tmax], with the mean displacement
// removed.  Returns 0 on success, 1 if the iteration cap was reached.
// bound (may be null): the bits of a time that other evaluations have already
// established as an upper bound of the minimum this evaluation contributes
// to; it is re-read every 8 advancement steps and lowers tmax.  A result of
// tmax then means "no impact before the bound", which leaves the minimum
// unchanged, so the minimum over all evaluations is exact whatever their
// timing.  d0_lp (may be null) receives the distance at t = 0 (-1 if not
// computed) and lp, the bound on the distance's rate of change: the distance
// at t is at least d0 - t lp.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int accd(int kind, const v3* xin, const v3* dx, double s, double tmax, int max_iter,
                                    double& toi, const unsigned long long* bound = nullptr,
                                    double2* d0_lp = nullptr) {
  v3 x[4], p[4];
  v3 mean;
  mean.x = __dmul_rn(__dadd_rn(__dadd_rn(dx[0].x, dx[1].x), __dadd_rn(dx[2].x, dx[3].x)), 0.25);
  mean.y = __dmul_rn(__dadd_rn(__dadd_rn(dx[0].y, dx[1].y), __dadd_rn(dx[2].y, dx[3].y)), 0.25);
  mean.z = __dmul_rn(__dadd_rn(__dadd_rn(dx[0].z, dx[1].z), __dadd_rn(dx[2].z, dx[3].z)), 0.25);
  double nrm[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    p[k] = csub(dx[k], mean);
    x[k] = xin[k];
    nrm[k] = __dsqrt_rn(cdot(p[k], p[k]));
  }
  double lp;
  if (kind == 0) {
    double m = nrm[1] > nrm[2] ? nrm[1] : nrm[2];
    m = m > nrm[3] ? m : nrm[3];
    lp = __dadd_rn(nrm[0], m);
  } else {
    double ma = nrm[0] > nrm[1] ? nrm[0] : nrm[1];
    double mb = nrm[2] > nrm[3] ? nrm[2] : nrm[3];
    lp = __dadd_rn(ma, mb);
  }
  if (d0_lp) *d0_lp = make_double2(-1.0, lp);  // distance not known yet: no bound
  if (lp == 0.0) {
    toi = tmax;
    return 0;
  }
  int type;
  double d = __dsqrt_rn(pair_dist2(kind, x, type));
  if (d0_lp) d0_lp->x = d;
  if (d == 0.0) {
    toi = 0.0;
    return 0;
  }
  const double g = __dmul_rn(s, d);
  double t = 0.0;
  double tl = __ddiv_rn(__dmul_rn(__dsub_rn(1.0, s), d), lp);
  for (int it = 0; it < max_iter; ++it) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      x[k].x = __dadd_rn(x[k].x, __dmul_rn(tl, p[k].x));
      x[k].y = __dadd_rn(x[k].y, __dmul_rn(tl, p[k].y));
      x[k].z = __dadd_rn(x[k].z, __dmul_rn(tl, p[k].z));
    }
    d = __dsqrt_rn(pair_dist2(kind, x, type));
    if (t > 0.0 && d < g) {
      toi = t;
      return 0;
    }
    t = __dadd_rn(t, tl);
    if (bound && (it & 7) == 7) {
      const double bt = __longlong_as_double((long long)*(const volatile unsigned long long*)bound);
      if (bt < tmax) tmax = bt;
    }
    if (t > tmax) {
      toi = tmax;
      return 0;
    }
    tl = __ddiv_rn(__dmul_rn(0.9, d), lp);
  }
  toi = t;
  return 1;
}

// ---------------------------------------------------------------------------
// clamped log barrier B(d) = -(d - dhat)^2 ln(d / dhat) and its derivatives
// ---------------------------------------------------------------------------
ABD_HD void barrier_derivs(double d, double dhat, double& B, double& B1, double& B2) {
  double t = d - dhat;
  double l = log(d / dhat);
  B = -t * t * l;
  B1 = -2.0 * t * l - t * t / d;
  B2 = -2.0 * l - 4.0 * t / d + (t * t) / (d * d);
}

// ---------------------------------------------------------------------------
// near-parallel edge-edge mollifier (IPC, Li et al. 2020): an edge-edge
// barrier is multiplied by m(c) = (2 - c/eps) c/eps while c = |e0 x e1|^2 is
// below eps = 1e-3 |rest e0|^2 |rest e1|^2, so that it fades out (C1) as the
// edges turn parallel and the line-line distance loses its conditioning.
// c and eps are formed in canonical order: the choice of branch matches the
// CPU reference bit for bit.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double ee_cross2(const v3* x) {
  v3 n = ccross(csub(x[1], x[0]), csub(x[3], x[2]));
  return cdot(n, n);
}
__device__ __forceinline__ double ee_eps(double l2i, double l2j) { return __dmul_rn(__dmul_rn(1e-3, l2i), l2j); }
// m(c) with its first and second derivatives (1, 0, 0 at and above eps)
ABD_HD double ee_mollifier(double c, double eps, double& dm, double& d2m) {
  if (!(c < eps)) {
    dm = d2m = 0.0;
    return 1.0;
  }
  double r = c / eps;
  dm = (2.0 - 2.0 * r) / eps;
  d2m = -2.0 / (eps * eps);
  return (2.0 - r) * r;
}

}  // namespace abd
