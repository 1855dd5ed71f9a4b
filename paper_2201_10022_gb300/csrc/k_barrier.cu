// Barrier terms of the active pairs (Sec. 4, Eq. barrier and Eq. clamped-b):
// energy kappa B(d), vertex gradient and PSD-projected vertex Hessian of every
// active point-triangle and edge-edge pair, written per term for the
// deterministic per-body-pair reduction.
//
// Every distance type's squared distance s is a function of m difference
// vectors r = C x (C a 4 x m matrix with entries in {-1, 0, 1}), so the 12x12
// vertex Hessian is T H_r T^T with T = C (x) I3.  With C^T C = Rm^T Rm (Rm
// upper triangular, Ri = Rm^-1) its PSD projection is exactly
//   T (Ri (x) I3) Proj((Rm (x) I3) H_r (Rm^T (x) I3)) (Ri^T (x) I3) T^T.
// C^T C depends only on the type's class (point-point, point-edge,
// point-plane, line-line), so Rm and Ri are per-class constants.
//
// The work is split by working dimension n = 3m after a classification pass
// that buckets the terms:
//   n = 3 (point-point): one thread per term.  H_r = 4 c_a e e^T + 2 c_g I
//     has the eigenvalue 4 c_a |e|^2 + 2 c_g along e and 2 c_g across it, so
//     its projection is in closed form.
//   n = 6, 9: one warp per term.  The lanes form the n x n entries of H_r
//     and of K = (Rm x I) H_r (Rm^T x I), find an eigenbasis of K by cyclic
//     Jacobi in FP32 with round-robin ordering (n/2 disjoint rotations per
//     round), then refine it in FP64: one Newton-Schulz step V (3I - V^T V)/2,
//     K' = V^T K V, a second FP32 Jacobi pass on K' (it resolves the lower
//     levels of the spectrum, which the first pass on K / max|K| cannot see;
//     scale-aware skip test, until a sweep takes no rotation) with the same
//     FP64 basis update, and FP64 round-robin Jacobi sweeps on the nearly
//     diagonal result until the couplings between its positive and
//     non-positive diagonal entries are below 1e-11 of the total (squares
//     below 1e-22); the clamp keeps the whole block on the positive entries.
// A mollified edge-edge pair (near-parallel edges) is worked in the line-line
// coordinates (n = 9) whatever its distance type.
#include <math.h>
#include <stddef.h>
#include <string.h>

#include "abd_internal.cuh"
#include "derivs.cuh"

namespace abd {

namespace {

constexpr unsigned kAll = 0xffffffffu;
constexpr int kBarWarps = 4;
// blocks of k_barrier that must fit on one SM (a register bound of
// 65536 / (32 kBarWarps kBarMinBlocks) per thread)
#ifndef ABD_BAR_MIN_BLOCKS
#define ABD_BAR_MIN_BLOCKS 1
#endif
constexpr int kBarMinBlocks = ABD_BAR_MIN_BLOCKS;

// Gram factors of the four reduced-coordinate classes: 0 point-point,
// 1 point-edge, 2 point-plane, 3 line-line (3x3 row-major, upper)
struct GramTables {
  double Rm[4][9];
  double Ri[4][9];
};

GramTables make_gram() {
  GramTables g;
  memset(&g, 0, sizeof(g));
  const int kinds[4] = {0, 0, 0, 1}, types[4] = {0, 3, 6, 8};
  v3 x[4] = {{0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
  for (int c = 0; c < 4; ++c) {
    Reduced R;
    reduce(kinds[c], types[c], x, R);
    const int m = R.m;
    double G[3][3], Rm[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}}, Ri[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    for (int a = 0; a < m; ++a)
      for (int b = 0; b < m; ++b) {
        double t = 0.0;
        for (int k = 0; k < 4; ++k) t += R.C[k][a] * R.C[k][b];
        G[a][b] = t;
      }
    for (int j = 0; j < m; ++j) {
      double t = G[j][j];
      for (int k = 0; k < j; ++k) t -= Rm[k][j] * Rm[k][j];
      Rm[j][j] = sqrt(t);
      for (int i = j + 1; i < m; ++i) {
        double u = G[j][i];
        for (int k = 0; k < j; ++k) u -= Rm[k][j] * Rm[k][i];
        Rm[j][i] = u / Rm[j][j];
      }
    }
    for (int i = m - 1; i >= 0; --i) {
      Ri[i][i] = 1.0 / Rm[i][i];
      for (int j = i + 1; j < m; ++j) {
        double t = 0.0;
        for (int k = i + 1; k <= j; ++k) t += Rm[i][k] * Ri[k][j];
        Ri[i][j] = -t / Rm[i][i];
      }
    }
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) {
        g.Rm[c][3 * a + b] = Rm[a][b];
        g.Ri[c][3 * a + b] = Ri[a][b];
      }
  }
  return g;
}

__device__ __forceinline__ int gram_class(int kind, int type, int moll) {
  if (moll) return 3;
  if (kind == 0) return type < 3 ? 0 : (type < 6 ? 1 : 2);
  return type < 4 ? 0 : (type < 8 ? 1 : 3);
}

// ---------------------------------------------------------------------------
// classification: vertex ids, type / mollifier flag and bucket of every term
// ---------------------------------------------------------------------------
__global__ void k_bar_classify(const DevStatus* __restrict__ cst, const int* aoff, const int4* act,
                               const double* act_d2, const int* tri, const int* edge, const double4* x,
                               const double* l2e, int maxc, long cap, int4* termv, int* tmeta, double* teps,
                               double* td2, int* tlist, DevStatus* st) {
  const int lane = threadIdx.x & 31;
  const int np = cst->np;
  const long nact = min((long)cst->nact, cap);
  const long stride = (long)gridDim.x * blockDim.x;
  for (long base = (long)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < nact; base += stride) {
    const long f = base + lane;
    int cls = -1;
    if (f < nact) {
      const int p = owner(aoff, np, (int)f);
      const size_t slot = (size_t)p * maxc + (f - aoff[p]);
      const int4 r = act[slot];
      const int kind = (unsigned)r.x >> 31, i = r.x & 0x7fffffff, type = r.z;
      int v[4];
      pair_vertices(kind, i, r.y, tri, edge, v);
      int moll = 0;
      double eps = 0.0;
      if (kind == 1) {
        v3 xs[4];
        for (int k = 0; k < 4; ++k) xs[k] = mk(x[v[k]]);
        eps = ee_eps(l2e[i], l2e[r.y]);
        moll = ee_cross2(xs) < eps;
      }
      const int g = gram_class(kind, type, moll);
      cls = g == 0 ? 0 : (g == 1 ? 1 : 2);
      termv[f] = make_int4(v[0], v[1], v[2], v[3]);
      tmeta[f] = kind | (type << 1) | (moll << 5);
      teps[f] = eps;
      td2[f] = act_d2[slot];
    }
    for (int k = 0; k < 3; ++k) {
      const unsigned m = __ballot_sync(kAll, cls == k);
      if (!m) continue;
      const int leader = __ffs(m) - 1;
      int pos0 = 0;
      if (lane == leader) pos0 = atomicAdd(&st->bar_cnt[k], __popc(m));
      pos0 = __shfl_sync(kAll, pos0, leader);
      if (cls == k) tlist[(size_t)k * cap + pos0 + __popc(m & ((1u << lane) - 1u))] = (int)f;
    }
  }
}

// ---------------------------------------------------------------------------
// per-form distance quantities of the type's reduced coordinates
// ---------------------------------------------------------------------------
struct TypeDist {
  int form, n;
  double s, iD, t, uu, vv, uv;
  v3 r0, r1, r2;
};

// s and its gradient gs; for forms 1 and 2 also the gradient gD of the
// denominator of s = N / D and (form 2) the gradient gt of the triple
// product.  Lane 0 writes the vectors to the warp's shared scratch.
__device__ __forceinline__ void type_dist(const Reduced& R, TypeDist& T, double* gs, double* gD, double* gt,
                                          int lane) {
  T.form = R.form;
  T.n = 3 * R.m;
  T.r0 = R.r[0];
  T.r1 = R.r[1];
  T.r2 = R.r[2];
  T.t = 0.0;
  T.uu = T.vv = T.uv = 0.0;
  T.iD = 1.0;
  double g[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0}, hD[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  double ht[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  if (R.form == 0) {
    const v3 e = R.r[0];
    T.s = dot(e, e);
    g[0] = 2.0 * e.x;
    g[1] = 2.0 * e.y;
    g[2] = 2.0 * e.z;
  } else if (R.form == 1) {
    const v3 u = R.r[0], v = R.r[1];
    T.uu = dot(u, u);
    T.vv = dot(v, v);
    T.uv = dot(u, v);
    const double N = T.uu * T.vv - T.uv * T.uv;
    const v3 e = v - u;
    const double D = dot(e, e);
    T.s = N / D;
    T.iD = 1.0 / D;
    const v3 gu = (2.0 * T.vv) * u - (2.0 * T.uv) * v, gv = (2.0 * T.uu) * v - (2.0 * T.uv) * u;
    hD[0] = -2.0 * e.x; hD[1] = -2.0 * e.y; hD[2] = -2.0 * e.z;
    hD[3] = 2.0 * e.x; hD[4] = 2.0 * e.y; hD[5] = 2.0 * e.z;
    const double gn[6] = {gu.x, gu.y, gu.z, gv.x, gv.y, gv.z};
    for (int k = 0; k < 6; ++k) g[k] = (gn[k] - T.s * hD[k]) * T.iD;
  } else {
    const v3 w = R.r[0], e1 = R.r[1], e2 = R.r[2];
    const v3 n = cross(e1, e2), g1 = cross(e2, w), g2 = cross(w, e1);
    T.t = dot(w, n);
    T.uu = dot(e1, e1);
    T.vv = dot(e2, e2);
    T.uv = dot(e1, e2);
    const double D = dot(n, n);
    T.s = (T.t * T.t) / D;
    T.iD = 1.0 / D;
    const v3 d1 = (2.0 * T.vv) * e1 - (2.0 * T.uv) * e2, d2 = (2.0 * T.uu) * e2 - (2.0 * T.uv) * e1;
    ht[0] = n.x; ht[1] = n.y; ht[2] = n.z;
    ht[3] = g1.x; ht[4] = g1.y; ht[5] = g1.z;
    ht[6] = g2.x; ht[7] = g2.y; ht[8] = g2.z;
    hD[3] = d1.x; hD[4] = d1.y; hD[5] = d1.z;
    hD[6] = d2.x; hD[7] = d2.y; hD[8] = d2.z;
    for (int k = 0; k < 9; ++k) g[k] = (2.0 * T.t * ht[k] - T.s * hD[k]) * T.iD;
  }
  if (lane == 0)
    for (int k = 0; k < 9; ++k) {
      gs[k] = g[k];
      gD[k] = hD[k];
      gt[k] = ht[k];
    }
}

// entry (I i, J j) of the Hessian of |u|^2 |v|^2 - (u.v)^2 (I, J: 0 = u, 1 = v)
__device__ __forceinline__ double lagr_entry(v3 u, v3 v, double uu, double vv, double uv, int I, int i, int J,
                                             int j) {
  const double ui = comp(u, i), uj = comp(u, j), vi = comp(v, i), vj = comp(v, j), dl = i == j ? 1.0 : 0.0;
  if (I == 0 && J == 0) return 2.0 * vv * dl - 2.0 * vi * vj;
  if (I == 1 && J == 1) return 2.0 * uu * dl - 2.0 * ui * uj;
  if (I == 0) return 4.0 * ui * vj - 2.0 * vi * uj - 2.0 * uv * dl;
  return 4.0 * vi * uj - 2.0 * ui * vj - 2.0 * uv * dl;
}

// entry (i, j) of the cross-product matrix [v]x
__device__ __forceinline__ double skew_entry(v3 v, int i, int j) {
  if (i == j) return 0.0;
  const double vk = comp(v, 3 - i - j);
  return ((j - i + 3) % 3 == 2) ? vk : -vk;
}

// entry (a, b) of the Hessian of s in the type's reduced coordinates
__device__ __forceinline__ double hs_entry(const TypeDist& T, const double* gs, const double* gD, const double* gt,
                                           int a, int b) {
  if (T.form == 0) return a == b ? 2.0 : 0.0;
  const int I = a / 3, i = a - 3 * I, J = b / 3, j = b - 3 * J;
  double HN, HD;
  if (T.form == 1) {
    HN = lagr_entry(T.r0, T.r1, T.uu, T.vv, T.uv, I, i, J, j);
    HD = i == j ? (I == J ? 2.0 : -2.0) : 0.0;
  } else {
    HN = 2.0 * gt[a] * gt[b];
    if (I != J) {
      // second derivatives of t = w . (e1 x e2): (w,e1) -[e2]x, (w,e2) [e1]x,
      // (e1,e2) -[w]x, and the transposed blocks with the opposite sign
      double sk;
      if (I + J == 1) sk = (I == 0 ? -1.0 : 1.0) * skew_entry(T.r2, i, j);
      else if (I + J == 2) sk = (I == 0 ? 1.0 : -1.0) * skew_entry(T.r1, i, j);
      else sk = (I == 1 ? -1.0 : 1.0) * skew_entry(T.r0, i, j);
      HN += 2.0 * T.t * sk;
    }
    HD = (I > 0 && J > 0) ? lagr_entry(T.r1, T.r2, T.uu, T.vv, T.uv, I - 1, i, J - 1, j) : 0.0;
  }
  return (HN - T.s * HD - gs[a] * gD[b] - gD[a] * gs[b]) * T.iD;
}

// ---------------------------------------------------------------------------
// round-robin Jacobi
// ---------------------------------------------------------------------------
// partner of index i in round r of the circle schedule over np (even) indices
__device__ __forceinline__ int rr_partner(int r, int i, int np) {
  const int last = np - 1;
  if (i == last) return r;
  if (i == r) return last;
  int j = (2 * r - i) % last;
  return j < 0 ? j + last : j;
}

__device__ __forceinline__ void rot32(float app, float aqq, float apq, float& c, float& s) {
  if (apq == 0.0f) {
    c = 1.0f;
    s = 0.0f;
    return;
  }
  const float theta = (aqq - app) / (2.0f * apq);
  float t;
  if (fabsf(theta) > 1e18f) t = 0.5f / theta;
  else t = copysignf(1.0f, theta) / (fabsf(theta) + sqrtf(theta * theta + 1.0f));
  c = rsqrtf(t * t + 1.0f);
  s = t * c;
}

// FP64 rotation; sc scales the entries into FP32 range (1 / max |K|)
__device__ __forceinline__ void rot64(double app, double aqq, double apq, double sc, double& c, double& s) {
  if (apq == 0.0 || apq * apq <= 1e-36 * fabs(app * aqq)) {  // negligible against its diagonal pair
    c = 1.0;
    s = 0.0;
    return;
  }
  const double dd = aqq - app;
  if (fabs(dd) > 2e4 * fabs(apq)) {
    // |theta| > 1e4: t = 1/(2 theta) (1 - 1/(4 theta^2)).  The quotient is
    // taken in FP32: the rotation stays orthogonal to FP64 rounding
    // (c = 1 - t^2/2 is exact to a relative 1e-17 here) and annihilates
    // K_pq up to a relative 1e-7, which the next sweep squares away.
    const double u = (double)(__fdividef((float)(apq * sc), (float)(dd * sc)));
    const double t = u * (1.0 - u * u);
    c = 1.0 - 0.5 * t * t;
    s = t * c;
    return;
  }
  const double theta = dd / (2.0 * apq);
  const double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
  c = 1.0 / sqrt(t * t + 1.0);
  s = t * c;
}

// one round: n/2 disjoint rotations J (J_pp = J_qq = c, J_pq = s, J_qp = -s)
// chosen to annihilate K_pq, applied as K <- J^T K J, V <- V J into the
// other buffers.  rc[i] = J_ii, rs[i] = J_{partner(i), i}.
// rel (FP32 only): skip a rotation whose off-diagonal entry is below 1e-7 of
// its diagonal pair (the scale-aware test of the second FP32 pass).  Returns
// whether any rotation of the round was taken.
template <int N, typename T, bool REL = false>
__device__ __forceinline__ bool jacobi_round(int r, int lane, const T* Kc, T* Kn, const T* Vc, T* Vn, T* rc, T* rs,
                                             double sc) {
  constexpr int NP = N + (N & 1), last = NP - 1;
  bool took = false;
  if (lane < NP / 2) {
    int p = lane == 0 ? r : (r + lane) % last;
    int q = lane == 0 ? last : (r - lane + last) % last;
    if (p > q) {
      const int t = p;
      p = q;
      q = t;
    }
    if (q < N) {
      T c, s;
      if constexpr (sizeof(T) == 4) {
        const float app = Kc[p * N + p], aqq = Kc[q * N + q], apq = Kc[p * N + q];
        if (REL && fabsf(apq) <= 1e-7f * sqrtf(fabsf(app * aqq))) {
          c = 1.0f;
          s = 0.0f;
        } else {
          rot32(app, aqq, apq, c, s);
        }
      } else {
        rot64(Kc[p * N + p], Kc[q * N + q], Kc[p * N + q], sc, c, s);
      }
      took = s != T(0);
      rc[p] = c;
      rc[q] = c;
      rs[p] = -s;
      rs[q] = s;
    } else {  // partner is the padding index
      rc[p] = T(1);
      rs[p] = T(0);
    }
  }
  __syncwarp();
  // the lane's entries computed together (independent chains), then stored
  constexpr int NE = (N * N + 31) / 32;
  T kn[NE], vn[NE];
#pragma unroll
  for (int it = 0; it < NE; ++it) {
    const int e = min(lane + 32 * it, N * N - 1);
    const int a = e / N, b = e - N * (e / N);
    int pa = rr_partner(r, a, NP), pb = rr_partner(r, b, NP);
    if (pa >= N) pa = a;  // rs[a] == 0 then
    if (pb >= N) pb = b;
    const T ca = rc[a], sa = rs[a], cb = rc[b], sb = rs[b];
    kn[it] = ca * (cb * Kc[a * N + b] + sb * Kc[a * N + pb]) + sa * (cb * Kc[pa * N + b] + sb * Kc[pa * N + pb]);
    vn[it] = cb * Vc[a * N + b] + sb * Vc[a * N + pb];
  }
#pragma unroll
  for (int it = 0; it < NE; ++it) {
    const int e = lane + 32 * it;
    if (e < N * N) {
      Kn[e] = kn[it];
      Vn[e] = vn[it];
    }
  }
  __syncwarp();
  return __ballot_sync(kAll, took) != 0;
}

// out[a N + b] = sum_k X[a xa + k xk] Y[k yk + b yb] (k ascending), the
// lane's entries accumulated together; out must not overlap X or Y
template <int N>
__device__ __forceinline__ void mat_prod(int lane, const double* X, int xa, int xk, const double* Y, int yk, int yb,
                                         double* out) {
  constexpr int NE = (N * N + 31) / 32;
  double acc[NE];
  int ia[NE], ib[NE];
#pragma unroll
  for (int it = 0; it < NE; ++it) {
    const int e = min(lane + 32 * it, N * N - 1);
    ia[it] = e / N;
    ib[it] = e - N * (e / N);
    acc[it] = 0.0;
  }
#pragma unroll
  for (int k = 0; k < N; ++k)
#pragma unroll
    for (int it = 0; it < NE; ++it) acc[it] += X[ia[it] * xa + k * xk] * Y[k * yk + ib[it] * yb];
  __syncwarp();
#pragma unroll
  for (int it = 0; it < NE; ++it) {
    const int e = lane + 32 * it;
    if (e < N * N) out[e] = acc[it];
  }
}

// block congruence out = (R x I) X (R^T x I) for an upper-triangular M x M
// R (3x3 blocks of an N = 3M matrix), per entry in the order c, e2 ascending
template <int N, typename TR>
__device__ __forceinline__ void block_congruence(int lane, const TR* R, const double* X, double* out) {
  constexpr int M = N / 3, NE = (N * N + 31) / 32;
  double acc[NE];
#pragma unroll
  for (int it = 0; it < NE; ++it) {
    const int e = min(lane + 32 * it, N * N - 1);
    const int a = e / N, b = e - N * (e / N);
    const int Ia = a / 3, i = a - 3 * Ia, Jb = b / 3, j = b - 3 * Jb;
    double t = 0.0;
    for (int c = Ia; c < M; ++c)
      for (int e2 = Jb; e2 < M; ++e2) t += R[3 * Ia + c] * R[3 * Jb + e2] * X[(3 * c + i) * N + 3 * e2 + j];
    acc[it] = t;
  }
  __syncwarp();
#pragma unroll
  for (int it = 0; it < NE; ++it) {
    const int e = lane + 32 * it;
    if (e < N * N) out[e] = acc[it];
  }
}

// Newton-Schulz step out = 1.5 V - 0.5 V S (k ascending per entry)
template <int N>
__device__ __forceinline__ void ns_step(int lane, const double* V, const double* S, double* out) {
  constexpr int NE = (N * N + 31) / 32;
  double acc[NE];
  int ia[NE], ib[NE];
#pragma unroll
  for (int it = 0; it < NE; ++it) {
    const int e = min(lane + 32 * it, N * N - 1);
    ia[it] = e / N;
    ib[it] = e - N * (e / N);
    acc[it] = 1.5 * V[ia[it] * N + ib[it]];
  }
#pragma unroll
  for (int k = 0; k < N; ++k)
#pragma unroll
    for (int it = 0; it < NE; ++it) acc[it] -= 0.5 * V[ia[it] * N + k] * S[k * N + ib[it]];
  __syncwarp();
#pragma unroll
  for (int it = 0; it < NE; ++it) {
    const int e = lane + 32 * it;
    if (e < N * N) out[e] = acc[it];
  }
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kAll, v, o);
  return v;
}

// off-diagonal and total sums of squares of an N x N matrix, over the warp
template <int N, typename T>
__device__ __forceinline__ void off_tot(const T* K, int lane, T& off, T& tot) {
  off = T(0);
  tot = T(0);
  for (int e = lane; e < N * N; e += 32) {
    const T v = K[e] * K[e];
    tot += v;
    if (e / N != e - N * (e / N)) off += v;
  }
  off = warp_sum(off);
  tot = warp_sum(tot);
}

// squares of the couplings between indices of opposite diagonal sign (the
// only off-diagonal entries that change the clamp), and the total
template <int N>
__device__ __forceinline__ void off_cross_tot(const double* K, int lane, double& off, double& tot) {
  off = 0.0;
  tot = 0.0;
  for (int e = lane; e < N * N; e += 32) {
    const int a = e / N, b = e - N * (e / N);
    const double v = K[e] * K[e];
    tot += v;
    if ((K[a * N + a] > 0.0) != (K[b * N + b] > 0.0)) off += v;
  }
  off = warp_sum(off);
  tot = warp_sum(tot);
}

// ---------------------------------------------------------------------------
// per-warp scratch
// ---------------------------------------------------------------------------
struct WarpScratch {
  double H[81];
  double Kd[2][81];
  double Vd[2][81];
  float K32[2][81];
  float V32[2][81];
  double vec[6][9];  // gs, gD, gt, gr, gb, gc
  double Rm[9], Ri[9], C[12], A[9];
  float Ri32[9];
  double rc[10], rs[10];
  float rc32[10], rs32[10];
};

// one 6- or 9-dimensional term by the whole warp
template <int N>
__device__ void warp_term(int f, int lane, WarpScratch& W, const int4* __restrict__ termv,
                          const int* __restrict__ tmeta, const double* __restrict__ teps,
                          const double* __restrict__ td2, const double4* x, double dhat, double kappa, int project,
                          int mixed, const GramTables& gram, double* term, DevStatus* st) {
  constexpr int M = N / 3;
  const int4 vv = termv[f];
  const int meta = tmeta[f];
  const int kind = meta & 1, type = (meta >> 1) & 15, moll = (meta >> 5) & 1;
  const v3 xs[4] = {mk(x[vv.x]), mk(x[vv.y]), mk(x[vv.z]), mk(x[vv.w])};
  Reduced R;  // working frame
  reduce(kind, moll ? 8 : type, xs, R);
  Reduced Rt;  // the type's own frame (differs from R only when mollified)
  reduce(kind, type, xs, Rt);
  double *gs = W.vec[0], *gD = W.vec[1], *gt = W.vec[2], *gr = W.vec[3], *gb = W.vec[4], *gc = W.vec[5];
  TypeDist T;
  type_dist(Rt, T, gs, gD, gt, lane);
  // the barrier's scalar factors at the canonical squared distance (the value
  // that decides membership); the derivatives of s come from the type's form
  const double sc = td2[f];
  const double d = sqrt(sc);
  double B, B1, B2;
  barrier_derivs(d, dhat, B, B1, B2);
  const double cg = kappa * B1 / (2.0 * d);
  const double ca = kappa * (B2 / (4.0 * sc) - B1 / (4.0 * d * sc));
  const double Eb = kappa * B;
  const int gcls = gram_class(kind, type, moll);
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
      for (int w = 0; w < 3; ++w) W.C[3 * k + w] = R.C[k][w];
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      W.Rm[k] = gcls == 1 ? gram.Rm[1][k] : (gcls == 2 ? gram.Rm[2][k] : gram.Rm[3][k]);
      W.Ri[k] = gcls == 1 ? gram.Ri[1][k] : (gcls == 2 ? gram.Ri[2][k] : gram.Ri[3][k]);
      W.Ri32[k] = (float)W.Ri[k];
    }
  }
  __syncwarp();
  double E;
  if (!moll) {
    {
      constexpr int NE = (N * N + 31) / 32;
      double h[NE];
#pragma unroll
      for (int it = 0; it < NE; ++it) {
        const int e = min(lane + 32 * it, N * N - 1);
        const int a = e / N, b = e - N * (e / N);
        h[it] = ca * gs[a] * gs[b] + cg * hs_entry(T, gs, gD, gt, a, b);
      }
#pragma unroll
      for (int it = 0; it < NE; ++it)
        if (lane + 32 * it < N * N) W.H[lane + 32 * it] = h[it];
    }
    if (lane < N) gr[lane] = cg * gs[lane];
    E = Eb;
  } else {
    // kappa B in the type's coordinates, pulled back to y = (w, e0, e1)
    const int nt = T.n, mt = nt / 3;
    double* Ht = W.Kd[1];
    for (int e = lane; e < nt * nt; e += 32) {
      const int a = e / nt, b = e - nt * (e / nt);
      Ht[e] = ca * gs[a] * gs[b] + cg * hs_entry(T, gs, gD, gt, a, b);
    }
    const v3 e0 = R.r[1], e1 = R.r[2];
    const double e00 = dot(e0, e0), e11 = dot(e1, e1), e01 = dot(e0, e1);
    if (lane == 0) {
      double A[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
#pragma unroll
      for (int w = 0; w < 3; ++w)
        if (w < mt) {
          A[w][0] = Rt.C[2][w] + Rt.C[3][w];
          A[w][1] = Rt.C[1][w];
          A[w][2] = Rt.C[3][w];
        }
#pragma unroll
      for (int k = 0; k < 9; ++k) W.A[k] = A[k / 3][k % 3];
#pragma unroll
      for (int J = 0; J < 3; ++J)
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          double t = 0.0;
#pragma unroll
          for (int w = 0; w < 3; ++w)
            if (w < mt) t += A[w][J] * gs[3 * w + i];
          gb[3 * J + i] = cg * t;
        }
      // c = |e0 x e1|^2 = |e0|^2 |e1|^2 - (e0.e1)^2 in slots e0 = 1, e1 = 2
      const v3 gu = (2.0 * e11) * e0 - (2.0 * e01) * e1, gv = (2.0 * e00) * e1 - (2.0 * e01) * e0;
      gc[0] = gc[1] = gc[2] = 0.0;
      gc[3] = gu.x; gc[4] = gu.y; gc[5] = gu.z;
      gc[6] = gv.x; gc[7] = gv.y; gc[8] = gv.z;
    }
    double dm, d2m;
    const double mv = ee_mollifier(ee_cross2(xs), teps[f], dm, d2m);
    __syncwarp();
    for (int e = lane; e < 81; e += 32) {
      const int a = e / 9, b = e - 9 * (e / 9);
      const int I = a / 3, i = a - 3 * I, J = b / 3, j = b - 3 * J;
      double Hb = 0.0;
      for (int w = 0; w < mt; ++w) {
        const double aw = W.A[3 * w + I];
        if (aw == 0.0) continue;
        for (int v = 0; v < mt; ++v) Hb += aw * W.A[3 * v + J] * Ht[(3 * w + i) * nt + 3 * v + j];
      }
      const double Hc = (I > 0 && J > 0) ? lagr_entry(e0, e1, e00, e11, e01, I - 1, i, J - 1, j) : 0.0;
      // product rule: m Hb + Eb (m'' gc gc^T + m' Hc) + m' (gc gb^T + gb gc^T)
      W.H[e] = mv * Hb + Eb * (d2m * gc[a] * gc[b] + dm * Hc) + dm * (gc[a] * gb[b] + gb[a] * gc[b]);
    }
    if (lane < 9) gr[lane] = mv * gb[lane] + Eb * dm * gc[lane];
    E = Eb * mv;
  }
  __syncwarp();
  const double* Hr = W.H;
  if (project) {
    double* K = W.Kd[0];
    block_congruence<N>(lane, W.Rm, W.H, K);
    __syncwarp();
    double mx = 0.0;
    for (int e = lane; e < N * N; e += 32) mx = fmax(mx, fabs(K[e]));
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(kAll, mx, o));
    double* P = W.H;  // projected K, then back in the difference coordinates
    if (mx > 0.0 && mx < INFINITY) {
      // FP32 eigenbasis of K / max|K|
      const double inv = 1.0 / mx;
      for (int e = lane; e < N * N; e += 32) {
        W.K32[0][e] = (float)(K[e] * inv);
        W.V32[0][e] = (e / N == e - N * (e / N)) ? 1.0f : 0.0f;
      }
      __syncwarp();
      constexpr int NP = N + (N & 1);
      int cur = 0, n32 = 0, n64 = 0, capped = 0;
      float prev = INFINITY;
      for (int sweep = 0; sweep < 12; ++sweep) {
        float off, tot;
        off_tot<N>(W.K32[cur], lane, off, tot);
        if (!(off > 1e-13f * tot)) break;
        if (off < 1e-9f * tot && off > 0.25f * prev) break;  // at the FP32 rounding floor
        prev = off;
        ++n32;
        for (int r = 0; r < NP - 1; ++r) {
          jacobi_round<N, float>(r, lane, W.K32[cur], W.K32[cur ^ 1], W.V32[cur], W.V32[cur ^ 1], W.rc32, W.rs32,
                                 1.0);
          cur ^= 1;
        }
      }
      if (mixed) {
        // mixed precision: the clamp from the FP32 eigenpairs, no FP64
        // refinement.  The factor G = (Ri x I) V sqrt(max(lambda, 0)) is
        // formed in FP32 and the clamped block as G G^T in FP64, so the block
        // is positive semidefinite to FP64 rounding (an FP32 product would
        // leave negative eigenvalues of ~1e-7 of the largest, enough to make
        // a light body's diagonal block indefinite)
        const float* Kc = W.K32[cur];
        const float* Vc = W.V32[cur];
        float* Gv = W.K32[cur ^ 1];
        for (int e = lane; e < N * N; e += 32) {  // V sqrt(lambda+)
          const int a = e / N, k = e - N * (e / N);
          const float lam = Kc[k * N + k];
          Gv[e] = lam > 0.0f ? Vc[a * N + k] * sqrtf(lam) : 0.0f;
        }
        __syncwarp();
        double* G = W.Vd[0];
        for (int e = lane; e < N * N; e += 32) {  // (Ri x I) V sqrt(lambda+)
          const int a = e / N, k = e - N * (e / N);
          const int Ia = a / 3, i = a - 3 * Ia;
          float t = 0.0f;
          for (int c = Ia; c < M; ++c) t += W.Ri32[3 * Ia + c] * Gv[(3 * c + i) * N + k];
          G[e] = (double)t;
        }
        __syncwarp();
        for (int e = lane; e < N * N; e += 32) {
          const int a = e / N, b = e - N * (e / N);
          double t = 0.0;
          for (int k = 0; k < N; ++k) t += G[a * N + k] * G[b * N + k];
          P[e] = t * mx;
        }
        if (lane == 0) atomicAdd(&st->jac[0], (unsigned long long)n32);
      } else {
      // FP64 refinement: V <- V (3I - V^T V) / 2, K' = V^T K V, FP64 sweeps
      double *V0 = W.Vd[0], *V1 = W.Vd[1], *S = W.H;
      for (int e = lane; e < N * N; e += 32) V0[e] = (double)W.V32[cur][e];
      __syncwarp();
      mat_prod<N>(lane, V0, 1, N, V0, N, 1, S);  // S = V0^T V0
      __syncwarp();
      ns_step<N>(lane, V0, S, V1);
      __syncwarp();
      double* KV = W.H;
      mat_prod<N>(lane, K, N, 1, V1, N, 1, KV);  // K V1
      __syncwarp();
      mat_prod<N>(lane, V1, 1, N, KV, N, 1, W.Kd[1]);  // V1^T (K V1)
      __syncwarp();
      for (int e = lane; e < N * N; e += 32) {
        const int a = e / N, b = e - N * (e / N);
        K[e] = 0.5 * (W.Kd[1][a * N + b] + W.Kd[1][b * N + a]);
      }
      __syncwarp();
      // second FP32 pass on K' (floating point keeps the lower levels of the
      // spectrum, which the first pass on K / max|K| could not resolve), a
      // scale-aware skip test, until a sweep takes no rotation; then the
      // basis update in FP64: V2 <- V2 (3I - V2^T V2) / 2, K'' = V2^T K' V2,
      // V = V' V2
      {
        double mx2 = 0.0;
        for (int e = lane; e < N * N; e += 32) mx2 = fmax(mx2, fabs(K[e]));
        for (int o = 16; o > 0; o >>= 1) mx2 = fmax(mx2, __shfl_xor_sync(kAll, mx2, o));
        const double inv2 = 1.0 / mx2;
        for (int e = lane; e < N * N; e += 32) {
          W.K32[0][e] = (float)(K[e] * inv2);
          W.V32[0][e] = (e / N == e - N * (e / N)) ? 1.0f : 0.0f;
        }
        __syncwarp();
        int c2 = 0;
        for (int sweep = 0; sweep < 5; ++sweep) {
          bool any = false;
          for (int r = 0; r < NP - 1; ++r) {
            any |= jacobi_round<N, float, true>(r, lane, W.K32[c2], W.K32[c2 ^ 1], W.V32[c2], W.V32[c2 ^ 1], W.rc32,
                                                W.rs32, 1.0);
            c2 ^= 1;
          }
          ++n32;
          if (!any) break;
        }
        double* V2 = W.Vd[0];  // free: the first basis lives in V1
        for (int e = lane; e < N * N; e += 32) V2[e] = (double)W.V32[c2][e];
        __syncwarp();
        mat_prod<N>(lane, V2, 1, N, V2, N, 1, W.H);  // S = V2^T V2 into H
        __syncwarp();
        double* V2n = W.Kd[1];
        ns_step<N>(lane, V2, W.H, V2n);
        __syncwarp();
        mat_prod<N>(lane, K, N, 1, V2n, N, 1, W.H);  // K' V2 into H
        __syncwarp();
        mat_prod<N>(lane, V2n, 1, N, W.H, N, 1, V2);  // K'' = V2^T (K' V2) into Vd[0]
        __syncwarp();
        mat_prod<N>(lane, V1, N, 1, V2n, N, 1, W.H);  // V = V' V2 into H
        __syncwarp();
        for (int e = lane; e < N * N; e += 32) {
          const int a = e / N, b = e - N * (e / N);
          K[e] = 0.5 * (V2[a * N + b] + V2[b * N + a]);
          V1[e] = W.H[e];
        }
      }
      // current: K in Kd[0], V in Vd[1]
      double* Kb[2] = {W.Kd[0], W.Kd[1]};
      double* Vb[2] = {W.Vd[1], W.Vd[0]};
      int c64 = 0;
      __syncwarp();
      for (int sweep = 0; sweep <= 8; ++sweep) {
        double off, tot;
        off_cross_tot<N>(Kb[c64], lane, off, tot);
        if (!(off > 1e-22 * tot)) break;
        if (sweep == 8) {  // cap reached: keep the last basis
          capped = 1;
          break;
        }
        ++n64;
        for (int r = 0; r < NP - 1; ++r) {
          jacobi_round<N, double>(r, lane, Kb[c64], Kb[c64 ^ 1], Vb[c64], Vb[c64 ^ 1], W.rc, W.rs, inv);
          c64 ^= 1;
        }
      }
      if (lane == 0) {
        atomicAdd(&st->jac[0], (unsigned long long)n32);
        atomicAdd(&st->jac[1], (unsigned long long)n64);
        if (capped) atomicAdd(&st->jac[2], 1ull);
      }
      // Proj = V P V^T with P the block of K'' on its positive diagonal
      // entries: couplings inside that block are kept exactly, couplings to
      // the clamped part are below the threshold above
      const double* Kf = Kb[c64];
      const double* Vf = Vb[c64];
      double* Pk = W.Kd[c64 ^ 1];
      for (int e = lane; e < N * N; e += 32) {  // T = V P into H
        const int a = e / N, l = e - N * (e / N);
        double t = 0.0;
        if (Kf[l * N + l] > 0.0)
          for (int k = 0; k < N; ++k)
            if (Kf[k * N + k] > 0.0) t += Vf[a * N + k] * Kf[k * N + l];
        W.H[e] = t;
      }
      __syncwarp();
      mat_prod<N>(lane, W.H, N, 1, Vf, 1, N, Pk);  // T V^T
      __syncwarp();
      // back to the difference coordinates: (Ri x I) Proj (Ri^T x I)
      block_congruence<N>(lane, W.Ri, Pk, P);
      }  // FP64 refinement
    } else {
      for (int e = lane; e < N * N; e += 32) P[e] = 0.0;
    }
    __syncwarp();
    Hr = P;
  }
  // vertex gradient, packed upper vertex Hessian H12 = T Hr T^T, energy
  double* Tt = term + (size_t)f * kTermStride;
  if (lane < 12) {
    const int k = lane / 3, ci = lane - 3 * k;
    double t = 0.0;
#pragma unroll
    for (int w = 0; w < M; ++w) t += W.C[3 * k + w] * gr[3 * w + ci];
    Tt[1 + lane] = t;
  }
  for (int e = lane; e < 78; e += 32) {
    int row = 0, rem = e;
    while (rem >= 12 - row) {
      rem -= 12 - row;
      ++row;
    }
    const int col = row + rem;
    const int k = row / 3, ci = row - 3 * k, l = col / 3, cj = col - 3 * l;
    double t = 0.0;
#pragma unroll
    for (int v = 0; v < M; ++v) {
      const double ckv = W.C[3 * k + v];
      if (ckv == 0.0) continue;
#pragma unroll
      for (int w = 0; w < M; ++w) t += ckv * W.C[3 * l + w] * Hr[(3 * v + ci) * N + 3 * w + cj];
    }
    Tt[13 + e] = t;
  }
  if (lane == 0) {
    Tt[0] = E;
    atomicAdd(&st->bar_terms[M], 1ull);
  }
  __syncwarp();  // the scratch is reused by the next term
}

// one point-point term by one thread (closed-form projection)
__device__ __forceinline__ void pp_term(int f, const int4* __restrict__ termv, const int* __restrict__ tmeta,
                                        const double* __restrict__ td2, const double4* x, double dhat, double kappa,
                                        int project, double* term) {
  const int4 vv = termv[f];
  const int meta = tmeta[f];
  const int kind = meta & 1, type = (meta >> 1) & 15;
  const v3 xs[4] = {mk(x[vv.x]), mk(x[vv.y]), mk(x[vv.z]), mk(x[vv.w])};
  Reduced R;
  reduce(kind, type, xs, R);
  const v3 e = R.r[0];
  const double s = dot(e, e);             // |e|^2 of the difference vector
  const double sc = td2[f], d = sqrt(sc);  // the canonical distance, for the barrier's factors
  double B, B1, B2;
  barrier_derivs(d, dhat, B, B1, B2);
  const double cg = kappa * B1 / (2.0 * d);
  const double ca = kappa * (B2 / (4.0 * sc) - B1 / (4.0 * d * sc));
  // H_r = h0 e e^T + h1 I
  double h0 = 4.0 * ca, h1 = 2.0 * cg;
  if (project) {
    const double lu = fmax(h0 * s + h1, 0.0), lp = fmax(h1, 0.0);
    h0 = (lu - lp) / s;
    h1 = lp;
  }
  double ck[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) ck[k] = R.C[k][0];
  const double ev[3] = {e.x, e.y, e.z};
  double* Tt = term + (size_t)f * kTermStride;
  Tt[0] = kappa * B;
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int i = 0; i < 3; ++i) Tt[1 + 3 * k + i] = ck[k] * (2.0 * cg * ev[i]);
  int idx = 13;
#pragma unroll
  for (int row = 0; row < 12; ++row)
#pragma unroll
    for (int col = row; col < 12; ++col) {
      const int k = row / 3, i = row % 3, l = col / 3, j = col % 3;
      Tt[idx++] = ck[k] * ck[l] * (h0 * ev[i] * ev[j] + (i == j ? h1 : 0.0));
    }
}

__global__ void __launch_bounds__(32 * kBarWarps, kBarMinBlocks) k_barrier(const DevStatus* __restrict__ cst, const int* tlist, long cap,
                                                            const int4* __restrict__ termv,
                                                            const int* __restrict__ tmeta,
                                                            const double* __restrict__ teps,
                                                            const double* __restrict__ td2, const double4* x,
                                                            double dhat, double kappa, int project, int mixed,
                                                            GramTables gram, double* term, DevStatus* st) {
  __shared__ WarpScratch scratch[kBarWarps];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  WarpScratch& W = scratch[warp];
  const int n3 = cst->bar_cnt[0], n6 = cst->bar_cnt[1], n9 = cst->bar_cnt[2];
  const int wpp = (n3 + 31) / 32;
  const long total = (long)n9 + n6 + wpp;
  const long nwarps = (long)gridDim.x * kBarWarps;
  // heaviest work first: 9-dimensional terms, then 6-dimensional, then
  // point-point terms 32 to a warp
  for (long t = (long)blockIdx.x * kBarWarps + warp; t < total; t += nwarps) {
    if (t < n9) {
      warp_term<9>(tlist[2 * cap + t], lane, W, termv, tmeta, teps, td2, x, dhat, kappa, project, mixed, gram, term,
                   st);
    } else if (t < n9 + n6) {
      warp_term<6>(tlist[cap + (t - n9)], lane, W, termv, tmeta, teps, td2, x, dhat, kappa, project, mixed, gram,
                   term, st);
    } else {
      const long k = (t - n9 - n6) * 32 + lane;
      const bool ok = k < n3;
      if (ok) pp_term(tlist[k], termv, tmeta, td2, x, dhat, kappa, project, term);
      const unsigned m = __ballot_sync(kAll, ok);
      if (lane == 0) atomicAdd(&st->bar_terms[1], (unsigned long long)__popc(m));
    }
  }
}

}  // namespace

void launch_barrier(Scene& s, int project, long cap) {
  static const GramTables gram = make_gram();
  counted(s, 2);
  ProfScope ps(s, PF_BARRIER);
  cudaMemsetAsync(reinterpret_cast<char*>(s.st) + offsetof(DevStatus, bar_cnt), 0, sizeof(int) * 4, s.stream);
  k_bar_classify<<<sm_grid(s, 8), 256, 0, s.stream>>>(s.st, s.aoff.p, s.act.p, s.act_d2.p, s.tri.p, s.edge.p, s.x.p,
                                                s.l2e.p, s.maxc, cap, s.termv.p, s.tmeta.p, s.teps.p, s.td2.p,
                                                s.tlist.p, s.st);
  k_barrier<<<sm_grid(s, 8), 32 * kBarWarps, 0, s.stream>>>(s.st, s.tlist.p, cap, s.termv.p, s.tmeta.p, s.teps.p, s.td2.p,
                                                      s.x.p,
                                                      s.prm.dhat, s.prm.kappa, project, s.fp32_proj ? 1 : 0,
                                                      gram, s.term.p, s.st);
}

}  // namespace abd
