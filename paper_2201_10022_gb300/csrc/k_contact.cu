// Contact kernels: primitive candidate enumeration per body pair with the
// d-hat box test (Sec. 4.2, i-AABB culling restated per body pair), additive
// CCD over linear trajectories (Sec. 4.1), active-set detection, barrier and
// friction terms (Sec. 4) and their energies.
#include <float.h>

#include "abd_internal.cuh"
#include "derivs.cuh"

namespace abd {

namespace {

constexpr int kWarpsPerBlock = 4;
constexpr int kChunk = 64;
constexpr unsigned kFull = 0xffffffffu;

struct Box {
  double lo[3], hi[3];
};

__device__ __forceinline__ void box_point(Box& b, const double4& p) {
  b.lo[0] = b.hi[0] = p.x;
  b.lo[1] = b.hi[1] = p.y;
  b.lo[2] = b.hi[2] = p.z;
}
__device__ __forceinline__ void box_add(Box& b, const double4& p) {
  b.lo[0] = fmin(b.lo[0], p.x);
  b.hi[0] = fmax(b.hi[0], p.x);
  b.lo[1] = fmin(b.lo[1], p.y);
  b.hi[1] = fmax(b.hi[1], p.y);
  b.lo[2] = fmin(b.lo[2], p.z);
  b.hi[2] = fmax(b.hi[2], p.z);
}
// canonical proximity test: on every axis lo_P - hi_Q <= dhat and lo_Q - hi_P <= dhat
__device__ __forceinline__ bool box_near(const double* plo, const double* phi, const double* qlo, const double* qhi,
                                         double dhat) {
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    if (!(__dsub_rn(plo[k], qhi[k]) <= dhat)) return false;
    if (!(__dsub_rn(qlo[k], phi[k]) <= dhat)) return false;
  }
  return true;
}

// box of primitive `id` of type t (0 vertex, 1 edge, 2 triangle)
__device__ __forceinline__ void prim_box(int t, int id, const int* tri, const int* edge, const double4* x,
                                         const double4* x1, Box& b) {
  int nvtx = t == 0 ? 1 : (t == 1 ? 2 : 3);
  int v0 = t == 0 ? id : (t == 1 ? edge[2 * id] : tri[3 * id]);
  box_point(b, x[v0]);
  if (x1) box_add(b, x1[v0]);
  for (int k = 1; k < nvtx; ++k) {
    int v = t == 1 ? edge[2 * id + k] : tri[3 * id + k];
    box_add(b, x[v]);
    if (x1) box_add(b, x1[v]);
  }
}

__device__ __forceinline__ void pair_vertices(int kind, int i, int j, const int* tri, const int* edge, int v[4]) {
  if (kind == 0) {
    v[0] = i;
    v[1] = tri[3 * j];
    v[2] = tri[3 * j + 1];
    v[3] = tri[3 * j + 2];
  } else {
    v[0] = edge[2 * i];
    v[1] = edge[2 * i + 1];
    v[2] = edge[2 * j];
    v[3] = edge[2 * j + 1];
  }
}

__device__ __forceinline__ void set_flag(DevStatus* st, unsigned f) { atomicOr(&st->flags, f); }

struct WarpLists {
  int pid[kChunk], qid[kChunk];
  double pb[kChunk][6], qb[kChunk][6];
};

// Fill a chunk of primitives of type t from [cur, hi) that pass the box test
// against the other body's box; returns the new cursor.
__device__ int fill_chunk(int t, int cur, int hi, const double* olo, const double* ohi, double dhat, const int* tri,
                          const int* edge, const double4* x, const double4* x1, int* ids, double (*boxes)[6],
                          int& n) {
  const int lane = threadIdx.x & 31;
  n = 0;
  while (cur < hi && n <= kChunk - 32) {
    int id = cur + lane;
    bool ok = false;
    Box b;
    if (id < hi) {
      prim_box(t, id, tri, edge, x, x1, b);
      ok = box_near(b.lo, b.hi, olo, ohi, dhat);
    }
    unsigned m = __ballot_sync(kFull, ok);
    if (ok) {
      int pos = n + __popc(m & ((1u << lane) - 1u));
      ids[pos] = id;
      for (int k = 0; k < 3; ++k) {
        boxes[pos][k] = b.lo[k];
        boxes[pos][3 + k] = b.hi[k];
      }
    }
    n += __popc(m);
    cur += 32;
  }
  __syncwarp();
  return cur;
}

// Enumerate the candidates of one kind between primitive ranges of two
// bodies.  P side: vertices (PT) or edges (EE) of body `pa`; Q side:
// triangles (PT) or edges (EE) of body `qa`.
__device__ void enum_kind(int kind, int p_lo, int p_hi, int q_lo, int q_hi, const Box& boxP, const Box& boxQ,
                          double dhat, const int* tri, const int* edge, const double4* x, const double4* x1,
                          const double4* dx, WarpLists& L, int2* out, int maxc, int& base, bool ccd, double ccd_s,
                          int ccd_max, double& tmin, DevStatus* st) {
  const int lane = threadIdx.x & 31;
  const int tp = kind == 0 ? 0 : 1, tq = kind == 0 ? 2 : 1;
  int qc = q_lo;
  while (qc < q_hi) {
    int nq;
    qc = fill_chunk(tq, qc, q_hi, boxP.lo, boxP.hi, dhat, tri, edge, x, x1, L.qid, L.qb, nq);
    if (nq == 0) continue;
    int pc = p_lo;
    while (pc < p_hi) {
      int npp;
      pc = fill_chunk(tp, pc, p_hi, boxQ.lo, boxQ.hi, dhat, tri, edge, x, x1, L.pid, L.pb, npp);
      const int tot = npp * nq;
      for (int t0 = 0; t0 < tot; t0 += 32) {
        int t = t0 + lane;
        bool c = false;
        int pi = 0, qi = 0;
        if (t < tot) {
          pi = t / nq;
          qi = t - pi * nq;
          c = box_near(L.pb[pi], L.pb[pi] + 3, L.qb[qi], L.qb[qi] + 3, dhat);
        }
        unsigned m = __ballot_sync(kFull, c);
        if (c) {
          int pos = base + __popc(m & ((1u << lane) - 1u));
          int i = L.pid[pi], j = L.qid[qi];
          if (pos < maxc) out[pos] = make_int2(i | (kind << 31), j);
          if (ccd) {
            int v[4];
            pair_vertices(kind, i, j, tri, edge, v);
            v3 xs[4], ds[4];
            for (int k = 0; k < 4; ++k) {
              xs[k] = mk(x[v[k]]);
              ds[k] = mk(dx[v[k]]);
            }
            double toi;
            if (accd(kind, xs, ds, ccd_s, 1.0, ccd_max, toi)) set_flag(st, ST_CCD_MAXITER);
            tmin = fmin(tmin, toi);
          }
        }
        base += __popc(m);
      }
      __syncwarp();
    }
  }
}

__global__ void k_enumerate(const int2* __restrict__ P, const DevStatus* __restrict__ cst, const int* vbeg,
                            const int* tbeg, const int* ebeg, const int* tri, const int* edge, const double4* x,
                            const double4* x1, const double4* dx, const double* bbox, double dhat, int maxc,
                            int2* cand, int* ccount, bool ccd, double ccd_s, int ccd_max, DevStatus* st) {
  __shared__ WarpLists lists[kWarpsPerBlock];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nwarps = gridDim.x * kWarpsPerBlock;
  const int np = cst->np;
  WarpLists& L = lists[warp];
  double tmin = 1.0;
  unsigned long long ncand = 0;
  for (int p = blockIdx.x * kWarpsPerBlock + warp; p < np; p += nwarps) {
    const int a = P[p].x, b = P[p].y;
    Box Ba, Bb;
    for (int k = 0; k < 3; ++k) {
      Ba.lo[k] = bbox[6 * a + k];
      Ba.hi[k] = bbox[6 * a + 3 + k];
      Bb.lo[k] = bbox[6 * b + k];
      Bb.hi[k] = bbox[6 * b + 3 + k];
    }
    int base = 0;
    int2* out = cand + (size_t)p * maxc;
    // vertices of a against triangles of b, vertices of b against triangles of a
    enum_kind(0, vbeg[a], vbeg[a + 1], tbeg[b], tbeg[b + 1], Ba, Bb, dhat, tri, edge, x, x1, dx, L, out, maxc, base,
              ccd, ccd_s, ccd_max, tmin, st);
    enum_kind(0, vbeg[b], vbeg[b + 1], tbeg[a], tbeg[a + 1], Bb, Ba, dhat, tri, edge, x, x1, dx, L, out, maxc, base,
              ccd, ccd_s, ccd_max, tmin, st);
    // edges of a against edges of b
    enum_kind(1, ebeg[a], ebeg[a + 1], ebeg[b], ebeg[b + 1], Ba, Bb, dhat, tri, edge, x, x1, dx, L, out, maxc, base,
              ccd, ccd_s, ccd_max, tmin, st);
    if (lane == 0) {
      ccount[p] = base;
      if (base > maxc) {
        set_flag(st, ST_CAP_CANDS);
        atomicMax(&st->need_cand, base);
      }
    }
    ncand += base;
  }
  if (ccd) {
    for (int o = 16; o > 0; o >>= 1) tmin = fmin(tmin, __shfl_xor_sync(kFull, tmin, o));
    if (lane == 0 && tmin < 1.0) atomicMin(&st->toi_bits, (unsigned long long)__double_as_longlong(tmin));
  }
  if (lane == 0 && ncand) atomicAdd(&st->n_cand, ncand);
}

// active pairs: canonical d^2 < dhat^2, compacted per body pair in slot order
__global__ void k_active(const int2* __restrict__ P, const DevStatus* __restrict__ cst, const int2* cand,
                         const int* ccount, const int* tri, const int* edge, const double4* x, double dhat, int maxc,
                         int4* act, double* act_d2, int* acount, DevStatus* st) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nwarps = gridDim.x * (blockDim.x >> 5);
  const int np = cst->np;
  const double dh2 = __dmul_rn(dhat, dhat);
  for (int p = blockIdx.x * (blockDim.x >> 5) + warp; p < np; p += nwarps) {
    const int n = min(ccount[p], maxc);
    int base = 0;
    for (int k0 = 0; k0 < n; k0 += 32) {
      int k = k0 + lane;
      bool a = false;
      int type = 0;
      double d2 = 0.0;
      int2 c = make_int2(0, 0);
      if (k < n) {
        c = cand[(size_t)p * maxc + k];
        int kind = (unsigned)c.x >> 31, i = c.x & 0x7fffffff;
        int v[4];
        pair_vertices(kind, i, c.y, tri, edge, v);
        v3 xs[4];
        for (int m = 0; m < 4; ++m) xs[m] = mk(x[v[m]]);
        d2 = pair_dist2(kind, xs, type);
        a = d2 < dh2;
        if (a && d2 == 0.0) set_flag(st, ST_INTERSECT);
        if (!(d2 == d2)) set_flag(st, ST_NONFINITE);
      }
      unsigned m = __ballot_sync(kFull, a);
      if (a) {
        int pos = base + __popc(m & ((1u << lane) - 1u));
        act[(size_t)p * maxc + pos] = make_int4(c.x, c.y, type, 0);
        act_d2[(size_t)p * maxc + pos] = d2;
      }
      base += __popc(m);
    }
    if (lane == 0) acount[p] = base;
  }
}

__device__ __forceinline__ int owner(const int* off, int n, int f) {
  // largest p with off[p] <= f (off has n+1 entries, nondecreasing)
  int lo = 0, hi = n;
  while (hi - lo > 1) {
    int mid = (lo + hi) >> 1;
    if (off[mid] <= f) lo = mid;
    else hi = mid;
  }
  return lo;
}

// barrier terms: energy, vertex gradient and projected vertex Hessian.
// Nine lanes work on one pair (three pairs per warp): lane 0 forms the
// Hessian in the type's reduced coordinates, then the lanes share the
// congruence with the Gram factor, the Jacobi rotations of the 9x9 (6x6, 3x3)
// eigenproblem (one matrix row per lane), the eigenvalue clamp and the
// expansion to the 12x12 vertex Hessian.
constexpr int kBarWarps = 4;
constexpr int kGroups = 3, kGroupLanes = 9;

struct BarrierShared {
  double H[kBarWarps][kGroups][81];
  double K[kBarWarps][kGroups][81];
  double V[kBarWarps][kGroups][81];
  float K32[kBarWarps][kGroups][81];
  float V32[kBarWarps][kGroups][81];
  double lam[kBarWarps][kGroups][9];
  double g[kBarWarps][kGroups][9];
  double red[kBarWarps][kGroups][2 * kGroupLanes];
  double E[kBarWarps][kGroups];
};

__global__ void __launch_bounds__(32 * kBarWarps) k_barrier(const DevStatus* __restrict__ cst, const int* aoff,
                                                            const int4* act, const int* tri, const int* edge,
                                                            const double4* x, const double* l2e, double dhat,
                                                            double kappa, int maxc, int project, long cap,
                                                            double* term, int4* termv, DevStatus* st) {
  __shared__ BarrierShared sh;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int grp = lane / kGroupLanes, gl = lane - grp * kGroupLanes;
  if (grp >= kGroups) return;  // lanes 27..31 idle
  const unsigned gmask = 0x1FFu << (kGroupLanes * grp);
  const int np = cst->np, nact = (int)min((long)cst->nact, cap);
  double* H = sh.H[warp][grp];
  double* K = sh.K[warp][grp];
  double* V = sh.V[warp][grp];
  double* red = sh.red[warp][grp];
  const long stride = (long)gridDim.x * kBarWarps * kGroups;
  for (long f = ((long)blockIdx.x * kBarWarps + warp) * kGroups + grp; f < nact; f += stride) {
    const int p = owner(aoff, np, (int)f);
    const int4 r = act[(size_t)p * maxc + (f - aoff[p])];
    const int kind = (unsigned)r.x >> 31, i = r.x & 0x7fffffff;
    int v[4];
    pair_vertices(kind, i, r.y, tri, edge, v);
    v3 xs[4];
    for (int m = 0; m < 4; ++m) xs[m] = mk(x[v[m]]);
    // a mollified edge-edge pair is worked in the line-line coordinates
    double c = 0.0, eps = 0.0;
    bool moll = false;
    if (kind == 1) {
      c = ee_cross2(xs);
      eps = ee_eps(l2e[i], l2e[r.y]);
      moll = c < eps;
    }
    Reduced R;
    reduce(kind, moll ? 8 : r.z, xs, R);
    const int m = R.m, n3 = 3 * m;
    if (gl == 0 && moll) {
      sh.E[warp][grp] = mollified_ee_term(r.z, xs, dhat, kappa, c, eps, sh.g[warp][grp], H);
    } else if (gl == 0) {
      double gs[9], Hs[81];
      const double s = reduced_dist2(R, gs, Hs);
      const double d = sqrt(s);
      double B, B1, B2;
      barrier_derivs(d, dhat, B, B1, B2);
      const double cg = kappa * B1 / (2.0 * d);
      const double ca = kappa * (B2 / (4.0 * s) - B1 / (4.0 * d * s));
      for (int a = 0; a < n3; ++a) {
        sh.g[warp][grp][a] = cg * gs[a];
        for (int b = 0; b < n3; ++b) H[a * n3 + b] = ca * gs[a] * gs[b] + cg * Hs[a * n3 + b];
      }
      sh.E[warp][grp] = kappa * B;
    }
    __syncwarp(gmask);
    // Gram factor of the difference map: C^T C = Rm^T Rm (Rm upper), Ri = Rm^-1
    double Rm[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}}, Ri[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    if (project) {
      double G[3][3];
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
        for (int ii = j + 1; ii < m; ++ii) {
          double u = G[j][ii];
          for (int k = 0; k < j; ++k) u -= Rm[k][j] * Rm[k][ii];
          Rm[j][ii] = u / Rm[j][j];
        }
      }
      for (int ii = m - 1; ii >= 0; --ii) {
        Ri[ii][ii] = 1.0 / Rm[ii][ii];
        for (int j = ii + 1; j < m; ++j) {
          double t = 0.0;
          for (int k = ii + 1; k <= j; ++k) t += Rm[ii][k] * Ri[k][j];
          Ri[ii][j] = -t / Rm[ii][ii];
        }
      }
      // K = (Rm x I) H (Rm^T x I): lane gl forms row gl
      if (gl < n3) {
        const int a = gl / 3, ci = gl % 3;
        for (int col = 0; col < n3; ++col) {
          const int b = col / 3, cj = col % 3;
          double t = 0.0;
          for (int c = a; c < m; ++c)
            for (int e = b; e < m; ++e) t += Rm[a][c] * H[(3 * c + ci) * n3 + 3 * e + cj] * Rm[b][e];
          K[gl * n3 + col] = t;
          V[gl * n3 + col] = gl == col ? 1.0 : 0.0;
        }
      }
      __syncwarp(gmask);
      // eigenvectors: cyclic Jacobi in FP32 first (one row per lane; FP32
      // rotations are cheap), then refined to FP64 accuracy below
      float* K32 = sh.K32[warp][grp];
      float* V32 = sh.V32[warp][grp];
      if (gl < n3)
        for (int c = 0; c < n3; ++c) {
          K32[gl * n3 + c] = (float)K[gl * n3 + c];
          V32[gl * n3 + c] = gl == c ? 1.0f : 0.0f;
        }
      __syncwarp(gmask);
      for (int sweep = 0; sweep < 20; ++sweep) {
        float off = 0.f, tot = 0.f;
        if (gl < n3)
          for (int c = 0; c < n3; ++c) {
            const float a2 = K32[gl * n3 + c] * K32[gl * n3 + c];
            tot += a2;
            if (c != gl) off += a2;
          }
        red[2 * gl] = off;
        red[2 * gl + 1] = tot;
        __syncwarp(gmask);
        off = 0.f;
        tot = 0.f;
        for (int k = 0; k < n3; ++k) {
          off += (float)red[2 * k];
          tot += (float)red[2 * k + 1];
        }
        __syncwarp(gmask);
        if (!(off > 1e-12f * tot)) break;
        for (int pp = 0; pp < n3 - 1; ++pp)
          for (int qq = pp + 1; qq < n3; ++qq) {
            const float apq = K32[pp * n3 + qq];
            if (fabsf(apq) <= 1e-7f * sqrtf(fabsf(K32[pp * n3 + pp] * K32[qq * n3 + qq]))) continue;
            const float theta = (K32[qq * n3 + qq] - K32[pp * n3 + pp]) / (2.f * apq);
            const float t = (theta >= 0.f ? 1.f : -1.f) / (fabsf(theta) + sqrtf(theta * theta + 1.f));
            const float c = rsqrtf(t * t + 1.f), sn = t * c;
            __syncwarp(gmask);
            if (gl < n3) {
              const float kp = K32[gl * n3 + pp], kq = K32[gl * n3 + qq];
              K32[gl * n3 + pp] = c * kp - sn * kq;
              K32[gl * n3 + qq] = sn * kp + c * kq;
              const float vp = V32[gl * n3 + pp], vq = V32[gl * n3 + qq];
              V32[gl * n3 + pp] = c * vp - sn * vq;
              V32[gl * n3 + qq] = sn * vp + c * vq;
            }
            __syncwarp(gmask);
            if (gl < n3) {
              const float kp = K32[pp * n3 + gl], kq = K32[qq * n3 + gl];
              K32[pp * n3 + gl] = c * kp - sn * kq;
              K32[qq * n3 + gl] = sn * kp + c * kq;
            }
            __syncwarp(gmask);
          }
      }
      // FP64 refinement: orthonormalise the FP32 basis by one Newton-Schulz
      // step V (3I - V^T V) / 2, rotate K into it (nearly diagonal), finish
      // with FP64 Jacobi sweeps (quadratic convergence from FP32 accuracy)
      if (gl < n3)
        for (int c = 0; c < n3; ++c) V[gl * n3 + c] = (double)V32[gl * n3 + c];
      __syncwarp(gmask);
      if (gl < n3)  // S = V^T V, row gl into H
        for (int c = 0; c < n3; ++c) {
          double t = 0.0;
          for (int k = 0; k < n3; ++k) t += V[k * n3 + gl] * V[k * n3 + c];
          H[gl * n3 + c] = t;
        }
      __syncwarp(gmask);
      double vrow[9];
      if (gl < n3)
        for (int c = 0; c < n3; ++c) {
          double t = 0.0;
          for (int k = 0; k < n3; ++k) t += V[gl * n3 + k] * ((k == c ? 1.5 : 0.0) - 0.5 * H[k * n3 + c]);
          vrow[c] = t;
        }
      __syncwarp(gmask);
      if (gl < n3)
        for (int c = 0; c < n3; ++c) V[gl * n3 + c] = vrow[c];
      __syncwarp(gmask);
      if (gl < n3)  // T = K V, row gl into H
        for (int c = 0; c < n3; ++c) {
          double t = 0.0;
          for (int k = 0; k < n3; ++k) t += K[gl * n3 + k] * V[k * n3 + c];
          H[gl * n3 + c] = t;
        }
      __syncwarp(gmask);
      double krow[9];
      if (gl < n3)  // K' = V^T T, row gl
        for (int c = 0; c < n3; ++c) {
          double t = 0.0;
          for (int k = 0; k < n3; ++k) t += V[k * n3 + gl] * H[k * n3 + c];
          krow[c] = t;
        }
      __syncwarp(gmask);
      if (gl < n3)
        for (int c = 0; c < n3; ++c) K[gl * n3 + c] = krow[c];
      __syncwarp(gmask);
      // symmetrise (K' is symmetric up to rounding)
      if (gl < n3)
        for (int c = gl + 1; c < n3; ++c) {
          const double a = 0.5 * (K[gl * n3 + c] + K[c * n3 + gl]);
          K[gl * n3 + c] = a;
          K[c * n3 + gl] = a;
        }
      __syncwarp(gmask);
      for (int sweep = 0; sweep < 20; ++sweep) {
        double off = 0.0, tot = 0.0;
        if (gl < n3)
          for (int c = 0; c < n3; ++c) {
            const double a2 = K[gl * n3 + c] * K[gl * n3 + c];
            tot += a2;
            if (c != gl) off += a2;
          }
        red[2 * gl] = off;
        red[2 * gl + 1] = tot;
        __syncwarp(gmask);
        off = 0.0;
        tot = 0.0;
        for (int k = 0; k < n3; ++k) {
          off += red[2 * k];
          tot += red[2 * k + 1];
        }
        __syncwarp(gmask);
        if (!(off > 1e-28 * tot)) break;
        for (int pp = 0; pp < n3 - 1; ++pp)
          for (int qq = pp + 1; qq < n3; ++qq) {
            const double apq = K[pp * n3 + qq];
            // negligible against its diagonal pair: no rotation
            if (fabs(apq) <= 1e-16 * sqrt(fabs(K[pp * n3 + pp] * K[qq * n3 + qq]))) continue;
            const double theta = (K[qq * n3 + qq] - K[pp * n3 + pp]) / (2.0 * apq);
            const double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
            const double c = 1.0 / sqrt(t * t + 1.0), sn = t * c;
            __syncwarp(gmask);
            if (gl < n3) {
              const double kp = K[gl * n3 + pp], kq = K[gl * n3 + qq];
              K[gl * n3 + pp] = c * kp - sn * kq;
              K[gl * n3 + qq] = sn * kp + c * kq;
              const double vp = V[gl * n3 + pp], vq = V[gl * n3 + qq];
              V[gl * n3 + pp] = c * vp - sn * vq;
              V[gl * n3 + qq] = sn * vp + c * vq;
            }
            __syncwarp(gmask);
            if (gl < n3) {
              const double kp = K[pp * n3 + gl], kq = K[qq * n3 + gl];
              K[pp * n3 + gl] = c * kp - sn * kq;
              K[qq * n3 + gl] = sn * kp + c * kq;
            }
            __syncwarp(gmask);
          }
      }
      if (gl < n3) sh.lam[warp][grp][gl] = K[gl * n3 + gl];
      __syncwarp(gmask);
      // Proj(K) = sum_k max(lambda_k, 0) v_k v_k^T, row gl into H
      if (gl < n3)
        for (int col = 0; col < n3; ++col) {
          double t = 0.0;
          for (int k = 0; k < n3; ++k) {
            const double lam = sh.lam[warp][grp][k];
            if (lam > 0.0) t += V[gl * n3 + k] * lam * V[col * n3 + k];
          }
          H[gl * n3 + col] = t;
        }
      __syncwarp(gmask);
      // back to the difference coordinates: (Ri x I) Proj(K) (Ri^T x I), row gl into K
      if (gl < n3) {
        const int a = gl / 3, ci = gl % 3;
        for (int col = 0; col < n3; ++col) {
          const int b = col / 3, cj = col % 3;
          double t = 0.0;
          for (int c = a; c < m; ++c)
            for (int e = b; e < m; ++e) t += Ri[a][c] * H[(3 * c + ci) * n3 + 3 * e + cj] * Ri[b][e];
          K[gl * n3 + col] = t;
        }
      }
      __syncwarp(gmask);
    }
    const double* Hr = project ? K : H;
    double* T = term + (size_t)f * kTermStride;
    // vertex gradient and packed upper vertex Hessian: H12 = T Hr T^T
    for (int o = gl; o < 12; o += kGroupLanes) {
      const int k = o / 3, ci = o % 3;
      double t = 0.0;
      for (int w = 0; w < m; ++w) t += R.C[k][w] * sh.g[warp][grp][3 * w + ci];
      T[1 + o] = t;
    }
    for (int e = gl; e < 78; e += kGroupLanes) {
      // packed index e -> (row, col), row <= col
      int row = 0, rem = e;
      while (rem >= 12 - row) {
        rem -= 12 - row;
        ++row;
      }
      const int col = row + rem;
      const int k = row / 3, ci = row % 3, l = col / 3, cj = col % 3;
      double t = 0.0;
      for (int vv = 0; vv < m; ++vv) {
        if (R.C[k][vv] == 0.0) continue;
        for (int w = 0; w < m; ++w) t += R.C[k][vv] * R.C[l][w] * Hr[(3 * vv + ci) * n3 + 3 * w + cj];
      }
      T[13 + e] = t;
    }
    if (gl == 0) {
      T[0] = sh.E[warp][grp];
      termv[f] = make_int4(v[0], v[1], v[2], v[3]);
      atomicAdd(&st->bar_terms[m], 1ull);
    }
    __syncwarp(gmask);
  }
}

// closest-point weights of a pair of the given distance type: point on the
// first primitive minus point on the second = sum gamma_k x_k
__device__ void closest_weights(int kind, int type, const v3* x, double* g) {
  auto seg = [](v3 p, v3 a, v3 b) { return dot(p - a, b - a) / dot(b - a, b - a); };
  g[0] = g[1] = g[2] = g[3] = 0.0;
  if (kind == 0) {
    double b1 = 0, b2 = 0, b3 = 0, t;
    switch (type) {
      case 0: b1 = 1; break;
      case 1: b2 = 1; break;
      case 2: b3 = 1; break;
      case 3: t = seg(x[0], x[1], x[2]); b1 = 1 - t; b2 = t; break;
      case 4: t = seg(x[0], x[2], x[3]); b2 = 1 - t; b3 = t; break;
      case 5: t = seg(x[0], x[3], x[1]); b3 = 1 - t; b1 = t; break;
      default: {
        v3 e1 = x[2] - x[1], e2 = x[3] - x[1], w = x[0] - x[1];
        double a11 = dot(e1, e1), a12 = dot(e1, e2), a22 = dot(e2, e2), r1 = dot(e1, w), r2 = dot(e2, w);
        double det = a11 * a22 - a12 * a12;
        b2 = (r1 * a22 - r2 * a12) / det;
        b3 = (a11 * r2 - a12 * r1) / det;
        b1 = 1 - b2 - b3;
      } break;
    }
    g[0] = 1.0;
    g[1] = -b1;
    g[2] = -b2;
    g[3] = -b3;
  } else {
    double s = 0, t = 0;
    switch (type) {
      case 0: break;
      case 1: t = 1; break;
      case 2: s = 1; break;
      case 3: s = 1; t = 1; break;
      case 4: t = seg(x[0], x[2], x[3]); break;
      case 5: s = 1; t = seg(x[1], x[2], x[3]); break;
      case 6: s = seg(x[2], x[0], x[1]); break;
      case 7: t = 1; s = seg(x[3], x[0], x[1]); break;
      default: {
        v3 e0 = x[1] - x[0], e1 = x[3] - x[2], w0 = x[0] - x[2];
        double A = dot(e0, e0), B = dot(e0, e1), C = dot(e1, e1), D = dot(e0, w0), E = dot(e1, w0);
        double den = A * C - B * B;
        s = (B * E - C * D) / den;
        t = (A * E - B * D) / den;
      } break;
    }
    g[0] = 1 - s;
    g[1] = s;
    g[2] = -(1 - t);
    g[3] = -t;
  }
}

// lag friction at the current positions: one record per active pair
// (lambda = -kappa B'(d), closest-point weights, normal, lagged offset)
__global__ void k_friction_lag(DevStatus* cst, const int2* P, const int* aoff, const int4* act,
                               const double* act_d2, const int* tri, const int* edge, const int* vbody,
                               const double4* x, const double* l2e, double dhat, double kappa, double mu, int maxc,
                               FricRec* fr) {
  const int np = cst->np, nact = cst->nact;
  if (blockIdx.x == 0 && threadIdx.x == 0) cst->nfr = nact;
  for (int f = blockIdx.x * blockDim.x + threadIdx.x; f < nact; f += gridDim.x * blockDim.x) {
    int p = owner(aoff, np, f);
    int k = f - aoff[p];
    int4 r = act[(size_t)p * maxc + k];
    int kind = (unsigned)r.x >> 31, i = r.x & 0x7fffffff;
    FricRec R;
    pair_vertices(kind, i, r.y, tri, edge, R.v);
    v3 xs[4];
    for (int m = 0; m < 4; ++m) xs[m] = mk(x[R.v[m]]);
    double d = sqrt(act_d2[(size_t)p * maxc + k]);
    double B, B1, B2;
    barrier_derivs(d, dhat, B, B1, B2);
    // normal force magnitude; a mollified edge-edge pair carries m(c)
    double mv = 1.0;
    if (kind == 1) {
      double dm, d2m;
      mv = ee_mollifier(ee_cross2(xs), ee_eps(l2e[i], l2e[r.y]), dm, d2m);
    }
    R.mu_lambda = mu * (-kappa * B1 * mv);
    closest_weights(kind, r.z, xs, R.gam);
    v3 w = (R.gam[0] * xs[0] + R.gam[1] * xs[1]) + (R.gam[2] * xs[2] + R.gam[3] * xs[3]);
    double nn = sqrt(dot(w, w));
    R.n[0] = w.x / nn;
    R.n[1] = w.y / nn;
    R.n[2] = w.z / nn;
    R.r[0] = w.x;
    R.r[1] = w.y;
    R.r[2] = w.z;
    R.a = P[p].x;
    R.b = P[p].y;
    R.kind = kind;
    R.i = i;
    R.j = r.y;
    R.type = r.z;
    fr[f] = R;
  }
}

__global__ void k_friction_eval(const DevStatus* __restrict__ cst, const FricRec* fr, const double4* x, double eps,
                                double* fterm, int4* ftermv, bool derivs) {
  const int nfr = cst->nfr;
  for (int f = blockIdx.x * blockDim.x + threadIdx.x; f < nfr; f += gridDim.x * blockDim.x) {
    const FricRec& R = fr[f];
    v3 xs[4];
    for (int m = 0; m < 4; ++m) xs[m] = mk(x[R.v[m]]);
    double* T = fterm + (size_t)f * kTermStride;
    double g12[12], H78[78];
    double e = friction_term(xs, R.gam, v3{R.n[0], R.n[1], R.n[2]}, v3{R.r[0], R.r[1], R.r[2]}, R.mu_lambda, eps,
                             g12, H78);
    T[0] = e;
    if (derivs) {
      for (int m = 0; m < 12; ++m) T[1 + m] = g12[m];
      for (int m = 0; m < 78; ++m) T[13 + m] = H78[m];
      ftermv[f] = make_int4(R.v[0], R.v[1], R.v[2], R.v[3]);
    }
  }
}

// energy of the barrier over the stored candidates at positions x: one value
// per body pair, summed in slot order (energy-only pass of the line search)
__global__ void k_pair_energy(const DevStatus* __restrict__ cst, const int2* cand, const int* ccount,
                              const int* tri, const int* edge, const double4* x, const double* l2e, double dhat,
                              double kappa, int maxc, double* Ep, DevStatus* st) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nwarps = gridDim.x * (blockDim.x >> 5);
  const int np = cst->np;
  const double dh2 = __dmul_rn(dhat, dhat);
  for (int p = blockIdx.x * (blockDim.x >> 5) + warp; p < np; p += nwarps) {
    const int n = min(ccount[p], maxc);
    double e = 0.0;
    for (int k = lane; k < n; k += 32) {
      int2 c = cand[(size_t)p * maxc + k];
      int kind = (unsigned)c.x >> 31, i = c.x & 0x7fffffff;
      int v[4];
      pair_vertices(kind, i, c.y, tri, edge, v);
      v3 xs[4];
      for (int m = 0; m < 4; ++m) xs[m] = mk(x[v[m]]);
      int type;
      double d2 = pair_dist2(kind, xs, type);
      if (d2 < dh2) {
        if (d2 == 0.0) set_flag(st, ST_INTERSECT);
        double B, B1, B2;
        barrier_derivs(sqrt(d2), dhat, B, B1, B2);
        double mv = 1.0;
        if (kind == 1) {
          double dm, d2m;
          mv = ee_mollifier(ee_cross2(xs), ee_eps(l2e[i], l2e[c.y]), dm, d2m);
        }
        e += kappa * B * mv;
      }
    }
    for (int o = 16; o > 0; o >>= 1) e += __shfl_down_sync(kFull, e, o);
    if (lane == 0) Ep[p] = e;
  }
}

int grid_for(long n, int per_block, int max_blocks) {
  long g = (n + per_block - 1) / per_block;
  if (g < 1) g = 1;
  if (g > max_blocks) g = max_blocks;
  return (int)g;
}

}  // namespace

void launch_enumerate(Scene& s, bool swept, bool ccd) {
  const int threads = 32 * kWarpsPerBlock;
  int grid = grid_for(s.last_np > 0 ? s.last_np : s.nb, kWarpsPerBlock, 152 * 16);
  counted(s);
  ProfScope ps(s, PF_ENUM);
  k_enumerate<<<grid, threads, 0, s.stream>>>(s.P.p, s.st, s.vbeg.p, s.tbeg.p, s.ebeg.p, s.tri.p, s.edge.p, s.x.p,
                                              swept ? s.x1.p : nullptr, s.dx.p, s.bbox.p, s.prm.dhat, s.maxc,
                                              s.cand.p, s.ccount.p, ccd, s.prm.ccd_s, s.prm.ccd_max, s.st);
}

void launch_active(Scene& s, const double4* x) {
  int grid = grid_for(s.last_np > 0 ? s.last_np : s.nb, 8, 152 * 16);
  counted(s);
  ProfScope ps(s, PF_ACTIVE);
  k_active<<<grid, 256, 0, s.stream>>>(s.P.p, s.st, s.cand.p, s.ccount.p, s.tri.p, s.edge.p, x, s.prm.dhat, s.maxc,
                                       s.act.p, s.act_d2.p, s.acount.p, s.st);
}

void launch_barrier(Scene& s, int project, long cap) {
  counted(s);
  ProfScope ps(s, PF_BARRIER);
  k_barrier<<<152 * 8, 32 * kBarWarps, 0, s.stream>>>(s.st, s.aoff.p, s.act.p, s.tri.p, s.edge.p, s.x.p, s.l2e.p,
                                          s.prm.dhat, s.prm.kappa, s.maxc, project, cap, s.term.p, s.termv.p, s.st);
}

void launch_friction_lag(Scene& s) {
  counted(s);
  k_friction_lag<<<152 * 4, 128, 0, s.stream>>>(s.st, s.P.p, s.aoff.p, s.act.p, s.act_d2.p, s.tri.p, s.edge.p,
                                               s.vbody.p, s.x.p, s.l2e.p, s.prm.dhat, s.prm.kappa, s.prm.mu, s.maxc,
                                               s.fric.p);
}

void launch_friction_eval(Scene& s, const double4* x, bool derivs) {
  counted(s);
  ProfScope ps(s, PF_FRICTION);
  k_friction_eval<<<152 * 4, 128, 0, s.stream>>>(s.st, s.fric.p, x, s.prm.eps_v * s.prm.dt, s.fterm.p,
                                                s.ftermv.p, derivs);
}

void launch_pair_energy(Scene& s, const double4* x) {
  int grid = grid_for(s.last_np > 0 ? s.last_np : s.nb, 8, 152 * 16);
  counted(s);
  k_pair_energy<<<grid, 256, 0, s.stream>>>(s.st, s.cand.p, s.ccount.p, s.tri.p, s.edge.p, x, s.l2e.p,
                                            s.prm.dhat, s.prm.kappa, s.maxc, s.Epair.p, s.st);
}

}  // namespace abd
