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

// order-preserving integer key of a double (non-NaN): min / max on keys is
// the exact min / max of the values, on the integer units rather than the
// (slow) FP64 pipe
__device__ __forceinline__ long long dkey(double d) {
  const long long b = __double_as_longlong(d);
  return b >= 0 ? b : b ^ 0x7FFFFFFFFFFFFFFFll;
}
__device__ __forceinline__ double dval(long long k) {
  return __longlong_as_double(k >= 0 ? k : k ^ 0x7FFFFFFFFFFFFFFFll);
}

struct KeyBox {
  long long lo[3], hi[3];
};
__device__ __forceinline__ void kbox_point(KeyBox& b, const double4& p) {
  b.lo[0] = b.hi[0] = dkey(p.x);
  b.lo[1] = b.hi[1] = dkey(p.y);
  b.lo[2] = b.hi[2] = dkey(p.z);
}
__device__ __forceinline__ void kbox_add(KeyBox& b, const double4& p) {
  const long long k[3] = {dkey(p.x), dkey(p.y), dkey(p.z)};
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    b.lo[c] = min(b.lo[c], k[c]);
    b.hi[c] = max(b.hi[c], k[c]);
  }
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

// box of primitive `id` of type t (0 vertex, 1 edge, 2 triangle): exact
// min / max of its vertices (and their end positions when swept)
__device__ __forceinline__ void prim_box(int t, int id, const int* tri, const int* edge, const double4* x,
                                         const double4* x1, Box& b) {
  int nvtx = t == 0 ? 1 : (t == 1 ? 2 : 3);
  int v0 = t == 0 ? id : (t == 1 ? edge[2 * id] : tri[3 * id]);
  KeyBox k;
  kbox_point(k, x[v0]);
  if (x1) kbox_add(k, x1[v0]);
  for (int j = 1; j < nvtx; ++j) {
    int v = t == 1 ? edge[2 * id + j] : tri[3 * id + j];
    kbox_add(k, x[v]);
    if (x1) kbox_add(k, x1[v]);
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    b.lo[c] = dval(k.lo[c]);
    b.hi[c] = dval(k.hi[c]);
  }
}

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
                          WarpLists& L, int2* out, int maxc, int& base, unsigned long long& tested) {
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
      tested += tot;
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
        }
        base += __popc(m);
      }
      __syncwarp();
    }
  }
}

__global__ void k_enumerate(const int2* __restrict__ P, const DevStatus* __restrict__ cst, const int* vbeg,
                            const int* tbeg, const int* ebeg, const int* tri, const int* edge, const double4* x,
                            const double4* x1, const double* bbox, double dhat, int maxc, int2* cand, int* ccount,
                            DevStatus* st) {
  __shared__ WarpLists lists[kWarpsPerBlock];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nwarps = gridDim.x * kWarpsPerBlock;
  const int np = cst->np;
  WarpLists& L = lists[warp];
  unsigned long long ncand = 0, nall = 0, ntested = 0;
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
    enum_kind(0, vbeg[a], vbeg[a + 1], tbeg[b], tbeg[b + 1], Ba, Bb, dhat, tri, edge, x, x1, L, out, maxc, base,
              ntested);
    enum_kind(0, vbeg[b], vbeg[b + 1], tbeg[a], tbeg[a + 1], Bb, Ba, dhat, tri, edge, x, x1, L, out, maxc, base,
              ntested);
    // edges of a against edges of b
    enum_kind(1, ebeg[a], ebeg[a + 1], ebeg[b], ebeg[b + 1], Ba, Bb, dhat, tri, edge, x, x1, L, out, maxc, base,
              ntested);
    nall += (unsigned long long)(vbeg[a + 1] - vbeg[a]) * (tbeg[b + 1] - tbeg[b]) +
            (unsigned long long)(vbeg[b + 1] - vbeg[b]) * (tbeg[a + 1] - tbeg[a]) +
            (unsigned long long)(ebeg[a + 1] - ebeg[a]) * (ebeg[b + 1] - ebeg[b]);
    if (lane == 0) {
      ccount[p] = base;
      if (base > maxc) {
        set_flag(st, ST_CAP_CANDS);
        atomicMax(&st->need_cand, base);
      }
    }
    ncand += base;
  }
  if (lane == 0 && ncand) atomicAdd(&st->n_cand, ncand);
  if (lane == 0 && nall) {
    atomicAdd(&st->cull[0], nall);
    atomicAdd(&st->cull[1], ntested);
    atomicAdd(&st->cull[2], ncand);
  }
}

// additive CCD (Sec. 4.1) over the stored swept candidates: one warp per
// (body pair, 32 candidates), the minimum time of impact by an atomic
// minimum on the bits of the positive double (exact, order-independent):
// over the scene, and over the body pair's contact island (the island of its
// dynamic body; every island's bound starts at 1).  Every candidate publishes
// its time as soon as it has it, and a candidate still advancing stops once
// its island's published bound is below its time (the island's minimum is
// unchanged by that, see accd): a sliding contact with a tiny gap no longer
// advances to t = 1 in thousands of steps when its island's step is already
// bounded far below.
__global__ void k_ccd_chunks(const DevStatus* __restrict__ cst, const int2* cand, const int* ccount, const int* tri,
                             const int* edge, const double4* x, const double4* dx, int maxc, int nch, double ccd_s,
                             int ccd_max, const int2* __restrict__ P, const uint8_t* __restrict__ is_static,
                             const int* __restrict__ isl, unsigned long long* isl_toi, double2* cdl,
                             const int* __restrict__ ework, DevStatus* st) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long nwarps = (long)gridDim.x * (blockDim.x >> 5);
  const long nw = cst->n_ework;  // the (body pair, chunk) slots holding candidates
  double tmin = 1.0;
  for (long tw = (long)blockIdx.x * (blockDim.x >> 5) + warp; tw < nw; tw += nwarps) {
    const int w = ework[tw];
    const int p = w / nch, c = w - p * nch;
    const int n = min(ccount[p], maxc);
    if (c * 32 >= n) continue;
    const int k = c * 32 + lane;
    double t = 1.0;
    if (k < n) {
      const int2 pr = P[p];
      unsigned long long* bound = isl_toi + (is_static[pr.x] ? isl[pr.y] : isl[pr.x]);
      const int2 cc = cand[(size_t)p * maxc + k];
      const int kind = (unsigned)cc.x >> 31, i = cc.x & 0x7fffffff;
      int v[4];
      pair_vertices(kind, i, cc.y, tri, edge, v);
      v3 xs[4], ds[4];
      for (int m = 0; m < 4; ++m) {
        xs[m] = mk(x[v[m]]);
        ds[m] = mk(dx[v[m]]);
      }
      if (accd(kind, xs, ds, ccd_s, 1.0, ccd_max, t, bound, cdl + (size_t)p * maxc + k))
        set_flag(st, ST_CCD_MAXITER);
      if (t < 1.0) atomicMin(bound, (unsigned long long)__double_as_longlong(t));
    }
    tmin = fmin(tmin, t);
  }
  for (int o = 16; o > 0; o >>= 1) tmin = fmin(tmin, __shfl_xor_sync(kFull, tmin, o));
  if (lane == 0 && tmin < 1.0) atomicMin(&st->toi_bits, (unsigned long long)__double_as_longlong(tmin));
}

// active pairs, pass 1: one warp per (body pair, 32 candidates): canonical
// d^2, type and membership d^2 < dhat^2 of every candidate in its own slot,
// and the chunk's membership mask
__global__ void k_active(const DevStatus* __restrict__ cst, const int2* cand, const int* ccount, const int* tri,
                         const int* edge, const double4* x, double dhat, int maxc, int nch, int4* act, double* act_d2,
                         unsigned* amask, const int* __restrict__ ework, DevStatus* st) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long nwarps = (long)gridDim.x * (blockDim.x >> 5);
  const long nw = cst->n_ework;  // the (body pair, chunk) slots holding candidates
  const double dh2 = __dmul_rn(dhat, dhat);
  for (long tw = (long)blockIdx.x * (blockDim.x >> 5) + warp; tw < nw; tw += nwarps) {
    const int w = ework[tw];
    const int p = w / nch, c = w - p * nch;
    const int n = min(ccount[p], maxc);
    if (c * 32 >= n) continue;
    const int k = c * 32 + lane;
    bool a = false;
    if (k < n) {
      const size_t slot = (size_t)p * maxc + k;
      const int2 cc = cand[slot];
      const int kind = (unsigned)cc.x >> 31, i = cc.x & 0x7fffffff;
      int v[4];
      pair_vertices(kind, i, cc.y, tri, edge, v);
      v3 xs[4];
      for (int m = 0; m < 4; ++m) xs[m] = mk(x[v[m]]);
      int type = 0;
      const double d2 = pair_dist2(kind, xs, type);
      a = d2 < dh2;
      if (a && d2 == 0.0) set_flag(st, ST_INTERSECT);
      if (!(d2 == d2)) set_flag(st, ST_NONFINITE);
      act[slot] = make_int4(cc.x, cc.y, type, 0);
      act_d2[slot] = d2;
    }
    const unsigned m = __ballot_sync(kFull, a);
    if (lane == 0) amask[(size_t)p * nch + c] = m;
  }
}

// active pairs, pass 2: one warp per body pair moves the active candidates to
// the front of the pair's slots in slot order and counts them.  In place: the
// targets of a chunk lie at or below its own slots (every lane reads before
// any writes), never in a later chunk.
__global__ void k_active_compact(const DevStatus* __restrict__ cst, const int* ccount, int maxc, int nch,
                                 const unsigned* amask, int4* act, double* act_d2, int* acount) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nwarps = gridDim.x * (blockDim.x >> 5);
  const int np = cst->np;
  for (int p = blockIdx.x * (blockDim.x >> 5) + warp; p < np; p += nwarps) {
    const int n = min(ccount[p], maxc);
    int base = 0;
    for (int c = 0; c * 32 < n; ++c) {
      const unsigned m = amask[(size_t)p * nch + c];
      if (m) {
        const bool bit = (m >> lane) & 1u;
        const size_t src = (size_t)p * maxc + c * 32 + lane;
        int4 v = make_int4(0, 0, 0, 0);
        double d = 0.0;
        if (bit) {
          v = act[src];
          d = act_d2[src];
        }
        __syncwarp();
        if (bit) {
          const size_t dst = (size_t)p * maxc + base + __popc(m & ((1u << lane) - 1u));
          act[dst] = v;
          act_d2[dst] = d;
        }
        __syncwarp();
      }
      base += __popc(m);
    }
    if (lane == 0) acount[p] = base;
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
                                double* fterm, int4* ftermv, bool derivs, const uint8_t* is_static, const int* isl,
                                const int* lstate) {
  const int nfr = cst->nfr;
  for (int f = blockIdx.x * blockDim.x + threadIdx.x; f < nfr; f += gridDim.x * blockDim.x) {
    const FricRec& R = fr[f];
    // line-search rounds: records of islands already accepted are not needed
    if (isl && lstate[2 * (is_static[R.a] ? isl[R.b] : isl[R.a])] != 0) continue;
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
// energy-only barrier sum over the stored candidates: one warp per (body
// pair, chunk of 32 candidates) so that a body pair with many candidates is
// spread over several warps; each warp writes its partial sum to its own
// slot (np x nch, summed later in a fixed order)
//
// With a work list (the line search), only the slots that hold candidates are
// visited (ework[0 .. n_ework)); the other slots are neither read nor written.
// In the line search every candidate also carries, from the CCD pass over
// the same step, its distance d0 at the iterate and the bound lp on the
// distance's rate of change along the step: at the island's trial step alpha
// the distance is at least d0 - alpha lp, so where that exceeds d-hat (with a
// margin of 1e-6 d-hat against rounding) the barrier is zero and the
// distance is not evaluated.
__global__ void k_pair_energy(const DevStatus* __restrict__ cst, const int2* cand, const int* ccount,
                              const int* tri, const int* edge, const double4* x, const double* l2e, double dhat,
                              double kappa, int maxc, int nch, double* Ep, const int2* P, const uint8_t* is_static,
                              const int* isl, const int* lstate, const int* ework, const double2* cdl,
                              const double* alpha, DevStatus* st) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long nwarps = (long)gridDim.x * (blockDim.x >> 5);
  const long nw = ework ? (long)cst->n_ework : (long)cst->np * nch;
  const double dh2 = __dmul_rn(dhat, dhat);
  for (long t = (long)blockIdx.x * (blockDim.x >> 5) + warp; t < nw; t += nwarps) {
    const long w = ework ? (long)ework[t] : t;
    const int p = (int)(w / nch), c = (int)(w - (long)p * nch);
    double a_isl = -1.0;
    if (isl) {  // line-search rounds: pairs of islands already accepted are not needed
      const int2 pr = P[p];
      const int is = is_static[pr.x] ? isl[pr.y] : isl[pr.x];
      if (lstate[2 * is] != 0) continue;
      if (cdl) a_isl = alpha[is];
    }
    const int n = min(ccount[p], maxc);
    const int k = c * 32 + lane;
    double e = 0.0;
    bool far = false;
    if (k < n && a_isl >= 0.0) {
      const double2 dl = cdl[(size_t)p * maxc + k];
      far = dl.x >= 0.0 && dl.x - a_isl * dl.y > dhat * (1.0 + 1e-6);
    }
    if (k < n && !far) {
      int2 cc = cand[(size_t)p * maxc + k];
      int kind = (unsigned)cc.x >> 31, i = cc.x & 0x7fffffff;
      int v[4];
      pair_vertices(kind, i, cc.y, tri, edge, v);
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
          mv = ee_mollifier(ee_cross2(xs), ee_eps(l2e[i], l2e[cc.y]), dm, d2m);
        }
        e = kappa * B * mv;
      }
    }
    if (c * 32 < n)
      for (int o = 16; o > 0; o >>= 1) e += __shfl_down_sync(kFull, e, o);
    if (lane == 0) Ep[w] = e;
  }
}

// the (body pair, chunk) slots holding candidates: ceil(min(count, maxc) / 32)
// per body pair, appended in any order (every slot's energy lands in its own
// place and the island sums are exact, so the order is immaterial)
__global__ void k_energy_worklist(const DevStatus* __restrict__ cst, const int* __restrict__ ccount, int maxc,
                                  int nch, int* ework, DevStatus* st) {
  const int np = cst->np;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < np; p += gridDim.x * blockDim.x) {
    const int nc = (min(ccount[p], maxc) + 31) / 32;
    if (nc == 0) continue;
    const int base = atomicAdd(&st->n_ework, nc);
    for (int c = 0; c < nc; ++c) ework[base + c] = p * nch + c;
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
  int grid = grid_for(2L * s.nb, kWarpsPerBlock, sm_grid(s, 16));  // grid-stride over the device's pair count
  counted(s);
  ProfScope ps(s, PF_ENUM);
  k_enumerate<<<grid, threads, 0, s.stream>>>(s.P.p, s.st, s.vbeg.p, s.tbeg.p, s.ebeg.p, s.tri.p, s.edge.p, s.x.p,
                                              swept ? s.x1.p : nullptr, s.bbox.p, s.prm.dhat, s.maxc, s.cand.p,
                                              s.ccount.p, s.st);
  launch_energy_worklist(s);  // the slots holding candidates, for every pass over them
  if (ccd) {
    const int nch = energy_chunks(s);
    counted(s);
    k_ccd_chunks<<<grid_for(2L * s.nb * nch, 8, sm_grid(s, 32)), 256, 0, s.stream>>>(
        s.st, s.cand.p, s.ccount.p, s.tri.p, s.edge.p, s.x.p, s.dx.p, s.maxc, nch, s.prm.ccd_s, s.prm.ccd_max, s.P.p,
        s.is_static.p, s.isl.p, s.isl_toi.p, s.cdl.p, s.ework.p, s.st);
  }
}

void launch_active(Scene& s, const double4* x) {
  const int nch = energy_chunks(s);
  counted(s, 2);
  ProfScope ps(s, PF_ACTIVE);
  // grid-stride over the device's pair count
  k_active<<<grid_for(2L * s.nb * nch, 8, sm_grid(s, 32)), 256, 0, s.stream>>>(
      s.st, s.cand.p, s.ccount.p, s.tri.p, s.edge.p, x, s.prm.dhat, s.maxc, nch, s.act.p, s.act_d2.p, s.amask.p,
      s.ework.p, s.st);
  k_active_compact<<<grid_for(2L * s.nb, 8, sm_grid(s, 16)), 256, 0, s.stream>>>(
      s.st, s.ccount.p, s.maxc, nch, s.amask.p, s.act.p, s.act_d2.p, s.acount.p);
}

void launch_friction_lag(Scene& s) {
  counted(s);
  k_friction_lag<<<sm_grid(s, 4), 128, 0, s.stream>>>(s.st, s.P.p, s.aoff.p, s.act.p, s.act_d2.p, s.tri.p, s.edge.p,
                                               s.vbody.p, s.x.p, s.l2e.p, s.prm.dhat, s.prm.kappa, s.prm.mu, s.maxc,
                                               s.fric.p);
}

void launch_friction_eval(Scene& s, const double4* x, bool derivs, bool pending_only) {
  counted(s);
  ProfScope ps(s, PF_FRICTION);
  k_friction_eval<<<sm_grid(s, 4), 128, 0, s.stream>>>(s.st, s.fric.p, x, s.prm.eps_v * s.prm.dt, s.fterm.p,
                                                s.ftermv.p, derivs, s.is_static.p,
                                                pending_only ? s.isl.p : nullptr, s.isl_state.p);
}

void launch_pair_energy(Scene& s, const double4* x, bool pending_only) {
  const int nch = energy_chunks(s);
  int grid = grid_for(2L * s.nb * nch, 8, sm_grid(s, 32));  // grid-stride over the device's pair count
  counted(s);
  k_pair_energy<<<grid, 256, 0, s.stream>>>(s.st, s.cand.p, s.ccount.p, s.tri.p, s.edge.p, x, s.l2e.p,
                                            s.prm.dhat, s.prm.kappa, s.maxc, nch, s.Epair.p, s.P.p,
                                            s.is_static.p, pending_only ? s.isl.p : nullptr, s.isl_state.p,
                                            pending_only ? s.ework.p : nullptr, pending_only ? s.cdl.p : nullptr,
                                            s.isl_alpha.p, s.st);
}

void launch_energy_worklist(Scene& s) {
  counted(s, 2);
  cudaMemsetAsync(&s.st->n_ework, 0, sizeof(int), s.stream);
  k_energy_worklist<<<grid_for(2L * s.nb, 256, sm_grid(s, 8)), 256, 0, s.stream>>>(s.st, s.ccount.p, s.maxc,
                                                                                   energy_chunks(s), s.ework.p, s.st);
}

}  // namespace abd
