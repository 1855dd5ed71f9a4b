// System kernels: mass integrals (Sec. 3.1), predictor (Sec. 4), vertex map
// (Sec. 3), body boxes and body-pair culling (Sec. 4.2), per-body inertia and
// orthogonality terms (Sec. 3.2 / Sec. 4), Hessian assembly by body-pair
// blocks (Sec. 4.3), block-Jacobi PCG, and deterministic reductions.
#include "abd_internal.cuh"
#include "derivs.cuh"

namespace abd {

namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ void set_flag(DevStatus* st, unsigned f) { atomicOr(&st->flags, f); }

// DOF of the coefficient multiplying w_u = (1, xbar)_u in x_c
__host__ __device__ __forceinline__ int dof(int u, int c) { return u == 0 ? c : 3 + 3 * c + (u - 1); }
__device__ __forceinline__ void inv_dof(int i, int& u, int& c) {
  if (i < 3) {
    u = 0;
    c = i;
  } else {
    u = 1 + (i - 3) % 3;
    c = (i - 3) / 3;
  }
}

// ---------------------------------------------------------------------------
// Sec. 3.1: volume, first and second moments by signed tetrahedra (0, v0, v1,
// v2) of the closed surface; M = rho [[vol I, I (x) m1^T], [I (x) m1, I (x) S]]
// ---------------------------------------------------------------------------
__global__ void k_mass_moments(int nb, const int* tbeg, const int* tri, const double4* xbar, const double* density,
                               const uint8_t* is_static, double* mass10, double* vol) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= nb) return;
  const int b = warp;
  double acc[10];
  for (int k = 0; k < 10; ++k) acc[k] = 0.0;
  if (!is_static[b]) {
    for (int t = tbeg[b] + lane; t < tbeg[b + 1]; t += 32) {
      double4 a = xbar[tri[3 * t]], c1 = xbar[tri[3 * t + 1]], c2 = xbar[tri[3 * t + 2]];
      double det = a.x * (c1.y * c2.z - c1.z * c2.y) - a.y * (c1.x * c2.z - c1.z * c2.x) + a.z * (c1.x * c2.y - c1.y * c2.x);
      double V = det / 6.0;
      double s[3] = {a.x + c1.x + c2.x, a.y + c1.y + c2.y, a.z + c1.z + c2.z};
      double v0[3] = {a.x, a.y, a.z}, v1[3] = {c1.x, c1.y, c1.z}, v2[3] = {c2.x, c2.y, c2.z};
      acc[0] += V;
      for (int k = 0; k < 3; ++k) acc[1 + k] += V * s[k] / 4.0;
      int idx = 4;
      for (int i = 0; i < 3; ++i)
        for (int j = i; j < 3; ++j)
          acc[idx++] += V / 20.0 * (v0[i] * v0[j] + v1[i] * v1[j] + v2[i] * v2[j] + s[i] * s[j]);
    }
  }
  for (int k = 0; k < 10; ++k)
    for (int o = 16; o > 0; o >>= 1) acc[k] += __shfl_down_sync(kFull, acc[k], o);
  if (lane == 0) {
    const double rho = density[b];
    for (int k = 0; k < 10; ++k) mass10[10 * b + k] = rho * acc[k];
    vol[b] = acc[0];
  }
}

// Sec. 4: qtilde = q^t + dt qdot^t + dt^2 M^-1 f with f = int rho J^T g.
// M (g, 0, 0, 0) = f for every body, so M^-1 f = (g, 0, 0, 0).
__global__ void k_predictor(int nb, const uint8_t* is_static, const double* qt, const double* qdot, double dt,
                            double gx, double gy, double gz, double* qtilde) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb) return;
  const double gv[3] = {gx, gy, gz};
  for (int k = 0; k < 12; ++k) {
    double q = qt[12 * b + k];
    if (is_static[b]) {
      qtilde[12 * b + k] = q;
      continue;
    }
    double f = k < 3 ? gv[k] : 0.0;
    qtilde[12 * b + k] = __dadd_rn(__dadd_rn(q, __dmul_rn(dt, qdot[12 * b + k])), __dmul_rn(__dmul_rn(dt, dt), f));
  }
}

// Sec. 3: x_c = fma(A[c][2], xbar2, fma(A[c][1], xbar1, fma(A[c][0], xbar0, p_c)))
__device__ __forceinline__ double4 affine(const double* q, double4 xb) {
  double4 r;
  r.x = __fma_rn(q[5], xb.z, __fma_rn(q[4], xb.y, __fma_rn(q[3], xb.x, q[0])));
  r.y = __fma_rn(q[8], xb.z, __fma_rn(q[7], xb.y, __fma_rn(q[6], xb.x, q[1])));
  r.z = __fma_rn(q[11], xb.z, __fma_rn(q[10], xb.y, __fma_rn(q[9], xb.x, q[2])));
  r.w = 0.0;
  return r;
}

__global__ void k_transform(int nv, const int* vbody, const double4* xbar, const double* q, double4* x) {
  int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= nv) return;
  x[v] = affine(q + 12 * vbody[v], xbar[v]);
}

__global__ void k_transform_dq(int nv, const int* vbody, const double4* xbar, const double* dq, const double4* x,
                               double4* dx, double4* x1) {
  int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= nv) return;
  double4 d = affine(dq + 12 * vbody[v], xbar[v]);
  double4 p = x[v];
  dx[v] = d;
  x1[v] = make_double4(__dadd_rn(p.x, d.x), __dadd_rn(p.y, d.y), __dadd_rn(p.z, d.z), 0.0);
}

__global__ void k_body_boxes(int nb, const int* vbeg, const double4* x, const double4* x1, double* bbox) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= nb) return;
  const int b = warp;
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  for (int v = vbeg[b] + lane; v < vbeg[b + 1]; v += 32) {
    double4 p = x[v];
    lo[0] = fmin(lo[0], p.x); hi[0] = fmax(hi[0], p.x);
    lo[1] = fmin(lo[1], p.y); hi[1] = fmax(hi[1], p.y);
    lo[2] = fmin(lo[2], p.z); hi[2] = fmax(hi[2], p.z);
    if (x1) {
      double4 r = x1[v];
      lo[0] = fmin(lo[0], r.x); hi[0] = fmax(hi[0], r.x);
      lo[1] = fmin(lo[1], r.y); hi[1] = fmax(hi[1], r.y);
      lo[2] = fmin(lo[2], r.z); hi[2] = fmax(hi[2], r.z);
    }
  }
  for (int k = 0; k < 3; ++k)
    for (int o = 16; o > 0; o >>= 1) {
      lo[k] = fmin(lo[k], __shfl_xor_sync(kFull, lo[k], o));
      hi[k] = fmax(hi[k], __shfl_xor_sync(kFull, hi[k], o));
    }
  if (lane == 0)
    for (int k = 0; k < 3; ++k) {
      bbox[6 * b + k] = lo[k];
      bbox[6 * b + 3 + k] = hi[k];
    }
}

// ---------------------------------------------------------------------------
// body pairs (a < b, not both static) whose boxes are within dhat, plus the
// lagged friction body pairs; one row per body a, sorted by b
// ---------------------------------------------------------------------------
__global__ void k_rows(int nb, const uint8_t* is_static, const double* bbox, double dhat, const int2* fpairs,
                       const DevStatus* cst, int maxn, int* nbr, int* ncount, DevStatus* st) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  const int nfp = cst->nfp;
  for (int a = warp; a < nb; a += nwarps) {
    double alo[3], ahi[3];
    for (int k = 0; k < 3; ++k) {
      alo[k] = bbox[6 * a + k];
      ahi[k] = bbox[6 * a + 3 + k];
    }
    const bool sa = is_static[a];
    int* out = nbr + (size_t)a * maxn;
    int base = 0;
    for (int b0 = a + 1; b0 < nb; b0 += 32) {
      int b = b0 + lane;
      bool keep = false;
      if (b < nb && !(sa && is_static[b])) {
        keep = true;
        for (int k = 0; k < 3; ++k) {
          if (!(__dsub_rn(alo[k], bbox[6 * b + 3 + k]) <= dhat)) keep = false;
          if (!(__dsub_rn(bbox[6 * b + k], ahi[k]) <= dhat)) keep = false;
        }
      }
      unsigned m = __ballot_sync(kFull, keep);
      if (keep) {
        int pos = base + __popc(m & ((1u << lane) - 1u));
        if (pos < maxn) out[pos] = b;
      }
      base += __popc(m);
    }
    if (lane == 0 && nfp > 0) {
      // friction neighbours of row a: fpairs entries with .x == a (sorted)
      int lo = 0, hi = nfp;
      while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (fpairs[mid].x < a) lo = mid + 1;
        else hi = mid;
      }
      for (int f = lo; f < nfp && fpairs[f].x == a; ++f) {
        int b = fpairs[f].y;
        int n = min(base, maxn);
        int pos = 0;
        while (pos < n && out[pos] < b) ++pos;
        if (pos < n && out[pos] == b) continue;
        if (base < maxn) {
          for (int k = n; k > pos; --k) out[k] = out[k - 1];
          out[pos] = b;
        }
        ++base;
      }
    }
    if (lane == 0) {
      ncount[a] = min(base, maxn);
      if (base > maxn) {
        set_flag(st, ST_CAP_ROWS);
        atomicMax(&st->need_row, base);
      }
    }
  }
}

__global__ void k_rows_compact(int nb, const int* nbr, const int* ncount, const int* rowoff, int maxn, int2* P,
                               long cap) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int a = warp; a < nb; a += nwarps) {
    const int n = ncount[a], o = rowoff[a];
    for (int k = lane; k < n; k += 32)
      if (o + k < cap) P[o + k] = make_int2(a, nbr[(size_t)a * maxn + k]);
  }
}

// single-block exclusive scan (fixed order)
__global__ void k_scan(const int* cnt, int* off, const int* n_dev, int n_const, int* total_dev, long cap,
                       unsigned flag, unsigned long long* need, DevStatus* st) {
  __shared__ long long sums[1024];
  const int n = n_dev ? *n_dev : n_const;
  const int t = threadIdx.x;
  const int chunk = (n + 1023) / 1024;
  const int beg = min(n, t * chunk), end = min(n, beg + chunk);
  long long local = 0;
  for (int i = beg; i < end; ++i) local += cnt[i];
  sums[t] = local;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {
    long long v = t >= o ? sums[t - o] : 0;
    __syncthreads();
    sums[t] += v;
    __syncthreads();
  }
  long long run = sums[t] - local;
  for (int i = beg; i < end; ++i) {
    off[i] = (int)run;
    run += cnt[i];
  }
  if (t == 1023) {
    long long total = sums[1023];
    off[n] = (int)total;
    if (total > cap) {
      set_flag(st, flag);
      atomicMax(need, (unsigned long long)total);
      *total_dev = (int)cap;
    } else {
      *total_dev = (int)total;
    }
  }
}

// incoming lists: body pairs whose second body is b, sorted by pair index
__global__ void k_in_count(const DevStatus* cst, const int2* P, int* cnt) {
  const int np = cst->np;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < np; p += gridDim.x * blockDim.x) atomicAdd(&cnt[P[p].y], 1);
}
__global__ void k_in_fill(const DevStatus* cst, const int2* P, const int* off, int* cur, int* list) {
  const int np = cst->np;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < np; p += gridDim.x * blockDim.x) {
    int b = P[p].y;
    int pos = atomicAdd(&cur[b], 1);
    list[off[b] + pos] = p;
  }
}
__global__ void k_in_sort(int nb, const int* off, int* list) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb) return;
  for (int i = off[b] + 1; i < off[b + 1]; ++i) {
    int v = list[i], j = i - 1;
    while (j >= off[b] && list[j] > v) {
      list[j + 1] = list[j];
      --j;
    }
    list[j + 1] = v;
  }
}

// friction body pairs: the body pairs that carry active pairs when friction is lagged
__global__ void k_flag_active(const DevStatus* cst, const int* acount, int* flag) {
  const int np = cst->np;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < np; p += gridDim.x * blockDim.x) flag[p] = acount[p] > 0;
}
__global__ void k_fpairs(const DevStatus* cst, const int2* P, const int* flag, const int* pos, const int* aoff,
                         int2* fpairs, int* fpoff) {
  const int np = cst->np;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < np; p += gridDim.x * blockDim.x)
    if (flag[p]) {
      fpairs[pos[p]] = P[p];
      fpoff[pos[p]] = aoff[p];
    }
  if (blockIdx.x == 0 && threadIdx.x == 0) fpoff[cst->nfp] = cst->nact;
}

// ---------------------------------------------------------------------------
// Sec. 4.3: per body pair, J^T H J of its contact terms in fixed order:
// off-diagonal block H_ab, diagonal parts for a and b, gradient parts, energies
// ---------------------------------------------------------------------------
__device__ int find_fpair(const int2* fp, int n, int a, int b) {
  int lo = 0, hi = n;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    int2 k = fp[mid];
    if (k.x < a || (k.x == a && k.y < b)) lo = mid + 1;
    else hi = mid;
  }
  return (lo < n && fp[lo].x == a && fp[lo].y == b) ? lo : -1;
}

__global__ void k_assemble(const DevStatus* __restrict__ cst, const int2* P, const int* aoff, const double* term,
                           const int4* termv, const int2* fpairs, const int* fpoff, const double* fterm,
                           const int4* ftermv, const int* vbody, const double4* xbar, double* pblk) {
  __shared__ double sH[8][kTermStride];
  __shared__ double sw[8][4][4];
  __shared__ int sside[8][4];
  const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  const int np = cst->np, nfp = cst->nfp, nact = cst->nact;
  for (int p = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; p < np; p += nwarps) {
    const int a = P[p].x, b = P[p].y;
    int t0 = aoff[p], t1 = min(aoff[p + 1], nact);
    int f0 = 0, f1 = 0;
    if (nfp > 0) {
      int q = find_fpair(fpairs, nfp, a, b);
      if (q >= 0) {
        f0 = fpoff[q];
        f1 = fpoff[q + 1];
      }
    }
    double acc[15];
    for (int k = 0; k < 15; ++k) acc[k] = 0.0;
    const int nterms = (t1 - t0) + (f1 - f0);
    for (int it = 0; it < nterms; ++it) {
      const bool fr = it >= (t1 - t0);
      const int t = fr ? f0 + (it - (t1 - t0)) : t0 + it;
      const double* T = (fr ? fterm : term) + (size_t)t * kTermStride;
      for (int k = lane; k < kTermStride; k += 32) sH[wib][k] = T[k];
      if (lane < 4) {
        int4 vv = fr ? ftermv[t] : termv[t];
        int v = lane == 0 ? vv.x : (lane == 1 ? vv.y : (lane == 2 ? vv.z : vv.w));
        sside[wib][lane] = vbody[v] == a ? 0 : 1;
        double4 xb = xbar[v];
        sw[wib][lane][0] = 1.0;
        sw[wib][lane][1] = xb.x;
        sw[wib][lane][2] = xb.y;
        sw[wib][lane][3] = xb.z;
      }
      __syncwarp();
      const double* H = sH[wib] + 13;
      const double* g = sH[wib] + 1;
      for (int k = 0; k < 15; ++k) {
        const int o = lane + 32 * k;
        if (o >= kBlkStride) break;
        double c = 0.0;
        if (o < 432) {
          const int region = o / 144, e = o % 144;
          const int sk = region == 2 ? 1 : 0, sl = region == 1 ? 0 : 1;
          int u, cc, u2, c2;
          inv_dof(e / 12, u, cc);
          inv_dof(e % 12, u2, c2);
          for (int kk = 0; kk < 4; ++kk) {
            if (sside[wib][kk] != sk) continue;
            const double wk = sw[wib][kk][u];
            for (int ll = 0; ll < 4; ++ll) {
              if (sside[wib][ll] != sl) continue;
              c += wk * sw[wib][ll][u2] * H[up12(3 * kk + cc, 3 * ll + c2)];
            }
          }
        } else if (o < 456) {
          const int gi = o - 432, sd = gi / 12;
          int u, cc;
          inv_dof(gi % 12, u, cc);
          for (int kk = 0; kk < 4; ++kk)
            if (sside[wib][kk] == sd) c += sw[wib][kk][u] * g[3 * kk + cc];
        } else if (o == 456) {
          c = fr ? 0.0 : sH[wib][0];
        } else {
          c = fr ? sH[wib][0] : 0.0;
        }
        acc[k] += c;
      }
      __syncwarp();
    }
    for (int k = 0; k < 15; ++k) {
      const int o = lane + 32 * k;
      if (o < kBlkStride) pblk[(size_t)p * kBlkStride + o] = acc[k];
    }
  }
}

// ---------------------------------------------------------------------------
// per-body inertia and orthogonality terms (Sec. 3.2, Sec. 4)
// ---------------------------------------------------------------------------
__global__ void k_body_terms(int nb, const uint8_t* is_static, const double* q, const double* qtilde,
                             const double* mass10, const double* vol, const double* kappa_b, double dt, bool hess,
                             double* Db, double* gb, double* Eb) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb) return;
  if (is_static[b]) {
    if (hess)
      for (int k = 0; k < 144; ++k) Db[144 * b + k] = (k % 13 == 0) ? 1.0 : 0.0;
    for (int k = 0; k < 12; ++k) gb[12 * b + k] = 0.0;
    Eb[2 * b] = Eb[2 * b + 1] = 0.0;
    return;
  }
  const double* m = mass10 + 10 * b;
  const double W[4][4] = {{m[0], m[1], m[2], m[3]}, {m[1], m[4], m[5], m[6]}, {m[2], m[5], m[7], m[8]},
                          {m[3], m[6], m[8], m[9]}};
  double qq[12], d[12], Md[12];
  for (int k = 0; k < 12; ++k) {
    qq[k] = q[12 * b + k];
    d[k] = qq[k] - qtilde[12 * b + k];
  }
  double Ein = 0.0;
  for (int c = 0; c < 3; ++c)
    for (int u = 0; u < 4; ++u) {
      double s = 0.0;
      for (int v = 0; v < 4; ++v) s += W[u][v] * d[dof(v, c)];
      Md[dof(u, c)] = s;
    }
  for (int k = 0; k < 12; ++k) Ein += 0.5 * d[k] * Md[k];
  // V = kappa nu sum_ij (a_i . a_j - delta_ij)^2, rows a_i of A
  const double kv = kappa_b[b] * vol[b];
  v3 a[3];
  for (int i = 0; i < 3; ++i) a[i] = v3{qq[3 + 3 * i], qq[4 + 3 * i], qq[5 + 3 * i]};
  double G[3][3];
  double V = 0.0;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      G[i][j] = dot(a[i], a[j]);
      double e = G[i][j] - (i == j ? 1.0 : 0.0);
      V += e * e;
    }
  V *= kv;
  const double dt2 = dt * dt;
  // gradient: 4 kv [(a_i.a_i - 1) a_i + sum_{j != i} (a_i.a_j) a_j]
  double gv[12] = {0, 0, 0};
  for (int i = 0; i < 3; ++i) {
    v3 t = (G[i][i] - 1.0) * a[i];
    for (int j = 0; j < 3; ++j)
      if (j != i) t = t + G[i][j] * a[j];
    gv[3 + 3 * i] = 4.0 * kv * t.x;
    gv[4 + 3 * i] = 4.0 * kv * t.y;
    gv[5 + 3 * i] = 4.0 * kv * t.z;
  }
  for (int k = 0; k < 12; ++k) gb[12 * b + k] = Md[k] + dt2 * gv[k];
  Eb[2 * b] = Ein;
  Eb[2 * b + 1] = dt2 * V;
  if (!hess) return;
  // Hessian blocks: (i,i) 4kv[2 a_i a_i^T + (|a_i|^2 - 1) I + sum_{j!=i} a_j a_j^T],
  //                 (i,j) 4kv[a_j a_i^T + (a_i.a_j) I]
  double A9[81];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
          double h;
          if (i == j) {
            h = 2.0 * comp(a[i], r) * comp(a[i], c) + (r == c ? G[i][i] - 1.0 : 0.0);
            for (int k = 0; k < 3; ++k)
              if (k != i) h += comp(a[k], r) * comp(a[k], c);
          } else {
            h = comp(a[j], r) * comp(a[i], c) + (r == c ? G[i][j] : 0.0);
          }
          A9[(3 * i + r) * 9 + 3 * j + c] = 4.0 * kv * h;
        }
  project_psd<9, double>(A9);
  double* D = Db + 144 * b;
  for (int k = 0; k < 144; ++k) D[k] = 0.0;
  for (int c = 0; c < 3; ++c)
    for (int u = 0; u < 4; ++u)
      for (int v = 0; v < 4; ++v) D[12 * dof(u, c) + dof(v, c)] = W[u][v];
  for (int i = 0; i < 9; ++i)
    for (int j = 0; j < 9; ++j) D[12 * (3 + i) + 3 + j] += dt2 * A9[9 * i + j];
}

// diagonal blocks and gradient: body terms plus the body's share of each of
// its body pairs, in pair order
__global__ void k_gather(int nb, const uint8_t* is_static, const int* rowoff, const int* in_off, const int* in_list,
                         const double* pblk, const double* Db, const double* gb, double* D, double* g,
                         const DevStatus* cst) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= nb) return;
  const int b = warp;
  const int np = cst->np;
  for (int o = lane; o < 156; o += 32) {
    double v = o < 144 ? Db[144 * b + o] : gb[12 * b + o - 144];
    if (!is_static[b]) {
      const int off_lo = o < 144 ? 144 + o : 432 + (o - 144);
      const int off_hi = o < 144 ? 288 + o : 444 + (o - 144);
      for (int p = rowoff[b]; p < min(rowoff[b + 1], np); ++p) v += pblk[(size_t)p * kBlkStride + off_lo];
      for (int k = in_off[b]; k < in_off[b + 1]; ++k) v += pblk[(size_t)in_list[k] * kBlkStride + off_hi];
    } else if (o >= 144) {
      v = 0.0;
    }
    if (o < 144) D[144 * b + o] = v;
    else g[12 * b + o - 144] = v;
  }
}

// block-Jacobi preconditioner: inverse of each dynamic diagonal block
__global__ void k_precond(int nb, const uint8_t* is_static, const double* D, double* Pinv, DevStatus* st) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb) return;
  double* Pi = Pinv + 144 * b;
  if (is_static[b]) {
    for (int k = 0; k < 144; ++k) Pi[k] = 0.0;
    return;
  }
  double L[144];
  for (int k = 0; k < 144; ++k) L[k] = D[144 * b + k];
  bool ok = true;
  for (int j = 0; j < 12 && ok; ++j) {
    double s = L[13 * j];
    for (int k = 0; k < j; ++k) s -= L[12 * j + k] * L[12 * j + k];
    if (!(s > 0.0)) {
      ok = false;
      break;
    }
    double l = sqrt(s);
    L[13 * j] = l;
    for (int i = j + 1; i < 12; ++i) {
      double t = L[12 * i + j];
      for (int k = 0; k < j; ++k) t -= L[12 * i + k] * L[12 * j + k];
      L[12 * i + j] = t / l;
    }
  }
  if (!ok) {
    set_flag(st, ST_PCG_BREAKDOWN);
    for (int k = 0; k < 144; ++k) Pi[k] = (k % 13 == 0) ? 1.0 / fabs(D[144 * b + k]) : 0.0;
    return;
  }
  // columns of the inverse: solve L L^T x = e_c
  for (int c = 0; c < 12; ++c) {
    double x[12];
    for (int i = 0; i < 12; ++i) {
      double s = (i == c) ? 1.0 : 0.0;
      for (int k = 0; k < i; ++k) s -= L[12 * i + k] * x[k];
      x[i] = s / L[13 * i];
    }
    for (int i = 11; i >= 0; --i) {
      double s = x[i];
      for (int k = i + 1; k < 12; ++k) s -= L[12 * k + i] * x[k];
      x[i] = s / L[13 * i];
    }
    for (int i = 0; i < 12; ++i) Pi[12 * i + c] = x[i];
  }
}

// ---------------------------------------------------------------------------
// PCG on the block system: y = H v from the diagonal blocks, the stored
// upper blocks of the body's rows and the transposed blocks of its incoming
// pairs; scalars live in the status word so no host round trip is needed
// ---------------------------------------------------------------------------
constexpr int kPcgThreads = 192;  // 16 bodies x 12 rows

__global__ void k_spmv(int nb, const uint8_t* is_static, const double* D, const int* rowoff, const int* in_off,
                       const int* in_list, const int2* P, const double* pblk, const double* v, double* y,
                       double* part, const DevStatus* cst) {
  __shared__ double red[kPcgThreads];
  if (cst->scal[6] != 0.0) return;
  const int np = cst->np;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int b = t / 12, i = t % 12;
  double acc = 0.0, pd = 0.0;
  if (b < nb && !is_static[b]) {
    const double* Di = D + 144 * b + 12 * i;
    for (int j = 0; j < 12; ++j) acc += Di[j] * v[12 * b + j];
    for (int p = rowoff[b]; p < min(rowoff[b + 1], np); ++p) {
      int o = P[p].y;
      if (is_static[o]) continue;
      const double* Hr = pblk + (size_t)p * kBlkStride + 12 * i;
      for (int j = 0; j < 12; ++j) acc += Hr[j] * v[12 * o + j];
    }
    for (int k = in_off[b]; k < in_off[b + 1]; ++k) {
      int p = in_list[k];
      int o = P[p].x;
      if (is_static[o]) continue;
      const double* Hc = pblk + (size_t)p * kBlkStride + i;
      for (int j = 0; j < 12; ++j) acc += Hc[12 * j] * v[12 * o + j];
    }
    pd = acc * v[12 * b + i];
  }
  if (b < nb) y[t] = acc;
  // block sum in fixed order: warp shuffles, then the warp partials in order
  for (int o = 16; o > 0; o >>= 1) pd += __shfl_down_sync(kFull, pd, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = pd;
  __syncthreads();
  if (threadIdx.x == 0) {
    double sum = 0.0;
    for (int w = 0; w < kPcgThreads / 32; ++w) sum += red[w];
    red[0] = sum;
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// fixed-order sum of n partials into st->scal[slot]
__device__ double block_sum(const double* v, int n) {
  __shared__ double red[256];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += 256) s += v[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  double r = red[0];
  __syncthreads();
  return r;
}

__global__ void k_pcg_alpha(const double* part, int n, DevStatus* st) {
  if (st->scal[6] != 0.0) return;
  double pAp = block_sum(part, n);
  if (threadIdx.x == 0) {
    st->scal[1] = pAp;
    if (!(pAp > 0.0)) {
      st->scal[6] = 2.0;  // breakdown
      set_flag(st, ST_PCG_BREAKDOWN);
    } else {
      st->scal[4] = st->scal[0] / pAp;
    }
  }
}

// x += alpha p; r -= alpha Ap; z = Pinv r; partial sums of r.z and r.r
__global__ void k_pcg_update(int nb, const uint8_t* is_static, const double* Pinv, const double* pv,
                             const double* Ap, double* x, double* r, double* z, double* part, const DevStatus* cst) {
  __shared__ double red[2][128];
  if (cst->scal[6] != 0.0) return;
  const double alpha = cst->scal[4];
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  double rz = 0.0, rr = 0.0;
  if (b < nb && !is_static[b]) {
    double rb[12];
    for (int k = 0; k < 12; ++k) {
      x[12 * b + k] += alpha * pv[12 * b + k];
      rb[k] = r[12 * b + k] - alpha * Ap[12 * b + k];
      r[12 * b + k] = rb[k];
      rr += rb[k] * rb[k];
    }
    const double* Pi = Pinv + 144 * b;
    for (int i = 0; i < 12; ++i) {
      double s = 0.0;
      for (int j = 0; j < 12; ++j) s += Pi[12 * i + j] * rb[j];
      z[12 * b + i] = s;
      rz += rb[i] * s;
    }
  }
  red[0][threadIdx.x] = rz;
  red[1][threadIdx.x] = rr;
  __syncthreads();
  for (int o = 64; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      red[0][threadIdx.x] += red[0][threadIdx.x + o];
      red[1][threadIdx.x] += red[1][threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = red[0][0];
    part[2 * blockIdx.x + 1] = red[1][0];
  }
}

__global__ void k_pcg_beta(const double* part, int n, double tol2, DevStatus* st) {
  __shared__ double red[2][256];
  if (st->scal[6] != 0.0) return;
  double a = 0.0, c = 0.0;
  for (int i = threadIdx.x; i < n; i += 256) {
    a += part[2 * i];
    c += part[2 * i + 1];
  }
  red[0][threadIdx.x] = a;
  red[1][threadIdx.x] = c;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      red[0][threadIdx.x] += red[0][threadIdx.x + o];
      red[1][threadIdx.x] += red[1][threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    double rz = red[0][0], rr = red[1][0];
    st->scal[5] = rz / st->scal[0];
    st->scal[0] = rz;
    st->scal[2] = rr;
    st->scal[7] += 1.0;
    if (rr <= tol2 * st->scal[3]) st->scal[6] = 1.0;
  }
}

__global__ void k_pcg_dir(long n, const double* z, double* pv, const DevStatus* cst) {
  if (cst->scal[6] != 0.0) return;
  const double beta = cst->scal[5];
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    pv[i] = z[i] + beta * pv[i];
}

// r = rhs (dynamic rows), x = 0, z = Pinv r, p = z; partials of r.z and r.r
__global__ void k_pcg_init(int nb, const uint8_t* is_static, const double* Pinv, const double* rhs, double* x,
                           double* r, double* z, double* pv, double* part) {
  __shared__ double red[2][128];
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  double rz = 0.0, rr = 0.0;
  if (b < nb) {
    const bool st = is_static[b];
    double rb[12];
    for (int k = 0; k < 12; ++k) {
      rb[k] = st ? 0.0 : rhs[12 * b + k];
      r[12 * b + k] = rb[k];
      x[12 * b + k] = 0.0;
      rr += rb[k] * rb[k];
    }
    const double* Pi = Pinv + 144 * b;
    for (int i = 0; i < 12; ++i) {
      double s = 0.0;
      for (int j = 0; j < 12; ++j) s += Pi[12 * i + j] * rb[j];
      z[12 * b + i] = s;
      pv[12 * b + i] = s;
      rz += rb[i] * s;
    }
  }
  red[0][threadIdx.x] = rz;
  red[1][threadIdx.x] = rr;
  __syncthreads();
  for (int o = 64; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      red[0][threadIdx.x] += red[0][threadIdx.x + o];
      red[1][threadIdx.x] += red[1][threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = red[0][0];
    part[2 * blockIdx.x + 1] = red[1][0];
  }
}

__global__ void k_pcg_start(const double* part, int n, DevStatus* st) {
  __shared__ double red[2][256];
  double a = 0.0, c = 0.0;
  for (int i = threadIdx.x; i < n; i += 256) {
    a += part[2 * i];
    c += part[2 * i + 1];
  }
  red[0][threadIdx.x] = a;
  red[1][threadIdx.x] = c;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      red[0][threadIdx.x] += red[0][threadIdx.x + o];
      red[1][threadIdx.x] += red[1][threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    st->scal[0] = red[0][0];
    st->scal[2] = red[1][0];
    st->scal[3] = red[1][0];
    st->scal[7] = 0.0;
    st->scal[6] = red[1][0] == 0.0 ? 1.0 : 0.0;
  }
}

// fixed-order sum: out = sum_i v[i * stride] for i < n
__global__ void k_reduce(const double* v, long stride, const int* n_dev, long n_const, double* out) {
  __shared__ double red[1024];
  const long n = n_dev ? *n_dev : n_const;
  double s = 0.0;
  for (long i = threadIdx.x; i < n; i += 1024) s += v[i * stride];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = 512; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}

__global__ void k_energy_sum(DevStatus* st) {
  st->energy[0] = ((st->energy[1] + st->energy[2]) + st->energy[3]) + st->energy[4];
}

__global__ void k_max_step(int nv, const int* vbody, const uint8_t* is_static, const double4* dx, DevStatus* st) {
  int v = blockIdx.x * blockDim.x + threadIdx.x;
  double m = 0.0;
  if (v < nv && !is_static[vbody[v]]) {
    double4 d = dx[v];
    m = sqrt(d.x * d.x + d.y * d.y + d.z * d.z);
  }
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(kFull, m, o));
  if ((threadIdx.x & 31) == 0 && m > 0.0) atomicMax(&st->step_bits, (unsigned long long)__double_as_longlong(m));
}

__global__ void k_trial(int n, const double* q, const double* dq, double alpha, double* qtrial) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) qtrial[k] = __dadd_rn(q[k], __dmul_rn(alpha, dq[k]));
}

__global__ void k_finish(int nb, const uint8_t* is_static, const double* q, double dt, double* qt, double* qdot) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb) return;
  for (int k = 0; k < 12; ++k) {
    if (is_static[b]) {
      qdot[12 * b + k] = 0.0;
      continue;
    }
    double v = __ddiv_rn(__dsub_rn(q[12 * b + k], qt[12 * b + k]), dt);
    qdot[12 * b + k] = v;
    qt[12 * b + k] = q[12 * b + k];
  }
}

int blocks(long n, int t) { return (int)((n + t - 1) / t > 0 ? (n + t - 1) / t : 1); }

}  // namespace

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
void launch_mass_moments(Scene& s) {
  counted(s);
  k_mass_moments<<<blocks(32L * s.nb, 256), 256, 0, s.stream>>>(s.nb, s.tbeg.p, s.tri.p, s.xbar.p,
                                                                 s.density.p, s.is_static.p, s.mass10.p,
                                                                 s.vol.p);
}

void launch_predictor(Scene& s) {
  counted(s);
  k_predictor<<<blocks(s.nb, 128), 128, 0, s.stream>>>(s.nb, s.is_static.p, s.qt.p, s.qdot.p, s.prm.dt,
                                                        s.prm.gravity[0], s.prm.gravity[1], s.prm.gravity[2],
                                                        s.qtilde.p);
}

void launch_transform(Scene& s, const double* q, double4* x) {
  counted(s);
  k_transform<<<blocks(s.nv, 256), 256, 0, s.stream>>>(s.nv, s.vbody.p, s.xbar.p, q, x);
}

void launch_transform_dq(Scene& s, const double* dq) {
  counted(s);
  k_transform_dq<<<blocks(s.nv, 256), 256, 0, s.stream>>>(s.nv, s.vbody.p, s.xbar.p, dq, s.x.p, s.dx.p, s.x1.p);
}

void launch_body_boxes(Scene& s, bool swept) {
  counted(s);
  k_body_boxes<<<blocks(32L * s.nb, 256), 256, 0, s.stream>>>(s.nb, s.vbeg.p, s.x.p, swept ? s.x1.p : nullptr,
                                                               s.bbox.p);
}

void launch_scan(Scene& s, const int* cnt, int* off, const int* n_dev, int* total_dev, long cap, unsigned flag_bit,
                 unsigned long long* need) {
  counted(s);
  k_scan<<<1, 1024, 0, s.stream>>>(cnt, off, n_dev, n_dev ? 0 : s.nb, total_dev, cap, flag_bit, need, s.st);
}

void launch_body_pairs(Scene& s) {
  counted(s);
  ProfScope pr(s, PF_ROWS);
  k_rows<<<blocks(32L * s.nb, 256), 256, 0, s.stream>>>(s.nb, s.is_static.p, s.bbox.p, s.prm.dhat, s.fpairs.p, s.st,
                                                        s.maxn, s.nbr.p, s.ncount.p, s.st);
  launch_scan(s, s.ncount.p, s.rowoff.p, nullptr, &s.st->np, (long)s.P.cap, ST_CAP_PAIRS, &s.st->need_pairs);
  counted(s);
  k_rows_compact<<<blocks(32L * s.nb, 256), 256, 0, s.stream>>>(s.nb, s.nbr.p, s.ncount.p, s.rowoff.p, s.maxn, s.P.p,
                                                                (long)s.P.cap);
}

void launch_incoming(Scene& s) {
  cudaMemsetAsync(s.in_cnt.p, 0, sizeof(int) * s.nb, s.stream);
  counted(s);
  k_in_count<<<152 * 4, 256, 0, s.stream>>>(s.st, s.P.p, s.in_cnt.p);
  counted(s);
  k_scan<<<1, 1024, 0, s.stream>>>(s.in_cnt.p, s.in_off.p, nullptr, s.nb, &s.st->pad, (long)s.P.cap, 0,
                                   &s.st->need_misc, s.st);
  cudaMemsetAsync(s.in_cnt.p, 0, sizeof(int) * s.nb, s.stream);
  counted(s);
  k_in_fill<<<152 * 4, 256, 0, s.stream>>>(s.st, s.P.p, s.in_off.p, s.in_cnt.p, s.in_list.p);
  counted(s);
  k_in_sort<<<blocks(s.nb, 128), 128, 0, s.stream>>>(s.nb, s.in_off.p, s.in_list.p);
}

void launch_fpairs(Scene& s) {
  counted(s);
  k_flag_active<<<152 * 4, 256, 0, s.stream>>>(s.st, s.acount.p, s.flagbuf.p);
  counted(s);
  k_scan<<<1, 1024, 0, s.stream>>>(s.flagbuf.p, s.posbuf.p, &s.st->np, 0, &s.st->nfp, (long)s.fpairs.cap,
                                   ST_CAP_PAIRS, &s.st->need_misc, s.st);
  counted(s);
  k_fpairs<<<152 * 4, 256, 0, s.stream>>>(s.st, s.P.p, s.flagbuf.p, s.posbuf.p, s.aoff.p, s.fpairs.p, s.fpoff.p);
}

__global__ void k_negate(long n, const double* in, double* out) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) out[i] = -in[i];
}

void launch_negate(Scene& s, const double* in, double* out, long n) {
  counted(s);
  k_negate<<<blocks(n, 256), 256, 0, s.stream>>>(n, in, out);
}

void launch_assemble(Scene& s) {
  counted(s);
  ProfScope pa(s, PF_ASSEMBLE);
  k_assemble<<<152 * 8, 256, 0, s.stream>>>(s.st, s.P.p, s.aoff.p, s.term.p, s.termv.p, s.fpairs.p, s.fpoff.p,
                                            s.fterm.p, s.ftermv.p, s.vbody.p, s.xbar.p, s.pblk.p);
}

void launch_body_terms(Scene& s, const double* q, bool hess) {
  counted(s);
  ProfScope pb(s, PF_BODY);
  k_body_terms<<<blocks(s.nb, 64), 64, 0, s.stream>>>(s.nb, s.is_static.p, q, s.qtilde.p, s.mass10.p, s.vol.p,
                                                       s.kappa_b.p, s.prm.dt, hess, s.Db.p, s.gb.p, s.Eb.p);
}

void launch_gather(Scene& s) {
  counted(s);
  k_gather<<<blocks(32L * s.nb, 256), 256, 0, s.stream>>>(s.nb, s.is_static.p, s.rowoff.p, s.in_off.p, s.in_list.p,
                                                          s.pblk.p, s.Db.p, s.gb.p, s.D.p, s.g.p, s.st);
}

void launch_precond(Scene& s) {
  counted(s);
  k_precond<<<blocks(s.nb, 64), 64, 0, s.stream>>>(s.nb, s.is_static.p, s.D.p, s.Pinv.p, s.st);
}

// energies of the last evaluation into st->energy: bodies, barrier terms or
// per-body-pair barrier energies (energy-only pass), friction terms
void launch_energy_total(Scene& s, bool from_terms) {
  counted(s);
  k_reduce<<<1, 1024, 0, s.stream>>>(s.Eb.p, 2, nullptr, s.nb, &s.st->energy[1]);
  counted(s);
  k_reduce<<<1, 1024, 0, s.stream>>>(s.Eb.p + 1, 2, nullptr, s.nb, &s.st->energy[2]);
  counted(s);
  if (from_terms) k_reduce<<<1, 1024, 0, s.stream>>>(s.term.p, kTermStride, &s.st->nact, 0, &s.st->energy[3]);
  else k_reduce<<<1, 1024, 0, s.stream>>>(s.Epair.p, 1, &s.st->np, 0, &s.st->energy[3]);
  counted(s);
  k_reduce<<<1, 1024, 0, s.stream>>>(s.fterm.p, kTermStride, &s.st->nfr, 0, &s.st->energy[4]);
  counted(s);
  k_energy_sum<<<1, 1, 0, s.stream>>>(s.st);
}

int run_pcg(Scene& s, const double* rhs, double* xout, int max_iter, double rel_tol, double* rel_res) {
  const int nbk = blocks(s.nb, 128);
  counted(s);
  k_pcg_init<<<nbk, 128, 0, s.stream>>>(s.nb, s.is_static.p, s.Pinv.p, rhs, xout, s.r.p, s.z.p, s.pv.p, s.part.p);
  counted(s);
  k_pcg_start<<<1, 256, 0, s.stream>>>(s.part.p, nbk, s.st);
  const int sblocks = blocks(12L * s.nb, kPcgThreads);
  const double tol2 = rel_tol * rel_tol;
  // algorithmic bytes of one product: every stored block once (diagonal and
  // upper off-diagonal, 144 doubles each), the vector read once and the
  // product written once, the pair list once
  const double spmv_bytes = 8.0 * 144.0 * (s.nb + (double)s.last_np) + 2.0 * 8.0 * 12.0 * s.nb + 8.0 * s.last_np;
  int it = 0;
  const int chunk = 16;
  while (true) {
    for (int k = 0; k < chunk; ++k) {
      counted(s);
      {
        ProfScope pv(s, PF_SPMV, spmv_bytes);
        k_spmv<<<sblocks, kPcgThreads, 0, s.stream>>>(s.nb, s.is_static.p, s.D.p, s.rowoff.p, s.in_off.p,
                                                      s.in_list.p, s.P.p, s.pblk.p, s.pv.p, s.Ap.p, s.part.p, s.st);
      }
      counted(s);
      k_pcg_alpha<<<1, 256, 0, s.stream>>>(s.part.p, sblocks, s.st);
      counted(s);
      k_pcg_update<<<nbk, 128, 0, s.stream>>>(s.nb, s.is_static.p, s.Pinv.p, s.pv.p, s.Ap.p, xout, s.r.p, s.z.p,
                                              s.part.p, s.st);
      counted(s);
      k_pcg_beta<<<1, 256, 0, s.stream>>>(s.part.p, nbk, tol2, s.st);
      counted(s);
      k_pcg_dir<<<blocks(12L * s.nb, 256), 256, 0, s.stream>>>(12L * s.nb, s.z.p, s.pv.p, s.st);
    }
    it += chunk;
    cudaMemcpyAsync(s.st_host, s.st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s.stream);
    cudaStreamSynchronize(s.stream);
    if (s.st_host->scal[6] != 0.0 || it >= max_iter) break;
  }
  double rr = s.st_host->scal[2], rr0 = s.st_host->scal[3];
  *rel_res = rr0 > 0 ? sqrt(rr / rr0) : 0.0;
  int iters = (int)s.st_host->scal[7];
  if (s.st_host->scal[6] == 2.0) return -2;
  if (s.st_host->scal[6] == 0.0) return -1;
  return iters;
}

void launch_max_step(Scene& s) {
  counted(s);
  k_max_step<<<blocks(s.nv, 256), 256, 0, s.stream>>>(s.nv, s.vbody.p, s.is_static.p, s.dx.p, s.st);
}

void launch_trial(Scene& s, double alpha) {
  counted(s);
  k_trial<<<blocks(12L * s.nb, 256), 256, 0, s.stream>>>(12 * s.nb, s.q.p, s.dq.p, alpha, s.qtrial.p);
}

void launch_finish_step(Scene& s) {
  counted(s);
  k_finish<<<blocks(s.nb, 128), 128, 0, s.stream>>>(s.nb, s.is_static.p, s.q.p, s.prm.dt, s.qt.p, s.qdot.p);
  launch_predictor(s);
}

}  // namespace abd
