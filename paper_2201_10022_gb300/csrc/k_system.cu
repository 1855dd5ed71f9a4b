// System kernels: mass integrals (Sec. 3.1), predictor (Sec. 4), vertex map
// (Sec. 3), body boxes and body-pair culling (Sec. 4.2), per-body inertia and
// orthogonality terms (Sec. 3.2 / Sec. 4), Hessian assembly by body-pair
// blocks (Sec. 4.3), block-Jacobi PCG, and deterministic reductions.
#include <stddef.h>

#include <algorithm>

#include "abd_internal.cuh"
#include "derivs.cuh"

namespace abd {

namespace {

constexpr unsigned kFull = 0xffffffffu;


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
// squared rest length of every edge, canonical order (edge-edge mollifier
// threshold eps = 1e-3 |rest e_i|^2 |rest e_j|^2)
__global__ void k_edge_rest(int ne, const int* edge, const double4* xbar, double* l2e) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < ne; e += gridDim.x * blockDim.x) {
    v3 d = csub(mk(xbar[edge[2 * e + 1]]), mk(xbar[edge[2 * e]]));
    l2e[e] = cdot(d, d);
  }
}

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

// vertex positions x = J(xbar) q; with isl (the line search's trial
// positions) only the vertices of bodies whose island is still pending
__global__ void k_transform(int nv, const int* vbody, const double4* xbar, const double* q, double4* x,
                            const int* isl, const int* lstate) {
  int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= nv) return;
  const int b = vbody[v];
  if (isl && lstate[2 * isl[b]] != 0) return;
  x[v] = affine(q + 12 * b, xbar[v]);
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

// order-preserving integer key of a double (non-NaN): min / max of keys is
// the exact min / max of the values, on the integer units instead of the
// (slow) FP64 pipe
__device__ __forceinline__ long long dkey(double d) {
  const long long b = __double_as_longlong(d);
  return b >= 0 ? b : b ^ 0x7FFFFFFFFFFFFFFFll;
}
__device__ __forceinline__ double dval(long long k) {
  return __longlong_as_double(k >= 0 ? k : k ^ 0x7FFFFFFFFFFFFFFFll);
}

__global__ void k_body_boxes(int nb, const int* vbeg, const double4* x, const double4* x1, double* bbox,
                             float* bbox32) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= nb) return;
  const int b = warp;
  const long long klo = dkey(1e300), khi = dkey(-1e300);  // an empty body keeps an empty box
  long long lo[3] = {klo, klo, klo}, hi[3] = {khi, khi, khi};
  for (int v = vbeg[b] + lane; v < vbeg[b + 1]; v += 32) {
    const double4 p = x[v];
    const long long k[3] = {dkey(p.x), dkey(p.y), dkey(p.z)};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      lo[c] = min(lo[c], k[c]);
      hi[c] = max(hi[c], k[c]);
    }
    if (x1) {
      const double4 r = x1[v];
      const long long kr[3] = {dkey(r.x), dkey(r.y), dkey(r.z)};
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        lo[c] = min(lo[c], kr[c]);
        hi[c] = max(hi[c], kr[c]);
      }
    }
  }
#pragma unroll
  for (int c = 0; c < 3; ++c)
    for (int o = 16; o > 0; o >>= 1) {
      lo[c] = min(lo[c], __shfl_xor_sync(kFull, lo[c], o));
      hi[c] = max(hi[c], __shfl_xor_sync(kFull, hi[c], o));
    }
  if (lane < 6) {  // FP64 box and its FP32 copy rounded outward
    const int c = lane % 3;
    const double v = dval(lane < 3 ? lo[c] : hi[c]);
    bbox[6 * b + lane] = v;
    bbox32[6 * b + lane] = lane < 3 ? __double2float_rd(v) : __double2float_ru(v);
  }
}

// ---------------------------------------------------------------------------
// body pairs (a < b, not both static) whose boxes are within dhat, plus the
// lagged friction body pairs; one row per body (the smaller index, or the
// non-large body), sorted by the other body.  A spatial hash over the bodies'
// d-hat-dilated boxes finds the neighbours of ordinary bodies; bodies whose
// box spans more than kMaxCells cells ("large", e.g. a ground slab) are tested
// directly against every body.
// ---------------------------------------------------------------------------
constexpr int kMaxCells = 64;

__device__ __forceinline__ int cell_of(double v, double inv_h) { return (int)floor(v * inv_h); }
__device__ __forceinline__ unsigned slot_of(int ix, int iy, int iz, unsigned mask) {
  return ((unsigned)ix * 73856093u ^ (unsigned)iy * 19349663u ^ (unsigned)iz * 83492791u) & mask;
}
__device__ __forceinline__ void cell_range(const double* bb, double dhat, double inv_h, int lo[3], int hi[3]) {
  for (int k = 0; k < 3; ++k) {
    lo[k] = cell_of(bb[k] - dhat, inv_h);
    hi[k] = cell_of(bb[3 + k] + dhat, inv_h);
  }
}
// conservative FP32 test on the outward-rounded boxes: true only if some
// axis is separated by more than dh32 (d-hat rounded up with a relative
// margin of 1e-6), in which case the exact FP64 predicate below is false too
__device__ __forceinline__ bool bodies_far32(const float* A, const float* B, float dh32) {
  bool far = false;
#pragma unroll
  for (int k = 0; k < 3; ++k) far = far || __fsub_rd(A[k], B[3 + k]) > dh32 || __fsub_rd(B[k], A[3 + k]) > dh32;
  return far;
}

__device__ __forceinline__ bool bodies_near(const double* A, const double* B, double dhat) {
  for (int k = 0; k < 3; ++k) {
    if (!(__dsub_rn(A[k], B[3 + k]) <= dhat)) return false;
    if (!(__dsub_rn(B[k], A[3 + k]) <= dhat)) return false;
  }
  return true;
}

__global__ void k_hash_count(int nb, const double* bbox, double dhat, double inv_h, int* count, int* large) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb) return;
  int lo[3], hi[3];
  cell_range(bbox + 6 * b, dhat, inv_h, lo, hi);
  long n = (long)(hi[0] - lo[0] + 1) * (hi[1] - lo[1] + 1) * (hi[2] - lo[2] + 1);
  const bool big = n > kMaxCells || n <= 0;
  large[b] = big ? 1 : 0;
  count[b] = big ? 0 : (int)n;
}

__global__ void k_large_list(int nb, const int* large, const int* pos, int* list) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < nb && large[b]) list[pos[b]] = b;
}

__global__ void k_hash_slots(int nb, const double* bbox, const int* large, double dhat, double inv_h, unsigned mask,
                             int* slot_cnt, const int* slot_off, int* entries, long cap, bool fill) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb || large[b]) return;
  int lo[3], hi[3];
  cell_range(bbox + 6 * b, dhat, inv_h, lo, hi);
  for (int ix = lo[0]; ix <= hi[0]; ++ix)
    for (int iy = lo[1]; iy <= hi[1]; ++iy)
      for (int iz = lo[2]; iz <= hi[2]; ++iz) {
        unsigned h = slot_of(ix, iy, iz, mask);
        int pos = atomicAdd(&slot_cnt[h], 1);
        if (fill && (long)slot_off[h] + pos < cap) entries[slot_off[h] + pos] = b;
      }
}

__global__ void k_rows(int nb, const uint8_t* is_static, const double* bbox, const float* bbox32, float dh32,
                       double dhat, double inv_h, unsigned mask,
                       const int* large, const int* large_list, const int* slot_off, const int* entries,
                       const int2* fpairs, const DevStatus* cst, int maxn, int* nbr, int* ncount, DevStatus* st) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  const int nfp = cst->nfp, nlarge = cst->nlarge;
  for (int a = warp; a < nb; a += nwarps) {
    const double* A = bbox + 6 * a;
    const bool sa = is_static[a];
    int* out = nbr + (size_t)a * maxn;
    int base = 0;
    auto emit = [&](bool keep, int b) {
      unsigned m = __ballot_sync(kFull, keep);
      if (keep) {
        int pos = base + __popc(m & ((1u << lane) - 1u));
        if (pos < maxn) out[pos] = b;
      }
      base += __popc(m);
    };
    if (large[a]) {
      continue;  // rows of large bodies: k_rows_large
    } else {
      int lo[3], hi[3];
      cell_range(A, dhat, inv_h, lo, hi);
      for (int ix = lo[0]; ix <= hi[0]; ++ix)
        for (int iy = lo[1]; iy <= hi[1]; ++iy)
          for (int iz = lo[2]; iz <= hi[2]; ++iz) {
            unsigned h = slot_of(ix, iy, iz, mask);
            const int e0 = slot_off[h], e1 = slot_off[h + 1];
            for (int k0 = e0; k0 < e1; k0 += 32) {
              int k = k0 + lane;
              bool keep = false;
              int b = -1;
              if (k < e1) {
                b = entries[k];
                const double* B = bbox + 6 * b;
                if (b > a && !(sa && is_static[b]) && !bodies_far32(bbox32 + 6 * a, bbox32 + 6 * b, dh32) &&
                    bodies_near(A, B, dhat)) {
                  // report the pair only in the cell of the low corner of the
                  // dilated boxes' overlap, so it is found once
                  keep = cell_of(fmax(A[0], B[0]) - dhat, inv_h) == ix && cell_of(fmax(A[1], B[1]) - dhat, inv_h) == iy &&
                         cell_of(fmax(A[2], B[2]) - dhat, inv_h) == iz;
                }
              }
              emit(keep, b);
            }
          }
      // large bodies after a
      for (int k0 = 0; k0 < nlarge; k0 += 32) {
        int k = k0 + lane;
        int b = k < nlarge ? large_list[k] : -1;
        bool keep = b > a && !(sa && is_static[b]) && !bodies_far32(bbox32 + 6 * a, bbox32 + 6 * b, dh32) &&
                    bodies_near(A, bbox + 6 * b, dhat);
        emit(keep, b);
      }
      // hash order is arbitrary: sort the row and drop repeats (a body
      // listed twice in one slot when two of its cells share the slot)
      if (lane == 0) {
        const int n = min(base, maxn);
        for (int i = 1; i < n; ++i) {
          int v = out[i], j = i - 1;
          while (j >= 0 && out[j] > v) {
            out[j + 1] = out[j];
            --j;
          }
          out[j + 1] = v;
        }
        int u = 0;
        for (int i = 0; i < n; ++i)
          if (u == 0 || out[i] != out[u - 1]) out[u++] = out[i];
        if (base <= maxn) base = u;
      }
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
    __syncwarp();
  }
}

// rows of large bodies: one block scans every body after the large one, in
// order, with a block-wide ordered compaction; then the friction merge
// rows of large bodies up to this many entries merge their missing friction
// neighbours in shared memory
constexpr int kRowMerge = 6144;

__global__ void k_rows_large(int nb, const uint8_t* is_static, const double* bbox, const float* bbox32, float dh32,
                             double dhat, const int* large_list,
                             const int2* fpairs, const DevStatus* cst, int maxn, int* nbr, int* ncount, DevStatus* st) {
  __shared__ int wcount[32];
  __shared__ int wbase[33];
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const int nlarge = cst->nlarge, nfp = cst->nfp;
  for (int li = blockIdx.x; li < nlarge; li += gridDim.x) {
    const int a = large_list[li];
    const double* A = bbox + 6 * a;
    const bool sa = is_static[a];
    int* out = nbr + (size_t)a * maxn;
    int base = 0;
    for (int b0 = a + 1; b0 < nb; b0 += 1024) {
      const int b = b0 + t;
      const bool keep = b < nb && !(sa && is_static[b]) && !bodies_far32(bbox32 + 6 * a, bbox32 + 6 * b, dh32) &&
                        bodies_near(A, bbox + 6 * b, dhat);
      const unsigned m = __ballot_sync(kFull, keep);
      if (lane == 0) wcount[w] = __popc(m);
      __syncthreads();
      if (w == 0) {  // warp offsets by an inclusive shuffle scan
        int x = wcount[lane];
        for (int o = 1; o < 32; o <<= 1) {
          const int y = __shfl_up_sync(kFull, x, o);
          if (lane >= o) x += y;
        }
        wbase[lane + 1] = x;
        if (lane == 0) wbase[0] = 0;
      }
      __syncthreads();
      if (keep) {
        const int pos = base + wbase[w] + __popc(m & ((1u << lane) - 1u));
        if (pos < maxn) out[pos] = b;
      }
      base += wbase[32];
      __syncthreads();
    }
    // friction neighbours of the row (fpairs entries with .x == a): the
    // threads check membership by binary search; the missing ones (at most
    // 256, the row and they at most kRowMerge entries) are merged into the
    // sorted row in parallel through shared memory, else inserted by one
    // thread
    __shared__ int frange[2], nmiss;
    __shared__ int miss[256], smiss[256];
    __shared__ int srow[kRowMerge];
    if (t < 2) {  // first entry with .x >= a (t = 0), first with .x > a (t = 1)
      int lo = 0, hi = nfp;
      while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (fpairs[mid].x < a + t) lo = mid + 1;
        else hi = mid;
      }
      frange[t] = lo;
    }
    if (t == 0) nmiss = 0;
    __syncthreads();
    const int n0 = min(base, maxn);
    for (int f = frange[0] + t; f < frange[1]; f += blockDim.x) {
      const int b = fpairs[f].y;
      int lo = 0, hi = n0;
      while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (out[mid] < b) lo = mid + 1;
        else hi = mid;
      }
      if (!(lo < n0 && out[lo] == b)) {
        int k = atomicAdd(&nmiss, 1);
        if (k < 256) miss[k] = b;
      }
    }
    __syncthreads();
    const int nm = nmiss;
    if (nm > 0 && nm <= 256 && base <= maxn && n0 + nm <= kRowMerge) {
      // sorted misses (distinct body ids: rank = number of smaller ones)
      for (int i = t; i < nm; i += blockDim.x) {
        int r = 0;
        for (int k = 0; k < nm; ++k) r += miss[k] < miss[i];
        smiss[r] = miss[i];
      }
      for (int k = t; k < n0; k += blockDim.x) srow[k] = out[k];
      __syncthreads();
      const int total = n0 + nm;
      // every entry's place in the merged row: its index plus the number of
      // entries of the other list below it
      for (int k = t; k < n0; k += blockDim.x) {
        const int v = srow[k];
        int lo = 0, hi = nm;
        while (lo < hi) {
          int mid = (lo + hi) >> 1;
          if (smiss[mid] < v) lo = mid + 1;
          else hi = mid;
        }
        if (k + lo < maxn) out[k + lo] = v;
      }
      for (int i = t; i < nm; i += blockDim.x) {
        const int v = smiss[i];
        int lo = 0, hi = n0;
        while (lo < hi) {
          int mid = (lo + hi) >> 1;
          if (srow[mid] < v) lo = mid + 1;
          else hi = mid;
        }
        if (i + lo < maxn) out[i + lo] = v;
      }
      if (t == 0) {
        ncount[a] = min(total, maxn);
        if (total > maxn) {
          set_flag(st, ST_CAP_ROWS);
          atomicMax(&st->need_row, total);
        }
      }
    } else if (t == 0) {
      // more misses than the buffer holds: walk every friction neighbour
      const bool all = nm > 256;
      const int nmw = all ? frange[1] - frange[0] : nm;
      for (int i = 0; i < nmw; ++i) {
        const int b = all ? fpairs[frange[0] + i].y : miss[i];
        const int n = min(base, maxn);
        int pos = 0;
        while (pos < n && out[pos] < b) ++pos;
        if (pos < n && out[pos] == b) continue;
        if (base < maxn) {
          for (int k = n; k > pos; --k) out[k] = out[k - 1];
          out[pos] = b;
        }
        ++base;
      }
      ncount[a] = min(base, maxn);
      if (base > maxn) {
        set_flag(st, ST_CAP_ROWS);
        atomicMax(&st->need_row, base);
      }
    }
    __syncthreads();
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

// single-block exclusive scan in tiles of 4096 (coalesced loads, fixed order)
__global__ void k_scan(const int* cnt, int* off, const int* n_dev, int n_const, int* total_dev, long cap,
                       unsigned flag, unsigned long long* need, DevStatus* st) {
  __shared__ long long wsum[32];
  __shared__ long long carry_s;
  const int n = n_dev ? *n_dev : n_const;
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  if (t == 0) carry_s = 0;
  __syncthreads();
  for (int base = 0; base < n; base += 4096) {
    int v[4];
    long long loc = 0;
    for (int k = 0; k < 4; ++k) {
      const int i = base + 4 * t + k;
      v[k] = i < n ? cnt[i] : 0;
      loc += v[k];
    }
    // inclusive scan of the per-thread sums: warp, then warp totals
    long long inc = loc;
    for (int o = 1; o < 32; o <<= 1) {
      long long u = __shfl_up_sync(kFull, inc, o);
      if (lane >= o) inc += u;
    }
    if (lane == 31) wsum[w] = inc;
    __syncthreads();
    if (w == 0) {
      long long x = wsum[lane];
      for (int o = 1; o < 32; o <<= 1) {
        long long u = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += u;
      }
      wsum[lane] = x;
    }
    __syncthreads();
    long long run = carry_s + (w ? wsum[w - 1] : 0) + inc - loc;
    for (int k = 0; k < 4; ++k) {
      const int i = base + 4 * t + k;
      if (i < n) off[i] = (int)run;
      run += v[k];
    }
    __syncthreads();
    if (t == 1023) carry_s += wsum[31];
    __syncthreads();
  }
  if (t == 0) {
    long long total = carry_s;
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

// two-phase exclusive scan for long arrays: tile sums (4096 entries a block),
// then every block scans its tile from the sum of the tiles before it; the
// last block writes off[n] and the clamped total
constexpr int kScanTile = 4096;

__global__ void k_scan_tiles(const int* cnt, int n, long long* part) {
  __shared__ long long ws[32];
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const int base = blockIdx.x * kScanTile;
  long long loc = 0;
  for (int k = 0; k < 4; ++k) {
    const int i = base + 4 * t + k;
    if (i < n) loc += cnt[i];
  }
  for (int o = 16; o > 0; o >>= 1) loc += __shfl_xor_sync(kFull, loc, o);
  if (lane == 0) ws[w] = loc;
  __syncthreads();
  if (w == 0) {
    long long x = ws[lane];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
    if (lane == 0) part[blockIdx.x] = x;
  }
}

__global__ void k_scan_apply(const int* cnt, int* off, int n, const long long* part, int* total_dev, long cap,
                             unsigned flag, unsigned long long* need, DevStatus* st) {
  __shared__ long long wsum[32];
  __shared__ long long carry_s;
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const int b = blockIdx.x, base = b * kScanTile;
  if (w == 0) {  // sum of the earlier tiles, in a fixed order
    long long c = 0;
    for (int k = lane; k < b; k += 32) c += part[k];
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(kFull, c, o);
    if (lane == 0) carry_s = c;
  }
  int v[4];
  long long loc = 0;
  for (int k = 0; k < 4; ++k) {
    const int i = base + 4 * t + k;
    v[k] = i < n ? cnt[i] : 0;
    loc += v[k];
  }
  long long inc = loc;
  for (int o = 1; o < 32; o <<= 1) {
    long long u = __shfl_up_sync(kFull, inc, o);
    if (lane >= o) inc += u;
  }
  if (lane == 31) wsum[w] = inc;
  __syncthreads();
  if (w == 0) {
    long long x = wsum[lane];
    for (int o = 1; o < 32; o <<= 1) {
      long long u = __shfl_up_sync(kFull, x, o);
      if (lane >= o) x += u;
    }
    wsum[lane] = x;
  }
  __syncthreads();
  long long run = carry_s + (w ? wsum[w - 1] : 0) + inc - loc;
  for (int k = 0; k < 4; ++k) {
    const int i = base + 4 * t + k;
    if (i < n) off[i] = (int)run;
    run += v[k];
  }
  if (b == gridDim.x - 1 && t == 1023) {
    const long long total = run;  // thread 1023 of the last tile ends past n
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

// A body pair's terms: its active barrier terms t0..t1 of term/termv, then
// its lagged friction records f0..f1 of fterm/ftermv.
struct PairTerms {
  int a, t0, t1, f0, f1;
  __device__ int count() const { return (t1 - t0) + (f1 - f0); }
};

__device__ __forceinline__ PairTerms pair_terms(const DevStatus* cst, const int2* P, const int* aoff,
                                                const int2* fpairs, const int* fpoff, int p) {
  const int nfp = cst->nfp, nact = cst->nact;
  const int a = P[p].x, b = P[p].y;
  PairTerms pt{a, aoff[p], min(aoff[p + 1], nact), 0, 0};
  if (nfp > 0) {
    int q = find_fpair(fpairs, nfp, a, b);
    if (q >= 0) {
      pt.f0 = fpoff[q];
      pt.f1 = fpoff[q + 1];
    }
  }
  return pt;
}

// One warp adds term number it of the pair to its lanes' accumulators.
// lanes 0..26: region r = lane / 9 (0: H_ab, 1: D_a, 2: D_b) and spatial
// component pair (c, c2) = ((lane % 9) / 3, lane % 3); each accumulates the
// 4x4 block over the weight indices (u, u2) of
//   sum_{k on side sk, l on side sl} w_k[u] w_l[u2] H_kl[c][c2]
// as two 4x4 products (T = W_sk^T H_c, then T W_sl) with the other side's
// weights zeroed; lanes 27..31: the 24 gradient entries and two energies.
// sH, sw, sside: this warp's staging in shared memory.
__device__ __forceinline__ void assemble_term(const PairTerms& pt, int it, const double* term, const int4* termv,
                                              const double* fterm, const int4* ftermv, const int* vbody,
                                              const double4* xbar, double* sHw, double (*sww)[4], int* ssidew,
                                              double (&acc)[16]) {
  const int lane = threadIdx.x & 31;
  const int a = pt.a, t0 = pt.t0, t1 = pt.t1, f0 = pt.f0;
  const int r = lane / 9, cc = (lane % 9) / 3, c2 = lane % 3;
  const int sk = r == 2 ? 1 : 0, sl = r == 1 ? 0 : 1;
    const bool fr = it >= (t1 - t0);
    const int t = fr ? f0 + (it - (t1 - t0)) : t0 + it;
    const double* T = (fr ? fterm : term) + (size_t)t * kTermStride;
    for (int k = lane; k < kTermStride; k += 32) sHw[k] = T[k];
    if (lane < 4) {
      int4 vv = fr ? ftermv[t] : termv[t];
      int v = lane == 0 ? vv.x : (lane == 1 ? vv.y : (lane == 2 ? vv.z : vv.w));
      ssidew[lane] = vbody[v] == a ? 0 : 1;
      double4 xb = xbar[v];
      sww[lane][0] = 1.0;
      sww[lane][1] = xb.x;
      sww[lane][2] = xb.y;
      sww[lane][3] = xb.z;
    }
    __syncwarp();
    const double* H = sHw + 13;
    const double* g = sHw + 1;
    if (lane < 27) {
      double wk[4][4], wl[4][4];
#pragma unroll
      for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          wk[k][u] = ssidew[k] == sk ? sww[k][u] : 0.0;
          wl[k][u] = ssidew[k] == sl ? sww[k][u] : 0.0;
        }
      double Tm[4][4];
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int l = 0; l < 4; ++l) {
          double x = 0.0;
#pragma unroll
          for (int k = 0; k < 4; ++k) x += wk[k][u] * H[up12(3 * k + cc, 3 * l + c2)];
          Tm[u][l] = x;
        }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int u2 = 0; u2 < 4; ++u2) {
          double x = acc[4 * u + u2];
#pragma unroll
          for (int l = 0; l < 4; ++l) x += Tm[u][l] * wl[l][u2];
          acc[4 * u + u2] = x;
        }
    } else {
#pragma unroll
      for (int j = 0; j < 6; ++j) {
        const int gi = (lane - 27) + 5 * j;
        double c = 0.0;
        if (gi < 24) {
          const int sd = gi / 12;
          int u, ci;
          inv_dof(gi % 12, u, ci);
          for (int k = 0; k < 4; ++k)
            if (ssidew[k] == sd) c += sww[k][u] * g[3 * k + ci];
        } else if (gi == 24) {
          c = fr ? 0.0 : sHw[0];
        } else if (gi == 25) {
          c = fr ? sHw[0] : 0.0;
        }
        acc[j] += c;
      }
    }
  __syncwarp();
}

// the pair's accumulated blocks, gradient parts and energies to its slot
__device__ __forceinline__ void assemble_write(double* pblk, int p, const double (&acc)[16]) {
  const int lane = threadIdx.x & 31;
  const int r = lane / 9, cc = (lane % 9) / 3, c2 = lane % 3;
  double* out = pblk + (size_t)p * kBlkStride;
  if (lane < 27) {
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int u2 = 0; u2 < 4; ++u2)
        out[144 * r + 12 * dof(u, cc) + dof(u2, c2)] = acc[4 * u + u2];
  } else {
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      const int gi = (lane - 27) + 5 * j;
      if (gi < 26) out[432 + gi] = acc[j];
    }
  }
}

// pairs with more terms than this go to k_assemble_large (a block per pair)
constexpr int kAssembleLarge = 12;
constexpr int kAssembleWarps = 8;

// a warp per body pair with at most kAssembleLarge terms (its terms in
// order); larger pairs are listed for k_assemble_large
__global__ void __launch_bounds__(128) k_assemble(const DevStatus* cst, const int2* P, const int* aoff,
                                                  const double* term, const int4* termv, const int2* fpairs,
                                                  const int* fpoff, const double* fterm, const int4* ftermv,
                                                  const int* vbody, const double4* xbar, double* pblk,
                                                  int* large_pairs, DevStatus* st) {
  __shared__ double sH[4][kTermStride];
  __shared__ double sw[4][4][4];
  __shared__ int sside[4][4];
  const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  const int np = cst->np;
  for (int p = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; p < np; p += nwarps) {
    const PairTerms pt = pair_terms(cst, P, aoff, fpairs, fpoff, p);
    const int nterms = pt.count();
    if (nterms > kAssembleLarge) {
      if (lane == 0) large_pairs[atomicAdd(&st->n_large_asm, 1)] = p;
      continue;
    }
    double acc[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) acc[k] = 0.0;
    for (int it = 0; it < nterms; ++it)
      assemble_term(pt, it, term, termv, fterm, ftermv, vbody, xbar, sH[wib], sw[wib], sside[wib], acc);
    assemble_write(pblk, p, acc);
  }
}

// a block of kAssembleWarps warps per listed pair: warp w takes terms w,
// w + kAssembleWarps, ...; the warps' sums are added in warp order (a fixed
// order, so results do not depend on timing)
__global__ void __launch_bounds__(32 * kAssembleWarps) k_assemble_large(
    const DevStatus* __restrict__ cst, const int2* P, const int* aoff, const double* term, const int4* termv,
    const int2* fpairs, const int* fpoff, const double* fterm, const int4* ftermv, const int* vbody,
    const double4* xbar, double* pblk, const int* large_pairs) {
  __shared__ double sH[kAssembleWarps][kTermStride];
  __shared__ double sw[kAssembleWarps][4][4];
  __shared__ int sside[kAssembleWarps][4];
  __shared__ double sacc[kAssembleWarps][16][33];
  const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nl = cst->n_large_asm;
  for (int k = blockIdx.x; k < nl; k += gridDim.x) {
    const int p = large_pairs[k];
    const PairTerms pt = pair_terms(cst, P, aoff, fpairs, fpoff, p);
    const int nterms = pt.count();
    double acc[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) acc[j] = 0.0;
    for (int it = wib; it < nterms; it += kAssembleWarps)
      assemble_term(pt, it, term, termv, fterm, ftermv, vbody, xbar, sH[wib], sw[wib], sside[wib], acc);
#pragma unroll
    for (int j = 0; j < 16; ++j) sacc[wib][j][lane] = acc[j];
    __syncthreads();
    if (wib == 0) {
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        double x = sacc[0][j][lane];
        for (int w = 1; w < kAssembleWarps; ++w) x += sacc[w][j][lane];
        acc[j] = x;
      }
      assemble_write(pblk, p, acc);
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// per-body inertia and orthogonality energies and gradients (Sec. 3.2,
// Sec. 4); the Hessian block is formed by k_body_hess
// ---------------------------------------------------------------------------
__global__ void k_body_terms(int nb, const uint8_t* is_static, const double* q, const double* qtilde,
                             const double* mass10, const double* vol, const double* kappa_b, double dt, double* gb,
                             double* Eb, const int* isl, const int* lstate) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb) return;
  // line-search rounds: bodies of islands already accepted are not needed
  if (isl && !is_static[b] && lstate[2 * isl[b]] != 0) return;
  if (is_static[b]) {
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

}

// one body per thread, 32 bodies per block: the blocks are staged through
// shared memory (rows padded to 145 doubles: conflict-free per-thread rows)
// with coalesced loads and stores, and factored in registers
constexpr int kBodyWarp = 32;

__device__ __forceinline__ constexpr int tri(int i, int j) { return i * (i + 1) / 2 + j; }  // j <= i

// in-register Cholesky of a 12x12 symmetric matrix held as its lower
// triangle: L receives the factor below the diagonal and 1 / L_ii on it;
// false if a pivot is not positive
__device__ __forceinline__ bool chol12(double* L) {
  bool ok = true;
#pragma unroll
  for (int j = 0; j < 12; ++j) {
    double d = L[tri(j, j)];
#pragma unroll
    for (int k = 0; k < j; ++k) d -= L[tri(j, k)] * L[tri(j, k)];
    ok = ok && d > 0.0;
    const double r = rsqrt(d);
    L[tri(j, j)] = r;
#pragma unroll
    for (int i = j + 1; i < 12; ++i) {
      double t = L[tri(i, j)];
#pragma unroll
      for (int k = 0; k < j; ++k) t -= L[tri(i, k)] * L[tri(j, k)];
      L[tri(i, j)] = t * r;
    }
  }
  return ok;
}

// Hessian block of the body terms (Sec. 3.2, Sec. 4): B = M + dt^2 hess V_ortho
// over q = (p, rows a_i of A), with the closed form
//   d2 V / da_k da_l = 4 kappa nu [C_kl I + delta_kl A^T A + a_l a_k^T],
//   C = A A^T - I,
// used as it is when it is positive definite (a Cholesky factorisation
// succeeds).  Otherwise C is replaced by its eigenvalue clamp C+ (3x3 cyclic
// Jacobi): the Gauss-Newton part of the sum of squares V = kappa nu |C|_F^2
// stays and the residual curvature is clamped, so the block is positive
// definite (M is) and equals the true one whenever C is positive
// semidefinite.  One body per thread; static bodies get I.
__device__ __forceinline__ int qcomp(int i) { return i < 3 ? i : (i - 3) / 3; }  // spatial row of dof i
__device__ __forceinline__ int qmono(int i) { return i < 3 ? 0 : 1 + (i - 3) % 3; }  // 1, xbar_x, xbar_y, xbar_z

__device__ __forceinline__ void body_block(const double W[4][4], const double A[3][3], const double C[3][3],
                                           double s4, double* B) {
#pragma unroll
  for (int i = 0; i < 12; ++i)
#pragma unroll
    for (int j = 0; j <= i; ++j) {
      double v = qcomp(i) == qcomp(j) ? W[qmono(i)][qmono(j)] : 0.0;
      if (i >= 3 && j >= 3) {
        const int k = qcomp(i), ck = qmono(i) - 1, l = qcomp(j), cl = qmono(j) - 1;
        double h = A[l][ck] * A[k][cl];
        if (ck == cl) h += C[k][l];
        if (k == l) h += A[0][ck] * A[0][cl] + A[1][ck] * A[1][cl] + A[2][ck] * A[2][cl];
        v += s4 * h;
      }
      B[tri(i, j)] = v;
    }
}

__global__ void __launch_bounds__(kBodyWarp) k_body_hess(int nb, const uint8_t* is_static, const double* q,
                                                         const double* mass10, const double* vol,
                                                         const double* kappa_b, double dt, int project, double* Db,
                                                         DevStatus* st) {
  __shared__ double S[kBodyWarp][145];
  const int t = threadIdx.x;
  const long b0 = (long)blockIdx.x * kBodyWarp, b = b0 + t;
  const bool live = b < nb && !is_static[b];
  double B[78];
  if (live) {
    const double* m = mass10 + 10 * b;
    const double W[4][4] = {{m[0], m[1], m[2], m[3]}, {m[1], m[4], m[5], m[6]}, {m[2], m[5], m[7], m[8]},
                            {m[3], m[6], m[8], m[9]}};
    double A[3][3], C[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int c = 0; c < 3; ++c) A[i][c] = q[12 * b + 3 + 3 * i + c];
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
      for (int l = 0; l < 3; ++l)
        C[k][l] = A[k][0] * A[l][0] + A[k][1] * A[l][1] + A[k][2] * A[l][2] - (k == l ? 1.0 : 0.0);
    const double s4 = dt * dt * 4.0 * kappa_b[b] * vol[b];
    body_block(W, A, C, s4, B);
    double L[78];
#pragma unroll
    for (int k = 0; k < 78; ++k) L[k] = B[k];
    if (project && !chol12(L)) {
      double Cm[9], V[9];
#pragma unroll
      for (int k = 0; k < 9; ++k) Cm[k] = C[k / 3][k % 3];
      jacobi_eig<3, double>(Cm, V);
      double Cp[3][3];
#pragma unroll
      for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int l = 0; l < 3; ++l) {
          double v = 0.0;
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            const double lam = Cm[4 * c];
            if (lam > 0.0) v += V[3 * k + c] * lam * V[3 * l + c];
          }
          Cp[k][l] = v;
        }
      body_block(W, A, Cp, s4, B);
      atomicAdd(&st->bh_fix, 1);
    }
  } else {
#pragma unroll
    for (int i = 0; i < 12; ++i)
#pragma unroll
      for (int j = 0; j <= i; ++j) B[tri(i, j)] = i == j ? 1.0 : 0.0;
  }
#pragma unroll
  for (int i = 0; i < 12; ++i)
#pragma unroll
    for (int j = 0; j <= i; ++j) {
      S[t][12 * i + j] = B[tri(i, j)];
      S[t][12 * j + i] = B[tri(i, j)];
    }
  __syncthreads();
  for (int k = t; k < kBodyWarp * 144; k += kBodyWarp) {
    const int bb = k / 144, e = k - 144 * bb;
    if (b0 + bb < nb) Db[144 * (b0 + bb) + e] = S[bb][e];
  }
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

// block-Jacobi preconditioner: the explicit inverse of each dynamic diagonal
// block, from its Cholesky factor (L^-1 in place, then L^-T L^-1), stored per
// body as a full symmetric 144-double block.  A block that is not positive
// definite falls back to the inverse of its diagonal (flagged); static bodies
// get a zero block (their rows stay zero).
__global__ void __launch_bounds__(kBodyWarp) k_precond(int nb, const uint8_t* is_static, const double* D,
                                                       double* Minv, DevStatus* st) {
  __shared__ double S[kBodyWarp][145];
  const int t = threadIdx.x;
  const long b0 = (long)blockIdx.x * kBodyWarp, b = b0 + t;
  for (int k = t; k < kBodyWarp * 144; k += kBodyWarp) {
    const int bb = k / 144, e = k - 144 * bb;
    S[bb][e] = b0 + bb < nb ? D[144 * (b0 + bb) + e] : 0.0;
  }
  __syncthreads();
  const bool live = b < nb && !is_static[b];
  double L[78];
#pragma unroll
  for (int i = 0; i < 12; ++i)
#pragma unroll
    for (int j = 0; j <= i; ++j) L[tri(i, j)] = S[t][12 * i + j];
  const bool fallback = live && !chol12(L);
  // L^-1 in place, column by column: the diagonal already holds 1 / L_jj;
  // entry (i, j) needs L(i, k) of columns k > j (not yet overwritten) and the
  // inverse's entries (k, j), k < i, of its own column (already written)
#pragma unroll
  for (int j = 0; j < 12; ++j)
#pragma unroll
    for (int i = j + 1; i < 12; ++i) {
      double acc = L[tri(i, j)] * L[tri(j, j)];
#pragma unroll
      for (int k = j + 1; k < i; ++k) acc += L[tri(i, k)] * L[tri(k, j)];
      L[tri(i, j)] = -acc * L[tri(i, i)];
    }
  // M^-1 = L^-T L^-1: entry (i, j), i >= j, = sum_{k >= i} Li(k, i) Li(k, j)
#pragma unroll
  for (int i = 0; i < 12; ++i)
#pragma unroll
    for (int j = 0; j <= i; ++j) {
      double v = 0.0;
#pragma unroll
      for (int k = i; k < 12; ++k) v += L[tri(k, i)] * L[tri(k, j)];
      if (!live) v = 0.0;
      if (fallback) {
        const double d = S[t][13 * i];
        v = i == j ? (d != 0.0 ? 1.0 / fabs(d) : 1.0) : 0.0;
      }
      S[t][12 * i + j] = v;
      S[t][12 * j + i] = v;
    }
  if (fallback) set_flag(st, ST_PCG_BREAKDOWN);
  __syncthreads();
  for (int k = t; k < kBodyWarp * 144; k += kBodyWarp) {
    const int bb = k / 144, e = k - 144 * bb;
    if (b0 + bb < nb) Minv[144 * (b0 + bb) + e] = S[bb][e];
  }
}

// the four energy components (inertia, orthogonality, barrier, friction) in
// fixed order: component k = blockIdx.y is cut into kEnergyParts contiguous
// ranges of equal length (a function of its count only, not of the grid);
// block x sums range x (strided per thread, then a shared-memory tree)
__global__ void __launch_bounds__(256) k_energies(const double* Eb, int nb, const double* bar, long bar_stride,
                                                  const int* nbar, int nbar_mul, const double* fterm, const int* nfr,
                                                  double* part) {
  __shared__ double red[256];
  const int k = blockIdx.y;
  const double* v = k == 0 ? Eb : (k == 1 ? Eb + 1 : (k == 2 ? bar : fterm));
  const long stride = k < 2 ? 2 : (k == 2 ? bar_stride : kTermStride);
  const long n = k < 2 ? nb : (k == 2 ? (long)*nbar * nbar_mul : *nfr);
  const long len = (n + kEnergyParts - 1) / kEnergyParts;
  for (int x = blockIdx.x; x < kEnergyParts; x += gridDim.x) {
    const long lo = x * len, hi = min(n, lo + len);
    double acc = 0.0;
    for (long i = lo + threadIdx.x; i < hi; i += 256) acc += v[i * stride];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
      if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
      __syncthreads();
    }
    if (threadIdx.x == 0) part[k * kEnergyParts + x] = red[0];
    __syncthreads();
  }
}

// components from their partial sums (warp k sums component k in fixed
// order), then the total; keep != 0 also stores it in energy[5] (the
// reference value of the line search, which later energy-only passes do not
// overwrite)
__global__ void k_energy_sum(const double* part, DevStatus* st, int keep) {
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double acc = 0.0;
  for (int i = lane; i < kEnergyParts; i += 32) acc += part[w * kEnergyParts + i];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(kFull, acc, o);
  if (lane == 0) st->energy[1 + w] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    st->energy[0] = ((st->energy[1] + st->energy[2]) + st->energy[3]) + st->energy[4];
    if (keep) st->energy[5] = st->energy[0];
  }
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

__global__ void k_trial(int n, const double* q, const double* dq, double alpha, const DevStatus* toi_from,
                        double* qtrial) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (toi_from) alpha = __longlong_as_double((long long)toi_from->toi_bits);
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

void launch_edge_rest(Scene& s) {
  if (s.ne == 0) return;
  counted(s);
  k_edge_rest<<<blocks(s.ne, 256), 256, 0, s.stream>>>(s.ne, s.edge.p, s.xbar.p, s.l2e.p);
}

void launch_predictor(Scene& s) {
  counted(s);
  k_predictor<<<blocks(s.nb, 128), 128, 0, s.stream>>>(s.nb, s.is_static.p, s.qt.p, s.qdot.p, s.prm.dt,
                                                        s.prm.gravity[0], s.prm.gravity[1], s.prm.gravity[2],
                                                        s.qtilde.p);
}

void launch_transform(Scene& s, const double* q, double4* x, bool pending_only) {
  counted(s);
  k_transform<<<blocks(s.nv, 256), 256, 0, s.stream>>>(s.nv, s.vbody.p, s.xbar.p, q, x,
                                                       pending_only ? s.isl.p : nullptr, s.isl_state.p);
}

void launch_transform_dq(Scene& s, const double* dq) {
  counted(s);
  k_transform_dq<<<blocks(s.nv, 256), 256, 0, s.stream>>>(s.nv, s.vbody.p, s.xbar.p, dq, s.x.p, s.dx.p, s.x1.p);
}

void launch_body_boxes(Scene& s, bool swept) {
  counted(s);
  k_body_boxes<<<blocks(32L * s.nb, 256), 256, 0, s.stream>>>(s.nb, s.vbeg.p, s.x.p, swept ? s.x1.p : nullptr,
                                                               s.bbox.p, s.bbox32.p);
}

void launch_scan(Scene& s, const int* cnt, int* off, const int* n_dev, int* total_dev, long cap, unsigned flag_bit,
                 unsigned long long* need) {
  counted(s);
  k_scan<<<1, 1024, 0, s.stream>>>(cnt, off, n_dev, n_dev ? 0 : s.nb, total_dev, cap, flag_bit, need, s.st);
}

// d-hat for the FP32 box prefilter: rounded up, with a relative margin
float dh32(const Scene& s) { return nextafterf((float)(s.prm.dhat * (1.0 + 1e-6)), INFINITY); }

void launch_body_pairs(Scene& s) {
  const double inv_h = 1.0 / s.cell_h;
  const unsigned mask = (unsigned)s.hash_T - 1u;
  const int nbk = blocks(s.nb, 128);
  counted(s, 2);
  ProfScope pr(s, PF_ROWS);
  k_hash_count<<<nbk, 128, 0, s.stream>>>(s.nb, s.bbox.p, s.prm.dhat, inv_h, s.hcount.p, s.large.p);
  launch_scan(s, s.large.p, s.large_pos.p, nullptr, &s.st->nlarge, (long)s.nb, 0, &s.st->need_misc);
  k_large_list<<<nbk, 128, 0, s.stream>>>(s.nb, s.large.p, s.large_pos.p, s.large_list.p);
  // rows of the large bodies (direct scan over all bodies, no hash) beside
  // the hash build and the hashed rows; both write disjoint rows
  counted(s);
  on_side(s, 1, 4, [&]() {
    k_rows_large<<<64, 1024, 0, s.stream>>>(s.nb, s.is_static.p, s.bbox.p, s.bbox32.p, dh32(s), s.prm.dhat,
                                            s.large_list.p, s.fpairs.p, s.st, s.maxn, s.nbr.p, s.ncount.p, s.st);
  });
  launch_scan(s, s.hcount.p, s.hoff.p, nullptr, &s.st->nent, (long)s.entries.cap, ST_CAP_HASH, &s.st->need_misc);
  cudaMemsetAsync(s.slot_cnt.p, 0, sizeof(int) * s.hash_T, s.stream);
  k_hash_slots<<<nbk, 128, 0, s.stream>>>(s.nb, s.bbox.p, s.large.p, s.prm.dhat, inv_h, mask, s.slot_cnt.p,
                                          s.slot_off.p, s.entries.p, (long)s.entries.cap, false);
  counted(s, 4);
  {
    const int tiles = (s.hash_T + kScanTile - 1) / kScanTile;
    k_scan_tiles<<<tiles, 1024, 0, s.stream>>>(s.slot_cnt.p, s.hash_T, s.scan_part.p);
    k_scan_apply<<<tiles, 1024, 0, s.stream>>>(s.slot_cnt.p, s.slot_off.p, s.hash_T, s.scan_part.p, &s.st->pad2[0],
                                               (long)s.entries.cap, ST_CAP_HASH, &s.st->need_misc, s.st);
  }
  cudaMemsetAsync(s.slot_cnt.p, 0, sizeof(int) * s.hash_T, s.stream);
  k_hash_slots<<<nbk, 128, 0, s.stream>>>(s.nb, s.bbox.p, s.large.p, s.prm.dhat, inv_h, mask, s.slot_cnt.p,
                                          s.slot_off.p, s.entries.p, (long)s.entries.cap, true);
  counted(s, 2);
  k_rows<<<blocks(32L * s.nb, 256), 256, 0, s.stream>>>(s.nb, s.is_static.p, s.bbox.p, s.bbox32.p, dh32(s),
                                                        s.prm.dhat, inv_h, mask,
                                                        s.large.p, s.large_list.p, s.slot_off.p, s.entries.p,
                                                        s.fpairs.p, s.st, s.maxn, s.nbr.p, s.ncount.p, s.st);
  join_side(s, 1, 4);
  launch_scan(s, s.ncount.p, s.rowoff.p, nullptr, &s.st->np, (long)s.P.cap, ST_CAP_PAIRS, &s.st->need_pairs);
  k_rows_compact<<<blocks(32L * s.nb, 256), 256, 0, s.stream>>>(s.nb, s.nbr.p, s.ncount.p, s.rowoff.p, s.maxn, s.P.p,
                                                                (long)s.P.cap);
}

void launch_incoming(Scene& s) {
  cudaMemsetAsync(s.in_cnt.p, 0, sizeof(int) * s.nb, s.stream);
  counted(s);
  k_in_count<<<sm_grid(s, 4), 256, 0, s.stream>>>(s.st, s.P.p, s.in_cnt.p);
  counted(s);
  k_scan<<<1, 1024, 0, s.stream>>>(s.in_cnt.p, s.in_off.p, nullptr, s.nb, &s.st->pad, (long)s.P.cap, 0,
                                   &s.st->need_misc, s.st);
  cudaMemsetAsync(s.in_cnt.p, 0, sizeof(int) * s.nb, s.stream);
  counted(s);
  k_in_fill<<<sm_grid(s, 4), 256, 0, s.stream>>>(s.st, s.P.p, s.in_off.p, s.in_cnt.p, s.in_list.p);
  counted(s);
  k_in_sort<<<blocks(s.nb, 128), 128, 0, s.stream>>>(s.nb, s.in_off.p, s.in_list.p);
}

void launch_fpairs(Scene& s) {
  counted(s);
  k_flag_active<<<sm_grid(s, 4), 256, 0, s.stream>>>(s.st, s.acount.p, s.flagbuf.p);
  counted(s);
  k_scan<<<1, 1024, 0, s.stream>>>(s.flagbuf.p, s.posbuf.p, &s.st->np, 0, &s.st->nfp, (long)s.fpairs.cap,
                                   ST_CAP_PAIRS, &s.st->need_misc, s.st);
  counted(s);
  k_fpairs<<<sm_grid(s, 4), 256, 0, s.stream>>>(s.st, s.P.p, s.flagbuf.p, s.posbuf.p, s.aoff.p, s.fpairs.p, s.fpoff.p);
}

__global__ void k_negate(long n, const double* in, double* out) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) out[i] = -in[i];
}

void launch_negate(Scene& s, const double* in, double* out, long n) {
  counted(s);
  k_negate<<<blocks(n, 256), 256, 0, s.stream>>>(n, in, out);
}

void launch_assemble(Scene& s) {
  counted(s, 3);
  ProfScope pa(s, PF_ASSEMBLE);
  cudaMemsetAsync(reinterpret_cast<char*>(s.st) + offsetof(DevStatus, n_large_asm), 0, sizeof(int), s.stream);
  k_assemble<<<sm_grid(s, 16), 128, 0, s.stream>>>(s.st, s.P.p, s.aoff.p, s.term.p, s.termv.p, s.fpairs.p, s.fpoff.p,
                                                   s.fterm.p, s.ftermv.p, s.vbody.p, s.xbar.p, s.pblk.p,
                                                   s.large_asm.p, s.st);
  k_assemble_large<<<sm_grid(s, 4), 32 * kAssembleWarps, 0, s.stream>>>(
      s.st, s.P.p, s.aoff.p, s.term.p, s.termv.p, s.fpairs.p, s.fpoff.p, s.fterm.p, s.ftermv.p, s.vbody.p, s.xbar.p,
      s.pblk.p, s.large_asm.p);
}

void launch_body_terms(Scene& s, const double* q, bool hess, bool project, bool pending_only) {
  counted(s);
  ProfScope pb(s, PF_BODY);
  k_body_terms<<<blocks(s.nb, 64), 64, 0, s.stream>>>(s.nb, s.is_static.p, q, s.qtilde.p, s.mass10.p, s.vol.p,
                                                       s.kappa_b.p, s.prm.dt, s.gb.p, s.Eb.p,
                                                       pending_only ? s.isl.p : nullptr, s.isl_state.p);
  if (hess) {
    counted(s, 2);
    cudaMemsetAsync(reinterpret_cast<char*>(s.st) + offsetof(DevStatus, bh_fix), 0, sizeof(int), s.stream);
    k_body_hess<<<blocks(s.nb, kBodyWarp), kBodyWarp, 0, s.stream>>>(s.nb, s.is_static.p, q, s.mass10.p, s.vol.p,
                                                                     s.kappa_b.p, s.prm.dt, project ? 1 : 0, s.Db.p,
                                                                     s.st);
  }
}

void launch_gather(Scene& s) {
  counted(s);
  k_gather<<<blocks(32L * s.nb, 256), 256, 0, s.stream>>>(s.nb, s.is_static.p, s.rowoff.p, s.in_off.p, s.in_list.p,
                                                          s.pblk.p, s.Db.p, s.gb.p, s.D.p, s.g.p, s.st);
}

void launch_precond(Scene& s) {
  counted(s);
  k_precond<<<blocks(s.nb, kBodyWarp), kBodyWarp, 0, s.stream>>>(s.nb, s.is_static.p, s.D.p, s.Pinv.p, s.st);
  launch_cluster_factor(s);
}

// the preconditioner, then the start of the Newton solve H dx = -g
void launch_precond_start(Scene& s, double* xout) {
  launch_precond(s);
  launch_pcg_fp32_blocks(s);
  launch_pcg_init(s, s.g.p, -1.0, xout);
}

// energies of the last evaluation into st->energy: bodies, barrier terms or
// per-body-pair barrier energies (energy-only pass), friction terms
void launch_energy_total(Scene& s, bool from_terms) {
  counted(s, 2);
  const dim3 grid(std::max(1, kEnergyParts / s.grid_div), 4);
  if (from_terms)
    k_energies<<<grid, 256, 0, s.stream>>>(s.Eb.p, s.nb, s.term.p, kTermStride, &s.st->nact, 1, s.fterm.p,
                                           &s.st->nfr, s.red.p);
  else
    k_energies<<<grid, 256, 0, s.stream>>>(s.Eb.p, s.nb, s.Epair.p, 1, &s.st->np, energy_chunks(s), s.fterm.p,
                                           &s.st->nfr, s.red.p);
  k_energy_sum<<<1, 128, 0, s.stream>>>(s.red.p, s.st, from_terms ? 1 : 0);
}

__global__ void k_set_u64(unsigned long long* p, unsigned long long v) { *p = v; }

// adjoint of a step: rhs = dL/dq_next + dL/dqdot_next / dt (dynamic rows)
__global__ void k_adj_rhs(int n, const uint8_t* is_static, const double* gq, const double* gqd, double dt,
                          double* rhs) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) rhs[i] = is_static[i / 12] ? 0.0 : gq[i] + gqd[i] / dt;
}

// adjoint of a step: M lam, then dL/dq_t = M lam - dL/dqdot_next / dt,
// dL/dqdot_t = dt M lam, dL/dkappa_b += -dt^2 lam_b . grad V_b / kappa_b
// with grad V / kappa = 4 nu sum_j (a_i . a_j - delta_ij) a_j at q_next
__global__ void k_adj_out(int nb, const uint8_t* is_static, const double* mass10, const double* vol,
                          const double* q, double dt, const double* lam, double* gq, double* gqd, double* gkappa) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb) return;
  if (is_static[b]) {
    for (int k = 0; k < 12; ++k) gq[12 * b + k] = gqd[12 * b + k] = 0.0;
    return;
  }
  const double* m = mass10 + 10 * b;
  const double W[4][4] = {{m[0], m[1], m[2], m[3]}, {m[1], m[4], m[5], m[6]}, {m[2], m[5], m[7], m[8]},
                          {m[3], m[6], m[8], m[9]}};
  double l[12], Ml[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) l[k] = lam[12 * b + k];
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      double t = 0.0;
#pragma unroll
      for (int v = 0; v < 4; ++v) t += W[u][v] * l[dof(v, c)];
      Ml[dof(u, c)] = t;
    }
  double A[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int c = 0; c < 3; ++c) A[i][c] = q[12 * b + 3 + 3 * i + c];
  double dot = 0.0;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      double gi = 0.0;
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const double Gij = A[i][0] * A[j][0] + A[i][1] * A[j][1] + A[i][2] * A[j][2] - (i == j ? 1.0 : 0.0);
        gi += Gij * A[j][c];
      }
      dot += l[3 + 3 * i + c] * 4.0 * vol[b] * gi;
    }
  gkappa[b] += -dt * dt * dot;
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    const double g_v = gqd[12 * b + k];
    gq[12 * b + k] = Ml[k] - g_v / dt;
    gqd[12 * b + k] = dt * Ml[k];
  }
}

void launch_adjoint_rhs(Scene& s, const double* gq, const double* gqd, double* rhs) {
  counted(s);
  k_adj_rhs<<<blocks(12L * s.nb, 256), 256, 0, s.stream>>>(12 * s.nb, s.is_static.p, gq, gqd, s.prm.dt, rhs);
}

void launch_adjoint_out(Scene& s, const double* q, const double* lam, double* gq, double* gqd, double* gkappa) {
  counted(s);
  k_adj_out<<<blocks(s.nb, 128), 128, 0, s.stream>>>(s.nb, s.is_static.p, s.mass10.p, s.vol.p, q, s.prm.dt, lam, gq,
                                                     gqd, gkappa);
}

// the CCD minimum starts at 1 (a whole step)
void launch_reset_toi(Scene& s) {
  counted(s);
  k_set_u64<<<1, 1, 0, s.stream>>>(&s.st->toi_bits, 0x3FF0000000000000ull);
}

void launch_max_step(Scene& s) {
  counted(s);
  k_max_step<<<blocks(s.nv, 256), 256, 0, s.stream>>>(s.nv, s.vbody.p, s.is_static.p, s.dx.p, s.st);
}

void launch_trial(Scene& s, double alpha, bool alpha_from_ccd) {
  counted(s);
  k_trial<<<blocks(12L * s.nb, 256), 256, 0, s.stream>>>(12 * s.nb, s.q.p, s.dq.p, alpha,
                                                          alpha_from_ccd ? s.st : nullptr, s.qtrial.p);
}

void launch_finish_step(Scene& s) {
  counted(s);
  k_finish<<<blocks(s.nb, 128), 128, 0, s.stream>>>(s.nb, s.is_static.p, s.q.p, s.prm.dt, s.qt.p, s.qdot.p);
  launch_predictor(s);
}

}  // namespace abd
