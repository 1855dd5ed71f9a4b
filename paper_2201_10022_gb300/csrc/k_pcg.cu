// Block-Jacobi preconditioned conjugate gradients on the Newton system
// H dq = rhs (the linear solve of each Newton iteration; the paper's direct
// LLT of Sec. 5 replaced by an iterative solve on the device).
//
// H is symmetric block-sparse with 12x12 blocks: the diagonal blocks D_b,
// and for every body pair (a, b), a < b, the upper block H_ab stored once
// (rows = DOFs of a).  Row b of the product is
//   y_b = D_b v_b + sum_{(b,c) upper} H_bc v_c + sum_{(c,b) incoming} H_cb^T v_c
// The preconditioner is the explicit inverse of each diagonal block.
//
// One persistent cooperative kernel runs the whole solve: every iteration is
// two phases separated by a grid barrier, and every block derives the
// scalars (alpha, beta, the convergence test) from the same per-body partial
// sums in the same order, so no host round trip is needed, the result is
// bit-identical run to run and independent of the grid size.  The grid
// barrier's wait is bounded: a block that waits longer than kBarrierTimeout
// cycles raises an abort word that releases every other block, and the solve
// reports the failure in the status word.
//
// Two precisions (the paper states none for its solve):
//  * FP64: blocks, vectors and products in FP64;
//  * mixed: the blocks and the preconditioner stored in FP32 and the inner
//    iterations in FP32 (FP32 blocks and vectors, FP64 dot products), inside
//    an FP64 iterative refinement: x (FP64) += the inner solution of
//    H32 d = r, then r = rhs - H32 x recomputed in FP64 arithmetic, until the
//    FP64 residual meets the tolerance.  The gradient, and so the Newton
//    minimiser, stay FP64; only the direction's solve uses the FP32 blocks.
//
// Layout of a block product: a warp takes one body row; lanes 0..11 and
// 16..27 are two groups of 12, one row DOF per lane, taking the row's blocks
// alternately.  Lane l of a group forms y_l = sum_i B(l, i) v_i (a block as
// stored: 12 consecutive entries) or sum_i B(i, l) v_i (transposed: the group
// reads 12 consecutive entries per i), with v_i broadcast by shuffles, so no
// cross-lane reduction of products is needed; the two groups' sums are added
// at the end of the row.
#include <stddef.h>

#include <algorithm>

#include "abd_internal.cuh"

namespace abd {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kThreads = 256;       // threads per block of the solve kernel
constexpr int kWarps = kThreads / 32;
constexpr long long kBarrierTimeout = 4000000000LL;  // cycles (about 2 s at 2 GHz)
constexpr int kRefineMax = 8;       // FP64 refinement rounds of the mixed solve
constexpr double kInnerTolMin = 1e-5;  // smallest relative reduction asked of one FP32 inner solve

struct PcgArgs {
  int nb, max_iter, mixed;
  double tol2;                      // squared relative residual tolerance
  const int* np;                    // body pairs in the list (device count; clamps the rows)
  const uint8_t* __restrict__ is_static;
  const double* __restrict__ D;     // nb x 144 diagonal blocks, row-major (FP64)
  const double* __restrict__ Minv;  // nb x 144 inverse diagonal blocks (FP64)
  const double* __restrict__ pblk;  // per pair kBlkStride doubles, H_ab first (FP64)
  const float* __restrict__ D32;    // mixed: the same blocks in FP32, pairs 144 apart
  const float* __restrict__ Minv32;
  const float* __restrict__ H32;
  const int* __restrict__ rowoff;   // nb + 1: upper pairs of each row in P
  const int* __restrict__ in_off;   // nb + 1: incoming pairs of each row
  const int* __restrict__ in_list;
  const int2* __restrict__ P;
  const double* rhs;                // mixed: the right-hand side (FP64)
  double* x;                        // the solution (FP64)
  // FP64 solve: residual, preconditioned residual, two alternating
  // directions, H p; mixed: the same five in FP32 (..f), r being the FP64
  // refinement residual
  double* r;
  double* z;
  double* p0;
  double* p1;
  double* Ap;
  float* rf;
  float* zf;
  float* p0f;
  float* p1f;
  float* Apf;
  float* xf;                        // mixed: the inner solution
  double* cpart;                    // 4 x nb per-body partials: p.Ap, r.z, r.r, FP64 r.r
  unsigned* bar;                    // grid barrier: arrivals, generation, abort
  DevStatus* st;
  // preconditioner clusters: members, bounds, factor offsets, factors, flags
  const int* nclu;
  const int* __restrict__ c_perm;
  const int* __restrict__ c_off;
  const long long* __restrict__ c_foff;
  const double* __restrict__ c_fac;
  const int* __restrict__ c_ok;
};

// ---- grid barrier ------------------------------------------------------------
__device__ __forceinline__ unsigned ld_volatile(const unsigned* p) { return *(volatile const unsigned*)p; }

// all blocks of the (co-resident, cooperatively launched) grid meet here;
// false on abort (a block timed out, or another block raised the abort word)
__device__ bool grid_barrier(unsigned* bar, unsigned& gen) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    const unsigned target = gen + 1;
    __threadfence();
    if (atomicAdd(&bar[0], 1u) == gridDim.x - 1) {
      atomicExch(&bar[0], 0u);
      __threadfence();
      atomicExch(&bar[1], target);
    } else {
      const long long t0 = clock64();
      while (ld_volatile(&bar[1]) != target) {
        if (ld_volatile(&bar[2])) {
          ok = 0;
          break;
        }
        if (clock64() - t0 > kBarrierTimeout) {
          atomicExch(&bar[2], 1u);
          ok = 0;
          break;
        }
        __nanosleep(32);
      }
    }
    if (ld_volatile(&bar[2])) ok = 0;
    __threadfence();
    gen = target;
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// ---- fixed-order sums --------------------------------------------------------
// sum over lanes 0..11 of v (fixed tree); valid in lane 0
__device__ __forceinline__ double sum12(double v) {
  const int lane = threadIdx.x & 31;
  double t = lane < 12 ? v : 0.0;
  t += __shfl_down_sync(kFull, t, 8);
  t += __shfl_down_sync(kFull, t, 4);
  t += __shfl_down_sync(kFull, t, 2);
  t += __shfl_down_sync(kFull, t, 1);
  return t;
}

// totals of K per-body partial arrays (stride n), by every thread of the
// block in an order that depends only on n: thread t adds entries t,
// t + kThreads, ...; a fixed butterfly in each warp; the warps in order
template <int K>
__device__ void block_totals(const double* part, int n, double* out) {
  __shared__ double s_red[4][kWarps];
  const int t = threadIdx.x;
  double acc[K];
#pragma unroll
  for (int k = 0; k < K; ++k) acc[k] = 0.0;
#pragma unroll 4
  for (int i = t; i < n; i += kThreads)
#pragma unroll
    for (int k = 0; k < K; ++k) acc[k] += part[(size_t)k * n + i];
#pragma unroll
  for (int k = 0; k < K; ++k) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc[k] += __shfl_xor_sync(kFull, acc[k], o);
    if ((t & 31) == 0) s_red[k][t >> 5] = acc[k];
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < K; ++k) {
    double v = 0.0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) v += s_red[k][w];
    out[k] = v;
  }
  __syncthreads();
}

// ---- one body row of a block product ----------------------------------------
// The row's blocks: the diagonal (index 0), the upper pairs, the incoming
// pairs (transposed).  Group g = lane / 16 takes blocks g, g + 2, ...; lane
// l = lane % 16 < 12 holds row DOF l.  For block j with column body c the
// column values v_i = vcol(c, i) are produced by lane i of the group and
// broadcast.  Returns y_l in lanes 0..11 (both groups' sums added).
template <typename TB, typename TA, typename VF>
__device__ __forceinline__ TA row_product(int b, int np, const PcgArgs& a, const TB* __restrict__ Dblk,
                                          const TB* __restrict__ Hblk, long hstride, bool diag_only, VF vcol) {
  const int lane = threadIdx.x & 31;
  const int g = lane >> 4, l = lane & 15;
  const int up0 = a.rowoff[b], nup = diag_only ? 0 : max(0, min(a.rowoff[b + 1], np) - up0);
  const int in0 = a.in_off[b], nin = diag_only ? 0 : a.in_off[b + 1] - in0;
  const int nblk = 1 + nup + nin;
  TA y = TA(0);
  for (int j0 = 0; j0 < nblk; j0 += 2) {
    const int j = j0 + g;
    // the block, its column body and orientation (uniform within a group)
    int c = b;
    bool trans = false;
    const TB* B = Dblk + (size_t)144 * b;
    if (j >= 1 && j < nblk) {
      int p;
      if (j - 1 < nup) {
        p = up0 + j - 1;
        c = a.P[p].y;
      } else {
        p = a.in_list[in0 + j - 1 - nup];
        c = a.P[p].x;
        trans = true;
      }
      B = Hblk + (size_t)p * hstride;
    }
    const bool live = j < nblk && !a.is_static[c];
    const TA vi = (live && l < 12) ? vcol(c, l) : TA(0);
    // every lane of the warp takes part in the shuffles (both groups)
    TA acc = TA(0);
#pragma unroll
    for (int i = 0; i < 12; ++i) {
      const TA v = __shfl_sync(kFull, vi, (g << 4) + i);
      if (live && l < 12) {
        const TB h = trans ? __ldg(B + 12 * i + l) : __ldg(B + 12 * l + i);
        acc = fma((TA)h, v, acc);
      }
    }
    y += acc;
  }
  y += __shfl_down_sync(kFull, y, 16);
  return y;
}

// ---- the phases ---------------------------------------------------------------
// Phase A of iteration k: p_k = z_k + beta p_{k-1} (formed on the fly for the
// row and every column it reads; p_0 = z_0 is given), Ap = H p_k, and the
// per-body partials of p_k . Ap.  Warp w of the grid takes rows w, w + W, ...
template <typename T>
__device__ void phase_spmv(const PcgArgs& a, int k, T beta, const T* __restrict__ Dblk,
                           const T* __restrict__ Hblk, long hstride, const T* z, T* p0, T* p1, T* Ap,
                           double* part) {
  const int lane = threadIdx.x & 31;
  const int wgrid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  const int np = *a.np;
  const T* pold = (k & 1) ? p0 : p1;  // p_{k-1}
  T* pnew = (k & 1) ? p1 : p0;        // p_k
  const bool fly = k > 0;
  for (int b = wgrid; b < a.nb; b += nw) {
    if (a.is_static[b]) {
      if (lane < 12) {
        Ap[12 * b + lane] = T(0);
        pnew[12 * b + lane] = T(0);
      }
      if (lane == 0) part[b] = 0.0;
      continue;
    }
    auto vcol = [&](int c, int i) -> T {
      return fly ? fma(beta, pold[12 * c + i], z[12 * c + i]) : pnew[12 * c + i];
    };
    const T y = row_product<T, T>(b, np, a, Dblk, Hblk, hstride, false, vcol);
    T pb = T(0);
    if (lane < 12) {
      pb = vcol(b, lane);
      Ap[12 * b + lane] = y;
    }
    // p_k of this row is written after the row's reads (other rows read only
    // p_{k-1} and z, never p_k, in this phase)
    __syncwarp();
    if (lane < 12 && fly) pnew[12 * b + lane] = pb;
    const double t = sum12((double)pb * (double)y);
    if (lane == 0) part[b] = t;
  }
}

// z = (L L^T)^-1 r over the N = 12 n DOFs of a cluster of n >= 2 bodies, L
// its Cholesky factor (packed lower rows: entry (i, j), j <= i, at
// i (i + 1) / 2 + j, reciprocal pivots on the diagonal); one warp, r and z in
// the rows of the members; ybuf: N doubles of the warp's shared memory.
// Forward substitution row by row (lane sums in a fixed order), back
// substitution column by column.  Row i of L is held in registers (lane l
// holds entries l, l + 32, ... below the diagonal: kRowChunks per lane for
// N <= 192; the diagonal entry in every lane), and the next row's loads are
// issued before the current row's dependent chain, so each step waits on
// shuffles and shared memory, not on a load from L2.
__device__ __forceinline__ long ptri(int i, int j) { return (long)i * (i + 1) / 2 + j; }

constexpr int kRowChunks = (12 * kClusterMax + 31) / 32;

// entries 0..len-1 of a packed row into lane-strided registers (zero beyond)
__device__ __forceinline__ void load_row(const double* Li, int len, int lane, double (&v)[kRowChunks]) {
#pragma unroll
  for (int q = 0; q < kRowChunks; ++q) {
    const int j = lane + 32 * q;
    v[q] = j < len ? Li[j] : 0.0;
  }
}

template <typename T>
__device__ void cluster_solve(const PcgArgs& a, int c, const T* r, T* z, double* ybuf) {
  const int lane = threadIdx.x & 31;
  const int m0 = a.c_off[c], n = a.c_off[c + 1] - m0, N = 12 * n;
  const double* L = a.c_fac + a.c_foff[c];
  for (int i = lane; i < N; i += 32) ybuf[i] = (double)r[12 * a.c_perm[m0 + i / 12] + i % 12];
  __syncwarp();
  // the row (off-diagonal entries) and its diagonal entry (the reciprocal
  // pivot, loaded by every lane) of the current and the next step
  double cur[kRowChunks], nxt[kRowChunks];
  double dcur = L[0], dnxt = 0.0;
  load_row(L, 0, lane, cur);
  for (int i = 0; i < N; ++i) {
    if (i + 1 < N) {
      load_row(L + ptri(i + 1, 0), i + 1, lane, nxt);
      dnxt = L[ptri(i + 1, i + 1)];
    }
    double t = 0.0;
#pragma unroll
    for (int q = 0; q < kRowChunks; ++q) {
      const int j = lane + 32 * q;
      if (j < i) t = fma(cur[q], ybuf[j], t);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(kFull, t, o);
    if (lane == 0) ybuf[i] = (ybuf[i] - t) * dcur;
    __syncwarp();
#pragma unroll
    for (int q = 0; q < kRowChunks; ++q) cur[q] = nxt[q];
    dcur = dnxt;
  }
  load_row(L + ptri(N - 1, 0), N - 1, lane, cur);
  dcur = L[ptri(N - 1, N - 1)];
  for (int i = N - 1; i >= 0; --i) {
    if (i > 0) {
      load_row(L + ptri(i - 1, 0), i - 1, lane, nxt);
      dnxt = L[ptri(i - 1, i - 1)];
    }
    const double zi = ybuf[i] * dcur;
    __syncwarp();
#pragma unroll
    for (int q = 0; q < kRowChunks; ++q) {
      const int j = lane + 32 * q;
      if (j < i) ybuf[j] = fma(-cur[q], zi, ybuf[j]);
    }
    if (lane == 0) ybuf[i] = zi;
    __syncwarp();
#pragma unroll
    for (int q = 0; q < kRowChunks; ++q) cur[q] = nxt[q];
    dcur = dnxt;
  }
  for (int i = lane; i < N; i += 32) z[12 * a.c_perm[m0 + i / 12] + i % 12] = (T)ybuf[i];
  __syncwarp();
}

// z = M^-1 r for the members of cluster c (r already in place): a singleton
// (or a cluster whose factorisation failed) by the inverse diagonal blocks,
// a larger cluster by its factor; then the members' partials of r.z and r.r
template <typename T>
__device__ void cluster_precond(const PcgArgs& a, int c, const T* __restrict__ Minv, const T* r, T* z,
                                double* part_rz, double* part_rr, double* ybuf) {
  const int lane = threadIdx.x & 31;
  const int m0 = a.c_off[c], n = a.c_off[c + 1] - m0;
  if (n >= 2 && a.c_ok[c]) {
    cluster_solve<T>(a, c, r, z, ybuf);
  } else {
    for (int i = 0; i < n; ++i) {
      const int b = a.c_perm[m0 + i];
      const T rb = lane < 12 ? r[12 * b + lane] : T(0);
      auto vcol = [&](int, int) -> T { return rb; };
      const T zb = row_product<T, T>(b, 0, a, Minv, Minv, 0, true, vcol);
      if (lane < 12) z[12 * b + lane] = zb;
    }
    __syncwarp();
  }
  for (int i = 0; i < n; ++i) {
    const int b = a.c_perm[m0 + i];
    const T rb = lane < 12 ? r[12 * b + lane] : T(0);
    const T zb = lane < 12 ? z[12 * b + lane] : T(0);
    const double rz = sum12((double)rb * (double)zb), rr = sum12((double)rb * (double)rb);
    if (lane == 0) {
      part_rz[b] = rz;
      part_rr[b] = rr;
    }
  }
}

// Phase B of iteration k: x += alpha p_k, r -= alpha Ap, z = M^-1 r, and the
// per-body partials of r.z (part[0..nb)) and r.r (part[nb..2nb)); warps take
// clusters (static bodies are in none; their partials stay zero)
template <typename T>
__device__ void phase_update(const PcgArgs& a, int k, T alpha, const T* __restrict__ Minv, T* x, T* r, T* z,
                             const T* p0, const T* p1, const T* Ap, double* part, double* ybuf) {
  const int lane = threadIdx.x & 31;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  const T* pk = (k & 1) ? p1 : p0;
  const int nclu = *a.nclu;
  // block-first order: consecutive clusters (listed largest first) go to
  // different blocks, hence different SMs
  for (int c = (threadIdx.x >> 5) * gridDim.x + blockIdx.x; c < nclu; c += nw) {
    const int m0 = a.c_off[c], n = a.c_off[c + 1] - m0;
    for (int i = 0; i < n; ++i) {
      const int b = a.c_perm[m0 + i];
      if (lane < 12) {
        const int q = 12 * b + lane;
        x[q] = fma(alpha, pk[q], x[q]);
        r[q] = fma(-alpha, Ap[q], r[q]);
      }
    }
    __syncwarp();
    cluster_precond<T>(a, c, Minv, r, z, part, part + a.nb, ybuf);
  }
}

// start of a solve: r = sign rhs (as T), x = 0, z = M^-1 r, p0 = z, and the
// per-body r.z (part[nb..2nb)) and r.r (part[2nb..3nb)); static bodies' rows
// and partials zero
template <typename T, typename TR>
__device__ void phase_start(const PcgArgs& a, const TR* rhs, double sign, const T* __restrict__ Minv, T* x, T* r,
                            T* z, T* p0, double* part, double* ybuf) {
  const int lane = threadIdx.x & 31;
  const int wgrid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int b = wgrid; b < a.nb; b += nw) {
    if (!a.is_static[b]) continue;
    if (lane < 12) {
      const int i = 12 * b + lane;
      r[i] = x[i] = z[i] = p0[i] = T(0);
    }
    if (lane == 0) part[a.nb + b] = part[2 * a.nb + b] = 0.0;
  }
  const int nclu = *a.nclu;
  // block-first order: consecutive clusters (listed largest first) go to
  // different blocks, hence different SMs
  for (int c = (threadIdx.x >> 5) * gridDim.x + blockIdx.x; c < nclu; c += nw) {
    const int m0 = a.c_off[c], n = a.c_off[c + 1] - m0;
    for (int i = 0; i < n; ++i) {
      const int b = a.c_perm[m0 + i];
      if (lane < 12) {
        const int q = 12 * b + lane;
        r[q] = (T)(sign * (double)rhs[q]);
        x[q] = T(0);
      }
    }
    __syncwarp();
    cluster_precond<T>(a, c, Minv, r, z, part + a.nb, part + 2 * a.nb, ybuf);
    for (int i = 0; i < n; ++i) {
      const int b = a.c_perm[m0 + i];
      if (lane < 12) p0[12 * b + lane] = z[12 * b + lane];
    }
  }
}

// iterations of one PCG solve from the state phase_start left; stops when
// r.r <= tol2 r.r_0 or after max_iter.  state: 1 converged, 0 cap,
// 2 breakdown, 3 barrier timeout.  Returns the iterations.
template <typename T>
__device__ int pcg_loop(const PcgArgs& a, double tol2, int max_iter, const T* Dblk, const T* Hblk, long hstride,
                        const T* Minv, T* x, T* r, T* z, T* p0, T* p1, T* Ap, double* part, double* ybuf,
                        unsigned& gen, int& state, double& rz_out, double& rr_out, double& rr0_out) {
  double tot[2];
  block_totals<2>(part + a.nb, a.nb, tot);
  double rz = tot[0], rr = tot[1], rz_prev = 0.0;
  const double rr0 = rr;
  int k = 0;
  state = rr0 == 0.0 ? 1 : 0;
  // Hazards: phase_spmv of iteration k+1 overwrites the p.Ap partials and
  // phase_update of k+1 the r.z / r.r partials; every block has finished
  // reading them before the barrier that precedes each of those phases.
  while (state == 0 && k < max_iter) {
    phase_spmv<T>(a, k, (T)(k > 0 ? rz / rz_prev : 0.0), Dblk, Hblk, hstride, z, p0, p1, Ap, part);
    if (!grid_barrier(a.bar, gen)) {
      state = 3;
      break;
    }
    block_totals<1>(part, a.nb, tot);
    const double pap = tot[0];
    if (!(pap > 0.0)) {
      state = 2;
      break;
    }
    phase_update<T>(a, k, (T)(rz / pap), Minv, x, r, z, p0, p1, Ap, part + a.nb, ybuf);
    if (!grid_barrier(a.bar, gen)) {
      state = 3;
      break;
    }
    block_totals<2>(part + a.nb, a.nb, tot);
    rz_prev = rz;
    rz = tot[0];
    rr = tot[1];
    ++k;
    if (rr <= tol2 * rr0) state = 1;
  }
  rz_out = rz;
  rr_out = rr;
  rr0_out = rr0;
  return k;
}

// FP64 refinement residual of the mixed solve: r = rhs - H32 x (FP64
// arithmetic on the FP32-stored blocks), per-body partials of r.r in part
__device__ void phase_residual64(const PcgArgs& a, double* part) {
  const int lane = threadIdx.x & 31;
  const int wgrid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  const int np = *a.np;
  for (int b = wgrid; b < a.nb; b += nw) {
    if (a.is_static[b]) {
      if (lane < 12) a.r[12 * b + lane] = 0.0;
      if (lane == 0) part[b] = 0.0;
      continue;
    }
    auto vcol = [&](int c, int i) -> double { return a.x[12 * c + i]; };
    const double y = row_product<float, double>(b, np, a, a.D32, a.H32, 144, false, vcol);
    double rb = 0.0;
    if (lane < 12) {
      rb = a.rhs[12 * b + lane] - y;
      a.r[12 * b + lane] = rb;
    }
    const double rr = sum12(rb * rb);
    if (lane == 0) part[b] = rr;
  }
}

// x += (FP64) inner solution
__device__ void phase_accumulate(const PcgArgs& a) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  for (int i = t; i < 12 * a.nb; i += gridDim.x * blockDim.x) a.x[i] += (double)a.xf[i];
}

// The whole solve.  FP64: on entry x, r, z, p0 = z hold the start (x = 0,
// r = rhs, z = Minv r) and part[nb..3nb) the partials of r.z and r.r.  Mixed:
// x = 0, r = rhs (FP64), part[3nb..4nb) the partials of rhs.rhs.  On exit
// st->scal: [0] r.z, [2] r.r, [3] r.r at the start, [6] 1 converged / 0 cap /
// 2 breakdown (p.Ap <= 0) / 3 barrier timeout, [7] iterations (inner
// iterations summed over the refinement rounds when mixed), [8] refinement
// rounds.
__global__ void __launch_bounds__(kThreads, 2) k_pcg_solve(PcgArgs a) {
  __shared__ double s_y[kWarps][12 * kClusterMax];
  double* ybuf = s_y[threadIdx.x >> 5];
  unsigned gen = 0;
  int state = 0, k = 0, rounds = 0;
  double rz = 0.0, rr = 0.0, rr0 = 0.0;
  if (!a.mixed) {
    k = pcg_loop<double>(a, a.tol2, a.max_iter, a.D, a.pblk, kBlkStride, a.Minv, a.x, a.r, a.z, a.p0, a.p1, a.Ap,
                         a.cpart, ybuf, gen, state, rz, rr, rr0);
  } else {
    double tot[1];
    block_totals<1>(a.cpart + 3 * a.nb, a.nb, tot);
    const double bb = tot[0];
    double r64 = bb;  // squared FP64 residual of the current x
    rr0 = bb;
    state = bb == 0.0 ? 1 : 0;
    while (state == 0 && rounds < kRefineMax && k < a.max_iter) {
      // inner FP32 solve of H32 d = r, asked for the reduction that would
      // meet the tolerance (not below what FP32 iterations attain)
      const double want = a.tol2 * bb / r64;
      const double inner = want > kInnerTolMin * kInnerTolMin ? want : kInnerTolMin * kInnerTolMin;
      phase_start<float, double>(a, a.r, 1.0, a.Minv32, a.xf, a.rf, a.zf, a.p0f, a.cpart, ybuf);
      if (!grid_barrier(a.bar, gen)) {
        state = 3;
        break;
      }
      int st_in = 0;
      double rzi, rri, rr0i;
      k += pcg_loop<float>(a, inner, a.max_iter - k, a.D32, a.H32, 144, a.Minv32, a.xf, a.rf, a.zf, a.p0f, a.p1f,
                           a.Apf, a.cpart, ybuf, gen, st_in, rzi, rri, rr0i);
      ++rounds;
      if (st_in == 3 || st_in == 2) {
        state = st_in;
        break;
      }
      phase_accumulate(a);
      if (!grid_barrier(a.bar, gen)) {
        state = 3;
        break;
      }
      phase_residual64(a, a.cpart + 3 * a.nb);
      if (!grid_barrier(a.bar, gen)) {
        state = 3;
        break;
      }
      block_totals<1>(a.cpart + 3 * a.nb, a.nb, tot);
      r64 = tot[0];
      rz = rzi;
      if (r64 <= a.tol2 * bb) state = 1;
    }
    rr = r64;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    a.st->scal[0] = rz;
    a.st->scal[2] = rr;
    a.st->scal[3] = rr0;
    a.st->scal[6] = (double)state;
    a.st->scal[7] = (double)k;
    a.st->scal[8] = (double)rounds;
    if (state == 2 || state == 3) atomicOr(&a.st->flags, ST_PCG_BREAKDOWN);
  }
}

// start of a solve from rhs (times sign): FP64 as phase_start; mixed: x = 0,
// r = sign rhs (FP64) and the partials of r.r
__global__ void k_pcg_init(PcgArgs a, const double* __restrict__ rhs, double sign) {
  __shared__ double s_y[kWarps][12 * kClusterMax];
  if (!a.mixed) {
    phase_start<double, double>(a, rhs, sign, a.Minv, a.x, a.r, a.z, a.p0, a.cpart, s_y[threadIdx.x >> 5]);
    return;
  }
  const int lane = threadIdx.x & 31;
  const int wgrid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int b = wgrid; b < a.nb; b += nw) {
    const bool st = a.is_static[b];
    double rb = 0.0;
    if (lane < 12) {
      const int i = 12 * b + lane;
      rb = st ? 0.0 : sign * rhs[i];
      a.r[i] = rb;
      a.x[i] = 0.0;
    }
    const double rr = sum12(rb * rb);
    if (lane == 0) a.cpart[3 * a.nb + b] = rr;
  }
}

// mixed: the rhs of the solve (FP64, kept for the refinement residual)
__global__ void k_pcg_rhs_copy(int n, const double* rhs, double sign, double* out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) out[i] = sign * rhs[i];
}

// mixed: FP32 copies of the diagonal blocks, the inverse diagonal blocks and
// the upper pair blocks (packed 144 apart)
__global__ void k_blocks_to_fp32(int nb, const DevStatus* cst, const double* D, const double* Minv,
                                 const double* pblk, float* D32, float* Minv32, float* H32) {
  const long nd = 144L * nb, nh = 144L * cst->np;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < 2 * nd + nh; i += (long)gridDim.x * blockDim.x) {
    if (i < nd) {
      D32[i] = (float)D[i];
    } else if (i < 2 * nd) {
      Minv32[i - nd] = (float)Minv[i - nd];
    } else {
      const long j = i - 2 * nd, p = j / 144;
      H32[j] = (float)pblk[p * kBlkStride + (j - 144 * p)];
    }
  }
}

// Cholesky factors of the preconditioner clusters of two or more bodies:
// one block per cluster builds the lower triangle of the cluster's dense
// matrix in shared memory (packed rows; the members' diagonal blocks and the
// upper blocks of the body pairs inside the cluster, placed below the
// diagonal by the members' local order), factors it (right-looking, the
// reciprocal pivots stored on the diagonal) and writes it to its slot.  The
// cluster matrix is a principal submatrix of the positive definite Newton
// Hessian, so a failure (a non-positive pivot) is a rounding accident: the
// cluster is flagged and falls back to its members' inverse diagonal blocks.
__global__ void __launch_bounds__(256) k_cluster_factor(const DevStatus* __restrict__ cst, const int* c_perm,
                                                        const int* c_off, const int* c_of, const int* c_loc,
                                                        const long long* c_foff, const double* D, const int* rowoff,
                                                        const int2* P, const double* pblk, double* fac, int* ok,
                                                        DevStatus* st) {
  extern __shared__ double A[];
  __shared__ int s_fail, s_npair;
  __shared__ int s_rows[kClusterMax + 1];
  __shared__ int3 s_pair[kClusterMax * (kClusterMax - 1) / 2];  // (pair, row member, column member)
  // block structure of the factor: bit J of s_mask[I] (J <= I) marks the
  // 12x12 block (I, J) as possibly nonzero (a body pair, or fill); bit I of
  // s_col[K] marks the blocks (I, K) of block column K
  __shared__ unsigned s_mask[kClusterMax], s_col[kClusterMax];
  const int tid = threadIdx.x, nt = blockDim.x;
  const int nclu = cst->n_clusters, np = cst->np;
  for (int c = blockIdx.x; c < nclu; c += gridDim.x) {
    const int m0 = c_off[c], n = c_off[c + 1] - m0;
    if (n < 2) continue;
    const int N = 12 * n;
    const long NT = ptri(N, 0);
    for (long i = tid; i < NT; i += nt) A[i] = 0.0;
    if (tid < n) s_mask[tid] = 1u << tid;
    if (tid == 0) {
      s_fail = 0;
      s_npair = 0;
      // the members' body-pair rows, concatenated
      s_rows[0] = 0;
      for (int i = 0; i < n; ++i) {
        const int b = c_perm[m0 + i];
        s_rows[i + 1] = s_rows[i] + max(0, min(rowoff[b + 1], np) - rowoff[b]);
      }
    }
    __syncthreads();
    for (int t = tid; t < n * 144; t += nt) {
      const int i = t / 144, e = t - 144 * i, r = e / 12, cc = e % 12;
      if (cc <= r) A[ptri(12 * i + r, 12 * i + cc)] = D[144L * c_perm[m0 + i] + e];
    }
    // the body pairs between members: every row of every member tested in
    // parallel (each pair is listed once, in the row of its first body)
    for (int t = tid; t < s_rows[n]; t += nt) {
      int i = 0;
      while (t >= s_rows[i + 1]) ++i;
      const int p = rowoff[c_perm[m0 + i]] + (t - s_rows[i]);
      const int o = P[p].y;
      if (c_of[o] == c) {
        const int j = c_loc[o];
        s_pair[atomicAdd(&s_npair, 1)] = make_int3(p, i, j);
        atomicOr(&s_mask[max(i, j)], 1u << min(i, j));
      }
    }
    __syncthreads();
    // symbolic factorisation: blocks (I, K) and (J, K) of a column K, K < J <=
    // I, fill block (I, J)
    if (tid == 0) {
      for (int K = 0; K < n; ++K) {
        unsigned col = 0;
        for (int I = K; I < n; ++I)
          if ((s_mask[I] >> K) & 1u) col |= 1u << I;
        s_col[K] = col;
        const unsigned below = col & ~((2u << K) - 1u);  // rows I > K
        for (unsigned m = below; m; m &= m - 1) {
          const int I = __ffs(m) - 1;
          s_mask[I] |= below & ((2u << I) - 1u);
        }
      }
    }
    // their blocks H_bo(r, cc) (row of b, column of o), lower triangle
    for (int t = tid; t < 144 * s_npair; t += nt) {
      const int k = t / 144, e = t - 144 * k;
      const int3 q = s_pair[k];
      const int i = q.y, j = q.z;
      const double h = pblk[(size_t)q.x * kBlkStride + e];
      const int r = e / 12, cc = e % 12;
      if (i > j) A[ptri(12 * i + r, 12 * j + cc)] = h;
      else A[ptri(12 * j + cc, 12 * i + r)] = h;
    }
    __syncthreads();
    // right-looking Cholesky by 12-column block columns (a body each).  For
    // every entry the updates come in the order of the columns, as in the
    // column-by-column algorithm, so the factor is the same; entries of blocks
    // outside the symbolic structure stay exactly zero, so their scaling and
    // updates (products with an exact zero) are skipped.
    const int lane = tid & 31, warp = tid >> 5, nwarp = nt >> 5;
    for (int K = 0; K < n; ++K) {
      const unsigned colk = s_col[K];
      const int o = 12 * K;
      // (1) the diagonal block, one warp: pivots (reciprocals stored on the
      // diagonal), column scaling and updates inside the block
      if (warp == 0) {
        for (int cc = 0; cc < 12; ++cc) {
          const int k = o + cc;
          if (lane == 0) {
            double d = A[ptri(k, k)];
            if (!(d > 0.0)) {
              s_fail = 1;
              d = 1.0;
            }
            A[ptri(k, k)] = 1.0 / sqrt(d);
          }
          __syncwarp();
          const double rk = A[ptri(k, k)];
          if (lane > cc && lane < 12) A[ptri(o + lane, k)] *= rk;
          __syncwarp();
          // entries (r, j) of the block with cc < j <= r < 12
          for (int e = lane; e < 144; e += 32) {
            const int r = e / 12, j = e - 12 * r;
            if (j > cc && j <= r) A[ptri(o + r, o + j)] = fma(-A[ptri(o + r, k)], A[ptri(o + j, k)], A[ptri(o + r, o + j)]);
          }
          __syncwarp();
        }
      }
      __syncthreads();
      // (2) the panel below: a thread per row of the column's blocks, its 12
      // entries solved in column order against the diagonal block
      for (int i = o + 12 + tid; i < N; i += nt) {
        if (!((colk >> (i / 12)) & 1u)) continue;
        double* Ai = A + ptri(i, 0);
        for (int cc = 0; cc < 12; ++cc) {
          const int k = o + cc;
          double x = Ai[k];
          const double* Ak = A + ptri(k, 0);
          for (int c2 = 0; c2 < cc; ++c2) x = fma(-Ai[o + c2], Ak[o + c2], x);
          Ai[k] = x * Ak[k];
        }
      }
      __syncthreads();
      // (3) the trailing blocks (I, J), K < J <= I, of the column's blocks: a
      // warp per row, lanes over the row's columns, the 12 updates in column
      // order
      for (int i = o + 12 + warp; i < N; i += nwarp) {
        if (!((colk >> (i / 12)) & 1u)) continue;
        const double* Ai = A + ptri(i, 0);
        double li[12];
#pragma unroll
        for (int cc = 0; cc < 12; ++cc) li[cc] = Ai[o + cc];
        double* Aw = A + ptri(i, 0);
        for (int j = o + 12 + lane; j <= i; j += 32) {
          if (!((colk >> (j / 12)) & 1u)) continue;
          const double* Aj = A + ptri(j, 0) + o;
          double x = Aw[j];
#pragma unroll
          for (int cc = 0; cc < 12; ++cc) x = fma(-li[cc], Aj[cc], x);
          Aw[j] = x;
        }
      }
      __syncthreads();
    }
    double* L = fac + c_foff[c];
    for (long t = tid; t < NT; t += nt) L[t] = A[t];
    if (tid == 0) {
      ok[c] = s_fail ? 0 : 1;
      if (s_fail) atomicAdd(&st->clu_fail, 1);
    }
    __syncthreads();
  }
}

}  // namespace

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static PcgArgs pcg_args(Scene& s, double* xout, int max_iter, double rel_tol) {
  PcgArgs a;
  a.nb = s.nb;
  a.max_iter = max_iter;
  a.mixed = s.pcg_mixed ? 1 : 0;
  a.tol2 = rel_tol * rel_tol;
  a.np = &s.st->np;
  a.is_static = s.is_static.p;
  a.D = s.D.p;
  a.Minv = s.Pinv.p;
  a.pblk = s.pblk.p;
  a.D32 = s.D32.p;
  a.Minv32 = s.Minv32.p;
  a.H32 = s.H32.p;
  a.rowoff = s.rowoff.p;
  a.in_off = s.in_off.p;
  a.in_list = s.in_list.p;
  a.P = s.P.p;
  a.rhs = s.rhs64.p;
  a.x = xout;
  a.r = s.r.p;
  a.z = s.z.p;
  a.p0 = s.pv.p;
  a.p1 = s.pv2.p;
  a.Ap = s.Ap.p;
  a.rf = s.vf.p;
  a.zf = s.vf.p ? s.vf.p + 12L * s.nb : nullptr;
  a.p0f = s.vf.p ? s.vf.p + 24L * s.nb : nullptr;
  a.p1f = s.vf.p ? s.vf.p + 36L * s.nb : nullptr;
  a.Apf = s.vf.p ? s.vf.p + 48L * s.nb : nullptr;
  a.xf = s.vf.p ? s.vf.p + 60L * s.nb : nullptr;
  a.cpart = s.part.p;
  a.bar = s.pcg_bar.p;
  a.st = s.st;
  a.nclu = &s.st->n_clusters;
  a.c_perm = s.c_perm.p;
  a.c_off = s.c_off.p;
  a.c_foff = s.c_foff.p;
  a.c_fac = s.c_fac.p;
  a.c_ok = s.c_ok.p;
  return a;
}

void launch_cluster_factor(Scene& s) {
  static const int kSmem = (12 * kClusterMax) * (12 * kClusterMax + 1) / 2 * (int)sizeof(double);
  if (!s.cluster_attr_set) {
    cudaFuncSetAttribute(k_cluster_factor, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
    s.cluster_attr_set = true;
  }
  counted(s);
  k_cluster_factor<<<sm_grid(s, 1), 256, kSmem, s.stream>>>(s.st, s.c_perm.p, s.c_off.p, s.c_of.p, s.c_loc.p,
                                                           s.c_foff.p, s.D.p, s.rowoff.p, s.P.p, s.pblk.p,
                                                           s.c_fac.p, s.c_ok.p, s.st);
}

// co-resident blocks of the solve kernel on this device (set once per scene)
static int pcg_grid(Scene& s) {
  if (s.pcg_blocks_per_sm <= 0) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pcg_solve, kThreads, 0) != cudaSuccess ||
        per_sm < 1) {
      cudaGetLastError();
      per_sm = 1;
    }
    s.pcg_blocks_per_sm = std::min(per_sm, 2);
  }
  // enough warps for the rows, at most one wave of co-resident blocks
  const int want = (s.nb + kWarps - 1) / kWarps;  // one warp per row or cluster
  const int cap = std::max(1, s.pcg_blocks_per_sm * s.num_sms / s.grid_div);
  return std::max(1, std::min(want, cap));
}

// mixed precision: FP32 copies of the assembled blocks (after the
// preconditioner's inverse blocks exist)
void launch_pcg_fp32_blocks(Scene& s) {
  if (!s.pcg_mixed) return;
  counted(s);
  k_blocks_to_fp32<<<sm_grid(s, 8), 256, 0, s.stream>>>(s.nb, s.st, s.D.p, s.Pinv.p, s.pblk.p, s.D32.p, s.Minv32.p,
                                                        s.H32.p);
}

void launch_pcg_init(Scene& s, const double* rhs, double sign, double* xout) {
  PcgArgs a = pcg_args(s, xout, 0, 0.0);
  if (a.mixed) {
    counted(s);
    k_pcg_rhs_copy<<<sm_grid(s, 4), 256, 0, s.stream>>>(12 * s.nb, rhs, sign, s.rhs64.p);
  }
  counted(s);
  const int grid = std::max(1, std::min((s.nb + kWarps - 1) / kWarps, 4 * s.num_sms));
  k_pcg_init<<<grid, kThreads, 0, s.stream>>>(a, rhs, sign);
}

// the solve from the state k_pcg_init left; enqueued only (the result is in
// the status word)
void launch_pcg_solve(Scene& s, double* xout, int max_iter, double rel_tol) {
  PcgArgs a = pcg_args(s, xout, max_iter, rel_tol);
  counted(s);
  cudaMemsetAsync(s.pcg_bar.p, 0, 4 * sizeof(unsigned), s.stream);
  const int grid = pcg_grid(s);
  ProfScope ps(s, PF_SPMV);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s.stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, k_pcg_solve, a);
}

// algorithmic bytes and operations of one (inner) iteration: every stored
// block once (diagonal, upper off-diagonal, inverse diagonal), the vectors
// p, z, Ap, x, r read or written once each, the pair list once; 8-byte
// entries in FP64, 4-byte in the mixed solve's inner iterations
double pcg_iter_bytes(const Scene& s, long np) {
  const double e = s.pcg_mixed ? 4.0 : 8.0;
  // the preconditioner's factors (packed lower triangles) or inverse blocks
  double pre = 0.0;
  const int* off = s.clu_host + s.nb;
  for (int c = 0; c < s.nclu; ++c) {
    const double n = off[c + 1] - off[c];
    pre += n >= 2 ? 8.0 * (12.0 * n) * (12.0 * n + 1.0) / 2.0 : e * 144.0 * n;
  }
  return e * 144.0 * (s.nb + (double)np) + pre + e * 12.0 * 8.0 * s.nb + 8.0 * np;
}
double pcg_iter_flops(const Scene& s, long np) {
  // block products: the diagonal once and each off-diagonal block twice (as
  // stored and transposed), 2 flops per entry; the preconditioner: a single
  // body's inverse block (2 x 144), a cluster's two triangular solves
  // (2 x N^2, N = 12 n); vector updates
  double pre = 0.0;
  const int* off = s.clu_host + s.nb;
  for (int c = 0; c < s.nclu; ++c) {
    const double n = off[c + 1] - off[c];
    pre += n >= 2 ? 2.0 * (12.0 * n) * (12.0 * n) : 2.0 * 144.0 * n;
  }
  return 2.0 * 144.0 * (s.nb + 2.0 * (double)np) + pre + 2.0 * 12.0 * 6.0 * s.nb;
}

// status of the last solve: iterations (>= 0) if converged, -1 at the cap,
// -2 on breakdown or barrier timeout; *rel_res the relative residual
int pcg_result(Scene& s, double* rel_res) {
  const double rr = s.st_host->scal[2], rr0 = s.st_host->scal[3];
  if (rel_res) *rel_res = rr0 > 0 ? sqrt(rr / rr0) : 0.0;
  const int iters = (int)s.st_host->scal[7];
  const double state = s.st_host->scal[6];
  if (state == 2.0 || state == 3.0) return -2;
  if (state == 0.0) return -1;
  return iters;
}

// with profiling on, the algorithmic bytes and operations of a finished
// solve (its iteration count is known only once the status word is read)
void pcg_account(Scene& s, int its) {
  if (!s.prof.on || its == -2 || s.dense_n) return;
  const double n = (double)(its == -1 ? (int)s.st_host->scal[7] : its);
  const long np = s.st_host->np;
  s.prof.slot[PF_SPMV].bytes += n * pcg_iter_bytes(s, np);
  s.prof.slot[PF_SPMV].flops += n * pcg_iter_flops(s, np);
}

int run_pcg(Scene& s, const double* rhs, double* xout, int max_iter, double rel_tol, double* rel_res,
            bool indefinite) {
  if (s.dense_n) {
    launch_dense_solve(s, rhs, xout, indefinite);
    cudaMemcpyAsync(s.st_host, s.st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s.stream);
    cudaStreamSynchronize(s.stream);
    return pcg_result(s, rel_res);
  }
  launch_pcg_fp32_blocks(s);
  launch_pcg_init(s, rhs, 1.0, xout);
  launch_pcg_solve(s, xout, max_iter, rel_tol);
  cudaMemcpyAsync(s.st_host, s.st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s.stream);
  cudaStreamSynchronize(s.stream);
  const int its = pcg_result(s, rel_res);
  pcg_account(s, its);
  return its;
}

}  // namespace abd
