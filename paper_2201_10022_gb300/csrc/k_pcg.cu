// Block-Jacobi preconditioned conjugate gradients on the Newton system
// H dq = rhs (the linear solve of each Newton iteration; the paper's direct
// LLT of Sec. 5 replaced by an iterative solve on the device).
//
// H is symmetric block-sparse with 12x12 blocks: the diagonal blocks D_b,
// and for every body pair (a, b), a < b, the upper block H_ab stored once in
// the pair's assembly record (rows = DOFs of a).  Row b of the product is
//   y_b = D_b v_b + sum_{(b,c) upper} H_bc v_c + sum_{(c,b) incoming} H_cb^T v_b'
// The preconditioner is the explicit inverse of each diagonal block.
//
// One persistent cooperative kernel runs the whole solve: every iteration is
// two phases separated by a grid barrier, and every block derives the
// scalars (alpha, beta, the convergence test) from the same chunk partial
// sums in the same order, so no host round trip is needed and the result is
// bit-identical run to run.  Partial sums are formed per chunk of kChunk
// bodies in body order (not per block), so the arithmetic does not depend on
// the grid size.  The grid barrier's wait is bounded: a block that waits
// longer than kBarrierTimeout cycles raises an abort word that releases
// every other block, and the solve reports the failure in the status word.
#include <stddef.h>

#include <algorithm>

#include "abd_internal.cuh"

namespace abd {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kChunk = 4;           // bodies per reduction chunk
constexpr int kThreads = 256;       // threads per block of the solve kernel
constexpr int kWarps = kThreads / 32;
constexpr long long kBarrierTimeout = 4000000000LL;  // cycles (about 2 s at 2 GHz)

struct PcgArgs {
  int nb, nchunk, max_iter;
  const int* np;                    // body pairs in the list (device count; clamps the rows)
  double tol2;                      // squared relative residual tolerance
  const uint8_t* __restrict__ is_static;
  const double* __restrict__ D;     // nb x 144 diagonal blocks, row-major
  const double* __restrict__ Minv;  // nb x 144 inverse diagonal blocks
  const int* __restrict__ rowoff;   // nb + 1: upper pairs of each row in P
  const int* __restrict__ in_off;   // nb + 1: incoming pairs of each row
  const int* __restrict__ in_list;
  const int2* __restrict__ P;
  const double* __restrict__ pblk;  // per pair kBlkStride doubles, H_ab first
  double* x;
  double* r;
  double* z;
  double* p0;                       // search directions, alternating by iteration
  double* p1;
  double* Ap;
  double* cpart;                    // 3 x nchunk chunk partials: p.Ap, r.z, r.r
  unsigned* bar;                    // grid barrier: arrivals, generation, abort
  DevStatus* st;
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
        __nanosleep(64);
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
// sum of the first 12 lanes' values (tree, fixed order); valid in lane 0
__device__ __forceinline__ double sum12(double v) {
  const int lane = threadIdx.x & 31;
  double t = lane < 12 ? v : 0.0;
  t += __shfl_down_sync(kFull, t, 8);   // lanes 0..3 gather 8..11
  t += __shfl_down_sync(kFull, t, 4);
  t += __shfl_down_sync(kFull, t, 2);
  t += __shfl_down_sync(kFull, t, 1);
  return t;
}

// the totals of K partial arrays (each nchunk long), by every thread of the
// block: thread t adds entries t, t + kThreads, ... (loads independent of one
// another), then a fixed tree over the block; the order depends only on
// nchunk, so every block of the grid forms the same totals
template <int K>
__device__ void block_totals(const double* part, int nchunk, double* out) {
  __shared__ double s_red[K][kWarps];
  const int t = threadIdx.x;
  double acc[K];
#pragma unroll
  for (int k = 0; k < K; ++k) acc[k] = 0.0;
#pragma unroll 4
  for (int i = t; i < nchunk; i += kThreads)
#pragma unroll
    for (int k = 0; k < K; ++k) acc[k] += part[(size_t)k * nchunk + i];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    // within the warp (fixed butterfly), then across the warps in order
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

// ---- warp-cooperative 12x12 block products --------------------------------
// Lane l holds entries e = l + 32 k (k < 5, e < 144) of every block it reads,
// so each block is read by the warp as contiguous 256-byte rows.  acc[k]
// collects entry e's products for row e / 12 (a block used as stored) and
// acct[k] for row e % 12 (a block used transposed); the 12 column values come
// from lanes 0..11 by shuffles.
struct BlockAcc {
  double acc[5], acct[5];
};

__device__ __forceinline__ void acc_block(BlockAcc& A, const double* __restrict__ blk, double vlane,
                                          bool transposed) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    const int e = lane + 32 * k;
    const int src = transposed ? e / 12 : e % 12;
    const double v = __shfl_sync(kFull, vlane, src < 12 ? src : 0);
    if (e < 144) {
      const double h = __ldg(blk + e);
      if (transposed) A.acct[k] = fma(h, v, A.acct[k]);
      else A.acc[k] = fma(h, v, A.acc[k]);
    }
  }
}

// row sums of the accumulated entries: lanes 0..11 receive y_l
__device__ __forceinline__ double row_sums(const BlockAcc& A, double* sbuf) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    const int e = lane + 32 * k;
    if (e < 144) {
      sbuf[e] = A.acc[k];
      sbuf[144 + e] = A.acct[k];
    }
  }
  __syncwarp();
  double y = 0.0;
  if (lane < 12) {
#pragma unroll
    for (int j = 0; j < 12; ++j) y += sbuf[12 * lane + j];
#pragma unroll
    for (int i = 0; i < 12; ++i) y += sbuf[144 + 12 * i + lane];
  }
  __syncwarp();
  return y;
}

// ---- the two phases of an iteration ------------------------------------------
// Phase A of iteration k: p_k = z_k + beta p_{k-1} (formed on the fly for the
// row and every column it reads; p_0 = z_0 is given), Ap = H p_k, and the
// chunk partials of p_k . Ap.  Warp w of the grid takes chunks w, w + W, ...
__device__ void phase_spmv(const PcgArgs& a, int k, double beta, double* sbuf) {
  const int lane = threadIdx.x & 31;
  const int wgrid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  const int np = *a.np;
  const double* pold = (k & 1) ? a.p0 : a.p1;  // p_{k-1}
  double* pnew = (k & 1) ? a.p1 : a.p0;        // p_k
  const bool fly = k > 0;
  for (int c = wgrid; c < a.nchunk; c += nw) {
    double pap = 0.0;
    for (int b = c * kChunk; b < min(a.nb, (c + 1) * kChunk); ++b) {
      if (a.is_static[b]) {
        if (lane < 12) {
          a.Ap[12 * b + lane] = 0.0;
          pnew[12 * b + lane] = 0.0;
        }
        continue;
      }
      // this row's direction (lanes 0..11)
      double pb = 0.0;
      if (lane < 12) {
        pb = fly ? fma(beta, pold[12 * b + lane], a.z[12 * b + lane]) : pnew[12 * b + lane];
      }
      BlockAcc A;
#pragma unroll
      for (int q = 0; q < 5; ++q) A.acc[q] = A.acct[q] = 0.0;
      acc_block(A, a.D + (size_t)144 * b, pb, false);
      for (int p = a.rowoff[b]; p < min(a.rowoff[b + 1], np); ++p) {
        const int o = a.P[p].y;
        if (a.is_static[o]) continue;
        double po = 0.0;
        if (lane < 12) po = fly ? fma(beta, pold[12 * o + lane], a.z[12 * o + lane]) : pnew[12 * o + lane];
        acc_block(A, a.pblk + (size_t)p * kBlkStride, po, false);
      }
      for (int q = a.in_off[b]; q < a.in_off[b + 1]; ++q) {
        const int p = a.in_list[q];
        const int o = a.P[p].x;
        if (a.is_static[o]) continue;
        double po = 0.0;
        if (lane < 12) po = fly ? fma(beta, pold[12 * o + lane], a.z[12 * o + lane]) : pnew[12 * o + lane];
        acc_block(A, a.pblk + (size_t)p * kBlkStride, po, true);
      }
      const double y = row_sums(A, sbuf);
      if (lane < 12) {
        a.Ap[12 * b + lane] = y;
        if (fly) pnew[12 * b + lane] = pb;
      }
      const double t = sum12(pb * y);
      pap += t;  // lane 0's value is the one used
    }
    if (lane == 0) a.cpart[c] = pap;
  }
}

// Phase B of iteration k: x += alpha p_k, r -= alpha Ap, z = Minv r, and the
// chunk partials of r.z and r.r
__device__ void phase_update(const PcgArgs& a, int k, double alpha, double* sbuf) {
  const int lane = threadIdx.x & 31;
  const int wgrid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  const double* pk = (k & 1) ? a.p1 : a.p0;
  for (int c = wgrid; c < a.nchunk; c += nw) {
    double rz = 0.0, rr = 0.0;
    for (int b = c * kChunk; b < min(a.nb, (c + 1) * kChunk); ++b) {
      if (a.is_static[b]) continue;
      double rb = 0.0;
      if (lane < 12) {
        const int i = 12 * b + lane;
        a.x[i] = fma(alpha, pk[i], a.x[i]);
        rb = fma(-alpha, a.Ap[i], a.r[i]);
        a.r[i] = rb;
      }
      BlockAcc A;
#pragma unroll
      for (int q = 0; q < 5; ++q) A.acc[q] = A.acct[q] = 0.0;
      acc_block(A, a.Minv + (size_t)144 * b, rb, false);
      const double zb = row_sums(A, sbuf);
      if (lane < 12) a.z[12 * b + lane] = zb;
      rz += sum12(rb * zb);
      rr += sum12(rb * rb);
    }
    if (lane == 0) {
      a.cpart[a.nchunk + c] = rz;
      a.cpart[2 * a.nchunk + c] = rr;
    }
  }
}

// The whole solve.  On entry x, r, z, p0 = z hold the start (x = 0, r = rhs,
// z = Minv r) and cpart[nchunk..3 nchunk) the chunk partials of r.z and r.r.
// On exit st->scal: [0] r.z, [2] r.r, [3] r.r at the start, [6] 1 converged /
// 0 iteration cap / 2 breakdown (p.Ap <= 0) / 3 barrier timeout, [7] iterations.
__global__ void __launch_bounds__(kThreads) k_pcg_solve(PcgArgs a) {
  __shared__ double sbuf[kWarps][288];
  double* wbuf = sbuf[threadIdx.x >> 5];
  unsigned gen = 0;
  double tot[3];
  block_totals<2>(a.cpart + a.nchunk, a.nchunk, tot);
  double rz = tot[0], rr = tot[1], rz_prev = 0.0;
  const double rr0 = rr;
  int k = 0;
  int state = rr0 == 0.0 ? 1 : 0;
  bool alive = true;
  // Hazards: phase_spmv of iteration k+1 overwrites the p.Ap partials and
  // phase_update of k+1 the r.z / r.r partials; every block has finished
  // reading them before the barrier that precedes each of those phases.
  while (state == 0 && k < a.max_iter) {
    phase_spmv(a, k, k > 0 ? rz / rz_prev : 0.0, wbuf);
    if (!(alive = grid_barrier(a.bar, gen))) break;
    block_totals<1>(a.cpart, a.nchunk, tot);
    const double pap = tot[0];
    if (!(pap > 0.0)) {
      state = 2;
      break;
    }
    phase_update(a, k, rz / pap, wbuf);
    if (!(alive = grid_barrier(a.bar, gen))) break;
    block_totals<2>(a.cpart + a.nchunk, a.nchunk, tot);
    rz_prev = rz;
    rz = tot[0];
    rr = tot[1];
    ++k;
    if (rr <= a.tol2 * rr0) state = 1;
  }
  if (!alive) state = 3;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    a.st->scal[0] = rz;
    a.st->scal[2] = rr;
    a.st->scal[3] = rr0;
    a.st->scal[6] = (double)state;
    a.st->scal[7] = (double)k;
    if (state == 2 || state == 3) atomicOr(&a.st->flags, ST_PCG_BREAKDOWN);
  }
}

// r = rhs (dynamic rows), x = 0, z = Minv r, p0 = z, chunk partials of r.z, r.r
__global__ void k_pcg_init(PcgArgs a, const double* __restrict__ rhs, double sign) {
  __shared__ double sbuf[kWarps][288];
  double* wbuf = sbuf[threadIdx.x >> 5];
  const int lane = threadIdx.x & 31;
  const int wgrid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int c = wgrid; c < a.nchunk; c += nw) {
    double rz = 0.0, rr = 0.0;
    for (int b = c * kChunk; b < min(a.nb, (c + 1) * kChunk); ++b) {
      const bool st = a.is_static[b];
      double rb = 0.0;
      if (lane < 12) {
        const int i = 12 * b + lane;
        rb = st ? 0.0 : sign * rhs[i];
        a.r[i] = rb;
        a.x[i] = 0.0;
      }
      double zb = 0.0;
      if (!st) {
        BlockAcc A;
#pragma unroll
        for (int q = 0; q < 5; ++q) A.acc[q] = A.acct[q] = 0.0;
        acc_block(A, a.Minv + (size_t)144 * b, rb, false);
        zb = row_sums(A, wbuf);
      }
      if (lane < 12) {
        a.z[12 * b + lane] = zb;
        a.p0[12 * b + lane] = zb;
      }
      rz += sum12(rb * zb);
      rr += sum12(rb * rb);
    }
    if (lane == 0) {
      a.cpart[a.nchunk + c] = rz;
      a.cpart[2 * a.nchunk + c] = rr;
    }
  }
}

}  // namespace

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static PcgArgs pcg_args(Scene& s, double* xout, int max_iter, double rel_tol) {
  PcgArgs a;
  a.nb = s.nb;
  a.nchunk = (s.nb + kChunk - 1) / kChunk;
  a.max_iter = max_iter;
  a.tol2 = rel_tol * rel_tol;
  a.is_static = s.is_static.p;
  a.D = s.D.p;
  a.Minv = s.Pinv.p;
  a.rowoff = s.rowoff.p;
  a.in_off = s.in_off.p;
  a.in_list = s.in_list.p;
  a.P = s.P.p;
  a.pblk = s.pblk.p;
  a.x = xout;
  a.r = s.r.p;
  a.z = s.z.p;
  a.p0 = s.pv.p;
  a.p1 = s.pv2.p;
  a.Ap = s.Ap.p;
  a.cpart = s.part.p;
  a.bar = s.pcg_bar.p;
  a.st = s.st;
  a.np = &s.st->np;
  return a;
}

int pcg_chunks(int nb) { return (nb + kChunk - 1) / kChunk; }

// co-resident blocks of the solve kernel on this device (set once per scene)
int pcg_grid(Scene& s) {
  if (s.pcg_blocks_per_sm <= 0) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pcg_solve, kThreads, 0) != cudaSuccess ||
        per_sm < 1) {
      cudaGetLastError();
      per_sm = 1;
    }
    s.pcg_blocks_per_sm = std::min(per_sm, 2);
  }
  // enough warps for the chunks, at most one wave of co-resident blocks
  const int want = (pcg_chunks(s.nb) + kWarps - 1) / kWarps;
  const int cap = std::max(1, s.pcg_blocks_per_sm * s.num_sms / s.grid_div);
  return std::max(1, std::min(want, cap));
}

void launch_pcg_init(Scene& s, const double* rhs, double sign, double* xout) {
  PcgArgs a = pcg_args(s, xout, 0, 0.0);
  counted(s);
  const int grid = std::max(1, std::min((a.nchunk + kWarps - 1) / kWarps, 4 * s.num_sms));
  k_pcg_init<<<grid, kThreads, 0, s.stream>>>(a, rhs, sign);
}

// the solve from the state k_pcg_init (or the preconditioner's fused start)
// left; enqueued only (the result is in the status word)
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

// algorithmic bytes and FP64 operations of one iteration: every stored block
// once (diagonal, upper off-diagonal), the inverse diagonal blocks once, the
// vectors p, z, Ap, x, r read or written once each, the pair list once
double pcg_iter_bytes(const Scene& s, long np) {
  return 8.0 * 144.0 * (2.0 * s.nb + (double)np) + 8.0 * 12.0 * 8.0 * s.nb + 8.0 * np;
}
double pcg_iter_flops(const Scene& s, long np) {
  // block products: diagonal and inverse once, each off-diagonal block twice
  // (as stored and transposed), 2 flops per entry; vector updates
  return 2.0 * 144.0 * (2.0 * s.nb + 2.0 * (double)np) + 2.0 * 12.0 * 6.0 * s.nb;
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

// with profiling on, the algorithmic bytes and FP64 operations of a finished
// solve (its iteration count is known only once the status word is read)
void pcg_account(Scene& s, int its) {
  if (!s.prof.on || its == -2 || s.dense_n) return;
  const double n = (double)(its == -1 ? (int)s.st_host->scal[7] : its);
  const long np = s.st_host->np;
  s.prof.slot[PF_SPMV].bytes += n * pcg_iter_bytes(s, np);
  s.prof.slot[PF_SPMV].flops += n * pcg_iter_flops(s, np);
}

int run_pcg(Scene& s, const double* rhs, double* xout, int max_iter, double rel_tol, double* rel_res) {
  if (s.dense_n) {
    launch_dense_solve(s, rhs, xout);
    cudaMemcpyAsync(s.st_host, s.st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s.stream);
    cudaStreamSynchronize(s.stream);
    return pcg_result(s, rel_res);
  }
  launch_pcg_init(s, rhs, 1.0, xout);
  launch_pcg_solve(s, xout, max_iter, rel_tol);
  cudaMemcpyAsync(s.st_host, s.st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s.stream);
  cudaStreamSynchronize(s.stream);
  const int its = pcg_result(s, rel_res);
  pcg_account(s, its);
  return its;
}

}  // namespace abd
