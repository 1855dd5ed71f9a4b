// Dense direct solve of the Newton system of a small scene: the block
// system (diagonal body blocks and body-pair blocks) is written into a dense
// symmetric matrix of order N (12 DOFs per body, padded to a multiple of 32
// with unit diagonal; static bodies decoupled with identity blocks and zero
// right-hand side), factored by a right-looking tiled Cholesky (32x32 tiles:
// the diagonal tile, the tiles below it, the trailing tiles, one launch each
// per tile column) and solved by forward and backward substitution in one
// block.  It replaces the block-Jacobi PCG of the paper's direct solver
// substitute (Sec. 5) where the PCG needs many iterations (stacks: long
// chains of stiff contacts).  A non-positive pivot marks the solve as a
// breakdown in the status word (scal[6] = 2), like the PCG's.
//
// The adjoint's unprojected Hessian may be indefinite at a converged state
// (a stationary point need not be a minimiser; the implicit function theorem
// wants it nonsingular only).  For it the factorisation is the signed
// Cholesky A = L S L^T, S = diag(s_j), s_j = sign of the j-th pivot, without
// pivoting (the LDL^T factorisation with D = L_jj^2 S); then only a zero or
// non-finite pivot is a breakdown.  dinv holds s_j / L_jj, positive
// throughout for the Newton system.
#include <cfloat>

#include "abd_internal.cuh"

namespace abd {

namespace {

constexpr int kT = 32;  // tile order

__global__ void k_dense_fill(int nb, int N, const uint8_t* is_static, const double* D, const int2* P,
                             const double* pblk, const DevStatus* cst, double* A) {
  const int np = cst->np;
  const long tid = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const long stride = (long)gridDim.x * blockDim.x;
  // diagonal blocks (identity for static bodies) and the padding diagonal
  for (long e = tid; e < 144L * nb; e += stride) {
    const int b = (int)(e / 144), k = (int)(e - 144L * b), i = k / 12, j = k - 12 * i;
    const double v = is_static[b] ? (i == j ? 1.0 : 0.0) : D[144L * b + k];
    A[(long)(12 * b + i) * N + 12 * b + j] = v;
  }
  for (long r = 12L * nb + tid; r < N; r += stride) A[r * N + r] = 1.0;
  // body-pair blocks H_ab (rows: DOFs of a) and their transposes
  for (long e = tid; e < 144L * np; e += stride) {
    const int p = (int)(e / 144), k = (int)(e - 144L * p), i = k / 12, j = k - 12 * i;
    const int a = P[p].x, b = P[p].y;
    if (is_static[a] || is_static[b]) continue;
    const double v = pblk[(size_t)p * kBlkStride + k];
    A[(long)(12 * a + i) * N + 12 * b + j] = v;
    A[(long)(12 * b + j) * N + 12 * a + i] = v;
  }
}

// Cholesky of the diagonal tile k (lower factor in place; s_j / L_jj in
// dinv).  Warp c holds column c of the tile, lane r its row r (the tile is
// staged transposed): every step's column scaling and rank-1 update are
// whole-warp instructions, and the pivot's reciprocal square root is one
// lane's work.  indefinite != 0 accepts negative pivots (signed Cholesky)
__global__ void __launch_bounds__(1024) k_dense_potrf(double* A, int N, int k, double* dinv, DevStatus* st,
                                                      int indefinite) {
  __shared__ double T[kT][kT + 1];  // T[c][r] = A(o + r, o + c)
  __shared__ double inv, sgn;
  __shared__ int bad;
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const long o = (long)kT * k;
  T[lane][w] = A[(o + w) * N + o + lane];  // coalesced rows, transposed into columns
  if (t == 0) bad = 0;
  __syncthreads();
  for (int j = 0; j < kT; ++j) {
    if (t == 0) {
      double d = T[j][j], sj = 1.0;
      if (indefinite && d < 0.0) {
        d = -d;
        sj = -1.0;
      }
      if (!(d > 0.0) || !(d <= DBL_MAX)) {
        bad = 1;
        d = 1.0;  // keep the factor finite; the solve is marked as failed
      }
      const double rs = rsqrt(d);
      T[j][j] = d * rs;
      inv = sj * rs;
      sgn = sj;
      dinv[o + j] = sj * rs;
    }
    __syncthreads();
    // L_ij = a_ij s_j / L_jj; the trailing update subtracts L_ij s_j L_wj
    if (w == j && lane > j) T[j][lane] *= inv;
    __syncthreads();
    if (w > j && lane >= w) T[w][lane] -= sgn * T[j][lane] * T[j][w];
    __syncthreads();
  }
  if (w >= lane) A[(o + w) * N + o + lane] = T[lane][w];
  if (t == 0 && bad) st->scal[6] = 2.0;
}

// tiles below the diagonal in column k: X = A_ik L_kk^-T S_k (warp c holds
// column c of X and of L, lane r row r)
__global__ void __launch_bounds__(1024) k_dense_trsm(double* A, int N, int k, const double* dinv) {
  __shared__ double L[kT][kT + 1], X[kT][kT + 1];  // transposed: [column][row]
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const long o = (long)kT * k, oi = (long)kT * (k + 1 + blockIdx.x);
  L[lane][w] = A[(o + w) * N + o + lane];
  X[lane][w] = A[(oi + w) * N + o + lane];
  __syncthreads();
  for (int j = 0; j < kT; ++j) {
    if (w == j) X[j][lane] *= fabs(dinv[o + j]);
    __syncthreads();
    if (w > j) X[w][lane] -= X[j][lane] * L[j][w];
    __syncthreads();
  }
  A[(oi + w) * N + o + lane] = dinv[o + lane] < 0.0 ? -X[lane][w] : X[lane][w];
}

// trailing tiles (i, j), k < j <= i: A_ij -= L_ik S_k L_jk^T
__global__ void __launch_bounds__(1024) k_dense_syrk(double* A, int N, int k, int nt, const double* dinv) {
  __shared__ double Li[kT][kT + 1], Lj[kT][kT + 1], S[kT];
  const int t = threadIdx.x, r = t / kT, c = t - kT * (t / kT);
  // blockIdx.x -> (ii, jj), jj <= ii, over the m = nt - k - 1 trailing tiles
  const int m = nt - k - 1;
  int idx = blockIdx.x, ii = 0;
  while (idx > ii) {
    idx -= ii + 1;
    ++ii;
  }
  const int jj = idx;
  if (ii >= m) return;
  const long o = (long)kT * k, oi = (long)kT * (k + 1 + ii), oj = (long)kT * (k + 1 + jj);
  Li[r][c] = A[(oi + r) * N + o + c];
  Lj[r][c] = A[(oj + r) * N + o + c];
  if (t < kT) S[t] = dinv[o + t] < 0.0 ? -1.0 : 1.0;
  __syncthreads();
  double s = 0.0;
#pragma unroll 8
  for (int q = 0; q < kT; ++q) s += Li[r][q] * S[q] * Lj[c][q];
  A[(oi + r) * N + oj + c] -= s;
}

// forward and backward substitution with the factor (one block): L y = b,
// z = S y, L^T x = z; static rows of the right-hand side are taken as zero,
// padding rows are zero
__global__ void __launch_bounds__(1024) k_dense_trsv(const double* A, int N, int n, const double* dinv,
                                                     const uint8_t* is_static, const double* rhs, double* x,
                                                     const DevStatus* cst) {
  extern __shared__ double y[];
  __shared__ double Dt[kT][kT + 1];
  const int t = threadIdx.x, lane = t & 31, w = t >> 5, nw = blockDim.x >> 5;
  for (int i = t; i < N; i += blockDim.x) y[i] = (i < n && !is_static[i / 12]) ? rhs[i] : 0.0;
  __syncthreads();
  const int nt = N / kT;
  // L y = b
  for (int k = 0; k < nt; ++k) {
    const long o = (long)kT * k;
    Dt[w][lane] = A[(o + w) * N + o + lane];  // the diagonal tile, staged
    __syncthreads();
    if (w == 0) {
      double v = y[o + lane];
      for (int j = 0; j < kT; ++j) {
        const double yj = __shfl_sync(0xffffffffu, v * fabs(dinv[o + j]), j);
        if (lane == j) v = yj;
        if (lane > j) v -= Dt[lane][j] * yj;
      }
      y[o + lane] = v;
    }
    __syncthreads();
    for (long i = o + kT + w; i < N; i += nw) {  // rows below: warp per row
      double s = A[i * N + o + lane] * y[o + lane];
      for (int q = 16; q > 0; q >>= 1) s += __shfl_xor_sync(0xffffffffu, s, q);
      if (lane == 0) y[i] -= s;
    }
    __syncthreads();
  }
  for (int i = t; i < N; i += blockDim.x)
    if (dinv[i] < 0.0) y[i] = -y[i];
  __syncthreads();
  // L^T x = y
  for (int k = nt - 1; k >= 0; --k) {
    const long o = (long)kT * k;
    Dt[w][lane] = A[(o + w) * N + o + lane];
    __syncthreads();
    if (w == 0) {
      double v = y[o + lane];
      for (int j = kT - 1; j >= 0; --j) {
        const double xj = __shfl_sync(0xffffffffu, v * fabs(dinv[o + j]), j);
        if (lane == j) v = xj;
        if (lane < j) v -= Dt[j][lane] * xj;
      }
      y[o + lane] = v;
    }
    __syncthreads();
    for (long i = t; i < o; i += blockDim.x) {  // rows above: column block of L^T
      double s = 0.0;
#pragma unroll 8
      for (int q = 0; q < kT; ++q) s += A[(o + q) * N + i] * y[o + q];
      y[i] -= s;
    }
    __syncthreads();
  }
  for (int i = t; i < n; i += blockDim.x) x[i] = is_static[i / 12] ? 0.0 : y[i];
  (void)cst;
}

// solver status in the PCG's slots: done (or breakdown, set by the
// factorisation), no iterations, residual not formed
__global__ void k_dense_status(DevStatus* st) {
  if (st->scal[6] != 2.0) st->scal[6] = 1.0;
  st->scal[7] = 0.0;
  st->scal[2] = 0.0;
  st->scal[3] = 0.0;
}

__global__ void k_dense_begin(DevStatus* st) { st->scal[6] = 0.0; }

}  // namespace

int dense_order(int nb, int max_dofs) {
  const long n = 12L * nb;
  if (max_dofs <= 0 || n > max_dofs) return 0;
  const long N = (n + kT - 1) / kT * kT;
  return N <= kDenseMaxOrder ? (int)N : 0;
}

void launch_dense_solve(Scene& s, const double* rhs, double* x, bool indefinite) {
  const int N = s.dense_n, nt = N / kT;
  double* A = s.dense.p;
  // algorithmic flops: the factorisation N^3 / 3 and two substitutions 2 N^2
  ProfScope pd(s, PF_DENSE, 0.0, (double)N * N * N / 3.0 + 2.0 * N * N);
  counted(s, 3);
  k_dense_begin<<<1, 1, 0, s.stream>>>(s.st);
  cudaMemsetAsync(A, 0, sizeof(double) * N * N, s.stream);
  k_dense_fill<<<sm_grid(s, 4), 256, 0, s.stream>>>(s.nb, N, s.is_static.p, s.D.p, s.P.p, s.pblk.p, s.st, A);
  for (int k = 0; k < nt; ++k) {
    counted(s);
    k_dense_potrf<<<1, 1024, 0, s.stream>>>(A, N, k, s.dense_dinv.p, s.st, indefinite ? 1 : 0);
    const int m = nt - k - 1;
    if (m > 0) {
      counted(s, 2);
      k_dense_trsm<<<m, 1024, 0, s.stream>>>(A, N, k, s.dense_dinv.p);
      k_dense_syrk<<<m * (m + 1) / 2, 1024, 0, s.stream>>>(A, N, k, nt, s.dense_dinv.p);
    }
  }
  counted(s, 2);
  k_dense_trsv<<<1, 1024, sizeof(double) * N, s.stream>>>(A, N, 12 * s.nb, s.dense_dinv.p, s.is_static.p, rhs, x,
                                                          s.st);
  k_dense_status<<<1, 1, 0, s.stream>>>(s.st);
}

}  // namespace abd
