// Contact islands and the per-island line search of a Newton iteration.
//
// The incremental potential (Sec. 4) is a sum of body terms and of pair terms
// (barrier and lagged friction), each pair term coupling two bodies.  Take the
// graph whose nodes are the dynamic bodies and whose edges are the body pairs
// of the swept broad phase (every pair whose d-hat-dilated boxes over the
// whole step x(q) -> x(q + dq) overlap) and the lagged friction pairs.  Its
// connected components -- islands -- share no term anywhere on the segment
// from q to q + dq: E(q + diag(alpha_i) dq) = sum_i E_i(q_i + alpha_i dq_i).
// So the CCD step bound and the backtracking line search (Sec. 4.1, the
// filtered Newton step) are taken per island: each island gets the minimum
// time of impact over its own swept pairs and halves its own step until its
// own energy does not increase.  An island that needs a short step no longer
// shortens the step of every other body in the scene; each island's sequence
// of iterates is the one a Newton loop on that island alone would produce, so
// the converged point is the same minimiser.
//
// Islands are labelled by union-find with the smaller root kept on every link,
// so each island's label is its smallest body id whatever the order of the
// links.  Island energies are accumulated exactly: every contribution is a
// non-negative double (inertia, orthogonality energy, barrier energy and
// friction energy are all >= 0 up to rounding), converted to a 128-bit
// fixed-point integer (units of 2^-64) whose four 32-bit digits are added
// with 64-bit integer atomics (negative ones into a second sum), so the sums
// are exact and independent of the order of the additions (bit-identical
// runs).
#include <stddef.h>

#include <algorithm>

#include "abd_internal.cuh"

namespace abd {

namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ int uf_find(int* parent, int x) {
  volatile int* p = parent;
  int px = p[x];
  while (px != x) {
    const int gp = p[px];
    if (gp != px) p[x] = gp;  // path halving: a grandparent is still an ancestor
    x = px;
    px = p[x];
  }
  return x;
}

__device__ __forceinline__ void uf_union(int* parent, int a, int b) {
  while (true) {
    a = uf_find(parent, a);
    b = uf_find(parent, b);
    if (a == b) return;
    const int lo = min(a, b), hi = max(a, b);
    if (atomicCAS(&parent[hi], hi, lo) == hi) return;
  }
}

// ---- exact non-negative sums ------------------------------------------------
// digits of floor(v * 2^64) (v >= 0, finite, < 2^64); false if v is out of range
__device__ __forceinline__ bool fx_digits(double v, unsigned long long d[4]) {
  d[0] = d[1] = d[2] = d[3] = 0ull;
  if (v == 0.0) return true;
  if (!(v > 0.0) || !(v < 18446744073709551616.0)) return false;
  const unsigned long long bits = (unsigned long long)__double_as_longlong(v);
  int ex = (int)((bits >> 52) & 0x7ff);
  unsigned long long m = bits & ((1ull << 52) - 1);
  if (ex == 0) ex = 1;
  else m |= 1ull << 52;
  const int sh = ex - 1075 + 64;  // floor(v 2^64) = m 2^sh
  unsigned long long lo = 0, hi = 0;
  if (sh >= 64) {
    hi = m << (sh - 64);
  } else if (sh > 0) {
    lo = m << sh;
    hi = m >> (64 - sh);
  } else if (sh == 0) {
    lo = m;
  } else if (sh > -64) {
    lo = m >> (-sh);
  }
  d[0] = lo & 0xffffffffull;
  d[1] = lo >> 32;
  d[2] = hi & 0xffffffffull;
  d[3] = hi >> 32;
  return true;
}

// value of four digit accumulators (each < 2^64): carries, then the double
// (the same integer always gives the same double)
__device__ __forceinline__ double fx_value(const unsigned long long* acc) {
  unsigned long long c = 0, dig[5];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const unsigned long long t = acc[k] + c;
    dig[k] = t & 0xffffffffull;
    c = t >> 32;
  }
  dig[4] = c;
  return ldexp((double)dig[4], 64) + ldexp((double)dig[3], 32) + (double)dig[2] + ldexp((double)dig[1], -32) +
         ldexp((double)dig[0], -64);
}

// add v to an island's accumulator: |v| to base[16 key + 4 (v < 0) + 0..3]
// (separate sums of the positive and the negative contributions, so that a
// contribution that rounding made slightly negative is still exact); lanes
// with the same key and sign first add their digits (integer adds, exact),
// so that each takes one atomic per digit and warp.  Called by whole warps
// (on selects the lanes that contribute); the loop over the contributing
// lanes has the same trip count in every lane.
__device__ __forceinline__ void fx_add(unsigned long long* base, int island, double v, bool on, DevStatus* st) {
  unsigned long long d[4];
  const bool neg = v < 0.0;
  const int key = 2 * island + (neg ? 1 : 0);
  if (on && !fx_digits(fabs(v), d)) {
    set_flag(st, ST_NONFINITE);
    on = false;
  }
  if (!on) d[0] = d[1] = d[2] = d[3] = 0ull;
  const unsigned act = __ballot_sync(kFull, on && v != 0.0);
  if (!act) return;
  const int lane = threadIdx.x & 31;
  const int mykey = ((act >> lane) & 1) ? key : -1;
  unsigned long long s[4] = {0ull, 0ull, 0ull, 0ull};
  unsigned lead = 0;  // lanes that lead a group of equal keys
  for (unsigned m = act; m; m &= m - 1) {
    const int src = __ffs(m) - 1;
    const int k = __shfl_sync(kFull, mykey, src);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const unsigned long long x = __shfl_sync(kFull, d[j], src);
      if (k == mykey) s[j] += x;
    }
    // the first contributing lane with this key leads its group
    const unsigned same = __ballot_sync(kFull, k == mykey) & act;
    if ((same & ((1u << src) - 1u)) == 0) lead |= 1u << src;
  }
  if (((lead >> lane) & 1) && ((act >> lane) & 1)) {
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if (s[j]) atomicAdd(base + 16L * island + 4 * (neg ? 1 : 0) + j, s[j]);
  }
}

}  // namespace

// ---- kernels ------------------------------------------------------------------
// every body its own root; per-root island state cleared
__global__ void k_isl_init(int nb, int* parent, unsigned long long* toi, unsigned long long* step,
                           unsigned long long* E, int* lstate) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += gridDim.x * blockDim.x) {
    parent[b] = b;
    toi[b] = 0x3ff0000000000000ull;  // bits of 1.0
    step[b] = 0ull;
    for (int k = 0; k < 16; ++k) E[16L * b + k] = 0ull;
    lstate[2 * b] = 0;
    lstate[2 * b + 1] = 0;
  }
}

// links: dynamic-dynamic body pairs of the list and the lagged friction pairs
__global__ void k_isl_link(const DevStatus* __restrict__ cst, const int2* P, const int2* fpairs,
                           const uint8_t* is_static, int* parent) {
  const int np = cst->np, nfp = cst->nfp;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < np + nfp; p += gridDim.x * blockDim.x) {
    const int2 e = p < np ? P[p] : fpairs[p - np];
    if (is_static[e.x] || is_static[e.y]) continue;
    uf_union(parent, e.x, e.y);
  }
}

// island label (smallest body id of the island) of every body
__global__ void k_isl_label(int nb, int* parent, int* isl) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += gridDim.x * blockDim.x) isl[b] = uf_find(parent, b);
}

// island of a body pair: that of its dynamic body (pairs of two static bodies
// are never listed)
__device__ __forceinline__ int pair_island(const int* isl, const uint8_t* is_static, int a, int b) {
  return is_static[a] ? isl[b] : isl[a];
}

// exact per-island energies.  which = 0: the reference energies E0 of the
// iterate, from the system's stored terms (body energies, barrier terms with
// their vertices, friction records); which = 1: the trial's, from the
// energy-only pass (body energies, the barrier partials of the (body pair,
// chunk) slots of the work list, friction records).  One thread per
// contribution.
__global__ void k_isl_energy(int which, int nb, const uint8_t* __restrict__ is_static, const int* __restrict__ isl,
                             const int* __restrict__ vbody, const double* __restrict__ Eb,
                             const DevStatus* __restrict__ cst, const double* __restrict__ term,
                             const int4* __restrict__ termv, const double* __restrict__ Epair, int nch,
                             const int2* __restrict__ P, const double* __restrict__ fterm,
                             const FricRec* __restrict__ fr, const int* __restrict__ lstate,
                             const int* __restrict__ ework, unsigned long long* E, DevStatus* st) {
  const long nbar = which == 0 ? (long)cst->nact : (long)cst->n_ework;
  const long nfr = cst->nfr;
  const long n = 2L * nb + nbar + nfr;
  unsigned long long* base = E + 8 * which;
  const long stride = (long)gridDim.x * blockDim.x;
  for (long i0 = (long)blockIdx.x * blockDim.x; i0 < n; i0 += stride) {
    const long i = i0 + threadIdx.x;
    bool on = i < n;
    int key = 0;
    double v = 0.0;
    if (on) {
      if (i < 2L * nb) {
        const int b = (int)(i >> 1);
        on = !is_static[b];
        if (on) {
          key = isl[b];
          v = Eb[i];
        }
      } else if (i < 2L * nb + nbar) {
        const long t = i - 2L * nb;
        if (which == 0) {
          const int4 vv = termv[t];
          key = pair_island(isl, is_static, vbody[vv.x], vbody[vv.w]);
          v = term[t * kTermStride];
        } else {
          const int w = ework[t];
          const int2 pr = P[w / nch];
          key = pair_island(isl, is_static, pr.x, pr.y);
          v = Epair[w];
        }
      } else {
        const long f = i - 2L * nb - nbar;
        key = pair_island(isl, is_static, fr[f].a, fr[f].b);
        v = fterm[f * kTermStride];
      }
    }
    // a trial's sums are read for the pending islands only
    if (which == 1 && on && lstate[2 * key] != 0) on = false;
    fx_add(base, key, v, on, st);
  }
}

// largest vertex step |J dq| of each island (the bits of non-negative
// doubles order like the doubles; lanes of one island first take their
// maximum together)
__global__ void k_isl_step(int nv, const int* vbody, const uint8_t* is_static, const int* isl, const double4* dx,
                           unsigned long long* step) {
  for (int v0 = blockIdx.x * blockDim.x; v0 < nv; v0 += gridDim.x * blockDim.x) {
    const int v = v0 + threadIdx.x;
    bool on = v < nv;
    int key = -1;
    unsigned long long bits = 0ull;
    if (on) {
      const int b = vbody[v];
      on = !is_static[b];
      if (on) {
        const double4 d = dx[v];
        key = isl[b];
        bits = (unsigned long long)__double_as_longlong(sqrt(d.x * d.x + d.y * d.y + d.z * d.z));
      }
    }
    const unsigned act = __ballot_sync(kFull, on);
    if (!on) continue;
    const unsigned peers = __match_any_sync(act, key);
    unsigned long long m = bits;
    for (unsigned q = peers; q; q &= q - 1) {
      const unsigned long long x = __shfl_sync(peers, bits, __ffs(q) - 1);
      m = x > m ? x : m;
    }
    if ((int)(threadIdx.x & 31) == __ffs(peers) - 1) atomicMax(&step[key], m);
  }
}

// start of the line search: each island's step = its CCD bound.  An island
// whose Newton step is already within the tolerance (converged: the step is
// a refinement inside the quadratic region) takes it, bounded by CCD,
// without the energy test, which at that scale measures rounding only.
__global__ void k_isl_start(int nb, const uint8_t* is_static, const int* isl, const unsigned long long* toi,
                            const unsigned long long* step, double tol, double* alpha, int* lstate) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += gridDim.x * blockDim.x) {
    if (is_static[b] || isl[b] != b) continue;
    const bool done = __longlong_as_double((long long)step[b]) <= tol;
    alpha[b] = __longlong_as_double((long long)toi[b]);
    lstate[2 * b] = done ? 1 : 0;  // 0 pending, 1 accepted
    lstate[2 * b + 1] = 0;         // halvings
  }
}

// trial state: q + alpha_island dq (static bodies keep q); with lstate (the
// halving rounds) only for the bodies of pending islands (an accepted
// island's trial state stays as accepted)
__global__ void k_isl_trial(int nb, const uint8_t* is_static, const int* isl, const double* alpha, const double* q,
                            const double* dq, const int* lstate, double* qtrial) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 12 * nb; i += gridDim.x * blockDim.x) {
    const int b = i / 12;
    if (is_static[b]) {
      qtrial[i] = q[i];
      continue;
    }
    const int is = isl[b];
    if (lstate && lstate[2 * is] != 0) continue;
    qtrial[i] = fma(alpha[is], dq[i], q[i]);
  }
}

// acceptance of each pending island: E_i(trial) <= E_i(q) + slack (|E_i(q)| + 1)
// accepts; otherwise the island's step is halved (at most ls_max times).  The
// trial accumulators of the islands that were pending (the only ones a trial
// adds to) are cleared for the next trial; the counts of pending islands, of
// islands and of failed islands go to the status word.
__global__ void k_isl_accept(int nb, const uint8_t* is_static, const int* isl, double slack_rel, int ls_max,
                             unsigned long long* E, double* alpha, int* lstate, DevStatus* st) {
  int pending = 0, islands = 0, failed = 0, halv = 0;
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += gridDim.x * blockDim.x) {
    if (is_static[b] || isl[b] != b) continue;
    ++islands;
    const bool was_pending = lstate[2 * b] == 0;
    if (was_pending) {
      const double e0 = fx_value(E + 16L * b) - fx_value(E + 16L * b + 4);
      const double et = fx_value(E + 16L * b + 8) - fx_value(E + 16L * b + 12);
      if (et <= e0 + slack_rel * (fabs(e0) + 1.0)) {
        lstate[2 * b] = 1;
      } else if (lstate[2 * b + 1] >= ls_max) {
        ++failed;
      } else {
        alpha[b] *= 0.5;
        lstate[2 * b + 1] += 1;
        ++pending;
      }
    }
    halv = max(halv, lstate[2 * b + 1]);
    // only pending islands accumulate trial sums: clear those
    if (was_pending) {
#pragma unroll
      for (int k = 8; k < 16; ++k) E[16L * b + k] = 0ull;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    pending += __shfl_xor_sync(kFull, pending, o);
    islands += __shfl_xor_sync(kFull, islands, o);
    failed += __shfl_xor_sync(kFull, failed, o);
    halv = max(halv, __shfl_xor_sync(kFull, halv, o));
  }
  if ((threadIdx.x & 31) == 0) {
    if (pending) atomicAdd(&st->ls_pending, pending);
    if (islands) atomicAdd(&st->n_islands, islands);
    if (failed) atomicAdd(&st->ls_failed, failed);
    if (halv) atomicMax(&st->ls_halv_max, halv);
  }
}

// start of a halving round of the device-side loop: the counts the acceptance
// pass accumulates are cleared, the round is counted
__global__ void k_ls_round_begin(DevStatus* st) {
  st->ls_pending = 0;
  st->n_islands = 0;
  st->ls_failed = 0;
  st->ls_halv_max = 0;
  st->ls_rounds += 1;
}

// condition of the device-side line-search loop (one thread)
__global__ void k_ls_condition(DevStatus* st, cudaGraphConditionalHandle h, int max_rounds, int first) {
  if (first) st->ls_rounds = 0;
  const bool more = st->ls_pending > 0 && st->ls_failed == 0 && !(st->flags & ST_INTERSECT) &&
                    st->ls_rounds < max_rounds;
  cudaGraphSetConditional(h, more ? 1u : 0u);
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
static int grid_n(long n, int t, int cap) {
  long g = (n + t - 1) / t;
  return (int)std::max(1L, std::min(g, (long)cap));
}

// islands of the current body-pair list (and the lagged friction pairs)
void launch_islands(Scene& s) {
  counted(s, 3);
  const int g = grid_n(s.nb, 256, sm_grid(s, 8));
  k_isl_init<<<g, 256, 0, s.stream>>>(s.nb, s.uf.p, s.isl_toi.p, s.isl_step.p, s.isl_E.p, s.isl_state.p);
  k_isl_link<<<sm_grid(s, 4), 256, 0, s.stream>>>(s.st, s.P.p, s.fpairs.p, s.is_static.p, s.uf.p);
  k_isl_label<<<g, 256, 0, s.stream>>>(s.nb, s.uf.p, s.isl.p);
}

void launch_island_energy(Scene& s, int which) {
  counted(s);
  k_isl_energy<<<sm_grid(s, 8), 256, 0, s.stream>>>(which, s.nb, s.is_static.p, s.isl.p, s.vbody.p, s.Eb.p, s.st,
                                                      s.term.p, s.termv.p, s.Epair.p, energy_chunks(s), s.P.p,
                                                      s.fterm.p, s.fric.p, s.isl_state.p, s.ework.p, s.isl_E.p,
                                                      s.st);
}

void launch_island_start(Scene& s) {
  counted(s, 2);
  // the Newton step per island (dx of this iteration, labels of this swept list)
  k_isl_step<<<grid_n(s.nv, 256, sm_grid(s, 8)), 256, 0, s.stream>>>(s.nv, s.vbody.p, s.is_static.p, s.isl.p,
                                                                      s.dx.p, s.isl_step.p);
  k_isl_start<<<grid_n(s.nb, 256, sm_grid(s, 8)), 256, 0, s.stream>>>(
      s.nb, s.is_static.p, s.isl.p, s.isl_toi.p, s.isl_step.p, s.newton_tol, s.isl_alpha.p, s.isl_state.p);
}

void launch_island_trial(Scene& s, bool pending_only) {
  counted(s);
  k_isl_trial<<<grid_n(12L * s.nb, 256, sm_grid(s, 8)), 256, 0, s.stream>>>(
      s.nb, s.is_static.p, s.isl.p, s.isl_alpha.p, s.q.p, s.dq.p, pending_only ? s.isl_state.p : nullptr,
      s.qtrial.p);
}

void launch_island_accept(Scene& s, bool reset) {
  counted(s, reset ? 2 : 1);
  if (reset) cudaMemsetAsync(&s.st->ls_pending, 0, 4 * sizeof(int), s.stream);
  k_isl_accept<<<grid_n(s.nb, 256, sm_grid(s, 4)), 256, 0, s.stream>>>(
      s.nb, s.is_static.p, s.isl.p, s.prm.ls_slack_rel, s.prm.ls_max, s.isl_E.p, s.isl_alpha.p, s.isl_state.p, s.st);
}

void launch_ls_round_begin(Scene& s) {
  counted(s);
  k_ls_round_begin<<<1, 1, 0, s.stream>>>(s.st);
}

void launch_ls_condition(Scene& s, cudaGraphConditionalHandle h, int max_rounds, bool first) {
  counted(s);
  k_ls_condition<<<1, 1, 0, s.stream>>>(s.st, h, max_rounds, first ? 1 : 0);
}

}  // namespace abd
