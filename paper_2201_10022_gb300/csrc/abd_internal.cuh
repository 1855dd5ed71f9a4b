// Internal declarations of the affine-body library: the device-resident
// scene, the device status word and the kernel launchers shared by the
// translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <utility>
#include <vector>

#include "../../include/abd.h"

namespace abd {

// ---- device status word ----------------------------------------------------
enum : unsigned {
  ST_CAP_ROWS = 1u << 0,       // body-pair row capacity exceeded
  ST_CAP_CANDS = 1u << 1,      // candidate slots per body pair exceeded
  ST_CAP_PAIRS = 1u << 2,      // body-pair list capacity exceeded
  ST_CAP_ACTIVE = 1u << 3,     // flat active-term storage exceeded
  ST_CCD_MAXITER = 1u << 4,
  ST_INTERSECT = 1u << 5,      // a pair at zero distance
  ST_NONFINITE = 1u << 6,
  ST_PCG_BREAKDOWN = 1u << 7,
  ST_CAP_HASH = 1u << 8,       // spatial-hash entry storage exceeded
};

struct DevStatus {
  unsigned flags;
  int need_row;                 // largest body-pair row seen
  int need_cand;                // largest candidate count of one body pair
  int np;                       // body pairs in the current list
  int nact;                     // active barrier terms
  int nfr;                      // lagged friction terms
  int nfp;                      // friction body pairs
  int pad;
  int nlarge;                   // bodies handled outside the spatial hash
  int nent;                     // spatial-hash entries
  int pad2[2];
  unsigned long long need_pairs;  // body pairs needed
  unsigned long long need_act;    // active terms needed
  unsigned long long need_misc;   // other scans
  unsigned long long toi_bits;  // min time of impact (bits of a positive double)
  unsigned long long step_bits; // max vertex step length (bits of a positive double)
  unsigned long long n_cand;    // candidates of the last enumeration
  unsigned long long bar_terms[4];  // barrier terms evaluated, by reduced dimension m = 1, 2, 3
  double scal[10];              // PCG scalars: 0 rz, 1 pAp, 2 rr, 3 rr0, 4 alpha, 5 beta, 6 done,
                                // 7 iterations, 8 rz of the previous iteration
  double energy[8];             // 0 total, 1 inertia, 2 ortho, 3 barrier, 4 friction
  int bar_cnt[4];               // active terms by working dimension 3, 6, 9 (classification pass)
  unsigned long long jac[3];    // Jacobi sweeps FP32, FP64, terms at the FP64 sweep cap (cumulative)
  int bh_fix;                   // body blocks that took the orthogonality surrogate (not positive definite)
  int pad3;
  // culling of the enumeration (cumulative): primitive pairs of the body
  // pairs, pairs left after restricting each side to the other body's box,
  // candidates passing the exact primitive box test
  unsigned long long cull[3];
  // per-island line search (k_island.cu): islands still pending after the
  // last acceptance pass, islands, islands past the halving cap, the largest
  // halving count of any island
  int ls_pending, n_islands, ls_failed, ls_halv_max;
  int n_clusters;               // preconditioner clusters of the current body-pair list
  int clu_fail;                 // clusters whose Cholesky factorisation failed (block-Jacobi used)
  int ls_rounds;                // halving rounds run by the device-side line-search loop
  int n_ework;                  // entries of the (body pair, chunk) work list
  int n_large_asm;              // body pairs assembled by a whole block (many terms)
  int pad5;
};

// ---- small device helpers shared by the kernel files -----------------------
#ifdef __CUDACC__
__device__ __forceinline__ void set_flag(DevStatus* st, unsigned f) { atomicOr(&st->flags, f); }

// vertices of a pair: point-triangle (vertex i, triangle j) or edge-edge
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

// largest p with off[p] <= f (off has n+1 entries, nondecreasing)
__device__ __forceinline__ int owner(const int* off, int n, int f) {
  int lo = 0, hi = n;
  while (hi - lo > 1) {
    int mid = (lo + hi) >> 1;
    if (off[mid] <= f) lo = mid;
    else hi = mid;
  }
  return lo;
}
#endif

// ---- allocation -------------------------------------------------------------
struct Alloc {
  abd_allocator a{};
  bool custom = false;
  cudaStream_t stream = nullptr;
  void* get(size_t bytes);
  void put(void* p);
};

template <typename T>
struct Buf {
  T* p = nullptr;
  size_t cap = 0;  // elements
};

// lagged friction record (one per friction term)
struct FricRec {
  int v[4];
  int a, b;        // body pair (a < b)
  double gam[4], n[3], r[3], mu_lambda;
  int kind, i, j, type;
};

// ---- optional per-kernel timing (CUDA events on the scene's stream) -----------
enum ProfSlot {
  PF_ENUM = 0, PF_ACTIVE, PF_BARRIER, PF_FRICTION, PF_ASSEMBLE, PF_BODY, PF_SPMV, PF_ROWS, PF_DENSE, PF_COUNT
};

struct Prof {
  bool on = false;
  std::vector<cudaEvent_t> pool;
  size_t used = 0;
  struct Slot {
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev;
    long launches = 0;
    double bytes = 0;  // algorithmic bytes of the recorded launches
    double flops = 0;  // algorithmic flops of the recorded launches (where known on the host)
  } slot[PF_COUNT];
  unsigned long long bar_terms0[4] = {0, 0, 0, 0};  // counters when profiling started
};

// ---- scene ------------------------------------------------------------------
constexpr int kClusterMax = 16;      // largest preconditioner cluster (bodies)
constexpr int kClusterDefault = 12;  // default run length (abd_tuning.cluster_max = 0)

struct Scene {
  abd_params prm{};
  int nb = 0, nv = 0, nt = 0, ne = 0, ndyn = 0;
  double newton_tol = 0;
  bool fp32_proj = false;  // barrier projection from the FP32 eigenbasis (mixed precision)

  // CUDA graphs of the two fixed launch sequences of a Newton iteration
  // (captured on a private stream, replayed on the scene's stream, captured
  // again whenever a buffer has been reallocated)
  struct Segment {
    cudaGraphExec_t exec = nullptr;
    long gen = -1;
    long nlaunch = 0;
    // a device-side while loop inside the segment (the line search's
    // halving rounds): its condition, its body graph while the segment is
    // being built, the launches of one pass of the body
    bool has_loop = false;
    cudaGraphConditionalHandle loop_cond = 0;
    cudaGraph_t loop_body = nullptr;
    long loop_nlaunch = 0;
  };
  std::vector<int> perm_tmp;     // host scratch of the cluster build
  Segment* capturing = nullptr;  // the segment being captured (run_segment)
  bool loop_graphs = true;       // device-side loops inside segments (off after a failed build)
  long gen = 0;  // bumped on every buffer (re)allocation
  bool graphs = true;
  cudaStream_t cap_stream = nullptr;
  // per Newton iteration: the system up to the assembled blocks (head), the
  // preconditioner and the PCG solve (tail; the host builds the clusters
  // while the head runs), the trial step and line search
  Segment seg_head[2], seg_tail[2], seg_trial;
  Alloc alloc;
  cudaStream_t stream = nullptr;
  // two side streams for the independent branches of a Newton iteration
  // (fork / join by events; inside a capture they become graph branches)
  cudaStream_t side[2] = {nullptr, nullptr};
  cudaEvent_t ev_fork[5] = {}, ev_join[5] = {};
  int device = 0;    // CUDA device the scene was created on
  int grid_div = 1;  // divisor of the device-sized grids (abd_tuning)
  int cluster_max = kClusterDefault;  // bodies per preconditioner cluster (abd_tuning)
  std::string err;

  // topology and body constants
  Buf<double4> xbar;   // nv (w unused)
  Buf<double> l2e;     // ne: squared rest length of every edge (edge-edge mollifier)
  Buf<int> vbody, tri, edge, vbeg, tbeg, ebeg;
  Buf<uint8_t> is_static;
  Buf<double> mass10;  // nb*10: rho*vol, rho*m1[3], rho*S[xx,xy,xz,yy,yz,zz]
  Buf<double> vol, kappa_b, density;

  // state
  Buf<double> q, qdot, qt, qtilde, dq, qtrial, qsave, qdotsave;
  Buf<double4> x, dx, x1, xt;
  Buf<double> bbox;    // nb*6
  Buf<float> bbox32;   // nb*6, the same boxes rounded outward to FP32 (prefilter)

  // spatial hash over body boxes
  double cell_h = 1.0;         // cell edge
  int hash_T = 1;              // slots (power of two)
  Buf<int> hcount, hoff, large, large_pos, large_list, slot_cnt, slot_off, entries;

  // body pairs
  int maxn = 0;        // neighbours per row
  Buf<int> nbr, ncount, rowoff;  // rows
  Buf<int2> P;                   // body pairs (a, b), a < b, row-major
  Buf<int> in_off, in_cnt, in_list;   // incoming lists (pairs whose b is the body)

  // candidates / actives per body pair
  int maxc = 0;
  Buf<int2> cand;      // np*maxc: (i | kind << 31, j)
  Buf<double2> cdl;    // np*maxc: swept candidates' distance at the iterate and its rate bound (CCD pass)
  Buf<int> ccount;
  Buf<int4> act;       // np*maxc: (i | kind << 31, j, type, unused)
  Buf<int> acount, aoff;
  Buf<double> act_d2;  // np*maxc
  Buf<unsigned> amask; // np*chunks: active-membership masks of 32-candidate chunks

  // per-term energy and derivatives: E, g12, H78 (kTermStride doubles) and
  // the term's four vertices
  Buf<double> term;    // barrier terms
  Buf<int4> termv;
  Buf<int> tmeta;      // barrier terms: kind | type << 1 | mollified << 5
  Buf<double> teps;    // barrier terms: edge-edge mollifier threshold
  Buf<double> td2;     // barrier terms: canonical squared distance
  Buf<int> tlist;      // barrier terms bucketed by working dimension 3, 6, 9 (3 x capacity)
  Buf<double> fterm;   // friction terms
  Buf<int4> ftermv;
  Buf<double> Epair;   // energy-only pass: barrier energy per (body pair, chunk of 32 candidates)
  Buf<int> ework;      // the (body pair, chunk) slots p * chunks + c that hold candidates (line search)
  Buf<int> large_asm;  // body pairs with many terms, assembled a block per pair

  // friction
  Buf<FricRec> fric;
  Buf<int2> fpairs;    // friction body pairs, sorted
  Buf<int> fpoff;      // nfp+1 ranges into fric
  Buf<int> flagbuf, posbuf;  // scan scratch (body-pair sized)

  // assembly
  Buf<double> pblk;    // np * (3*144 + 24 + 2): Hab, Dlo, Dhi, glo, ghi, Eb, Ef
  Buf<double> Db, gb, Eb;   // body terms
  Buf<double> D, g, Pinv;   // assembled diagonal, gradient, preconditioner
  Buf<double> red;     // reduction scratch
  int dense_n = 0;           // order of the dense system (0: PCG)
  Buf<double> dense, dense_dinv;  // dense_n^2 matrix / factor, reciprocal pivots
  Buf<long long> scan_part;  // tile sums of the two-phase scan

  // contact islands (k_island.cu): union-find parents, labels (smallest body
  // id of the island), per-island CCD bound (bits), exact energy accumulators
  // (16 per island: 4 digits each of the positive and negative parts of E at
  // the iterate, then of the trial), line-search
  // state (accepted, halvings) and step
  Buf<int> uf, isl, isl_state;
  Buf<unsigned long long> isl_toi, isl_step, isl_E;
  Buf<double> isl_alpha;

  // PCG: residual, preconditioned residual, two alternating directions, H p,
  // chunk partial sums, the solve kernel's grid-barrier words
  Buf<double> r, z, pv, pv2, Ap, part;
  Buf<unsigned> pcg_bar;
  // mixed-precision solve (precision = 1): FP32 copies of the diagonal, the
  // inverse diagonal and the upper pair blocks, the FP64 right-hand side, and
  // six FP32 vectors (r, z, two directions, H p, the inner solution)
  bool pcg_mixed = false;
  Buf<float> D32, Minv32, H32, vf;
  Buf<double> rhs64;
  // preconditioner clusters (k_pcg.cu): the dynamic bodies of every contact
  // island in body order, cut into runs of at most kClusterMax bodies; per
  // cluster its members (c_off into c_perm), per body its cluster and local
  // index, per cluster the offset of its dense Cholesky factor in c_fac and a
  // flag (factorisation succeeded); host staging of the island labels and of
  // the cluster arrays
  int nclu = 0;
  Buf<int> c_perm, c_off, c_of, c_loc, c_ok;
  Buf<long long> c_foff;
  Buf<double> c_fac;
  int* isl_host = nullptr;
  int* clu_host = nullptr;       // c_perm | c_off | c_of | c_loc | count, then c_foff (long long)
  std::vector<int2> pairs_host;  // the body pairs (cluster adjacency)
  std::vector<uint8_t> is_static_host;
  bool cluster_attr_set = false;
  int num_sms = 152;          // multiprocessors of the scene's device
  int pcg_blocks_per_sm = 0;  // co-resident blocks of the solve kernel (0: not yet queried)

  long nlaunch = 0;              // kernels launched by the library
  long cand_last = 0;            // candidates of the last enumeration
  Prof prof;

  DevStatus* st = nullptr;       // device
  DevStatus* st_host = nullptr;  // pinned mirror
  long last_np = 0;
  bool have_hess = false;
};

constexpr int kTermStride = 91;

// algorithmic FP64 operations of one barrier term by reduced dimension m.
// m = 1: derivatives, closed-form clamp, 91 outputs.  m = 2, 3: the n x n
// Hessian entries, the Gram congruence, two FP64 basis updates (Newton-Schulz
// and the change of basis, after each FP32 pass), the clamp as two products,
// the inverse congruence and the expansion to 12x12 (the FP32 passes and the
// rare FP64 sweeps are not counted)
constexpr double kBarrierFlops[4] = {0.0, 380.0, 7000.0, 22100.0};

// launch bookkeeping: count every kernel; with profiling on, bracket the
// launches of a slot with events
cudaEvent_t prof_event(Scene& s);
inline void counted(Scene& s, int n = 1) { s.nlaunch += n; }

// chunks of 32 candidate slots per body pair (energy-only pass partial sums)
inline int energy_chunks(const Scene& s) { return (s.maxc + 31) / 32; }

// run `body` on side stream k, after the work enqueued so far on the scene's
// stream (fork point f); join_side makes the scene's stream wait for it
template <typename F>
void on_side(Scene& s, int k, int f, F body) {
  cudaEventRecord(s.ev_fork[f], s.stream);
  cudaStreamWaitEvent(s.side[k], s.ev_fork[f], 0);
  cudaStream_t main = s.stream;
  s.stream = s.side[k];
  body();
  s.stream = main;
}
inline void join_side(Scene& s, int k, int f) {
  cudaEventRecord(s.ev_join[f], s.side[k]);
  cudaStreamWaitEvent(s.stream, s.ev_join[f], 0);
}

// grid of a kernel that grid-strides over a count held on the device:
// per_sm blocks on each of the 152 SMs, divided by the scene's grid_div
constexpr int kNumSMs = 152;
// ranges per energy component in the two-stage energy reduction
constexpr int kEnergyParts = 256;
inline int sm_grid(const Scene& s, int per_sm) {
  const int g = kNumSMs * per_sm / s.grid_div;
  return g < 1 ? 1 : g;
}
struct ProfScope {
  Scene& s;
  int slot;
  cudaEvent_t a = nullptr;
  double bytes, flops;
  ProfScope(Scene& sc, int sl, double b = 0, double f = 0) : s(sc), slot(sl), bytes(b), flops(f) {
    if (s.prof.on) {
      a = prof_event(s);
      cudaEventRecord(a, s.stream);
    }
  }
  ~ProfScope() {
    if (a) {
      cudaEvent_t e = prof_event(s);
      cudaEventRecord(e, s.stream);
      s.prof.slot[slot].ev.emplace_back(a, e);
      s.prof.slot[slot].launches++;
      s.prof.slot[slot].bytes += bytes;
      s.prof.slot[slot].flops += flops;
    }
  }
};
constexpr int kBlkStride = 3 * 144 + 24 + 2;

// ---- launchers (k_system.cu) -----------------------------------------------
void launch_mass_moments(Scene& s);
void launch_edge_rest(Scene& s);
void launch_predictor(Scene& s);
// pending_only: the line search's trial positions, only for bodies of
// pending islands
void launch_transform(Scene& s, const double* q, double4* x, bool pending_only = false);
void launch_transform_dq(Scene& s, const double* dq);   // dx = J dq, x1 = x + dx
void launch_body_boxes(Scene& s, bool swept);
void launch_body_pairs(Scene& s);                       // rows -> P (uses friction pairs)
void launch_incoming(Scene& s);
void launch_assemble(Scene& s);
// pending_only: line-search rounds, only the bodies / pairs / records of the
// islands whose step is not yet accepted
void launch_body_terms(Scene& s, const double* q, bool hess, bool project = true, bool pending_only = false);
void launch_adjoint_rhs(Scene& s, const double* gq, const double* gqd, double* rhs);
void launch_adjoint_out(Scene& s, const double* q, const double* lam, double* gq, double* gqd, double* gkappa);
void launch_gather(Scene& s);
void launch_precond(Scene& s);
void launch_energy_total(Scene& s, bool with_pairs);
// block-Jacobi PCG (k_pcg.cu): r = sign * rhs, x = 0, z, p and the partial
// sums of the start (launch_pcg_init); the whole solve in one persistent
// launch (launch_pcg_solve); its outcome from the status word read back
// (pcg_result: iterations, -1 at the cap, -2 breakdown); run_pcg does all
// three and synchronises
void launch_pcg_init(Scene& s, const double* rhs, double sign, double* xout);
void launch_pcg_solve(Scene& s, double* xout, int max_iter, double rel_tol);
int pcg_result(Scene& s, double* rel_res);
void pcg_account(Scene& s, int its);
// indefinite: the dense branch factors by signed Cholesky (the adjoint's
// unprojected system); the PCG branch is unchanged
int run_pcg(Scene& s, const double* rhs, double* xout, int max_iter, double rel_tol, double* rel_res,
            bool indefinite = false);
void launch_pcg_fp32_blocks(Scene& s);  // mixed precision: FP32 copies of the blocks
// factors of the preconditioner clusters (after the assembly)
void launch_cluster_factor(Scene& s);
double pcg_iter_bytes(const Scene& s, long np);
double pcg_iter_flops(const Scene& s, long np);
// dense direct solve (small scenes): order of the padded matrix, 0 if off
constexpr int kDenseMaxOrder = 3072;
int dense_order(int nb, int max_dofs);
// indefinite: signed Cholesky (negative pivots accepted), for the adjoint
void launch_dense_solve(Scene& s, const double* rhs, double* x, bool indefinite = false);
// the preconditioner (inverse diagonal blocks), then the PCG start on H dx = -g
void launch_precond_start(Scene& s, double* xout);
void launch_reset_toi(Scene& s);
void launch_max_step(Scene& s);
void launch_trial(Scene& s, double alpha, bool alpha_from_ccd);
void launch_finish_step(Scene& s);
// exclusive scan of cnt[0..*n_dev) into off[0..*n_dev] (off[n] = total), total
// also to *total_dev; if the total exceeds cap, flag_bit is raised.
void launch_scan(Scene& s, const int* cnt, int* off, const int* n_dev, int* total_dev, long cap, unsigned flag_bit,
                 unsigned long long* need);
void launch_fpairs(Scene& s);
void launch_negate(Scene& s, const double* in, double* out, long n);

// ---- launchers (k_contact.cu) ------------------------------------------------
void launch_enumerate(Scene& s, bool swept, bool ccd);
void launch_active(Scene& s, const double4* x);
void launch_barrier(Scene& s, int project, long cap);
void launch_friction_lag(Scene& s);
void launch_friction_eval(Scene& s, const double4* x, bool derivs, bool pending_only = false);
void launch_pair_energy(Scene& s, const double4* x, bool pending_only = false);  // energy only, over candidates
// the (body pair, chunk) slots that hold candidates, for every pass over
// the candidates (CCD, active set, the line search's energy passes); part of
// every enumeration
void launch_energy_worklist(Scene& s);

// ---- launchers (k_island.cu) -------------------------------------------------
void launch_islands(Scene& s);                 // labels of the current body-pair list
void launch_island_energy(Scene& s, int which); // 0: E at the iterate from the terms; 1: the trial's
void launch_island_start(Scene& s);            // each island's step = its CCD bound
// qtrial = q + alpha_island dq (pending_only: the halving rounds)
void launch_island_trial(Scene& s, bool pending_only = false);
// accept or halve each pending island; reset: clear the counts first (else a
// preceding launch_ls_round_begin has)
void launch_island_accept(Scene& s, bool reset = true);
void launch_ls_round_begin(Scene& s);          // clear the counts, count the round
// sets the loop condition: islands pending, none failed, no zero distance,
// fewer than max_rounds rounds; first: the evaluation before the loop (clears
// the round count)
void launch_ls_condition(Scene& s, cudaGraphConditionalHandle h, int max_rounds, bool first);

}  // namespace abd
