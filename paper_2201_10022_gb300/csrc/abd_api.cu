// C ABI of the affine-body library and the host driver of the time step:
// Newton iterations on the incremental potential (Sec. 4) with the linear
// solve, the CCD step bound (Sec. 4.1) and a backtracking line search, all
// enqueued on the scene's stream; the host reads the device status word
// once per Newton iteration and once per line-search trial.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <numeric>
#include <thread>
#include <vector>

#include "abd_internal.cuh"

namespace abd {

cudaEvent_t prof_event(Scene& s) {
  if (s.prof.used == s.prof.pool.size()) {
    cudaEvent_t e;
    cudaEventCreate(&e);
    s.prof.pool.push_back(e);
  }
  return s.prof.pool[s.prof.used++];
}

void* Alloc::get(size_t bytes) {
  if (bytes == 0) bytes = 16;
  if (custom) return a.alloc(bytes, (void*)stream, a.ctx);
  void* p = nullptr;
  if (cudaMalloc(&p, bytes) != cudaSuccess) return nullptr;
  return p;
}

void Alloc::put(void* p) {
  if (!p) return;
  if (custom) a.free(p, (void*)stream, a.ctx);
  else cudaFree(p);
}

namespace {

struct OomError {};

template <typename T>
void grow(Scene& s, Buf<T>& b, size_t n) {
  if (b.cap >= n && b.p) return;
  if (b.p) {
    cudaStreamSynchronize(s.stream);
    s.alloc.put(b.p);
  }
  b.p = (T*)s.alloc.get(sizeof(T) * (n ? n : 1));
  b.cap = n;
  ++s.gen;
  if (!b.p) throw OomError{};
}

template <typename T>
void release(Scene& s, Buf<T>& b) {
  s.alloc.put(b.p);
  b.p = nullptr;
  b.cap = 0;
  ++s.gen;
}

// buffers whose size follows the body-pair capacity, the candidates per pair
// and the active-term capacity
void size_pair_buffers(Scene& s, size_t pcap) {
  grow(s, s.P, pcap);
  grow(s, s.ccount, pcap);
  grow(s, s.acount, pcap);
  grow(s, s.aoff, pcap + 1);
  grow(s, s.in_list, pcap);
  grow(s, s.pblk, pcap * kBlkStride);
  grow(s, s.fpairs, pcap);
  grow(s, s.fpoff, pcap + 1);
  grow(s, s.flagbuf, pcap);
  if (s.prm.precision == 1) grow(s, s.H32, pcap * 144);
  grow(s, s.posbuf, pcap + 1);
  grow(s, s.Epair, pcap * (size_t)energy_chunks(s));
  grow(s, s.ework, pcap * (size_t)energy_chunks(s));
  grow(s, s.large_asm, pcap);
  grow(s, s.cand, pcap * (size_t)s.maxc);
  grow(s, s.cdl, pcap * (size_t)s.maxc);
  grow(s, s.act, pcap * (size_t)s.maxc);
  grow(s, s.act_d2, pcap * (size_t)s.maxc);
  grow(s, s.amask, pcap * (size_t)energy_chunks(s));
}

void size_term_buffers(Scene& s, size_t tcap) {
  grow(s, s.term, tcap * kTermStride);
  grow(s, s.termv, tcap);
  grow(s, s.tmeta, tcap);
  grow(s, s.teps, tcap);
  grow(s, s.td2, tcap);
  grow(s, s.tlist, 3 * tcap);
  grow(s, s.fric, tcap);
  grow(s, s.fterm, tcap * kTermStride);
  grow(s, s.ftermv, tcap);
}

size_t term_cap(const Scene& s) { return s.termv.cap; }

void reset_status(Scene& s) {
  // clear flags and per-pass counters, keep np / nact / nfr / nfp
  DevStatus h;
  memset(&h, 0, sizeof(h));
  cudaMemcpyAsync(s.st_host, s.st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s.stream);
  cudaStreamSynchronize(s.stream);
  h = *s.st_host;
  h.flags = 0;
  h.need_row = h.need_cand = 0;
  h.need_pairs = h.need_act = h.need_misc = 0;
  double one = 1.0;
  memcpy(&h.toi_bits, &one, 8);
  h.step_bits = 0;
  h.n_cand = 0;
  *s.st_host = h;
  cudaMemcpyAsync(s.st, s.st_host, sizeof(DevStatus), cudaMemcpyHostToDevice, s.stream);
}

void read_status(Scene& s) {
  cudaMemcpyAsync(s.st_host, s.st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s.stream);
  cudaStreamSynchronize(s.stream);
}

void set_counter(Scene& s, int* field, int v) { cudaMemcpyAsync(field, &v, sizeof(int), cudaMemcpyHostToDevice, s.stream); }

double bits_to_double(unsigned long long b) {
  double d;
  memcpy(&d, &b, 8);
  return d;
}

// grow every buffer whose capacity flag is raised; returns true if any grew
bool handle_capacity(Scene& s) {
  const DevStatus& h = *s.st_host;
  bool grew = false;
  if (h.flags & ST_CAP_ROWS) {
    s.maxn = std::max(2 * s.maxn, h.need_row + 16);
    grow(s, s.nbr, (size_t)s.nb * s.maxn);
    grew = true;
  }
  size_t pcap = s.P.cap;
  if (h.flags & ST_CAP_PAIRS) {
    pcap = std::max<size_t>(2 * pcap, (size_t)(1.5 * (double)std::max(h.need_pairs, h.need_misc)) + 64);
    grew = true;
  }
  if (h.flags & ST_CAP_CANDS) {
    s.maxc = std::max(2 * s.maxc, h.need_cand + 64);
    release(s, s.cand);
    release(s, s.act);
    release(s, s.act_d2);
    grew = true;
  }
  if (grew) size_pair_buffers(s, pcap);
  if (h.flags & ST_CAP_ACTIVE) {
    size_term_buffers(s, std::max<size_t>(2 * term_cap(s), (size_t)(1.5 * (double)h.need_act) + 64));
    grew = true;
  }
  if (h.flags & ST_CAP_HASH) {
    grow(s, s.entries, std::max<size_t>(2 * s.entries.cap, (size_t)(1.5 * (double)h.need_misc) + 64));
    grew = true;
  }
  return grew;
}

abd_status check_cuda(Scene& s) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    s.err = std::string("CUDA error: ") + cudaGetErrorString(e);
    return ABD_ERR_CUDA;
  }
  return ABD_OK;
}

// Preconditioner clusters from the island labels in s.isl_host (and the
// body pairs, read here): the dynamic bodies of each island in breadth-first
// order over the island's dynamic body pairs (from its smallest body id,
// neighbours in pair order), cut into consecutive runs of at most
// kClusterMax bodies, so that a cluster is a compact piece of the contact
// graph (a stack of bodies rather than a row of neighbours).  Deterministic;
// uploaded with the cluster count; the factor pool grows when needed.
// the body pairs of the current list to the host (after a synchronisation:
// s.st_host holds their count); build_clusters_host uses them and the island
// labels in s.isl_host
void fetch_pairs_host(Scene& s) {
  const long np = std::max(0, s.st_host->np);
  s.pairs_host.resize(np);
  if (np) cudaMemcpy(s.pairs_host.data(), s.P.p, sizeof(int2) * np, cudaMemcpyDeviceToHost);
}

void build_clusters_host(Scene& s) {
  const int nb = s.nb;
  int* perm = s.clu_host;
  int* off = perm + nb;
  int* cof = off + nb + 1;
  int* loc = cof + nb;
  int* ncl = loc + nb;
  long long* foff = reinterpret_cast<long long*>(s.clu_host + 4 * nb + 2);
  // adjacency of the dynamic bodies (pair order)
  std::vector<int> deg(nb + 1, 0), adj;
  for (const int2& e : s.pairs_host)
    if (!s.is_static_host[e.x] && !s.is_static_host[e.y]) {
      deg[e.x + 1]++;
      deg[e.y + 1]++;
    }
  for (int b = 0; b < nb; ++b) deg[b + 1] += deg[b];
  adj.resize(deg[nb]);
  {
    std::vector<int> fill(deg.begin(), deg.end() - 1);
    for (const int2& e : s.pairs_host)
      if (!s.is_static_host[e.x] && !s.is_static_host[e.y]) {
        adj[fill[e.x]++] = e.y;
        adj[fill[e.y]++] = e.x;
      }
  }
  // breadth-first order of each island from its label (its smallest body)
  std::vector<char> seen(nb, 0);
  int nd = 0;
  for (int b = 0; b < nb; ++b) {
    cof[b] = -1;
    loc[b] = 0;
  }
  std::vector<int> island_start;
  for (int b = 0; b < nb; ++b) {
    if (s.is_static_host[b] || s.isl_host[b] != b) continue;  // b is an island's label
    island_start.push_back(nd);
    int head = nd;
    perm[nd++] = b;
    seen[b] = 1;
    while (head < nd) {
      const int u = perm[head++];
      for (int k = deg[u]; k < deg[u + 1]; ++k)
        if (!seen[adj[k]]) {
          seen[adj[k]] = 1;
          perm[nd++] = adj[k];
        }
    }
  }
  island_start.push_back(nd);
  // runs of at most cluster_max bodies of each island's order; the clusters
  // are then listed largest first (stable), so that the largest ones, which
  // set the time of the factorisation and of every preconditioner
  // application, go to different SMs (the kernels stride over clusters by
  // block first); each cluster's result does not depend on its place
  std::vector<int2> runs;  // (first index into the island order, members)
  for (size_t k = 0; k + 1 < island_start.size(); ++k)
    for (int c0 = island_start[k]; c0 < island_start[k + 1]; c0 += s.cluster_max)
      runs.push_back(make_int2(c0, std::min(s.cluster_max, island_start[k + 1] - c0)));
  std::stable_sort(runs.begin(), runs.end(), [](const int2& u, const int2& v) { return u.y > v.y; });
  s.perm_tmp.assign(perm, perm + nd);
  int nc = 0, m = 0;
  long long fo = 0;
  for (const int2& r : runs) {
    const int n = r.y;
    off[nc] = m;
    foff[nc] = fo;
    if (n >= 2) fo += (long long)(12 * n) * (12 * n + 1) / 2;
    for (int i = 0; i < n; ++i) {
      const int b = s.perm_tmp[r.x + i];
      perm[m + i] = b;
      cof[b] = nc;
      loc[b] = i;
    }
    m += n;
    ++nc;
  }
  off[nc] = nd;
  foff[nc] = fo;
  *ncl = nc;
  s.nclu = nc;
  if ((size_t)fo > s.c_fac.cap) grow(s, s.c_fac, std::max<size_t>((size_t)fo, 2 * s.c_fac.cap));
  cudaMemcpyAsync(s.c_perm.p, perm, sizeof(int) * nb, cudaMemcpyHostToDevice, s.stream);
  cudaMemcpyAsync(s.c_off.p, off, sizeof(int) * (nc + 1), cudaMemcpyHostToDevice, s.stream);
  cudaMemcpyAsync(s.c_of.p, cof, sizeof(int) * nb, cudaMemcpyHostToDevice, s.stream);
  cudaMemcpyAsync(s.c_loc.p, loc, sizeof(int) * nb, cudaMemcpyHostToDevice, s.stream);
  cudaMemcpyAsync(s.c_foff.p, foff, sizeof(long long) * (nc + 1), cudaMemcpyHostToDevice, s.stream);
  cudaMemcpyAsync(&s.st->n_clusters, ncl, sizeof(int), cudaMemcpyHostToDevice, s.stream);
}

// islands of the current body-pair list, their labels to the host, and the
// preconditioner clusters built from them (synchronises the stream)
void prepare_clusters(Scene& s) {
  launch_islands(s);
  cudaMemcpyAsync(s.isl_host, s.isl.p, sizeof(int) * s.nb, cudaMemcpyDeviceToHost, s.stream);
  cudaMemcpyAsync(s.st_host, s.st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s.stream);
  cudaStreamSynchronize(s.stream);
  fetch_pairs_host(s);
  build_clusters_host(s);
}

// ---- pipeline stages --------------------------------------------------------

// body pairs and their candidate pairs at s.x (static) or over s.x -> s.x1
// (swept, with additive CCD when ccd is set)
void broad_and_enumerate(Scene& s, bool swept, bool ccd) {
  cudaMemsetAsync(&s.st->n_cand, 0, sizeof(unsigned long long), s.stream);
  launch_body_boxes(s, swept);
  launch_body_pairs(s);
  if (ccd) launch_islands(s);  // the CCD bound is taken per contact island
  launch_enumerate(s, swept, ccd);
}

// actives, terms, assembly and preconditioner at positions s.x (from q):
// the body terms and the incoming-pair lists (which need only q and the
// body pairs) and the friction terms (only x) run beside the active set and
// the barrier terms, and join before the assembly
// head: everything up to the assembled blocks and the gathered gradient;
// tail: the preconditioner (with the PCG's start when newton_x is given) and
// the energy total.  eval_system runs both.
void eval_system_head(Scene& s, const double* q, int project) {
  on_side(s, 0, 0, [&]() {
    launch_body_terms(s, q, true, project != 0);
    launch_incoming(s);
  });
  on_side(s, 1, 1, [&]() { launch_friction_eval(s, s.x.p, true); });
  launch_active(s, s.x.p);
  launch_scan(s, s.acount.p, s.aoff.p, &s.st->np, &s.st->nact, (long)term_cap(s), ST_CAP_ACTIVE, &s.st->need_act);
  launch_barrier(s, project, (long)term_cap(s));
  join_side(s, 0, 0);
  join_side(s, 1, 1);
  launch_assemble(s);
  launch_gather(s);
}

void eval_system_tail(Scene& s, double* newton_x) {
  if (newton_x)  // and the PCG's start on H dx = -g
    launch_precond_start(s, newton_x);
  else
    launch_precond(s);
  launch_energy_total(s, true);
}

void eval_system(Scene& s, const double* q, int project, double* newton_x = nullptr) {
  eval_system_head(s, q, project);
  eval_system_tail(s, newton_x);
}

// energy only at positions s.xt (from qv), over the stored candidates; the
// body and friction terms run beside the pair energies.  In the per-island
// line search only the islands whose step is not yet accepted are evaluated
// (their island sums are all that is read) and the scene totals are skipped.
void eval_energy(Scene& s, const double* qv, bool line_search = false) {
  on_side(s, 0, 2, [&]() { launch_body_terms(s, qv, false, true, line_search); });
  on_side(s, 1, 3, [&]() { launch_friction_eval(s, s.xt.p, false, line_search); });
  launch_pair_energy(s, s.xt.p, line_search);
  join_side(s, 0, 2);
  join_side(s, 1, 3);
  if (!line_search) launch_energy_total(s, false);
}

// lag friction at q^t: proximity pairs at x(q^t), one record per active pair
void lag_friction(Scene& s) {
  set_counter(s, &s.st->nfp, 0);
  set_counter(s, &s.st->nfr, 0);
  if (!(s.prm.mu > 0.0)) return;
  launch_transform(s, s.qt.p, s.x.p);
  broad_and_enumerate(s, false, false);
  launch_active(s, s.x.p);
  launch_scan(s, s.acount.p, s.aoff.p, &s.st->np, &s.st->nact, (long)term_cap(s), ST_CAP_ACTIVE, &s.st->need_act);
  launch_friction_lag(s);
  launch_fpairs(s);
}

abd_status flags_to_status(Scene& s, unsigned f) {
  if (f & ST_INTERSECT) {
    s.err = "a contact pair reached zero distance";
    return ABD_ERR_INITIAL_INTERSECTION;
  }
  if (f & ST_NONFINITE) {
    s.err = "non-finite value in the state or the system";
    return ABD_ERR_NONFINITE;
  }
  if (f & ST_CCD_MAXITER) {
    s.err = "additive CCD iteration cap reached";
    return ABD_ERR_CCD_MAXITER;
  }
  return ABD_OK;
}

const unsigned kCapFlags = ST_CAP_ROWS | ST_CAP_CANDS | ST_CAP_PAIRS | ST_CAP_ACTIVE | ST_CAP_HASH;

// run fn until no capacity flag is raised (buffers grow in between)
template <typename F>
abd_status with_capacity(Scene& s, F fn) {
  for (int attempt = 0; attempt < 12; ++attempt) {
    reset_status(s);
    abd_status r = fn();
    if (r != ABD_OK && r != ABD_ERR_CAPACITY) return r;
    read_status(s);
    if (abd_status c = check_cuda(s)) return c;
    if (!(s.st_host->flags & kCapFlags)) return r;
    handle_capacity(s);
  }
  s.err = "buffer capacity did not converge";
  return ABD_ERR_CAPACITY;
}

// candidates of the enumeration that produced the current candidate set
long cand_total(Scene& s) { return s.cand_last; }

// Run a fixed launch sequence: as a CUDA graph (captured on a private stream
// the first time and after any buffer reallocation, then replayed on the
// scene's stream), or directly while profiling or if capture is unavailable.
// The sequence must not read device results on the host.  A sequence may hold
// one device-side while loop: the body calls loop_node() where it goes, and
// loop() enqueues one pass of the loop's body, ending with the launch that
// sets the loop's condition (Scene::Segment::loop_cond).  Returns true if the
// loop ran on the device; otherwise (direct launches, or graph conditionals
// unavailable) the caller runs it from the host.
template <typename F, typename L>
bool run_segment_loop(Scene& s, Scene::Segment& g, F body, L loop) {
  if (!s.graphs || s.prof.on) {
    body();
    return false;
  }
  if (!g.exec || g.gen != s.gen) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    g.exec = nullptr;
    if (!s.cap_stream && cudaStreamCreateWithFlags(&s.cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      s.graphs = false;
      body();
      return false;
    }
    cudaStream_t user = s.stream;
    const long n0 = s.nlaunch;
    cudaGraph_t gr = nullptr;
    g.has_loop = false;
    g.loop_body = nullptr;
    g.loop_nlaunch = 0;
    bool ok = cudaStreamBeginCapture(s.cap_stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
      s.stream = s.cap_stream;
      s.capturing = &g;
      body();
      s.capturing = nullptr;
      s.stream = user;
      ok = cudaStreamEndCapture(s.cap_stream, &gr) == cudaSuccess && gr;
    }
    g.nlaunch = s.nlaunch - n0;
    // the loop's body, captured into the conditional node's body graph
    if (ok && g.has_loop) {
      ok = cudaStreamBeginCaptureToGraph(s.cap_stream, g.loop_body, nullptr, nullptr, 0,
                                         cudaStreamCaptureModeThreadLocal) == cudaSuccess;
      if (ok) {
        const long n1 = s.nlaunch;
        s.stream = s.cap_stream;
        loop();
        s.stream = user;
        cudaGraph_t lb = nullptr;
        ok = cudaStreamEndCapture(s.cap_stream, &lb) == cudaSuccess;
        g.loop_nlaunch = s.nlaunch - n1;
      }
    }
    s.nlaunch = n0;
    if (ok) ok = cudaGraphInstantiate(&g.exec, gr, 0) == cudaSuccess;
    if (gr) cudaGraphDestroy(gr);
    if (!ok) {  // nothing of the captured body ran
      cudaGetLastError();
      g.exec = nullptr;
      if (g.has_loop && s.loop_graphs) {  // again without the device-side loop
        s.loop_graphs = false;
        g.has_loop = false;
        return run_segment_loop(s, g, body, loop);
      }
      s.graphs = false;  // run it directly from now on
      body();
      return false;
    }
    g.gen = s.gen;
  }
  cudaGraphLaunch(g.exec, s.stream);
  s.nlaunch += g.nlaunch;
  return g.has_loop;
}

template <typename F>
void run_segment(Scene& s, Scene::Segment& g, F body) {
  run_segment_loop(s, g, body, []() {});
}

// Inside a segment's body while it is captured: a while-loop node at this
// point of the sequence, entered while the condition (set by a launch just
// before it, and by the last launch of each pass) is non-zero.  Outside a
// capture, or if graph conditionals are unavailable, nothing: the caller's
// host loop runs the passes.
void loop_node(Scene& s, int max_rounds) {
  Scene::Segment* g = s.capturing;
  if (!g || !s.loop_graphs) return;
  cudaStreamCaptureStatus cs;
  cudaGraph_t G = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  const cudaGraphEdgeData* ed = nullptr;
  size_t nd = 0;
  cudaGraphConditionalHandle h;
  if (cudaStreamGetCaptureInfo(s.stream, &cs, nullptr, &G, &deps, &ed, &nd) != cudaSuccess ||
      cs != cudaStreamCaptureStatusActive || cudaGraphConditionalHandleCreate(&h, G, 0, 0) != cudaSuccess) {
    cudaGetLastError();
    s.loop_graphs = false;
    return;
  }
  launch_ls_condition(s, h, max_rounds, true);
  // zero-initialised parameter block (the struct's default constructor is
  // deleted: it holds a union of node kinds)
  alignas(cudaGraphNodeParams) unsigned char raw[sizeof(cudaGraphNodeParams)];
  memset(raw, 0, sizeof(raw));
  cudaGraphNodeParams& np = *reinterpret_cast<cudaGraphNodeParams*>(raw);
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = h;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t node = nullptr;
  if (cudaStreamGetCaptureInfo(s.stream, &cs, nullptr, &G, &deps, &ed, &nd) != cudaSuccess ||
      cudaGraphAddNode(&node, G, deps, ed, nd, &np) != cudaSuccess ||
      cudaStreamUpdateCaptureDependencies(s.stream, &node, nullptr, 1, cudaStreamSetCaptureDependencies) !=
          cudaSuccess) {
    // the capture is left invalid: its end fails and the segment is built
    // again without the loop
    cudaGetLastError();
    g->has_loop = true;
    g->loop_body = nullptr;
    return;
  }
  g->has_loop = true;
  g->loop_cond = h;
  g->loop_body = np.conditional.phGraph_out[0];
}

// one implicit-Euler step from (q^t, qdot^t); on error the state is unchanged
abd_status newton_step(Scene& s, abd_step_stats* stats) {
  const size_t qb = sizeof(double) * 12 * s.nb;
  cudaMemcpyAsync(s.q.p, s.qt.p, qb, cudaMemcpyDeviceToDevice, s.stream);
  abd_step_stats loc;
  memset(&loc, 0, sizeof(loc));
  loc.toi_min = 1.0;
  launch_transform(s, s.q.p, s.x.p);
  broad_and_enumerate(s, false, false);
  prepare_clusters(s);  // the clusters of the first system
  bool clusters_due = false;
  read_status(s);
  s.cand_last = (long)s.st_host->n_cand;
  s.last_np = s.st_host->np;
  abd_status status = ABD_ERR_NEWTON_MAXITER;
  // mixed precision iterates with the FP32-basis projection; once its step
  // passes the convergence test, the test is repeated with the FP64-refined
  // projection at the same iterate, so both modes stop on the same criterion
  bool hp = s.prm.precision == 0;
  s.pcg_mixed = s.prm.precision == 1;  // FP32 blocks and inner PCG, FP64 refinement
  for (int it = 0; it < s.prm.newton_max; ++it) {
    s.fp32_proj = !hp;
    // system at q and the Newton direction H dq = -g, enqueued as one
    // sequence with the whole PCG solve (one persistent launch); the status word read
    // back at its end also carries the system's flags and energies, checked
    // before the direction is used (every kernel bounds its work by the
    // clamped counts, so an overflowed system is only discarded)
    const int pv = s.fp32_proj ? 1 : 0;
    run_segment(s, s.seg_head[pv], [&]() {
      launch_transform(s, s.q.p, s.x.p);
      eval_system_head(s, s.q.p, 1);
    });
    // the clusters of the last swept pair list, built on the host while the
    // head runs (the head reads none of the cluster buffers; their uploads
    // are queued behind it)
    if (clusters_due) {
      build_clusters_host(s);
      clusters_due = false;
    }
    run_segment(s, s.seg_tail[pv], [&]() {
      if (s.dense_n) {
        eval_system_tail(s, nullptr);
        launch_negate(s, s.g.p, s.qsave.p, 12L * s.nb);
        launch_dense_solve(s, s.qsave.p, s.dq.p);
      } else {
        eval_system_tail(s, s.dq.p);
        launch_pcg_solve(s, s.dq.p, s.prm.pcg_max, s.prm.pcg_rel_tol);
      }
      cudaMemcpyAsync(s.st_host, s.st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s.stream);
    });
    cudaStreamSynchronize(s.stream);
    double rel;
    int its = pcg_result(s, &rel);
    pcg_account(s, its);
    if (s.st_host->flags & kCapFlags) return ABD_ERR_CAPACITY;
    if (abd_status r = flags_to_status(s, s.st_host->flags)) return r;
    loc.n_active = s.st_host->nact;
    loc.candidates_tested += cand_total(s);
    loc.active_evaluated += s.st_host->nact;
    loc.n_candidates = cand_total(s);
    if (its == -2) {
      s.err = s.st_host->scal[6] == 3.0 ? "PCG grid barrier timed out" : "PCG breakdown (p.Hp <= 0)";
      return ABD_ERR_PCG_BREAKDOWN;
    }
    loc.pcg_iters += its == -1 ? s.prm.pcg_max : std::max(its, 0);
    // step length for the convergence test, then (in the same batch) the CCD
    // bound over the swept candidates and the first trial at alpha = bound;
    // the swept candidates also serve the next iteration
    // the halving rounds of the line search, while any island is pending:
    // on the device (a while loop in the segment's graph) or from the host
    const int max_rounds = s.prm.ls_max + 2;
    auto ls_round = [&](bool device) {
      if (device) launch_ls_round_begin(s);
      launch_island_trial(s, true);
      launch_transform(s, s.qtrial.p, s.xt.p, true);
      eval_energy(s, s.qtrial.p, true);
      launch_island_energy(s, 1);
      launch_island_accept(s, !device);
      if (device) launch_ls_condition(s, s.seg_trial.loop_cond, max_rounds, false);
    };
    const bool device_ls = run_segment_loop(s, s.seg_trial, [&]() {
      launch_transform_dq(s, s.dq.p);
      cudaMemsetAsync(&s.st->step_bits, 0, sizeof(unsigned long long), s.stream);
      // the step length beside the broad phase; eval_energy's join of side
      // stream 0 (queued behind it) also joins it
      on_side(s, 0, 0, [&]() { launch_max_step(s); });
      launch_reset_toi(s);
      broad_and_enumerate(s, true, true);
      // per contact island: E at q from the system's terms (before the
      // trial's energy pass overwrites the body and friction energies), the
      // step = the island's CCD bound, the first trial and its acceptance
      launch_island_energy(s, 0);
      launch_island_start(s);
      launch_island_trial(s);
      launch_transform(s, s.qtrial.p, s.xt.p, true);
      eval_energy(s, s.qtrial.p, true);
      launch_island_energy(s, 1);
      launch_island_accept(s);
      loop_node(s, max_rounds);
      cudaMemcpyAsync(s.isl_host, s.isl.p, sizeof(int) * s.nb, cudaMemcpyDeviceToHost, s.stream);
      cudaMemcpyAsync(s.st_host, s.st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s.stream);
    }, [&]() { ls_round(true); });
    cudaStreamSynchronize(s.stream);
    if (device_ls) {
      loc.ls_halvings += s.st_host->ls_rounds;
      s.nlaunch += s.seg_trial.loop_nlaunch * s.st_host->ls_rounds;
    }
    // the islands of this swept pair list are those of the next system:
    // its preconditioner clusters (built during the next system's head)
    fetch_pairs_host(s);
    clusters_due = true;
    double step = bits_to_double(s.st_host->step_bits);
    loc.last_step = step;
    if (!(step == step)) {
      s.err = "non-finite Newton step";
      return ABD_ERR_NONFINITE;
    }
    if (step <= s.newton_tol) {
      if (hp) {
        status = ABD_OK;
        break;
      }
      hp = true;  // verify with the FP64-refined projection (the swept set covers x)
      s.cand_last = (long)s.st_host->n_cand;
      s.last_np = s.st_host->np;
      continue;
    }
    loc.newton_iters++;
    s.cand_last = (long)s.st_host->n_cand;
    s.last_np = s.st_host->np;
    if (s.st_host->flags & kCapFlags) return ABD_ERR_CAPACITY;
    if (abd_status r = flags_to_status(s, s.st_host->flags & ~ST_INTERSECT)) return r;
    const double alpha = bits_to_double(s.st_host->toi_bits);  // smallest island bound
    loc.n_swept = (long)s.st_host->n_cand;
    loc.candidates_tested += (long)s.st_host->n_cand;
    loc.toi_min = std::min(loc.toi_min, alpha);
    if (alpha < 1.0) loc.ccd_limited++;
    {
      int bin = 0;
      for (double edge = 1.0; bin < 5 && alpha < edge; edge *= 0.1) ++bin;
      loc.toi_hist[bin]++;
    }
    loc.n_islands = s.st_host->n_islands;
    // line search per island: E_i(q + alpha_i dq) <= E_i(q) + slack; islands
    // that fail halve their own step and are tried again (the rounds the
    // device-side loop left, if any)
    for (int round = 0; s.st_host->ls_pending > 0 && !s.st_host->ls_failed; ++round) {
      if (s.st_host->flags & ST_INTERSECT) break;
      ls_round(false);
      read_status(s);
      loc.ls_halvings++;
    }
    if (s.st_host->flags & ST_INTERSECT) {
      s.err = "line search reached zero distance";
      return ABD_ERR_INITIAL_INTERSECTION;
    }
    loc.ls_island_halvings_max = std::max(loc.ls_island_halvings_max, s.st_host->ls_halv_max);
    if (s.st_host->ls_failed) {
      s.err = "line search did not decrease the energy";
      return ABD_ERR_LINESEARCH;
    }
    // accept the trial (a copy, not a pointer swap: the captured sequences
    // keep their buffers)
    cudaMemcpyAsync(s.q.p, s.qtrial.p, qb, cudaMemcpyDeviceToDevice, s.stream);
  }
  if (status != ABD_OK) {
    if (s.err.empty()) s.err = "Newton iteration cap reached";
    return status;
  }
  launch_finish_step(s);
  if (stats) {
    loc.kernel_launches = stats->kernel_launches;
    loc.candidates_tested += stats->candidates_tested;
    loc.active_evaluated += stats->active_evaluated;
    *stats = loc;
  }
  return ABD_OK;
}

}  // namespace
}  // namespace abd

using namespace abd;

struct abd_scene {
  Scene s;
};

extern "C" {

void abd_default_params(abd_params* p) {
  memset(p, 0, sizeof(*p));
  p->dt = 0.01;
  p->dhat = 1e-3;
  p->kappa = 1e8;
  p->gravity[2] = -9.8;
  p->mu = 0.0;
  p->eps_v = 1e-3;
  p->newton_tol = 0.0;
  p->pcg_rel_tol = 1e-4;
  p->ls_slack_rel = 1e-12;
  p->ccd_s = 0.1;
  p->newton_max = 500;
  p->pcg_max = 20000;
  p->ls_max = 30;
  p->ccd_max = 10000;
  p->precision = 0;
}

static bool grouped(const int* owner, int n, int nb, std::vector<int>& beg) {
  beg.assign(nb + 1, 0);
  int prev = 0;
  std::vector<int> cnt(nb, 0);
  for (int k = 0; k < n; ++k) {
    int b = owner[k];
    if (b < 0 || b >= nb || b < prev) return false;
    prev = b;
    cnt[b]++;
  }
  for (int b = 0; b < nb; ++b) beg[b + 1] = beg[b] + cnt[b];
  return true;
}

abd_status abd_create_scene(const abd_scene_desc* d, const abd_params* prm, const abd_allocator* alloc,
                            void* stream, abd_scene** out) {
  if (!d || !prm || !out || d->nb <= 0 || d->nv <= 0 || d->nt < 0 || d->ne < 0 || !d->xbar || !d->vbody ||
      !d->q0 || !d->qdot0 || !d->density || !d->kappa_body || !d->is_static || (d->nt && !d->tri) ||
      (d->ne && !d->edge))
    return ABD_ERR_INVALID_ARG;
  if (!(prm->dt > 0) || !(prm->dhat > 0) || !(prm->kappa > 0) || prm->newton_max <= 0 || prm->pcg_max <= 0 ||
      prm->ls_max < 0 || prm->ccd_max <= 0 || !(prm->ccd_s > 0 && prm->ccd_s < 1) || (prm->precision != 0 && prm->precision != 1))
    return ABD_ERR_INVALID_ARG;
  const int nb = d->nb, nv = d->nv, nt = d->nt, ne = d->ne;
  std::vector<int> vbeg, tbeg, ebeg, towner(nt), eowner(ne);
  for (int t = 0; t < nt; ++t) {
    for (int k = 0; k < 3; ++k)
      if (d->tri[3 * t + k] < 0 || d->tri[3 * t + k] >= nv) return ABD_ERR_INVALID_ARG;
    towner[t] = d->vbody[d->tri[3 * t]];
    if (d->vbody[d->tri[3 * t + 1]] != towner[t] || d->vbody[d->tri[3 * t + 2]] != towner[t])
      return ABD_ERR_INVALID_ARG;
  }
  for (int e = 0; e < ne; ++e) {
    for (int k = 0; k < 2; ++k)
      if (d->edge[2 * e + k] < 0 || d->edge[2 * e + k] >= nv) return ABD_ERR_INVALID_ARG;
    eowner[e] = d->vbody[d->edge[2 * e]];
    if (d->vbody[d->edge[2 * e + 1]] != eowner[e]) return ABD_ERR_INVALID_ARG;
  }
  if (!grouped(d->vbody, nv, nb, vbeg) || !grouped(towner.data(), nt, nb, tbeg) ||
      !grouped(eowner.data(), ne, nb, ebeg))
    return ABD_ERR_INVALID_ARG;
  for (int k = 0; k < 12 * nb; ++k)
    if (!std::isfinite(d->q0[k]) || !std::isfinite(d->qdot0[k])) return ABD_ERR_NONFINITE;

  abd_scene* S = new abd_scene();
  Scene& s = S->s;
  s.prm = *prm;
  s.nb = nb;
  s.nv = nv;
  s.nt = nt;
  s.ne = ne;
  s.stream = (cudaStream_t)stream;
  s.alloc.stream = s.stream;
  cudaGetDevice(&s.device);
  if (cudaDeviceGetAttribute(&s.num_sms, cudaDevAttrMultiProcessorCount, s.device) != cudaSuccess || s.num_sms < 1) {
    cudaGetLastError();
    s.num_sms = kNumSMs;
  }
  for (cudaStream_t& x : s.side)
    if (cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      for (cudaStream_t y : s.side)
        if (y) cudaStreamDestroy(y);
      delete S;
      return ABD_ERR_CUDA;
    }
  for (int k = 0; k < 5; ++k) {
    cudaEventCreateWithFlags(&s.ev_fork[k], cudaEventDisableTiming);
    cudaEventCreateWithFlags(&s.ev_join[k], cudaEventDisableTiming);
  }
  if (alloc && alloc->alloc && alloc->free) {
    s.alloc.a = *alloc;
    s.alloc.custom = true;
  }
  try {
    grow(s, s.xbar, nv);
    grow(s, s.red, 4L * kEnergyParts);
    s.dense_n = dense_order(nb, prm->dense_max_dofs);
    if (s.dense_n) {
      grow(s, s.dense, (size_t)s.dense_n * s.dense_n);
      grow(s, s.dense_dinv, (size_t)s.dense_n);
    }
    grow(s, s.vbody, nv);
    grow(s, s.tri, 3L * nt + 1);
    grow(s, s.edge, 2L * ne + 1);
    grow(s, s.l2e, ne + 1L);
    grow(s, s.vbeg, nb + 1);
    grow(s, s.tbeg, nb + 1);
    grow(s, s.ebeg, nb + 1);
    grow(s, s.is_static, nb);
    grow(s, s.mass10, 10L * nb);
    grow(s, s.vol, nb);
    grow(s, s.kappa_b, nb);
    grow(s, s.density, nb);
    for (Buf<double>* b : {&s.q, &s.qdot, &s.qt, &s.qtilde, &s.dq, &s.qtrial, &s.qsave, &s.qdotsave, &s.gb, &s.g,
                           &s.r, &s.z, &s.pv, &s.pv2, &s.Ap})
      grow(s, *b, 12L * nb);
    grow(s, s.pcg_bar, 4);
    grow(s, s.uf, nb);
    for (Buf<int>* b : {&s.c_perm, &s.c_of, &s.c_loc, &s.c_ok}) grow(s, *b, nb);
    grow(s, s.c_off, nb + 1L);
    grow(s, s.c_foff, nb + 1L);
    grow(s, s.c_fac, 576L * nb);
    grow(s, s.isl, nb);
    grow(s, s.isl_state, 2L * nb);
    grow(s, s.isl_toi, nb);
    grow(s, s.isl_step, nb);
    grow(s, s.isl_E, 16L * nb);
    grow(s, s.isl_alpha, nb);
    grow(s, s.Eb, 2L * nb);
    for (Buf<double>* b : {&s.Db, &s.D, &s.Pinv}) grow(s, *b, 144L * nb);
    grow(s, s.part, 4L * nb + 1024);
    if (prm->precision == 1) {
      grow(s, s.D32, 144L * nb);
      grow(s, s.Minv32, 144L * nb);
      grow(s, s.vf, 72L * nb);
      grow(s, s.rhs64, 12L * nb);
    }
    for (Buf<double4>* b : {&s.x, &s.dx, &s.x1, &s.xt}) grow(s, *b, nv);
    grow(s, s.bbox, 6L * nb);
    grow(s, s.bbox32, 6L * nb);
    s.maxn = 64;
    grow(s, s.nbr, (size_t)nb * s.maxn);
    grow(s, s.ncount, nb);
    grow(s, s.rowoff, nb + 1);
    grow(s, s.in_off, nb + 1);
    grow(s, s.in_cnt, nb);
    grow(s, s.hcount, nb);
    grow(s, s.hoff, nb + 1);
    grow(s, s.large, nb);
    grow(s, s.large_pos, nb + 1);
    grow(s, s.large_list, nb);
    {
      long t = 1024;
      while (t < 16L * nb) t <<= 1;
      s.hash_T = (int)t;
    }
    grow(s, s.slot_cnt, (size_t)s.hash_T);
    grow(s, s.scan_part, (size_t)s.hash_T / 4096 + 1);
    grow(s, s.slot_off, (size_t)s.hash_T + 1);
    grow(s, s.entries, 16L * nb + 1024);
    s.maxc = 256;
    size_pair_buffers(s, std::max<size_t>(1024, 8L * nb));
    size_term_buffers(s, std::max<size_t>(4096, 16L * nb));
    if (cudaMalloc(&s.st, sizeof(DevStatus)) != cudaSuccess) throw OomError{};
    if (cudaMallocHost(&s.st_host, sizeof(DevStatus)) != cudaSuccess) throw OomError{};
    if (cudaMallocHost(&s.isl_host, sizeof(int) * nb) != cudaSuccess) throw OomError{};
    if (cudaMallocHost(&s.clu_host, sizeof(int) * (4L * nb + 2) + sizeof(long long) * (nb + 1L)) != cudaSuccess)
      throw OomError{};
  } catch (OomError&) {
    abd_destroy(S);
    return ABD_ERR_OOM;
  }
  std::vector<double4> xb(nv);
  for (int v = 0; v < nv; ++v) xb[v] = make_double4(d->xbar[3 * v], d->xbar[3 * v + 1], d->xbar[3 * v + 2], 0.0);
  // spatial-hash cell: the largest rest-frame box diagonal of the dynamic
  // bodies, so every dynamic body's box spans at most 2 cells per axis
  {
    std::vector<double> diam;
    for (int b = 0; b < nb; ++b) {
      if (d->is_static[b] || vbeg[b] == vbeg[b + 1]) continue;
      double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
      for (int v = vbeg[b]; v < vbeg[b + 1]; ++v)
        for (int k = 0; k < 3; ++k) {
          lo[k] = std::min(lo[k], d->xbar[3 * v + k]);
          hi[k] = std::max(hi[k], d->xbar[3 * v + k]);
        }
      diam.push_back(sqrt((hi[0] - lo[0]) * (hi[0] - lo[0]) + (hi[1] - lo[1]) * (hi[1] - lo[1]) +
                          (hi[2] - lo[2]) * (hi[2] - lo[2])));
    }
    double big = 1.0;
    if (!diam.empty()) big = *std::max_element(diam.begin(), diam.end());
    s.cell_h = std::max(big, 4.0 * prm->dhat) + 2.0 * prm->dhat;
  }
  cudaMemcpyAsync(s.xbar.p, xb.data(), sizeof(double4) * nv, cudaMemcpyHostToDevice, s.stream);
  cudaMemcpyAsync(s.vbody.p, d->vbody, sizeof(int) * nv, cudaMemcpyHostToDevice, s.stream);
  if (nt) cudaMemcpyAsync(s.tri.p, d->tri, sizeof(int) * 3 * nt, cudaMemcpyHostToDevice, s.stream);
  if (ne) cudaMemcpyAsync(s.edge.p, d->edge, sizeof(int) * 2 * ne, cudaMemcpyHostToDevice, s.stream);
  cudaMemcpyAsync(s.vbeg.p, vbeg.data(), sizeof(int) * (nb + 1), cudaMemcpyHostToDevice, s.stream);
  cudaMemcpyAsync(s.tbeg.p, tbeg.data(), sizeof(int) * (nb + 1), cudaMemcpyHostToDevice, s.stream);
  cudaMemcpyAsync(s.ebeg.p, ebeg.data(), sizeof(int) * (nb + 1), cudaMemcpyHostToDevice, s.stream);
  cudaMemcpyAsync(s.is_static.p, d->is_static, nb, cudaMemcpyHostToDevice, s.stream);
  s.is_static_host.assign(d->is_static, d->is_static + nb);
  cudaMemcpyAsync(s.kappa_b.p, d->kappa_body, sizeof(double) * nb, cudaMemcpyHostToDevice, s.stream);
  cudaMemcpyAsync(s.density.p, d->density, sizeof(double) * nb, cudaMemcpyHostToDevice, s.stream);
  DevStatus z;
  memset(&z, 0, sizeof(z));
  *s.st_host = z;
  cudaMemcpyAsync(s.st, s.st_host, sizeof(DevStatus), cudaMemcpyHostToDevice, s.stream);
  launch_mass_moments(s);
  launch_edge_rest(s);
  s.ndyn = 0;
  for (int b = 0; b < nb; ++b) s.ndyn += d->is_static[b] ? 0 : 1;
  // Newton tolerance (the paper states none): IPC's rule |dx|_inf <= 1e-5 l dt,
  // l the diagonal of the dynamic bodies' box at q0
  s.newton_tol = prm->newton_tol;
  if (!(s.newton_tol > 0)) {
    cudaMemcpyAsync(s.qt.p, d->q0, sizeof(double) * 12 * nb, cudaMemcpyHostToDevice, s.stream);
    launch_transform(s, s.qt.p, s.x.p);
    launch_body_boxes(s, false);
    std::vector<double> bb(6L * nb);
    cudaMemcpyAsync(bb.data(), s.bbox.p, sizeof(double) * 6 * nb, cudaMemcpyDeviceToHost, s.stream);
    cudaStreamSynchronize(s.stream);
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (int b = 0; b < nb; ++b) {
      if (d->is_static[b]) continue;
      for (int k = 0; k < 3; ++k) {
        lo[k] = std::min(lo[k], bb[6 * b + k]);
        hi[k] = std::max(hi[k], bb[6 * b + 3 + k]);
      }
    }
    double l2 = 0;
    for (int k = 0; k < 3; ++k) l2 += s.ndyn ? (hi[k] - lo[k]) * (hi[k] - lo[k]) : 0.0;
    s.newton_tol = 1e-5 * std::max(sqrt(l2), 1e-3) * prm->dt;
  }
  abd_status r = abd_set_state(S, d->q0, d->qdot0, 0);
  if (r != ABD_OK) {
    abd_destroy(S);
    return r;
  }
  // no pair may start at zero distance
  r = with_capacity(s, [&]() {
    launch_transform(s, s.qt.p, s.x.p);
    broad_and_enumerate(s, false, false);
    launch_active(s, s.x.p);
    return ABD_OK;
  });
  if (r == ABD_OK && (s.st_host->flags & ST_INTERSECT)) r = ABD_ERR_INITIAL_INTERSECTION;
  if (r == ABD_OK) r = check_cuda(s);
  if (r != ABD_OK) {
    abd_destroy(S);
    return r;
  }
  *out = S;
  return ABD_OK;
}

void abd_destroy(abd_scene* S) {
  if (!S) return;
  Scene& s = S->s;
  if (s.stream || s.st) cudaStreamSynchronize(s.stream);
  for (Scene::Segment* g : {&s.seg_head[0], &s.seg_head[1], &s.seg_tail[0], &s.seg_tail[1], &s.seg_trial})
    if (g->exec) cudaGraphExecDestroy(g->exec);
  if (s.cap_stream) cudaStreamDestroy(s.cap_stream);
  for (cudaStream_t x : s.side)
    if (x) cudaStreamDestroy(x);
  for (int k = 0; k < 5; ++k) {
    if (s.ev_fork[k]) cudaEventDestroy(s.ev_fork[k]);
    if (s.ev_join[k]) cudaEventDestroy(s.ev_join[k]);
  }
  release(s, s.xbar);
  release(s, s.l2e);
  release(s, s.scan_part);
  release(s, s.amask);
  release(s, s.bbox32);
  release(s, s.vbody);
  release(s, s.tri);
  release(s, s.edge);
  release(s, s.vbeg);
  release(s, s.tbeg);
  release(s, s.ebeg);
  release(s, s.is_static);
  release(s, s.mass10);
  release(s, s.vol);
  release(s, s.kappa_b);
  release(s, s.density);
  release(s, s.pcg_bar);
  for (Buf<float>* b : {&s.D32, &s.Minv32, &s.H32, &s.vf}) release(s, *b);
  release(s, s.rhs64);
  release(s, s.uf);
  for (Buf<int>* b : {&s.c_perm, &s.c_of, &s.c_loc, &s.c_ok, &s.c_off}) release(s, *b);
  release(s, s.c_foff);
  release(s, s.c_fac);
  release(s, s.isl);
  release(s, s.isl_state);
  release(s, s.isl_toi);
  release(s, s.isl_step);
  release(s, s.isl_E);
  release(s, s.isl_alpha);
  for (Buf<double>* b : {&s.q, &s.qdot, &s.qt, &s.qtilde, &s.dq, &s.qtrial, &s.qsave, &s.qdotsave, &s.gb, &s.g, &s.r,
                         &s.z, &s.pv, &s.pv2, &s.Ap, &s.Eb, &s.Db, &s.D, &s.Pinv, &s.part, &s.bbox, &s.term, &s.fterm,
                         &s.pblk, &s.Epair, &s.act_d2, &s.red, &s.dense, &s.dense_dinv})
    release(s, *b);
  for (Buf<double4>* b : {&s.x, &s.dx, &s.x1, &s.xt}) release(s, *b);
  for (Buf<int>* b : {&s.nbr, &s.ncount, &s.rowoff, &s.in_off, &s.in_cnt, &s.in_list, &s.ccount, &s.acount, &s.aoff,
                      &s.fpoff, &s.flagbuf, &s.posbuf, &s.hcount, &s.hoff, &s.large, &s.large_pos, &s.large_list,
                      &s.slot_cnt, &s.slot_off, &s.entries, &s.ework, &s.large_asm})
    release(s, *b);
  release(s, s.P);
  release(s, s.fpairs);
  release(s, s.cand);
  release(s, s.cdl);
  release(s, s.act);
  release(s, s.termv);
  release(s, s.tmeta);
  release(s, s.teps);
  release(s, s.td2);
  release(s, s.tlist);
  release(s, s.ftermv);
  release(s, s.fric);
  for (cudaEvent_t e : s.prof.pool) cudaEventDestroy(e);
  if (s.st) cudaFree(s.st);
  if (s.st_host) cudaFreeHost(s.st_host);
  if (s.isl_host) cudaFreeHost(s.isl_host);
  if (s.clu_host) cudaFreeHost(s.clu_host);
  delete S;
}

abd_status abd_set_state(abd_scene* S, const double* q, const double* qdot, int on_device) {
  if (!S || !q || !qdot) return ABD_ERR_INVALID_ARG;
  Scene& s = S->s;
  s.err.clear();
  const size_t qb = sizeof(double) * 12 * s.nb;
  cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  cudaMemcpyAsync(s.qt.p, q, qb, k, s.stream);
  cudaMemcpyAsync(s.qdot.p, qdot, qb, k, s.stream);
  launch_predictor(s);
  s.have_hess = false;
  abd_status r = with_capacity(s, [&]() {
    lag_friction(s);
    return ABD_OK;
  });
  if (r == ABD_OK) r = check_cuda(s);
  return r;
}

abd_status abd_get_state(abd_scene* S, double* q, double* qdot, int on_device) {
  if (!S) return ABD_ERR_INVALID_ARG;
  Scene& s = S->s;
  const size_t qb = sizeof(double) * 12 * s.nb;
  cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (q) cudaMemcpyAsync(q, s.qt.p, qb, k, s.stream);
  if (qdot) cudaMemcpyAsync(qdot, s.qdot.p, qb, k, s.stream);
  cudaStreamSynchronize(s.stream);
  return check_cuda(s);
}

abd_status abd_energy_grad_hess(abd_scene* S, const double* q_dev, double* E_host, double* g_dev,
                                abd_pair_counts* counts) {
  if (!S || !q_dev) return ABD_ERR_INVALID_ARG;
  Scene& s = S->s;
  s.err.clear();
  abd_status r = with_capacity(s, [&]() {
    launch_transform(s, q_dev, s.x.p);
    broad_and_enumerate(s, false, false);
    prepare_clusters(s);
    s.fp32_proj = s.prm.precision == 1;
    eval_system(s, q_dev, 1);
    return ABD_OK;
  });
  if (r != ABD_OK) return r;
  if (abd_status f = flags_to_status(s, s.st_host->flags & ~ST_CCD_MAXITER)) return f;
  s.have_hess = true;
  s.last_np = s.st_host->np;
  if (E_host)
    for (int k = 0; k < 5; ++k) E_host[k] = s.st_host->energy[k];
  if (g_dev) cudaMemcpyAsync(g_dev, s.g.p, sizeof(double) * 12 * s.nb, cudaMemcpyDeviceToDevice, s.stream);
  if (counts) {
    counts->n_candidates = (long)s.st_host->n_cand;
    counts->n_active = s.st_host->nact;
    counts->n_friction = s.st_host->nfr;
    counts->n_body_pairs = s.st_host->np;
  }
  cudaStreamSynchronize(s.stream);
  return check_cuda(s);
}

abd_status abd_get_hessian(abd_scene* S, double* diag, int* bi, int* bj, double* blocks, long cap, long* nblocks) {
  if (!S) return ABD_ERR_INVALID_ARG;
  Scene& s = S->s;
  if (!s.have_hess) {
    s.err = "no Hessian: call abd_energy_grad_hess first";
    return ABD_ERR_INVALID_ARG;
  }
  read_status(s);
  const long np = s.st_host->np;
  if (nblocks) *nblocks = np;
  if (diag) cudaMemcpyAsync(diag, s.D.p, sizeof(double) * 144 * s.nb, cudaMemcpyDeviceToHost, s.stream);
  const long n = std::min(np, cap);
  if (n > 0 && (bi || bj)) {
    std::vector<int2> P(n);
    cudaMemcpyAsync(P.data(), s.P.p, sizeof(int2) * n, cudaMemcpyDeviceToHost, s.stream);
    cudaStreamSynchronize(s.stream);
    for (long k = 0; k < n; ++k) {
      if (bi) bi[k] = P[k].x;
      if (bj) bj[k] = P[k].y;
    }
  }
  if (n > 0 && blocks)
    cudaMemcpy2DAsync(blocks, sizeof(double) * 144, s.pblk.p, sizeof(double) * kBlkStride, sizeof(double) * 144, n,
                      cudaMemcpyDeviceToHost, s.stream);
  cudaStreamSynchronize(s.stream);
  return check_cuda(s);
}

abd_status abd_get_pairs(abd_scene* S, int which, int* kind, int* i, int* j, int* type, double* d2, long cap,
                         long* n) {
  if (!S || which < 0 || which > 2) return ABD_ERR_INVALID_ARG;
  Scene& s = S->s;
  read_status(s);
  if (which == 2) {
    const long nf = s.st_host->nfr;
    if (n) *n = nf;
    if (!kind && !i && !j && !type && !d2) return ABD_OK;
    std::vector<FricRec> F(nf);
    if (nf) cudaMemcpy(F.data(), s.fric.p, sizeof(FricRec) * nf, cudaMemcpyDeviceToHost);
    for (long k = 0; k < std::min(nf, cap); ++k) {
      if (kind) kind[k] = F[k].kind;
      if (i) i[k] = F[k].i;
      if (j) j[k] = F[k].j;
      if (type) type[k] = F[k].type;
      if (d2) d2[k] = F[k].mu_lambda;
    }
    return check_cuda(s);
  }
  if (!s.have_hess) {
    s.err = "no pair sets: call abd_energy_grad_hess first";
    return ABD_ERR_INVALID_ARG;
  }
  const long np = s.st_host->np;
  std::vector<int> cnt(np);
  if (np) cudaMemcpy(cnt.data(), which == 0 ? s.ccount.p : s.acount.p, sizeof(int) * np, cudaMemcpyDeviceToHost);
  long total = 0;
  for (long p = 0; p < np; ++p) total += std::min(cnt[p], s.maxc);
  if (n) *n = total;
  if (!kind && !i && !j && !type && !d2) return check_cuda(s);
  long o = 0;
  std::vector<int2> C;
  std::vector<int4> A;
  std::vector<double> D2;
  for (long p = 0; p < np && o < cap; ++p) {
    const int c = std::min(cnt[p], s.maxc);
    if (!c) continue;
    if (which == 0) {
      C.resize(c);
      cudaMemcpy(C.data(), s.cand.p + p * s.maxc, sizeof(int2) * c, cudaMemcpyDeviceToHost);
    } else {
      A.resize(c);
      D2.resize(c);
      cudaMemcpy(A.data(), s.act.p + p * s.maxc, sizeof(int4) * c, cudaMemcpyDeviceToHost);
      cudaMemcpy(D2.data(), s.act_d2.p + p * s.maxc, sizeof(double) * c, cudaMemcpyDeviceToHost);
    }
    for (int k = 0; k < c && o < cap; ++k, ++o) {
      int x = which == 0 ? C[k].x : A[k].x, y = which == 0 ? C[k].y : A[k].y;
      if (kind) kind[o] = (unsigned)x >> 31;
      if (i) i[o] = x & 0x7fffffff;
      if (j) j[o] = y;
      if (type) type[o] = which == 0 ? -1 : A[k].z;
      if (d2) d2[o] = which == 0 ? 0.0 : D2[k];
    }
  }
  return check_cuda(s);
}

abd_status abd_get_friction(abd_scene* S, double* gamma, double* normal, double* offset, long cap, long* n) {
  if (!S || cap < 0) return ABD_ERR_INVALID_ARG;
  Scene& s = S->s;
  read_status(s);
  const long nf = s.st_host->nfr;
  if (n) *n = nf;
  if (!gamma && !normal && !offset) return check_cuda(s);
  std::vector<FricRec> F(nf);
  if (nf) cudaMemcpy(F.data(), s.fric.p, sizeof(FricRec) * nf, cudaMemcpyDeviceToHost);
  for (long k = 0; k < std::min(nf, cap); ++k) {
    for (int m = 0; m < 4; ++m)
      if (gamma) gamma[4 * k + m] = F[k].gam[m];
    for (int m = 0; m < 3; ++m) {
      if (normal) normal[3 * k + m] = F[k].n[m];
      if (offset) offset[3 * k + m] = F[k].r[m];
    }
  }
  return check_cuda(s);
}

abd_status abd_solve(abd_scene* S, const double* rhs_dev, double* dq_dev, abd_solve_stats* stats) {
  if (!S || !rhs_dev || !dq_dev) return ABD_ERR_INVALID_ARG;
  Scene& s = S->s;
  if (!s.have_hess) {
    s.err = "no Hessian: call abd_energy_grad_hess first";
    return ABD_ERR_INVALID_ARG;
  }
  double rel;
  s.pcg_mixed = s.prm.precision == 1;
  int its = run_pcg(s, rhs_dev, dq_dev, s.prm.pcg_max, s.prm.pcg_rel_tol, &rel);
  if (stats) {
    stats->iterations = its < 0 ? s.prm.pcg_max : its;
    stats->rel_residual = rel;
  }
  if (abd_status c = check_cuda(s)) return c;
  if (its == -2) {
    s.err = "PCG breakdown";
    return ABD_ERR_PCG_BREAKDOWN;
  }
  if (its == -1) {
    s.err = "PCG iteration cap reached";
    return ABD_ERR_PCG_MAXITER;
  }
  return ABD_OK;
}

abd_status abd_ccd_toi(abd_scene* S, const double* q_dev, const double* dq_dev, double* toi_host) {
  if (!S || !q_dev || !dq_dev || !toi_host) return ABD_ERR_INVALID_ARG;
  Scene& s = S->s;
  s.err.clear();
  abd_status r = with_capacity(s, [&]() {
    launch_transform(s, q_dev, s.x.p);
    launch_transform_dq(s, dq_dev);
    broad_and_enumerate(s, true, true);
    return ABD_OK;
  });
  if (r != ABD_OK) return r;
  s.have_hess = false;
  if (abd_status f = flags_to_status(s, s.st_host->flags)) return f;
  *toi_host = bits_to_double(s.st_host->toi_bits);
  return ABD_OK;
}

abd_status abd_step(abd_scene* S, int nsteps, abd_step_stats* stats) {
  if (!S || nsteps < 0) return ABD_ERR_INVALID_ARG;
  Scene& s = S->s;
  s.err.clear();
  s.have_hess = false;
  const size_t qb = sizeof(double) * 12 * s.nb;
  const long launches0 = s.nlaunch;
  abd_step_stats acc;
  memset(&acc, 0, sizeof(acc));
  for (int k = 0; k < nsteps; ++k) {
    cudaMemcpyAsync(s.qdotsave.p, s.qdot.p, qb, cudaMemcpyDeviceToDevice, s.stream);
    abd_status r = ABD_ERR_CAPACITY;
    for (int attempt = 0; attempt < 12 && r == ABD_ERR_CAPACITY; ++attempt) {
      reset_status(s);
      try {
        abd_step_stats one;
        memset(&one, 0, sizeof(one));
        r = newton_step(s, &one);
        if (r == ABD_OK) {
          long tested = acc.candidates_tested + one.candidates_tested;
          long evald = acc.active_evaluated + one.active_evaluated;
          int ni = acc.newton_iters + one.newton_iters, pi = acc.pcg_iters + one.pcg_iters;
          int lh = acc.ls_halvings + one.ls_halvings;
          double tmin = k ? std::min(acc.toi_min, one.toi_min) : one.toi_min;
          int cl = acc.ccd_limited + one.ccd_limited;
          int hist[6];
          for (int m = 0; m < 6; ++m) hist[m] = acc.toi_hist[m] + one.toi_hist[m];
          int lhm = std::max(acc.ls_island_halvings_max, one.ls_island_halvings_max);
          acc = one;
          acc.ccd_limited = cl;
          for (int m = 0; m < 6; ++m) acc.toi_hist[m] = hist[m];
          acc.ls_island_halvings_max = lhm;
          acc.candidates_tested = tested;
          acc.active_evaluated = evald;
          acc.newton_iters = ni;
          acc.pcg_iters = pi;
          acc.ls_halvings = lh;
          acc.toi_min = tmin;
        }
      } catch (OomError&) {
        r = ABD_ERR_OOM;
      }
      if (r == ABD_ERR_CAPACITY) {
        read_status(s);
        handle_capacity(s);
        // grown buffers lose their contents: rebuild the friction set at q^t
        abd_status lr = with_capacity(s, [&]() {
          lag_friction(s);
          return ABD_OK;
        });
        if (lr != ABD_OK) r = lr;
      }
    }
    if (r == ABD_OK)  // the new q^t: lag friction for the next step
      r = with_capacity(s, [&]() {
        lag_friction(s);
        return ABD_OK;
      });
    if (r != ABD_OK) {
      // transactional: q^t was never modified before the step completed; the
      // velocity and the lagged friction set are restored from the copy
      cudaMemcpyAsync(s.qdot.p, s.qdotsave.p, qb, cudaMemcpyDeviceToDevice, s.stream);
      launch_predictor(s);
      with_capacity(s, [&]() {
        lag_friction(s);
        return ABD_OK;
      });
      cudaStreamSynchronize(s.stream);
      return r;
    }
  }
  cudaStreamSynchronize(s.stream);
  acc.kernel_launches = s.nlaunch - launches0;
  if (stats) *stats = acc;
  return check_cuda(s);
}

abd_status abd_set_tuning(abd_scene* S, const abd_tuning* t) {
  if (!S || !t || t->grid_div < 1 || t->grid_div > 64 || t->cluster_max < 0 || t->cluster_max > kClusterMax)
    return ABD_ERR_INVALID_ARG;
  Scene& s = S->s;
  s.cluster_max = t->cluster_max ? t->cluster_max : kClusterDefault;
  if (t->grid_div != s.grid_div) {
    s.grid_div = t->grid_div;
    ++s.gen;  // the captured sequences hold the old grids
  }
  return ABD_OK;
}

abd_status abd_get_tuning(const abd_scene* S, abd_tuning* t) {
  if (!S || !t) return ABD_ERR_INVALID_ARG;
  memset(t, 0, sizeof(*t));
  t->grid_div = S->s.grid_div;
  t->cluster_max = S->s.cluster_max;
  return ABD_OK;
}

abd_status abd_step_batch(abd_scene* const* scenes, int n, int nsteps, int nworkers, abd_status* status,
                          abd_step_stats* stats) {
  if (n < 0 || nsteps < 0 || nworkers < 1 || nworkers > 256 || (n > 0 && !scenes)) return ABD_ERR_INVALID_ARG;
  std::vector<abd_scene*> uniq(scenes, scenes + n);
  std::sort(uniq.begin(), uniq.end());
  if (n && !uniq[0]) return ABD_ERR_INVALID_ARG;
  if (std::adjacent_find(uniq.begin(), uniq.end()) != uniq.end()) return ABD_ERR_INVALID_ARG;
  // largest scenes first: the longest jobs start early (list scheduling)
  std::vector<int> order(n);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return scenes[a]->s.nb > scenes[b]->s.nb; });
  std::vector<abd_status> res(n, ABD_OK);
  std::atomic<int> next{0};
  auto work = [&]() {
    int dev = -1;
    for (;;) {
      const int k = next.fetch_add(1);
      if (k >= n) break;
      const int i = order[k];
      Scene& s = scenes[i]->s;
      try {
        if (s.device != dev) {
          cudaSetDevice(s.device);
          dev = s.device;
        }
        res[i] = abd_step(scenes[i], nsteps, stats ? &stats[i] : nullptr);
      } catch (...) {
        s.err = "host allocation failed";
        res[i] = ABD_ERR_OOM;
      }
    }
  };
  const int nw = std::min(nworkers, n);
  if (nw <= 1) {
    int dev0 = 0;
    cudaGetDevice(&dev0);
    work();
    cudaSetDevice(dev0);
  } else {
    std::vector<std::thread> pool;
    pool.reserve(nw);
    for (int w = 0; w < nw; ++w) pool.emplace_back(work);
    for (auto& t : pool) t.join();
  }
  abd_status first = ABD_OK;
  for (int i = 0; i < n; ++i) {
    if (status) status[i] = res[i];
    if (first == ABD_OK && res[i] != ABD_OK) first = res[i];
  }
  return first;
}

static const char* kSlotNames[PF_COUNT] = {"enumerate_ccd", "active_set", "barrier_terms", "friction_terms",
                                           "assemble_blocks", "body_terms", "pcg_solve", "body_pairs",
                                           "dense_solve"};

abd_status abd_set_profiling(abd_scene* S, int on) {
  if (!S) return ABD_ERR_INVALID_ARG;
  Scene& s = S->s;
  cudaStreamSynchronize(s.stream);
  s.prof.on = on != 0;
  s.prof.used = 0;
  for (auto& sl : s.prof.slot) sl = Prof::Slot();
  read_status(s);
  for (int m = 0; m < 4; ++m) s.prof.bar_terms0[m] = s.st_host->bar_terms[m];
  return check_cuda(s);
}

abd_status abd_get_profile(abd_scene* S, abd_kernel_profile* out, int cap, int* n) {
  if (!S) return ABD_ERR_INVALID_ARG;
  Scene& s = S->s;
  cudaStreamSynchronize(s.stream);
  read_status(s);
  double bar_flops = 0.0;
  for (int m = 1; m < 4; ++m) bar_flops += kBarrierFlops[m] * (double)(s.st_host->bar_terms[m] - s.prof.bar_terms0[m]);
  if (n) *n = PF_COUNT;
  for (int k = 0; k < PF_COUNT && k < cap && out; ++k) {
    double ms = 0.0;
    for (auto& e : s.prof.slot[k].ev) {
      float t = 0.f;
      cudaEventElapsedTime(&t, e.first, e.second);
      ms += t;
    }
    out[k].name = kSlotNames[k];
    out[k].launches = s.prof.slot[k].launches;
    out[k].total_ms = ms;
    out[k].bytes = s.prof.slot[k].bytes;
    out[k].flops = k == PF_BARRIER ? bar_flops : s.prof.slot[k].flops;
  }
  return check_cuda(s);
}

abd_status abd_adjoint_step(abd_scene* S, const double* q_t, const double* qdot_t, const double* q_next, double* gq,
                            double* gqdot, double* gkappa, double rel_tol, abd_solve_stats* stats) {
  if (!S || !q_t || !qdot_t || !q_next || !gq || !gqdot || !gkappa || !(rel_tol > 0.0)) return ABD_ERR_INVALID_ARG;
  Scene& s = S->s;
  if (abd_status r = abd_set_state(S, q_t, qdot_t, 1)) return r;
  // unprojected system of the step at its end state
  abd_status r = with_capacity(s, [&]() {
    launch_transform(s, q_next, s.x.p);
    broad_and_enumerate(s, false, false);
    prepare_clusters(s);
    s.fp32_proj = false;
    eval_system(s, q_next, 0);
    return ABD_OK;
  });
  if (r != ABD_OK) return r;
  if (abd_status f = flags_to_status(s, s.st_host->flags & ~ST_CCD_MAXITER)) return f;
  s.have_hess = false;  // not the projected system abd_solve expects
  s.last_np = s.st_host->np;
  launch_adjoint_rhs(s, gq, gqdot, s.qsave.p);
  double rel;
  s.pcg_mixed = false;  // the adjoint's solves stay FP64
  // the unprojected Hessian may be indefinite at the converged state: the
  // dense solve takes signed pivots; the PCG reports a breakdown there
  const int its = run_pcg(s, s.qsave.p, s.dq.p, s.prm.pcg_max, rel_tol, &rel, true);
  launch_adjoint_out(s, q_next, s.dq.p, gq, gqdot, gkappa);
  cudaStreamSynchronize(s.stream);
  if (stats) {
    stats->iterations = its < 0 ? s.prm.pcg_max : its;
    stats->rel_residual = rel;
  }
  if (abd_status c = check_cuda(s)) return c;
  if (its == -2) {
    s.err = s.dense_n ? "dense adjoint solve: zero or non-finite pivot (singular Hessian)"
                      : "PCG breakdown (Hessian not positive definite along the iterates)";
    return ABD_ERR_PCG_BREAKDOWN;
  }
  if (its == -1) {
    s.err = "PCG iteration cap reached";
    return ABD_ERR_PCG_MAXITER;
  }
  return ABD_OK;
}

abd_status abd_get_counters(abd_scene* S, abd_counters* out) {
  if (!S || !out) return ABD_ERR_INVALID_ARG;
  Scene& s = S->s;
  read_status(s);
  for (int m = 0; m < 4; ++m) out->barrier_terms[m] = s.st_host->bar_terms[m];
  out->sweeps_fp32 = s.st_host->jac[0];
  out->sweeps_fp64 = s.st_host->jac[1];
  out->capped_fp64 = s.st_host->jac[2];
  out->prim_pairs_body = s.st_host->cull[0];
  out->prim_pairs_iaabb = s.st_host->cull[1];
  out->prim_pairs_cand = s.st_host->cull[2];
  return check_cuda(s);
}

const char* abd_last_error(const abd_scene* S) { return S ? S->s.err.c_str() : "null scene"; }

}  // extern "C"
