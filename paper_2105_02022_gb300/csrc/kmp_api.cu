// C ABI of libkmp (declared in include/kmp.h) and the deep multilevel driver
// (Algorithm 1): coarsening with size-constrained LP and contraction until
// <= 2C nodes or convergence, then per level on the way up recursive
// bipartitioning of the blocks until k_i blocks exist (Algorithm 2, Section 3
// "Handling General k"), balancing and LP refinement, projection.
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "kmp_internal.cuh"

namespace kmp {

void set_last_error(const std::string &s);
const char *last_error();

static thread_local kmp_stats g_last_stats;

template <class F>
static int guarded(F &&f) {
  try {
    ensure_init();
    set_last_error("");
    f();
    return KMP_OK;
  } catch (const Error &e) {
    set_last_error(e.msg);
    return e.code;
  } catch (const std::bad_alloc &) {
    set_last_error("host allocation failed");
    return KMP_ERR_NOMEM;
  } catch (...) {
    set_last_error("unknown error");
    return KMP_ERR_CUDA;
  }
}

// ---------------------------------------------------------- validation
__global__ void k_validate(int32_t n, const int64_t *xadj, const int32_t *adj, const int32_t *vw,
                           const int32_t *ew, int64_t m, unsigned long long *bad,
                           unsigned long long *ewsum) {
  unsigned long long s = 0;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    int64_t b = xadj[v], e = xadj[v + 1];
    if (b > e || b < 0 || e > m) {
      atomicOr(bad, 1ull);
      continue;
    }
    if (vw && vw[v] <= 0) atomicOr(bad, 2ull);
    for (int64_t q = b; q < e; ++q) {
      int32_t u = adj[q];
      if (u < 0 || u >= n) atomicOr(bad, 4ull);
      else if (u == v) atomicOr(bad, 8ull);
      int32_t w = ew ? ew[q] : 1;
      if (w <= 0) atomicOr(bad, 16ull);
      s += (unsigned long long)(w > 0 ? w : 0);
    }
  }
#pragma unroll
  for (int mm = 16; mm > 0; mm >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, mm);
  if ((threadIdx.x & 31) == 0 && s) atomicAdd(ewsum, s);
}

__global__ void k_check_range(int64_t n, const int32_t *a, int32_t lo, int32_t hi,
                              unsigned long long *bad) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    if (a[i] < lo || a[i] >= hi) atomicOr(bad, 1ull);
}

static void check_range(int64_t n, const int32_t *a, int32_t lo, int32_t hi, const char *what) {
  if (n <= 0) return;
  DBuf<unsigned long long> bad(1);
  bad.zero();
  k_check_range<<<grid_for(n, 256), 256, 0, ctx().stream>>>(n, a, lo, hi, bad);
  KMP_LAUNCHED("check_range");
  if (read1(bad.p)) fail(KMP_ERR_ARG, std::string(what) + ": value out of range");
}

static Graph make_graph(int32_t n, const int64_t *xadj, const int32_t *adj, const int32_t *vw,
                        const int32_t *ew, bool is_device) {
  if (n < 0) fail(KMP_ERR_ARG, "n < 0");
  if (!xadj || (n > 0 && !adj && !is_device)) fail(KMP_ERR_ARG, "xadj/adjncy missing");
  cudaStream_t s = ctx().stream;
  Graph g;
  g.n = n;
  g.owned = true;
  int64_t m = 0;
  if (is_device) {
    KMP_CUDA(cudaMemcpyAsync(&m, xadj + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    KMP_CUDA(cudaStreamSynchronize(s));
  } else {
    if (xadj[0] != 0) fail(KMP_ERR_ARG, "xadj[0] != 0");
    m = xadj[n];
  }
  if (m < 0) fail(KMP_ERR_ARG, "negative edge count");
  g.m = m;
  cudaMemcpyKind kind = is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  g.xadj = static_cast<int64_t *>(dmalloc((size_t)(n + 1) * sizeof(int64_t)));
  g.adj = static_cast<int32_t *>(dmalloc((size_t)(m > 0 ? m : 1) * sizeof(int32_t)));
  KMP_CUDA(cudaMemcpyAsync(g.xadj, xadj, (size_t)(n + 1) * sizeof(int64_t), kind, s));
  if (m > 0) KMP_CUDA(cudaMemcpyAsync(g.adj, adj, (size_t)m * sizeof(int32_t), kind, s));
  if (vw) {
    g.vw = static_cast<int32_t *>(dmalloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t)));
    if (n > 0) KMP_CUDA(cudaMemcpyAsync(g.vw, vw, (size_t)n * sizeof(int32_t), kind, s));
  }
  if (ew) {
    g.ew = static_cast<int32_t *>(dmalloc((size_t)(m > 0 ? m : 1) * sizeof(int32_t)));
    if (m > 0) KMP_CUDA(cudaMemcpyAsync(g.ew, ew, (size_t)m * sizeof(int32_t), kind, s));
  }
  DBuf<unsigned long long> chk(2);
  chk.zero();
  if (n > 0) {
    k_validate<<<grid_for(n, 256), 256, 0, s>>>(n, g.xadj, g.adj, g.vw, g.ew, m, chk, chk.p + 1);
    KMP_LAUNCHED("validate");
  }
  unsigned long long h[2];
  to_host(h, chk.p, 2);
  if (h[0] || (h[1] / 2) >= (1ull << 31)) {
    Graph t = g;
    free_graph(t);
    if (h[0] & 1) fail(KMP_ERR_ARG, "xadj is not a valid offset array");
    if (h[0] & 2) fail(KMP_ERR_ARG, "node weights must be > 0");
    if (h[0] & 4) fail(KMP_ERR_ARG, "adjncy entry out of range");
    if (h[0] & 8) fail(KMP_ERR_ARG, "self-loop in adjncy");
    if (h[0] & 16) fail(KMP_ERR_ARG, "edge weights must be > 0");
    fail(KMP_ERR_UNSUPPORTED, "total edge weight must stay below 2^31");
  }
  compute_facts(g);
  if (g.total_vw >= (1ll << 31)) {
    Graph t = g;
    free_graph(t);
    fail(KMP_ERR_UNSUPPORTED, "total node weight must stay below 2^31");
  }
  return g;
}

// ------------------------------------------------------------------- caps
static int32_t ceil_log2(int32_t f) {
  int32_t j = 0;
  while ((1 << j) < f) ++j;
  return j;
}

void split_caps(double eps, int64_t cV, int32_t k, int64_t cB, int32_t fB, int32_t *t0,
                int32_t *t1, int32_t *L0, int32_t *L1) {
  int32_t f0 = fB / 2, f1 = fB - fB / 2;
  int64_t a = (cB * f0 + fB - 1) / fB, b = (cB * f1 + fB - 1) / fB;
  double e = 0.0;
  if (cB > 0) {
    double base = ((1.0 + eps) * (double)cV * (double)fB) / ((double)k * (double)cB);
    e = std::pow(base, 1.0 / (double)ceil_log2(fB)) - 1.0;
  }
  if (e < 0.0) e = 0.0;
  *t0 = (int32_t)a;
  *t1 = (int32_t)b;
  *L0 = (int32_t)std::floor((1.0 + e) * (double)a);
  *L1 = (int32_t)std::floor((1.0 + e) * (double)b);
}

int32_t block_cap(double eps, int64_t cV, int32_t k, int32_t fb, int32_t maxc) {
  double a = (1.0 + eps) * (double)cV * (double)fb / (double)k;
  double b = (double)cV * (double)fb / (double)k + (double)maxc;
  return (int32_t)std::floor(a > b ? a : b);
}

__global__ void k_bw_to_i32(int32_t k, const int64_t *bw64, int32_t *bw) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < k; i += gridDim.x * blockDim.x)
    bw[i] = (int32_t)bw64[i];
}

int64_t refine(const Graph &g, int32_t k, const int32_t *caps_host, int32_t rounds, uint64_t seed,
               int32_t *part, LPStats *st, bool want_cut) {
  cudaStream_t s = ctx().stream;
  DBuf<int64_t> bw64(k);
  DBuf<int32_t> bw(k), cap(k);
  to_dev(cap.p, caps_host, k);
  block_weights(g, part, k, bw64);
  k_bw_to_i32<<<grid_for(k, 256), 256, 0, s>>>(k, bw64, bw);
  KMP_LAUNCHED("bw_to_i32");
  lp_run(g, part, bw, k, cap, 0, rounds, key_of(seed, {DOM_REFINE}), nullptr, st);
  if (!want_cut) return 0;
  DBuf<int64_t> cut(1);
  cut_and_weights(g, part, k, bw64, cut);
  return read1(cut.p);
}

// --------------------------------------------------------------- driver
struct Timer {
  cudaEvent_t a, b;
  Timer() {
    KMP_CUDA(cudaEventCreate(&a));
    KMP_CUDA(cudaEventCreate(&b));
    KMP_CUDA(cudaEventRecord(a, ctx().stream));
  }
  float stop() {
    KMP_CUDA(cudaEventRecord(b, ctx().stream));
    KMP_CUDA(cudaEventSynchronize(b));
    float ms = 0;
    KMP_CUDA(cudaEventElapsedTime(&ms, a, b));
    return ms;
  }
  ~Timer() {
    cudaEventDestroy(a);
    cudaEventDestroy(b);
  }
};

__global__ void k_zero_i32(int64_t n, int32_t *p) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    p[i] = 0;
}

// D4 feasibility of a partition of one level (block caps by final counts)
static bool level_feasible(const Graph &g, const int32_t *part, int32_t nblocks, const std::vector<int32_t> &f,
                           double eps, int64_t cV, int32_t k, int64_t *cut_out) {
  DBuf<int64_t> bw(nblocks), cut(1);
  cut_and_weights(g, part, nblocks, bw, cut);
  std::vector<int64_t> hbw(nblocks);
  to_host(hbw.data(), bw.p, nblocks);
  *cut_out = read1(cut.p);
  for (int32_t b = 0; b < nblocks; ++b)
    if (hbw[b] > block_cap(eps, cV, k, f[b], g.max_vw)) return false;
  return true;
}

struct DeepOut {
  DBuf<int32_t> part;  // on the hierarchy's first graph
  int32_t nblocks = 1;
  std::vector<int32_t> f;
};

// Algorithm 1 on the hierarchy that starts at g0.  Coarsening stops at
// n <= max(R, 2) C; with R >= 2 the coarsest graph's partition is the better
// of two copies solved recursively with R / 2 under their own seeds
// (Section 3, "Parallelization"); `input`: g0 is the input graph (k blocks
// there); `top`: record the level statistics.
static void deep(const Graph &g0, int32_t R, uint64_t seed, bool input, bool top, int32_t n_in, int32_t k,
                 double eps, int64_t cV, kmp_stats *st, DeepOut &out) {
  Context &C = ctx();
  const kmp_config &cfg = C.cfg;
  std::vector<Graph> lv;
  std::vector<DBuf<int32_t>> maps;
  lv.push_back(g0);
  lv[0].owned = false;
  int64_t kp = n_in / cfg.C;
  if (kp > k) kp = k;
  if (kp < 1) kp = 1;
  const int64_t stop = (int64_t)(R > 2 ? R : 2) * cfg.C;
  while (lv.size() < 63 && lv.back().n > stop) {
    const Graph &cur = lv.back();
    while (kp > 1 && 2 * (int64_t)cur.n <= kp * cfg.C) kp /= 2;
    int64_t U = (int64_t)std::floor(eps * (double)cV / (double)kp);
    if (U < cur.max_vw) U = cur.max_vw;
    if (U < 1) U = 1;
    if (top) {
      st->level_kp[lv.size() - 1] = (int32_t)kp;
      st->level_U[lv.size() - 1] = U;
      st->clustered = (int32_t)lv.size();
    }
    DBuf<int32_t> label(cur.n);
    LPStats ls;
    float ms_other = 0;
    int level = (int)lv.size() - 1;
    int32_t nc = cluster_level(cur, (int32_t)U, cfg.lp_rounds, key_of(seed, {DOM_COARSEN, (uint64_t)level}),
                               cfg.two_hop != 0, label, nullptr, &ls, &ms_other);
    st->lp_scanned += ls.scanned;
    st->lp_rounds_run += ls.rounds;
    st->ms_lp += ls.ms;
    st->ms_cluster_other += ms_other;
    if (top && level == 0) {
      st->ms_lp_level0 = ls.ms;
      st->lp_scanned_level0 = ls.scanned;
      st->lp_rounds_level0 = ls.rounds;
    }
    if (nc == cur.n) break;
    DBuf<int32_t> map(cur.n);
    Timer tc;
    Graph coarse = contract_graph(cur, label, map);
    st->ms_contract += tc.stop();
    int32_t nprev = cur.n;
    lv.push_back(coarse);
    maps.push_back(std::move(map));
    if ((int64_t)cfg.conv_den * coarse.n > (int64_t)cfg.conv_num * nprev) break;
  }
  int L = (int)lv.size();
  if (top) {
    st->levels = L;
    for (int l = 0; l < L && l < 64; ++l) {
      st->level_n[l] = lv[l].n;
      st->level_m[l] = lv[l].m;
    }
  }
  std::vector<int32_t> f(1, k);
  int32_t nblocks = 1;
  DBuf<int32_t> part;
  if (R >= 2) {
    // the coarsest graph's partition: the better of two recursive copies
    const Graph &gc = lv[L - 1];
    DeepOut o[2];
    bool fe[2];
    int64_t ct[2];
    for (int c = 0; c < 2; ++c) {
      deep(gc, R / 2, key_of(seed, {DOM_REPLICA, (uint64_t)c}), false, false, n_in, k, eps, cV, st, o[c]);
      fe[c] = level_feasible(gc, o[c].part, o[c].nblocks, o[c].f, eps, cV, k, &ct[c]);
    }
    int pick = (fe[0] != fe[1]) ? (fe[0] ? 0 : 1) : (ct[1] < ct[0] ? 1 : 0);
    part = std::move(o[pick].part);
    nblocks = o[pick].nblocks;
    f = o[pick].f;
  } else {
    part.alloc(lv[L - 1].n);
    part.zero();
  }
  for (int l = L - 1; l >= 0; --l) {
    Graph &g = lv[l];
    if (l < L - 1) {
      Timer tp;
      DBuf<int32_t> fine(g.n);
      project(g.n, maps[l], part, fine);
      part = std::move(fine);
      st->ms_project += tp.stop();
    }
    int64_t ki;
    if (input && l == 0) {
      ki = k;
    } else {
      ki = 1;
      while (ki * cfg.C < g.n) ki *= 2;
    }
    if (ki > k) ki = k;
    if (ki < 2) ki = 2;
    {
      Timer ti;
      for (int j = 0; nblocks < ki; ++j) {
        int32_t items = 0;
        nblocks = bipartition_blocks(g, part, nblocks, f, eps, cV, k,
                                     key_of(seed, {DOM_IP, (uint64_t)l, (uint64_t)j}), &items);
        st->ip_items += items;
      }
      st->ms_ip += ti.stop();
    }
    if (top) st->level_k[l] = nblocks;
    std::vector<int32_t> caps(nblocks);
    for (int b = 0; b < nblocks; ++b) caps[b] = block_cap(eps, cV, k, f[b], g.max_vw);
    {
      Timer tb;
      BalStats bs;
      balance(g, nblocks, caps.data(), part, &bs);
      st->bal_over_blocks += bs.over_blocks;
      st->bal_moves += bs.moves;
      st->bal_spec_moves += bs.spec_moves;
      st->bal_exact_batches += bs.exact_batches;
      st->bal_exact_cands += bs.exact_cands;
      st->bal_exact_entries += bs.exact_entries;
      st->ms_balance += tb.stop();
    }
    LPStats rs;
    refine(g, nblocks, caps.data(), cfg.refine_rounds, key_of(seed, {DOM_REFINE_LEVEL, (uint64_t)l}),
           part, &rs, false);
    st->refine_scanned += rs.scanned;
    st->ms_refine += rs.ms;
  }
  for (int l = 1; l < L; ++l) free_graph(lv[l]);
  out.part = std::move(part);
  out.nblocks = nblocks;
  out.f = f;
}

static void partition_graph(const Graph &g0, int32_t k, double eps, uint64_t seed, int32_t *part_out,
                            kmp_stats *st) {
  Context &C = ctx();
  const kmp_config &cfg = C.cfg;
  cudaStream_t s = C.stream;
  memset(st, 0, sizeof(*st));
  int64_t launches0 = C.launches;
  Timer total;
  int32_t n = g0.n;
  if (k <= 1 || n == 0) {
    if (n > 0) {
      k_zero_i32<<<grid_for(n, 256), 256, 0, s>>>(n, part_out);
      KMP_LAUNCHED("zero");
    }
    st->levels = 1;
    st->level_n[0] = n;
    st->level_m[0] = g0.m;
    st->feasible = 1;
    st->ms_total = total.stop();
    st->gpu_launches = (int32_t)(C.launches - launches0);
    return;
  }
  int64_t cV = g0.total_vw;
  DeepOut o;
  deep(g0, cfg.replicas > 1 ? cfg.replicas : 1, seed, true, true, n, k, eps, cV, st, o);
  KMP_CUDA(cudaMemcpyAsync(part_out, o.part.p, (size_t)n * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
  DBuf<int64_t> bw(k), cut(1);
  cut_and_weights(g0, part_out, k, bw, cut);
  std::vector<int64_t> hbw(k);
  to_host(hbw.data(), bw.p, k);
  st->cut = read1(cut.p);
  int64_t Lk = (int64_t)std::floor((1.0 + eps) * (double)((cV + k - 1) / k));
  st->feasible = 1;
  for (int b = 0; b < k; ++b)
    if (hbw[b] > Lk) st->feasible = 0;
  sync_and_check("partition");
  st->ms_total = total.stop();
  st->gpu_launches = (int32_t)(C.launches - launches0);
}

}  // namespace kmp

using namespace kmp;

// ------------------------------------------------------------------ C ABI
extern "C" {

void kmp_config_default(kmp_config *c) {
  if (!c) return;
  c->C = 160;
  c->lp_rounds = 5;
  c->refine_rounds = 5;
  c->subrounds = 8;
  c->two_hop = 1;
  c->conv_num = 19;
  c->conv_den = 20;
  c->ip_C = 16;
  c->ip_lp_rounds = 5;
  c->rep_random = 4;
  c->rep_bfs = 4;
  c->rep_ggg = 8;
  c->fm_passes = 8;
  c->fm_stop = 64;
  c->learned = 0;
  c->lrep_random = 0;
  c->lrep_bfs = 0;
  c->lrep_ggg = 1;
  c->replicas = 1;
  c->adaptive = 0;
}

int kmp_set_config(const kmp_config *c) {
  return guarded([&] {
    if (!c) fail(KMP_ERR_ARG, "config is NULL");
    bool pow2 = c->subrounds >= 1 && c->subrounds <= 8 && (c->subrounds & (c->subrounds - 1)) == 0;
    if (c->C < 1 || c->lp_rounds < 0 || c->lp_rounds > 64 || c->refine_rounds < 0 ||
        c->refine_rounds > 64 || !pow2 || c->conv_den <= 0 || c->conv_num < 0 || c->ip_C < 1 ||
        c->ip_lp_rounds < 0 || c->ip_lp_rounds > 64 || c->rep_random < 0 || c->rep_bfs < 0 ||
        c->rep_ggg < 0 || c->rep_random + c->rep_bfs + c->rep_ggg < 1 ||
        c->rep_random + c->rep_bfs + c->rep_ggg > 64 || c->fm_passes < 0 || c->fm_stop < 1 ||
        c->learned < 0 || c->learned > 2 || c->lrep_random < 0 || c->lrep_bfs < 0 || c->lrep_ggg < 0 ||
        c->replicas < 1 || c->replicas > 64 || (c->replicas & (c->replicas - 1)) != 0 ||
        c->adaptive < 0 || c->adaptive > 1)
      fail(KMP_ERR_ARG, "invalid configuration");
    ctx().cfg = *c;
  });
}

int kmp_get_config(kmp_config *c) {
  return guarded([&] {
    if (!c) fail(KMP_ERR_ARG, "config is NULL");
    *c = ctx().cfg;
  });
}

int kmp_set_stream(void *stream) {
  return guarded([&] { ctx().stream = static_cast<cudaStream_t>(stream); });
}

const char *kmp_last_error(void) { return last_error(); }

int kmp_graph_create(kmp_vid n, const kmp_eid *xadj, const kmp_vid *adjncy, const kmp_wgt *vwgt,
                     const kmp_wgt *adjwgt, int is_device, kmp_graph **out) {
  return guarded([&] {
    if (!out) fail(KMP_ERR_ARG, "out is NULL");
    *out = nullptr;
    Graph g = make_graph(n, xadj, adjncy, vwgt, adjwgt, is_device != 0);
    kmp_graph *h = new kmp_graph;
    h->g = g;
    *out = h;
  });
}

int kmp_graph_free(kmp_graph *g) {
  return guarded([&] {
    if (!g) return;
    free_graph(g->g);
    KMP_CUDA(cudaStreamSynchronize(ctx().stream));
    delete g;
  });
}

int kmp_graph_get(const kmp_graph *g, kmp_vid *n, kmp_eid *m, const kmp_eid **xadj,
                  const kmp_vid **adjncy, const kmp_wgt **vwgt, const kmp_wgt **adjwgt) {
  return guarded([&] {
    if (!g) fail(KMP_ERR_ARG, "graph is NULL");
    if (n) *n = g->g.n;
    if (m) *m = g->g.m;
    if (xadj) *xadj = g->g.xadj;
    if (adjncy) *adjncy = g->g.adj;
    if (vwgt) *vwgt = g->g.vw;
    if (adjwgt) *adjwgt = g->g.ew;
  });
}

int kmp_graph_copy_to_host(const kmp_graph *g, kmp_eid *xadj, kmp_vid *adjncy, kmp_wgt *vwgt,
                           kmp_wgt *adjwgt) {
  return guarded([&] {
    if (!g) fail(KMP_ERR_ARG, "graph is NULL");
    const Graph &G = g->g;
    if (xadj) to_host(xadj, G.xadj, (size_t)G.n + 1);
    if (adjncy) to_host(adjncy, G.adj, (size_t)G.m);
    if (vwgt) {
      if (G.vw) to_host(vwgt, G.vw, (size_t)G.n);
      else for (int32_t v = 0; v < G.n; ++v) vwgt[v] = 1;
    }
    if (adjwgt) {
      if (G.ew) to_host(adjwgt, G.ew, (size_t)G.m);
      else for (int64_t e = 0; e < G.m; ++e) adjwgt[e] = 1;
    }
  });
}

int kmp_coarsen_level(const kmp_graph *g, int64_t U, int32_t rounds, uint64_t seed, int32_t level,
                      kmp_vid *label_out, kmp_vid *fav_out) {
  return guarded([&] {
    if (!g || !label_out) fail(KMP_ERR_ARG, "graph or label_out is NULL");
    if (U < g->g.max_vw || U >= (1ll << 31)) fail(KMP_ERR_ARG, "max_cluster_weight out of range");
    if (rounds < 0 || rounds > 64) fail(KMP_ERR_ARG, "rounds out of range");
    if (g->g.n == 0) return;
    cluster_level(g->g, (int32_t)U, rounds, key_of(seed, {DOM_COARSEN, (uint64_t)(uint32_t)level}),
                  ctx().cfg.two_hop != 0, label_out, fav_out, nullptr, nullptr);
    sync_and_check("coarsen_level");
  });
}

int kmp_contract(const kmp_graph *g, const kmp_vid *label, kmp_graph **coarse_out, kmp_vid *map_out) {
  return guarded([&] {
    if (!g || !label || !coarse_out || !map_out) fail(KMP_ERR_ARG, "NULL argument");
    *coarse_out = nullptr;
    check_range(g->g.n, label, 0, g->g.n, "label");
    Graph c = contract_graph(g->g, label, map_out);
    sync_and_check("contract");
    kmp_graph *h = new kmp_graph;
    h->g = c;
    *coarse_out = h;
  });
}

int kmp_refine(const kmp_graph *g, int32_t k, const int64_t *mbw, int32_t rounds, uint64_t seed,
               kmp_vid *part, int64_t *cut_out) {
  return guarded([&] {
    if (!g || !mbw || !part) fail(KMP_ERR_ARG, "NULL argument");
    if (k < 1) fail(KMP_ERR_ARG, "k < 1");
    if (rounds < 0 || rounds > 64) fail(KMP_ERR_ARG, "rounds out of range");
    std::vector<int32_t> caps(k);
    for (int b = 0; b < k; ++b) {
      if (mbw[b] < 0 || mbw[b] >= (1ll << 31)) fail(KMP_ERR_ARG, "max_block_weight out of range");
      caps[b] = (int32_t)mbw[b];
    }
    check_range(g->g.n, part, 0, k, "part");
    int64_t c = refine(g->g, k, caps.data(), rounds, seed, part, nullptr);
    sync_and_check("refine");
    if (cut_out) *cut_out = c;
  });
}

int kmp_balance(const kmp_graph *g, int32_t k, const int64_t *mbw, kmp_vid *part, int64_t *moved_out) {
  return guarded([&] {
    if (!g || !mbw || !part) fail(KMP_ERR_ARG, "NULL argument");
    if (k < 1) fail(KMP_ERR_ARG, "k < 1");
    std::vector<int32_t> caps(k);
    for (int b = 0; b < k; ++b) {
      if (mbw[b] < 0 || mbw[b] >= (1ll << 31)) fail(KMP_ERR_ARG, "max_block_weight out of range");
      caps[b] = (int32_t)mbw[b];
    }
    check_range(g->g.n, part, 0, k, "part");
    int64_t mv = balance(g->g, k, caps.data(), part);
    sync_and_check("balance");
    if (moved_out) *moved_out = mv;
  });
}

int kmp_project(kmp_vid n_fine, const kmp_vid *map, const kmp_vid *pc, kmp_vid *pf) {
  return guarded([&] {
    if (n_fine < 0 || (n_fine > 0 && (!map || !pc || !pf))) fail(KMP_ERR_ARG, "NULL argument");
    if (n_fine == 0) return;
    project(n_fine, map, pc, pf);
    sync_and_check("project");
  });
}

int kmp_cut(const kmp_graph *g, const kmp_vid *part, int32_t k, int64_t *cut_out, int64_t *bw_out) {
  return guarded([&] {
    if (!g || !part) fail(KMP_ERR_ARG, "NULL argument");
    if (k < 1) fail(KMP_ERR_ARG, "k < 1");
    check_range(g->g.n, part, 0, k, "part");
    DBuf<int64_t> bw(k), cut(1);
    cut_and_weights(g->g, part, k, bw, cut);
    if (bw_out) to_host(bw_out, bw.p, k);
    int64_t c = read1(cut.p);
    sync_and_check("cut");
    if (cut_out) *cut_out = c;
  });
}

int kmp_bipartition_blocks(const kmp_graph *g, int32_t nblocks, const int32_t *f, double eps,
                           int64_t cV, int32_t k, uint64_t roundkey, kmp_vid *part,
                           int32_t *nblocks_out, int32_t *f_out) {
  return guarded([&] {
    if (!g || !f || !part || !nblocks_out || !f_out) fail(KMP_ERR_ARG, "NULL argument");
    if (nblocks < 1 || k < 1 || !(eps > 0.0) || cV < 1) fail(KMP_ERR_ARG, "invalid arguments");
    check_range(g->g.n, part, 0, nblocks, "part");
    std::vector<int32_t> fv(f, f + nblocks);
    for (int32_t x : fv)
      if (x < 1) fail(KMP_ERR_ARG, "final block counts must be >= 1");
    int32_t items = 0;
    int32_t nb = bipartition_blocks(g->g, part, nblocks, fv, eps, cV, k, roundkey, &items);
    sync_and_check("bipartition_blocks");
    *nblocks_out = nb;
    for (int32_t i = 0; i < nb; ++i) f_out[i] = fv[i];
  });
}

int kmp_bipartition_each(const kmp_graph *g, int32_t nblocks, const int32_t *caps, uint64_t roundkey,
                         kmp_vid *part) {
  return guarded([&] {
    if (!g || !caps || !part) fail(KMP_ERR_ARG, "NULL argument");
    if (nblocks < 1) fail(KMP_ERR_ARG, "nblocks < 1");
    for (int32_t b = 0; b < nblocks; ++b) {
      const int32_t *c = caps + 4 * b;
      if (c[0] < 0 || c[1] < 0 || c[2] < 1 || c[3] < 1) fail(KMP_ERR_ARG, "invalid caps");
    }
    check_range(g->g.n, part, 0, nblocks, "part");
    std::vector<int32_t> fv(nblocks, 2);
    int32_t items = 0;
    bipartition_blocks(g->g, part, nblocks, fv, 0.0, 1, 1, roundkey, &items, caps);
    sync_and_check("bipartition_each");
  });
}

int kmp_partition_graph(const kmp_graph *g, int32_t k, double eps, uint64_t seed, kmp_vid *part_out,
                        kmp_stats *stats) {
  int rc = guarded([&] {
    if (!g || !part_out) fail(KMP_ERR_ARG, "NULL argument");
    if (k < 1) fail(KMP_ERR_ARG, "k < 1");
    if (!(eps > 0.0) || eps > 1e6) fail(KMP_ERR_ARG, "eps must be > 0");
    if (g->g.n < 1) fail(KMP_ERR_ARG, "n < 1");
    kmp_stats st;
    partition_graph(g->g, k, eps, seed, part_out, &st);
    g_last_stats = st;
    if (stats) *stats = st;
  });
  if (rc == KMP_OK && !g_last_stats.feasible) {
    set_last_error("partition violates L_k");
    return KMP_ERR_INFEASIBLE;
  }
  return rc;
}

int kmp_partition(kmp_vid n, const kmp_eid *xadj, const kmp_vid *adjncy, const kmp_wgt *vwgt,
                  const kmp_wgt *adjwgt, int32_t k, double eps, uint64_t seed, kmp_vid *part_out) {
  bool feasible = true;
  int rc = guarded([&] {
    if (n < 1 || !xadj || !adjncy || !part_out) fail(KMP_ERR_ARG, "invalid arguments");
    if (k < 1) fail(KMP_ERR_ARG, "k < 1");
    if (!(eps > 0.0) || eps > 1e6) fail(KMP_ERR_ARG, "eps must be > 0");
    Graph g = make_graph(n, xadj, adjncy, vwgt, adjwgt, false);
    struct Holder {
      Graph g;
      ~Holder() {
        try { free_graph(g); } catch (...) {}
      }
    } hold{g};
    DBuf<int32_t> part(n);
    kmp_stats st;
    partition_graph(hold.g, k, eps, seed, part, &st);
    to_host(part_out, part.p, (size_t)n);
    g_last_stats = st;
    feasible = st.feasible != 0;
  });
  if (rc == KMP_OK && !feasible) {
    set_last_error("partition violates L_k");
    return KMP_ERR_INFEASIBLE;
  }
  return rc;
}

int kmp_last_stats(kmp_stats *stats) {
  if (!stats) return KMP_ERR_ARG;
  *stats = g_last_stats;
  return KMP_OK;
}

int kmp_set_tuning(const kmp_tuning *t) {
  return guarded([&] {
    if (!t) fail(KMP_ERR_ARG, "tuning is NULL");
    bool pow2 = t->hub_chunk > 0 && (t->hub_chunk & (t->hub_chunk - 1)) == 0;
    if (t->rate_blocks_per_sm < 2 || t->rate_blocks_per_sm > 16 || t->hub_degree < 256 ||
        t->hub_degree > 2048 || !pow2 || t->hub_chunk < 256 || t->hub_chunk > 65536 ||
        t->ip_blocks_per_sm < 1 || t->ip_blocks_per_sm > 8 || t->dense_hub_degree < 512 ||
        t->dense_hub_degree > (1 << 30) || t->lp_graphs < 0 || t->lp_graphs > 1 ||
        (t->hub_bucket != 0 && (t->hub_bucket < 32 || t->hub_bucket > (1 << 20))) ||
        t->dense_labels < 0 || t->dense_labels > 57344)
      fail(KMP_ERR_ARG, "invalid tuning");
    ctx().tune = *t;
  });
}

int kmp_get_tuning(kmp_tuning *t) {
  return guarded([&] {
    if (!t) fail(KMP_ERR_ARG, "tuning is NULL");
    *t = ctx().tune;
  });
}

int kmp_autotune(const kmp_graph *g, int32_t k, double eps, uint64_t seed, kmp_tuning *best) {
  return guarded([&] {
    if (!g || !best) fail(KMP_ERR_ARG, "NULL argument");
    if (k < 1 || !(eps > 0.0)) fail(KMP_ERR_ARG, "invalid k or eps");
    Context &C = ctx();
    const Graph &G = g->g;
    kmp_tuning keep = C.tune, bestt = C.tune;
    float bestms = -1.f;
    int64_t kp = G.n / C.cfg.C;
    if (kp > k) kp = k;
    if (kp < 1) kp = 1;
    int64_t U = (int64_t)std::floor(eps * (double)G.total_vw / (double)kp);
    if (U < G.max_vw) U = G.max_vw;
    if (U < 1) U = 1;
    DBuf<int32_t> label(G.n > 0 ? G.n : 1);
    const int grids[3] = {4, 6, 8};
    const int hubs[2] = {1024, 2048};
    const int chunks[2] = {512, 2048};
    for (int gi : grids)
      for (int hd : hubs)
        for (int hc : chunks) {
          C.tune = kmp_tuning{gi, hd, hc, keep.ip_blocks_per_sm, keep.dense_hub_degree, keep.lp_graphs,
                                keep.hub_bucket, keep.dense_labels};
          LPStats st;
          cluster_level(G, (int32_t)U, C.cfg.lp_rounds, key_of(seed, {DOM_COARSEN, 0}), false, label,
                        nullptr, &st, nullptr);
          if (bestms < 0 || st.ms < bestms) {
            bestms = st.ms;
            bestt = C.tune;
          }
        }
    C.tune = bestt;
    sync_and_check("autotune");
    *best = bestt;
  });
}

int kmp_set_profiling(int on) {
  return guarded([&] { ctx().profile = on != 0; });
}

int kmp_profile_read(double *rate_ms, double *rate_bytes, int64_t *rate_launches, int reset) {
  return guarded([&] {
    Context &C = ctx();
    if (rate_ms) *rate_ms = C.prof_rate_ms;
    if (rate_bytes) *rate_bytes = C.prof_rate_bytes;
    if (rate_launches) *rate_launches = C.prof_rate_launches;
    if (reset) {
      C.prof_rate_ms = 0;
      C.prof_rate_bytes = 0;
      C.prof_rate_launches = 0;
    }
  });
}

int kmp_profile_read_stage(double *stage_ms, double *stage_bytes, int64_t *spans, int reset) {
  return guarded([&] {
    Context &C = ctx();
    if (stage_ms) *stage_ms = C.prof_stage_ms;
    if (stage_bytes) *stage_bytes = C.prof_stage_bytes;
    if (spans) *spans = C.prof_stage_spans;
    if (reset) {
      C.prof_stage_ms = 0;
      C.prof_stage_bytes = 0;
      C.prof_stage_spans = 0;
    }
  });
}

}  // extern "C"
