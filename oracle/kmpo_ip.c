/*
 * CPU oracle, part 2: initial bipartitioning of one (sub)graph (Section 4.2):
 * multilevel LP coarsening, a portfolio of random / BFS / greedy graph growing
 * bipartitions, 2-way FM on every level.  Brute-force bisection for pins.
 * Test infrastructure only (see kmpo.h).
 *
 * Readings (the paper gives the components, not their parameters):
 *  B1 Coarsening inside the bipartitioner: the same deterministic LP as
 *     coarsening (readings R1-R7 of part 1, no two-hop) with cluster cap
 *     U_B = max(floor(c(B)/ip_C), max_v c(v)) ("the value used in KaHIP" is
 *     not stated), repeated while a level still contracts and shrinks by at
 *     least conv_num/conv_den.
 *  B2 Portfolio order: rep_random random, rep_bfs BFS, rep_ggg greedy graph
 *     growing runs; each is FM-refined on the coarsest graph; the winner is the
 *     first run with the best (infeasible?, overload if infeasible, cut).
 *  B3 Random: nodes in ascending (step(key, v), v) order join block 0 while it
 *     stays <= target0 (first fit); BFS: same fill rule in BFS order from the
 *     node with the smallest key, neighbours enqueued in adjacency order, new
 *     root (smallest key) when a component is exhausted; greedy graph growing
 *     (Karypis-Kumar): start node as BFS, then repeatedly the block-1 node with
 *     the largest gain (ties: smallest id) that still fits.
 *  B5 Caps per level of the bipartitioner: max(L_j, t_j + max_v c(v)) for side
 *     j with target t_j -- the balance criterion of Fiduccia-Mattheyses (one
 *     maximum cell weight of slack), the 2-way analogue of L_max,k (Section 2).
 *  B4 2-way FM (Fiduccia-Mattheyses): gains from integer connectivity; each
 *     step looks at the top node (gain desc, id asc) of each side among
 *     unlocked nodes; it moves the better feasible top (destination stays <=
 *     its cap); if neither top is feasible both are locked.  A pass stops when
 *     no unlocked node is left or fm_stop moves passed without a new best; the
 *     pass is rolled back to its best prefix, ordered by (infeasible?,
 *     overload if infeasible, cut).  Passes repeat (<= fm_passes) while they
 *     improve.
 *  B6 Learned mode (cfg->learned with a proposer set, kmpo_mpnn.c): the
 *     candidates are the learned start (nodes by network score, first fit to
 *     target0; key step(itemkey, DOM_LEARNED)) followed by the first
 *     lrep_random random, lrep_bfs BFS and lrep_ggg greedy graph growing
 *     repetitions of B2 (same keys).  Only if the best of these is infeasible
 *     do the remaining repetitions of B2 run, in B2's order.  Every candidate
 *     is FM-refined and compared exactly as in B2 (first best wins).
 *  B8 Learned item mode (cfg->learned == 2 with a proposer set; an addition
 *     to the method): the network scores the item graph itself (M1-M3, key
 *     step(itemkey, DOM_LEARNED)), the learned start fills block 0 first fit
 *     in score order (as in B6), and 2-way FM (B4) refines it on the item
 *     graph with the caps of B5.  The item's own coarsening, portfolio and
 *     intermediate levels are skipped.  If the refined start breaks a cap, the
 *     item is bipartitioned by the plain method (B1-B5, the fixed portfolio).
 *  B7 Adaptive portfolio (cfg->adaptive, plain mode only; Section 4.2 names
 *     the adaptive algorithm selection of Mt-KaHyPar without describing it).
 *     Stage 1 runs the first ceil(R_a / 2) repetitions of every algorithm a,
 *     in B2's order.  Then each algorithm is judged once, on the FM-refined
 *     cuts of its feasible stage-1 runs (f runs, sum S1, sum of squares S2):
 *     it keeps running only while it can plausibly still win, i.e. its mean
 *     minus two standard deviations (population) is at most the best feasible
 *     cut b so far: S1 - f b <= 2 sqrt(f S2 - S1^2), evaluated exactly in
 *     integers; an algorithm without a feasible run stops.  Stage 2 runs the
 *     remaining repetitions of the algorithms kept, in B2's order.  With no
 *     feasible run at all after stage 1, every algorithm is kept.  The winner
 *     is the first candidate (stage 1, then stage 2) with the best key of B2.
 */
#include <stdlib.h>
#include <string.h>

#include "kmpo.h"

enum { DOM_IP_LP = 4, DOM_RANDOM = 5, DOM_BFS = 6, DOM_GGG = 7, DOM_LEARNED = 9 };

const float *kmpo_proposer(void);
void kmpo_learned_initial(int32_t n, const int64_t *xadj, const int32_t *adj, const int32_t *vw,
                          const int32_t *ew, int32_t target0, uint64_t key, const float *W,
                          int32_t *side);

uint64_t kmpo_step(uint64_t x, uint64_t w);
int32_t kmpo_cluster_key(int32_t n, const int64_t *xadj, const int32_t *adj, const int32_t *vw,
                         const int32_t *ew, int32_t U, int32_t rounds, int32_t S,
                         uint64_t basekey, int32_t *label);

static int32_t vwt(const int32_t *vw, int32_t v) { return vw ? vw[v] : 1; }
static int32_t ewt(const int32_t *ew, int64_t e) { return ew ? ew[e] : 1; }

/* state order of B2/B4: smaller is better */
typedef struct {
  int32_t inf;
  int64_t ov;
  int64_t cut;
} fmkey_t;

static fmkey_t make_key(int64_t W0, int64_t W1, int64_t L0, int64_t L1, int64_t cut) {
  fmkey_t k;
  int64_t o0 = W0 - L0, o1 = W1 - L1;
  int64_t ov = o0 > o1 ? o0 : o1;
  k.inf = ov > 0;
  k.ov = k.inf ? ov : 0;
  k.cut = cut;
  return k;
}

static int key_less(fmkey_t a, fmkey_t b) {
  if (a.inf != b.inf) return a.inf < b.inf;
  if (a.ov != b.ov) return a.ov < b.ov;
  return a.cut < b.cut;
}

static int64_t cut2(int32_t n, const int64_t *xadj, const int32_t *adj, const int32_t *ew,
                    const int32_t *side) {
  int64_t s = 0;
  for (int32_t v = 0; v < n; ++v)
    for (int64_t e = xadj[v]; e < xadj[v + 1]; ++e)
      if (side[adj[e]] != side[v]) s += ewt(ew, e);
  return s / 2;
}

/* B4 */
int64_t kmpo_fm(int32_t n, const int64_t *xadj, const int32_t *adj, const int32_t *vw,
                const int32_t *ew, int32_t L0, int32_t L1, const kmpo_config *cfg,
                int32_t *side) {
  int64_t L[2] = {L0, L1};
  int64_t *gain = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  char *locked = (char *)malloc((size_t)(n > 0 ? n : 1));
  int32_t *moves = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  int64_t cut = cut2(n, xadj, adj, ew, side);
  for (int32_t pass = 0; pass < cfg->fm_passes; ++pass) {
    int64_t W[2] = {0, 0};
    for (int32_t v = 0; v < n; ++v) {
      W[side[v]] += vwt(vw, v);
      int64_t g = 0;
      for (int64_t e = xadj[v]; e < xadj[v + 1]; ++e)
        g += (side[adj[e]] != side[v]) ? ewt(ew, e) : -(int64_t)ewt(ew, e);
      gain[v] = g;
      locked[v] = 0;
    }
    fmkey_t best = make_key(W[0], W[1], L[0], L[1], cut);
    int32_t best_step = 0, nsteps = 0;
    int64_t best_cut = cut;
    for (;;) {
      int32_t top[2] = {-1, -1};
      for (int32_t v = 0; v < n; ++v) {
        if (locked[v]) continue;
        int32_t s = side[v];
        if (top[s] < 0 || gain[v] > gain[top[s]]) top[s] = v; /* ties: first = smallest id */
      }
      if (top[0] < 0 && top[1] < 0) break;
      int32_t feas[2];
      for (int32_t s = 0; s < 2; ++s)
        feas[s] = top[s] >= 0 && W[1 - s] + vwt(vw, top[s]) <= L[1 - s];
      int32_t v = -1;
      if (feas[0] && feas[1]) {
        int32_t a = top[0], b = top[1];
        v = (gain[a] > gain[b] || (gain[a] == gain[b] && a < b)) ? a : b;
      } else if (feas[0]) {
        v = top[0];
      } else if (feas[1]) {
        v = top[1];
      } else {
        if (top[0] >= 0) locked[top[0]] = 1;
        if (top[1] >= 0) locked[top[1]] = 1;
        continue;
      }
      int32_t from = side[v], to = 1 - from;
      side[v] = to;
      W[from] -= vwt(vw, v);
      W[to] += vwt(vw, v);
      cut -= gain[v];
      locked[v] = 1;
      for (int64_t e = xadj[v]; e < xadj[v + 1]; ++e) {
        int32_t w = adj[e];
        if (side[w] == to) gain[w] -= 2 * (int64_t)ewt(ew, e);
        else gain[w] += 2 * (int64_t)ewt(ew, e);
      }
      gain[v] = -gain[v];
      moves[nsteps++] = v;
      fmkey_t k = make_key(W[0], W[1], L[0], L[1], cut);
      if (key_less(k, best)) {
        best = k;
        best_step = nsteps;
        best_cut = cut;
      }
      if (nsteps - best_step >= cfg->fm_stop) break;
    }
    for (int32_t i = nsteps - 1; i >= best_step; --i) side[moves[i]] = 1 - side[moves[i]];
    cut = best_cut;
    if (best_step == 0) break;
  }
  free(gain); free(locked); free(moves);
  return cut;
}

typedef struct {
  uint64_t h;
  int32_t v;
} hv_t;

static int cmp_hv(const void *a, const void *b) {
  const hv_t *x = (const hv_t *)a, *y = (const hv_t *)b;
  if (x->h != y->h) return x->h < y->h ? -1 : 1;
  return x->v < y->v ? -1 : (x->v > y->v);
}

/* B3 */
void kmpo_initial(int32_t algo, int32_t n, const int64_t *xadj, const int32_t *adj,
                  const int32_t *vw, const int32_t *ew, int32_t target0, uint64_t key,
                  int32_t *side) {
  hv_t *ord = (hv_t *)malloc(sizeof(hv_t) * (size_t)(n > 0 ? n : 1));
  for (int32_t v = 0; v < n; ++v) {
    ord[v].h = kmpo_step(key, (uint64_t)(uint32_t)v);
    ord[v].v = v;
  }
  qsort(ord, (size_t)n, sizeof(hv_t), cmp_hv);
  int64_t W0 = 0;
  for (int32_t v = 0; v < n; ++v) side[v] = 1;
  if (algo == 0) {
    for (int32_t i = 0; i < n; ++i) {
      int32_t v = ord[i].v;
      if (W0 + vwt(vw, v) <= target0) {
        side[v] = 0;
        W0 += vwt(vw, v);
      }
    }
  } else if (algo == 1) {
    char *vis = (char *)calloc((size_t)(n > 0 ? n : 1), 1);
    int32_t *q = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int32_t qh = 0, qt = 0, nextroot = 0;
    while (qh < n) {
      if (qh == qt) {
        while (vis[ord[nextroot].v]) ++nextroot;
        vis[ord[nextroot].v] = 1;
        q[qt++] = ord[nextroot].v;
      }
      int32_t v = q[qh++];
      if (W0 + vwt(vw, v) <= target0) {
        side[v] = 0;
        W0 += vwt(vw, v);
      }
      for (int64_t e = xadj[v]; e < xadj[v + 1]; ++e)
        if (!vis[adj[e]]) {
          vis[adj[e]] = 1;
          q[qt++] = adj[e];
        }
    }
    free(vis); free(q);
  } else {
    int64_t *gain = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    for (int32_t v = 0; v < n; ++v) {
      int64_t g = 0;
      for (int64_t e = xadj[v]; e < xadj[v + 1]; ++e) g -= ewt(ew, e);
      gain[v] = g; /* gain of moving v from block 1 to block 0 */
    }
    /* start node (smallest key) enters block 0 if it fits */
    int32_t v = (n > 0 && vwt(vw, ord[0].v) <= target0) ? ord[0].v : -1;
    for (;;) {
      if (v >= 0) {
        side[v] = 0;
        W0 += vwt(vw, v);
        for (int64_t e = xadj[v]; e < xadj[v + 1]; ++e) gain[adj[e]] += 2 * (int64_t)ewt(ew, e);
      }
      v = -1;
      for (int32_t w = 0; w < n; ++w) {
        if (side[w] == 0 || W0 + vwt(vw, w) > target0) continue;
        if (v < 0 || gain[w] > gain[v]) v = w;
      }
      if (v < 0) break;
    }
    free(gain);
  }
  free(ord);
}

/* B7: does an algorithm whose feasible runs have the cuts x_1..x_f (sum s1,
 * sum of squares s2) keep running, given the best feasible cut b?  Exactly
 * mean - 2 sd <= b with the population standard deviation:
 * s1 - f b <= 2 sqrt(f s2 - s1^2); no feasible run: no. */
static int adaptive_keep(int64_t f, int64_t s1, __int128 s2, int64_t b) {
  if (f <= 0) return 0;
  const __int128 D = (__int128)s1 - (__int128)f * b;
  if (D <= 0) return 1;
  const __int128 var = (__int128)f * s2 - (__int128)s1 * s1; /* f^2 times the variance */
  return D * D <= 4 * var;
}

/* the rule of B7 on an explicit list of feasible cuts (for the pins) */
int32_t kmpo_adaptive_keep(int32_t f, const int64_t *cuts, int64_t best) {
  int64_t s1 = 0;
  __int128 s2 = 0;
  for (int32_t i = 0; i < f; ++i) {
    s1 += cuts[i];
    s2 += (__int128)cuts[i] * cuts[i];
  }
  return adaptive_keep(f, s1, s2, best);
}

/* one level of the bipartitioner's hierarchy */
typedef struct {
  int32_t n;
  int64_t *xadj;
  int32_t *adj, *vw, *ew, *map; /* map: this level -> next coarser */
} lvl_t;

static int32_t level_cap(int32_t L, int32_t t, int32_t maxc) {
  int64_t b = (int64_t)t + maxc;
  return b > L ? (int32_t)b : L;
}

static int32_t max_w(int32_t n, const int32_t *vw) {
  int32_t m = 0;
  for (int32_t v = 0; v < n; ++v)
    if (vwt(vw, v) > m) m = vwt(vw, v);
  return m;
}

int64_t kmpo_bipartition(int32_t n, const int64_t *xadj, const int32_t *adj, const int32_t *vw,
                         const int32_t *ew, int32_t L0, int32_t L1, int32_t target0,
                         int32_t target1, uint64_t itemkey, const kmpo_config *cfg,
                         int32_t *side_out) {
  if (n == 0) return 0;
  if (cfg->learned == 2 && kmpo_proposer()) {
    /* B8: learned start on the item graph, FM there, plain method if infeasible */
    const int32_t mx = max_w(n, vw);
    const int32_t c0 = level_cap(L0, target0, mx), c1 = level_cap(L1, target1, mx);
    kmpo_learned_initial(n, xadj, adj, vw, ew, target0, kmpo_step(itemkey, DOM_LEARNED),
                         kmpo_proposer(), side_out);
    int64_t cut = kmpo_fm(n, xadj, adj, vw, ew, c0, c1, cfg, side_out);
    int64_t W0 = 0, W1 = 0;
    for (int32_t v = 0; v < n; ++v) {
      if (side_out[v] == 0) W0 += vwt(vw, v);
      else W1 += vwt(vw, v);
    }
    if (W0 <= c0 && W1 <= c1) return cut;
    kmpo_config plain = *cfg;
    plain.learned = 0;
    return kmpo_bipartition(n, xadj, adj, vw, ew, L0, L1, target0, target1, itemkey, &plain, side_out);
  }
  lvl_t lv[64];
  int32_t nl = 1;
  lv[0].n = n;
  lv[0].xadj = (int64_t *)xadj;
  lv[0].adj = (int32_t *)adj;
  lv[0].vw = (int32_t *)vw;
  lv[0].ew = (int32_t *)ew;
  lv[0].map = NULL;
  int64_t cB = 0;
  for (int32_t v = 0; v < n; ++v) cB += vwt(vw, v);
  uint64_t lpkey = kmpo_step(itemkey, DOM_IP_LP);
  /* B1: coarsen */
  while (nl < 63) {
    lvl_t *g = &lv[nl - 1];
    if (g->n <= 1) break;
    int32_t maxc = 0;
    for (int32_t v = 0; v < g->n; ++v)
      if (vwt(g->vw, v) > maxc) maxc = vwt(g->vw, v);
    int64_t UB = cB / cfg->ip_C;
    if (UB < maxc) UB = maxc;
    if (UB < 1) UB = 1;
    int32_t *label = (int32_t *)malloc(sizeof(int32_t) * (size_t)g->n);
    int32_t nc = kmpo_cluster_key(g->n, g->xadj, g->adj, g->vw, g->ew, (int32_t)UB,
                                  cfg->ip_lp_rounds, cfg->subrounds,
                                  kmpo_step(lpkey, (uint64_t)(nl - 1)), label);
    if (nc == g->n) {
      free(label);
      break;
    }
    g->map = (int32_t *)malloc(sizeof(int32_t) * (size_t)g->n);
    kmpo_graph cg;
    kmpo_contract(g->n, g->xadj, g->adj, g->vw, g->ew, label, g->map, &cg);
    free(label);
    lv[nl].n = cg.n;
    lv[nl].xadj = cg.xadj;
    lv[nl].adj = cg.adj;
    lv[nl].vw = cg.vw;
    lv[nl].ew = cg.ew;
    lv[nl].map = NULL;
    ++nl;
    if ((int64_t)cfg->conv_den * cg.n > (int64_t)cfg->conv_num * g->n) break;
  }
  /* B2: portfolio on the coarsest level */
  lvl_t *h = &lv[nl - 1];
  int32_t hm = max_w(h->n, h->vw);
  int32_t hL0 = level_cap(L0, target0, hm), hL1 = level_cap(L1, target1, hm);
  int32_t *side = (int32_t *)malloc(sizeof(int32_t) * (size_t)h->n);
  int32_t *best = (int32_t *)malloc(sizeof(int32_t) * (size_t)h->n);
  int32_t have = 0;
  fmkey_t bestk = {0, 0, 0};
  int32_t reps[3] = {cfg->rep_random, cfg->rep_bfs, cfg->rep_ggg};
  uint64_t doms[3] = {DOM_RANDOM, DOM_BFS, DOM_GGG};
  const float *W = cfg->learned ? kmpo_proposer() : NULL;
  /* B6: in learned mode the first pass takes the proposal and a prefix of
   * each algorithm's repetitions, the second the rest if still infeasible */
  int32_t first[3] = {reps[0], reps[1], reps[2]};
  const int adaptive = cfg->adaptive && !W;
  if (W) {
    first[0] = cfg->lrep_random < reps[0] ? cfg->lrep_random : reps[0];
    first[1] = cfg->lrep_bfs < reps[1] ? cfg->lrep_bfs : reps[1];
    first[2] = cfg->lrep_ggg < reps[2] ? cfg->lrep_ggg : reps[2];
  } else if (adaptive) {
    for (int32_t a = 0; a < 3; ++a) first[a] = (reps[a] + 1) / 2;
  }
  /* B7: per algorithm, the feasible stage-1 runs and their cut sums */
  int64_t fa[3] = {0, 0, 0}, s1[3] = {0, 0, 0};
  __int128 s2[3] = {0, 0, 0};
  int keep[3] = {1, 1, 1};
  for (int32_t pass = 0; pass < 2; ++pass) {
    if (pass == 1) {
      if (adaptive) {
        if (have && !bestk.inf)
          for (int32_t a = 0; a < 3; ++a) keep[a] = adaptive_keep(fa[a], s1[a], s2[a], bestk.cut);
      } else if (!W || (have && !bestk.inf)) {
        break;
      }
    }
    for (int32_t a = (pass == 0 && W) ? -1 : 0; a < 3; ++a) {
      int32_t r0 = a < 0 ? 0 : (pass == 0 ? 0 : first[a]);
      int32_t r1 = a < 0 ? 1 : (pass == 0 ? first[a] : reps[a]);
      if (pass == 1 && a >= 0 && !keep[a]) continue;
      for (int32_t r = r0; r < r1; ++r) {
        if (a < 0) {
          kmpo_learned_initial(h->n, h->xadj, h->adj, h->vw, h->ew, target0,
                               kmpo_step(itemkey, DOM_LEARNED), W, side);
        } else {
          uint64_t key = kmpo_step(kmpo_step(itemkey, doms[a]), (uint64_t)r);
          kmpo_initial(a, h->n, h->xadj, h->adj, h->vw, h->ew, target0, key, side);
        }
        int64_t cut = kmpo_fm(h->n, h->xadj, h->adj, h->vw, h->ew, hL0, hL1, cfg, side);
        int64_t W0 = 0, W1 = 0;
        for (int32_t v = 0; v < h->n; ++v) {
          if (side[v] == 0) W0 += vwt(h->vw, v);
          else W1 += vwt(h->vw, v);
        }
        fmkey_t k = make_key(W0, W1, hL0, hL1, cut);
        if (pass == 0 && a >= 0 && !k.inf) {
          fa[a] += 1;
          s1[a] += cut;
          s2[a] += (__int128)cut * cut;
        }
        if (!have || key_less(k, bestk)) {
          have = 1;
          bestk = k;
          memcpy(best, side, sizeof(int32_t) * (size_t)h->n);
        }
      }
    }
  }
  /* uncoarsen with FM on every level */
  int64_t cut = 0;
  int32_t *cur = best;
  for (int32_t l = nl - 2; l >= 0; --l) {
    int32_t *fine = (int32_t *)malloc(sizeof(int32_t) * (size_t)lv[l].n);
    for (int32_t v = 0; v < lv[l].n; ++v) fine[v] = cur[lv[l].map[v]];
    free(cur);
    cur = fine;
    int32_t lm = max_w(lv[l].n, lv[l].vw);
    kmpo_fm(lv[l].n, lv[l].xadj, lv[l].adj, lv[l].vw, lv[l].ew, level_cap(L0, target0, lm),
            level_cap(L1, target1, lm), cfg, cur);
  }
  cut = cut2(n, xadj, adj, ew, cur);
  memcpy(side_out, cur, sizeof(int32_t) * (size_t)n);
  free(cur);
  free(side);
  for (int32_t l = 0; l < nl; ++l) {
    free(lv[l].map);
    if (l > 0) {
      free(lv[l].xadj); free(lv[l].adj); free(lv[l].vw); free(lv[l].ew);
    }
  }
  return cut;
}

/* exhaustive minimum bisection under caps; side 0 holds the set bits */
int64_t kmpo_brute_bisection(int32_t n, const int64_t *xadj, const int32_t *adj,
                             const int32_t *vw, const int32_t *ew, int64_t L0, int64_t L1,
                             int32_t *side_out) {
  if (n > 24) return -2;
  int64_t best = -1;
  uint32_t bestmask = 0;
  int32_t *side = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  for (uint32_t mask = 0; mask < (1u << n); ++mask) {
    int64_t W0 = 0, W1 = 0;
    for (int32_t v = 0; v < n; ++v) {
      side[v] = (mask >> v) & 1u ? 0 : 1;
      if (side[v] == 0) W0 += vwt(vw, v);
      else W1 += vwt(vw, v);
    }
    if (W0 > L0 || W1 > L1) continue;
    int64_t c = cut2(n, xadj, adj, ew, side);
    if (best < 0 || c < best) {
      best = c;
      bestmask = mask;
    }
  }
  if (side_out && best >= 0)
    for (int32_t v = 0; v < n; ++v) side_out[v] = (bestmask >> v) & 1u ? 0 : 1;
  free(side);
  return best;
}
