/*
 * CPU oracle, part 1: keys, cut, size-constrained label propagation,
 * isolated-node packing, two-hop clustering, contraction, LP refinement.
 * Test infrastructure only (see kmpo.h).
 *
 * Readings of the paper fixed here (the CUDA path reproduces each exactly):
 *  R1 Randomness (Section 4.1 randomises traversal; no generator is given):
 *     every random choice is a pure function of counters through the SplitMix64
 *     finaliser (Steele, Lea, Flood 2014) chained over words.
 *  R2 Parallel LP (Section 4.1 "Parallelization" uses racy atomic updates and
 *     an arbitrary visit order): replaced by S deterministic sub-rounds per
 *     round.  Node u belongs to sub-round step(roundkey, u) mod S.  Within a
 *     sub-round every node reads the state at the start of that sub-round.
 *  R3 "Most neighbours" (Section 2) is the largest summed edge weight r(K).
 *     Candidates are the clusters of u's neighbours; K is admissible when
 *     w(K) + c(u) <= cap(K).  The best admissible K != own is chosen by
 *     (r desc, perm32(roundkey, K) asc), perm32 being a bijection, and u
 *     proposes K only when r(K) > r(own) (own wins ties).
 *  R4 Commit: proposals to the same target are ordered by (gain desc, u asc);
 *     a proposal is accepted when w_start(T) + prefix weight <= cap(T).  All
 *     accepted moves are then applied.  The cap therefore holds exactly, as
 *     Section 4.3 requires for refinement (coarsening in the paper tolerates
 *     small overshoots; here it does not).
 *  R5 Active set (Section 4.1): round 0 rates every node; round r > 0 rates u
 *     only if a neighbour moved during round r-1.  Stop after a round without
 *     moves.
 *  R6 Favoured cluster (Section 4.1, two-hop): recorded when u's best cluster
 *     ignoring the cap beats its own but no admissible one does, and when u's
 *     proposal to T is rejected at commit (fav = T).
 *  R7 Isolated nodes (degree 0; the paper is silent): packed in id order into
 *     chunks of weight <= U: with P the exclusive prefix weight, node v goes
 *     to chunk floor(P/U) unless it straddles a chunk boundary (then it stays
 *     alone); a chunk takes the label of its first member.
 *  R8 Two-hop (Section 4.1): if more than n/2 clusters remain, singleton
 *     clusters with a favoured cluster are sorted by (fav, id); inside each fav
 *     group members 2i and 2i+1 form a pair when their weights sum to <= U;
 *     pairs are taken in (fav, i) order until floor(n/2) clusters remain; the
 *     second member joins the first one's cluster.
 *  R9 Contraction (Section 2): coarse ids follow ascending cluster label; the
 *     coarse rows are sorted by neighbour id; edges inside a cluster vanish.
 */
#include <stdlib.h>
#include <string.h>

#include "kmpo.h"

#define GOLDEN 0x9E3779B97F4A7C15ull
enum { DOM_COARSEN = 1, DOM_REFINE = 2 };

static uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

uint64_t kmpo_step(uint64_t x, uint64_t w) { return mix64(x ^ mix64(w + GOLDEN)); }

uint64_t kmpo_key(uint64_t seed, int32_t nwords, const uint64_t *words) {
  uint64_t x = mix64(seed + GOLDEN);
  for (int32_t i = 0; i < nwords; ++i) x = kmpo_step(x, words[i]);
  return x;
}

/* MurmurHash3 32-bit finaliser (Appleby): a bijection on 32-bit words */
static uint32_t fmix32(uint32_t h) {
  h ^= h >> 16;
  h *= 0x85EBCA6Bu;
  h ^= h >> 13;
  h *= 0xC2B2AE35u;
  h ^= h >> 16;
  return h;
}

uint32_t kmpo_perm32(uint64_t roundkey, int32_t label) {
  return fmix32((uint32_t)label ^ (uint32_t)(roundkey >> 32));
}

int32_t kmpo_subround(uint64_t roundkey, int32_t v, int32_t S) {
  return (int32_t)(kmpo_step(roundkey, (uint64_t)(uint32_t)v) & (uint64_t)(S - 1));
}

static int32_t vwt(const int32_t *vw, int32_t v) { return vw ? vw[v] : 1; }
static int32_t ewt(const int32_t *ew, int64_t e) { return ew ? ew[e] : 1; }

int64_t kmpo_cut(int32_t n, const int64_t *xadj, const int32_t *adj, const int32_t *ew,
                 const int32_t *part) {
  int64_t s = 0;
  for (int32_t v = 0; v < n; ++v)
    for (int64_t e = xadj[v]; e < xadj[v + 1]; ++e)
      if (part[adj[e]] != part[v]) s += ewt(ew, e);
  return s / 2;
}

/* ------------------------------------------------------------------ LP -- */
typedef struct {
  int32_t u, target, own;
  int64_t gain;
} prop_t;

static int cmp_prop(const void *a, const void *b) {
  const prop_t *x = (const prop_t *)a, *y = (const prop_t *)b;
  if (x->target != y->target) return x->target < y->target ? -1 : 1;
  if (x->gain != y->gain) return x->gain > y->gain ? -1 : 1;
  return x->u < y->u ? -1 : (x->u > y->u);
}

/*
 * One run of size-constrained LP (Section 2) under readings R2-R6.
 * label[n] in/out, wt[nlab] label weights in/out, cap per label (NULL: U).
 */
static int32_t lp_run(int32_t n, const int64_t *xadj, const int32_t *adj, const int32_t *vw,
                      const int32_t *ew, int32_t *label, int64_t *wt, int32_t nlab,
                      const int32_t *cap, int32_t U, int32_t rounds, int32_t S,
                      uint64_t basekey, int32_t *fav, kmpo_lp_stats *st, int32_t sample,
                      int32_t sample_nodes) {
  int64_t *rating = (int64_t *)calloc((size_t)(nlab > 0 ? nlab : 1), sizeof(int64_t));
  char *active = (char *)malloc((size_t)(n > 0 ? n : 1));
  char *moved = (char *)malloc((size_t)(n > 0 ? n : 1));
  prop_t *props = (prop_t *)malloc(sizeof(prop_t) * (size_t)(n > 0 ? n : 1));
  int64_t maxdeg = 0;
  for (int32_t v = 0; v < n; ++v)
    if (xadj[v + 1] - xadj[v] > maxdeg) maxdeg = xadj[v + 1] - xadj[v];
  int32_t *cand = (int32_t *)malloc(sizeof(int32_t) * (size_t)(maxdeg + 1));
  for (int32_t v = 0; v < n; ++v) active[v] = 1;
  int32_t r;
  if (st) memset(st, 0, sizeof(*st));
  for (r = 0; r < rounds; ++r) {
    uint64_t rk = kmpo_step(basekey, (uint64_t)r);
    memset(moved, 0, (size_t)n);
    int64_t nmoved = 0, scanned = 0;
    for (int32_t s = 0; s < S; ++s) {
      if (sample > 0 && r * S + s >= sample) break;
      int32_t np = 0;
      const int32_t un = sample > 0 && sample_nodes > 0 && sample_nodes < n ? sample_nodes : n;
      for (int32_t u = 0; u < un; ++u) {
        if (!active[u] || kmpo_subround(rk, u, S) != s) continue;
        int64_t deg = xadj[u + 1] - xadj[u];
        if (deg == 0) continue;
        scanned += deg;
        int32_t own = label[u];
        /* r(K): summed edge weight from u to cluster K */
        int32_t nc = 0;
        for (int64_t e = xadj[u]; e < xadj[u + 1]; ++e) {
          int32_t K = label[adj[e]];
          if (rating[K] == 0) cand[nc++] = K;
          rating[K] += ewt(ew, e);
        }
        int64_t r_own = rating[own];
        int32_t best_c = -1, best_u = -1;
        for (int32_t i = 0; i < nc; ++i) {
          int32_t K = cand[i];
          if (K == own) continue;
          /* unconstrained best among K != own */
          if (best_u < 0 || rating[K] > rating[best_u] ||
              (rating[K] == rating[best_u] && kmpo_perm32(rk, K) < kmpo_perm32(rk, best_u)))
            best_u = K;
          int64_t capK = cap ? cap[K] : U;
          if (wt[K] + vwt(vw, u) > capK) continue;
          if (best_c < 0 || rating[K] > rating[best_c] ||
              (rating[K] == rating[best_c] && kmpo_perm32(rk, K) < kmpo_perm32(rk, best_c)))
            best_c = K;
        }
        if (best_c >= 0 && rating[best_c] > r_own) {
          props[np].u = u;
          props[np].target = best_c;
          props[np].own = own;
          props[np].gain = rating[best_c] - r_own;
          ++np;
        } else if (fav && best_u >= 0 && rating[best_u] > r_own) {
          fav[u] = best_u;
        }
        for (int32_t i = 0; i < nc; ++i) rating[cand[i]] = 0;
      }
      /* commit (R4): accept a prefix per target, against start-of-sub-round weights */
      qsort(props, (size_t)np, sizeof(prop_t), cmp_prop);
      char *acc = (char *)calloc((size_t)(np > 0 ? np : 1), 1);
      int32_t i = 0;
      while (i < np) {
        int32_t T = props[i].target, j = i;
        int64_t capT = cap ? cap[T] : U;
        int64_t pre = wt[T];
        while (j < np && props[j].target == T) {
          pre += vwt(vw, props[j].u);
          acc[j] = (pre <= capT);
          ++j;
        }
        i = j;
      }
      for (int32_t q = 0; q < np; ++q) {
        int32_t u = props[q].u;
        if (acc[q]) {
          wt[props[q].own] -= vwt(vw, u);
          wt[props[q].target] += vwt(vw, u);
          label[u] = props[q].target;
          moved[u] = 1;
          ++nmoved;
        } else if (fav) {
          fav[u] = props[q].target;
        }
      }
      free(acc);
    }
    if (st && r < 16) {
      st->moved[r] = nmoved;
      st->scanned[r] = scanned;
    }
    if (nmoved == 0) {
      ++r;
      break;
    }
    memset(active, 0, (size_t)n);
    for (int32_t v = 0; v < n; ++v)
      if (moved[v])
        for (int64_t e = xadj[v]; e < xadj[v + 1]; ++e) active[adj[e]] = 1;
  }
  if (st) st->rounds = r;
  free(rating); free(active); free(moved); free(props); free(cand);
  return r;
}

/* R7: pack isolated nodes in id order into chunks of weight <= U */
static void pack_isolated(int32_t n, const int64_t *xadj, const int32_t *vw, int32_t U,
                          int32_t *label) {
  int64_t P = 0;
  int64_t cur_chunk = -1;
  int32_t cur_label = -1;
  for (int32_t v = 0; v < n; ++v) {
    if (xadj[v + 1] != xadj[v]) continue;
    int64_t c = vwt(vw, v);
    int64_t q = P / U, q_end = (P + c - 1) / U;
    P += c;
    if (q != q_end) continue; /* straddles a chunk boundary: stays alone */
    if (q != cur_chunk) {
      cur_chunk = q;
      cur_label = label[v];
    }
    label[v] = cur_label;
  }
}

typedef struct {
  int32_t fav, u;
} favu_t;

static int cmp_favu(const void *a, const void *b) {
  const favu_t *x = (const favu_t *)a, *y = (const favu_t *)b;
  if (x->fav != y->fav) return x->fav < y->fav ? -1 : 1;
  return x->u < y->u ? -1 : (x->u > y->u);
}

static int32_t count_clusters(int32_t n, const int32_t *label) {
  char *used = (char *)calloc((size_t)(n > 0 ? n : 1), 1);
  int32_t c = 0;
  for (int32_t v = 0; v < n; ++v)
    if (!used[label[v]]) { used[label[v]] = 1; ++c; }
  free(used);
  return c;
}

/* R8: two-hop merging of singleton clusters that share a favoured cluster */
static void two_hop(int32_t n, const int32_t *vw, int32_t U, const int32_t *fav,
                    int32_t *label) {
  if (n <= 0) return;
  int32_t nc = count_clusters(n, label);
  if (2 * (int64_t)nc <= n) return;
  int64_t need = (int64_t)nc - n / 2;
  int32_t *size = (int32_t *)calloc((size_t)n, sizeof(int32_t));
  for (int32_t v = 0; v < n; ++v) size[label[v]]++;
  favu_t *c = (favu_t *)malloc(sizeof(favu_t) * (size_t)n);
  int32_t nc2 = 0;
  for (int32_t u = 0; u < n; ++u)
    if (size[label[u]] == 1 && fav[u] >= 0) {
      c[nc2].fav = fav[u];
      c[nc2].u = u;
      ++nc2;
    }
  qsort(c, (size_t)nc2, sizeof(favu_t), cmp_favu);
  int32_t i = 0;
  int64_t done = 0;
  while (i < nc2 && done < need) {
    int32_t j = i;
    while (j < nc2 && c[j].fav == c[i].fav) ++j;
    for (int32_t p = i; p + 1 < j && done < need; p += 2) {
      int32_t a = c[p].u, b = c[p + 1].u;
      if ((int64_t)vwt(vw, a) + vwt(vw, b) <= U) {
        label[b] = label[a];
        ++done;
      }
    }
    i = j;
  }
  free(size);
  free(c);
}

int32_t kmpo_cluster(int32_t n, const int64_t *xadj, const int32_t *adj, const int32_t *vw,
                     const int32_t *ew, int32_t U, int32_t rounds, uint64_t seed, int32_t level,
                     const kmpo_config *cfg, int32_t do_isolated, int32_t do_two_hop,
                     int32_t *label, int32_t *fav_out, kmpo_lp_stats *st) {
  uint64_t w[2] = {DOM_COARSEN, (uint64_t)(uint32_t)level};
  uint64_t basekey = kmpo_key(seed, 2, w);
  int64_t *wt = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  int32_t *fav = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  for (int32_t v = 0; v < n; ++v) {
    label[v] = v;
    wt[v] = vwt(vw, v);
    fav[v] = -1;
  }
  lp_run(n, xadj, adj, vw, ew, label, wt, n, NULL, U, rounds, cfg->subrounds, basekey, fav, st,
         cfg->sample_subrounds, cfg->sample_nodes);
  if (do_isolated) pack_isolated(n, xadj, vw, U, label);
  if (do_two_hop) two_hop(n, vw, U, fav, label);
  if (fav_out) memcpy(fav_out, fav, sizeof(int32_t) * (size_t)n);
  free(wt);
  free(fav);
  return count_clusters(n, label);
}

/* core used by the bipartitioner: LP + isolated packing with an explicit key */
int32_t kmpo_cluster_key(int32_t n, const int64_t *xadj, const int32_t *adj, const int32_t *vw,
                         const int32_t *ew, int32_t U, int32_t rounds, int32_t S,
                         uint64_t basekey, int32_t *label) {
  int64_t *wt = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  for (int32_t v = 0; v < n; ++v) {
    label[v] = v;
    wt[v] = vwt(vw, v);
  }
  lp_run(n, xadj, adj, vw, ew, label, wt, n, NULL, U, rounds, S, basekey, NULL, NULL, 0, 0);
  pack_isolated(n, xadj, vw, U, label);
  free(wt);
  return count_clusters(n, label);
}

/* ----------------------------------------------------------- contraction -- */
typedef struct {
  int32_t a, b, w;
} trip_t;

static int cmp_trip(const void *x, const void *y) {
  const trip_t *p = (const trip_t *)x, *q = (const trip_t *)y;
  if (p->a != q->a) return p->a < q->a ? -1 : 1;
  return p->b < q->b ? -1 : (p->b > q->b);
}

int32_t kmpo_contract(int32_t n, const int64_t *xadj, const int32_t *adj, const int32_t *vw,
                      const int32_t *ew, const int32_t *label, int32_t *map, kmpo_graph *out) {
  int32_t *cid = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  for (int32_t v = 0; v < n; ++v) cid[v] = 0;
  for (int32_t v = 0; v < n; ++v) cid[label[v]] = 1;
  int32_t nn = 0;
  for (int32_t v = 0; v < n; ++v) {
    int32_t f = cid[v];
    cid[v] = nn;
    nn += f;
  }
  for (int32_t v = 0; v < n; ++v) map[v] = cid[label[v]];
  free(cid);
  out->n = nn;
  out->vw = (int32_t *)calloc((size_t)(nn > 0 ? nn : 1), sizeof(int32_t));
  for (int32_t v = 0; v < n; ++v) out->vw[map[v]] += vwt(vw, v);
  int64_t M = xadj[n];
  trip_t *t = (trip_t *)malloc(sizeof(trip_t) * (size_t)(M > 0 ? M : 1));
  int64_t nt = 0;
  for (int32_t v = 0; v < n; ++v)
    for (int64_t e = xadj[v]; e < xadj[v + 1]; ++e) {
      int32_t a = map[v], b = map[adj[e]];
      if (a == b) continue;
      t[nt].a = a;
      t[nt].b = b;
      t[nt].w = ewt(ew, e);
      ++nt;
    }
  qsort(t, (size_t)nt, sizeof(trip_t), cmp_trip);
  out->xadj = (int64_t *)calloc((size_t)nn + 1, sizeof(int64_t));
  out->adj = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nt > 0 ? nt : 1));
  out->ew = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nt > 0 ? nt : 1));
  int64_t m = 0;
  for (int64_t i = 0; i < nt; ++i) {
    if (i > 0 && t[i - 1].a == t[i].a && t[i - 1].b == t[i].b) {
      out->ew[m - 1] += t[i].w;
    } else {
      out->adj[m] = t[i].b;
      out->ew[m] = t[i].w;
      out->xadj[t[i].a + 1]++;
      ++m;
    }
  }
  for (int32_t x = 0; x < nn; ++x) out->xadj[x + 1] += out->xadj[x];
  free(t);
  return nn;
}

void kmpo_graph_free(kmpo_graph *g) {
  if (!g) return;
  free(g->xadj); free(g->adj); free(g->vw); free(g->ew);
  g->xadj = NULL; g->adj = NULL; g->vw = NULL; g->ew = NULL;
}

/* ------------------------------------------------------------ refinement -- */
/* Section 4.3 "Local Improvement": the same LP over blocks with strict caps */
int64_t kmpo_refine(int32_t n, const int64_t *xadj, const int32_t *adj, const int32_t *vw,
                    const int32_t *ew, int32_t k, const int32_t *cap, int32_t rounds,
                    uint64_t seed, const kmpo_config *cfg, int32_t *part, kmpo_lp_stats *st) {
  uint64_t w[1] = {DOM_REFINE};
  uint64_t basekey = kmpo_key(seed, 1, w);
  int64_t *bw = (int64_t *)calloc((size_t)(k > 0 ? k : 1), sizeof(int64_t));
  for (int32_t v = 0; v < n; ++v) bw[part[v]] += vwt(vw, v);
  lp_run(n, xadj, adj, vw, ew, part, bw, k, cap, 0, rounds, cfg->subrounds, basekey, NULL, st, 0, 0);
  free(bw);
  return kmpo_cut(n, xadj, adj, ew, part);
}

/* ------------------------------------------- sequential asynchronous LP -- */
/* Quality reference: the paper's sequential semantics (Section 2), each move
 * applied immediately with the cap checked against the current weights, ties
 * kept by the own cluster then the smaller id.  Visiting order per round
 * (Section 4.1, "Iteration Order and Cache Locality"): exponentially spaced
 * degree buckets in increasing order, a seeded random order inside each
 * bucket (a fresh one every round). */
typedef struct {
  uint64_t key;
  int32_t v;
} vorder_t;

static int cmp_vorder(const void *x, const void *y) {
  const vorder_t *a = (const vorder_t *)x, *b = (const vorder_t *)y;
  if (a->key != b->key) return a->key < b->key ? -1 : 1;
  return a->v < b->v ? -1 : (a->v > b->v);
}

static uint64_t deg_bucket(int64_t d) {
  uint64_t b = 0;
  while (d > 0) {
    ++b;
    d >>= 1;
  }
  return b;  /* 0 for isolated nodes, else 1 + floor(log2 d) */
}

int32_t kmpo_async_cluster(int32_t n, const int64_t *xadj, const int32_t *adj,
                           const int32_t *vw, const int32_t *ew, int32_t U, int32_t rounds,
                           uint64_t seed, int32_t *label) {
  vorder_t *ord = (vorder_t *)malloc(sizeof(vorder_t) * (size_t)(n > 0 ? n : 1));
  int64_t *wt = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  int64_t *rating = (int64_t *)calloc((size_t)(n > 0 ? n : 1), sizeof(int64_t));
  int64_t maxdeg = 0;
  for (int32_t v = 0; v < n; ++v)
    if (xadj[v + 1] - xadj[v] > maxdeg) maxdeg = xadj[v + 1] - xadj[v];
  int32_t *cand = (int32_t *)malloc(sizeof(int32_t) * (size_t)(maxdeg + 1));
  for (int32_t v = 0; v < n; ++v) {
    label[v] = v;
    wt[v] = vwt(vw, v);
  }
  for (int32_t r = 0; r < rounds; ++r) {
    int64_t moved = 0;
    uint64_t rk = kmpo_step(seed, (uint64_t)r);
    for (int32_t v = 0; v < n; ++v) {
      ord[v].key = (deg_bucket(xadj[v + 1] - xadj[v]) << 32) | (uint64_t)kmpo_perm32(rk, v);
      ord[v].v = v;
    }
    qsort(ord, (size_t)n, sizeof(vorder_t), cmp_vorder);
    for (int32_t i = 0; i < n; ++i) {
      const int32_t u = ord[i].v;
      int32_t nc = 0, own = label[u];
      for (int64_t e = xadj[u]; e < xadj[u + 1]; ++e) {
        int32_t K = label[adj[e]];
        if (rating[K] == 0) cand[nc++] = K;
        rating[K] += ewt(ew, e);
      }
      int32_t best = own;
      for (int32_t i = 0; i < nc; ++i) {
        int32_t K = cand[i];
        if (K == own || wt[K] + vwt(vw, u) > U) continue;
        if (rating[K] > rating[best] || (rating[K] == rating[best] && best != own && K < best))
          best = K;
      }
      if (best != own) {
        wt[own] -= vwt(vw, u);
        wt[best] += vwt(vw, u);
        label[u] = best;
        ++moved;
      }
      for (int32_t i = 0; i < nc; ++i) rating[cand[i]] = 0;
    }
    if (!moved) break;
  }
  pack_isolated(n, xadj, vw, U, label);
  free(wt); free(rating); free(cand); free(ord);
  return count_clusters(n, label);
}
