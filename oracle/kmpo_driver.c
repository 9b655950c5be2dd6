/*
 * CPU oracle, part 3: balance caps, adaptive imbalance, k-way balancing and
 * the deep multilevel driver (Algorithm 1 and 2).  Test infrastructure only.
 *
 * Readings:
 *  D1 Coarsening schedule (Section 4.1): k' = max(min(k, floor(n/C)), 1);
 *     while k' > 1 and n_i <= (k'/2) C, k' is halved; U = max(floor(eps c(V)
 *     / k'), max_v c(v)) at every level.  Coarsening stops at n_i <= 2C, when
 *     a clustering contracts nothing, or after a level that shrank by less
 *     than conv_num/conv_den (Algorithm 1 "has not converged").
 *  D2 Blocks per level (Algorithm 1, invariant (P)): k_i = k on the input
 *     graph, else ceil2(n_i / C), clamped to [2, k]; while fewer blocks exist
 *     every block with final count f_B >= 2 is bipartitioned into
 *     f = (floor(f_B/2), ceil(f_B/2)) (Section 3, "Handling General k"); new
 *     ids are handed out in ascending old id, child 0 first.
 *  D3 Adaptive imbalance (Algorithm 2 generalised by f_B):
 *     eps' = ((1+eps) c(V) f_B / (k c(B)))^(1/ceil(log2 f_B)) - 1, clamped at
 *     0; child targets t_j = ceil(c(B) f_j / f_B) and caps
 *     L_j = floor((1+eps') t_j) (Section 4.2, L_2 = (1+eps') ceil(c(V')/2)).
 *  D4 Block cap L(b) = floor(max((1+eps) c(V) f_b / k, c(V) f_b / k +
 *     max_v c(v))) (Section 2, L_max,k, scaled by the block's final count).
 *  D5 Balancing (Section 4.3): one pass over the starting state initialises
 *     the candidates (the paper's priority-queue initialisation): every node
 *     of an initially overloaded block that has an admissible other block gets
 *     d = max over admissible blocks of conn - conn(own) and the relative gain
 *     d*c(v) (d >= 0) or d/c(v) (d < 0), compared exactly.  Then the
 *     overloaded blocks are emptied one after the other in ascending id: nodes
 *     in (relative gain desc, id asc) order, each moved at its turn to the
 *     admissible block of largest current connectivity (ties: lowest id)
 *     until the block fits.
 *  D6 Final feasibility uses L_k = floor((1+eps) ceil(c(V)/k)) (Section 2,
 *     footnote; Section 5).
 *  D7 Replication (Section 3, "Parallelization"), with R = cfg->replicas
 *     standing for the PEs p: coarsening stops at n_i <= max(R, 2) C instead
 *     of 2C.  For R >= 2 the coarsest graph G_C is then taken by two copies,
 *     each solved recursively with R/2 from G_C under its own seed
 *     key(seed, {10, copy}): it coarsens further (with R/2, the same k'
 *     schedule and U), partitions and uncoarsens back to G_C, where its
 *     blocks follow the G_C rule k_i = ceil2(n_C / C).  The better of the two
 *     partitions of G_C is kept: the feasible one if only one is feasible
 *     under the D4 caps, else the one with the smaller cut, the first copy on
 *     a tie.  From G_C on the run continues as before (split rounds if
 *     applicable, balancing, refinement, then the finer levels).  R = 1 is
 *     the plain method.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <time.h>

#include "kmpo.h"

enum { DOM_COARSEN = 1, DOM_IP = 3, DOM_REFINE_LEVEL = 8, DOM_REPLICA = 10 };

uint64_t kmpo_step(uint64_t x, uint64_t w);

static int32_t vwt(const int32_t *vw, int32_t v) { return vw ? vw[v] : 1; }
static int32_t ewt(const int32_t *ew, int64_t e) { return ew ? ew[e] : 1; }

static double now_s(void) {
  struct timespec ts;
  clock_gettime(CLOCK_MONOTONIC, &ts);
  return (double)ts.tv_sec + 1e-9 * (double)ts.tv_nsec;
}

void kmpo_config_default(kmpo_config *c) {
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
  c->async_lp = 0;
  c->sample_subrounds = 0;
  c->sample_nodes = 0;
  c->adaptive = 0;
}

static int32_t ceil_log2(int32_t f) {
  int32_t j = 0;
  while ((1 << j) < f) ++j;
  return j;
}

double kmpo_eps_prime(double eps, int64_t cV, int32_t k, int64_t cB, int32_t fB) {
  double base = ((1.0 + eps) * (double)cV * (double)fB) / ((double)k * (double)cB);
  return pow(base, 1.0 / (double)ceil_log2(fB)) - 1.0;
}

void kmpo_split_caps(double eps, int64_t cV, int32_t k, int64_t cB, int32_t fB,
                     int32_t *target0, int32_t *target1, int32_t *L0, int32_t *L1) {
  int32_t f0 = fB / 2, f1 = fB - fB / 2;
  int64_t t0 = (cB * f0 + fB - 1) / fB, t1 = (cB * f1 + fB - 1) / fB;
  double e = cB > 0 ? kmpo_eps_prime(eps, cV, k, cB, fB) : 0.0;
  if (e < 0.0) e = 0.0;
  *target0 = (int32_t)t0;
  *target1 = (int32_t)t1;
  *L0 = (int32_t)floor((1.0 + e) * (double)t0);
  *L1 = (int32_t)floor((1.0 + e) * (double)t1);
}

int32_t kmpo_block_cap(double eps, int64_t cV, int32_t k, int32_t fb, int32_t maxc) {
  double a = (1.0 + eps) * (double)cV * (double)fb / (double)k;
  double b = (double)cV * (double)fb / (double)k + (double)maxc;
  return (int32_t)floor(a > b ? a : b);
}

/* ------------------------------------------------------------- balance -- */
typedef struct {
  int64_t d, c;
  int32_t v;
} rg_t;

/* relative gain order: descending, exact (D5) */
static int cmp_rg(const void *x, const void *y) {
  const rg_t *a = (const rg_t *)x, *b = (const rg_t *)y;
  int sa = a->d >= 0, sb = b->d >= 0;
  int c;
  if (sa != sb) c = sa ? -1 : 1;
  else if (sa) {
    int64_t p = a->d * a->c, q = b->d * b->c;
    c = p > q ? -1 : (p < q ? 1 : 0);
  } else {
    int64_t p = a->d * b->c, q = b->d * a->c; /* a.d/a.c vs b.d/b.c */
    c = p > q ? -1 : (p < q ? 1 : 0);
  }
  if (c) return c;
  return a->v < b->v ? -1 : (a->v > b->v);
}

int64_t kmpo_balance(int32_t n, const int64_t *xadj, const int32_t *adj, const int32_t *vw,
                     const int32_t *ew, int32_t k, const int32_t *cap, int32_t *part) {
  int64_t *bw = (int64_t *)calloc((size_t)k, sizeof(int64_t));
  int64_t *conn = (int64_t *)calloc((size_t)k, sizeof(int64_t));
  char *over = (char *)calloc((size_t)k, 1);
  for (int32_t v = 0; v < n; ++v) bw[part[v]] += vwt(vw, v);
  int32_t nover = 0;
  for (int32_t b = 0; b < k; ++b)
    if (bw[b] > cap[b]) { over[b] = 1; ++nover; }
  rg_t *cand = (rg_t *)malloc(sizeof(rg_t) * (size_t)(n > 0 ? n : 1));
  int32_t *cb = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  int64_t moved = 0;
  if (nover == 0) goto done;
  /* initialisation from the starting state: every node of an overloaded block
   * with an admissible other block becomes a candidate of its block */
  int32_t nc = 0;
  for (int32_t v = 0; v < n; ++v) {
    int32_t B = part[v];
    if (!over[B]) continue;
    for (int64_t e = xadj[v]; e < xadj[v + 1]; ++e) conn[part[adj[e]]] += ewt(ew, e);
    int64_t bestc = -1;
    for (int32_t b = 0; b < k; ++b) {
      if (b == B || bw[b] + vwt(vw, v) > cap[b]) continue;
      if (conn[b] > bestc) bestc = conn[b];
    }
    if (bestc >= 0) {
      cand[nc].d = bestc - conn[B];
      cand[nc].c = vwt(vw, v);
      cand[nc].v = v;
      ++nc;
    }
    for (int64_t e = xadj[v]; e < xadj[v + 1]; ++e) conn[part[adj[e]]] = 0;
    conn[B] = 0;
  }
  /* group by block (stable in id order), then order each group by relative gain */
  {
    int32_t *cnt = (int32_t *)calloc((size_t)k + 1, sizeof(int32_t));
    for (int32_t i = 0; i < nc; ++i) cnt[part[cand[i].v] + 1]++;
    for (int32_t b = 0; b < k; ++b) cnt[b + 1] += cnt[b];
    rg_t *tmp = (rg_t *)malloc(sizeof(rg_t) * (size_t)(nc > 0 ? nc : 1));
    int32_t *pos = (int32_t *)malloc(sizeof(int32_t) * (size_t)k);
    for (int32_t b = 0; b < k; ++b) pos[b] = cnt[b];
    for (int32_t i = 0; i < nc; ++i) tmp[pos[part[cand[i].v]]++] = cand[i];
    for (int32_t B = 0; B < k; ++B) {
      if (!over[B]) continue;
      int32_t lo = cnt[B], hi = cnt[B + 1];
      qsort(tmp + lo, (size_t)(hi - lo), sizeof(rg_t), cmp_rg);
      for (int32_t i = lo; i < hi && bw[B] > cap[B]; ++i) {
        int32_t v = tmp[i].v;
        for (int64_t e = xadj[v]; e < xadj[v + 1]; ++e) conn[part[adj[e]]] += ewt(ew, e);
        int32_t t = -1;
        for (int32_t b = 0; b < k; ++b) {
          if (b == B || bw[b] + vwt(vw, v) > cap[b]) continue;
          if (t < 0 || conn[b] > conn[t]) t = b;
        }
        for (int64_t e = xadj[v]; e < xadj[v + 1]; ++e) conn[part[adj[e]]] = 0;
        if (t < 0) continue;
        part[v] = t;
        bw[B] -= vwt(vw, v);
        bw[t] += vwt(vw, v);
        ++moved;
      }
    }
    free(cnt); free(tmp); free(pos);
  }
done:
  free(bw); free(conn); free(cand); free(cb); free(over);
  return moved;
}

/* --------------------------------------------------------------- driver -- */
typedef struct {
  int32_t n;
  int64_t *xadj;
  int32_t *adj, *vw, *ew, *map;
  int32_t owned;
} glvl_t;

static int32_t max_vw(int32_t n, const int32_t *vw) {
  int32_t m = 0;
  for (int32_t v = 0; v < n; ++v)
    if (vwt(vw, v) > m) m = vwt(vw, v);
  return m;
}

/* Algorithm 2: bipartition every block with f >= 2 (one split round) */
static void bipartition_blocks(const glvl_t *g, int32_t *part, int32_t *nblocks, int32_t *f,
                               double eps, int64_t cV, int32_t k, uint64_t roundkey,
                               const kmpo_config *cfg) {
  int32_t nb = *nblocks;
  int32_t *newid = (int32_t *)malloc(sizeof(int32_t) * (size_t)nb);
  int32_t *nf = (int32_t *)malloc(sizeof(int32_t) * (size_t)(2 * nb));
  int32_t nn = 0;
  for (int32_t b = 0; b < nb; ++b) {
    newid[b] = nn;
    if (f[b] >= 2) {
      nf[nn] = f[b] / 2;
      nf[nn + 1] = f[b] - f[b] / 2;
      nn += 2;
    } else {
      nf[nn] = f[b];
      nn += 1;
    }
  }
  /* members of each block in ascending id */
  int32_t *cnt = (int32_t *)calloc((size_t)nb + 1, sizeof(int32_t));
  for (int32_t v = 0; v < g->n; ++v) cnt[part[v] + 1]++;
  for (int32_t b = 0; b < nb; ++b) cnt[b + 1] += cnt[b];
  int32_t *mem = (int32_t *)malloc(sizeof(int32_t) * (size_t)(g->n > 0 ? g->n : 1));
  int32_t *pos = (int32_t *)malloc(sizeof(int32_t) * (size_t)nb);
  for (int32_t b = 0; b < nb; ++b) pos[b] = cnt[b];
  for (int32_t v = 0; v < g->n; ++v) mem[pos[part[v]]++] = v;
  int32_t *loc = (int32_t *)malloc(sizeof(int32_t) * (size_t)(g->n > 0 ? g->n : 1));
  int32_t *newpart = (int32_t *)malloc(sizeof(int32_t) * (size_t)(g->n > 0 ? g->n : 1));
  for (int32_t b = 0; b < nb; ++b)
    for (int32_t i = cnt[b]; i < cnt[b + 1]; ++i) loc[mem[i]] = i - cnt[b];
  for (int32_t b = 0; b < nb; ++b) {
    int32_t nbv = cnt[b + 1] - cnt[b];
    if (f[b] < 2) {
      for (int32_t i = cnt[b]; i < cnt[b + 1]; ++i) newpart[mem[i]] = newid[b];
      continue;
    }
    /* induced subgraph G[V_b] with local ids in ascending global id */
    int64_t *sx = (int64_t *)calloc((size_t)nbv + 1, sizeof(int64_t));
    int64_t tot = 0;
    for (int32_t i = 0; i < nbv; ++i) {
      int32_t v = mem[cnt[b] + i];
      for (int64_t e = g->xadj[v]; e < g->xadj[v + 1]; ++e)
        if (part[g->adj[e]] == b) ++tot;
    }
    int32_t *sa = (int32_t *)malloc(sizeof(int32_t) * (size_t)(tot > 0 ? tot : 1));
    int32_t *se = (int32_t *)malloc(sizeof(int32_t) * (size_t)(tot > 0 ? tot : 1));
    int32_t *sv = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nbv > 0 ? nbv : 1));
    int64_t m = 0, cB = 0;
    for (int32_t i = 0; i < nbv; ++i) {
      int32_t v = mem[cnt[b] + i];
      sv[i] = vwt(g->vw, v);
      cB += sv[i];
      for (int64_t e = g->xadj[v]; e < g->xadj[v + 1]; ++e)
        if (part[g->adj[e]] == b) {
          sa[m] = loc[g->adj[e]];
          se[m] = ewt(g->ew, e);
          ++m;
        }
      sx[i + 1] = m;
    }
    int32_t t0, t1, L0, L1;
    kmpo_split_caps(eps, cV, k, cB, f[b], &t0, &t1, &L0, &L1);
    int32_t *side = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nbv > 0 ? nbv : 1));
    kmpo_bipartition(nbv, sx, sa, sv, se, L0, L1, t0, t1, kmpo_step(roundkey, (uint64_t)b),
                     cfg, side);
    for (int32_t i = 0; i < nbv; ++i) newpart[mem[cnt[b] + i]] = newid[b] + side[i];
    free(sx); free(sa); free(se); free(sv); free(side);
  }
  memcpy(part, newpart, sizeof(int32_t) * (size_t)g->n);
  memcpy(f, nf, sizeof(int32_t) * (size_t)nn);
  *nblocks = nn;
  free(newid); free(nf); free(cnt); free(mem); free(pos); free(loc); free(newpart);
}

int32_t kmpo_bipartition_blocks(int32_t n, const int64_t *xadj, const int32_t *adj,
                                const int32_t *vw, const int32_t *ew, int32_t nblocks,
                                const int32_t *f_in, double eps, int64_t cV, int32_t k,
                                uint64_t roundkey, const kmpo_config *cfg, int32_t *part,
                                int32_t *f_out) {
  glvl_t g;
  g.n = n;
  g.xadj = (int64_t *)xadj;
  g.adj = (int32_t *)adj;
  g.vw = (int32_t *)vw;
  g.ew = (int32_t *)ew;
  g.map = NULL;
  g.owned = 0;
  int32_t *f = (int32_t *)malloc(sizeof(int32_t) * (size_t)(2 * nblocks + 2));
  memcpy(f, f_in, sizeof(int32_t) * (size_t)nblocks);
  int32_t nb = nblocks;
  bipartition_blocks(&g, part, &nb, f, eps, cV, k, roundkey, cfg);
  memcpy(f_out, f, sizeof(int32_t) * (size_t)nb);
  free(f);
  return nb;
}

/* D4 feasibility of a partition of one level */
static int level_feasible(const glvl_t *g, const int32_t *part, int32_t nblocks, const int32_t *f,
                          double eps, int64_t cV, int32_t k) {
  int64_t *bw = (int64_t *)calloc((size_t)nblocks, sizeof(int64_t));
  for (int32_t v = 0; v < g->n; ++v) bw[part[v]] += vwt(g->vw, v);
  int32_t maxc = max_vw(g->n, g->vw);
  int ok = 1;
  for (int32_t b = 0; b < nblocks; ++b)
    if (bw[b] > kmpo_block_cap(eps, cV, k, f[b], maxc)) ok = 0;
  free(bw);
  return ok;
}

typedef struct {
  int32_t *part;  /* on the hierarchy's first graph */
  int32_t nblocks;
  int32_t *f;     /* final block counts, 2k + 2 entries */
} deep_out;

/* Algorithm 1 on the hierarchy that starts at G0 (D1, D2, D7); `input`: G0 is
 * the input graph (k_i = k there); `top`: record the level statistics */
static void deep(const glvl_t *G0, int32_t R, uint64_t seed, int input, int top, int32_t n_in,
                 int32_t k, double eps, int64_t cV, const kmpo_config *cfg, kmpo_stats *st,
                 double *tip, double *tref, deep_out *out) {
  glvl_t lv[64];
  int32_t nl = 1;
  lv[0] = *G0;
  lv[0].map = NULL;
  lv[0].owned = 0;
  int64_t kp = n_in / cfg->C;
  if (kp > k) kp = k;
  if (kp < 1) kp = 1;
  const int64_t stop = (int64_t)(R > 2 ? R : 2) * cfg->C;
  /* D1: coarsening */
  while (nl < 63 && lv[nl - 1].n > stop) {
    glvl_t *g = &lv[nl - 1];
    while (kp > 1 && 2 * (int64_t)g->n <= kp * cfg->C) kp /= 2;
    int64_t U = (int64_t)floor(eps * (double)cV / (double)kp);
    int32_t maxc = max_vw(g->n, g->vw);
    if (U < maxc) U = maxc;
    if (U < 1) U = 1;
    if (top) {
      st->level_kp[nl - 1] = (int32_t)kp;
      st->level_U[nl - 1] = U;
      st->clustered = nl;
    }
    int32_t *label = (int32_t *)malloc(sizeof(int32_t) * (size_t)g->n);
    kmpo_lp_stats ls;
    int32_t nc;
    if (cfg->async_lp) {  /* quality reference: sequential asynchronous LP */
      uint64_t w[2] = {DOM_COARSEN, (uint64_t)(nl - 1)};
      nc = kmpo_async_cluster(g->n, g->xadj, g->adj, g->vw, g->ew, (int32_t)U, cfg->lp_rounds,
                              kmpo_key(seed, 2, w), label);
    } else {
      nc = kmpo_cluster(g->n, g->xadj, g->adj, g->vw, g->ew, (int32_t)U, cfg->lp_rounds, seed, nl - 1, cfg,
                        1, cfg->two_hop, label, NULL, &ls);
      for (int32_t r = 0; r < ls.rounds && r < 16; ++r) st->lp_scanned += ls.scanned[r];
    }
    if (nc == g->n) {
      free(label);
      break;
    }
    g->map = (int32_t *)malloc(sizeof(int32_t) * (size_t)g->n);
    kmpo_graph cg;
    double tc = now_s();
    kmpo_contract(g->n, g->xadj, g->adj, g->vw, g->ew, label, g->map, &cg);
    st->t_contract += now_s() - tc;
    free(label);
    lv[nl].n = cg.n;
    lv[nl].xadj = cg.xadj;
    lv[nl].adj = cg.adj;
    lv[nl].vw = cg.vw;
    lv[nl].ew = cg.ew;
    lv[nl].map = NULL;
    lv[nl].owned = 1;
    ++nl;
    if ((int64_t)cfg->conv_den * cg.n > (int64_t)cfg->conv_num * g->n) break;
  }
  if (top) {
    st->levels = nl;
    for (int32_t l = 0; l < nl && l < 64; ++l) {
      st->level_n[l] = lv[l].n;
      st->level_m[l] = lv[l].xadj[lv[l].n];
    }
  }
  /* D7: the coarsest graph's partition from two recursive copies, or {V} */
  int32_t *f = (int32_t *)malloc(sizeof(int32_t) * (size_t)(2 * k + 2));
  int32_t *cap = (int32_t *)malloc(sizeof(int32_t) * (size_t)(2 * k + 2));
  int32_t nblocks = 1;
  int32_t *part;
  const glvl_t *gc = &lv[nl - 1];
  if (R >= 2) {
    deep_out o[2];
    int fe[2];
    int64_t ct[2];
    for (int c = 0; c < 2; ++c) {
      uint64_t w[2] = {DOM_REPLICA, (uint64_t)c};
      deep(gc, R / 2, kmpo_key(seed, 2, w), 0, 0, n_in, k, eps, cV, cfg, st, tip, tref, &o[c]);
      fe[c] = level_feasible(gc, o[c].part, o[c].nblocks, o[c].f, eps, cV, k);
      ct[c] = kmpo_cut(gc->n, gc->xadj, gc->adj, gc->ew, o[c].part);
    }
    int pick = (fe[0] != fe[1]) ? (fe[0] ? 0 : 1) : (ct[1] < ct[0] ? 1 : 0);
    part = o[pick].part;
    nblocks = o[pick].nblocks;
    memcpy(f, o[pick].f, sizeof(int32_t) * (size_t)nblocks);
    free(o[1 - pick].part);
    free(o[0].f);
    free(o[1].f);
  } else {
    part = (int32_t *)calloc((size_t)gc->n, sizeof(int32_t));
    f[0] = k;
  }
  /* D2: uncoarsening with recursive bipartitioning, balancing, refinement */
  for (int32_t l = nl - 1; l >= 0; --l) {
    glvl_t *g = &lv[l];
    if (l < nl - 1) {
      int32_t *fine = (int32_t *)malloc(sizeof(int32_t) * (size_t)g->n);
      for (int32_t v = 0; v < g->n; ++v) fine[v] = part[g->map[v]];
      free(part);
      part = fine;
    }
    int64_t ki;
    if (input && l == 0) {
      ki = k;
    } else {
      ki = 1;
      while (ki * cfg->C < g->n) ki *= 2;
    }
    if (ki > k) ki = k;
    if (ki < 2) ki = 2;
    double a = now_s();
    for (int32_t j = 0; nblocks < ki; ++j) {
      uint64_t w[3] = {DOM_IP, (uint64_t)l, (uint64_t)j};
      bipartition_blocks(g, part, &nblocks, f, eps, cV, k, kmpo_key(seed, 3, w), cfg);
    }
    double b = now_s();
    *tip += b - a;
    if (top) st->level_k[l] = nblocks;
    int32_t maxc = max_vw(g->n, g->vw);
    for (int32_t i = 0; i < nblocks; ++i) cap[i] = kmpo_block_cap(eps, cV, k, f[i], maxc);
    double tb = now_s();
    kmpo_balance(g->n, g->xadj, g->adj, g->vw, g->ew, nblocks, cap, part);
    st->t_balance += now_s() - tb;
    uint64_t w2[2] = {DOM_REFINE_LEVEL, (uint64_t)l};
    kmpo_lp_stats ls;
    kmpo_refine(g->n, g->xadj, g->adj, g->vw, g->ew, nblocks, cap, cfg->refine_rounds,
                kmpo_key(seed, 2, w2), cfg, part, &ls);
    for (int32_t r = 0; r < ls.rounds && r < 16; ++r) st->refine_scanned += ls.scanned[r];
    *tref += now_s() - b;
  }
  free(cap);
  for (int32_t l = 0; l < nl; ++l) {
    free(lv[l].map);
    if (lv[l].owned) {
      free(lv[l].xadj); free(lv[l].adj); free(lv[l].vw); free(lv[l].ew);
    }
  }
  out->part = part;
  out->nblocks = nblocks;
  out->f = f;
}

int32_t kmpo_partition(int32_t n, const int64_t *xadj, const int32_t *adj, const int32_t *vw,
                       const int32_t *ew, int32_t k, double eps, uint64_t seed,
                       const kmpo_config *cfg, int32_t *part_out, kmpo_stats *st) {
  double t0 = now_s();
  kmpo_stats dummy;
  if (!st) st = &dummy;
  memset(st, 0, sizeof(*st));
  if (k <= 1) {
    for (int32_t v = 0; v < n; ++v) part_out[v] = 0;
    st->feasible = 1;
    return 0;
  }
  int64_t cV = 0;
  for (int32_t v = 0; v < n; ++v) cV += vwt(vw, v);
  glvl_t g0;
  g0.n = n;
  g0.xadj = (int64_t *)xadj;
  g0.adj = (int32_t *)adj;
  g0.vw = (int32_t *)vw;
  g0.ew = (int32_t *)ew;
  g0.map = NULL;
  g0.owned = 0;
  double tip = 0, tref = 0;
  deep_out o;
  deep(&g0, cfg->replicas > 1 ? cfg->replicas : 1, seed, 1, 1, n, k, eps, cV, cfg, st, &tip, &tref, &o);
  memcpy(part_out, o.part, sizeof(int32_t) * (size_t)n);
  free(o.part);
  free(o.f);
  /* D6 */
  int64_t Lk = (int64_t)floor((1.0 + eps) * (double)((cV + k - 1) / k));
  int64_t *bw = (int64_t *)calloc((size_t)k, sizeof(int64_t));
  for (int32_t v = 0; v < n; ++v) bw[part_out[v]] += vwt(vw, v);
  int32_t feas = 1;
  for (int32_t b = 0; b < k; ++b)
    if (bw[b] > Lk) feas = 0;
  free(bw);
  st->cut = kmpo_cut(n, xadj, adj, ew, part_out);
  st->feasible = feas;
  st->t_ip = tip;
  st->t_refine = tref;
  st->t_total = now_s() - t0;
  st->t_coarsen = st->t_total - tip - tref;
  return feas ? 0 : -5;
}
