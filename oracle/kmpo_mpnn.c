/*
 * CPU oracle, part 4: the learned seed proposer for the bipartitioner's
 * coarsest graphs (test infrastructure only).  The paper repeats simple
 * bipartitioning algorithms several times and keeps the best (Section 4.2);
 * here a small message-passing network scores the nodes of a coarsest graph
 * and the score order seeds one bipartition that then goes through the same
 * 2-way FM and the same feasible/lower-cut selection as the portfolio.
 *
 * Network (fp64 here): per node features x (8), two layers
 *   m_v = sum_u w(v,u) h_u / sum_u w(v,u)      (0 for isolated nodes)
 *   h'_v = relu(W_self h_v + W_nbr m_v + b)    (8 -> 64 -> 64)
 * and a linear read-out s_v = w_o . h2_v + b_o.
 * Features: 1; c(v)/mean c; deg/max deg; weighted degree /
 * mean; BFS hops from anchor a (smallest key) and from anchor b (farthest from
 * a, smallest id), each divided by (max hops + 1), unreachable = 1; two
 * +-1 key bits (symmetry breaking).
 * Loss: per graph min over the two block orientations of the mean binary
 * cross-entropy of sigmoid(s) against the best-of-portfolio sides.
 * Proposal: nodes by (score desc, id asc) join block 0 while it stays within
 * its target (first fit), like the random start with a learned order.
 * Every feature is an integer sum or a correctly rounded quotient of integer
 * sums (no transcendental function), so a GPU computes the same values.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "kmpo.h"

#define F_IN 8
#define HID 64
/* parameter layout */
#define P_W1S 0
#define P_W1N (P_W1S + HID * F_IN)
#define P_B1 (P_W1N + HID * F_IN)
#define P_W2S (P_B1 + HID)
#define P_W2N (P_W2S + HID * HID)
#define P_B2 (P_W2N + HID * HID)
#define P_WO (P_B2 + HID)
#define P_BO (P_WO + HID)
#define P_TOTAL (P_BO + 1)

uint64_t kmpo_step(uint64_t x, uint64_t w);

int32_t kmpo_mpnn_num_params(void) { return P_TOTAL; }

static double ewt(const int32_t *ew, int64_t e) { return ew ? (double)ew[e] : 1.0; }

static void bfs(int32_t n, const int64_t *xadj, const int32_t *adj, int32_t src, int32_t *dist,
                int32_t *q) {
  for (int32_t v = 0; v < n; ++v) dist[v] = -1;
  int32_t h = 0, t = 0;
  dist[src] = 0;
  q[t++] = src;
  while (h < t) {
    int32_t v = q[h++];
    for (int64_t e = xadj[v]; e < xadj[v + 1]; ++e)
      if (dist[adj[e]] < 0) {
        dist[adj[e]] = dist[v] + 1;
        q[t++] = adj[e];
      }
  }
}

void kmpo_mpnn_features(int32_t n, const int64_t *xadj, const int32_t *adj, const int32_t *vw,
                        const int32_t *ew, uint64_t key, double *X) {
  if (n <= 0) return;
  double cs = 0, ws = 0;
  int64_t maxdeg = 0;
  for (int32_t v = 0; v < n; ++v) {
    cs += vw ? vw[v] : 1;
    for (int64_t e = xadj[v]; e < xadj[v + 1]; ++e) ws += ewt(ew, e);
    if (xadj[v + 1] - xadj[v] > maxdeg) maxdeg = xadj[v + 1] - xadj[v];
  }
  double meanc = cs / n, meanw = ws / n;
  int32_t *d1 = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
  int32_t *d2 = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
  int32_t *q = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
  int32_t a = 0;
  uint64_t best = kmpo_step(key, 0);
  for (int32_t v = 1; v < n; ++v) {
    uint64_t h = kmpo_step(key, (uint64_t)(uint32_t)v);
    if (h < best) { best = h; a = v; }
  }
  bfs(n, xadj, adj, a, d1, q);
  int32_t b = a, D1 = 0;
  for (int32_t v = 0; v < n; ++v)
    if (d1[v] > D1) { D1 = d1[v]; b = v; }
  bfs(n, xadj, adj, b, d2, q);
  int32_t D2 = 0;
  for (int32_t v = 0; v < n; ++v)
    if (d2[v] > D2) D2 = d2[v];
  for (int32_t v = 0; v < n; ++v) {
    double wd = 0;
    for (int64_t e = xadj[v]; e < xadj[v + 1]; ++e) wd += ewt(ew, e);
    double *x = X + (size_t)v * F_IN;
    int64_t deg = xadj[v + 1] - xadj[v];
    uint64_t h = kmpo_step(key, (uint64_t)(uint32_t)v);
    x[0] = 1.0;
    x[1] = (vw ? vw[v] : 1) / meanc;
    x[2] = maxdeg > 0 ? (double)deg / (double)maxdeg : 0.0;
    x[3] = meanw > 0 ? wd / meanw : 0.0;
    x[4] = d1[v] >= 0 ? (double)d1[v] / (double)(D1 + 1) : 1.0;
    x[5] = d2[v] >= 0 ? (double)d2[v] / (double)(D2 + 1) : 1.0;
    x[6] = ((h >> 1) & 1) ? 1.0 : -1.0;
    x[7] = ((h >> 2) & 1) ? 1.0 : -1.0;
  }
  free(d1); free(d2); free(q);
}

/* neighbour mean of a d-dimensional node signal */
static void nbr_mean(int32_t n, const int64_t *xadj, const int32_t *adj, const int32_t *ew,
                     const double *Hin, int32_t d, double *M) {
  for (int32_t v = 0; v < n; ++v) {
    double *m = M + (size_t)v * d;
    for (int32_t j = 0; j < d; ++j) m[j] = 0;
    double ws = 0;
    for (int64_t e = xadj[v]; e < xadj[v + 1]; ++e) {
      double w = ewt(ew, e);
      ws += w;
      const double *hu = Hin + (size_t)adj[e] * d;
      for (int32_t j = 0; j < d; ++j) m[j] += w * hu[j];
    }
    if (ws > 0)
      for (int32_t j = 0; j < d; ++j) m[j] /= ws;
  }
}

/* cache layout (per node): M0[8] A1[64] H1[64] M1[64] A2[64] H2[64] */
#define C_STRIDE (F_IN + 5 * HID)

void kmpo_mpnn_forward(int32_t n, const int64_t *xadj, const int32_t *adj, const int32_t *ew,
                       const double *X, const double *P, double *S, double *cache) {
  double *M0 = (double *)malloc(sizeof(double) * (size_t)n * F_IN + 8);
  double *H1 = (double *)malloc(sizeof(double) * (size_t)n * HID + 8);
  double *A1 = (double *)malloc(sizeof(double) * (size_t)n * HID + 8);
  double *M1 = (double *)malloc(sizeof(double) * (size_t)n * HID + 8);
  double *A2 = (double *)malloc(sizeof(double) * (size_t)n * HID + 8);
  double *H2 = (double *)malloc(sizeof(double) * (size_t)n * HID + 8);
  nbr_mean(n, xadj, adj, ew, X, F_IN, M0);
  for (int32_t v = 0; v < n; ++v)
    for (int32_t o = 0; o < HID; ++o) {
      double a = P[P_B1 + o];
      for (int32_t i = 0; i < F_IN; ++i)
        a += P[P_W1S + o * F_IN + i] * X[(size_t)v * F_IN + i] +
             P[P_W1N + o * F_IN + i] * M0[(size_t)v * F_IN + i];
      A1[(size_t)v * HID + o] = a;
      H1[(size_t)v * HID + o] = a > 0 ? a : 0;
    }
  nbr_mean(n, xadj, adj, ew, H1, HID, M1);
  for (int32_t v = 0; v < n; ++v) {
    double s = P[P_BO];
    for (int32_t o = 0; o < HID; ++o) {
      double a = P[P_B2 + o];
      for (int32_t i = 0; i < HID; ++i)
        a += P[P_W2S + o * HID + i] * H1[(size_t)v * HID + i] +
             P[P_W2N + o * HID + i] * M1[(size_t)v * HID + i];
      A2[(size_t)v * HID + o] = a;
      H2[(size_t)v * HID + o] = a > 0 ? a : 0;
      s += P[P_WO + o] * H2[(size_t)v * HID + o];
    }
    S[v] = s;
  }
  if (cache)
    for (int32_t v = 0; v < n; ++v) {
      double *c = cache + (size_t)v * C_STRIDE;
      memcpy(c, M0 + (size_t)v * F_IN, sizeof(double) * F_IN);
      memcpy(c + F_IN, A1 + (size_t)v * HID, sizeof(double) * HID);
      memcpy(c + F_IN + HID, H1 + (size_t)v * HID, sizeof(double) * HID);
      memcpy(c + F_IN + 2 * HID, M1 + (size_t)v * HID, sizeof(double) * HID);
      memcpy(c + F_IN + 3 * HID, A2 + (size_t)v * HID, sizeof(double) * HID);
      memcpy(c + F_IN + 4 * HID, H2 + (size_t)v * HID, sizeof(double) * HID);
    }
  free(M0); free(H1); free(A1); free(M1); free(A2); free(H2);
}

static double softplus(double z) { return z > 0 ? z + log1p(exp(-z)) : log1p(exp(z)); }

/* symmetric BCE over one graph; writes dL/ds into gS; returns the loss */
double kmpo_mpnn_loss(int32_t n, const double *S, const int32_t *side, double *gS) {
  if (n <= 0) return 0;
  double l0 = 0, l1 = 0;
  for (int32_t v = 0; v < n; ++v) {
    double y = side[v] == 0 ? 1.0 : 0.0; /* target: block 0 */
    l0 += softplus(S[v]) - y * S[v];
    l1 += softplus(S[v]) - (1.0 - y) * S[v];
  }
  int flip = l1 < l0;
  for (int32_t v = 0; v < n; ++v) {
    double y = side[v] == 0 ? 1.0 : 0.0;
    if (flip) y = 1.0 - y;
    double p = 1.0 / (1.0 + exp(-S[v]));
    if (gS) gS[v] = (p - y) / n;
  }
  return (flip ? l1 : l0) / n;
}

void kmpo_mpnn_backward(int32_t n, const int64_t *xadj, const int32_t *adj, const int32_t *ew,
                        const double *X, const double *P, const double *gS, double *gP) {
  double *cache = (double *)malloc(sizeof(double) * (size_t)n * C_STRIDE + 8);
  double *S = (double *)malloc(sizeof(double) * (size_t)n + 8);
  kmpo_mpnn_forward(n, xadj, adj, ew, X, P, S, cache);
  memset(gP, 0, sizeof(double) * P_TOTAL);
  double *gA2 = (double *)calloc((size_t)n * HID + 8, sizeof(double));
  double *gM1 = (double *)calloc((size_t)n * HID + 8, sizeof(double));
  double *gH1 = (double *)calloc((size_t)n * HID + 8, sizeof(double));
  double *wdeg = (double *)calloc((size_t)n + 1, sizeof(double));
  for (int32_t v = 0; v < n; ++v)
    for (int64_t e = xadj[v]; e < xadj[v + 1]; ++e) wdeg[v] += ewt(ew, e);
  for (int32_t v = 0; v < n; ++v) {
    const double *c = cache + (size_t)v * C_STRIDE;
    const double *A2 = c + F_IN + 3 * HID, *H2 = c + F_IN + 4 * HID;
    const double *H1 = c + F_IN + HID, *M1 = c + F_IN + 2 * HID;
    gP[P_BO] += gS[v];
    for (int32_t o = 0; o < HID; ++o) {
      gP[P_WO + o] += gS[v] * H2[o];
      double g = A2[o] > 0 ? gS[v] * P[P_WO + o] : 0.0;
      gA2[(size_t)v * HID + o] = g;
      gP[P_B2 + o] += g;
      for (int32_t i = 0; i < HID; ++i) {
        gP[P_W2S + o * HID + i] += g * H1[i];
        gP[P_W2N + o * HID + i] += g * M1[i];
      }
    }
    for (int32_t i = 0; i < HID; ++i) {
      double gs = 0, gm = 0;
      for (int32_t o = 0; o < HID; ++o) {
        gs += P[P_W2S + o * HID + i] * gA2[(size_t)v * HID + o];
        gm += P[P_W2N + o * HID + i] * gA2[(size_t)v * HID + o];
      }
      gH1[(size_t)v * HID + i] += gs;
      gM1[(size_t)v * HID + i] = gm;
    }
  }
  /* m1_v = sum_u w(v,u)/wdeg(v) h1_u  =>  gH1_u += sum_v w(v,u)/wdeg(v) gM1_v */
  for (int32_t v = 0; v < n; ++v) {
    if (wdeg[v] <= 0) continue;
    for (int64_t e = xadj[v]; e < xadj[v + 1]; ++e) {
      double f = ewt(ew, e) / wdeg[v];
      int32_t u = adj[e];
      for (int32_t i = 0; i < HID; ++i) gH1[(size_t)u * HID + i] += f * gM1[(size_t)v * HID + i];
    }
  }
  for (int32_t v = 0; v < n; ++v) {
    const double *c = cache + (size_t)v * C_STRIDE;
    const double *M0 = c, *A1 = c + F_IN;
    for (int32_t o = 0; o < HID; ++o) {
      double g = A1[o] > 0 ? gH1[(size_t)v * HID + o] : 0.0;
      gP[P_B1 + o] += g;
      for (int32_t i = 0; i < F_IN; ++i) {
        gP[P_W1S + o * F_IN + i] += g * X[(size_t)v * F_IN + i];
        gP[P_W1N + o * F_IN + i] += g * M0[i];
      }
    }
  }
  free(cache); free(S); free(gA2); free(gM1); free(gH1); free(wdeg);
}

typedef struct {
  double s;
  int32_t v;
} sv_t;

static int cmp_sv(const void *a, const void *b) {
  const sv_t *x = (const sv_t *)a, *y = (const sv_t *)b;
  if (x->s != y->s) return x->s > y->s ? -1 : 1;
  return x->v < y->v ? -1 : (x->v > y->v);
}

void kmpo_mpnn_propose(int32_t n, const int32_t *vw, const double *S, int32_t target0, int32_t *side) {
  sv_t *o = (sv_t *)malloc(sizeof(sv_t) * (size_t)(n > 0 ? n : 1));
  for (int32_t v = 0; v < n; ++v) {
    o[v].s = S[v];
    o[v].v = v;
  }
  qsort(o, (size_t)n, sizeof(sv_t), cmp_sv);
  int64_t W0 = 0;
  for (int32_t v = 0; v < n; ++v) side[v] = 1;
  for (int32_t i = 0; i < n; ++i) {
    int32_t v = o[i].v;
    int64_t c = vw ? vw[v] : 1;
    if (W0 + c <= target0) {
      side[v] = 0;
      W0 += c;
    }
  }
  free(o);
}

/* ----------------------------------------------------------------------
 * Inference in the kernel's precision.  The score order decides an integer
 * result (the proposal), so both sides take that decision in the same
 * arithmetic: features in fp64 from integer sums (exact) and correctly
 * rounded divisions, rounded once to fp32; layers in fp32 with every
 * product-accumulate a fused multiply-add in this fixed order:
 *   neighbour mean:  s = fma(w(v,u), h_u, s) over v's row in CSR order,
 *                    then s / sum w (0 for isolated nodes)
 *   pre-activation:  a = b_o; for i: a = fma(Ws[o][i], h[i], a);
 *                                    a = fma(Wn[o][i], m[i], a)
 *   read-out:        s = b_o; for o: s = fma(w_o[o], h2[o], s)
 * W holds the network's parameters as fp32 values (BF16-representable).
 */
static void nbr_mean_f32(int32_t n, const int64_t *xadj, const int32_t *adj, const int32_t *ew,
                         const float *Hin, int32_t d, float *M) {
  for (int32_t v = 0; v < n; ++v)
    for (int32_t j = 0; j < d; ++j) {
      float s = 0.f, ws = 0.f;
      for (int64_t e = xadj[v]; e < xadj[v + 1]; ++e) {
        float w = ew ? (float)ew[e] : 1.f;
        ws += w;
        s = fmaf(w, Hin[(size_t)adj[e] * d + j], s);
      }
      M[(size_t)v * d + j] = ws > 0.f ? s / ws : 0.f;
    }
}

static void layer_f32(int32_t n, const float *W, int32_t ws, int32_t wn, int32_t b, int32_t din,
                      const float *Hin, const float *M, float *H) {
  for (int32_t v = 0; v < n; ++v)
    for (int32_t o = 0; o < HID; ++o) {
      float a = W[b + o];
      for (int32_t i = 0; i < din; ++i) {
        a = fmaf(W[ws + o * din + i], Hin[(size_t)v * din + i], a);
        a = fmaf(W[wn + o * din + i], M[(size_t)v * din + i], a);
      }
      H[(size_t)v * HID + o] = a > 0.f ? a : 0.f;
    }
}

void kmpo_mpnn_scores_f32(int32_t n, const int64_t *xadj, const int32_t *adj, const int32_t *vw,
                          const int32_t *ew, uint64_t key, const float *W, float *S) {
  if (n <= 0) return;
  double *Xd = (double *)malloc(sizeof(double) * (size_t)n * F_IN);
  float *X = (float *)malloc(sizeof(float) * (size_t)n * F_IN);
  float *M0 = (float *)malloc(sizeof(float) * (size_t)n * F_IN);
  float *H1 = (float *)malloc(sizeof(float) * (size_t)n * HID);
  float *M1 = (float *)malloc(sizeof(float) * (size_t)n * HID);
  float *H2 = (float *)malloc(sizeof(float) * (size_t)n * HID);
  kmpo_mpnn_features(n, xadj, adj, vw, ew, key, Xd);
  for (size_t i = 0; i < (size_t)n * F_IN; ++i) X[i] = (float)Xd[i];
  nbr_mean_f32(n, xadj, adj, ew, X, F_IN, M0);
  layer_f32(n, W, P_W1S, P_W1N, P_B1, F_IN, X, M0, H1);
  nbr_mean_f32(n, xadj, adj, ew, H1, HID, M1);
  layer_f32(n, W, P_W2S, P_W2N, P_B2, HID, H1, M1, H2);
  for (int32_t v = 0; v < n; ++v) {
    float s = W[P_BO];
    for (int32_t o = 0; o < HID; ++o) s = fmaf(W[P_WO + o], H2[(size_t)v * HID + o], s);
    S[v] = s;
  }
  free(Xd); free(X); free(M0); free(H1); free(M1); free(H2);
}

/* order key of a score for the proposal: ascending key = descending score;
 * -0 and +0 are the same score */
uint32_t kmpo_mpnn_score_key(float s) {
  uint32_t u = 0;
  if (s != 0.f) memcpy(&u, &s, sizeof u);
  u = (u & 0x80000000u) ? ~u : (u | 0x80000000u); /* ascending in s */
  return ~u;
}

/* the proposer the bipartitioner uses in learned mode (copied; NULL clears) */
static float g_prop[P_TOTAL];
static int g_have_prop;

void kmpo_set_proposer(const float *W) {
  g_have_prop = W != NULL;
  if (W) memcpy(g_prop, W, sizeof g_prop);
}

const float *kmpo_proposer(void) { return g_have_prop ? g_prop : NULL; }

/* learned start: nodes by (score key asc, id asc) join block 0 while it stays
 * within target0 (first fit) */
typedef struct {
  uint32_t k;
  int32_t v;
} kv_t;

static int cmp_kv(const void *a, const void *b) {
  const kv_t *x = (const kv_t *)a, *y = (const kv_t *)b;
  if (x->k != y->k) return x->k < y->k ? -1 : 1;
  return x->v < y->v ? -1 : (x->v > y->v);
}

void kmpo_learned_initial(int32_t n, const int64_t *xadj, const int32_t *adj, const int32_t *vw,
                          const int32_t *ew, int32_t target0, uint64_t key, const float *W,
                          int32_t *side) {
  float *S = (float *)malloc(sizeof(float) * (size_t)(n > 0 ? n : 1));
  kv_t *o = (kv_t *)malloc(sizeof(kv_t) * (size_t)(n > 0 ? n : 1));
  kmpo_mpnn_scores_f32(n, xadj, adj, vw, ew, key, W, S);
  for (int32_t v = 0; v < n; ++v) {
    o[v].k = kmpo_mpnn_score_key(S[v]);
    o[v].v = v;
  }
  qsort(o, (size_t)n, sizeof(kv_t), cmp_kv);
  int64_t W0 = 0;
  for (int32_t v = 0; v < n; ++v) side[v] = 1;
  for (int32_t i = 0; i < n; ++i) {
    int32_t v = o[i].v;
    int64_t c = vw ? vw[v] : 1;
    if (W0 + c <= target0) {
      side[v] = 0;
      W0 += c;
    }
  }
  free(S);
  free(o);
}
