// Device side of the learned seed proposer (shared by the training kernels
// and by the bipartitioner, which scores its coarsest graphs in place).
//
// Network: features x (8 per node), two layers
//   m_v = sum_u w(v,u) h_u / sum_u w(v,u)   (0 for isolated nodes)
//   h'_v = relu(W_self h_v + W_nbr m_v + b)  (8 -> 64 -> 64)
// and the read-out s_v = w_o . h2_v + b_o; BF16 weights, FP32 arithmetic.
// Features: 1; c(v)/mean c; deg/max deg; weighted degree over its mean; BFS
// hops from anchor a (smallest key, then id) and from anchor b (farthest
// from a, smallest id), each over (max hops + 1), unreachable 1; two +-1 key
// bits.  Features come from exact integer sums and correctly rounded fp64
// quotients; every product-accumulate of a layer is one fused multiply-add in
// a fixed order (CSR order for neighbour sums; for output o: b_o, then
// W_self[o][i] h_i and W_nbr[o][i] m_i for i = 0, 1, ...; read-out: b_o, then
// w_o[o] h2_o).  The scores are thus a fixed function of graph, key and
// weights, and the proposal order they induce is reproducible exactly.
#pragma once
#include <cuda_bf16.h>

#include "kmp_internal.cuh"

namespace kmp {

constexpr int MF = 8, MH = 64;
constexpr int P_W1S = 0, P_W1N = P_W1S + MH * MF, P_B1 = P_W1N + MH * MF, P_W2S = P_B1 + MH,
              P_W2N = P_W2S + MH * MH, P_B2 = P_W2N + MH * MH, P_WO = P_B2 + MH, P_BO = P_WO + MH,
              P_TOTAL = P_BO + 1;

// a graph seen through local node ids 0..n-1: row v is [xadj[v], xadj[v+1])
// of the edge arrays; a neighbour's local id is adj[e] - abase
template <class XT>
struct GView {
  int32_t n;
  const XT *xadj;
  const int32_t *adj;
  int32_t abase;
  const int32_t *vw;  // local index, nullable
  const int32_t *ew;  // edge index, nullable
};

__device__ __forceinline__ float wbf(const __nv_bfloat16 *W, int i) { return __bfloat162float(W[i]); }

// features of one graph by one CTA; d1, d2: scratch of n ints (local index)
template <class XT>
__device__ void mp_features(const GView<XT> &G, uint64_t key, float *X, int32_t *d1, int32_t *d2) {
  __shared__ double s_c, s_w;
  __shared__ unsigned long long s_md;
  int32_t n = G.n;
  if (threadIdx.x == 0) {
    s_c = 0;
    s_w = 0;
    s_md = 0;
  }
  __syncthreads();
  double lc = 0, lw = 0;
  unsigned long long md = 0;
  for (int32_t v = threadIdx.x; v < n; v += blockDim.x) {
    lc += G.vw ? G.vw[v] : 1;
    for (XT e = G.xadj[v]; e < G.xadj[v + 1]; ++e) lw += G.ew ? G.ew[e] : 1;
    unsigned long long d = (unsigned long long)(G.xadj[v + 1] - G.xadj[v]);
    md = d > md ? d : md;
  }
  atomicAdd(&s_c, lc);
  atomicAdd(&s_w, lw);
  atomicMax(&s_md, md);
  __syncthreads();
  // anchor a: smallest key, then smallest id
  __shared__ unsigned long long s_kmin;
  __shared__ int32_t s_src, s_D[2], s_chg[3];
  if (threadIdx.x == 0) {
    s_kmin = ~0ull;
    s_src = INT32_MAX;
  }
  __syncthreads();
  for (int32_t v = threadIdx.x; v < n; v += blockDim.x)
    atomicMin(&s_kmin, (unsigned long long)key_step(key, (uint64_t)(uint32_t)v));
  __syncthreads();
  for (int32_t v = threadIdx.x; v < n; v += blockDim.x)
    if (key_step(key, (uint64_t)(uint32_t)v) == s_kmin) atomicMin(&s_src, v);
  __syncthreads();
  // hop distances from a, then from b (farthest from a, smallest id), by
  // parallel relaxation d(v) = min(d(v), d(u) + 1) to the fixpoint (= BFS)
  for (int pass = 0; pass < 2 && n > 0; ++pass) {
    volatile int32_t *d = pass == 0 ? d1 : d2;
    int32_t src = s_src;
    for (int32_t v = threadIdx.x; v < n; v += blockDim.x) d[v] = v == src ? 0 : INT32_MAX;
    if (threadIdx.x == 0) {
      s_chg[0] = s_chg[1] = s_chg[2] = 0;
      s_D[pass] = 0;
    }
    __syncthreads();
    // at most n + 1 sweeps: every sweep that changes something lowers a distance
    for (int32_t it = 0; it <= n; ++it) {
      for (int32_t v = threadIdx.x; v < n; v += blockDim.x) {
        int32_t dv = d[v], best = dv;
        for (XT e = G.xadj[v]; e < G.xadj[v + 1]; ++e) {
          int32_t du = d[G.adj[e] - G.abase];
          if (du != INT32_MAX && du + 1 < best) best = du + 1;
        }
        if (best < dv) {
          d[v] = best;
          s_chg[it % 3] = 1;
        }
      }
      // flag (it + 1) % 3 was last read two sweeps ago: safe to clear now
      if (threadIdx.x == 0) s_chg[(it + 1) % 3] = 0;
      __syncthreads();
      if (!s_chg[it % 3]) break;
    }
    for (int32_t v = threadIdx.x; v < n; v += blockDim.x) {
      if (d[v] == INT32_MAX) d[v] = -1;
      else atomicMax(&s_D[pass], d[v]);
    }
    __syncthreads();
    if (pass == 0) {
      if (threadIdx.x == 0) s_src = INT32_MAX;
      __syncthreads();
      for (int32_t v = threadIdx.x; v < n; v += blockDim.x)
        if (d[v] == s_D[0]) atomicMin(&s_src, v);
      __syncthreads();
    }
  }
  int32_t s_D1 = s_D[0], s_D2 = s_D[1];
  double meanc = s_c / (n > 0 ? n : 1), meanw = s_w / (n > 0 ? n : 1);
  for (int32_t v = threadIdx.x; v < n; v += blockDim.x) {
    double wd = 0;
    for (XT e = G.xadj[v]; e < G.xadj[v + 1]; ++e) wd += G.ew ? G.ew[e] : 1;
    double deg = (double)(G.xadj[v + 1] - G.xadj[v]);
    uint64_t h = key_step(key, (uint64_t)(uint32_t)v);
    float *x = X + (int64_t)v * MF;
    x[0] = 1.f;
    x[1] = (float)((G.vw ? G.vw[v] : 1) / meanc);
    x[2] = s_md > 0 ? (float)(deg / (double)s_md) : 0.f;
    x[3] = meanw > 0 ? (float)(wd / meanw) : 0.f;
    x[4] = d1[v] >= 0 ? (float)((double)d1[v] / (double)(s_D1 + 1)) : 1.f;
    x[5] = d2[v] >= 0 ? (float)((double)d2[v] / (double)(s_D2 + 1)) : 1.f;
    x[6] = ((h >> 1) & 1) ? 1.f : -1.f;
    x[7] = ((h >> 2) & 1) ? 1.f : -1.f;
  }
  __syncthreads();
}

// neighbour mean of channel c of node v (d channels per node)
template <class XT>
__device__ __forceinline__ float mp_nbr_mean(const GView<XT> &G, const float *H, int d, int32_t v, int c) {
  float s = 0.f, ws = 0.f;
  for (XT e = G.xadj[v]; e < G.xadj[v + 1]; ++e) {
    float w = G.ew ? (float)G.ew[e] : 1.f;
    ws += w;
    s = __fmaf_rn(w, H[(int64_t)(G.adj[e] - G.abase) * d + c], s);
  }
  return ws > 0.f ? s / ws : 0.f;
}

// pre-activation of output o of a layer for node v
__device__ __forceinline__ float mp_preact(const __nv_bfloat16 *W, int ws_off, int wn_off, int b_off,
                                           int din, const float *hin, const float *min, int o) {
  float a = wbf(W, b_off + o);
  for (int i = 0; i < din; ++i) {
    a = __fmaf_rn(wbf(W, ws_off + o * din + i), hin[i], a);
    a = __fmaf_rn(wbf(W, wn_off + o * din + i), min[i], a);
  }
  return a;
}

__device__ __forceinline__ float mp_readout(const __nv_bfloat16 *W, const float *h2) {
  float s = wbf(W, P_BO);
  for (int o = 0; o < MH; ++o) s = __fmaf_rn(wbf(W, P_WO + o), h2[o], s);
  return s;
}

// forward of one graph by one CTA (inference): scores S[n]; scratch: n*(MF + 3*MH) floats
template <class XT>
__device__ void mp_forward_cta(const GView<XT> &G, const __nv_bfloat16 *W, const float *X, float *scr,
                               float *S) {
  int32_t n = G.n;
  float *M0 = scr, *H1 = M0 + (int64_t)n * MF, *M1 = H1 + (int64_t)n * MH, *H2 = M1 + (int64_t)n * MH;
  for (int64_t t = threadIdx.x; t < (int64_t)n * MF; t += blockDim.x)
    M0[t] = mp_nbr_mean(G, X, MF, (int32_t)(t / MF), (int)(t % MF));
  __syncthreads();
  for (int64_t t = threadIdx.x; t < (int64_t)n * MH; t += blockDim.x) {
    int32_t v = (int32_t)(t / MH);
    int o = (int)(t % MH);
    float a = mp_preact(W, P_W1S, P_W1N, P_B1, MF, X + (int64_t)v * MF, M0 + (int64_t)v * MF, o);
    H1[t] = a > 0.f ? a : 0.f;
  }
  __syncthreads();
  for (int64_t t = threadIdx.x; t < (int64_t)n * MH; t += blockDim.x)
    M1[t] = mp_nbr_mean(G, H1, MH, (int32_t)(t / MH), (int)(t % MH));
  __syncthreads();
  for (int64_t t = threadIdx.x; t < (int64_t)n * MH; t += blockDim.x) {
    int32_t v = (int32_t)(t / MH);
    int o = (int)(t % MH);
    float a = mp_preact(W, P_W2S, P_W2N, P_B2, MH, H1 + (int64_t)v * MH, M1 + (int64_t)v * MH, o);
    H2[t] = a > 0.f ? a : 0.f;
  }
  __syncthreads();
  for (int32_t v = threadIdx.x; v < n; v += blockDim.x) S[v] = mp_readout(W, H2 + (int64_t)v * MH);
  __syncthreads();
}

// order key of a score for the proposal: ascending key = descending score;
// -0 and +0 are the same score
__device__ __forceinline__ uint32_t mp_score_key(float s) {
  uint32_t u = s == 0.f ? 0u : __float_as_uint(s);
  u = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
  return ~u;
}

// the model the bipartitioner uses in learned mode (null: plain portfolio)
struct Proposer {
  const __nv_bfloat16 *W = nullptr;
};
Proposer &proposer();

// recorder of the bipartitioner's coarsest graphs and their winning sides
// (training data); device arrays, filled by reservation with atomics
struct SampleSink {
  unsigned long long *counters = nullptr;  // graphs, nodes, entries, dropped
  int64_t *rec = nullptr;                  // per graph: node base, n, entry base, m, key
  int32_t *deg = nullptr, *vw = nullptr, *side = nullptr;  // per node
  int32_t *adj = nullptr, *ew = nullptr;   // per entry, graph-local ids
  int32_t max_graphs = 0;
  int64_t max_nodes = 0, max_entries = 0;
  int32_t item_level = 0;  // 0: each item's coarsest graph and portfolio winner; 1: the item
                           // graph and its final bipartition
};
SampleSink &sample_sink();

}  // namespace kmp
