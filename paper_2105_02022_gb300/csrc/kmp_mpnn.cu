// Learned seed proposer: training and batched inference kernels.
//
// The paper bipartitions a coarsest graph by repeating simple algorithms
// several times and keeping the best (Section 4.2).  Here a small
// message-passing network (kmp_mpnn.cuh) scores the nodes; the score order
// seeds one extra bipartition in the bipartitioner, which goes through the
// same 2-way FM and the same feasible/lower-cut selection as the portfolio.
//
// A batch is one disjoint union of graphs in CSR form (union node ids) plus
// the node offset of each graph: layers are node-parallel over the union,
// features and loss work per graph.  Training keeps fp32 master weights and
// Adam moments and uses a BF16 copy of the weights in every kernel.
#include <algorithm>
#include <cmath>
#include <vector>

#include "kmp_mpnn.cuh"

struct kmp_mpnn {
  float *master = nullptr;
  __nv_bfloat16 *wbf = nullptr;
  float *am = nullptr, *av = nullptr, *grad = nullptr;
  int64_t step = 0;
};

static_assert(kmp::P_TOTAL == KMP_MPNN_PARAMS, "parameter layout of kmp.h");

namespace kmp {

static Proposer g_proposer;
Proposer &proposer() { return g_proposer; }
static SampleSink g_sink;
SampleSink &sample_sink() { return g_sink; }

static void sink_release() {
  SampleSink &K = g_sink;
  for (void *p : {(void *)K.counters, (void *)K.rec, (void *)K.deg, (void *)K.vw, (void *)K.side,
                  (void *)K.adj, (void *)K.ew})
    if (p) dfree(p);
  K = SampleSink{};
}

struct Batch {
  int32_t ng = 0, N = 0;
  int64_t E = 0;
  DBuf<int32_t> noff, adj, vw, ew, side;
  DBuf<int64_t> xadj;
  DBuf<uint64_t> keys;
};

// ---------------------------------------------------------------- kernels
__global__ void k_mp_features(int32_t ng, const int32_t *noff, const int64_t *xadj, const int32_t *adj,
                              const int32_t *vw, const int32_t *ew, const uint64_t *keys, float *X,
                              int32_t *d1, int32_t *d2) {
  for (int32_t g = blockIdx.x; g < ng; g += gridDim.x) {
    int32_t v0 = noff[g];
    GView<int64_t> G{noff[g + 1] - v0, xadj + v0, adj, v0, vw ? vw + v0 : nullptr, ew};
    mp_features(G, keys[g], X + (int64_t)v0 * MF, d1 + v0, d2 + v0);
  }
}

// one layer over the union: A (pre-activation) and H = relu(A); M = neighbour mean of Hin
__global__ void k_mp_nbr(int32_t N, const int64_t *xadj, const int32_t *adj, const int32_t *ew,
                         const float *Hin, int d, float *M) {
  GView<int64_t> G{N, xadj, adj, 0, nullptr, ew};
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < (int64_t)N * d;
       t += (int64_t)gridDim.x * blockDim.x)
    M[t] = mp_nbr_mean(G, Hin, d, (int32_t)(t / d), (int)(t % d));
}

__global__ void k_mp_layer(int32_t N, const __nv_bfloat16 *W, int ws, int wn, int b, int din,
                           const float *Hin, const float *M, float *A, float *H) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < (int64_t)N * MH;
       t += (int64_t)gridDim.x * blockDim.x) {
    int32_t v = (int32_t)(t / MH);
    int o = (int)(t % MH);
    float a = mp_preact(W, ws, wn, b, din, Hin + (int64_t)v * din, M + (int64_t)v * din, o);
    A[t] = a;
    H[t] = a > 0.f ? a : 0.f;
  }
}

__global__ void k_mp_readout(int32_t N, const __nv_bfloat16 *W, const float *H2, float *S) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < N;
       v += (int64_t)gridDim.x * blockDim.x) {
    S[v] = mp_readout(W, H2 + v * MH);
  }
}

__device__ __forceinline__ float softplusf(float z) { return z > 0.f ? z + log1pf(expf(-z)) : log1pf(expf(z)); }

// per graph: orientation-symmetric BCE, gS = dL/ds with L = mean over graphs;
// lossg[g] = graph g's share of L (summed on the host in graph order)
__global__ void k_mp_loss(int32_t ng, const int32_t *noff, const float *S, const int32_t *side, float *gS,
                          float *lossg) {
  __shared__ float r0[32], r1[32];
  for (int32_t g = blockIdx.x; g < ng; g += gridDim.x) {
    int32_t v0 = noff[g], n = noff[g + 1] - v0;
    float l0 = 0, l1 = 0;
    for (int32_t v = threadIdx.x; v < n; v += blockDim.x) {
      float s = S[v0 + v], y = side[v0 + v] == 0 ? 1.f : 0.f, sp = softplusf(s);
      l0 += sp - y * s;
      l1 += sp - (1.f - y) * s;
    }
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) {
      l0 += __shfl_xor_sync(0xFFFFFFFFu, l0, m);
      l1 += __shfl_xor_sync(0xFFFFFFFFu, l1, m);
    }
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) {
      r0[w] = l0;
      r1[w] = l1;
    }
    __syncthreads();
    float t0 = 0, t1 = 0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
      t0 += r0[i];
      t1 += r1[i];
    }
    bool flip = t1 < t0;
    float scale = 1.f / ((float)(n > 0 ? n : 1) * (float)ng);
    for (int32_t v = threadIdx.x; v < n; v += blockDim.x) {
      float y = side[v0 + v] == 0 ? 1.f : 0.f;
      if (flip) y = 1.f - y;
      float p = 1.f / (1.f + expf(-S[v0 + v]));
      gS[v0 + v] = (p - y) * scale;
    }
    if (threadIdx.x == 0) lossg[g] = (flip ? t1 : t0) * scale;
    __syncthreads();
  }
}

// read-out backward to the layer-2 pre-activations: gA2 = relu'(A2) gS w_o
__global__ void k_mp_bw_out(int32_t N, const __nv_bfloat16 *W, const float *gS, const float *A2, float *gA2) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < (int64_t)N * MH;
       t += (int64_t)gridDim.x * blockDim.x) {
    int o = (int)(t % MH);
    gA2[t] = A2[t] > 0.f ? gS[t / MH] * wbf(W, P_WO + o) : 0.f;
  }
}

// Weight gradients without atomics, so training is deterministic: CTA c sums
// tiles c, c + G, c + 2G, ... of MP_TILE nodes in order and writes its
// partial sums of dW_self[o][i] = sum_v gA[v][o] Hin[v][i], dW_nbr (with M)
// and db[o] = sum_v gA[v][o] to part[c][...]; k_mp_reduce adds the G
// partials in order.  dout = 64 for a layer, 1 for the read-out (no M).
constexpr int MP_TILE = 64;
constexpr int MP_T = 256;
constexpr int MP_PER = MH * MH / MP_T;  // weight pairs per thread at most
__global__ void __launch_bounds__(MP_T) k_mp_wgrad(int32_t N, int din, int dout, const float *gA,
                                                   const float *Hin, const float *M, float *part, int ws,
                                                   int wn, int b) {
  __shared__ float sgA[MP_TILE][MH];
  __shared__ float sH[MP_TILE][MH];
  __shared__ float sM[MP_TILE][MH];
  int npairs = dout * din;
  float accs[MP_PER], accn[MP_PER], accb = 0.f;
#pragma unroll
  for (int j = 0; j < MP_PER; ++j) accs[j] = accn[j] = 0.f;
  for (int64_t base = (int64_t)blockIdx.x * MP_TILE; base < N; base += (int64_t)gridDim.x * MP_TILE) {
    int cnt = (int)(N - base < MP_TILE ? N - base : MP_TILE);
    for (int t = threadIdx.x; t < MP_TILE * MH; t += MP_T) {
      int r = t / MH, c = t % MH;
      bool ok = r < cnt;
      if (c < dout) sgA[r][c] = ok ? gA[(base + r) * dout + c] : 0.f;
      if (c < din) {
        sH[r][c] = ok ? Hin[(base + r) * din + c] : 0.f;
        sM[r][c] = ok && M ? M[(base + r) * din + c] : 0.f;
      }
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < MP_PER; ++j) {
      int pr = threadIdx.x + j * MP_T;
      if (pr < npairs) {
        int o = pr / din, i = pr % din;
        for (int r = 0; r < cnt; ++r) {
          accs[j] = __fmaf_rn(sgA[r][o], sH[r][i], accs[j]);
          accn[j] = __fmaf_rn(sgA[r][o], sM[r][i], accn[j]);
        }
      }
    }
    if (threadIdx.x < dout)
      for (int r = 0; r < cnt; ++r) accb += sgA[r][threadIdx.x];
    __syncthreads();
  }
  float *pc = part + (int64_t)blockIdx.x * P_TOTAL;
#pragma unroll
  for (int j = 0; j < MP_PER; ++j) {
    int pr = threadIdx.x + j * MP_T;
    if (pr < npairs) {
      pc[ws + pr] = accs[j];
      if (wn >= 0) pc[wn + pr] = accn[j];
    }
  }
  if (threadIdx.x < dout) pc[b + threadIdx.x] = accb;
}

__global__ void k_mp_reduce(int32_t G, const float *part, float *grad) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < P_TOTAL; p += gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int32_t c = 0; c < G; ++c) s += part[(int64_t)c * P_TOTAL + p];
    grad[p] = s;
  }
}

// input gradients of layer 2: gH1s[v][i] = sum_o W2s[o][i] gA2[v][o], gM1[v][i] likewise with W2n
__global__ void k_mp_bw_input(int32_t N, const __nv_bfloat16 *W, const float *gA2, float *gH1,
                              float *gM1) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < (int64_t)N * MH;
       t += (int64_t)gridDim.x * blockDim.x) {
    int32_t v = (int32_t)(t / MH);
    int i = (int)(t % MH);
    float a = 0, c = 0;
    for (int o = 0; o < MH; ++o) {
      float g = gA2[(int64_t)v * MH + o];
      a += wbf(W, P_W2S + o * MH + i) * g;
      c += wbf(W, P_W2N + o * MH + i) * g;
    }
    gH1[t] = a;
    gM1[t] = c;
  }
}

// gA1[u][i] = relu'(A1) * (gH1s[u][i] + sum_{v in N(u)} w(u,v)/wdeg(v) gM1[v][i])
__global__ void k_mp_bw_agg(int32_t N, const int64_t *xadj, const int32_t *adj, const int32_t *ew,
                            const float *wdeg, const float *gH1, const float *gM1, const float *A1,
                            float *gA1) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < (int64_t)N * MH;
       t += (int64_t)gridDim.x * blockDim.x) {
    int32_t u = (int32_t)(t / MH);
    int i = (int)(t % MH);
    float s = gH1[t];
    for (int64_t e = xadj[u]; e < xadj[u + 1]; ++e) {
      int32_t v = adj[e];
      float w = ew ? (float)ew[e] : 1.f;
      if (wdeg[v] > 0.f) s += w / wdeg[v] * gM1[(int64_t)v * MH + i];
    }
    gA1[t] = A1[t] > 0.f ? s : 0.f;
  }
}

__global__ void k_mp_wdeg(int32_t N, const int64_t *xadj, const int32_t *ew, float *wdeg) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < N;
       v += (int64_t)gridDim.x * blockDim.x) {
    float s = 0;
    for (int64_t e = xadj[v]; e < xadj[v + 1]; ++e) s += ew ? (float)ew[e] : 1.f;
    wdeg[v] = s;
  }
}

__global__ void k_mp_adam(int32_t P, float *master, float *grad, float *am, float *av, __nv_bfloat16 *wbfo,
                          float lr, float b1, float b2, float epsa, float c1, float c2) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P; i += gridDim.x * blockDim.x) {
    float g = grad[i];
    float m = b1 * am[i] + (1.f - b1) * g;
    float v = b2 * av[i] + (1.f - b2) * g * g;
    am[i] = m;
    av[i] = v;
    float w = master[i] - lr * (m / c1) / (sqrtf(v / c2) + epsa);
    master[i] = w;
    wbfo[i] = __float2bfloat16(w);
    grad[i] = 0.f;
  }
}

__global__ void k_mp_tobf(int32_t P, const float *master, __nv_bfloat16 *wbfo) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P; i += gridDim.x * blockDim.x)
    wbfo[i] = __float2bfloat16(master[i]);
}

__global__ void k_mp_frombf(int32_t P, const __nv_bfloat16 *w, float *out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P; i += gridDim.x * blockDim.x)
    out[i] = __bfloat162float(w[i]);
}

// ------------------------------------------------------------------ host
static void upload_batch(Batch &b, int32_t ng, const int32_t *noff, const int64_t *xadj, const int32_t *adj,
                         const int32_t *vw, const int32_t *ew, const uint64_t *keys, const int32_t *side) {
  b.ng = ng;
  b.N = noff[ng];
  b.E = xadj[b.N];
  b.noff.alloc(ng + 1);
  to_dev(b.noff.p, noff, ng + 1);
  b.xadj.alloc(b.N + 1);
  to_dev(b.xadj.p, xadj, b.N + 1);
  b.adj.alloc(b.E);
  to_dev(b.adj.p, adj, b.E);
  if (vw) {
    b.vw.alloc(b.N);
    to_dev(b.vw.p, vw, b.N);
  }
  if (ew) {
    b.ew.alloc(b.E);
    to_dev(b.ew.p, ew, b.E);
  }
  b.keys.alloc(ng);
  to_dev(b.keys.p, keys, ng);
  if (side) {
    b.side.alloc(b.N);
    to_dev(b.side.p, side, b.N);
  }
}

struct Acts {
  DBuf<float> X, M0, A1, H1, M1, A2, H2, S, wdeg;
  DBuf<int32_t> d1, d2;
};

static void forward(const kmp_mpnn *m, const Batch &b, Acts &a) {
  cudaStream_t s = ctx().stream;
  int32_t N = b.N;
  a.X.alloc((int64_t)N * MF);
  a.M0.alloc((int64_t)N * MF);
  a.A1.alloc((int64_t)N * MH);
  a.H1.alloc((int64_t)N * MH);
  a.M1.alloc((int64_t)N * MH);
  a.A2.alloc((int64_t)N * MH);
  a.H2.alloc((int64_t)N * MH);
  a.S.alloc(N);
  a.d1.alloc(N);
  a.d2.alloc(N);
  const int32_t *vw = b.vw.p, *ew = b.ew.p;
  k_mp_features<<<grid_for(b.ng, 1, 8), 256, 0, s>>>(b.ng, b.noff, b.xadj, b.adj, vw, ew, b.keys, a.X, a.d1,
                                                     a.d2);
  KMP_LAUNCHED("mp_features");
  int gl = grid_for((int64_t)N * MH, 256, 8);
  k_mp_nbr<<<gl, 256, 0, s>>>(N, b.xadj, b.adj, ew, a.X, MF, a.M0);
  KMP_LAUNCHED("mp_nbr");
  k_mp_layer<<<gl, 256, 0, s>>>(N, m->wbf, P_W1S, P_W1N, P_B1, MF, a.X, a.M0, a.A1, a.H1);
  KMP_LAUNCHED("mp_layer");
  k_mp_nbr<<<gl, 256, 0, s>>>(N, b.xadj, b.adj, ew, a.H1, MH, a.M1);
  KMP_LAUNCHED("mp_nbr");
  k_mp_layer<<<gl, 256, 0, s>>>(N, m->wbf, P_W2S, P_W2N, P_B2, MH, a.H1, a.M1, a.A2, a.H2);
  KMP_LAUNCHED("mp_layer");
  k_mp_readout<<<grid_for(N, 256), 256, 0, s>>>(N, m->wbf, a.H2, a.S);
  KMP_LAUNCHED("mp_readout");
}

// loss and its gradient (written to m->grad); returns the loss
static float backward(kmp_mpnn *m, const Batch &b, Acts &a) {
  cudaStream_t s = ctx().stream;
  int32_t N = b.N;
  DBuf<float> gS(N), lossg(b.ng), gA2((int64_t)N * MH), gH1((int64_t)N * MH), gM1((int64_t)N * MH),
      gA1((int64_t)N * MH);
  a.wdeg.alloc(N);
  const int32_t *ew = b.ew.p;
  k_mp_loss<<<grid_for(b.ng, 1, 8), 256, 0, s>>>(b.ng, b.noff, a.S, b.side, gS, lossg);
  KMP_LAUNCHED("mp_loss");
  int gl = grid_for((int64_t)N * MH, 256, 8);
  k_mp_bw_out<<<gl, 256, 0, s>>>(N, m->wbf, gS, a.A2, gA2);
  KMP_LAUNCHED("mp_bw_out");
  // a fixed number of partial sums (not tied to the GPU) keeps results identical everywhere
  int32_t G = (int32_t)std::min<int64_t>(ceil_div(std::max(N, 1), MP_TILE), 256);
  DBuf<float> part((int64_t)G * P_TOTAL);
  k_mp_wgrad<<<G, MP_T, 0, s>>>(N, MH, 1, gS, a.H2, nullptr, part, P_WO, -1, P_BO);
  KMP_LAUNCHED("mp_wgrad");
  k_mp_wgrad<<<G, MP_T, 0, s>>>(N, MH, MH, gA2, a.H1, a.M1, part, P_W2S, P_W2N, P_B2);
  KMP_LAUNCHED("mp_wgrad");
  k_mp_bw_input<<<gl, 256, 0, s>>>(N, m->wbf, gA2, gH1, gM1);
  KMP_LAUNCHED("mp_bw_input");
  k_mp_wdeg<<<grid_for(N, 256), 256, 0, s>>>(N, b.xadj, ew, a.wdeg);
  KMP_LAUNCHED("mp_wdeg");
  k_mp_bw_agg<<<gl, 256, 0, s>>>(N, b.xadj, b.adj, ew, a.wdeg, gH1, gM1, a.A1, gA1);
  KMP_LAUNCHED("mp_bw_agg");
  k_mp_wgrad<<<G, MP_T, 0, s>>>(N, MF, MH, gA1, a.X, a.M0, part, P_W1S, P_W1N, P_B1);
  KMP_LAUNCHED("mp_wgrad");
  k_mp_reduce<<<grid_for(P_TOTAL, 256), 256, 0, s>>>(G, part, m->grad);
  KMP_LAUNCHED("mp_reduce");
  std::vector<float> hl(b.ng);
  to_host(hl.data(), lossg.p, b.ng);
  float l = 0.f;
  for (float x : hl) l += x;
  return l;
}

template <class F>
static int guarded_mp(F &&f) {
  try {
    ensure_init();
    set_last_error("");
    f();
    return KMP_OK;
  } catch (const Error &e) {
    set_last_error(e.msg);
    return e.code;
  } catch (...) {
    set_last_error("unknown error");
    return KMP_ERR_CUDA;
  }
}

static void check_batch(int32_t ng, const int32_t *noff, const int64_t *xadj) {
  if (ng < 1 || !noff || !xadj) fail(KMP_ERR_ARG, "invalid batch");
  if (noff[0] != 0) fail(KMP_ERR_ARG, "noff[0] != 0");
  for (int32_t g = 0; g < ng; ++g)
    if (noff[g + 1] < noff[g]) fail(KMP_ERR_ARG, "noff must be non-decreasing");
}

}  // namespace kmp

using namespace kmp;

extern "C" {

int kmp_mpnn_num_params(void) { return P_TOTAL; }

int kmp_mpnn_create(uint64_t seed, kmp_mpnn **out) {
  return guarded_mp([&] {
    if (!out) fail(KMP_ERR_ARG, "out is NULL");
    kmp_mpnn *m = new kmp_mpnn;
    m->master = static_cast<float *>(dmalloc(P_TOTAL * sizeof(float)));
    m->wbf = static_cast<__nv_bfloat16 *>(dmalloc(P_TOTAL * sizeof(__nv_bfloat16)));
    m->am = static_cast<float *>(dmalloc(P_TOTAL * sizeof(float)));
    m->av = static_cast<float *>(dmalloc(P_TOTAL * sizeof(float)));
    m->grad = static_cast<float *>(dmalloc(P_TOTAL * sizeof(float)));
    // He-style uniform initialisation from the counter-based generator
    std::vector<float> h(P_TOTAL, 0.f);
    auto uni = [&](int i) {
      return (double)(key_step(mix64(seed + 0x9E3779B97F4A7C15ull), (uint64_t)i) >> 11) * 0x1.0p-53 * 2.0 - 1.0;
    };
    for (int i = 0; i < MH * MF; ++i) {
      h[P_W1S + i] = (float)(uni(P_W1S + i) * std::sqrt(6.0 / (2 * MF)));
      h[P_W1N + i] = (float)(uni(P_W1N + i) * std::sqrt(6.0 / (2 * MF)));
    }
    for (int i = 0; i < MH * MH; ++i) {
      h[P_W2S + i] = (float)(uni(P_W2S + i) * std::sqrt(6.0 / (2 * MH)));
      h[P_W2N + i] = (float)(uni(P_W2N + i) * std::sqrt(6.0 / (2 * MH)));
    }
    for (int i = 0; i < MH; ++i) h[P_WO + i] = (float)(uni(P_WO + i) * std::sqrt(6.0 / MH));
    to_dev(m->master, h.data(), P_TOTAL);
    KMP_CUDA(cudaMemsetAsync(m->am, 0, P_TOTAL * sizeof(float), ctx().stream));
    KMP_CUDA(cudaMemsetAsync(m->av, 0, P_TOTAL * sizeof(float), ctx().stream));
    KMP_CUDA(cudaMemsetAsync(m->grad, 0, P_TOTAL * sizeof(float), ctx().stream));
    k_mp_tobf<<<grid_for(P_TOTAL, 256), 256, 0, ctx().stream>>>(P_TOTAL, m->master, m->wbf);
    KMP_LAUNCHED("mp_tobf");
    sync_and_check("mpnn_create");
    *out = m;
  });
}

int kmp_mpnn_free(kmp_mpnn *m) {
  return guarded_mp([&] {
    if (!m) return;
    if (proposer().W == m->wbf) proposer().W = nullptr;
    dfree(m->master);
    dfree(m->wbf);
    dfree(m->am);
    dfree(m->av);
    dfree(m->grad);
    KMP_CUDA(cudaStreamSynchronize(ctx().stream));
    delete m;
  });
}

int kmp_mpnn_get_params(const kmp_mpnn *m, float *params) {
  return guarded_mp([&] {
    if (!m || !params) fail(KMP_ERR_ARG, "NULL argument");
    DBuf<float> t(P_TOTAL);
    k_mp_frombf<<<grid_for(P_TOTAL, 256), 256, 0, ctx().stream>>>(P_TOTAL, m->wbf, t);
    KMP_LAUNCHED("mp_frombf");
    to_host(params, t.p, P_TOTAL);
  });
}

int kmp_mpnn_set_params(kmp_mpnn *m, const float *params) {
  return guarded_mp([&] {
    if (!m || !params) fail(KMP_ERR_ARG, "NULL argument");
    to_dev(m->master, params, P_TOTAL);
    k_mp_tobf<<<grid_for(P_TOTAL, 256), 256, 0, ctx().stream>>>(P_TOTAL, m->master, m->wbf);
    KMP_LAUNCHED("mp_tobf");
    sync_and_check("mpnn_set_params");
  });
}

int kmp_mpnn_forward(kmp_mpnn *m, int32_t ng, const int32_t *noff, const int64_t *xadj, const int32_t *adj,
                     const int32_t *vw, const int32_t *ew, const uint64_t *keys, float *scores,
                     float *features) {
  return guarded_mp([&] {
    if (!m || !scores) fail(KMP_ERR_ARG, "NULL argument");
    check_batch(ng, noff, xadj);
    Batch b;
    upload_batch(b, ng, noff, xadj, adj, vw, ew, keys, nullptr);
    Acts a;
    forward(m, b, a);
    to_host(scores, a.S.p, b.N);
    if (features) to_host(features, a.X.p, (size_t)b.N * MF);
    sync_and_check("mpnn_forward");
  });
}

int kmp_mpnn_gradients(kmp_mpnn *m, int32_t ng, const int32_t *noff, const int64_t *xadj, const int32_t *adj,
                       const int32_t *vw, const int32_t *ew, const uint64_t *keys, const int32_t *side,
                       float *loss_out, float *grad_out) {
  return guarded_mp([&] {
    if (!m || !side) fail(KMP_ERR_ARG, "NULL argument");
    check_batch(ng, noff, xadj);
    Batch b;
    upload_batch(b, ng, noff, xadj, adj, vw, ew, keys, side);
    Acts a;
    forward(m, b, a);
    KMP_CUDA(cudaMemsetAsync(m->grad, 0, P_TOTAL * sizeof(float), ctx().stream));
    float l = backward(m, b, a);
    if (grad_out) to_host(grad_out, m->grad, P_TOTAL);
    KMP_CUDA(cudaMemsetAsync(m->grad, 0, P_TOTAL * sizeof(float), ctx().stream));
    sync_and_check("mpnn_gradients");
    if (loss_out) *loss_out = l;
  });
}

int kmp_mpnn_train(kmp_mpnn *m, int32_t ng, const int32_t *noff, const int64_t *xadj, const int32_t *adj,
                   const int32_t *vw, const int32_t *ew, const uint64_t *keys, const int32_t *side,
                   int32_t epochs, float lr, float *loss_per_epoch) {
  return guarded_mp([&] {
    if (!m || !side || epochs < 0 || !(lr > 0.f)) fail(KMP_ERR_ARG, "invalid arguments");
    check_batch(ng, noff, xadj);
    Batch b;
    upload_batch(b, ng, noff, xadj, adj, vw, ew, keys, side);
    for (int32_t ep = 0; ep < epochs; ++ep) {
      Acts a;
      forward(m, b, a);
      float l = backward(m, b, a);
      m->step += 1;
      const float b1 = 0.9f, b2 = 0.999f;
      float c1 = 1.f - std::pow(b1, (float)m->step), c2 = 1.f - std::pow(b2, (float)m->step);
      k_mp_adam<<<grid_for(P_TOTAL, 256), 256, 0, ctx().stream>>>(P_TOTAL, m->master, m->grad, m->am, m->av,
                                                                 m->wbf, lr, b1, b2, 1e-8f, c1, c2);
      KMP_LAUNCHED("mp_adam");
      if (loss_per_epoch) loss_per_epoch[ep] = l;
    }
    sync_and_check("mpnn_train");
  });
}

int kmp_set_proposer(const kmp_mpnn *m) {
  return guarded_mp([&] { proposer().W = m ? m->wbf : nullptr; });
}

int kmp_sample_sink_level(int32_t item_level) {
  return guarded_mp([&] {
    if (item_level < 0 || item_level > 1) fail(KMP_ERR_ARG, "sink level must be 0 or 1");
    sample_sink().item_level = item_level;
  });
}

int kmp_sample_sink_open(int32_t max_graphs, int64_t max_nodes, int64_t max_entries) {
  return guarded_mp([&] {
    if (max_graphs < 1 || max_nodes < 1 || max_entries < 0) fail(KMP_ERR_ARG, "invalid sink capacity");
    sink_release();
    SampleSink &K = sample_sink();
    cudaStream_t s = ctx().stream;
    K.max_graphs = max_graphs;
    K.max_nodes = max_nodes;
    K.max_entries = max_entries;
    K.counters = static_cast<unsigned long long *>(dmalloc(4 * sizeof(unsigned long long)));
    K.rec = static_cast<int64_t *>(dmalloc((size_t)max_graphs * 5 * sizeof(int64_t)));
    K.deg = static_cast<int32_t *>(dmalloc((size_t)max_nodes * sizeof(int32_t)));
    K.vw = static_cast<int32_t *>(dmalloc((size_t)max_nodes * sizeof(int32_t)));
    K.side = static_cast<int32_t *>(dmalloc((size_t)max_nodes * sizeof(int32_t)));
    K.adj = static_cast<int32_t *>(dmalloc((size_t)std::max<int64_t>(max_entries, 1) * sizeof(int32_t)));
    K.ew = static_cast<int32_t *>(dmalloc((size_t)std::max<int64_t>(max_entries, 1) * sizeof(int32_t)));
    KMP_CUDA(cudaMemsetAsync(K.counters, 0, 4 * sizeof(unsigned long long), s));
    KMP_CUDA(cudaMemsetAsync(K.rec, 0xFF, (size_t)max_graphs * 5 * sizeof(int64_t), s));
    sync_and_check("sample_sink_open");
  });
}

int kmp_sample_sink_count(int32_t *graphs, int64_t *nodes, int64_t *entries, int64_t *dropped) {
  return guarded_mp([&] {
    SampleSink &K = sample_sink();
    if (!K.counters) fail(KMP_ERR_ARG, "no sample sink is open");
    unsigned long long c[4];
    to_host(c, K.counters, 4);
    int64_t kept = (int64_t)c[0] - (int64_t)c[3];
    // kept records sit at reservation indices below max_graphs; their node
    // and entry totals are summed from the records themselves
    std::vector<int64_t> rec((size_t)K.max_graphs * 5);
    to_host(rec.data(), K.rec, rec.size());
    int64_t nn = 0, ne = 0;
    int32_t ng = 0;
    for (int32_t g = 0; g < K.max_graphs; ++g)
      if (rec[5 * g + 1] >= 0) {
        ++ng;
        nn += rec[5 * g + 1];
        ne += rec[5 * g + 3];
      }
    if (ng != kept) fail(KMP_ERR_CUDA, "sample sink records inconsistent");
    if (graphs) *graphs = ng;
    if (nodes) *nodes = nn;
    if (entries) *entries = ne;
    if (dropped) *dropped = (int64_t)c[3];
  });
}

int kmp_sample_sink_read(int32_t *noff, int64_t *xadj, int32_t *adj, int32_t *vw, int32_t *ew,
                         uint64_t *keys, int32_t *side) {
  return guarded_mp([&] {
    SampleSink &K = sample_sink();
    if (!K.counters) fail(KMP_ERR_ARG, "no sample sink is open");
    if (!noff || !xadj || !adj || !vw || !ew || !keys || !side) fail(KMP_ERR_ARG, "NULL argument");
    std::vector<int64_t> rec((size_t)K.max_graphs * 5);
    to_host(rec.data(), K.rec, rec.size());
    std::vector<int32_t> idx;
    for (int32_t g = 0; g < K.max_graphs; ++g)
      if (rec[5 * g + 1] >= 0) idx.push_back(g);
    // deterministic order: by item key (unique per item and round), then size
    std::sort(idx.begin(), idx.end(), [&](int32_t a, int32_t b) {
      uint64_t ka = (uint64_t)rec[5 * a + 4], kb = (uint64_t)rec[5 * b + 4];
      if (ka != kb) return ka < kb;
      return rec[5 * a + 1] < rec[5 * b + 1];
    });
    int64_t nmax = 0, emax = 0;
    for (int32_t g : idx) {
      nmax = std::max(nmax, rec[5 * g] + rec[5 * g + 1]);
      emax = std::max(emax, rec[5 * g + 2] + rec[5 * g + 3]);
    }
    std::vector<int32_t> hdeg(nmax), hvw(nmax), hside(nmax), hadj(emax), hew(emax);
    to_host(hdeg.data(), K.deg, nmax);
    to_host(hvw.data(), K.vw, nmax);
    to_host(hside.data(), K.side, nmax);
    to_host(hadj.data(), K.adj, emax);
    to_host(hew.data(), K.ew, emax);
    int64_t nb = 0, eb = 0;
    noff[0] = 0;
    xadj[0] = 0;
    for (size_t i = 0; i < idx.size(); ++i) {
      const int64_t *r = &rec[5 * idx[i]];
      int64_t n0 = r[0], n = r[1], e0 = r[2], m = r[3];
      keys[i] = (uint64_t)r[4];
      for (int64_t v = 0; v < n; ++v) {
        xadj[nb + v + 1] = xadj[nb + v] + hdeg[n0 + v];
        vw[nb + v] = hvw[n0 + v];
        side[nb + v] = hside[n0 + v];
      }
      for (int64_t e = 0; e < m; ++e) {
        adj[eb + e] = (int32_t)(hadj[e0 + e] + nb);
        ew[eb + e] = hew[e0 + e];
      }
      nb += n;
      eb += m;
      noff[i + 1] = (int32_t)nb;
    }
  });
}

int kmp_sample_sink_close(void) {
  return guarded_mp([&] {
    KMP_CUDA(cudaStreamSynchronize(ctx().stream));
    sink_release();
  });
}

}  // extern "C"
