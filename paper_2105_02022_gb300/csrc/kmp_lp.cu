// Size-constrained label propagation on the GPU (Section 2 "Size-Constrained
// Label Propagation", Section 4.1 coarsening, Section 4.3 refinement).
//
// Each round visits the active nodes in S deterministic sub-rounds; a node's
// sub-round is step(roundkey, u) mod S.  Per sub-round:
//   rate     : every node of the sub-round sums the edge weight to each
//              neighbouring cluster (degree-binned: 4..32-lane groups with
//              shuffles, a warp with a shared-memory hash table, a CTA with a
//              shared-memory table, a CTA with a global table for very high
//              degrees), picks the best admissible cluster K with
//              w(K) + c(u) <= cap(K) by (rating desc, perm32 asc) and proposes
//              it when it beats the own cluster.
//   classify : a target whose total proposed weight fits is accepted whole;
//              otherwise its proposals are bucketed ("contested").
//   resolve  : per contested target, proposals ordered by (gain desc, u asc)
//              are accepted while the start weight plus the prefix fits
//              (warp shuffles for <= 32 proposals, a block radix select above).
//   apply    : labels and weights are updated, neighbours of moved nodes are
//              marked active for the next round.
// The cap holds exactly and the result is independent of scheduling.
#include <cstdio>

#include "kmp_internal.cuh"

namespace kmp {

constexpr int NB = 7;           // degree bins
constexpr int BIN_TILE = 2048;  // nodes per binning tile
constexpr int RATE_T = 256;
constexpr int WARP_TAB = 512;   // per-warp hash table (bin 4: degree <= 256)
constexpr int CTA_TAB = 4096;   // per-CTA shared table (bin 5: degree <= 2048)
constexpr int64_t HUGE_DEG_MAX = CTA_TAB / 2;  // largest degree a shared CTA table serves
static_assert(HUGE_DEG_MAX == 2048, "upper bound of kmp_tuning.hub_degree");

__host__ __device__ __forceinline__ int deg_bin(int64_t d, int64_t huge) {
  if (d <= 4) return 0;
  if (d <= 8) return 1;
  if (d <= 16) return 2;
  if (d <= 32) return 3;
  if (d <= 256) return 4;
  if (d <= huge) return 5;
  return 6;
}

// per-round values, read by the kernels from device memory so that one
// captured round can be replayed for every round of a run
struct LPRound {
  uint64_t rk;     // round key
  uint32_t rk_hi;  // its high word (tie-break permutation)
  int32_t r;       // round index; its parity selects the active-flag buffers
  int32_t next;    // index of the next round
  int32_t pad;
};

struct LPArgs {
  int32_t n;
  const int64_t *xadj;
  const int32_t *adj;
  const int32_t *vw;
  const int32_t *ew;
  int32_t *label;
  int32_t *wt;
  const int32_t *cap;
  int32_t U;
  int32_t *fav;
  uint8_t *act0, *act1;       // active flags: round r reads act_{r&1}, marks act_{1-(r&1)}
  int32_t *vlist;
  int32_t *boff;  // [S*NB+1]
  int32_t *prop_t;
  int32_t *prop_g;
  uint8_t *acc;
  int32_t *pos_in_t;
  int32_t *tsum;
  int32_t *tcnt;
  int32_t *tcur;
  int32_t *tslot;
  int32_t *slot_t;
  int32_t *slot_base;
  int32_t *bucket;
  int32_t *ctr;                // [0] slots, [1] bucket top, [2] big movers
  int32_t *bigmove;            // high-degree nodes that moved in this sub-round
  unsigned long long *ctr64;   // 18 per round: [0] scanned entries, [1] moved nodes, [2+s]
                               // degree sum of sub-round s, [10+s] the same over bin 6 (hubs)
  // bin 6 (degree > huge_deg) with many labels: the sub-round's hub entries
  // are hashed by label into buckets of about hub_bucket entries, scattered
  // into bucket order and aggregated one bucket per warp in shared memory
  const int32_t *hubs;         // hub node ids, ascending
  int32_t nhubs;
  unsigned long long *hkc;     // best admissible key per hub
  unsigned long long *hku;     // best key per hub
  int32_t *hrown;              // rating of the hub's own cluster
  int32_t *hlab;               // neighbour labels of the sub-round's hub entries (entry order)
  int32_t *hslab;              // the same in bucket order (~label once aggregated)
  int32_t *hsw;                // their edge weights in bucket order (weighted graphs)
  int32_t *hbcnt;              // entries per bucket (zeroed by the bucket kernel after use)
  int32_t *hbcur;              // scatter cursor per bucket (zeroed likewise)
  int32_t *hboff;              // bucket offsets: exclusive scan of hbcnt
  int32_t hub_bucket;          // target entries per bucket
  int32_t *plan_h;             // per sub-round hub plan: hub index of each bin-6 entry,
  int64_t *plan_e;             // exclusive prefix of its edge chunks,
  int64_t *plan_x;             // of its entries (degree),
  int64_t *plan_b;             // of its buckets,
  int64_t *plan_tot;           // [0] edge chunks, [1] buckets, [2] entries
  int32_t small_labels;        // all labels fit a CTA table: bin 6 handled like bin 5
  int32_t *hdense;             // few labels: bin-6 entry i of a sub-round owns row i of
                               // a [hubs][nlab] rating array filled by many CTAs
  int64_t huge_deg;            // degree above which a node is a hub (many labels: <= HUGE_DEG_MAX)
  int64_t hub_chunk;           // edges per hub insert work unit
  int32_t nlab;
  int32_t S;
  LPRound *R;                  // current round (written by k_round_begin)
  unsigned long long *tmin;    // profiling (nullable): per k_rate launch (round * S + sub-round)
  unsigned long long *tmax;    // the earliest CTA start and the latest CTA end, global-timer ns
  unsigned long long *smax;    // latest CTA end of the sub-round's whole rating stage (k_rate
                               // and the hub kernels after it)
};

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ uint32_t rkh(const LPArgs &A) { return __ldg(&A.R->rk_hi); }
__device__ __forceinline__ uint64_t rkey(const LPArgs &A) { return __ldg(&A.R->rk); }
__device__ __forceinline__ uint8_t *act_cur(const LPArgs &A) { return (__ldg(&A.R->r) & 1) ? A.act1 : A.act0; }
__device__ __forceinline__ uint8_t *act_nxt(const LPArgs &A) { return (__ldg(&A.R->r) & 1) ? A.act0 : A.act1; }
__device__ __forceinline__ unsigned long long *ctr_cur(const LPArgs &A) {
  return A.ctr64 + 18 * __ldg(&A.R->r);
}

// profiling: this round's bin offsets into its slot of boff_all
__global__ void k_save_boff(LPArgs A, int32_t *boff_all) {
  int32_t m = A.S * NB + 1;
  int32_t *dst = boff_all + (int64_t)m * __ldg(&A.R->r);
  for (int32_t i = threadIdx.x; i < m; i += blockDim.x) dst[i] = A.boff[i];
}

// the next round's key and index (one thread, first launch of every round)
__global__ void k_round_begin(LPArgs A, uint64_t basekey) {
  LPRound *R = A.R;
  int32_t r = R->next;
  uint64_t rk = key_step(basekey, (uint64_t)r);
  R->r = r;
  R->rk = rk;
  R->rk_hi = (uint32_t)(rk >> 32);
  R->next = r + 1;
}

// inverse of perm32: the label whose tie-break rank is p
__device__ __forceinline__ int32_t perm32_inv(uint32_t rk_hi, uint32_t p) {
  uint32_t h = p;
  h ^= h >> 16;
  h *= 0x7ED1B41Du;  // inverse of 0xC2B2AE35 modulo 2^32
  h ^= (h >> 13) ^ (h >> 26);
  h *= 0xA5CB9243u;  // inverse of 0x85EBCA6B modulo 2^32
  h ^= h >> 16;
  return (int32_t)(h ^ rk_hi);
}
__device__ __forceinline__ int32_t label_of_key(uint32_t rk_hi, uint64_t key) {
  return perm32_inv(rk_hi, 0xFFFFFFFFu - (uint32_t)key);
}
__device__ __forceinline__ uint32_t table_cap(int64_t deg, int32_t nlab) {
  int64_t d = deg < nlab ? deg : nlab;
  uint32_t c = 32;
  while ((int64_t)c < 2 * d) c <<= 1;
  return c;
}

__device__ __forceinline__ int32_t node_w(const LPArgs &A, int32_t v) { return A.vw ? A.vw[v] : 1; }
__device__ __forceinline__ int32_t edge_w(const LPArgs &A, int64_t e) { return A.ew ? A.ew[e] : 1; }
__device__ __forceinline__ int64_t cap_of(const LPArgs &A, int32_t K) {
  return A.cap ? (int64_t)A.cap[K] : (int64_t)A.U;
}
__device__ __forceinline__ uint64_t rate_key(const LPArgs &A, int32_t K, int32_t r) {
  return ((uint64_t)(uint32_t)r << 32) | (uint64_t)(0xFFFFFFFFu - perm32(rkh(A), K));
}

// final decision for node u given the best constrained / unconstrained keys
__device__ __forceinline__ void emit(const LPArgs &A, int32_t u, int32_t pos, int32_t r_own,
                                     uint64_t kc, int32_t lc, uint64_t ku, int32_t lu) {
  int32_t rc = (int32_t)(kc >> 32);
  if (kc != 0 && rc > r_own) {
    A.prop_t[pos] = lc;
    A.prop_g[pos] = rc - r_own;
    atomicAdd(&A.tsum[lc], node_w(A, u));
    atomicAdd(&A.tcnt[lc], 1);
  } else {
    A.prop_t[pos] = -1;
    int32_t ru = (int32_t)(ku >> 32);
    if (A.fav && ku != 0 && ru > r_own) A.fav[u] = lu;
  }
}

// ------------------------------------------------------------------ binning
__global__ void __launch_bounds__(256) k_bin_count(LPArgs A, int32_t *cnt, int64_t ntiles) {
  __shared__ int32_t c[8 * NB];
  __shared__ unsigned long long scanned;
  for (int i = threadIdx.x; i < A.S * NB; i += blockDim.x) c[i] = 0;
  if (threadIdx.x == 0) scanned = 0;
  __syncthreads();
  int64_t base = (int64_t)blockIdx.x * BIN_TILE;
  unsigned long long my = 0;
  __shared__ unsigned long long sdeg[8], sdeg6[8];
  if (threadIdx.x < 8) {
    sdeg[threadIdx.x] = 0;
    sdeg6[threadIdx.x] = 0;
  }
  __syncthreads();
  const uint8_t *act = act_cur(A);
  const uint64_t rk = rkey(A);
  for (int i = threadIdx.x; i < BIN_TILE; i += blockDim.x) {
    int64_t v = base + i;
    if (v >= A.n || !act[v]) continue;
    int64_t d = A.xadj[v + 1] - A.xadj[v];
    if (d == 0) continue;
    int s = (int)(key_step(rk, (uint64_t)(uint32_t)v) & (uint64_t)(A.S - 1));
    int bin = deg_bin(d, A.huge_deg);
    atomicAdd(&c[s * NB + bin], 1);
    atomicAdd(&sdeg[s], (unsigned long long)d);
    if (bin == 6) atomicAdd(&sdeg6[s], (unsigned long long)d);
    my += (unsigned long long)d;
  }
  atomicAdd(&scanned, my);
  __syncthreads();
  for (int i = threadIdx.x; i < A.S * NB; i += blockDim.x) cnt[(int64_t)i * ntiles + blockIdx.x] = c[i];
  unsigned long long *ctr = ctr_cur(A);
  if (threadIdx.x == 0) atomicAdd(&ctr[0], scanned);
  if (threadIdx.x < A.S && sdeg[threadIdx.x]) atomicAdd(&ctr[2 + threadIdx.x], sdeg[threadIdx.x]);
  if (threadIdx.x < A.S && sdeg6[threadIdx.x]) atomicAdd(&ctr[10 + threadIdx.x], sdeg6[threadIdx.x]);
}

__global__ void k_bin_boff(LPArgs A, const int32_t *off, const int32_t *total, int64_t ntiles) {
  int i = threadIdx.x;
  if (i < A.S * NB) A.boff[i] = off[(int64_t)i * ntiles];
  if (i == 0) A.boff[A.S * NB] = *total;
}

// stable scatter of the active nodes into (sub-round, bin) order; consumes act[]
__global__ void __launch_bounds__(256) k_bin_scatter(LPArgs A, const int32_t *off, int64_t ntiles) {
  constexpr int W = 8;
  __shared__ uint8_t key[BIN_TILE];
  __shared__ int32_t wcnt[W][8 * NB];
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int nk = A.S * NB;
  for (int i = threadIdx.x; i < W * 8 * NB; i += blockDim.x) (&wcnt[0][0])[i] = 0;
  __syncthreads();
  int64_t base = (int64_t)blockIdx.x * BIN_TILE;
  uint8_t *act = act_cur(A);
  const uint64_t rk = rkey(A);
  // pass 1: keys and per-warp counts; warp w owns nodes [w*256, w*256+256) of the tile
  for (int it = 0; it < BIN_TILE / (W * 32); ++it) {
    int li = w * (BIN_TILE / W) + it * 32 + lane;
    int64_t v = base + li;
    int k = 255;
    if (v < A.n && act[v]) {
      int64_t d = A.xadj[v + 1] - A.xadj[v];
      if (d > 0) {
        int s = (int)(key_step(rk, (uint64_t)(uint32_t)v) & (uint64_t)(A.S - 1));
        k = s * NB + deg_bin(d, A.huge_deg);
      }
    }
    if (v < A.n) act[v] = 0;
    key[li] = (uint8_t)k;
    unsigned peers = __match_any_sync(0xFFFFFFFFu, k);
    if (k != 255 && (peers & ((1u << lane) - 1u)) == 0) wcnt[w][k] += __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  if (threadIdx.x < nk) {
    int32_t s = 0;
    for (int ww = 0; ww < W; ++ww) {
      int32_t c = wcnt[ww][threadIdx.x];
      wcnt[ww][threadIdx.x] = s;
      s += c;
    }
  }
  __syncthreads();
  // pass 2: positions
  for (int it = 0; it < BIN_TILE / (W * 32); ++it) {
    int li = w * (BIN_TILE / W) + it * 32 + lane;
    int k = key[li];
    unsigned peers = __match_any_sync(0xFFFFFFFFu, k);
    int rank = __popc(peers & ((1u << lane) - 1u));
    if (k != 255) {
      int32_t p = off[(int64_t)k * ntiles + blockIdx.x] + wcnt[w][k] + rank;
      A.vlist[p] = (int32_t)(base + li);
    }
    __syncwarp();
    if (k != 255 && rank == 0) wcnt[w][k] += __popc(peers);
    __syncwarp();
  }
}

// ------------------------------------------------------------------- rating
// G lanes per node (G in 4, 8, 16, 32), degree <= G: one neighbour per lane.
template <int G>
__device__ __forceinline__ void rate_group(const LPArgs &A, int32_t u, int32_t pos, int lane) {
  int gl = lane & (G - 1);
  unsigned gmask = (G == 32) ? 0xFFFFFFFFu : (((1u << G) - 1u) << (lane & ~(G - 1)));
  int64_t beg = 0;
  int32_t deg = 0, own = -1, cu = 0;
  if (u >= 0) {
    beg = A.xadj[u];
    deg = (int32_t)(A.xadj[u + 1] - beg);
    own = A.label[u];
    cu = node_w(A, u);
  }
  int32_t l = -1, w = 0;
  if (gl < deg) {
    l = A.label[A.adj[beg + gl]];
    w = edge_w(A, beg + gl);
  }
  // lanes of one group holding the same label form a peer set; its weight sum
  // is the rating r(label)
  uint64_t mkey = ((uint64_t)(uint32_t)(lane / G) << 32) | (uint32_t)l;
  unsigned peers = __match_any_sync(0xFFFFFFFFu, mkey);
  int32_t r = __reduce_add_sync(peers, w);
  unsigned bown = __ballot_sync(0xFFFFFFFFu, l >= 0 && l == own) & gmask;
  int32_t rown = __shfl_sync(0xFFFFFFFFu, r, bown ? __ffs(bown) - 1 : lane);
  if (!bown) rown = 0;
  bool valid = l >= 0 && l != own;
  uint64_t ku = valid ? rate_key(A, l, r) : 0ull;
  bool adm = valid && ((int64_t)A.wt[l] + cu <= cap_of(A, l));
  uint64_t kc = adm ? ku : 0ull;
  uint64_t mc = group_max64<G>(kc), mu = group_max64<G>(ku);
  unsigned bc = __ballot_sync(0xFFFFFFFFu, mc != 0 && kc == mc) & gmask;
  unsigned bu = __ballot_sync(0xFFFFFFFFu, mu != 0 && ku == mu) & gmask;
  int32_t lc = __shfl_sync(0xFFFFFFFFu, l, bc ? __ffs(bc) - 1 : lane);
  int32_t lu = __shfl_sync(0xFFFFFFFFu, l, bu ? __ffs(bu) - 1 : lane);
  if (gl == 0 && u >= 0) emit(A, u, pos, rown, mc, lc, mu, lu);
}

// slot of a table insert, when this insert occupied it (else -1)
__device__ __forceinline__ int32_t ht_add_fresh(int32_t *keys, int32_t *vals, uint32_t mask, int32_t k,
                                                int32_t w) {
  uint32_t h = fmix32((uint32_t)k) & mask;
  for (uint32_t probe = 0; probe <= mask; ++probe) {
    int32_t old = atomicCAS(&keys[h], HT_EMPTY, k);
    if (old == HT_EMPTY || old == k) {
      atomicAdd(&vals[h], w);
      return old == HT_EMPTY ? (int32_t)h : -1;
    }
    h = (h + 1) & mask;
  }
  return -1;
}

// The shared tables of the warp and CTA bins start empty (cleared once per
// launch) and every node leaves them empty: its inserts record the slots they
// occupy in a list (at most cap / 2 distinct labels), and the selection pass
// walks only that list, clearing each slot after reading it.  Table size and
// hashing are unchanged, so per-node work scales with the distinct labels,
// not with the table capacity.

// Best keys over a table's held slots (one thread's share: list[i0], i0 +
// step, ... < held): ku over every label but `own`, kc over the admissible
// ones (target weight + c(u) <= cap).  Admissibility needs the target's
// weight, a random read, so a thread checks its own best label first; the
// caller reduces those to kc0, the best admissible top of the group, and only
// a thread whose top failed then checks its other labels above kc0
// (select_rest).  The result is the plain maximum over admissible labels:
// a thread whose top passed holds nothing above it.
struct SelTop {
  uint64_t ku = 0, kc = 0;
  int32_t lu = -1, lc = -1;
  bool failed = false;  // the thread's top label is not admissible
};
__device__ __forceinline__ SelTop select_top(const LPArgs &A, const int32_t *keys, const int32_t *vals,
                                             const uint16_t *list, int32_t i0, int32_t step, int32_t held,
                                             int32_t own, int32_t cu, int32_t &rown) {
  SelTop T;
  for (int32_t i = i0; i < held; i += step) {
    const int32_t sl = list[i];
    const int32_t K = keys[sl], r = vals[sl];
    if (K == own) {
      rown = r;
      continue;
    }
    const uint64_t k = rate_key(A, K, r);
    if (k > T.ku) {
      T.ku = k;
      T.lu = K;
    }
  }
  if (T.lu >= 0) {
    if ((int64_t)A.wt[T.lu] + cu <= cap_of(A, T.lu)) {
      T.kc = T.ku;
      T.lc = T.lu;
    } else {
      T.failed = true;
    }
  }
  return T;
}
// the labels above kc0 of a thread whose top failed; the slots are cleared
__device__ __forceinline__ void select_rest(const LPArgs &A, int32_t *keys, int32_t *vals, const uint16_t *list,
                                            int32_t i0, int32_t step, int32_t held, int32_t own, int32_t cu,
                                            uint64_t kc0, SelTop &T) {
  for (int32_t i = i0; i < held; i += step) {
    const int32_t sl = list[i];
    const int32_t K = keys[sl], r = vals[sl];
    keys[sl] = HT_EMPTY;
    vals[sl] = 0;
    if (!T.failed || K == own || K == T.lu) continue;
    const uint64_t k = rate_key(A, K, r);
    if (k > kc0 && (int64_t)A.wt[K] + cu <= cap_of(A, K) && k > T.kc) {
      T.kc = k;
      T.lc = K;
    }
  }
}

// one node per warp, neighbours aggregated in a shared-memory table of WARP_TAB
__device__ __forceinline__ void rate_warp(const LPArgs &A, int32_t u, int32_t pos, int lane,
                                          int32_t *keys, int32_t *vals, uint16_t *list) {
  int64_t beg = A.xadj[u];
  int32_t deg = (int32_t)(A.xadj[u + 1] - beg);
  uint32_t tcap = table_cap(deg, A.nlab);  // <= WARP_TAB for degree <= 256
  int32_t own = A.label[u], cu = node_w(A, u);
  int32_t cnt = 0;
  for (int32_t e0 = 0; e0 < deg; e0 += 32) {
    int32_t e = e0 + lane;
    int32_t sl = e < deg ? ht_add_fresh(keys, vals, tcap - 1, A.label[A.adj[beg + e]], edge_w(A, beg + e)) : -1;
    unsigned m = __ballot_sync(0xFFFFFFFFu, sl >= 0);
    if (sl >= 0) list[cnt + __popc(m & ((1u << lane) - 1u))] = (uint16_t)sl;
    cnt += __popc(m);
  }
  __syncwarp();
  int32_t rown = 0;
  SelTop T = select_top(A, keys, vals, list, lane, 32, cnt, own, cu, rown);
  select_rest(A, keys, vals, list, lane, 32, cnt, own, cu, group_max64<32>(T.kc), T);
  const uint64_t kc = T.kc, ku = T.ku;
  int32_t lc = T.lc, lu = T.lu;
  rown = (int32_t)__reduce_max_sync(0xFFFFFFFFu, (uint32_t)rown);
  uint64_t mc = group_max64<32>(kc), mu = group_max64<32>(ku);
  unsigned bc = __ballot_sync(0xFFFFFFFFu, mc != 0 && kc == mc);
  unsigned bu = __ballot_sync(0xFFFFFFFFu, mu != 0 && ku == mu);
  lc = __shfl_sync(0xFFFFFFFFu, lc, bc ? __ffs(bc) - 1 : 0);
  lu = __shfl_sync(0xFFFFFFFFu, lu, bu ? __ffs(bu) - 1 : 0);
  if (lane == 0) emit(A, u, pos, rown, mc, lc, mu, lu);
  __syncwarp();
}

// one node per CTA with a shared table of `mask+1` entries
__device__ void rate_cta(const LPArgs &A, int32_t u, int32_t pos, int32_t *keys, int32_t *vals,
                         uint16_t *list, uint32_t mask) {
  __shared__ uint64_t red_c[RATE_T / 32], red_u[RATE_T / 32];
  __shared__ int32_t lab_c, lab_u, s_cnt, s_rown;
  if (threadIdx.x == 0) {
    lab_c = -1;
    lab_u = -1;
    s_cnt = 0;
    s_rown = 0;
  }
  __syncthreads();
  int64_t beg = A.xadj[u];
  int64_t deg = A.xadj[u + 1] - beg;
  int32_t own = A.label[u], cu = node_w(A, u);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int64_t e0 = threadIdx.x & ~31; e0 < deg; e0 += blockDim.x) {
    int64_t e = e0 + lane;
    int32_t sl = e < deg ? ht_add_fresh(keys, vals, mask, A.label[A.adj[beg + e]], edge_w(A, beg + e)) : -1;
    unsigned m = __ballot_sync(0xFFFFFFFFu, sl >= 0);
    if (m) {
      int32_t at = 0;
      if (lane == 0) at = atomicAdd(&s_cnt, __popc(m));
      at = __shfl_sync(0xFFFFFFFFu, at, 0);
      if (sl >= 0) list[at + __popc(m & ((1u << lane) - 1u))] = (uint16_t)sl;
    }
  }
  __syncthreads();
  const int32_t cnt = s_cnt;
  int32_t rown = -1;
  SelTop T = select_top(A, keys, vals, list, threadIdx.x, blockDim.x, cnt, own, cu, rown);
  if (rown >= 0) s_rown = rown;
  {
    const uint64_t w0 = group_max64<32>(T.kc);
    if (lane == 0) red_c[w] = w0;
    __syncthreads();
    uint64_t kc0 = 0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) kc0 = red_c[i] > kc0 ? red_c[i] : kc0;
    select_rest(A, keys, vals, list, threadIdx.x, blockDim.x, cnt, own, cu, kc0, T);
    __syncthreads();  // red_c is reused below
  }
  const uint64_t kc = T.kc, ku = T.ku;
  const int32_t lc = T.lc, lu = T.lu;
  uint64_t wc = group_max64<32>(kc), wu = group_max64<32>(ku);
  if (lane == 0) { red_c[w] = wc; red_u[w] = wu; }
  __syncthreads();
  uint64_t mc = 0, mu = 0;
  for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
    mc = red_c[i] > mc ? red_c[i] : mc;
    mu = red_u[i] > mu ? red_u[i] : mu;
  }
  if (mc != 0 && kc == mc) lab_c = lc;  // unique label per key: benign identical writes
  if (mu != 0 && ku == mu) lab_u = lu;
  __syncthreads();
  if (threadIdx.x == 0) emit(A, u, pos, s_rown, mc, lab_c, mu, lab_u);
  __syncthreads();
}

__device__ __forceinline__ int32_t hub_index(const LPArgs &A, int32_t u);

__global__ void __launch_bounds__(RATE_T, 6) k_rate(LPArgs A, int s) {
  __shared__ int32_t tkeys[CTA_TAB];
  __shared__ int32_t tvals[CTA_TAB];
  __shared__ uint16_t tlist[CTA_TAB / 2];
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    A.ctr[0] = 0;
    A.ctr[1] = 0;
    A.ctr[2] = 0;
  }
  const int64_t tslot = A.tmin ? (int64_t)__ldg(&A.R->r) * A.S + s : 0;
  if (A.tmin && threadIdx.x == 0) atomicMin(&A.tmin[tslot], global_ns());
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int64_t gw = (int64_t)blockIdx.x * (RATE_T / 32) + w;
  int64_t nw = (int64_t)gridDim.x * (RATE_T / 32);
  const int32_t *bo = A.boff + s * NB;
  if ((int64_t)bo[4] + (int64_t)blockIdx.x * (RATE_T / 32) < bo[5] ||
      (int64_t)bo[5] + blockIdx.x < ((A.small_labels && !A.hdense) ? bo[7] : bo[6])) {
    for (int i = threadIdx.x; i < CTA_TAB; i += blockDim.x) {  // only blocks with table work
      tkeys[i] = HT_EMPTY;
      tvals[i] = 0;
    }
  }
  __syncthreads();
#define KMP_GROUP_BIN(BIN, G)                                                  \
  {                                                                            \
    int32_t lo = bo[BIN], hi = bo[BIN + 1];                                    \
    constexpr int per = 32 / G;                                                \
    for (int64_t b0 = lo + gw * per; b0 < hi; b0 += nw * per) {               \
      int64_t idx = b0 + lane / G;                                             \
      int32_t u = idx < hi ? A.vlist[idx] : -1;                                \
      rate_group<G>(A, u, (int32_t)idx, lane);                                 \
    }                                                                          \
  }
  KMP_GROUP_BIN(0, 4)
  KMP_GROUP_BIN(1, 8)
  KMP_GROUP_BIN(2, 16)
  KMP_GROUP_BIN(3, 32)
#undef KMP_GROUP_BIN
  {
    int32_t lo = bo[4], hi = bo[5];
    for (int64_t idx = lo + gw; idx < hi; idx += nw)
      rate_warp(A, A.vlist[idx], (int32_t)idx, lane, tkeys + w * WARP_TAB, tvals + w * WARP_TAB,
                tlist + w * (WARP_TAB / 2));
  }
  __syncthreads();
  {
    // bin 5, and bin 6 as well when every label set fits a shared table and
    // no dense hub array is in use
    int32_t lo = bo[5], hi = (A.small_labels && !A.hdense) ? bo[7] : bo[6];
    for (int64_t idx = lo + blockIdx.x; idx < hi; idx += gridDim.x) {
      int32_t u = A.vlist[idx];
      uint32_t cap = table_cap(A.xadj[u + 1] - A.xadj[u], A.nlab);
      rate_cta(A, u, (int32_t)idx, tkeys, tvals, tlist, cap - 1);
    }
  }
  if (A.tmin) {
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned long long t = global_ns();
      atomicMax(&A.tmax[tslot], t);
      atomicMax(&A.smax[tslot], t);
    }
  }
}

// profiling: the end of the rating stage of sub-round s (its last kernel)
__device__ __forceinline__ void stamp_stage_end(const LPArgs &A, int s) {
  if (!A.tmin) return;
  __syncthreads();
  if (threadIdx.x == 0) atomicMax(&A.smax[(int64_t)__ldg(&A.R->r) * A.S + s], global_ns());
}

// ---- hubs (bin 6) with many labels: insert / reduce / emit

__device__ __forceinline__ int32_t hub_index(const LPArgs &A, int32_t u) {
  int32_t lo = 0, hi = A.nhubs - 1;
  while (lo < hi) {
    int32_t mid = (lo + hi) >> 1;
    if (A.hubs[mid] < u) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ int32_t find_seg(const int64_t *off, int32_t cnt, int64_t x) {
  int32_t lo = 0, hi = cnt - 1;  // last index with off[idx] <= x
  while (lo < hi) {
    int32_t mid = (lo + hi + 1) >> 1;
    if (off[mid] <= x) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// buckets of a hub of degree deg, and the bucket of label L among them
__device__ __forceinline__ int64_t hub_nbuckets(const LPArgs &A, int64_t deg) {
  return ceil_div(deg, (int64_t)A.hub_bucket);
}
__device__ __forceinline__ int64_t hub_bucket_of(int32_t L, int64_t nb) {
  // a mix decorrelated from the table slots' fmix32(L)
  return (int64_t)(((uint64_t)fmix32((uint32_t)L ^ 0x5BD1E995u) * (uint64_t)nb) >> 32);
}

// work plan of one sub-round: the hubs it rates, with exclusive prefixes of
// their edge chunks, entries and buckets (one block, any number of hubs)
__global__ void __launch_bounds__(1024) k_hub_plan(LPArgs A, int s) {
  __shared__ int64_t we[32], wx[32], wb[32];
  __shared__ int64_t carry_e, carry_x, carry_b;
  const int32_t *bo = A.boff + s * NB;
  int32_t lo = bo[6], cnt = bo[7] - bo[6];
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (threadIdx.x == 0) { carry_e = 0; carry_x = 0; carry_b = 0; }
  __syncthreads();
  for (int32_t base = 0; base < cnt; base += blockDim.x) {
    int32_t i = base + threadIdx.x;
    int64_t ne = 0, nx = 0, nb = 0;
    int32_t h = 0;
    if (i < cnt) {
      int32_t u = A.vlist[lo + i];
      h = A.hubs ? hub_index(A, u) : i;
      int64_t deg = A.xadj[u + 1] - A.xadj[u];
      ne = ceil_div(deg, A.hub_chunk);
      nx = deg;
      nb = A.hub_bucket > 0 ? hub_nbuckets(A, deg) : 0;
    }
    int64_t xe = ne, xx = nx, xb = nb;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      int64_t ye = (int64_t)__shfl_up_sync(0xFFFFFFFFu, (unsigned long long)xe, d);
      int64_t yx = (int64_t)__shfl_up_sync(0xFFFFFFFFu, (unsigned long long)xx, d);
      int64_t yb = (int64_t)__shfl_up_sync(0xFFFFFFFFu, (unsigned long long)xb, d);
      if (lane >= d) { xe += ye; xx += yx; xb += yb; }
    }
    if (lane == 31) { we[w] = xe; wx[w] = xx; wb[w] = xb; }
    __syncthreads();
    int64_t pe = carry_e, px = carry_x, pb = carry_b, te = 0, tx = 0, tb = 0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
      if (k < w) { pe += we[k]; px += wx[k]; pb += wb[k]; }
      te += we[k];
      tx += wx[k];
      tb += wb[k];
    }
    if (i < cnt) {
      A.plan_h[i] = h;
      A.plan_e[i] = pe + xe - ne;
      A.plan_x[i] = px + xx - nx;
      A.plan_b[i] = pb + xb - nb;
    }
    __syncthreads();
    if (threadIdx.x == 0) { carry_e += te; carry_x += tx; carry_b += tb; }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    A.plan_tot[0] = carry_e;
    A.plan_tot[1] = carry_b;
    A.plan_tot[2] = carry_x;
  }
}

// A CTA takes its work units in pieces of HP entries (HP_PER per thread) and
// counts each piece's entries per bucket in a shared table first, so one
// global atomic serves all of a piece's entries of one bucket.
constexpr int HP_PER = 8;
constexpr int HP_T = 256;
constexpr int HP = HP_T * HP_PER;
constexpr int HP_TAB = 2 * HP;  // bucket slots (at most HP keys: load <= 1/2)
struct HubPieceTable {
  int32_t key[HP_TAB];  // bucket (relative to the hub's first) or HT_EMPTY
  int32_t val[HP_TAB];  // entries of the piece in it; then their first position
  uint16_t list[HP];    // occupied slots
  int32_t n;
};

__device__ void hp_clear_all(HubPieceTable &T) {
  for (int x = threadIdx.x; x < HP_TAB; x += blockDim.x) {
    T.key[x] = HT_EMPTY;
    T.val[x] = 0;
  }
  if (threadIdx.x == 0) T.n = 0;
}

// slot of bucket b (inserted if new) and the entry's rank among the piece's
// entries of b
__device__ __forceinline__ int32_t hp_insert(HubPieceTable &T, int32_t b, int32_t &rank) {
  uint32_t h = (uint32_t)b & (HP_TAB - 1);
  for (int probe = 0; probe < HP_TAB; ++probe) {
    const int32_t old = atomicCAS(&T.key[h], HT_EMPTY, b);
    if (old == HT_EMPTY || old == b) {
      rank = atomicAdd(&T.val[h], 1);
      if (old == HT_EMPTY) T.list[atomicAdd(&T.n, 1)] = (uint16_t)h;
      return (int32_t)h;
    }
    h = (h + 1) & (HP_TAB - 1);
  }
  rank = 0;
  return -1;  // unreachable: a piece has at most HP_TAB / 2 buckets
}

// The hub of every work unit: each CTA (warp) takes a contiguous range of
// units, finds the first one's hub by binary search and then only moves
// forward (the units of one hub are consecutive).
struct HubCursor {
  int32_t i = -1;   // hub position in the sub-round's plan
  int64_t next = 0; // first unit of hub i + 1
  int32_t u = 0;
  int64_t b = 0, deg = 0, nb = 0, gb = 0, xo = 0, e_first = 0;
  __device__ void seek(const LPArgs &A, const int64_t *units, int32_t cnt, int64_t total, int64_t c) {
    if (i < 0 || c >= next) {
      if (i < 0 || c >= next + 64) {
        i = find_seg(units, cnt, c);
      } else {
        do ++i;
        while (i + 1 < cnt && units[i + 1] <= c);
      }
      next = i + 1 < cnt ? units[i + 1] : total;
      u = A.hubs[A.plan_h[i]];
      b = A.xadj[u];
      deg = A.xadj[u + 1] - b;
      nb = A.hub_bucket > 0 ? hub_nbuckets(A, deg) : 0;
      gb = A.plan_b[i];
      xo = A.plan_x[i] - b;
      e_first = units[i];
    }
  }
};

// work units: edge chunks of the sub-round's hubs; every entry's neighbour
// label is gathered once (kept in entry order) and counted in its bucket
__global__ void __launch_bounds__(HP_T) k_hub_count(LPArgs A, int s) {
  __shared__ HubPieceTable T;
  hp_clear_all(T);
  __syncthreads();
  const int32_t *bo = A.boff + s * NB;
  int32_t cnt = bo[7] - bo[6];
  int64_t total = A.plan_tot[0];
  const int64_t per = ceil_div(total, (int64_t)gridDim.x);
  const int64_t c0 = (int64_t)blockIdx.x * per, c1 = c0 + per < total ? c0 + per : total;
  HubCursor H;
  for (int64_t c = c0; c < c1; ++c) {
    H.seek(A, A.plan_e, cnt, total, c);
    const int64_t b = H.b, deg = H.deg, nb = H.nb, gb = H.gb, xo = H.xo;
    int64_t e0 = b + (c - H.e_first) * A.hub_chunk, e1 = e0 + A.hub_chunk < b + deg ? e0 + A.hub_chunk : b + deg;
    for (int64_t p0 = e0; p0 < e1; p0 += HP) {
      int32_t nbr[HP_PER], L[HP_PER];
#pragma unroll
      for (int r = 0; r < HP_PER; ++r) {
        const int64_t e = p0 + r * HP_T + threadIdx.x;
        nbr[r] = e < e1 ? A.adj[e] : -1;
      }
#pragma unroll
      for (int r = 0; r < HP_PER; ++r) L[r] = nbr[r] >= 0 ? A.label[nbr[r]] : -1;
#pragma unroll
      for (int r = 0; r < HP_PER; ++r)
        if (nbr[r] >= 0) {
          A.hlab[xo + p0 + r * HP_T + threadIdx.x] = L[r];
          int32_t rk;
          hp_insert(T, (int32_t)hub_bucket_of(L[r], nb), rk);
        }
      __syncthreads();
      const int32_t nt = T.n;
      for (int32_t x = threadIdx.x; x < nt; x += HP_T) {
        const int32_t h = T.list[x];
        atomicAdd(&A.hbcnt[gb + T.key[h]], T.val[h]);
        T.key[h] = HT_EMPTY;
        T.val[h] = 0;
      }
      __syncthreads();
      if (threadIdx.x == 0) T.n = 0;
      __syncthreads();
    }
  }
}

// the same work units: entries into bucket order (positions inside a bucket
// are arbitrary; the aggregation below does not depend on them)
// one piece in bucket order: each staged entry's index in the piece and its
// table slot (the label and weight are read again, from cache, when written)
struct HubPieceStage {
  uint16_t idx[HP];
  uint16_t slot[HP];
  int32_t wsum[HP_T / 32];
};

__global__ void __launch_bounds__(HP_T) k_hub_scatter(LPArgs A, int s) {
  __shared__ HubPieceTable T;
  __shared__ HubPieceStage P;
  hp_clear_all(T);
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int32_t *bo = A.boff + s * NB;
  int32_t cnt = bo[7] - bo[6];
  int64_t total = A.plan_tot[0];
  const int64_t per = ceil_div(total, (int64_t)gridDim.x);
  const int64_t c0 = (int64_t)blockIdx.x * per, c1 = c0 + per < total ? c0 + per : total;
  HubCursor H;
  for (int64_t c = c0; c < c1; ++c) {
    H.seek(A, A.plan_e, cnt, total, c);
    const int64_t b = H.b, deg = H.deg, nb = H.nb, gb = H.gb, xo = H.xo;
    int64_t e0 = b + (c - H.e_first) * A.hub_chunk, e1 = e0 + A.hub_chunk < b + deg ? e0 + A.hub_chunk : b + deg;
    for (int64_t p0 = e0; p0 < e1; p0 += HP) {
      const int32_t pc = e1 - p0 < HP ? (int32_t)(e1 - p0) : HP;  // entries of the piece
      int32_t L[HP_PER], sl[HP_PER], rk[HP_PER];
#pragma unroll
      for (int r = 0; r < HP_PER; ++r) {
        const int64_t e = p0 + r * HP_T + threadIdx.x;
        L[r] = e < e1 ? A.hlab[xo + e] : -1;
      }
#pragma unroll
      for (int r = 0; r < HP_PER; ++r)
        sl[r] = L[r] >= 0 ? hp_insert(T, (int32_t)hub_bucket_of(L[r], nb), rk[r]) : -1;
      __syncthreads();
      // the occupied slots in list order get consecutive staging ranges
      // (exclusive prefix of their counts) and one global claim each; the
      // slot's key becomes the claimed position, its value the staging offset
      const int32_t nt = T.n;
      {
        int32_t cnts[HP_PER], sum = 0;
#pragma unroll
        for (int q = 0; q < HP_PER; ++q) {
          const int32_t x = threadIdx.x * HP_PER + q;
          cnts[q] = x < nt ? T.val[T.list[x]] : 0;
          sum += cnts[q];
        }
        int32_t inc = sum;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
          const int32_t o = __shfl_up_sync(0xFFFFFFFFu, inc, d);
          if (lane >= d) inc += o;
        }
        if (lane == 31) P.wsum[wid] = inc;
        __syncthreads();
        int32_t run = inc - sum;
        for (int k = 0; k < wid; ++k) run += P.wsum[k];
#pragma unroll
        for (int q = 0; q < HP_PER; ++q) {
          const int32_t x = threadIdx.x * HP_PER + q;
          if (x < nt) {
            const int32_t h = T.list[x];
            const int64_t g = gb + T.key[h];
            T.key[h] = A.hboff[g] + atomicAdd(&A.hbcur[g], cnts[q]);
            T.val[h] = run;
            run += cnts[q];
          }
        }
      }
      __syncthreads();
#pragma unroll
      for (int r = 0; r < HP_PER; ++r)
        if (sl[r] >= 0) {
          const int32_t lp = T.val[sl[r]] + rk[r];
          P.idx[lp] = (uint16_t)(r * HP_T + threadIdx.x);
          P.slot[lp] = (uint16_t)sl[r];
        }
      __syncthreads();
      // consecutive threads write consecutive positions of a bucket's run
      for (int32_t t = threadIdx.x; t < pc; t += HP_T) {
        const int32_t h = P.slot[t];
        const int64_t pos = (int64_t)T.key[h] + (t - T.val[h]);
        const int64_t e = p0 + P.idx[t];
        A.hslab[pos] = A.hlab[xo + e];
        if (A.ew) A.hsw[pos] = A.ew[e];
      }
      __syncthreads();
      for (int32_t x = threadIdx.x; x < nt; x += HP_T) {
        const int32_t h = T.list[x];
        T.key[h] = HT_EMPTY;
        T.val[h] = 0;
      }
      if (threadIdx.x == 0) T.n = 0;
      __syncthreads();
    }
  }
}

// add w to key k's slot if k is in the table (no insert)
__device__ __forceinline__ bool ht_find_add(int32_t *keys, int32_t *vals, uint32_t mask, int32_t k, int32_t w) {
  uint32_t h = fmix32((uint32_t)k) & mask;
  for (uint32_t probe = 0; probe <= mask; ++probe) {
    int32_t c = keys[h];
    if (c == k) {
      atomicAdd(&vals[h], w);
      return true;
    }
    if (c == HT_EMPTY) return false;
    h = (h + 1) & mask;
  }
  return false;
}

constexpr int64_t DENSE_ROWS_MAX_BYTES = 4ll << 30;  // dense hub rows of one LP run
constexpr int DENSE_LABELS_MAX = 57344;              // a CTA's shared counters (224 KB)

constexpr int HB_TAB = 1024;               // per-warp table of the bucket kernel
constexpr int HB_LIMIT = HB_TAB / 2 - 32;  // labels admitted per round (load <= 1/2)

// One warp per bucket: its entries are aggregated by label in the warp's
// shared table, every lane adding its own entry (shared-memory atomics; a
// warp-level pre-aggregation was slower).  A round admits new labels while
// fewer than HB_LIMIT are held and keeps adding to labels already held after
// that; entries whose label came too late wait for the next round (a label's
// entries therefore all land in the round that admitted it).  The next round
// starts at the first chunk that came after the table filled, so only the
// entries consumed after that point are marked.  Every round ends with the
// selection pass over the occupied slots; the bucket's best keys go to its
// hub by atomicMax, the own cluster's rating (in exactly one bucket) is
// stored.  Counts and cursors are cleared for the next sub-round.
constexpr int HB_W = 8;  // warps per CTA of k_hub_bucket
constexpr size_t HB_SMEM = (size_t)HB_W * (2 * HB_TAB * sizeof(int32_t) + HB_TAB / 2 * sizeof(uint16_t));

__global__ void __launch_bounds__(HB_W * 32) k_hub_bucket(LPArgs A, int s) {
  constexpr int W = HB_W;
  extern __shared__ __align__(16) unsigned char hb_smem[];  // HB_SMEM bytes (opt-in above 48 KB)
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int32_t *keys = reinterpret_cast<int32_t *>(hb_smem) + (size_t)w * 2 * HB_TAB;
  int32_t *vals = keys + HB_TAB;
  uint16_t *list = reinterpret_cast<uint16_t *>(hb_smem + (size_t)W * 2 * HB_TAB * sizeof(int32_t)) +
                   (size_t)w * (HB_TAB / 2);
  for (int x = lane; x < HB_TAB; x += 32) {
    keys[x] = HT_EMPTY;
    vals[x] = 0;
  }
  __syncwarp();
  const int32_t *bo = A.boff + s * NB;
  const int32_t cnt = bo[7] - bo[6];
  const int64_t NBt = A.plan_tot[1];
  const uint32_t mask = HB_TAB - 1;
  const int64_t gw = (int64_t)blockIdx.x * W + w, nw = (int64_t)gridDim.x * W;
  const int64_t per = ceil_div(NBt, nw);
  const int64_t g0 = gw * per, g1 = g0 + per < NBt ? g0 + per : NBt;
  HubCursor H;
  int32_t h = -1, own = 0, cu = 0;
  for (int64_t g = g0; g < g1; ++g) {
    const int32_t ne = A.hbcnt[g];
    if (ne == 0) continue;
    H.seek(A, A.plan_b, cnt, NBt, g);
    if (A.plan_h[H.i] != h) {
      h = A.plan_h[H.i];
      own = A.label[H.u];
      cu = node_w(A, H.u);
    }
    const int64_t beg = A.hboff[g];
    uint64_t kc = 0, ku = 0;
    int32_t start = 0;  // first entry of this round; every entry before it is consumed
    while (start < ne) {
      int32_t held = 0, next = ne;
      bool mine_left = false;
      for (int32_t e0 = start; e0 < ne; e0 += 32) {
        const int32_t e = e0 + lane;
        int32_t L = e < ne ? A.hslab[beg + e] : -1;
        const bool live = L >= 0;
        const int32_t wt = live ? (A.ew ? A.hsw[beg + e] : 1) : 0;
        if (next == ne) {
          // admitting: every entry of the chunk lands in this round
          int32_t sl = live ? ht_add_fresh(keys, vals, mask, L, wt) : -1;
          unsigned m = __ballot_sync(0xFFFFFFFFu, sl >= 0);
          if (sl >= 0) list[held + __popc(m & ((1u << lane) - 1u))] = (uint16_t)sl;
          held += __popc(m);
          if (held > HB_LIMIT) next = e0 + 32;
        } else {
          // full: only labels already held; those entries are marked, as the
          // next round starts at `next`
          const bool found = live && ht_find_add(keys, vals, mask, L, wt);
          if (live && found) A.hslab[beg + e] = ~L;
          if (live && !found) mine_left = true;
        }
      }
      start = __any_sync(0xFFFFFFFFu, mine_left) ? next : ne;
      __syncwarp();
      int32_t rown = -1;
      SelTop T = select_top(A, keys, vals, list, lane, 32, held, own, cu, rown);
      if (rown >= 0) A.hrown[h] = rown;
      const uint64_t thr = group_max64<32>(T.kc > kc ? T.kc : kc);  // best admissible so far
      select_rest(A, keys, vals, list, lane, 32, held, own, cu, thr, T);
      ku = T.ku > ku ? T.ku : ku;
      kc = T.kc > kc ? T.kc : kc;
      __syncwarp();
    }
    kc = group_max64<32>(kc);
    ku = group_max64<32>(ku);
    if (lane == 0) {
      if (kc) atomicMax(&A.hkc[h], kc);
      if (ku) atomicMax(&A.hku[h], ku);
      A.hbcnt[g] = 0;
      A.hbcur[g] = 0;
    }
    __syncwarp();
  }
}


__global__ void __launch_bounds__(256) k_hub_emit(LPArgs A, int s) {
  const int32_t *bo = A.boff + s * NB;
  int32_t lo = bo[6], hi = bo[7];
  for (int64_t p = lo + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < hi;
       p += (int64_t)gridDim.x * blockDim.x) {
    int32_t u = A.vlist[p];
    int32_t h = hub_index(A, u);
    uint64_t kc = A.hkc[h], ku = A.hku[h];
    int32_t rown = A.hrown[h];
    emit(A, u, (int32_t)p, rown, kc, kc ? label_of_key(rkh(A), kc) : -1, ku,
         ku ? label_of_key(rkh(A), ku) : -1);
    A.hkc[h] = 0;
    A.hku[h] = 0;
    A.hrown[h] = 0;
  }
  stamp_stage_end(A, s);
}

// ---- hubs with few labels (refinement): dense rating rows
// work units: edge chunks of the sub-round's hubs; every CTA takes a
// contiguous range of chunks and sums them per label in shared memory (lanes
// of a warp that hit the same label add first); the non-zero sums go to the
// hub's row whenever the next chunk belongs to another hub, and at the end
__global__ void __launch_bounds__(256) k_hubd_insert(LPArgs A, int s) {
  extern __shared__ int32_t cnt_s[];
  const int32_t *bo = A.boff + s * NB;
  const int32_t lo = bo[6], cnt = bo[7] - bo[6];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t total = A.plan_tot[0];
  const int64_t per = ceil_div(total, (int64_t)gridDim.x);
  const int64_t c0 = (int64_t)blockIdx.x * per, c1 = c0 + per < total ? c0 + per : total;
  for (int32_t l = threadIdx.x; l < A.nlab; l += blockDim.x) cnt_s[l] = 0;
  __syncthreads();
  int32_t i = -1;
  int64_t next = 0, b = 0, deg = 0, efirst = 0;
  auto flush = [&]() {
    __syncthreads();
    int32_t *row = A.hdense + (int64_t)i * A.nlab;
    for (int32_t l = threadIdx.x; l < A.nlab; l += blockDim.x)
      if (cnt_s[l]) {
        atomicAdd(&row[l], cnt_s[l]);
        cnt_s[l] = 0;
      }
    __syncthreads();
  };
  for (int64_t c = c0; c < c1; ++c) {
    if (i < 0 || c >= next) {
      if (i >= 0) flush();
      if (i < 0 || c >= next + 64) {
        i = find_seg(A.plan_e, cnt, c);
      } else {
        do ++i;
        while (i + 1 < cnt && A.plan_e[i + 1] <= c);
      }
      next = i + 1 < cnt ? A.plan_e[i + 1] : total;
      const int32_t u = A.vlist[lo + i];
      b = A.xadj[u];
      deg = A.xadj[u + 1] - b;
      efirst = A.plan_e[i];
    }
    const int64_t e0 = b + (c - efirst) * A.hub_chunk;
    const int64_t e1 = e0 + A.hub_chunk < b + deg ? e0 + A.hub_chunk : b + deg;
    for (int64_t base = e0 + 32 * w; base < e1; base += blockDim.x) {
      int64_t e = base + lane;
      bool ok = e < e1;
      int32_t L = ok ? A.label[A.adj[e]] : -1;
      int32_t x = ok ? edge_w(A, e) : 0;
      unsigned peers = __match_any_sync(0xFFFFFFFFu, L);
      int32_t sum = __reduce_add_sync(peers, x);
      if (ok && lane == __ffs(peers) - 1) atomicAdd(&cnt_s[L], sum);
    }
  }
  if (i >= 0) flush();
}

// one CTA per hub of the sub-round: best labels from its row (cleared for
// the next use), then the same decision as every other bin
__global__ void __launch_bounds__(256) k_hubd_reduce(LPArgs A, int s) {
  __shared__ unsigned long long red_c[8], red_u[8];
  __shared__ int32_t s_rown;
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int32_t *bo = A.boff + s * NB;
  int32_t lo = bo[6], cnt = bo[7] - bo[6];
  for (int32_t i = blockIdx.x; i < cnt; i += gridDim.x) {
    int32_t u = A.vlist[lo + i];
    int32_t own = A.label[u], cu = node_w(A, u);
    int32_t *row = A.hdense + (int64_t)i * A.nlab;
    if (threadIdx.x == 0) s_rown = 0;
    __syncthreads();
    uint64_t kc = 0, ku = 0;
    for (int32_t K = threadIdx.x; K < A.nlab; K += blockDim.x) {
      int32_t r = row[K];
      if (r == 0) continue;
      row[K] = 0;
      if (K == own) {
        s_rown = r;
        continue;
      }
      uint64_t k = rate_key(A, K, r);
      ku = k > ku ? k : ku;
      if ((int64_t)A.wt[K] + cu <= cap_of(A, K) && k > kc) kc = k;
    }
    kc = group_max64<32>(kc);
    ku = group_max64<32>(ku);
    if (lane == 0) {
      red_c[w] = kc;
      red_u[w] = ku;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int x = 1; x < (int)(blockDim.x >> 5); ++x) {
        kc = red_c[x] > kc ? red_c[x] : kc;
        ku = red_u[x] > ku ? red_u[x] : ku;
      }
      emit(A, u, lo + i, s_rown, kc, kc ? label_of_key(rkh(A), kc) : -1, ku,
           ku ? label_of_key(rkh(A), ku) : -1);
    }
    __syncthreads();
  }
  stamp_stage_end(A, s);
}

__global__ void k_hub_flags(int32_t n, const int64_t *xadj, int64_t huge, uint8_t *flag) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x)
    flag[v] = (xadj[v + 1] - xadj[v]) > huge ? 1 : 0;
}

// hub ids in ascending order and their degrees
__global__ void k_hub_list(int32_t n, const int64_t *xadj, const uint8_t *flag, const int32_t *pos,
                           int32_t *hubs, int64_t *hdeg) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x)
    if (flag[v]) {
      hubs[pos[v]] = (int32_t)v;
      hdeg[pos[v]] = xadj[v + 1] - xadj[v];
    }
}

// ------------------------------------------------------------------- commit
__global__ void __launch_bounds__(256) k_classify(LPArgs A, int s) {
  int32_t lo = A.boff[s * NB], hi = A.boff[(s + 1) * NB];
  for (int64_t pos = lo + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; pos < hi;
       pos += (int64_t)gridDim.x * blockDim.x) {
    int32_t T = A.prop_t[pos];
    if (T < 0) continue;
    if ((int64_t)A.wt[T] + A.tsum[T] <= cap_of(A, T)) {
      A.acc[pos] = 1;
    } else {
      A.acc[pos] = 0;
      int32_t r = atomicAdd(&A.tcur[T], 1);
      A.pos_in_t[pos] = r;
      if (r == 0) {
        int32_t sl = atomicAdd(&A.ctr[0], 1);
        A.slot_t[sl] = T;
        A.slot_base[sl] = atomicAdd(&A.ctr[1], A.tcnt[T]);
        A.tslot[T] = sl;
      }
    }
  }
}

__global__ void __launch_bounds__(256) k_bucket(LPArgs A, int s) {
  if (A.ctr[0] == 0) return;
  int32_t lo = A.boff[s * NB], hi = A.boff[(s + 1) * NB];
  for (int64_t pos = lo + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; pos < hi;
       pos += (int64_t)gridDim.x * blockDim.x) {
    int32_t T = A.prop_t[pos];
    if (T < 0 || A.acc[pos]) continue;
    int32_t sl = A.tslot[T];
    A.bucket[A.slot_base[sl] + A.pos_in_t[pos]] = (int32_t)pos;
  }
}

__device__ __forceinline__ uint64_t commit_key(const LPArgs &A, int32_t pos) {
  return ((uint64_t)(uint32_t)(0x7FFFFFFF - A.prop_g[pos]) << 32) | (uint32_t)A.vlist[pos];
}

__global__ void __launch_bounds__(256) k_resolve(LPArgs A) {
  int32_t nslots = A.ctr[0];
  if (nslots == 0) return;
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int64_t gw = (int64_t)blockIdx.x * (blockDim.x / 32) + w;
  int64_t nw = (int64_t)gridDim.x * (blockDim.x / 32);
  // small contested targets: one warp each
  for (int64_t sl = gw; sl < nslots; sl += nw) {
    int32_t T = A.slot_t[sl];
    int32_t cnt = A.tcnt[T];
    if (cnt > 32) continue;
    int32_t base = A.slot_base[sl];
    uint64_t key = ~0ull;
    int32_t c = 0, pos = -1;
    if (lane < cnt) {
      pos = A.bucket[base + lane];
      key = commit_key(A, pos);
      c = node_w(A, A.vlist[pos]);
    }
    int64_t pre = 0;
    for (int j = 0; j < 32; ++j) {
      uint64_t kj = __shfl_sync(0xFFFFFFFFu, key, j);
      int32_t cj = __shfl_sync(0xFFFFFFFFu, c, j);
      if (j < cnt && kj <= key) pre += cj;
    }
    int64_t R = cap_of(A, T) - A.wt[T];
    if (lane < cnt) A.acc[pos] = (pre <= R) ? 1 : 0;
  }
  // large contested targets: one block each, radix select of the accepted prefix
  __shared__ unsigned long long hist[256];
  __shared__ uint64_t prefix;
  __shared__ long long accw;
  for (int64_t sl = blockIdx.x; sl < nslots; sl += gridDim.x) {
    int32_t T = A.slot_t[sl];
    int32_t cnt = A.tcnt[T];
    if (cnt <= 32) continue;
    int32_t base = A.slot_base[sl];
    int64_t R = cap_of(A, T) - A.wt[T];
    if (R < 0) continue;  // nothing fits (acc already 0)
    // skip the leading digits that every key shares (all gains of a target
    // are usually small, so the top bytes agree): common prefix of min..max
    __shared__ unsigned long long kmin, kmax;
    if (threadIdx.x == 0) { kmin = ~0ull; kmax = 0; }
    __syncthreads();
    {
      unsigned long long lmin = ~0ull, lmax = 0;
      for (int32_t i = threadIdx.x; i < cnt; i += blockDim.x) {
        unsigned long long k = commit_key(A, A.bucket[base + i]);
        lmin = k < lmin ? k : lmin;
        lmax = k > lmax ? k : lmax;
      }
      atomicMin(&kmin, lmin);
      atomicMax(&kmax, lmax);
    }
    __syncthreads();
    int p0 = 0;
    {
      unsigned long long diff = kmin ^ kmax;  // != 0: keys are distinct and cnt > 32
      int top = 63 - __clzll((long long)diff);
      p0 = (63 - top) / 8;                     // first byte (from the top) that differs
    }
    if (threadIdx.x == 0) {
      prefix = p0 > 0 ? (kmin >> (64 - 8 * p0)) : 0;
      accw = 0;
    }
    __syncthreads();
    for (int p = p0; p < 8; ++p) {
      int sh = 56 - 8 * p;
      for (int i = threadIdx.x; i < 256; i += blockDim.x) hist[i] = 0;
      __syncthreads();
      uint64_t pf = prefix;
      int lane2 = threadIdx.x & 31;
      for (int32_t i0 = 0; i0 < cnt; i0 += blockDim.x) {
        int32_t i = i0 + threadIdx.x;
        int d = 256 + lane2;  // unique per lane when not counted
        unsigned long long wgt = 0;
        if (i < cnt) {
          int32_t ps = A.bucket[base + i];
          uint64_t k = commit_key(A, ps);
          if (p == 0 || (k >> (sh + 8)) == pf) {
            d = (int)((k >> sh) & 255u);
            wgt = (unsigned long long)node_w(A, A.vlist[ps]);
          }
        }
        // lanes with the same digit add their weights first: one atomic per digit and warp
        unsigned peers = __match_any_sync(0xFFFFFFFFu, d);
        unsigned long long sum = 0;
        for (int j = 0; j < 32; ++j) {
          unsigned long long wj = __shfl_sync(0xFFFFFFFFu, wgt, j);
          if ((peers >> j) & 1u) sum += wj;
        }
        if (d < 256 && (peers & ((1u << lane2) - 1u)) == 0) atomicAdd(&hist[d], sum);
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        long long run = accw;
        int dstar = 255;
        for (int d = 0; d < 256; ++d) {
          if (run + (long long)hist[d] <= R) {
            run += (long long)hist[d];
          } else {
            dstar = d;
            break;
          }
        }
        accw = run;
        prefix = (pf << 8) | (uint64_t)dstar;
      }
      __syncthreads();
    }
    uint64_t thr = prefix;  // key of the first rejected proposal
    for (int32_t i = threadIdx.x; i < cnt; i += blockDim.x) {
      int32_t ps = A.bucket[base + i];
      A.acc[ps] = commit_key(A, ps) < thr ? 1 : 0;
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(256) k_apply(LPArgs A, int s) {
  int32_t lo = A.boff[s * NB], hi = A.boff[(s + 1) * NB];
  uint8_t *nxt = act_nxt(A);
  unsigned long long moved = 0;
  for (int64_t pos = lo + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; pos < hi;
       pos += (int64_t)gridDim.x * blockDim.x) {
    int32_t T = A.prop_t[pos];
    if (T < 0) continue;
    int32_t u = A.vlist[pos];
    if (A.acc[pos]) {
      int32_t own = A.label[u], c = node_w(A, u);
      A.label[u] = T;
      atomicAdd(&A.wt[T], c);
      atomicSub(&A.wt[own], c);
      ++moved;
      int64_t b = A.xadj[u], e1 = A.xadj[u + 1];
      if (e1 - b > 64) {
        A.bigmove[atomicAdd(&A.ctr[2], 1)] = u;  // neighbours marked by k_scatter_big
      } else {
        for (int64_t e = b; e < e1; ++e) nxt[A.adj[e]] = 1;
      }
    } else if (A.fav) {
      A.fav[u] = T;
    }
    A.tsum[T] = 0;
    A.tcnt[T] = 0;
    A.tcur[T] = 0;
  }
#pragma unroll
  for (int m = 16; m > 0; m >>= 1) moved += __shfl_xor_sync(0xFFFFFFFFu, moved, m);
  if ((threadIdx.x & 31) == 0 && moved) atomicAdd(&ctr_cur(A)[1], moved);
}

// neighbours of high-degree nodes that moved become active: one block per node
__global__ void __launch_bounds__(256) k_scatter_big(LPArgs A) {
  int32_t nb = A.ctr[2];
  uint8_t *nxt = act_nxt(A);
  for (int32_t i = blockIdx.x; i < nb; i += gridDim.x) {
    int32_t u = A.bigmove[i];
    for (int64_t e = A.xadj[u] + threadIdx.x; e < A.xadj[u + 1]; e += blockDim.x) nxt[A.adj[e]] = 1;
  }
}

__global__ void k_fill_i32(int32_t *p, int64_t n, int32_t v) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    p[i] = v;
}

// ------------------------------------------------------------------- driver
void lp_run(const Graph &g, int32_t *label, int32_t *wt, int32_t nlab, const int32_t *cap,
            int32_t U, int32_t rounds, uint64_t basekey, int32_t *fav, LPStats *st) {
  Context &C = ctx();
  const int S = C.cfg.subrounds;
  cudaStream_t stream = C.stream;
  int32_t n = g.n;
  LPStats local;
  if (!st) st = &local;
  *st = LPStats();
  if (n == 0 || rounds <= 0) return;
  cudaEvent_t e0, e1;
  KMP_CUDA(cudaEventCreate(&e0));
  KMP_CUDA(cudaEventCreate(&e1));
  KMP_CUDA(cudaEventRecord(e0, stream));

  int64_t ntiles = ceil_div(n, BIN_TILE);
  DBuf<uint8_t> act(n), act_next(n), acc(n);
  DBuf<int32_t> vlist(n), boff(S * NB + 1), prop_t(n), prop_g(n), pos_in_t(n);
  DBuf<int32_t> tsum(nlab), tcnt(nlab), tcur(nlab), tslot(nlab);
  DBuf<int32_t> slot_t(n), slot_base(n), bucket(n), ctr(8), bigmove(n);
  DBuf<int32_t> bcnt(S * NB * ntiles), boffs(S * NB * ntiles), btotal(1);
  act.fill_bytes(1);
  act_next.zero();
  tsum.zero();
  tcnt.zero();
  tcur.zero();
  ctr.zero();

  // hubs: with few labels (refinement) a shared-memory table always fits;
  // otherwise every sub-round's hub entries are aggregated in label buckets
  // (entry buffers sized by the hubs' total degree, one count, cursor and
  // offset per bucket)
  bool small_labels = 2 * (int64_t)nlab <= CTA_TAB;
  const int64_t huge = small_labels ? C.tune.dense_hub_degree : C.tune.hub_degree;
  bool hub_path = !small_labels && g.maxdeg > huge;
  bool dense_hubs = small_labels && g.maxdeg > huge;
  // with more labels than a CTA table holds but at most tune.dense_labels of
  // them, hubs may rate into dense rows of nlab counters (the paper's dense
  // vector for high-degree nodes) when all rows fit DENSE_ROWS_MAX_BYTES
  if (hub_path && C.tune.dense_labels > 0 && nlab <= C.tune.dense_labels) {
    DBuf<uint8_t> flag(n);
    DBuf<int32_t> pos(n), cnt(1);
    k_hub_flags<<<grid_for(n, 256), 256, 0, stream>>>(n, g.xadj, huge, flag);
    KMP_LAUNCHED("hub_flags");
    scan_excl_u8_to_i32(flag, pos, n, cnt);
    const int64_t nh = read1(cnt.p);
    if (nh * (int64_t)nlab * (int64_t)sizeof(int32_t) <= DENSE_ROWS_MAX_BYTES) {
      hub_path = false;
      dense_hubs = true;
    }
  }
  const int32_t hub_bucket = C.tune.hub_bucket > 0 ? C.tune.hub_bucket : 256;
  int32_t nhubs = 0;
  int64_t nbmax = 0;
  DBuf<int32_t> hubs, hrown, plan_h, hdense, hlab, hslab, hsw, hbcnt, hbcur, hboff, hbsum;
  DBuf<int64_t> plan_e, plan_x, plan_b, plan_tot;
  DBuf<unsigned long long> hkc, hku;
  if (hub_path) {
    DBuf<uint8_t> flag(n);
    DBuf<int32_t> pos(n), cnt(1);
    k_hub_flags<<<grid_for(n, 256), 256, 0, stream>>>(n, g.xadj, huge, flag);
    KMP_LAUNCHED("hub_flags");
    scan_excl_u8_to_i32(flag, pos, n, cnt);
    nhubs = read1(cnt.p);
    hubs.alloc(nhubs);
    DBuf<int64_t> hdeg(nhubs), hdoff(nhubs), tot(1);
    k_hub_list<<<grid_for(n, 256), 256, 0, stream>>>(n, g.xadj, flag, pos, hubs, hdeg);
    KMP_LAUNCHED("hub_list");
    scan_excl_i64(hdeg, hdoff, nhubs, tot);
    const int64_t Dhub = read1(tot.p);  // bounds the entries of any sub-round
    nbmax = Dhub / hub_bucket + nhubs;  // bounds its buckets (ceil per hub)
    hlab.alloc(Dhub);
    hslab.alloc(Dhub);
    if (g.ew) hsw.alloc(Dhub);
    hbcnt.alloc(nbmax);
    hbcur.alloc(nbmax);
    hboff.alloc(nbmax);
    hbsum.alloc(scan_tmp_count(nbmax));
    hbcnt.zero();
    hbcur.zero();
    hkc.alloc(nhubs);
    hku.alloc(nhubs);
    hrown.alloc(nhubs);
    hkc.zero();
    hku.zero();
    hrown.zero();
    plan_h.alloc(nhubs);
    plan_e.alloc(nhubs + 1);
    plan_x.alloc(nhubs + 1);
    plan_b.alloc(nhubs + 1);
    plan_tot.alloc(3);
    static bool hb_attr = false;  // before any capture: the bucket kernel's tables exceed 48 KB
    if (!hb_attr) {
      KMP_CUDA(cudaFuncSetAttribute(k_hub_bucket, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)HB_SMEM));
      hb_attr = true;
    }
  } else if (dense_hubs) {
    DBuf<uint8_t> flag(n);
    DBuf<int32_t> pos(n), cnt(1);
    k_hub_flags<<<grid_for(n, 256), 256, 0, stream>>>(n, g.xadj, huge, flag);
    KMP_LAUNCHED("hub_flags");
    scan_excl_u8_to_i32(flag, pos, n, cnt);
    nhubs = read1(cnt.p);
    hdense.alloc((int64_t)nhubs * nlab);
    hdense.zero();
    static bool hd_attr = false;  // before any capture: counters of up to DENSE_LABELS_MAX labels
    if (!hd_attr) {
      KMP_CUDA(cudaFuncSetAttribute(k_hubd_insert, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    DENSE_LABELS_MAX * (int)sizeof(int32_t)));
      hd_attr = true;
    }
    plan_h.alloc(nhubs);
    plan_e.alloc(nhubs + 1);
    plan_x.alloc(nhubs + 1);
    plan_b.alloc(nhubs + 1);
    plan_tot.alloc(3);
  }

  LPArgs A{};
  A.n = n;
  A.xadj = g.xadj;
  A.adj = g.adj;
  A.vw = g.vw;
  A.ew = g.ew;
  A.label = label;
  A.wt = wt;
  A.cap = cap;
  A.U = U;
  A.fav = fav;
  A.act0 = act;
  A.act1 = act_next;
  A.vlist = vlist;
  A.boff = boff;
  A.prop_t = prop_t;
  A.prop_g = prop_g;
  A.acc = acc;
  A.pos_in_t = pos_in_t;
  A.tsum = tsum;
  A.tcnt = tcnt;
  A.tcur = tcur;
  A.tslot = tslot;
  A.slot_t = slot_t;
  A.slot_base = slot_base;
  A.bucket = bucket;
  A.ctr = ctr;
  A.bigmove = bigmove;
  A.hubs = hubs.p;
  A.nhubs = nhubs;

  A.hkc = hkc.p;
  A.hku = hku.p;
  A.hrown = hrown.p;
  A.hlab = hlab.p;
  A.hslab = hslab.p;
  A.hsw = hsw.p;
  A.hbcnt = hbcnt.p;
  A.hbcur = hbcur.p;
  A.hboff = hboff.p;
  A.hub_bucket = dense_hubs ? 0 : hub_bucket;
  A.plan_h = plan_h.p;
  A.plan_e = plan_e.p;
  A.plan_x = plan_x.p;
  A.plan_b = plan_b.p;
  A.plan_tot = plan_tot.p;
  A.small_labels = small_labels ? 1 : 0;
  A.hdense = dense_hubs ? hdense.p : nullptr;
  A.huge_deg = huge;
  A.hub_chunk = C.tune.hub_chunk;
  A.nlab = nlab;
  A.S = S;

  int grid_rate = C.tune.rate_blocks_per_sm * C.sms;
  int grid_hub = 4 * C.sms;
  int grid_bucket = 3 * C.sms;  // k_hub_bucket: 72 KB of tables per CTA
  int grid_commit = grid_for(ceil_div(n, S), 256, 8);
  // per-round state and counters in device memory (18 counters a round)
  DBuf<LPRound> rstate(1);
  DBuf<unsigned long long> ctr_all((size_t)18 * rounds);
  DBuf<int32_t> sbsum(scan_tmp_count((int64_t)S * NB * ntiles));
  rstate.zero();
  ctr_all.zero();
  A.R = rstate;
  A.ctr64 = ctr_all;
  // profiling: the span of every k_rate launch on the device's global timer
  // (first CTA start to last CTA end; stamps taken inside the kernel, so the
  // replayed graph needs no extra nodes) and each round's bin offsets, all
  // read after the run
  DBuf<int32_t> boff_all;
  DBuf<unsigned long long> tmin, tmax, smax;
  if (C.profile) {
    boff_all.alloc((size_t)(S * NB + 1) * rounds);
    tmin.alloc((size_t)S * rounds);
    tmax.alloc((size_t)S * rounds);
    smax.alloc((size_t)S * rounds);
    tmin.fill_bytes(0xFF);
    tmax.zero();
    smax.zero();
    A.tmin = tmin;
    A.tmax = tmax;
    A.smax = smax;
  }
  // one LP round: binning, then per sub-round rating, hub rating and commit
  auto launch_round = [&](cudaStream_t st) {
    k_round_begin<<<1, 1, 0, st>>>(A, basekey);
    KMP_LAUNCHED("round_begin");
    k_bin_count<<<(unsigned)ntiles, 256, 0, st>>>(A, bcnt, ntiles);
    KMP_LAUNCHED("bin_count");
    scan_excl_i32_on(bcnt, boffs, (int64_t)S * NB * ntiles, btotal, sbsum, st);
    k_bin_boff<<<1, 64, 0, st>>>(A, boffs, btotal, ntiles);
    KMP_LAUNCHED("bin_boff");
    k_bin_scatter<<<(unsigned)ntiles, 256, 0, st>>>(A, boffs, ntiles);
    KMP_LAUNCHED("bin_scatter");
    if (C.profile) {
      k_save_boff<<<1, 128, 0, st>>>(A, boff_all);
      KMP_LAUNCHED("save_boff");
    }
    for (int s = 0; s < S; ++s) {
      k_rate<<<grid_rate, RATE_T, 0, st>>>(A, s);
      KMP_LAUNCHED("rate");
      if (hub_path) {
        k_hub_plan<<<1, 1024, 0, st>>>(A, s);
        KMP_LAUNCHED("hub_plan");
        k_hub_count<<<grid_hub, HP_T, 0, st>>>(A, s);
        KMP_LAUNCHED("hub_count");
        scan_excl_i32_on(hbcnt, hboff, nbmax, nullptr, hbsum, st);
        k_hub_scatter<<<grid_hub, HP_T, 0, st>>>(A, s);
        KMP_LAUNCHED("hub_scatter");
        k_hub_bucket<<<grid_bucket, HB_W * 32, HB_SMEM, st>>>(A, s);
        KMP_LAUNCHED("hub_bucket");
        k_hub_emit<<<grid_for(nhubs, 256), 256, 0, st>>>(A, s);
        KMP_LAUNCHED("hub_emit");
      } else if (dense_hubs) {
        k_hub_plan<<<1, 1024, 0, st>>>(A, s);
        KMP_LAUNCHED("hub_plan");
        k_hubd_insert<<<grid_hub, 256, nlab * sizeof(int32_t), st>>>(A, s);
        KMP_LAUNCHED("hubd_insert");
        k_hubd_reduce<<<std::min(nhubs, grid_hub), 256, 0, st>>>(A, s);
        KMP_LAUNCHED("hubd_reduce");
      }
      k_classify<<<grid_commit, 256, 0, st>>>(A, s);
      KMP_LAUNCHED("classify");
      k_bucket<<<grid_commit, 256, 0, st>>>(A, s);
      KMP_LAUNCHED("bucket");
      k_resolve<<<grid_commit, 256, 0, st>>>(A);
      KMP_LAUNCHED("resolve");
      k_apply<<<grid_commit, 256, 0, st>>>(A, s);
      KMP_LAUNCHED("apply");
      if (g.maxdeg > 64) {
        k_scatter_big<<<2 * C.sms, 256, 0, st>>>(A);
        KMP_LAUNCHED("scatter_big");
      }
    }
  };
  // profiling: k_rate times and algorithmic bytes of rounds [0, nr) (per edge
  // visit adjncy + neighbour label (+ edge weight); per rated node xadj, list
  // entry, own label, proposal (target, gain) (+ node weight); hubs rated by
  // the hub kernels are not k_rate's work)
  auto profile_rounds = [&](int nr) {
    std::vector<unsigned long long> h((size_t)18 * nr), t0((size_t)S * nr), t1((size_t)S * nr),
        t2((size_t)S * nr);
    std::vector<int32_t> hb((size_t)(S * NB + 1) * nr);
    to_host(h.data(), ctr_all.p, h.size());
    to_host(hb.data(), boff_all.p, hb.size());
    to_host(t0.data(), tmin.p, t0.size());
    to_host(t1.data(), tmax.p, t1.size());
    to_host(t2.data(), smax.p, t2.size());
    bool hubs_outside = hub_path || dense_hubs;
    const double per_entry = 8.0 + (g.ew ? 4.0 : 0.0), per_node = 24.0 + (g.vw ? 4.0 : 0.0);
    for (int r = 0; r < nr; ++r) {
      const int32_t *hboff = hb.data() + (size_t)(S * NB + 1) * r;
      for (int s = 0; s < S; ++s) {
        const double Vall = (double)(hboff[(s + 1) * NB] - hboff[s * NB]);
        const double Dall = (double)h[18 * r + 2 + s];
        double V = Vall, D = Dall;
        if (hubs_outside) {
          V -= (double)(hboff[s * NB + 7] - hboff[s * NB + 6]);
          D -= (double)h[18 * r + 10 + s];
        }
        size_t i = (size_t)S * r + s;
        C.prof_rate_ms += t1[i] > t0[i] ? (double)(t1[i] - t0[i]) * 1e-6 : 0.0;
        C.prof_rate_launches += 1;
        C.prof_rate_bytes += D * per_entry + V * per_node;
        C.prof_stage_ms += t2[i] > t0[i] ? (double)(t2[i] - t0[i]) * 1e-6 : 0.0;
        C.prof_stage_spans += 1;
        C.prof_stage_bytes += Dall * per_entry + Vall * per_node;
      }
    }
  };
  if (C.tune.lp_graphs) {
    // one captured round, replayed for every round: its kernels read the
    // round's key, buffers and counters from device memory.  A round after
    // one that moved nothing has no active node and changes nothing, so all
    // rounds can be queued without reading the move counts in between.
    if (!C.capture_stream) KMP_CUDA(cudaStreamCreateWithFlags(&C.capture_stream, cudaStreamNonBlocking));
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int64_t before = C.launches;
    KMP_CUDA(cudaStreamBeginCapture(C.capture_stream, cudaStreamCaptureModeThreadLocal));
    try {
      launch_round(C.capture_stream);
    } catch (...) {
      cudaStreamEndCapture(C.capture_stream, &graph);
      if (graph) cudaGraphDestroy(graph);
      throw;
    }
    KMP_CUDA(cudaStreamEndCapture(C.capture_stream, &graph));
    int64_t per_round = C.launches - before;
    cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    KMP_CUDA(ie);
    cudaError_t le = cudaSuccess;
    for (int r = 0; r < rounds && le == cudaSuccess; ++r) {
      le = cudaGraphLaunch(exec, stream);
      if (r > 0) C.launches += per_round;
    }
    // an executable graph still in flight is released when it completes
    cudaGraphExecDestroy(exec);
    KMP_CUDA(le);
    if (C.profile) profile_rounds(rounds);
  } else {
    int r = 0;
    for (; r < rounds; ++r) {
      launch_round(stream);
      unsigned long long mv = read1(ctr_all.p + 18 * r + 1);
      if (mv == 0) {
        ++r;
        break;
      }
    }
    if (C.profile) profile_rounds(r);
  }
  // statistics: rounds up to and including the first that moved nothing
  std::vector<unsigned long long> hall((size_t)18 * rounds);
  to_host(hall.data(), ctr_all.p, hall.size());
  for (int r = 0; r < rounds; ++r) {
    st->rounds = r + 1;
    st->scanned += (int64_t)hall[18 * r];
    st->moved_total += (int64_t)hall[18 * r + 1];
    if (hall[18 * r + 1] == 0) break;
  }
  KMP_CUDA(cudaEventRecord(e1, stream));
  KMP_CUDA(cudaEventSynchronize(e1));
  float ms = 0;
  KMP_CUDA(cudaEventElapsedTime(&ms, e0, e1));
  st->ms = ms;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
}

// ------------------------------------------------ clustering of one level
__global__ void k_init_cluster(int32_t n, const int32_t *vw, int32_t *label, int32_t *wt,
                               int32_t *fav) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    label[v] = (int32_t)v;
    wt[v] = vw ? vw[v] : 1;
    fav[v] = -1;
  }
}

__global__ void k_iso_w(int32_t n, const int64_t *xadj, const int32_t *vw, int32_t *w) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x)
    w[v] = (xadj[v + 1] == xadj[v]) ? (vw ? vw[v] : 1) : 0;
}

// isolated node v with exclusive prefix weight P joins chunk floor(P/U) unless it straddles
__global__ void k_iso_chunk(int32_t n, const int64_t *xadj, const int32_t *vw, const int64_t *P,
                            int32_t U, int32_t *first, int pass, int32_t *label) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    if (xadj[v + 1] != xadj[v]) continue;
    int64_t c = vw ? vw[v] : 1;
    int64_t q = P[v] / U, qe = (P[v] + c - 1) / U;
    if (q != qe) continue;
    if (pass == 0) atomicMin(&first[q], label[v]);
    else label[v] = first[q];
  }
}

__global__ void k_mark_used(int32_t n, const int32_t *label, uint8_t *used) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x)
    used[label[v]] = 1;
}

__global__ void k_count_u8(int64_t n, const uint8_t *f, unsigned long long *out) {
  unsigned long long s = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    s += f[i];
#pragma unroll
  for (int m = 16; m > 0; m >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, m);
  if ((threadIdx.x & 31) == 0 && s) atomicAdd(out, s);
}

static int32_t count_clusters(int32_t n, const int32_t *label) {
  cudaStream_t s = ctx().stream;
  DBuf<uint8_t> used(n);
  used.zero();
  DBuf<unsigned long long> cnt(1);
  cnt.zero();
  int grid = grid_for(n, 256);
  k_mark_used<<<grid, 256, 0, s>>>(n, label, used);
  KMP_LAUNCHED("mark_used");
  k_count_u8<<<grid, 256, 0, s>>>(n, used, cnt);
  KMP_LAUNCHED("count_u8");
  return (int32_t)read1(cnt.p);
}

// two-hop: candidates are singleton clusters with a favoured cluster
__global__ void k_cluster_size(int32_t n, const int32_t *label, int32_t *size) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(&size[label[v]], 1);
}

__global__ void k_twohop_cand(int32_t n, const int32_t *label, const int32_t *size,
                              const int32_t *fav, int bits, uint64_t *keys, int32_t *count) {
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n;
       u += (int64_t)gridDim.x * blockDim.x) {
    if (size[label[u]] != 1 || fav[u] < 0) continue;
    int32_t p = atomicAdd(count, 1);
    keys[p] = ((uint64_t)(uint32_t)fav[u] << bits) | (uint64_t)u;
  }
}

__global__ void k_twohop_heads(int32_t N, const uint64_t *keys, int bits, uint8_t *head) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x)
    head[i] = (i == 0 || (keys[i] >> bits) != (keys[i - 1] >> bits)) ? 1 : 0;
}

__global__ void k_twohop_headpos(int32_t N, const uint8_t *head, const int32_t *hidx, int32_t *H) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x)
    if (head[i]) H[hidx[i]] = (int32_t)i;
}

__global__ void k_twohop_valid(int32_t N, const uint64_t *keys, int bits, const int32_t *H,
                               int32_t nh, const int32_t *vw, int32_t U, uint8_t *valid) {
  uint64_t mask = (bits >= 64) ? ~0ull : ((1ull << bits) - 1ull);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    // group start: largest head position <= i
    int32_t lo = 0, hi = nh - 1;
    while (lo < hi) {
      int32_t mid = (lo + hi + 1) >> 1;
      if (H[mid] <= i) lo = mid;
      else hi = mid - 1;
    }
    int64_t off = i - H[lo];
    uint8_t ok = 0;
    if ((off & 1) == 0 && i + 1 < N && (keys[i] >> bits) == (keys[i + 1] >> bits)) {
      int32_t a = (int32_t)(keys[i] & mask), b = (int32_t)(keys[i + 1] & mask);
      int64_t w = (int64_t)(vw ? vw[a] : 1) + (vw ? vw[b] : 1);
      ok = w <= U ? 1 : 0;
    }
    valid[i] = ok;
  }
}

__global__ void k_twohop_apply(int32_t N, const uint64_t *keys, int bits, const uint8_t *valid,
                               const int32_t *rank, int32_t need, int32_t *label) {
  uint64_t mask = (1ull << bits) - 1ull;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (!valid[i] || rank[i] >= need) continue;
    int32_t a = (int32_t)(keys[i] & mask), b = (int32_t)(keys[i + 1] & mask);
    label[b] = label[a];
  }
}

static void two_hop(const Graph &g, int32_t U, const int32_t *fav, int32_t *label, int32_t nc) {
  int32_t n = g.n;
  if (2 * (int64_t)nc <= n) return;
  int32_t need = nc - n / 2;
  cudaStream_t s = ctx().stream;
  int grid = grid_for(n, 256);
  DBuf<int32_t> size(n), count(1);
  size.zero();
  count.zero();
  int bits = 1;
  while ((1ll << bits) < (int64_t)n) ++bits;
  DBuf<uint64_t> keys(n), tmp(n);
  k_cluster_size<<<grid, 256, 0, s>>>(n, label, size);
  KMP_LAUNCHED("cluster_size");
  k_twohop_cand<<<grid, 256, 0, s>>>(n, label, size, fav, bits, keys, count);
  KMP_LAUNCHED("twohop_cand");
  int32_t N = read1(count.p);
  if (N < 2) return;
  radix_sort_u64(keys, tmp, N, 2 * bits);
  int gN = grid_for(N, 256);
  DBuf<uint8_t> head(N), valid(N);
  DBuf<int32_t> hidx(N), H(N), rank(N), nh(1), nvalid(1);
  k_twohop_heads<<<gN, 256, 0, s>>>(N, keys, bits, head);
  KMP_LAUNCHED("twohop_heads");
  scan_excl_u8_to_i32(head, hidx, N, nh);
  k_twohop_headpos<<<gN, 256, 0, s>>>(N, head, hidx, H);
  KMP_LAUNCHED("twohop_headpos");
  int32_t nhh = read1(nh.p);
  k_twohop_valid<<<gN, 256, 0, s>>>(N, keys, bits, H, nhh, g.vw, U, valid);
  KMP_LAUNCHED("twohop_valid");
  scan_excl_u8_to_i32(valid, rank, N, nvalid);
  k_twohop_apply<<<gN, 256, 0, s>>>(N, keys, bits, valid, rank, need, label);
  KMP_LAUNCHED("twohop_apply");
}

int32_t cluster_level(const Graph &g, int32_t U, int32_t rounds, uint64_t basekey, bool do_two_hop,
                      int32_t *label, int32_t *fav_out, LPStats *st, float *ms_other) {
  Context &C = ctx();
  cudaStream_t s = C.stream;
  int32_t n = g.n;
  DBuf<int32_t> wt(n), favb;
  int32_t *fav = fav_out;
  if (!fav) {
    favb.alloc(n);
    fav = favb;
  }
  int grid = grid_for(n, 256);
  k_init_cluster<<<grid, 256, 0, s>>>(n, g.vw, label, wt, fav);
  KMP_LAUNCHED("init_cluster");
  lp_run(g, label, wt, n, nullptr, U, rounds, basekey, fav, st);
  cudaEvent_t e0, e1;
  KMP_CUDA(cudaEventCreate(&e0));
  KMP_CUDA(cudaEventCreate(&e1));
  KMP_CUDA(cudaEventRecord(e0, s));
  if (g.n_isolated > 0) {
    DBuf<int32_t> w(n), first(n + 1);
    DBuf<int64_t> P(n);
    k_iso_w<<<grid, 256, 0, s>>>(n, g.xadj, g.vw, w);
    KMP_LAUNCHED("iso_w");
    scan_excl_i32_to_i64(w, P, n, nullptr);
    k_fill_i32<<<grid_for(n + 1, 256), 256, 0, s>>>(first, n + 1, INT32_MAX);
    KMP_LAUNCHED("fill");
    k_iso_chunk<<<grid, 256, 0, s>>>(n, g.xadj, g.vw, P, U, first, 0, label);
    KMP_LAUNCHED("iso_chunk");
    k_iso_chunk<<<grid, 256, 0, s>>>(n, g.xadj, g.vw, P, U, first, 1, label);
    KMP_LAUNCHED("iso_chunk");
  }
  int32_t nc = count_clusters(n, label);
  if (do_two_hop && 2 * (int64_t)nc > n) {
    two_hop(g, U, fav, label, nc);
    nc = count_clusters(n, label);
  }
  KMP_CUDA(cudaEventRecord(e1, s));
  KMP_CUDA(cudaEventSynchronize(e1));
  float ms = 0;
  KMP_CUDA(cudaEventElapsedTime(&ms, e0, e1));
  if (ms_other) *ms_other += ms;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return nc;
}

}  // namespace kmp
