// Batched multilevel initial bipartitioning (Section 4.2) for Algorithm 2
// (bipartitionBlocks): every block that must be split becomes one work item;
// all items of a split round run in ONE persistent launch whose CTAs take
// items from a device work queue (largest first).  Per item, one CTA:
//   1. coarsens the induced subgraph G[B] with the deterministic sub-round LP
//      (CTA-parallel rating with per-warp hash tables, commit by a bitonic
//      sort of (target, gain desc, node) keys and a segmented prefix sum),
//      packs isolated nodes, and contracts (sort of (cu, cv) pairs, run sums),
//      level after level until nothing contracts or the shrink stalls;
//   2. runs the portfolio -- random, BFS and greedy graph growing starts, each
//      refined by 2-way FM -- with one warp per repetition; in learned mode
//      the CTA first scores the coarsest graph with the message-passing
//      network (kmp_mpnn.cuh) and its score order is one more start, ahead of
//      a reduced portfolio; the rest of the portfolio runs only if the best so
//      far is infeasible;
//   3. projects the best bipartition up the item's hierarchy and runs 2-way FM
//      (one warp) on every level.
// Scratch comes from a per-item region through a bump allocator; if a region
// is too small the launch reports it and the host repeats the round with
// larger regions, so results never depend on scratch sizes.
#include <algorithm>
#include <cmath>
#include <numeric>

#include "kmp_internal.cuh"
#include "kmp_mpnn.cuh"

namespace kmp {

constexpr int IPT = 256;
constexpr int IPW = IPT / 32;
constexpr int IP_WTAB = 512;       // per-warp shared table: degree <= 256
constexpr int IP_MAXL = 63;
constexpr int32_t IP_MAX_N = 65535;
// dynamic shared memory per bipartitioner CTA, at most (words): 184 KB, which
// with the kernel's 40 KB of static shared memory stays within the 227 KB a
// CTA may use
constexpr int32_t IP_DYN_MAX_WORDS = 46000;
constexpr int32_t IP_DYN_SHARED_WORDS = 18000;  // 72 KB: two CTAs per SM

struct ItemDesc {
  int64_t vbase;  // first member position
  int64_t ebase;  // first induced edge
  int64_t sbase;  // scratch region (int32 units)
  int64_t ssize;
  uint64_t key;
  int32_t n, m;
  int32_t t0, t1, L0, L1;
  int32_t pad0, pad1;
};

struct IPArgs {
  const ItemDesc *items;
  const int32_t *order;   // item processing order
  int32_t nitems;
  int32_t *queue;         // work counter
  int32_t *oom;           // set when a scratch region was too small
  const int64_t *gx;      // induced CSR offsets over all members (n+1)
  const int32_t *sadj;    // local neighbour ids
  const int32_t *sew;
  const int32_t *svw;
  int32_t *side_out;      // per member position
  int32_t *scratch;
  // configuration
  int32_t S, ip_C, ip_lp_rounds, rep_random, rep_bfs, rep_ggg, fm_passes, fm_stop;
  int32_t conv_num, conv_den;
  // learned mode: proposer weights (null: plain portfolio) and reduced repetitions
  const __nv_bfloat16 *W;
  int32_t lrep_random, lrep_bfs, lrep_ggg;
  int32_t adaptive;  // adaptive portfolio (plain mode only)
  int32_t learned_item;  // learned item mode (W set): start on the item graph, FM there
  SampleSink sink;  // counters null: no recording
  int32_t dyn_words;  // dynamic shared memory per CTA (int32 words) for FM and portfolio state
};

struct LG {
  int32_t n, m;
  int32_t *xadj, *adj, *ew, *vw;
  int32_t maxdeg, maxc;
};

struct Bump {
  int32_t *base;
  int64_t cap, top;
  bool oom;
  __device__ int32_t *take(int64_t cnt) {
    int64_t t = (top + 1) & ~1ll;
    if (oom || t + cnt > cap) {
      oom = true;
      return base;  // never dereferenced: callers check oom
    }
    top = t + cnt;
    return base + t;
  }
};

// ------------------------------------------------------- block helpers
__device__ int64_t block_sum64(int64_t v) {
  __shared__ int64_t red[IPW];
  v = warp_sum64(v);
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  int64_t s = 0;
  for (int i = 0; i < IPW; ++i) s += red[i];
  __syncthreads();
  return s;
}

__device__ int32_t block_max32(int32_t v) {
  __shared__ int32_t red[IPW];
#pragma unroll
  for (int m = 16; m > 0; m >>= 1) v = max(v, __shfl_xor_sync(0xFFFFFFFFu, v, m));
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  int32_t s = red[0];
  for (int i = 1; i < IPW; ++i) s = max(s, red[i]);
  __syncthreads();
  return s;
}

// exclusive scan of in[0..n) into out (may alias), returns total
template <class T>
__device__ T block_scan_excl(const T *in, T *out, int32_t n) {
  __shared__ T wsum[IPW];
  __shared__ T carry;
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int32_t base = 0; base < n; base += IPT) {
    int32_t i = base + threadIdx.x;
    T v = i < n ? in[i] : T(0);
    T x = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      T y = __shfl_up_sync(0xFFFFFFFFu, x, d);
      if (lane >= d) x += y;
    }
    if (lane == 31) wsum[w] = x;
    __syncthreads();
    T pre = carry;
    for (int k = 0; k < w; ++k) pre += wsum[k];
    T tot = 0;
    for (int k = 0; k < IPW; ++k) tot += wsum[k];
    if (i < n) out[i] = pre + x - v;
    __syncthreads();
    if (threadIdx.x == 0) carry += tot;
    __syncthreads();
  }
  T r = carry;
  __syncthreads();
  return r;
}

// bitonic sort of P (power of two) keys ascending, optional values; block-wide
__device__ void block_bitonic(uint64_t *key, int32_t *val, int32_t P) {
  for (int32_t k = 2; k <= P; k <<= 1)
    for (int32_t j = k >> 1; j > 0; j >>= 1) {
      for (int32_t i = threadIdx.x; i < P; i += IPT) {
        int32_t l = i ^ j;
        if (l > i) {
          uint64_t x = key[i], y = key[l];
          bool up = (i & k) == 0;
          if ((x > y) == up) {
            key[i] = y;
            key[l] = x;
            if (val) {
              int32_t t = val[i];
              val[i] = val[l];
              val[l] = t;
            }
          }
        }
      }
      __syncthreads();
    }
}

// warp bitonic of P pairs (h, v) ascending by (h, v)
__device__ void warp_bitonic_hv(uint64_t *h, int32_t *v, int32_t P) {
  int lane = threadIdx.x & 31;
  for (int32_t k = 2; k <= P; k <<= 1)
    for (int32_t j = k >> 1; j > 0; j >>= 1) {
      for (int32_t i = lane; i < P; i += 32) {
        int32_t l = i ^ j;
        if (l > i) {
          uint64_t a = h[i], b = h[l];
          int32_t va = v[i], vb = v[l];
          bool gt = a > b || (a == b && va > vb);
          bool up = (i & k) == 0;
          if (gt == up) {
            h[i] = b; h[l] = a;
            v[i] = vb; v[l] = va;
          }
        }
      }
      __syncwarp();
    }
}

// warp bitonic of P (power of two) 64-bit keys ascending
__device__ void warp_bitonic_u64(uint64_t *a, int32_t P) {
  int lane = threadIdx.x & 31;
  for (int32_t k = 2; k <= P; k <<= 1)
    for (int32_t j = k >> 1; j > 0; j >>= 1) {
      for (int32_t i = lane; i < P; i += 32) {
        int32_t l = i ^ j;
        if (l > i) {
          uint64_t x = a[i], y = a[l];
          if ((x > y) == ((i & k) == 0)) {
            a[i] = y;
            a[l] = x;
          }
        }
      }
      __syncwarp();
    }
}

__device__ __forceinline__ int32_t pow2_at_least(int32_t x) {
  int32_t p = 1;
  while (p < x) p <<= 1;
  return p;
}

// ------------------------------------------------------ item clustering
// rating of node u by one warp; returns (via lane 0) proposal target or -1
__device__ void item_rate(const LG &g, int32_t u, const int32_t *label, const int32_t *wt, int32_t U,
                          uint32_t rk_hi, int32_t *skeys, int32_t *svals, int32_t *gkeys,
                          int32_t *gvals, int32_t *out_t, int32_t *out_g) {
  int lane = threadIdx.x & 31;
  int32_t b = g.xadj[u], e = g.xadj[u + 1], deg = e - b;
  uint32_t cap = 32;
  while ((int64_t)cap < 2ll * deg) cap <<= 1;
  uint32_t mask = cap - 1;
  // shared-memory table unless this node's table does not fit there
  int32_t *keys = cap <= (uint32_t)IP_WTAB ? skeys : gkeys;
  int32_t *vals = cap <= (uint32_t)IP_WTAB ? svals : gvals;
  for (uint32_t i = lane; i < cap; i += 32) {
    keys[i] = HT_EMPTY;
    vals[i] = 0;
  }
  __syncwarp();
  for (int32_t q = b + lane; q < e; q += 32) ht_add(keys, vals, mask, label[g.adj[q]], g.ew[q]);
  __syncwarp();
  int32_t own = label[u], cu = g.vw[u];
  int32_t rown = ht_get(keys, vals, mask, own);
  uint64_t kc = 0;
  int32_t lc = -1;
  for (uint32_t i = lane; i < cap; i += 32) {
    int32_t K = keys[i];
    if (K == HT_EMPTY || K == own) continue;
    if ((int64_t)wt[K] + cu > U) continue;
    uint64_t k = ((uint64_t)(uint32_t)vals[i] << 32) | (uint64_t)(0xFFFFFFFFu - perm32(rk_hi, K));
    if (k > kc) { kc = k; lc = K; }
  }
  uint64_t mc = group_max64<32>(kc);
  unsigned bc = __ballot_sync(0xFFFFFFFFu, mc != 0 && kc == mc);
  lc = __shfl_sync(0xFFFFFFFFu, lc, bc ? __ffs(bc) - 1 : 0);
  if (lane == 0) {
    int32_t rc = (int32_t)(mc >> 32);
    if (mc != 0 && rc > rown) {
      *out_t = lc;
      *out_g = rc - rown;
    } else {
      *out_t = -1;
    }
  }
  __syncwarp();
}

// rating of 32 / G nodes by one warp, G lanes per node (degree <= G, one
// neighbour per lane; u < 0: no node): lanes of a group holding the same
// label form a peer set whose weight sum is that label's rating.  Same
// decision as item_rate.
// loads of one group node: neighbour label and edge weight of this lane,
// own label and node weight (u < 0: no node)
struct GroupIn {
  int32_t l, x, own, cu;
};
template <int G>
__device__ __forceinline__ GroupIn item_group_load(const LG &g, int32_t u, const int32_t *label) {
  const int gl = (threadIdx.x & 31) & (G - 1);
  GroupIn r{-1, 0, -1, 0};
  if (u >= 0) {
    int32_t b = g.xadj[u], deg = g.xadj[u + 1] - b;
    r.own = label[u];
    r.cu = g.vw[u];
    if (gl < deg) {
      r.l = label[g.adj[b + gl]];
      r.x = g.ew[b + gl];
    }
  }
  return r;
}

// rating of 32 / G nodes by one warp, G lanes per node (degree <= G, one
// neighbour per lane): lanes of a group holding the same label form a peer
// set whose weight sum is that label's rating.  Same decision as item_rate.
template <int G>
__device__ __forceinline__ void item_group_rate(const GroupIn &in, int32_t u, const int32_t *wt, int32_t U,
                                                uint32_t rk_hi, int32_t *pt, int32_t *pg) {
  const int lane = threadIdx.x & 31, gl = lane & (G - 1);
  const unsigned gmask = (G == 32) ? 0xFFFFFFFFu : (((1u << G) - 1u) << (lane & ~(G - 1)));
  const int32_t l = in.l;
  unsigned peers = __match_any_sync(0xFFFFFFFFu, ((uint64_t)(uint32_t)(lane / G) << 32) | (uint32_t)l);
  int32_t r = __reduce_add_sync(peers, in.x);
  unsigned bown = __ballot_sync(0xFFFFFFFFu, l >= 0 && l == in.own) & gmask;
  int32_t rown = __shfl_sync(0xFFFFFFFFu, r, bown ? __ffs(bown) - 1 : lane);
  if (!bown) rown = 0;
  bool adm = l >= 0 && l != in.own && (int64_t)wt[l] + in.cu <= U;
  uint64_t k = adm ? ((uint64_t)(uint32_t)r << 32) | (uint64_t)(0xFFFFFFFFu - perm32(rk_hi, l)) : 0ull;
  uint64_t mc = group_max64<G>(k);
  unsigned bc = __ballot_sync(0xFFFFFFFFu, mc != 0 && k == mc) & gmask;
  int32_t lc = __shfl_sync(0xFFFFFFFFu, l, bc ? __ffs(bc) - 1 : lane);
  if (gl == 0 && u >= 0) {
    int32_t rc = (int32_t)(mc >> 32);
    if (mc != 0 && rc > rown) {
      pt[u] = lc;
      pg[u] = rc - rown;
    } else {
      pt[u] = -1;
    }
  }
}

// the nodes sl[lo..hi) rated 32 / G per warp step
template <int G>
__device__ __forceinline__ void item_rate_groups(const LG &g, const int32_t *sl, int32_t lo, int32_t hi,
                                                 const int32_t *label, const int32_t *wt, int32_t U,
                                                 uint32_t rk_hi, int32_t *pt, int32_t *pg) {
  constexpr int per = 32 / G;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int32_t i0 = lo + per * w; i0 < hi; i0 += per * IPW) {
    int32_t i = i0 + lane / G;
    int32_t u = i < hi ? sl[i] : -1;
    GroupIn a = item_group_load<G>(g, u, label);
    item_group_rate<G>(a, u, wt, U, rk_hi, pt, pg);
  }
}

// degree class of a node for the item rating schedule: 0 (<= 16, two nodes
// per warp), 1 (<= 32, one node per warp, no table), 2 (table)
__device__ __forceinline__ int32_t item_deg_class(int32_t deg) { return deg <= 16 ? 0 : (deg <= 32 ? 1 : 2); }

// segmented inclusive scan in shared memory (one element per thread)
__device__ int64_t block_seg_scan(int64_t x, bool head) {
  __shared__ int64_t sv[IPT];
  __shared__ int32_t sf[IPT];
  int t = threadIdx.x;
  sv[t] = x;
  sf[t] = head ? 1 : 0;
  __syncthreads();
  for (int d = 1; d < IPT; d <<= 1) {
    int64_t v = sv[t];
    int32_t f = sf[t];
    if (t >= d && !f) {
      v += sv[t - d];
      f |= sf[t - d];
    }
    __syncthreads();
    sv[t] = v;
    sf[t] = f;
    __syncthreads();
  }
  int64_t r = sv[t];
  __syncthreads();
  return r;
}

// LP clustering of one item level + isolated packing; returns #clusters
__device__ int32_t item_cluster(const IPArgs &A, const LG &g, int32_t U, uint64_t basekey,
                                int32_t *label, Bump &B, int32_t *wkeys, int32_t *wvals, int32_t *dyn,
                                int32_t dyn_words) {
  __shared__ int32_t s_cnt, s_fast;
  __shared__ int32_t s_moved;
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int32_t n = g.n;
  int64_t mark = B.top;
  int32_t P = pow2_at_least(n > 1 ? n : 2);
  // working arrays: in shared memory when the level fits (every phase of a
  // sub-round reads them), else in the item's scratch; labels are written
  // to `label` at the end either way.  The sort space of contested proposals
  // sits in shared memory behind them when a sub-round's proposals fit
  // there, else in the scratch (pl_g, always reserved).
  int32_t *lab, *wt, *pt, *pg, *sl, *fl, *tsum;
  uint8_t *act, *act2;  // active flags
  uint64_t *pl_s = nullptr;
  int32_t pl_cap = 0;   // entries of pl_s
  uint64_t *pl_g = reinterpret_cast<uint64_t *>(B.take(2ll * P));
  const int64_t flag_words = (n + 3) / 4;
  const bool fast = 7ll * n + 2 * flag_words + 2 + 128 <= dyn_words;
  if (fast) {
    int32_t *q = dyn;
    lab = q; q += n;
    wt = q; q += n;
    pt = q; q += n;
    pg = q; q += n;
    sl = q; q += n;
    fl = q; q += n;
    tsum = q; q += n;
    act = reinterpret_cast<uint8_t *>(q); q += flag_words;
    act2 = reinterpret_cast<uint8_t *>(q); q += flag_words;
    q += (q - dyn) & 1;  // 8-byte alignment
    pl_s = reinterpret_cast<uint64_t *>(q);
    pl_cap = (int32_t)((dyn_words - (q - dyn)) / 2);
  } else {
    lab = label;
    wt = B.take(n);
    act = reinterpret_cast<uint8_t *>(B.take(flag_words));
    act2 = reinterpret_cast<uint8_t *>(B.take(flag_words));
    pt = B.take(n);
    pg = B.take(n);
    sl = B.take(n);    // the round's nodes by sub-round
    fl = B.take(n);    // accepted proposals of uncontested targets
    tsum = B.take(n);  // proposed weight per target (kept zero between uses)
  }
  int32_t *gtab = nullptr;
  uint32_t gcap = 0;
  if (g.maxdeg > IP_WTAB / 2) {
    gcap = 32;
    while ((int64_t)gcap < 2ll * g.maxdeg) gcap <<= 1;
    gtab = B.take(2ll * gcap * IPW);
  }
  if (B.oom) return -1;
  for (int32_t v = threadIdx.x; v < n; v += IPT) {
    lab[v] = v;
    wt[v] = g.vw[v];
    act[v] = 1;
    tsum[v] = 0;
  }
  __syncthreads();
  int32_t *mk = wkeys + w * IP_WTAB, *mv = wvals + w * IP_WTAB;
  int32_t *gk = nullptr, *gv = nullptr;
  if (gtab) {
    gk = gtab + (int64_t)w * 2 * gcap;
    gv = gk + gcap;
  }
  for (int32_t r = 0; r < A.ip_lp_rounds; ++r) {
    uint64_t rk = key_step(basekey, (uint64_t)r);
    uint32_t rk_hi = (uint32_t)(rk >> 32);
    // the round's active nodes (with edges) bucketed by sub-round and, inside
    // a sub-round, by degree class (the rating schedule; any order inside a
    // sub-round gives the same result)
    __shared__ int32_t s_soff[3 * 8 + 1], s_fill[3 * 8];
    if (threadIdx.x < 3 * 8) s_fill[threadIdx.x] = 0;
    if (threadIdx.x == 0) s_moved = 0;
    __syncthreads();
    for (int32_t v = threadIdx.x; v < n; v += IPT) {
      act2[v] = 0;
      int32_t d = g.xadj[v + 1] - g.xadj[v];
      if (act[v] && d > 0)
        atomicAdd(&s_fill[3 * (int32_t)(key_step(rk, (uint64_t)(uint32_t)v) & (uint64_t)(A.S - 1)) +
                          item_deg_class(d)],
                  1);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      s_soff[0] = 0;
      for (int32_t x = 0; x < 3 * A.S; ++x) {
        s_soff[x + 1] = s_soff[x] + s_fill[x];
        s_fill[x] = 0;
      }
    }
    __syncthreads();
    for (int32_t v = threadIdx.x; v < n; v += IPT) {
      int32_t d = g.xadj[v + 1] - g.xadj[v];
      if (act[v] && d > 0) {
        int32_t x = 3 * (int32_t)(key_step(rk, (uint64_t)(uint32_t)v) & (uint64_t)(A.S - 1)) + item_deg_class(d);
        sl[s_soff[x] + atomicAdd(&s_fill[x], 1)] = v;
      }
    }
    __syncthreads();
    for (int32_t s = 0; s < A.S; ++s) {
      const int32_t lo = s_soff[3 * s], hi = s_soff[3 * s + 3];
      const int32_t m1 = s_soff[3 * s + 1], m2 = s_soff[3 * s + 2];
      // contested proposals are at most the sub-round's nodes
      uint64_t *pl = pow2_at_least(hi - lo > 1 ? hi - lo : 2) <= pl_cap ? pl_s : pl_g;
      // rating: two nodes per warp, then one per warp without a table, then
      // one per warp with a table
      item_rate_groups<16>(g, sl, lo, m1, lab, wt, U, rk_hi, pt, pg);
      item_rate_groups<32>(g, sl, m1, m2, lab, wt, U, rk_hi, pt, pg);
      for (int32_t i = m2 + w; i < hi; i += IPW) {
        int32_t u = sl[i];
        item_rate(g, u, lab, wt, U, rk_hi, mk, mv, gk, gv, &pt[u], &pg[u]);
      }
      if (threadIdx.x == 0) {
        s_cnt = 0;
        s_fast = 0;
      }
      __syncthreads();
      // proposed weight per target
      for (int32_t i = lo + threadIdx.x; i < hi; i += IPT) {
        int32_t u = sl[i], T = pt[u];
        if (T >= 0) atomicAdd(&tsum[T], g.vw[u]);
      }
      __syncthreads();
      // a target whose proposals all fit takes them all; only the proposals
      // of contested targets need the (target, gain desc, node) order
      for (int32_t i = lo + threadIdx.x; i < hi; i += IPT) {
        int32_t u = sl[i], T = pt[u];
        if (T < 0) continue;
        if ((int64_t)wt[T] + tsum[T] <= U) {
          fl[atomicAdd(&s_fast, 1)] = u;
        } else {
          int32_t p = atomicAdd(&s_cnt, 1);
          pl[p] = ((uint64_t)(uint32_t)T << 47) | ((uint64_t)(uint32_t)(0x7FFFFFFF - pg[u]) << 16) |
                  (uint64_t)(uint32_t)u;
        }
      }
      __syncthreads();
      for (int32_t i = lo + threadIdx.x; i < hi; i += IPT) {
        int32_t T = pt[sl[i]];
        if (T >= 0) tsum[T] = 0;  // every reader is past the barrier above
      }
      int32_t np = s_cnt, nf = s_fast;
      if (np > 0) {
        int32_t Pp = pow2_at_least(np);
        for (int32_t i = np + threadIdx.x; i < Pp; i += IPT) pl[i] = ~0ull;
        __syncthreads();
        block_bitonic(pl, nullptr, Pp);
        // accepted prefix per target: start weight + segmented prefix <= U
        __shared__ int64_t carry;
        __shared__ int32_t carryT;
        if (threadIdx.x == 0) { carry = 0; carryT = -1; }
        __syncthreads();
        for (int32_t base = 0; base < np; base += IPT) {
          int32_t i = base + threadIdx.x;
          bool ok = i < np;
          uint64_t k = ok ? pl[i] : 0;
          int32_t T = ok ? (int32_t)(k >> 47) : -1;
          int32_t u = ok ? (int32_t)(k & 0xFFFF) : 0;
          // only threads holding a proposal look at their predecessor (i - 1 < np)
          int32_t Tprev = (!ok || i == 0) ? -1 : (int32_t)((pl[i - 1] >> 47) & 0xFFFF);
          bool head = !ok || i == 0 || T != Tprev;
          int64_t c = ok ? g.vw[u] : 0;
          int64_t pre = block_seg_scan(c, head || threadIdx.x == 0);
          // the chunk's first segment continues the previous chunk's last one
          bool cont = ok && base > 0 && T == carryT;
          __shared__ int32_t firsthead;
          if (threadIdx.x == 0) firsthead = IPT;
          __syncthreads();
          if (ok && threadIdx.x > 0 && head) atomicMin(&firsthead, (int32_t)threadIdx.x);
          __syncthreads();
          if (cont && (int32_t)threadIdx.x < firsthead) pre += carry;
          if (ok) {
            bool acc = (int64_t)wt[T] + pre <= U;
            if (acc) pl[i] = k | (1ull << 63);
          }
          __syncthreads();
          int32_t last = min(IPT, np - base) - 1;
          if ((int32_t)threadIdx.x == last) {
            carry = pre;
            carryT = T;
          }
          __syncthreads();
        }
      }
      // apply: one warp per accepted move; lane 0 moves the node, the lanes
      // mark its neighbours active for the next round
      int32_t mv_local = 0;
      for (int32_t i = w; i < nf + np; i += IPW) {
        int32_t u, T;
        if (i < nf) {
          u = fl[i];
          T = pt[u];
        } else {
          uint64_t k = pl[i - nf];
          if (!(k >> 63)) continue;
          T = (int32_t)((k >> 47) & 0xFFFF);
          u = (int32_t)(k & 0xFFFF);
        }
        if (lane == 0) {
          int32_t own = lab[u], c = g.vw[u];
          lab[u] = T;
          atomicAdd(&wt[T], c);
          atomicSub(&wt[own], c);
          ++mv_local;
        }
        for (int32_t q = g.xadj[u] + lane; q < g.xadj[u + 1]; q += 32) act2[g.adj[q]] = 1;
      }
      if (mv_local) atomicAdd(&s_moved, mv_local);
      __syncthreads();
    }
    int32_t moved = s_moved;
    uint8_t *t = act;
    act = act2;
    act2 = t;
    __syncthreads();
    if (moved == 0) break;
  }
  // isolated packing in id order
  int32_t *iw = pg;  // reuse: weights of isolated nodes, then prefix
  for (int32_t v = threadIdx.x; v < n; v += IPT) iw[v] = (g.xadj[v + 1] == g.xadj[v]) ? g.vw[v] : 0;
  __syncthreads();
  block_scan_excl<int32_t>(iw, iw, n);
  int32_t *first = sl;
  for (int32_t v = threadIdx.x; v < n; v += IPT) first[v] = INT32_MAX;
  __syncthreads();
  for (int32_t v = threadIdx.x; v < n; v += IPT) {
    if (g.xadj[v + 1] != g.xadj[v]) continue;
    int64_t P0 = iw[v], c = g.vw[v];
    int64_t q = P0 / U, qe = (P0 + c - 1) / U;
    if (q == qe) atomicMin(&first[q], lab[v]);
  }
  __syncthreads();
  for (int32_t v = threadIdx.x; v < n; v += IPT) {
    if (g.xadj[v + 1] != g.xadj[v]) continue;
    int64_t P0 = iw[v], c = g.vw[v];
    int64_t q = P0 / U, qe = (P0 + c - 1) / U;
    if (q == qe) lab[v] = first[q];
  }
  __syncthreads();
  // count clusters
  int32_t *used = pt;
  for (int32_t v = threadIdx.x; v < n; v += IPT) used[v] = 0;
  __syncthreads();
  for (int32_t v = threadIdx.x; v < n; v += IPT) used[lab[v]] = 1;
  __syncthreads();
  int64_t c = 0;
  for (int32_t v = threadIdx.x; v < n; v += IPT) c += used[v];
  int32_t nc = (int32_t)block_sum64(c);
  if (fast) {
    for (int32_t v = threadIdx.x; v < n; v += IPT) label[v] = lab[v];
    __syncthreads();
  }
  B.top = mark;
  return nc;
}

// contraction of one item level; fills *out (arrays allocated from B)
__device__ void item_contract(const LG &g, const int32_t *label, int32_t *map, LG *out, Bump &B,
                              int32_t *wkeys, int32_t *wvals) {
  int32_t n = g.n;
  int32_t *cid = B.take(n + 1);
  if (B.oom) return;
  for (int32_t v = threadIdx.x; v < n; v += IPT) cid[v] = 0;
  __syncthreads();
  for (int32_t v = threadIdx.x; v < n; v += IPT) cid[label[v]] = 1;
  __syncthreads();
  int32_t nc = block_scan_excl<int32_t>(cid, cid, n);
  for (int32_t v = threadIdx.x; v < n; v += IPT) map[v] = cid[label[v]];
  __syncthreads();
  // coarse arrays (kept); rows hold at most the cross entries of the level
  int32_t *cvw = B.take(nc);
  int32_t *cx = B.take(nc + 1);
  int64_t cnt = 0;
  for (int32_t v = threadIdx.x; v < n; v += IPT)
    for (int32_t q = g.xadj[v]; q < g.xadj[v + 1]; ++q) cnt += (map[v] != map[g.adj[q]]);
  int32_t np = (int32_t)block_sum64(cnt);
  int32_t *cadj = B.take(np);
  int32_t *cew = B.take(np);
  int64_t mark = B.top;
  // members grouped by coarse node; members' total degree per coarse node
  int32_t *moff = B.take(nc + 1), *mcur = B.take(nc), *members = B.take(n);
  int32_t *ub = B.take(nc + 1), *toff = B.take(nc + 1), *rowlen = B.take(nc + 1);
  int32_t *tadj = B.take(g.m > 0 ? g.m : 1), *tw = B.take(g.m > 0 ? g.m : 1);
  if (B.oom) return;
  for (int32_t x = threadIdx.x; x <= nc; x += IPT) {
    if (x < nc) {
      cvw[x] = 0;
      mcur[x] = 0;
    }
    moff[x] = 0;
    ub[x] = 0;
  }
  __syncthreads();
  for (int32_t v = threadIdx.x; v < n; v += IPT) {
    int32_t x = map[v];
    atomicAdd(&cvw[x], g.vw[v]);
    atomicAdd(&moff[x], 1);
    atomicAdd(&ub[x], g.xadj[v + 1] - g.xadj[v]);
  }
  __syncthreads();
  block_scan_excl<int32_t>(moff, moff, nc + 1);
  int32_t maxub = 0;
  for (int32_t x = threadIdx.x; x < nc; x += IPT) maxub = max(maxub, ub[x]);
  maxub = block_max32(maxub);
  block_scan_excl<int32_t>(ub, toff, nc + 1);
  for (int32_t v = threadIdx.x; v < n; v += IPT) {
    int32_t x = map[v];
    members[moff[x] + atomicAdd(&mcur[x], 1)] = v;
  }
  // per-warp global table and sort list for rows that do not fit shared memory
  int32_t dmax = maxub < nc ? maxub : nc;
  int32_t gcap = 32;
  while (gcap < 2 * dmax) gcap <<= 1;
  int32_t lcap = pow2_at_least(dmax > 1 ? dmax : 2);
  int32_t *gtab = gcap > IP_WTAB ? B.take(2ll * gcap * IPW) : nullptr;
  uint64_t *lbuf = reinterpret_cast<uint64_t *>(B.take(2ll * lcap * IPW));
  __syncthreads();
  if (B.oom) return;
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint64_t *L = lbuf + (int64_t)w * lcap;
  // one warp per coarse node: aggregate, compact, sort by neighbour, write the row
  for (int32_t x = w; x < nc; x += IPW) {
    int32_t d = ub[x] < nc ? ub[x] : nc;
    uint32_t cap = 32;
    while ((int32_t)cap < 2 * d) cap <<= 1;
    int32_t *K = cap <= (uint32_t)IP_WTAB ? wkeys + w * IP_WTAB : gtab + (int64_t)w * 2 * gcap;
    int32_t *V = cap <= (uint32_t)IP_WTAB ? wvals + w * IP_WTAB : K + gcap;
    for (uint32_t i = lane; i < cap; i += 32) {
      K[i] = HT_EMPTY;
      V[i] = 0;
    }
    __syncwarp();
    // up to 32 members at a time spread their edges over the lanes: a warp
    // prefix of their degrees, and each lane finds the member of its edge
    for (int32_t c0 = moff[x]; c0 < moff[x + 1]; c0 += 32) {
      int32_t d = 0, b = 0;
      if (c0 + lane < moff[x + 1]) {
        int32_t v = members[c0 + lane];
        b = g.xadj[v];
        d = g.xadj[v + 1] - b;
      }
      int32_t inc = d;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        int32_t t = __shfl_up_sync(0xFFFFFFFFu, inc, o);
        if (lane >= o) inc += t;
      }
      const int32_t tot = __shfl_sync(0xFFFFFFFFu, inc, 31);
      for (int32_t e0 = 0; e0 < tot; e0 += 32) {
        const int32_t e = e0 + lane;
        int32_t j = 0;  // members before the owner of edge e
#pragma unroll
        for (int st = 16; st > 0; st >>= 1) {
          int32_t t = __shfl_sync(0xFFFFFFFFu, inc, j + st - 1);
          if (t <= e) j += st;
        }
        int32_t bj = __shfl_sync(0xFFFFFFFFu, b, j & 31);
        int32_t ej = __shfl_sync(0xFFFFFFFFu, inc - d, j & 31);
        if (e < tot) {
          int32_t q = bj + (e - ej);
          int32_t y = map[g.adj[q]];
          if (y != x) ht_add(K, V, cap - 1, y, g.ew[q]);
        }
      }
    }
    __syncwarp();
    int32_t c = 0;
    for (uint32_t i0 = 0; i0 < cap; i0 += 32) {
      uint32_t i = i0 + lane;
      bool has = K[i] != HT_EMPTY;
      unsigned bal = __ballot_sync(0xFFFFFFFFu, has);
      if (has) L[c + __popc(bal & ((1u << lane) - 1u))] = ((uint64_t)(uint32_t)K[i] << 32) | (uint32_t)V[i];
      c += __popc(bal);
    }
    int32_t P = pow2_at_least(c > 1 ? c : 2);
    for (int32_t i = c + lane; i < P; i += 32) L[i] = ~0ull;
    __syncwarp();
    warp_bitonic_u64(L, P);
    for (int32_t i = lane; i < c; i += 32) {
      tadj[toff[x] + i] = (int32_t)(L[i] >> 32);
      tw[toff[x] + i] = (int32_t)(uint32_t)L[i];
    }
    if (lane == 0) rowlen[x] = c;
    __syncwarp();
  }
  __syncthreads();
  if (threadIdx.x == 0) rowlen[nc] = 0;
  __syncthreads();
  int32_t m2 = block_scan_excl<int32_t>(rowlen, cx, nc + 1);
  for (int32_t x = w; x < nc; x += IPW)
    for (int32_t i = lane; i < cx[x + 1] - cx[x]; i += 32) {
      cadj[cx[x] + i] = tadj[toff[x] + i];
      cew[cx[x] + i] = tw[toff[x] + i];
    }
  __syncthreads();
  B.top = mark;
  out->n = nc;
  out->m = m2;
  out->xadj = cx;
  out->adj = cadj;
  out->ew = cew;
  out->vw = cvw;
  __syncthreads();
}

// ------------------------------------------------------------ warp FM
// FM state: gains, locks, the move log, and per side the selection key of
// every node of that side that may still move (0 otherwise), so that finding
// the top of a side is a branch-free max over one array
struct FMBuf {
  int32_t *gain, *locked, *moves;
  uint64_t *key0, *key1;
};

__device__ __forceinline__ uint64_t fm_key(int32_t gain, int32_t v) {
  return ((uint64_t)((uint32_t)gain ^ 0x80000000u) << 32) | (0xFFFFFFFFu - (uint32_t)v);
}

__device__ __forceinline__ bool fm_less(int32_t ia, int64_t oa, int64_t ca, int32_t ib, int64_t ob,
                                        int64_t cb) {
  if (ia != ib) return ia < ib;
  if (oa != ob) return oa < ob;
  return ca < cb;
}

// 2-way FM by one warp (same decisions as the oracle); returns the final cut
// the moves of one FM pass by one warp, from gains and locks already set:
// repeatedly the better feasible top of the two sides (gain desc, id asc),
// until no unlocked node is left or fm_stop moves bring no new best; then
// the pass is rolled back to its best prefix.  Returns the kept moves (0: the
// pass found nothing better) and updates cut.
__device__ int32_t fm_pass_moves(const IPArgs &A, const LG &g, int32_t *side, int64_t L0, int64_t L1,
                                 FMBuf fb, int64_t W0, int64_t W1, int64_t &cut) {
  int lane = threadIdx.x & 31;
  int32_t n = g.n;
  auto mk = [&](int32_t &inf, int64_t &ov) {
    int64_t o0 = W0 - L0, o1 = W1 - L1;
    int64_t o = o0 > o1 ? o0 : o1;
    inf = o > 0;
    ov = inf ? o : 0;
  };
  int32_t binf;
  int64_t bov;
  mk(binf, bov);
  int64_t bcut = cut;
  int32_t best_step = 0, nsteps = 0;
  for (;;) {
    uint64_t t0 = 0, t1 = 0;  // (gain biased, ~id): larger is better; 0 = none
#pragma unroll 4
    for (int32_t v = lane; v < n; v += 32) {
      uint64_t a = fb.key0[v], b = fb.key1[v];
      t0 = a > t0 ? a : t0;
      t1 = b > t1 ? b : t1;
    }
    t0 = group_max64<32>(t0);
    t1 = group_max64<32>(t1);
    if (t0 == 0 && t1 == 0) break;
    int32_t v0 = t0 ? (int32_t)(0xFFFFFFFFu - (uint32_t)t0) : -1;
    int32_t v1 = t1 ? (int32_t)(0xFFFFFFFFu - (uint32_t)t1) : -1;
    // both candidates' weights and row bounds in one round of loads
    int32_t c0 = 0, c1 = 0, b0 = 0, e0 = 0, b1 = 0, e1 = 0;
    if (v0 >= 0) {
      c0 = g.vw[v0];
      b0 = g.xadj[v0];
      e0 = g.xadj[v0 + 1];
    }
    if (v1 >= 0) {
      c1 = g.vw[v1];
      b1 = g.xadj[v1];
      e1 = g.xadj[v1 + 1];
    }
    bool f0 = v0 >= 0 && W1 + c0 <= L1;
    bool f1 = v1 >= 0 && W0 + c1 <= L0;
    int32_t v;
    if (f0 && f1) v = (t0 > t1) ? v0 : v1;
    else if (f0) v = v0;
    else if (f1) v = v1;
    else {
      if (lane == 0) {
        if (v0 >= 0) {
          fb.locked[v0] = 1;
          fb.key0[v0] = 0;
        }
        if (v1 >= 0) {
          fb.locked[v1] = 1;
          fb.key1[v1] = 0;
        }
      }
      __syncwarp();
      continue;
    }
    int32_t from = side[v], to = 1 - from;
    int32_t gv = fb.gain[v];
    __syncwarp();
    if (lane == 0) {
      side[v] = to;
      fb.locked[v] = 1;
      fb.key0[v] = 0;
      fb.key1[v] = 0;
    }
    const bool is0 = v == v0;
    int32_t c = is0 ? c0 : c1;
    if (from == 0) { W0 -= c; W1 += c; } else { W1 -= c; W0 += c; }
    cut -= gv;
    const int32_t qe = is0 ? e0 : e1;
    for (int32_t q = (is0 ? b0 : b1) + lane; q < qe; q += 32) {
      int32_t x = g.adj[q];
      int32_t sx = side[x];
      int32_t gx = fb.gain[x] + (sx == to ? -2 * g.ew[q] : 2 * g.ew[q]);
      fb.gain[x] = gx;
      if (!fb.locked[x]) {
        if (sx == 0) fb.key0[x] = fm_key(gx, x);
        else fb.key1[x] = fm_key(gx, x);
      }
    }
    __syncwarp();
    if (lane == 0) {
      fb.gain[v] = -gv;
      fb.moves[nsteps] = v;
    }
    ++nsteps;
    __syncwarp();
    int32_t inf;
    int64_t ov;
    mk(inf, ov);
    if (fm_less(inf, ov, cut, binf, bov, bcut)) {
      binf = inf;
      bov = ov;
      bcut = cut;
      best_step = nsteps;
    }
    if (nsteps - best_step >= A.fm_stop) break;
  }
  for (int32_t i = best_step + lane; i < nsteps; i += 32) side[fb.moves[i]] ^= 1;
  __syncwarp();
  cut = bcut;
  return best_step;
}

__device__ int64_t warp_fm(const IPArgs &A, const LG &g, int32_t *side, int64_t L0, int64_t L1,
                           FMBuf fb) {
  int lane = threadIdx.x & 31;
  int32_t n = g.n;
  int64_t cut = 0;
  for (int32_t v = lane; v < n; v += 32)
    for (int32_t q = g.xadj[v]; q < g.xadj[v + 1]; ++q)
      if (side[g.adj[q]] != side[v]) cut += g.ew[q];
  cut = warp_sum64(cut) / 2;
  for (int32_t pass = 0; pass < A.fm_passes; ++pass) {
    int64_t W0 = 0, W1 = 0;
    for (int32_t v = lane; v < n; v += 32) {
      if (side[v] == 0) W0 += g.vw[v];
      else W1 += g.vw[v];
      int32_t gsum = 0;
      for (int32_t q = g.xadj[v]; q < g.xadj[v + 1]; ++q)
        gsum += (side[g.adj[q]] != side[v]) ? g.ew[q] : -g.ew[q];
      fb.gain[v] = gsum;
      fb.locked[v] = 0;
      fb.key0[v] = side[v] == 0 ? fm_key(gsum, v) : 0;
      fb.key1[v] = side[v] == 0 ? 0 : fm_key(gsum, v);
    }
    W0 = warp_sum64(W0);
    W1 = warp_sum64(W1);
    __syncwarp();
    if (fm_pass_moves(A, g, side, L0, L1, fb, W0, W1, cut) == 0) break;
  }
  return cut;
}

// the same FM with the whole CTA: cut, gains and weights of every pass by all
// warps (a half-warp per node, its 16 lanes over the row), the moves by warp 0
__device__ int64_t cta_fm(const IPArgs &A, const LG &g, int32_t *side, int64_t L0, int64_t L1, FMBuf fb) {
  __shared__ int64_t s_cut;
  __shared__ int32_t s_kept;
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int hl = lane & 15, hf = lane >> 4;
  int32_t n = g.n;
  int64_t c = 0;
  for (int32_t v = 2 * w + hf; v < n; v += 2 * IPW) {
    int32_t sv = side[v];
    for (int32_t q = g.xadj[v] + hl; q < g.xadj[v + 1]; q += 16)
      if (side[g.adj[q]] != sv) c += g.ew[q];
  }
  int64_t cut = block_sum64(c) / 2;
  for (int32_t pass = 0; pass < A.fm_passes; ++pass) {
    int64_t W0 = 0, W1 = 0;
    for (int32_t v = threadIdx.x; v < n; v += IPT) {
      if (side[v] == 0) W0 += g.vw[v];
      else W1 += g.vw[v];
    }
    for (int32_t v0 = 2 * w; v0 < n; v0 += 2 * IPW) {
      const int32_t v = v0 + hf;
      int32_t sv = 0, gs = 0;
      if (v < n) {
        sv = side[v];
        for (int32_t q = g.xadj[v] + hl; q < g.xadj[v + 1]; q += 16)
          gs += (side[g.adj[q]] != sv) ? g.ew[q] : -g.ew[q];
      }
#pragma unroll
      for (int m = 8; m > 0; m >>= 1) gs += __shfl_xor_sync(0xFFFFFFFFu, gs, m);  // within the half
      if (hl == 0 && v < n) {
        fb.gain[v] = gs;
        fb.locked[v] = 0;
        fb.key0[v] = sv == 0 ? fm_key(gs, v) : 0;
        fb.key1[v] = sv == 0 ? 0 : fm_key(gs, v);
      }
    }
    W0 = block_sum64(W0);  // its barriers also publish the gains
    W1 = block_sum64(W1);
    if (w == 0) {
      int32_t kept = fm_pass_moves(A, g, side, L0, L1, fb, W0, W1, cut);
      if (lane == 0) {
        s_kept = kept;
        s_cut = cut;
      }
    }
    __syncthreads();
    cut = s_cut;
    int32_t kept = s_kept;
    __syncthreads();
    if (kept == 0) break;
  }
  return cut;
}

// portfolio initial bipartition by one warp: algo 0 random, 1 BFS, 2 GGG
// algo 0 random, 1 BFS, 2 greedy graph growing, 3 learned (first fit in the
// order of `score`, like random with a learned order)
__device__ void warp_initial(int algo, const LG &g, int32_t t0, uint64_t key, int32_t *side,
                             uint64_t *oh, int32_t *ov, int32_t *gain, int32_t *vis, int32_t *queue,
                             const float *score) {
  int lane = threadIdx.x & 31;
  int32_t n = g.n;
  int32_t P = pow2_at_least(n > 1 ? n : 2);
  for (int32_t i = lane; i < P; i += 32) {
    if (i < n) {
      oh[i] = algo == 3 ? (uint64_t)mp_score_key(score[i]) : key_step(key, (uint64_t)(uint32_t)i);
      ov[i] = i;
    } else {
      oh[i] = ~0ull;
      ov[i] = INT32_MAX;
    }
  }
  for (int32_t v = lane; v < n; v += 32) side[v] = 1;
  __syncwarp();
  warp_bitonic_hv(oh, ov, P);
  if (algo == 0 || algo == 3) {
    if (lane == 0) {
      int64_t W0 = 0;
      for (int32_t i = 0; i < n; ++i) {
        int32_t v = ov[i];
        if (W0 + g.vw[v] <= t0) {
          side[v] = 0;
          W0 += g.vw[v];
        }
      }
    }
  } else if (algo == 1) {
    for (int32_t v = lane; v < n; v += 32) vis[v] = 0;
    __syncwarp();
    if (lane == 0) {
      int64_t W0 = 0;
      int32_t qh = 0, qt = 0, nr = 0;
      while (qh < n) {
        if (qh == qt) {
          while (vis[ov[nr]]) ++nr;
          vis[ov[nr]] = 1;
          queue[qt++] = ov[nr];
        }
        int32_t v = queue[qh++];
        if (W0 + g.vw[v] <= t0) {
          side[v] = 0;
          W0 += g.vw[v];
        }
        for (int32_t q = g.xadj[v]; q < g.xadj[v + 1]; ++q) {
          int32_t x = g.adj[q];
          if (!vis[x]) {
            vis[x] = 1;
            queue[qt++] = x;
          }
        }
      }
    }
  } else {
    for (int32_t v = lane; v < n; v += 32) {
      int32_t s = 0;
      for (int32_t q = g.xadj[v]; q < g.xadj[v + 1]; ++q) s -= g.ew[q];
      gain[v] = s;
    }
    __syncwarp();
    int64_t W0 = 0;
    int32_t v = (n > 0 && g.vw[ov[0]] <= t0) ? ov[0] : -1;
    for (;;) {
      if (v >= 0) {
        if (lane == 0) side[v] = 0;
        W0 += g.vw[v];
        for (int32_t q = g.xadj[v] + lane; q < g.xadj[v + 1]; q += 32) gain[g.adj[q]] += 2 * g.ew[q];
        __syncwarp();
      }
      uint64_t best = 0;
      for (int32_t x = lane; x < n; x += 32) {
        if (side[x] == 0 || W0 + g.vw[x] > t0) continue;
        uint64_t k = ((uint64_t)((uint32_t)gain[x] ^ 0x80000000u) << 32) | (0xFFFFFFFFu - (uint32_t)x);
        best = k > best ? k : best;
      }
      best = group_max64<32>(best);
      if (best == 0) break;
      v = (int32_t)(0xFFFFFFFFu - (uint32_t)best);
    }
  }
  __syncwarp();
}

__device__ __forceinline__ int32_t level_cap(int32_t L, int32_t t, int32_t maxc) {
  int64_t b = (int64_t)t + maxc;
  return b > L ? (int32_t)b : L;
}

// append the coarsest graph of an item and its winning sides to the sink
// (skipped and counted as dropped when the sink is full)
__device__ void record_sample(const SampleSink &K, const LG &h, const int32_t *side, uint64_t key) {
  __shared__ unsigned long long s_nb, s_eb;
  __shared__ int32_t s_ok;
  if (threadIdx.x == 0) {
    unsigned long long gi = atomicAdd(&K.counters[0], 1ull);
    unsigned long long nb = atomicAdd(&K.counters[1], (unsigned long long)h.n);
    unsigned long long eb = atomicAdd(&K.counters[2], (unsigned long long)h.m);
    bool ok = gi < (unsigned long long)K.max_graphs && nb + h.n <= (unsigned long long)K.max_nodes &&
              eb + h.m <= (unsigned long long)K.max_entries;
    if (ok) {
      int64_t *r = K.rec + 5 * gi;
      r[0] = (int64_t)nb;
      r[1] = h.n;
      r[2] = (int64_t)eb;
      r[3] = h.m;
      r[4] = (int64_t)key;
    } else {
      atomicAdd(&K.counters[3], 1ull);
    }
    s_ok = ok;
    s_nb = nb;
    s_eb = eb;
  }
  __syncthreads();
  if (s_ok) {
    for (int32_t v = threadIdx.x; v < h.n; v += IPT) {
      K.deg[s_nb + v] = h.xadj[v + 1] - h.xadj[v];
      K.vw[s_nb + v] = h.vw[v];
      K.side[s_nb + v] = side[v];
    }
    for (int32_t e = threadIdx.x; e < h.m; e += IPT) {
      K.adj[s_eb + e] = h.adj[e];
      K.ew[s_eb + e] = h.ew[e];
    }
  }
  __syncthreads();
}

// Learned item mode: the network scores the item graph itself, the learned
// start (first fit in score order, warp 0) is refined by the CTA's 2-way FM on
// the item graph with the finest level's caps.  1: feasible, written to
// side_out; 0: a cap is broken (the caller runs the plain method); -1: the
// item's scratch is too small.
__device__ int item_learned(const IPArgs &A, const ItemDesc &D, const LG &g, Bump &B, int32_t *dyn) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int32_t n = g.n;
  const int32_t P = pow2_at_least(n > 1 ? n : 2);
  float *X = reinterpret_cast<float *>(B.take((int64_t)n * MF));
  int32_t *d1 = B.take(n), *d2 = B.take(n);
  float *scr = reinterpret_cast<float *>(B.take((int64_t)n * (MF + 3 * MH)));
  float *sc = reinterpret_cast<float *>(B.take(n));
  int32_t *side = B.take(n);
  uint64_t *oh = reinterpret_cast<uint64_t *>(B.take(2ll * P));
  int32_t *ov = B.take(P);
  int32_t *fmbuf = B.take(7ll * n + 2);
  if (B.oom) return -1;
  GView<int32_t> G{n, g.xadj, g.adj, 0, g.vw, g.ew};
  mp_features(G, key_step(D.key, DOM_LEARNED), X, d1, d2);
  mp_forward_cta(G, A.W, X, scr, sc);
  __syncthreads();
  if (w == 0) warp_initial(3, g, D.t0, 0, side, oh, ov, nullptr, nullptr, nullptr, sc);
  __syncthreads();
  const int64_t c0 = level_cap(D.L0, D.t0, g.maxc), c1 = level_cap(D.L1, D.t1, g.maxc);
  // FM's state (sides, gains, locks, moves) in shared memory when it fits
  const bool in_smem = 8ll * n + 2 <= A.dyn_words;
  int32_t *fs = in_smem ? dyn : side;
  if (in_smem) {
    for (int32_t v = threadIdx.x; v < n; v += IPT) fs[v] = side[v];
    __syncthreads();
  }
  {
    uint64_t *k0 = reinterpret_cast<uint64_t *>(dyn + 4ll * n + 2 - ((4ll * n) & 1));
    FMBuf sb{dyn + n, dyn + 2ll * n, dyn + 3ll * n, k0, k0 + n};
    FMBuf fb{fmbuf, fmbuf + n, fmbuf + 2ll * n, reinterpret_cast<uint64_t *>(fmbuf + 3ll * n + (n & 1)),
             reinterpret_cast<uint64_t *>(fmbuf + 3ll * n + (n & 1)) + n};
    cta_fm(A, g, fs, c0, c1, in_smem ? sb : fb);
  }
  __syncthreads();
  int64_t W0 = 0, W1 = 0;
  for (int32_t v = threadIdx.x; v < n; v += IPT) {
    if (fs[v] == 0) W0 += g.vw[v];
    else W1 += g.vw[v];
  }
  W0 = block_sum64(W0);
  W1 = block_sum64(W1);
  if (W0 > c0 || W1 > c1) return 0;
  for (int32_t v = threadIdx.x; v < n; v += IPT) A.side_out[D.vbase + v] = fs[v];
  __syncthreads();
  (void)lane;
  return 1;
}

__device__ void run_item(const IPArgs &A, int32_t it, int32_t *wkeys, int32_t *wvals, int32_t *dyn) {
  __shared__ LG lv[IP_MAXL + 1];
  __shared__ int32_t *maps[IP_MAXL + 1];
  __shared__ int64_t s_wk[IPW][3];
  __shared__ int32_t s_wrep[IPW];
  // adaptive portfolio: per warp and algorithm, the feasible stage-1 runs,
  // their cut sum and sum of squares; the repetitions kept for stage 2
  __shared__ int32_t s_fa[IPW][3];
  __shared__ int64_t s_s1[IPW][3];
  __shared__ unsigned __int128 s_s2[IPW][3];
  __shared__ int32_t s_rest[3];
  const ItemDesc D = A.items[it];
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (D.n == 0) return;
  Bump B{A.scratch + D.sbase, D.ssize, 0, false};
  int32_t n0 = D.n;
  int32_t *x0 = B.take(n0 + 1);
  if (B.oom) {
    if (threadIdx.x == 0) atomicExch(A.oom, 1);
    return;
  }
  const int64_t eb = A.gx[D.vbase];
  for (int32_t v = threadIdx.x; v <= n0; v += IPT) x0[v] = (int32_t)(A.gx[D.vbase + v] - eb);
  int64_t cB = 0;
  int32_t md = 0, mc = 0;
  for (int32_t v = threadIdx.x; v < n0; v += IPT) {
    cB += A.svw[D.vbase + v];
    md = max(md, (int32_t)(A.gx[D.vbase + v + 1] - A.gx[D.vbase + v]));
    mc = max(mc, A.svw[D.vbase + v]);
  }
  cB = block_sum64(cB);
  md = block_max32(md);
  mc = block_max32(mc);
  if (threadIdx.x == 0) {
    LG g0;
    g0.n = n0;
    g0.m = D.m;
    g0.xadj = x0;
    g0.adj = const_cast<int32_t *>(A.sadj + eb);
    g0.ew = const_cast<int32_t *>(A.sew + eb);
    g0.vw = const_cast<int32_t *>(A.svw + D.vbase);
    g0.maxdeg = md;
    g0.maxc = mc;
    lv[0] = g0;
  }
  __syncthreads();
  if (A.learned_item) {
    const int64_t mark = B.top;
    const int r = item_learned(A, D, lv[0], B, dyn);
    if (r < 0) {
      if (threadIdx.x == 0) atomicExch(A.oom, 1);
      return;
    }
    if (r == 1) return;
    B.top = mark;  // infeasible: the plain method from here, in the same scratch
  }
  // 1. coarsen
  uint64_t lpkey = key_step(D.key, DOM_IP_LP);
  int32_t nl = 1;
  while (nl < IP_MAXL) {
    LG g = lv[nl - 1];
    if (g.n <= 1) break;
    int64_t UB = cB / A.ip_C;
    if (UB < g.maxc) UB = g.maxc;
    if (UB < 1) UB = 1;
    int32_t *label = B.take(g.n);
    if (B.oom) break;
    int32_t nc = item_cluster(A, g, (int32_t)UB, key_step(lpkey, (uint64_t)(nl - 1)), label, B, wkeys, wvals,
                              dyn, A.dyn_words);
    if (B.oom) break;
    if (nc == g.n) break;
    int32_t *map = B.take(g.n);
    LG c;
    item_contract(g, label, map, &c, B, wkeys, wvals);
    if (B.oom) break;
    int32_t cmd = 0, cmc = 0;
    for (int32_t x = threadIdx.x; x < c.n; x += IPT) {
      cmd = max(cmd, c.xadj[x + 1] - c.xadj[x]);
      cmc = max(cmc, c.vw[x]);
    }
    cmd = block_max32(cmd);
    cmc = block_max32(cmc);
    c.maxdeg = cmd;
    c.maxc = cmc;
    if (threadIdx.x == 0) {
      lv[nl] = c;
      maps[nl - 1] = map;
    }
    __syncthreads();
    ++nl;
    if ((int64_t)A.conv_den * c.n > (int64_t)A.conv_num * g.n) break;
  }
  if (B.oom) {
    if (threadIdx.x == 0) atomicExch(A.oom, 1);
    return;
  }
  // 2. portfolio on the coarsest level, one warp per repetition
  LG h = lv[nl - 1];
  int32_t nH = h.n;
  int32_t PH = pow2_at_least(nH > 1 ? nH : 2);
  int32_t hL0 = level_cap(D.L0, D.t0, h.maxc), hL1 = level_cap(D.L1, D.t1, h.maxc);
  int64_t per_warp = 12ll * nH + 3ll * PH + 16;  // even: keeps every warp's 64-bit areas aligned
  // the portfolio's working state lives in shared memory when it fits
  int32_t *wbuf = per_warp * IPW <= A.dyn_words ? dyn : B.take(per_warp * IPW);
  int32_t *fin = B.take(nH);
  if (B.oom) {
    if (threadIdx.x == 0) atomicExch(A.oom, 1);
    return;
  }
  // learned mode: scores of the coarsest graph's nodes (whole CTA)
  const float *score = nullptr;
  if (A.W && !A.learned_item) {
    float *X = reinterpret_cast<float *>(B.take((int64_t)nH * MF));
    int32_t *d1 = B.take(nH), *d2 = B.take(nH);
    float *scr = reinterpret_cast<float *>(B.take((int64_t)nH * (MF + 3 * MH)));
    float *sc = reinterpret_cast<float *>(B.take(nH));
    if (B.oom) {
      if (threadIdx.x == 0) atomicExch(A.oom, 1);
      return;
    }
    GView<int32_t> G{nH, h.xadj, h.adj, 0, h.vw, h.ew};
    mp_features(G, key_step(D.key, DOM_LEARNED), X, d1, d2);
    mp_forward_cta(G, A.W, X, scr, sc);
    score = sc;
  }
  __shared__ int32_t s_bw;
  {
    int32_t *base = wbuf + per_warp * w;
    int32_t *side = base;
    int32_t *best = side + nH;
    int32_t *gain = best + nH;
    int32_t *locked = gain + nH;
    int32_t *moves = locked + nH;
    int32_t *queue = moves + nH;
    int32_t *ov = queue + nH;
    uint64_t *oh = reinterpret_cast<uint64_t *>(ov + PH);  // offset 6 nH + PH: even
    int32_t reps[3] = {A.rep_random, A.rep_bfs, A.rep_ggg};
    uint64_t doms[3] = {DOM_RANDOM, DOM_BFS, DOM_GGG};
    // candidates in order: [learned], the first `first[a]` repetitions of each
    // algorithm, then (learned mode, best still infeasible) the rest
    int32_t nlrn = score ? 1 : 0;
    int32_t first[3] = {reps[0], reps[1], reps[2]};
    const bool adaptive = A.adaptive && !score;
    if (score) {
      first[0] = min(A.lrep_random, reps[0]);
      first[1] = min(A.lrep_bfs, reps[1]);
      first[2] = min(A.lrep_ggg, reps[2]);
    } else if (adaptive) {
      for (int a = 0; a < 3; ++a) first[a] = (reps[a] + 1) / 2;  // stage 1
    }
    int32_t rest[3] = {reps[0] - first[0], reps[1] - first[1], reps[2] - first[2]};
    int32_t R0 = nlrn + first[0] + first[1] + first[2];
    int32_t R1 = rest[0] + rest[1] + rest[2];
    bool have = false;
    int32_t binf = 0, brep = -1;
    int64_t bov = 0, bcut = 0;
    int32_t fa[3] = {0, 0, 0};
    int64_t s1[3] = {0, 0, 0};
    unsigned __int128 s2[3] = {0, 0, 0};
    for (int phase = 0; phase < 2; ++phase) {
      if (phase == 1) {
        if (adaptive) {
          // stage 2 keeps an algorithm while mean - 2 sd (population) of its
          // feasible stage-1 cuts is at most the best feasible cut, exactly:
          // s1 - f b <= 2 sqrt(f s2 - s1^2); everything stays when no run is
          // feasible yet
          if (threadIdx.x == 0) {
            const bool feas = s_wk[s_bw][0] == 0;
            const int64_t b = s_wk[s_bw][2];
            for (int a = 0; a < 3; ++a) {
              int32_t f = 0;
              int64_t t1 = 0;
              unsigned __int128 t2 = 0;
              for (int x = 0; x < IPW; ++x) {
                f += s_fa[x][a];
                t1 += s_s1[x][a];
                t2 += s_s2[x][a];
              }
              bool keep = true;
              if (feas) {
                if (f == 0) {
                  keep = false;
                } else {
                  const __int128 D = (__int128)t1 - (__int128)f * b;
                  const __int128 var = (__int128)f * (__int128)t2 - (__int128)t1 * t1;
                  keep = D <= 0 || D * D <= 4 * var;
                }
              }
              s_rest[a] = keep ? reps[a] - first[a] : 0;
            }
          }
          __syncthreads();
          rest[0] = s_rest[0];
          rest[1] = s_rest[1];
          rest[2] = s_rest[2];
          R1 = rest[0] + rest[1] + rest[2];
          if (R1 == 0) break;
        } else if (R1 == 0 || s_wk[s_bw][0] == 0) {
          break;
        }
      }
      int32_t Rp = phase == 0 ? R0 : R1;
      const int32_t *cnt = phase == 0 ? first : rest;
      for (int32_t q = w; q < Rp; q += IPW) {
        int a, r;
        if (phase == 0 && q < nlrn) {
          a = 3;
          r = 0;
        } else {
          int32_t x = phase == 0 ? q - nlrn : q;
          a = x < cnt[0] ? 0 : (x < cnt[0] + cnt[1] ? 1 : 2);
          r = a == 0 ? x : (a == 1 ? x - cnt[0] : x - cnt[0] - cnt[1]);
          if (phase == 1) r += first[a];
        }
        uint64_t key = a == 3 ? 0 : key_step(key_step(D.key, doms[a]), (uint64_t)r);
        warp_initial(a, h, D.t0, key, side, oh, ov, gain, locked, queue, score);
        FMBuf fb{gain, locked, moves, oh + PH, oh + PH + nH};
        int64_t cut = warp_fm(A, h, side, hL0, hL1, fb);
        int64_t W0 = 0, W1 = 0;
        for (int32_t v = lane; v < nH; v += 32) {
          if (side[v] == 0) W0 += h.vw[v];
          else W1 += h.vw[v];
        }
        W0 = warp_sum64(W0);
        W1 = warp_sum64(W1);
        int64_t o0 = W0 - hL0, o1 = W1 - hL1;
        int64_t o = o0 > o1 ? o0 : o1;
        int32_t inf = o > 0;
        int64_t ovv = inf ? o : 0;
        if (phase == 0 && a < 3 && !inf) {
          fa[a] += 1;
          s1[a] += cut;
          s2[a] += (unsigned __int128)((uint64_t)cut) * (uint64_t)cut;
        }
        if (!have || fm_less(inf, ovv, cut, binf, bov, bcut)) {
          have = true;
          binf = inf;
          bov = ovv;
          bcut = cut;
          brep = phase == 0 ? q : R0 + q;
          for (int32_t v = lane; v < nH; v += 32) best[v] = side[v];
        }
        __syncwarp();
      }
      if (lane == 0) {
        s_wk[w][0] = have ? binf : 2;
        s_wk[w][1] = bov;
        s_wk[w][2] = bcut;
        s_wrep[w] = have ? brep : INT32_MAX;
        for (int a = 0; a < 3; ++a) {
          s_fa[w][a] = fa[a];
          s_s1[w][a] = s1[a];
          s_s2[w][a] = s2[a];
        }
      }
      __syncthreads();
      // the first candidate with the best (infeasible?, overload, cut) wins
      if (threadIdx.x == 0) {
        int32_t bw_ = 0;
        for (int32_t x = 1; x < IPW; ++x) {
          bool better = fm_less((int32_t)s_wk[x][0], s_wk[x][1], s_wk[x][2], (int32_t)s_wk[bw_][0],
                                s_wk[bw_][1], s_wk[bw_][2]);
          bool tie = !better && !fm_less((int32_t)s_wk[bw_][0], s_wk[bw_][1], s_wk[bw_][2],
                                         (int32_t)s_wk[x][0], s_wk[x][1], s_wk[x][2]);
          if (better || (tie && s_wrep[x] < s_wrep[bw_])) bw_ = x;
        }
        s_bw = bw_;
      }
      __syncthreads();
    }
  }
  {
    int32_t *bsrc = wbuf + per_warp * s_bw + nH;
    for (int32_t v = threadIdx.x; v < nH; v += IPT) fin[v] = bsrc[v];
  }
  __syncthreads();
  if (A.sink.counters && !A.sink.item_level) record_sample(A.sink, h, fin, D.key);
  // 3. uncoarsen with FM on every level (warp 0)
  int32_t *cur = fin;
  int32_t *fmbuf = B.take(7ll * n0 + 2);
  if (B.oom) {
    if (threadIdx.x == 0) atomicExch(A.oom, 1);
    return;
  }
  FMBuf fb{fmbuf, fmbuf + n0, fmbuf + 2ll * n0, reinterpret_cast<uint64_t *>(fmbuf + 3ll * n0 + (n0 & 1)),
           reinterpret_cast<uint64_t *>(fmbuf + 3ll * n0 + (n0 & 1)) + n0};
  for (int32_t l = nl - 2; l >= 0; --l) {
    LG g = lv[l];
    int32_t *fine = B.take(g.n);
    if (B.oom) {
      if (threadIdx.x == 0) atomicExch(A.oom, 1);
      return;
    }
    const int32_t *map = maps[l];
    // FM's state (sides, gains, locks, moves) in shared memory when it fits:
    // every FM step scans all nodes
    bool in_smem = 8ll * g.n + 2 <= A.dyn_words;
    int32_t *fs = in_smem ? dyn : fine;
    for (int32_t v = threadIdx.x; v < g.n; v += IPT) fs[v] = cur[map[v]];
    __syncthreads();
    {
      uint64_t *k0 = reinterpret_cast<uint64_t *>(dyn + 4ll * g.n + 2 - ((4ll * g.n) & 1));
      FMBuf sb{dyn + g.n, dyn + 2ll * g.n, dyn + 3ll * g.n, k0, k0 + g.n};
      cta_fm(A, g, fs, level_cap(D.L0, D.t0, g.maxc), level_cap(D.L1, D.t1, g.maxc), in_smem ? sb : fb);
    }
    __syncthreads();
    if (in_smem) {
      for (int32_t v = threadIdx.x; v < g.n; v += IPT) fine[v] = fs[v];
      __syncthreads();
    }
    cur = fine;
  }
  for (int32_t v = threadIdx.x; v < n0; v += IPT) A.side_out[D.vbase + v] = cur[v];
  __syncthreads();
  if (A.sink.counters && A.sink.item_level) record_sample(A.sink, lv[0], cur, D.key);
}

__global__ void __launch_bounds__(IPT) k_ip_items(IPArgs A) {
  __shared__ int32_t wkeys[IPW * IP_WTAB];
  __shared__ int32_t wvals[IPW * IP_WTAB];
  __shared__ int32_t s_it;
  extern __shared__ __align__(16) int32_t ipdyn[];
  for (;;) {
    if (threadIdx.x == 0) s_it = atomicAdd(A.queue, 1);
    __syncthreads();
    int32_t q = s_it;
    __syncthreads();
    if (q >= A.nitems) break;
    run_item(A, A.order[q], wkeys, wvals, ipdyn);
  }
}

// ------------------------------------------------------ extraction (host side kernels)
__global__ void k_block_keys(int32_t n, const int32_t *part, int bits, uint64_t *keys) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x)
    keys[v] = ((uint64_t)(uint32_t)part[v] << bits) | (uint64_t)v;
}

__global__ void k_block_stats(int32_t n, const int64_t *xadj, const int32_t *adj, const int32_t *vw,
                              const int32_t *part, const uint64_t *keys, uint64_t mask, int32_t *members,
                              int32_t *bcount, unsigned long long *bweight, int32_t *ideg,
                              unsigned long long *becount) {
  // a warp takes 32 consecutive positions and walks their rows one by one
  int lane = threadIdx.x & 31;
  int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t base = gw * 32; base < n; base += nw * 32) {
    int64_t i = base + lane;
    int32_t v = -1, b = -1;
    if (i < n) {
      v = (int32_t)(keys[i] & mask);
      members[i] = v;
      b = part[v];
    }
    int32_t myd = 0;
    int jmax = (int)(n - base < 32 ? n - base : 32);
    for (int j = 0; j < jmax; ++j) {
      int32_t vj = __shfl_sync(0xFFFFFFFFu, v, j), bj = __shfl_sync(0xFFFFFFFFu, b, j);
      int32_t d = 0;
      for (int64_t q = xadj[vj] + lane; q < xadj[vj + 1]; q += 32) d += (part[adj[q]] == bj);
      d = warp_sum32(d);
      if (lane == j) myd = d;
    }
    if (i < n) {
      atomicAdd(&bcount[b], 1);
      atomicAdd(&bweight[b], (unsigned long long)(vw ? vw[v] : 1));
      ideg[i] = myd;
      atomicAdd(&becount[b], (unsigned long long)myd);
    }
  }
}

__global__ void k_local_ids(int32_t n, const int32_t *members, const int32_t *part, const int32_t *boff,
                            int32_t *loc) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    int32_t v = members[i];
    loc[v] = (int32_t)(i - boff[part[v]]);
  }
}

__global__ void k_fill_sub(int32_t n, const int64_t *xadj, const int32_t *adj, const int32_t *vw,
                           const int32_t *ew, const int32_t *part, const int32_t *members,
                           const int32_t *loc, const int64_t *gx, int32_t *sadj, int32_t *sew,
                           int32_t *svw) {
  // a warp per row, order-preserving compaction of the entries inside the block
  int lane = threadIdx.x & 31;
  int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = gw; i < n; i += nw) {
    int32_t v = members[i];
    int32_t b = part[v];
    if (lane == 0) svw[i] = vw ? vw[v] : 1;
    int64_t o = gx[i];
    for (int64_t q0 = xadj[v]; q0 < xadj[v + 1]; q0 += 32) {
      int64_t q = q0 + lane;
      bool keep = false;
      int32_t u = 0;
      if (q < xadj[v + 1]) {
        u = adj[q];
        keep = part[u] == b;
      }
      unsigned bal = __ballot_sync(0xFFFFFFFFu, keep);
      if (keep) {
        int64_t p = o + __popc(bal & ((1u << lane) - 1u));
        sadj[p] = loc[u];
        sew[p] = ew ? ew[q] : 1;
      }
      o += __popc(bal);
    }
  }
}

__global__ void k_set_last(int64_t *a, int64_t idx, const int64_t *v) { a[idx] = *v; }

__global__ void k_write_parts(int32_t n, const int32_t *members, const int32_t *part_old,
                              const int32_t *newid, const int32_t *split, const int32_t *side,
                              int32_t *part) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    int32_t v = members[i];
    int32_t b = part_old[v];
    part[v] = newid[b] + (split[b] ? side[i] : 0);
  }
}

// caps4 (host, nullable): explicit (t0, t1, L0, L1) per block instead of the
// caps Algorithm 2 derives from (eps, cV, k, f)
int32_t bipartition_blocks(const Graph &g, int32_t *part, int32_t nblocks, std::vector<int32_t> &f,
                           double eps, int64_t cV, int32_t k, uint64_t roundkey, int32_t *items_out,
                           const int32_t *caps4) {
  Context &C = ctx();
  const kmp_config &cfg = C.cfg;
  cudaStream_t s = C.stream;
  int32_t n = g.n;
  // new ids, child final counts
  std::vector<int32_t> newid(nblocks), split(nblocks), nf;
  int32_t nn = 0;
  for (int32_t b = 0; b < nblocks; ++b) {
    newid[b] = nn;
    if (f[b] >= 2) {
      split[b] = 1;
      nf.push_back(f[b] / 2);
      nf.push_back(f[b] - f[b] / 2);
      nn += 2;
    } else {
      split[b] = 0;
      nf.push_back(f[b]);
      nn += 1;
    }
  }
  if (items_out) *items_out = 0;
  if (n == 0) {
    f = nf;
    return nn;
  }
  int bitsN = 1;
  while ((1ll << bitsN) < (int64_t)n) ++bitsN;
  int bitsB = 1;
  while ((1ll << bitsB) < (int64_t)nblocks) ++bitsB;
  int grid = grid_for(n, 256);
  DBuf<uint64_t> keys(n), tmp(n);
  k_block_keys<<<grid, 256, 0, s>>>(n, part, bitsN, keys);
  KMP_LAUNCHED("block_keys");
  // keys are written in ascending node order, so a stable sort by the block
  // bits alone leaves every block's members in ascending id
  radix_sort_u64(keys, tmp, n, bitsB, bitsN);
  DBuf<int32_t> members(n), bcount(nblocks + 1), ideg(n), boff(nblocks + 1), loc(n);
  DBuf<unsigned long long> bweight(nblocks), becount(nblocks);
  bcount.zero();
  bweight.zero();
  becount.zero();
  k_block_stats<<<grid, 256, 0, s>>>(n, g.xadj, g.adj, g.vw, part, keys, (1ull << bitsN) - 1ull, members,
                                     bcount, bweight, ideg, becount);
  KMP_LAUNCHED("block_stats");
  scan_excl_i32(bcount, boff, nblocks + 1, nullptr);
  k_local_ids<<<grid, 256, 0, s>>>(n, members, part, boff, loc);
  KMP_LAUNCHED("local_ids");
  DBuf<int64_t> gx(n + 1), etot(1);
  scan_excl_i32_to_i64(ideg, gx, n, etot);
  k_set_last<<<1, 1, 0, s>>>(gx, n, etot);
  KMP_LAUNCHED("set_last");
  int64_t E = read1(etot.p);
  DBuf<int32_t> sadj(E), sew(E), svw(n);
  k_fill_sub<<<grid, 256, 0, s>>>(n, g.xadj, g.adj, g.vw, g.ew, part, members, loc, gx, sadj, sew, svw);
  KMP_LAUNCHED("fill_sub");
  std::vector<int32_t> hcount(nblocks + 1), hoff(nblocks + 1);
  std::vector<unsigned long long> hw(nblocks), he(nblocks);
  to_host(hcount.data(), bcount.p, nblocks);
  to_host(hoff.data(), boff.p, nblocks + 1);
  to_host(hw.data(), bweight.p, nblocks);
  to_host(he.data(), becount.p, nblocks);
  // item descriptors
  std::vector<ItemDesc> items;
  int64_t ebase = 0;
  for (int32_t b = 0; b < nblocks; ++b) {
    int64_t eb = ebase;
    ebase += (int64_t)he[b];
    if (!split[b] || hcount[b] == 0) continue;
    if (hcount[b] > IP_MAX_N)
      fail(KMP_ERR_UNSUPPORTED, "block of " + std::to_string(hcount[b]) +
                                    " nodes exceeds the bipartitioner's item limit");
    ItemDesc d{};
    d.vbase = hoff[b];
    d.ebase = eb;
    d.n = hcount[b];
    d.m = (int32_t)he[b];
    if (caps4) {
      d.t0 = caps4[4 * b];
      d.t1 = caps4[4 * b + 1];
      d.L0 = caps4[4 * b + 2];
      d.L1 = caps4[4 * b + 3];
    } else {
      split_caps(eps, cV, k, (int64_t)hw[b], f[b], &d.t0, &d.t1, &d.L0, &d.L1);
    }
    d.key = key_step(roundkey, (uint64_t)b);
    items.push_back(d);
  }
  if (items_out) *items_out = (int32_t)items.size();
  DBuf<int32_t> side(n);
  side.zero();
  if (!items.empty()) {
    // largest items first (work queue order does not change results)
    std::vector<int32_t> order(items.size());
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b2) {
      return (int64_t)items[a].n + items[a].m > (int64_t)items[b2].n + items[b2].m;
    });
    DBuf<int32_t> dorder(items.size()), q(2);
    to_dev(dorder.p, order.data(), order.size());
    bool learned = cfg.learned && proposer().W;
    int64_t mult = 1;
    for (int attempt = 0; attempt < 6; ++attempt, mult *= 4) {
      int64_t total = 0;
      for (auto &d : items) {
        int64_t nP = next_pow2((uint64_t)std::max(d.n, 2));
        int64_t mP = next_pow2((uint64_t)std::max(d.m, 2));
        d.sbase = total;
        d.ssize = mult * (104ll * d.n + 64ll * nP + 16ll * d.m + 8ll * mP + 2048 +
                          (learned ? (int64_t)(2 * MF + 3 * MH + 4) * d.n + 64 : 0));
        total += d.ssize;
      }
      DBuf<ItemDesc> ditems(items.size());
      DBuf<int32_t> scratch(total);
      to_dev(ditems.p, items.data(), items.size());
      q.zero();
      IPArgs A;
      A.items = ditems;
      A.order = dorder;
      A.nitems = (int32_t)items.size();
      A.queue = q.p;
      A.oom = q.p + 1;
      A.gx = gx;
      A.sadj = sadj;
      A.sew = sew;
      A.svw = svw;
      A.side_out = side;
      A.scratch = scratch;
      A.S = cfg.subrounds;
      A.ip_C = cfg.ip_C;
      A.ip_lp_rounds = cfg.ip_lp_rounds;
      A.rep_random = cfg.rep_random;
      A.rep_bfs = cfg.rep_bfs;
      A.rep_ggg = cfg.rep_ggg;
      A.fm_passes = cfg.fm_passes;
      A.fm_stop = cfg.fm_stop;
      A.conv_num = cfg.conv_num;
      A.conv_den = cfg.conv_den;
      A.W = cfg.learned ? proposer().W : nullptr;
      A.lrep_random = cfg.lrep_random;
      A.lrep_bfs = cfg.lrep_bfs;
      A.lrep_ggg = cfg.lrep_ggg;
      A.adaptive = (cfg.adaptive && !A.W) ? 1 : 0;
      A.learned_item = (cfg.learned == 2 && A.W) ? 1 : 0;
      A.sink = sample_sink();
      // dynamic shared memory: the LP working arrays (7.5 words a node plus
      // sort space) and then the FM state (8 words a node) of the largest item of the round,
      // at least 16 KB (the portfolio of small coarsest graphs), at most what
      // the SM offers next to the kernel's static shared memory when the round
      // has no more items than SMs (its items are then on the critical path,
      // one CTA per SM), else at most 72 KB (two CTAs per SM); an item that
      // does not fit works in its global scratch
      int64_t maxn = 0;
      for (auto &d : items) maxn = std::max<int64_t>(maxn, d.n);
      int32_t cap_words = (int64_t)items.size() <= C.sms ? IP_DYN_MAX_WORDS : IP_DYN_SHARED_WORDS;
      A.dyn_words = (int32_t)std::min<int64_t>(std::max<int64_t>(8 * maxn + 2 + 2 * maxn / 4, 4096), cap_words);
      size_t dyn_bytes = (size_t)A.dyn_words * sizeof(int32_t);
      static bool attr_set = false;
      if (!attr_set) {
        KMP_CUDA(cudaFuncSetAttribute(k_ip_items, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      IP_DYN_MAX_WORDS * (int)sizeof(int32_t)));
        attr_set = true;
      }
      int gridip = (int)std::min<int64_t>((int64_t)items.size(), (int64_t)C.sms * C.tune.ip_blocks_per_sm);
      k_ip_items<<<gridip, IPT, dyn_bytes, s>>>(A);
      KMP_LAUNCHED("ip_items");
      int32_t oom = 0;
      to_host(&oom, q.p + 1, 1);
      if (!oom) break;
      if (attempt == 5) fail(KMP_ERR_NOMEM, "bipartitioner scratch could not be sized");
    }
  }
  DBuf<int32_t> dnew(nblocks), dsplit(nblocks), old(n);
  to_dev(dnew.p, newid.data(), nblocks);
  to_dev(dsplit.p, split.data(), nblocks);
  KMP_CUDA(cudaMemcpyAsync(old.p, part, (size_t)n * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
  k_write_parts<<<grid, 256, 0, s>>>(n, members, old, dnew, dsplit, side, part);
  KMP_LAUNCHED("write_parts");
  f = nf;
  return nn;
}

}  // namespace kmp
