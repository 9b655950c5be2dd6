// k-way balancing (Section 4.3, "Balancing").
//
// Deterministic reading: the starting state initialises the candidates of
// every overloaded block at once (the paper's priority-queue initialisation):
// a node v of an overloaded block B with some admissible other block gets
// d = max over admissible blocks of conn(v, b) - conn(v, B) and the relative
// gain d*c(v) (d >= 0) or d/c(v) (d < 0).  Then the overloaded blocks are
// emptied in ascending id, candidates in (relative gain desc, id asc) order,
// each moved at its turn to the admissible block of largest current
// connectivity (ties: lowest id) until the block fits.
//
// GPU mapping: candidates of all overloaded blocks in one full-GPU pass (one
// warp per node, connectivity in a per-warp hash table); grouping by block
// with a radix sort of (block, node) keys; one CTA per overloaded block sorts
// its candidates by the exact rational order; then every overloaded block
// speculates its moves at once (one warp each, as if it were emptied first),
// and one CTA commits in block order: a speculated move stands while its
// target still fits, everything else is decided again exactly, in batches
// whose members are evaluated at once and committed while they provably do
// not interact.
#include <algorithm>
#include <climits>

#include "kmp_internal.cuh"

namespace kmp {

constexpr int BAL_T = 256;
constexpr int BAL_W = BAL_T / 32;
constexpr int BAL_STAB = 512;  // per-warp shared table entries

struct BalArgs {
  int32_t n, k;
  const int64_t *xadj;
  const int32_t *adj;
  const int32_t *vw;
  const int32_t *ew;
  int32_t *part;
  int64_t *bw;
  const int32_t *cap;
  const uint8_t *over;
  const int32_t *olist;  // the overloaded blocks, ascending
  int32_t nover;
  int64_t max_room;      // the largest cap - weight over all blocks at the start
  int64_t *cand_d;       // [n] d of candidate nodes
  uint64_t *keys;        // (block << bitsN | node) of candidates
  int32_t *ncand;
  int bitsN;
  int32_t *seg_lo;       // [k] candidate segment of each block
  int32_t *seg_hi;
  uint64_t *sortbuf;     // per-block sort space (2 * ncand)
  int32_t *gtab;         // per-warp global tables when labels do not fit shared memory
  uint32_t gcap;
  unsigned long long *moved;
  // speculation: per overloaded block (index in olist) up to SPEC_MAX moves
  int32_t *spec_v, *spec_t;  // [nover][SPEC_MAX]
  int32_t *spec_n;           // moves recorded
  int32_t *spec_end;         // candidate position where the speculation stopped
  int32_t *spec_sat;         // 1: the block fits after its recorded moves
};

constexpr int SPEC_MAX = 16;

__device__ __forceinline__ int32_t bw_node(const BalArgs &A, int32_t v) { return A.vw ? A.vw[v] : 1; }

// table size for v's connectivity: a power of two >= 2 * (distinct blocks
// among its neighbours, at most min(degree, k)), at least 32
__device__ __forceinline__ uint32_t conn_cap(const BalArgs &A, int32_t v) {
  int64_t d = A.xadj[v + 1] - A.xadj[v];
  if (d > A.k) d = A.k;
  uint32_t cap = 32;
  while ((int64_t)cap < 2 * d) cap <<= 1;
  return cap;
}

// connectivity of v to the blocks of its neighbours, aggregated by one warp
__device__ int64_t conn_table(const BalArgs &A, int32_t v, int32_t *K, int32_t *V, uint32_t &mask) {
  int lane = threadIdx.x & 31;
  int64_t b = A.xadj[v], e = A.xadj[v + 1];
  uint32_t cap = conn_cap(A, v);
  mask = cap - 1;
  for (uint32_t i = lane; i < cap; i += 32) {
    K[i] = HT_EMPTY;
    V[i] = 0;
  }
  __syncwarp();
  // 128 entries per pass (four gathers in flight per lane); lanes that hit the
  // same block add their weights first, so a hub's many entries into one block
  // cost one atomic per pass instead of one per entry
  for (int64_t base = b; base < e; base += 128) {
    int32_t u[4], wt[4], blk[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      int64_t q = base + r * 32 + lane;
      bool ok = q < e;
      u[r] = ok ? A.adj[q] : -1;
      wt[r] = ok ? (A.ew ? A.ew[q] : 1) : 0;
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) blk[r] = u[r] >= 0 ? A.part[u[r]] : HT_EMPTY;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      unsigned peers = __match_any_sync(0xFFFFFFFFu, blk[r]);
      int32_t s = __reduce_add_sync(peers, wt[r]);
      if (blk[r] != HT_EMPTY && lane == __ffs(peers) - 1) ht_add(K, V, mask, blk[r], s);
    }
  }
  __syncwarp();
  return ht_get(K, V, mask, A.part[v]);
}

// some block has room for weight c (the overloaded block itself has none);
// candidates are rated from the starting state, so the starting room decides
__device__ __forceinline__ bool room_somewhere(const BalArgs &A, int64_t c) { return A.max_room >= c; }

// Candidates of the overloaded blocks, one warp per node with the warp's
// shared-memory table.  Nodes whose table would not fit it are listed in
// big[] for k_bal_cand_big.
__global__ void __launch_bounds__(BAL_T) k_bal_cand(BalArgs A, int32_t *big, int32_t *nbig) {
  __shared__ int32_t sk[BAL_W][BAL_STAB], sv[BAL_W][BAL_STAB];
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int64_t gw = (int64_t)blockIdx.x * BAL_W + w, nw = (int64_t)gridDim.x * BAL_W;
  int32_t *K = sk[w], *V = sv[w];
  for (int64_t v = gw; v < A.n; v += nw) {
    int32_t B = A.part[v];
    if (!A.over[B]) continue;
    if (conn_cap(A, (int32_t)v) > (uint32_t)BAL_STAB) {
      if (lane == 0) big[atomicAdd(nbig, 1)] = (int32_t)v;
      continue;
    }
    uint32_t mask;
    int64_t cown = conn_table(A, (int32_t)v, K, V, mask);
    int64_t c = bw_node(A, (int32_t)v);
    int64_t best = -1;
    int32_t nadj = 0;
    for (uint32_t i = lane; i <= mask; i += 32) {
      int32_t b = K[i];
      if (b == HT_EMPTY || b == B) continue;
      if (A.bw[b] + c > A.cap[b]) continue;
      ++nadj;
      if (V[i] > best) best = V[i];
    }
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) {
      int64_t o = (int64_t)shfl_xor64((uint64_t)best, m);
      best = o > best ? o : best;
      nadj += __shfl_xor_sync(0xFFFFFFFFu, nadj, m);
    }
    if (best < 0 && room_somewhere(A, c)) best = 0;  // an admissible block without neighbours
    if (lane == 0 && best >= 0) {
      A.cand_d[v] = best - cown;
      int32_t p = atomicAdd(A.ncand, 1);
      A.keys[p] = ((uint64_t)(uint32_t)B << A.bitsN) | (uint64_t)v;
    }
    __syncwarp();
  }
}

// Candidates among the listed high-degree nodes: one CTA per node, the node's
// row spread over all threads into the CTA's own global table region
// (2 * gcap words; the node uses the power of two >= 2 min(degree, k)).
__global__ void __launch_bounds__(BAL_T) k_bal_cand_big(BalArgs A, const int32_t *big, const int32_t *nbig) {
  __shared__ int64_t s_best[BAL_W];
  __shared__ int32_t s_nadj[BAL_W];
  __shared__ int64_t s_cown;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int32_t *K = A.gtab + (int64_t)blockIdx.x * 2 * A.gcap, *V = K + A.gcap;
  const int32_t nb = *nbig;
  for (int32_t i = blockIdx.x; i < nb; i += gridDim.x) {
    const int32_t v = big[i], B = A.part[v];
    const uint32_t cap = conn_cap(A, v), mask = cap - 1;
    for (uint32_t x = threadIdx.x; x < cap; x += BAL_T) {
      K[x] = HT_EMPTY;
      V[x] = 0;
    }
    if (threadIdx.x == 0) s_cown = 0;
    __syncthreads();
    const int64_t b = A.xadj[v], e = A.xadj[v + 1];
    for (int64_t base = b + 32 * w; base < e; base += BAL_T) {
      const int64_t q = base + lane;
      const bool ok = q < e;
      const int32_t u = ok ? A.adj[q] : -1;
      const int32_t wt = ok ? (A.ew ? A.ew[q] : 1) : 0;
      const int32_t blk = ok ? A.part[u] : HT_EMPTY;
      const unsigned peers = __match_any_sync(0xFFFFFFFFu, blk);
      const int32_t sm = __reduce_add_sync(peers, wt);
      if (blk != HT_EMPTY && lane == __ffs(peers) - 1) ht_add(K, V, mask, blk, sm);
    }
    __syncthreads();
    const int64_t c = bw_node(A, v);
    int64_t best = -1;
    int32_t nadj = 0;
    for (uint32_t x = threadIdx.x; x < cap; x += BAL_T) {
      const int32_t blk = K[x];
      if (blk == HT_EMPTY) continue;
      if (blk == B) {
        s_cown = V[x];
        continue;
      }
      if (A.bw[blk] + c > A.cap[blk]) continue;
      ++nadj;
      if (V[x] > best) best = V[x];
    }
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) {
      int64_t o = (int64_t)shfl_xor64((uint64_t)best, m);
      best = o > best ? o : best;
      nadj += __shfl_xor_sync(0xFFFFFFFFu, nadj, m);
    }
    if (lane == 0) {
      s_best[w] = best;
      s_nadj[w] = nadj;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      int64_t bb = -1;
      int32_t na = 0;
      for (int x = 0; x < BAL_W; ++x) {
        bb = s_best[x] > bb ? s_best[x] : bb;
        na += s_nadj[x];
      }
      if (bb < 0 && room_somewhere(A, c)) bb = 0;  // an admissible block without neighbours
      if (bb >= 0) {
        A.cand_d[v] = bb - s_cown;
        int32_t p = atomicAdd(A.ncand, 1);
        A.keys[p] = ((uint64_t)(uint32_t)B << A.bitsN) | (uint64_t)v;
      }
    }
    __syncthreads();
  }
}

__global__ void k_bal_segments(BalArgs A, int32_t N) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    int32_t B = (int32_t)(A.keys[i] >> A.bitsN);
    if (i == 0 || (int32_t)(A.keys[i - 1] >> A.bitsN) != B) A.seg_lo[B] = (int32_t)i;
    if (i == N - 1 || (int32_t)(A.keys[i + 1] >> A.bitsN) != B) A.seg_hi[B] = (int32_t)i + 1;
  }
}

// "a before b" in (relative gain desc, node asc); exact with 64-bit products
__device__ __forceinline__ bool rg_before(int64_t d1, int64_t c1, int32_t v1, int64_t d2, int64_t c2,
                                          int32_t v2) {
  bool s1 = d1 >= 0, s2 = d2 >= 0;
  if (s1 != s2) return s1;
  int64_t p = s1 ? d1 * c1 : d1 * c2, q = s1 ? d2 * c2 : d2 * c1;
  if (p != q) return p > q;
  return v1 < v2;
}

// one CTA per overloaded block: bitonic sort of its candidates
__global__ void __launch_bounds__(BAL_T) k_bal_sort(BalArgs A) {
  int32_t B = A.olist[blockIdx.x];
  int32_t lo = A.seg_lo[B], hi = A.seg_hi[B];
  int32_t len = hi - lo;
  if (len <= 1) return;
  int32_t P = 1;
  while (P < len) P <<= 1;
  uint64_t mask = (1ull << A.bitsN) - 1ull;
  int32_t *vv = reinterpret_cast<int32_t *>(A.sortbuf + 2ll * lo);  // 2*len >= P slots
  for (int32_t i = threadIdx.x; i < P; i += blockDim.x)
    vv[i] = i < len ? (int32_t)(A.keys[lo + i] & mask) : -1;
  __syncthreads();
  for (int32_t kk = 2; kk <= P; kk <<= 1)
    for (int32_t j = kk >> 1; j > 0; j >>= 1) {
      for (int32_t i = threadIdx.x; i < P; i += blockDim.x) {
        int32_t l = i ^ j;
        if (l > i) {
          int32_t a = vv[i], b = vv[l];
          // padding (-1) sorts last
          bool b_first;
          if (a < 0) b_first = b >= 0;
          else if (b < 0) b_first = false;
          else b_first = rg_before(A.cand_d[b], bw_node(A, b), b, A.cand_d[a], bw_node(A, a), a);
          if (b_first == ((i & kk) == 0)) {
            vv[i] = b;
            vv[l] = a;
          }
        }
      }
      __syncthreads();
    }
  for (int32_t i = threadIdx.x; i < len; i += blockDim.x)
    A.keys[lo + i] = ((uint64_t)(uint32_t)B << A.bitsN) | (uint64_t)(uint32_t)vv[i];
}

// Moves in candidate order, evaluated in batches of up to 32.  A batch holds
// the shortest prefix of the remaining candidates whose weights cover the
// overload (it may need more moves, never fewer).  The batch's adjacency
// rows are walked at once (by warp 0 alone for a small batch, else by the
// whole CTA), building one connectivity table per member and marking which
// members are neighbours of each other; each member's target is picked from
// the state at the start of the batch, and one thread commits in order.
// While a block is emptied, every other block only gains
// weight, so a target that is still admissible is still the best (or still
// the lowest-id admissible one), and "no admissible target" stays true; only
// a move of a neighbour changes connectivity.  A member passes iff its target
// still fits and no earlier move of the batch was its neighbour; at the first
// one that does not, the next batch starts there (its first member always
// passes).  The result equals one move at a time.
constexpr int BM_T = 1024;
constexpr int BM_W = BM_T / 32;

// Speculation, one warp per overloaded block B, all blocks at once: B's moves
// in candidate order as if B were the first block emptied (every other block
// at its starting weight, plus B's own recorded moves).  A decision is only
// recorded when nothing an earlier block does can change it: blocks other
// than the overloaded ones only gain weight, so a better block that does not
// fit keeps not fitting, and the chosen block is checked again at commit; an
// earlier overloaded block, however, loses weight (it may start to fit) and
// its moved nodes change their neighbours' connectivity, so a node adjacent
// to an earlier overloaded block stops the speculation, as does a node that
// would need the lowest-id fallback.
__global__ void __launch_bounds__(BAL_T) k_bal_spec(BalArgs A) {
  __shared__ int32_t sk[BAL_W][BAL_STAB], sv[BAL_W][BAL_STAB];
  __shared__ int32_t mv_v[BAL_W][SPEC_MAX], mv_t[BAL_W][SPEC_MAX], mv_c[BAL_W][SPEC_MAX];
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int64_t gw = (int64_t)blockIdx.x * BAL_W + w, nw = (int64_t)gridDim.x * BAL_W;
  int32_t *K = sk[w], *V = sv[w];
  uint64_t vmask = (1ull << A.bitsN) - 1ull;
  for (int64_t ob = gw; ob < A.nover; ob += nw) {
    int32_t B = A.olist[ob];
    int32_t lo = A.seg_lo[B], hi = A.seg_hi[B];
    int64_t wB = A.bw[B];
    int32_t nm = 0, i = lo, sat = 0;
    for (; i < hi; ++i) {
      if (wB <= A.cap[B]) {
        sat = 1;
        break;
      }
      if (nm == SPEC_MAX) break;
      int32_t v = (int32_t)(A.keys[i] & vmask);
      // a node whose table does not fit shared memory is left to the exact commit
      if (conn_cap(A, v) > (uint32_t)BAL_STAB) break;
      int64_t c = bw_node(A, v);
      uint32_t mask;
      conn_table(A, v, K, V, mask);
      // B's own recorded moves of neighbours; neighbours in earlier overloaded blocks
      bool fragile = false;
      for (int64_t q = A.xadj[v] + lane; q < A.xadj[v + 1]; q += 32) {
        int32_t u = A.adj[q], bu = A.part[u];
        if (bu != B && bu < B && A.over[bu]) fragile = true;
        if (bu == B)
          for (int j = 0; j < nm; ++j)
            if (mv_v[w][j] == u) ht_add(K, V, mask, mv_t[w][j], A.ew ? A.ew[q] : 1);
      }
      __syncwarp();
      fragile = __any_sync(0xFFFFFFFFu, fragile);
      uint64_t bestk = 0;  // (conn, ~block): largest connectivity, then lowest id
      if (!fragile)
        for (uint32_t x = lane; x <= mask; x += 32) {
          int32_t b = K[x];
          if (b == HT_EMPTY || b == B) continue;
          int64_t wb = A.bw[b];
          for (int j = 0; j < nm; ++j)
            if (mv_t[w][j] == b) wb += mv_c[w][j];
          if (wb + c > A.cap[b]) continue;
          uint64_t key = ((uint64_t)(uint32_t)V[x] << 32) | (0xFFFFFFFFu - (uint32_t)b);
          bestk = key > bestk ? key : bestk;
        }
      bestk = group_max64<32>(bestk);
      if (fragile || bestk == 0) break;  // left to the exact commit
      int32_t t = (int32_t)(0xFFFFFFFFu - (uint32_t)bestk);
      if (lane == 0) {
        mv_v[w][nm] = v;
        mv_t[w][nm] = t;
        mv_c[w][nm] = (int32_t)c;
        A.spec_v[ob * SPEC_MAX + nm] = v;
        A.spec_t[ob * SPEC_MAX + nm] = t;
      }
      __syncwarp();
      ++nm;
      wB -= c;
    }
    if (i >= hi && wB <= A.cap[B]) sat = 1;
    if (lane == 0) {
      A.spec_n[ob] = nm;
      A.spec_end[ob] = i;
      A.spec_sat[ob] = sat;
    }
    __syncwarp();
  }
}

// A batch with at most WS_E adjacency entries and WS_T table slots is
// evaluated by warp 0 alone, in shared-memory tables, with no CTA barrier.
constexpr int WS_E = 256;
constexpr int WS_T = 2048;
constexpr int WS_R = 4;  // entries per lane whose loads are issued together

// Lowest-id admissible block for a member of weight c (>= 1) with no
// admissible neighbouring block (one warp).  *hint is the lowest block that
// may have room: every block below it has cap - weight < 1.  Blocks only gain
// weight during the commit, except the block being emptied (the commit lowers
// the hint to it when it gets room), so the scan starts there and moves the
// hint up past the full blocks it passes.  The overloaded block B has no room.
constexpr int LA_U = 8;  // chunks of 32 blocks checked per round trip
__device__ int32_t lowest_admissible(const BalArgs &A, int32_t B, int64_t c, int lane, int32_t *hint) {
  int32_t h1 = -1, res = -1;
  for (int32_t base = *hint & ~31; base < A.k && res < 0; base += 32 * LA_U) {
    int32_t room[LA_U];  // cap - weight, clamped to int32 (only >= 1 and >= c matter)
#pragma unroll
    for (int u = 0; u < LA_U; ++u) {
      const int32_t b = base + 32 * u + lane;
      const int32_t bb = b < A.k ? b : A.k - 1;
      const int64_t r = (int64_t)A.cap[bb] - A.bw[bb];
      room[u] = r < INT32_MIN ? INT32_MIN : (r > INT32_MAX ? INT32_MAX : (int32_t)r);
    }
#pragma unroll
    for (int u = 0; u < LA_U; ++u) {
      const int32_t b = base + 32 * u + lane;
      const unsigned m1 = __ballot_sync(0xFFFFFFFFu, b < A.k && room[u] >= 1);
      const unsigned mc = __ballot_sync(0xFFFFFFFFu, b < A.k && b != B && (int64_t)room[u] >= c);
      if (h1 < 0 && m1) h1 = base + 32 * u + __ffs(m1) - 1;
      if (res < 0 && mc) res = base + 32 * u + __ffs(mc) - 1;
    }
  }
  // blocks in [*hint, h1) were seen without room (h1 = k: none has room)
  if (lane == 0) atomicMax(hint, h1 >= 0 ? h1 : A.k);
  __syncwarp();
  return res;
}


// the in-order commit of an evaluated batch (one thread); returns the members
// decided, `stop` when the block fits
__device__ int32_t commit_batch(const BalArgs &A, int32_t B, int32_t nb, const int32_t *s_v, const int32_t *s_t,
                                const int64_t *s_c, const int64_t *s_bwt, const int64_t *s_capt,
                                const uint32_t *s_adj, int64_t E, int32_t &stop, int32_t *hint, int64_t &wB,
                                int32_t capB) {
  // only this CTA changes weights, so the block's and the targets' weights are
  // tracked here (a target's weight is its start weight plus the moves of this
  // batch into it)
  uint32_t moved_mask = 0;
  int32_t j = 0, moves = 0;
  stop = 0;
  for (; j < nb; ++j) {
    if (wB <= capB) {
      stop = 1;
      break;
    }
    const int32_t t = s_t[j];
    const int64_t c = s_c[j];
    int64_t wt = 0;
    if (t >= 0) {
      wt = s_bwt[j];
      for (int32_t x = 0; x < j; ++x)
        if (((moved_mask >> x) & 1u) && s_t[x] == t) wt += s_c[x];
    }
    if (j > 0 && ((s_adj[j] & moved_mask) || (t >= 0 && wt + c > s_capt[j]))) break;
    if (t >= 0) {
      A.part[s_v[j]] = t;
      A.bw[t] = wt + c;
      wB -= c;
      ++moves;
      moved_mask |= 1u << j;
    }
  }
  A.bw[B] = wB;
  if ((int64_t)capB - wB >= 1 && B < *hint) *hint = B;
  if (moves) atomicAdd(A.moved, (unsigned long long)moves);
  atomicAdd(A.moved + 2, 1ull);  // an exact batch
  atomicAdd(A.moved + 3, (unsigned long long)nb);
  atomicAdd(A.moved + 4, (unsigned long long)E);
  return j;
}

// the fixed data of overloaded block o's speculation (lane j: its move j)
struct SpecAhead {
  int32_t B = 0, nm = 0, v = 0, t = 0;
};
__device__ __forceinline__ SpecAhead spec_ahead(const BalArgs &A, int32_t o, int lane) {
  SpecAhead S;
  S.B = A.olist[o];
  S.nm = A.spec_n[o];
  if (lane < S.nm) {
    S.v = A.spec_v[(int64_t)o * SPEC_MAX + lane];
    S.t = A.spec_t[(int64_t)o * SPEC_MAX + lane];
  }
  return S;
}

// Warp 0 drives the commit: it applies the speculated moves that stand,
// sets up every exact batch, and evaluates and commits the small ones alone;
// the whole CTA joins only for a batch beyond WS_E entries or WS_T slots.
__global__ void __launch_bounds__(BM_T) k_bal_moves(BalArgs A, int32_t *inbatch) {
  __shared__ int32_t s_v[BM_W], s_t[BM_W];
  __shared__ int64_t s_c[BM_W], s_eoff[BM_W + 1], s_beg[BM_W], s_bwt[BM_W], s_capt[BM_W];
  __shared__ uint32_t s_adj[BM_W], s_mask[BM_W], s_toff[BM_W + 1];
  __shared__ unsigned long long s_best[BM_W];
  __shared__ int32_t wk[WS_T], wv[WS_T];  // warp 0's tables (empty between batches)
  __shared__ int32_t s_nb, s_B, s_ob, s_i, s_phase, s_done, s_hint, s_capB;
  __shared__ int64_t s_wB;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const uint64_t vmask = (1ull << A.bitsN) - 1ull;
  const uint32_t gcap = A.gcap;  // stride of the per-member table regions
  for (int x = threadIdx.x; x < WS_T; x += BM_T) {
    wk[x] = HT_EMPTY;
    wv[x] = 0;
  }
  if (threadIdx.x == 0) {
    s_ob = 0;
    s_i = 0;
    s_phase = 0;
    s_done = 0;
    s_hint = 0;
  }
  __syncthreads();
  for (;;) {
    if (w == 0) {
      int32_t ob = s_ob, i = s_i, phase = s_phase;
      for (;;) {
        if (phase == 0) {
          // Run ahead over the blocks: a block's speculated moves stand, in
          // order, while their targets still fit under the weights left by
          // the blocks before.  One lane per move checks its target against
          // the current weight plus what the block's earlier moves add to
          // it; the moves before the first that does not fit are applied at
          // once.  Stop at the first block that still needs exact batches.
          // What does not change during the commit (the block, its speculated
          // moves, caps, node weights) is read one block ahead; only the
          // weights are read when the block's turn comes.
          int32_t o = ob, resume = 0;
          SpecAhead nx;
          if (o < A.nover) nx = spec_ahead(A, o, lane);
          for (; o < A.nover; ++o) {
            const SpecAhead cur = nx;
            if (o + 1 < A.nover) nx = spec_ahead(A, o + 1, lane);
            const int32_t B = cur.B, nm = cur.nm, v = cur.v, t = cur.t;
            const int32_t lo = A.seg_lo[B], hi = A.seg_hi[B], capB = A.cap[B];
            const int32_t sat = A.spec_sat[o], send = A.spec_end[o];
            const int64_t bwB = A.bw[B];  // no move below targets B
            int64_t c = 0, bt = 0, ct = 0;
            if (lane < nm) {
              c = bw_node(A, v);
              bt = A.bw[t];
              ct = A.cap[t];
            }
            int64_t pre = 0;  // this block's earlier moves into the same target
#pragma unroll
            for (int j = 0; j < SPEC_MAX; ++j) {
              const int32_t tj = __shfl_sync(0xFFFFFFFFu, t, j);
              const long long cj = __shfl_sync(0xFFFFFFFFu, (long long)c, j);
              if (j < lane && j < nm && tj == t) pre += cj;
            }
            const unsigned bad = __ballot_sync(0xFFFFFFFFu, lane < nm && bt + pre + c > ct);
            const int32_t f = bad ? __ffs(bad) - 1 : nm;  // moves [0, f) stand
            if (lane < f) {
              A.part[v] = t;
              atomicAdd(reinterpret_cast<unsigned long long *>(&A.bw[t]), (unsigned long long)c);
            }
            const int64_t bwB2 = bwB - warp_sum64(lane < f ? c : 0);
            if (lane == 0 && f > 0) {
              A.bw[B] = bwB2;
              if ((int64_t)capB - bwB2 >= 1 && B < s_hint) s_hint = B;  // the block got room
              atomicAdd(A.moved, (unsigned long long)f);
              atomicAdd(A.moved + 1, (unsigned long long)f);  // speculated moves that stood
            }
            __syncwarp();
            resume = f < nm ? lo + f : (sat ? hi : send);
            if (resume < hi && bwB2 > capB) break;  // exact batches take over here
          }
          if (o >= A.nover) {
            if (lane == 0) s_done = 1;
            break;
          }
          ob = o;
          i = resume;
          phase = 1;
        }
        const int32_t B = A.olist[ob];
        const int32_t hi = A.seg_hi[B];
        const int64_t wB = A.bw[B];
        const int32_t capB = A.cap[B];
        if (i >= hi || wB <= capB) {
          ++ob;
          phase = 0;
          continue;
        }
        if (lane == 0) {
          s_wB = wB;  // for the commit, which comes after several warp barriers
          s_capB = capB;
        }
        // the next batch: the shortest prefix of the remaining candidates
        // whose weights cover the overload
        {
          int32_t avail = hi - i < BM_W ? hi - i : BM_W;
          int32_t v = lane < avail ? (int32_t)(A.keys[i + lane] & vmask) : 0;
          int64_t c = lane < avail ? bw_node(A, v) : 0;
          const int64_t rb = lane < avail ? A.xadj[v] : 0;
          int64_t deg = lane < avail ? A.xadj[v + 1] - rb : 0;
          const int64_t own = deg < A.k ? deg : A.k;
          // inclusive prefix sums of weights and degrees
#pragma unroll
          for (int m = 1; m < 32; m <<= 1) {
            int64_t oc = (int64_t)__shfl_up_sync(0xFFFFFFFFu, (unsigned long long)c, m);
            int64_t od = (int64_t)__shfl_up_sync(0xFFFFFFFFu, (unsigned long long)deg, m);
            if (lane >= m) {
              c += oc;
              deg += od;
            }
          }
          unsigned enough = __ballot_sync(0xFFFFFFFFu, lane < avail && c >= wB - capB);
          int32_t nb = enough ? __ffs(enough) : avail;
          // member table sized by the member's own distinct blocks (at most
          // min(degree, k)), so low-degree members never touch a hub-sized
          // table; the tables' slots are numbered across the batch (s_toff)
          uint32_t cap = 32;
          while ((int64_t)cap < 2 * own) cap <<= 1;
          uint32_t tpre = lane < nb ? cap : 0;
#pragma unroll
          for (int m = 1; m < 32; m <<= 1) {
            const uint32_t o = __shfl_up_sync(0xFFFFFFFFu, tpre, m);
            if (lane >= m) tpre += o;
          }
          if (lane < nb) {
            s_v[lane] = v;
            s_beg[lane] = rb;
            s_eoff[lane + 1] = deg;
            s_adj[lane] = 0;
            s_mask[lane] = cap - 1;
            s_toff[lane + 1] = tpre;
            s_best[lane] = 0;
            inbatch[v] = lane + 1;
          }
          if (lane == 0) {
            s_eoff[0] = 0;
            s_toff[0] = 0;
            s_nb = nb;
          }
        }
        __syncwarp();
        const int32_t nb = s_nb;
        const int64_t E = s_eoff[nb];
        const uint32_t TT = s_toff[nb];
        if (E > WS_E || TT > WS_T) {
          if (lane == 0) {
            s_B = B;
            s_ob = ob;
            s_i = i;
          }
          break;  // the whole CTA evaluates this batch
        }
        // ---- warp 0 alone: connectivity tables in shared memory, entries in
        // rounds of WS_R per lane (their loads issued together)
        {
          int32_t j = 0;
          for (int64_t t0 = 0; t0 < E; t0 += 32 * WS_R) {
            int32_t uu[WS_R], wt[WS_R], jm[WS_R];
#pragma unroll
            for (int r = 0; r < WS_R; ++r) {
              const int64_t t = t0 + lane + 32 * r;
              uu[r] = -1;
              if (t < E) {
                while (s_eoff[j + 1] <= t) ++j;
                const int64_t q = s_beg[j] + (t - s_eoff[j]);
                uu[r] = A.adj[q];
                wt[r] = A.ew ? A.ew[q] : 1;
                jm[r] = j;
              }
            }
            int32_t bk[WS_R], ib[WS_R];
#pragma unroll
            for (int r = 0; r < WS_R; ++r)
              if (uu[r] >= 0) {
                bk[r] = A.part[uu[r]];
                ib[r] = inbatch[uu[r]];
              }
#pragma unroll
            for (int r = 0; r < WS_R; ++r)
              if (uu[r] >= 0) {
                if (ib[r] > 0) atomicOr(&s_adj[jm[r]], 1u << (ib[r] - 1));
                ht_add(wk + s_toff[jm[r]], wv + s_toff[jm[r]], s_mask[jm[r]], bk[r], wt[r]);
              }
          }
        }
        __syncwarp();
        // best admissible block of every member, (conn, ~block); the tables
        // are emptied on the way (every table spans whole 32-slot chunks)
        // (the lane that holds a member's best so far also records that
        // block's weight and cap, the target's state at the start of the batch)
        {
          int32_t j = 0;
          for (uint32_t base = 0; base < TT; base += 32) {
            while (s_toff[j + 1] <= base) ++j;
            const uint32_t x = base + lane;
            const int32_t b = wk[x], cv = wv[x];
            wk[x] = HT_EMPTY;
            wv[x] = 0;
            uint64_t key = 0;
            int64_t bwb = 0;
            int32_t capb = 0;
            if (b != HT_EMPTY && b != B) {
              bwb = A.bw[b];
              capb = A.cap[b];
              if (bwb + bw_node(A, s_v[j]) <= capb)
                key = ((uint64_t)(uint32_t)cv << 32) | (0xFFFFFFFFu - (uint32_t)b);
            }
            const uint64_t top = group_max64<32>(key);
            if (top != 0 && key == top && top > s_best[j]) {
              s_best[j] = top;
              s_bwt[j] = bwb;
              s_capt[j] = capb;
            }
            __syncwarp();
          }
        }
        if (lane < nb) {
          const uint64_t bkey = s_best[lane];
          s_t[lane] = bkey ? (int32_t)(0xFFFFFFFFu - (uint32_t)bkey) : -1;
          s_c[lane] = bw_node(A, s_v[lane]);
        }
        __syncwarp();
        for (int32_t j = 0; j < nb; ++j)
          if (s_t[j] < 0) {
            const int32_t t = lowest_admissible(A, B, s_c[j], lane, &s_hint);
            __syncwarp();
            if (lane == 0) {
              s_t[j] = t;
              s_bwt[j] = t >= 0 ? A.bw[t] : 0;
              s_capt[j] = t >= 0 ? A.cap[t] : 0;
            }
            __syncwarp();
          }
        int32_t next = 0, stop = 0;
        if (lane == 0) {
          int64_t w = s_wB;
          next = commit_batch(A, B, nb, s_v, s_t, s_c, s_bwt, s_capt, s_adj, E, stop, &s_hint, w, s_capB);
        }
        next = __shfl_sync(0xFFFFFFFFu, next, 0);
        stop = __shfl_sync(0xFFFFFFFFu, stop, 0);
        if (lane < nb) inbatch[s_v[lane]] = 0;
        __syncwarp();
        i += next;
        if (stop) {
          ++ob;
          phase = 0;
        }
      }
    }
    __syncthreads();
    if (s_done) break;
    // ---- a large batch, evaluated by the whole CTA
    const int32_t B = s_B, nb = s_nb;
    // every table size is a multiple of 32, so a warp's 32 slots lie in one table
    const uint32_t TT = s_toff[nb];
    {
      int32_t j = 0;
      for (uint32_t t = threadIdx.x; t < TT; t += BM_T) {
        while (s_toff[j + 1] <= t) ++j;
        int32_t *K = A.gtab + (int64_t)j * 2 * gcap;
        const uint32_t x = t - s_toff[j];
        K[x] = HT_EMPTY;
        K[gcap + x] = 0;
      }
    }
    __syncthreads();
    const int64_t E = s_eoff[nb];
    {
      int32_t jm = 0;  // this thread's entries only move forward through the members
      for (int64_t base = 0; base < E; base += BM_T) {
        int64_t t = base + threadIdx.x;
        bool ok = t < E;
        if (ok)
          while (s_eoff[jm + 1] <= t) ++jm;
        int32_t blk = HT_EMPTY, wt = 0;
        if (ok) {
          int64_t q = s_beg[jm] + (t - s_eoff[jm]);
          int32_t u = A.adj[q];
          blk = A.part[u];
          wt = A.ew ? A.ew[q] : 1;
          int32_t jj = inbatch[u];
          if (jj > 0) atomicOr(&s_adj[jm], 1u << (jj - 1));
        }
        uint64_t key = ok ? ((uint64_t)(uint32_t)jm << 32) | (uint32_t)blk : ~0ull;
        unsigned peers = __match_any_sync(0xFFFFFFFFu, key);
        int32_t s = __reduce_add_sync(peers, wt);
        if (ok && lane == __ffs(peers) - 1) {
          int32_t *K = A.gtab + (int64_t)jm * 2 * gcap;
          ht_add(K, K + gcap, s_mask[jm], blk, s);
        }
      }
    }
    __syncthreads();
    {
      // best admissible block of every member: (conn, ~block), largest
      // connectivity, then lowest id; a warp's slots belong to one member
      int32_t jj = 0;
      for (uint32_t base = 0; base < TT; base += BM_T) {
        const uint32_t t = base + threadIdx.x;
        if (base + (threadIdx.x & ~31u) >= TT) break;  // warp-uniform
        while (s_toff[jj + 1] <= t) ++jj;
        const int32_t *K = A.gtab + (int64_t)jj * 2 * gcap;
        const uint32_t x = t - s_toff[jj];
        const int32_t b = K[x];
        uint64_t key = 0;
        if (b != HT_EMPTY && b != B && A.bw[b] + bw_node(A, s_v[jj]) <= A.cap[b])
          key = ((uint64_t)(uint32_t)K[gcap + x] << 32) | (0xFFFFFFFFu - (uint32_t)b);
        key = group_max64<32>(key);
        if (lane == 0 && key) atomicMax(&s_best[jj], key);
      }
    }
    __syncthreads();
    if (w < nb) {
      const int64_t c = bw_node(A, s_v[w]);
      const uint64_t bestk = s_best[w];
      int32_t t = bestk ? (int32_t)(0xFFFFFFFFu - (uint32_t)bestk) : -1;
      if (t < 0) t = lowest_admissible(A, B, c, lane, &s_hint);
      if (lane == 0) {
        s_t[w] = t;
        s_c[w] = c;
        s_bwt[w] = t >= 0 ? A.bw[t] : 0;  // the target's weight at the start of the batch
        s_capt[w] = t >= 0 ? A.cap[t] : 0;
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      int32_t stop = 0;
      int64_t wB = A.bw[B];
      const int32_t next =
          commit_batch(A, B, nb, s_v, s_t, s_c, s_bwt, s_capt, s_adj, E, stop, &s_hint, wB, A.cap[B]);
      s_i += next;
      if (stop) {
        ++s_ob;
        s_phase = 0;
      } else {
        s_phase = 1;
      }
    }
    __syncthreads();
    if (threadIdx.x < nb) inbatch[s_v[threadIdx.x]] = 0;
    __syncthreads();
  }
}

int64_t balance(const Graph &g, int32_t k, const int32_t *caps_host, int32_t *part, BalStats *bs) {
  Context &C = ctx();
  cudaStream_t s = C.stream;
  int32_t n = g.n;
  DBuf<int64_t> bw(k);
  block_weights(g, part, k, bw);
  std::vector<int64_t> hbw(k);
  to_host(hbw.data(), bw.p, k);
  std::vector<uint8_t> hover(k, 0);
  std::vector<int32_t> holist;
  int64_t max_room = INT64_MIN;
  for (int32_t b = 0; b < k; ++b) {
    if (hbw[b] > caps_host[b]) {
      hover[b] = 1;
      holist.push_back(b);
    }
    max_room = std::max<int64_t>(max_room, (int64_t)caps_host[b] - hbw[b]);
  }
  if (holist.empty() || n == 0) return 0;
  int bitsN = 1;
  while ((1ll << bitsN) < (int64_t)n) ++bitsN;
  int bitsK = 1;
  while ((1ll << bitsK) < (int64_t)k) ++bitsK;
  DBuf<int32_t> cap(k), ncand(1), seg_lo(k), seg_hi(k);
  DBuf<uint8_t> over(k);
  DBuf<int64_t> cand_d(n);
  DBuf<uint64_t> keys(n), tmp(n), sortbuf(2ll * n);
  // moves, speculated moves that stood, exact batches, their candidates and adjacency entries
  DBuf<unsigned long long> moved(5);
  to_dev(cap.p, caps_host, k);
  to_dev(over.p, hover.data(), k);
  DBuf<int32_t> olist(holist.size());
  to_dev(olist.p, holist.data(), holist.size());
  ncand.zero();
  moved.zero();
  seg_lo.zero();
  seg_hi.zero();
  int64_t dmax = std::min<int64_t>(g.maxdeg, k);
  uint32_t gcap = 32;
  while ((int64_t)gcap < 2 * dmax) gcap <<= 1;
  const int grid = grid_for((int64_t)n * 32, BAL_T, 8);
  int grid_big = 0;
  DBuf<int32_t> gtab;
  BalArgs A;
  A.n = n;
  A.k = k;
  A.xadj = g.xadj;
  A.adj = g.adj;
  A.vw = g.vw;
  A.ew = g.ew;
  A.part = part;
  A.bw = bw;
  A.cap = cap;
  A.over = over;
  A.olist = olist;
  A.nover = (int32_t)holist.size();
  A.max_room = max_room;
  A.cand_d = cand_d;
  A.keys = keys;
  A.ncand = ncand;
  A.bitsN = bitsN;
  A.seg_lo = seg_lo;
  A.seg_hi = seg_hi;
  A.sortbuf = sortbuf;
  A.gtab = nullptr;
  A.gcap = gcap;
  A.moved = moved;
  // nodes with more distinct neighbour blocks than a warp's shared table
  // holds have degree > BAL_STAB / 2, so there are at most m / 257 of them
  DBuf<int32_t> big(g.m / (BAL_STAB / 2 + 1) + 1), nbig(1);
  nbig.zero();
  k_bal_cand<<<grid, BAL_T, 0, s>>>(A, big, nbig);
  KMP_LAUNCHED("bal_cand");
  if (gcap > BAL_STAB) {
    const int32_t nb = read1(nbig.p);
    if (nb > 0) {
      // one CTA per listed node, each with its own global table region,
      // bounded to about 256 MB in all
      int64_t per_cta = 2ll * gcap * (int64_t)sizeof(int32_t);
      int64_t gmax = std::max<int64_t>(1, (256ll << 20) / per_cta);
      grid_big = (int)std::min<int64_t>(std::min<int64_t>(nb, gmax), (int64_t)C.sms * 8);
      gtab.alloc(2ll * gcap * (int64_t)grid_big);
      A.gtab = gtab;
      k_bal_cand_big<<<grid_big, BAL_T, 0, s>>>(A, big, nbig);
      KMP_LAUNCHED("bal_cand_big");
    }
  }
  int32_t N = read1(ncand.p);
  if (N == 0) return 0;
  // grouped by block only: k_bal_sort orders every block's candidates by a
  // strict total order (relative gain, then id), whatever order they arrive in
  radix_sort_u64(keys, tmp, N, bitsK, bitsN);
  k_bal_segments<<<grid_for(N, 256), 256, 0, s>>>(A, N);
  KMP_LAUNCHED("bal_segments");
  k_bal_sort<<<A.nover, BAL_T, 0, s>>>(A);
  KMP_LAUNCHED("bal_sort");
  // speculation over all overloaded blocks (tables as for the candidates)
  int32_t nover = (int32_t)holist.size();
  DBuf<int32_t> spec_v((size_t)nover * SPEC_MAX), spec_t((size_t)nover * SPEC_MAX), spec_n(nover),
      spec_end(nover), spec_sat(nover);
  A.spec_v = spec_v;
  A.spec_t = spec_t;
  A.spec_n = spec_n;
  A.spec_end = spec_end;
  A.spec_sat = spec_sat;
  {
    int sgrid = (int)ceil_div(nover, BAL_W);
    A.gtab = nullptr;
    k_bal_spec<<<sgrid, BAL_T, 0, s>>>(A);
    KMP_LAUNCHED("bal_spec");
  }
  // one global table per warp of the move kernel, and the batch membership marks
  DBuf<int32_t> gtab1(2ll * gcap * BM_W), inbatch(n);
  inbatch.zero();
  A.gtab = gtab1;
  k_bal_moves<<<1, BM_T, 0, s>>>(A, inbatch);
  KMP_LAUNCHED("bal_moves");
  unsigned long long hm[5];
  to_host(hm, moved.p, 5);
  if (bs) {
    bs->over_blocks += nover;
    bs->moves += (int64_t)hm[0];
    bs->spec_moves += (int64_t)hm[1];
    bs->exact_batches += (int64_t)hm[2];
    bs->exact_cands += (int64_t)hm[3];
    bs->exact_entries += (int64_t)hm[4];
  }
  return (int64_t)hm[0];
}

}  // namespace kmp
