// Contraction (Section 2, "Multilevel Graph Partitioning"): each cluster
// becomes one coarse node whose weight is the sum of its members' weights;
// the coarse edge between two clusters carries the summed weight of the fine
// edges between them; edges inside a cluster vanish.
//
// GPU layout: coarse ids = exclusive scan of "label used" flags (ascending
// label); members grouped by a counting sort.  A coarse node whose members'
// total degree is <= 512 is aggregated by one warp in a shared-memory hash
// table (four bins by size: 64, 128, 256, 512) and sorted by a warp bitonic
// network; one whose total degree is <= 8192 by one CTA in a shared-memory
// table sized for it (three bins: 2048, 4096, 8192), ordered by a bitmap rank
// or a block bitonic network; larger rows are aggregated by all their
// members' warps in parallel into global tables, and the distinct entries of
// all large rows are ordered by one GPU-wide key-value radix sort of
// (row, neighbour).  Rows go to temporary space at upper-bound offsets; a
// prefix sum of the row lengths then places them into the final CSR.
// Also: projection (Algorithm 1), cut and block weights (Section 2), and the
// per-graph facts the other kernels need (max degree, isolated nodes, weights).
#include "kmp_internal.cuh"

namespace kmp {

constexpr int CW_UB = 512;            // warp path: members' total degree <= CW_UB
constexpr int CB_UB = 8192;           // block path: members' total degree <= CB_UB
constexpr int NCLASS = 8;             // four warp bins, three block bins, global path
constexpr int CLS_GLOBAL = NCLASS - 1;

// row class by members' total degree ub: warp bins 64 / 128 / 256 / 512, block
// bins 2048 / 4096 / 8192, then the global path
__host__ __device__ __forceinline__ int row_class(unsigned long long ub) {
  return ub <= 64ull    ? 0
         : ub <= 128ull  ? 1
         : ub <= 256ull  ? 2
         : ub <= (unsigned long long)CW_UB ? 3
         : ub <= 2048ull ? 4
         : ub <= 4096ull ? 5
         : ub <= 8192ull ? 6
                         : CLS_GLOBAL;
}

__global__ void k_map_used(int32_t n, const int32_t *label, uint8_t *used) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x)
    used[label[v]] = 1;
}

__global__ void k_map(int32_t n, const int32_t *label, const int32_t *cid, int32_t *map) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x)
    map[v] = cid[label[v]];
}

__global__ void k_contract_prep(int32_t n, const int64_t *xadj, const int32_t *vw,
                                const int32_t *map, int32_t *cvw, int32_t *csize,
                                unsigned long long *cub) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    int32_t x = map[v];
    atomicAdd(&cvw[x], vw ? vw[v] : 1);
    atomicAdd(&csize[x], 1);
    atomicAdd(&cub[x], (unsigned long long)(xadj[v + 1] - xadj[v]));
  }
}

__global__ void k_members(int32_t n, const int32_t *map, const int32_t *moff, int32_t *mcur,
                          int32_t *members) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    int32_t x = map[v];
    members[moff[x] + atomicAdd(&mcur[x], 1)] = (int32_t)v;
  }
}

// split coarse nodes by row class: list c holds its rows at lists + c * nc
__global__ void k_split_ub(int32_t nc, const unsigned long long *cub, int32_t *lists, int32_t *counts) {
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < nc;
       x += (int64_t)gridDim.x * blockDim.x) {
    int c = row_class(cub[x]);
    lists[(int64_t)c * nc + atomicAdd(&counts[c], 1)] = (int32_t)x;
  }
}

__global__ void k_ub_to_i64(int32_t nc, const unsigned long long *cub, int64_t *ub64) {
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < nc;
       x += (int64_t)gridDim.x * blockDim.x)
    ub64[x] = (int64_t)cub[x];
}

// bitonic sort (ascending) of P = power-of-two entries by `nt` cooperating
// threads with index t; sync() separates the steps
template <bool BLOCK>
__device__ __forceinline__ void bitonic(uint64_t *a, uint32_t P, uint32_t t, uint32_t nt) {
  for (uint32_t k = 2; k <= P; k <<= 1) {
    for (uint32_t j = k >> 1; j > 0; j >>= 1) {
      for (uint32_t i = t; i < P; i += nt) {
        uint32_t l = i ^ j;
        if (l > i) {
          uint64_t x = a[i], y = a[l];
          bool up = (i & k) == 0;
          if ((x > y) == up) {
            a[i] = y;
            a[l] = x;
          }
        }
      }
      if (BLOCK) __syncthreads();
      else __syncwarp();
    }
  }
}

// warp path: one coarse node per warp for rows whose members' total degree
// ub is at most TABW / 2.  The table packs (neighbour << 32 | weight) per slot
// (key and weight updated as the two 32-bit halves), is sized to the power of
// two >= 2 ub, and is compacted in place into the sort list, since every entry
// moves to a slot at or below its own.  Up to 32 members at a time spread
// their edges over the lanes (a warp prefix sum of their degrees; each lane
// finds the member of its edge by a five-step search over the prefixes).
template <int TABW, int WARPS>
__global__ void __launch_bounds__(WARPS * 32) k_aggregate_warp(
    const int32_t *list, int32_t nrows, const unsigned long long *cub, const int64_t *xadj,
    const int32_t *adj, const int32_t *ew, const int32_t *map, const int32_t *members,
    const int32_t *moff, const int64_t *toff, int32_t *tadj, int32_t *tw, int32_t *cdeg) {
  __shared__ uint64_t tab[WARPS][TABW];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint64_t *T = tab[w];
  int32_t *H = reinterpret_cast<int32_t *>(T);  // H[2 j] weight, H[2 j + 1] key of slot j
  const int64_t gw = (int64_t)blockIdx.x * WARPS + w, nw = (int64_t)gridDim.x * WARPS;
  for (int64_t i = gw; i < nrows; i += nw) {
    const int32_t x = list[i];
    const uint32_t ub = (uint32_t)cub[x];
    uint32_t tsz = 64;
    while (tsz < 2 * ub) tsz <<= 1;
    const uint32_t mask = tsz - 1;
    for (uint32_t j = lane; j < tsz; j += 32) T[j] = (uint64_t)(uint32_t)HT_EMPTY << 32;
    __syncwarp();
    const int32_t m1 = moff[x + 1];
    for (int32_t c0 = moff[x]; c0 < m1; c0 += 32) {
      int32_t d = 0;
      int64_t b = 0;
      if (c0 + lane < m1) {
        int32_t v = members[c0 + lane];
        b = xadj[v];
        d = (int32_t)(xadj[v + 1] - b);
      }
      int32_t inc = d;
      for (int o = 1; o < 32; o <<= 1) {
        int32_t t = __shfl_up_sync(0xFFFFFFFFu, inc, o);
        if (lane >= o) inc += t;
      }
      const int32_t tot = __shfl_sync(0xFFFFFFFFu, inc, 31);
      for (int32_t e0 = 0; e0 < tot; e0 += 32) {
        const int32_t e = e0 + lane;
        int32_t j = 0;  // members before the owner of edge e: their inclusive prefix is <= e
        for (int st = 16; st > 0; st >>= 1) {
          int32_t t = __shfl_sync(0xFFFFFFFFu, inc, j + st - 1);
          if (t <= e) j += st;
        }
        int64_t bj = __shfl_sync(0xFFFFFFFFu, b, j & 31);
        int32_t ej = __shfl_sync(0xFFFFFFFFu, inc - d, j & 31);
        if (e < tot) {
          int64_t q = bj + (e - ej);
          int32_t y = map[adj[q]];
          if (y != x) {
            int32_t wq = ew ? ew[q] : 1;
            uint32_t h = fmix32((uint32_t)y) & mask;
            for (uint32_t probe = 0; probe <= mask; ++probe) {
              int32_t old = atomicCAS(&H[2 * h + 1], HT_EMPTY, y);
              if (old == HT_EMPTY || old == y) {
                atomicAdd(&H[2 * h], wq);
                break;
              }
              h = (h + 1) & mask;
            }
          }
        }
      }
    }
    __syncwarp();
    // in-place compaction: entry j goes to slot cnt + rank <= j
    int32_t cnt = 0;
    for (uint32_t j0 = 0; j0 < tsz; j0 += 32) {
      uint64_t ent = T[j0 + lane];
      bool has = (int32_t)(ent >> 32) != HT_EMPTY;
      unsigned bal = __ballot_sync(0xFFFFFFFFu, has);
      __syncwarp();
      if (has) T[cnt + __popc(bal & ((1u << lane) - 1u))] = ent;
      cnt += __popc(bal);
      __syncwarp();
    }
    uint32_t P = 1;
    while (P < (uint32_t)cnt) P <<= 1;
    for (uint32_t j = cnt + lane; j < P; j += 32) T[j] = ~0ull;
    __syncwarp();
    bitonic<false>(T, P, lane, 32);
    const int64_t o = toff[x];
    for (int32_t j = lane; j < cnt; j += 32) {
      tadj[o + j] = (int32_t)(T[j] >> 32);
      tw[o + j] = (int32_t)(uint32_t)T[j];
    }
    if (lane == 0) cdeg[x] = cnt;
    __syncwarp();
  }
}

template <int TABW, int WARPS>
void launch_aggregate_warp(const int32_t *list, int32_t nrows, const unsigned long long *cub, const Graph &g,
                           const int32_t *map, const int32_t *members, const int32_t *moff,
                           const int64_t *toff, int32_t *tadj, int32_t *tw, int32_t *cdeg) {
  static_assert(TABW >= 64 && TABW * WARPS * sizeof(uint64_t) <= 48 * 1024, "bin shape");
  constexpr int per_sm_smem = (int)((227u << 10) / (TABW * WARPS * sizeof(uint64_t) + 1024));
  constexpr int per_sm = per_sm_smem < 64 / WARPS ? per_sm_smem : 64 / WARPS;
  k_aggregate_warp<TABW, WARPS><<<grid_for(nrows, WARPS, per_sm), WARPS * 32, 0, ctx().stream>>>(
      list, nrows, cub, g.xadj, g.adj, g.ew, map, members, moff, toff, tadj, tw, cdeg);
  KMP_LAUNCHED("aggregate_warp");
}

// block path: one coarse node per CTA for rows whose members' total degree ub
// is at most TAB / 2.  The row's table is the power of two >= 2 ub (load
// factor <= 1/2); its distinct entries (at most ub) are sorted by neighbour id.
// The members' edges are spread evenly over all NT threads (up to NT members
// at a time: a prefix sum of their degrees, each thread finds the member of
// its edge by binary search), so one high-degree member does not serialise
// the row on one warp.  Ordering: when the row's neighbour ids span at most
// 32 TAB values (and not far more than the entries), each entry's position is
// the number of smaller ids, read from a bitmap of the span and a prefix sum
// of its word popcounts (the freed table is the space); else the entries are
// sorted by a block bitonic network.
// exclusive prefix sum of v over the NT threads of the block (all threads call it)
template <int NT>
__device__ __forceinline__ int32_t block_scan_excl(int32_t v, int32_t *s_wsum /* NT / 32 */) {
  constexpr int NW = NT / 32;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int32_t inc = v;
  for (int o = 1; o < 32; o <<= 1) {
    int32_t t = __shfl_up_sync(0xFFFFFFFFu, inc, o);
    if (lane >= o) inc += t;
  }
  if (lane == 31) s_wsum[w] = inc;
  __syncthreads();
  if (w == 0) {
    int32_t t = lane < NW ? s_wsum[lane] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      int32_t u = __shfl_up_sync(0xFFFFFFFFu, t, o);
      if (lane >= o) t += u;
    }
    if (lane < NW) s_wsum[lane] = t;
  }
  __syncthreads();
  int32_t r = inc - v + (w > 0 ? s_wsum[w - 1] : 0);
  __syncthreads();  // s_wsum may be reused
  return r;
}

template <int TAB, int NT>
constexpr size_t cta_smem_bytes() {
  return (size_t)TAB / 2 * sizeof(uint64_t) + (size_t)TAB * 2 * sizeof(int32_t);
}

template <int TAB, int NT>
__global__ void __launch_bounds__(NT) k_aggregate_cta(
    const int32_t *list, int32_t nrows, const unsigned long long *cub, const int64_t *xadj,
    const int32_t *adj, const int32_t *ew, const int32_t *map, const int32_t *members,
    const int32_t *moff, const int64_t *toff, int32_t *tadj, int32_t *tw, int32_t *cdeg) {
  extern __shared__ __align__(16) unsigned char cta_smem[];
  uint64_t *L = reinterpret_cast<uint64_t *>(cta_smem);      // TAB / 2 sort entries
  int32_t *K = reinterpret_cast<int32_t *>(L + TAB / 2);     // TAB keys
  int32_t *V = K + TAB;                                       // TAB weights
  __shared__ int32_t s_cnt, s_ymin, s_ymax;
  __shared__ int32_t s_pre[NT + 1];
  __shared__ int64_t s_b[NT];
  __shared__ int32_t s_wsum[NT / 32];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  for (int32_t i = blockIdx.x; i < nrows; i += gridDim.x) {
    int32_t x = list[i];
    uint32_t ub = (uint32_t)cub[x];
    uint32_t tsz = 64;
    while (tsz < 2 * ub) tsz <<= 1;
    for (uint32_t j = tid; j < tsz; j += NT) {
      K[j] = HT_EMPTY;
      V[j] = 0;
    }
    if (tid == 0) {
      s_cnt = 0;
      s_ymin = INT32_MAX;
      s_ymax = -1;
    }
    __syncthreads();
    const int32_t m1 = moff[x + 1];
    for (int32_t c0 = moff[x]; c0 < m1; c0 += NT) {
      const int32_t cn = m1 - c0 < NT ? m1 - c0 : NT;
      int32_t d = 0;
      int64_t b = 0;
      if (tid < cn) {
        int32_t v = members[c0 + tid];
        b = xadj[v];
        d = (int32_t)(xadj[v + 1] - b);
      }
      s_pre[tid + 1] = block_scan_excl<NT>(d, s_wsum) + d;
      s_b[tid] = b;
      if (tid == 0) s_pre[0] = 0;
      __syncthreads();
      const int32_t tot = s_pre[cn];
      for (int32_t e = tid; e < tot; e += NT) {
        int32_t lo = 0, hi = cn - 1;  // the last member whose prefix is <= e owns edge e
        while (lo < hi) {
          int32_t mid = (lo + hi + 1) >> 1;
          if (s_pre[mid] <= e) lo = mid;
          else hi = mid - 1;
        }
        int64_t q = s_b[lo] + (e - s_pre[lo]);
        int32_t y = map[adj[q]];
        if (y != x) ht_add(K, V, tsz - 1, y, ew ? ew[q] : 1);
      }
      __syncthreads();  // the next chunk rewrites the prefix
    }
    // compact into L (order arbitrary; tsz is a multiple of 32)
    for (uint32_t j0 = (uint32_t)w * 32; j0 < tsz; j0 += NT) {
      uint32_t j = j0 + lane;
      bool has = K[j] != HT_EMPTY;
      unsigned bal = __ballot_sync(0xFFFFFFFFu, has);
      int32_t p0 = 0;
      if (lane == 0 && bal) p0 = atomicAdd(&s_cnt, __popc(bal));
      p0 = __shfl_sync(0xFFFFFFFFu, p0, 0);
      if (has) L[p0 + __popc(bal & ((1u << lane) - 1u))] = ((uint64_t)(uint32_t)K[j] << 32) | (uint32_t)V[j];
      int32_t mn = __reduce_min_sync(0xFFFFFFFFu, has ? K[j] : INT32_MAX);
      int32_t mx = __reduce_max_sync(0xFFFFFFFFu, has ? K[j] : -1);
      if (lane == 0 && bal) {
        atomicMin(&s_ymin, mn);
        atomicMax(&s_ymax, mx);
      }
    }
    __syncthreads();
    const int32_t cnt = s_cnt, ymin = s_ymin;
    uint32_t P = 1;
    while (P < (uint32_t)cnt) P <<= 1;
    const int32_t W = cnt > 0 ? ((s_ymax - ymin) >> 5) + 1 : 0;
    int64_t o = toff[x];
    if (W <= TAB && (uint32_t)W <= 16 * P) {
      uint32_t *Bm = reinterpret_cast<uint32_t *>(K);  // bitmap of ids ymin.. (W words)
      int32_t *Pf = V;                                 // popcount prefix per word
      for (int32_t j = tid; j < W; j += NT) Bm[j] = 0;
      __syncthreads();
      for (int32_t j = tid; j < cnt; j += NT) {
        int32_t d = (int32_t)(L[j] >> 32) - ymin;
        atomicOr(&Bm[d >> 5], 1u << (d & 31));
      }
      __syncthreads();
      const int32_t seg = (W + NT - 1) / NT, a = tid * seg < W ? tid * seg : W, b = a + seg < W ? a + seg : W;
      int32_t loc = 0;
      for (int32_t j = a; j < b; ++j) loc += __popc(Bm[j]);
      int32_t base = block_scan_excl<NT>(loc, s_wsum);
      for (int32_t j = a; j < b; ++j) {
        Pf[j] = base;
        base += __popc(Bm[j]);
      }
      __syncthreads();
      for (int32_t j = tid; j < cnt; j += NT) {
        uint64_t ent = L[j];
        int32_t y = (int32_t)(ent >> 32), d = y - ymin;
        int32_t r = Pf[d >> 5] + __popc(Bm[d >> 5] & ((1u << (d & 31)) - 1u));
        tadj[o + r] = y;
        tw[o + r] = (int32_t)(uint32_t)ent;
      }
    } else {
      for (uint32_t j = cnt + tid; j < P; j += NT) L[j] = ~0ull;
      __syncthreads();
      bitonic<true>(L, P, tid, NT);
      for (int32_t j = tid; j < cnt; j += NT) {
        tadj[o + j] = (int32_t)(L[j] >> 32);
        tw[o + j] = (int32_t)(uint32_t)L[j];
      }
    }
    if (tid == 0) cdeg[x] = cnt;
    __syncthreads();  // the next row reuses the tables and the counter
  }
}

template <int TAB, int NT>
void launch_aggregate_cta(const int32_t *list, int32_t nrows, const unsigned long long *cub, const Graph &g,
                          const int32_t *map, const int32_t *members, const int32_t *moff,
                          const int64_t *toff, int32_t *tadj, int32_t *tw, int32_t *cdeg) {
  static_assert(TAB / 2 >= NT && TAB % NT == 0, "bin shape");
  constexpr size_t bytes = cta_smem_bytes<TAB, NT>();
  static bool attr = false;
  if (!attr) {
    KMP_CUDA(cudaFuncSetAttribute(k_aggregate_cta<TAB, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)bytes));
    attr = true;
  }
  int per_sm = (int)((227u << 10) / (bytes + 1024));
  if (per_sm < 1) per_sm = 1;
  int blocks = std::min<int64_t>(nrows, (int64_t)ctx().sms * per_sm);
  k_aggregate_cta<TAB, NT><<<blocks, NT, bytes, ctx().stream>>>(list, nrows, cub, g.xadj, g.adj, g.ew, map,
                                                                members, moff, toff, tadj, tw, cdeg);
  KMP_LAUNCHED("aggregate_cta");
}

// ---- large rows (members' total degree > CW_UB)
__global__ void k_large_sizes(int32_t nc, const unsigned long long *cub, int64_t *tsz) {
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < nc;
       x += (int64_t)gridDim.x * blockDim.x) {
    unsigned long long ub = cub[x];
    if (ub <= (unsigned long long)CB_UB) {
      tsz[x] = 0;
    } else {
      int64_t d = (int64_t)ub < nc ? (int64_t)ub : nc;  // distinct neighbours < nc
      int64_t c = 32;
      while (c < 2 * d) c <<= 1;
      tsz[x] = c;
    }
  }
}

// work units: chunks of LARGE_CHUNK entries of the rows of members of large
// coarse nodes (so one very high-degree member is spread over many warps)
constexpr int64_t LARGE_CHUNK = 512;

__global__ void k_large_chunks(int32_t n, const int64_t *xadj, const int32_t *map,
                               const unsigned long long *cub, int64_t *nch) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x)
    nch[v] = cub[map[v]] > (unsigned long long)CB_UB ? ceil_div(xadj[v + 1] - xadj[v], LARGE_CHUNK) : 0;
}

// the node owning every chunk
__global__ void k_large_owner(int32_t n, const int64_t *nch, const int64_t *choff, int32_t *owner) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x)
    for (int64_t c = 0; c < nch[v]; ++c) owner[choff[v] + c] = (int32_t)v;
}

__global__ void __launch_bounds__(256) k_large_insert(int64_t total, const int32_t *owner, const int64_t *choff,
                                                      const int64_t *xadj, const int32_t *adj,
                                                      const int32_t *ew, const int32_t *map,
                                                      const int64_t *ltoff, const int64_t *tsz, int32_t *lk,
                                                      int32_t *lv) {
  int lane = threadIdx.x & 31;
  int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t c = gw; c < total; c += nw) {
    int32_t v = owner[c], x = map[v];
    int32_t *K = lk + ltoff[x], *V = lv + ltoff[x];
    uint32_t mask = (uint32_t)(tsz[x] - 1);
    int64_t b = xadj[v] + (c - choff[v]) * LARGE_CHUNK;
    int64_t e = b + LARGE_CHUNK < xadj[v + 1] ? b + LARGE_CHUNK : xadj[v + 1];
    for (int64_t q = b + lane; q < e; q += 32) {
      int32_t y = map[adj[q]];
      if (y != x) ht_add(K, V, mask, y, ew ? ew[q] : 1);
    }
  }
}

// Tables are powers of two >= 32 laid out back to back, so every aligned tile
// of 32 entries belongs to one row: the row of every tile (a warp per large
// row writes its tiles)
__global__ void k_large_tiles(const int32_t *large_list, const int32_t *nlarge, const int64_t *ltoff,
                              const int64_t *tsz, int32_t *tile_row) {
  int lane = threadIdx.x & 31;
  int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = gw; i < *nlarge; i += nw) {
    int32_t x = large_list[i];
    for (int64_t t = ltoff[x] / 32 + lane; t < (ltoff[x] + tsz[x]) / 32; t += 32) tile_row[t] = x;
  }
}

// distinct entries of every large row into its own temporary row (positions
// within the row from its entry counter; the row is sorted afterwards)
__global__ void __launch_bounds__(256) k_large_compact(int64_t LT, const int32_t *tile_row,
                                                       const int32_t *lk, const int32_t *lv,
                                                       const int64_t *toff, int32_t *tadj, int32_t *tw,
                                                       int32_t *cdeg) {
  int lane = threadIdx.x & 31;
  int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t t = gw; t * 32 < LT; t += nw) {
    int64_t e = t * 32;
    int32_t x = tile_row[t];
    int32_t y = lk[e + lane];
    bool has = y != HT_EMPTY;
    unsigned bal = __ballot_sync(0xFFFFFFFFu, has);
    if (bal == 0) continue;
    int32_t p0 = 0;
    if (lane == 0) p0 = atomicAdd(&cdeg[x], __popc(bal));
    p0 = __shfl_sync(0xFFFFFFFFu, p0, 0);
    if (has) {
      const int64_t p = toff[x] + p0 + __popc(bal & ((1u << lane) - 1u));
      tadj[p] = y;
      tw[p] = lv[e + lane];
    }
  }
}

// large rows by their distinct entries: up to SORT_S (one CTA of 256 threads
// sorts in shared memory), up to SORT_L (1024 threads), more (radix sort)
constexpr int32_t SORT_S = 2048;
constexpr int32_t SORT_L = 16384;
__global__ void k_large_split(const int32_t *rows, const int32_t *nrows, const int32_t *cdeg, int32_t cap,
                              int32_t *lists, int32_t *counts) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < *nrows;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t x = rows[i], d = cdeg[x];
    const int c = d <= SORT_S ? 0 : d <= SORT_L ? 1 : 2;
    lists[(int64_t)c * cap + atomicAdd(&counts[c], 1)] = x;
  }
}

// one CTA per row: (neighbour << 32 | weight) sorted in shared memory; the
// neighbours of a row are distinct, so the order is by neighbour
template <int P, int NT>
__global__ void __launch_bounds__(NT) k_large_sort_smem(const int32_t *rows, int32_t nrows, const int64_t *toff,
                                                        const int32_t *cdeg, int32_t *tadj, int32_t *tw) {
  extern __shared__ uint64_t srt[];  // P entries
  const uint32_t tid = threadIdx.x;
  for (int64_t i = blockIdx.x; i < nrows; i += gridDim.x) {
    const int32_t x = rows[i];
    const int64_t o = toff[x];
    const int32_t d = cdeg[x];
    uint32_t Q = 32;
    while ((int32_t)Q < d) Q <<= 1;
    for (uint32_t j = tid; j < Q; j += NT)
      srt[j] = (int32_t)j < d ? ((uint64_t)(uint32_t)tadj[o + j] << 32) | (uint32_t)tw[o + j] : ~0ull;
    __syncthreads();
    bitonic<true>(srt, Q, tid, NT);
    for (uint32_t j = tid; (int32_t)j < d; j += NT) {
      tadj[o + j] = (int32_t)(srt[j] >> 32);
      tw[o + j] = (int32_t)(uint32_t)srt[j];
    }
    __syncthreads();  // the next row reuses the array
  }
}

template <int P, int NT>
void launch_large_sort_smem(const int32_t *rows, int32_t nrows, const int64_t *toff, const int32_t *cdeg,
                            int32_t *tadj, int32_t *tw) {
  constexpr size_t bytes = (size_t)P * sizeof(uint64_t);
  static bool attr = false;
  if (!attr) {
    KMP_CUDA(cudaFuncSetAttribute(k_large_sort_smem<P, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)bytes));
    attr = true;
  }
  int per_sm = (int)((227u << 10) / (bytes + 1024));
  if (per_sm < 1) per_sm = 1;
  if (per_sm > 2048 / NT) per_sm = 2048 / NT;
  int blocks = std::min<int64_t>(nrows, (int64_t)ctx().sms * per_sm);
  k_large_sort_smem<P, NT><<<blocks, NT, bytes, ctx().stream>>>(rows, nrows, toff, cdeg, tadj, tw);
  KMP_LAUNCHED("large_sort_smem");
}

// rows too long for shared memory: their entries as (rank << bits | neighbour,
// weight), a warp per row, at the row's offset among them
__global__ void k_large_gather(const int32_t *rows, int32_t nrows, const int64_t *boff, const int64_t *toff,
                               const int32_t *tadj, const int32_t *tw, const int32_t *cdeg, int bits,
                               uint64_t *ek, int32_t *ev) {
  const int lane = threadIdx.x & 31;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = gw; r < nrows; r += nw) {
    const int32_t x = rows[r], d = cdeg[x];
    const int64_t o = toff[x], b = boff[r];
    for (int32_t j = lane; j < d; j += 32) {
      ek[b + j] = ((uint64_t)r << bits) | (uint64_t)(uint32_t)tadj[o + j];
      ev[b + j] = tw[o + j];
    }
  }
}

// The longer rows' entries (rank r << bits | neighbour) are ordered by a
// counting sort on (r, neighbour >> SEG_LO): every such segment holds at most
// 2^SEG_LO distinct neighbours of one row, and one CTA then sorts it in shared
// memory by the low bits.
constexpr int SEG_LO = 14;
static_assert((1 << SEG_LO) == SORT_L, "a segment fits the larger shared-memory sort");
__global__ void k_seg_hist(int64_t N, const uint64_t *ek, int bits, int32_t *hist) {
  const int hb = bits - SEG_LO;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t k = ek[i];
    atomicAdd(&hist[((k >> bits) << hb) | ((k & ((1ull << bits) - 1ull)) >> SEG_LO)], 1);
  }
}
__global__ void k_seg_scatter(int64_t N, const uint64_t *ek, const int32_t *ev, int bits, const int32_t *off,
                              int32_t *cur, uint64_t *ek2, int32_t *ev2) {
  const int hb = bits - SEG_LO;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t k = ek[i];
    const int64_t x = (int64_t)(((k >> bits) << hb) | ((k & ((1ull << bits) - 1ull)) >> SEG_LO));
    const int64_t p = (int64_t)off[x] + atomicAdd(&cur[x], 1);
    ek2[p] = k;
    ev2[p] = ev[i];
  }
}
// non-empty segments by size: up to SORT_S entries (list 0) and up to SORT_L (list 1)
__global__ void k_seg_split(int64_t X, const int32_t *hist, int32_t *lists, int32_t *counts, int64_t cap) {
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < X;
       x += (int64_t)gridDim.x * blockDim.x) {
    const int32_t len = hist[x];
    if (len == 0) continue;
    const int c = len <= SORT_S ? 0 : 1;
    lists[(int64_t)c * cap + atomicAdd(&counts[c], 1)] = (int32_t)x;
  }
}
// one CTA per segment: (low SEG_LO bits << 32 | weight) sorted in shared memory
template <int P, int NT>
__global__ void __launch_bounds__(NT) k_seg_sort(const int32_t *segs, int32_t nseg, const int32_t *off,
                                                 const int32_t *hist, uint64_t *ek, int32_t *ev) {
  extern __shared__ uint64_t srt[];  // P entries
  const uint32_t tid = threadIdx.x;
  const uint64_t lo_mask = (1ull << SEG_LO) - 1ull;
  for (int64_t i = blockIdx.x; i < nseg; i += gridDim.x) {
    const int32_t x = segs[i];
    const int64_t o = off[x];
    const int32_t d = hist[x];
    const uint64_t hi = ek[o] & ~lo_mask;
    uint32_t Q = 32;
    while ((int32_t)Q < d) Q <<= 1;
    for (uint32_t j = tid; j < Q; j += NT)
      srt[j] = (int32_t)j < d ? ((ek[o + j] & lo_mask) << 32) | (uint32_t)ev[o + j] : ~0ull;
    __syncthreads();
    bitonic<true>(srt, Q, tid, NT);
    for (uint32_t j = tid; (int32_t)j < d; j += NT) {
      ek[o + j] = hi | (srt[j] >> 32);
      ev[o + j] = (int32_t)(uint32_t)srt[j];
    }
    __syncthreads();  // the next segment reuses the array
  }
}
template <int P, int NT>
void launch_seg_sort(const int32_t *segs, int32_t nseg, const int32_t *off, const int32_t *hist, uint64_t *ek,
                     int32_t *ev) {
  constexpr size_t bytes = (size_t)P * sizeof(uint64_t);
  static bool attr = false;
  if (!attr) {
    KMP_CUDA(cudaFuncSetAttribute(k_seg_sort<P, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    attr = true;
  }
  int per_sm = (int)((227u << 10) / (bytes + 1024));
  if (per_sm < 1) per_sm = 1;
  if (per_sm > 2048 / NT) per_sm = 2048 / NT;
  int blocks = std::min<int64_t>(nseg, (int64_t)ctx().sms * per_sm);
  k_seg_sort<P, NT><<<blocks, NT, bytes, ctx().stream>>>(segs, nseg, off, hist, ek, ev);
  KMP_LAUNCHED("seg_sort");
}

// sorted entries back into their rows (rank r's entries fill [boff[r], boff[r + 1]))
__global__ void k_large_place(int64_t N, const uint64_t *ek, const int32_t *ev, int bits, const int32_t *rows,
                              const int64_t *boff, const int64_t *toff, int32_t *tadj, int32_t *tw) {
  const uint64_t mask = (1ull << bits) - 1ull;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = (int64_t)(ek[i] >> bits);
    const int64_t p = toff[rows[r]] + (i - boff[r]);
    tadj[p] = (int32_t)(ek[i] & mask);
    tw[p] = ev[i];
  }
}

__global__ void k_gather_deg(const int32_t *rows, int32_t nrows, const int32_t *cdeg, int64_t *out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nrows;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = cdeg[rows[i]];
}

// rows from their upper-bound offsets into the final CSR; four loads per lane
// are issued before their stores
__global__ void k_copy_rows(int32_t nc, const int64_t *__restrict__ toff, const int64_t *__restrict__ cx,
                            const int32_t *__restrict__ tadj, const int32_t *__restrict__ tw,
                            int32_t *__restrict__ adj, int32_t *__restrict__ ew) {
  int lane = threadIdx.x & 31;
  int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t x = gw; x < nc; x += nw) {
    int64_t o = toff[x], p = cx[x], d = cx[x + 1] - p;
    for (int64_t j = lane; j < d; j += 128) {
      int32_t a[4], c[4];
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (j + 32 * u < d) {
          a[u] = tadj[o + j + 32 * u];
          c[u] = tw[o + j + 32 * u];
        }
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (j + 32 * u < d) {
          adj[p + j + 32 * u] = a[u];
          ew[p + j + 32 * u] = c[u];
        }
    }
  }
}

__global__ void k_set_last_i64(int64_t *a, int64_t idx, const int64_t *v) { a[idx] = *v; }

// graph facts: max degree, isolated nodes, max and total node weight, total edge weight
__global__ void k_graph_facts(int32_t n, const int64_t *xadj, const int32_t *vw,
                              unsigned long long *out /* [maxdeg, iso, maxvw, totvw] */) {
  unsigned long long md = 0, iso = 0, mw = 0, tw = 0;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    unsigned long long d = (unsigned long long)(xadj[v + 1] - xadj[v]);
    md = d > md ? d : md;
    iso += d == 0;
    unsigned long long w = vw ? (unsigned long long)vw[v] : 1ull;
    mw = w > mw ? w : mw;
    tw += w;
  }
#pragma unroll
  for (int m = 16; m > 0; m >>= 1) {
    unsigned long long a = __shfl_xor_sync(0xFFFFFFFFu, md, m);
    md = a > md ? a : md;
    iso += __shfl_xor_sync(0xFFFFFFFFu, iso, m);
    unsigned long long b = __shfl_xor_sync(0xFFFFFFFFu, mw, m);
    mw = b > mw ? b : mw;
    tw += __shfl_xor_sync(0xFFFFFFFFu, tw, m);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(&out[0], md);
    atomicAdd(&out[1], iso);
    atomicMax(&out[2], mw);
    atomicAdd(&out[3], tw);
  }
}

void compute_facts(Graph &g) {
  DBuf<unsigned long long> f(4);
  f.zero();
  k_graph_facts<<<grid_for(g.n, 256), 256, 0, ctx().stream>>>(g.n, g.xadj, g.vw, f);
  KMP_LAUNCHED("graph_facts");
  unsigned long long h[4];
  to_host(h, f.p, 4);
  g.maxdeg = (int64_t)h[0];
  g.n_isolated = (int64_t)h[1];
  g.max_vw = (int32_t)h[2];
  g.total_vw = (int64_t)h[3];
}

void free_graph(Graph &g) {
  if (g.owned) {
    dfree(g.xadj);
    dfree(g.adj);
    dfree(g.vw);
    dfree(g.ew);
  }
  g = Graph();
}

Graph contract_graph(const Graph &g, const int32_t *label, int32_t *map) {
  Context &C = ctx();
  cudaStream_t s = C.stream;
  int32_t n = g.n;
  int grid = grid_for(n, 256);
  DBuf<uint8_t> used(n);
  used.zero();
  DBuf<int32_t> cid(n), ncd(1);
  k_map_used<<<grid, 256, 0, s>>>(n, label, used);
  KMP_LAUNCHED("map_used");
  scan_excl_u8_to_i32(used, cid, n, ncd);
  k_map<<<grid, 256, 0, s>>>(n, label, cid, map);
  KMP_LAUNCHED("map");
  int32_t nc = read1(ncd.p);

  Graph out;
  out.n = nc;
  out.owned = true;
  DBuf<int32_t> cvw(nc), csize(nc + 1), moff(nc + 1), mcur(nc), members(n);
  DBuf<unsigned long long> cub(nc);
  cvw.zero();
  csize.zero();
  mcur.zero();
  cub.zero();
  k_contract_prep<<<grid, 256, 0, s>>>(n, g.xadj, g.vw, map, cvw, csize, cub);
  KMP_LAUNCHED("contract_prep");
  scan_excl_i32(csize, moff, nc + 1, nullptr);
  k_members<<<grid, 256, 0, s>>>(n, map, moff, mcur, members);
  KMP_LAUNCHED("members");
  // temporary rows at upper-bound offsets
  DBuf<int64_t> ub64(nc + 1), toff(nc + 1), ttot(1);
  int gridc = grid_for(nc, 256);
  k_ub_to_i64<<<gridc, 256, 0, s>>>(nc, cub, ub64);
  KMP_LAUNCHED("ub_copy");
  scan_excl_i64(ub64, toff, nc, ttot);
  int64_t tot = read1(ttot.p);
  DBuf<int32_t> tadj(tot), tw(tot), cdeg(nc + 1);
  cdeg.zero();
  DBuf<int32_t> lists((int64_t)NCLASS * nc), counts(NCLASS);
  counts.zero();
  k_split_ub<<<gridc, 256, 0, s>>>(nc, cub, lists, counts);
  KMP_LAUNCHED("split_ub");
  int32_t hc[NCLASS];
  to_host(hc, counts.p, NCLASS);
  const int32_t *large_list = lists.p + (int64_t)CLS_GLOBAL * nc;
  auto L = [&](int c) { return lists.p + (int64_t)c * nc; };
  if (hc[4] > 0) launch_aggregate_cta<4096, 256>(L(4), hc[4], cub, g, map, members, moff, toff, tadj, tw, cdeg);
  if (hc[5] > 0) launch_aggregate_cta<8192, 512>(L(5), hc[5], cub, g, map, members, moff, toff, tadj, tw, cdeg);
  if (hc[6] > 0)
    launch_aggregate_cta<16384, 1024>(L(6), hc[6], cub, g, map, members, moff, toff, tadj, tw, cdeg);
  if (hc[0] > 0) launch_aggregate_warp<128, 8>(L(0), hc[0], cub, g, map, members, moff, toff, tadj, tw, cdeg);
  if (hc[1] > 0) launch_aggregate_warp<256, 8>(L(1), hc[1], cub, g, map, members, moff, toff, tadj, tw, cdeg);
  if (hc[2] > 0) launch_aggregate_warp<512, 8>(L(2), hc[2], cub, g, map, members, moff, toff, tadj, tw, cdeg);
  if (hc[3] > 0) launch_aggregate_warp<1024, 4>(L(3), hc[3], cub, g, map, members, moff, toff, tadj, tw, cdeg);
  if (hc[CLS_GLOBAL] > 0) {
    // large rows: every member inserts in parallel into its coarse node's global
    // table; each row's distinct entries are compacted into its temporary row
    // and sorted there by neighbour: in shared memory by one CTA per row when
    // they fit; the longer rows' entries by a key-value radix sort of (row
    // rank, neighbour's high bits) and then per segment in shared memory
    int bits = 1;
    while ((1ll << bits) < (int64_t)nc) ++bits;
    DBuf<int64_t> tsz(nc), ltoff(nc), ltot(1);
    k_large_sizes<<<gridc, 256, 0, s>>>(nc, cub, tsz);
    KMP_LAUNCHED("large_sizes");
    scan_excl_i64(tsz, ltoff, nc, ltot);
    int64_t LT = read1(ltot.p);
    DBuf<int32_t> lk(LT), lv(LT);
    lk.fill_bytes(0xFF);
    lv.zero();
    DBuf<int64_t> nch(n), choff(n), chtot(1);
    k_large_chunks<<<grid, 256, 0, s>>>(n, g.xadj, map, cub, nch);
    KMP_LAUNCHED("large_chunks");
    scan_excl_i64(nch, choff, n, chtot);
    int64_t CT = read1(chtot.p);
    DBuf<int32_t> owner(CT + 1);
    k_large_owner<<<grid, 256, 0, s>>>(n, nch, choff, owner);
    KMP_LAUNCHED("large_owner");
    k_large_insert<<<grid_for(CT * 32, 256, 8), 256, 0, s>>>(CT, owner, choff, g.xadj, g.adj, g.ew, map,
                                                             ltoff, tsz, lk, lv);
    KMP_LAUNCHED("large_insert");
    DBuf<int32_t> tile_row(LT / 32 + 1);
    k_large_tiles<<<grid_for((int64_t)hc[CLS_GLOBAL] * 32, 256), 256, 0, s>>>(large_list, counts.p + CLS_GLOBAL, ltoff, tsz,
                                                                     tile_row);
    KMP_LAUNCHED("large_tiles");
    k_large_compact<<<grid_for(LT, 256, 8), 256, 0, s>>>(LT, tile_row, lk, lv, toff, tadj, tw, cdeg);
    KMP_LAUNCHED("large_compact");
    const int32_t nlarge = hc[CLS_GLOBAL];
    DBuf<int32_t> slists(3ll * nlarge), scounts(3);
    scounts.zero();
    k_large_split<<<grid_for(nlarge, 256), 256, 0, s>>>(large_list, counts.p + CLS_GLOBAL, cdeg, nlarge, slists,
                                                       scounts);
    KMP_LAUNCHED("large_split");
    int32_t sc[3];
    to_host(sc, scounts.p, 3);
    if (sc[0] > 0) launch_large_sort_smem<SORT_S, 256>(slists.p, sc[0], toff, cdeg, tadj, tw);
    if (sc[1] > 0) launch_large_sort_smem<SORT_L, 1024>(slists.p + nlarge, sc[1], toff, cdeg, tadj, tw);
    if (sc[2] > 0) {
      const int32_t nbig = sc[2];
      const int32_t *brows = slists.p + 2ll * nlarge;
      DBuf<int64_t> bdeg(nbig), boff(nbig), btot(1);
      k_gather_deg<<<grid_for(nbig, 256), 256, 0, s>>>(brows, nbig, cdeg, bdeg);
      KMP_LAUNCHED("gather_deg");
      scan_excl_i64(bdeg, boff, nbig, btot);
      const int64_t NE = read1(btot.p);
      DBuf<uint64_t> ek(NE), ektmp(NE);
      DBuf<int32_t> ev(NE), evtmp(NE);
      k_large_gather<<<grid_for((int64_t)nbig * 32, 256), 256, 0, s>>>(brows, nbig, boff, toff, tadj, tw, cdeg,
                                                                      bits, ek, ev);
      KMP_LAUNCHED("large_gather");
      // counting sort by (rank, neighbour >> SEG_LO), then every segment by the
      // low bits in shared memory (a row above SORT_L entries has more than
      // 2^SEG_LO distinct neighbours, so bits > SEG_LO here)
      const int hb = bits - SEG_LO;
      const int64_t X = (int64_t)nbig << hb;
      if (X > (int64_t)INT32_MAX / 2) {
        // counters beyond int32 indexing (coarse graphs near 2^31 nodes): one
        // key-value radix sort of (rank, neighbour) instead
        int rbits = 1;
        while ((1ll << rbits) < (int64_t)nbig) ++rbits;
        radix_sort_kv(ek, ev, ektmp, evtmp, NE, rbits + bits);
        KMP_CUDA(cudaMemcpyAsync(ektmp, ek, NE * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
        KMP_CUDA(cudaMemcpyAsync(evtmp, ev, NE * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
      } else {
        DBuf<int32_t> hist(X), off(X), cur(X), htot(1);
        hist.zero();
        cur.zero();
        k_seg_hist<<<grid_for(NE, 256), 256, 0, s>>>(NE, ek, bits, hist);
        KMP_LAUNCHED("seg_hist");
        scan_excl_i32(hist, off, X, htot);
        k_seg_scatter<<<grid_for(NE, 256), 256, 0, s>>>(NE, ek, ev, bits, off, cur, ektmp, evtmp);
        KMP_LAUNCHED("seg_scatter");
        DBuf<int32_t> slists(2 * X), scnt(2);
        scnt.zero();
        k_seg_split<<<grid_for(X, 256), 256, 0, s>>>(X, hist, slists, scnt, X);
        KMP_LAUNCHED("seg_split");
        int32_t sc2[2];
        to_host(sc2, scnt.p, 2);
        if (sc2[0] > 0) launch_seg_sort<SORT_S, 256>(slists.p, sc2[0], off, hist, ektmp, evtmp);
        if (sc2[1] > 0) launch_seg_sort<SORT_L, 1024>(slists.p + X, sc2[1], off, hist, ektmp, evtmp);
      }
      k_large_place<<<grid_for(NE, 256), 256, 0, s>>>(NE, ektmp, evtmp, bits, brows, boff, toff, tadj, tw);
      KMP_LAUNCHED("large_place");
    }
  }
  DBuf<int64_t> mtot(1);
  out.xadj = static_cast<int64_t *>(dmalloc((nc + 1) * sizeof(int64_t)));
  scan_excl_i32_to_i64(cdeg, out.xadj, nc, mtot);
  k_set_last_i64<<<1, 1, 0, s>>>(out.xadj, nc, mtot);
  KMP_LAUNCHED("set_last");
  out.m = read1(mtot.p);
  out.adj = static_cast<int32_t *>(dmalloc((out.m > 0 ? out.m : 1) * sizeof(int32_t)));
  out.ew = static_cast<int32_t *>(dmalloc((out.m > 0 ? out.m : 1) * sizeof(int32_t)));
  if (nc > 0) {
    k_copy_rows<<<grid_for((int64_t)nc * 32, 256), 256, 0, s>>>(nc, toff, out.xadj, tadj, tw,
                                                                out.adj, out.ew);
    KMP_LAUNCHED("copy_rows");
  }
  out.vw = cvw.release();
  compute_facts(out);
  return out;
}

__global__ void k_project(int32_t n, const int32_t *map, const int32_t *pc, int32_t *pf) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x)
    pf[v] = pc[map[v]];
}

void project(int32_t n_fine, const int32_t *map, const int32_t *part_c, int32_t *part_f) {
  k_project<<<grid_for(n_fine, 256), 256, 0, ctx().stream>>>(n_fine, map, part_c, part_f);
  KMP_LAUNCHED("project");
}

// Each warp takes 32 consecutive nodes and walks their rows one after the
// other with its lanes over the entries (balanced for any degree mix); block
// weights are accumulated in shared memory when k is small.
constexpr int CUT_SBW = 2048;
__global__ void __launch_bounds__(256) k_cut_bw(int32_t n, int32_t k, const int64_t *xadj,
                                                const int32_t *adj, const int32_t *vw, const int32_t *ew,
                                                const int32_t *part, unsigned long long *bw,
                                                unsigned long long *cut) {
  __shared__ unsigned long long sbw[CUT_SBW];
  bool local = k <= CUT_SBW;
  if (local)
    for (int i = threadIdx.x; i < k; i += blockDim.x) sbw[i] = 0;
  __syncthreads();
  int lane = threadIdx.x & 31;
  int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  unsigned long long c = 0;
  for (int64_t base = gw * 32; base < n; base += nw * 32) {
    int64_t my = base + lane;
    int32_t p = my < n ? part[my] : -1;
    if (p >= 0) {
      unsigned long long w = (unsigned long long)(vw ? vw[my] : 1);
      if (local) atomicAdd(&sbw[p], w);
      else atomicAdd(&bw[p], w);
    }
    int jmax = (int)(n - base < 32 ? n - base : 32);
    for (int j = 0; j < jmax; ++j) {
      int64_t v = base + j;
      int32_t pv = __shfl_sync(0xFFFFFFFFu, p, j);
      for (int64_t q = xadj[v] + lane; q < xadj[v + 1]; q += 32)
        if (part[adj[q]] != pv) c += (unsigned long long)(ew ? ew[q] : 1);
    }
  }
#pragma unroll
  for (int m = 16; m > 0; m >>= 1) c += __shfl_xor_sync(0xFFFFFFFFu, c, m);
  if (lane == 0 && c) atomicAdd(cut, c);
  __syncthreads();
  if (local)
    for (int i = threadIdx.x; i < k; i += blockDim.x)
      if (sbw[i]) atomicAdd(&bw[i], sbw[i]);
}

__global__ void k_half(int64_t *c) { *c /= 2; }

// block weights only (no edge traffic)
__global__ void __launch_bounds__(256) k_bw_only(int32_t n, int32_t k, const int32_t *vw,
                                                 const int32_t *part, unsigned long long *bw) {
  __shared__ unsigned long long sbw[CUT_SBW];
  bool local = k <= CUT_SBW;
  if (local)
    for (int i = threadIdx.x; i < k; i += blockDim.x) sbw[i] = 0;
  __syncthreads();
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    unsigned long long w = (unsigned long long)(vw ? vw[v] : 1);
    if (local) atomicAdd(&sbw[part[v]], w);
    else atomicAdd(&bw[part[v]], w);
  }
  __syncthreads();
  if (local)
    for (int i = threadIdx.x; i < k; i += blockDim.x)
      if (sbw[i]) atomicAdd(&bw[i], sbw[i]);
}

void block_weights(const Graph &g, const int32_t *part, int32_t k, int64_t *bw_dev) {
  cudaStream_t s = ctx().stream;
  KMP_CUDA(cudaMemsetAsync(bw_dev, 0, (size_t)k * sizeof(int64_t), s));
  if (g.n == 0) return;
  k_bw_only<<<grid_for(g.n, 256, 4), 256, 0, s>>>(g.n, k, g.vw, part,
                                                  reinterpret_cast<unsigned long long *>(bw_dev));
  KMP_LAUNCHED("bw_only");
}

void cut_and_weights(const Graph &g, const int32_t *part, int32_t k, int64_t *bw_dev,
                     int64_t *cut_dev) {
  cudaStream_t s = ctx().stream;
  KMP_CUDA(cudaMemsetAsync(bw_dev, 0, (size_t)k * sizeof(int64_t), s));
  KMP_CUDA(cudaMemsetAsync(cut_dev, 0, sizeof(int64_t), s));
  k_cut_bw<<<grid_for((int64_t)g.n, 256, 8), 256, 0, s>>>(
      g.n, k, g.xadj, g.adj, g.vw, g.ew, part, reinterpret_cast<unsigned long long *>(bw_dev),
      reinterpret_cast<unsigned long long *>(cut_dev));
  KMP_LAUNCHED("cut_bw");
  k_half<<<1, 1, 0, s>>>(cut_dev);
  KMP_LAUNCHED("half");
}

}  // namespace kmp
