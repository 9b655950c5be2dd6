// Internal declarations shared by the CUDA translation units of libkmp.
// Device helpers (counter-based keys, warp reductions, hash tables), the
// library context (stream, configuration, allocator, launch counter), the
// device graph handle and the host-side entry points of each component.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "kmp.h"

namespace kmp {

// ------------------------------------------------------------------ errors
struct Error {
  int code;
  std::string msg;
};

[[noreturn]] void fail(int code, const std::string &msg);
void set_last_error(const std::string &s);  // message kmp_last_error returns
void check_cuda(cudaError_t e, const char *what);
#define KMP_CUDA(call) ::kmp::check_cuda((call), #call)
// after a kernel launch: launch errors only (no sync)
#define KMP_LAUNCHED(name)                   \
  do {                                       \
    ::kmp::check_cuda(cudaGetLastError(), name); \
    ::kmp::ctx().launches++;                 \
  } while (0)

// ----------------------------------------------------------------- context
struct Context {
  cudaStream_t stream = 0;
  kmp_config cfg{};
  int sms = 152;
  int device = 0;
  int64_t launches = 0;
  int *d_status = nullptr;  // device status word: 0 ok, else KMP_ERR_* set by kernels
  // schedule parameters (never change results); see kmp_autotune
  kmp_tuning tune{8, 2048, 2048, 4, 8192, 1, 256, 0};
  // live profiling of the LP rating launches (CUDA events on `stream`)
  bool profile = false;
  cudaStream_t capture_stream = nullptr;  // created on first use: CUDA graph capture of LP rounds
  double prof_rate_ms = 0, prof_rate_bytes = 0;
  int64_t prof_rate_launches = 0;
  double prof_stage_ms = 0, prof_stage_bytes = 0;  // whole rating stage per sub-round
  int64_t prof_stage_spans = 0;
};
Context &ctx();
void ensure_init();
void noalloc_prepare();  // resolves kmp_cut_noalloc's scratch array on the current device
void sync_and_check(const char *what);  // drain the stream and read the status word

// ---------------------------------------------------------- device memory
void *dmalloc(size_t bytes);
void dfree(void *p);

template <class T>
struct DBuf {
  T *p = nullptr;
  size_t n = 0;
  DBuf() = default;
  explicit DBuf(size_t count) { alloc(count); }
  DBuf(const DBuf &) = delete;
  DBuf &operator=(const DBuf &) = delete;
  DBuf(DBuf &&o) noexcept : p(o.p), n(o.n) { o.p = nullptr; o.n = 0; }
  DBuf &operator=(DBuf &&o) noexcept {
    reset();
    p = o.p; n = o.n; o.p = nullptr; o.n = 0;
    return *this;
  }
  ~DBuf() { reset(); }
  void alloc(size_t count) {
    reset();
    n = count;
    p = static_cast<T *>(dmalloc((count > 0 ? count : 1) * sizeof(T)));
  }
  void ensure(size_t count) {
    if (count > n || p == nullptr) alloc(count);
  }
  void zero() { KMP_CUDA(cudaMemsetAsync(p, 0, (n > 0 ? n : 1) * sizeof(T), ctx().stream)); }
  void fill_bytes(int v) { KMP_CUDA(cudaMemsetAsync(p, v, (n > 0 ? n : 1) * sizeof(T), ctx().stream)); }
  void reset() {
    if (p) dfree(p);
    p = nullptr;
    n = 0;
  }
  T *release() { T *q = p; p = nullptr; n = 0; return q; }
  operator T *() const { return p; }
};

template <class T>
void to_host(T *h, const T *d, size_t count) {
  if (count == 0) return;
  KMP_CUDA(cudaMemcpyAsync(h, d, count * sizeof(T), cudaMemcpyDeviceToHost, ctx().stream));
  KMP_CUDA(cudaStreamSynchronize(ctx().stream));
}
template <class T>
void to_dev(T *d, const T *h, size_t count) {
  if (count == 0) return;
  KMP_CUDA(cudaMemcpyAsync(d, h, count * sizeof(T), cudaMemcpyHostToDevice, ctx().stream));
}
template <class T>
T read1(const T *d) {
  T v;
  to_host(&v, d, 1);
  return v;
}

// ------------------------------------------------------------ graph handle
struct Graph {
  int32_t n = 0;
  int64_t m = 0;            // directed entries
  int64_t *xadj = nullptr;  // device
  int32_t *adj = nullptr;
  int32_t *vw = nullptr;    // nullable: unit
  int32_t *ew = nullptr;    // nullable: unit
  int64_t total_vw = 0;     // host copies of graph facts
  int32_t max_vw = 1;
  int64_t maxdeg = 0;
  int64_t n_isolated = 0;
  bool owned = true;
};

// ------------------------------------------------------- counter-based keys
// SplitMix64 finaliser (Steele, Lea, Flood, OOPSLA 2014) chained over words.
__host__ __device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__host__ __device__ __forceinline__ uint64_t key_step(uint64_t x, uint64_t w) {
  return mix64(x ^ mix64(w + 0x9E3779B97F4A7C15ull));
}
inline uint64_t key_of(uint64_t seed, std::initializer_list<uint64_t> words) {
  uint64_t x = mix64(seed + 0x9E3779B97F4A7C15ull);
  for (uint64_t w : words) x = key_step(x, w);
  return x;
}
// MurmurHash3 fmix32 (a bijection of 32-bit words)
__host__ __device__ __forceinline__ uint32_t fmix32(uint32_t h) {
  h ^= h >> 16;
  h *= 0x85EBCA6Bu;
  h ^= h >> 13;
  h *= 0xC2B2AE35u;
  h ^= h >> 16;
  return h;
}
// tie-break rank of a label in one LP round (smaller wins)
__device__ __forceinline__ uint32_t perm32(uint32_t rk_hi, int32_t label) {
  return fmix32((uint32_t)label ^ rk_hi);
}

// domains of the random choices
enum : uint64_t {
  DOM_COARSEN = 1,
  DOM_REFINE = 2,
  DOM_IP = 3,
  DOM_IP_LP = 4,
  DOM_RANDOM = 5,
  DOM_BFS = 6,
  DOM_GGG = 7,
  DOM_REFINE_LEVEL = 8,
  DOM_LEARNED = 9,
  DOM_REPLICA = 10
};

// ----------------------------------------------------------- warp helpers
__device__ __forceinline__ uint64_t shfl_xor64(uint64_t v, int m, int width = 32) {
  uint32_t lo = __shfl_xor_sync(0xFFFFFFFFu, (uint32_t)v, m, width);
  uint32_t hi = __shfl_xor_sync(0xFFFFFFFFu, (uint32_t)(v >> 32), m, width);
  return ((uint64_t)hi << 32) | lo;
}
template <int W>
__device__ __forceinline__ uint64_t group_max64(uint64_t v) {
#pragma unroll
  for (int m = W / 2; m > 0; m >>= 1) {
    uint64_t o = shfl_xor64(v, m, W);
    v = o > v ? o : v;
  }
  return v;
}
__device__ __forceinline__ int64_t warp_sum64(int64_t v) {
#pragma unroll
  for (int m = 16; m > 0; m >>= 1) v += (int64_t)shfl_xor64((uint64_t)v, m);
  return v;
}
__device__ __forceinline__ int32_t warp_sum32(int32_t v) {
#pragma unroll
  for (int m = 16; m > 0; m >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, m);
  return v;
}

// open-addressing (key -> summed weight) table; EMPTY key = -1.  Works on
// shared or global memory through generic pointers.
constexpr int32_t HT_EMPTY = -1;
__device__ __forceinline__ void ht_add(int32_t *keys, int32_t *vals, uint32_t mask, int32_t k,
                                       int32_t w) {
  uint32_t h = fmix32((uint32_t)k) & mask;
  for (uint32_t probe = 0; probe <= mask; ++probe) {
    int32_t old = atomicCAS(&keys[h], HT_EMPTY, k);
    if (old == HT_EMPTY || old == k) {
      atomicAdd(&vals[h], w);
      return;
    }
    h = (h + 1) & mask;
  }
}
__device__ __forceinline__ int32_t ht_get(const int32_t *keys, const int32_t *vals, uint32_t mask,
                                          int32_t k) {
  uint32_t h = fmix32((uint32_t)k) & mask;
  for (uint32_t probe = 0; probe <= mask; ++probe) {
    int32_t c = keys[h];
    if (c == k) return vals[h];
    if (c == HT_EMPTY) return 0;
    h = (h + 1) & mask;
  }
  return 0;
}

__host__ __device__ __forceinline__ int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
inline uint64_t next_pow2(uint64_t x) {
  uint64_t p = 1;
  while (p < x) p <<= 1;
  return p;
}
__device__ __forceinline__ uint32_t next_pow2_dev(int64_t x) {
  uint32_t p = 1;
  while ((int64_t)p < x) p <<= 1;
  return p;
}

// ------------------------------------------------------ shared primitives
// exclusive scan of n values; out[i] = sum in[0..i), *total_dev (device, nullable) = sum
void scan_excl_i32_to_i64(const int32_t *in, int64_t *out, int64_t n, int64_t *total_dev);
void scan_excl_i32(const int32_t *in, int32_t *out, int64_t n, int32_t *total_dev);
// the same on stream s with caller-provided block sums (scan_tmp_count(n) entries):
// no allocation, so it can be captured into a CUDA graph
int64_t scan_tmp_count(int64_t n);
void scan_excl_i32_on(const int32_t *in, int32_t *out, int64_t n, int32_t *total_dev, int32_t *bsum,
                      cudaStream_t s);
void scan_excl_i64(const int64_t *in, int64_t *out, int64_t n, int64_t *total_dev);
void scan_excl_u8_to_i32(const uint8_t *in, int32_t *out, int64_t n, int32_t *total_dev);
// stable LSD radix sort of 64-bit keys by bits [lo_bit, lo_bit + bits) (in place via tmp);
// keys equal in those bits keep their order
void radix_sort_u64(uint64_t *keys, uint64_t *tmp, int64_t n, int bits, int lo_bit = 0);
// same with an int32 payload moved along with each key
void radix_sort_kv(uint64_t *keys, int32_t *vals, uint64_t *tmpk, int32_t *tmpv, int64_t n, int bits,
                   int lo_bit = 0);
int grid_for(int64_t work, int per_block, int max_blocks_per_sm = 8);

// -------------------------------------------------------------- components
struct LPStats {
  int32_t rounds = 0;
  int64_t scanned = 0;
  int64_t moved_total = 0;
  float ms = 0.f;
};

// Size-constrained LP (coarsening when cap == nullptr, else refinement over
// nlab blocks with per-block caps).  label/wt are device arrays that are
// updated in place; fav nullable.
void lp_run(const Graph &g, int32_t *label, int32_t *wt, int32_t nlab, const int32_t *cap,
            int32_t U, int32_t rounds, uint64_t basekey, int32_t *fav, LPStats *st);
// one coarsening level: LP + isolated packing + two-hop; returns #clusters
int32_t cluster_level(const Graph &g, int32_t U, int32_t rounds, uint64_t basekey, bool two_hop,
                      int32_t *label, int32_t *fav_out, LPStats *st, float *ms_other);
// contraction; returns the coarse graph (owned), writes map
Graph contract_graph(const Graph &g, const int32_t *label, int32_t *map);
void free_graph(Graph &g);
void compute_facts(Graph &g);
void project(int32_t n_fine, const int32_t *map, const int32_t *part_c, int32_t *part_f);
// cut and block weights (device out arrays: bw int64[k], cut int64[1])
void cut_and_weights(const Graph &g, const int32_t *part, int32_t k, int64_t *bw_dev,
                     int64_t *cut_dev);
// block weights only (device out int64[k])
void block_weights(const Graph &g, const int32_t *part, int32_t k, int64_t *bw_dev);
// refinement wrapper: caps host int32[k]; returns the cut when want_cut, else 0
int64_t refine(const Graph &g, int32_t k, const int32_t *caps_host, int32_t rounds,
               uint64_t seed, int32_t *part, LPStats *st, bool want_cut = true);
struct BalStats {
  int64_t over_blocks = 0, moves = 0, spec_moves = 0, exact_batches = 0, exact_cands = 0, exact_entries = 0;
};
// k-way balancing; bs (nullable) accumulates where the work went
int64_t balance(const Graph &g, int32_t k, const int32_t *caps_host, int32_t *part, BalStats *bs = nullptr);
// Algorithm 2, one split round; f in/out (host), returns new block count
int32_t bipartition_blocks(const Graph &g, int32_t *part, int32_t nblocks, std::vector<int32_t> &f,
                           double eps, int64_t cV, int32_t k, uint64_t roundkey,
                           int32_t *items_out, const int32_t *caps4 = nullptr);
// caps (host)
void split_caps(double eps, int64_t cV, int32_t k, int64_t cB, int32_t fB, int32_t *t0,
                int32_t *t1, int32_t *L0, int32_t *L1);
int32_t block_cap(double eps, int64_t cV, int32_t k, int32_t fb, int32_t maxc);

}  // namespace kmp

// the opaque handle of include/kmp.h: a device graph
struct kmp_graph {
  kmp::Graph g;
};
