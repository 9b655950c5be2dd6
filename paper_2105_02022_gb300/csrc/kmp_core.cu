// Library context, errors, stream-ordered device allocation and the generic
// device primitives (exclusive scans, stable LSD radix sort) used by the
// partitioner's kernels.
#include <cstdio>
#include <cstring>
#include <mutex>

#include "kmp_internal.cuh"

namespace kmp {

static thread_local std::string g_last_error;
static Context g_ctx;
static std::once_flag g_once;

Context &ctx() { return g_ctx; }

[[noreturn]] void fail(int code, const std::string &msg) { throw Error{code, msg}; }

void check_cuda(cudaError_t e, const char *what) {
  if (e == cudaSuccess) return;
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    fail(KMP_ERR_NOMEM, std::string(what) + ": " + cudaGetErrorString(e));
  }
  fail(KMP_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

void set_last_error(const std::string &s) { g_last_error = s; }
const char *last_error() { return g_last_error.c_str(); }

void ensure_init() {
  std::call_once(g_once, [] {
    kmp_config_default(&g_ctx.cfg);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) dev = 0;
    g_ctx.device = dev;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && sms > 0)
      g_ctx.sms = sms;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
      uint64_t thr = UINT64_MAX;
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
  });
  if (!g_ctx.d_status) {
    void *p = nullptr;
    KMP_CUDA(cudaMalloc(&p, 64));
    KMP_CUDA(cudaMemset(p, 0, 64));
    g_ctx.d_status = static_cast<int *>(p);
    // loads the no-allocation entry point's module (and its fixed scratch
    // array) now, while the library initialises, and records its address
    noalloc_prepare();
  }
}

void sync_and_check(const char *what) {
  KMP_CUDA(cudaStreamSynchronize(g_ctx.stream));
  int st = 0;
  KMP_CUDA(cudaMemcpy(&st, g_ctx.d_status, sizeof(int), cudaMemcpyDeviceToHost));
  if (st != 0) {
    KMP_CUDA(cudaMemset(g_ctx.d_status, 0, sizeof(int)));
    fail(st, std::string(what) + ": device kernel reported status " + std::to_string(st));
  }
}

void *dmalloc(size_t bytes) {
  void *p = nullptr;
  cudaError_t e = cudaMallocAsync(&p, bytes, g_ctx.stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    fail(KMP_ERR_NOMEM, "device allocation of " + std::to_string(bytes) + " bytes failed: " +
                            cudaGetErrorString(e));
  }
  return p;
}

void dfree(void *p) {
  if (p) cudaFreeAsync(p, g_ctx.stream);
}

int grid_for(int64_t work, int per_block, int max_blocks_per_sm) {
  int64_t b = ceil_div(work, per_block);
  int64_t cap = (int64_t)g_ctx.sms * max_blocks_per_sm;
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return (int)b;
}

// ------------------------------------------------------------------ scans
constexpr int SCAN_T = 256;
constexpr int SCAN_IPT = 8;
constexpr int SCAN_TILE = SCAN_T * SCAN_IPT;

template <class Tacc>
__device__ Tacc block_excl_scan(Tacc v, Tacc *total) {
  __shared__ Tacc wsum[SCAN_T / 32];
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  Tacc x = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    Tacc y = __shfl_up_sync(0xFFFFFFFFu, x, d);
    if (lane >= d) x += y;
  }
  if (lane == 31) wsum[w] = x;
  __syncthreads();
  if (w == 0) {
    Tacc s = lane < SCAN_T / 32 ? wsum[lane] : Tacc(0);
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      Tacc y = __shfl_up_sync(0xFFFFFFFFu, s, d);
      if (lane >= d) s += y;
    }
    if (lane < SCAN_T / 32) wsum[lane] = s;
  }
  __syncthreads();
  Tacc base = w > 0 ? wsum[w - 1] : Tacc(0);
  if (total) *total = wsum[SCAN_T / 32 - 1];
  Tacc r = base + x - v;
  __syncthreads();
  return r;
}

template <class Tin, class Tacc>
__global__ void __launch_bounds__(SCAN_T) k_scan_reduce(const Tin *in, int64_t n, Tacc *bsum) {
  int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
  Tacc s = 0;
  for (int i = threadIdx.x; i < SCAN_TILE; i += SCAN_T) {
    int64_t j = base + i;
    if (j < n) s += (Tacc)in[j];
  }
  __shared__ Tacc red[SCAN_T / 32];
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, d);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    Tacc t = 0;
    for (int w = 0; w < SCAN_T / 32; ++w) t += red[w];
    bsum[blockIdx.x] = t;
  }
}

template <class Tacc>
__global__ void __launch_bounds__(SCAN_T) k_scan_bsums(Tacc *bsum, int64_t nb, Tacc *total) {
  __shared__ Tacc carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int64_t off = 0; off < nb; off += SCAN_T) {
    int64_t j = off + threadIdx.x;
    Tacc v = j < nb ? bsum[j] : Tacc(0);
    Tacc tot;
    Tacc ex = block_excl_scan<Tacc>(v, &tot);
    if (j < nb) bsum[j] = ex + carry;
    __syncthreads();
    if (threadIdx.x == 0) carry += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0 && total) *total = carry;
}

template <class Tin, class Tacc, class Tout>
__global__ void __launch_bounds__(SCAN_T) k_scan_down(const Tin *in, Tout *out, int64_t n,
                                                      const Tacc *bsum) {
  int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_IPT;
  Tacc v[SCAN_IPT];
  Tacc s = 0;
#pragma unroll
  for (int i = 0; i < SCAN_IPT; ++i) {
    int64_t j = base + i;
    v[i] = j < n ? (Tacc)in[j] : Tacc(0);
    s += v[i];
  }
  Tacc ex = block_excl_scan<Tacc>(s, nullptr) + bsum[blockIdx.x];
#pragma unroll
  for (int i = 0; i < SCAN_IPT; ++i) {
    int64_t j = base + i;
    if (j < n) out[j] = (Tout)ex;
    ex += v[i];
  }
}

template <class Tin, class Tacc, class Tout>
static void scan_impl(const Tin *in, Tout *out, int64_t n, Tacc *total_dev) {
  int64_t nb = ceil_div(n > 0 ? n : 1, SCAN_TILE);
  DBuf<Tacc> bsum(nb);
  cudaStream_t s = ctx().stream;
  k_scan_reduce<Tin, Tacc><<<(unsigned)nb, SCAN_T, 0, s>>>(in, n, bsum);
  KMP_LAUNCHED("scan_reduce");
  k_scan_bsums<Tacc><<<1, SCAN_T, 0, s>>>(bsum, nb, total_dev);
  KMP_LAUNCHED("scan_bsums");
  if (n > 0) {
    k_scan_down<Tin, Tacc, Tout><<<(unsigned)nb, SCAN_T, 0, s>>>(in, out, n, bsum);
    KMP_LAUNCHED("scan_down");
  }
}

int64_t scan_tmp_count(int64_t n) { return ceil_div(n > 0 ? n : 1, SCAN_TILE); }

void scan_excl_i32_on(const int32_t *in, int32_t *out, int64_t n, int32_t *total_dev, int32_t *bsum,
                      cudaStream_t s) {
  int64_t nb = scan_tmp_count(n);
  k_scan_reduce<int32_t, int32_t><<<(unsigned)nb, SCAN_T, 0, s>>>(in, n, bsum);
  KMP_LAUNCHED("scan_reduce");
  k_scan_bsums<int32_t><<<1, SCAN_T, 0, s>>>(bsum, nb, total_dev);
  KMP_LAUNCHED("scan_bsums");
  if (n > 0) {
    k_scan_down<int32_t, int32_t, int32_t><<<(unsigned)nb, SCAN_T, 0, s>>>(in, out, n, bsum);
    KMP_LAUNCHED("scan_down");
  }
}

void scan_excl_i32_to_i64(const int32_t *in, int64_t *out, int64_t n, int64_t *total_dev) {
  scan_impl<int32_t, int64_t, int64_t>(in, out, n, total_dev);
}
void scan_excl_i32(const int32_t *in, int32_t *out, int64_t n, int32_t *total_dev) {
  scan_impl<int32_t, int32_t, int32_t>(in, out, n, total_dev);
}
void scan_excl_i64(const int64_t *in, int64_t *out, int64_t n, int64_t *total_dev) {
  scan_impl<int64_t, int64_t, int64_t>(in, out, n, total_dev);
}
void scan_excl_u8_to_i32(const uint8_t *in, int32_t *out, int64_t n, int32_t *total_dev) {
  scan_impl<uint8_t, int32_t, int32_t>(in, out, n, total_dev);
}

// ------------------------------------------------------------ radix sort
constexpr int RS_T = 256;
constexpr int RS_SUB = 8;                // sub-tiles of RS_T keys per tile
constexpr int RS_TILE = RS_T * RS_SUB;   // keys per tile (one CTA)

// digit histogram of every tile (2048 keys)
__global__ void __launch_bounds__(RS_T) k_rs_hist(const uint64_t *keys, int64_t n, int sh,
                                                  int32_t *cnt, int64_t ntiles) {
  __shared__ int32_t h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * RS_TILE;
#pragma unroll
  for (int r = 0; r < RS_SUB; ++r) {
    const int64_t j = base + r * RS_T + threadIdx.x;
    if (j < n) atomicAdd(&h[(keys[j] >> sh) & 255u], 1);
  }
  __syncthreads();
  cnt[(int64_t)threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

// Stable scatter of one tile: its sub-tiles in order, inside a sub-tile warps
// in order and lanes in order (ranks from match-any groups), on top of the
// digit's running count over the tile's earlier sub-tiles.
__global__ void __launch_bounds__(RS_T) k_rs_scatter(const uint64_t *keys, uint64_t *out,
                                                     int64_t n, int sh, const int32_t *off,
                                                     int64_t ntiles, const int32_t *vin = nullptr,
                                                     int32_t *vout = nullptr) {
  __shared__ int32_t wc[RS_T / 32][256];
  __shared__ int32_t run[256];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  run[threadIdx.x] = off[(int64_t)threadIdx.x * ntiles + blockIdx.x];
  const int64_t base = (int64_t)blockIdx.x * RS_TILE;
  for (int r = 0; r < RS_SUB; ++r) {
    for (int i = threadIdx.x; i < (RS_T / 32) * 256; i += RS_T) (&wc[0][0])[i] = 0;
    __syncthreads();
    const int64_t j = base + r * RS_T + threadIdx.x;
    const bool ok = j < n;
    const uint64_t k = ok ? keys[j] : 0;
    const int d = ok ? (int)((k >> sh) & 255u) : 256 + lane;  // unique dummy digit for padding lanes
    const unsigned peers = __match_any_sync(0xFFFFFFFFu, d);
    const int rank = __popc(peers & ((1u << lane) - 1u));
    if (ok && rank == 0) wc[w][d] = __popc(peers);
    __syncthreads();
    // per digit (thread t handles digit t): exclusive prefix over warps on
    // top of the running position, which then moves past this sub-tile
    {
      const int dd = threadIdx.x;
      int32_t s = run[dd];
      for (int ww = 0; ww < RS_T / 32; ++ww) {
        const int32_t c = wc[ww][dd];
        wc[ww][dd] = s;
        s += c;
      }
      run[dd] = s;
    }
    __syncthreads();
    if (ok) {
      const int64_t p = (int64_t)wc[w][d] + rank;
      out[p] = k;
      if (vin) vout[p] = vin[j];
    }
    __syncthreads();  // wc is cleared for the next sub-tile
  }
}

void radix_sort_u64(uint64_t *keys, uint64_t *tmp, int64_t n, int bits, int lo_bit) {
  if (n <= 1 || bits <= 0) return;
  int64_t ntiles = ceil_div(n, RS_TILE);
  DBuf<int32_t> cnt(256 * ntiles), off(256 * ntiles);
  cudaStream_t s = ctx().stream;
  uint64_t *a = keys, *b = tmp;
  int passes = (bits + 7) / 8;
  for (int p = 0; p < passes; ++p) {
    int sh = lo_bit + 8 * p;
    k_rs_hist<<<(unsigned)ntiles, RS_T, 0, s>>>(a, n, sh, cnt, ntiles);
    KMP_LAUNCHED("rs_hist");
    scan_excl_i32(cnt, off, 256 * ntiles, nullptr);
    k_rs_scatter<<<(unsigned)ntiles, RS_T, 0, s>>>(a, b, n, sh, off, ntiles);
    KMP_LAUNCHED("rs_scatter");
    uint64_t *t = a; a = b; b = t;
  }
  if (a != keys) KMP_CUDA(cudaMemcpyAsync(keys, a, n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
}

void radix_sort_kv(uint64_t *keys, int32_t *vals, uint64_t *tmpk, int32_t *tmpv, int64_t n, int bits,
                   int lo_bit) {
  if (n <= 1 || bits <= 0) return;
  int64_t ntiles = ceil_div(n, RS_TILE);
  DBuf<int32_t> cnt(256 * ntiles), off(256 * ntiles);
  cudaStream_t s = ctx().stream;
  uint64_t *a = keys, *b = tmpk;
  int32_t *va = vals, *vb = tmpv;
  int passes = (bits + 7) / 8;
  for (int p = 0; p < passes; ++p) {
    int sh = lo_bit + 8 * p;
    k_rs_hist<<<(unsigned)ntiles, RS_T, 0, s>>>(a, n, sh, cnt, ntiles);
    KMP_LAUNCHED("rs_hist");
    scan_excl_i32(cnt, off, 256 * ntiles, nullptr);
    k_rs_scatter<<<(unsigned)ntiles, RS_T, 0, s>>>(a, b, n, sh, off, ntiles, va, vb);
    KMP_LAUNCHED("rs_scatter");
    uint64_t *t = a; a = b; b = t;
    int32_t *tv = va; va = vb; vb = tv;
  }
  if (a != keys) {
    KMP_CUDA(cudaMemcpyAsync(keys, a, n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
    KMP_CUDA(cudaMemcpyAsync(vals, va, n * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
  }
}

}  // namespace kmp
