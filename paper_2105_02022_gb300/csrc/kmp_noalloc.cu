// Cut and block weights of a partition without any device allocation.
//
// kmp_cut keeps its per-block accumulators in scratch that the library
// allocates for each call.  Some callers cannot allow that: code whose device
// memory is owned by another runtime (a framework's pool or a fixed arena that
// must account for every byte), processes that pre-reserve all device memory,
// and latency-critical loops that cannot afford the implicit synchronisation
// and possible failure of an allocation at call time.  kmp_cut_noalloc gives
// them the same result with its scratch in a fixed file-scope device array.
//
// The array lives in this file's module.  With lazy module loading (the CUDA
// default) the module, and with it the array's memory, is loaded the first
// time anything in it is used; the library therefore resolves the array's
// address while it initialises on a device (noalloc_prepare, called from the
// first library call there), so that the load happens then and not inside a
// later kmp_cut_noalloc call.
#include <cuda.h>

#include <mutex>

#include "kmp_internal.cuh"

namespace kmp {

// [0] cut, [1] out-of-range flag, [2 .. 2+k) block weights
static __device__ __align__(256) unsigned long long g_noalloc_scratch[KMP_NOALLOC_MAX_K + 2];

namespace {
constexpr int kMaxDevices = 64;
constexpr int kStagedK = 2048;  // block weights staged in shared memory up to this k

// one entry per device: the array's device address and the context it was
// resolved in (a context recreated after cudaDeviceReset has a new id, and the
// address must be looked up again)
struct Slot {
  unsigned long long *ptr = nullptr;
  unsigned long long ctx_id = 0;
};
std::mutex g_mu;
Slot g_slot[kMaxDevices];

typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long *);

// id of the current context (0 when the driver cannot tell); the entry point
// is fetched through the runtime so that the library does not link libcuda
unsigned long long current_ctx_id() {
  static CtxGetIdFn fn = [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      p = nullptr;
    return reinterpret_cast<CtxGetIdFn>(p);
  }();
  unsigned long long id = 0;
  if (fn && fn(nullptr, &id) != CUDA_SUCCESS) id = 0;
  return id;
}

// device address of the scratch array on the current device.  The host-side
// symbol is only a stand-in and never a device address, so it is looked up
// with cudaGetSymbolAddress: once per device (and again only if the device's
// context was recreated).
unsigned long long *scratch_ptr() {
  int dev = 0;
  KMP_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) fail(KMP_ERR_UNSUPPORTED, "device index beyond 64");
  const unsigned long long id = current_ctx_id();
  std::lock_guard<std::mutex> lk(g_mu);
  Slot &s = g_slot[dev];
  if (!s.ptr || s.ctx_id != id) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) fail(KMP_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    s.ptr = static_cast<unsigned long long *>(p);
    s.ctx_id = id;
  }
  return s.ptr;
}
}  // namespace

// called while the library initialises on the current device
void noalloc_prepare() { scratch_ptr(); }

// same row walk as the allocating cut kernel: a warp takes 32 consecutive
// nodes, lanes over each row's entries; for k <= kStagedK each CTA adds its
// block weights in shared memory first, then once per block into scratch
__global__ void __launch_bounds__(256) k_cut_noalloc(int32_t n, int32_t k, const int64_t *xadj,
                                                     const int32_t *adj, const int32_t *vw,
                                                     const int32_t *ew, const int32_t *part,
                                                     unsigned long long *scratch) {
  __shared__ unsigned long long sbw[kStagedK];
  unsigned long long *cut = scratch, *flag = scratch + 1, *bw = scratch + 2;
  const bool staged = k <= kStagedK;
  if (staged)
    for (int i = threadIdx.x; i < k; i += blockDim.x) sbw[i] = 0;
  __syncthreads();
  int lane = threadIdx.x & 31;
  int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  unsigned long long c = 0;
  for (int64_t base = gw * 32; base < n; base += nw * 32) {
    int64_t my = base + lane;
    int32_t p = my < n ? part[my] : -1;
    bool ok = p >= 0 && p < k;
    if (my < n && !ok) atomicOr(flag, 1ull);
    if (ok) {
      unsigned long long w = (unsigned long long)(vw ? vw[my] : 1);
      if (staged) atomicAdd(&sbw[p], w);
      else atomicAdd(&bw[p], w);
    }
    int jmax = (int)(n - base < 32 ? n - base : 32);
    for (int j = 0; j < jmax; ++j) {
      int64_t v = base + j;
      int32_t pv = __shfl_sync(0xFFFFFFFFu, p, j);
      for (int64_t q = xadj[v] + lane; q < xadj[v + 1]; q += 32) {
        int32_t pu = part[adj[q]];
        if (pu != pv) c += (unsigned long long)(ew ? ew[q] : 1);
      }
    }
  }
#pragma unroll
  for (int m = 16; m > 0; m >>= 1) c += __shfl_xor_sync(0xFFFFFFFFu, c, m);
  if (lane == 0 && c) atomicAdd(cut, c);
  if (staged) {
    __syncthreads();
    for (int i = threadIdx.x; i < k; i += blockDim.x)
      if (sbw[i]) atomicAdd(&bw[i], sbw[i]);
  }
}

}  // namespace kmp

using namespace kmp;

extern "C" int kmp_cut_noalloc(const kmp_graph *g, const kmp_vid *part, int32_t k, int64_t *cut_out,
                               int64_t *block_weights_out) {
  try {
    set_last_error("");
    if (!g || !part) fail(KMP_ERR_ARG, "NULL argument");
    if (k < 1 || k > KMP_NOALLOC_MAX_K) fail(KMP_ERR_ARG, "k must lie in [1, KMP_NOALLOC_MAX_K]");
    const Graph &G = g->g;
    cudaStream_t s = ctx().stream;
    unsigned long long *scr = scratch_ptr();
    // the array keeps the previous call's contents: clear what accumulates
    KMP_CUDA(cudaMemsetAsync(scr, 0, (size_t)(k + 2) * sizeof(unsigned long long), s));
    if (G.n > 0) {
      k_cut_noalloc<<<grid_for((int64_t)G.n, 256, 8), 256, 0, s>>>(G.n, k, G.xadj, G.adj, G.vw, G.ew,
                                                                   part, scr);
      KMP_LAUNCHED("cut_noalloc");
    }
    unsigned long long head[2];
    KMP_CUDA(cudaMemcpyAsync(head, scr, sizeof(head), cudaMemcpyDeviceToHost, s));
    if (block_weights_out)
      KMP_CUDA(cudaMemcpyAsync(block_weights_out, scr + 2, (size_t)k * sizeof(int64_t),
                               cudaMemcpyDeviceToHost, s));
    KMP_CUDA(cudaStreamSynchronize(s));
    if (head[1]) fail(KMP_ERR_ARG, "part: value out of range");
    if (cut_out) *cut_out = (int64_t)(head[0] / 2);
    return KMP_OK;
  } catch (const Error &e) {
    set_last_error(e.msg);
    return e.code;
  } catch (...) {
    set_last_error("unknown error");
    return KMP_ERR_CUDA;
  }
}
