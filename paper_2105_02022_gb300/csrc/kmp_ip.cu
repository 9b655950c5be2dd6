// Batched multilevel initial bipartitioning (Section 4.2) and k-way balancing
// (Section 4.3).
#include "kmp_internal.cuh"

namespace kmp {

int32_t bipartition_blocks(const Graph &g, int32_t *part, int32_t nblocks, std::vector<int32_t> &f,
                           double eps, int64_t cV, int32_t k, uint64_t roundkey, int32_t *items_out) {
  fail(KMP_ERR_UNSUPPORTED, "bipartitioner not built yet");
}

int64_t balance(const Graph &g, int32_t k, const int32_t *caps_host, int32_t *part) {
  fail(KMP_ERR_UNSUPPORTED, "balancer not built yet");
}

}  // namespace kmp
