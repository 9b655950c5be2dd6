/*
 * kmp.h -- C ABI of the GB300 (sm_103a) deep multilevel graph partitioner.
 *
 * Problem (Section 2, "Notation and Definitions"): an undirected graph
 * G = (V, E, c, w) with positive integer node weights c and edge weights w is
 * split into k blocks V_1..V_k, every block obeying the balance constraint
 * c(V_i) <= L, while the cut (total weight of edges between blocks) is
 * minimised.  The method is deep multilevel graph partitioning (Section 3,
 * Algorithm 1 and 2) with size-constrained label propagation for coarsening
 * and refinement (Section 4.1, 4.3), contraction (Section 2) and multilevel
 * recursive bipartitioning of the blocks (Section 4.2).  Every step runs in
 * CUDA kernels on one GPU; there is no CPU fallback.
 *
 * Graphs are CSR: xadj[n+1] (int64 offsets), adjncy[xadj[n]] (int32 ids),
 * vwgt[n] and adjwgt[xadj[n]] (int32, > 0; NULL means all ones).  The CSR must
 * be symmetric with equal weights in both directions and no self-loops.
 * Limits: n < 2^31, sum of node weights < 2^31, sum of edge weights over
 * undirected edges < 2^31 (every rating and gain then fits in int32).
 *
 * Results are deterministic for fixed (input, k, eps, seed, config) and equal,
 * bit for bit, to those of the project's CPU oracle.
 *
 * Errors: every entry point returns KMP_OK (0) or a negative code; the text of
 * the last error of the calling thread is available from kmp_last_error().  No
 * C++ exception crosses this boundary.  Device pointers are plain
 * cudaMalloc-style global memory pointers on the current device; all work is
 * issued on the stream set with kmp_set_stream (default: the legacy stream)
 * and every call returns after that stream has drained, unless noted.
 */
#ifndef KMP_H
#define KMP_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t kmp_vid; /* vertex id */
typedef int64_t kmp_eid; /* CSR offset */
typedef int32_t kmp_wgt; /* node / edge weight */

#define KMP_OK 0
#define KMP_ERR_ARG -1         /* invalid argument or CSR */
#define KMP_ERR_NOMEM -2       /* device or host allocation failed */
#define KMP_ERR_CUDA -3        /* a CUDA call or kernel failed */
#define KMP_ERR_TIMEOUT -4     /* a bounded device wait expired */
#define KMP_ERR_INFEASIBLE -5  /* result violates L_k (result still written) */
#define KMP_ERR_UNSUPPORTED -6 /* input beyond a documented limit */

/*
 * Parameters of the method.  Values the paper gives: lp_rounds = 5 and
 * refine_rounds = 5 (Section 4.1, 4.3).  The others are readings of passages
 * the paper leaves open (C is not given; "the same value used in KaHIP" for
 * the bipartitioner's cluster cap; the number of portfolio repetitions; FM
 * details); kmp_config_default documents the defaults.
 */
typedef struct {
  int32_t C;             /* coarsening stops at <= 2C nodes; k_i = ceil2(n_i/C) (default 160) */
  int32_t lp_rounds;     /* coarsening LP rounds (5) */
  int32_t refine_rounds; /* refinement LP rounds (5) */
  int32_t subrounds;     /* S deterministic sub-rounds per LP round, power of two (8) */
  int32_t two_hop;       /* two-hop clustering on/off (1) */
  int32_t conv_num;      /* coarsening converged when conv_den*n' > conv_num*n (19) */
  int32_t conv_den;      /* (20) */
  int32_t ip_C;          /* bipartitioner cluster cap floor(c(B)/ip_C) (16) */
  int32_t ip_lp_rounds;  /* LP rounds per bipartitioner level (5) */
  int32_t rep_random;    /* portfolio repetitions: random (4) */
  int32_t rep_bfs;       /* BFS (4) */
  int32_t rep_ggg;       /* greedy graph growing (8) */
  int32_t fm_passes;     /* 2-way FM passes per level (8) */
  int32_t fm_stop;       /* fruitless FM moves that end a pass (64) */
  int32_t learned;       /* learned mode (0 = off), with the proposer set by kmp_set_proposer:
                            1: the proposal seeds one bipartition of each item's coarsest graph
                            first, then a reduced portfolio runs; the rest of the plain portfolio
                            runs only if the best so far is infeasible;
                            2: the proposal is made on the item graph itself and refined there by
                            2-way FM, skipping the item's coarsening and portfolio; the plain
                            method runs only if that breaks a cap */
  int32_t lrep_random;   /* learned-mode repetitions (each at most its rep_*): random (0) */
  int32_t lrep_bfs;      /* BFS (0) */
  int32_t lrep_ggg;      /* greedy graph growing (1) */
  int32_t replicas;      /* R, a power of two in 1..64 (1 = off): the coarsest graph is taken by
                            two copies, each coarsened further and partitioned on its own with
                            R/2 under its own seed, and the better partition is kept (feasible
                            first, then the smaller cut); coarsening stops at max(R, 2) C nodes
                            (Section 3, "Parallelization", with R in the role of the PEs) */
  int32_t adaptive;      /* 1: adaptive portfolio (plain mode only): the first ceil(R/2) runs of
                            every algorithm, then the rest only of algorithms whose feasible cuts
                            have mean - 2 sd <= the best feasible cut so far (Section 4.2, the
                            adaptive algorithm selection it names); 0: the fixed portfolio */
} kmp_config;

/* Per-call measurements of kmp_partition / kmp_partition_graph (CUDA events). */
typedef struct {
  int32_t levels;            /* graphs in the hierarchy, input included */
  int32_t level_n[64];
  int64_t level_m[64];       /* directed CSR entries per level */
  int64_t lp_scanned;        /* directed entries rated by coarsening LP (all rounds) */
  int64_t refine_scanned;    /* same for refinement LP */
  int64_t lp_rounds_run;     /* coarsening LP rounds executed, all levels */
  int64_t cut;
  int32_t feasible;
  int32_t ip_items;          /* bipartitioner work items */
  float ms_lp;               /* coarsening LP (rating + commit) */
  float ms_cluster_other;    /* isolated packing + two-hop */
  float ms_contract;
  float ms_ip;               /* batched initial bipartitioning incl. extraction */
  float ms_balance;
  float ms_refine;
  float ms_project;
  float ms_total;            /* whole call on the device stream */
  float ms_lp_level0;        /* coarsening LP of the input level alone */
  int64_t lp_scanned_level0; /* entries rated there */
  int32_t lp_rounds_level0;
  int32_t gpu_launches;      /* kernels launched by the call */
  /* the schedule of the top hierarchy (Section 4.1, Algorithm 1): k' and the
   * cluster cap U used to cluster level i (clustered entries; the last one
   * may be a clustering that contracted nothing and stopped coarsening), and
   * the number of blocks of level i's partition after its split rounds */
  int32_t clustered;
  int32_t level_kp[64];
  int64_t level_U[64];
  int32_t level_k[64];
  /* k-way balancing (Section 4.3), summed over the levels: overloaded blocks,
   * moves, moves decided by the parallel speculation that stood at commit,
   * and batches the exact in-order commit evaluated */
  int64_t bal_over_blocks, bal_moves, bal_spec_moves, bal_exact_batches;
  /* candidates the exact batches evaluated, and the adjacency entries they read */
  int64_t bal_exact_cands, bal_exact_entries;
} kmp_stats;

/* opaque handle to a CSR graph resident in device memory */
typedef struct kmp_graph kmp_graph;

void kmp_config_default(kmp_config *cfg);
/* process-wide configuration used by all later calls; KMP_ERR_ARG if invalid */
int kmp_set_config(const kmp_config *cfg);
int kmp_get_config(kmp_config *cfg);
/* stream (cudaStream_t) used by later calls of this thread's process */
int kmp_set_stream(void *stream);
/* message of the last failed call on this thread ("" if none) */
const char *kmp_last_error(void);

/*
 * Create a device graph.  is_device = 0: the arrays are host memory and are
 * copied; 1: they are device memory and are copied device-to-device.  The
 * library owns the copy; free with kmp_graph_free.  vwgt/adjwgt may be NULL
 * (unit weights).  Validates offsets and ranges (KMP_ERR_ARG); symmetry is
 * the caller's contract.
 */
int kmp_graph_create(kmp_vid n, const kmp_eid *xadj, const kmp_vid *adjncy,
                     const kmp_wgt *vwgt, const kmp_wgt *adjwgt, int is_device,
                     kmp_graph **out);
int kmp_graph_free(kmp_graph *g);
/* device pointers of a graph (vwgt/adjwgt NULL when unit) */
int kmp_graph_get(const kmp_graph *g, kmp_vid *n, kmp_eid *m_directed, const kmp_eid **xadj,
                  const kmp_vid **adjncy, const kmp_wgt **vwgt, const kmp_wgt **adjwgt);

/* copy a device graph to host arrays (xadj[n+1], adjncy[m], vwgt[n],
 * adjwgt[m]; any may be NULL to skip; unit weights are written as ones) */
int kmp_graph_copy_to_host(const kmp_graph *g, kmp_eid *xadj, kmp_vid *adjncy, kmp_wgt *vwgt,
                           kmp_wgt *adjwgt);

/*
 * One level of coarsening (Section 4.1): size-constrained label propagation
 * with cluster cap U = max_cluster_weight for `rounds` rounds in S
 * deterministic sub-rounds, packing of isolated nodes, and two-hop clustering
 * when fewer than half of the nodes were clustered away (config.two_hop).
 * label_out: device int32[n], cluster id of each node (a node id).
 * fav_out: device int32[n] or NULL, favoured cluster (-1 if none).
 * Random choices depend on (seed, level).  KMP_ERR_ARG if U < max c(v).
 */
int kmp_coarsen_level(const kmp_graph *g, int64_t max_cluster_weight, int32_t rounds,
                      uint64_t seed, int32_t level, kmp_vid *label_out, kmp_vid *fav_out);

/*
 * Contraction (Section 2, "Multilevel Graph Partitioning"): every cluster of
 * `label` (device int32[n]) becomes one coarse node of summed weight; parallel
 * edges are summed, edges inside a cluster vanish.  Coarse ids follow
 * ascending label; coarse rows are sorted by neighbour id.  *coarse_out is
 * allocated by the library (free with kmp_graph_free); map_out: device
 * int32[n], coarse id of each node.
 */
int kmp_contract(const kmp_graph *g, const kmp_vid *label, kmp_graph **coarse_out,
                 kmp_vid *map_out);

/*
 * LP refinement (Section 4.3, "Local Improvement"): label propagation over
 * the k blocks of part_inout (device int32[n], values in [0,k)) that never
 * lets a block exceed max_block_weight[b] (host int64[k]).  `rounds` rounds,
 * early stop when nothing moved.  cut_out (host, nullable) receives the cut.
 */
int kmp_refine(const kmp_graph *g, int32_t k, const int64_t *max_block_weight, int32_t rounds,
               uint64_t seed, kmp_vid *part_inout, int64_t *cut_out);

/*
 * k-way balancing (Section 4.3, "Balancing"): moves nodes out of every block
 * heavier than max_block_weight[b] (host int64[k]) by relative gain until it
 * fits or no node can move.  moved_out (host, nullable): nodes moved.
 */
int kmp_balance(const kmp_graph *g, int32_t k, const int64_t *max_block_weight,
                kmp_vid *part_inout, int64_t *moved_out);

/* projection (Algorithm 1): part_fine[v] = part_coarse[map[v]], device arrays */
int kmp_project(kmp_vid n_fine, const kmp_vid *map, const kmp_vid *part_coarse,
                kmp_vid *part_fine);

/* cut and block weights of a partition (Section 2); block_weights_out host int64[k] or NULL */
int kmp_cut(const kmp_graph *g, const kmp_vid *part, int32_t k, int64_t *cut_out,
            int64_t *block_weights_out);

/*
 * One round of Algorithm 2 (bipartitionBlocks): every block b of part_inout
 * (device int32[n], nblocks blocks) with final count f[b] >= 2 (host int32)
 * is split by the multilevel bipartitioner of Section 4.2, all blocks in one
 * batched launch; blocks are renumbered in ascending order, child 0 first.
 * f_out (host int32[2*nblocks]) and *nblocks_out receive the new counts.
 * eps, total weight cV and final k define the adaptive imbalance; roundkey
 * selects the random choices.
 */
int kmp_bipartition_blocks(const kmp_graph *g, int32_t nblocks, const int32_t *f, double eps,
                           int64_t cV, int32_t k, uint64_t roundkey, kmp_vid *part_inout,
                           int32_t *nblocks_out, int32_t *f_out);

/*
 * The bipartitioner of Section 4.2 on every block of part (device int32[n],
 * values in [0, nblocks)) with explicit caps: caps is host int32[4*nblocks],
 * (target0, target1, L0, L1) of block b at 4b (targets >= 0, caps >= 1).
 * Blocks are the items of one batched launch, item key step(roundkey, b) as
 * in kmp_bipartition_blocks; on return node v of block b is in block
 * 2b + side.  For bipartitioning many independent subgraphs at once (give
 * the disjoint union and the subgraph index as part).
 */
int kmp_bipartition_each(const kmp_graph *g, int32_t nblocks, const int32_t *caps, uint64_t roundkey,
                         kmp_vid *part);

/*
 * Full deep multilevel partition (Algorithm 1) of a host CSR into k blocks
 * with imbalance eps.  part_out: host int32[n].  Returns KMP_ERR_INFEASIBLE
 * (result still written) when a block exceeds L_k = floor((1+eps) ceil(c(V)/k)).
 */
int kmp_partition(kmp_vid n, const kmp_eid *xadj, const kmp_vid *adjncy, const kmp_wgt *vwgt,
                  const kmp_wgt *adjwgt, int32_t k, double eps, uint64_t seed,
                  kmp_vid *part_out);

/* same on a device graph; part_out is device int32[n]; stats (host) nullable */
int kmp_partition_graph(const kmp_graph *g, int32_t k, double eps, uint64_t seed,
                        kmp_vid *part_out, kmp_stats *stats);

/* stats of the last kmp_partition / kmp_partition_graph call of this thread */
int kmp_last_stats(kmp_stats *stats);

/*
 * Live profiling of the LP rating stage (Section 4.1 and 4.3: the rating of
 * every LP sub-round, the dominant work of coarsening and refinement).  When
 * on, the rating kernel k_rate stamps the device's global timer: its first
 * CTA's start and its last CTA's end give the launch's duration (stamps are
 * taken inside the kernels, so the replayed CUDA graph of an LP round needs
 * no extra nodes).  Algorithmic bytes are counted per directed entry rated:
 * adjncy 4 + neighbour label 4 (+ edge weight 4 when weighted); per rated
 * node: xadj 8 + list entry 4 + own label 4 + proposal 8 (+ node weight 4).
 * kmp_profile_read: k_rate alone (nodes rated by the hub kernels excluded),
 * sums since the last reset (milliseconds, bytes, launches).
 * kmp_profile_read_stage: the whole rating stage of each sub-round, from
 * k_rate's first CTA start to the last CTA end of the last hub kernel after
 * it (hub nodes and entries included): milliseconds, bytes, spans.
 * Host pointers, each nullable; reset != 0 zeroes the sums after reading.
 */
int kmp_set_profiling(int on);
int kmp_profile_read(double *rate_ms, double *rate_bytes, int64_t *rate_launches, int reset);
int kmp_profile_read_stage(double *stage_ms, double *stage_bytes, int64_t *spans, int reset);

/*
 * Schedule parameters of the GPU kernels.  They decide which kernel variant
 * handles a node or work item and how grids are sized; they never change a
 * result (the parity tests run every setting against the CPU oracle).
 */
typedef struct {
  int32_t rate_blocks_per_sm; /* LP rating grid = this * SMs (2..16) */
  int32_t hub_degree;         /* degree above which coarsening rates a node with the
                                 multi-CTA hub kernels (256..2048) */
  int32_t hub_chunk;          /* edges per hub work unit (256..65536, power of two;
                                 default 2048) */
  int32_t ip_blocks_per_sm;   /* bipartitioner CTAs per SM (1..8) */
  int32_t dense_hub_degree;   /* with few labels (refinement: labels are block ids), degree
                                 above which a node's rating is split over many CTAs into a
                                 dense per-label row instead of one CTA (512..2^30) */
  int32_t lp_graphs;          /* 1: each LP run captures one round as a CUDA graph and replays
                                 it for every round; 0: direct launches (default 1) */
  int32_t hub_bucket;         /* hub ratings with many labels: target entries per label bucket
                                 aggregated by one warp (32..2^20; 0 = default 256) */
  int32_t dense_labels;       /* an LP run with more than 2048 but at most this many labels rates
                                 its hubs into dense per-hub rows of label counters (the dense
                                 vector of Section 5) when the rows fit 4 GB; 0 = never (label
                                 buckets); at most 57344 */
} kmp_tuning;

int kmp_set_tuning(const kmp_tuning *t);
int kmp_get_tuning(kmp_tuning *t);
/*
 * Autotuner: times candidate schedules on the level-0 coarsening LP of `g`
 * (one run per candidate, cap derived from k and eps as the partitioner
 * does), keeps the fastest with kmp_set_tuning and returns it in *best.
 * Candidates: rating grid {4, 6, 8} x SMs, hub degree {1024, 2048}, hub chunk
 * {512, 2048}.
 */
int kmp_autotune(const kmp_graph *g, int32_t k, double eps, uint64_t seed, kmp_tuning *best);

/*
 * Learned seed proposer for the bipartitioner (learned mode of kmp_config).
 * The paper bipartitions a coarsest graph by repeating random, BFS and
 * greedy-graph-growing starts and keeping the best (Section 4.2); in learned
 * mode a message-passing network scores the coarsest graph's nodes first and
 * its score order (first fit to block 0's target, like the random start)
 * becomes one more start, FM-refined and compared exactly like the others,
 * ahead of a reduced portfolio; the rest of the portfolio runs only if the
 * best so far is infeasible.  So every result is still FM-refined and
 * balance-checked by the method itself.
 *
 * Network: 8 node features (1; c(v)/mean c; deg/max deg; weighted degree /
 * mean; BFS hops from two anchors over (max hops + 1); two +-1 key bits),
 * two layers h' = relu(W_self h + W_nbr mean_w(h_nbr) + b) of width 64, and a
 * linear read-out.  Parameters: KMP_MPNN_PARAMS floats in the order W1_self
 * [64][8], W1_nbr [64][8], b1 [64], W2_self [64][64], W2_nbr [64][64], b2 [64],
 * w_out [64], b_out.  The model keeps fp32 master weights and Adam moments;
 * every kernel computes with the BF16-rounded weights and fp32 arithmetic
 * (fixed-order fused multiply-adds, so scores are reproducible exactly).
 *
 * Batches (forward, gradients, train): ng graphs as one disjoint union in
 * HOST arrays: noff[ng+1] node offsets (noff[0] = 0), xadj[N+1] (int64), adj
 * (union node ids; symmetric, no self-loops), vw[N] and ew[E] (NULL: ones),
 * keys[ng] (the key of each graph's features), side[N] (0/1 labels, e.g. the
 * best-of-portfolio sides from the sample sink).  Loss: per graph the mean
 * binary cross-entropy of sigmoid(score) against side (block 0 = 1) under
 * the better of the two block orientations, averaged over graphs.
 */
#define KMP_MPNN_PARAMS 9409
typedef struct kmp_mpnn kmp_mpnn;
int kmp_mpnn_num_params(void);
/* new model with He-uniform weights from seed; free with kmp_mpnn_free */
int kmp_mpnn_create(uint64_t seed, kmp_mpnn **out);
int kmp_mpnn_free(kmp_mpnn *m);
/* params: host float[KMP_MPNN_PARAMS]; get returns the BF16 weights as floats */
int kmp_mpnn_get_params(const kmp_mpnn *m, float *params);
int kmp_mpnn_set_params(kmp_mpnn *m, const float *params);
/* scores[N] (host); features[N*8] (host, nullable) */
int kmp_mpnn_forward(kmp_mpnn *m, int32_t ng, const int32_t *noff, const int64_t *xadj,
                     const int32_t *adj, const int32_t *vw, const int32_t *ew, const uint64_t *keys,
                     float *scores, float *features);
/* loss and its gradient with respect to the (BF16) weights; grad_out host
 * float[KMP_MPNN_PARAMS] or NULL; the model is not changed */
int kmp_mpnn_gradients(kmp_mpnn *m, int32_t ng, const int32_t *noff, const int64_t *xadj,
                       const int32_t *adj, const int32_t *vw, const int32_t *ew,
                       const uint64_t *keys, const int32_t *side, float *loss_out, float *grad_out);
/* `epochs` full-batch Adam steps (beta 0.9/0.999) at learning rate lr;
 * loss_per_epoch host float[epochs] or NULL (loss before each step) */
int kmp_mpnn_train(kmp_mpnn *m, int32_t ng, const int32_t *noff, const int64_t *xadj,
                   const int32_t *adj, const int32_t *vw, const int32_t *ew, const uint64_t *keys,
                   const int32_t *side, int32_t epochs, float lr, float *loss_per_epoch);
/* proposer used by learned mode from now on (NULL: none, learned mode then
 * runs the plain portfolio); the model must outlive its use */
int kmp_set_proposer(const kmp_mpnn *m);

/*
 * Sample sink: while open, every item of the batched bipartitioner (the
 * blocks split by kmp_bipartition_blocks, kmp_partition and friends) appends
 * its coarsest graph and the winning bipartition of the portfolio there --
 * the training data of the proposer, generated by the method itself.  Items
 * beyond the capacity are dropped and counted.  read: the kept samples as
 * one union (format of the batches above) ordered by item key; the host
 * arrays must hold count's totals (noff graphs+1, xadj nodes+1, adj/ew
 * entries, vw/side nodes, keys graphs).  open replaces an open sink.
 */
int kmp_sample_sink_open(int32_t max_graphs, int64_t max_nodes, int64_t max_entries);
int kmp_sample_sink_count(int32_t *graphs, int64_t *nodes, int64_t *entries, int64_t *dropped);
int kmp_sample_sink_read(int32_t *noff, int64_t *xadj, int32_t *adj, int32_t *vw, int32_t *ew,
                         uint64_t *keys, int32_t *side);
int kmp_sample_sink_close(void);
/* what the sink records from now on: 0 (default) each item's coarsest graph
 * and the winning portfolio bipartition there (training data for learned
 * mode 1); 1 each item graph and its final bipartition by the plain method
 * (training data for learned mode 2).  KMP_ERR_ARG for other values. */
int kmp_sample_sink_level(int32_t item_level);

/*
 * Cut and block weights without any device allocation.  The paper has no
 * counterpart: this is a library-side variant of kmp_cut for callers that
 * cannot let the library allocate device memory at call time: code whose
 * device memory belongs to another allocator or to a fixed arena that must
 * account for every byte, processes that reserve all device memory up front,
 * and loops that cannot take the implicit synchronisation or the possible
 * failure of an allocation.  Its scratch is one fixed device array of
 * KMP_NOALLOC_MAX_K + 2 64-bit words (about 512 KB) inside the library, held
 * on every device that loads the library until the process exits.
 *
 * g: graph handle; part: DEVICE int32[n] with values in [0, k); k in
 * [1, KMP_NOALLOC_MAX_K] (else KMP_ERR_ARG, nothing launched); cut_out (host,
 * nullable): the cut; block_weights_out (host int64[k], nullable): c(V_b).
 * A part value outside [0, k) gives KMP_ERR_ARG (outputs unspecified).
 * Runs on the stream of kmp_set_stream and returns after it drained.
 *
 * Set-up: the array's module is loaded, and its device address looked up,
 * while the library initialises on a device (the first library call there,
 * e.g. kmp_graph_create).  That module load is the only device memory this
 * entry point ever causes to be committed, and it happens before the first
 * kmp_cut_noalloc call; make that first library call before any stream
 * capture.  If the device's context is recreated (cudaDeviceReset), the next
 * call looks the address up again.  Each call clears the part of the array it
 * accumulates into; overlapping calls (from several host threads or streams)
 * share the one array and race: serialise them.
 */
#define KMP_NOALLOC_MAX_K 65536
int kmp_cut_noalloc(const kmp_graph *g, const kmp_vid *part, int32_t k, int64_t *cut_out,
                    int64_t *block_weights_out);

#ifdef __cplusplus
}
#endif
#endif
