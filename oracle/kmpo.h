/*
 * kmpo -- CPU ORACLE for deep multilevel graph partitioning (test
 * infrastructure only).
 *
 * A plain, slow, single-threaded C restatement of what the method computes:
 * size-constrained label propagation (Section 2 and 4.1), two-hop clustering
 * (Section 4.1), contraction (Section 2, "Multilevel Graph Partitioning"),
 * deep multilevel partitioning with recursive bipartitioning of blocks
 * (Algorithm 1, Algorithm 2, Section 3 "Handling General k"), multilevel
 * initial bipartitioning with a portfolio and 2-way FM (Section 4.2), k-way
 * balancing and LP refinement (Section 4.3).  Where the paper leaves a detail
 * open, the oracle follows one fixed deterministic reading that the CUDA path
 * must reproduce bit for bit; those readings are listed at the top of each
 * source file.
 *
 * Only the test suite, the smoke check and the benchmark's CPU-baseline leg
 * may load this library.  It shares no code with the CUDA path.
 */
#ifndef KMPO_H
#define KMPO_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int32_t C;             /* contraction limit: coarsen until <= 2C nodes */
  int32_t lp_rounds;     /* coarsening LP rounds (Section 4.1: 5) */
  int32_t refine_rounds; /* refinement LP rounds (Section 4.3: 5) */
  int32_t subrounds;     /* S: deterministic sub-rounds per round (power of 2) */
  int32_t two_hop;       /* enable two-hop clustering (Section 4.1) */
  int32_t conv_num;      /* coarsening converged when conv_den*n' > conv_num*n */
  int32_t conv_den;
  int32_t ip_C;          /* bipartitioner cluster cap: floor(c(B)/ip_C) */
  int32_t ip_lp_rounds;  /* LP rounds per bipartitioner coarsening level */
  int32_t rep_random;    /* portfolio repetitions (Section 4.2) */
  int32_t rep_bfs;
  int32_t rep_ggg;
  int32_t fm_passes;     /* 2-way FM passes per level */
  int32_t fm_stop;       /* a pass ends after this many moves without a new best */
  int32_t learned;       /* learned mode: proposal first, reduced portfolio (B6) */
  int32_t lrep_random;   /* portfolio repetitions in learned mode */
  int32_t lrep_bfs;
  int32_t lrep_ggg;
  int32_t replicas;      /* R, copies of the coarsest graph (Section 3, "Parallelization"): 1 = off */
  int32_t async_lp;      /* quality reference only (no GPU counterpart): coarsen with the sequential
                            asynchronous LP (kmpo_async_cluster, no two-hop) instead of the
                            deterministic sub-rounds (0) */
  int32_t sample_subrounds; /* timing samples only: kmpo_cluster's LP ends after this many
                               sub-rounds (0: no limit); the sub-rounds that run are unchanged */
  int32_t adaptive;      /* adaptive portfolio (B7, kmpo_ip.c): 0 = the fixed portfolio of B2 */
  int32_t sample_nodes;  /* timing samples only: with sample_subrounds, the sampled sub-rounds rate
                            only nodes u < sample_nodes (0: all) */
} kmpo_config;

/* graph owned by the oracle (returned by kmpo_contract) */
typedef struct {
  int32_t n;
  int64_t *xadj;
  int32_t *adj;
  int32_t *vw;
  int32_t *ew;
} kmpo_graph;

typedef struct {
  int32_t rounds;            /* LP rounds executed */
  int64_t moved[16];         /* vertices moved per round */
  int64_t scanned[16];       /* directed entries scanned per round */
} kmpo_lp_stats;

typedef struct {
  int32_t levels;            /* number of coarse levels built */
  int32_t level_n[64];       /* vertices per level */
  int64_t level_m[64];       /* directed entries per level */
  int64_t lp_scanned;        /* total directed entries scanned by coarsening LP */
  int64_t refine_scanned;    /* same for refinement LP */
  int64_t cut;
  int32_t feasible;
  double t_coarsen, t_ip, t_refine, t_total; /* seconds (coarsening includes contraction) */
  /* the schedule of the top hierarchy (D1, D2): k' and U used to cluster
   * level i (i < levels; the last entry is the clustering that stopped
   * coarsening, if one ran), and the block count of level i's partition after
   * its split rounds */
  int32_t level_kp[64];
  int64_t level_U[64];
  int32_t level_k[64];
  int32_t clustered;         /* number of clusterings run (entries of level_kp/U) */
  double t_contract, t_balance; /* seconds, parts of t_coarsen and t_refine */
} kmpo_stats;

void kmpo_config_default(kmpo_config *cfg);

/* counter-based keys (SplitMix64 finaliser chained over words) */
uint64_t kmpo_key(uint64_t seed, int32_t nwords, const uint64_t *words);
uint64_t kmpo_step(uint64_t x, uint64_t w);
uint32_t kmpo_perm32(uint64_t roundkey, int32_t label);
int32_t kmpo_subround(uint64_t roundkey, int32_t v, int32_t S);

/* cut (Section 2: sum of weights of edges between different blocks) */
int64_t kmpo_cut(int32_t n, const int64_t *xadj, const int32_t *adj, const int32_t *ew,
                 const int32_t *part);

/*
 * LP clustering of one level: LP (rounds) + isolated-node packing +
 * two-hop merging (if cfg->two_hop).  Keys: kmpo_key(seed, {1, level}).
 * Returns the number of clusters.  fav_out nullable.
 */
int32_t kmpo_cluster(int32_t n, const int64_t *xadj, const int32_t *adj, const int32_t *vw,
                     const int32_t *ew, int32_t U, int32_t rounds, uint64_t seed, int32_t level,
                     const kmpo_config *cfg, int32_t do_isolated, int32_t do_two_hop,
                     int32_t *label_out, int32_t *fav_out, kmpo_lp_stats *st);

/* contraction; allocates *out (free with kmpo_graph_free). map_out[n]. */
int32_t kmpo_contract(int32_t n, const int64_t *xadj, const int32_t *adj, const int32_t *vw,
                      const int32_t *ew, const int32_t *label, int32_t *map_out, kmpo_graph *out);
void kmpo_graph_free(kmpo_graph *g);

/* LP refinement over k blocks with per-block caps; returns the cut afterwards */
int64_t kmpo_refine(int32_t n, const int64_t *xadj, const int32_t *adj, const int32_t *vw,
                    const int32_t *ew, int32_t k, const int32_t *cap, int32_t rounds,
                    uint64_t seed, const kmpo_config *cfg, int32_t *part, kmpo_lp_stats *st);

/* k-way balancing (Section 4.3); returns number of moved nodes */
int64_t kmpo_balance(int32_t n, const int64_t *xadj, const int32_t *adj, const int32_t *vw,
                     const int32_t *ew, int32_t k, const int32_t *cap, int32_t *part);

/* multilevel 2-way bipartitioner of one (sub)graph (Section 4.2); returns cut */
int64_t kmpo_bipartition(int32_t n, const int64_t *xadj, const int32_t *adj, const int32_t *vw,
                         const int32_t *ew, int32_t L0, int32_t L1, int32_t target0,
                         int32_t target1, uint64_t itemkey, const kmpo_config *cfg,
                         int32_t *side_out);

/* 2-way FM on a given bipartition (in place); returns the cut */
int64_t kmpo_fm(int32_t n, const int64_t *xadj, const int32_t *adj, const int32_t *vw,
                const int32_t *ew, int32_t L0, int32_t L1, const kmpo_config *cfg,
                int32_t *side);

/* portfolio initial bipartitions: algo 0 random, 1 BFS, 2 greedy graph growing */
void kmpo_initial(int32_t algo, int32_t n, const int64_t *xadj, const int32_t *adj,
                  const int32_t *vw, const int32_t *ew, int32_t target0, uint64_t key,
                  int32_t *side);

/* adaptive imbalance and child caps for splitting a block (Section 2, Alg. 2) */
double kmpo_eps_prime(double eps, int64_t cV, int32_t k, int64_t cB, int32_t fB);
void kmpo_split_caps(double eps, int64_t cV, int32_t k, int64_t cB, int32_t fB,
                     int32_t *target0, int32_t *target1, int32_t *L0, int32_t *L1);
/* per-block cap L(b) = floor(max((1+eps) cV f/k, cV f/k + maxc)) */
int32_t kmpo_block_cap(double eps, int64_t cV, int32_t k, int32_t fb, int32_t maxc);

/* one split round of Algorithm 2: every block b with f_in[b] >= 2 is
 * bipartitioned; blocks renumbered in ascending order, child 0 first;
 * returns the new block count, f_out receives the new final counts */
int32_t kmpo_bipartition_blocks(int32_t n, const int64_t *xadj, const int32_t *adj,
                                const int32_t *vw, const int32_t *ew, int32_t nblocks,
                                const int32_t *f_in, double eps, int64_t cV, int32_t k,
                                uint64_t roundkey, const kmpo_config *cfg, int32_t *part,
                                int32_t *f_out);

/* full deep multilevel partition (Algorithm 1).  Returns 0, or -5 when the
 * result violates L_k = floor((1+eps) ceil(c(V)/k)) (result still written). */
int32_t kmpo_partition(int32_t n, const int64_t *xadj, const int32_t *adj, const int32_t *vw,
                       const int32_t *ew, int32_t k, double eps, uint64_t seed,
                       const kmpo_config *cfg, int32_t *part_out, kmpo_stats *st);

/* the adaptive portfolio's rule (B7): 1 if an algorithm whose f feasible
 * runs have these cuts keeps running given the best feasible cut */
int32_t kmpo_adaptive_keep(int32_t f, const int64_t *cuts, int64_t best);

/* brute-force minimum cut bisection (n <= 24) with caps on both sides;
 * returns -1 if no feasible bisection exists */
int64_t kmpo_brute_bisection(int32_t n, const int64_t *xadj, const int32_t *adj,
                             const int32_t *vw, const int32_t *ew, int64_t L0, int64_t L1,
                             int32_t *side_out);

/* sequential asynchronous (Gauss-Seidel) LP clustering: the paper's sequential
 * semantics of size-constrained LP, nodes visited by degree bucket in a seeded
 * random order per round; used only as a quality reference */
int32_t kmpo_async_cluster(int32_t n, const int64_t *xadj, const int32_t *adj,
                           const int32_t *vw, const int32_t *ew, int32_t U, int32_t rounds,
                           uint64_t seed, int32_t *label_out);

/* learned seed proposer (kmpo_mpnn.c): parameters in fp64, layout documented there */
int32_t kmpo_mpnn_num_params(void);
void kmpo_mpnn_features(int32_t n, const int64_t *xadj, const int32_t *adj, const int32_t *vw,
                        const int32_t *ew, uint64_t key, double *X);
void kmpo_mpnn_forward(int32_t n, const int64_t *xadj, const int32_t *adj, const int32_t *ew,
                       const double *X, const double *P, double *S, double *cache);
double kmpo_mpnn_loss(int32_t n, const double *S, const int32_t *side, double *gS);
void kmpo_mpnn_backward(int32_t n, const int64_t *xadj, const int32_t *adj, const int32_t *ew,
                        const double *X, const double *P, const double *gS, double *gP);
void kmpo_mpnn_propose(int32_t n, const int32_t *vw, const double *S, int32_t target0,
                       int32_t *side);
/* inference in the kernel's precision (fp32, fused multiply-adds in a fixed
 * order); W: parameters as fp32 values */
void kmpo_mpnn_scores_f32(int32_t n, const int64_t *xadj, const int32_t *adj, const int32_t *vw,
                          const int32_t *ew, uint64_t key, const float *W, float *S);
uint32_t kmpo_mpnn_score_key(float s);
/* proposer used by learned mode (copied; NULL clears) */
void kmpo_set_proposer(const float *W);
const float *kmpo_proposer(void);
/* learned start: first fit to target0 in (score key, id) order */
void kmpo_learned_initial(int32_t n, const int64_t *xadj, const int32_t *adj, const int32_t *vw,
                          const int32_t *ew, int32_t target0, uint64_t key, const float *W,
                          int32_t *side);

#ifdef __cplusplus
}
#endif
#endif
