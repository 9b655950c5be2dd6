/*
 * Seeded synthetic graph generators (input side only).
 *
 * This module produces the inputs that both the CUDA path and the CPU oracle
 * consume.  It holds none of the partitioning method's arithmetic: it only
 * builds undirected weighted graphs in CSR form G = (V, E, c, w) with positive
 * integer node and edge weights (the problem statement of Section 2).
 *
 * Randomness: one counter-based generator, SplitMix64's output function
 * (Steele, Lea, Flood, "Fast splittable pseudorandom number generators",
 * OOPSLA 2014) applied to seed-derived counters, so every value is a pure
 * function of (seed, stream, index) and identical on every host.
 *
 * Every returned CSR is symmetric, has no self-loops, no duplicate entries,
 * rows sorted by neighbour id, and equal weights on both directions.
 *
 * The large loops may run on several host threads (OpenMP, when the build
 * has it); every value is a pure function of its index and every parallel
 * step keeps the sequential order, so the output does not depend on the
 * thread count.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static uint64_t sm64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

/* value number i of stream s for a given seed */
static uint64_t draw(uint64_t seed, uint64_t s, uint64_t i) {
  return sm64(sm64(seed ^ sm64(s * 0x632BE59BD9B4E019ull)) + i);
}

static double unit(uint64_t seed, uint64_t s, uint64_t i) {
  return (double)(draw(seed, s, i) >> 11) * (1.0 / 9007199254740992.0);
}

#ifdef _OPENMP
#include <omp.h>
static int nthreads(int64_t work) { return work < (1 << 20) ? 1 : omp_get_max_threads(); }
static int thread_id(void) { return omp_get_thread_num(); }
static int team_size(void) { return omp_get_num_threads(); }
#else
static int nthreads(int64_t work) { (void)work; return 1; }
static int thread_id(void) { return 0; }
static int team_size(void) { return 1; }
#endif

/* The work is split into T fixed chunks before a parallel region starts.  The
 * runtime may give the region fewer threads than asked for (a thread limit,
 * dynamic teams, a nested region), so every region walks all T chunks with
 * the threads it actually has: chunk t goes to thread t mod (team size). */
#define FOR_EACH_CHUNK(t, T) for (int t = thread_id(); t < (T); t += team_size())

/* ---------------- LSD radix sort of uint64 keys (host helper) ---------------- */
/* Stable 16-bit digits; with T threads each thread owns a contiguous chunk
 * and scatters it to the offsets of (digit, thread) in that order, which is
 * exactly the sequential placement. */
static void sort_u64(uint64_t *a, int64_t n) {
  if (n < 2) return;
  uint64_t *tmp = (uint64_t *)malloc((size_t)n * sizeof(uint64_t));
  const int T = nthreads(n);
  int64_t *cnt = (int64_t *)malloc(sizeof(int64_t) * 65536 * (size_t)T);
  for (int pass = 0; pass < 4; ++pass) {
    int sh = pass * 16;
    memset(cnt, 0, sizeof(int64_t) * 65536 * (size_t)T);
#pragma omp parallel num_threads(T)
    FOR_EACH_CHUNK(t, T) {
      const int64_t lo = n * t / T, hi = n * (t + 1) / T;
      int64_t *c = cnt + (size_t)t * 65536;
      for (int64_t i = lo; i < hi; ++i) c[(a[i] >> sh) & 0xFFFF]++;
    }
    int64_t s = 0;
    for (int d = 0; d < 65536; ++d)
      for (int t = 0; t < T; ++t) {
        int64_t c = cnt[(size_t)t * 65536 + d];
        cnt[(size_t)t * 65536 + d] = s;
        s += c;
      }
#pragma omp parallel num_threads(T)
    FOR_EACH_CHUNK(t, T) {
      const int64_t lo = n * t / T, hi = n * (t + 1) / T;
      int64_t *c = cnt + (size_t)t * 65536;
      for (int64_t i = lo; i < hi; ++i) tmp[c[(a[i] >> sh) & 0xFFFF]++] = a[i];
    }
    uint64_t *t = a; a = tmp; tmp = t;
  }
  /* 4 passes: result is back in the original buffer */
  free(cnt);
  free(tmp);
}

/*
 * Build CSR from a list of (u << 32 | v) directed keys: symmetrises, removes
 * self-loops and duplicates.  Writes xadj[n+1]; returns the adjacency through
 * *adj_out (malloc'd) and the number of directed entries.
 */
static int64_t keys_to_csr(int32_t n, uint64_t *keys, int64_t nk, int64_t *xadj,
                           int32_t **adj_out) {
  /* symmetrise into a doubled buffer (per-chunk counts keep the order) */
  uint64_t *k2 = (uint64_t *)malloc((size_t)(2 * nk + 1) * sizeof(uint64_t));
  const int T = nthreads(nk);
  int64_t *off = (int64_t *)calloc((size_t)T + 1, sizeof(int64_t));
#pragma omp parallel num_threads(T)
  FOR_EACH_CHUNK(t, T) {
    const int64_t lo = nk * t / T, hi = nk * (t + 1) / T;
    int64_t c = 0;
    for (int64_t i = lo; i < hi; ++i) c += (uint32_t)(keys[i] >> 32) != (uint32_t)keys[i];
    off[t + 1] = 2 * c;
  }
  for (int t = 0; t < T; ++t) off[t + 1] += off[t];
  const int64_t m = off[T];
#pragma omp parallel num_threads(T)
  FOR_EACH_CHUNK(t, T) {
    const int64_t lo = nk * t / T, hi = nk * (t + 1) / T;
    int64_t p = off[t];
    for (int64_t i = lo; i < hi; ++i) {
      uint32_t u = (uint32_t)(keys[i] >> 32), v = (uint32_t)keys[i];
      if (u == v) continue;
      k2[p++] = ((uint64_t)u << 32) | v;
      k2[p++] = ((uint64_t)v << 32) | u;
    }
  }
  free(off);
  sort_u64(k2, m);
  int64_t w = 0;
  for (int64_t i = 0; i < m; ++i)
    if (w == 0 || k2[i] != k2[w - 1]) k2[w++] = k2[i];
  int32_t *adj = (int32_t *)malloc((size_t)(w > 0 ? w : 1) * sizeof(int32_t));
  for (int32_t v = 0; v <= n; ++v) xadj[v] = 0;
  for (int64_t i = 0; i < w; ++i) {
    xadj[(k2[i] >> 32) + 1]++;
    adj[i] = (int32_t)(uint32_t)k2[i];
  }
  for (int32_t v = 0; v < n; ++v) xadj[v + 1] += xadj[v];
  free(k2);
  *adj_out = adj;
  return w;
}

/* ---------------- 2D random geometric graph ---------------- */
/*
 * n points uniform in the unit square; an edge joins two points at Euclidean
 * distance < r with r = sqrt(avg_deg / (pi n)).  Vertex ids are assigned in
 * order of (cell row, cell column, x) on a grid of cell side >= r, which gives
 * the spatial locality that real meshes have.
 * Returns the number of directed CSR entries; *adj_out is malloc'd.
 */
int64_t gg_rgg(int32_t n, double avg_deg, uint64_t seed, int64_t *xadj,
               int32_t **adj_out) {
  double r = sqrt(avg_deg / (M_PI * (double)n));
  int32_t g = (int32_t)floor(1.0 / r);
  if (g < 1) g = 1;
  double *px = (double *)malloc((size_t)n * sizeof(double));
  double *py = (double *)malloc((size_t)n * sizeof(double));
  uint64_t *key = (uint64_t *)malloc((size_t)n * sizeof(uint64_t));
  for (int32_t i = 0; i < n; ++i) {
    px[i] = unit(seed, 1, (uint64_t)i);
    py[i] = unit(seed, 2, (uint64_t)i);
  }
  /* order by (cy, cx): key = cell id << 32 | point index */
  for (int32_t i = 0; i < n; ++i) {
    int64_t cx = (int64_t)(px[i] * g), cy = (int64_t)(py[i] * g);
    if (cx >= g) cx = g - 1;
    if (cy >= g) cy = g - 1;
    uint64_t cell = (uint64_t)(cy * g + cx);
    key[i] = (cell << 32) | (uint32_t)i; /* stable within cell by index */
  }
  /* sort by cell, then re-sort each cell by x */
  sort_u64(key, n);
  int32_t *perm = (int32_t *)malloc((size_t)n * sizeof(int32_t));
  double *sx = (double *)malloc((size_t)n * sizeof(double));
  double *sy = (double *)malloc((size_t)n * sizeof(double));
  int64_t *cstart = (int64_t *)calloc((size_t)g * g + 1, sizeof(int64_t));
  for (int32_t i = 0; i < n; ++i) cstart[(key[i] >> 32) + 1]++;
  for (int64_t c = 0; c < (int64_t)g * g; ++c) cstart[c + 1] += cstart[c];
  for (int32_t i = 0; i < n; ++i) perm[i] = (int32_t)(uint32_t)key[i];
  /* insertion sort inside each cell by x (cells hold ~avg_deg/pi points) */
  for (int64_t c = 0; c < (int64_t)g * g; ++c) {
    for (int64_t a = cstart[c] + 1; a < cstart[c + 1]; ++a) {
      int32_t t = perm[a];
      int64_t b = a - 1;
      while (b >= cstart[c] && (px[perm[b]] > px[t] ||
                                (px[perm[b]] == px[t] && perm[b] > t))) {
        perm[b + 1] = perm[b];
        --b;
      }
      perm[b + 1] = t;
    }
  }
  for (int32_t i = 0; i < n; ++i) { sx[i] = px[perm[i]]; sy[i] = py[perm[i]]; }
  free(px); free(py); free(perm);
  /* neighbour search over 3x3 cells; points are now grouped by cell */
  double r2 = r * r;
  int64_t cap = (int64_t)((double)n * (0.5 * avg_deg + 2.0 * sqrt(avg_deg) + 4.0));
  uint64_t *ek = (uint64_t *)malloc((size_t)cap * sizeof(uint64_t));
  int64_t ne = 0;
  for (int32_t cy = 0; cy < g; ++cy)
    for (int32_t cx = 0; cx < g; ++cx) {
      int64_t c = (int64_t)cy * g + cx;
      for (int64_t a = cstart[c]; a < cstart[c + 1]; ++a)
        for (int32_t dy = -1; dy <= 1; ++dy)
          for (int32_t dx = -1; dx <= 1; ++dx) {
            int32_t ny = cy + dy, nx = cx + dx;
            if (ny < 0 || nx < 0 || ny >= g || nx >= g) continue;
            int64_t c2 = (int64_t)ny * g + nx;
            if (c2 < c) continue; /* each unordered cell pair once */
            for (int64_t b = cstart[c2]; b < cstart[c2 + 1]; ++b) {
              if (c2 == c && b <= a) continue;
              double ddx = sx[a] - sx[b], ddy = sy[a] - sy[b];
              if (ddx * ddx + ddy * ddy < r2) {
                if (ne >= cap) {
                  cap = cap * 2;
                  ek = (uint64_t *)realloc(ek, (size_t)cap * sizeof(uint64_t));
                }
                ek[ne++] = ((uint64_t)a << 32) | (uint64_t)b;
              }
            }
          }
    }
  free(sx); free(sy); free(cstart); free(key);
  int64_t m = keys_to_csr(n, ek, ne, xadj, adj_out);
  free(ek);
  return m;
}

/* ---------------- R-MAT ---------------- */
/*
 * R-MAT (Chakrabarti, Zhan, Faloutsos, SDM 2004): edge_factor * 2^scale edge
 * samples, each choosing one quadrant per bit with probabilities (a, b, c, d).
 * The result is symmetrised, deduplicated, self-loops removed, and vertex ids
 * are relabelled by a seeded random permutation.
 */
int64_t gg_rmat(int32_t scale, int32_t edge_factor, double a, double b,
                double c, uint64_t seed, int64_t *xadj, int32_t **adj_out) {
  int32_t n = 1 << scale;
  int64_t ns = (int64_t)edge_factor * (int64_t)n;
  uint64_t *ek = (uint64_t *)malloc((size_t)ns * sizeof(uint64_t));
  double ab = a + b, abc = a + b + c;
#pragma omp parallel for schedule(static) num_threads(nthreads(ns))
  for (int64_t e = 0; e < ns; ++e) {
    uint32_t u = 0, v = 0;
    for (int32_t l = 0; l < scale; ++l) {
      double p = unit(seed, 16 + (uint64_t)l, (uint64_t)e);
      uint32_t bu = 0, bv = 0;
      if (p < a) { bu = 0; bv = 0; }
      else if (p < ab) { bu = 0; bv = 1; }
      else if (p < abc) { bu = 1; bv = 0; }
      else { bu = 1; bv = 1; }
      u = (u << 1) | bu;
      v = (v << 1) | bv;
    }
    ek[e] = ((uint64_t)u << 32) | v;
  }
  /* random permutation of ids: sort (random key, id) pairs */
  uint64_t *pk = (uint64_t *)malloc((size_t)n * sizeof(uint64_t));
  for (int32_t i = 0; i < n; ++i)
    pk[i] = (draw(seed, 7, (uint64_t)i) & 0xFFFFFFFF00000000ull) | (uint32_t)i;
  sort_u64(pk, n);
  int32_t *newid = (int32_t *)malloc((size_t)n * sizeof(int32_t));
  for (int32_t i = 0; i < n; ++i) newid[(uint32_t)pk[i]] = i;
#pragma omp parallel for schedule(static) num_threads(nthreads(ns))
  for (int64_t e = 0; e < ns; ++e) {
    uint32_t u = (uint32_t)(ek[e] >> 32), v = (uint32_t)ek[e];
    ek[e] = ((uint64_t)(uint32_t)newid[u] << 32) | (uint32_t)newid[v];
  }
  free(pk); free(newid);
  int64_t m = keys_to_csr(n, ek, ns, xadj, adj_out);
  free(ek);
  return m;
}

/* ---------------- small structured graphs ---------------- */
/* a x b grid, vertex (i, j) has id i*b + j */
int64_t gg_grid(int32_t a, int32_t b, int64_t *xadj, int32_t **adj_out) {
  int32_t n = a * b;
  uint64_t *ek = (uint64_t *)malloc((size_t)(2 * (int64_t)n + 1) * sizeof(uint64_t));
  int64_t ne = 0;
  for (int32_t i = 0; i < a; ++i)
    for (int32_t j = 0; j < b; ++j) {
      uint32_t v = (uint32_t)(i * b + j);
      if (j + 1 < b) ek[ne++] = ((uint64_t)v << 32) | (v + 1);
      if (i + 1 < a) ek[ne++] = ((uint64_t)v << 32) | (uint32_t)(v + b);
    }
  int64_t m = keys_to_csr(n, ek, ne, xadj, adj_out);
  free(ek);
  return m;
}

/*
 * Erdos-Renyi-like random graph with m_samples edge draws among n vertices
 * (duplicates and self-loops dropped).  Used for small fuzz cases.
 */
int64_t gg_random(int32_t n, int64_t m_samples, uint64_t seed, int64_t *xadj,
                  int32_t **adj_out) {
  uint64_t *ek = (uint64_t *)malloc((size_t)(m_samples + 1) * sizeof(uint64_t));
  for (int64_t e = 0; e < m_samples; ++e) {
    uint32_t u = (uint32_t)(draw(seed, 3, (uint64_t)e) % (uint64_t)n);
    uint32_t v = (uint32_t)(draw(seed, 4, (uint64_t)e) % (uint64_t)n);
    ek[e] = ((uint64_t)u << 32) | v;
  }
  int64_t m = keys_to_csr(n, ek, m_samples, xadj, adj_out);
  free(ek);
  return m;
}

/*
 * Hub graph: n vertices; vertex i < nhubs is a hub joined to a random subset
 * of size hub_deg[i]; the rest get a sparse random background of bg_samples
 * edges.  Exercises every degree class of the LP kernels.
 */
int64_t gg_hubs(int32_t n, int32_t nhubs, const int32_t *hub_deg,
                int64_t bg_samples, uint64_t seed, int64_t *xadj,
                int32_t **adj_out) {
  int64_t tot = bg_samples;
  for (int32_t h = 0; h < nhubs; ++h) tot += hub_deg[h];
  uint64_t *ek = (uint64_t *)malloc((size_t)(tot + 1) * sizeof(uint64_t));
  int64_t ne = 0;
  for (int32_t h = 0; h < nhubs; ++h)
    for (int32_t j = 0; j < hub_deg[h]; ++j) {
      uint32_t v = (uint32_t)(draw(seed, 100 + (uint64_t)h, (uint64_t)j) % (uint64_t)n);
      ek[ne++] = ((uint64_t)(uint32_t)h << 32) | v;
    }
  for (int64_t e = 0; e < bg_samples; ++e) {
    uint32_t u = (uint32_t)(draw(seed, 5, (uint64_t)e) % (uint64_t)n);
    uint32_t v = (uint32_t)(draw(seed, 6, (uint64_t)e) % (uint64_t)n);
    ek[ne++] = ((uint64_t)u << 32) | v;
  }
  int64_t m = keys_to_csr(n, ek, ne, xadj, adj_out);
  free(ek);
  return m;
}

/*
 * Symmetric random integer weights: vertex weights in [1, vmax] and edge
 * weights in [1, emax] with w(u,v) = w(v,u) (drawn from the unordered pair).
 */
void gg_weights(int32_t n, const int64_t *xadj, const int32_t *adj, int32_t vmax,
                int32_t emax, uint64_t seed, int32_t *vwgt, int32_t *adjwgt) {
  if (vwgt)
    for (int32_t v = 0; v < n; ++v)
      vwgt[v] = 1 + (int32_t)(draw(seed, 8, (uint64_t)v) % (uint64_t)vmax);
  if (adjwgt)
    for (int32_t v = 0; v < n; ++v)
      for (int64_t e = xadj[v]; e < xadj[v + 1]; ++e) {
        uint32_t a = (uint32_t)v, b = (uint32_t)adj[e];
        uint64_t lo = a < b ? a : b, hi = a < b ? b : a;
        adjwgt[e] = 1 + (int32_t)(draw(seed, 9, (lo << 32) | hi) % (uint64_t)emax);
      }
}

void gg_free(void *p) { free(p); }
