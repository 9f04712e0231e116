/*
 * Seeded synthetic graph inputs: R-MAT edge generation, symmetrisation and CSR assembly.
 *
 * This file generates INPUTS only.  It holds none of the eigensolver's or the SpMM's
 * arithmetic; both the CPU oracle tests and the CUDA tests/benchmarks read the graphs it
 * produces.
 *
 * R-MAT (Chakrabarti, Zhan, Faloutsos, SDM 2004): every edge descends `scale` levels of the
 * adjacency matrix, choosing one of four quadrants with probabilities a, b, c, d = 1-a-b-c.
 * The stand-in recipe for the paper's power-law graphs (Section 4, Table "graphs"): edge factor
 * 16, a/b/c/d = 0.57/0.19/0.19/0.05, a seeded random relabelling of the vertices (so hubs are
 * spread over the id range, as in real graphs whose vertex connection is nearly random), then
 * symmetrise, drop self-loops and duplicate edges, 0/1 pattern-only CSR.  Directed graphs
 * (the SVD path; the paper's page graph, Section 4.3.2) keep the draws as out-edges.
 *
 * Randomness: SplitMix64 (Steele, Lea, Flood, OOPSLA 2014) used as a counter-based hash of
 * (seed, stream, counter), so the graph depends only on the seed, not on the thread count.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static inline uint64_t sm64_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
/* counter-based draw: the i-th output of a SplitMix64 sequence whose state starts at a
 * seed- and stream-dependent value (state_i = state_0 + (i+1) * golden gamma). */
static inline uint64_t sm64_at(uint64_t seed, uint64_t stream, uint64_t i) {
  uint64_t s0 = sm64_mix(seed * 0x9E3779B97F4A7C15ull + stream * 0xD1B54A32D192ED03ull + 0x632BE59BD9B4E019ull);
  return sm64_mix(s0 + (i + 1) * 0x9E3779B97F4A7C15ull);
}
static inline double u01(uint64_t z) { return (double)(z >> 11) * (1.0 / 9007199254740992.0); }

/* Fisher-Yates permutation of [0, n) driven by the counter-based stream 1. */
static void make_perm(int64_t n, uint64_t seed, int32_t* perm) {
  for (int64_t i = 0; i < n; ++i) perm[i] = (int32_t)i;
  for (int64_t i = n - 1; i > 0; --i) {
    uint64_t j = sm64_at(seed, 1, (uint64_t)i) % (uint64_t)(i + 1);
    int32_t t = perm[i]; perm[i] = perm[j]; perm[j] = t;
  }
}

static int cmp_i32(const void* a, const void* b) {
  int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
  return (x > y) - (x < y);
}
static void sort_small(int32_t* v, int64_t len) {
  if (len > 48) { qsort(v, (size_t)len, sizeof(int32_t), cmp_i32); return; }
  for (int64_t i = 1; i < len; ++i) {
    int32_t x = v[i]; int64_t j = i - 1;
    while (j >= 0 && v[j] > x) { v[j + 1] = v[j]; --j; }
    v[j + 1] = x;
  }
}

/*
 * CSR of a directed edge list (src[e] -> dst[e]) with self-loops and duplicate edges
 * dropped and sorted column indices.  symmetric != 0 stores every edge in both directions
 * (an undirected graph); otherwise row u holds the out-neighbours of u.  Returns 0 on
 * success, -1 on allocation failure.  *rowptr_out (n+1 int64) and *colidx_out (nnz int32)
 * are malloc'ed; free with fe_gen_free.
 */
static int build_csr(int64_t n, int64_t m, const int32_t* src, const int32_t* dst, int symmetric,
                     int64_t** rowptr_out, int32_t** colidx_out, int64_t* nnz_out) {
  int64_t* cnt = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
  if (!cnt) return -1;
  #pragma omp parallel for schedule(static)
  for (int64_t e = 0; e < m; ++e) {
    int32_t u = src[e], v = dst[e];
    if (u == v) continue;
    #pragma omp atomic
    cnt[u + 1]++;
    if (symmetric) {
      #pragma omp atomic
      cnt[v + 1]++;
    }
  }
  for (int64_t i = 0; i < n; ++i) cnt[i + 1] += cnt[i];
  int64_t total = cnt[n];
  int32_t* tmp = (int32_t*)malloc((size_t)(total > 0 ? total : 1) * sizeof(int32_t));
  int64_t* cur = (int64_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
  if (!tmp || !cur) { free(cnt); free(tmp); free(cur); return -1; }
  memcpy(cur, cnt, (size_t)n * sizeof(int64_t));
  #pragma omp parallel for schedule(static)
  for (int64_t e = 0; e < m; ++e) {
    int32_t u = src[e], v = dst[e];
    if (u == v) continue;
    int64_t pu;
    #pragma omp atomic capture
    pu = cur[u]++;
    tmp[pu] = v;
    if (symmetric) {
      int64_t pv;
      #pragma omp atomic capture
      pv = cur[v]++;
      tmp[pv] = u;
    }
  }
  free(cur);
  /* sort + unique each row in place, record unique counts */
  int64_t* ucnt = (int64_t*)malloc((size_t)(n + 1) * sizeof(int64_t));
  if (!ucnt) { free(cnt); free(tmp); return -1; }
  ucnt[0] = 0;
  #pragma omp parallel for schedule(dynamic, 1024)
  for (int64_t i = 0; i < n; ++i) {
    int32_t* row = tmp + cnt[i];
    int64_t len = cnt[i + 1] - cnt[i];
    sort_small(row, len);
    int64_t k = 0;
    for (int64_t j = 0; j < len; ++j)
      if (k == 0 || row[j] != row[k - 1]) row[k++] = row[j];
    ucnt[i + 1] = k;
  }
  for (int64_t i = 0; i < n; ++i) ucnt[i + 1] += ucnt[i];
  int64_t nnz = ucnt[n];
  int32_t* col = (int32_t*)malloc((size_t)(nnz > 0 ? nnz : 1) * sizeof(int32_t));
  if (!col) { free(cnt); free(tmp); free(ucnt); return -1; }
  #pragma omp parallel for schedule(dynamic, 1024)
  for (int64_t i = 0; i < n; ++i)
    memcpy(col + ucnt[i], tmp + cnt[i], (size_t)(ucnt[i + 1] - ucnt[i]) * sizeof(int32_t));
  free(tmp);
  free(cnt);
  *rowptr_out = ucnt;
  *colidx_out = col;
  *nnz_out = nnz;
  return 0;
}

/* Undirected graph of an edge list (both directions stored). */
int fe_gen_symmetrize(int64_t n, int64_t m, const int32_t* src, const int32_t* dst,
                      int64_t** rowptr_out, int32_t** colidx_out, int64_t* nnz_out) {
  return build_csr(n, m, src, dst, 1, rowptr_out, colidx_out, nnz_out);
}

/* Directed graph of an edge list (row u = out-neighbours of u). */
int fe_gen_directed(int64_t n, int64_t m, const int32_t* src, const int32_t* dst,
                    int64_t** rowptr_out, int32_t** colidx_out, int64_t* nnz_out) {
  return build_csr(n, m, src, dst, 0, rowptr_out, colidx_out, nnz_out);
}

/*
 * Generate an R-MAT graph with n = 2^scale vertices and edge_factor * n directed draws.
 * permute != 0 applies the seeded vertex relabelling; directed != 0 keeps the draws as
 * directed edges (row u = out-neighbours), otherwise the graph is symmetrised.
 */
int fe_gen_rmat_ex(int scale, int64_t edge_factor, double a, double b, double c, uint64_t seed,
                   int permute, int directed, int64_t* n_out, int64_t** rowptr_out,
                   int32_t** colidx_out, int64_t* nnz_out) {
  if (scale < 1 || scale > 30 || edge_factor < 1) return -2;
  int64_t n = (int64_t)1 << scale;
  int64_t m = edge_factor * n;
  int32_t* src = (int32_t*)malloc((size_t)m * sizeof(int32_t));
  int32_t* dst = (int32_t*)malloc((size_t)m * sizeof(int32_t));
  int32_t* perm = permute ? (int32_t*)malloc((size_t)n * sizeof(int32_t)) : NULL;
  if (!src || !dst || (permute && !perm)) { free(src); free(dst); free(perm); return -1; }
  if (permute) make_perm(n, seed, perm);
  const double ab = a + b, abc = a + b + c;
  #pragma omp parallel for schedule(static)
  for (int64_t e = 0; e < m; ++e) {
    int64_t u = 0, v = 0;
    for (int l = 0; l < scale; ++l) {
      double r = u01(sm64_at(seed, 2, (uint64_t)e * 64u + (uint64_t)l));
      int bu, bv;
      if (r < a) { bu = 0; bv = 0; }
      else if (r < ab) { bu = 0; bv = 1; }
      else if (r < abc) { bu = 1; bv = 0; }
      else { bu = 1; bv = 1; }
      u = (u << 1) | bu;
      v = (v << 1) | bv;
    }
    src[e] = permute ? perm[u] : (int32_t)u;
    dst[e] = permute ? perm[v] : (int32_t)v;
  }
  free(perm);
  int rc = build_csr(n, m, src, dst, directed ? 0 : 1, rowptr_out, colidx_out, nnz_out);
  free(src);
  free(dst);
  if (rc == 0) *n_out = n;
  return rc;
}

/* Symmetrised R-MAT graph (see fe_gen_rmat_ex). */
int fe_gen_rmat(int scale, int64_t edge_factor, double a, double b, double c, uint64_t seed,
                int permute, int64_t* n_out, int64_t** rowptr_out, int32_t** colidx_out,
                int64_t* nnz_out) {
  return fe_gen_rmat_ex(scale, edge_factor, a, b, c, seed, permute, 0, n_out, rowptr_out,
                        colidx_out, nnz_out);
}

void fe_gen_free(void* p) { free(p); }

/* Seeded uniform [0,1) draws from the same counter-based generator (stream 3). */
void fe_gen_uniform(uint64_t seed, int64_t count, double* out) {
  #pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < count; ++i) out[i] = u01(sm64_at(seed, 3, (uint64_t)i));
}
