/*
 * CAPS CPU oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, sequential-by-definition restatement of CAPS (Constrained
 * Approximate Partitioned Search, arXiv 2308.15014) used to check the CUDA
 * path.  Only the test suite, the smoke check and the benchmark's CPU-baseline
 * leg may load this library; the product path never does.  It shares no code,
 * header, table or helper with the CUDA library.
 *
 * Conventions (each a reading of a point the paper leaves open):
 *   - Query filter (Def. 1) with variable constraints (Sec. 6.1): a query field
 *     set to -1 is unconstrained.  Sparse label sets: the filter holds when
 *     every required label is present.
 *   - Distances are computed in fp32 in a fixed order (j = 0..d-1, one fused
 *     multiply-add per coordinate).  Every integer decision (partition
 *     assignment, probe order, top-k order) is taken on that fp32 value, with
 *     ties broken towards the lower index.  An fp64 twin is provided for
 *     ground truth and error reports.
 *   - Inner product: larger is better; k-means on inner product normalises
 *     each centroid (spherical k-means).
 *   - k-means (Sec. 5.2): Lloyd iterations from given seed points, centroid
 *     = fp64 mean of members summed in id order, rounded to fp32; an empty
 *     partition keeps its centroid; a final assignment follows the last
 *     update.
 *   - Attribute frequency tree (Alg. 1): the most frequent code among the
 *     points not yet peeled, tie towards the lowest code; -1 tags once no
 *     point (or no code) remains.
 *   - Sub-partition selection (Alg. 2): j* = first tag carried by the query;
 *     select every block j <= j* whose tag does not contradict the query, and
 *     the remainder block only when no tag matches.  This is the smallest
 *     tag-determined block set that holds every valid point of the bin.
 *
 * Parity status: every function below is pinned by the test suite against
 * hand-worked examples, closed forms, invariants or brute force.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_L2 0
#define ORC_IP 1

typedef struct {
  int L;                 /* dense fields (0 for sparse) */
  const int32_t* A;      /* [N*L] dense values */
  const int32_t* vocab;  /* [L] */
  const int64_t* sp_off; /* [N+1] sparse CSR offsets */
  const int32_t* sp_lab; /* sorted labels */
  int32_t sp_vocab;
} attrs_t;

static attrs_t mk_attrs(int L, const int32_t* A, const int32_t* vocab,
                        const int64_t* sp_off, const int32_t* sp_lab,
                        int32_t sp_vocab) {
  attrs_t a;
  a.L = L;
  a.A = A;
  a.vocab = vocab;
  a.sp_off = sp_off;
  a.sp_lab = sp_lab;
  a.sp_vocab = sp_vocab;
  return a;
}

static int is_dense(const attrs_t* a) { return a->A != NULL; }

/* Total number of distinct attribute codes: a dense (field, value) pair is
 * the code off[field] + value, a sparse label is its own code. */
static int64_t n_codes(const attrs_t* a) {
  if (!is_dense(a)) return a->sp_vocab;
  int64_t s = 0;
  for (int f = 0; f < a->L; f++) s += a->vocab[f];
  return s;
}

static int64_t field_offset(const attrs_t* a, int f) {
  int64_t s = 0;
  for (int g = 0; g < f; g++) s += a->vocab[g];
  return s;
}

/* Does point i carry code c? */
static int carries(const attrs_t* a, int64_t i, int64_t c) {
  if (is_dense(a)) {
    for (int f = 0; f < a->L; f++)
      if (field_offset(a, f) + a->A[i * a->L + f] == c) return 1;
    return 0;
  }
  for (int64_t r = a->sp_off[i]; r < a->sp_off[i + 1]; r++)
    if (a->sp_lab[r] == c) return 1;
  return 0;
}

/* ---- Def. 1: query filter -------------------------------------------- */

int orc_filter_dense(const int32_t* a, const int32_t* b, int L) {
  for (int f = 0; f < L; f++)
    if (b[f] >= 0 && a[f] != b[f]) return 0;
  return 1;
}

int orc_filter_sparse(const int32_t* a, int64_t na, const int32_t* b,
                      int64_t nb) {
  for (int64_t u = 0; u < nb; u++) {
    int found = 0;
    for (int64_t v = 0; v < na; v++)
      if (a[v] == b[u]) found = 1;
    if (!found) return 0;
  }
  return 1;
}

/* C(b, a_i) for data point i and query qi. */
static int filter_point(const attrs_t* a, int64_t i, const int32_t* Qb,
                        const int64_t* q_off, const int32_t* q_lab, int64_t qi) {
  if (is_dense(a)) return orc_filter_dense(a->A + i * a->L, Qb + qi * a->L, a->L);
  return orc_filter_sparse(a->sp_lab + a->sp_off[i], a->sp_off[i + 1] - a->sp_off[i],
                           q_lab + q_off[qi], q_off[qi + 1] - q_off[qi]);
}

/* ---- distances --------------------------------------------------------- */

float orc_dist32(const float* x, const float* q, int d, int metric) {
  float acc = 0.0f;
  if (metric == ORC_L2) {
    for (int j = 0; j < d; j++) {
      float t = x[j] - q[j];
      acc = fmaf(t, t, acc);
    }
  } else {
    for (int j = 0; j < d; j++) acc = fmaf(x[j], q[j], acc);
  }
  return acc;
}

double orc_dist64(const float* x, const float* q, int d, int metric) {
  double acc = 0.0;
  if (metric == ORC_L2) {
    for (int j = 0; j < d; j++) {
      double t = (double)x[j] - (double)q[j];
      acc += t * t;
    }
  } else {
    for (int j = 0; j < d; j++) acc += (double)x[j] * (double)q[j];
  }
  return acc;
}

/* Is (s1, i1) strictly better than (s2, i2)?  L2: smaller; IP: larger;
 * ties towards the lower index. */
static int better(double s1, int64_t i1, double s2, int64_t i2, int metric) {
  if (s1 != s2) return metric == ORC_L2 ? (s1 < s2) : (s1 > s2);
  return i1 < i2;
}

/* ---- Alg. 1, first level: f(x) = best centroid --------------------------- */

void orc_assign(const float* X, int64_t N, int d, const float* C, int B,
                int metric, int32_t* bin) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < N; i++) {
    int best = 0;
    float bs = orc_dist32(X + i * d, C, d, metric);
    for (int c = 1; c < B; c++) {
      float s = orc_dist32(X + i * d, C + (int64_t)c * d, d, metric);
      if (better(s, c, bs, best, metric)) {
        best = c;
        bs = s;
      }
    }
    bin[i] = best;
  }
}

/* Centroid update: fp64 mean of the members in id order (spherical for IP). */
void orc_centroid_update(const float* X, int64_t N, int d, const int32_t* bin,
                         int B, int metric, float* C) {
  double* sum = (double*)calloc((size_t)B * d, sizeof(double));
  int64_t* cnt = (int64_t*)calloc((size_t)B, sizeof(int64_t));
  for (int64_t i = 0; i < N; i++) {
    int c = bin[i];
    cnt[c] += 1;
    for (int j = 0; j < d; j++) sum[(int64_t)c * d + j] += (double)X[i * d + j];
  }
  for (int c = 0; c < B; c++) {
    if (cnt[c] == 0) continue; /* empty partition keeps its centroid */
    double* s = sum + (int64_t)c * d;
    for (int j = 0; j < d; j++) s[j] = s[j] / (double)cnt[c];
    if (metric == ORC_IP) {
      double nrm = 0.0;
      for (int j = 0; j < d; j++) nrm += s[j] * s[j];
      nrm = sqrt(nrm);
      if (nrm > 0.0)
        for (int j = 0; j < d; j++) s[j] = s[j] / nrm;
    }
    for (int j = 0; j < d; j++) C[(int64_t)c * d + j] = (float)s[j];
  }
  free(sum);
  free(cnt);
}

void orc_kmeans(const float* X, int64_t N, int d, int B, int iters,
                const int64_t* init_idx, int metric, float* C, int32_t* bin) {
  for (int c = 0; c < B; c++)
    memcpy(C + (int64_t)c * d, X + init_idx[c] * d, sizeof(float) * d);
  for (int it = 0; it < iters; it++) {
    orc_assign(X, N, d, C, B, metric, bin);
    orc_centroid_update(X, N, d, bin, B, metric, C);
  }
  orc_assign(X, N, d, C, B, metric, bin);
}

/* ---- Alg. 1, second level: attribute frequency tree ----------------------- */

int orc_aft(const int32_t* bin, int64_t N, int B, int h, int L, const int32_t* A,
            const int32_t* vocab, const int64_t* sp_off, const int32_t* sp_lab,
            int32_t sp_vocab, int32_t* tags, uint8_t* key) {
  attrs_t a = mk_attrs(L, A, vocab, sp_off, sp_lab, sp_vocab);
  int64_t V = n_codes(&a);
  int64_t* count = (int64_t*)malloc(sizeof(int64_t) * (size_t)(V > 0 ? V : 1));
  uint8_t* peeled = (uint8_t*)calloc((size_t)(N > 0 ? N : 1), 1);
  /* P_bin as id-ordered member lists */
  int64_t* start = (int64_t*)calloc((size_t)B + 1, sizeof(int64_t));
  int64_t* members = (int64_t*)malloc(sizeof(int64_t) * (size_t)(N > 0 ? N : 1));
  for (int64_t i = 0; i < N; i++) start[bin[i] + 1]++;
  for (int b = 0; b < B; b++) start[b + 1] += start[b];
  int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)B + 1);
  for (int b = 0; b < B; b++) fill[b] = start[b];
  for (int64_t i = 0; i < N; i++) members[fill[bin[i]]++] = i;
  for (int b = 0; b < B; b++) {
    int done = 0;
    for (int j = 1; j <= h; j++) {
      int32_t t = -1;
      if (!done) {
        /* t = top-attribute(P_bin - S): most frequent code, lowest on ties */
        memset(count, 0, sizeof(int64_t) * (size_t)V);
        int64_t remaining = 0;
        for (int64_t u = start[b]; u < start[b + 1]; u++) {
          int64_t i = members[u];
          if (peeled[i]) continue;
          remaining++;
          if (is_dense(&a)) {
            for (int f = 0; f < L; f++) count[field_offset(&a, f) + A[i * L + f]]++;
          } else {
            for (int64_t r = sp_off[i]; r < sp_off[i + 1]; r++) count[sp_lab[r]]++;
          }
        }
        int64_t best = 0;
        for (int64_t c = 0; c < V; c++)
          if (count[c] > count[best]) best = c;
        if (remaining > 0 && V > 0 && count[best] > 0) t = (int32_t)best;
        else done = 1;
      }
      tags[(int64_t)b * h + (j - 1)] = t;
      if (t < 0) continue;
      /* p_j = points of P_bin - S carrying t; S = S + p_j */
      for (int64_t u = start[b]; u < start[b + 1]; u++) {
        int64_t i = members[u];
        if (peeled[i]) continue;
        if (carries(&a, i, t)) {
          key[i] = (uint8_t)j;
          peeled[i] = 1;
        }
      }
    }
    /* p_{h+1} = P_bin - S */
    for (int64_t u = start[b]; u < start[b + 1]; u++)
      if (!peeled[members[u]]) key[members[u]] = (uint8_t)(h + 1);
  }
  free(fill);
  free(members);
  free(start);
  free(count);
  free(peeled);
  return 0;
}

/* ---- contiguous layout: order points by (bin, block, id) ----------------- */

static const int32_t* g_sort_bin;
static const uint8_t* g_sort_key;
static int cmp_layout(const void* pa, const void* pb) {
  int64_t i = *(const int64_t*)pa, j = *(const int64_t*)pb;
  if (g_sort_bin[i] != g_sort_bin[j]) return g_sort_bin[i] < g_sort_bin[j] ? -1 : 1;
  if (g_sort_key[i] != g_sort_key[j]) return g_sort_key[i] < g_sort_key[j] ? -1 : 1;
  return (i > j) - (i < j);
}

void orc_layout(const int32_t* bin, const uint8_t* key, int64_t N, int B, int h,
                int32_t* perm, int32_t* offsets) {
  int64_t* idx = (int64_t*)malloc(sizeof(int64_t) * (size_t)(N > 0 ? N : 1));
  for (int64_t i = 0; i < N; i++) idx[i] = i;
  g_sort_bin = bin;
  g_sort_key = key;
  qsort(idx, (size_t)N, sizeof(int64_t), cmp_layout);
  for (int64_t r = 0; r < N; r++) perm[r] = (int32_t)idx[r];
  int64_t nseg = (int64_t)B * (h + 1);
  int64_t* cnt = (int64_t*)calloc((size_t)nseg, sizeof(int64_t));
  for (int64_t i = 0; i < N; i++) cnt[(int64_t)bin[i] * (h + 1) + (key[i] - 1)]++;
  int64_t run = 0;
  for (int64_t s = 0; s < nseg; s++) {
    offsets[s] = (int32_t)run;
    run += cnt[s];
  }
  offsets[nseg] = (int32_t)run;
  free(cnt);
  free(idx);
}

/* ---- Alg. 2: probe, sub-partition selection, attribute + vector match ------ */

typedef struct {
  double s;
  int64_t i;
  float s32;
  double s64;
} cand_t;

/* qsort's comparator reads the metric from a global; each thread sorts its
 * own array, so the global is thread-private. */
static int g_metric_cmp;
#ifdef _OPENMP
#pragma omp threadprivate(g_metric_cmp)
#endif
static int cmp_cand(const void* pa, const void* pb) {
  const cand_t* a = (const cand_t*)pa;
  const cand_t* b = (const cand_t*)pb;
  if (better(a->s, a->i, b->s, b->i, g_metric_cmp)) return -1;
  if (better(b->s, b->i, a->s, a->i, g_metric_cmp)) return 1;
  return 0;
}

void orc_probe(const float* Q, int64_t nq, int d, const float* C, int B,
               int metric, int m, int32_t* probe) {
#pragma omp parallel
  {
    cand_t* s = (cand_t*)malloc(sizeof(cand_t) * (size_t)B);
    g_metric_cmp = metric;
#pragma omp for schedule(dynamic, 4)
    for (int64_t q = 0; q < nq; q++) {
      for (int c = 0; c < B; c++) {
        s[c].s32 = orc_dist32(Q + q * d, C + (int64_t)c * d, d, metric);
        s[c].s = s[c].s32;
        s[c].i = c;
      }
      qsort(s, (size_t)B, sizeof(cand_t), cmp_cand);
      for (int r = 0; r < m; r++) probe[q * m + r] = (int32_t)s[r].i;
    }
    free(s);
  }
}

/* Code -> (field, value) for dense attributes. */
static void code_field(const attrs_t* a, int64_t code, int* f, int32_t* v) {
  int g = 0;
  while (g + 1 < a->L && field_offset(a, g + 1) <= code) g++;
  *f = g;
  *v = (int32_t)(code - field_offset(a, g));
}

/* Does the query (dense row b, or sparse list) require code t? */
static int query_has(const attrs_t* a, const int32_t* b, const int32_t* lab,
                     int64_t nlab, int64_t t) {
  if (is_dense(a)) {
    int f;
    int32_t v;
    code_field(a, t, &f, &v);
    return b[f] == v;
  }
  for (int64_t u = 0; u < nlab; u++)
    if (lab[u] == t) return 1;
  return 0;
}

/* May a point carrying code t still satisfy the query? */
static int query_compatible(const attrs_t* a, const int32_t* b, int64_t t) {
  if (!is_dense(a)) return 1;
  int f;
  int32_t v;
  code_field(a, t, &f, &v);
  return b[f] < 0 || b[f] == v;
}

static uint64_t select_blocks(const attrs_t* a, const int32_t* tags, int h,
                              int32_t b_bin, const int32_t* b, const int32_t* lab,
                              int64_t nlab) {
  const int32_t* t = tags + (int64_t)b_bin * h;
  int jstar = h + 1;
  for (int j = 1; j <= h; j++) {
    if (t[j - 1] < 0) break;
    if (query_has(a, b, lab, nlab, t[j - 1])) {
      jstar = j;
      break;
    }
  }
  uint64_t sel = 0;
  int jmax = jstar < h ? jstar : h;
  for (int j = 1; j <= jmax; j++) {
    if (t[j - 1] < 0) continue;
    if (query_compatible(a, b, t[j - 1])) sel |= (uint64_t)1 << (j - 1);
  }
  if (jstar == h + 1) sel |= (uint64_t)1 << h;
  return sel;
}

/* Selected-block bitmask (bit j-1 = block j) for each (query, probed bin). */
void orc_select(const int32_t* tags, int h, int L, const int32_t* vocab,
                int32_t sp_vocab, const int32_t* probe, int64_t nq, int m,
                const int32_t* Qb, const int64_t* q_off, const int32_t* q_lab,
                uint64_t* sel) {
  attrs_t a = mk_attrs(L, Qb /* non-NULL marks dense */, vocab, NULL, NULL, sp_vocab);
  for (int64_t q = 0; q < nq; q++) {
    const int32_t* b = Qb ? Qb + q * L : NULL;
    const int32_t* lab = Qb ? NULL : q_lab + q_off[q];
    int64_t nlab = Qb ? 0 : q_off[q + 1] - q_off[q];
    for (int r = 0; r < m; r++)
      sel[q * m + r] = select_blocks(&a, tags, h, probe[q * m + r], b, lab, nlab);
  }
}

static void emit_topk(cand_t* c, int64_t nc, int k, int metric, int64_t* ids,
                      float* d32, double* d64) {
  qsort(c, (size_t)nc, sizeof(cand_t), cmp_cand);
  for (int r = 0; r < k; r++) {
    if (r < nc) {
      ids[r] = c[r].i;
      if (d32) d32[r] = c[r].s32;
      if (d64) d64[r] = c[r].s64;
    } else {
      ids[r] = -1;
      if (d32) d32[r] = metric == ORC_L2 ? INFINITY : -INFINITY;
      if (d64) d64[r] = metric == ORC_L2 ? INFINITY : -INFINITY;
    }
  }
}

/* Full CAPS query (Alg. 2) for nq queries.  n_scan[q] counts rows whose
 * attributes were tested, n_match[q] rows that passed the filter. */
void orc_search(const float* X, int64_t N, int d, int L, const int32_t* A,
                const int32_t* vocab, const int64_t* sp_off, const int32_t* sp_lab,
                int32_t sp_vocab, const float* C, int B, int metric,
                const int32_t* tags, int h, const int32_t* perm,
                const int32_t* offsets, const float* Q, int64_t nq,
                const int32_t* Qb, const int64_t* q_off, const int32_t* q_lab,
                int k, int m, int64_t* out_ids, float* out_dist, int64_t* n_scan,
                int64_t* n_match, const int32_t* probe_in) {
  /* probe_in (optional [nq*m]): partitions to probe (a learned f(q)); else
     the m nearest centroids */
  attrs_t a = mk_attrs(L, A, vocab, sp_off, sp_lab, sp_vocab);
  (void)N;
#pragma omp parallel
  {
    int32_t* probe = (int32_t*)malloc(sizeof(int32_t) * (size_t)m);
    int64_t cap = 1024;
    cand_t* cand = (cand_t*)malloc(sizeof(cand_t) * (size_t)cap);
    g_metric_cmp = metric;
#pragma omp for schedule(dynamic, 1)
    for (int64_t q = 0; q < nq; q++) {
      if (probe_in) memcpy(probe, probe_in + q * m, sizeof(int32_t) * (size_t)m);
      else orc_probe(Q + q * d, 1, d, C, B, metric, m, probe);
      const int32_t* b = A ? Qb + q * L : NULL;
      const int32_t* lab = A ? NULL : q_lab + q_off[q];
      int64_t nlab = A ? 0 : q_off[q + 1] - q_off[q];
      int64_t nc = 0, ns = 0;
      for (int r = 0; r < m; r++) {
        int32_t bn = probe[r];
        uint64_t sel = select_blocks(&a, tags, h, bn, b, lab, nlab);
        for (int j = 1; j <= h + 1; j++) {
          if (!((sel >> (j - 1)) & 1)) continue;
          int64_t s = (int64_t)bn * (h + 1) + (j - 1);
          for (int64_t row = offsets[s]; row < offsets[s + 1]; row++) {
            int64_t i = perm[row];
            ns++;
            if (!filter_point(&a, i, Qb, q_off, q_lab, q)) continue;
            if (nc == cap) {
              cap *= 2;
              cand = (cand_t*)realloc(cand, sizeof(cand_t) * (size_t)cap);
            }
            cand[nc].s32 = orc_dist32(X + i * d, Q + q * d, d, metric);
            cand[nc].s = cand[nc].s32;
            cand[nc].s64 = orc_dist64(X + i * d, Q + q * d, d, metric);
            cand[nc].i = i;
            nc++;
          }
        }
      }
      if (n_scan) n_scan[q] = ns;
      if (n_match) n_match[q] = nc;
      emit_topk(cand, nc, k, metric, out_ids + q * k, out_dist ? out_dist + q * k : NULL,
                NULL);
    }
    free(cand);
    free(probe);
  }
}

/* ---- dynamic insertion (Table 1 claims it; the mechanism is not given) ----
 * A new point x goes to partition f(x) and, inside it, to the first block j
 * (1..h) whose tag t_j it carries, else to the remainder block h+1: the block
 * the attribute-frequency peel of Alg. 1 gives a point, with the partition's
 * tags kept as they are.  key[i] = that block for point i of bins[i]. */
void orc_block_of(const int32_t* tags, int h, int L, const int32_t* A, const int32_t* vocab,
                  const int64_t* sp_off, const int32_t* sp_lab, int32_t sp_vocab,
                  const int32_t* bins, int64_t n, uint8_t* key) {
  attrs_t a = mk_attrs(L, A, vocab, sp_off, sp_lab, sp_vocab);
  for (int64_t i = 0; i < n; i++) {
    const int32_t* t = tags + (int64_t)bins[i] * h;
    int j = 1;
    for (; j <= h; j++) {
      if (t[j - 1] < 0) {
        j = h + 1;
        break;
      }
      if (carries(&a, i, t[j - 1])) break;
    }
    key[i] = (uint8_t)j;
  }
}

/* ---- disjunctive (OR) constraints (Sec. 5.3: several constraints map to
 * several sub-partitions) ---------------------------------------------------
 * Field f of query q allows the values vals[voff[q*L+f] .. voff[q*L+f+1]);
 * an empty list leaves the field unconstrained.  The filter holds when every
 * constrained field's value is in its list.  In a probed partition the
 * blocks scanned are the union, over every single-valued query of the cross
 * product of the lists, of the blocks Alg. 2 selects for it.  Dense
 * attributes only. */
static int filter_or(const int32_t* arow, int L, const int64_t* voff, const int32_t* vals,
                     int64_t q) {
  for (int f = 0; f < L; f++) {
    const int64_t b = voff[q * L + f], e = voff[q * L + f + 1];
    if (b == e) continue;
    int hit = 0;
    for (int64_t u = b; u < e; u++)
      if (vals[u] >= 0 && vals[u] == arow[f]) hit = 1;
    if (!hit) return 0;
  }
  return 1;
}

/* Union of Alg. 2's block selections over the cross product of the lists:
 * a mixed-radix count over the constrained fields walks every single-valued
 * query once. */
static uint64_t select_blocks_or(const attrs_t* a, const int32_t* tags, int h, int32_t b_bin,
                                 int L, const int64_t* voff, const int32_t* vals, int64_t q) {
  int32_t b[64];
  int64_t pos[64];
  for (int f = 0; f < L; f++) {
    pos[f] = voff[q * L + f];
    b[f] = pos[f] < voff[q * L + f + 1] ? vals[pos[f]] : -1;
  }
  uint64_t sel = 0;
  for (;;) {
    sel |= select_blocks(a, tags, h, b_bin, b, NULL, 0);
    int f = 0;
    for (; f < L; f++) {
      const int64_t e = voff[q * L + f + 1];
      if (voff[q * L + f] == e) continue;
      if (++pos[f] < e) {
        b[f] = vals[pos[f]];
        break;
      }
      pos[f] = voff[q * L + f];
      b[f] = vals[pos[f]];
    }
    if (f == L) break;
  }
  return sel;
}

void orc_select_or(const int32_t* tags, int h, int L, const int32_t* vocab,
                   const int32_t* probe, int64_t nq, int m, const int64_t* voff,
                   const int32_t* vals, uint64_t* sel) {
  attrs_t a = mk_attrs(L, vocab /* non-NULL marks dense */, vocab, NULL, NULL, 0);
  for (int64_t q = 0; q < nq; q++)
    for (int r = 0; r < m; r++)
      sel[q * m + r] = select_blocks_or(&a, tags, h, probe[q * m + r], L, voff, vals, q);
}

/* Alg. 2 with disjunctive constraints: probe (the m nearest centroids, or
 * probe_in), the union block selection above, the OR filter, distances and
 * the exact top-k (ties to the lower id). */
void orc_search_or(const float* X, int64_t N, int d, int L, const int32_t* A,
                   const int32_t* vocab, const float* C, int B, int metric,
                   const int32_t* tags, int h, const int32_t* perm, const int32_t* offsets,
                   const float* Q, int64_t nq, const int64_t* voff, const int32_t* vals, int k,
                   int m, int64_t* out_ids, float* out_dist, const int32_t* probe_in) {
  attrs_t a = mk_attrs(L, A, vocab, NULL, NULL, 0);
  (void)N;
#pragma omp parallel
  {
    int32_t* probe = (int32_t*)malloc(sizeof(int32_t) * (size_t)m);
    int64_t cap = 1024;
    cand_t* cand = (cand_t*)malloc(sizeof(cand_t) * (size_t)cap);
    g_metric_cmp = metric;
#pragma omp for schedule(dynamic, 1)
    for (int64_t q = 0; q < nq; q++) {
      if (probe_in) memcpy(probe, probe_in + q * m, sizeof(int32_t) * (size_t)m);
      else orc_probe(Q + q * d, 1, d, C, B, metric, m, probe);
      int64_t nc = 0;
      for (int r = 0; r < m; r++) {
        const int32_t bn = probe[r];
        const uint64_t sel = select_blocks_or(&a, tags, h, bn, L, voff, vals, q);
        for (int j = 1; j <= h + 1; j++) {
          if (!((sel >> (j - 1)) & 1)) continue;
          const int64_t s = (int64_t)bn * (h + 1) + (j - 1);
          for (int64_t row = offsets[s]; row < offsets[s + 1]; row++) {
            const int64_t i = perm[row];
            if (!filter_or(A + i * L, L, voff, vals, q)) continue;
            if (nc == cap) {
              cap *= 2;
              cand = (cand_t*)realloc(cand, sizeof(cand_t) * (size_t)cap);
            }
            cand[nc].s32 = orc_dist32(X + i * d, Q + q * d, d, metric);
            cand[nc].s = cand[nc].s32;
            cand[nc].s64 = orc_dist64(X + i * d, Q + q * d, d, metric);
            cand[nc].i = i;
            nc++;
          }
        }
      }
      emit_topk(cand, nc, k, metric, out_ids + q * k, out_dist ? out_dist + q * k : NULL, NULL);
    }
    free(cand);
    free(probe);
  }
}

/* Exact filtered kNN (Def. 2; ground truth): filter every point, rank by the
 * fp64 distance (order64 = 1) or by the canonical fp32 one (order64 = 0). */
void orc_bruteforce(const float* X, int64_t N, int d, int L, const int32_t* A,
                    const int32_t* vocab, const int64_t* sp_off,
                    const int32_t* sp_lab, int32_t sp_vocab, const float* Q,
                    int64_t nq, const int32_t* Qb, const int64_t* q_off,
                    const int32_t* q_lab, int k, int metric, int order64,
                    int64_t* out_ids, float* out_d32, double* out_d64,
                    int64_t* out_count) {
  attrs_t a = mk_attrs(L, A, vocab, sp_off, sp_lab, sp_vocab);
#pragma omp parallel
  {
    int64_t cap = 1024;
    cand_t* cand = (cand_t*)malloc(sizeof(cand_t) * (size_t)cap);
    g_metric_cmp = metric;
#pragma omp for schedule(dynamic, 1)
    for (int64_t q = 0; q < nq; q++) {
      int64_t nc = 0;
      for (int64_t i = 0; i < N; i++) {
        if (!filter_point(&a, i, Qb, q_off, q_lab, q)) continue;
        if (nc == cap) {
          cap *= 2;
          cand = (cand_t*)realloc(cand, sizeof(cand_t) * (size_t)cap);
        }
        cand[nc].s32 = orc_dist32(X + i * d, Q + q * d, d, metric);
        cand[nc].s64 = orc_dist64(X + i * d, Q + q * d, d, metric);
        cand[nc].s = order64 ? cand[nc].s64 : (double)cand[nc].s32;
        cand[nc].i = i;
        nc++;
      }
      if (out_count) out_count[q] = nc;
      emit_topk(cand, nc, k, metric, out_ids + q * k, out_d32 ? out_d32 + q * k : NULL,
                out_d64 ? out_d64 + q * k : NULL);
    }
    free(cand);
  }
}

int orc_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}

/* ---- Sec. 5.2 learned partitioner (BLISS-style MLP) ------------------------
 * f(x) = W2 relu(W1 x + b1) + b2, W1 [H x d], b1 [H], W2 [B x H], b2 [B]
 * (row-major, output index first).  Training minimises the mean softmax
 * cross-entropy between f(x_s) and a label distribution Y[s] over the B
 * partitions; the partition of x is argmax f(x) (ties to the lower index). */

/* fp64 forward: Z [n x B]; Hd [n x H] (post-ReLU) if not NULL */
void orc_mlp_forward64(const float* X, int64_t n, int d, int H, int B,
                       const double* W1, const double* b1, const double* W2,
                       const double* b2, double* Z, double* Hd) {
  double* h = (double*)malloc(sizeof(double) * (size_t)H);
  for (int64_t i = 0; i < n; i++) {
    for (int u = 0; u < H; u++) {
      double a = b1[u];
      for (int j = 0; j < d; j++) a += W1[(int64_t)u * d + j] * (double)X[i * d + j];
      h[u] = a > 0.0 ? a : 0.0;
      if (Hd) Hd[i * H + u] = h[u];
    }
    for (int c = 0; c < B; c++) {
      double a = b2[c];
      for (int u = 0; u < H; u++) a += W2[(int64_t)c * H + u] * h[u];
      Z[i * B + c] = a;
    }
  }
  free(h);
}

/* Mean softmax cross-entropy and its gradients (fp64). */
double orc_mlp_loss_grad(const float* X, int64_t n, int d, int H, int B,
                         const double* W1, const double* b1, const double* W2,
                         const double* b2, const float* Y, double* gW1, double* gb1,
                         double* gW2, double* gb2) {
  double* Z = (double*)malloc(sizeof(double) * (size_t)(n * B));
  double* Hd = (double*)malloc(sizeof(double) * (size_t)(n * H));
  double* dz = (double*)malloc(sizeof(double) * (size_t)B);
  double* dh = (double*)malloc(sizeof(double) * (size_t)H);
  orc_mlp_forward64(X, n, d, H, B, W1, b1, W2, b2, Z, Hd);
  memset(gW1, 0, sizeof(double) * (size_t)H * d);
  memset(gb1, 0, sizeof(double) * (size_t)H);
  memset(gW2, 0, sizeof(double) * (size_t)B * H);
  memset(gb2, 0, sizeof(double) * (size_t)B);
  double loss = 0.0;
  for (int64_t i = 0; i < n; i++) {
    const double* z = Z + i * B;
    double mx = z[0];
    for (int c = 1; c < B; c++) mx = z[c] > mx ? z[c] : mx;
    double se = 0.0;
    for (int c = 0; c < B; c++) se += exp(z[c] - mx);
    const double lse = mx + log(se);
    double ysum = 0.0;
    for (int c = 0; c < B; c++) ysum += (double)Y[i * B + c];
    for (int c = 0; c < B; c++) {
      const double p = exp(z[c] - lse);
      loss -= (double)Y[i * B + c] * (z[c] - lse);
      /* d/dz of -sum_c y_c log p_c = p * sum(y) - y */
      dz[c] = (p * ysum - (double)Y[i * B + c]) / (double)n;
    }
    const double* h = Hd + i * H;
    for (int c = 0; c < B; c++) {
      gb2[c] += dz[c];
      for (int u = 0; u < H; u++) gW2[(int64_t)c * H + u] += dz[c] * h[u];
    }
    for (int u = 0; u < H; u++) {
      double a = 0.0;
      for (int c = 0; c < B; c++) a += dz[c] * W2[(int64_t)c * H + u];
      dh[u] = h[u] > 0.0 ? a : 0.0;
    }
    for (int u = 0; u < H; u++) {
      gb1[u] += dh[u];
      for (int j = 0; j < d; j++) gW1[(int64_t)u * d + j] += dh[u] * (double)X[i * d + j];
    }
  }
  free(Z);
  free(Hd);
  free(dz);
  free(dh);
  return loss / (double)n;
}

/* Nearest bf16 value of v (8 significant bits, ties to the even one): with
 * v = m 2^e, 1/2 <= |m| < 1, the result is rint(m 2^8) 2^(e-8).  Finite
 * values inside the bf16 normal range only. */
double orc_bf16(double v) {
  if (v == 0.0 || !isfinite(v)) return v;
  int e;
  const double m = frexp(v, &e);
  return ldexp(nearbyint(ldexp(m, 8)), e - 8);
}

/* The training step with bf16 weights and activations (the learned
 * partitioner's "BF16 weights with FP32 master weights" form): the same mean
 * softmax cross-entropy, with every operand of a matrix product rounded to
 * bf16 first -- x and W1 in W1 x, the hidden activations h and W2 in W2 h,
 * dz and h in the W2 gradient, dz and W2 in the back-propagated dh, dh and x
 * in the W1 gradient -- each product then summed exactly (fp64 here).  Biases,
 * the ReLU mask, the softmax and the bias gradients (sums of the unrounded dz
 * and dh) stay at full precision.  The masters (W1, b1, W2, b2) are what the
 * optimizer updates. */
double orc_mlp_loss_grad_bf16(const float* X, int64_t n, int d, int H, int B,
                              const double* W1, const double* b1, const double* W2,
                              const double* b2, const float* Y, double* gW1, double* gb1,
                              double* gW2, double* gb2) {
  double* w1 = (double*)malloc(sizeof(double) * (size_t)H * d);
  double* w2 = (double*)malloc(sizeof(double) * (size_t)B * H);
  double* x = (double*)malloc(sizeof(double) * (size_t)d);
  double* h = (double*)malloc(sizeof(double) * (size_t)H);   /* relu(W1 x + b1) */
  double* hr = (double*)malloc(sizeof(double) * (size_t)H);  /* bf16(h) */
  double* z = (double*)malloc(sizeof(double) * (size_t)B);
  double* dz = (double*)malloc(sizeof(double) * (size_t)B);
  double* dzr = (double*)malloc(sizeof(double) * (size_t)B);
  double* dh = (double*)malloc(sizeof(double) * (size_t)H);
  for (int64_t i = 0; i < (int64_t)H * d; i++) w1[i] = orc_bf16(W1[i]);
  for (int64_t i = 0; i < (int64_t)B * H; i++) w2[i] = orc_bf16(W2[i]);
  memset(gW1, 0, sizeof(double) * (size_t)H * d);
  memset(gb1, 0, sizeof(double) * (size_t)H);
  memset(gW2, 0, sizeof(double) * (size_t)B * H);
  memset(gb2, 0, sizeof(double) * (size_t)B);
  double loss = 0.0;
  for (int64_t i = 0; i < n; i++) {
    for (int j = 0; j < d; j++) x[j] = orc_bf16((double)X[i * d + j]);
    for (int u = 0; u < H; u++) {
      double a = 0.0;
      for (int j = 0; j < d; j++) a += w1[(int64_t)u * d + j] * x[j];
      a += b1[u];
      h[u] = a > 0.0 ? a : 0.0;
      hr[u] = orc_bf16(h[u]);
    }
    for (int c = 0; c < B; c++) {
      double a = 0.0;
      for (int u = 0; u < H; u++) a += w2[(int64_t)c * H + u] * hr[u];
      z[c] = a + b2[c];
    }
    double mx = z[0];
    for (int c = 1; c < B; c++) mx = z[c] > mx ? z[c] : mx;
    double se = 0.0;
    for (int c = 0; c < B; c++) se += exp(z[c] - mx);
    const double lse = mx + log(se);
    double ysum = 0.0;
    for (int c = 0; c < B; c++) ysum += (double)Y[i * B + c];
    for (int c = 0; c < B; c++) {
      const double p = exp(z[c] - lse);
      loss -= (double)Y[i * B + c] * (z[c] - lse);
      dz[c] = (p * ysum - (double)Y[i * B + c]) / (double)n;
      dzr[c] = orc_bf16(dz[c]);
    }
    for (int c = 0; c < B; c++) {
      gb2[c] += dz[c];
      for (int u = 0; u < H; u++) gW2[(int64_t)c * H + u] += dzr[c] * hr[u];
    }
    for (int u = 0; u < H; u++) {
      double a = 0.0;
      for (int c = 0; c < B; c++) a += dzr[c] * w2[(int64_t)c * H + u];
      dh[u] = h[u] > 0.0 ? a : 0.0;
    }
    for (int u = 0; u < H; u++) {
      gb1[u] += dh[u];
      const double r = orc_bf16(dh[u]);
      for (int j = 0; j < d; j++) gW1[(int64_t)u * d + j] += r * x[j];
    }
  }
  free(w1);
  free(w2);
  free(x);
  free(h);
  free(hr);
  free(z);
  free(dz);
  free(dzr);
  free(dh);
  return loss / (double)n;
}

/* Adam (Kingma & Ba 2015) with bias correction; t counts from 1. */
void orc_adam(double* w, const double* g, double* m, double* v, int64_t n, double lr,
              double beta1, double beta2, double eps, int t) {
  const double c1 = 1.0 - pow(beta1, t), c2 = 1.0 - pow(beta2, t);
  for (int64_t i = 0; i < n; i++) {
    m[i] = beta1 * m[i] + (1.0 - beta1) * g[i];
    v[i] = beta2 * v[i] + (1.0 - beta2) * g[i] * g[i];
    w[i] -= lr * (m[i] / c1) / (sqrt(v[i] / c2) + eps);
  }
}

/* Balanced assignment of the learned partitioner's rounds (BLISS-style, Sec.
 * 5.2 "iterative learning scheme"): top[i*R .. i*R+R) lists point i's R best
 * partitions by fp32 logit, best first (ties to the lower partition).
 * Points are taken in id order; each goes to the candidate with the least
 * load so far (ties to the earlier candidate) and adds one to its load.
 * load0 (optional, [B]) gives the loads before the first point. */
void orc_balanced_assign(const int32_t* top, int64_t n, int R, int B, const int64_t* load0,
                         int32_t* bins) {
  int64_t* load = (int64_t*)calloc((size_t)B, sizeof(int64_t));
  if (load0) memcpy(load, load0, sizeof(int64_t) * (size_t)B);
  for (int64_t i = 0; i < n; i++) {
    int32_t best = top[i * R];
    for (int r = 1; r < R; r++) {
      const int32_t c = top[i * R + r];
      if (load[c] < load[best]) best = c;
    }
    bins[i] = best;
    load[best]++;
  }
  free(load);
}

/* fp32 forward in a fixed order (bias, then coordinates in order with one
 * fma each; ReLU), used to take the argmax decision the GPU takes. */
void orc_mlp_assign32(const float* X, int64_t n, int d, int H, int B, const float* W1,
                      const float* b1, const float* W2, const float* b2, int32_t* bin) {
#pragma omp parallel
  {
    float* h = (float*)malloc(sizeof(float) * (size_t)H);
#pragma omp for schedule(static)
    for (int64_t i = 0; i < n; i++) {
      for (int u = 0; u < H; u++) {
        float a = 0.0f;
        for (int j = 0; j < d; j++) a = fmaf(W1[(int64_t)u * d + j], X[i * d + j], a);
        a = a + b1[u];
        h[u] = a > 0.0f ? a : 0.0f;
      }
      int best = 0;
      float bs = 0.0f;
      for (int c = 0; c < B; c++) {
        float a = 0.0f;
        for (int u = 0; u < H; u++) a = fmaf(W2[(int64_t)c * H + u], h[u], a);
        a = a + b2[c];
        if (c == 0 || a > bs) {
          bs = a;
          best = c;
        }
      }
      bin[i] = best;
    }
    free(h);
  }
}

/* fp32 logits in the same fixed order (queries' partition scores). */
void orc_mlp_logits32(const float* X, int64_t n, int d, int H, int B, const float* W1,
                      const float* b1, const float* W2, const float* b2, float* Z) {
#pragma omp parallel
  {
    float* h = (float*)malloc(sizeof(float) * (size_t)H);
#pragma omp for schedule(static)
    for (int64_t i = 0; i < n; i++) {
      for (int u = 0; u < H; u++) {
        float a = 0.0f;
        for (int j = 0; j < d; j++) a = fmaf(W1[(int64_t)u * d + j], X[i * d + j], a);
        a = a + b1[u];
        h[u] = a > 0.0f ? a : 0.0f;
      }
      for (int c = 0; c < B; c++) {
        float a = 0.0f;
        for (int u = 0; u < H; u++) a = fmaf(W2[(int64_t)c * H + u], h[u], a);
        Z[i * B + c] = a + b2[c];
      }
    }
    free(h);
  }
}
