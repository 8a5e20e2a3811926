/*
 * Seeded synthetic bipartite edge lists.
 *
 * Input generation only: nothing in this file counts wedges or butterflies.
 * Both the CPU oracle and the CUDA library consume what it writes; neither
 * shares any other code.
 *
 * Random numbers: the k-th output of the SplitMix64 sequence (Steele, Lea and
 * Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014) seeded
 * with a per-stream key,
 *     r(key, k) = mix64(key + (k + 1) * 0x9E3779B97F4A7C15),
 * where mix64 is SplitMix64's output finaliser.  Being counter-based, any draw
 * can be recomputed independently, so the result does not depend on the number
 * of threads.
 *
 * Edges are drawn as candidate pairs (u, v) one after another; duplicates are
 * rejected and the first m distinct pairs, in draw order, are the output.
 * Bipartite ids: u in [0, nU), v in [0, nV).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define GOLDEN 0x9E3779B97F4A7C15ULL

static inline uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

/* k-th draw of the stream with key `key`. */
static inline uint64_t ctr(uint64_t key, uint64_t k) { return mix64(key + (k + 1) * GOLDEN); }

/* Key of sub-stream `s` of a seed. */
static inline uint64_t stream_key(uint64_t seed, uint64_t s) {
  return mix64(seed ^ mix64(0xD1B54A32D192ED03ULL * (s + 1)));
}

/* Uniform integer in [0, n) from the high 32 bits of r (n < 2^32). */
static inline uint32_t below(uint64_t r, uint32_t n) {
  return (uint32_t)(((r >> 32) * (uint64_t)n) >> 32);
}

uint64_t synth_draw(uint64_t seed, uint64_t stream, uint64_t k) {
  return ctr(stream_key(seed, stream), k);
}

/* ------------------------------------------------------------------ */
/* Walker/Vose alias table (Vose, IEEE TSE 1991) over weights p[0..n). */
typedef struct {
  uint32_t n;
  double *prob;
  uint32_t *alias;
} alias_t;

static int alias_build(alias_t *a, const double *w, uint32_t n) {
  a->n = n;
  a->prob = (double *)malloc(sizeof(double) * n);
  a->alias = (uint32_t *)malloc(sizeof(uint32_t) * n);
  uint32_t *small = (uint32_t *)malloc(sizeof(uint32_t) * n);
  uint32_t *large = (uint32_t *)malloc(sizeof(uint32_t) * n);
  double *q = (double *)malloc(sizeof(double) * n);
  if (!a->prob || !a->alias || !small || !large || !q) {
    free(small); free(large); free(q);
    return -1;
  }
  double tot = 0.0;
  for (uint32_t i = 0; i < n; i++) tot += w[i];
  uint32_t ns = 0, nl = 0;
  for (uint32_t i = 0; i < n; i++) {
    q[i] = w[i] * (double)n / tot;
    if (q[i] < 1.0) small[ns++] = i; else large[nl++] = i;
  }
  while (ns > 0 && nl > 0) {
    uint32_t s = small[--ns], l = large[--nl];
    a->prob[s] = q[s];
    a->alias[s] = l;
    q[l] = (q[l] + q[s]) - 1.0;
    if (q[l] < 1.0) small[ns++] = l; else large[nl++] = l;
  }
  while (nl > 0) { uint32_t l = large[--nl]; a->prob[l] = 1.0; a->alias[l] = l; }
  while (ns > 0) { uint32_t s = small[--ns]; a->prob[s] = 1.0; a->alias[s] = s; }
  free(small); free(large); free(q);
  return 0;
}

static inline uint32_t alias_draw(const alias_t *a, uint64_t r) {
  uint32_t i = below(r, a->n);
  double coin = (double)(uint32_t)(r & 0xFFFFFFFFu) * (1.0 / 4294967296.0);
  return coin < a->prob[i] ? i : a->alias[i];
}

static void alias_free(alias_t *a) { free(a->prob); free(a->alias); }

/* Seeded Fisher-Yates permutation of [0, n). */
static uint32_t *make_perm(uint64_t key, uint32_t n) {
  uint32_t *p = (uint32_t *)malloc(sizeof(uint32_t) * (n ? n : 1));
  if (!p) return NULL;
  for (uint32_t i = 0; i < n; i++) p[i] = i;
  for (uint32_t i = n; i > 1; i--) {
    uint32_t j = below(ctr(key, i), i);
    uint32_t t = p[i - 1]; p[i - 1] = p[j]; p[j] = t;
  }
  return p;
}

/* ------------------------------------------------------------------ */
/* Candidate drawing, in parallel over contiguous index ranges. */
typedef struct {
  int kind; /* 0 = uniform (Erdos-Renyi), 1 = alias tables (Chung-Lu) */
  uint32_t nU, nV;
  uint64_t keyU, keyV;
  const alias_t *aU, *aV;
  const uint32_t *permU, *permV;
} drawer_t;

static inline void draw_pair(const drawer_t *d, uint64_t k, uint32_t *u, uint32_t *v) {
  uint64_t ru = ctr(d->keyU, k), rv = ctr(d->keyV, k);
  if (d->kind == 0) {
    *u = below(ru, d->nU);
    *v = below(rv, d->nV);
  } else {
    uint32_t a = alias_draw(d->aU, ru), b = alias_draw(d->aV, rv);
    *u = d->permU ? d->permU[a] : a;
    *v = d->permV ? d->permV[b] : b;
  }
}

typedef struct {
  const drawer_t *d;
  uint64_t k0, k1;
  uint32_t *cu, *cv;
} draw_job_t;

static void *draw_worker(void *arg) {
  draw_job_t *j = (draw_job_t *)arg;
  for (uint64_t k = j->k0; k < j->k1; k++) draw_pair(j->d, k, &j->cu[k], &j->cv[k]);
  return NULL;
}

/* ------------------------------------------------------------------ */
/* First-occurrence deduplication, partitioned by a hash of the pair so that
 * partitions run in parallel; within a partition candidates stay in draw
 * order, so "first" means smallest draw index regardless of thread count. */
#define NPART 256

typedef struct {
  int t, nthreads;
  uint64_t K;
  const uint32_t *cu, *cv;
  uint64_t *cnt;      /* [nthreads][NPART] */
  uint64_t *pos;      /* [nthreads][NPART] write cursors */
  uint64_t *pkey;     /* partitioned keys */
  uint64_t *pidx;     /* partitioned draw indices */
  uint64_t *pstart;   /* [NPART+1] */
  uint8_t *first;     /* [K] */
  int phase;
  int err;
} dd_job_t;

static inline uint64_t pair_key(uint32_t u, uint32_t v) { return ((uint64_t)u << 32) | v; }
static inline uint32_t part_of(uint64_t key) { return (uint32_t)(mix64(key ^ 0x5851F42D4C957F2DULL) >> 56); }

static void *dd_worker(void *arg) {
  dd_job_t *j = (dd_job_t *)arg;
  uint64_t lo = j->K * (uint64_t)j->t / (uint64_t)j->nthreads;
  uint64_t hi = j->K * (uint64_t)(j->t + 1) / (uint64_t)j->nthreads;
  if (j->phase == 0) {
    uint64_t *c = j->cnt + (size_t)j->t * NPART;
    for (uint64_t k = lo; k < hi; k++) c[part_of(pair_key(j->cu[k], j->cv[k]))]++;
  } else if (j->phase == 1) {
    uint64_t *p = j->pos + (size_t)j->t * NPART;
    for (uint64_t k = lo; k < hi; k++) {
      uint64_t key = pair_key(j->cu[k], j->cv[k]);
      uint64_t at = p[part_of(key)]++;
      j->pkey[at] = key;
      j->pidx[at] = k;
    }
  } else {
    /* partitions t, t + nthreads, ... */
    for (uint32_t part = (uint32_t)j->t; part < NPART; part += (uint32_t)j->nthreads) {
      uint64_t s = j->pstart[part], e = j->pstart[part + 1], len = e - s;
      if (len == 0) continue;
      uint64_t cap = 16;
      while (cap < 2 * len) cap <<= 1;
      uint64_t *tab = (uint64_t *)malloc(sizeof(uint64_t) * cap);
      if (!tab) { j->err = 1; return NULL; }
      memset(tab, 0xFF, sizeof(uint64_t) * cap); /* all-ones is never a pair key: v < 2^32-1 */
      for (uint64_t a = s; a < e; a++) {
        uint64_t key = j->pkey[a];
        uint64_t h = mix64(key) & (cap - 1);
        for (;;) {
          if (tab[h] == key) break;
          if (tab[h] == ~0ULL) { tab[h] = key; j->first[j->pidx[a]] = 1; break; }
          h = (h + 1) & (cap - 1);
        }
      }
      free(tab);
    }
  }
  return NULL;
}

static int run_threads(int nthreads, void *(*fn)(void *), void *jobs, size_t job_size) {
  pthread_t th[256];
  int n = nthreads;
  for (int t = 1; t < n; t++)
    if (pthread_create(&th[t], NULL, fn, (char *)jobs + job_size * t) != 0) return -1;
  fn(jobs);
  for (int t = 1; t < n; t++) pthread_join(th[t], NULL);
  return 0;
}

/* Draw candidates until m distinct pairs exist; write the first m, in draw order. */
static int sample_distinct(const drawer_t *d, uint64_t m, int nthreads, uint32_t *u_out, uint32_t *v_out) {
  if (nthreads < 1) nthreads = 1;
  if (nthreads > 256) nthreads = 256;
  if (m == 0) return 0;
  uint64_t K = m + m / 16 + 1024, Kdone = 0;
  uint32_t *cu = NULL, *cv = NULL;
  for (int round = 0; round < 64; round++) {
    uint32_t *nu = (uint32_t *)realloc(cu, sizeof(uint32_t) * K);
    if (!nu) { free(cu); free(cv); return -2; }
    cu = nu;
    uint32_t *nv = (uint32_t *)realloc(cv, sizeof(uint32_t) * K);
    if (!nv) { free(cu); free(cv); return -2; }
    cv = nv;
    /* draw [Kdone, K) */
    draw_job_t dj[256];
    for (int t = 0; t < nthreads; t++) {
      dj[t].d = d; dj[t].cu = cu; dj[t].cv = cv;
      dj[t].k0 = Kdone + (K - Kdone) * (uint64_t)t / (uint64_t)nthreads;
      dj[t].k1 = Kdone + (K - Kdone) * (uint64_t)(t + 1) / (uint64_t)nthreads;
    }
    run_threads(nthreads, draw_worker, dj, sizeof(draw_job_t));
    Kdone = K;
    /* dedupe all K candidates */
    uint64_t *cnt = (uint64_t *)calloc((size_t)nthreads * NPART, sizeof(uint64_t));
    uint64_t *pos = (uint64_t *)calloc((size_t)nthreads * NPART, sizeof(uint64_t));
    uint64_t *pkey = (uint64_t *)malloc(sizeof(uint64_t) * K);
    uint64_t *pidx = (uint64_t *)malloc(sizeof(uint64_t) * K);
    uint8_t *first = (uint8_t *)calloc(K, 1);
    uint64_t pstart[NPART + 1];
    if (!cnt || !pos || !pkey || !pidx || !first) {
      free(cnt); free(pos); free(pkey); free(pidx); free(first); free(cu); free(cv);
      return -2;
    }
    dd_job_t jj[256];
    for (int t = 0; t < nthreads; t++) {
      jj[t].t = t; jj[t].nthreads = nthreads; jj[t].K = K; jj[t].cu = cu; jj[t].cv = cv;
      jj[t].cnt = cnt; jj[t].pos = pos; jj[t].pkey = pkey; jj[t].pidx = pidx;
      jj[t].pstart = pstart; jj[t].first = first; jj[t].phase = 0; jj[t].err = 0;
    }
    run_threads(nthreads, dd_worker, jj, sizeof(dd_job_t));
    uint64_t acc = 0;
    for (uint32_t p = 0; p < NPART; p++) {
      pstart[p] = acc;
      for (int t = 0; t < nthreads; t++) {
        pos[(size_t)t * NPART + p] = acc;
        acc += cnt[(size_t)t * NPART + p];
      }
    }
    pstart[NPART] = acc;
    for (int t = 0; t < nthreads; t++) jj[t].phase = 1;
    run_threads(nthreads, dd_worker, jj, sizeof(dd_job_t));
    for (int t = 0; t < nthreads; t++) jj[t].phase = 2;
    run_threads(nthreads, dd_worker, jj, sizeof(dd_job_t));
    int err = 0;
    for (int t = 0; t < nthreads; t++) err |= jj[t].err;
    free(cnt); free(pos); free(pkey); free(pidx);
    if (err) { free(first); free(cu); free(cv); return -2; }
    uint64_t D = 0;
    for (uint64_t k = 0; k < K; k++) D += first[k];
    if (D >= m) {
      uint64_t w = 0;
      for (uint64_t k = 0; k < K && w < m; k++)
        if (first[k]) { u_out[w] = cu[k]; v_out[w] = cv[k]; w++; }
      free(first); free(cu); free(cv);
      return 0;
    }
    free(first);
    /* grow by the deficit, scaled by the observed distinct rate */
    double rate = (double)D / (double)K;
    if (rate < 1e-6) rate = 1e-6;
    uint64_t need = (uint64_t)((double)(m - D) / rate * 1.15) + 1024;
    K += need;
  }
  free(cu); free(cv);
  return -3; /* could not reach m distinct pairs */
}

/* ------------------------------------------------------------------ */
int synth_er(uint64_t seed, uint32_t nU, uint32_t nV, uint64_t m, int nthreads,
             uint32_t *u, uint32_t *v) {
  if (nU == 0 || nV == 0) return m == 0 ? 0 : -1;
  if ((double)m > 0.5 * (double)nU * (double)nV) return -1;
  drawer_t d;
  memset(&d, 0, sizeof d);
  d.kind = 0; d.nU = nU; d.nV = nV;
  d.keyU = stream_key(seed, 1); d.keyV = stream_key(seed, 2);
  return sample_distinct(&d, m, nthreads, u, v);
}

/* Expected-degree weights: w_i = min(cap, c * (i+1)^(-1/(gamma-1))) with c
 * chosen (bisection on log c) so that sum_i w_i = m. */
static int chung_lu_weights(uint32_t n, uint64_t m, double gamma, double cap, double *w) {
  if (gamma <= 1.0 || n == 0) return -1;
  if (cap * (double)n < (double)m) return -1;
  double s = 1.0 / (gamma - 1.0);
  for (uint32_t i = 0; i < n; i++) w[i] = pow((double)i + 1.0, -s);
  double lo = -50.0, hi = 80.0;
  for (int it = 0; it < 200; it++) {
    double mid = 0.5 * (lo + hi), c = exp(mid), tot = 0.0;
    for (uint32_t i = 0; i < n; i++) { double x = c * w[i]; tot += x < cap ? x : cap; }
    if (tot < (double)m) lo = mid; else hi = mid;
  }
  double c = exp(hi);
  for (uint32_t i = 0; i < n; i++) { double x = c * w[i]; w[i] = x < cap ? x : cap; }
  return 0;
}

int synth_chung_lu(uint64_t seed, uint32_t nU, uint32_t nV, uint64_t m, double gammaU,
                   double gammaV, double capU, double capV, int permute, int nthreads,
                   uint32_t *u, uint32_t *v) {
  if (nU == 0 || nV == 0) return m == 0 ? 0 : -1;
  if ((double)m > 0.5 * (double)nU * (double)nV) return -1;
  double *wU = (double *)malloc(sizeof(double) * nU);
  double *wV = (double *)malloc(sizeof(double) * nV);
  if (!wU || !wV) { free(wU); free(wV); return -2; }
  if (chung_lu_weights(nU, m, gammaU, capU, wU) || chung_lu_weights(nV, m, gammaV, capV, wV)) {
    free(wU); free(wV);
    return -1;
  }
  alias_t aU, aV;
  if (alias_build(&aU, wU, nU) || alias_build(&aV, wV, nV)) { free(wU); free(wV); return -2; }
  free(wU); free(wV);
  uint32_t *pU = NULL, *pV = NULL;
  if (permute) {
    pU = make_perm(stream_key(seed, 3), nU);
    pV = make_perm(stream_key(seed, 4), nV);
  }
  drawer_t d;
  memset(&d, 0, sizeof d);
  d.kind = 1; d.nU = nU; d.nV = nV;
  d.keyU = stream_key(seed, 1); d.keyV = stream_key(seed, 2);
  d.aU = &aU; d.aV = &aV; d.permU = pU; d.permV = pV;
  int rc = sample_distinct(&d, m, nthreads, u, v);
  alias_free(&aU); alias_free(&aV);
  free(pU); free(pV);
  return rc;
}

/* Seeded shuffle of an edge list (used to present duplicate-bearing or
 * reordered inputs to both implementations). */
void synth_shuffle_pairs(uint64_t seed, uint64_t m, uint32_t *u, uint32_t *v) {
  uint64_t key = stream_key(seed, 5);
  for (uint64_t i = m; i > 1; i--) {
    uint64_t r = ctr(key, i);
    uint64_t j = (uint64_t)(((unsigned __int128)r * i) >> 64);
    uint32_t t = u[i - 1]; u[i - 1] = u[j]; u[j] = t;
    t = v[i - 1]; v[i - 1] = v[j]; v[j] = t;
  }
}
