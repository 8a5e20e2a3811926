/*
 * TEST INFRASTRUCTURE ONLY -- plain CPU oracle for exact butterfly counting.
 *
 * Only the tests, the smoke check and the benchmark's CPU-baseline leg may
 * load this file.  It shares no code with the CUDA library.
 *
 * It follows "Parallel Algorithms for Butterfly Computations" (Shi & Shun),
 * step by step and in the paper's order:
 *   - duplicate edges are removed (Sec. "Experiments / Environment");
 *   - PREPROCESS (Algorithm 1): vertices sorted by the rank function f, renamed
 *     to their rank, each adjacency list sorted by decreasing rank;
 *   - GET-WEDGES (Algorithm 2): for every x1, every y in N(x1) with
 *     rank(y) > rank(x1), every x2 in N(y) with rank(x2) > rank(x1), the wedge
 *     ((x1, x2), y);
 *   - GET-FREQ with the simple batching option (Sec. "Wedge aggregation"):
 *     x1 aggregates its wedges in a dense array indexed by the second endpoint;
 *   - butterfly aggregation with atomic adds (Sec. "Butterfly aggregation"):
 *     global += C(d,2); per vertex, both endpoints += C(d,2) and each center
 *     += d - 1 (Algorithm 3, Eq. 1); per edge, both wedge edges += d - 1
 *     (Algorithm 4, Eq. 2).
 * It also gives the exact retrieved-wedge count W under a ranking, and the
 * per-edge count of single edges straight from Eq. 2 (no ranking at all).
 *
 * Vertex ids: U = [0, nU), V = [nU, nU + nV) ("global id").
 * Readings where the paper is silent (all listed in the design notes):
 *   degree order: key (-deg, global id); approximate degree order: key
 *   (-floor(log2 deg), global id) with degree-0 vertices last; side order:
 *   the side whose vertices as endpoints give fewer wedges comes first
 *   (ties: U), decreasing degree within a side (ties by id); complement
 *   degeneracy orders: peeling rounds, ties within a round by global id.
 *   rank 0 is first.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { ORC_RANK_SIDE = 0, ORC_RANK_DEGREE = 1, ORC_RANK_APPROX_DEGREE = 2, ORC_RANK_CODEGEN = 3,
       ORC_RANK_APPROX_CODEGEN = 4 };
enum { ORC_OK = 0, ORC_ERR_INVALID = 1, ORC_ERR_NOMEM = 2, ORC_ERR_OVERFLOW = 6 };

/* ------------------------------------------------------------------ */
/* Deduplicated bipartite graph, CSR of U -> V with canonical edge ids. */
typedef struct {
  uint32_t nU, nV;
  uint64_t m;          /* distinct edges */
  uint64_t *uoff;      /* nU + 1 */
  uint32_t *uadj;      /* m: V-side id (0-based within V), ascending per list */
  uint64_t *in2e;      /* m_in: canonical edge id of each input edge */
  uint32_t *deg;       /* n: degree by global id */
} bgraph_t;

static void bgraph_free(bgraph_t *g) {
  free(g->uoff); free(g->uadj); free(g->in2e); free(g->deg);
  memset(g, 0, sizeof *g);
}

typedef struct { uint32_t v; uint64_t idx; } vent_t;

static int cmp_vent(const void *a, const void *b) {
  const vent_t *x = (const vent_t *)a, *y = (const vent_t *)b;
  if (x->v != y->v) return x->v < y->v ? -1 : 1;
  return x->idx < y->idx ? -1 : (x->idx > y->idx);
}

/* Remove duplicate (u, v) pairs; canonical edge ids follow (u, v) order. */
static int bgraph_build(uint32_t nU, uint32_t nV, uint64_t m_in, const uint32_t *u,
                        const uint32_t *v, bgraph_t *g) {
  memset(g, 0, sizeof *g);
  g->nU = nU; g->nV = nV;
  for (uint64_t k = 0; k < m_in; k++)
    if (u[k] >= nU || v[k] >= nV) return ORC_ERR_INVALID;
  uint64_t *cnt = (uint64_t *)calloc((size_t)nU + 1, sizeof(uint64_t));
  vent_t *ent = (vent_t *)malloc(sizeof(vent_t) * (m_in ? m_in : 1));
  g->uoff = (uint64_t *)calloc((size_t)nU + 1, sizeof(uint64_t));
  g->in2e = (uint64_t *)malloc(sizeof(uint64_t) * (m_in ? m_in : 1));
  g->deg = (uint32_t *)calloc((size_t)nU + nV + 1, sizeof(uint32_t));
  if (!cnt || !ent || !g->uoff || !g->in2e || !g->deg) {
    free(cnt); free(ent); bgraph_free(g);
    return ORC_ERR_NOMEM;
  }
  for (uint64_t k = 0; k < m_in; k++) cnt[u[k] + 1]++;
  for (uint32_t i = 0; i < nU; i++) cnt[i + 1] += cnt[i];
  uint64_t *cur = (uint64_t *)malloc(sizeof(uint64_t) * ((size_t)nU + 1));
  if (!cur) { free(cnt); free(ent); bgraph_free(g); return ORC_ERR_NOMEM; }
  memcpy(cur, cnt, sizeof(uint64_t) * ((size_t)nU + 1));
  for (uint64_t k = 0; k < m_in; k++) {
    uint64_t at = cur[u[k]]++;
    ent[at].v = v[k];
    ent[at].idx = k;
  }
  free(cur);
  /* sort each U-list by v; keep the first of every run of equal v */
  uint64_t m = 0;
  for (uint32_t i = 0; i < nU; i++) {
    uint64_t s = cnt[i], e = cnt[i + 1];
    qsort(ent + s, e - s, sizeof(vent_t), cmp_vent);
    for (uint64_t a = s; a < e; a++) {
      if (a == s || ent[a].v != ent[a - 1].v) m++;
    }
  }
  g->m = m;
  g->uadj = (uint32_t *)malloc(sizeof(uint32_t) * (m ? m : 1));
  if (!g->uadj) { free(cnt); free(ent); bgraph_free(g); return ORC_ERR_NOMEM; }
  uint64_t e_id = 0;
  for (uint32_t i = 0; i < nU; i++) {
    uint64_t s = cnt[i], e = cnt[i + 1];
    g->uoff[i] = e_id;
    for (uint64_t a = s; a < e; a++) {
      if (a == s || ent[a].v != ent[a - 1].v) {
        g->uadj[e_id] = ent[a].v;
        g->deg[i]++;
        g->deg[nU + ent[a].v]++;
        e_id++;
      }
      g->in2e[ent[a].idx] = e_id - 1;
    }
  }
  g->uoff[nU] = e_id;
  free(cnt); free(ent);
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Rank functions f (Sec. "Ranking"); PREPROCESS sorts by them. */
typedef struct { uint64_t key; uint32_t id; } rkey_t;

static int cmp_rkey(const void *a, const void *b) {
  const rkey_t *x = (const rkey_t *)a, *y = (const rkey_t *)b;
  if (x->key != y->key) return x->key < y->key ? -1 : 1;
  return x->id < y->id ? -1 : (x->id > y->id);
}

static uint32_t floor_log2_u32(uint32_t d) {
  uint32_t r = 0;
  while (d >>= 1) r++;
  return r;
}

/* Complement degeneracy order (Sec. "Ranking"): peeling rounds, each removing
 * every remaining vertex whose current degree (in the subgraph induced by the
 * remaining vertices) is the largest -- or, for the approximate order, whose
 * current floor(log2 degree) is the largest, degree 0 below every class.
 * Vertices removed in the same round are ranked in global-id order. */
static int codegen_rank(const bgraph_t *g, int approx, uint32_t *rank) {
  uint32_t nU = g->nU, nV = g->nV;
  uint64_t n = (uint64_t)nU + nV;
  uint64_t *off = (uint64_t *)calloc(n + 1, sizeof(uint64_t));
  uint32_t *nb = (uint32_t *)malloc(sizeof(uint32_t) * (2 * g->m + 1));
  uint64_t *cur = (uint64_t *)malloc(sizeof(uint64_t) * (n + 1));
  uint32_t *d = (uint32_t *)malloc(sizeof(uint32_t) * (n ? n : 1));
  uint8_t *gone = (uint8_t *)calloc(n ? n : 1, 1);
  uint32_t *front = (uint32_t *)malloc(sizeof(uint32_t) * (n ? n : 1));
  if (!off || !nb || !cur || !d || !gone || !front) {
    free(off); free(nb); free(cur); free(d); free(gone); free(front);
    return ORC_ERR_NOMEM;
  }
  for (uint64_t x = 0; x < n; x++) off[x + 1] = off[x] + g->deg[x];
  memcpy(cur, off, sizeof(uint64_t) * (n + 1));
  for (uint32_t i = 0; i < nU; i++)
    for (uint64_t e = g->uoff[i]; e < g->uoff[i + 1]; e++) {
      uint32_t j = nU + g->uadj[e];
      nb[cur[i]++] = j;
      nb[cur[j]++] = i;
    }
  for (uint64_t x = 0; x < n; x++) d[x] = g->deg[x];
  uint64_t next = 0;
  while (next < n) {
    int64_t best = -2;
    for (uint64_t x = 0; x < n; x++) {
      if (gone[x]) continue;
      int64_t key = approx ? (d[x] ? (int64_t)floor_log2_u32(d[x]) : -1) : (int64_t)d[x];
      if (key > best) best = key;
    }
    uint64_t nf = 0;
    for (uint64_t x = 0; x < n; x++) {
      if (gone[x]) continue;
      int64_t key = approx ? (d[x] ? (int64_t)floor_log2_u32(d[x]) : -1) : (int64_t)d[x];
      if (key == best) front[nf++] = (uint32_t)x;
    }
    for (uint64_t f = 0; f < nf; f++) { rank[front[f]] = (uint32_t)(next + f); gone[front[f]] = 1; }
    next += nf;
    for (uint64_t f = 0; f < nf; f++) {
      uint32_t x = front[f];
      for (uint64_t a = off[x]; a < off[x + 1]; a++)
        if (!gone[nb[a]]) d[nb[a]]--;
    }
  }
  free(off); free(nb); free(cur); free(d); free(gone); free(front);
  return ORC_OK;
}

/* rank[id] for id in [0, n). */
static int make_rank(const bgraph_t *g, int kind, uint32_t *rank) {
  uint32_t nU = g->nU, nV = g->nV;
  uint64_t n = (uint64_t)nU + nV;
  if (kind == ORC_RANK_CODEGEN || kind == ORC_RANK_APPROX_CODEGEN)
    return codegen_rank(g, kind == ORC_RANK_APPROX_CODEGEN, rank);
  if (kind == ORC_RANK_SIDE) {
    /* Wedges retrieved when side X holds the endpoints: every pair of
     * neighbours of a centre on the other side, i.e. sum over centres y not in
     * X of C(deg y, 2). */
    unsigned __int128 wU = 0, wV = 0; /* endpoints in U / endpoints in V */
    for (uint32_t i = 0; i < nU; i++) { uint64_t d = g->deg[i]; if (d) wV += (unsigned __int128)d * (d - 1) / 2; }
    for (uint32_t j = 0; j < nV; j++) { uint64_t d = g->deg[nU + j]; if (d) wU += (unsigned __int128)d * (d - 1) / 2; }
    int u_first = wU <= wV;
    /* Within a side: decreasing degree, ties by id.  The paper fixes only which
     * side comes first; every wedge with endpoints on that side is retrieved
     * once whatever the order inside it, so W and the counts do not depend on
     * this choice. */
    rkey_t *k = (rkey_t *)malloc(sizeof(rkey_t) * (n ? n : 1));
    if (!k) return ORC_ERR_NOMEM;
    for (uint64_t x = 0; x < n; x++) {
      uint64_t second = (x < nU) ? !u_first : u_first; /* 1 for the side placed second */
      k[x].key = (second << 32) | (uint64_t)(0xFFFFFFFFu - g->deg[x]);
      k[x].id = (uint32_t)x;
    }
    qsort(k, n, sizeof(rkey_t), cmp_rkey);
    for (uint64_t r = 0; r < n; r++) rank[k[r].id] = (uint32_t)r;
    free(k);
    return ORC_OK;
  }
  rkey_t *k = (rkey_t *)malloc(sizeof(rkey_t) * (n ? n : 1));
  if (!k) return ORC_ERR_NOMEM;
  for (uint64_t x = 0; x < n; x++) {
    uint32_t d = g->deg[x];
    uint64_t key;
    if (kind == ORC_RANK_DEGREE) key = (uint64_t)(0xFFFFFFFFu - d); /* decreasing degree */
    else key = d == 0 ? 64 : (uint64_t)(31 - floor_log2_u32(d));   /* decreasing log-degree */
    k[x].key = key;
    k[x].id = (uint32_t)x;
  }
  qsort(k, n, sizeof(rkey_t), cmp_rkey);
  for (uint64_t r = 0; r < n; r++) rank[k[r].id] = (uint32_t)r;
  free(k);
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* PREPROCESS output: general graph in rank space, lists by decreasing rank. */
typedef struct {
  uint64_t n;
  uint64_t *off;    /* n + 1 */
  uint32_t *nbr;    /* 2m: neighbour rank */
  uint64_t *eid;    /* 2m: canonical edge id of the entry */
} rgraph_t;

typedef struct { uint32_t y; uint64_t e; } rent_t;

static int cmp_rent_desc(const void *a, const void *b) {
  const rent_t *x = (const rent_t *)a, *y = (const rent_t *)b;
  return x->y > y->y ? -1 : (x->y < y->y);
}

static void rgraph_free(rgraph_t *r) { free(r->off); free(r->nbr); free(r->eid); memset(r, 0, sizeof *r); }

static int preprocess(const bgraph_t *g, const uint32_t *rank, rgraph_t *r) {
  uint64_t n = (uint64_t)g->nU + g->nV, m = g->m;
  r->n = n;
  r->off = (uint64_t *)calloc(n + 1, sizeof(uint64_t));
  rent_t *ent = (rent_t *)malloc(sizeof(rent_t) * (2 * m + 1));
  r->nbr = (uint32_t *)malloc(sizeof(uint32_t) * (2 * m + 1));
  r->eid = (uint64_t *)malloc(sizeof(uint64_t) * (2 * m + 1));
  uint64_t *cur = (uint64_t *)malloc(sizeof(uint64_t) * (n + 1));
  if (!r->off || !ent || !r->nbr || !r->eid || !cur) {
    free(ent); free(cur); rgraph_free(r);
    return ORC_ERR_NOMEM;
  }
  for (uint64_t x = 0; x < n; x++) r->off[rank[x] + 1] = g->deg[x];
  for (uint64_t x = 0; x < n; x++) r->off[x + 1] += r->off[x];
  memcpy(cur, r->off, sizeof(uint64_t) * (n + 1));
  for (uint32_t i = 0; i < g->nU; i++) {
    for (uint64_t e = g->uoff[i]; e < g->uoff[i + 1]; e++) {
      uint32_t ru = rank[i], rv = rank[g->nU + g->uadj[e]];
      uint64_t a = cur[ru]++, b = cur[rv]++;
      ent[a].y = rv; ent[a].e = e;
      ent[b].y = ru; ent[b].e = e;
    }
  }
  free(cur);
  for (uint64_t x = 0; x < n; x++)
    qsort(ent + r->off[x], r->off[x + 1] - r->off[x], sizeof(rent_t), cmp_rent_desc);
  for (uint64_t s = 0; s < 2 * m; s++) { r->nbr[s] = ent[s].y; r->eid[s] = ent[s].e; }
  free(ent);
  return ORC_OK;
}

/* Number of entries of x's list with rank > t (a prefix, lists are descending). */
static inline uint64_t prefix_above(const rgraph_t *r, uint64_t x, uint32_t t) {
  uint64_t s = r->off[x], e = r->off[x + 1], k = s;
  while (k < e && r->nbr[k] > t) k++;
  return k - s;
}

/* ------------------------------------------------------------------ */
/* Counting: every x1 aggregates its wedges in a dense array (simple batching)
 * and adds its butterflies with atomic adds. */
typedef struct {
  const rgraph_t *r;
  uint64_t *next;       /* shared x1 cursor */
  uint64_t hi;          /* first x1 not counted */
  uint64_t *pv;         /* n, rank space, or NULL */
  uint64_t *pe;         /* m, canonical edge ids, or NULL */
  unsigned __int128 global;
  uint64_t wedges;
} cnt_job_t;

#define X1_CHUNK 64

static void *count_worker(void *arg) {
  cnt_job_t *j = (cnt_job_t *)arg;
  const rgraph_t *r = j->r;
  uint64_t n = r->n;
  uint32_t *A = (uint32_t *)calloc(n ? n : 1, sizeof(uint32_t));
  uint32_t *touched = (uint32_t *)malloc(sizeof(uint32_t) * (n ? n : 1));
  if (!A || !touched) { free(A); free(touched); j->wedges = ~0ULL; return NULL; }
  for (;;) {
    uint64_t lo = __atomic_fetch_add(j->next, X1_CHUNK, __ATOMIC_RELAXED);
    if (lo >= j->hi) break;
    uint64_t hi = lo + X1_CHUNK < j->hi ? lo + X1_CHUNK : j->hi;
    for (uint64_t x1 = lo; x1 < hi; x1++) {
      uint64_t nt = 0;
      uint64_t s1 = r->off[x1], k1 = prefix_above(r, x1, (uint32_t)x1);
      /* GET-WEDGES feeding GET-FREQ: d(x1, x2) accumulates in A[x2] */
      for (uint64_t i = 0; i < k1; i++) {
        uint32_t y = r->nbr[s1 + i];
        uint64_t sy = r->off[y], ky = prefix_above(r, y, (uint32_t)x1);
        for (uint64_t t = 0; t < ky; t++) {
          uint32_t x2 = r->nbr[sy + t];
          if (A[x2]++ == 0) touched[nt++] = x2;
        }
        j->wedges += ky;
      }
      /* endpoints: C(d, 2) to the global count, x1 and x2 */
      uint64_t own = 0;
      for (uint64_t t = 0; t < nt; t++) {
        uint64_t d = A[touched[t]];
        uint64_t b = d * (d - 1) / 2;
        j->global += b;
        own += b;
        if (j->pv && b) __atomic_fetch_add(&j->pv[touched[t]], b, __ATOMIC_RELAXED);
      }
      if (j->pv && own) __atomic_fetch_add(&j->pv[x1], own, __ATOMIC_RELAXED);
      /* centres and edges: second pass over the same wedges, d - 1 each */
      if (j->pv || j->pe) {
        for (uint64_t i = 0; i < k1; i++) {
          uint32_t y = r->nbr[s1 + i];
          uint64_t sy = r->off[y], ky = prefix_above(r, y, (uint32_t)x1);
          uint64_t s = 0;
          for (uint64_t t = 0; t < ky; t++) {
            uint64_t c = (uint64_t)A[r->nbr[sy + t]] - 1;
            s += c;
            if (j->pe && c) __atomic_fetch_add(&j->pe[r->eid[sy + t]], c, __ATOMIC_RELAXED);
          }
          if (j->pv && s) __atomic_fetch_add(&j->pv[y], s, __ATOMIC_RELAXED);
          if (j->pe && s) __atomic_fetch_add(&j->pe[r->eid[s1 + i]], s, __ATOMIC_RELAXED);
        }
      }
      for (uint64_t t = 0; t < nt; t++) A[touched[t]] = 0;
    }
  }
  free(A); free(touched);
  return NULL;
}

static int run_count(const rgraph_t *r, int nthreads, uint64_t x_lo, uint64_t x_hi, uint64_t *W,
                     unsigned __int128 *global, uint64_t *pv_rank, uint64_t *pe) {
  if (nthreads < 1) nthreads = 1;
  if (nthreads > 512) nthreads = 512;
  uint64_t next = x_lo;
  cnt_job_t *jobs = (cnt_job_t *)calloc((size_t)nthreads, sizeof(cnt_job_t));
  pthread_t *th = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
  if (!jobs || !th) { free(jobs); free(th); return ORC_ERR_NOMEM; }
  for (int t = 0; t < nthreads; t++) {
    jobs[t].r = r; jobs[t].next = &next; jobs[t].hi = x_hi; jobs[t].pv = pv_rank; jobs[t].pe = pe;
  }
  for (int t = 1; t < nthreads; t++) pthread_create(&th[t], NULL, count_worker, &jobs[t]);
  count_worker(&jobs[0]);
  for (int t = 1; t < nthreads; t++) pthread_join(th[t], NULL);
  uint64_t w = 0;
  unsigned __int128 gsum = 0;
  int bad = 0;
  for (int t = 0; t < nthreads; t++) {
    if (jobs[t].wedges == ~0ULL) bad = 1;
    w += jobs[t].wedges;
    gsum += jobs[t].global;
  }
  free(jobs); free(th);
  if (bad) return ORC_ERR_NOMEM;
  *W = w;
  *global = gsum;
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Public entry points (ctypes). */

int orc_rank(uint32_t nU, uint32_t nV, uint64_t m_in, const uint32_t *u, const uint32_t *v,
             int kind, uint32_t *rank_out) {
  bgraph_t g;
  int rc = bgraph_build(nU, nV, m_in, u, v, &g);
  if (rc) return rc;
  if (kind < 0 || kind > 4) { bgraph_free(&g); return ORC_ERR_INVALID; }
  rc = make_rank(&g, kind, rank_out);
  bgraph_free(&g);
  return rc;
}

/* Counts under ranking `kind`, or under the given rank[] (a permutation of
 * [0, n)) when rank_in is not NULL.  Outputs may be NULL:
 *   pv_out[n]    per-vertex counts by global id (U then V);
 *   pe_out[m_in] per-edge counts in input order (duplicates share their edge's);
 *   m_out        number of distinct edges. */
/* As orc_count, restricted to first endpoints with rank in [x_lo, x_hi): the
 * partial counts of those wedges (Algorithm 2's outer loop is over
 * independent first endpoints, so the parts of a partition add up). */
int orc_count_range(uint32_t nU, uint32_t nV, uint64_t m_in, const uint32_t *u, const uint32_t *v,
                    int kind, const uint32_t *rank_in, int nthreads, uint64_t x_lo, uint64_t x_hi,
                    uint64_t *W_out, uint64_t *global_out, uint64_t *pv_out, uint64_t *pe_out,
                    uint64_t *m_out);

int orc_count(uint32_t nU, uint32_t nV, uint64_t m_in, const uint32_t *u, const uint32_t *v,
              int kind, const uint32_t *rank_in, int nthreads, uint64_t *W_out,
              uint64_t *global_out, uint64_t *pv_out, uint64_t *pe_out, uint64_t *m_out) {
  return orc_count_range(nU, nV, m_in, u, v, kind, rank_in, nthreads, 0, UINT64_MAX, W_out, global_out,
                         pv_out, pe_out, m_out);
}

int orc_count_range(uint32_t nU, uint32_t nV, uint64_t m_in, const uint32_t *u, const uint32_t *v,
                    int kind, const uint32_t *rank_in, int nthreads, uint64_t x_lo, uint64_t x_hi,
                    uint64_t *W_out, uint64_t *global_out, uint64_t *pv_out, uint64_t *pe_out,
                    uint64_t *m_out) {
  bgraph_t g;
  int rc = bgraph_build(nU, nV, m_in, u, v, &g);
  if (rc) return rc;
  uint64_t n = (uint64_t)nU + nV;
  uint32_t *rank = (uint32_t *)malloc(sizeof(uint32_t) * (n ? n : 1));
  if (!rank) { bgraph_free(&g); return ORC_ERR_NOMEM; }
  if (rank_in) {
    uint8_t *seen = (uint8_t *)calloc(n ? n : 1, 1);
    if (!seen) { free(rank); bgraph_free(&g); return ORC_ERR_NOMEM; }
    for (uint64_t x = 0; x < n; x++) {
      if (rank_in[x] >= n || seen[rank_in[x]]) { free(seen); free(rank); bgraph_free(&g); return ORC_ERR_INVALID; }
      seen[rank_in[x]] = 1;
      rank[x] = rank_in[x];
    }
    free(seen);
  } else {
    if (kind < 0 || kind > 4) { free(rank); bgraph_free(&g); return ORC_ERR_INVALID; }
    rc = make_rank(&g, kind, rank);
    if (rc) { free(rank); bgraph_free(&g); return rc; }
  }
  rgraph_t r;
  rc = preprocess(&g, rank, &r);
  if (rc) { free(rank); bgraph_free(&g); return rc; }
  uint64_t *pv_rank = pv_out ? (uint64_t *)calloc(n ? n : 1, sizeof(uint64_t)) : NULL;
  uint64_t *pe = pe_out ? (uint64_t *)calloc(g.m ? g.m : 1, sizeof(uint64_t)) : NULL;
  if ((pv_out && !pv_rank) || (pe_out && !pe)) {
    free(pv_rank); free(pe); rgraph_free(&r); free(rank); bgraph_free(&g);
    return ORC_ERR_NOMEM;
  }
  uint64_t W = 0;
  unsigned __int128 glob = 0;
  if (x_hi > n) x_hi = n;
  if (x_lo > x_hi) x_lo = x_hi;
  rc = run_count(&r, nthreads, x_lo, x_hi, &W, &glob, pv_rank, pe);
  if (rc == ORC_OK) {
    if (glob > (unsigned __int128)UINT64_MAX) rc = ORC_ERR_OVERFLOW;
    if (W_out) *W_out = W;
    if (global_out) *global_out = (uint64_t)glob;
    if (m_out) *m_out = g.m;
    if (pv_out) for (uint64_t x = 0; x < n; x++) pv_out[x] = pv_rank[rank[x]];
    if (pe_out) for (uint64_t k = 0; k < m_in; k++) pe_out[k] = pe[g.in2e[k]];
  }
  free(pv_rank); free(pe); rgraph_free(&r); free(rank); bgraph_free(&g);
  return rc;
}

/* Retrieved-wedge count W under a ranking, without aggregating:
 * sum over x1 and y in N(x1) with rank(y) > rank(x1) of |N_{x1}(y)|. */
int orc_wedges(uint32_t nU, uint32_t nV, uint64_t m_in, const uint32_t *u, const uint32_t *v,
               int kind, const uint32_t *rank_in, uint64_t *W_out) {
  bgraph_t g;
  int rc = bgraph_build(nU, nV, m_in, u, v, &g);
  if (rc) return rc;
  uint64_t n = (uint64_t)nU + nV;
  uint32_t *rank = (uint32_t *)malloc(sizeof(uint32_t) * (n ? n : 1));
  if (!rank) { bgraph_free(&g); return ORC_ERR_NOMEM; }
  if (rank_in) memcpy(rank, rank_in, sizeof(uint32_t) * n);
  else if ((rc = make_rank(&g, kind, rank)) != ORC_OK) { free(rank); bgraph_free(&g); return rc; }
  rgraph_t r;
  rc = preprocess(&g, rank, &r);
  if (rc) { free(rank); bgraph_free(&g); return rc; }
  /* |N_{x1}(y)| is the position of x1 in y's descending list */
  uint64_t W = 0;
  for (uint64_t y = 0; y < n; y++) {
    for (uint64_t s = r.off[y]; s < r.off[y + 1]; s++) {
      if (r.nbr[s] < y) W += s - r.off[y];
    }
  }
  *W_out = W;
  rgraph_free(&r); free(rank); bgraph_free(&g);
  return ORC_OK;
}

/* Wedges of each first endpoint, by rank: wx[r] for r in [0, n). */
int orc_owner_wedges(uint32_t nU, uint32_t nV, uint64_t m_in, const uint32_t *u, const uint32_t *v,
                     int kind, const uint32_t *rank_in, uint64_t *wx) {
  bgraph_t g;
  int rc = bgraph_build(nU, nV, m_in, u, v, &g);
  if (rc) return rc;
  uint64_t n = (uint64_t)nU + nV;
  uint32_t *rank = (uint32_t *)malloc(sizeof(uint32_t) * (n ? n : 1));
  if (!rank) { bgraph_free(&g); return ORC_ERR_NOMEM; }
  if (rank_in) memcpy(rank, rank_in, sizeof(uint32_t) * n);
  else if ((rc = make_rank(&g, kind, rank)) != ORC_OK) { free(rank); bgraph_free(&g); return rc; }
  rgraph_t r;
  rc = preprocess(&g, rank, &r);
  if (rc) { free(rank); bgraph_free(&g); return rc; }
  for (uint64_t x = 0; x < n; x++) {
    uint64_t k1 = prefix_above(&r, x, (uint32_t)x), w = 0;
    for (uint64_t i = 0; i < k1; i++) w += prefix_above(&r, r.nbr[r.off[x] + i], (uint32_t)x);
    wx[x] = w;
  }
  rgraph_free(&r); free(rank); bgraph_free(&g);
  return ORC_OK;
}

/* Eq. 2 evaluated directly for selected input edges, no ranking:
 * count(u, v) = sum over u' in N(v), u' != u, of (|N(u) n N(u')| - 1). */
int orc_edge_eq2(uint32_t nU, uint32_t nV, uint64_t m_in, const uint32_t *u, const uint32_t *v,
                 uint64_t nq, const uint64_t *query, int nthreads, uint64_t *out) {
  (void)nthreads;
  bgraph_t g;
  int rc = bgraph_build(nU, nV, m_in, u, v, &g);
  if (rc) return rc;
  /* V -> U lists, ascending */
  uint64_t *voff = (uint64_t *)calloc((size_t)nV + 1, sizeof(uint64_t));
  uint32_t *vadj = (uint32_t *)malloc(sizeof(uint32_t) * (g.m ? g.m : 1));
  if (!voff || !vadj) { free(voff); free(vadj); bgraph_free(&g); return ORC_ERR_NOMEM; }
  for (uint64_t e = 0; e < g.m; e++) voff[g.uadj[e] + 1]++;
  for (uint32_t j = 0; j < nV; j++) voff[j + 1] += voff[j];
  uint64_t *cur = (uint64_t *)malloc(sizeof(uint64_t) * ((size_t)nV + 1));
  if (!cur) { free(voff); free(vadj); bgraph_free(&g); return ORC_ERR_NOMEM; }
  memcpy(cur, voff, sizeof(uint64_t) * ((size_t)nV + 1));
  for (uint32_t i = 0; i < nU; i++)
    for (uint64_t e = g.uoff[i]; e < g.uoff[i + 1]; e++) vadj[cur[g.uadj[e]]++] = i;
  free(cur);
  for (uint64_t q = 0; q < nq; q++) {
    uint64_t k = query[q];
    if (k >= m_in) { rc = ORC_ERR_INVALID; break; }
    uint32_t a = u[k], b = v[k];
    uint64_t tot = 0;
    for (uint64_t p = voff[b]; p < voff[b + 1]; p++) {
      uint32_t a2 = vadj[p];
      if (a2 == a) continue;
      /* |N(a) n N(a2)| by merging two ascending lists */
      uint64_t x = g.uoff[a], xe = g.uoff[a + 1], y = g.uoff[a2], ye = g.uoff[a2 + 1], c = 0;
      while (x < xe && y < ye) {
        if (g.uadj[x] < g.uadj[y]) x++;
        else if (g.uadj[x] > g.uadj[y]) y++;
        else { c++; x++; y++; }
      }
      tot += c - 1; /* b itself is in both lists, so c >= 1 */
    }
    out[q] = tot;
  }
  free(voff); free(vadj); bgraph_free(&g);
  return rc;
}

/* Eq. 1 evaluated directly for selected vertices (global ids), no ranking:
 * count(x) = sum over x' != x on x's side of C(|N(x) n N(x')|, 2); the
 * intersection sizes come from walking every 2-path x - y - x'. */
int orc_vertex_eq1(uint32_t nU, uint32_t nV, uint64_t m_in, const uint32_t *u, const uint32_t *v,
                   uint64_t nq, const uint64_t *query, uint64_t *out) {
  bgraph_t g;
  int rc = bgraph_build(nU, nV, m_in, u, v, &g);
  if (rc) return rc;
  uint64_t n = (uint64_t)nU + nV;
  /* adjacency of both sides by global id */
  uint64_t *off = (uint64_t *)calloc(n + 1, sizeof(uint64_t));
  uint32_t *nb = (uint32_t *)malloc(sizeof(uint32_t) * (2 * g.m + 1));
  uint64_t *cur = (uint64_t *)malloc(sizeof(uint64_t) * (n + 1));
  uint32_t *cnt = (uint32_t *)calloc(n ? n : 1, sizeof(uint32_t));
  uint32_t *touched = (uint32_t *)malloc(sizeof(uint32_t) * (n ? n : 1));
  if (!off || !nb || !cur || !cnt || !touched) {
    free(off); free(nb); free(cur); free(cnt); free(touched); bgraph_free(&g);
    return ORC_ERR_NOMEM;
  }
  for (uint64_t x = 0; x < n; x++) off[x + 1] = off[x] + g.deg[x];
  memcpy(cur, off, sizeof(uint64_t) * (n + 1));
  for (uint32_t i = 0; i < nU; i++)
    for (uint64_t e = g.uoff[i]; e < g.uoff[i + 1]; e++) {
      uint32_t j = nU + g.uadj[e];
      nb[cur[i]++] = j;
      nb[cur[j]++] = i;
    }
  for (uint64_t q = 0; q < nq && rc == ORC_OK; q++) {
    uint64_t x = query[q];
    if (x >= n) { rc = ORC_ERR_INVALID; break; }
    uint64_t nt = 0, tot = 0;
    for (uint64_t a = off[x]; a < off[x + 1]; a++) {
      uint32_t y = nb[a];
      for (uint64_t b = off[y]; b < off[y + 1]; b++) {
        uint32_t x2 = nb[b];
        if (x2 == x) continue;
        if (cnt[x2]++ == 0) touched[nt++] = x2;
      }
    }
    for (uint64_t t = 0; t < nt; t++) {
      uint64_t c = cnt[touched[t]];
      tot += c * (c - 1) / 2;
      cnt[touched[t]] = 0;
    }
    out[q] = tot;
  }
  free(off); free(nb); free(cur); free(cnt); free(touched); bgraph_free(&g);
  return rc;
}

