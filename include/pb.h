/*
 * pb.h -- C ABI of the GB300 (sm_103a) exact butterfly-counting library.
 *
 * Implements the counting framework of Shi & Shun, "Parallel Algorithms for
 * Butterfly Computations": rank the vertices (Sec. "Ranking"), retrieve the
 * wedges whose centre and second endpoint rank above the first endpoint
 * (Algorithm 2), aggregate them by endpoint pair (Sec. "Wedge aggregation"),
 * and turn the group sizes d into global, per-vertex (Algorithm 3, Eq. 1) and
 * per-edge (Algorithm 4, Eq. 2) butterfly counts with atomic adds
 * (Sec. "Butterfly aggregation").  All counts are exact uint64.
 *
 * Conventions shared by every entry point:
 *  - Every call returns a pb_status and never aborts the process; on failure
 *    pb_last_error() gives a message (thread-local, valid until the next call
 *    on the same thread).
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Every call enqueues its device work on that stream and returns
 *    after the stream has completed it, so outputs are ready on return.
 *  - Pointers marked "host or device" are device pointers when the matching
 *    on_device / out_on_device flag is non-zero, else host pointers.  Callers
 *    own their inputs and outputs; the library copies inputs and owns the
 *    graph and all scratch memory, which pb_graph_free releases.
 *  - A pb_graph is bound to the device that was current when it was created;
 *    calls on it make that device current.  Calls on one graph must not run
 *    concurrently; distinct graphs may be used from different threads.
 *  - Vertex ids are per side: u in [0, nU), v in [0, nV).  Internally vertex
 *    x has a "global id" (u, or nU + v) and, after ranking, a rank in [0, n).
 *  - Limits: nU + nV < 2^31 and at most 2^31 - 1 distinct edges.
 */
#ifndef PB_H
#define PB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pb_graph pb_graph; /* opaque, library-owned */

/* Ranking functions f of Sec. "Ranking" (PREPROCESS, Algorithm 1 sorts the
 * vertices by f; rank 0 comes first and is the first endpoint x1 of the
 * wedges it retrieves).
 *  SIDE:          every vertex of one side before the other; the side placed
 *                 first is the one whose vertices, as endpoints, give fewer
 *                 wedges (ties: U); within a side decreasing degree, ties by
 *                 id (the order inside a side changes neither W nor counts).
 *  DEGREE:        decreasing degree (Chiba-Nishizeki); ties by global id.
 *  APPROX_DEGREE: decreasing floor(log2 degree); ties keep global-id order;
 *                 degree-0 vertices last.
 *  COMPLEMENT_DEGENERACY: peeling rounds; each round ranks next every
 *                 remaining vertex whose degree in the subgraph induced by
 *                 the remaining vertices is the largest (ties: global id).
 *  APPROX_COMPLEMENT_DEGENERACY: the same with floor(log2 degree) classes
 *                 (at most 33 rounds). */
typedef enum {
  PB_RANK_SIDE = 0,
  PB_RANK_DEGREE = 1,
  PB_RANK_APPROX_DEGREE = 2,
  PB_RANK_COMPLEMENT_DEGENERACY = 3,
  PB_RANK_APPROX_COMPLEMENT_DEGENERACY = 4
} pb_rank_kind;

/* Wedge aggregation methods of Sec. "Wedge aggregation".
 *  SORT:  wedge keys (x1, x2) are materialised chunk by chunk (the paper's
 *         limit on wedges held in memory), radix-sorted on the device and
 *         grouped; group sizes are d(x1, x2).
 *  HASH:  open-addressing hash tables keyed by the second endpoint, one per
 *         first endpoint: in shared memory for first endpoints with few
 *         wedges, in device memory (atomic-add combining) for heavy ones.
 *  HIST:  as HASH for first endpoints with few wedges; heavy ones count
 *         their wedges in a dense histogram over the range of labels their
 *         second endpoints can take, the most frequent part of it in shared
 *         memory; the largest ones share a histogram among a thread-block
 *         cluster.
 *  BATCH: dense arrays over the range of second endpoints, one per
 *         concurrently processed first endpoint, as many as the scratch
 *         budget holds (simple batching), one block each; first endpoints are
 *         taken in decreasing order of wedge count (wedge-aware).  First
 *         endpoints with at most 4096 wedges use shared-memory tables.
 *  AUTO:  chosen per graph from degree and wedge statistics. */
typedef enum {
  PB_AGG_SORT = 0,
  PB_AGG_HASH = 1,
  PB_AGG_HIST = 2,
  PB_AGG_BATCH = 3,
  PB_AGG_AUTO = 4
} pb_agg;

/* Which endpoint of a wedge owns it during aggregation.
 *  LOW:  the lower-ranked endpoint x1 (Algorithm 2): x1 walks its neighbours y
 *        ranked above it and, for each, the entries of y's list ranked above
 *        x1, and groups them by the second endpoint.
 *  HIGH: the higher-ranked endpoint (the cache optimisation of Wang et al.
 *        described in Sec. "Other options"): the same wedges, each grouped at
 *        its higher-ranked endpoint by the lower one.  Owners then have far
 *        fewer wedges each, and the grouping keys concentrate on the few
 *        lowest-ranked (highest-degree) vertices.
 *  AUTO: HIGH unless its largest owner holds more wedges than LOW's.
 *  Counts and the wedge total W are the same either way. */
typedef enum {
  PB_RETRIEVE_LOW = 0,
  PB_RETRIEVE_HIGH = 1,
  PB_RETRIEVE_AUTO = 2
} pb_retrieval;

/* Butterfly aggregation (Sec. "Butterfly aggregation"): how the per-vertex and
 * per-edge contributions found by wedge aggregation reach their counters.
 *  ATOMIC: each contribution is added with an atomic add (the default; the
 *          paper's recommended option).
 *  SORT:   re-aggregation: contributions are written out as (vertex or edge,
 *          value) pairs, radix-sorted by key and summed per key, and every
 *          counter is then written once per chunk of wedges, without atomics.
 *          Needs wedge aggregation PB_AGG_SORT; counts are identical. */
typedef enum {
  PB_BFLY_ATOMIC = 0,
  PB_BFLY_SORT = 1
} pb_bfly_agg;

typedef enum {
  PB_OK = 0,
  PB_ERR_INVALID = 1,  /* bad argument, id out of range, size over a limit */
  PB_ERR_NOMEM = 2,    /* device or host allocation failed */
  PB_ERR_CUDA = 3,     /* a CUDA runtime call failed */
  PB_ERR_SCRATCH = 4,  /* scratch budget too small for one unit of work */
  PB_ERR_TIMEOUT = 5,  /* a bounded device wait ran out */
  PB_ERR_OVERFLOW = 6  /* a count does not fit in uint64 */
} pb_status;

/* Graph statistics (filled by pb_graph_info). */
typedef struct {
  uint32_t nU, nV;
  uint64_t m_in;       /* edges given, duplicates included */
  uint64_t m;          /* distinct edges */
  uint32_t max_deg_U, max_deg_V;
  int32_t rank_kind;   /* pb_rank_kind, 5 = custom ranking, -1 = not ranked */
  uint64_t W;          /* wedges retrieved under the current ranking */
  uint64_t max_wedges_x1; /* largest wedge count of one lower-ranked endpoint */
  uint64_t device_bytes;  /* device memory held by the graph (scratch included) */
} pb_graph_info_t;

/* Builds a graph from m edge pairs (u[k], v[k]) (preliminaries: bipartite CSR;
 * Sec. "Experiments / Environment": duplicate edges removed).  u and v are
 * host or device arrays of m uint32 each (on_device selects).  Duplicated
 * pairs collapse into one edge; per-edge outputs still have one entry per
 * input pair, in input order.  Returns PB_ERR_INVALID if u[k] >= nU or
 * v[k] >= nV for any k, or if nU + nV = 0.  The graph is ranked with PB_RANK_SIDE until pb_rank
 * is called; that ranking is computed on the first call that needs one (a
 * count, pb_wedge_count, pb_graph_info, ...), so pb_rank straight after this
 * call runs PREPROCESS once.  Calls without a stream argument that trigger it
 * use the legacy default stream.  *out receives the handle (NULL on failure). */
pb_status pb_graph_from_edges(uint32_t nU, uint32_t nV, uint64_t m, const uint32_t *u,
                              const uint32_t *v, int on_device, void *stream,
                              pb_graph **out);

/* PREPROCESS (Algorithm 1): ranks the vertices with f = kind, renames them to
 * their ranks, sorts every adjacency list by decreasing rank and stores, for
 * every adjacency entry (x, y), deg_x(y) = |N_x(y)| (the number of y's
 * neighbours ranked above x), plus the wedge count of every first endpoint
 * and their prefix sum (the work split of Algorithm 2). */
pb_status pb_rank(pb_graph *g, pb_rank_kind kind, void *stream);

/* As pb_rank with an explicit ranking: rank_of[x] for global id x (U ids
 * then V ids), a permutation of [0, nU + nV) (host or device, on_device
 * selects).  PB_ERR_INVALID if it is not a permutation.  Counts do not depend
 * on the ranking (Sec. "Preprocessing"); only the retrieved wedges do. */
pb_status pb_rank_custom(pb_graph *g, const uint32_t *rank_of, int on_device, void *stream);

/* Selects the wedge owner used by later counts on g (default AUTO). */
pb_status pb_set_retrieval(pb_graph *g, pb_retrieval r);

/* Selects the butterfly aggregation used by later counts on g (default
 * ATOMIC).  PB_ERR_INVALID for an unknown value; a later count with
 * PB_BFLY_SORT and a wedge aggregation other than PB_AGG_SORT fails with
 * PB_ERR_INVALID. */
pb_status pb_set_butterfly_aggregation(pb_graph *g, pb_bfly_agg b);

/* Writes rank_of[x] for every global id x (host or device). */
pb_status pb_graph_ranks(const pb_graph *g, uint32_t *rank_of, int out_on_device, void *stream);

/* Total butterfly count: sum over endpoint pairs of C(d, 2) (footnote of
 * Sec. "Butterfly aggregation").  *out is a host uint64.
 * scratch_bytes bounds the aggregation scratch (0 = library default, 16 GiB
 * or less); work is chunked to fit, PB_ERR_SCRATCH if one first endpoint
 * cannot fit alone. */
pb_status pb_count_global(pb_graph *g, pb_agg agg, uint64_t scratch_bytes, uint64_t *out,
                          void *stream);

/* Per-vertex counts (Algorithm 3 / Eq. 1): out_U[nU] and out_V[nV], uint64,
 * host or device (out_on_device selects); either may be NULL. */
pb_status pb_count_vertex(pb_graph *g, pb_agg agg, uint64_t scratch_bytes, uint64_t *out_U,
                          uint64_t *out_V, int out_on_device, void *stream);

/* Per-edge counts (Algorithm 4 / Eq. 2): out_E[m_in], uint64, one entry per
 * input pair in input order (duplicates repeat their edge's count). */
pb_status pb_count_edge(pb_graph *g, pb_agg agg, uint64_t scratch_bytes, uint64_t *out_E,
                        int out_on_device, void *stream);

/* All three in one wedge pass: any output may be NULL.  out_global is a host
 * uint64; out_U, out_V, out_E follow out_on_device. */
pb_status pb_count_all(pb_graph *g, pb_agg agg, uint64_t scratch_bytes, uint64_t *out_global,
                       uint64_t *out_U, uint64_t *out_V, uint64_t *out_E, int out_on_device,
                       void *stream);

/* Counts restricted to the wedges owned by labels in [owner_lo, owner_hi)
 * (labels: U vertices [0, nU), V vertices [nU, nU + nV), each side in rank
 * order; the owner is the endpoint pb_set_retrieval selects).  The outer loop
 * of Algorithm 2 is over independent owners, so the outputs of a partition of
 * [0, n) into ranges sum, element by element, to those of pb_count_all: a
 * graph can be split over devices or processes this way and the parts added.
 * Outputs as for pb_count_all (partial counts). */
pb_status pb_count_owner_range(pb_graph *g, pb_agg agg, uint64_t scratch_bytes, uint32_t owner_lo,
                               uint32_t owner_hi, uint64_t *out_global, uint64_t *out_U,
                               uint64_t *out_V, uint64_t *out_E, int out_on_device, void *stream);

/* Exclusive prefix sum over labels of the wedges each owner holds under the
 * current retrieval: out[n + 1] uint64 (host or device).  out[n] = W.  Input
 * for splitting the owners into ranges of equal wedge mass. */
pb_status pb_wedge_prefix(const pb_graph *g, uint64_t *out, int out_on_device, void *stream);

/* Number of wedges Algorithm 2 retrieves under the current ranking. */
pb_status pb_wedge_count(const pb_graph *g, uint64_t *W);

/* Statistics of the graph (host struct). */
pb_status pb_graph_info(const pb_graph *g, pb_graph_info_t *info);

/* Sparsification for approximate total counts (Sec. "Approximate counting").
 *  EDGE:  keep each edge with probability p; the total butterfly count of the
 *         kept graph divided by p^4 is an unbiased estimate of the total.
 *  COLOR: colourful sparsification: each vertex gets one of c = ceil(1/p)
 *         colours, edges whose two endpoints share a colour are kept; a
 *         butterfly survives with probability c^-3 (p^3 when 1/p is an
 *         integer), so the kept count times c^3 is unbiased.
 * Decisions hash the pair (u, v) or the vertex (SplitMix64's output function,
 * seeded), so duplicate pairs share one decision and results are
 * reproducible.  Writes the kept pairs, in input order, to out_u / out_v
 * (m entries of room; host or device as on_device) and their number to
 * *out_m (host).  Build a graph from them with pb_graph_from_edges. */
typedef enum { PB_SPARSIFY_EDGE = 0, PB_SPARSIFY_COLOR = 1 } pb_sparsify_kind;
pb_status pb_sparsify(uint32_t nU, uint32_t nV, uint64_t m, const uint32_t *u, const uint32_t *v,
                      int on_device, pb_sparsify_kind kind, double p, uint64_t seed, uint32_t *out_u,
                      uint32_t *out_v, uint64_t *out_m, void *stream);

/* Approximate total butterfly count (Sec. "Approximate counting"): the m
 * pairs (host or device, on_device selects) are sparsified on the device as
 * pb_sparsify does, the kept graph is built, ranked with `rank` and counted
 * exactly with aggregation `agg` (scratch_bytes as for pb_count_global), and
 * the device scales the exact count: by p^-4 (EDGE) or ceil(1/p)^3 (COLOR).
 * *estimate (host) receives the estimate; *kept_count the exact butterfly
 * count of the kept graph and *kept_edges the number of kept input pairs
 * (either may be NULL).  PB_ERR_INVALID for p outside (0, 1], an unknown kind
 * or out-of-range ids; all intermediate graphs and buffers are released
 * before the call returns. */
pb_status pb_count_approx(uint32_t nU, uint32_t nV, uint64_t m, const uint32_t *u, const uint32_t *v,
                          int on_device, pb_sparsify_kind kind, double p, uint64_t seed, pb_rank_kind rank,
                          pb_agg agg, uint64_t scratch_bytes, double *estimate, uint64_t *kept_count,
                          uint64_t *kept_edges, void *stream);

/* Autotuner: a counting plan from the graph's degree and wedge statistics,
 * for a scratch budget (scratch_bytes as for pb_count_global, 0 = 16 GiB).
 *  rank_kind: f_side = (W_side - W_rank) / W_side, W_side the wedges of side
 *    order (the fewer of sum C(deg v, 2) over V and over U), W_rank those of
 *    the current ranking: the paper's ranking-choice metric (Sec.
 *    "Experiments", Table 3); side order is recommended when f_side < 0.1.
 *  retrieval: the endpoint that gives the smaller largest per-owner wedge
 *    count (load balance; the higher-ranked one almost always).
 *  Work tiers, from the per-owner wedge counts under that retrieval: owners
 *    with at most light_max wedges (<= 768) are counted one warp each in a
 *    shared-memory hash table; those up to med_max (<= 4096) one 512-thread
 *    block each in a shared-memory hash table; those up to large_max
 *    (<= 65535) one 256-thread block each (eight per SM), with 16-bit counts
 *    of the first 8192 labels of a side in shared memory and the rest in a
 *    small hash table in device memory; the rest ("heavy") one 1024-thread
 *    block each with the counts of the first `hot` labels of a side in shared
 *    memory and the rest in device-memory scratch.  hot is the size whose share of
 *    wedge endpoints (hot_hit) pays for its shared memory: 16384 labels, or
 *    49152 when the smaller range catches under 90 % of the endpoints.
 *    The autotuner sets light_max = 768 and large_max = 4096; med_max is
 *    4096 (the hash tier takes the mid-size owners) unless their mean wedges
 *    per neighbour (mid_segment, over the owners of more than light_max and at
 *    most 65535 wedges) is at least 80, when med_max = light_max and the
 *    hot-range tier takes them: a warp then walks whole segments instead of
 *    locating every wedge.
 *  agg (used by PB_AGG_AUTO), from the heavy owners' scratch per slot against
 *    the budget and the device's resident blocks:
 *    BATCH when one dense histogram per resident block fits the budget;
 *    HASH (the dense histogram's cold part replaced by a hash table sized by
 *    the owner's distinct bound) when only those smaller slots fit;
 *    HIST when a single owner holds more than eight times a block's share of
 *    the heavy wedges: owners of at least hub_min wedges then take a
 *    cluster of hub_cluster blocks (hub_min = UINT64_MAX when no owner needs
 *    one).
 *    SORT is never chosen (on the GPU it trails the others several-fold).
 *    With fit_d and fit_h the dense and hashed slots the budget holds and
 *    want = min(resident_blocks, heavy owners): BATCH if fit_d >= want or
 *    fit_d >= fit_h, else HASH.
 *  heavy_slots / slot_bytes: concurrently processed heavy owners and the
 *    device memory each takes under that choice.
 * pb_count_* with PB_AGG_AUTO follow this plan (computed per call unless one
 * is pinned with pb_set_plan); explicit aggregations keep their own heavy
 * path and take light_max, med_max and hot from it. */
typedef struct {
  int32_t rank_kind;    /* recommended pb_rank_kind */
  int32_t retrieval;    /* pb_retrieval (LOW or HIGH) */
  int32_t agg;          /* pb_agg for PB_AGG_AUTO: BATCH, HASH or HIST */
  uint32_t hub_cluster;
  uint64_t hub_min;
  double f_side;
  uint64_t W_side, W_rank;
  uint64_t max_owner_wedges;  /* under the chosen retrieval */
  uint32_t light_max, med_max, large_max, hot, heavy_slots;
  double hot_hit;             /* share of wedges whose second endpoint is hot */
  uint64_t owners[4];         /* light, medium, large, heavy owners */
  uint64_t wedges[4];         /* their wedges */
  uint64_t slot_bytes;        /* device memory per heavy slot under agg */
  uint64_t slot_bytes_dense;  /* ... with a dense histogram (BATCH, HIST) */
  uint64_t slot_bytes_hash;   /* ... with a hashed cold part (HASH) */
  uint32_t resident_blocks;   /* resident blocks of the heavy kernel */
  double mid_segment;         /* wedges per neighbour of the owners above light_max, up to 65535 wedges */
  uint64_t scratch_bytes;     /* the budget the plan was made for */
} pb_plan_t;
pb_status pb_autotune(const pb_graph *g, uint64_t scratch_bytes, pb_plan_t *plan);

/* Pins a plan for later PB_AGG_AUTO counts on g (NULL returns to planning
 * per call).  light_max is clamped to [1, 768], med_max to [light_max, 4096],
 * large_max to [med_max, 65535],
 * hot to [0, 49152]; PB_ERR_INVALID for an agg other than BATCH, HASH or
 * HIST, a retrieval other than LOW or HIGH, or hub_cluster outside [1, 16].
 * Counts are exact under every plan. */
pb_status pb_set_plan(pb_graph *g, const pb_plan_t *plan);

/* Batched counting: many ranked graphs counted by one persistent kernel per
 * work tier over all their owners, the launches captured once in a CUDA
 * graph and replayed by every pb_batch_run (global and, with want_vertex,
 * per-vertex counts).  Each graph's owner direction follows pb_autotune.
 * The graphs must stay alive and unchanged while the batch exists.
 * scratch_bytes bounds the shared dense-histogram slots (0 = 16 GiB). */
typedef struct pb_batch pb_batch;
pb_status pb_batch_create(pb_graph *const *graphs, uint32_t ng, int want_vertex, uint64_t scratch_bytes,
                          void *stream, pb_batch **out);
pb_status pb_batch_run(pb_batch *b, void *stream);
/* out[ng] host: global count of each graph after the last run. */
pb_status pb_batch_globals(const pb_batch *b, uint64_t *out, void *stream);
/* Per-vertex counts of graph i after the last run (as pb_count_vertex). */
pb_status pb_batch_vertex(const pb_batch *b, uint32_t i, uint64_t *out_U, uint64_t *out_V, int out_on_device,
                          void *stream);
/* Total wedges of all graphs in the batch (under their chosen owners). */
pb_status pb_batch_wedges(const pb_batch *b, uint64_t *W);
pb_status pb_batch_free(pb_batch *b);

/* Copies the graph's PREPROCESS output (Algorithm 1) -- the layout that
 * pb_count_noalloc takes -- into caller-owned buffers (host or device, as
 * out_on_device selects; any may be NULL): off[n + 1] CSR offsets by label,
 * adj[2m] neighbour labels in decreasing rank order, cpos[2m] (deg_x(y) for
 * the entry holding y in x's list), degp[n] (deg_x(x)), and label_of[n], the
 * label of every global id.  Ranks the graph by side order first if it has
 * no ranking. */
pb_status pb_graph_layout(const pb_graph *g, uint32_t *off, uint32_t *adj, uint32_t *cpos, uint32_t *degp,
                          uint32_t *label_of, int out_on_device, void *stream);

/* Upper bound on the device memory a count on g with these arguments will
 * allocate (outputs, tier lists, heavy-tier scratch, download staging), for
 * admission control: the library's stream-ordered pool rounds each allocation
 * up, which the bound includes.  Runs the planner's statistics pass on the
 * legacy default stream, into memory of its own; like pb_autotune it only
 * reads a ranked graph, so it may run while that graph is counted. */
pb_status pb_count_bytes(pb_graph *g, pb_agg agg, uint64_t scratch_bytes, int want_vertex, int want_edge,
                         int out_on_device, uint64_t *bytes);

/* The persistent tier kernels of later counts on g take this share, in
 * (0, 1], of the device's resident blocks (default 1).  Counts running at the
 * same time on other streams then share the SMs instead of waiting for a
 * kernel that holds all of them.  Results do not depend on it. */
pb_status pb_set_grid_share(pb_graph *g, double share);

/* Memory of the current device's default stream-ordered pool, which every
 * library allocation comes from: bytes in use now and the high-water mark
 * since the last reset (reset_peak != 0 resets it to the current use first).
 * Measurement support for checking pb_count_bytes. */
pb_status pb_device_memory(int reset_peak, uint64_t *used, uint64_t *peak);

/* Releases the graph and every device buffer it holds.  NULL is accepted. */
pb_status pb_graph_free(pb_graph *g);

/* Counting without any device allocation.  The paper has no counterpart:
 * this entry point exists for callers that cannot let a library allocate
 * device memory -- a host runtime that owns all device memory through its own
 * pool and forbids driver allocations after start-up, or a latency-critical
 * loop that must not risk the implicit synchronisation of cudaMalloc/cudaFree.
 * It calls no cudaMalloc, cudaFree or allocating library routine.
 *
 * Input: an already preprocessed graph in device memory, caller-owned, in the
 * layout PREPROCESS produces: n vertices labelled so that U is [0, nU) and V
 * is [nU, n), each side in increasing rank order; off[n + 1] (uint32) CSR
 * offsets by label; adj[off[n]] neighbour labels, each list in decreasing
 * rank order; cpos[off[n]], for the entry holding y in x's list, the position
 * of x in y's list (the number of y's neighbours ranked above x); degp[n], the
 * number of x's neighbours ranked above x.
 * Output (device, caller-owned): *out_global, and out_pv[n] per label when
 * out_pv is not NULL (butterflies per vertex).  Both are cleared by the call.
 *
 * Scratch: a file-scope device array of 128 MiB in the library, held by every
 * GPU that loads the library until the process exits.  A side (nU or n - nU)
 * of more than 16,777,184 vertices does not fit and is rejected with
 * PB_ERR_INVALID.  The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress) with that device current; make that first
 * call before any stream capture.  `stream` must belong to the current device
 * (PB_ERR_INVALID otherwise).  Every call shares the array and leaves its
 * contents behind; the call clears what must start at zero.  Calls whose
 * device work overlaps (other streams, other threads) race on the array and
 * must be serialised by the caller.
 *
 * The layout is checked on the device before it is used (offsets start at 0
 * and never decrease, neighbour labels lie below n on the other side, no
 * deg_x(y) or deg_x(x) entry exceeds the degree): a violation returns
 * PB_ERR_INVALID and writes nothing but the cleared outputs.  off[n] must be
 * the length of adj and cpos.  PB_ERR_OVERFLOW if the global count, or any
 * partial sum of it, exceeds 2^64 - 1; no per-vertex count can exceed the
 * global count, so this also covers out_pv.  Like every entry point, the call
 * returns after its stream has completed the work. */
pb_status pb_count_noalloc(uint64_t n, uint32_t nU, const uint32_t *off, const uint32_t *adj,
                           const uint32_t *cpos, const uint32_t *degp, uint64_t *out_global,
                           uint64_t *out_pv, void *stream);

/* Measurement support, not part of the counting path: the current device's
 * throughput of 64-bit atomic adds whose result is unused (performed in L2),
 * in operations per second, over a 64 MiB array of counters.  scattered = 0:
 * the 32 lanes of a warp add to 32 consecutive counters (the per-edge counter
 * pattern); scattered != 0: every lane adds to a hashed counter (the
 * per-vertex pattern).  Allocates and frees 64 MiB; takes a few ms. */
pb_status pb_calibrate_atomics(int scattered, double *ops_per_s, void *stream);

/* Number of device kernels the library has launched in this process (all
 * graphs, all devices); used to report launch counts. */
uint64_t pb_kernel_launches(void);

/* Phase profiling (process-wide).  While enabled, every call records CUDA
 * events on its stream around each phase below and accumulates the elapsed
 * device time, the kernel launches and the wedges the phase processed.
 * Recording adds two events per phase and nothing else; results are exact
 * either way. */
enum {
  PB_PHASE_BUILD = 0,    /* pb_graph_from_edges: upload, validation, dedupe */
  PB_PHASE_RANK = 1,     /* PREPROCESS: rank, relabel, adjacency, work split */
  PB_PHASE_CLASSIFY = 2, /* binning first endpoints by wedge count */
  PB_PHASE_LIGHT = 3,    /* warp-per-endpoint shared-memory hash kernel */
  PB_PHASE_MEDIUM = 4,   /* block-per-endpoint shared-memory hash kernel */
  PB_PHASE_HEAVY = 5,    /* block-per-endpoint hot-range kernel, 1024 threads (or clusters) */
  PB_PHASE_SORT = 6,     /* sort aggregation (all its kernels) */
  PB_PHASE_OUTPUT = 7,   /* rank space -> id space / input order, downloads */
  PB_PHASE_LARGE = 8,    /* block-per-endpoint hot-range kernel, 256 threads */
  PB_NPHASE = 9
};
typedef struct {
  double ms[PB_NPHASE];         /* accumulated device time */
  uint64_t launches[PB_NPHASE]; /* kernels launched */
  uint64_t wedges[PB_NPHASE];   /* wedges aggregated (counting phases) */
  uint64_t records[PB_NPHASE];  /* phase executions */
} pb_profile_t;

void pb_profile_enable(int on);
void pb_profile_reset(void);
pb_status pb_profile_read(pb_profile_t *out);

const char *pb_last_error(void);
const char *pb_status_string(pb_status s);

#ifdef __cplusplus
}
#endif

#endif /* PB_H */
