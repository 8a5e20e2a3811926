// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <cstdio>
#include <string>

#include "pb.h"

// The opaque graph handle of the C ABI.
struct pb_graph {
  int device = 0;
  uint32_t nU = 0, nV = 0;
  uint64_t n = 0;
  uint64_t m_in = 0;  // input pairs
  uint64_t m = 0;     // distinct edges
  int bitsN = 1;      // bits to hold a vertex index in [0, n)
  uint32_t maxdegU = 0, maxdegV = 0;

  // Bipartite graph after deduplication (device).
  uint32_t *in2c = nullptr;  // [m_in] canonical edge of each input pair
  uint32_t *eu = nullptr;    // [m] U id of canonical edge (sorted by (u, v))
  uint32_t *ev = nullptr;    // [m] V id (0-based within V)
  uint32_t *deg = nullptr;   // [n] degree by global id

  // PREPROCESS output (device).  Vertices are renamed to "labels": U
  // vertices get [0, nU) and V vertices [nU, n), each side in increasing rank
  // order.  Wedge endpoints always share a side, so aggregation over second
  // endpoints touches one side's contiguous label range; comparisons between
  // vertices are by rank and are all folded into cpos / degp below.
  // Slot s of vertex x is off[x] + i.
  int rank_kind = -1;
  uint32_t *rank = nullptr;   // [n] rank of global id
  uint32_t *order = nullptr;  // [n] global id at rank
  uint32_t *label = nullptr;  // [n] label of global id
  uint32_t *off = nullptr;    // [n + 1] by label
  uint32_t *adj = nullptr;    // [2m] neighbour labels, decreasing rank within a list
  uint32_t *cpos = nullptr;   // [2m] for slot (x, y): position of x in y's list = deg_x(y)
  uint32_t *degp = nullptr;   // [n] deg_x(x): neighbours ranked above x
  uint64_t *wpre = nullptr;   // [n + 1] exclusive prefix of wedges per lower-ranked endpoint
  uint64_t *wpre_rev = nullptr;  // [n + 1] the same per higher-ranked endpoint
  uint32_t *slotA = nullptr;  // [m] slot of canonical edge e in its U endpoint's list
  uint32_t *slotB = nullptr;  // [m] slot of e in its V endpoint's list
  uint64_t W = 0;
  uint64_t maxw = 0;          // max wedges of one lower-ranked endpoint
  uint64_t maxw_rev = 0;      // max wedges of one higher-ranked endpoint
  int retrieval = PB_RETRIEVE_AUTO;
  int butterfly_agg = PB_BFLY_ATOMIC;
  uint64_t w_side_U = 0, w_side_V = 0;  // wedges with endpoints in U / in V (side order)

  // Aggregation scratch, grown on demand and kept until pb_graph_free.
  void *scratch = nullptr;
  size_t scratch_cap = 0;
  void *scratch2 = nullptr;  // the medium tier's slots
  size_t scratch2_cap = 0;
  // Count outputs in rank space (kept to avoid reallocating per call).
  uint64_t *pv = nullptr;     // [n]
  uint64_t *es = nullptr;     // [2m] per-slot edge partial counts
  uint32_t *es32 = nullptr;   // [2m] per-slot 32-bit partials (carries go to es)
  unsigned long long *acc = nullptr;  // [8] global sum, overflow word, work queues
  unsigned long long *tstat = nullptr;  // autotuner statistics of the owners
  // A plan pinned by pb_set_plan (used by PB_AGG_AUTO counts instead of one
  // computed per call).
  bool has_plan = false;
  pb_plan_t plan = {};
  double grid_share = 1.0;  // share of resident blocks the tier kernels take (pb_set_grid_share)
};

namespace pb {

constexpr uint32_t FULL = 0xffffffffu;
constexpr uint32_t EMPTY = 0xffffffffu;

// ---- errors ---------------------------------------------------------------
pb_status fail(pb_status s, const char *fmt, ...);
pb_status cuda_fail(cudaError_t e, const char *what, const char *file, int line);
void clear_error();
void count_launch(uint64_t k = 1);

#define PB_CUDA(call)                                                     \
  do {                                                                    \
    cudaError_t e_ = (call);                                              \
    if (e_ != cudaSuccess) return ::pb::cuda_fail(e_, #call, __FILE__, __LINE__); \
  } while (0)

#define PB_TRY(call)                 \
  do {                               \
    pb_status s_ = (call);           \
    if (s_ != PB_OK) return s_;      \
  } while (0)

// Kernel launch with accounting and an immediate launch-error check.
#define PB_LAUNCH(kernel, grid, block, smem, stream, ...)               \
  do {                                                                  \
    kernel<<<(grid), (block), (smem), (stream)>>>(__VA_ARGS__);         \
    ::pb::count_launch();                                               \
    PB_CUDA(cudaGetLastError());                                        \
  } while (0)

// ---- phase profiling (pb_api.cu) ------------------------------------------
// PhaseScope records a start event on construction and an end event on
// finish(); elapsed times are folded in by prof_flush() after a stream sync.
bool prof_on();
struct PhaseScope {
  int phase;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  uint64_t launches0 = 0, wedges = 0;
  bool active = false, done = false;
  PhaseScope(int ph, cudaStream_t s);
  void finish(cudaStream_t s, uint64_t wedges_processed = 0);
  ~PhaseScope();
};
void prof_flush();  // call after the stream has been synchronised

// ---- device memory --------------------------------------------------------
pb_status dalloc(void **p, size_t bytes, cudaStream_t s);  // stream-ordered
void dfree(void *p, cudaStream_t s);
template <class T>
inline pb_status dalloc_t(T **p, size_t count, cudaStream_t s) {
  return dalloc(reinterpret_cast<void **>(p), count * sizeof(T), s);
}
pb_status ensure_scratch(pb_graph *g, size_t bytes, cudaStream_t s);
pb_status ensure_scratch2(pb_graph *g, size_t bytes, cudaStream_t s);
int sm_count(int device);

// ---- primitives (pb_prim.cu) ---------------------------------------------
// out[i] = sum_{j<i} in[j] for i in [0, n]; out has n + 1 entries.
pb_status scan_u32(const uint32_t *in, uint32_t *out, size_t n, cudaStream_t s);
pb_status scan_u64(const uint64_t *in, uint64_t *out, size_t n, cudaStream_t s);
pb_status scan_u32_to_u64(const uint32_t *in, uint64_t *out, size_t n, cudaStream_t s);
// Stable LSD radix sort of keys (bits [0, bits)) with optional payload; the
// result is left in keys/vals.
pb_status radix_sort(uint64_t *keys, uint32_t *vals, size_t n, int bits, cudaStream_t s);
// Exact uint64 sum of an array into *out (device).
pb_status sum_u64(const uint64_t *in, size_t n, unsigned long long *out, cudaStream_t s);

inline int bits_for(uint64_t maxval) {  // bits to represent [0, maxval]
  int b = 1;
  while (b < 64 && (maxval >> b) != 0) b++;
  return b;
}

inline unsigned grid_for(size_t n, unsigned block, unsigned cap = 1u << 20) {
  size_t g = (n + block - 1) / block;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return static_cast<unsigned>(g);
}

// ---- stages (pb_graph.cu / pb_count.cu) -------------------------------------
pb_status build_graph(pb_graph *g, const uint32_t *u, const uint32_t *v, int on_device,
                      cudaStream_t s);
pb_status rank_graph(pb_graph *g, int kind, const uint32_t *rank_of, int on_device,
                     cudaStream_t s);
void free_ranked(pb_graph *g, cudaStream_t s);
// Ranks g by side order if it has no ranking yet (pb_api.cu); asynchronous on s.
pb_status ensure_ranked(const pb_graph *g, cudaStream_t s);
struct CountOut {
  uint64_t *global = nullptr;  // host
  uint64_t *U = nullptr, *V = nullptr, *E = nullptr;
  int on_device = 0;
  uint64_t owner_lo = 0, owner_hi = UINT64_MAX;  // owners (labels) whose wedges are counted
};
pb_status count_all(pb_graph *g, int agg, uint64_t scratch_bytes, const CountOut &o,
                    cudaStream_t s);
void make_plan_basic(const pb_graph *g, pb_plan_t *plan);
pb_status make_plan(pb_graph *g, uint64_t budget, cudaStream_t s, pb_plan_t *plan);

// head[i] = 1 where keys[i] starts a run of equal keys (pb_graph.cu).
__global__ void k_heads(const uint64_t *__restrict__ keys, size_t m, uint32_t *__restrict__ head);

// ---- device helpers ---------------------------------------------------------
__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31u; }
__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm volatile("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

template <class T>
__device__ __forceinline__ T warp_incl_scan(T x) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T y = __shfl_up_sync(FULL, x, o);
    if (static_cast<int>(lane_id()) >= o) x += y;
  }
  return x;
}

template <class T>
__device__ __forceinline__ T warp_sum(T x) {
#pragma unroll
  for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(FULL, x, o);
  return x;
}

// Inclusive scan of one value per thread across the block; s_warp holds 33
// entries (one per warp, plus the block total).  Returns the inclusive prefix; *total gets the block sum.
template <class T>
__device__ __forceinline__ T block_incl_scan(T x, T *s_warp, T *total) {
  const uint32_t lane = lane_id(), wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  T inc = warp_incl_scan(x);
  if (lane == 31) s_warp[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    T t = lane < nw ? s_warp[lane] : T(0);
    T ti = warp_incl_scan(t);
    if (lane < nw) s_warp[lane] = ti - t;  // exclusive warp offsets
    if (lane == nw - 1) s_warp[32] = ti;
  }
  __syncthreads();
  T res = inc + s_warp[wid];
  *total = s_warp[32];
  __syncthreads();
  return res;
}

template <class T>
__device__ __forceinline__ T block_sum(T x, T *s_warp) {
  T tot;
  block_incl_scan(x, s_warp, &tot);
  return tot;
}

}  // namespace pb
