// The C ABI (include/pb.h): argument checks, device selection, memory
// helpers, error reporting.  Every entry point returns a status; none aborts.
#include <cstdarg>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "pb_common.cuh"

namespace pb {

static thread_local std::string t_err;
static std::atomic<uint64_t> g_launches{0};

pb_status fail(pb_status s, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  t_err = buf;
  return s;
}

pb_status cuda_fail(cudaError_t e, const char *what, const char *file, int line) {
  cudaGetLastError();  // clear a sticky launch error where possible
  if (e == cudaErrorMemoryAllocation)
    return fail(PB_ERR_NOMEM, "%s: out of device memory (%s:%d)", what, file, line);
  return fail(PB_ERR_CUDA, "%s: %s (%s:%d)", what, cudaGetErrorString(e), file, line);
}

void clear_error() { t_err.clear(); }
void count_launch(uint64_t k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

// ---- phase profiling
static std::atomic<bool> g_prof_on{false};
static std::mutex g_prof_mu;
static pb_profile_t g_prof;
struct PendingPhase {
  int phase;
  cudaEvent_t e0, e1;
  uint64_t launches, wedges;
};
static thread_local std::vector<PendingPhase> t_pending;

bool prof_on() { return g_prof_on.load(std::memory_order_relaxed); }

PhaseScope::PhaseScope(int ph, cudaStream_t s) : phase(ph) {
  if (!prof_on()) return;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  launches0 = g_launches.load(std::memory_order_relaxed);
  cudaEventRecord(e0, s);
  active = true;
}

void PhaseScope::finish(cudaStream_t s, uint64_t wedges_processed) {
  if (!active || done) return;
  cudaEventRecord(e1, s);
  t_pending.push_back({phase, e0, e1, g_launches.load(std::memory_order_relaxed) - launches0, wedges_processed});
  e0 = e1 = nullptr;
  done = true;
}

PhaseScope::~PhaseScope() {
  if (active && !done) {  // abandoned (error path): drop the events
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
  }
}

void prof_flush() {
  if (t_pending.empty()) return;
  std::lock_guard<std::mutex> lk(g_prof_mu);
  for (auto &p : t_pending) {
    float ms = 0.f;
    if (cudaEventSynchronize(p.e1) == cudaSuccess && cudaEventElapsedTime(&ms, p.e0, p.e1) == cudaSuccess) {
      g_prof.ms[p.phase] += ms;
      g_prof.launches[p.phase] += p.launches;
      g_prof.wedges[p.phase] += p.wedges;
      g_prof.records[p.phase] += 1;
    }
    cudaEventDestroy(p.e0);
    cudaEventDestroy(p.e1);
  }
  cudaGetLastError();
  t_pending.clear();
}

// Stream-ordered allocation from the device's default pool.  The pool keeps
// freed memory (release threshold raised once per device) so repeated calls do
// not return memory to the driver between calls.
static std::mutex g_pool_mu;
static bool g_pool_ready[64];

pb_status dalloc(void **p, size_t bytes, cudaStream_t s) {
  *p = nullptr;
  if (bytes == 0) bytes = 16;
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 0 && dev < 64) {
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (!g_pool_ready[dev]) {
      cudaMemPool_t pool;
      if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t thr = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
      }
      cudaGetLastError();
      g_pool_ready[dev] = true;
    }
  }
  cudaError_t e = cudaMallocAsync(p, bytes, s);
  if (e != cudaSuccess) {
    *p = nullptr;
    return cuda_fail(e, "cudaMallocAsync", __FILE__, __LINE__);
  }
  return PB_OK;
}

void dfree(void *p, cudaStream_t s) {
  if (p) cudaFreeAsync(p, s);
}

pb_status ensure_scratch(pb_graph *g, size_t bytes, cudaStream_t s) {
  if (g->scratch_cap >= bytes) return PB_OK;
  dfree(g->scratch, s);
  g->scratch = nullptr;
  g->scratch_cap = 0;
  PB_TRY(dalloc(&g->scratch, bytes, s));
  g->scratch_cap = bytes;
  return PB_OK;
}

pb_status ensure_scratch2(pb_graph *g, size_t bytes, cudaStream_t s) {
  if (g->scratch2_cap >= bytes) return PB_OK;
  dfree(g->scratch2, s);
  g->scratch2 = nullptr;
  g->scratch2_cap = 0;
  PB_TRY(dalloc(&g->scratch2, bytes, s));
  g->scratch2_cap = bytes;
  return PB_OK;
}

int sm_count(int device) {
  static int cached[64] = {0};
  if (device >= 0 && device < 64 && cached[device]) return cached[device];
  int v = 0;
  cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, device);
  if (v <= 0) v = 1;
  if (device >= 0 && device < 64) cached[device] = v;
  return v;
}

static void free_graph(pb_graph *g) {
  if (!g) return;
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(g->device);
  // All work on the graph is complete (every call synchronises its stream);
  // pool frees on the legacy stream make the memory reusable by later calls.
  cudaStream_t s = 0;
  free_ranked(g, s);
  dfree(g->in2c, s); dfree(g->eu, s); dfree(g->ev, s); dfree(g->deg, s);
  dfree(g->scratch, s); dfree(g->scratch2, s); dfree(g->pv, s); dfree(g->es, s); dfree(g->es32, s); dfree(g->acc, s); dfree(g->tstat, s);
  cudaStreamSynchronize(s);
  cudaGetLastError();
  cudaSetDevice(cur);
  delete g;
}

// Makes g's device current for the duration of a call.
struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    cudaGetDevice(&cur);
    if (prev >= 0 && cur != prev) cudaSetDevice(prev);
  }
};

pb_status ensure_ranked(const pb_graph *cg, cudaStream_t s) {
  pb_graph *g = const_cast<pb_graph *>(cg);  // ranking on first use does not change what the graph is
  if (g->rank_kind >= 0) return PB_OK;
  DeviceGuard dg(g->device);
  PhaseScope ph(PB_PHASE_RANK, s);
  PB_TRY(rank_graph(g, PB_RANK_SIDE, nullptr, 0, s));
  ph.finish(s);
  return PB_OK;
}
}  // namespace pb

using namespace pb;

extern "C" {

const char *pb_last_error(void) { return t_err.c_str(); }

const char *pb_status_string(pb_status s) {
  switch (s) {
    case PB_OK: return "PB_OK";
    case PB_ERR_INVALID: return "PB_ERR_INVALID";
    case PB_ERR_NOMEM: return "PB_ERR_NOMEM";
    case PB_ERR_CUDA: return "PB_ERR_CUDA";
    case PB_ERR_SCRATCH: return "PB_ERR_SCRATCH";
    case PB_ERR_TIMEOUT: return "PB_ERR_TIMEOUT";
    case PB_ERR_OVERFLOW: return "PB_ERR_OVERFLOW";
  }
  return "PB_ERR_UNKNOWN";
}

uint64_t pb_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

void pb_profile_enable(int on) { g_prof_on.store(on != 0); }

void pb_profile_reset(void) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  std::memset(&g_prof, 0, sizeof g_prof);
}

pb_status pb_profile_read(pb_profile_t *out) {
  if (!out) return fail(PB_ERR_INVALID, "out is NULL");
  std::lock_guard<std::mutex> lk(g_prof_mu);
  *out = g_prof;
  return PB_OK;
}

pb_status pb_graph_from_edges(uint32_t nU, uint32_t nV, uint64_t m, const uint32_t *u, const uint32_t *v,
                              int on_device, void *stream, pb_graph **out) {
  clear_error();
  if (!out) return fail(PB_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (m > 0 && (!u || !v)) return fail(PB_ERR_INVALID, "u or v is NULL");
  uint64_t n = static_cast<uint64_t>(nU) + nV;
  if (n == 0) return fail(PB_ERR_INVALID, "graph has no vertices");
  if (n >= (uint64_t(1) << 31)) return fail(PB_ERR_INVALID, "nU + nV must be below 2^31");
  if (m >= (uint64_t(1) << 32) - 1) return fail(PB_ERR_INVALID, "too many input edges (m >= 2^32-1)");
  pb_graph *g = new (std::nothrow) pb_graph();
  if (!g) return fail(PB_ERR_NOMEM, "host allocation failed");
  if (cudaGetDevice(&g->device) != cudaSuccess) {
    delete g;
    return fail(PB_ERR_CUDA, "no CUDA device");
  }
  g->nU = nU;
  g->nV = nV;
  g->n = n;
  g->m_in = m;
  g->bitsN = bits_for(n - 1);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  pb_status st;
  {
    PhaseScope ph(PB_PHASE_BUILD, s);
    st = build_graph(g, u, v, on_device, s);
    if (st == PB_OK) ph.finish(s);
  }
  // The side ranking is computed on first use (ensure_ranked), so that a
  // pb_rank right after this call runs PREPROCESS once.
  cudaError_t e = cudaStreamSynchronize(s);
  prof_flush();
  if (st == PB_OK && e != cudaSuccess) st = cuda_fail(e, "graph build", __FILE__, __LINE__);
  if (st != PB_OK) {
    std::string keep = t_err;
    free_graph(g);
    t_err = keep;
    return st;
  }
  *out = g;
  return PB_OK;
}

pb_status pb_rank(pb_graph *g, pb_rank_kind kind, void *stream) {
  clear_error();
  if (!g) return fail(PB_ERR_INVALID, "graph is NULL");
  if (kind < PB_RANK_SIDE || kind > PB_RANK_APPROX_COMPLEMENT_DEGENERACY)
    return fail(PB_ERR_INVALID, "unknown rank kind %d", (int)kind);
  DeviceGuard dg(g->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  {
    PhaseScope ph(PB_PHASE_RANK, s);
    PB_TRY(rank_graph(g, kind, nullptr, 0, s));
    ph.finish(s);
  }
  PB_CUDA(cudaStreamSynchronize(s));
  prof_flush();
  return PB_OK;
}

pb_status pb_rank_custom(pb_graph *g, const uint32_t *rank_of, int on_device, void *stream) {
  clear_error();
  if (!g || !rank_of) return fail(PB_ERR_INVALID, "graph or rank_of is NULL");
  DeviceGuard dg(g->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  {
    PhaseScope ph(PB_PHASE_RANK, s);
    PB_TRY(rank_graph(g, 5, rank_of, on_device, s));
    ph.finish(s);
  }
  PB_CUDA(cudaStreamSynchronize(s));
  prof_flush();
  return PB_OK;
}

pb_status pb_set_retrieval(pb_graph *g, pb_retrieval r) {
  clear_error();
  if (!g) return fail(PB_ERR_INVALID, "graph is NULL");
  if (r < PB_RETRIEVE_LOW || r > PB_RETRIEVE_AUTO) return fail(PB_ERR_INVALID, "unknown retrieval %d", (int)r);
  g->retrieval = r;
  return PB_OK;
}

pb_status pb_set_butterfly_aggregation(pb_graph *g, pb_bfly_agg b) {
  clear_error();
  if (!g) return fail(PB_ERR_INVALID, "graph is NULL");
  if (b != PB_BFLY_ATOMIC && b != PB_BFLY_SORT) return fail(PB_ERR_INVALID, "unknown butterfly aggregation %d", (int)b);
  g->butterfly_agg = b;
  return PB_OK;
}

pb_status pb_graph_ranks(const pb_graph *g, uint32_t *rank_of, int out_on_device, void *stream) {
  clear_error();
  if (!g || !rank_of) return fail(PB_ERR_INVALID, "graph or rank_of is NULL");
  DeviceGuard dg(g->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  PB_TRY(ensure_ranked(g, s));
  PB_CUDA(cudaMemcpyAsync(rank_of, g->rank, g->n * sizeof(uint32_t),
                          out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
  PB_CUDA(cudaStreamSynchronize(s));
  return PB_OK;
}

pb_status pb_count_all(pb_graph *g, pb_agg agg, uint64_t scratch_bytes, uint64_t *out_global, uint64_t *out_U,
                       uint64_t *out_V, uint64_t *out_E, int out_on_device, void *stream) {
  clear_error();
  if (!g) return fail(PB_ERR_INVALID, "graph is NULL");
  DeviceGuard dg(g->device);
  CountOut o;
  o.global = out_global;
  o.U = out_U;
  o.V = out_V;
  o.E = out_E;
  o.on_device = out_on_device;
  pb_status st = count_all(g, static_cast<int>(agg), scratch_bytes, o, static_cast<cudaStream_t>(stream));
  prof_flush();
  return st;
}

pb_status pb_count_owner_range(pb_graph *g, pb_agg agg, uint64_t scratch_bytes, uint32_t owner_lo,
                               uint32_t owner_hi, uint64_t *out_global, uint64_t *out_U, uint64_t *out_V,
                               uint64_t *out_E, int out_on_device, void *stream) {
  clear_error();
  if (!g) return fail(PB_ERR_INVALID, "graph is NULL");
  if (owner_lo > owner_hi || owner_hi > g->n) return fail(PB_ERR_INVALID, "owner range [%u, %u) outside [0, %llu)",
                                                           owner_lo, owner_hi, (unsigned long long)g->n);
  DeviceGuard dg(g->device);
  CountOut o;
  o.global = out_global;
  o.U = out_U;
  o.V = out_V;
  o.E = out_E;
  o.on_device = out_on_device;
  o.owner_lo = owner_lo;
  o.owner_hi = owner_hi;
  pb_status st = count_all(g, static_cast<int>(agg), scratch_bytes, o, static_cast<cudaStream_t>(stream));
  prof_flush();
  return st;
}

pb_status pb_wedge_prefix(const pb_graph *g, uint64_t *out, int out_on_device, void *stream) {
  clear_error();
  if (!g || !out) return fail(PB_ERR_INVALID, "graph or out is NULL");
  DeviceGuard dg(g->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  PB_TRY(ensure_ranked(g, s));
  const uint64_t *src = g->retrieval == PB_RETRIEVE_LOW ? g->wpre : g->wpre_rev;
  PB_CUDA(cudaMemcpyAsync(out, src, (g->n + 1) * sizeof(uint64_t),
                          out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
  PB_CUDA(cudaStreamSynchronize(s));
  return PB_OK;
}

pb_status pb_count_global(pb_graph *g, pb_agg agg, uint64_t scratch_bytes, uint64_t *out, void *stream) {
  if (!out) return fail(PB_ERR_INVALID, "out is NULL");
  return pb_count_all(g, agg, scratch_bytes, out, nullptr, nullptr, nullptr, 0, stream);
}

pb_status pb_count_vertex(pb_graph *g, pb_agg agg, uint64_t scratch_bytes, uint64_t *out_U, uint64_t *out_V,
                          int out_on_device, void *stream) {
  if (!out_U && !out_V) return fail(PB_ERR_INVALID, "both outputs are NULL");
  return pb_count_all(g, agg, scratch_bytes, nullptr, out_U, out_V, nullptr, out_on_device, stream);
}

pb_status pb_count_edge(pb_graph *g, pb_agg agg, uint64_t scratch_bytes, uint64_t *out_E, int out_on_device,
                        void *stream) {
  if (!out_E) return fail(PB_ERR_INVALID, "out_E is NULL");
  return pb_count_all(g, agg, scratch_bytes, nullptr, nullptr, nullptr, out_E, out_on_device, stream);
}

pb_status pb_wedge_count(const pb_graph *g, uint64_t *W) {
  clear_error();
  if (!g || !W) return fail(PB_ERR_INVALID, "graph or W is NULL");
  PB_TRY(ensure_ranked(g, nullptr));
  PB_CUDA(cudaStreamSynchronize(nullptr));
  *W = g->W;
  return PB_OK;
}

pb_status pb_graph_info(const pb_graph *g, pb_graph_info_t *info) {
  clear_error();
  if (!g || !info) return fail(PB_ERR_INVALID, "graph or info is NULL");
  PB_TRY(ensure_ranked(g, nullptr));
  PB_CUDA(cudaStreamSynchronize(nullptr));
  info->nU = g->nU;
  info->nV = g->nV;
  info->m_in = g->m_in;
  info->m = g->m;
  info->max_deg_U = g->maxdegU;
  info->max_deg_V = g->maxdegV;
  info->rank_kind = g->rank_kind;
  info->W = g->W;
  info->max_wedges_x1 = g->maxw;
  uint64_t b = 0;
  b += (g->m_in + 1) * 4 + 2 * (g->m + 1) * 4 + (g->n + 1) * 4;            // input map, edges, degrees
  if (g->rank_kind >= 0) b += 4 * (g->n + 1) * 4 + (g->n + 1) * 8 + 2 * (2 * g->m + 1) * 4 + 2 * (g->m + 1) * 4;
  if (g->pv) b += (g->n + 1) * 8;
  if (g->es) b += (2 * g->m + 1) * 8;
  if (g->es32) b += (2 * g->m + 1) * 4;
  b += g->scratch_cap + g->scratch2_cap;
  info->device_bytes = b;
  return PB_OK;
}

pb_status pb_graph_layout(const pb_graph *g, uint32_t *off, uint32_t *adj, uint32_t *cpos, uint32_t *degp,
                          uint32_t *label_of, int out_on_device, void *stream) {
  clear_error();
  if (!g) return fail(PB_ERR_INVALID, "graph is NULL");
  DeviceGuard dg(g->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  PB_TRY(ensure_ranked(g, s));
  const cudaMemcpyKind k = out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  const size_t na = 2 * g->m;
  if (off) PB_CUDA(cudaMemcpyAsync(off, g->off, (g->n + 1) * sizeof(uint32_t), k, s));
  if (adj && na) PB_CUDA(cudaMemcpyAsync(adj, g->adj, na * sizeof(uint32_t), k, s));
  if (cpos && na) PB_CUDA(cudaMemcpyAsync(cpos, g->cpos, na * sizeof(uint32_t), k, s));
  if (degp) PB_CUDA(cudaMemcpyAsync(degp, g->degp, g->n * sizeof(uint32_t), k, s));
  if (label_of) PB_CUDA(cudaMemcpyAsync(label_of, g->label, g->n * sizeof(uint32_t), k, s));
  PB_CUDA(cudaStreamSynchronize(s));
  return PB_OK;
}

pb_status pb_set_grid_share(pb_graph *g, double share) {
  clear_error();
  if (!g) return fail(PB_ERR_INVALID, "graph is NULL");
  if (!(share > 0.0 && share <= 1.0)) return fail(PB_ERR_INVALID, "share must be in (0, 1]");
  g->grid_share = share;
  return PB_OK;
}

pb_status pb_device_memory(int reset_peak, uint64_t *used, uint64_t *peak) {
  clear_error();
  int dev = 0;
  PB_CUDA(cudaGetDevice(&dev));
  cudaMemPool_t pool;
  PB_CUDA(cudaDeviceGetDefaultMemPool(&pool, dev));
  unsigned long long u = 0, h = 0;  // the pool attributes are 64-bit
  PB_CUDA(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &u));
  if (reset_peak) {
    unsigned long long zero = 0;
    PB_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrUsedMemHigh, &zero));
  }
  PB_CUDA(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemHigh, &h));
  if (used) *used = u;
  if (peak) *peak = h;
  return PB_OK;
}

pb_status pb_graph_free(pb_graph *g) {
  clear_error();
  free_graph(g);
  return PB_OK;
}

}  // extern "C"
