// pb_count_noalloc: butterfly counting that allocates no device memory.
//
// Some callers cannot let a library call cudaMalloc: a host runtime that owns
// every byte of device memory through its own pool and forbids driver
// allocations once it has started, or a latency-critical loop that must not
// risk the implicit device synchronisation cudaMalloc/cudaFree can cause.
// This entry point serves them.  It is a variant of the library's dense
// batching kernel (one block per first endpoint, a dense per-block histogram
// of second endpoints and a list of the entries it touched), but its scratch
// is the file-scope array below instead of memory from cudaMalloc.  Every GPU
// that loads the library holds that array until the process exits.
#include <mutex>

#include "pb_common.cuh"

namespace pb {
namespace {

// Scratch size: 128 MiB.  Each concurrently processed first endpoint needs a
// histogram and a touched list of one side's size (2 x 4 B per vertex of the
// larger side), so sides of up to about 16.7 million vertices fit.
constexpr size_t NA_SCRATCH_BYTES = size_t(128) << 20;
constexpr size_t NA_CTRL_BYTES = 256;  // call counters, before the slots
constexpr int NA_THREADS = 1024;
constexpr int NA_BATCH = 4;

static __device__ __align__(256) uint32_t g_na_scratch[NA_SCRATCH_BYTES / sizeof(uint32_t)];

// Device addresses of g_na_scratch, looked up once per device.
std::mutex g_na_mu;
void *g_na_addr[64];

struct NaCtrl {                 // at the start of the scratch
  unsigned long long queue;     // next first endpoint to take
  unsigned long long overflow;  // a sum wrapped past 2^64
  unsigned long long bad;       // the input layout failed validation
};

// Checks the caller's layout before any of it is used as an index: offsets
// start at 0 and never decrease; every neighbour label is below n and on the
// other side; every deg_x(y) entry is at most y's degree; every deg_x(x) at
// most x's degree.  One warp per label.  On a violation the flag is set and the
// counting kernel does nothing, so a malformed layout yields an error status
// rather than an out-of-range access (off[n] must still be the length of adj
// and cpos, which the library cannot see).
__global__ void k_na_validate(uint64_t n, uint32_t nU, const uint32_t *__restrict__ off,
                              const uint32_t *__restrict__ adj, const uint32_t *__restrict__ cpos,
                              const uint32_t *__restrict__ degp, unsigned long long *bad) {
  const uint64_t warps = (static_cast<uint64_t>(gridDim.x) * blockDim.x) >> 5;
  const uint32_t lane = lane_id();
  for (uint64_t x = (static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; x < n; x += warps) {
    const uint32_t o0 = off[x], o1 = off[x + 1];
    bool ok = o1 >= o0 && (x > 0 || o0 == 0) && degp[x] <= o1 - o0;
    const bool xu = x < nU;
    if (ok) {
      for (uint32_t sl = o0 + lane; sl < o1; sl += 32) {
        const uint32_t y = adj[sl];
        if (y >= n || (y < nU) == xu) { ok = false; break; }
        const uint32_t dy0 = off[y], dy1 = off[y + 1];
        if (dy1 < dy0 || cpos[sl] > dy1 - dy0) { ok = false; break; }
      }
    }
    if (!__all_sync(FULL, ok) && lane == 0) atomicOr(bad, 1ull);
  }
}

// a + b, flagging a wrap past 2^64
__device__ __forceinline__ unsigned long long na_add(unsigned long long a, unsigned long long b, bool &wrap) {
  const unsigned long long r = a + b;
  if (r < a) wrap = true;
  return r;
}

__device__ __forceinline__ uint32_t na_find(const uint32_t *s_incl, uint32_t wi) {
  uint32_t lo = 0, hi = NA_THREADS - 1;  // first index with s_incl > wi
  while (lo < hi) {
    uint32_t mid = (lo + hi) >> 1;
    if (s_incl[mid] > wi) hi = mid;
    else lo = mid + 1;
  }
  return lo;
}

// One block per first endpoint x1 (a work queue over all labels): wedges of
// x1 (Algorithm 2) are counted per second endpoint in the block's dense
// histogram, then C(d, 2) is added to the global count and, with PV, to both
// endpoints, and d - 1 to every centre (Algorithm 3); the touched entries are
// reset to zero before the next x1.  Histogram entries are updated by L2
// atomics and read back through L2 (ld.global.cg).
template <bool PV>
__global__ void __launch_bounds__(NA_THREADS) k_noalloc(uint64_t n, uint32_t nU, const uint32_t *__restrict__ off,
                                                        const uint32_t *__restrict__ adj,
                                                        const uint32_t *__restrict__ cpos,
                                                        const uint32_t *__restrict__ degp, uint32_t *scratch,
                                                        uint64_t side, unsigned long long *out_global,
                                                        unsigned long long *out_pv) {
  NaCtrl *ctrl = reinterpret_cast<NaCtrl *>(scratch);
  uint32_t *A = scratch + NA_CTRL_BYTES / sizeof(uint32_t) + static_cast<size_t>(blockIdx.x) * 2 * side;
  uint32_t *T = A + side;
  __shared__ uint32_t s_incl[NA_THREADS], s_ex[NA_THREADS], s_oy[NA_THREADS];
  __shared__ unsigned long long s_sum[NA_THREADS];
  __shared__ uint32_t s_w[33];
  __shared__ unsigned long long s_own;
  __shared__ uint32_t s_item, s_nt, s_wrap;
  const uint32_t tid = threadIdx.x;
  unsigned long long gacc = 0;
  bool wrap = false;  // this thread saw a sum wrap past 2^64
  if (__ldcg(&ctrl->bad)) return;  // the layout failed validation
  if (PV) s_sum[tid] = 0;
  if (tid == 0) {
    s_nt = 0;
    s_own = 0;
    s_wrap = 0;
  }
  for (;;) {
    if (tid == 0) s_item = static_cast<uint32_t>(atomicAdd(&ctrl->queue, 1ull));
    __syncthreads();
    const uint32_t x1 = s_item;
    if (x1 >= n) break;
    const uint32_t base = x1 < nU ? 0u : nU;
    const uint32_t xbase = off[x1], dp = degp[x1];
    // ---- aggregate
    for (uint32_t k0 = 0; k0 < dp; k0 += NA_THREADS) {
      const uint32_t i = k0 + tid;
      const bool v = i < dp;
      const uint32_t y = v ? adj[xbase + i] : 0, c = v ? cpos[xbase + i] : 0;
      uint32_t tot;
      const uint32_t incl = block_incl_scan(c, s_w, &tot);
      s_incl[tid] = incl;
      s_ex[tid] = incl - c;
      s_oy[tid] = v ? off[y] : 0;
      __syncthreads();
      for (uint32_t wb = 0; wb < tot; wb += NA_BATCH * NA_THREADS) {
        uint32_t x2v[NA_BATCH], old[NA_BATCH];
#pragma unroll
        for (int q = 0; q < NA_BATCH; q++) {
          const uint32_t wi = wb + q * NA_THREADS + tid;
          x2v[q] = 0;
          if (wi < tot) {
            const uint32_t src = na_find(s_incl, wi);
            x2v[q] = adj[s_oy[src] + (wi - s_ex[src])];
          }
        }
#pragma unroll
        for (int q = 0; q < NA_BATCH; q++)
          old[q] = wb + q * NA_THREADS + tid < tot ? atomicAdd(&A[x2v[q] - base], 1u) : 1u;
#pragma unroll
        for (int q = 0; q < NA_BATCH; q++)
          if (old[q] == 0u) T[atomicAdd(&s_nt, 1u)] = x2v[q];
      }
      __syncthreads();
    }
    const uint32_t nt = s_nt;
    // ---- endpoints
    // Every per-vertex count is at most the global count, so checking every
    // partial sum of the global count for a wrap covers the per-vertex sums.
    unsigned long long own = 0;
    for (uint32_t t = tid; t < nt; t += NA_THREADS) {
      const uint32_t x2 = T[t];
      unsigned long long d = __ldcg(&A[x2 - base]), b = d * (d - 1) / 2;
      own = na_add(own, b, wrap);
      if (PV && b) atomicAdd(&out_pv[x2], b);
    }
    if (own) {
      const unsigned long long before = atomicAdd(&s_own, own);
      if (before + own < before) wrap = true;
    }
    __syncthreads();
    if (tid == 0) {
      own = s_own;
      s_own = 0;
      gacc = na_add(gacc, own, wrap);
      if (PV && own) atomicAdd(&out_pv[x1], own);
    }
    // ---- centres: d - 1 per wedge, summed per neighbour
    if (PV) {
      for (uint32_t k0 = 0; k0 < dp; k0 += NA_THREADS) {
        const uint32_t i = k0 + tid;
        const bool v = i < dp;
        const uint32_t y = v ? adj[xbase + i] : 0, c = v ? cpos[xbase + i] : 0;
        uint32_t tot;
        const uint32_t incl = block_incl_scan(c, s_w, &tot);
        s_incl[tid] = incl;
        s_ex[tid] = incl - c;
        s_oy[tid] = v ? off[y] : 0;
        __syncthreads();
        for (uint32_t wi = tid; wi < tot; wi += NA_THREADS) {
          const uint32_t src = na_find(s_incl, wi);
          const uint32_t d = __ldcg(&A[adj[s_oy[src] + (wi - s_ex[src])] - base]);
          if (d > 1) atomicAdd(&s_sum[src], static_cast<unsigned long long>(d - 1));
        }
        __syncthreads();
        if (v && s_sum[tid]) {
          atomicAdd(&out_pv[y], s_sum[tid]);
          s_sum[tid] = 0;
        }
        __syncthreads();
      }
    }
    // ---- reset the touched entries for the next first endpoint
    for (uint32_t t = tid; t < nt; t += NA_THREADS) A[T[t] - base] = 0;
    __syncthreads();
    if (tid == 0) s_nt = 0;
  }
  if (wrap) atomicOr(&s_wrap, 1u);
  __syncthreads();
  if (tid == 0) {
    if (gacc) {
      const unsigned long long old = atomicAdd(out_global, gacc);
      if (old + gacc < old) s_wrap = 1;
    }
    if (s_wrap) atomicAdd(&ctrl->overflow, 1ull);
  }
}

pb_status na_scratch_address(uint32_t **out) {
  int dev = 0;
  PB_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return fail(PB_ERR_INVALID, "device index %d out of range", dev);
  std::lock_guard<std::mutex> lk(g_na_mu);
  if (!g_na_addr[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_na_scratch);
    if (e != cudaSuccess || !p) return cuda_fail(e, "cudaGetSymbolAddress(no-allocation scratch)", __FILE__, __LINE__);
    g_na_addr[dev] = p;
  }
  *out = static_cast<uint32_t *>(g_na_addr[dev]);
  return PB_OK;
}

}  // namespace
}  // namespace pb

using namespace pb;

extern "C" pb_status pb_count_noalloc(uint64_t n, uint32_t nU, const uint32_t *off, const uint32_t *adj,
                                      const uint32_t *cpos, const uint32_t *degp, uint64_t *out_global,
                                      uint64_t *out_pv, void *stream) {
  clear_error();
  if (n == 0 || nU > n) return fail(PB_ERR_INVALID, "need n > 0 and nU <= n");
  if (n >= (uint64_t(1) << 31)) return fail(PB_ERR_INVALID, "n must be below 2^31");
  if (!off || !adj || !cpos || !degp || !out_global) return fail(PB_ERR_INVALID, "NULL input or output");
  const uint64_t side = nU > n - nU ? nU : n - nU;
  const uint64_t slot_bytes = 2 * side * sizeof(uint32_t);
  const uint64_t room = NA_SCRATCH_BYTES - NA_CTRL_BYTES;
  if (slot_bytes > room)
    return fail(PB_ERR_INVALID, "a side of %llu vertices exceeds the no-allocation scratch (%llu MiB: at most %llu "
                "vertices per side)", (unsigned long long)side, (unsigned long long)(NA_SCRATCH_BYTES >> 20),
                (unsigned long long)(room / (2 * sizeof(uint32_t))));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int dev = 0, sdev = 0, per_sm = 0;
  PB_CUDA(cudaGetDevice(&dev));
  PB_CUDA(cudaStreamGetDevice(s, &sdev));
  if (sdev != dev)
    return fail(PB_ERR_INVALID, "the stream belongs to device %d but device %d is current; make the stream's "
                "device current before the call", sdev, dev);
  uint32_t *scratch = nullptr;
  PB_TRY(na_scratch_address(&scratch));
  auto kern = out_pv ? k_noalloc<true> : k_noalloc<false>;
  PB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NA_THREADS, 0));
  uint64_t nslots = static_cast<uint64_t>(sm_count(dev)) * (per_sm > 0 ? per_sm : 1);
  if (nslots > room / slot_bytes) nslots = room / slot_bytes;
  if (nslots > n) nslots = n;
  // Start state: counters and outputs zero, histograms zero (a previous call
  // leaves them zero, but the array is shared and a failed call might not).
  PB_CUDA(cudaMemsetAsync(scratch, 0, NA_CTRL_BYTES + nslots * slot_bytes, s));
  PB_CUDA(cudaMemsetAsync(out_global, 0, sizeof(uint64_t), s));
  if (out_pv) PB_CUDA(cudaMemsetAsync(out_pv, 0, n * sizeof(uint64_t), s));
  NaCtrl *ctrl = reinterpret_cast<NaCtrl *>(scratch);
  k_na_validate<<<grid_for(n * 32, 256, 8192), 256, 0, s>>>(n, nU, off, adj, cpos, degp, &ctrl->bad);
  count_launch();
  kern<<<static_cast<unsigned>(nslots), NA_THREADS, 0, s>>>(n, nU, off, adj, cpos, degp, scratch, side,
                                                            reinterpret_cast<unsigned long long *>(out_global),
                                                            reinterpret_cast<unsigned long long *>(out_pv));
  count_launch();
  PB_CUDA(cudaGetLastError());
  NaCtrl h = {};
  PB_CUDA(cudaMemcpyAsync(&h, ctrl, sizeof(h), cudaMemcpyDeviceToHost, s));
  PB_CUDA(cudaStreamSynchronize(s));
  if (h.bad)
    return fail(PB_ERR_INVALID, "malformed layout: offsets not starting at 0 or decreasing, a neighbour label out of "
                "range or on the same side, or a deg_x(y) / deg_x(x) entry above the degree");
  if (h.overflow) return fail(PB_ERR_OVERFLOW, "global butterfly count exceeds 2^64");
  return PB_OK;
}
