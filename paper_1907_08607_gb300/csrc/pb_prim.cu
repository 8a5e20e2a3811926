// Device primitives: exclusive scans, a stable LSD radix sort, a uint64 sum.
// These are the prefix-sum and integer-sort building blocks of the paper's
// preliminaries ("Parallel primitives"), written for the GPU.
#include "pb_common.cuh"

namespace pb {

// ---------------------------------------------------------------------------
// Exclusive scan, three phases: per-tile sums, a recursive scan of the tile
// sums, and a per-tile scan with the tile offset added.
constexpr int SC_THREADS = 512;
constexpr int SC_IPT = 8;
constexpr int SC_TILE = SC_THREADS * SC_IPT;

template <class Tin, class Tout>
__global__ void __launch_bounds__(SC_THREADS) k_scan_tilesum(const Tin *__restrict__ in, size_t n,
                                                           Tout *__restrict__ tsum) {
  __shared__ Tout s_w[33];
  size_t base = static_cast<size_t>(blockIdx.x) * SC_TILE;
  Tout acc = 0;
#pragma unroll
  for (int k = 0; k < SC_IPT; k++) {
    size_t i = base + static_cast<size_t>(k) * SC_THREADS + threadIdx.x;
    if (i < n) acc += static_cast<Tout>(in[i]);
  }
  Tout tot = block_sum(acc, s_w);
  if (threadIdx.x == 0) tsum[blockIdx.x] = tot;
}

template <class Tin, class Tout>
__global__ void __launch_bounds__(SC_THREADS) k_scan_tile(const Tin *__restrict__ in, size_t n,
                                                        Tout *__restrict__ out,
                                                        const Tout *__restrict__ toff) {
  __shared__ Tout s_v[SC_TILE];
  __shared__ Tout s_w[33];
  size_t base = static_cast<size_t>(blockIdx.x) * SC_TILE;
  // coalesced load into shared memory, then each thread scans a contiguous run
#pragma unroll
  for (int k = 0; k < SC_IPT; k++) {
    size_t i = base + static_cast<size_t>(k) * SC_THREADS + threadIdx.x;
    s_v[k * SC_THREADS + threadIdx.x] = i < n ? static_cast<Tout>(in[i]) : Tout(0);
  }
  __syncthreads();
  Tout run[SC_IPT];
  Tout acc = 0;
#pragma unroll
  for (int k = 0; k < SC_IPT; k++) {
    run[k] = acc;
    acc += s_v[threadIdx.x * SC_IPT + k];
  }
  Tout tot;
  Tout incl = block_incl_scan(acc, s_w, &tot);
  Tout off = incl - acc + (toff ? toff[blockIdx.x] : Tout(0));
#pragma unroll
  for (int k = 0; k < SC_IPT; k++) s_v[threadIdx.x * SC_IPT + k] = run[k] + off;
  __syncthreads();
#pragma unroll
  for (int k = 0; k < SC_IPT; k++) {
    size_t i = base + static_cast<size_t>(k) * SC_THREADS + threadIdx.x;
    if (i < n) out[i] = s_v[k * SC_THREADS + threadIdx.x];
  }
  // out[n] = grand total, written by the tile holding the last element
  if (threadIdx.x == SC_THREADS - 1 && base + SC_TILE >= n) out[n] = off + acc;
}

template <class Tin, class Tout>
static pb_status scan_impl(const Tin *in, Tout *out, size_t n, cudaStream_t s) {
  if (n == 0) {
    PB_CUDA(cudaMemsetAsync(out, 0, sizeof(Tout), s));
    return PB_OK;
  }
  size_t tiles = (n + SC_TILE - 1) / SC_TILE;
  if (tiles == 1) {
    PB_LAUNCH((k_scan_tile<Tin, Tout>), 1, SC_THREADS, 0, s, in, n, out, (const Tout *)nullptr);
    return PB_OK;
  }
  Tout *tsum = nullptr, *toff = nullptr;
  PB_TRY(dalloc_t(&tsum, tiles, s));
  PB_TRY(dalloc_t(&toff, tiles + 1, s));
  pb_status st = PB_OK;
  do {
    k_scan_tilesum<Tin, Tout><<<(unsigned)tiles, SC_THREADS, 0, s>>>(in, n, tsum);
    count_launch();
    if (cudaGetLastError() != cudaSuccess) { st = fail(PB_ERR_CUDA, "scan tile sums launch failed"); break; }
    st = scan_impl<Tout, Tout>(tsum, toff, tiles, s);
    if (st != PB_OK) break;
    k_scan_tile<Tin, Tout><<<(unsigned)tiles, SC_THREADS, 0, s>>>(in, n, out, toff);
    count_launch();
    if (cudaGetLastError() != cudaSuccess) { st = fail(PB_ERR_CUDA, "scan tile launch failed"); break; }
  } while (0);
  dfree(tsum, s);
  dfree(toff, s);
  return st;
}

pb_status scan_u32(const uint32_t *in, uint32_t *out, size_t n, cudaStream_t s) {
  return scan_impl<uint32_t, uint32_t>(in, out, n, s);
}
pb_status scan_u64(const uint64_t *in, uint64_t *out, size_t n, cudaStream_t s) {
  return scan_impl<uint64_t, uint64_t>(in, out, n, s);
}
pb_status scan_u32_to_u64(const uint32_t *in, uint64_t *out, size_t n, cudaStream_t s) {
  return scan_impl<uint32_t, uint64_t>(in, out, n, s);
}

// ---------------------------------------------------------------------------
// Stable LSD radix sort, 8-bit digits.  Per pass: per-tile digit histograms
// (digit-major so that one exclusive scan gives every tile's output offset),
// then a scatter in which each warp ranks its keys with match_any so that the
// order of equal digits is the input order.
constexpr int RS_THREADS = 256;
constexpr int RS_WARPS = RS_THREADS / 32;
// Keys per thread: eight, so that five blocks share an SM (the scatter is
// latency-bound; 20M x 60M build + PREPROCESS 150.3 ms with sixteen keys and
// three blocks per SM, 147.0 with twelve and four, 142.8 with eight and five).
constexpr int RS_IPT = 8;
constexpr int RS_TILE = RS_THREADS * RS_IPT;
constexpr int RS_BINS = 256;
static_assert(RS_THREADS == RS_BINS, "one thread per digit in the scatter prefix");
constexpr int RS_SMEM_KEYS = RS_TILE * 8;
constexpr int RS_SMEM_VALS = RS_TILE * 12;

__global__ void __launch_bounds__(RS_THREADS) k_rs_hist(const uint64_t *__restrict__ keys, size_t n,
                                                      int shift, uint32_t *__restrict__ counts,
                                                      uint32_t ntiles) {
  __shared__ uint32_t h[RS_BINS];
  for (int i = threadIdx.x; i < RS_BINS; i += RS_THREADS) h[i] = 0;
  __syncthreads();
  size_t base = static_cast<size_t>(blockIdx.x) * RS_TILE;
#pragma unroll 4
  for (int k = 0; k < RS_IPT; k++) {
    size_t i = base + static_cast<size_t>(k) * RS_THREADS + threadIdx.x;
    if (i < n) atomicAdd(&h[(keys[i] >> shift) & (RS_BINS - 1)], 1u);
  }
  __syncthreads();
  for (int d = threadIdx.x; d < RS_BINS; d += RS_THREADS)
    counts[static_cast<size_t>(d) * ntiles + blockIdx.x] = h[d];
}

// Scatter of one pass.  Each warp ranks its keys with match_any so that equal
// digits keep input order; the tile is then staged in shared memory in
// digit-sorted order and written out in runs, so consecutive threads write
// consecutive output positions.
template <bool VALS>
__global__ void __launch_bounds__(RS_THREADS, 5) k_rs_scatter(
    const uint64_t *__restrict__ kin, const uint32_t *__restrict__ vin, uint64_t *__restrict__ kout,
    uint32_t *__restrict__ vout, size_t n, int shift, const uint32_t *__restrict__ offs,
    uint32_t ntiles) {
  extern __shared__ __align__(16) unsigned char rs_smem[];
  uint64_t *skey = reinterpret_cast<uint64_t *>(rs_smem);
  uint32_t *sval = reinterpret_cast<uint32_t *>(skey + RS_TILE);
  __shared__ uint32_t wcnt[RS_WARPS][RS_BINS];
  __shared__ uint32_t tstart[RS_BINS];
  __shared__ uint32_t gbase[RS_BINS];
  __shared__ uint32_t s_w[33];
  const uint32_t lane = lane_id(), w = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < RS_WARPS * RS_BINS; i += RS_THREADS) (&wcnt[0][0])[i] = 0;
  __syncthreads();
  // warp w owns keys [base + w*32*IPT, base + (w+1)*32*IPT), round r lane l
  // takes key base + w*32*IPT + r*32 + l: (w, r, l) order is the input order.
  const size_t tbase = static_cast<size_t>(blockIdx.x) * RS_TILE;
  const size_t wbase = tbase + static_cast<size_t>(w) * 32 * RS_IPT;
  uint64_t k[RS_IPT];
  uint32_t lr[RS_IPT];
  // all of the thread's keys are loaded before the ranking starts (the warp
  // barriers of the ranking would otherwise hold each load back)
  uint32_t vv[VALS ? RS_IPT : 1];
#pragma unroll
  for (int r = 0; r < RS_IPT; r++) {
    size_t i = wbase + static_cast<size_t>(r) * 32 + lane;
    k[r] = i < n ? kin[i] : 0;
    if (VALS) vv[r] = i < n ? vin[i] : 0;
  }
#pragma unroll
  for (int r = 0; r < RS_IPT; r++) {
    size_t i = wbase + static_cast<size_t>(r) * 32 + lane;
    bool valid = i < n;
    uint32_t d = valid ? static_cast<uint32_t>((k[r] >> shift) & (RS_BINS - 1)) : 0xffffffffu;
    uint32_t peers = __match_any_sync(FULL, d);
    uint32_t cur = valid ? wcnt[w][d] : 0;
    __syncwarp();
    if (valid && lane == static_cast<uint32_t>(__ffs(peers) - 1)) wcnt[w][d] = cur + __popc(peers);
    __syncwarp();
    lr[r] = cur + __popc(peers & lanemask_lt());
  }
  __syncthreads();
  {
    // thread d (RS_THREADS == RS_BINS): exclusive prefix over warps, then over digits
    const int d = threadIdx.x;
    uint32_t run = 0;
#pragma unroll
    for (int ww = 0; ww < RS_WARPS; ww++) {
      uint32_t c = wcnt[ww][d];
      wcnt[ww][d] = run;
      run += c;
    }
    uint32_t tot;
    uint32_t incl = block_incl_scan(run, s_w, &tot);
    tstart[d] = incl - run;
    gbase[d] = offs[static_cast<size_t>(d) * ntiles + blockIdx.x] - (incl - run);
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < RS_IPT; r++) {
    size_t i = wbase + static_cast<size_t>(r) * 32 + lane;
    if (i < n) {
      uint32_t d = static_cast<uint32_t>((k[r] >> shift) & (RS_BINS - 1));
      uint32_t lp = tstart[d] + wcnt[w][d] + lr[r];
      skey[lp] = k[r];
      if (VALS) sval[lp] = vv[r];
    }
  }
  __syncthreads();
  const uint32_t nvalid = n - tbase < RS_TILE ? static_cast<uint32_t>(n - tbase) : RS_TILE;
  for (uint32_t i = threadIdx.x; i < nvalid; i += RS_THREADS) {
    uint64_t key = skey[i];
    uint32_t d = static_cast<uint32_t>((key >> shift) & (RS_BINS - 1));
    size_t pos = static_cast<size_t>(gbase[d]) + i;
    kout[pos] = key;
    if (VALS) vout[pos] = sval[i];
  }
}

pb_status radix_sort(uint64_t *keys, uint32_t *vals, size_t n, int bits, cudaStream_t s) {
  if (n <= 1 || bits <= 0) return PB_OK;
  if (n >= (size_t(1) << 32)) return fail(PB_ERR_INVALID, "radix_sort: n too large");
  size_t ntiles = (n + RS_TILE - 1) / RS_TILE;
  uint64_t *k2 = nullptr;
  uint32_t *v2 = nullptr, *counts = nullptr, *offs = nullptr;
  PB_TRY(dalloc_t(&k2, n, s));
  pb_status st = PB_OK;
  if (vals) st = dalloc_t(&v2, n, s);
  if (st == PB_OK) st = dalloc_t(&counts, ntiles * RS_BINS, s);
  if (st == PB_OK) st = dalloc_t(&offs, ntiles * RS_BINS + 1, s);
  static bool attr_set = false;  // per process; the attribute is per function
  if (!attr_set) {
    cudaFuncSetAttribute(k_rs_scatter<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, RS_SMEM_VALS);
    cudaFuncSetAttribute(k_rs_scatter<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, RS_SMEM_KEYS);
    attr_set = true;
  }
  uint64_t *ka = keys, *kb = k2;
  uint32_t *va = vals, *vb = v2;
  int passes = (bits + 7) / 8;
  for (int p = 0; p < passes && st == PB_OK; p++) {
    int shift = p * 8;
    k_rs_hist<<<(unsigned)ntiles, RS_THREADS, 0, s>>>(ka, n, shift, counts, (uint32_t)ntiles);
    count_launch();
    if (cudaGetLastError() != cudaSuccess) { st = fail(PB_ERR_CUDA, "radix hist launch failed"); break; }
    st = scan_u32(counts, offs, ntiles * RS_BINS, s);
    if (st != PB_OK) break;
    if (vals)
      k_rs_scatter<true><<<(unsigned)ntiles, RS_THREADS, RS_SMEM_VALS, s>>>(ka, va, kb, vb, n, shift, offs,
                                                                           (uint32_t)ntiles);
    else
      k_rs_scatter<false><<<(unsigned)ntiles, RS_THREADS, RS_SMEM_KEYS, s>>>(ka, va, kb, vb, n, shift, offs,
                                                                            (uint32_t)ntiles);
    count_launch();
    if (cudaGetLastError() != cudaSuccess) { st = fail(PB_ERR_CUDA, "radix scatter launch failed"); break; }
    uint64_t *tk = ka; ka = kb; kb = tk;
    uint32_t *tv = va; va = vb; vb = tv;
  }
  if (st == PB_OK && ka != keys) {
    cudaError_t e = cudaMemcpyAsync(keys, ka, n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess && vals)
      e = cudaMemcpyAsync(vals, va, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) st = cuda_fail(e, "radix_sort copy-back", __FILE__, __LINE__);
  }
  dfree(k2, s);
  dfree(v2, s);
  dfree(counts, s);
  dfree(offs, s);
  return st;
}

// ---------------------------------------------------------------------------
__global__ void k_sum_u64(const uint64_t *__restrict__ in, size_t n, unsigned long long *out) {
  __shared__ unsigned long long s_w[33];
  unsigned long long acc = 0;
  for (size_t i = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += static_cast<size_t>(gridDim.x) * blockDim.x)
    acc += in[i];
  unsigned long long tot = block_sum(acc, s_w);
  if (threadIdx.x == 0 && tot) atomicAdd(out, tot);
}

pb_status sum_u64(const uint64_t *in, size_t n, unsigned long long *out, cudaStream_t s) {
  PB_CUDA(cudaMemsetAsync(out, 0, sizeof(unsigned long long), s));
  if (n == 0) return PB_OK;
  PB_LAUNCH(k_sum_u64, grid_for(n, 256, 4096), 256, 0, s, in, n, out);
  return PB_OK;
}

}  // namespace pb
