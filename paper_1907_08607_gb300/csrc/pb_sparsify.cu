// Graph sparsification for approximate global counts (Sec. "Approximate
// counting"): edge sparsification keeps each edge with probability p (the
// count of the kept graph divided by p^4 estimates the total); colourful
// sparsification gives every vertex one of c = ceil(1/p) colours and keeps the
// edges whose endpoints share a colour.  A butterfly survives colouring when
// its three other vertices take the colour of the first, with probability
// c^-3 (= p^3 when 1/p is an integer), so the kept count is multiplied by c^3.
//
// Randomness is a hash of the edge or the vertex, so duplicate input pairs
// get the same decision: SplitMix64's output function (Steele, Lea & Flood,
// OOPSLA 2014) applied as h = mix(mix(seed ^ a * 0x9E3779B97F4A7C15) + b),
// with (a, b) = (u, v) for an edge and (global id, 0x5BD1E995) for a colour;
// the uniform draw is (h >> 11) * 2^-53.
#include "pb_common.cuh"

namespace pb {

__device__ __forceinline__ uint64_t sp_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

__device__ __forceinline__ double sp_uniform(uint64_t seed, uint64_t a, uint64_t b) {
  uint64_t h = sp_mix(sp_mix(seed ^ (a * 0x9E3779B97F4A7C15ULL)) + b);
  return static_cast<double>(h >> 11) * (1.0 / 9007199254740992.0);
}

__global__ void k_sparsify_keep(const uint32_t *__restrict__ u, const uint32_t *__restrict__ v, uint64_t m,
                                uint32_t nU, int kind, double p, uint64_t colors, uint64_t seed,
                                uint32_t *__restrict__ keep) {
  for (size_t k = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x; k < m;
       k += static_cast<size_t>(gridDim.x) * blockDim.x) {
    bool kp;
    if (kind == PB_SPARSIFY_EDGE) {
      kp = sp_uniform(seed, u[k], v[k]) < p;
    } else {
      uint64_t cu = static_cast<uint64_t>(sp_uniform(seed, u[k], 0x5BD1E995ULL) * static_cast<double>(colors));
      uint64_t cv = static_cast<uint64_t>(sp_uniform(seed, static_cast<uint64_t>(nU) + v[k], 0x5BD1E995ULL) *
                                          static_cast<double>(colors));
      kp = cu == cv;
    }
    keep[k] = kp ? 1u : 0u;
  }
}

__global__ void k_sparsify_compact(const uint32_t *__restrict__ u, const uint32_t *__restrict__ v, uint64_t m,
                                   const uint32_t *__restrict__ keep, const uint32_t *__restrict__ pos,
                                   uint32_t *__restrict__ ou, uint32_t *__restrict__ ov) {
  for (size_t k = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x; k < m;
       k += static_cast<size_t>(gridDim.x) * blockDim.x) {
    if (keep[k]) {
      ou[pos[k]] = u[k];
      ov[pos[k]] = v[k];
    }
  }
}

// estimate = count * scale, with the exact count read from the counting
// accumulator on the device.
__global__ void k_approx_scale(const unsigned long long *__restrict__ count, double scale, double *__restrict__ out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) out[0] = static_cast<double>(count[0]) * scale;
}

// Filters the m pairs (device arrays) into the device arrays ou / ov (m
// entries of room); *kept receives the number kept (host).
static pb_status sparsify_device(uint32_t nU, uint64_t m, const uint32_t *du, const uint32_t *dv, int kind, double p,
                                 uint64_t seed, uint32_t *ou, uint32_t *ov, uint32_t *kept, cudaStream_t s) {
  *kept = 0;
  if (m == 0) return PB_OK;
  const uint64_t colors = static_cast<uint64_t>(ceil(1.0 / p));
  uint32_t *keep = nullptr, *pos = nullptr;
  pb_status st = PB_OK;
  do {
    if ((st = dalloc_t(&keep, m, s)) != PB_OK || (st = dalloc_t(&pos, m + 1, s)) != PB_OK) break;
    k_sparsify_keep<<<grid_for(m, 256, 8192), 256, 0, s>>>(du, dv, m, nU, kind, p, colors, seed, keep);
    count_launch();
    if ((st = scan_u32(keep, pos, m, s)) != PB_OK) break;
    k_sparsify_compact<<<grid_for(m, 256, 8192), 256, 0, s>>>(du, dv, m, keep, pos, ou, ov);
    count_launch();
    if (cudaMemcpyAsync(kept, pos + m, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) st = fail(PB_ERR_CUDA, "kept-edge count readback");
  } while (0);
  dfree(keep, s);
  dfree(pos, s);
  return st;
}

}  // namespace pb

using namespace pb;

extern "C" pb_status pb_sparsify(uint32_t nU, uint32_t nV, uint64_t m, const uint32_t *u, const uint32_t *v,
                                 int on_device, pb_sparsify_kind kind, double p, uint64_t seed, uint32_t *out_u,
                                 uint32_t *out_v, uint64_t *out_m, void *stream) {
  clear_error();
  if (!out_m || (m > 0 && (!u || !v || !out_u || !out_v))) return fail(PB_ERR_INVALID, "NULL argument");
  if (!(p > 0.0 && p <= 1.0)) return fail(PB_ERR_INVALID, "p must be in (0, 1]");
  if (kind != PB_SPARSIFY_EDGE && kind != PB_SPARSIFY_COLOR) return fail(PB_ERR_INVALID, "unknown kind");
  if (m >= (uint64_t(1) << 32) - 1) return fail(PB_ERR_INVALID, "too many edges");
  (void)nV;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  *out_m = 0;
  if (m == 0) return PB_OK;
  const uint64_t colors = static_cast<uint64_t>(ceil(1.0 / p));
  uint32_t *du = nullptr, *dv = nullptr, *keep = nullptr, *pos = nullptr;
  const uint32_t *cu = u, *cv = v;
  pb_status st = PB_OK;
  uint32_t hm = 0;
  do {
    if (!on_device) {
      if ((st = dalloc_t(&du, m, s)) != PB_OK || (st = dalloc_t(&dv, m, s)) != PB_OK) break;
      if (cudaMemcpyAsync(du, u, m * 4, cudaMemcpyHostToDevice, s) != cudaSuccess ||
          cudaMemcpyAsync(dv, v, m * 4, cudaMemcpyHostToDevice, s) != cudaSuccess) { st = fail(PB_ERR_CUDA, "upload"); break; }
      cu = du;
      cv = dv;
    }
    if ((st = dalloc_t(&keep, m, s)) != PB_OK || (st = dalloc_t(&pos, m + 1, s)) != PB_OK) break;
    k_sparsify_keep<<<grid_for(m, 256, 8192), 256, 0, s>>>(cu, cv, m, nU, kind, p, colors, seed, keep);
    count_launch();
    if ((st = scan_u32(keep, pos, m, s)) != PB_OK) break;
    if (cudaMemcpyAsync(&hm, pos + m, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) { st = fail(PB_ERR_CUDA, "count readback"); break; }
    uint32_t *ou = out_u, *ov = out_v, *tu = nullptr, *tv = nullptr;
    if (!on_device) {
      if ((st = dalloc_t(&tu, hm + 1, s)) != PB_OK || (st = dalloc_t(&tv, hm + 1, s)) != PB_OK) break;
      ou = tu;
      ov = tv;
    }
    k_sparsify_compact<<<grid_for(m, 256, 8192), 256, 0, s>>>(cu, cv, m, keep, pos, ou, ov);
    count_launch();
    if (!on_device && hm) {
      if (cudaMemcpyAsync(out_u, tu, hm * 4ull, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
          cudaMemcpyAsync(out_v, tv, hm * 4ull, cudaMemcpyDeviceToHost, s) != cudaSuccess) st = fail(PB_ERR_CUDA, "download");
    }
    dfree(tu, s);
    dfree(tv, s);
  } while (0);
  dfree(du, s); dfree(dv, s); dfree(keep, s); dfree(pos, s);
  cudaError_t e = cudaStreamSynchronize(s);
  if (st != PB_OK) return st;
  if (e != cudaSuccess) return cuda_fail(e, "sparsify", __FILE__, __LINE__);
  *out_m = hm;
  return PB_OK;
}

extern "C" pb_status pb_count_approx(uint32_t nU, uint32_t nV, uint64_t m, const uint32_t *u, const uint32_t *v,
                                     int on_device, pb_sparsify_kind kind, double p, uint64_t seed,
                                     pb_rank_kind rank, pb_agg agg, uint64_t scratch_bytes, double *estimate,
                                     uint64_t *kept_count, uint64_t *kept_edges, void *stream) {
  clear_error();
  if (!estimate || (m > 0 && (!u || !v))) return fail(PB_ERR_INVALID, "NULL argument");
  if (!(p > 0.0 && p <= 1.0)) return fail(PB_ERR_INVALID, "p must be in (0, 1]");
  if (kind != PB_SPARSIFY_EDGE && kind != PB_SPARSIFY_COLOR) return fail(PB_ERR_INVALID, "unknown kind");
  if (m >= (uint64_t(1) << 32) - 1) return fail(PB_ERR_INVALID, "too many edges");
  if (static_cast<uint64_t>(nU) + nV == 0) return fail(PB_ERR_INVALID, "graph has no vertices");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  double scale;
  if (kind == PB_SPARSIFY_EDGE) {
    scale = 1.0 / (p * p * p * p);
  } else {
    const double c = ceil(1.0 / p);
    scale = c * c * c;
  }
  uint32_t *du = nullptr, *dv = nullptr, *ou = nullptr, *ov = nullptr;
  double *dest = nullptr;
  pb_graph *g = nullptr;
  uint32_t kept = 0;
  uint64_t cnt = 0;
  pb_status st = PB_OK;
  do {
    const uint32_t *cu = u, *cv = v;
    if (m > 0 && !on_device) {
      if ((st = dalloc_t(&du, m, s)) != PB_OK || (st = dalloc_t(&dv, m, s)) != PB_OK) break;
      if (cudaMemcpyAsync(du, u, m * 4, cudaMemcpyHostToDevice, s) != cudaSuccess ||
          cudaMemcpyAsync(dv, v, m * 4, cudaMemcpyHostToDevice, s) != cudaSuccess) { st = fail(PB_ERR_CUDA, "upload"); break; }
      cu = du;
      cv = dv;
    }
    if ((st = dalloc_t(&ou, m + 1, s)) != PB_OK || (st = dalloc_t(&ov, m + 1, s)) != PB_OK) break;
    if ((st = dalloc_t(&dest, 1, s)) != PB_OK) break;
    if ((st = sparsify_device(nU, m, cu, cv, kind, p, seed, ou, ov, &kept, s)) != PB_OK) break;
    if ((st = pb_graph_from_edges(nU, nV, kept, ou, ov, 1, stream, &g)) != PB_OK) break;
    if ((st = pb_rank(g, rank, stream)) != PB_OK) break;
    if ((st = pb_count_global(g, agg, scratch_bytes, &cnt, stream)) != PB_OK) break;
    {
      int cur = 0;
      cudaGetDevice(&cur);
      if (cur != g->device) cudaSetDevice(g->device);
      k_approx_scale<<<1, 32, 0, s>>>(g->acc, scale, dest);
      count_launch();
      cudaError_t e = cudaMemcpyAsync(estimate, dest, sizeof(double), cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (cur != g->device) cudaSetDevice(cur);
      if (e != cudaSuccess) { st = cuda_fail(e, "approximate count scaling", __FILE__, __LINE__); break; }
    }
  } while (0);
  if (g) {
    std::string keep_err = pb_last_error();
    pb_graph_free(g);
    if (st != PB_OK) fail(st, "%s", keep_err.c_str());
  }
  dfree(du, s); dfree(dv, s); dfree(ou, s); dfree(ov, s); dfree(dest, s);
  cudaError_t e = cudaStreamSynchronize(s);
  if (st != PB_OK) return st;
  if (e != cudaSuccess) return cuda_fail(e, "approximate count", __FILE__, __LINE__);
  if (kept_count) *kept_count = cnt;
  if (kept_edges) *kept_edges = kept;
  return PB_OK;
}
