// Graph sparsification for approximate global counts (Sec. "Approximate
// counting"): edge sparsification keeps each edge with probability p (the
// count of the kept graph divided by p^4 estimates the total); colourful
// sparsification gives every vertex one of ceil(1/p) colours and keeps the
// edges whose endpoints share a colour (divide by p^3).
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
