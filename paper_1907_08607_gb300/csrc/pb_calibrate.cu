// Measurement support (not on the counting path): the device's throughput of
// 64-bit atomic adds whose result is unused (reductions performed in L2), the
// operation the counting kernels use for every per-vertex and per-edge
// contribution (Sec. "Butterfly aggregation", atomic adds).  The figure is the
// second ceiling, beside HBM bandwidth, that the counting kernels' rates are
// compared with.
//
// Two address patterns, both over a 64 MiB array that stays resident in L2:
//  COALESCED: lane i of a warp adds to word base + i (32 consecutive 8-byte
//             words, 8 sectors per warp instruction), as the per-edge
//             counters of one neighbour's list are updated;
//  SCATTERED: every lane adds to a word picked by a hash of its index, as the
//             per-vertex counters of second endpoints are updated.
#include "pb_common.cuh"

namespace pb {

constexpr size_t CAL_WORDS = size_t(8) << 20;  // 64 MiB of 8-byte counters

__device__ __forceinline__ uint32_t cal_hash(uint32_t x) {
  x ^= x >> 16;
  x *= 0x7feb352dU;
  x ^= x >> 15;
  x *= 0x846ca68bU;
  x ^= x >> 16;
  return x;
}

template <bool SCATTER>
__global__ void __launch_bounds__(512) k_cal_red(unsigned long long *__restrict__ a, uint32_t rounds) {
  const uint32_t gtid = blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t nthreads = gridDim.x * blockDim.x;
  const uint32_t mask = static_cast<uint32_t>(CAL_WORDS - 1);
#pragma unroll 4
  for (uint32_t r = 0; r < rounds; r++) {
    const uint32_t i = r * nthreads + gtid;
    const uint32_t w = SCATTER ? cal_hash(i) & mask : i & mask;
    atomicAdd(&a[w], 1ull);  // result unused: compiled to a reduction
  }
}

}  // namespace pb

using namespace pb;

extern "C" pb_status pb_calibrate_atomics(int scattered, double *ops_per_s, void *stream) {
  clear_error();
  if (!ops_per_s) return fail(PB_ERR_INVALID, "ops_per_s is NULL");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int dev = 0;
  PB_CUDA(cudaGetDevice(&dev));
  unsigned long long *a = nullptr;
  PB_TRY(dalloc_t(&a, CAL_WORDS, s));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  pb_status st = PB_OK;
  do {
    if (cudaMemsetAsync(a, 0, CAL_WORDS * 8, s) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
      st = fail(PB_ERR_CUDA, "calibration set-up: %s", cudaGetErrorString(cudaGetLastError()));
      break;
    }
    const unsigned grid = static_cast<unsigned>(sm_count(dev) * 4), block = 512;
    const uint32_t rounds = 256;
    auto kern = scattered ? k_cal_red<true> : k_cal_red<false>;
    for (int w = 0; w < 2; w++) kern<<<grid, block, 0, s>>>(a, rounds);  // warm-up
    cudaEventRecord(e0, s);
    const int reps = 10;
    for (int r = 0; r < reps; r++) kern<<<grid, block, 0, s>>>(a, rounds);
    cudaEventRecord(e1, s);
    count_launch(2 + reps);
    cudaError_t e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e != cudaSuccess || ms <= 0.f) {
      st = cuda_fail(e, "calibration kernels", __FILE__, __LINE__);
      break;
    }
    *ops_per_s = static_cast<double>(grid) * block * rounds * reps / (ms * 1e-3);
  } while (0);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  dfree(a, s);
  cudaStreamSynchronize(s);
  return st;
}
