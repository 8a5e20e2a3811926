// Wedge retrieval (Algorithm 2) fused with wedge aggregation (GET-FREQ,
// Sec. "Wedge aggregation") and butterfly aggregation with atomic adds
// (Sec. "Butterfly aggregation"; Algorithms 3 and 4).
//
// For a first endpoint x1 the wedges are ((x1, x2), y) with y in the first
// deg_x1(x1) slots of x1's list and x2 in the first deg_x1(y) slots of y's
// list (lists are sorted by decreasing rank).  The wedges of x1 are grouped by
// x2; the group size d(x1, x2) = |N(x1) n N(x2)| restricted to centres ranked
// above x1.  Then, per group:
//   global += C(d, 2); pv[x1] += C(d, 2); pv[x2] += C(d, 2)          (Eq. 1)
// and per wedge (second pass over the same wedges, d still in scratch):
//   pv[y] += d - 1; e(x1, y) += d - 1; e(x2, y) += d - 1             (Eq. 2)
// Edge contributions land on adjacency slots: e(x2, y) on the slot of x2 in
// y's list, e(x1, y) on the slot of y in x1's list; an edge's count is the sum
// of its two slots.
//
// Work split: first endpoints are binned by their wedge count (prefix sums of
// the PREPROCESS step):
//   light  (<= 512 wedges)   one warp per x1, hash table in shared memory;
//   medium (<= 4096 wedges)  one block per x1, hash table in shared memory;
//   heavy                    one thread-block cluster per x1, aggregation in
//                            device memory: a dense histogram over all second
//                            endpoints with a touched list, or an
//                            open-addressing hash table.
// Inside a warp / block / cluster the wedges of a chunk of neighbours are
// flattened with a prefix sum over deg_x1(y) and spread evenly over threads.
#include <cooperative_groups.h>

#include <cmath>
#include <cstdlib>
#include <new>
#include <string>
#include <type_traits>
#include <vector>

#include "pb_common.cuh"

namespace cg = cooperative_groups;

namespace pb {

struct CArgs {
  const uint32_t *__restrict__ off;
  const uint32_t *__restrict__ adj;
  const uint32_t *__restrict__ cpos;
  const uint32_t *__restrict__ degp;
  const uint64_t *__restrict__ wpre;
  uint64_t n;
  uint32_t nU;              // labels [0, nU) are U vertices, [nU, n) V vertices
  int rev;                  // 1: wedges are owned by their higher-ranked endpoint
  unsigned long long *pv;   // [n] by label, or null
  unsigned long long *es;   // [2m] per slot, or null
  unsigned int *es32;       // [2m] per-slot 32-bit partials of the per-wedge contributions, or null
  uint32_t nlim[2];         // y's list takes 32-bit partials when deg(y) - 1 <= nlim[side of its entries]
  unsigned long long *acc;  // [0] global, [1] overflow, [2..] work queues
};

// Accumulator words: the global count and its overflow word, the work queues
// of the block tiers, the list cursors of the tier split, an error word.
enum { ACC_GLOBAL = 0, ACC_OVF = 1, ACC_QMED = 2, ACC_QHEAVY = 3, ACC_NLIGHT = 4, ACC_NMED = 5,
       ACC_NLARGE = 6, ACC_NHEAVY = 7, ACC_ERR = 8, ACC_NHUB = 9, ACC_QLARGE = 10, ACC_WORDS = 16 };

// Probe loops are bounded by the table size; running past it (impossible at
// load <= 1/2 unless scratch is corrupt) records an error instead of spinning.

constexpr uint32_t LIGHT_MAX = 768;   // wedges of a light first endpoint
constexpr int LW_THREADS = 512;
constexpr int LW_WARPS = LW_THREADS / 32;
constexpr int LW_CAP = 1024;          // per-warp table entries (> LIGHT_MAX: never full)
constexpr int LW_LG = 10;
constexpr uint32_t MED_MAX = 4096;
constexpr int MB_THREADS = 512;
constexpr int MB_WARPS = MB_THREADS / 32;
constexpr int MB_CAP = 8192;          // per-block table entries (>= 2 * MED_MAX)
// medium-tier dynamic shared memory: keys, 16-bit counts, 16-bit table position per wedge
constexpr size_t MB_SMEM = (MB_CAP + MB_CAP / 2) * sizeof(uint32_t) + MED_MAX * sizeof(uint16_t);
constexpr int HB_THREADS = 1024;

// Per-wedge edge contributions of the heavy tiers go to 32-bit per-slot
// partial counters where they cannot wrap: the count of edge (x2, y) is at
// most (deg(x2) - 1)(deg(y) - 1) (a butterfly through the edge picks one other
// neighbour of each endpoint), so every slot of y's list is safe when
// deg(y) - 1 <= nlim, nlim = (2^32 - 1) / (largest degree on x2's side - 1).
// On an array far larger than L2, where most reductions miss, a 4-byte
// reduction moves half the sector bytes of an 8-byte one.  The lists of the
// few centres above the limit keep 64-bit counters.  An edge's count is the
// sum of both arrays over its two slots.
__device__ __forceinline__ bool es_narrow(const CArgs &a, uint32_t x1, uint32_t dy) {
  return dy - 1 <= (x1 < a.nU ? a.nlim[0] : a.nlim[1]);  // constant indices keep a copy of CArgs in registers
}

__device__ __forceinline__ void es_add_wedge(const CArgs &a, uint32_t sl, uint32_t t, bool narrow) {
  if (narrow) atomicAdd(&a.es32[sl], t);
  else atomicAdd(&a.es[sl], static_cast<unsigned long long>(t));
}

__device__ __forceinline__ void add_global(unsigned long long *acc, unsigned long long v) {
  if (!v) return;
  unsigned long long old = atomicAdd(&acc[ACC_GLOBAL], v);
  if (old + v < old) atomicAdd(&acc[ACC_OVF], 1ull);
}

// Per-vertex counts of the lowest labels of each side (the highest-degree
// vertices under degree-like rankings) are hit by many owners at once when
// owners are the higher-ranked endpoints.  Blocks add them into a shared
// array first and flush it once at the end.
constexpr int HUBK = 512;  // cached labels per side

__device__ __forceinline__ void pv_add(unsigned long long *s_hub, const CArgs &a, uint32_t x,
                                       unsigned long long b) {
  if (s_hub) {
    const uint32_t side = x < a.nU ? 0u : 1u;
    const uint32_t o = x - (side ? a.nU : 0u);
    if (o < HUBK) {
      atomicAdd(&s_hub[side * HUBK + o], b);
      return;
    }
  }
  atomicAdd(&a.pv[x], b);
}

__device__ __forceinline__ void hub_zero(unsigned long long *s_hub) {
  for (uint32_t t = threadIdx.x; t < 2 * HUBK; t += blockDim.x) s_hub[t] = 0;
}

// Called by the whole block after its last owner.
__device__ __forceinline__ void hub_flush(unsigned long long *s_hub, const CArgs &a) {
  for (uint32_t t = threadIdx.x; t < 2 * HUBK; t += blockDim.x) {
    unsigned long long v = s_hub[t];
    if (!v) continue;
    const uint64_t x = t < HUBK ? t : static_cast<uint64_t>(a.nU) + (t - HUBK);
    if (x < a.n) atomicAdd(&a.pv[x], v);
  }
}

__device__ __forceinline__ uint32_t hash_home(uint32_t x, int lg) {
  return (x * 0x9E3779B1u) >> (32 - lg);
}

// Shared-memory open addressing (linear probing, atomic-add combine).
__device__ __forceinline__ void sh_add(uint32_t *key, uint32_t *cnt, int lg, uint32_t x,
                                       unsigned long long *err) {
  const uint32_t mask = (1u << lg) - 1;
  uint32_t h = hash_home(x, lg);
  for (uint32_t probe = 0;; probe++) {
    if (probe > mask) { atomicOr(err, 1ull); return; }
    uint32_t k = reinterpret_cast<volatile uint32_t *>(key)[h];
    if (k == x) break;
    if (k == EMPTY) {
      uint32_t prev = atomicCAS(&key[h], EMPTY, x);
      if (prev == EMPTY || prev == x) break;
    }
    h = (h + 1) & mask;
  }
  atomicAdd(&cnt[h], 1u);
}

__device__ __forceinline__ uint32_t sh_get(const uint32_t *key, const uint32_t *cnt, int lg, uint32_t x,
                                           unsigned long long *err) {
  const uint32_t mask = (1u << lg) - 1;
  uint32_t h = hash_home(x, lg);
  for (uint32_t probe = 0; key[h] != x; probe++) {
    if (probe > mask) { atomicOr(err, 2ull); return 0; }
    h = (h + 1) & mask;
  }
  return cnt[h];
}

// Bound on the distinct other endpoints of an owner x: its wedges, and the
// vertices of its own side on the far side of it in rank order (labels above x
// up to the side's end when x owns as the lower endpoint, labels below x down
// to the side's start when it owns as the higher one).
__device__ __forceinline__ uint64_t distinct_bound(uint64_t wc, uint64_t n, uint32_t nU, uint32_t x, int rev) {
  uint64_t side_end = x < nU ? nU : n, side_begin = x < nU ? 0 : nU;
  uint64_t room = rev ? x - side_begin : side_end - 1 - x;
  return wc < room ? wc : room;
}

// Neighbour i of owner x (slot xbase + i): its label y, the number c of
// wedges through y that x owns, and the slot oy in y's list where their other
// endpoints start.  Owning as the lower endpoint (Algorithm 2): the first
// deg_x(y) entries of y's list.  Owning as the higher endpoint (the cache
// optimisation of Sec. "Other options"): the entries of y's list ranked below
// both y and x, a suffix starting after deg_y(y) and after x's own position.
__device__ __forceinline__ void owner_nbr(const CArgs &a, uint32_t xbase, uint32_t i, bool v, uint32_t &y,
                                          uint32_t &c, uint32_t &oy) {
  if (!v) {
    y = 0; c = 0; oy = 0;
    return;
  }
  const uint32_t sl = xbase + i;
  y = a.adj[sl];
  const uint32_t p = a.cpos[sl];
  const uint32_t o0 = a.off[y];
  if (!a.rev) {
    c = p;
    oy = o0;
    return;
  }
  const uint32_t dy = a.off[y + 1] - o0;
  uint32_t st = a.degp[y];
  if (p + 1 > st) st = p + 1;
  c = dy > st ? dy - st : 0;
  oy = o0 + st;
}

// First label a dense histogram of owner x1 covers: its second endpoints are
// the labels of its side below x1 (owner = higher-ranked endpoint) or above
// it (owner = lower-ranked endpoint), so a histogram of the owner's range of
// labels suffices.
__device__ __forceinline__ uint32_t dense_base(const CArgs &a, uint32_t x1) {
  return a.rev ? (x1 < a.nU ? 0u : a.nU) : x1 + 1;
}

// Number of neighbours of owner x that can carry its wedges.
__device__ __forceinline__ uint32_t owner_span(const CArgs &a, uint32_t x) {
  return a.rev ? a.off[x + 1] - a.off[x] : a.degp[x];
}

// The same table with 16-bit counts, two per 32-bit word (cnt16 holds cap/2
// words).  Only for owners whose wedge count, and so every group size d, is
// below 2^16: the light tier.
__device__ __forceinline__ uint32_t sh_add16(uint32_t *key, uint32_t *cnt16, int lg, uint32_t x,
                                             unsigned long long *err) {
  const uint32_t mask = (1u << lg) - 1;
  uint32_t h = hash_home(x, lg);
  for (uint32_t probe = 0;; probe++) {
    if (probe > mask) { atomicOr(err, 1ull); return 0; }
    uint32_t k = reinterpret_cast<volatile uint32_t *>(key)[h];
    if (k == x) break;
    if (k == EMPTY) {
      uint32_t prev = atomicCAS(&key[h], EMPTY, x);
      if (prev == EMPTY || prev == x) break;
    }
    h = (h + 1) & mask;
  }
  atomicAdd(&cnt16[h >> 1], 1u << ((h & 1u) << 4));
  return h;
}

// As sh_add16, returning the table position with bit 15 set for the first
// insertion of x (its count was 0).  Tables of at most 2^15 entries.
__device__ __forceinline__ uint32_t sh_add16f(uint32_t *key, uint32_t *cnt16, int lg, uint32_t x,
                                              unsigned long long *err) {
  const uint32_t mask = (1u << lg) - 1;
  uint32_t h = hash_home(x, lg);
  for (uint32_t probe = 0;; probe++) {
    if (probe > mask) { atomicOr(err, 1ull); return 0; }
    uint32_t k = reinterpret_cast<volatile uint32_t *>(key)[h];
    if (k == x) break;
    if (k == EMPTY) {
      uint32_t prev = atomicCAS(&key[h], EMPTY, x);
      if (prev == EMPTY || prev == x) break;
    }
    h = (h + 1) & mask;
  }
  const uint32_t sh = (h & 1u) << 4;
  const uint32_t old = atomicAdd(&cnt16[h >> 1], 1u << sh);
  return h | (((old >> sh) & 0xffffu) == 0 ? 0x8000u : 0u);
}

// As sh_add16, also setting bit h of the occupancy bitmap occ when x takes a
// new entry h.
__device__ __forceinline__ void sh_add16m(uint32_t *key, uint32_t *cnt16, uint32_t *occ, int lg, uint32_t x,
                                          unsigned long long *err) {
  const uint32_t mask = (1u << lg) - 1;
  uint32_t h = hash_home(x, lg);
  for (uint32_t probe = 0;; probe++) {
    if (probe > mask) { atomicOr(err, 1ull); return; }
    uint32_t k = reinterpret_cast<volatile uint32_t *>(key)[h];
    if (k == x) break;
    if (k == EMPTY) {
      uint32_t prev = atomicCAS(&key[h], EMPTY, x);
      if (prev == EMPTY) {
        atomicOr(&occ[h >> 5], 1u << (h & 31u));
        break;
      }
      if (prev == x) break;
    }
    h = (h + 1) & mask;
  }
  atomicAdd(&cnt16[h >> 1], 1u << ((h & 1u) << 4));
}

__device__ __forceinline__ uint32_t cnt16_at(const uint32_t *cnt16, uint32_t h) {
  return (cnt16[h >> 1] >> ((h & 1u) << 4)) & 0xffffu;
}

__device__ __forceinline__ uint32_t sh_get16(const uint32_t *key, const uint32_t *cnt16, int lg, uint32_t x,
                                             unsigned long long *err) {
  const uint32_t mask = (1u << lg) - 1;
  uint32_t h = hash_home(x, lg);
  for (uint32_t probe = 0; key[h] != x; probe++) {
    if (probe > mask) { atomicOr(err, 2ull); return 0; }
    h = (h + 1) & mask;
  }
  return cnt16_at(cnt16, h);
}

// Table size: a power of two at least twice the bound on distinct second
// endpoints (load factor at most 1/2).
__device__ __forceinline__ int table_lg(uint64_t wc, uint64_t n, uint32_t nU, uint32_t x1, int rev) {
  uint64_t dmax = distinct_bound(wc, n, nU, x1, rev);
  int lg = 5;
  while ((uint64_t(1) << lg) < 2 * dmax) lg++;
  return lg;
}

// Warp-level: which lane's neighbour owns flattened wedge index wi, and the
// adjacency slot of that wedge's second endpoint.
__device__ __forceinline__ void warp_locate(uint32_t incl, uint32_t c, uint32_t oy, uint32_t wi,
                                            uint32_t &src, uint32_t &slot) {
  int lo = 0;
#pragma unroll
  for (int step = 16; step; step >>= 1) {
    uint32_t v = __shfl_sync(FULL, incl, lo + step - 1);
    if (v <= wi) lo += step;
  }
  uint32_t s_incl = __shfl_sync(FULL, incl, lo);
  uint32_t s_c = __shfl_sync(FULL, c, lo);
  uint32_t s_oy = __shfl_sync(FULL, oy, lo);
  src = static_cast<uint32_t>(lo);
  slot = s_oy + (wi - (s_incl - s_c));
}

// Adds v into acc[key] for every lane, combining lanes whose keys are equal
// and adjacent (keys are non-decreasing across the warp, as the flattened
// wedges of a neighbour chunk are): one shared atomic per run of equal keys
// instead of one per lane.  All 32 lanes must call it; inactive lanes pass
// v = 0.
__device__ __forceinline__ void warp_run_add(unsigned long long *acc, uint32_t key, unsigned long long v) {
  const uint32_t lane = lane_id();
  const uint32_t prev = __shfl_up_sync(FULL, key, 1);
  const bool head = lane == 0 || prev != key;
  const uint32_t heads = __ballot_sync(FULL, head);
  // segmented inclusive scan from the right: each run head gets its run's sum
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    unsigned long long u = __shfl_down_sync(FULL, v, o);
    // lane + o is in this lane's run iff no run head lies in (lane, lane + o]
    if (lane + o < 32 && (heads & (((1u << o) - 1u) << (lane + 1))) == 0) v += u;
  }
  if (head && v) atomicAdd(&acc[key], v);
}

// As warp_run_add, for v < 2^32: each run's lanes reduce over their own lane
// mask (the 16-bit halves separately, so no partial sum overflows 32 bits).
// Faster than the shuffle scan in the light tier, slower in the others.
__device__ __forceinline__ void warp_run_add_rx(unsigned long long *acc, uint32_t key, unsigned long long v) {
  const uint32_t lane = lane_id();
  const uint32_t prev = __shfl_up_sync(FULL, key, 1);
  const bool head = lane == 0 || prev != key;
  const uint32_t heads = __ballot_sync(FULL, head);
  const uint32_t upto = 0xffffffffu >> (31 - lane);             // lanes 0..lane
  const uint32_t start = 31 - __clz(heads & upto);               // this lane's run head
  const uint32_t after = heads & ~upto;                          // heads beyond this lane
  const uint32_t below_end = after ? (1u << (__ffs(after) - 1)) - 1u : 0xffffffffu;
  const uint32_t run = below_end & ~((1u << start) - 1u);
  const uint32_t v32 = static_cast<uint32_t>(v);
  const uint32_t lo = __reduce_add_sync(run, v32 & 0xffffu), hi = __reduce_add_sync(run, v32 >> 16);
  const unsigned long long sum = static_cast<unsigned long long>(lo) + (static_cast<unsigned long long>(hi) << 16);
  if (head && sum) atomicAdd(&acc[key], sum);
}

// ---------------------------------------------------------------------------
// Light tier: one warp per owner, per-warp table with 16-bit counts.  Light
// owners have few neighbours with long segments (the 1/16 copy of 20M x 60M:
// two to three non-empty segments of ~95 wedges per owner, 95 % of the light
// wedges in segments of 32 or more), so the warp walks one segment at a time
// with its lanes (coalesced adjacency reads, LW_ILP loads per lane in flight)
// and sums a segment's d - 1 in registers: no per-wedge search for the
// wedge's neighbour and no per-wedge run reduction.
constexpr int LW_ILP = 4;

// Centre walk of one segment (positions [0, c) of the list at oy): d - 1 of
// every wedge added to its edge slot (32-bit partials when NARROW), the sum
// over the segment returned to every lane.  d <= LIGHT_MAX, so the sum fits
// 32 bits.
template <bool PE, bool NARROW>
__device__ __forceinline__ uint32_t light_centre_walk(const CArgs &a, const uint32_t *key, const uint32_t *cnt,
                                                      int lg, uint32_t oy, uint32_t c, unsigned long long *err) {
  uint32_t sum = 0;
  for (uint32_t e0 = lane_id(); e0 < c; e0 += 32 * LW_ILP) {
    uint32_t x2v[LW_ILP];
#pragma unroll
    for (int q = 0; q < LW_ILP; q++) x2v[q] = e0 + 32 * q < c ? a.adj[oy + e0 + 32 * q] : 0u;
#pragma unroll
    for (int q = 0; q < LW_ILP; q++) {
      const uint32_t e = e0 + 32 * q;
      if (e >= c) break;
      const uint32_t d = sh_get16(key, cnt, lg, x2v[q], err);
      if (d > 1) {
        sum += d - 1;
        if (PE) {
          if (NARROW) atomicAdd(&a.es32[oy + e], d - 1);
          else atomicAdd(&a.es[oy + e], static_cast<unsigned long long>(d - 1));
        }
      }
    }
  }
  return warp_sum(sum);
}

template <bool PV, bool PE, bool MULTI>
__global__ void __launch_bounds__(LW_THREADS, 2) k_light(CArgs a0, const uint32_t *__restrict__ list,
                                                      uint32_t nlist, const uint64_t *__restrict__ items,
                                                      const CArgs *__restrict__ tab) {
  extern __shared__ uint32_t dsm[];  // per warp: LW_CAP keys, then LW_CAP / 2 count words
  __shared__ uint32_t s_occ[LW_WARPS][LW_CAP / 32];  // per warp: occupied table entries
  __shared__ unsigned long long s_hubarr[2 * HUBK];
  unsigned long long *s_hub = (PV && !MULTI) ? s_hubarr : nullptr;
  const uint32_t lane = lane_id(), w = threadIdx.x >> 5;
  uint32_t *key = dsm + w * (LW_CAP + LW_CAP / 2), *cnt = key + LW_CAP, *occ = s_occ[w];
  static_assert(LW_CAP == 32 * 32, "one bitmap word of 32 entries per lane");
  unsigned long long *err = &a0.acc[ACC_ERR];
  unsigned long long gacc = 0;
  if (s_hub) hub_zero(s_hub);
  // The table always has LW_CAP entries and is cleared once; each owner marks
  // the entries it takes in occ, and its endpoint phase and reset visit only
  // those (lane l owns entries [32 l, 32 l + 32) and count words [16 l, 16 l + 16)).
  for (uint32_t t = lane; t < LW_CAP; t += 32) key[t] = EMPTY;
  for (uint32_t t = lane; t < LW_CAP / 2; t += 32) cnt[t] = 0;
  occ[lane] = 0;
  __syncthreads();
  for (uint32_t it = blockIdx.x * LW_WARPS + w; it < nlist; it += gridDim.x * LW_WARPS) {
    uint32_t x1;
    CArgs a;  // this item's graph
    if (MULTI) {
      const uint64_t item = items[it];
      a = tab[item >> 32];
      x1 = static_cast<uint32_t>(item);
    } else {
      a = a0;
      x1 = list[it];
    }
    const int lg = LW_LG;
    const uint32_t base = a.off[x1], dp = owner_span(a, x1);
    // An owner with at most 32 neighbours has one chunk: its neighbour data
    // stay in registers for the second pass.
    uint32_t ky = 0, kc = 0, koy = 0;
    for (uint32_t k0 = 0; k0 < dp; k0 += 32) {
      const uint32_t i = k0 + lane;
      uint32_t y, c, oy;
      owner_nbr(a, base, i, i < dp, y, c, oy);
      ky = y; kc = c; koy = oy;
      for (uint32_t bm = __ballot_sync(FULL, c > 0); bm; bm &= bm - 1) {
        const int j = __ffs(bm) - 1;
        const uint32_t cj = __shfl_sync(FULL, c, j), oyj = __shfl_sync(FULL, oy, j);
        for (uint32_t e0 = lane; e0 < cj; e0 += 32 * LW_ILP) {
          uint32_t x2v[LW_ILP];
#pragma unroll
          for (int q = 0; q < LW_ILP; q++) x2v[q] = e0 + 32 * q < cj ? a.adj[oyj + e0 + 32 * q] : 0u;
#pragma unroll
          for (int q = 0; q < LW_ILP; q++) {
            if (e0 + 32 * q >= cj) break;
            sh_add16m(key, cnt, occ, lg, x2v[q], err);
          }
        }
      }
    }
    __syncwarp();
    unsigned long long own = 0;
    for (uint32_t bits = occ[lane]; bits; bits &= bits - 1) {
      const uint32_t t = lane * 32 + (__ffs(bits) - 1);
      unsigned long long d = cnt16_at(cnt, t), b = d * (d - 1) / 2;
      own += b;
      if (PV && b) pv_add(s_hub, a, key[t], b);
    }
    own = warp_sum(own);
    if (lane == 0) {
      if (MULTI) add_global(a.acc, own);
      else gacc += own;
      if (PV && own) atomicAdd(&a.pv[x1], own);
    }
    if (PV || PE) {
      for (uint32_t k0 = 0; k0 < dp; k0 += 32) {
        const uint32_t i = k0 + lane;
        const bool v = i < dp;
        uint32_t y = ky, c = kc, oy = koy;
        if (dp > 32) owner_nbr(a, base, i, v, y, c, oy);
        const bool nar = PE && v && es_narrow(a, x1, a.off[y + 1] - a.off[y]);
        uint32_t mine = 0;  // the sum over neighbour i's segment
        for (uint32_t bm = __ballot_sync(FULL, c > 0); bm; bm &= bm - 1) {
          const int j = __ffs(bm) - 1;
          const uint32_t cj = __shfl_sync(FULL, c, j), oyj = __shfl_sync(FULL, oy, j);
          const uint32_t sj = __shfl_sync(FULL, static_cast<uint32_t>(nar), j)
                                  ? light_centre_walk<PE, true>(a, key, cnt, lg, oyj, cj, err)
                                  : light_centre_walk<PE, false>(a, key, cnt, lg, oyj, cj, err);
          if (lane == static_cast<uint32_t>(j)) mine = sj;
        }
        if (mine) {
          if (PV) pv_add(s_hub, a, y, mine);
          if (PE) atomicAdd(&a.es[base + i], static_cast<unsigned long long>(mine));
        }
      }
    }
    __syncwarp();
    // reset the entries this owner took (lane l: its 32 entries, its 16 count words)
    for (uint32_t bits = occ[lane]; bits; bits &= bits - 1) key[lane * 32 + (__ffs(bits) - 1)] = EMPTY;
    if (occ[lane]) {
      for (uint32_t t = 0; t < 16; t++) cnt[lane * 16 + t] = 0;
      occ[lane] = 0;
    }
    __syncwarp();
  }
  if (!MULTI && lane == 0) add_global(a0.acc, gacc);
  __syncthreads();
  if (s_hub) hub_flush(s_hub, a0);
}

// ---------------------------------------------------------------------------
// Block-level flattening of a chunk of neighbours.
__device__ __forceinline__ uint32_t block_find(const uint32_t *s_incl, uint32_t nb, uint32_t wi) {
  uint32_t lo = 0, hi = nb - 1;  // first index with s_incl > wi
  while (lo < hi) {
    uint32_t mid = (lo + hi) >> 1;
    if (s_incl[mid] > wi) hi = mid;
    else lo = mid + 1;
  }
  return lo;
}

// Medium tier: one block per owner, table in (dynamic) shared memory.  Up to
// MB_THREADS neighbours of the owner are loaded at once (one per thread) and
// flattened 32 at a time with warp scans into shared memory; the wedges of
// each 32-neighbour chunk are then dealt out to all warps (wedge wi to thread
// wi mod MB_THREADS), each located with the shuffle search of the light tier,
// MB_BATCH wedges in flight per thread.  With per-vertex or per-edge outputs
// the first pass records each wedge's table position, so the second pass
// reads its group size directly, and an owner with at most MB_THREADS
// neighbours keeps its flattening for the second pass.  The table always has
// MB_CAP entries and is cleared once per block: the endpoint phase and the
// reset visit only the entries the owner used (the wedges that inserted a new
// key are flagged in the recorded positions), so per-owner work scales with
// its wedges, not with the table.
constexpr int MB_BATCH = 4;
constexpr int MB_LG = 13;
static_assert((1 << MB_LG) == MB_CAP, "medium table size");

// Chunk ch of the staged neighbours as seen by one lane: inclusive wedge
// count, wedge count and first slot of the lane's neighbour.
__device__ __forceinline__ void mb_chunk(const uint32_t *s_incl, const uint32_t *s_oy, uint32_t ch, uint32_t lane,
                                         uint32_t &incl, uint32_t &c, uint32_t &oy) {
  incl = s_incl[ch * 32 + lane];
  const uint32_t prev = __shfl_up_sync(FULL, incl, 1);
  c = lane ? incl - prev : incl;
  oy = s_oy[ch * 32 + lane];
}

template <bool PV, bool PE, bool MULTI>
__global__ void __launch_bounds__(MB_THREADS, 3) k_medium(CArgs a0, const uint32_t *__restrict__ list,
                                                       uint32_t nlist, const uint64_t *__restrict__ items,
                                                       const CArgs *__restrict__ tab) {
  // MB_CAP keys, MB_CAP / 2 words of 16-bit counts, then MED_MAX 16-bit table positions
  extern __shared__ uint32_t dsm[];
  uint32_t *key = dsm, *cnt = dsm + MB_CAP;
  uint16_t *pos = reinterpret_cast<uint16_t *>(dsm + MB_CAP + MB_CAP / 2);
  __shared__ unsigned long long s_hubarr[2 * HUBK];
  unsigned long long *s_hub = (PV && !MULTI) ? s_hubarr : nullptr;
  __shared__ uint32_t s_incl[MB_THREADS], s_oy[MB_THREADS];  // per 32-chunk inclusive counts, first slots
  __shared__ unsigned long long s_sum[MB_THREADS];
  __shared__ uint32_t s_item;
  const uint32_t tid = threadIdx.x, lane = lane_id(), w = tid >> 5;
  unsigned long long *err = &a0.acc[ACC_ERR];
  unsigned long long gacc = 0;
  if (PV || PE) s_sum[tid] = 0;
  if (s_hub) hub_zero(s_hub);
  for (uint32_t t = tid; t < MB_CAP; t += MB_THREADS) key[t] = EMPTY;
  for (uint32_t t = tid; t < MB_CAP / 2; t += MB_THREADS) cnt[t] = 0;
  // The next owner is fetched by thread 0 during the previous owner's reset
  // and published by the barrier that ends it.
  if (tid == 0) s_item = static_cast<uint32_t>(atomicAdd(&a0.acc[ACC_QMED], 1ull));
  __syncthreads();
  for (;;) {
    const uint32_t it = s_item;
    if (it >= nlist) break;
    uint32_t x1;
    CArgs a;  // this item's graph
    if (MULTI) {
      const uint64_t item = items[it];
      a = tab[item >> 32];
      x1 = static_cast<uint32_t>(item);
    } else {
      a = a0;
      x1 = list[it];
    }
    const uint64_t wc = a.wpre[x1 + 1] - a.wpre[x1];
    if (wc > MED_MAX) {  // the tier split guarantees wc <= MED_MAX
      __syncthreads();  // every thread has read s_item
      if (tid == 0) {
        atomicOr(err, 16ull);
        s_item = static_cast<uint32_t>(atomicAdd(&a0.acc[ACC_QMED], 1ull));
      }
      __syncthreads();
      continue;
    }
    const uint32_t base = a.off[x1], dp = owner_span(a, x1);
    uint32_t my_y = 0;  // this thread's neighbour in the current group of MB_THREADS
    uint32_t done = 0;  // wedges of the chunks before the current one
    for (uint32_t s0 = 0; s0 < dp; s0 += MB_THREADS) {
      {
        uint32_t c, oy;
        owner_nbr(a, base, s0 + tid, s0 + tid < dp, my_y, c, oy);
        s_incl[tid] = warp_incl_scan(c);
        s_oy[tid] = oy;
      }
      __syncthreads();  // also orders the table reset before the first insert
      const uint32_t left = dp - s0, nch = left >= MB_THREADS ? MB_WARPS : (left + 31) / 32;
      for (uint32_t ch = 0; ch < nch; ch++) {
        uint32_t incl, c, oy;
        mb_chunk(s_incl, s_oy, ch, lane, incl, c, oy);
        const uint32_t tot = __shfl_sync(FULL, incl, 31);
        for (uint32_t wb = 0; wb < tot; wb += MB_BATCH * MB_THREADS) {
          uint32_t x2v[MB_BATCH];
#pragma unroll
          for (int q = 0; q < MB_BATCH; q++) {
            const uint32_t wi = wb + q * MB_THREADS + tid;
            x2v[q] = 0;
            if (wb + q * MB_THREADS + w * 32 < tot) {  // warp-uniform
              uint32_t src, slot;
              warp_locate(incl, c, oy, wi < tot ? wi : tot - 1, src, slot);
              if (wi < tot) x2v[q] = a.adj[slot];
            }
          }
#pragma unroll
          for (int q = 0; q < MB_BATCH; q++) {
            const uint32_t wi = wb + q * MB_THREADS + tid;
            if (wi < tot) pos[done + wi] = static_cast<uint16_t>(sh_add16f(key, cnt, MB_LG, x2v[q], err));
          }
        }
        done += tot;
      }
      __syncthreads();
    }
    const uint32_t nw = done;  // the owner's wedges
    unsigned long long own = 0;
    for (uint32_t j = tid; j < nw; j += MB_THREADS) {
      const uint32_t p = pos[j];
      if (p & 0x8000u) {  // one flagged wedge per distinct second endpoint
        const uint32_t h = p & 0x7fffu;
        unsigned long long d = cnt16_at(cnt, h), b = d * (d - 1) / 2;
        own += b;
        if (PV && b) pv_add(s_hub, a, key[h], b);
      }
    }
    own = warp_sum(own);  // per warp: no block barrier
    if (lane == 0 && own) {
      if (MULTI) add_global(a.acc, own);
      else gacc += own;
      if (PV) atomicAdd(&a.pv[x1], own);
    }
    if (PV || PE) {
      done = 0;
      for (uint32_t s0 = 0; s0 < dp; s0 += MB_THREADS) {
        if (dp > MB_THREADS) {  // otherwise the first pass's flattening is still in place
          uint32_t c, oy;
          owner_nbr(a, base, s0 + tid, s0 + tid < dp, my_y, c, oy);
          s_incl[tid] = warp_incl_scan(c);
          s_oy[tid] = oy;
          __syncthreads();
        }
        const uint32_t left = dp - s0, nch = left >= MB_THREADS ? MB_WARPS : (left + 31) / 32;
        for (uint32_t ch = 0; ch < nch; ch++) {
          uint32_t incl, c, oy;
          mb_chunk(s_incl, s_oy, ch, lane, incl, c, oy);
          const uint32_t tot = __shfl_sync(FULL, incl, 31);
          for (uint32_t wb = 0; wb < tot; wb += MB_BATCH * MB_THREADS) {
#pragma unroll
            for (int q = 0; q < MB_BATCH; q++) {
              const uint32_t wi = wb + q * MB_THREADS + tid;
              if (wb + q * MB_THREADS + w * 32 < tot) {  // warp-uniform
                uint32_t src, slot;
                warp_locate(incl, c, oy, wi < tot ? wi : tot - 1, src, slot);
                unsigned long long t = 0;
                if (wi < tot) {
                  const uint32_t d = cnt16_at(cnt, pos[done + wi] & 0x7fffu);
                  if (d > 1) {
                    t = d - 1;
                    if (PE) atomicAdd(&a.es[slot], t);
                  }
                }
                warp_run_add(s_sum + ch * 32, src, t);
              }
            }
          }
          done += tot;
        }
        __syncthreads();
        if (s0 + tid < dp) {
          unsigned long long sm = s_sum[tid];
          if (sm) {
            if (PV) pv_add(s_hub, a, my_y, sm);
            if (PE) atomicAdd(&a.es[base + s0 + tid], sm);
            s_sum[tid] = 0;
          }
        }
        if (s0 + MB_THREADS < dp) __syncthreads();  // before the next group is staged
      }
    }
    // Reset the entries this owner used.  Entry h is read in the endpoint
    // phase only by the thread of its flagged wedge, the one that resets it;
    // the second pass ended with a barrier.
    for (uint32_t j = tid; j < nw; j += MB_THREADS) {
      const uint32_t p = pos[j];
      if (p & 0x8000u) {
        const uint32_t h = p & 0x7fffu;
        key[h] = EMPTY;
        atomicAnd(&cnt[h >> 1], (h & 1u) ? 0x0000ffffu : 0xffff0000u);
      }
    }
    if (tid == 0) s_item = static_cast<uint32_t>(atomicAdd(&a0.acc[ACC_QMED], 1ull));
    __syncthreads();
  }
  if (!MULTI && lane == 0) add_global(a0.acc, gacc);
  __syncthreads();
  if (s_hub) hub_flush(s_hub, a0);
}

// ---------------------------------------------------------------------------
// Heavy tier, clustered or hashed (k_heavy): one cluster per first endpoint;
// each cluster owns one slot of device-memory scratch.  Used for hubs (a
// cluster of blocks each), for slots shared by a cluster when the scratch
// budget holds fewer slots than there are SMs, for hash tables (HASH) and for
// batches; a dense slot owned by one block uses k_heavy1 below.  The blocks of
// the cluster walk the same neighbour chunks and take equal shares of every
// chunk's wedges; inside a block consecutive threads take consecutive wedges
// and every thread keeps HB_BATCH of them in flight.  Phases are separated by
// cluster barriers (release/acquire at cluster scope); scratch written by
// other blocks is read through L2 (ld.global.cg).
// Dense slots are indexed by the second endpoint's offset within its side.
constexpr int HB_BATCH = 4;
// Shared-memory histogram of the first labels of a side: with the cache
// optimisation the second endpoints are the lower-ranked ones, so nearly all
// of a heavy owner's wedges land there (the highest-degree vertices).
constexpr uint32_t HB_HOT = 16384;

struct HeavySlots {
  uint32_t *A;        // dense: [nslots][side] counts (all zero between uses)
  uint32_t *T;        // dense: [nslots][tcap] touched second endpoints
  uint32_t *hkey;     // hash:  [nslots][hcap] keys (EMPTY between uses)
  uint32_t *hval;     // hash:  [nslots][hcap] counts
  uint32_t *tcnt;     // [nslots][2] touched counters (alternating)
  uint32_t *item;     // [nslots] current work item of the slot
  uint64_t side, tcap, hcap;
  uint32_t hot;       // k_heavy1: labels [0, hot) of the side counted in shared memory
};

// Appends second endpoints seen for the first time to the touched list
// (warp-aggregated: one counter atomic per warp).
__device__ __forceinline__ void dense_touch(const HeavySlots &h, uint32_t *T, uint32_t *tc, uint32_t x2, bool isnew,
                                            unsigned long long *err) {
  uint32_t bm = __ballot_sync(FULL, isnew);
  if (bm) {
    uint32_t leader = __ffs(bm) - 1, b0 = 0;
    if (lane_id() == leader) b0 = atomicAdd(tc, static_cast<uint32_t>(__popc(bm)));
    b0 = __shfl_sync(FULL, b0, leader);
    if (isnew) {
      uint32_t pos = b0 + __popc(bm & lanemask_lt());
      if (pos < h.tcap) T[pos] = x2;
      else atomicOr(err, 16ull);
    }
  }
}

template <bool DENSE>
__device__ __forceinline__ void heavy_insert(const HeavySlots &h, uint32_t slot, uint32_t *A, uint32_t *T,
                                             uint32_t *tc, int lg, uint32_t x2, uint32_t base, bool act,
                                             unsigned long long *err) {
  if (DENSE) {
    bool isnew = false;
    if (act) isnew = atomicAdd(&A[x2 - base], 1u) == 0u;
    uint32_t bm = __ballot_sync(FULL, isnew);
    if (bm) {
      uint32_t leader = __ffs(bm) - 1, b0 = 0;
      if (lane_id() == leader) b0 = atomicAdd(tc, static_cast<uint32_t>(__popc(bm)));
      b0 = __shfl_sync(FULL, b0, leader);
      if (isnew) {
        uint32_t pos = b0 + __popc(bm & lanemask_lt());
        if (pos < h.tcap) T[pos] = x2;
        else atomicOr(err, 16ull);
      }
    }
  } else if (act) {
    uint32_t *key = h.hkey + static_cast<size_t>(slot) * h.hcap;
    uint32_t *val = h.hval + static_cast<size_t>(slot) * h.hcap;
    const uint32_t mask = (1u << lg) - 1;
    uint32_t p = hash_home(x2, lg);
    for (uint32_t probe = 0;; probe++) {
      if (probe > mask) { atomicOr(err, 4ull); return; }
      uint32_t k = __ldcg(&key[p]);
      if (k == EMPTY) k = atomicCAS(&key[p], EMPTY, x2);
      if (k == EMPTY || k == x2) break;
      p = (p + 1) & mask;
    }
    atomicAdd(&val[p], 1u);
  }
}

template <bool DENSE>
__device__ __forceinline__ uint32_t heavy_get(const HeavySlots &h, uint32_t slot, const uint32_t *A, int lg,
                                              uint32_t x2, uint32_t base, unsigned long long *err) {
  if (DENSE) return __ldcg(&A[x2 - base]);
  const uint32_t *key = h.hkey + static_cast<size_t>(slot) * h.hcap;
  const uint32_t *val = h.hval + static_cast<size_t>(slot) * h.hcap;
  const uint32_t mask = (1u << lg) - 1;
  uint32_t p = hash_home(x2, lg);
  for (uint32_t probe = 0; __ldcg(&key[p]) != x2; probe++) {
    if (probe > mask) { atomicOr(err, 8ull); return 0; }
    p = (p + 1) & mask;
  }
  return __ldcg(&val[p]);
}

template <bool PV, bool PE, bool DENSE, bool MULTI>
__global__ void __launch_bounds__(HB_THREADS) k_heavy(CArgs a0, const uint32_t *__restrict__ list,
                                                      uint32_t nlist, HeavySlots h, const uint64_t *__restrict__ items,
                                                      const CArgs *__restrict__ tab) {
  cg::cluster_group cl = cg::this_cluster();
  const uint32_t crank = cl.block_rank(), csize = cl.num_blocks();
  const uint32_t slot = blockIdx.x / csize;
  const uint32_t tid = threadIdx.x;
  __shared__ uint32_t s_incl[HB_THREADS], s_ex[HB_THREADS], s_oy[HB_THREADS];
  __shared__ uint8_t s_nar[HB_THREADS];  // the neighbour's list takes 32-bit edge partials
  __shared__ unsigned long long s_sum[HB_THREADS];
  __shared__ uint32_t s_w[33];
  __shared__ unsigned long long s_w64[33];
  __shared__ unsigned long long s_hubarr[2 * HUBK];
  unsigned long long *s_hub = (PV && !MULTI) ? s_hubarr : nullptr;
  uint32_t *A = DENSE ? h.A + static_cast<size_t>(slot) * h.side : nullptr;
  uint32_t *T = DENSE ? h.T + static_cast<size_t>(slot) * h.tcap : nullptr;
  unsigned long long *err = &a0.acc[ACC_ERR];
  unsigned long long gacc = 0;
  if (PV || PE) s_sum[tid] = 0;
  if (s_hub) hub_zero(s_hub);
  for (uint32_t k = 0;; k++) {
    if (crank == 0 && tid == 0) h.item[slot] = static_cast<uint32_t>(atomicAdd(&a0.acc[ACC_QHEAVY], 1ull));
    cl.sync();
    const uint32_t it = __ldcg(&h.item[slot]);
    if (it >= nlist) break;
    uint32_t *tc = &h.tcnt[2 * slot + (k & 1)];
    if (crank == 0 && tid == 0) h.tcnt[2 * slot + ((k + 1) & 1)] = 0;
    uint32_t x1;
    CArgs a;  // this item's graph
    if (MULTI) {
      const uint64_t item = items[it];
      a = tab[item >> 32];
      x1 = static_cast<uint32_t>(item);
    } else {
      a = a0;
      x1 = list[it];
    }
    const uint32_t base = dense_base(a, x1);  // label of histogram entry 0
    const uint64_t wc = a.wpre[x1 + 1] - a.wpre[x1];
    const int lg = DENSE ? 0 : table_lg(wc, a.n, a.nU, x1, a.rev);
    const uint32_t xbase = a.off[x1], dp = owner_span(a, x1);
    // ---- aggregate
    for (uint32_t k0 = 0; k0 < dp; k0 += HB_THREADS) {
      const uint32_t i = k0 + tid;
      const bool v = i < dp;
      uint32_t y, c, oy;
      owner_nbr(a, xbase, i, v, y, c, oy);
      uint32_t tot;
      const uint32_t incl = block_incl_scan(c, s_w, &tot);
      s_incl[tid] = incl;
      s_ex[tid] = incl - c;
      s_oy[tid] = oy;
      __syncthreads();
      const uint32_t lo = static_cast<uint32_t>(static_cast<uint64_t>(tot) * crank / csize);
      const uint32_t hi = static_cast<uint32_t>(static_cast<uint64_t>(tot) * (crank + 1) / csize);
      // interleaved: consecutive threads take consecutive wedges (coalesced
      // adjacency reads); HB_BATCH wedges per thread are in flight at once
      for (uint32_t wb = lo; wb < hi; wb += HB_BATCH * HB_THREADS) {
        uint32_t x2v[HB_BATCH];
#pragma unroll
        for (int q = 0; q < HB_BATCH; q++) {
          const uint32_t wi = wb + q * HB_THREADS + tid;
          x2v[q] = 0;
          if (wi < hi) {
            const uint32_t src = block_find(s_incl, HB_THREADS, wi);
            x2v[q] = a.adj[s_oy[src] + (wi - s_ex[src])];
          }
        }
        if (DENSE) {
          // issue every atomic of the batch before any result is used
          uint32_t old[HB_BATCH];
#pragma unroll
          for (int q = 0; q < HB_BATCH; q++)
            old[q] = wb + q * HB_THREADS + tid < hi ? atomicAdd(&A[x2v[q] - base], 1u) : 1u;
#pragma unroll
          for (int q = 0; q < HB_BATCH; q++) dense_touch(h, T, tc, x2v[q], old[q] == 0u, err);
        } else {
#pragma unroll
          for (int q = 0; q < HB_BATCH; q++)
            heavy_insert<DENSE>(h, slot, A, T, tc, lg, x2v[q], base, wb + q * HB_THREADS + tid < hi, err);
        }
      }
      __syncthreads();
    }
    cl.sync();
    // ---- endpoints: C(d, 2) per distinct second endpoint
    unsigned long long own = 0;
    if (DENSE) {
      const uint32_t nt = __ldcg(tc);
      for (uint32_t t = crank * HB_THREADS + tid; t < nt; t += csize * HB_THREADS) {
        uint32_t x2 = __ldcg(&T[t]);
        unsigned long long d = __ldcg(&A[x2 - base]), b = d * (d - 1) / 2;
        own += b;
        if (PV && b) pv_add(s_hub, a, x2, b);
      }
    } else {
      const uint32_t *key = h.hkey + static_cast<size_t>(slot) * h.hcap;
      const uint32_t *val = h.hval + static_cast<size_t>(slot) * h.hcap;
      const uint32_t cap = 1u << lg;
      for (uint32_t t = crank * HB_THREADS + tid; t < cap; t += csize * HB_THREADS) {
        uint32_t kk = __ldcg(&key[t]);
        if (kk != EMPTY) {
          unsigned long long d = __ldcg(&val[t]), b = d * (d - 1) / 2;
          own += b;
          if (PV && b) pv_add(s_hub, a, kk, b);
        }
      }
    }
    own = block_sum(own, s_w64);
    if (tid == 0) {
      if (MULTI) add_global(a.acc, own);
      else gacc += own;
      if (PV && own) atomicAdd(&a.pv[x1], own);
    }
    // ---- centres and edges
    if (PV || PE) {
      for (uint32_t k0 = 0; k0 < dp; k0 += HB_THREADS) {
        const uint32_t i = k0 + tid;
        const bool v = i < dp;
        uint32_t y, c, oy;
        owner_nbr(a, xbase, i, v, y, c, oy);
        if (PE) s_nar[tid] = v && es_narrow(a, x1, a.off[y + 1] - a.off[y]);
        uint32_t tot;
        const uint32_t incl = block_incl_scan(c, s_w, &tot);
        s_incl[tid] = incl;
        s_ex[tid] = incl - c;
        s_oy[tid] = oy;
        __syncthreads();
        const uint32_t lo = static_cast<uint32_t>(static_cast<uint64_t>(tot) * crank / csize);
        const uint32_t hi = static_cast<uint32_t>(static_cast<uint64_t>(tot) * (crank + 1) / csize);
        for (uint32_t wb = lo; wb < hi; wb += HB_BATCH * HB_THREADS) {
          uint32_t x2v[HB_BATCH], slv[HB_BATCH], srcv[HB_BATCH], dv[HB_BATCH];
#pragma unroll
          for (int q = 0; q < HB_BATCH; q++) {
            const uint32_t wi = wb + q * HB_THREADS + tid;
            x2v[q] = 0;
            srcv[q] = 0;
            slv[q] = 0;
            if (wi < hi) {
              srcv[q] = block_find(s_incl, HB_THREADS, wi);
              slv[q] = s_oy[srcv[q]] + (wi - s_ex[srcv[q]]);
              x2v[q] = a.adj[slv[q]];
            }
          }
#pragma unroll
          for (int q = 0; q < HB_BATCH; q++)
            dv[q] = wb + q * HB_THREADS + tid < hi ? heavy_get<DENSE>(h, slot, A, lg, x2v[q], base, err) : 0;
#pragma unroll
          for (int q = 0; q < HB_BATCH; q++) {
            unsigned long long t = dv[q] > 1 ? dv[q] - 1 : 0;
            if (PE && t) es_add_wedge(a, slv[q], static_cast<uint32_t>(t), s_nar[srcv[q]]);
            warp_run_add(s_sum, srcv[q], t);
          }
        }
        __syncthreads();
        if (v) {
          unsigned long long sm = s_sum[tid];
          if (sm) {
            if (PV) pv_add(s_hub, a, y, sm);
            if (PE) atomicAdd(&a.es[xbase + i], sm);
            s_sum[tid] = 0;
          }
        }
        __syncthreads();
      }
    }
    cl.sync();
    // ---- restore the slot to all-zero / all-empty
    if (DENSE) {
      const uint32_t nt = __ldcg(tc);
      for (uint32_t t = crank * HB_THREADS + tid; t < nt; t += csize * HB_THREADS) A[__ldcg(&T[t]) - base] = 0;
    } else {
      uint32_t *key = h.hkey + static_cast<size_t>(slot) * h.hcap;
      uint32_t *val = h.hval + static_cast<size_t>(slot) * h.hcap;
      const uint32_t cap = 1u << lg;
      for (uint32_t t = crank * HB_THREADS + tid; t < cap; t += csize * HB_THREADS) {
        key[t] = EMPTY;
        val[t] = 0;
      }
    }
  }
  if (!MULTI && tid == 0) add_global(a0.acc, gacc);
  __syncthreads();
  if (s_hub) hub_flush(s_hub, a0);
}

// ---------------------------------------------------------------------------
// Heavy tier, one block per owner and slot (no cluster): the owner's
// neighbours are staged HB_THREADS at a time, and each warp takes whole
// neighbours from a shared counter and walks the neighbour's segment of
// second endpoints with its lanes (coalesced adjacency reads).  Counts of the
// first h.hot labels of the side live in shared memory; the rest ("cold"
// second endpoints) live in the slot's device memory, either as a dense
// histogram over the owner's label range (HCOLD = false) or as an
// open-addressing hash table sized by the owner's bound on distinct second
// endpoints (HCOLD = true, a few times smaller, so that more slots fit a
// scratch budget).  A touched list (device memory, counter in shared memory)
// records each distinct second endpoint once: its label (dense) or its hot
// offset / table position with the top bit set (hashed).  The second pass sums
// d - 1 over a segment in registers and adds it to the centre once.
constexpr uint32_t TCOLD = 0x80000000u;  // touched-list tag of a hash-table position

// Inserts cold second endpoint x2 into the slot's hash table; returns its
// position and whether it was new.
__device__ __forceinline__ uint32_t cold_insert(uint32_t *key, uint32_t *val, int lg, uint32_t x2, bool &isnew,
                                                unsigned long long *err) {
  const uint32_t mask = (1u << lg) - 1;
  uint32_t p = hash_home(x2, lg);
  for (uint32_t probe = 0;; probe++) {
    if (probe > mask) { atomicOr(err, 4ull); isnew = false; return TCOLD - 1; }
    uint32_t k = __ldcg(&key[p]);
    if (k == EMPTY) k = atomicCAS(&key[p], EMPTY, x2);
    if (k == EMPTY || k == x2) break;
    p = (p + 1) & mask;
  }
  isnew = atomicAdd(&val[p], 1u) == 0u;
  return p;
}

__device__ __forceinline__ uint32_t cold_get(const uint32_t *key, const uint32_t *val, int lg, uint32_t x2,
                                             unsigned long long *err) {
  const uint32_t mask = (1u << lg) - 1;
  uint32_t p = hash_home(x2, lg);
  for (uint32_t probe = 0; __ldcg(&key[p]) != x2; probe++) {
    if (probe > mask) { atomicOr(err, 8ull); return 0; }
    p = (p + 1) & mask;
  }
  return __ldcg(&val[p]);
}

// Shared-memory hot counts: 32-bit, or 16-bit two to a word for owners whose
// wedge count (and so every group size) is below 2^16.
template <bool HOT16>
__device__ __forceinline__ bool hot_inc(uint32_t *hot, uint32_t r) {
  if (HOT16) {
    const uint32_t sh = (r & 1u) << 4;
    return ((atomicAdd(&hot[r >> 1], 1u << sh) >> sh) & 0xffffu) == 0u;
  }
  return atomicAdd(&hot[r], 1u) == 0u;
}
template <bool HOT16>
__device__ __forceinline__ uint32_t hot_get(const uint32_t *hot, uint32_t r) {
  if (HOT16) return (hot[r >> 1] >> ((r & 1u) << 4)) & 0xffffu;
  return hot[r];
}
template <bool HOT16>
__device__ __forceinline__ void hot_clear(uint32_t *hot, uint32_t r) {
  // Only this entry's half: the other half of the word may belong to an entry
  // another thread is still reading (with global counts alone, no barrier
  // separates the endpoint phase from the reset).
  if (HOT16) atomicAnd(&hot[r >> 1], (r & 1u) ? 0x0000ffffu : 0xffff0000u);
  else hot[r] = 0;
}
__host__ __device__ constexpr uint32_t hot_words(uint32_t hot, bool hot16) { return hot16 ? (hot + 1) / 2 : hot; }
// Count without the first-occurrence test (owners whose hot range is read
// whole afterwards).
template <bool HOT16>
__device__ __forceinline__ void hot_add(uint32_t *hot, uint32_t r) {
  if (HOT16) atomicAdd(&hot[r >> 1], 1u << ((r & 1u) << 4));
  else atomicAdd(&hot[r], 1u);
}

// Owners with at least hot_words / HOT_SCAN_DIV wedges keep no record of
// which hot labels they touched: after counting, the block reads the whole hot
// range (four words per thread and load) for the endpoint sums, and clears it
// after the centre pass.  Below that the touched list is cheaper than the read
// (the record costs a vote and a compare per wedge, the read a fixed few
// instructions per hot word).
constexpr uint32_t HOT_SCAN_DIV = 4;

// C(d, 2) of the counts in hot word w (one count, or two 16-bit ones), with
// the per-vertex contribution of each second endpoint base + entry.
template <bool PV, bool HOT16>
__device__ __forceinline__ unsigned long long hot_word_sum(uint32_t v, uint32_t w, uint32_t base,
                                                           unsigned long long *s_hub, const CArgs &a) {
  if (!v) return 0;
  unsigned long long s = 0;
#pragma unroll
  for (int k = 0; k < (HOT16 ? 2 : 1); k++) {
    const unsigned long long d = HOT16 ? (v >> (16 * k)) & 0xffffu : v;
    const unsigned long long b = d * (d - 1) / 2;
    s += b;
    if (PV && b) pv_add(s_hub, a, base + (HOT16 ? 2 * w + k : w), b);
  }
  return s;
}

// Work unit of the one-block kernels: a neighbour's whole segment of second
// endpoints, or -- when some staged segment is longer than twice the owner's
// chunk size -- up to that many consecutive endpoints of one segment, so that
// an owner whose wedges sit in a few long segments (through hub centres)
// spreads them over all its warps.  The chunk size is the owner's wedges per
// warp, rounded up to a power of two, at least SEG_CHUNK.
constexpr uint32_t SEG_CHUNK = 256;
// Adjacency loads per lane in flight in a segment walk (20M x 60M heavy tier:
// 823 ms with one, 668 with two, 623 with four), per block size.
constexpr int OWNER_ILP_HEAVY = 4, OWNER_ILP_LARGE = 4;
__host__ __device__ constexpr int owner_ilp(int nt) { return nt >= 1024 ? OWNER_ILP_HEAVY : OWNER_ILP_LARGE; }

// Chunk j of the staged neighbours: the neighbour k it belongs to (first k
// with ck[k] > j), the end c of the chunk's range in that segment (its
// length, capped at the chunk end), the segment's first slot oy and the
// chunk's first position e_lo.
template <int NT>
__device__ __forceinline__ uint32_t seg_chunk(const uint32_t *ck, const uint32_t *cs, const uint32_t *oys, uint32_t j,
                                              uint32_t ch, uint32_t &c, uint32_t &oy, uint32_t &e_lo) {
  uint32_t lo = 0, hi = NT - 1;
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if (ck[mid] > j) hi = mid;
    else lo = mid + 1;
  }
  const uint32_t len = cs[lo];
  const uint32_t first = ck[lo] - (len + ch - 1) / ch;  // the neighbour's first chunk
  e_lo = (j - first) * ch;
  c = e_lo + ch < len ? e_lo + ch : len;
  oy = oys[lo];
  return lo;
}

// The next work unit of a warp: chunk j of the staged neighbours when the
// segments are split (split != 0), else the whole segment of neighbour j.
// Returns the neighbour, or NT when the staged work is done.
template <int NT>
__device__ __forceinline__ uint32_t next_unit(uint32_t *s_next, const uint32_t *ck, const uint32_t *cs,
                                              const uint32_t *oys, int split, uint32_t units, uint32_t ch,
                                              uint32_t &c, uint32_t &oy, uint32_t &e_lo) {
  uint32_t j = 0;
  if (lane_id() == 0) j = atomicAdd(s_next, 1u);
  j = __shfl_sync(FULL, j, 0);
  if (j >= units) return NT;
  if (split) return seg_chunk<NT>(ck, cs, oys, j, ch, c, oy, e_lo);
  c = cs[j];
  oy = oys[j];
  e_lo = 0;
  return j;
}

// Counting walk of one work unit (positions [e_lo, c) of the segment at oy)
// for owners that read their hot range whole: no first-occurrence record for
// hot labels, so lanes walk independently; a cold label seen for the first
// time is appended to the touched list with its own shared-memory add (cold
// labels are a small share of the wedges).
template <bool HOT16, bool HCOLD, int ILP>
__device__ __forceinline__ void owner_count_scan(const CArgs &a, uint32_t *hb_hot, const HeavySlots &h, uint32_t *A,
                                                 uint32_t *hkey, uint32_t *hval, uint32_t *T, uint32_t *s_nt, int lg,
                                                 uint32_t base, uint32_t oy, uint32_t e_lo, uint32_t c,
                                                 unsigned long long *err) {
  for (uint32_t e0 = e_lo + lane_id(); e0 < c; e0 += 32 * ILP) {
    uint32_t x2v[ILP];
#pragma unroll
    for (int q = 0; q < ILP; q++) x2v[q] = e0 + 32 * q < c ? a.adj[oy + e0 + 32 * q] : 0u;
#pragma unroll
    for (int q = 0; q < ILP; q++) {
      if (e0 + 32 * q >= c) break;
      const uint32_t x2 = x2v[q], r = x2 - base;
      if (r < h.hot) {
        hot_add<HOT16>(hb_hot, r);
        continue;
      }
      bool isnew;
      uint32_t tag;
      if (HCOLD) {
        tag = TCOLD | cold_insert(hkey, hval, lg, x2, isnew, err);
      } else {
        isnew = atomicAdd(&A[r], 1u) == 0u;
        tag = x2;
      }
      if (isnew) {
        const uint32_t at = atomicAdd(s_nt, 1u);
        if (at < h.tcap) T[at] = tag;
        else atomicOr(err, 16ull);
      }
    }
  }
}

// Centre walk of one work unit: the count d of every wedge's second endpoint,
// d - 1 added to the wedge's edge slot (32-bit partials when NARROW) and
// summed for the centre.  Returns this lane's sum.  With 16-bit hot counts
// every owner has fewer than 2^16 wedges, so a 32-bit sum cannot wrap.
template <bool PE, bool HOT16, bool HCOLD, bool NARROW, int ILP>
__device__ __forceinline__ unsigned long long owner_centre_walk(const CArgs &a, const uint32_t *hb_hot,
                                                                const HeavySlots &h, const uint32_t *A,
                                                                const uint32_t *hkey, const uint32_t *hval, int lg,
                                                                uint32_t base, uint32_t oy, uint32_t e_lo, uint32_t c,
                                                                unsigned long long *err) {
  using S = typename std::conditional<HOT16, uint32_t, unsigned long long>::type;
  S sum = 0;
  for (uint32_t e0 = e_lo + lane_id(); e0 < c; e0 += 32 * ILP) {
    uint32_t x2v[ILP];
#pragma unroll
    for (int q = 0; q < ILP; q++) x2v[q] = e0 + 32 * q < c ? a.adj[oy + e0 + 32 * q] : 0u;
#pragma unroll
    for (int q = 0; q < ILP; q++) {
      const uint32_t e = e0 + 32 * q;
      if (e >= c) break;
      const uint32_t x2 = x2v[q], r = x2 - base;
      uint32_t d;
      if (r < h.hot) d = hot_get<HOT16>(hb_hot, r);
      else if (HCOLD) d = cold_get(hkey, hval, lg, x2, err);
      else d = __ldcg(&A[r]);
      if (d > 1) {
        sum += d - 1;
        if (PE) {
          if (NARROW) atomicAdd(&a.es32[oy + e], d - 1);
          else atomicAdd(&a.es[oy + e], static_cast<unsigned long long>(d - 1));
        }
      }
    }
  }
  return warp_sum(sum);
}

// One block of NT threads per owner and slot: the heavy tier (NT = 1024,
// 32-bit hot counts, cold part dense or hashed) and the medium tier (NT =
// 256, 16-bit hot counts, cold part hashed).  The owner's neighbours are
// staged NT at a time, and each warp takes whole neighbours from a shared
// counter and walks the neighbour's segment of second endpoints with its
// lanes (coalesced adjacency reads).  Counts of the first h.hot labels of the
// side live in shared memory; the rest ("cold" second endpoints) live in the
// slot's device memory, either as a dense histogram over the owner's label
// range (HCOLD = false) or as an open-addressing hash table sized by the
// owner's bound on distinct second endpoints (HCOLD = true).  A touched list
// (device memory, counter in shared memory) records each distinct second
// endpoint once: its label (dense) or its hot offset / table position with
// the top bit set (hashed).  The second pass sums d - 1 over a segment in
// registers and adds it to the centre once.  Owners come from the work queue
// acc[QUEUE].
// Block sizes of the one-block owner kernels: the heavy tier's (32-bit hot
// counts of the plan's hot range) and the large tier's (16-bit counts of
// MH_HOT labels).  Owners are latency-bound (a chain of dependent loads to
// stage the neighbours, block barriers between passes), so the large tier is
// sized for a full SM: eight 256-thread blocks, whose 16 KB of hot counts fit
// eight to an SM (20M x 60M large tier: 413 ms with 16,384 labels and six
// blocks per SM, 324 ms with 8,192 and eight; 128-thread blocks with 8,192
// labels, 331 ms; 64-thread blocks, 385 ms).
constexpr int H1_THREADS = HB_THREADS;
constexpr int MH_THREADS = 256;
constexpr uint32_t MH_HOT = 8192;  // large tier: labels counted in shared memory (16-bit)
constexpr int owner_min_blocks(int nt) { return 2048 / nt; }

template <bool PV, bool PE, bool MULTI, bool HCOLD, int NT, bool HOT16, int QUEUE>
__global__ void __launch_bounds__(NT, owner_min_blocks(NT)) k_owner(CArgs a0, const uint32_t *__restrict__ list, uint32_t nlist,
                                              HeavySlots h, const uint64_t *__restrict__ items,
                                              const CArgs *__restrict__ tab) {
  extern __shared__ __align__(16) uint32_t hb_hot[];
  __shared__ uint32_t s_c[NT], s_oy[NT], s_y[NT];
  __shared__ uint32_t s_ck[NT];  // inclusive prefix of the staged neighbours' chunk counts
  __shared__ uint32_t s_w[33];
  __shared__ uint8_t s_nar[NT];  // the neighbour's list takes 32-bit edge partials
  __shared__ unsigned long long s_hubarr[(PV && !MULTI) ? 2 * HUBK : 1];
  __shared__ uint32_t s_item, s_next, s_nt;
  unsigned long long *s_hub = (PV && !MULTI) ? s_hubarr : nullptr;
  const uint32_t slot = blockIdx.x, tid = threadIdx.x, lane = lane_id();
  uint32_t *A = HCOLD ? nullptr : h.A + static_cast<size_t>(slot) * h.side;
  uint32_t *hkey = HCOLD ? h.hkey + static_cast<size_t>(slot) * h.hcap : nullptr;
  uint32_t *hval = HCOLD ? h.hval + static_cast<size_t>(slot) * h.hcap : nullptr;
  uint32_t *T = h.T + static_cast<size_t>(slot) * h.tcap;
  unsigned long long *err = &a0.acc[ACC_ERR];
  unsigned long long gacc = 0;
  constexpr int ILP = owner_ilp(NT);
  const uint32_t hw = hot_words(h.hot, HOT16), hw4 = hw & ~3u;
  if (s_hub) hub_zero(s_hub);
  for (uint32_t t = tid; t < hw; t += NT) hb_hot[t] = 0;
  // The next owner is fetched by thread 0 during the previous owner's reset
  // and published by the barrier that ends it (one barrier between owners).
  if (tid == 0) s_item = static_cast<uint32_t>(atomicAdd(&a0.acc[QUEUE], 1ull));
  __syncthreads();
  for (;;) {
    const uint32_t it = s_item;
    if (it >= nlist) break;
    if (tid == 0) s_nt = 0;  // every thread read the previous count before the last barrier
    uint32_t x1;
    CArgs a;  // this item's graph
    if (MULTI) {
      const uint64_t item = items[it];
      a = tab[item >> 32];
      x1 = static_cast<uint32_t>(item);
    } else {
      a = a0;
      x1 = list[it];
    }
    const uint32_t base = dense_base(a, x1);  // label of histogram entry 0
    const uint32_t xbase = a.off[x1], dp = owner_span(a, x1);
    const uint64_t wc = a.wpre[x1 + 1] - a.wpre[x1];
    if (HOT16 && wc > 0xffffu) {  // the tier split guarantees 16-bit counts suffice
      __syncthreads();            // every thread has read s_item
      if (tid == 0) {
        atomicOr(err, 16ull);
        s_item = static_cast<uint32_t>(atomicAdd(&a0.acc[QUEUE], 1ull));
      }
      __syncthreads();
      continue;
    }
    const int lg = HCOLD ? table_lg(wc, a.n, a.nU, x1, a.rev) : 0;
    // hot labels go unrecorded and the hot range is read whole (block-uniform)
    const bool scan = wc * HOT_SCAN_DIV >= hw;
    // ---- aggregate
    uint32_t ch = SEG_CHUNK;
    while (static_cast<uint64_t>(ch) * (NT / 32) < wc) ch <<= 1;
    uint32_t units = 0;  // work units of the staged neighbours
    int split = 0;       // some staged segment is longer than a chunk
    for (uint32_t s0 = 0; s0 < dp; s0 += NT) {
      {
        uint32_t y, c, oy;
        const bool v = s0 + tid < dp;
        owner_nbr(a, xbase, s0 + tid, v, y, c, oy);
        s_c[tid] = c;
        s_oy[tid] = oy;
        s_y[tid] = y;
        if (PE && dp <= NT) s_nar[tid] = v && es_narrow(a, x1, a.off[y + 1] - a.off[y]);
        if (tid == 0) s_next = 0;
        split = __syncthreads_or(c > 2 * ch);
        if (split) s_ck[tid] = block_incl_scan((c + ch - 1) / ch, s_w, &units);  // barriers inside
        else units = dp - s0 < NT ? dp - s0 : NT;
      }
      __syncthreads();
      for (;;) {
        uint32_t c, oy, e_lo;
        if (next_unit<NT>(&s_next, s_ck, s_c, s_oy, split, units, ch, c, oy, e_lo) == NT) break;
        if (scan) {
          owner_count_scan<HOT16, HCOLD, ILP>(a, hb_hot, h, A, hkey, hval, T, &s_nt, lg, base, oy, e_lo, c, err);
          continue;
        }
        // ILP adjacency loads per lane in flight before their counts
        for (uint32_t e0 = e_lo; e0 < c; e0 += 32 * ILP) {
          uint32_t x2v[ILP];
#pragma unroll
          for (int q = 0; q < ILP; q++) {
            const uint32_t e = e0 + 32 * q + lane;
            x2v[q] = e < c ? a.adj[oy + e] : 0u;
          }
#pragma unroll
          for (int q = 0; q < ILP; q++) {
            if (e0 + 32 * q >= c) break;  // warp-uniform
            const bool act = e0 + 32 * q + lane < c;
            uint32_t tag = 0;
            bool isnew = false;
            if (act) {
              const uint32_t x2 = x2v[q];
              const uint32_t r = x2 - base;
              if (r < h.hot) {
                isnew = hot_inc<HOT16>(hb_hot, r);
                tag = HCOLD ? r : x2;
              } else if (HCOLD) {
                tag = TCOLD | cold_insert(hkey, hval, lg, x2, isnew, err);
              } else {
                isnew = atomicAdd(&A[r], 1u) == 0u;
                tag = x2;
              }
            }
            const uint32_t bm = __ballot_sync(FULL, isnew);
            if (bm) {
              uint32_t b0 = 0;
              if (lane == 0) b0 = atomicAdd(&s_nt, static_cast<uint32_t>(__popc(bm)));
              b0 = __shfl_sync(FULL, b0, 0);
              if (isnew) {
                const uint32_t at = b0 + __popc(bm & lanemask_lt());
                if (at < h.tcap) T[at] = tag;
                else atomicOr(err, 16ull);
              }
            }
          }
        }
      }
      __syncthreads();
    }
    const uint32_t nt = s_nt < h.tcap ? s_nt : static_cast<uint32_t>(h.tcap);
    // ---- endpoints: C(d, 2) per distinct second endpoint
    unsigned long long own = 0;
    if (scan) {  // the hot range whole; with global counts alone it is cleared on the way
      for (uint32_t w = 4 * tid; w < hw4; w += 4 * NT) {
        uint4 &q4 = *reinterpret_cast<uint4 *>(&hb_hot[w]);
        const uint4 v4 = q4;
        if ((v4.x | v4.y | v4.z | v4.w) == 0u) continue;  // most quads of a smaller owner are empty
        if (!PV && !PE) q4 = make_uint4(0u, 0u, 0u, 0u);
        own += hot_word_sum<PV, HOT16>(v4.x, w, base, s_hub, a) + hot_word_sum<PV, HOT16>(v4.y, w + 1, base, s_hub, a) +
               hot_word_sum<PV, HOT16>(v4.z, w + 2, base, s_hub, a) + hot_word_sum<PV, HOT16>(v4.w, w + 3, base, s_hub, a);
      }
      for (uint32_t w = hw4 + tid; w < hw; w += NT) {
        own += hot_word_sum<PV, HOT16>(hb_hot[w], w, base, s_hub, a);
        if (!PV && !PE) hb_hot[w] = 0;
      }
    }
    for (uint32_t t = tid; t < nt; t += NT) {  // recorded labels (cold ones only when scanning)
      const uint32_t v = T[t];
      uint32_t x2;
      unsigned long long d;
      if (HCOLD) {
        if (v & TCOLD) {
          const uint32_t p = v & ~TCOLD;
          x2 = __ldcg(&hkey[p]);
          d = __ldcg(&hval[p]);
        } else {
          x2 = base + v;
          d = hot_get<HOT16>(hb_hot, v);
        }
      } else {
        x2 = v;
        const uint32_t r = x2 - base;
        d = r < h.hot ? hot_get<HOT16>(hb_hot, r) : __ldcg(&A[r]);
      }
      const unsigned long long b = d * (d - 1) / 2;
      own += b;
      if (PV && b) pv_add(s_hub, a, x2, b);
    }
    own = warp_sum(own);  // per warp: no block barrier
    if (lane == 0 && own) {
      if (MULTI) add_global(a.acc, own);
      else gacc += own;
      if (PV) atomicAdd(&a.pv[x1], own);
    }
    // ---- centres and edges: d - 1 per wedge
    if (PV || PE) {
      for (uint32_t s0 = 0; s0 < dp; s0 += NT) {
        if (tid == 0) s_next = 0;
        if (dp > NT) {  // otherwise the first pass's staging is still in place
          uint32_t y, c, oy;
          const bool v = s0 + tid < dp;
          owner_nbr(a, xbase, s0 + tid, v, y, c, oy);
          if (PE) s_nar[tid] = v && es_narrow(a, x1, a.off[y + 1] - a.off[y]);
          s_c[tid] = c;
          s_oy[tid] = oy;
          s_y[tid] = y;
          split = __syncthreads_or(c > 2 * ch);
          if (split) s_ck[tid] = block_incl_scan((c + ch - 1) / ch, s_w, &units);  // barriers inside
          else units = dp - s0 < NT ? dp - s0 : NT;
        }
        __syncthreads();
        for (;;) {
          uint32_t c, oy, e_lo;
          const uint32_t k = next_unit<NT>(&s_next, s_ck, s_c, s_oy, split, units, ch, c, oy, e_lo);
          if (k == NT) break;
          const unsigned long long sum =
              (PE && s_nar[k]) ? owner_centre_walk<PE, HOT16, HCOLD, true, ILP>(a, hb_hot, h, A, hkey, hval, lg, base, oy, e_lo, c, err)
                               : owner_centre_walk<PE, HOT16, HCOLD, false, ILP>(a, hb_hot, h, A, hkey, hval, lg, base, oy, e_lo, c, err);
          if (lane == 0 && sum) {
            if (PV) pv_add(s_hub, a, s_y[k], sum);
            if (PE) atomicAdd(&a.es[xbase + s0 + k], sum);
          }
        }
        __syncthreads();
      }
    }
    // ---- reset the slot's used entries (every thread has passed the first
    // pass's staging barrier, so all have read s_item: fetch the next owner)
    if (tid == 0) s_item = static_cast<uint32_t>(atomicAdd(&a0.acc[QUEUE], 1ull));
    if (scan && (PV || PE)) {
      for (uint32_t w = 4 * tid; w < hw4; w += 4 * NT) *reinterpret_cast<uint4 *>(&hb_hot[w]) = make_uint4(0u, 0u, 0u, 0u);
      for (uint32_t w = hw4 + tid; w < hw; w += NT) hb_hot[w] = 0;
    }
    for (uint32_t t = tid; t < nt; t += NT) {
      const uint32_t v = T[t];
      if (HCOLD) {
        if (v & TCOLD) {
          const uint32_t p = v & ~TCOLD;
          hkey[p] = EMPTY;
          hval[p] = 0;
        } else {
          hot_clear<HOT16>(hb_hot, v);
        }
      } else {
        const uint32_t r = v - base;
        if (r < h.hot) hot_clear<HOT16>(hb_hot, r);
        else A[r] = 0;
      }
    }
    __syncthreads();
  }
  if (!MULTI && lane == 0) add_global(a0.acc, gacc);
  __syncthreads();
  if (s_hub) hub_flush(s_hub, a0);
}

// The heavy tier's instance (1024 threads, 32-bit hot counts, dense or hashed
// cold part) and the large tier's (MH_THREADS threads, 16-bit hot counts,
// hashed cold part).
template <bool PV, bool PE, bool MULTI, bool HCOLD>
constexpr auto k_heavy1 = k_owner<PV, PE, MULTI, HCOLD, H1_THREADS, false, ACC_QHEAVY>;
constexpr uint32_t LARGE_LIMIT = 0xffff;  // the large tier's 16-bit counts bound its owners' wedges
// The large tier is off by default (large_max = med_max): with work split into
// chunks, the 1024-thread kernel counts owners of 4K-16K wedges as fast as the
// 256-thread one (20M x 60M: 1420 vs 1425 ms per count) or faster (1M x 4M:
// 47.8 vs 54.3 ms), on every graph measured.  Pinned plans can still use it.
constexpr uint32_t LARGE_MAX = MED_MAX;
// Mean wedges per neighbour of the mid-size owners from which the hot-range
// tier counts them faster than the shared-memory hash tier.  Measured (mid-size
// tier ms, per-edge counts, hash / hot range): Chung-Lu 2M x 2M gamma 2.5,
// 9.5 wedges per neighbour: 3.05 / 4.78; 1M x 4M quarter copy, 30: 2.58 / 3.08;
// 1M x 4M, 42: 14.2 / 18.0; 100k x 300k gamma 2.0, 51: 1.05 / 1.65; 20M x 60M
// 1/16 copy, 105: 9.26 / 7.47; 20M x 60M, 399: 492.6 / 420.5.
constexpr double MID_SEGMENT = 80.0;
template <bool PV, bool PE, bool MULTI>
constexpr auto k_large = k_owner<PV, PE, MULTI, true, MH_THREADS, true, ACC_QLARGE>;

// ---------------------------------------------------------------------------
// Sort aggregation: the wedges of a chunk of first endpoints [lo, hi) are
// materialised as keys ((x1 - lo) << bitsN) | x2, radix-sorted, and grouped;
// a group's length is d(x1, x2).  The chunk is sized so that its wedges fit
// the scratch budget (the paper's limit on wedges processed at once).  The
// second pass re-walks the chunk's wedges and finds d by binary search in the
// sorted group keys of its first endpoint.

__device__ __forceinline__ uint32_t lower_bound_u64(const uint64_t *a, uint32_t lo, uint32_t hi, uint64_t k) {
  while (lo < hi) {
    uint32_t mid = lo + ((hi - lo) >> 1);
    if (a[mid] < k) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// Butterfly aggregation by re-aggregation (Sec. "Butterfly aggregation", the
// alternative to atomic adds): contributions are appended as (key, value)
// pairs, then sorted by key and summed per key, so each counter is written
// once.  Keys are vertex labels (per-vertex) or adjacency slots (per-edge).
struct Sink {
  uint64_t *vkey, *ekey;
  unsigned long long *vval, *eval;
  unsigned long long *vcnt, *ecnt;  // append cursors
  uint64_t vcap, ecap;
};

// Warp-aggregated append; every lane of the warp calls it.
__device__ __forceinline__ void sink_put(uint64_t *keys, unsigned long long *vals, unsigned long long *cursor,
                                         uint64_t cap, uint64_t key, unsigned long long v, bool act,
                                         unsigned long long *err) {
  const uint32_t bm = __ballot_sync(FULL, act);
  if (!bm) return;
  const uint32_t leader = __ffs(bm) - 1;
  unsigned long long b0 = 0;
  if (lane_id() == leader) b0 = atomicAdd(cursor, static_cast<unsigned long long>(__popc(bm)));
  b0 = __shfl_sync(FULL, b0, leader);
  if (act) {
    const unsigned long long at = b0 + __popc(bm & lanemask_lt());
    if (at < cap) {
      keys[at] = key;
      vals[at] = v;
    } else {
      atomicOr(err, 64ull);
    }
  }
}

template <bool PV, bool PE, bool EMIT, bool RE>
__global__ void __launch_bounds__(MB_THREADS) k_sort_walk(CArgs a, uint32_t lo, uint32_t hi, uint64_t wbase,
                                                          int bitsN, uint64_t *__restrict__ keys,
                                                          const uint64_t *__restrict__ ukey,
                                                          const uint32_t *__restrict__ ud,
                                                          const uint32_t *__restrict__ seg, Sink sk) {
  __shared__ uint32_t s_incl[MB_THREADS], s_ex[MB_THREADS], s_oy[MB_THREADS];
  __shared__ unsigned long long s_sum[MB_THREADS];
  __shared__ uint32_t s_w[33];
  __shared__ uint32_t s_item;
  const uint32_t tid = threadIdx.x;
  if (!EMIT) s_sum[tid] = 0;
  for (;;) {
    if (tid == 0) s_item = lo + static_cast<uint32_t>(atomicAdd(&a.acc[ACC_QMED], 1ull));
    __syncthreads();
    const uint32_t x1 = s_item;
    if (x1 >= hi) break;
    if (a.wpre[x1 + 1] == a.wpre[x1]) {  // no wedges here (or counted in shared memory: k_sort_small)
      __syncthreads();                    // every thread has read s_item
      continue;
    }
    const uint64_t kx = static_cast<uint64_t>(x1 - lo) << bitsN;
    const uint32_t base = a.off[x1], dp = owner_span(a, x1);
    uint64_t *out = EMIT ? keys + (a.wpre[x1] - wbase) : nullptr;
    uint32_t s0 = 0, s1 = 0;
    if (!EMIT) { s0 = seg[x1 - lo]; s1 = seg[x1 - lo + 1]; }
    uint64_t done = 0;
    for (uint32_t k0 = 0; k0 < dp; k0 += MB_THREADS) {
      const uint32_t i = k0 + tid;
      const bool v = i < dp;
      uint32_t y, c, oy;
      owner_nbr(a, base, i, v, y, c, oy);
      uint32_t tot;
      const uint32_t incl = block_incl_scan(c, s_w, &tot);
      s_incl[tid] = incl;
      s_ex[tid] = incl - c;
      s_oy[tid] = oy;
      __syncthreads();
      for (uint32_t wb = 0; wb < tot; wb += MB_THREADS) {
        const uint32_t wi = wb + tid;
        uint32_t src = 0, slot = 0;
        unsigned long long t = 0;
        if (wi < tot) {
          src = block_find(s_incl, MB_THREADS, wi);
          slot = s_oy[src] + (wi - s_ex[src]);
          uint32_t x2 = a.adj[slot];
          if (EMIT) {
            out[done + wi] = kx | x2;
          } else {
            uint32_t r = lower_bound_u64(ukey, s0, s1, kx | x2);
            uint32_t d = (r < s1 && ukey[r] == (kx | x2)) ? ud[r] : 0;
            if (d == 0) atomicOr(&a.acc[ACC_ERR], 32ull);
            if (d > 1) {
              t = d - 1;
              if (PE && !RE) atomicAdd(&a.es[slot], t);
            }
          }
        }
        if (!EMIT) {
          if (PE && RE) sink_put(sk.ekey, sk.eval, sk.ecnt, sk.ecap, slot, t, t != 0, &a.acc[ACC_ERR]);
          warp_run_add(s_sum, src, t);
        }
      }
      __syncthreads();
      if (!EMIT) {
        unsigned long long sm = v ? s_sum[tid] : 0;
        if (RE) {
          if (PV) sink_put(sk.vkey, sk.vval, sk.vcnt, sk.vcap, y, sm, sm != 0, &a.acc[ACC_ERR]);
          if (PE) sink_put(sk.ekey, sk.eval, sk.ecnt, sk.ecap, base + i, sm, sm != 0, &a.acc[ACC_ERR]);
        } else if (sm) {
          if (PV) atomicAdd(&a.pv[y], sm);
          if (PE) atomicAdd(&a.es[base + i], sm);
        }
        if (v) s_sum[tid] = 0;
      }
      done += tot;
      __syncthreads();
    }
  }
}

// Sort aggregation for first endpoints with at most SS_MAX wedges: the
// owner's second endpoints are gathered into shared memory and sorted there
// (a bitonic network over the next power of two); a run of equal keys is one
// group, of size d (its last position finds its first by binary search).  The
// second pass finds each wedge's d by binary search in the sorted keys.
constexpr int SS_THREADS = 512;
constexpr uint32_t SS_MAX = 4096;

__device__ __forceinline__ uint32_t lower_bound_u32(const uint32_t *k, uint32_t lo, uint32_t hi, uint32_t key) {
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if (k[mid] < key) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ uint32_t upper_bound_u32(const uint32_t *k, uint32_t lo, uint32_t hi, uint32_t key) {
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if (k[mid] <= key) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

template <bool PV, bool PE>
__global__ void __launch_bounds__(SS_THREADS) k_sort_small(CArgs a, uint32_t lo, uint32_t hi) {
  __shared__ uint32_t K[SS_MAX];
  __shared__ uint32_t s_incl[SS_THREADS], s_ex[SS_THREADS], s_oy[SS_THREADS];
  __shared__ unsigned long long s_sum[SS_THREADS];
  __shared__ uint32_t s_w[33];
  __shared__ unsigned long long s_w64[33];
  __shared__ uint32_t s_item;
  const uint32_t tid = threadIdx.x;
  unsigned long long gacc = 0;
  if (PV || PE) s_sum[tid] = 0;
  for (;;) {
    if (tid == 0) s_item = lo + static_cast<uint32_t>(atomicAdd(&a.acc[ACC_QLARGE], 1ull));
    __syncthreads();
    const uint32_t x1 = s_item;
    if (x1 >= hi) break;
    const uint64_t wc = a.wpre[x1 + 1] - a.wpre[x1];
    if (wc == 0 || wc > SS_MAX) {  // no wedges, or sorted in device memory (k_sort_walk)
      __syncthreads();             // every thread has read s_item
      continue;
    }
    const uint32_t n_w = static_cast<uint32_t>(wc);
    const uint32_t base = a.off[x1], dp = owner_span(a, x1);
    // ---- gather the owner's second endpoints
    uint32_t done = 0;
    for (uint32_t k0 = 0; k0 < dp; k0 += SS_THREADS) {
      const uint32_t i = k0 + tid;
      uint32_t y, c, oy;
      owner_nbr(a, base, i, i < dp, y, c, oy);
      uint32_t tot;
      const uint32_t incl = block_incl_scan(c, s_w, &tot);
      s_incl[tid] = incl;
      s_ex[tid] = incl - c;
      s_oy[tid] = oy;
      __syncthreads();
      for (uint32_t wi = tid; wi < tot; wi += SS_THREADS) {
        const uint32_t src = block_find(s_incl, SS_THREADS, wi);
        const uint32_t at = done + wi;
        if (at < SS_MAX) K[at] = a.adj[s_oy[src] + (wi - s_ex[src])];
      }
      done += tot;
      __syncthreads();
    }
    if (done != n_w) {  // the wedge split and the adjacency disagree: record, skip
      if (tid == 0) atomicOr(&a.acc[ACC_ERR], 32ull);
      __syncthreads();
      continue;
    }
    uint32_t P = 2;
    while (P < n_w) P <<= 1;
    for (uint32_t t = n_w + tid; t < P; t += SS_THREADS) K[t] = 0xffffffffu;
    __syncthreads();
    // ---- bitonic sort of K[0, P)
    for (uint32_t k = 2; k <= P; k <<= 1) {
      for (uint32_t j = k >> 1; j > 0; j >>= 1) {
        for (uint32_t t = tid; t < P / 2; t += SS_THREADS) {
          const uint32_t i = (t / j) * 2 * j + (t % j), l = i + j;
          const uint32_t ki = K[i], kl = K[l];
          if ((ki > kl) == ((i & k) == 0)) {
            K[i] = kl;
            K[l] = ki;
          }
        }
        __syncthreads();
      }
    }
    // ---- groups: C(d, 2) to the global count and both endpoints
    unsigned long long own = 0;
    for (uint32_t t = tid; t < n_w; t += SS_THREADS) {
      const uint32_t key = K[t];
      if (t + 1 == n_w || K[t + 1] != key) {
        const unsigned long long d = t + 1 - lower_bound_u32(K, 0, t, key), b = d * (d - 1) / 2;
        own += b;
        if (PV && b) atomicAdd(&a.pv[key], b);
      }
    }
    own = block_sum(own, s_w64);
    if (tid == 0) {
      gacc += own;
      if (PV && own) atomicAdd(&a.pv[x1], own);
    }
    // ---- centres and edges: d - 1 per wedge
    if (PV || PE) {
      for (uint32_t k0 = 0; k0 < dp; k0 += SS_THREADS) {
        const uint32_t i = k0 + tid;
        const bool v = i < dp;
        uint32_t y, c, oy;
        owner_nbr(a, base, i, v, y, c, oy);
        uint32_t tot;
        const uint32_t incl = block_incl_scan(c, s_w, &tot);
        s_incl[tid] = incl;
        s_ex[tid] = incl - c;
        s_oy[tid] = oy;
        __syncthreads();
        for (uint32_t wb = 0; wb < tot; wb += SS_THREADS) {  // block-uniform trip count
          const uint32_t wi = wb + tid;
          uint32_t src = 0;
          unsigned long long t = 0;
          if (wi < tot) {
            src = block_find(s_incl, SS_THREADS, wi);
            const uint32_t slot = s_oy[src] + (wi - s_ex[src]), x2 = a.adj[slot];
            const uint32_t lb = lower_bound_u32(K, 0, n_w, x2);
            const uint32_t d = upper_bound_u32(K, lb, n_w, x2) - lb;
            if (d > 1) {
              t = d - 1;
              if (PE) atomicAdd(&a.es[slot], t);
            }
          }
          warp_run_add(s_sum, src, t);
        }
        __syncthreads();
        if (v) {
          const unsigned long long sm = s_sum[tid];
          if (sm) {
            if (PV) atomicAdd(&a.pv[y], sm);
            if (PE) atomicAdd(&a.es[base + i], sm);
            s_sum[tid] = 0;
          }
        }
        __syncthreads();
      }
    }
  }
  if (tid == 0 && gacc) add_global(a.acc, gacc);
}

// wl[x] = the wedges of owner x when they are too many for k_sort_small, else 0.
__global__ void k_wedges_large(const uint64_t *__restrict__ wpre, uint64_t n, uint64_t *__restrict__ wl) {
  for (size_t x = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x; x < n;
       x += static_cast<size_t>(gridDim.x) * blockDim.x) {
    const uint64_t w = wpre[x + 1] - wpre[x];
    wl[x] = w > SS_MAX ? w : 0;
  }
}

__global__ void k_runs(const uint64_t *__restrict__ keys, const uint32_t *__restrict__ head,
                       const uint32_t *__restrict__ cid, uint64_t cnt, uint64_t *__restrict__ ukey,
                       uint32_t *__restrict__ rstart) {
  for (size_t i = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < cnt;
       i += static_cast<size_t>(gridDim.x) * blockDim.x) {
    if (head[i]) {
      uint32_t r = cid[i];
      ukey[r] = keys[i];
      rstart[r] = static_cast<uint32_t>(i);
    }
  }
}

template <bool PV, bool RE>
__global__ void k_run_sums(CArgs a, const uint64_t *__restrict__ ukey, const uint32_t *__restrict__ rstart,
                           uint32_t nr, uint32_t cnt, uint32_t lo, int bitsN, uint32_t *__restrict__ ud, Sink sk) {
  __shared__ unsigned long long s_w64[33];
  const uint64_t mask = (uint64_t(1) << bitsN) - 1;
  unsigned long long acc = 0;
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t rb = blockIdx.x * blockDim.x; rb < nr; rb += stride) {  // block-uniform trip count
    const uint32_t r = rb + threadIdx.x;
    unsigned long long b = 0;
    uint32_t k1 = 0, k2 = 0;
    if (r < nr) {
      uint32_t d = (r + 1 < nr ? rstart[r + 1] : cnt) - rstart[r];
      ud[r] = d;
      b = static_cast<unsigned long long>(d) * (d - 1) / 2;
      acc += b;
      k1 = lo + static_cast<uint32_t>(ukey[r] >> bitsN);
      k2 = static_cast<uint32_t>(ukey[r] & mask);
    }
    if (PV && RE) {
      sink_put(sk.vkey, sk.vval, sk.vcnt, sk.vcap, k1, b, b != 0, &a.acc[ACC_ERR]);
      sink_put(sk.vkey, sk.vval, sk.vcnt, sk.vcap, k2, b, b != 0, &a.acc[ACC_ERR]);
    } else if (PV && b) {
      atomicAdd(&a.pv[k1], b);
      atomicAdd(&a.pv[k2], b);
    }
  }
  unsigned long long tot = block_sum(acc, s_w64);
  if (threadIdx.x == 0) add_global(a.acc, tot);
}

__global__ void k_segments(const uint64_t *__restrict__ ukey, uint32_t nr, uint32_t nseg, int bitsN,
                           uint32_t *__restrict__ seg) {
  for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j <= nseg; j += gridDim.x * blockDim.x)
    seg[j] = lower_bound_u64(ukey, 0, nr, static_cast<uint64_t>(j) << bitsN);
}

// Largest hi in (lo, n] with wpre[hi] - wpre[lo] <= cap (at least lo + 1).
__global__ void k_chunk_end(const uint64_t *__restrict__ wpre, uint64_t n, uint32_t lo, uint64_t cap,
                            unsigned long long *out) {
  uint64_t base = wpre[lo];
  uint64_t l = lo + 1, h = n;  // answer in [lo+1, n]
  while (l < h) {
    uint64_t mid = (l + h + 1) >> 1;
    if (wpre[mid] - base <= cap) l = mid;
    else h = mid - 1;
  }
  out[0] = l;
  out[1] = wpre[l] - base;
}

// ---------------------------------------------------------------------------
// Tier classification.
// Writes each owner to its tier's list; the lists hold cap[t] entries (the
// counts of the statistics pass), and an owner past them sets an error bit
// instead of being written.
struct TierCaps {
  uint64_t cap[4];
};

__global__ void k_classify(const uint64_t *__restrict__ wpre, uint64_t n, uint64_t olo, uint64_t ohi,
                           uint64_t light_max, uint64_t med_max, uint64_t large_max, uint64_t hub_min,
                           uint32_t *__restrict__ light, uint32_t *__restrict__ med, uint32_t *__restrict__ large,
                           uint64_t *__restrict__ heavy_keys, int bitsN, unsigned long long *acc, TierCaps caps) {
  size_t stride = static_cast<size_t>(gridDim.x) * blockDim.x;
  size_t iters = (n + stride - 1) / stride;
  for (size_t itn = 0; itn < iters; itn++) {
    size_t x = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x + itn * stride;
    uint64_t wc = (x < n && x >= olo && x < ohi) ? wpre[x + 1] - wpre[x] : 0;
    int tier = wc == 0 ? 0 : (wc <= light_max ? 1 : (wc <= med_max ? 2 : (wc <= large_max ? 3 : 4)));
    uint32_t hubs = __popc(__ballot_sync(FULL, tier == 4 && wc >= hub_min));
    if (lane_id() == 0 && hubs) atomicAdd(&acc[ACC_NHUB], (unsigned long long)hubs);
#pragma unroll
    for (int t = 1; t <= 4; t++) {
      uint32_t bm = __ballot_sync(FULL, tier == t);
      if (!bm) continue;
      uint32_t leader = __ffs(bm) - 1;
      unsigned long long b0 = 0;
      if (lane_id() == leader) b0 = atomicAdd(&acc[ACC_NLIGHT + t - 1], (unsigned long long)__popc(bm));
      b0 = __shfl_sync(FULL, b0, leader);
      if (tier == t) {
        uint64_t at = b0 + __popc(bm & lanemask_lt());
        if (at >= caps.cap[t - 1]) {
          atomicOr(&acc[ACC_ERR], 128ull);
          continue;
        }
        if (t == 1) light[at] = static_cast<uint32_t>(x);
        else if (t == 2) med[at] = static_cast<uint32_t>(x);
        else if (t == 3) large[at] = static_cast<uint32_t>(x);
        else {
          // Owners by power-of-two band of wedge count, largest band first
          // (the biggest owners start early), and by label within a band:
          // owners of nearby rank read nearly the same suffixes of the hub
          // lists and update the same edge slots, so the owners in flight
          // share those lines in L2 (20M x 60M heavy tier: 538 ms by wedge
          // count, 516 ms by band then label).
          heavy_keys[at] = (static_cast<uint64_t>(__clzll(wc)) << bitsN) | x;
        }
      }
    }
  }
}

__global__ void k_keys_low(const uint64_t *__restrict__ keys, uint32_t nk, int bitsN, uint32_t *__restrict__ out) {
  const uint64_t mask = (uint64_t(1) << bitsN) - 1;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nk; i += gridDim.x * blockDim.x)
    out[i] = static_cast<uint32_t>(keys[i] & mask);
}

// out[0] = the largest bound on distinct second endpoints over the listed
// owners; out[1] = the largest range of labels their second endpoints can
// take (the length of a dense histogram for them).
__global__ void k_max_wedges_list(const uint32_t *__restrict__ list, uint32_t nl, const uint64_t *__restrict__ wpre,
                                  uint64_t n, uint32_t nU, int rev, unsigned long long *out) {
  unsigned long long mx = 0, mr = 0;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nl; i += gridDim.x * blockDim.x) {
    uint32_t x = list[i];
    unsigned long long dm = distinct_bound(wpre[x + 1] - wpre[x], n, nU, x, rev);
    unsigned long long rm = distinct_bound(~0ull, n, nU, x, rev);
    mx = dm > mx ? dm : mx;
    mr = rm > mr ? rm : mr;
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    unsigned long long y = __shfl_xor_sync(FULL, mx, o), z = __shfl_xor_sync(FULL, mr, o);
    mx = y > mx ? y : mx;
    mr = z > mr ? z : mr;
  }
  if (lane_id() == 0 && mx) atomicMax(&out[0], mx);
  if (lane_id() == 0 && mr) atomicMax(&out[1], mr);
}


// ---------------------------------------------------------------------------
// Outputs back in id space / input order.
__global__ void k_out_vertex(const unsigned long long *__restrict__ pv, const uint32_t *__restrict__ label,
                             uint32_t nU, uint32_t nV, uint64_t *__restrict__ outU, uint64_t *__restrict__ outV) {
  const uint64_t n = static_cast<uint64_t>(nU) + nV;
  for (size_t x = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x; x < n;
       x += static_cast<size_t>(gridDim.x) * blockDim.x) {
    uint64_t c = pv[label[x]];
    if (x < nU) {
      if (outU) outU[x] = c;
    } else if (outV) {
      outV[x - nU] = c;
    }
  }
}

// Per-edge count of canonical edge e = the sums on its two adjacency slots.
// Canonical edges are ordered by U endpoint, so slotA reads stay within one
// list for runs of edges.
__global__ void k_edge_sums(const unsigned long long *__restrict__ es, const unsigned int *__restrict__ es32,
                            const uint32_t *__restrict__ slotA, const uint32_t *__restrict__ slotB, uint64_t m,
                            uint64_t *__restrict__ E) {
  for (size_t e = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < m;
       e += static_cast<size_t>(gridDim.x) * blockDim.x) {
    const uint32_t sa = slotA[e], sb = slotB[e];
    E[e] = es[sa] + es[sb] + es32[sa] + es32[sb];
  }
}

// Input pair k reports the count of its canonical edge.
__global__ void k_out_edge(const uint64_t *__restrict__ E, const uint32_t *__restrict__ in2c, uint64_t m_in,
                           uint64_t *__restrict__ outE) {
  for (size_t k = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x; k < m_in;
       k += static_cast<size_t>(gridDim.x) * blockDim.x)
    outE[k] = E[in2c[k]];
}

// ---------------------------------------------------------------------------
// Host orchestration.

template <class K, class... Args>
static pb_status launch_cluster(K kernel, unsigned grid, unsigned block, unsigned cl, size_t smem, cudaStream_t s,
                                Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cl;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  PB_CUDA(cudaLaunchKernelEx(&cfg, kernel, args...));
  count_launch();
  return PB_OK;
}

template <class K>
static int max_clusters(K kernel, unsigned block, unsigned cl, size_t smem) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(cl * 256);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cl;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int nc = 0;
  if (cudaOccupancyMaxActiveClusters(&nc, kernel, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return nc;
}

// Autotuner statistics of the owners in [olo, ohi) under one owner direction:
// owners and wedges per tier, the heavy owners' largest wedge count, label
// range (the length of a dense histogram for them) and distinct bound, the
// largest wedge count overall, the heavy owners above the hub threshold, and
// the prefix sums of second-endpoint wedges at the candidate hot-range sizes
// (wother is the other direction's wedge prefix: a wedge's second endpoint is
// the owner of that wedge in the other direction).
constexpr uint32_t HOT_SMALL = 16384, HOT_LARGE = 49152;  // candidate hot-range sizes
constexpr uint64_t LARGE_LIMIT_D = 0xffff;                 // the large tier's bound (16-bit counts)
enum { TS_N = 0, TS_W = 4, TS_HMAXW = 8, TS_HRANGE = 9, TS_HDIST = 10, TS_MAXW = 11, TS_NHUB = 12, TS_PRE = 13,
       TS_SPAN = 17, TS_WMID = 18, TS_WORDS = 20 };

__global__ void k_tier_stats(const uint64_t *__restrict__ wpre, const uint64_t *__restrict__ wother, uint64_t n,
                             uint32_t nU, int rev, uint64_t olo, uint64_t ohi, uint64_t light_max, uint64_t med_max,
                             uint64_t large_max, uint64_t hub_min, const uint32_t *__restrict__ off,
                             const uint32_t *__restrict__ degp, unsigned long long *out) {
  unsigned long long cnt[4] = {0, 0, 0, 0}, ws[4] = {0, 0, 0, 0}, hmaxw = 0, hrange = 0, hdist = 0, maxw = 0,
                     nhub = 0, span = 0, wmid = 0;
  for (size_t x = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x; x < n;
       x += static_cast<size_t>(gridDim.x) * blockDim.x) {
    const uint64_t wc = wpre[x + 1] - wpre[x];
    if (wc == 0 || x < olo || x >= ohi) continue;
    const int t = wc <= light_max ? 0 : (wc <= med_max ? 1 : (wc <= large_max ? 2 : 3));
    cnt[t]++;
    ws[t] += wc;
    maxw = wc > maxw ? wc : maxw;
    // neighbours of the owners between light_max and the large tier's limit:
    // their wedges per neighbour (mean segment length) choose the tier of the
    // mid-size owners
    if (wc > light_max && wc <= LARGE_LIMIT_D) {
      span += rev ? off[x + 1] - off[x] : degp[x];
      wmid += wc;
    }
    if (t == 3) {
      const uint32_t xl = static_cast<uint32_t>(x);
      const unsigned long long r = distinct_bound(~0ull, n, nU, xl, rev), d = distinct_bound(wc, n, nU, xl, rev);
      hmaxw = wc > hmaxw ? wc : hmaxw;
      hrange = r > hrange ? r : hrange;
      hdist = d > hdist ? d : hdist;
      if (wc >= hub_min) nhub++;
    }
  }
#pragma unroll
  for (int t = 0; t < 4; t++) {
    const unsigned long long c = warp_sum(cnt[t]), w = warp_sum(ws[t]);
    if (lane_id() == 0 && c) {
      atomicAdd(&out[TS_N + t], c);
      atomicAdd(&out[TS_W + t], w);
    }
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    hmaxw = max(hmaxw, __shfl_xor_sync(FULL, hmaxw, o));
    hrange = max(hrange, __shfl_xor_sync(FULL, hrange, o));
    hdist = max(hdist, __shfl_xor_sync(FULL, hdist, o));
    maxw = max(maxw, __shfl_xor_sync(FULL, maxw, o));
  }
  nhub = warp_sum(nhub);
  span = warp_sum(span);
  wmid = warp_sum(wmid);
  if (lane_id() == 0 && span) {
    atomicAdd(&out[TS_SPAN], span);
    atomicAdd(&out[TS_WMID], wmid);
  }
  if (lane_id() == 0) {
    if (hmaxw) atomicMax(&out[TS_HMAXW], hmaxw);
    if (hrange) atomicMax(&out[TS_HRANGE], hrange);
    if (hdist) atomicMax(&out[TS_HDIST], hdist);
    if (maxw) atomicMax(&out[TS_MAXW], maxw);
    if (nhub) atomicAdd(&out[TS_NHUB], nhub);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const uint64_t nV = n - nU;
#pragma unroll
    for (int k = 0; k < 2; k++) {
      const uint64_t H = k == 0 ? HOT_SMALL : HOT_LARGE;
      const uint64_t hu = H < nU ? H : nU, hv = H < nV ? H : nV;
      out[TS_PRE + 2 * k] = wother[hu] - wother[0];
      out[TS_PRE + 2 * k + 1] = wother[nU + hv] - wother[nU];
    }
  }
}

struct TierStats {  // tiers: light, medium, large, heavy
  uint64_t n[4] = {0, 0, 0, 0}, w[4] = {0, 0, 0, 0};
  uint64_t hmaxw = 0, hrange = 0, hdist = 0, maxw = 0, nhub = 0;
  uint64_t pre[4] = {0, 0, 0, 0};
  uint64_t span_mid = 0, w_mid = 0;  // neighbours and wedges of the owners with med_max < wedges <= LARGE_LIMIT
};

// Owners given a cluster when hubs get one: at least HUB_MIN wedges.  A power
// of two, so that the hubs are exactly the first bands of the heavy list.
constexpr uint64_t HUB_MIN = uint64_t(1) << 18;
constexpr uint64_t HUB_MAX = uint64_t(1) << 20;  // hubs get clusters only past this many wedges

// Statistics into buf (TS_WORDS words of device memory; the graph's own
// buffer when buf is NULL).  Planning calls that may run while the graph is
// being counted (pb_autotune, pb_count_bytes) pass a buffer of their own.
static pb_status tier_stats(pb_graph *g, int rev, uint64_t olo, uint64_t ohi, uint64_t light_max, uint64_t med_max,
                            uint64_t large_max, cudaStream_t s, TierStats *ts, unsigned long long *buf = nullptr) {
  if (!buf) {
    if (!g->tstat) PB_TRY(dalloc_t(&g->tstat, TS_WORDS, s));
    buf = g->tstat;
  }
  PB_CUDA(cudaMemsetAsync(buf, 0, TS_WORDS * sizeof(unsigned long long), s));
  const uint64_t *wp = rev ? g->wpre_rev : g->wpre, *wo = rev ? g->wpre : g->wpre_rev;
  k_tier_stats<<<grid_for(g->n, 256, 4096), 256, 0, s>>>(wp, wo, g->n, g->nU, rev, olo, ohi, light_max, med_max,
                                                        large_max, HUB_MIN, g->off, g->degp, buf);
  count_launch();
  unsigned long long h[TS_WORDS];
  PB_CUDA(cudaMemcpyAsync(h, buf, sizeof(h), cudaMemcpyDeviceToHost, s));
  PB_CUDA(cudaStreamSynchronize(s));
  for (int t = 0; t < 4; t++) {
    ts->n[t] = h[TS_N + t];
    ts->w[t] = h[TS_W + t];
  }
  ts->hmaxw = h[TS_HMAXW];
  ts->hrange = h[TS_HRANGE];
  ts->hdist = h[TS_HDIST];
  ts->maxw = h[TS_MAXW];
  ts->nhub = h[TS_NHUB];
  ts->span_mid = h[TS_SPAN];
  ts->w_mid = h[TS_WMID];
  for (int k = 0; k < 4; k++) ts->pre[k] = h[TS_PRE + k];
  return PB_OK;
}

// Device memory of one heavy slot: a dense histogram over the heavy owners'
// label range (or a hash table for their cold second endpoints) and a touched
// list bounded by their distinct second endpoints.
static uint64_t dense_slot_bytes(const pb_graph *g, const TierStats &ts, uint64_t *side, uint64_t *tcap) {
  uint64_t sd = g->nU > g->nV ? g->nU : g->nV;
  if (ts.hrange && ts.hrange < sd) sd = ts.hrange;
  const uint64_t tc = ts.hdist < sd ? ts.hdist : sd;
  if (side) *side = sd;
  if (tcap) *tcap = tc;
  return (sd + tc) * sizeof(uint32_t);
}

static uint64_t hash_slot_bytes(const pb_graph *g, const TierStats &ts, uint64_t *hcap, uint64_t *tcap) {
  uint64_t sd = g->nU > g->nV ? g->nU : g->nV;
  const uint64_t tc = ts.hdist < sd ? ts.hdist : sd;
  uint64_t cap = 32;
  while (cap < 2 * tc) cap <<= 1;
  if (hcap) *hcap = cap;
  if (tcap) *tcap = tc;
  return (2 * cap + tc) * sizeof(uint32_t);
}

// Resident blocks of the one-block heavy kernel with `hot` shared-memory labels.
static uint64_t heavy1_resident(int device, uint32_t hot) {
  int per_sm = 0;
  const size_t smem = hot * sizeof(uint32_t);
  cudaFuncSetAttribute(k_heavy1<false, true, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_heavy1<false, true, false, false>, H1_THREADS,
                                                    smem) != cudaSuccess)
    cudaGetLastError();
  return static_cast<uint64_t>(sm_count(device)) * (per_sm > 0 ? per_sm : 1);
}

// Large-tier slot: a hash table for the cold second endpoints of an owner of
// at most large_max wedges (load at most 1/2) and its touched list.
static void large_slot_shape(uint64_t large_max, HeavySlots *hm) {
  uint64_t cap = 32;
  while (cap < 2 * large_max) cap <<= 1;
  hm->hcap = cap;
  hm->tcap = large_max;
  hm->hot = MH_HOT;
}
static uint64_t large_slot_bytes(const HeavySlots &hm) { return (2 * hm.hcap + hm.tcap) * sizeof(uint32_t); }

// The statistics part of the plan: tiers, hot range, and the aggregation that
// PB_AGG_AUTO uses (rules documented with pb_plan_t).
static void plan_from_stats(const pb_graph *g, TierStats &ts, uint64_t budget, pb_plan_t *plan) {
  // Mid-size owners (light_max < wedges <= med_max): the shared-memory hash
  // tier, or -- when their wedges sit in long segments (mean wedges per
  // neighbour at least MID_SEGMENT) -- the 256-thread hot-range tier, which
  // walks a segment with a whole warp instead of locating every wedge.  The
  // owners and wedges of the medium tier then move to the large one.
  plan->mid_segment = ts.span_mid ? static_cast<double>(ts.w_mid) / static_cast<double>(ts.span_mid) : 0.0;
  if (plan->mid_segment >= MID_SEGMENT && plan->med_max > plan->light_max) {
    if (plan->large_max < plan->med_max) plan->large_max = plan->med_max;
    plan->med_max = plan->light_max;
    ts.n[2] += ts.n[1];
    ts.w[2] += ts.w[1];
    ts.n[1] = ts.w[1] = 0;
  }
  for (int t = 0; t < 4; t++) {
    plan->owners[t] = ts.n[t];
    plan->wedges[t] = ts.w[t];
  }
  plan->max_owner_wedges = ts.maxw;
  plan->scratch_bytes = budget;
  const double W = g->W ? static_cast<double>(g->W) : 1.0;
  const double hit16 = static_cast<double>(ts.pre[0] + ts.pre[1]) / W;
  const double hit48 = static_cast<double>(ts.pre[2] + ts.pre[3]) / W;
  plan->hot = hit16 < 0.9 ? HOT_LARGE : HOT_SMALL;
  plan->hot_hit = plan->hot == HOT_LARGE ? hit48 : hit16;
  const uint64_t nh = ts.n[3];
  plan->hub_min = UINT64_MAX;
  plan->hub_cluster = 1;
  plan->heavy_slots = 0;
  plan->slot_bytes = 0;
  if (nh == 0) {
    plan->agg = PB_AGG_BATCH;
    return;
  }
  const uint64_t resident = heavy1_resident(g->device, plan->hot);
  const uint64_t want = nh < resident ? nh : resident;
  const uint64_t dslot = dense_slot_bytes(g, ts, nullptr, nullptr), hslot = hash_slot_bytes(g, ts, nullptr, nullptr);
  const uint64_t fit_d = budget / (dslot + 16), fit_h = budget / (hslot + 16);
  plan->slot_bytes_dense = dslot;
  plan->slot_bytes_hash = hslot;
  plan->resident_blocks = static_cast<uint32_t>(resident);
  if (ts.hmaxw > HUB_MAX && ts.hmaxw * want > 8 * ts.w[3]) {
    // one owner would hold a block far past the others: hubs share a cluster
    plan->agg = PB_AGG_HIST;
    plan->hub_min = HUB_MIN;
    plan->hub_cluster = 2;
    plan->slot_bytes = dslot;
    plan->heavy_slots = static_cast<uint32_t>(fit_d < want ? fit_d : want);
  } else if (fit_d >= want || fit_d >= fit_h) {
    plan->agg = PB_AGG_BATCH;
    plan->slot_bytes = dslot;
    plan->heavy_slots = static_cast<uint32_t>(fit_d < want ? fit_d : want);
  } else {
    plan->agg = PB_AGG_HASH;
    plan->slot_bytes = hslot;
    plan->heavy_slots = static_cast<uint32_t>(fit_h < want ? fit_h : want);
  }
}

// What one count runs: the tier bounds, and the heavy tier's path.
struct Plan {
  bool pv, pe;
  uint64_t light_max, med_max, large_max;
  int heavy;          // PB_AGG_HIST / PB_AGG_BATCH: dense; PB_AGG_HASH: hashed
  uint32_t hot;       // shared-memory labels of the one-block heavy kernel
  unsigned cluster;   // blocks per hub owner (1: no hub clusters)
  uint64_t owner_lo, owner_hi;  // owners counted
};

template <bool PV, bool PE>
static pb_status run_tiers(pb_graph *g, const CArgs &a, const Plan &p, const TierStats &ts, uint64_t budget,
                           cudaStream_t s) {
  const uint64_t n = g->n;
  uint32_t *light = nullptr, *med = nullptr, *large = nullptr, *heavy = nullptr;
  uint64_t *hkeys = nullptr;
  pb_status st = PB_OK;
  const int sms = sm_count(g->device);
  // Every launch below is sized from the statistics read before the count, so
  // the host does not wait on the device again until the outputs are ready.
  const uint32_t nl = static_cast<uint32_t>(ts.n[0]), nm = static_cast<uint32_t>(ts.n[1]),
                 nq = static_cast<uint32_t>(ts.n[2]), nh = static_cast<uint32_t>(ts.n[3]);
  // The persistent tier kernels take this share of the device's resident
  // blocks (pb_set_grid_share): concurrent counts on other streams then run
  // side by side instead of waiting for a kernel that holds every SM.
  auto share = [&](uint64_t resident) -> uint64_t {
    const double f = g->grid_share > 0.0 && g->grid_share < 1.0 ? g->grid_share : 1.0;
    const uint64_t r = static_cast<uint64_t>(std::ceil(f * static_cast<double>(resident)));
    return r < 1 ? 1 : r;
  };
  do {
    if ((st = dalloc_t(&light, nl + 1, s)) != PB_OK) break;
    if ((st = dalloc_t(&med, nm + 1, s)) != PB_OK) break;
    if ((st = dalloc_t(&large, nq + 1, s)) != PB_OK) break;
    if ((st = dalloc_t(&hkeys, nh + 1, s)) != PB_OK) break;
    {
      PhaseScope ph(PB_PHASE_CLASSIFY, s);
      const TierCaps caps = {{nl, nm, nq, nh}};
      k_classify<<<grid_for(n, 256, 8192), 256, 0, s>>>(a.wpre, n, p.owner_lo, p.owner_hi, p.light_max, p.med_max,
                                                        p.large_max, HUB_MIN, light, med, large, hkeys, g->bitsN,
                                                        a.acc, caps);
      count_launch();
      ph.finish(s);
    }
    if (nl) {
      PhaseScope ph(PB_PHASE_LIGHT, s);
      const size_t smem = LW_WARPS * (LW_CAP + LW_CAP / 2) * sizeof(uint32_t);
      PB_CUDA(cudaFuncSetAttribute(k_light<PV, PE, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      int per_sm = 0;
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_light<PV, PE, false>, LW_THREADS, smem);
      unsigned grid = static_cast<unsigned>(share(static_cast<uint64_t>(sms) * (per_sm > 0 ? per_sm : 1)));
      unsigned need = (nl + LW_WARPS - 1) / LW_WARPS;
      PB_LAUNCH((k_light<PV, PE, false>), grid < need ? grid : need, LW_THREADS, smem, s, a, light, nl,
                (const uint64_t *)nullptr, (const CArgs *)nullptr);
      ph.finish(s, ts.w[0]);
    }
    if (nm) {
      PhaseScope ph(PB_PHASE_MEDIUM, s);
      const size_t smem = MB_SMEM;
      PB_CUDA(cudaFuncSetAttribute(k_medium<PV, PE, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      int per_sm = 0;
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_medium<PV, PE, false>, MB_THREADS, smem);
      unsigned grid = static_cast<unsigned>(share(static_cast<uint64_t>(sms) * (per_sm > 0 ? per_sm : 1)));
      PB_LAUNCH((k_medium<PV, PE, false>), grid < nm ? grid : nm, MB_THREADS, smem, s, a, med, nm,
                (const uint64_t *)nullptr, (const CArgs *)nullptr);
      ph.finish(s, ts.w[1]);
    }
    if (nq) {
      // One MH_THREADS block per owner: 16-bit counts of the first MH_HOT
      // labels in shared memory, the rest in a small hash table per slot.
      PhaseScope ph(PB_PHASE_LARGE, s);
      HeavySlots hm = {};
      large_slot_shape(p.large_max, &hm);
      const size_t smem = hot_words(hm.hot, true) * sizeof(uint32_t);
      auto kern = k_large<PV, PE, false>;
      PB_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      int per_sm = 0;
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, MH_THREADS, smem);
      uint64_t nslots = share(static_cast<uint64_t>(sms) * (per_sm > 0 ? per_sm : 1));
      if (nslots > nq) nslots = nq;
      if ((st = ensure_scratch2(g, nslots * large_slot_bytes(hm), s)) != PB_OK) break;
      hm.hkey = static_cast<uint32_t *>(g->scratch2);
      hm.hval = hm.hkey + nslots * hm.hcap;
      hm.T = hm.hval + nslots * hm.hcap;
      if (cudaMemsetAsync(hm.hkey, 0xff, nslots * hm.hcap * sizeof(uint32_t), s) != cudaSuccess ||
          cudaMemsetAsync(hm.hval, 0, nslots * hm.hcap * sizeof(uint32_t), s) != cudaSuccess) { st = fail(PB_ERR_CUDA, "memset"); break; }
      PB_LAUNCH(kern, static_cast<unsigned>(nslots), MH_THREADS, smem, s, a, large, nq, hm, (const uint64_t *)nullptr,
                (const CArgs *)nullptr);
      ph.finish(s, ts.w[2]);
    }
    if (nh) {
      if ((st = radix_sort(hkeys, nullptr, nh, g->bitsN + 7, s)) != PB_OK) break;  // band (<= 63) above the label
      if ((st = dalloc_t(&heavy, nh, s)) != PB_OK) break;
      k_keys_low<<<grid_for(nh, 256, 4096), 256, 0, s>>>(hkeys, nh, g->bitsN, heavy);
      count_launch();
      const bool hashed = p.heavy == PB_AGG_HASH;
      HeavySlots hs = {};
      uint64_t slot_bytes = hashed ? hash_slot_bytes(g, ts, &hs.hcap, &hs.tcap)
                                   : dense_slot_bytes(g, ts, &hs.side, &hs.tcap);
      // Hubs (the head of the largest-first list) get one cluster each; the
      // rest one block each.
      const uint32_t nhub = p.cluster > 1 ? static_cast<uint32_t>(ts.nhub) : 0;
      unsigned hub_cl = p.cluster, rest_cl = 1;
      const uint64_t fit = budget / (slot_bytes + 16);
      if (fit == 0) { st = fail(PB_ERR_SCRATCH, "scratch budget %llu B below one heavy slot (%llu B)", (unsigned long long)budget, (unsigned long long)slot_bytes); break; }
      // The one-block kernel (shared-memory hot range) serves the non-hub
      // owners when at least one slot per SM fits the budget; otherwise
      // slots are shared by clusters of blocks so that every SM works.
      if (fit < static_cast<uint64_t>(sms)) {
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_heavy<PV, PE, true, false>, HB_THREADS, 0);
        const uint64_t resident = static_cast<uint64_t>(sms) * (per_sm > 0 ? per_sm : 1);
        uint64_t want = (resident + fit - 1) / fit;
        unsigned c = 1;
        while (c < want && c < 8) c <<= 1;
        rest_cl = c;
        if (hub_cl < c) hub_cl = c;
      }
      struct Part { const uint32_t *list; uint32_t cnt; unsigned cl; };
      Part parts[2] = {{heavy, nhub, hub_cl}, {heavy + nhub, nh - nhub, rest_cl}};
      PhaseScope ph(PB_PHASE_HEAVY, s);
      for (const Part &pt : parts) {
        if (pt.cnt == 0) continue;
        const unsigned cl = pt.cl;
        const bool one = cl == 1;  // one block per slot: k_heavy1 with the hot range
        auto ckern = hashed ? k_heavy<PV, PE, false, false> : k_heavy<PV, PE, true, false>;
        auto okern = hashed ? k_heavy1<PV, PE, false, true> : k_heavy1<PV, PE, false, false>;
        if (cl > 8) PB_CUDA(cudaFuncSetAttribute(ckern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
        hs.hot = one ? p.hot : 0;
        const size_t hsmem = hs.hot * sizeof(uint32_t);
        int nc = 0;
        if (one) {
          PB_CUDA(cudaFuncSetAttribute(okern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)hsmem));
          int per_sm = 0;
          cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, okern, H1_THREADS, hsmem);
          nc = sms * (per_sm > 0 ? per_sm : 1);
        } else {
          nc = max_clusters(ckern, HB_THREADS, cl, hsmem);
        }
        if (nc <= 0) nc = sms / static_cast<int>(cl);
        uint64_t nslots = share(static_cast<uint64_t>(nc));
        if (nslots > fit) nslots = fit;
        if (nslots > pt.cnt) nslots = pt.cnt;
        // the touched list is used by k_heavy1 in both modes, by k_heavy in dense mode
        const uint64_t tlist = (one || !hashed) ? hs.tcap : 0;
        size_t need = nslots * slot_bytes + nslots * 3 * sizeof(uint32_t) + 64;
        if ((st = ensure_scratch(g, need, s)) != PB_OK) break;
        char *sp = static_cast<char *>(g->scratch);
        if (!hashed) {
          hs.A = reinterpret_cast<uint32_t *>(sp);
          hs.T = hs.A + nslots * hs.side;
          hs.tcnt = hs.T + nslots * hs.tcap;
          if (cudaMemsetAsync(hs.A, 0, nslots * hs.side * sizeof(uint32_t), s) != cudaSuccess) { st = fail(PB_ERR_CUDA, "memset"); break; }
        } else {
          hs.hkey = reinterpret_cast<uint32_t *>(sp);
          hs.hval = hs.hkey + nslots * hs.hcap;
          hs.T = hs.hval + nslots * hs.hcap;
          hs.tcnt = hs.T + nslots * tlist;
          if (cudaMemsetAsync(hs.hkey, 0xff, nslots * hs.hcap * sizeof(uint32_t), s) != cudaSuccess ||
              cudaMemsetAsync(hs.hval, 0, nslots * hs.hcap * sizeof(uint32_t), s) != cudaSuccess) { st = fail(PB_ERR_CUDA, "memset"); break; }
        }
        hs.item = hs.tcnt + 2 * nslots;
        if (cudaMemsetAsync(hs.tcnt, 0, 3 * nslots * sizeof(uint32_t), s) != cudaSuccess ||
            cudaMemsetAsync(a.acc + ACC_QHEAVY, 0, sizeof(unsigned long long), s) != cudaSuccess) { st = fail(PB_ERR_CUDA, "memset"); break; }
        if (one) {
          PB_LAUNCH(okern, static_cast<unsigned>(nslots), H1_THREADS, hsmem, s, a, pt.list, pt.cnt, hs,
                    (const uint64_t *)nullptr, (const CArgs *)nullptr);
        } else if ((st = launch_cluster(ckern, static_cast<unsigned>(nslots * cl), HB_THREADS, cl, hsmem, s, a, pt.list,
                                        pt.cnt, hs, (const uint64_t *)nullptr, (const CArgs *)nullptr)) != PB_OK) {
          break;
        }
      }
      if (st != PB_OK) break;
      ph.finish(s, ts.w[3]);
    }
  } while (0);
  dfree(light, s); dfree(med, s); dfree(large, s); dfree(heavy, s); dfree(hkeys, s);
  return st;
}

__global__ void k_iota(uint32_t *__restrict__ a, uint64_t n) {
  for (size_t i = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += static_cast<size_t>(gridDim.x) * blockDim.x)
    a[i] = static_cast<uint32_t>(i);
}

__global__ void k_gather_u64(const unsigned long long *__restrict__ v, const uint32_t *__restrict__ idx, uint64_t n,
                             uint64_t *__restrict__ out) {
  for (size_t i = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += static_cast<size_t>(gridDim.x) * blockDim.x)
    out[i] = v[idx[i]];
}

// Run r (keys equal, sorted) adds its sum -- a difference of the prefix sums
// -- to target[key]; keys are unique per run, so no atomics.
__global__ void k_apply_runs(const uint64_t *__restrict__ ukey, const uint32_t *__restrict__ rstart, uint32_t nr,
                             uint64_t cnt, const uint64_t *__restrict__ pre, unsigned long long *__restrict__ target) {
  for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < nr; r += gridDim.x * blockDim.x) {
    const uint64_t b = rstart[r], e = r + 1 < nr ? rstart[r + 1] : cnt;
    target[ukey[r]] += pre[e] - pre[b];
  }
}

// Sorts (key, value) pairs by key and adds each key's total into target.
static pb_status reaggregate(uint64_t *keys, unsigned long long *vals, uint64_t cnt, int bits,
                             unsigned long long *target, cudaStream_t s) {
  if (cnt == 0) return PB_OK;
  uint32_t *idx = nullptr, *head = nullptr, *cid = nullptr, *rstart = nullptr;
  uint64_t *sv = nullptr, *pre = nullptr, *ukey = nullptr;
  pb_status st = PB_OK;
  do {
    if ((st = dalloc_t(&idx, cnt, s)) != PB_OK || (st = dalloc_t(&sv, cnt, s)) != PB_OK ||
        (st = dalloc_t(&pre, cnt + 1, s)) != PB_OK || (st = dalloc_t(&head, cnt, s)) != PB_OK ||
        (st = dalloc_t(&cid, cnt + 1, s)) != PB_OK || (st = dalloc_t(&ukey, cnt, s)) != PB_OK ||
        (st = dalloc_t(&rstart, cnt, s)) != PB_OK) break;
    k_iota<<<grid_for(cnt, 256, 8192), 256, 0, s>>>(idx, cnt);
    count_launch();
    if ((st = radix_sort(keys, idx, cnt, bits, s)) != PB_OK) break;
    k_gather_u64<<<grid_for(cnt, 256, 8192), 256, 0, s>>>(vals, idx, cnt, sv);
    count_launch();
    if ((st = scan_u64(sv, pre, cnt, s)) != PB_OK) break;
    k_heads<<<grid_for(cnt, 256, 8192), 256, 0, s>>>(keys, cnt, head);
    count_launch();
    if ((st = scan_u32(head, cid, cnt, s)) != PB_OK) break;
    uint32_t nr = 0;
    if (cudaMemcpyAsync(&nr, cid + cnt, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) { st = fail(PB_ERR_CUDA, "re-aggregation readback"); break; }
    k_runs<<<grid_for(cnt, 256, 8192), 256, 0, s>>>(keys, head, cid, cnt, ukey, rstart);
    count_launch();
    k_apply_runs<<<grid_for(nr, 256, 8192), 256, 0, s>>>(ukey, rstart, nr, cnt, pre, target);
    count_launch();
  } while (0);
  dfree(idx, s); dfree(sv, s); dfree(pre, s); dfree(head, s); dfree(cid, s); dfree(ukey, s); dfree(rstart, s);
  return st;
}

template <bool PV, bool PE, bool RE>
static pb_status run_sort_global(pb_graph *g, const CArgs &a, uint64_t budget, uint64_t olo, uint64_t ohi,
                                 cudaStream_t s) {
  const uint64_t n = g->n;
  const int bitsN = g->bitsN;
  // bytes per wedge: key, radix ping-pong key, head, run id, run key, run start, run d
  uint64_t per_wedge = 8 + 8 + 4 + 4 + 8 + 4 + 4;
  // Re-aggregation: at most 2 (key, value) pairs per wedge per output (run
  // sums give 2 per run of >= 2 wedges; centres give one per wedge and one per
  // (owner, centre) pair), plus reaggregate()'s temporaries for one sink
  // (index, value, prefix, head, run id, run key, run start, radix ping-pong).
  const uint64_t SINK_PER_WEDGE = 2;
  if (RE) per_wedge += SINK_PER_WEDGE * (16 * ((PV ? 1 : 0) + (PE ? 1 : 0)) + 4 + 8 + 8 + 4 + 4 + 8 + 4 + 12);
  uint64_t cap = budget / per_wedge;
  if (cap > (uint64_t(1) << 31)) cap = uint64_t(1) << 31;
  const uint64_t maxw = a.rev ? g->maxw_rev : g->maxw;
  if (cap < maxw) return fail(PB_ERR_SCRATCH, "sort aggregation: one owner has %llu wedges, budget holds %llu",
                              (unsigned long long)maxw, (unsigned long long)cap);
  unsigned long long *dchunk = nullptr;
  uint64_t *keys = nullptr, *ukey = nullptr;
  uint32_t *head = nullptr, *cid = nullptr, *rstart = nullptr, *ud = nullptr, *seg = nullptr;
  pb_status st = PB_OK;
  uint64_t cap_alloc = cap < g->W ? cap : g->W;
  if (cap_alloc == 0) return PB_OK;
  Sink sk{};
  do {
    if ((st = dalloc_t(&dchunk, 2, s)) != PB_OK) break;
    if ((st = dalloc_t(&keys, cap_alloc, s)) != PB_OK) break;
    if ((st = dalloc_t(&head, cap_alloc, s)) != PB_OK) break;
    if ((st = dalloc_t(&cid, cap_alloc + 1, s)) != PB_OK) break;
    if ((st = dalloc_t(&ukey, cap_alloc, s)) != PB_OK) break;
    if ((st = dalloc_t(&rstart, cap_alloc, s)) != PB_OK) break;
    if ((st = dalloc_t(&ud, cap_alloc, s)) != PB_OK) break;
    if (RE) {
      sk.vcap = PV ? SINK_PER_WEDGE * cap_alloc : 0;
      sk.ecap = PE ? SINK_PER_WEDGE * cap_alloc : 0;
      if ((st = dalloc_t(&sk.vcnt, 2, s)) != PB_OK) break;
      sk.ecnt = sk.vcnt + 1;
      if (PV && ((st = dalloc_t(&sk.vkey, sk.vcap, s)) != PB_OK || (st = dalloc_t(&sk.vval, sk.vcap, s)) != PB_OK))
        break;
      if (PE && ((st = dalloc_t(&sk.ekey, sk.ecap, s)) != PB_OK || (st = dalloc_t(&sk.eval, sk.ecap, s)) != PB_OK))
        break;
    }
    const int sms = sm_count(g->device);
    uint32_t lo = static_cast<uint32_t>(olo);
    while (lo < ohi && st == PB_OK) {
      k_chunk_end<<<1, 1, 0, s>>>(a.wpre, ohi, lo, cap, dchunk);
      count_launch();
      unsigned long long hc[2];
      if (cudaMemcpyAsync(hc, dchunk, sizeof(hc), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
          cudaStreamSynchronize(s) != cudaSuccess) { st = fail(PB_ERR_CUDA, "chunk readback"); break; }
      const uint32_t hi = static_cast<uint32_t>(hc[0]);
      const uint64_t cnt = hc[1];
      if (cnt > 0) {
        uint64_t wbase = 0;
        if (cudaMemcpyAsync(&wbase, a.wpre + lo, sizeof(uint64_t), cudaMemcpyDeviceToHost, s) != cudaSuccess) { st = fail(PB_ERR_CUDA, "readback"); break; }
        cudaStreamSynchronize(s);
        if (cudaMemsetAsync(a.acc + ACC_QMED, 0, sizeof(unsigned long long), s) != cudaSuccess) { st = fail(PB_ERR_CUDA, "memset"); break; }
        if (RE && cudaMemsetAsync(sk.vcnt, 0, 2 * sizeof(unsigned long long), s) != cudaSuccess) { st = fail(PB_ERR_CUDA, "memset"); break; }
        unsigned grid = static_cast<unsigned>(sms * 4);
        if (grid > hi - lo) grid = hi - lo;
        k_sort_walk<PV, PE, true, false><<<grid, MB_THREADS, 0, s>>>(a, lo, hi, wbase, bitsN, keys, nullptr, nullptr,
                                                                     nullptr, sk);
        count_launch();
        int kbits = bits_for(hi - lo - 1) + bitsN;
        if ((st = radix_sort(keys, nullptr, cnt, kbits, s)) != PB_OK) break;
        k_heads<<<grid_for(cnt, 256, 8192), 256, 0, s>>>(keys, cnt, head);
        count_launch();
        if ((st = scan_u32(head, cid, cnt, s)) != PB_OK) break;
        uint32_t nr = 0;
        if (cudaMemcpyAsync(&nr, cid + cnt, sizeof(uint32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) { st = fail(PB_ERR_CUDA, "run count readback"); break; }
        k_runs<<<grid_for(cnt, 256, 8192), 256, 0, s>>>(keys, head, cid, cnt, ukey, rstart);
        count_launch();
        k_run_sums<PV, RE><<<grid_for(nr, 256, 4096), 256, 0, s>>>(a, ukey, rstart, nr, static_cast<uint32_t>(cnt),
                                                                   lo, bitsN, ud, sk);
        count_launch();
        if (PV || PE) {
          dfree(seg, s);
          seg = nullptr;
          if ((st = dalloc_t(&seg, (hi - lo) + 1, s)) != PB_OK) break;
          k_segments<<<grid_for(hi - lo + 1, 256, 4096), 256, 0, s>>>(ukey, nr, hi - lo, bitsN, seg);
          count_launch();
          if (cudaMemsetAsync(a.acc + ACC_QMED, 0, sizeof(unsigned long long), s) != cudaSuccess) { st = fail(PB_ERR_CUDA, "memset"); break; }
          k_sort_walk<PV, PE, false, RE><<<grid, MB_THREADS, 0, s>>>(a, lo, hi, wbase, bitsN, nullptr, ukey, ud, seg,
                                                                     sk);
          count_launch();
        }
        if (RE && (PV || PE)) {
          // Butterfly re-aggregation of this chunk: sort the emitted pairs by
          // key and add each key's total once.
          unsigned long long hn[2] = {0, 0};
          if (cudaMemcpyAsync(hn, sk.vcnt, sizeof(hn), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
              cudaStreamSynchronize(s) != cudaSuccess) { st = fail(PB_ERR_CUDA, "sink count readback"); break; }
          if (hn[0] > sk.vcap || hn[1] > sk.ecap) { st = fail(PB_ERR_SCRATCH, "re-aggregation sink overflow"); break; }
          if (PV && (st = reaggregate(sk.vkey, sk.vval, hn[0], bits_for(n), a.pv, s)) != PB_OK) break;
          if (PE && (st = reaggregate(sk.ekey, sk.eval, hn[1], bits_for(2 * g->m), a.es, s)) != PB_OK) break;
        }
        if (cudaGetLastError() != cudaSuccess) { st = fail(PB_ERR_CUDA, "sort aggregation kernels failed to launch"); break; }
      }
      lo = hi;
    }
  } while (0);
  dfree(dchunk, s); dfree(keys, s); dfree(head, s); dfree(cid, s); dfree(ukey, s); dfree(rstart, s);
  dfree(ud, s); dfree(seg, s);
  dfree(sk.vcnt, s); dfree(sk.vkey, s); dfree(sk.vval, s); dfree(sk.ekey, s); dfree(sk.eval, s);
  return st;
}

// Sort aggregation: owners of at most SS_MAX wedges sort in shared memory
// (k_sort_small); the rest materialise their wedge keys chunk by chunk under
// the budget and sort them in device memory (run_sort_global), over a wedge
// prefix that counts only those owners.  Re-aggregation keeps every owner on
// the device-wide path (its contributions go through the sorted sinks).
template <bool PV, bool PE, bool RE>
static pb_status run_sort(pb_graph *g, const CArgs &a, uint64_t budget, uint64_t olo, uint64_t ohi,
                          cudaStream_t s) {
  if (RE) return run_sort_global<PV, PE, RE>(g, a, budget, olo, ohi, s);
  const uint64_t n = g->n;
  if (ohi > olo) {
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sort_small<PV, PE>, SS_THREADS, 0);
    uint64_t grid = static_cast<uint64_t>(sm_count(g->device)) * (per_sm > 0 ? per_sm : 1);
    if (grid > ohi - olo) grid = ohi - olo;
    PB_CUDA(cudaMemsetAsync(a.acc + ACC_QLARGE, 0, sizeof(unsigned long long), s));
    PB_LAUNCH((k_sort_small<PV, PE>), static_cast<unsigned>(grid), SS_THREADS, 0, s, a, static_cast<uint32_t>(olo),
              static_cast<uint32_t>(ohi));
  }
  uint64_t *wl = nullptr, *wpl = nullptr;
  pb_status st = PB_OK;
  do {
    if ((st = dalloc_t(&wl, n + 1, s)) != PB_OK || (st = dalloc_t(&wpl, n + 1, s)) != PB_OK) break;
    k_wedges_large<<<grid_for(n, 256, 8192), 256, 0, s>>>(a.wpre, n, wl);
    count_launch();
    if ((st = scan_u64(wl, wpl, n, s)) != PB_OK) break;
    CArgs al = a;
    al.wpre = wpl;
    st = run_sort_global<PV, PE, false>(g, al, budget, olo, ohi, s);
  } while (0);
  dfree(wl, s);
  dfree(wpl, s);
  return st;
}

pb_status count_all(pb_graph *g, int agg, uint64_t scratch_bytes, const CountOut &o, cudaStream_t s) {
  PB_TRY(ensure_ranked(g, s));
  if (agg < 0 || agg > PB_AGG_AUTO) return fail(PB_ERR_INVALID, "unknown aggregation %d", agg);
  if (g->butterfly_agg == PB_BFLY_SORT && agg != PB_AGG_SORT)
    return fail(PB_ERR_INVALID, "butterfly re-aggregation by sorting needs wedge aggregation PB_AGG_SORT");
  const uint64_t n = g->n, na = 2 * g->m;
  const bool want_pv = o.U || o.V, want_pe = o.E != nullptr;
  uint64_t budget = scratch_bytes ? scratch_bytes : (uint64_t(16) << 30);
  if (!g->acc) PB_TRY(dalloc_t(&g->acc, ACC_WORDS, s));
  PB_CUDA(cudaMemsetAsync(g->acc, 0, ACC_WORDS * sizeof(unsigned long long), s));
  if (want_pv) {
    if (!g->pv) PB_TRY(dalloc_t(&g->pv, n + 1, s));
    PB_CUDA(cudaMemsetAsync(g->pv, 0, (n + 1) * sizeof(uint64_t), s));
  }
  if (want_pe) {
    if (!g->es) PB_TRY(dalloc_t(&g->es, na + 1, s));
    PB_CUDA(cudaMemsetAsync(g->es, 0, (na + 1) * sizeof(uint64_t), s));
    if (!g->es32) PB_TRY(dalloc_t(&g->es32, na + 1, s));
    PB_CUDA(cudaMemsetAsync(g->es32, 0, (na + 1) * sizeof(uint32_t), s));
  }
  CArgs a;
  // Owner of each wedge: its lower-ranked endpoint (Algorithm 2) or, with the
  // cache optimisation, its higher-ranked one.  Same wedges either way.
  pb_plan_t plan;
  if (g->has_plan) plan = g->plan;  // pinned by pb_set_plan
  else make_plan_basic(g, &plan);
  a.rev = g->retrieval == PB_RETRIEVE_AUTO ? plan.retrieval == PB_RETRIEVE_HIGH : g->retrieval == PB_RETRIEVE_HIGH;
  a.off = g->off; a.adj = g->adj; a.cpos = g->cpos; a.degp = g->degp; a.n = n;
  a.wpre = a.rev ? g->wpre_rev : g->wpre;
  a.nU = g->nU;
  a.pv = want_pv ? reinterpret_cast<unsigned long long *>(g->pv) : nullptr;
  a.es = want_pe ? reinterpret_cast<unsigned long long *>(g->es) : nullptr;
  a.es32 = want_pe ? reinterpret_cast<unsigned int *>(g->es32) : nullptr;
  // y's list takes 32-bit partials when (deg(y) - 1)(largest degree on the
  // entries' side - 1) stays within 32 bits
  a.nlim[0] = g->maxdegU > 1 ? static_cast<uint32_t>(0xffffffffull / (g->maxdegU - 1)) : 0xffffffffu;
  a.nlim[1] = g->maxdegV > 1 ? static_cast<uint32_t>(0xffffffffull / (g->maxdegV - 1)) : 0xffffffffu;
  a.acc = g->acc;
  if (g->W > 0) {
    Plan p;
    p.pv = want_pv;
    p.pe = want_pe;
    p.owner_lo = o.owner_lo < n ? o.owner_lo : n;
    p.owner_hi = o.owner_hi < n ? o.owner_hi : n;
    pb_status st;
    if (agg == PB_AGG_SORT) {
      PhaseScope ph(PB_PHASE_SORT, s);
      const bool re = g->butterfly_agg == PB_BFLY_SORT;
      if (want_pv && want_pe)
        st = re ? run_sort<true, true, true>(g, a, budget, p.owner_lo, p.owner_hi, s)
                : run_sort<true, true, false>(g, a, budget, p.owner_lo, p.owner_hi, s);
      else if (want_pv)
        st = re ? run_sort<true, false, true>(g, a, budget, p.owner_lo, p.owner_hi, s)
                : run_sort<true, false, false>(g, a, budget, p.owner_lo, p.owner_hi, s);
      else if (want_pe)
        st = re ? run_sort<false, true, true>(g, a, budget, p.owner_lo, p.owner_hi, s)
                : run_sort<false, true, false>(g, a, budget, p.owner_lo, p.owner_hi, s);
      else st = run_sort<false, false, false>(g, a, budget, p.owner_lo, p.owner_hi, s);
      if (st == PB_OK) ph.finish(s, g->W);
    } else {
      // The plan's tier bounds; the statistics under them (one readback, the
      // only host wait before the outputs); the rest of the plan from them
      // unless one is pinned.
      p.light_max = plan.light_max;
      p.med_max = plan.med_max;
      p.large_max = plan.large_max;
      TierStats ts;
      PB_TRY(tier_stats(g, a.rev, p.owner_lo, p.owner_hi, p.light_max, p.med_max, p.large_max, s, &ts));
      if (!g->has_plan) {
        plan_from_stats(g, ts, budget, &plan);
        p.med_max = plan.med_max;  // the plan may move the mid-size owners to the large tier
        p.large_max = plan.large_max;
      }
      p.hot = plan.hot;
      const int heavy = agg == PB_AGG_AUTO ? plan.agg : agg;
      p.heavy = heavy;
      p.cluster = 1;
      if (heavy == PB_AGG_HIST) {
        // HIST gives hubs a cluster: the pinned or planned size, else two
        // blocks once the largest owner passes HUB_MAX wedges
        if (agg == PB_AGG_AUTO) p.cluster = plan.hub_cluster;
        else if (ts.hmaxw > HUB_MAX) p.cluster = 2;
      }
      if (p.cluster < 1) p.cluster = 1;
      if (p.cluster > 16) p.cluster = 16;
      if (want_pv && want_pe) st = run_tiers<true, true>(g, a, p, ts, budget, s);
      else if (want_pv) st = run_tiers<true, false>(g, a, p, ts, budget, s);
      else if (want_pe) st = run_tiers<false, true>(g, a, p, ts, budget, s);
      else st = run_tiers<false, false>(g, a, p, ts, budget, s);
    }
    PB_TRY(st);
  }
  unsigned long long hacc[ACC_WORDS] = {0};
  PB_CUDA(cudaMemcpyAsync(hacc, g->acc, sizeof(hacc), cudaMemcpyDeviceToHost, s));
  // outputs
  uint64_t *dU = o.U, *dV = o.V, *dE = o.E, *tmp = nullptr;
  if (!o.on_device && (want_pv || want_pe)) {
    size_t cnt = (want_pv ? n : 0) + (want_pe ? g->m_in : 0);
    PB_TRY(dalloc_t(&tmp, cnt + 1, s));
    uint64_t *q = tmp;
    if (want_pv) { dU = o.U ? q : nullptr; dV = o.V ? q + g->nU : nullptr; q += n; }
    if (want_pe) dE = q;
  }
  pb_status st = PB_OK;
  PhaseScope ph_out(PB_PHASE_OUTPUT, s);
  if (want_pv && n) {
    k_out_vertex<<<grid_for(n, 256, 8192), 256, 0, s>>>(reinterpret_cast<unsigned long long *>(g->pv), g->label,
                                                         g->nU, g->nV, dU, dV);
    count_launch();
  }
  uint64_t *Ecan = nullptr;
  if (want_pe && g->m_in) {
    st = dalloc_t(&Ecan, g->m + 1, s);
    if (st == PB_OK) {
      k_edge_sums<<<grid_for(g->m, 256, 8192), 256, 0, s>>>(reinterpret_cast<unsigned long long *>(g->es),
                                                            reinterpret_cast<unsigned int *>(g->es32), g->slotA,
                                                            g->slotB, g->m, Ecan);
      count_launch();
      k_out_edge<<<grid_for(g->m_in, 256, 8192), 256, 0, s>>>(Ecan, g->in2c, g->m_in, dE);
      count_launch();
    }
  }
  if (cudaGetLastError() != cudaSuccess) st = fail(PB_ERR_CUDA, "output kernels failed to launch");
  if (st == PB_OK && !o.on_device) {
    cudaError_t e = cudaSuccess;
    if (o.U && n) e = cudaMemcpyAsync(o.U, dU, g->nU * sizeof(uint64_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && o.V && n) e = cudaMemcpyAsync(o.V, dV, g->nV * sizeof(uint64_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && o.E && g->m_in) e = cudaMemcpyAsync(o.E, dE, g->m_in * sizeof(uint64_t), cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) st = cuda_fail(e, "output download", __FILE__, __LINE__);
  }
  dfree(Ecan, s);
  dfree(tmp, s);
  if (st == PB_OK) ph_out.finish(s);
  cudaError_t e = cudaStreamSynchronize(s);
  if (st != PB_OK) return st;
  if (e != cudaSuccess) return cuda_fail(e, "counting kernels", __FILE__, __LINE__);
  if (hacc[ACC_ERR]) return fail(PB_ERR_SCRATCH, "aggregation table overflow (code %llu)", hacc[ACC_ERR]);
  if (hacc[ACC_OVF]) return fail(PB_ERR_OVERFLOW, "global butterfly count exceeds 2^64");
  if (o.global) *o.global = hacc[0];
  return PB_OK;
}

}  // namespace pb

namespace pb {

// ---------------------------------------------------------------------------
// Autotuner (rules from degree and wedge statistics).  The part that needs no
// device pass: ranking recommendation, owner direction, default tiers.
void make_plan_basic(const pb_graph *g, pb_plan_t *plan) {
  *plan = pb_plan_t{};
  const uint64_t w_side = g->w_side_U < g->w_side_V ? g->w_side_U : g->w_side_V;
  plan->W_side = w_side;
  plan->W_rank = g->W;
  plan->f_side = w_side ? (static_cast<double>(w_side) - static_cast<double>(g->W)) / static_cast<double>(w_side) : 0.0;
  // side order when the ranking saves under 10% of its wedges (Table 3's rule)
  plan->rank_kind = plan->f_side < 0.1 ? PB_RANK_SIDE : (g->rank_kind >= 0 && g->rank_kind <= 4 ? g->rank_kind
                                                                                                   : PB_RANK_DEGREE);
  const bool high = g->maxw_rev <= g->maxw;
  plan->retrieval = high ? PB_RETRIEVE_HIGH : PB_RETRIEVE_LOW;
  plan->max_owner_wedges = high ? g->maxw_rev : g->maxw;
  plan->agg = PB_AGG_BATCH;
  plan->light_max = LIGHT_MAX;
  plan->med_max = MED_MAX;
  plan->large_max = LARGE_MAX;
  plan->hot = HOT_SMALL;
  plan->hub_min = UINT64_MAX;
  plan->hub_cluster = 1;
}

// The whole plan (pb_autotune): the basic part, then the statistics of the
// owners under the chosen direction.
pb_status make_plan(pb_graph *g, uint64_t budget, cudaStream_t s, pb_plan_t *plan) {
  make_plan_basic(g, plan);
  if (g->W == 0) {
    plan->scratch_bytes = budget;
    return PB_OK;
  }
  TierStats ts;
  unsigned long long *buf = nullptr;
  PB_TRY(dalloc_t(&buf, TS_WORDS, s));
  const pb_status st = tier_stats(g, plan->retrieval == PB_RETRIEVE_HIGH, 0, g->n, plan->light_max, plan->med_max,
                                  plan->large_max, s, &ts, buf);
  dfree(buf, s);
  PB_TRY(st);
  plan_from_stats(g, ts, budget, plan);
  return PB_OK;
}

}  // namespace pb

// ---------------------------------------------------------------------------
// Batched counting across graphs.
struct pb_batch {
  int device = 0;
  uint32_t ng = 0;
  bool pv = false;
  std::vector<pb_graph *> graphs;
  std::vector<uint64_t> pv_off;          // start of each graph's counts in pvbuf
  pb::CArgs *tab = nullptr;               // [ng] device
  unsigned long long *acc = nullptr;      // [ng][ACC_WORDS] per-graph accumulators
  unsigned long long *bacc = nullptr;     // [ACC_WORDS] batch work queues
  unsigned long long *pvbuf = nullptr;    // per-vertex counts, all graphs
  uint64_t pv_total = 0;
  uint64_t *light = nullptr, *med = nullptr, *large = nullptr, *heavy = nullptr, *heavy_h = nullptr;
  uint32_t nl = 0, nm = 0, nq = 0, nh = 0, nhh = 0;  // nh: dense heavy owners, nhh: hashed heavy owners
  pb::HeavySlots hs = {}, hsh = {};          // dense and hashed heavy slots
  void *scratch = nullptr, *scratch_h = nullptr, *scratch_m = nullptr;
  pb::HeavySlots hsm = {};                   // large-tier slots
  uint64_t nslots_m = 0;
  uint64_t nslots = 0, slot_bytes = 0, nslots_h = 0, slot_bytes_h = 0;
  std::vector<int32_t> agg;                  // per graph: the heavy path its plan chose
  uint64_t W = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

namespace pb {

__global__ void k_tag_items(const uint32_t *__restrict__ list, uint32_t cnt, uint32_t gid,
                            uint64_t *__restrict__ out) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += gridDim.x * blockDim.x)
    out[i] = (static_cast<uint64_t>(gid) << 32) | list[i];
}

static void batch_release(pb_batch *b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  cudaStream_t s = 0;
  dfree(b->tab, s); dfree(b->acc, s); dfree(b->bacc, s); dfree(b->pvbuf, s);
  dfree(b->light, s); dfree(b->med, s); dfree(b->large, s); dfree(b->heavy, s); dfree(b->scratch, s);
  dfree(b->heavy_h, s); dfree(b->scratch_h, s); dfree(b->scratch_m, s);
  cudaStreamSynchronize(s);
  cudaGetLastError();
  delete b;
}

template <bool PV>
static pb_status batch_capture_on(pb_batch *b, cudaStream_t s);

// The launches are recorded on a private stream (the legacy default stream
// cannot be captured); the resulting graph is launched on any stream.
template <bool PV>
static pb_status batch_capture(pb_batch *b) {
  cudaStream_t cs = nullptr;
  PB_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  pb_status st = batch_capture_on<PV>(b, cs);
  cudaStreamDestroy(cs);
  return st;
}

template <bool PV>
static pb_status batch_capture_on(pb_batch *b, cudaStream_t s) {
  const int sms = sm_count(b->device);
  CArgs a0 = {};
  a0.acc = b->bacc;
  PB_CUDA(cudaFuncSetAttribute(k_light<PV, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)(LW_WARPS * (LW_CAP + LW_CAP / 2) * sizeof(uint32_t))));
  PB_CUDA(cudaFuncSetAttribute(k_medium<PV, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)MB_SMEM));
  PB_CUDA(cudaFuncSetAttribute(k_large<PV, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)(hot_words(MH_HOT, true) * sizeof(uint32_t))));
  PB_CUDA(cudaFuncSetAttribute(k_heavy1<PV, false, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)(b->hs.hot * sizeof(uint32_t))));
  PB_CUDA(cudaFuncSetAttribute(k_heavy1<PV, false, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)(b->hsh.hot * sizeof(uint32_t))));
  PB_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  pb_status st = PB_OK;
  do {
    cudaError_t e1 = cudaMemsetAsync(b->acc, 0, sizeof(unsigned long long) * ACC_WORDS * b->ng, s);
    if (e1 != cudaSuccess) { st = cuda_fail(e1, "batch memset (accumulators)", __FILE__, __LINE__); break; }
    e1 = cudaMemsetAsync(b->bacc, 0, sizeof(unsigned long long) * ACC_WORDS, s);
    if (e1 != cudaSuccess) { st = cuda_fail(e1, "batch memset (queues)", __FILE__, __LINE__); break; }
    if (PV) {
      e1 = cudaMemsetAsync(b->pvbuf, 0, sizeof(unsigned long long) * (b->pv_total + 1), s);
      if (e1 != cudaSuccess) { st = cuda_fail(e1, "batch memset (per-vertex)", __FILE__, __LINE__); break; }
    }
    if (b->nl) {
      const size_t smem = LW_WARPS * (LW_CAP + LW_CAP / 2) * sizeof(uint32_t);
      int per_sm = 0;
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_light<PV, false, true>, LW_THREADS, smem);
      unsigned grid = static_cast<unsigned>(sms * (per_sm > 0 ? per_sm : 1));
      unsigned need = (b->nl + LW_WARPS - 1) / LW_WARPS;
      k_light<PV, false, true><<<grid < need ? grid : need, LW_THREADS, smem, s>>>(a0, nullptr, b->nl, b->light, b->tab);
      count_launch();
      e1 = cudaGetLastError();
      if (e1 != cudaSuccess) { st = cuda_fail(e1, "batch light launch", __FILE__, __LINE__); break; }
    }
    if (b->nm) {
      const size_t smem = MB_SMEM;
      int per_sm = 0;
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_medium<PV, false, true>, MB_THREADS, smem);
      unsigned grid = static_cast<unsigned>(sms * (per_sm > 0 ? per_sm : 1));
      k_medium<PV, false, true><<<grid < b->nm ? grid : b->nm, MB_THREADS, smem, s>>>(a0, nullptr, b->nm, b->med, b->tab);
      count_launch();
      e1 = cudaGetLastError();
      if (e1 != cudaSuccess) { st = cuda_fail(e1, "batch medium launch", __FILE__, __LINE__); break; }
    }
    if (b->nq) {
      const size_t hb = b->nslots_m * b->hsm.hcap * sizeof(uint32_t);
      e1 = cudaMemsetAsync(b->hsm.hkey, 0xff, hb, s);
      if (e1 == cudaSuccess) e1 = cudaMemsetAsync(b->hsm.hval, 0, hb, s);
      if (e1 != cudaSuccess) { st = cuda_fail(e1, "batch memset (large slots)", __FILE__, __LINE__); break; }
      k_large<PV, false, true><<<static_cast<unsigned>(b->nslots_m), MH_THREADS,
                                 hot_words(MH_HOT, true) * sizeof(uint32_t), s>>>(a0, nullptr, b->nq, b->hsm, b->large,
                                                                                   b->tab);
      count_launch();
      e1 = cudaGetLastError();
      if (e1 != cudaSuccess) { st = cuda_fail(e1, "batch large launch", __FILE__, __LINE__); break; }
    }
    if (b->nh) {
      e1 = cudaMemsetAsync(b->scratch, 0, b->nslots * b->slot_bytes + b->nslots * 7 * sizeof(uint32_t) + 64, s);
      if (e1 != cudaSuccess) { st = cuda_fail(e1, "batch memset (slots)", __FILE__, __LINE__); break; }
      k_heavy1<PV, false, true, false><<<static_cast<unsigned>(b->nslots), H1_THREADS, b->hs.hot * sizeof(uint32_t),
                                         s>>>(a0, nullptr, b->nh, b->hs, b->heavy, b->tab);
      count_launch();
      e1 = cudaGetLastError();
      if (e1 != cudaSuccess) { st = cuda_fail(e1, "batch heavy launch", __FILE__, __LINE__); break; }
    }
    if (b->nhh) {  // graphs whose plan hashes the heavy owners' cold endpoints: own slots, own queue
      const size_t hb = b->nslots_h * b->hsh.hcap * sizeof(uint32_t);
      e1 = cudaMemsetAsync(b->hsh.hkey, 0xff, hb, s);
      if (e1 == cudaSuccess) e1 = cudaMemsetAsync(b->hsh.hval, 0, hb, s);
      if (e1 == cudaSuccess) e1 = cudaMemsetAsync(b->hsh.tcnt, 0, 3 * b->nslots_h * sizeof(uint32_t), s);
      if (e1 == cudaSuccess) e1 = cudaMemsetAsync(b->bacc + ACC_QHEAVY, 0, sizeof(unsigned long long), s);
      if (e1 != cudaSuccess) { st = cuda_fail(e1, "batch memset (hashed slots)", __FILE__, __LINE__); break; }
      k_heavy1<PV, false, true, true><<<static_cast<unsigned>(b->nslots_h), H1_THREADS,
                                        b->hsh.hot * sizeof(uint32_t), s>>>(a0, nullptr, b->nhh, b->hsh, b->heavy_h,
                                                                            b->tab);
      count_launch();
      e1 = cudaGetLastError();
      if (e1 != cudaSuccess) { st = cuda_fail(e1, "batch hashed heavy launch", __FILE__, __LINE__); break; }
    }
  } while (0);
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamEndCapture(s, &graph);
  if (st != PB_OK) {
    if (graph) cudaGraphDestroy(graph);
    return st;
  }
  if (e != cudaSuccess) return cuda_fail(e, "batch capture", __FILE__, __LINE__);
  b->graph = graph;
  PB_CUDA(cudaGraphInstantiate(&b->exec, graph, 0));
  return PB_OK;
}

static pb_status batch_build(pb_batch *b, uint64_t budget, cudaStream_t s) {
  const uint32_t ng = b->ng;
  // per-graph argument table and output buffers
  std::vector<CArgs> host_tab(ng);
  b->pv_off.resize(ng);
  b->agg.assign(ng, PB_AGG_BATCH);
  uint64_t total_n = 0, max_side = 1;
  for (uint32_t i = 0; i < ng; i++) {
    pb_graph *g = b->graphs[i];
    b->pv_off[i] = total_n;
    total_n += g->n;
    uint64_t side = g->nU > g->nV ? g->nU : g->nV;
    if (side > max_side) max_side = side;
  }
  b->pv_total = total_n;
  PB_TRY(dalloc_t(&b->acc, static_cast<size_t>(ng) * ACC_WORDS, s));
  PB_TRY(dalloc_t(&b->bacc, ACC_WORDS, s));
  PB_TRY(dalloc_t(&b->pvbuf, total_n + 1, s));
  PB_TRY(dalloc_t(&b->light, total_n + 1, s));
  PB_TRY(dalloc_t(&b->med, total_n + 1, s));
  PB_TRY(dalloc_t(&b->large, total_n + 1, s));
  PB_TRY(dalloc_t(&b->heavy, total_n + 1, s));
  PB_TRY(dalloc_t(&b->heavy_h, total_n + 1, s));
  uint32_t *tl = nullptr, *tm = nullptr, *tq = nullptr;
  uint64_t *th = nullptr;
  unsigned long long *tacc = nullptr;
  pb_status st = PB_OK;
  // slot sizes over the graphs of each heavy path
  TierStats dmax, hmax;
  uint64_t large_max_all = 1;
  do {
    if ((st = dalloc_t(&tacc, ACC_WORDS, s)) != PB_OK) break;
    for (uint32_t i = 0; i < ng && st == PB_OK; i++) {
      pb_graph *g = b->graphs[i];
      // Each graph's own plan: owner direction, tier bounds and heavy path
      // from its statistics (or the plan pinned on it).
      pb_plan_t plan;
      if (g->has_plan) plan = g->plan;
      else make_plan_basic(g, &plan);
      CArgs &a = host_tab[i];
      a.rev = g->retrieval == PB_RETRIEVE_AUTO ? plan.retrieval == PB_RETRIEVE_HIGH : g->retrieval == PB_RETRIEVE_HIGH;
      a.off = g->off; a.adj = g->adj; a.cpos = g->cpos; a.degp = g->degp; a.n = g->n; a.nU = g->nU;
      a.wpre = a.rev ? g->wpre_rev : g->wpre;
      a.pv = b->pv ? b->pvbuf + b->pv_off[i] : nullptr;
      a.es = nullptr;
      a.es32 = nullptr;
      a.nlim[0] = a.nlim[1] = 0;
      a.acc = b->acc + static_cast<size_t>(i) * ACC_WORDS;
      b->W += g->W;
      if (g->W == 0) continue;
      const uint64_t n = g->n;
      TierStats ts;
      if ((st = tier_stats(g, a.rev, 0, n, plan.light_max, plan.med_max, plan.large_max, s, &ts)) != PB_OK) break;
      if (!g->has_plan) plan_from_stats(g, ts, budget, &plan);
      // a batch runs one kernel per tier over every graph: hub clusters are
      // not used, a graph's heavy owners take the dense or the hashed path
      const bool hashed = plan.agg == PB_AGG_HASH;
      b->agg[i] = hashed ? PB_AGG_HASH : PB_AGG_BATCH;
      const uint32_t cl = static_cast<uint32_t>(ts.n[0]), cm = static_cast<uint32_t>(ts.n[1]),
                     cq = static_cast<uint32_t>(ts.n[2]), ch = static_cast<uint32_t>(ts.n[3]);
      if ((st = dalloc_t(&tl, cl + 1, s)) != PB_OK || (st = dalloc_t(&tm, cm + 1, s)) != PB_OK ||
          (st = dalloc_t(&tq, cq + 1, s)) != PB_OK || (st = dalloc_t(&th, ch + 1, s)) != PB_OK) break;
      if (cudaMemsetAsync(tacc, 0, sizeof(unsigned long long) * ACC_WORDS, s) != cudaSuccess) { st = fail(PB_ERR_CUDA, "memset"); break; }
      const TierCaps caps = {{cl, cm, cq, ch}};
      k_classify<<<grid_for(n, 256, 8192), 256, 0, s>>>(a.wpre, n, 0, n, plan.light_max, plan.med_max, plan.large_max,
                                                        UINT64_MAX, tl, tm, tq, th, g->bitsN, tacc, caps);
      count_launch();
      if (cl) { k_tag_items<<<grid_for(cl, 256, 1024), 256, 0, s>>>(tl, cl, i, b->light + b->nl); count_launch(); }
      if (cm) { k_tag_items<<<grid_for(cm, 256, 1024), 256, 0, s>>>(tm, cm, i, b->med + b->nm); count_launch(); }
      if (cq) { k_tag_items<<<grid_for(cq, 256, 1024), 256, 0, s>>>(tq, cq, i, b->large + b->nq); count_launch(); }
      if (ch) {
        dfree(tl, s);
        tl = nullptr;
        if ((st = dalloc_t(&tl, ch + 1, s)) != PB_OK) break;
        k_keys_low<<<grid_for(ch, 256, 1024), 256, 0, s>>>(th, ch, g->bitsN, tl);
        count_launch();
        TierStats &mx = hashed ? hmax : dmax;
        const uint64_t side = g->nU > g->nV ? g->nU : g->nV;
        const uint64_t hr = ts.hrange ? ts.hrange : side;
        if (hr > mx.hrange) mx.hrange = hr;
        if (ts.hdist > mx.hdist) mx.hdist = ts.hdist;
        if (hashed) {
          k_tag_items<<<grid_for(ch, 256, 1024), 256, 0, s>>>(tl, ch, i, b->heavy_h + b->nhh);
          b->nhh += ch;
        } else {
          k_tag_items<<<grid_for(ch, 256, 1024), 256, 0, s>>>(tl, ch, i, b->heavy + b->nh);
          b->nh += ch;
        }
        count_launch();
      }
      b->nl += cl; b->nm += cm; b->nq += cq;
      if (cq && plan.large_max > large_max_all) large_max_all = plan.large_max;
      // the temporary lists are reused by the next graph only after these kernels
      if (cudaStreamSynchronize(s) != cudaSuccess) { st = fail(PB_ERR_CUDA, "batch classify"); break; }
      dfree(tl, s); dfree(tm, s); dfree(tq, s); dfree(th, s);
      tl = tm = tq = nullptr; th = nullptr;
    }
  } while (0);
  dfree(tl, s); dfree(tm, s); dfree(tq, s); dfree(th, s); dfree(tacc, s);
  if (st != PB_OK) return st;
  PB_TRY(dalloc_t(&b->tab, ng, s));
  PB_CUDA(cudaMemcpyAsync(b->tab, host_tab.data(), sizeof(CArgs) * ng, cudaMemcpyHostToDevice, s));
  const uint64_t resident = heavy1_resident(b->device, HB_HOT);
  if (b->nq) {
    large_slot_shape(large_max_all, &b->hsm);
    const size_t smem = hot_words(MH_HOT, true) * sizeof(uint32_t);
    PB_CUDA(cudaFuncSetAttribute(k_large<true, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem));
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_large<true, false, true>, MH_THREADS, smem);
    uint64_t ns = static_cast<uint64_t>(sm_count(b->device)) * (per_sm > 0 ? per_sm : 1);
    if (ns > b->nq) ns = b->nq;
    b->nslots_m = ns;
    PB_TRY(dalloc(&b->scratch_m, ns * large_slot_bytes(b->hsm) + 64, s));
    b->hsm.hkey = static_cast<uint32_t *>(b->scratch_m);
    b->hsm.hval = b->hsm.hkey + ns * b->hsm.hcap;
    b->hsm.T = b->hsm.hval + ns * b->hsm.hcap;
  }
  if (b->nh) {
    b->hs.side = dmax.hrange < max_side ? dmax.hrange : max_side;  // dense histograms span the owners' label ranges
    b->hs.tcap = dmax.hdist < b->hs.side ? dmax.hdist : b->hs.side;
    b->slot_bytes = (b->hs.side + b->hs.tcap) * sizeof(uint32_t);
    b->hs.hot = HB_HOT;
    uint64_t ns = resident;
    uint64_t fit = budget / (b->slot_bytes + 32);
    if (fit == 0) return fail(PB_ERR_SCRATCH, "batch scratch budget below one slot");
    if (ns > fit) ns = fit;
    if (ns > b->nh) ns = b->nh;
    b->nslots = ns;
    PB_TRY(dalloc(&b->scratch, ns * b->slot_bytes + ns * 7 * sizeof(uint32_t) + 64, s));
    char *sp = static_cast<char *>(b->scratch);
    b->hs.A = reinterpret_cast<uint32_t *>(sp);
    b->hs.T = b->hs.A + ns * b->hs.side;
    b->hs.tcnt = b->hs.T + ns * b->hs.tcap;
    b->hs.item = b->hs.tcnt + 2 * ns;
  }
  if (b->nhh) {
    b->hsh.tcap = hmax.hdist < max_side ? hmax.hdist : max_side;
    uint64_t cap = 32;
    while (cap < 2 * b->hsh.tcap) cap <<= 1;
    b->hsh.hcap = cap;
    b->slot_bytes_h = (2 * cap + b->hsh.tcap) * sizeof(uint32_t);
    b->hsh.hot = HB_HOT;
    uint64_t ns = resident;
    uint64_t fit = budget / (b->slot_bytes_h + 32);
    if (fit == 0) return fail(PB_ERR_SCRATCH, "batch scratch budget below one hashed slot");
    if (ns > fit) ns = fit;
    if (ns > b->nhh) ns = b->nhh;
    b->nslots_h = ns;
    PB_TRY(dalloc(&b->scratch_h, ns * b->slot_bytes_h + ns * 7 * sizeof(uint32_t) + 64, s));
    uint32_t *sp = static_cast<uint32_t *>(b->scratch_h);
    b->hsh.hkey = sp;
    b->hsh.hval = sp + ns * cap;
    b->hsh.T = b->hsh.hval + ns * cap;
    b->hsh.tcnt = b->hsh.T + ns * b->hsh.tcap;
    b->hsh.item = b->hsh.tcnt + 2 * ns;
  }
  PB_CUDA(cudaStreamSynchronize(s));
  return b->pv ? batch_capture<true>(b) : batch_capture<false>(b);
}

}  // namespace pb

using namespace pb;

extern "C" {

pb_status pb_autotune(const pb_graph *cg, uint64_t scratch_bytes, pb_plan_t *plan) {
  clear_error();
  if (!cg || !plan) return fail(PB_ERR_INVALID, "graph or plan is NULL");
  pb_graph *g = const_cast<pb_graph *>(cg);  // planning reads the graph; only its statistics buffer is written
  int cur = -1;
  cudaGetDevice(&cur);
  if (cur != g->device) cudaSetDevice(g->device);
  pb_status st = ensure_ranked(g, nullptr);
  if (st == PB_OK) st = make_plan(g, scratch_bytes ? scratch_bytes : (uint64_t(16) << 30), nullptr, plan);
  if (st == PB_OK && cudaStreamSynchronize(nullptr) != cudaSuccess) st = fail(PB_ERR_CUDA, "autotune");
  if (cur >= 0 && cur != g->device) cudaSetDevice(cur);
  return st;
}

pb_status pb_count_bytes(pb_graph *g, pb_agg agg, uint64_t scratch_bytes, int want_vertex, int want_edge,
                         int out_on_device, uint64_t *bytes) {
  clear_error();
  if (!g || !bytes) return fail(PB_ERR_INVALID, "graph or bytes is NULL");
  if (agg < PB_AGG_SORT || agg > PB_AGG_AUTO) return fail(PB_ERR_INVALID, "unknown aggregation %d", (int)agg);
  int cur = -1;
  cudaGetDevice(&cur);
  if (cur != g->device) cudaSetDevice(g->device);
  const uint64_t budget = scratch_bytes ? scratch_bytes : (uint64_t(16) << 30);
  const uint64_t n = g->n, m = g->m, na = 2 * m;
  constexpr uint64_t SLACK = uint64_t(2) << 20;  // per allocation: the pool's rounding
  uint64_t b = 0, allocs = 0;
  auto add = [&](uint64_t x) { b += x; allocs++; };
  pb_status st = ensure_ranked(g, nullptr);
  do {
    if (st != PB_OK) break;
    add(2 * TS_WORDS * 8);                       // counters and statistics
    if (want_vertex) add((n + 1) * 8);            // per-vertex accumulators
    if (want_edge) { add((na + 1) * 8); add((na + 1) * 4); add((m + 1) * 8); }  // per-slot, canonical edges
    if (!out_on_device && (want_vertex || want_edge))
      add(((want_vertex ? n : 0) + (want_edge ? g->m_in : 0) + 1) * 8);           // download staging
    if (g->W == 0) break;
    if (agg == PB_AGG_SORT) {
      add(budget);                               // the wedge chunk never exceeds the budget
      break;
    }
    pb_plan_t plan;
    if (g->has_plan) plan = g->plan;
    else make_plan_basic(g, &plan);
    const int rev = g->retrieval == PB_RETRIEVE_AUTO ? plan.retrieval == PB_RETRIEVE_HIGH
                                                      : g->retrieval == PB_RETRIEVE_HIGH;
    TierStats ts;
    unsigned long long *buf = nullptr;
    if ((st = dalloc_t(&buf, TS_WORDS, nullptr)) != PB_OK) break;
    st = tier_stats(g, rev, 0, n, plan.light_max, plan.med_max, plan.large_max, nullptr, &ts, buf);
    dfree(buf, nullptr);
    if (st != PB_OK) break;
    if (!g->has_plan) plan_from_stats(g, ts, budget, &plan);
    const uint64_t nl = ts.n[0], nm = ts.n[1], nq = ts.n[2], nh = ts.n[3];
    add((nl + 1) * 4); add((nm + 1) * 4); add((nq + 1) * 4); add((nh + 1) * 8);   // tier lists
    if (nq) {                                                   // large-tier slots (grow only)
      HeavySlots hm = {};
      large_slot_shape(plan.large_max, &hm);
      const uint64_t sc = static_cast<uint64_t>(sm_count(g->device)) * 8 * large_slot_bytes(hm);
      add(sc > g->scratch2_cap ? sc : 0);
    }
    if (nh) {
      add(nh * 4);                                              // heavy list
      const uint64_t tiles = (nh + 4095) / 4096;
      add(nh * 8); add(tiles * 256 * 4); add(tiles * 256 * 4 + 4); add(64 << 10);  // its radix sort
      const int heavy = agg == PB_AGG_AUTO ? plan.agg : agg;
      const uint64_t slot = heavy == PB_AGG_HASH ? hash_slot_bytes(g, ts, nullptr, nullptr)
                                                 : dense_slot_bytes(g, ts, nullptr, nullptr);
      uint64_t fit = budget / (slot + 16);
      const uint64_t resident = heavy1_resident(g->device, HOT_SMALL);
      uint64_t ns = fit < resident ? fit : resident;
      if (ns < 1) ns = 1;
      const uint64_t sc = ns * slot + ns * 12 + 64;
      add(sc > g->scratch_cap ? sc : 0);                        // scratch grows only
    }
  } while (0);
  if (cur >= 0 && cur != g->device) cudaSetDevice(cur);
  if (st != PB_OK) return st;
  *bytes = b + allocs * SLACK;
  return PB_OK;
}

pb_status pb_set_plan(pb_graph *g, const pb_plan_t *plan) {
  clear_error();
  if (!g) return fail(PB_ERR_INVALID, "graph is NULL");
  if (!plan) {
    g->has_plan = false;
    return PB_OK;
  }
  if (plan->agg != PB_AGG_BATCH && plan->agg != PB_AGG_HASH && plan->agg != PB_AGG_HIST)
    return fail(PB_ERR_INVALID, "plan aggregation must be BATCH, HASH or HIST (got %d)", plan->agg);
  if (plan->retrieval != PB_RETRIEVE_LOW && plan->retrieval != PB_RETRIEVE_HIGH)
    return fail(PB_ERR_INVALID, "plan retrieval must be LOW or HIGH (got %d)", plan->retrieval);
  if (plan->hub_cluster < 1 || plan->hub_cluster > 16)
    return fail(PB_ERR_INVALID, "plan hub_cluster must be in [1, 16] (got %u)", plan->hub_cluster);
  pb_plan_t p = *plan;
  if (p.light_max < 1) p.light_max = 1;
  if (p.light_max > LIGHT_MAX) p.light_max = LIGHT_MAX;
  if (p.med_max < p.light_max) p.med_max = p.light_max;
  if (p.med_max > MED_MAX) p.med_max = MED_MAX;
  if (p.large_max < p.med_max) p.large_max = p.med_max;
  if (p.large_max > LARGE_LIMIT) p.large_max = LARGE_LIMIT;
  if (p.hot > HOT_LARGE) p.hot = HOT_LARGE;
  g->plan = p;
  g->has_plan = true;
  return PB_OK;
}

pb_status pb_batch_create(pb_graph *const *graphs, uint32_t ng, int want_vertex, uint64_t scratch_bytes,
                          void *stream, pb_batch **out) {
  clear_error();
  if (!out || (ng && !graphs)) return fail(PB_ERR_INVALID, "NULL argument");
  *out = nullptr;
  pb_batch *b = new (std::nothrow) pb_batch();
  if (!b) return fail(PB_ERR_NOMEM, "host allocation failed");
  cudaGetDevice(&b->device);
  b->ng = ng;
  b->pv = want_vertex != 0;
  for (uint32_t i = 0; i < ng; i++) {
    if (!graphs[i] || graphs[i]->device != b->device) {
      delete b;
      return fail(PB_ERR_INVALID, "graph %u is NULL or on another device", i);
    }
    pb_status rs = ensure_ranked(graphs[i], static_cast<cudaStream_t>(stream));
    if (rs != PB_OK) { delete b; return rs; }
    if (graphs[i]->n >= (uint64_t(1) << 32)) { delete b; return fail(PB_ERR_INVALID, "graph too large"); }
    b->graphs.push_back(graphs[i]);
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  pb_status st = batch_build(b, scratch_bytes ? scratch_bytes : (uint64_t(16) << 30), s);
  if (st != PB_OK) {
    std::string keep = pb_last_error();
    batch_release(b);
    fail(st, "%s", keep.c_str());
    return st;
  }
  *out = b;
  return PB_OK;
}

pb_status pb_batch_run(pb_batch *b, void *stream) {
  clear_error();
  if (!b) return fail(PB_ERR_INVALID, "batch is NULL");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  PhaseScope ph(PB_PHASE_HEAVY, s);
  PB_CUDA(cudaGraphLaunch(b->exec, s));
  count_launch((b->nl ? 1 : 0) + (b->nm ? 1 : 0) + (b->nq ? 1 : 0) + (b->nh ? 1 : 0) + (b->nhh ? 1 : 0));
  ph.finish(s, b->W);
  PB_CUDA(cudaStreamSynchronize(s));
  prof_flush();
  return PB_OK;
}

pb_status pb_batch_globals(const pb_batch *b, uint64_t *out, void *stream) {
  clear_error();
  if (!b || !out) return fail(PB_ERR_INVALID, "NULL argument");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  std::vector<unsigned long long> h(static_cast<size_t>(b->ng) * ACC_WORDS);
  if (b->ng) {
    PB_CUDA(cudaMemcpyAsync(h.data(), b->acc, h.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
    PB_CUDA(cudaStreamSynchronize(s));
  }
  for (uint32_t i = 0; i < b->ng; i++) {
    const unsigned long long *r = &h[static_cast<size_t>(i) * ACC_WORDS];
    if (r[ACC_ERR]) return fail(PB_ERR_SCRATCH, "graph %u: aggregation table overflow", i);
    if (r[ACC_OVF]) return fail(PB_ERR_OVERFLOW, "graph %u: global count exceeds 2^64", i);
    out[i] = r[ACC_GLOBAL];
  }
  return PB_OK;
}

pb_status pb_batch_vertex(const pb_batch *b, uint32_t i, uint64_t *out_U, uint64_t *out_V, int out_on_device,
                          void *stream) {
  clear_error();
  if (!b || i >= b->ng || !b->pv) return fail(PB_ERR_INVALID, "bad batch, index or no per-vertex counts");
  const pb_graph *g = b->graphs[i];
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  uint64_t *dU = out_U, *dV = out_V, *tmp = nullptr;
  if (!out_on_device) {
    PB_TRY(dalloc_t(&tmp, g->n + 1, s));
    dU = out_U ? tmp : nullptr;
    dV = out_V ? tmp + g->nU : nullptr;
  }
  k_out_vertex<<<grid_for(g->n, 256, 8192), 256, 0, s>>>(b->pvbuf + b->pv_off[i], g->label, g->nU, g->nV, dU, dV);
  count_launch();
  pb_status st = PB_OK;
  if (!out_on_device) {
    if ((out_U && cudaMemcpyAsync(out_U, dU, g->nU * 8ull, cudaMemcpyDeviceToHost, s) != cudaSuccess) ||
        (out_V && cudaMemcpyAsync(out_V, dV, g->nV * 8ull, cudaMemcpyDeviceToHost, s) != cudaSuccess))
      st = fail(PB_ERR_CUDA, "download");
  }
  dfree(tmp, s);
  cudaError_t e = cudaStreamSynchronize(s);
  if (st != PB_OK) return st;
  if (e != cudaSuccess) return cuda_fail(e, "batch vertex output", __FILE__, __LINE__);
  return PB_OK;
}

pb_status pb_batch_wedges(const pb_batch *b, uint64_t *W) {
  clear_error();
  if (!b || !W) return fail(PB_ERR_INVALID, "NULL argument");
  *W = b->W;
  return PB_OK;
}

pb_status pb_batch_free(pb_batch *b) {
  clear_error();
  batch_release(b);
  return PB_OK;
}

}  // extern "C"

