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

#include <cstdlib>
#include <new>
#include <string>
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
  unsigned long long *acc;  // [0] global, [1] overflow, [2..] work queues
};

enum { ACC_GLOBAL = 0, ACC_OVF = 1, ACC_QMED = 2, ACC_QHEAVY = 3, ACC_NLIGHT = 4, ACC_NMED = 5,
       ACC_NHEAVY = 6, ACC_ERR = 7, ACC_WLIGHT = 8, ACC_WMED = 9, ACC_WHEAVY = 10, ACC_NHUB = 11,
       ACC_WORDS = 16 };

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
// Light tier: one warp per owner; per-warp table with 16-bit counts; LW_BATCH
// steps of 32 wedges in flight per warp.
constexpr int LW_BATCH = 2;

template <bool PV, bool PE, bool MULTI>
__global__ void __launch_bounds__(LW_THREADS, 2) k_light(CArgs a0, const uint32_t *__restrict__ list,
                                                      uint32_t nlist, const uint64_t *__restrict__ items,
                                                      const CArgs *__restrict__ tab) {
  extern __shared__ uint32_t dsm[];  // per warp: LW_CAP keys, then LW_CAP / 2 count words
  __shared__ unsigned long long s_sum[LW_WARPS][32];
  __shared__ uint32_t s_occ[LW_WARPS][LW_CAP / 32];  // per warp: occupied table entries
  __shared__ unsigned long long s_hubarr[2 * HUBK];
  unsigned long long *s_hub = (PV && !MULTI) ? s_hubarr : nullptr;
  const uint32_t lane = lane_id(), w = threadIdx.x >> 5;
  uint32_t *key = dsm + w * (LW_CAP + LW_CAP / 2), *cnt = key + LW_CAP, *occ = s_occ[w];
  static_assert(LW_CAP == 32 * 32, "one bitmap word of 32 entries per lane");
  unsigned long long *err = &a0.acc[ACC_ERR];
  unsigned long long gacc = 0;
  if (PV || PE) s_sum[w][lane] = 0;
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
    uint32_t ky = 0, kc = 0, koy = 0, kincl = 0;
    for (uint32_t k0 = 0; k0 < dp; k0 += 32) {
      const uint32_t i = k0 + lane;
      const bool v = i < dp;
      uint32_t y, c, oy;
      owner_nbr(a, base, i, v, y, c, oy);
      const uint32_t incl = warp_incl_scan(c), tot = __shfl_sync(FULL, incl, 31);
      ky = y; kc = c; koy = oy; kincl = incl;
      for (uint32_t wb = 0; wb < tot; wb += LW_BATCH * 32) {
        uint32_t x2v[LW_BATCH];
#pragma unroll
        for (int q = 0; q < LW_BATCH; q++) {
          const uint32_t wi = wb + q * 32 + lane;
          uint32_t src, slot;
          warp_locate(incl, c, oy, wi < tot ? wi : tot - 1, src, slot);
          x2v[q] = wi < tot ? a.adj[slot] : 0;
        }
#pragma unroll
        for (int q = 0; q < LW_BATCH; q++)
          if (wb + q * 32 + lane < tot) sh_add16m(key, cnt, occ, lg, x2v[q], err);
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
        uint32_t y = ky, c = kc, oy = koy, incl = kincl;
        if (dp > 32) {
          owner_nbr(a, base, i, v, y, c, oy);
          incl = warp_incl_scan(c);
        }
        const uint32_t tot = __shfl_sync(FULL, incl, 31);
        for (uint32_t wb = 0; wb < tot; wb += LW_BATCH * 32) {
          uint32_t x2v[LW_BATCH], srcv[LW_BATCH], slv[LW_BATCH], dv[LW_BATCH];
#pragma unroll
          for (int q = 0; q < LW_BATCH; q++) {
            const uint32_t wi = wb + q * 32 + lane;
            warp_locate(incl, c, oy, wi < tot ? wi : tot - 1, srcv[q], slv[q]);
            x2v[q] = wi < tot ? a.adj[slv[q]] : 0;
          }
#pragma unroll
          for (int q = 0; q < LW_BATCH; q++)
            dv[q] = wb + q * 32 + lane < tot ? sh_get16(key, cnt, lg, x2v[q], err) : 0;
#pragma unroll
          for (int q = 0; q < LW_BATCH; q++) {
            unsigned long long t = dv[q] > 1 ? dv[q] - 1 : 0;
            if (PE && t) atomicAdd(&a.es[slv[q]], t);
            warp_run_add_rx(s_sum[w], srcv[q], t);
          }
        }
        __syncwarp();
        if (v) {
          unsigned long long sm = s_sum[w][lane];
          if (sm) {
            if (PV) pv_add(s_hub, a, y, sm);
            if (PE) atomicAdd(&a.es[base + i], sm);
            s_sum[w][lane] = 0;
          }
        }
        __syncwarp();
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
            if (PE && t) atomicAdd(&a.es[slv[q]], t);
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
// Heavy tier, one block per owner with a dense slot (no cluster): the owner's
// neighbours are staged HB_THREADS at a time, and each warp takes whole
// neighbours from a shared counter and walks the neighbour's segment of
// second endpoints with its lanes (coalesced adjacency reads).  Counts of the
// first h.hot labels of the side live in shared memory, the rest in the
// slot's device-memory histogram; a touched list (device memory, counter in
// shared memory) records each distinct second endpoint once.  The second
// pass sums d - 1 over a segment in registers and adds it to the centre once.
template <bool PV, bool PE, bool MULTI>
__global__ void __launch_bounds__(HB_THREADS) k_heavy1(CArgs a0, const uint32_t *__restrict__ list, uint32_t nlist,
                                                       HeavySlots h, const uint64_t *__restrict__ items,
                                                       const CArgs *__restrict__ tab) {
  extern __shared__ uint32_t hb_hot[];
  __shared__ uint32_t s_c[HB_THREADS], s_oy[HB_THREADS], s_y[HB_THREADS];
  __shared__ unsigned long long s_hubarr[2 * HUBK];
  __shared__ uint32_t s_item, s_next, s_nt;
  unsigned long long *s_hub = (PV && !MULTI) ? s_hubarr : nullptr;
  const uint32_t slot = blockIdx.x, tid = threadIdx.x, lane = lane_id();
  uint32_t *A = h.A + static_cast<size_t>(slot) * h.side;
  uint32_t *T = h.T + static_cast<size_t>(slot) * h.tcap;
  unsigned long long *err = &a0.acc[ACC_ERR];
  unsigned long long gacc = 0;
  if (s_hub) hub_zero(s_hub);
  for (uint32_t t = tid; t < h.hot; t += HB_THREADS) hb_hot[t] = 0;
  if (tid == 0) s_nt = 0;
  for (;;) {
    if (tid == 0) s_item = static_cast<uint32_t>(atomicAdd(&a0.acc[ACC_QHEAVY], 1ull));
    __syncthreads();
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
    const uint32_t base = dense_base(a, x1);  // label of histogram entry 0
    const uint32_t xbase = a.off[x1], dp = owner_span(a, x1);
    // ---- aggregate
    for (uint32_t s0 = 0; s0 < dp; s0 += HB_THREADS) {
      {
        uint32_t y, c, oy;
        owner_nbr(a, xbase, s0 + tid, s0 + tid < dp, y, c, oy);
        s_c[tid] = c;
        s_oy[tid] = oy;
        s_y[tid] = y;
      }
      if (tid == 0) s_next = 0;
      __syncthreads();
      const uint32_t nn = dp - s0 < HB_THREADS ? dp - s0 : HB_THREADS;
      for (;;) {
        uint32_t j = 0;
        if (lane == 0) j = atomicAdd(&s_next, 1u);
        j = __shfl_sync(FULL, j, 0);
        if (j >= nn) break;
        const uint32_t c = s_c[j], oy = s_oy[j];
        for (uint32_t e0 = 0; e0 < c; e0 += 32) {
          const bool act = e0 + lane < c;
          uint32_t x2 = 0;
          bool isnew = false;
          if (act) {
            x2 = a.adj[oy + e0 + lane];
            const uint32_t r = x2 - base;
            isnew = (r < h.hot ? atomicAdd(&hb_hot[r], 1u) : atomicAdd(&A[r], 1u)) == 0u;
          }
          const uint32_t bm = __ballot_sync(FULL, isnew);
          if (bm) {
            uint32_t b0 = 0;
            if (lane == 0) b0 = atomicAdd(&s_nt, static_cast<uint32_t>(__popc(bm)));
            b0 = __shfl_sync(FULL, b0, 0);
            if (isnew) {
              const uint32_t at = b0 + __popc(bm & lanemask_lt());
              if (at < h.tcap) T[at] = x2;
              else atomicOr(err, 16ull);
            }
          }
        }
      }
      __syncthreads();
    }
    const uint32_t nt = s_nt < h.tcap ? s_nt : static_cast<uint32_t>(h.tcap);
    // ---- endpoints: C(d, 2) per distinct second endpoint
    unsigned long long own = 0;
    for (uint32_t t = tid; t < nt; t += HB_THREADS) {
      const uint32_t x2 = T[t], r = x2 - base;
      unsigned long long d = r < h.hot ? hb_hot[r] : __ldcg(&A[r]), b = d * (d - 1) / 2;
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
      for (uint32_t s0 = 0; s0 < dp; s0 += HB_THREADS) {
        if (dp > HB_THREADS) {  // otherwise the first pass's staging is still in place
          uint32_t y, c, oy;
          owner_nbr(a, xbase, s0 + tid, s0 + tid < dp, y, c, oy);
          s_c[tid] = c;
          s_oy[tid] = oy;
          s_y[tid] = y;
        }
        if (tid == 0) s_next = 0;
        __syncthreads();
        const uint32_t nn = dp - s0 < HB_THREADS ? dp - s0 : HB_THREADS;
        for (;;) {
          uint32_t j = 0;
          if (lane == 0) j = atomicAdd(&s_next, 1u);
          j = __shfl_sync(FULL, j, 0);
          if (j >= nn) break;
          const uint32_t c = s_c[j], oy = s_oy[j];
          unsigned long long sum = 0;
          for (uint32_t e = lane; e < c; e += 32) {
            const uint32_t sl = oy + e, r = a.adj[sl] - base;
            const uint32_t d = r < h.hot ? hb_hot[r] : __ldcg(&A[r]);
            if (d > 1) {
              sum += d - 1;
              if (PE) atomicAdd(&a.es[sl], static_cast<unsigned long long>(d - 1));
            }
          }
          sum = warp_sum(sum);
          if (lane == 0 && sum) {
            if (PV) pv_add(s_hub, a, s_y[j], sum);
            if (PE) atomicAdd(&a.es[xbase + s0 + j], sum);
          }
        }
        __syncthreads();
      }
    }
    // ---- reset the slot's used entries
    for (uint32_t t = tid; t < nt; t += HB_THREADS) {
      const uint32_t r = T[t] - base;
      if (r < h.hot) hb_hot[r] = 0;
      else A[r] = 0;
    }
    __syncthreads();
    if (tid == 0) s_nt = 0;
  }
  if (!MULTI && lane == 0) add_global(a0.acc, gacc);
  __syncthreads();
  if (s_hub) hub_flush(s_hub, a0);
}

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
__global__ void k_classify(const uint64_t *__restrict__ wpre, uint64_t n, uint64_t olo, uint64_t ohi,
                           uint64_t light_max, uint64_t med_max,
                           uint64_t hub_min, uint32_t *__restrict__ light, uint32_t *__restrict__ med,
                           uint64_t *__restrict__ heavy_keys, int bitsN, unsigned long long *acc) {
  size_t stride = static_cast<size_t>(gridDim.x) * blockDim.x;
  size_t iters = (n + stride - 1) / stride;
  for (size_t itn = 0; itn < iters; itn++) {
    size_t x = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x + itn * stride;
    uint64_t wc = (x < n && x >= olo && x < ohi) ? wpre[x + 1] - wpre[x] : 0;
    int tier = wc == 0 ? 0 : (wc <= light_max ? 1 : (wc <= med_max ? 2 : 3));
    uint32_t hubs = __popc(__ballot_sync(FULL, tier == 3 && wc > hub_min));
    if (lane_id() == 0 && hubs) atomicAdd(&acc[ACC_NHUB], (unsigned long long)hubs);
#pragma unroll
    for (int t = 1; t <= 3; t++) {
      unsigned long long ws = warp_sum(static_cast<unsigned long long>(tier == t ? wc : 0));
      if (lane_id() == 0 && ws) atomicAdd(&acc[ACC_WLIGHT + t - 1], ws);
      uint32_t bm = __ballot_sync(FULL, tier == t);
      if (!bm) continue;
      uint32_t leader = __ffs(bm) - 1;
      unsigned long long b0 = 0;
      if (lane_id() == leader) b0 = atomicAdd(&acc[ACC_NLIGHT + t - 1], (unsigned long long)__popc(bm));
      b0 = __shfl_sync(FULL, b0, leader);
      if (tier == t) {
        uint64_t at = b0 + __popc(bm & lanemask_lt());
        if (t == 1) light[at] = static_cast<uint32_t>(x);
        else if (t == 2) med[at] = static_cast<uint32_t>(x);
        else {
          // decreasing wedge count first (largest-first scheduling)
          const uint64_t cmax = (uint64_t(1) << (63 - bitsN)) - 1;
          uint64_t cw = wc < cmax ? wc : cmax;
          heavy_keys[at] = ((cmax - cw) << bitsN) | x;
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
__global__ void k_edge_sums(const unsigned long long *__restrict__ es, const uint32_t *__restrict__ slotA,
                            const uint32_t *__restrict__ slotB, uint64_t m, uint64_t *__restrict__ E) {
  for (size_t e = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < m;
       e += static_cast<size_t>(gridDim.x) * blockDim.x)
    E[e] = es[slotA[e]] + es[slotB[e]];
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

struct Plan {
  int agg;
  bool pv, pe;
  uint64_t light_max, med_max;
  bool dense;         // heavy tier uses dense histograms
  unsigned cluster;   // blocks per heavy first endpoint
  uint64_t max_slots; // cap on concurrently processed hubs (0 = resident clusters)
  uint64_t hub_min;   // heavy first endpoints above this many wedges get a cluster each
  uint64_t owner_lo, owner_hi;  // owners counted
};

// Tuning knobs (environment): PB_HEAVY_CLUSTER, PB_HEAVY_SLOTS, PB_HUB_MIN.
static uint64_t env_u64(const char *name, uint64_t dflt) {
  const char *v = getenv(name);
  if (!v || !*v) return dflt;
  return strtoull(v, nullptr, 10);
}

template <bool PV, bool PE>
static pb_status run_tiers(pb_graph *g, const CArgs &a, const Plan &p, uint64_t budget, cudaStream_t s) {
  const uint64_t n = g->n;
  unsigned long long hcnt[ACC_WORDS] = {0};
  uint32_t *light = nullptr, *med = nullptr, *heavy = nullptr;
  uint64_t *hkeys = nullptr;
  unsigned long long *dmx = nullptr;
  pb_status st = PB_OK;
  const int sms = sm_count(g->device);
  do {
    if ((st = dalloc_t(&light, n + 1, s)) != PB_OK) break;
    if ((st = dalloc_t(&med, n + 1, s)) != PB_OK) break;
    if ((st = dalloc_t(&hkeys, n + 1, s)) != PB_OK) break;
    {
      PhaseScope ph(PB_PHASE_CLASSIFY, s);
      k_classify<<<grid_for(n, 256, 8192), 256, 0, s>>>(a.wpre, n, p.owner_lo, p.owner_hi, p.light_max, p.med_max,
                                                        p.hub_min, light, med,
                                                        hkeys, g->bitsN, a.acc);
      count_launch();
      ph.finish(s);
    }
    if (cudaMemcpyAsync(hcnt, a.acc, sizeof(hcnt), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) { st = fail(PB_ERR_CUDA, "tier readback: %s", cudaGetErrorString(cudaGetLastError())); break; }
    const uint32_t nl = static_cast<uint32_t>(hcnt[ACC_NLIGHT]), nm = static_cast<uint32_t>(hcnt[ACC_NMED]),
                   nh = static_cast<uint32_t>(hcnt[ACC_NHEAVY]);
    if (nl) {
      PhaseScope ph(PB_PHASE_LIGHT, s);
      const size_t smem = LW_WARPS * (LW_CAP + LW_CAP / 2) * sizeof(uint32_t);
      PB_CUDA(cudaFuncSetAttribute(k_light<PV, PE, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      int per_sm = 0;
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_light<PV, PE, false>, LW_THREADS, smem);
      unsigned grid = static_cast<unsigned>(sms * (per_sm > 0 ? per_sm : 1));
      unsigned need = (nl + LW_WARPS - 1) / LW_WARPS;
      PB_LAUNCH((k_light<PV, PE, false>), grid < need ? grid : need, LW_THREADS, smem, s, a, light, nl,
                (const uint64_t *)nullptr, (const CArgs *)nullptr);
      ph.finish(s, hcnt[ACC_WLIGHT]);
    }
    if (nm) {
      PhaseScope ph(PB_PHASE_MEDIUM, s);
      const size_t smem = MB_SMEM;
      PB_CUDA(cudaFuncSetAttribute(k_medium<PV, PE, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      int per_sm = 0;
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_medium<PV, PE, false>, MB_THREADS, smem);
      unsigned grid = static_cast<unsigned>(sms * (per_sm > 0 ? per_sm : 1));
      PB_LAUNCH((k_medium<PV, PE, false>), grid < nm ? grid : nm, MB_THREADS, smem, s, a, med, nm,
                (const uint64_t *)nullptr, (const CArgs *)nullptr);
      ph.finish(s, hcnt[ACC_WMED]);
    }
    if (nh) {
      if ((st = radix_sort(hkeys, nullptr, nh, 64 - 1, s)) != PB_OK) break;
      if ((st = dalloc_t(&heavy, nh, s)) != PB_OK) break;
      k_keys_low<<<grid_for(nh, 256, 4096), 256, 0, s>>>(hkeys, nh, g->bitsN, heavy);
      count_launch();
      if ((st = dalloc_t(&dmx, 2, s)) != PB_OK) break;
      if (cudaMemsetAsync(dmx, 0, 2 * sizeof(unsigned long long), s) != cudaSuccess) { st = fail(PB_ERR_CUDA, "memset"); break; }
      k_max_wedges_list<<<grid_for(nh, 256, 4096), 256, 0, s>>>(heavy, nh, a.wpre, n, g->nU, a.rev, dmx);
      count_launch();
      unsigned long long hdm2[2] = {0, 0};
      if (cudaMemcpyAsync(hdm2, dmx, sizeof(hdm2), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
          cudaStreamSynchronize(s) != cudaSuccess) { st = fail(PB_ERR_CUDA, "heavy readback"); break; }
      const unsigned long long hdm = hdm2[0];
      HeavySlots hs = {};
      hs.side = g->nU > g->nV ? g->nU : g->nV;
      if (hdm2[1] && hdm2[1] < hs.side) hs.side = hdm2[1];  // dense histograms span the owners' label ranges
      size_t slot_bytes;
      if (p.dense) {
        hs.tcap = hdm < hs.side ? hdm : hs.side;
        slot_bytes = (hs.side + hs.tcap) * sizeof(uint32_t);
      } else {
        uint64_t cap = 32;
        while (cap < 2 * hdm) cap <<= 1;
        hs.hcap = cap;
        slot_bytes = 2 * cap * sizeof(uint32_t);
      }
      auto kern = p.dense ? k_heavy<PV, PE, true, false> : k_heavy<PV, PE, false, false>;
      // Hubs (wedges > hub_min, the head of the largest-first list) get one
      // cluster each; the rest one block each (plain batching).
      uint32_t nhub = p.cluster > 1 ? static_cast<uint32_t>(hcnt[ACC_NHUB]) : 0;
      unsigned hub_cl = p.cluster, rest_cl = 1;
      uint64_t fit = budget / (slot_bytes + 16);
      if (fit == 0) { st = fail(PB_ERR_SCRATCH, "scratch budget %llu B below one heavy slot (%llu B)", (unsigned long long)budget, (unsigned long long)slot_bytes); break; }
      {
        // When the budget holds fewer slots than there are resident blocks,
        // every slot is shared by a cluster of blocks so that all SMs work.
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_heavy<PV, PE, true, false>, HB_THREADS, 0);
        const uint64_t resident = static_cast<uint64_t>(sms) * (per_sm > 0 ? per_sm : 1);
        if (fit < resident) {
          uint64_t want = (resident + fit - 1) / fit;
          unsigned c = 1;
          while (c < want && c < 8) c <<= 1;
          rest_cl = c;
          if (hub_cl < c) hub_cl = c;
        }
      }
      struct Part { const uint32_t *list; uint32_t cnt; unsigned cl; };
      Part parts[2] = {{heavy, nhub, hub_cl}, {heavy + nhub, nh - nhub, rest_cl}};
      PhaseScope ph(PB_PHASE_HEAVY, s);
      for (const Part &pt : parts) {
        if (pt.cnt == 0) continue;
        const unsigned cl = pt.cl;
        if (cl > 8) PB_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
        // A slot processed by one block keeps the counts of the first HB_HOT
        // labels of the side in shared memory (dense mode).
        const bool one = p.dense && cl == 1;  // one block per dense slot: k_heavy1
        const uint32_t hot = one ? HB_HOT : 0;
        const size_t hsmem = hot * sizeof(uint32_t);
        hs.hot = hot;
        int nc = 0;
        if (one) {
          PB_CUDA(cudaFuncSetAttribute(k_heavy1<PV, PE, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)hsmem));
          int per_sm = 0;
          cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_heavy1<PV, PE, false>, HB_THREADS, hsmem);
          nc = sms * (per_sm > 0 ? per_sm : 1);
        } else {
          nc = max_clusters(kern, HB_THREADS, cl, hsmem);
        }
        if (nc <= 0) nc = sms / static_cast<int>(cl);
        uint64_t nslots = static_cast<uint64_t>(nc);
        if (&pt == &parts[0] && p.max_slots && nslots > p.max_slots) nslots = p.max_slots;
        if (nslots > fit) nslots = fit;
        if (nslots > pt.cnt) nslots = pt.cnt;
        size_t need = nslots * slot_bytes + nslots * 3 * sizeof(uint32_t) + 64;
        if ((st = ensure_scratch(g, need, s)) != PB_OK) break;
        char *sp = static_cast<char *>(g->scratch);
        if (p.dense) {
          hs.A = reinterpret_cast<uint32_t *>(sp);
          hs.T = hs.A + nslots * hs.side;
          hs.tcnt = hs.T + nslots * hs.tcap;
          if (cudaMemsetAsync(hs.A, 0, nslots * hs.side * sizeof(uint32_t), s) != cudaSuccess) { st = fail(PB_ERR_CUDA, "memset"); break; }
        } else {
          hs.hkey = reinterpret_cast<uint32_t *>(sp);
          hs.hval = hs.hkey + nslots * hs.hcap;
          hs.tcnt = hs.hval + nslots * hs.hcap;
          if (cudaMemsetAsync(hs.hkey, 0xff, nslots * hs.hcap * sizeof(uint32_t), s) != cudaSuccess ||
              cudaMemsetAsync(hs.hval, 0, nslots * hs.hcap * sizeof(uint32_t), s) != cudaSuccess) { st = fail(PB_ERR_CUDA, "memset"); break; }
        }
        hs.item = hs.tcnt + 2 * nslots;
        if (cudaMemsetAsync(hs.tcnt, 0, 3 * nslots * sizeof(uint32_t), s) != cudaSuccess ||
            cudaMemsetAsync(a.acc + ACC_QHEAVY, 0, sizeof(unsigned long long), s) != cudaSuccess) { st = fail(PB_ERR_CUDA, "memset"); break; }
        if (one) {
          PB_LAUNCH((k_heavy1<PV, PE, false>), static_cast<unsigned>(nslots), HB_THREADS, hsmem, s, a, pt.list, pt.cnt,
                    hs, (const uint64_t *)nullptr, (const CArgs *)nullptr);
        } else if ((st = launch_cluster(kern, static_cast<unsigned>(nslots * cl), HB_THREADS, cl, hsmem, s, a, pt.list,
                                        pt.cnt, hs, (const uint64_t *)nullptr, (const CArgs *)nullptr)) != PB_OK) {
          break;
        }
      }
      if (st != PB_OK) break;
      ph.finish(s, hcnt[ACC_WHEAVY]);
    }
  } while (0);
  dfree(light, s); dfree(med, s); dfree(heavy, s); dfree(hkeys, s); dfree(dmx, s);
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
static pb_status run_sort(pb_graph *g, const CArgs &a, uint64_t budget, uint64_t olo, uint64_t ohi,
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
  }
  CArgs a;
  // Owner of each wedge: its lower-ranked endpoint (Algorithm 2) or, with the
  // cache optimisation, its higher-ranked one.  Same wedges either way.
  pb_plan_t plan;
  make_plan(g, &plan);
  a.rev = g->retrieval == PB_RETRIEVE_AUTO ? plan.retrieval == PB_RETRIEVE_HIGH : g->retrieval == PB_RETRIEVE_HIGH;
  a.off = g->off; a.adj = g->adj; a.cpos = g->cpos; a.degp = g->degp; a.n = n;
  a.wpre = a.rev ? g->wpre_rev : g->wpre;
  a.nU = g->nU;
  a.pv = want_pv ? reinterpret_cast<unsigned long long *>(g->pv) : nullptr;
  a.es = want_pe ? reinterpret_cast<unsigned long long *>(g->es) : nullptr;
  a.acc = g->acc;
  if (g->W > 0) {
    Plan p;
    p.agg = agg;
    p.pv = want_pv;
    p.pe = want_pe;
    p.light_max = LIGHT_MAX;
    p.med_max = MED_MAX;
    p.owner_lo = o.owner_lo < n ? o.owner_lo : n;
    p.owner_hi = o.owner_hi < n ? o.owner_hi : n;
    p.dense = agg != PB_AGG_HASH;
    p.cluster = static_cast<unsigned>(env_u64("PB_HEAVY_CLUSTER", plan.hub_cluster));
    p.max_slots = env_u64("PB_HEAVY_SLOTS", 0);
    p.hub_min = env_u64("PB_HUB_MIN", plan.hub_min);
    if (agg == PB_AGG_BATCH) {
      // One dense array per concurrently processed heavy first endpoint, no
      // clusters; first endpoints with at most MED_MAX wedges keep the
      // shared-memory tiers (a dense array each would exhaust the budget).
      p.cluster = 1;
      p.max_slots = 0;
      p.hub_min = UINT64_MAX;
    }
    if (p.cluster < 1) p.cluster = 1;
    if (p.cluster > 16) p.cluster = 16;
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
    } else if (want_pv && want_pe) st = run_tiers<true, true>(g, a, p, budget, s);
    else if (want_pv) st = run_tiers<true, false>(g, a, p, budget, s);
    else if (want_pe) st = run_tiers<false, true>(g, a, p, budget, s);
    else st = run_tiers<false, false>(g, a, p, budget, s);
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
      k_edge_sums<<<grid_for(g->m, 256, 8192), 256, 0, s>>>(reinterpret_cast<unsigned long long *>(g->es), g->slotA,
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
// Autotuner (rules from degree and wedge statistics).
void make_plan(const pb_graph *g, pb_plan_t *plan) {
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
  plan->agg = PB_AGG_AUTO;
  // owners past 2^20 wedges would keep one block busy for milliseconds:
  // give owners past 2^18 a pair of blocks
  if (plan->max_owner_wedges > (uint64_t(1) << 20)) {
    plan->hub_min = uint64_t(1) << 18;
    plan->hub_cluster = 2;
  } else {
    plan->hub_min = UINT64_MAX;
    plan->hub_cluster = 1;
  }
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
  uint64_t *light = nullptr, *med = nullptr, *heavy = nullptr;
  uint32_t nl = 0, nm = 0, nh = 0;
  pb::HeavySlots hs = {};
  void *scratch = nullptr;
  uint64_t nslots = 0, slot_bytes = 0;
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
  dfree(b->light, s); dfree(b->med, s); dfree(b->heavy, s); dfree(b->scratch, s);
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
  PB_CUDA(cudaFuncSetAttribute(k_heavy1<PV, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)(b->hs.hot * sizeof(uint32_t))));
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
    if (b->nh) {
      e1 = cudaMemsetAsync(b->scratch, 0, b->nslots * b->slot_bytes + b->nslots * 7 * sizeof(uint32_t) + 64, s);
      if (e1 != cudaSuccess) { st = cuda_fail(e1, "batch memset (slots)", __FILE__, __LINE__); break; }
      k_heavy1<PV, false, true><<<static_cast<unsigned>(b->nslots), HB_THREADS, b->hs.hot * sizeof(uint32_t), s>>>(
          a0, nullptr, b->nh, b->hs, b->heavy, b->tab);
      count_launch();
      e1 = cudaGetLastError();
      if (e1 != cudaSuccess) { st = cuda_fail(e1, "batch heavy launch", __FILE__, __LINE__); break; }
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
  PB_TRY(dalloc_t(&b->heavy, total_n + 1, s));
  uint32_t *tl = nullptr, *tm = nullptr;
  uint64_t *th = nullptr;
  unsigned long long *tacc = nullptr;
  pb_status st = PB_OK;
  uint64_t max_bound = 1, max_room = 1;
  do {
    if ((st = dalloc_t(&tacc, ACC_WORDS, s)) != PB_OK) break;
    for (uint32_t i = 0; i < ng && st == PB_OK; i++) {
      pb_graph *g = b->graphs[i];
      pb_plan_t plan;
      make_plan(g, &plan);
      CArgs &a = host_tab[i];
      a.rev = g->retrieval == PB_RETRIEVE_AUTO ? plan.retrieval == PB_RETRIEVE_HIGH : g->retrieval == PB_RETRIEVE_HIGH;
      a.off = g->off; a.adj = g->adj; a.cpos = g->cpos; a.degp = g->degp; a.n = g->n; a.nU = g->nU;
      a.wpre = a.rev ? g->wpre_rev : g->wpre;
      a.pv = b->pv ? b->pvbuf + b->pv_off[i] : nullptr;
      a.es = nullptr;
      a.acc = b->acc + static_cast<size_t>(i) * ACC_WORDS;
      b->W += g->W;
      if (g->W == 0) continue;
      const uint64_t n = g->n;
      if ((st = dalloc_t(&tl, n + 1, s)) != PB_OK || (st = dalloc_t(&tm, n + 1, s)) != PB_OK ||
          (st = dalloc_t(&th, n + 1, s)) != PB_OK) break;
      if (cudaMemsetAsync(tacc, 0, sizeof(unsigned long long) * ACC_WORDS, s) != cudaSuccess) { st = fail(PB_ERR_CUDA, "memset"); break; }
      k_classify<<<grid_for(n, 256, 8192), 256, 0, s>>>(a.wpre, n, 0, n, LIGHT_MAX, MED_MAX, UINT64_MAX, tl, tm, th,
                                                        g->bitsN, tacc);
      count_launch();
      unsigned long long hc[ACC_WORDS];
      if (cudaMemcpyAsync(hc, tacc, sizeof(hc), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
          cudaStreamSynchronize(s) != cudaSuccess) { st = fail(PB_ERR_CUDA, "classify readback"); break; }
      const uint32_t cl = static_cast<uint32_t>(hc[ACC_NLIGHT]), cm = static_cast<uint32_t>(hc[ACC_NMED]),
                     ch = static_cast<uint32_t>(hc[ACC_NHEAVY]);
      if (cl) { k_tag_items<<<grid_for(cl, 256, 1024), 256, 0, s>>>(tl, cl, i, b->light + b->nl); count_launch(); }
      if (cm) { k_tag_items<<<grid_for(cm, 256, 1024), 256, 0, s>>>(tm, cm, i, b->med + b->nm); count_launch(); }
      if (ch) {
        k_keys_low<<<grid_for(ch, 256, 1024), 256, 0, s>>>(th, ch, g->bitsN, tl);
        count_launch();
        k_tag_items<<<grid_for(ch, 256, 1024), 256, 0, s>>>(tl, ch, i, b->heavy + b->nh);
        count_launch();
        // distinct bound of this graph's heavy owners
        if (cudaMemsetAsync(tacc, 0, 2 * sizeof(unsigned long long), s) != cudaSuccess) { st = fail(PB_ERR_CUDA, "memset"); break; }
        k_max_wedges_list<<<grid_for(ch, 256, 1024), 256, 0, s>>>(tl, ch, a.wpre, n, g->nU, a.rev, tacc);
        count_launch();
        unsigned long long bd[2] = {0, 0};
        if (cudaMemcpyAsync(bd, tacc, sizeof(bd), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) { st = fail(PB_ERR_CUDA, "readback"); break; }
        if (bd[0] > max_bound) max_bound = bd[0];
        if (bd[1] > max_room) max_room = bd[1];
      }
      b->nl += cl; b->nm += cm; b->nh += ch;
      dfree(tl, s); dfree(tm, s); dfree(th, s);
      tl = tm = nullptr; th = nullptr;
    }
  } while (0);
  dfree(tl, s); dfree(tm, s); dfree(th, s); dfree(tacc, s);
  if (st != PB_OK) return st;
  PB_TRY(dalloc_t(&b->tab, ng, s));
  PB_CUDA(cudaMemcpyAsync(b->tab, host_tab.data(), sizeof(CArgs) * ng, cudaMemcpyHostToDevice, s));
  if (b->nh) {
    b->hs.side = max_room < max_side ? max_room : max_side;  // dense histograms span the owners' label ranges
    b->hs.tcap = max_bound < max_side ? max_bound : max_side;
    b->slot_bytes = (b->hs.side + b->hs.tcap) * sizeof(uint32_t);
    b->hs.hot = HB_HOT;
    const size_t hsmem = HB_HOT * sizeof(uint32_t);
    PB_CUDA(cudaFuncSetAttribute(k_heavy1<true, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)hsmem));
    PB_CUDA(cudaFuncSetAttribute(k_heavy1<false, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)hsmem));
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_heavy1<true, false, true>, HB_THREADS, hsmem);
    uint64_t ns = static_cast<uint64_t>(sm_count(b->device)) * (per_sm > 0 ? per_sm : 1);
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
  PB_CUDA(cudaStreamSynchronize(s));
  return b->pv ? batch_capture<true>(b) : batch_capture<false>(b);
}

}  // namespace pb

using namespace pb;

extern "C" {

pb_status pb_autotune(const pb_graph *g, pb_plan_t *plan) {
  clear_error();
  if (!g || !plan) return fail(PB_ERR_INVALID, "graph or plan is NULL");
  PB_TRY(ensure_ranked(g, nullptr));
  PB_CUDA(cudaStreamSynchronize(nullptr));
  make_plan(g, plan);
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
  count_launch((b->nl ? 1 : 0) + (b->nm ? 1 : 0) + (b->nh ? 1 : 0));
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

