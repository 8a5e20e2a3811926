// Graph construction (bipartite CSR input, duplicate removal) and PREPROCESS
// (Algorithm 1): rank keys, device radix sorts, renaming, adjacency sorted by
// decreasing rank, the modified degrees deg_x(y), and the per-first-endpoint
// wedge counts with their prefix sum (the work split of Algorithm 2).
#include "pb_common.cuh"

namespace pb {

// ---------------------------------------------------------------------------
// Input validation and duplicate removal.

__global__ void k_validate(const uint32_t *__restrict__ u, const uint32_t *__restrict__ v, size_t m,
                           uint32_t nU, uint32_t nV, unsigned long long *bad) {
  for (size_t i = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < m;
       i += static_cast<size_t>(gridDim.x) * blockDim.x)
    if (u[i] >= nU || v[i] >= nV) atomicAdd(bad, 1ull);
}

__global__ void k_pair_keys(const uint32_t *__restrict__ u, const uint32_t *__restrict__ v, size_t m,
                            int bitsV, uint64_t *__restrict__ keys, uint32_t *__restrict__ idx) {
  for (size_t i = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < m;
       i += static_cast<size_t>(gridDim.x) * blockDim.x) {
    keys[i] = (static_cast<uint64_t>(u[i]) << bitsV) | v[i];
    idx[i] = static_cast<uint32_t>(i);
  }
}

__global__ void k_heads(const uint64_t *__restrict__ keys, size_t m, uint32_t *__restrict__ head) {
  for (size_t i = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < m;
       i += static_cast<size_t>(gridDim.x) * blockDim.x)
    head[i] = (i == 0 || keys[i] != keys[i - 1]) ? 1u : 0u;
}

__global__ void k_canon(const uint64_t *__restrict__ keys, const uint32_t *__restrict__ idx,
                        const uint32_t *__restrict__ head, const uint32_t *__restrict__ cid, size_t m,
                        int bitsV, uint32_t nU, uint32_t *__restrict__ in2c, uint32_t *__restrict__ eu,
                        uint32_t *__restrict__ ev, uint32_t *__restrict__ deg) {
  const uint64_t maskV = (uint64_t(1) << bitsV) - 1;
  const size_t stride = static_cast<size_t>(gridDim.x) * blockDim.x;
  const size_t start = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const size_t iters = (m + stride - 1) / stride;
  for (size_t itn = 0; itn < iters; itn++) {  // uniform trip count: the whole warp reaches the matches
    const size_t i = start + itn * stride;
    uint32_t du = 0xffffffffu, dv = 0xffffffffu;  // degree targets of this canonical edge
    if (i < m) {
      uint32_t r = cid[i] + head[i] - 1;
      in2c[idx[i]] = r;
      if (head[i]) {
        uint32_t a = static_cast<uint32_t>(keys[i] >> bitsV), b = static_cast<uint32_t>(keys[i] & maskV);
        eu[r] = a;
        ev[r] = b;
        du = a;
        dv = nU + b;
      }
    }
    // keys are sorted by u, so a warp's edges mostly share u: one atomic per distinct vertex
    uint32_t peers = __match_any_sync(FULL, du);
    if (du != 0xffffffffu && lane_id() == static_cast<uint32_t>(__ffs(peers) - 1)) atomicAdd(&deg[du], __popc(peers));
    peers = __match_any_sync(FULL, dv);
    if (dv != 0xffffffffu && lane_id() == static_cast<uint32_t>(__ffs(peers) - 1)) atomicAdd(&deg[dv], __popc(peers));
  }
}

__global__ void k_maxdeg(const uint32_t *__restrict__ deg, uint64_t n, uint32_t nU, uint32_t *out2) {
  uint32_t mu = 0, mv = 0;
  for (size_t i = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += static_cast<size_t>(gridDim.x) * blockDim.x) {
    if (i < nU) mu = max(mu, deg[i]);
    else mv = max(mv, deg[i]);
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    mu = max(mu, __shfl_xor_sync(FULL, mu, o));
    mv = max(mv, __shfl_xor_sync(FULL, mv, o));
  }
  if (lane_id() == 0) {
    atomicMax(&out2[0], mu);
    atomicMax(&out2[1], mv);
  }
}

pb_status build_graph(pb_graph *g, const uint32_t *u_in, const uint32_t *v_in, int on_device,
                      cudaStream_t s) {
  const size_t m = g->m_in;
  const uint64_t n = g->n;
  PB_TRY(dalloc_t(&g->deg, n + 1, s));
  PB_CUDA(cudaMemsetAsync(g->deg, 0, (n + 1) * sizeof(uint32_t), s));
  PB_TRY(dalloc_t(&g->in2c, m + 1, s));
  unsigned long long *flag = nullptr;
  PB_TRY(dalloc_t(&flag, 2, s));
  const uint32_t *u = u_in, *v = v_in;
  uint32_t *du = nullptr, *dv = nullptr, *idx = nullptr, *head = nullptr, *cid = nullptr;
  uint64_t *keys = nullptr;
  pb_status st = PB_OK;
  unsigned long long hbad = 0;
  uint32_t hm = 0, hmax[2] = {0, 0};
  uint32_t *dmax = nullptr;
  do {
    if (m > 0 && !on_device) {
      if ((st = dalloc_t(&du, m, s)) != PB_OK) break;
      if ((st = dalloc_t(&dv, m, s)) != PB_OK) break;
      cudaError_t e = cudaMemcpyAsync(du, u_in, m * sizeof(uint32_t), cudaMemcpyHostToDevice, s);
      if (e == cudaSuccess) e = cudaMemcpyAsync(dv, v_in, m * sizeof(uint32_t), cudaMemcpyHostToDevice, s);
      if (e != cudaSuccess) { st = cuda_fail(e, "edge upload", __FILE__, __LINE__); break; }
      u = du;
      v = dv;
    }
    if (cudaMemsetAsync(flag, 0, 2 * sizeof(unsigned long long), s) != cudaSuccess) { st = fail(PB_ERR_CUDA, "memset"); break; }
    if (m > 0) {
      k_validate<<<grid_for(m, 256, 8192), 256, 0, s>>>(u, v, m, g->nU, g->nV, flag);
      count_launch();
    }
    if (cudaMemcpyAsync(&hbad, flag, sizeof(hbad), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) { st = fail(PB_ERR_CUDA, "validation readback failed: %s", cudaGetErrorString(cudaGetLastError())); break; }
    if (hbad) { st = fail(PB_ERR_INVALID, "%llu edge(s) have u >= nU or v >= nV", hbad); break; }
    if (m == 0) { g->m = 0; break; }
    const int bitsU = bits_for(g->nU ? g->nU - 1 : 0), bitsV = bits_for(g->nV ? g->nV - 1 : 0);
    if ((st = dalloc_t(&keys, m, s)) != PB_OK) break;
    if ((st = dalloc_t(&idx, m, s)) != PB_OK) break;
    k_pair_keys<<<grid_for(m, 256, 8192), 256, 0, s>>>(u, v, m, bitsV, keys, idx);
    count_launch();
    if ((st = radix_sort(keys, idx, m, bitsU + bitsV, s)) != PB_OK) break;
    if ((st = dalloc_t(&head, m, s)) != PB_OK) break;
    if ((st = dalloc_t(&cid, m + 1, s)) != PB_OK) break;
    k_heads<<<grid_for(m, 256, 8192), 256, 0, s>>>(keys, m, head);
    count_launch();
    if ((st = scan_u32(head, cid, m, s)) != PB_OK) break;
    if (cudaMemcpyAsync(&hm, cid + m, sizeof(uint32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) { st = fail(PB_ERR_CUDA, "dedupe readback failed"); break; }
    g->m = hm;
    if (g->m >= (uint64_t(1) << 31)) { st = fail(PB_ERR_INVALID, "more than 2^31-1 distinct edges"); break; }
    if ((st = dalloc_t(&g->eu, g->m, s)) != PB_OK) break;
    if ((st = dalloc_t(&g->ev, g->m, s)) != PB_OK) break;
    k_canon<<<grid_for(m, 256, 8192), 256, 0, s>>>(keys, idx, head, cid, m, bitsV, g->nU, g->in2c,
                                                    g->eu, g->ev, g->deg);
    count_launch();
    if (cudaGetLastError() != cudaSuccess) { st = fail(PB_ERR_CUDA, "canonical edge kernel failed"); break; }
  } while (0);
  if (st == PB_OK && n > 0) {
    do {
      if ((st = dalloc_t(&dmax, 2, s)) != PB_OK) break;
      if (cudaMemsetAsync(dmax, 0, 2 * sizeof(uint32_t), s) != cudaSuccess) { st = fail(PB_ERR_CUDA, "memset"); break; }
      k_maxdeg<<<grid_for(n, 256, 2048), 256, 0, s>>>(g->deg, n, g->nU, dmax);
      count_launch();
      if (cudaMemcpyAsync(hmax, dmax, sizeof(hmax), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
          cudaStreamSynchronize(s) != cudaSuccess) { st = fail(PB_ERR_CUDA, "degree readback failed"); break; }
      g->maxdegU = hmax[0];
      g->maxdegV = hmax[1];
    } while (0);
  }
  dfree(du, s); dfree(dv, s); dfree(keys, s); dfree(idx, s); dfree(head, s); dfree(cid, s);
  dfree(flag, s); dfree(dmax, s);
  return st;
}

// ---------------------------------------------------------------------------
// Rank keys (Sec. "Ranking").  Sorting (class << bitsN | global id) ascending
// gives the order; ties fall back to the global id.

__global__ void k_side_wedges(const uint32_t *__restrict__ deg, uint64_t n, uint32_t nU,
                              unsigned long long *w2) {
  // w2[0]: wedges with endpoints in U = sum over v of C(deg v, 2)
  // w2[1]: wedges with endpoints in V = sum over u of C(deg u, 2)
  unsigned long long a = 0, b = 0;
  for (size_t i = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += static_cast<size_t>(gridDim.x) * blockDim.x) {
    unsigned long long d = deg[i], c = d ? d * (d - 1) / 2 : 0;
    if (i < nU) b += c;
    else a += c;
  }
  a = warp_sum(a);
  b = warp_sum(b);
  if (lane_id() == 0) {
    if (a) atomicAdd(&w2[0], a);
    if (b) atomicAdd(&w2[1], b);
  }
}

// Side order: the first side (u_first) before the other, and within a side
// decreasing degree; the paper fixes only which side comes first, and W and
// the counts do not depend on the order inside a side.
__global__ void k_rank_keys(const uint32_t *__restrict__ deg, uint64_t n, uint32_t nU, int kind, int u_first,
                            uint32_t maxdeg, int dbits, int bitsN, uint64_t *__restrict__ keys) {
  for (size_t x = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x; x < n;
       x += static_cast<size_t>(gridDim.x) * blockDim.x) {
    uint32_t d = deg[x];
    uint64_t cls;
    if (kind == PB_RANK_DEGREE) {
      cls = maxdeg - d;                                          // decreasing degree
    } else if (kind == PB_RANK_SIDE) {
      const uint64_t second = (x < nU) ? !u_first : u_first;     // 1 for the side placed second
      cls = (second << dbits) | (maxdeg - d);
    } else {
      cls = d == 0 ? 32u : 31u - (31u - __clz(d));               // decreasing floor(log2 d), 0 last
    }
    keys[x] = (cls << bitsN) | x;
  }
}

__global__ void k_rank_from_keys(const uint64_t *__restrict__ keys, uint64_t n, int bitsN,
                                 uint32_t *__restrict__ rank, uint32_t *__restrict__ order) {
  const uint64_t mask = (uint64_t(1) << bitsN) - 1;
  for (size_t r = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x; r < n;
       r += static_cast<size_t>(gridDim.x) * blockDim.x) {
    uint32_t x = static_cast<uint32_t>(keys[r] & mask);
    order[r] = x;
    rank[x] = static_cast<uint32_t>(r);
  }
}

__global__ void k_custom_rank(const uint32_t *__restrict__ rank_of, uint64_t n, uint32_t *__restrict__ rank,
                              uint32_t *__restrict__ order, uint32_t *__restrict__ seen,
                              unsigned long long *bad) {
  for (size_t x = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x; x < n;
       x += static_cast<size_t>(gridDim.x) * blockDim.x) {
    uint32_t r = rank_of[x];
    rank[x] = r;
    if (r >= n || atomicAdd(&seen[r], 1u) != 0) {
      atomicAdd(bad, 1ull);
    } else {
      order[r] = static_cast<uint32_t>(x);
    }
  }
}

// ---------------------------------------------------------------------------
// Complement degeneracy orders (peeling rounds on the device, driven from the
// host: at most 33 rounds for the approximate order).

__global__ void k_id_csr(const uint32_t *__restrict__ eu, const uint32_t *__restrict__ ev, uint64_t m, uint32_t nU,
                         uint32_t *__restrict__ cur, uint32_t *__restrict__ nb) {
  for (size_t e = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < m;
       e += static_cast<size_t>(gridDim.x) * blockDim.x) {
    uint32_t a = eu[e], b = nU + ev[e];
    nb[atomicAdd(&cur[a], 1u)] = b;
    nb[atomicAdd(&cur[b], 1u)] = a;
  }
}

__device__ __forceinline__ uint32_t cd_key(uint32_t d, int approx) {
  return approx ? (d ? 32u - __clz(d) : 0u) : d;  // floor(log2 d) + 1, 0 for degree 0
}

__global__ void k_cd_max(const uint32_t *__restrict__ d, const uint32_t *__restrict__ rank, uint64_t n, int approx,
                         uint32_t *out) {
  uint32_t mx = 0;
  bool any = false;
  for (size_t x = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x; x < n;
       x += static_cast<size_t>(gridDim.x) * blockDim.x)
    if (rank[x] == 0xffffffffu) {
      uint32_t k = cd_key(d[x], approx);
      mx = k > mx ? k : mx;
      any = true;
    }
#pragma unroll
  for (int o = 16; o; o >>= 1) mx = max(mx, __shfl_xor_sync(FULL, mx, o));
  if (__any_sync(FULL, any) && lane_id() == 0) atomicMax(out, mx + 1);  // +1: 0 means nothing left
}

__global__ void k_cd_flag(const uint32_t *__restrict__ d, const uint32_t *__restrict__ rank, uint64_t n, int approx,
                          uint32_t best, uint32_t *__restrict__ flag) {
  for (size_t x = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x; x < n;
       x += static_cast<size_t>(gridDim.x) * blockDim.x)
    flag[x] = (rank[x] == 0xffffffffu && cd_key(d[x], approx) == best) ? 1u : 0u;
}

__global__ void k_cd_assign(const uint32_t *__restrict__ flag, const uint32_t *__restrict__ pos, uint64_t n,
                            uint32_t base, uint32_t *__restrict__ rank, uint32_t *__restrict__ order) {
  for (size_t x = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x; x < n;
       x += static_cast<size_t>(gridDim.x) * blockDim.x)
    if (flag[x]) {
      uint32_t r = base + pos[x];
      rank[x] = r;
      order[r] = static_cast<uint32_t>(x);
    }
}

// One warp per vertex peeled this round: its remaining neighbours lose a degree.
__global__ void k_cd_peel(const uint32_t *__restrict__ flag, const uint32_t *__restrict__ off,
                          const uint32_t *__restrict__ nb, const uint32_t *__restrict__ rank, uint64_t n,
                          uint32_t *__restrict__ d) {
  const uint64_t warps = static_cast<uint64_t>(gridDim.x) * blockDim.x / 32;
  for (uint64_t x = (static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x) / 32; x < n; x += warps) {
    if (!flag[x]) continue;
    for (uint32_t a = off[x] + lane_id(); a < off[x + 1]; a += 32) {
      uint32_t z = nb[a];
      if (rank[z] == 0xffffffffu) atomicSub(&d[z], 1u);
    }
  }
}

static pb_status codegen_rank(pb_graph *g, int approx, cudaStream_t s) {
  const uint64_t n = g->n, m = g->m;
  uint32_t *off = nullptr, *cur = nullptr, *nb = nullptr, *d = nullptr, *flag = nullptr, *pos = nullptr,
           *dmax = nullptr;
  pb_status st = PB_OK;
  do {
    if ((st = dalloc_t(&off, n + 1, s)) != PB_OK || (st = dalloc_t(&cur, n + 1, s)) != PB_OK ||
        (st = dalloc_t(&nb, 2 * m + 1, s)) != PB_OK || (st = dalloc_t(&d, n + 1, s)) != PB_OK ||
        (st = dalloc_t(&flag, n + 1, s)) != PB_OK || (st = dalloc_t(&pos, n + 1, s)) != PB_OK ||
        (st = dalloc_t(&dmax, 1, s)) != PB_OK) break;
    if ((st = scan_u32(g->deg, off, n, s)) != PB_OK) break;
    if (cudaMemcpyAsync(cur, off, (n + 1) * 4, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(d, g->deg, n * 4, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
        cudaMemsetAsync(g->rank, 0xff, (n + 1) * 4, s) != cudaSuccess) { st = fail(PB_ERR_CUDA, "copy"); break; }
    if (m) {
      k_id_csr<<<grid_for(m, 256, 8192), 256, 0, s>>>(g->eu, g->ev, m, g->nU, cur, nb);
      count_launch();
    }
    uint64_t done = 0;
    for (uint64_t round = 0; done < n; round++) {
      if (round > n + 1) { st = fail(PB_ERR_CUDA, "peeling made no progress"); break; }
      uint32_t best1 = 0, cnt = 0;
      if (cudaMemsetAsync(dmax, 0, 4, s) != cudaSuccess) { st = fail(PB_ERR_CUDA, "memset"); break; }
      k_cd_max<<<grid_for(n, 256, 4096), 256, 0, s>>>(d, g->rank, n, approx, dmax);
      count_launch();
      if (cudaMemcpyAsync(&best1, dmax, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
          cudaStreamSynchronize(s) != cudaSuccess) { st = fail(PB_ERR_CUDA, "round readback"); break; }
      if (best1 == 0) { st = fail(PB_ERR_CUDA, "peeling lost vertices"); break; }
      k_cd_flag<<<grid_for(n, 256, 8192), 256, 0, s>>>(d, g->rank, n, approx, best1 - 1, flag);
      count_launch();
      if ((st = scan_u32(flag, pos, n, s)) != PB_OK) break;
      k_cd_assign<<<grid_for(n, 256, 8192), 256, 0, s>>>(flag, pos, n, static_cast<uint32_t>(done), g->rank,
                                                         g->order);
      count_launch();
      k_cd_peel<<<grid_for(n * 32, 256, 8192), 256, 0, s>>>(flag, off, nb, g->rank, n, d);
      count_launch();
      if (cudaMemcpyAsync(&cnt, pos + n, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
          cudaStreamSynchronize(s) != cudaSuccess) { st = fail(PB_ERR_CUDA, "round readback"); break; }
      if (cnt == 0) { st = fail(PB_ERR_CUDA, "empty peeling round"); break; }
      done += cnt;
    }
  } while (0);
  dfree(off, s); dfree(cur, s); dfree(nb, s); dfree(d, s); dfree(flag, s); dfree(pos, s); dfree(dmax, s);
  return st;
}

// ---------------------------------------------------------------------------
// Renaming + adjacency.  Labels: U vertices [0, nU), V vertices [nU, n), each
// side in rank order.  Every canonical edge e = (u, v) gives two arcs: 2e from
// u to v and 2e+1 back.  Keys (label(src) << bitsN) | (maxrank - rank(nbr))
// sort the arcs by source, then by decreasing neighbour rank.

__global__ void k_is_u(const uint32_t *__restrict__ order, uint64_t n, uint32_t nU, uint32_t *__restrict__ f) {
  for (size_t r = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x; r < n;
       r += static_cast<size_t>(gridDim.x) * blockDim.x)
    f[r] = order[r] < nU ? 1u : 0u;
}

__global__ void k_labels(const uint32_t *__restrict__ order, const uint32_t *__restrict__ cu, uint64_t n,
                         uint32_t nU, const uint32_t *__restrict__ deg, uint32_t *__restrict__ label,
                         uint32_t *__restrict__ lrank, uint32_t *__restrict__ rlab, uint32_t *__restrict__ degl) {
  for (size_t r = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x; r < n;
       r += static_cast<size_t>(gridDim.x) * blockDim.x) {
    uint32_t x = order[r];
    uint32_t l = x < nU ? cu[r] : nU + static_cast<uint32_t>(r - cu[r]);
    label[x] = l;
    lrank[l] = static_cast<uint32_t>(r);
    rlab[r] = l;
    degl[l] = deg[x];
  }
}

// The two arcs of every canonical edge, keyed (label(src), maxrank -
// rank(nbr)), and in the same pass deg_x(x) (degp: the neighbours of x ranked
// above it): each edge adds one to its lower-ranked endpoint, warp-aggregated
// since edges come grouped by U endpoint.
__global__ void k_arc_keys(const uint32_t *__restrict__ eu, const uint32_t *__restrict__ ev, uint64_t m,
                           uint32_t nU, const uint32_t *__restrict__ rank, const uint32_t *__restrict__ label,
                           int bitsN, uint64_t *__restrict__ keys, uint32_t *__restrict__ vals,
                           uint32_t *__restrict__ degp) {
  const uint64_t mask = (uint64_t(1) << bitsN) - 1;
  const size_t stride = static_cast<size_t>(gridDim.x) * blockDim.x;
  const size_t start = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const size_t iters = (m + stride - 1) / stride;
  for (size_t itn = 0; itn < iters; itn++) {  // uniform trip count: the whole warp reaches the match
    const size_t e = start + itn * stride;
    uint32_t t = 0xffffffffu;
    if (e < m) {
      const uint32_t a = eu[e], b = nU + ev[e];
      const uint32_t ra = rank[a], rb = rank[b], la = label[a], lb = label[b];
      keys[2 * e] = (static_cast<uint64_t>(la) << bitsN) | (mask - rb);
      vals[2 * e] = static_cast<uint32_t>(2 * e);
      keys[2 * e + 1] = (static_cast<uint64_t>(lb) << bitsN) | (mask - ra);
      vals[2 * e + 1] = static_cast<uint32_t>(2 * e + 1);
      t = rb > ra ? la : lb;
    }
    const uint32_t peers = __match_any_sync(FULL, t);
    if (t != 0xffffffffu && lane_id() == static_cast<uint32_t>(__ffs(peers) - 1)) atomicAdd(&degp[t], __popc(peers));
  }
}

// Slot s holds the arc of sort key keys[s]: its neighbour's label comes from
// the rank in the key (rlab: label of each rank, a table that stays in L2),
// and the arc's edge learns its slot.
__global__ void k_arcs_out(const uint64_t *__restrict__ keys, const uint32_t *__restrict__ vals, uint64_t na,
                           int bitsN, const uint32_t *__restrict__ rlab, uint32_t *__restrict__ adj,
                           uint32_t *__restrict__ slotA, uint32_t *__restrict__ slotB) {
  const uint64_t mask = (uint64_t(1) << bitsN) - 1;
  for (size_t s = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x; s < na;
       s += static_cast<size_t>(gridDim.x) * blockDim.x) {
    const uint32_t a = vals[s], e = a >> 1;
    adj[s] = rlab[mask - (keys[s] & mask)];
    if (a & 1u) slotB[e] = static_cast<uint32_t>(s);  // arc from v to u
    else slotA[e] = static_cast<uint32_t>(s);
  }
}

// cpos[s] = position of the list owner x in y's list (= deg_x(y), the number
// of y's neighbours ranked above x, since lists are strictly decreasing in
// rank).  The same pass counts the wedges of every owner in both directions
// (warp-aggregated atomics):
//   wc[x]  (x the lower-ranked endpoint, Algorithm 2): cpos over the first
//          degp[x] slots of x;
//   wcr[x] (x the higher-ranked endpoint): for every neighbour y (slot s),
//          the entries of y's list ranked below both y and x.
__global__ void k_cpos_wedges(const uint64_t *__restrict__ keys, const uint32_t *__restrict__ vals,
                              uint64_t na, int bitsN, const uint32_t *__restrict__ off,
                              const uint32_t *__restrict__ adj, const uint32_t *__restrict__ slotA,
                              const uint32_t *__restrict__ slotB, const uint32_t *__restrict__ lrank,
                              const uint32_t *__restrict__ degp, uint32_t *__restrict__ cpos,
                              unsigned long long *__restrict__ wc, unsigned long long *__restrict__ wcr) {
  const uint64_t mask = (uint64_t(1) << bitsN) - 1;
  const size_t stride = static_cast<size_t>(gridDim.x) * blockDim.x;
  const size_t start = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const size_t iters = (na + stride - 1) / stride;
  for (size_t itn = 0; itn < iters; itn++) {  // uniform trip count: the whole warp reaches the match
    const size_t s = start + itn * stride;
    const bool valid = s < na;
    uint32_t x = 0xffffffffu;
    unsigned long long c = 0, cr = 0;
    if (valid) {
      const uint32_t a = vals[s], y = adj[s];
      const uint32_t other = (a & 1u) ? slotA[a >> 1] : slotB[a >> 1];
      const uint32_t oy = off[y], cp = other - oy;
      cpos[s] = cp;
      x = static_cast<uint32_t>(keys[s] >> bitsN);
      const uint32_t rx = lrank[x], ry = static_cast<uint32_t>(mask - (keys[s] & mask));
      if (ry > rx) c = cp;
      const uint32_t dy = off[y + 1] - oy;
      uint32_t st = degp[y];
      if (cp + 1 > st) st = cp + 1;
      cr = dy > st ? dy - st : 0;
    }
    const uint32_t peers = __match_any_sync(FULL, x);
    unsigned long long tot = 0, totr = 0;
    for (uint32_t q = peers; q; q &= q - 1) {
      const int l = __ffs(q) - 1;
      tot += __shfl_sync(peers, c, l);
      totr += __shfl_sync(peers, cr, l);
    }
    if (valid && lane_id() == static_cast<uint32_t>(__ffs(peers) - 1)) {
      if (tot) atomicAdd(&wc[x], tot);
      if (totr) atomicAdd(&wcr[x], totr);
    }
  }
}

__global__ void k_max_u64(const unsigned long long *__restrict__ a, uint64_t n, unsigned long long *out) {
  unsigned long long mx = 0;
  for (size_t i = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += static_cast<size_t>(gridDim.x) * blockDim.x)
    mx = a[i] > mx ? a[i] : mx;
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    unsigned long long y = __shfl_xor_sync(FULL, mx, o);
    mx = y > mx ? y : mx;
  }
  if (lane_id() == 0 && mx) atomicMax(out, mx);
}

void free_ranked(pb_graph *g, cudaStream_t s) {
  dfree(g->rank, s); dfree(g->order, s); dfree(g->label, s); dfree(g->off, s); dfree(g->adj, s);
  dfree(g->cpos, s); dfree(g->degp, s); dfree(g->wpre, s); dfree(g->wpre_rev, s); dfree(g->slotA, s);
  dfree(g->slotB, s);
  g->rank = g->order = g->label = g->off = g->adj = g->cpos = g->degp = g->slotA = g->slotB = nullptr;
  g->wpre = g->wpre_rev = nullptr;
  g->rank_kind = -1;
  g->W = g->maxw = g->maxw_rev = 0;
}

static pb_status alloc_ranked(pb_graph *g, cudaStream_t s) {
  const uint64_t n = g->n, na = 2 * g->m;
  PB_TRY(dalloc_t(&g->rank, n + 1, s));
  PB_TRY(dalloc_t(&g->order, n + 1, s));
  PB_TRY(dalloc_t(&g->label, n + 1, s));
  PB_TRY(dalloc_t(&g->off, n + 1, s));
  PB_TRY(dalloc_t(&g->adj, na + 1, s));
  PB_TRY(dalloc_t(&g->cpos, na + 1, s));
  PB_TRY(dalloc_t(&g->degp, n + 1, s));
  PB_TRY(dalloc_t(&g->wpre, n + 1, s));
  PB_TRY(dalloc_t(&g->wpre_rev, n + 1, s));
  PB_TRY(dalloc_t(&g->slotA, g->m + 1, s));
  PB_TRY(dalloc_t(&g->slotB, g->m + 1, s));
  return PB_OK;
}

pb_status rank_graph(pb_graph *g, int kind, const uint32_t *rank_of, int on_device, cudaStream_t s) {
  free_ranked(g, s);
  const uint64_t n = g->n, m = g->m, na = 2 * m;
  const int bitsN = g->bitsN;
  pb_status st = alloc_ranked(g, s);
  if (st != PB_OK) { free_ranked(g, s); return st; }
  uint64_t *keys = nullptr;
  uint32_t *vals = nullptr, *tmp = nullptr, *drank = nullptr, *lrank = nullptr, *cu = nullptr, *rlab = nullptr;
  unsigned long long *acc = nullptr, *wc = nullptr;
  unsigned long long hacc[2] = {0, 0};
  do {
    if ((st = dalloc_t(&acc, 2, s)) != PB_OK) break;
    if (cudaMemsetAsync(acc, 0, 2 * sizeof(unsigned long long), s) != cudaSuccess) { st = fail(PB_ERR_CUDA, "memset"); break; }
    // ---- 0. wedges of side order (input to the ranking choice)
    if (n) {
      k_side_wedges<<<grid_for(n, 256, 2048), 256, 0, s>>>(g->deg, n, g->nU, acc);
      count_launch();
    }
    if (cudaMemcpyAsync(hacc, acc, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) { st = fail(PB_ERR_CUDA, "side wedge readback"); break; }
    g->w_side_U = hacc[0];
    g->w_side_V = hacc[1];
    if (cudaMemsetAsync(acc, 0, 2 * sizeof(unsigned long long), s) != cudaSuccess) { st = fail(PB_ERR_CUDA, "memset"); break; }
    // ---- 1. the ranking
    if (rank_of) {
      const uint32_t *src = rank_of;
      if (!on_device) {
        if ((st = dalloc_t(&drank, n + 1, s)) != PB_OK) break;
        if (cudaMemcpyAsync(drank, rank_of, n * sizeof(uint32_t), cudaMemcpyHostToDevice, s) != cudaSuccess) { st = fail(PB_ERR_CUDA, "rank upload"); break; }
        src = drank;
      }
      if ((st = dalloc_t(&tmp, n + 1, s)) != PB_OK) break;
      if (cudaMemsetAsync(tmp, 0, (n + 1) * sizeof(uint32_t), s) != cudaSuccess) { st = fail(PB_ERR_CUDA, "memset"); break; }
      if (n) {
        k_custom_rank<<<grid_for(n, 256, 8192), 256, 0, s>>>(src, n, g->rank, g->order, tmp, acc);
        count_launch();
      }
      if (cudaMemcpyAsync(hacc, acc, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
          cudaStreamSynchronize(s) != cudaSuccess) { st = fail(PB_ERR_CUDA, "rank check readback"); break; }
      if (hacc[0]) { st = fail(PB_ERR_INVALID, "rank_of is not a permutation of [0, %llu)", (unsigned long long)n); break; }
      dfree(tmp, s);
      tmp = nullptr;
    } else if (kind == PB_RANK_COMPLEMENT_DEGENERACY || kind == PB_RANK_APPROX_COMPLEMENT_DEGENERACY) {
      if ((st = codegen_rank(g, kind == PB_RANK_APPROX_COMPLEMENT_DEGENERACY, s)) != PB_OK) break;
    } else {
      const int u_first = g->w_side_U <= g->w_side_V;
      uint32_t maxdeg = g->maxdegU > g->maxdegV ? g->maxdegU : g->maxdegV;
      const int dbits = bits_for(maxdeg);
      int cbits = kind == PB_RANK_DEGREE ? dbits : (kind == PB_RANK_SIDE ? dbits + 1 : 6);
      if ((st = dalloc_t(&keys, n + 1, s)) != PB_OK) break;
      if (n) {
        k_rank_keys<<<grid_for(n, 256, 8192), 256, 0, s>>>(g->deg, n, g->nU, kind, u_first, maxdeg, dbits, bitsN,
                                                            keys);
        count_launch();
      }
      if ((st = radix_sort(keys, nullptr, n, bitsN + cbits, s)) != PB_OK) break;
      if (n) {
        k_rank_from_keys<<<grid_for(n, 256, 8192), 256, 0, s>>>(keys, n, bitsN, g->rank, g->order);
        count_launch();
      }
      dfree(keys, s);
      keys = nullptr;
    }
    // ---- 2. labels (side-major, rank order within a side) and offsets
    if ((st = dalloc_t(&tmp, n + 1, s)) != PB_OK) break;
    if ((st = dalloc_t(&cu, n + 1, s)) != PB_OK) break;
    if ((st = dalloc_t(&lrank, n + 1, s)) != PB_OK) break;
    if ((st = dalloc_t(&rlab, n + 1, s)) != PB_OK) break;
    if (n) {
      k_is_u<<<grid_for(n, 256, 8192), 256, 0, s>>>(g->order, n, g->nU, tmp);
      count_launch();
    }
    if ((st = scan_u32(tmp, cu, n, s)) != PB_OK) break;
    if (n) {
      k_labels<<<grid_for(n, 256, 8192), 256, 0, s>>>(g->order, cu, n, g->nU, g->deg, g->label, lrank, rlab, tmp);
      count_launch();
    }
    if ((st = scan_u32(tmp, g->off, n, s)) != PB_OK) break;
    dfree(tmp, s);
    tmp = nullptr;
    if (cudaMemsetAsync(g->degp, 0, (n + 1) * sizeof(uint32_t), s) != cudaSuccess) { st = fail(PB_ERR_CUDA, "memset"); break; }
    if ((st = dalloc_t(&wc, 2 * (n + 1), s)) != PB_OK) break;  // both directions
    if (cudaMemsetAsync(wc, 0, 2 * (n + 1) * sizeof(unsigned long long), s) != cudaSuccess) { st = fail(PB_ERR_CUDA, "memset"); break; }
    unsigned long long *wcr = wc + (n + 1);
    if (na > 0) {
      // ---- 3. arcs sorted by (source, decreasing neighbour)
      if ((st = dalloc_t(&keys, na, s)) != PB_OK) break;
      if ((st = dalloc_t(&vals, na, s)) != PB_OK) break;
      k_arc_keys<<<grid_for(m, 256, 8192), 256, 0, s>>>(g->eu, g->ev, m, g->nU, g->rank, g->label, bitsN, keys,
                                                         vals, g->degp);
      count_launch();
      if ((st = radix_sort(keys, vals, na, 2 * bitsN, s)) != PB_OK) break;
      k_arcs_out<<<grid_for(na, 256, 8192), 256, 0, s>>>(keys, vals, na, bitsN, rlab, g->adj, g->slotA, g->slotB);
      count_launch();
      // ---- 4. (same pass) wedges per owner in both directions, then the work split prefixes
      k_cpos_wedges<<<grid_for(na, 256, 8192), 256, 0, s>>>(keys, vals, na, bitsN, g->off, g->adj, g->slotA,
                                                             g->slotB, lrank, g->degp, g->cpos, wc, wcr);
      count_launch();
    }
    if ((st = scan_u64(reinterpret_cast<uint64_t *>(wc), g->wpre, n, s)) != PB_OK) break;
    if (cudaMemsetAsync(acc, 0, 2 * sizeof(unsigned long long), s) != cudaSuccess) { st = fail(PB_ERR_CUDA, "memset"); break; }
    if (n) {
      k_max_u64<<<grid_for(n, 256, 2048), 256, 0, s>>>(wc, n, acc);
      count_launch();
    }
    // the same wedges counted at their higher-ranked endpoint
    if ((st = scan_u64(reinterpret_cast<uint64_t *>(wcr), g->wpre_rev, n, s)) != PB_OK) break;
    if (n) {
      k_max_u64<<<grid_for(n, 256, 2048), 256, 0, s>>>(wcr, n, acc + 1);
      count_launch();
    }
    uint64_t hW = 0, hWr = 0;
    if (cudaMemcpyAsync(&hW, g->wpre + n, sizeof(uint64_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(&hWr, g->wpre_rev + n, sizeof(uint64_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(hacc, acc, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) { st = fail(PB_ERR_CUDA, "wedge count readback: %s", cudaGetErrorString(cudaGetLastError())); break; }
    if (hW != hWr) { st = fail(PB_ERR_CUDA, "wedge totals disagree (%llu vs %llu)", (unsigned long long)hW, (unsigned long long)hWr); break; }
    g->W = hW;
    g->maxw = hacc[0];
    g->maxw_rev = hacc[1];
    g->rank_kind = rank_of ? 5 : kind;
  } while (0);
  dfree(keys, s); dfree(vals, s); dfree(tmp, s); dfree(drank, s); dfree(acc, s); dfree(wc, s);
  dfree(lrank, s); dfree(cu, s); dfree(rlab, s);
  if (st != PB_OK) free_ranked(g, s);
  return st;
}

}  // namespace pb
