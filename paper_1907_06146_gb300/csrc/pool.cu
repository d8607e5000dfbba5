// Candidate pools (Alg. 3: for each neighbour n of node i, add n and the neighbours of n;
// drop repeats; stop once the pool holds >= l ids) and the SSG prune of each pool.
//
// One warp per node.  Ids are gathered a kNN row at a time (coalesced int32 row reads);
// a shared-memory open-addressing hash set removes repeats; the fp32 distances to node i
// are computed by teams of 8 lanes with float4 loads; a warp bitonic sort orders the
// pool by (d2, id), and near-equal fp32 distances are re-ordered in fp64 so that the
// order equals the exact one.
#include "common.cuh"
#include "graph_dev.cuh"
#include "knn.cuh"

namespace ssg {

__device__ __forceinline__ uint32_t hash_slot(int32_t id, int log2cap) {
  return ((uint32_t)id * 2654435761u) >> (32 - log2cap);
}

// Insert id into the set; true if it was not there.  Distinct ids may be inserted
// concurrently by different lanes.
__device__ __forceinline__ bool hash_insert(int32_t* h, int log2cap, int32_t id) {
  const uint32_t mask = (1u << log2cap) - 1;
  uint32_t s = hash_slot(id, log2cap);
  for (;;) {
    int32_t old = atomicCAS(h + s, -1, id);
    if (old == -1) return true;
    if (old == id) return false;
    s = (s + 1) & mask;
  }
}

// keys[0, m): node i's candidate ids.  Orders them by (d2, id) -- fp32 distances, runs of
// near-equal values re-sorted in fp64 unless the data are exact -- and writes the first
// L as node i's pool.  keys has room for the next power of two >= m; d64 for m doubles.
__device__ __forceinline__ void pool_finish(uint64_t* keys, int m, int L, int exact, double* d64,
                                            const float* __restrict__ X,
                                            const uint8_t* __restrict__ X8, int ld, int d,
                                            int64_t i, float rel, int32_t* __restrict__ pool_id,
                                            float* __restrict__ pool_d2,
                                            int32_t* __restrict__ pool_len,
                                            unsigned long long* __restrict__ n_order) {
  const int lane = lane_id();
  const float* xi = X + i * ld;
  if (X8)
    warp_fill_dist_keys_u8(keys, m, X8, ld, X8 + i * ld);
  else
    warp_fill_dist_keys(keys, m, X, ld, xi);
  int mp = 1;
  while (mp < m) mp <<= 1;
  for (int t = m + lane; t < mp; t += 32) keys[t] = KEY_NONE;
  __syncwarp();
  warp_sort_keys_wide(keys, mp);
  const int keep = m < L ? m : L;
  if (!exact && m > 1) {
    int f = warp_fix_runs(keys, m, keep, d64, X, ld, d, xi, rel);
    for (int o = 16; o > 0; o >>= 1) f += __shfl_xor_sync(0xffffffffu, f, o);
    if (lane == 0 && f) atomicAdd(n_order, (unsigned long long)f);
  }
  for (int t = lane; t < L; t += 32) {
    const bool v = t < keep;
    pool_id[i * L + t] = v ? key_id(keys[t]) : -1;
    pool_d2[i * L + t] = v ? key_dist(keys[t]) : __int_as_float(0x7f800000);
  }
  if (lane == 0) pool_len[i] = keep;
}

// Node i's candidate ids, in the order of Alg. 3's loop (or its own-row-first reading),
// repeats and i itself dropped, into keys[0, m); returns m.  One warp; hset (1 << log2h
// entries) must hold -1 everywhere.
__device__ __forceinline__ int warp_collect_pool(int64_t i, const int32_t* __restrict__ knn,
                                                 int K, int L, int own_first, int log2h,
                                                 int32_t* hset, uint64_t* keys) {
  const int lane = lane_id();
  int m = 0;
  if (own_first) {
    // the node's own row whole, then its neighbours' rows while the pool holds < L ids
    for (int t = -1; t < K; ++t) {
      if (t >= 0 && m >= L) break;
      const int32_t src = t < 0 ? (int32_t)i : knn[i * K + t];
      if (src < 0) break;  // a row of an approximate graph with fewer than K neighbours
      for (int c = 0; c < K; c += 32) {
        const int idx = c + lane;
        const int32_t id = idx < K ? knn[(int64_t)src * K + idx] : -1;
        bool fresh = id >= 0 && id != (int32_t)i && hash_insert(hset, log2h, id);
        const unsigned bal = __ballot_sync(0xffffffffu, fresh);
        if (fresh) keys[m + __popc(bal & lanemask_lt())] = (uint64_t)(uint32_t)id;
        m += __popc(bal);
      }
    }
  } else {
    for (int t = 0; t < K; ++t) {
      const int32_t nb = knn[i * K + t];
      if (nb < 0) break;  // a row of an approximate graph with fewer than K neighbours
      for (int c = 0; c <= K; c += 32) {  // the batch {nb} + knn(nb): K + 1 distinct ids
        const int idx = c + lane;
        int32_t id = -1;
        if (idx <= K) id = idx == 0 ? nb : knn[(int64_t)nb * K + idx - 1];
        bool fresh = id >= 0 && id != (int32_t)i && hash_insert(hset, log2h, id);
        const unsigned bal = __ballot_sync(0xffffffffu, fresh);
        if (fresh) keys[m + __popc(bal & lanemask_lt())] = (uint64_t)(uint32_t)id;
        m += __popc(bal);
      }
      if (m >= L) break;
    }
  }
  __syncwarp();
  return m;
}

__global__ void k_pool(const float* __restrict__ X, const uint8_t* __restrict__ X8, int ld, int d,
                       int64_t n,
                       const int32_t* __restrict__ knn, int K, int L, int cap, int log2h,
                       int hbytes, int own_first, int exact, float rel,
                       int32_t* __restrict__ pool_id,
                       float* __restrict__ pool_d2, int32_t* __restrict__ pool_len,
                       unsigned long long* __restrict__ n_order) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  const int wpb = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = lane_id();
  const int hcap = 1 << log2h;
  const size_t per_warp = (size_t)cap * 8 + (size_t)hbytes;
  uint64_t* keys = (uint64_t*)(sm_raw + warp * per_warp);
  int32_t* hset = (int32_t*)(keys + cap);
  const int64_t i = (int64_t)blockIdx.x * wpb + warp;
  if (i >= n) return;

  for (int t = lane; t < hcap; t += 32) hset[t] = -1;
  __syncwarp();
  const int m = warp_collect_pool(i, knn, K, L, own_first, log2h, hset, keys);
  __syncwarp();
  pool_finish(keys, m, L, exact, (double*)hset, X, X8, ld, d, i, rel, pool_id, pool_d2, pool_len,
              n_order);
}

// The same pools for nodes with long rows (above 256 values), one node per block of eight
// warps: at these widths the distances (some L rows of d floats per node) are nearly all
// of the work, and a warp per node with its key and hash buffers beside it leaves the SM
// with too few warps to cover the row loads.  Warp 0 gathers the ids exactly as k_pool
// does, the eight warps share the distances, the block sorts, warp 0 re-sorts near-equal
// runs; the pool is k_pool's, entry for entry.
constexpr int POOLW_WARPS = 8;
__global__ void __launch_bounds__(POOLW_WARPS * 32)
    k_pool_wide(const float* __restrict__ X, int ld, int d, int64_t n,
                const int32_t* __restrict__ knn, int K, int L, int cap, int log2h, int own_first,
                int exact, float rel, int32_t* __restrict__ pool_id, float* __restrict__ pool_d2,
                int32_t* __restrict__ pool_len, unsigned long long* __restrict__ n_order) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  __shared__ int s_m;
  const int warp = threadIdx.x >> 5, lane = lane_id();
  const int hcap = 1 << log2h;
  uint64_t* keys = (uint64_t*)sm_raw;
  int32_t* hset = (int32_t*)(keys + cap);
  for (int64_t i = blockIdx.x; i < n; i += gridDim.x) {
    __syncthreads();  // the previous node's readers are done
    for (int t = threadIdx.x; t < hcap; t += blockDim.x) hset[t] = -1;
    __syncthreads();
    if (warp == 0) {
      const int m0 = warp_collect_pool(i, knn, K, L, own_first, log2h, hset, keys);
      if (lane == 0) s_m = m0;
    }
    __syncthreads();
    const int m = s_m;
    const float* xi = X + i * ld;
    warp_fill_dist_keys_steps(keys, m, X, ld, xi, 8 * warp, 8 * POOLW_WARPS);
    int mp = 1;
    while (mp < m) mp <<= 1;
    for (int t = m + threadIdx.x; t < mp; t += blockDim.x) keys[t] = KEY_NONE;
    __syncthreads();
    block_sort_keys(keys, mp);
    const int keep = m < L ? m : L;
    if (warp == 0 && !exact && m > 1) {
      int f = warp_fix_runs(keys, m, keep, (double*)hset, X, ld, d, xi, rel);
      for (int o = 16; o > 0; o >>= 1) f += __shfl_xor_sync(0xffffffffu, f, o);
      if (lane == 0 && f) atomicAdd(n_order, (unsigned long long)f);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < L; t += blockDim.x) {
      const bool v = t < keep;
      pool_id[i * L + t] = v ? key_id(keys[t]) : -1;
      pool_d2[i * L + t] = v ? key_dist(keys[t]) : __int_as_float(0x7f800000);
    }
    if (threadIdx.x == 0) pool_len[i] = keep;
  }
}

// Pools from given candidates: row i's pool is the L nearest of its KS candidate ids
// (cand [n][KS], -1 padded; i itself skipped), ordered as k_pool orders them.
__global__ void k_pool_cand(const float* __restrict__ X, const uint8_t* __restrict__ X8, int ld,
                            int d, int64_t n,
                            const int32_t* __restrict__ cand, int KS, int L, int cap, int exact,
                            float rel, int32_t* __restrict__ pool_id, float* __restrict__ pool_d2,
                            int32_t* __restrict__ pool_len, unsigned long long* __restrict__ n_order) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  const int wpb = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = lane_id();
  uint64_t* keys = (uint64_t*)(sm_raw + (size_t)warp * cap * 16);
  double* d64 = (double*)(keys + cap);
  const int64_t i = (int64_t)blockIdx.x * wpb + warp;
  if (i >= n) return;
  int m = 0;
  for (int c = 0; c < KS; c += 32) {
    const int t = c + lane;
    const int32_t id = t < KS ? cand[i * KS + t] : -1;
    const bool v = id >= 0 && id != (int32_t)i;
    const unsigned bal = __ballot_sync(0xffffffffu, v);
    if (v) keys[m + __popc(bal & lanemask_lt())] = (uint64_t)(uint32_t)id;
    m += __popc(bal);
  }
  __syncwarp();
  pool_finish(keys, m, L, exact, d64, X, X8, ld, d, i, rel, pool_id, pool_d2, pool_len, n_order);
}

void pool_run(const float* X, const uint8_t* X8, int ld, int d, int64_t n, const int32_t* knn,
              int K, int L, int exact, int32_t* pool_id, float* pool_d2, int32_t* pool_len,
              Counters* dctr, cudaStream_t st, int own_first) {
  const int cap = next_pow2(L + K + 1);
  // after the keys: the id hash set (load factor at most 0.6), reused as the fp64 scratch of
  // the run re-sorts (one double per pool entry)
  const int mmax = L + K + 1;
  int log2h = 0;
  while ((1 << log2h) * 3 < 5 * mmax) ++log2h;
  const size_t hbytes =
      ((std::max<size_t>(((size_t)1 << log2h) * 4, (size_t)mmax * 8) + 15) / 16) * 16;
  const size_t per_warp = (size_t)cap * 8 + hbytes;
  if (!X8 && ((d + 3) & ~3) > 256) {
    // long float rows: a block per node
    ensure_smem((const void*)k_pool_wide, per_warp);
    int per_sm = 0;
    SSG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pool_wide, POOLW_WARPS * 32,
                                                           per_warp));
    const int64_t grid = std::min<int64_t>(std::max<int64_t>(n, 1),
                                           (int64_t)std::max(1, per_sm) * num_sms());
    SSG_LAUNCH(k_pool_wide, (unsigned)grid, POOLW_WARPS * 32, per_warp, st, X, ld, d, n, knn, K, L,
               cap, log2h, own_first, exact, dist_rel_team8c(ld), pool_id, pool_d2, pool_len,
               &dctr->order_fp64);
    return;
  }
  int wpb = (int)std::max<size_t>(1, std::min<size_t>(8, (96 * 1024) / per_warp));
  const size_t smem = per_warp * wpb;
  ensure_smem((const void*)k_pool, smem);
  SSG_LAUNCH(k_pool, (unsigned)ceil_div(n, wpb), wpb * 32, smem, st, X, X8, ld, d, n, knn, K, L, cap,
             log2h, (int)hbytes, own_first, exact, dist_rel_team8c(ld), pool_id, pool_d2, pool_len,
             &dctr->order_fp64);
}

void pool_from_candidates(const float* X, const uint8_t* X8, int ld, int d, int64_t n,
                          const int32_t* cand, int KS, int L, int exact, int32_t* pool_id,
                          float* pool_d2, int32_t* pool_len, Counters* dctr, cudaStream_t st) {
  const int cap = next_pow2(KS);
  const int wpb = 8;
  const size_t smem = (size_t)cap * 16 * wpb;
  ensure_smem((const void*)k_pool_cand, smem);
  SSG_LAUNCH(k_pool_cand, (unsigned)ceil_div(n, wpb), wpb * 32, smem, st, X, X8, ld, d, n, cand, KS,
             L, cap, exact, dist_rel_team8c(ld), pool_id, pool_d2, pool_len, &dctr->order_fp64);
}

// ---------------------------------------------------------------------------------------
// Prune (Alg. 2 selection on each pool, Alg. 3).
// ---------------------------------------------------------------------------------------
// One warp per node.  Vg == nullptr: the kept vectors sit in shared memory
// (warp_prune_node); otherwise each warp of the (persistent) grid owns the global slot
// Vg + warp_index * (R + 1) * d4 for wide rows (warp_prune_node_wide).
__global__ void k_prune(const float* __restrict__ X, int ld, int d, int64_t n,
                        const int32_t* __restrict__ pool_id, const int32_t* __restrict__ pool_len,
                        int L, int R, float cosA32, double cosA64, float margin,
                        int32_t* __restrict__ adj, int32_t* __restrict__ deg,
                        unsigned long long* __restrict__ n64, float* __restrict__ Vg,
                        double border, unsigned long long* __restrict__ nborder) {
  extern __shared__ __align__(16) float smf[];
  const int wpb = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = lane_id();
  const int64_t gwarp = (int64_t)blockIdx.x * wpb + warp;
  const int64_t nwarps = (int64_t)gridDim.x * wpb;
  const int d4 = (d + 3) & ~3;
  const int D1 = prune_row_stride(d);
  float* base = smf + (size_t)warp * (Vg ? prune_wide_smem_floats(d, R) : prune_smem_floats(d, R));
  for (int64_t i = gwarp; i < n; i += nwarps) {
    int32_t* out = adj + i * R;
    int kept;
    if (Vg) {
      kept = warp_prune_node_wide(X, ld, d, i, pool_id + i * L, pool_len[i], R, cosA32, cosA64,
                                  margin, Vg + (size_t)gwarp * (R + 1) * d4, base, base + d4,
                                  base + 2 * d4, out, n64, border, nborder);
    } else {
      float* xs = base + (size_t)(R + 1) * D1;
      kept = warp_prune_node(X, ld, d, i, pool_id + i * L, pool_len[i], R, cosA32, cosA64, margin,
                             base, D1, xs, xs + D1, out, n64, border, nborder);
    }
    for (int t = kept + lane; t < R; t += 32) out[t] = -1;
    if (lane == 0) deg[i] = kept;
    __syncwarp();
  }
}

void prune_run(const float* X, int ld, int d, int64_t n, const int32_t* pool_id,
               const int32_t* pool_len, int L, int R, double cos_a, double border, int32_t* adj,
               int32_t* deg, Counters* dctr, cudaStream_t st, int wide_blocks) {
  const bool wide = prune_is_wide(d, R);
  if (prune_block_preferred(d, R)) {
    prune_run_wide(X, ld, d, n, pool_id, pool_len, L, R, cos_a, border, adj, deg, dctr, st,
                   wide_blocks);
    return;
  }
  const size_t per_warp =
      (wide ? prune_wide_smem_floats(d, R) : prune_smem_floats(d, R)) * sizeof(float);
  int wpb = (int)std::max<size_t>(1, std::min<size_t>(8, (96 * 1024) / per_warp));
  const size_t smem = per_warp * wpb;
  ensure_smem((const void*)k_prune, smem);
  int blocks_per_sm = 0;
  SSG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, k_prune, wpb * 32, smem));
  // wide rows: a persistent grid (one device slot per warp); otherwise one warp per node
  const int64_t grid =
      wide ? std::min<int64_t>(ceil_div(n, wpb), (int64_t)std::max(1, blocks_per_sm) * num_sms())
           : ceil_div(n, wpb);
  Scratch<float> Vg;
  if (wide) Vg.alloc((size_t)grid * wpb * (R + 1) * ((d + 3) & ~3), st);
  SSG_LAUNCH(k_prune, (unsigned)grid, wpb * 32, smem, st, X, ld, d, n, pool_id, pool_len, L, R,
             (float)cos_a, cos_a, angle_margin_fp32(d) + (float)border, adj, deg, &dctr->angle_fp64,
             Vg.p, border, &dctr->angle_border);
}

}  // namespace ssg

// ---------------------------------------------------------------------------------------
// The prune of many indices at once (the batched build): one persistent launch per row
// shape class over work items (index, node).  The items are bucketed by pool length and
// handed out longest pools first from one atomic counter, so indices of very different
// sizes and nodes of very different pool lengths share the GPU without a tail; every node
// is pruned by the same warp routine as prune_run, so the adjacency is the same bit for bit.
// ---------------------------------------------------------------------------------------
namespace ssg {

__global__ void k_prune_batched(const PruneJob* __restrict__ jobs, const int2* __restrict__ items,
                                int64_t nitems, unsigned long long* __restrict__ next,
                                float* __restrict__ Vg, size_t vg_stride, size_t warp_floats,
                                int wide) {
  extern __shared__ __align__(16) float smf[];
  const int wpb = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = lane_id();
  const int64_t gwarp = (int64_t)blockIdx.x * wpb + warp;
  float* base = smf + (size_t)warp * warp_floats;
  for (;;) {
    unsigned long long it = 0;
    if (lane == 0) it = atomicAdd(next, 1ull);
    it = __shfl_sync(0xffffffffu, it, 0);
    if (it >= (unsigned long long)nitems) break;
    const int2 w = items[it];
    const PruneJob& jb = jobs[w.x];
    const int64_t i = w.y;
    int32_t* out = jb.adj + i * jb.R;
    const int32_t* cand = jb.pool_id + i * jb.L;
    const int len = jb.pool_len[i];
    int kept;
    if (wide) {
      const int d4 = (jb.d + 3) & ~3;
      kept = warp_prune_node_wide(jb.X, jb.ld, jb.d, i, cand, len, jb.R, jb.cosA32, jb.cosA64,
                                  jb.margin, Vg + (size_t)gwarp * vg_stride, base, base + d4,
                                  base + 2 * d4, out, jb.n64, jb.border, jb.nborder);
    } else {
      const int D1 = prune_row_stride(jb.d);
      float* xs = base + (size_t)(jb.R + 1) * D1;
      kept = warp_prune_node(jb.X, jb.ld, jb.d, i, cand, len, jb.R, jb.cosA32, jb.cosA64,
                             jb.margin, base, D1, xs, xs + D1, out, jb.n64, jb.border,
                             jb.nborder);
    }
    for (int t = kept + lane; t < jb.R; t += 32) out[t] = -1;
    if (lane == 0) jb.deg[i] = kept;
    __syncwarp();
  }
}

// Bucket of a pool length: buckets of `width` lengths, the longest first.
__device__ __forceinline__ int pool_bucket(int len, int width, int nb) {
  const int b = len / width;
  return nb - 1 - (b < nb - 1 ? b : nb - 1);
}

// The job of flattened node g (first[j] = the first flattened node of job j).
__device__ __forceinline__ int job_of(const int64_t* first, int njobs, int64_t g) {
  int lo = 0, hi = njobs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (first[mid] <= g) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__global__ void k_bucket_count(const PruneJob* __restrict__ jobs, const int64_t* __restrict__ first,
                               int njobs, int64_t total, int width, int nb,
                               unsigned long long* __restrict__ counts) {
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < total;
       g += (int64_t)gridDim.x * blockDim.x) {
    const int j = job_of(first, njobs, g);
    const int len = jobs[j].pool_len[g - first[j]];
    atomicAdd(counts + pool_bucket(len, width, nb), 1ull);
  }
}

__global__ void k_bucket_scatter(const PruneJob* __restrict__ jobs, const int64_t* __restrict__ first,
                                 int njobs, int64_t total, int width, int nb,
                                 unsigned long long* __restrict__ cursor, int2* __restrict__ items) {
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < total;
       g += (int64_t)gridDim.x * blockDim.x) {
    const int j = job_of(first, njobs, g);
    const int64_t i = g - first[j];
    const int len = jobs[j].pool_len[i];
    const unsigned long long p = atomicAdd(cursor + pool_bucket(len, width, nb), 1ull);
    items[p] = make_int2(j, (int)i);
  }
}

double prune_run_batched(const std::vector<PruneJob>& jobs, const PruneTune& tune, cudaStream_t st) {
  if (jobs.empty()) return 0.0;
  // one launch per row shape class: rows the warp prune takes with its R + 1 kept vectors
  // in shared memory, rows it takes with them in a device slot per warp (wider than 1,024
  // values), and rows the block prune takes (prune_block_preferred: 96 values and more)
  std::vector<PruneJob> cls[3];
  for (const PruneJob& j : jobs)
    cls[prune_block_preferred(j.d, j.R) ? 2 : (prune_is_wide(j.d, j.R) ? 1 : 0)].push_back(j);
  const int width = std::max(1, tune.bucket_width);
  struct Prepared {
    Scratch<PruneJob> dj;
    Scratch<int2> items;
    Scratch<float> Vg;
    int64_t nitems = 0;
    size_t warp_floats = 0, vg_stride = 0;
    int wpb = 1, grid = 1;
  } prep[3];
  WideBatchPlan plan;
  Scratch<unsigned long long> cnt(64, st), next(3, st);
  for (int w = 0; w < 3; ++w) {
    const std::vector<PruneJob>& js = cls[w];
    if (js.empty()) continue;
    Prepared& P = prep[w];
    const int njobs = (int)js.size();
    std::vector<int64_t> first((size_t)njobs);
    int64_t total = 0;
    int Lmax = 1, Rmax = 1, d4max = 4;
    for (int j = 0; j < njobs; ++j) {
      first[j] = total;
      total += js[j].n;
      Lmax = std::max(Lmax, js[j].L);
      Rmax = std::max(Rmax, js[j].R);
      d4max = std::max(d4max, (js[j].d + 3) & ~3);
      P.warp_floats = std::max(P.warp_floats, w == 1 ? prune_wide_smem_floats(js[j].d, js[j].R)
                                                     : prune_smem_floats(js[j].d, js[j].R));
    }
    SSG_REQUIRE(total < (1ll << 31), SSG_EINVAL, "batched prune: more than 2^31 nodes");
    const int nb = std::min(64, (Lmax + width) / width);
    P.nitems = total;
    P.dj.alloc((size_t)njobs, st);
    SSG_CUDA(cudaMemcpyAsync(P.dj.p, js.data(), sizeof(PruneJob) * njobs, cudaMemcpyHostToDevice, st));
    Scratch<int64_t> dfirst((size_t)njobs, st);
    SSG_CUDA(cudaMemcpyAsync(dfirst.p, first.data(), sizeof(int64_t) * njobs, cudaMemcpyHostToDevice,
                             st));
    SSG_CUDA(cudaMemsetAsync(cnt.p, 0, sizeof(unsigned long long) * 64, st));
    const int g = 8 * num_sms();
    SSG_LAUNCH(k_bucket_count, g, 256, 0, st, P.dj.p, dfirst.p, njobs, total, width, nb, cnt.p);
    unsigned long long hc[64];
    SSG_CUDA(cudaMemcpyAsync(hc, cnt.p, sizeof(hc), cudaMemcpyDeviceToHost, st));
    SSG_CUDA(cudaStreamSynchronize(st));
    unsigned long long off[64], acc = 0;
    for (int b = 0; b < nb; ++b) {
      off[b] = acc;
      acc += hc[b];
    }
    SSG_CUDA(cudaMemcpyAsync(cnt.p, off, sizeof(unsigned long long) * nb, cudaMemcpyHostToDevice, st));
    P.items.alloc((size_t)total, st);
    SSG_LAUNCH(k_bucket_scatter, g, 256, 0, st, P.dj.p, dfirst.p, njobs, total, width, nb, cnt.p,
               P.items.p);
    if (w == 2) {
      prune_wide_batched_prepare(js, plan, st);
      continue;
    }
    const size_t per_warp = P.warp_floats * sizeof(float);
    P.wpb = tune.warps > 0 ? tune.warps
                           : (int)std::max<size_t>(1, std::min<size_t>(8, (96 * 1024) / per_warp));
    const size_t smem = per_warp * P.wpb;
    SSG_REQUIRE(smem <= 225 * 1024, SSG_EINVAL, "batched prune: %d warps per block need %zu bytes",
                P.wpb, smem);
    ensure_smem((const void*)k_prune_batched, smem);
    int per_sm = 0;
    SSG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_prune_batched, P.wpb * 32, smem));
    P.grid = std::max(1, per_sm) * num_sms();
    if (w) {
      P.vg_stride = (size_t)(Rmax + 1) * d4max;
      P.Vg.alloc((size_t)P.grid * P.wpb * P.vg_stride, st);
    }
    SSG_CUDA(cudaStreamSynchronize(st));  // the scatter done and every buffer in place
  }
  // the launches themselves, recorded once into a CUDA graph and replayed (no allocation
  // or host synchronisation inside)
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  SSG_CUDA(cudaEventCreate(&e0));
  SSG_CUDA(cudaEventCreate(&e1));
  struct Cleanup {
    cudaGraph_t& g;
    cudaGraphExec_t& x;
    cudaEvent_t& a;
    cudaEvent_t& b;
    ~Cleanup() {
      if (x) cudaGraphExecDestroy(x);
      if (g) cudaGraphDestroy(g);
      if (a) cudaEventDestroy(a);
      if (b) cudaEventDestroy(b);
    }
  } cleanup{graph, exec, e0, e1};
  SSG_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
  cudaError_t cap = cudaSuccess;
  try {
    SSG_CUDA(cudaMemsetAsync(next.p, 0, 3 * sizeof(unsigned long long), st));
    for (int w = 0; w < 3; ++w) {
      Prepared& P = prep[w];
      if (P.nitems == 0) continue;
      if (w == 2) {
        prune_wide_batched_launch(plan, P.items.p, P.nitems, next.p + 2, st);
        continue;
      }
      SSG_LAUNCH(k_prune_batched, P.grid, P.wpb * 32, P.warp_floats * sizeof(float) * P.wpb, st,
                 P.dj.p, P.items.p, P.nitems, next.p + w, P.Vg.p, P.vg_stride, P.warp_floats, w);
    }
  } catch (...) {
    cap = cudaErrorUnknown;
  }
  const cudaError_t ec = cudaStreamEndCapture(st, &graph);
  SSG_REQUIRE(cap == cudaSuccess, SSG_ECUDA, "batched prune: a launch failed during capture");
  SSG_CUDA(ec);
  SSG_CUDA(cudaGraphInstantiate(&exec, graph, 0));
  SSG_CUDA(cudaEventRecord(e0, st));
  SSG_CUDA(cudaGraphLaunch(exec, st));
  SSG_CUDA(cudaEventRecord(e1, st));
  SSG_CUDA(cudaEventSynchronize(e1));
  float ms = 0.f;
  SSG_CUDA(cudaEventElapsedTime(&ms, e0, e1));
  return (double)ms;
}

}  // namespace ssg
