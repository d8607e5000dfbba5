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
  warp_sort_keys(keys, mp);
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

__global__ void k_pool(const float* __restrict__ X, const uint8_t* __restrict__ X8, int ld, int d,
                       int64_t n,
                       const int32_t* __restrict__ knn, int K, int L, int cap, int log2h,
                       int own_first, int exact, float rel, int32_t* __restrict__ pool_id,
                       float* __restrict__ pool_d2, int32_t* __restrict__ pool_len,
                       unsigned long long* __restrict__ n_order) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  const int wpb = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = lane_id();
  const int hcap = 1 << log2h;
  const size_t per_warp = (size_t)cap * 8 + (size_t)hcap * 4;
  uint64_t* keys = (uint64_t*)(sm_raw + warp * per_warp);
  int32_t* hset = (int32_t*)(keys + cap);
  const int64_t i = (int64_t)blockIdx.x * wpb + warp;
  if (i >= n) return;

  for (int t = lane; t < hcap; t += 32) hset[t] = -1;
  __syncwarp();
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
  pool_finish(keys, m, L, exact, (double*)hset, X, X8, ld, d, i, rel, pool_id, pool_d2, pool_len,
              n_order);
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
  int log2h = 0;
  while ((1 << log2h) < 2 * cap) ++log2h;
  const size_t per_warp = (size_t)cap * 8 + ((size_t)1 << log2h) * 4;
  int wpb = (int)std::max<size_t>(1, std::min<size_t>(8, (96 * 1024) / per_warp));
  const size_t smem = per_warp * wpb;
  ensure_smem((const void*)k_pool, smem);
  SSG_LAUNCH(k_pool, (unsigned)ceil_div(n, wpb), wpb * 32, smem, st, X, X8, ld, d, n, knn, K, L, cap,
             log2h, own_first, exact, dist_rel_team8(ld), pool_id, pool_d2, pool_len, &dctr->order_fp64);
}

void pool_from_candidates(const float* X, const uint8_t* X8, int ld, int d, int64_t n,
                          const int32_t* cand, int KS, int L, int exact, int32_t* pool_id,
                          float* pool_d2, int32_t* pool_len, Counters* dctr, cudaStream_t st) {
  const int cap = next_pow2(KS);
  const int wpb = 8;
  const size_t smem = (size_t)cap * 16 * wpb;
  ensure_smem((const void*)k_pool_cand, smem);
  SSG_LAUNCH(k_pool_cand, (unsigned)ceil_div(n, wpb), wpb * 32, smem, st, X, X8, ld, d, n, cand, KS,
             L, cap, exact, dist_rel_team8(ld), pool_id, pool_d2, pool_len, &dctr->order_fp64);
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
               int32_t* deg, Counters* dctr, cudaStream_t st) {
  const bool wide = prune_is_wide(d, R);
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
