// Reverse-neighbour merge (Alg. 3, reverse neighbour checking; Sec. 4.1).
//
// Order-free batch reading: from the pruned graph adj0 as a whole, every node j gets the
// candidates adj0[j] united with its in-neighbours {i : j in adj0[i]}, sorted by
// (d2(j, .), id), and the same SSG prune with the same cap R.  The transpose is a
// histogram (atomic in-degree count), an exclusive scan to 64-bit offsets, and an atomic
// scatter; the scatter order inside a node's in-list does not matter because the list is
// sorted afterwards.  Nodes whose candidate count exceeds the per-warp capacity (hubs)
// are processed by a second launch with one warp and a large shared-memory buffer each.
#include "common.cuh"
#include "graph_dev.cuh"
#include "knn.cuh"

namespace ssg {

__global__ void k_indeg(const int32_t* __restrict__ adj0, const int32_t* __restrict__ deg0, int R,
                        int64_t n, int* __restrict__ indeg) {
  const int64_t total = n * R;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / R;
    const int t = (int)(e - i * R);
    if (t < deg0[i]) atomicAdd(indeg + adj0[e], 1);
  }
}

__global__ void k_scatter(const int32_t* __restrict__ adj0, const int32_t* __restrict__ deg0, int R,
                          int64_t n, const int64_t* __restrict__ off, int* __restrict__ fill,
                          int32_t* __restrict__ rev) {
  const int64_t total = n * R;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / R;
    const int t = (int)(e - i * R);
    if (t < deg0[i]) {
      const int32_t j = adj0[e];
      rev[off[j] + atomicAdd(fill + j, 1)] = (int32_t)i;
    }
  }
}

// ---- exclusive scan of int32 counts into int64 offsets (out has n + 1 entries) ----------
constexpr int SCAN_B = 1024;

__global__ void k_scan_block(const int* __restrict__ in, const int64_t* __restrict__ in64,
                             int64_t n, int64_t* __restrict__ out, int64_t* __restrict__ sums) {
  __shared__ int64_t ws[32];
  const int64_t idx = (int64_t)blockIdx.x * SCAN_B + threadIdx.x;
  int64_t v = idx < n ? (in ? (int64_t)in[idx] : in64[idx]) : 0;
  const int lane = lane_id(), warp = threadIdx.x >> 5;
  int64_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int64_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) ws[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int64_t w = ws[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int64_t y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    ws[lane] = w;
  }
  __syncthreads();
  const int64_t incl = x + (warp > 0 ? ws[warp - 1] : 0);
  if (idx < n) out[idx] = incl - v;
  if (threadIdx.x == SCAN_B - 1) sums[blockIdx.x] = incl;
}

__global__ void k_scan_add(int64_t* __restrict__ out, int64_t n, const int64_t* __restrict__ boff) {
  const int64_t idx = (int64_t)blockIdx.x * SCAN_B + threadIdx.x;
  if (idx < n) out[idx] += boff[blockIdx.x];
}

// Exclusive scan; returns the total on the host (synchronises the stream).
static int64_t exclusive_scan(const int* in32, const int64_t* in64, int64_t n, int64_t* out,
                              cudaStream_t st) {
  const int64_t nb = ceil_div(n, SCAN_B);
  Scratch<int64_t> sums((size_t)nb, st);
  SSG_LAUNCH(k_scan_block, (unsigned)nb, SCAN_B, 0, st, in32, in64, n, out, sums.p);
  int64_t total = 0;
  if (nb > 1) {
    Scratch<int64_t> boff((size_t)nb + 1, st);
    total = exclusive_scan(nullptr, sums.p, nb, boff.p, st);
    SSG_LAUNCH(k_scan_add, (unsigned)nb, SCAN_B, 0, st, out, n, boff.p);
  } else {
    SSG_CUDA(cudaMemcpyAsync(&total, sums.p, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    SSG_CUDA(cudaStreamSynchronize(st));
  }
  SSG_CUDA(cudaMemcpyAsync(out + n, &total, sizeof(int64_t), cudaMemcpyHostToDevice, st));
  SSG_CUDA(cudaStreamSynchronize(st));
  return total;
}

// ---- merge + prune ----------------------------------------------------------------------
// One warp per node, persistent over count nodes.  Vg == nullptr: the prune keeps its
// vectors in shared memory; otherwise each warp owns the global slot
// Vg + warp_index * (R + 1) * d4 for wide rows.
__host__ __device__ inline size_t merge_prune_bytes(int d, int R, bool wide) {
  const size_t f = wide ? prune_wide_smem_floats(d, R) : prune_smem_floats(d, R);
  return (f * sizeof(float) + 15) & ~(size_t)15;
}

__global__ void k_reverse_merge(const float* __restrict__ X, const uint8_t* __restrict__ X8,
                                int ld, int d, int64_t n,
                                const int32_t* __restrict__ adj0, const int32_t* __restrict__ deg0,
                                int R, const int64_t* __restrict__ off,
                                const int32_t* __restrict__ rev,
                                const int32_t* __restrict__ node_list, int64_t count, int cap,
                                int limit,
                                int exact, float rel, float cosA32, double cosA64, float margin,
                                int32_t* __restrict__ adj1, int32_t* __restrict__ deg1,
                                int32_t* __restrict__ big_list, int* __restrict__ big_count,
                                unsigned long long* __restrict__ n_order,
                                unsigned long long* __restrict__ n_angle, float* __restrict__ Vg,
                                int32_t* __restrict__ lists, int32_t* __restrict__ list_len,
                                int lstride, double border,
                                unsigned long long* __restrict__ n_border) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  const int wpb = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = lane_id();
  // merge only (lists != nullptr): no prune state
  const size_t per_warp =
      (size_t)cap * 20 + (lists ? 0 : merge_prune_bytes(d, R, Vg != nullptr));
  unsigned char* base = sm_raw + warp * per_warp;
  uint64_t* keys = (uint64_t*)base;
  double* d64 = (double*)(keys + cap);
  int32_t* cand = (int32_t*)(d64 + cap);
  float* P = (float*)(base + (size_t)cap * 20);
  const int D1 = prune_row_stride(d);
  const int d4 = (d + 3) & ~3;
  const int64_t gwarp = (int64_t)blockIdx.x * wpb + warp;
  const int64_t nwarps = (int64_t)gridDim.x * wpb;

  for (int64_t w = gwarp; w < count; w += nwarps) {
    const int64_t j = node_list ? node_list[w] : w;
    const int d0 = deg0[j];
    const int64_t r0 = off[j], r1 = off[j + 1];
    if (d0 + (r1 - r0) > limit) {
      if (lane == 0) {
        big_list[atomicAdd(big_count, 1)] = (int32_t)j;
        if (list_len) list_len[j] = 0;
      }
      continue;
    }
    for (int t = lane; t < d0; t += 32) keys[t] = (uint64_t)(uint32_t)adj0[j * R + t];
    __syncwarp();
    int m = d0;
    for (int64_t c = r0; c < r1; c += 32) {
      const int64_t p = c + lane;
      int32_t id = p < r1 ? rev[p] : -1;
      bool fresh = id >= 0;
      for (int t = 0; t < d0 && fresh; ++t)
        if (key_id(keys[t]) == id) fresh = false;
      const unsigned bal = __ballot_sync(0xffffffffu, fresh);
      if (fresh) keys[m + __popc(bal & lanemask_lt())] = (uint64_t)(uint32_t)id;
      m += __popc(bal);
    }
    __syncwarp();
    const float* xj = X + j * ld;
    if (X8)
      warp_fill_dist_keys_u8(keys, m, X8, ld, X8 + j * ld);
    else
      warp_fill_dist_keys(keys, m, X, ld, xj);
    int mp = 1;
    while (mp < m) mp <<= 1;
    for (int t = m + lane; t < mp; t += 32) keys[t] = KEY_NONE;
    __syncwarp();
    warp_sort_keys(keys, mp);
    if (!exact && m > 1) {
      int f = warp_fix_runs(keys, m, m, d64, X, ld, d, xj, rel);
      for (int o = 16; o > 0; o >>= 1) f += __shfl_xor_sync(0xffffffffu, f, o);
      if (lane == 0 && f) atomicAdd(n_order, (unsigned long long)f);
    }
    if (lists) {
      // merge only: the sorted list goes to the tensor-core or the block prune
      for (int t = lane; t < m; t += 32) lists[j * lstride + t] = key_id(keys[t]);
      if (lane == 0) list_len[j] = m;
      __syncwarp();
      continue;
    }
    for (int t = lane; t < m; t += 32) cand[t] = key_id(keys[t]);
    __syncwarp();
    int32_t* out = adj1 + j * R;
    int kept;
    if (Vg) {
      kept = warp_prune_node_wide(X, ld, d, j, cand, m, R, cosA32, cosA64, margin,
                                  Vg + (size_t)gwarp * (R + 1) * d4, P, P + d4, P + 2 * d4, out,
                                  n_angle, border, n_border);
    } else {
      float* xs = P + (size_t)(R + 1) * D1;
      kept = warp_prune_node(X, ld, d, j, cand, m, R, cosA32, cosA64, margin, P, D1, xs, xs + D1,
                             out, n_angle, border, n_border);
    }
    for (int t = kept + lane; t < R; t += 32) out[t] = -1;
    if (lane == 0) deg1[j] = kept;
    __syncwarp();
  }
}

__global__ void k_max_int(const int* __restrict__ v, int64_t n, int* __restrict__ out) {
  int m = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    m = max(m, v[i]);
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (lane_id() == 0) atomicMax(out, m);
}

int reverse_run(const float* X, const uint8_t* X8, int ld, int d, int64_t n,
                const int32_t* adj0, const int32_t* deg0, int R, double cos_a, double border,
                int exact, bool tc, int32_t* adj1, int32_t* deg1, Counters* dctr,
                cudaStream_t st, int wide_blocks) {
  const int grid = 8 * num_sms();
  Scratch<int> indeg((size_t)n, st), fill((size_t)n, st), small(2, st);
  SSG_CUDA(cudaMemsetAsync(indeg.p, 0, sizeof(int) * n, st));
  SSG_CUDA(cudaMemsetAsync(fill.p, 0, sizeof(int) * n, st));
  SSG_CUDA(cudaMemsetAsync(small.p, 0, sizeof(int) * 2, st));
  SSG_LAUNCH(k_indeg, grid, 256, 0, st, adj0, deg0, R, n, indeg.p);
  SSG_LAUNCH(k_max_int, grid, 256, 0, st, indeg.p, n, small.p + 1);
  Scratch<int64_t> off((size_t)n + 1, st);
  const int64_t total = exclusive_scan(indeg.p, nullptr, n, off.p, st);
  Scratch<int32_t> rev((size_t)std::max<int64_t>(total, 1), st);
  SSG_LAUNCH(k_scatter, grid, 256, 0, st, adj0, deg0, R, n, off.p, fill.p, rev.p);

  const bool wide = prune_is_wide(d, R);
  const size_t prune_bytes = merge_prune_bytes(d, R, wide);
  const float rel = dist_rel_team8c(ld), margin = angle_margin_fp32(d) + (float)border;
  const int d4 = (d + 3) & ~3;
  // Tensor-core path (data exact in bf16): the warps only merge and sort, lists of up to
  // 127 candidates go to the Gram prune, longer ones to the warp prune below.
  const bool use_tc = tc && exact && prune_tc_available(d, 127, R);
  if (!use_tc && prune_wide_available(d) && (wide || d4 >= 192)) {
    // long rows: the warps merge and sort every list, the block prune prunes them (the
    // merged lists are short, so below 192 values the warp prune inside the merge stays
    // faster: 200,000 16-centre float points, R = 32: d = 128 8.6 ms against 13.4, d = 256
    // 23.2 against 15.6)
    int h[2];
    SSG_CUDA(cudaMemcpyAsync(h, small.p, sizeof(h), cudaMemcpyDeviceToHost, st));
    SSG_CUDA(cudaStreamSynchronize(st));
    const int Lr = R + std::max(h[1], 1);
    Scratch<int32_t> lists((size_t)n * Lr, st), list_len((size_t)n, st), big((size_t)n, st);
    const size_t smem_max = 220 * 1024;
    ensure_smem((const void*)k_reverse_merge, smem_max);
    int cap1 = 32;
    while (cap1 < Lr && cap1 < 1024) cap1 *= 2;
    const int wpb1 = (int)std::max<size_t>(1, std::min<size_t>(8, (96 * 1024) / ((size_t)cap1 * 20)));
    SSG_LAUNCH(k_reverse_merge, (unsigned)ceil_div(n, wpb1), wpb1 * 32, (size_t)cap1 * 20 * wpb1, st, X,
               X8, ld, d, n, adj0, deg0, R, off.p, rev.p, (const int32_t*)nullptr, n, cap1, cap1, exact,
               rel, (float)cos_a, cos_a, margin, adj1, deg1, big.p, small.p, &dctr->order_fp64,
               &dctr->angle_fp64, (float*)nullptr, lists.p, list_len.p, Lr, border,
               &dctr->angle_border);
    SSG_CUDA(cudaMemcpyAsync(h, small.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    SSG_CUDA(cudaStreamSynchronize(st));
    if (h[0] > 0) {
      int cap_big = cap1;
      while (cap_big < Lr) cap_big *= 2;
      SSG_REQUIRE((size_t)cap_big * 20 <= smem_max, SSG_EINTERNAL,
                  "reverse merge: a node has %d candidates, more than the %zu supported", Lr,
                  smem_max / 20);
      Scratch<int> small2(2, st);
      SSG_CUDA(cudaMemsetAsync(small2.p, 0, sizeof(int) * 2, st));
      SSG_LAUNCH(k_reverse_merge, (unsigned)std::min<int64_t>(h[0], 8 * num_sms()), 32,
                 (size_t)cap_big * 20, st, X, X8, ld, d, n, adj0, deg0, R, off.p, rev.p, big.p,
                 (int64_t)h[0], cap_big, cap_big, exact, rel, (float)cos_a, cos_a, margin, adj1, deg1,
                 big.p, small2.p, &dctr->order_fp64, &dctr->angle_fp64, (float*)nullptr, lists.p,
                 list_len.p, Lr, border, &dctr->angle_border);
    }
    prune_run_wide(X, ld, d, n, lists.p, list_len.p, Lr, R, cos_a, border, adj1, deg1, dctr, st,
                   wide_blocks);
    return h[1];
  }
  // warp path: per-warp buffers of cap keys (a power of two, for the sort); lists longer
  // than limit go to the second pass
  const int cap = use_tc ? 128 : 256;
  const int limit = use_tc ? 127 : cap;
  // merge-only warps (the tensor-core path) keep no prune state
  const size_t per_warp = (size_t)cap * 20 + (use_tc ? 0 : prune_bytes);
  SSG_REQUIRE((cap & (cap - 1)) == 0 && (cap * 20) % 16 == 0 && limit <= cap, SSG_EINTERNAL,
              "reverse merge: bad buffer layout (cap %d, limit %d)", cap, limit);
  const int wpb = (int)std::max<size_t>(1, std::min<size_t>(8, (96 * 1024) / per_warp));
  const size_t smem = per_warp * wpb;
  const size_t smem_big_max = 220 * 1024;
  ensure_smem((const void*)k_reverse_merge, smem_big_max);
  int blocks_per_sm = 0;
  SSG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, k_reverse_merge, wpb * 32,
                                                         smem));
  // wide rows: a persistent grid (one device slot per warp); otherwise one warp per node
  const int64_t mgrid =
      wide ? std::min<int64_t>(ceil_div(n, wpb), (int64_t)std::max(1, blocks_per_sm) * num_sms())
           : ceil_div(n, wpb);
  Scratch<float> Vg;
  if (wide) Vg.alloc((size_t)mgrid * wpb * (R + 1) * d4, st);
  Scratch<int32_t> big((size_t)n, st);
  Scratch<int32_t> lists, list_len;
  if (use_tc) {
    lists.alloc((size_t)n * limit, st);
    list_len.alloc((size_t)n, st);
  }
  SSG_LAUNCH(k_reverse_merge, (unsigned)mgrid, wpb * 32, smem, st, X, X8, ld, d, n, adj0, deg0, R, off.p,
             rev.p, (const int32_t*)nullptr, n, cap, limit, exact, rel, (float)cos_a, cos_a, margin, adj1,
             deg1, big.p, small.p, &dctr->order_fp64, &dctr->angle_fp64, Vg.p, lists.p, list_len.p,
             limit, border, &dctr->angle_border);
  if (use_tc)
    prune_run_tc(X, ld, d, n, lists.p, list_len.p, limit, R, cos_a, border, adj1, deg1, dctr, st,
                 true);
  int h[2];
  SSG_CUDA(cudaMemcpyAsync(h, small.p, sizeof(h), cudaMemcpyDeviceToHost, st));
  SSG_CUDA(cudaStreamSynchronize(st));
  if (h[0] > 0) {
    int cap_big = 1;
    while ((size_t)(cap_big * 2) * 20 + prune_bytes <= smem_big_max) cap_big *= 2;
    SSG_REQUIRE(h[1] + R <= cap_big, SSG_EINTERNAL,
                "reverse merge: a node has %d candidates, more than the %d supported", h[1] + R,
                cap_big);
    const size_t smem_big = (size_t)cap_big * 20 + prune_bytes;
    // every listed node fits cap_big, so the second launch appends to no list; one warp per
    // block, so the wide slots of the first launch (>= this many warps) are reused
    const int grid_big = (int)std::min<int64_t>(h[0], mgrid * wpb);
    Scratch<int32_t> none(1, st);
    Scratch<int> small2(2, st);
    SSG_CUDA(cudaMemsetAsync(small2.p, 0, sizeof(int) * 2, st));
    SSG_LAUNCH(k_reverse_merge, grid_big, 32, smem_big, st, X, X8, ld, d, n, adj0, deg0, R, off.p, rev.p,
               big.p, (int64_t)h[0], cap_big, cap_big, exact, rel, (float)cos_a, cos_a, margin, adj1, deg1,
               none.p, small2.p, &dctr->order_fp64, &dctr->angle_fp64, Vg.p, (int32_t*)nullptr,
               (int32_t*)nullptr, 0, border, &dctr->angle_border);
  }
  return h[1];
}

}  // namespace ssg
