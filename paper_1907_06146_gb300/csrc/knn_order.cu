// Near-first column order for the exact kNN graph.
//
// A streaming top-K keeps a row's threshold at the K-th smallest distance seen so far; the
// sooner its true nearest neighbours are seen, the fewer candidates pass the threshold and
// the fewer buffer compactions follow.  The rows are clustered (a few Lloyd steps of
// k-means on a sample, centroids started at evenly spaced rows, then one assignment of
// every row), stored cluster by cluster, and every block of query rows visits the column
// tiles of the stored order nearest cluster first: a tile is visited with the first
// cluster in the block's order that it overlaps.  The order only changes how fast the
// threshold drops: every tile is still visited exactly once, candidate keys carry original
// ids, and the threshold admits ties, so the selected neighbours are the exact (distance,
// id) top-K in any order.
#include <vector>

#include "common.cuh"
#include "knn.cuh"

namespace ssg {

__global__ void k_init_centroids(const float* __restrict__ X, int ld, int d, int64_t n, int ncl,
                                 int dc, float* __restrict__ C) {
  const int c = blockIdx.x;
  const int64_t src = (int64_t)c * n / ncl;
  for (int t = threadIdx.x; t < dc; t += blockDim.x) C[(int64_t)c * dc + t] = t < d ? X[src * ld + t] : 0.f;
}

// Squared norms of the centroids.
__global__ void k_centroid_norms(const float* __restrict__ C, int ncl, int dc, float* __restrict__ cn) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncl) return;
  float s = 0.f;
  for (int t = 0; t < dc; ++t) s = fmaf(C[(int64_t)c * dc + t], C[(int64_t)c * dc + t], s);
  cn[c] = s;
}

// Nearest centroid of each of m visited rows (row r of them is row r * n / m of X; m = n:
// every row), tiled: a block takes 128 rows and walks the centroids 64 at a time through
// shared memory, 32 coordinates per step; thread (row group, centroid group) scores 4 rows
// x 8 centroids by |c|^2 - 2 x.c (the row's own |x|^2 does not change the argmin), and the
// 8 threads of a row group agree on each row's smallest (ties to the lower centroid).
// counts (nullable) gets the cluster sizes.
constexpr int AS_ROWS = 128, AS_CENT = 64, AS_DIMS = 32;
__global__ void __launch_bounds__(256) k_assign_tiled(const float* __restrict__ X, int ld, int d,
                                                      int64_t n, int64_t m,
                                                      const float* __restrict__ C,
                                                      const float* __restrict__ cn, int ncl, int dc,
                                                      int32_t* __restrict__ label,
                                                      int* __restrict__ counts) {
  __shared__ float xs[AS_DIMS][AS_ROWS + 4];
  __shared__ __align__(16) float cs[AS_DIMS][AS_CENT];
  const int t = threadIdx.x;
  const int rg = t >> 3, g = t & 7;  // rows rg * 4 .. + 3, centroids g * 8 .. + 7 of a chunk
  const int64_t row0 = (int64_t)blockIdx.x * AS_ROWS;
  float best[4];
  int bc[4];
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    best[r] = __int_as_float(0x7f800000);
    bc[r] = 0;
  }
  for (int c0 = 0; c0 < ncl; c0 += AS_CENT) {
    float acc[4][8];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int j = 0; j < 8; ++j) acc[r][j] = 0.f;
    for (int d0 = 0; d0 < d; d0 += AS_DIMS) {
      __syncthreads();
      for (int i = t; i < AS_ROWS * AS_DIMS; i += 256) {
        const int rr = i / AS_DIMS, kk = i % AS_DIMS;
        const int64_t row = row0 + rr;
        const int64_t src = m == n ? row : row * n / m;
        xs[kk][rr] = (row < m && d0 + kk < d) ? X[src * ld + d0 + kk] : 0.f;
      }
      for (int i = t; i < AS_DIMS * AS_CENT; i += 256) {
        const int kk = i / AS_CENT, cc = i % AS_CENT;
        cs[kk][cc] = (c0 + cc < ncl && d0 + kk < d) ? C[(int64_t)(c0 + cc) * dc + d0 + kk] : 0.f;
      }
      __syncthreads();
#pragma unroll 4
      for (int kk = 0; kk < AS_DIMS; ++kk) {
        const float4 xv = *(const float4*)&xs[kk][rg * 4];
        const float4 a = *(const float4*)&cs[kk][g * 8];
        const float4 b = *(const float4*)&cs[kk][g * 8 + 4];
        const float xr[4] = {xv.x, xv.y, xv.z, xv.w};
        const float cv[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
          for (int j = 0; j < 8; ++j) acc[r][j] = fmaf(xr[r], cv[j], acc[r][j]);
      }
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int c = c0 + g * 8 + j;
      if (c < ncl) {
        const float nc = cn[c];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          const float sc = fmaf(-2.f, acc[r][j], nc);
          if (sc < best[r]) {
            best[r] = sc;
            bc[r] = c;
          }
        }
      }
    }
  }
  // the 8 threads of a row group are 8 consecutive lanes
#pragma unroll
  for (int r = 0; r < 4; ++r) {
#pragma unroll
    for (int o = 1; o < 8; o <<= 1) {
      const float ob = __shfl_xor_sync(0xffffffffu, best[r], o);
      const int oc = __shfl_xor_sync(0xffffffffu, bc[r], o);
      if (ob < best[r] || (ob == best[r] && oc < bc[r])) {
        best[r] = ob;
        bc[r] = oc;
      }
    }
  }
  if (g < 4) {
    const int64_t row = row0 + rg * 4 + g;
    int c = bc[0];
#pragma unroll
    for (int r = 1; r < 4; ++r)
      if (r == g) c = bc[r];
    if (row < m) {
      label[row] = c;
      if (counts) atomicAdd(counts + c, 1);
    }
  }
}

// Per-cluster coordinate sums and sizes of the m visited rows (as in k_assign_tiled).
__global__ void k_accum(const float* __restrict__ X, int ld, int d, int64_t n, int64_t m,
                        const int32_t* __restrict__ label, int dc, float* __restrict__ sums,
                        int* __restrict__ counts) {
  const int64_t total = m * (int64_t)d;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / d;
    const int t = (int)(e - r * d);
    const int l = label[r];
    atomicAdd(sums + (int64_t)l * dc + t, X[(m == n ? r : r * n / m) * ld + t]);
    if (t == 0) atomicAdd(counts + l, 1);
  }
}

__global__ void k_update(float* __restrict__ C, const float* __restrict__ sums,
                         const int* __restrict__ counts, int ncl, int dc) {
  const int c = blockIdx.x;
  const int k = counts[c];
  if (k == 0) return;
  for (int t = threadIdx.x; t < dc; t += blockDim.x)
    C[(int64_t)c * dc + t] = sums[(int64_t)c * dc + t] / (float)k;
}

// Cluster sizes; a label outside [0, ncl) (a row whose distances were all NaN) becomes 0.
__global__ void k_count_labels(int32_t* __restrict__ label, int64_t n, int ncl,
                               int* __restrict__ counts) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    int32_t l = label[i];
    if ((uint32_t)l >= (uint32_t)ncl) {
      l = 0;
      label[i] = 0;
    }
    atomicAdd(counts + l, 1);
  }
}

__global__ void k_scatter_perm(const int32_t* __restrict__ label, int64_t n, int* __restrict__ cursor,
                               int32_t* __restrict__ perm, int32_t* __restrict__ inv) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int pos = atomicAdd(cursor + label[i], 1);
    perm[pos] = (int32_t)i;
    inv[i] = pos;
  }
}

// Row c of the table: all clusters by (centroid distance from c, id); c itself first.
__global__ void k_cluster_order(const float* __restrict__ C, int ncl, int dc, int ncl_p2,
                                int32_t* __restrict__ order) {
  extern __shared__ uint64_t keys[];
  const int c = blockIdx.x;
  for (int t = threadIdx.x; t < ncl_p2; t += blockDim.x) {
    uint64_t key = KEY_NONE;
    if (t < ncl) {
      float s = 0.f;
      for (int u = 0; u < dc; ++u) {
        const float v = C[(int64_t)c * dc + u] - C[(int64_t)t * dc + u];
        s = fmaf(v, v, s);
      }
      key = make_key(t == c ? -1.f : s, t);
    }
    keys[t] = key;
  }
  __syncthreads();
  block_sort_keys(keys, ncl_p2);
  for (int t = threadIdx.x; t < ncl; t += blockDim.x) order[(int64_t)c * ncl + t] = key_id(keys[t]);
}

__global__ void k_rb_cluster(const int32_t* __restrict__ label, const int32_t* __restrict__ perm,
                             int64_t n, int BM, int64_t nrb, int32_t* __restrict__ rbc) {
  for (int64_t rb = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; rb < nrb;
       rb += (int64_t)gridDim.x * blockDim.x) {
    int64_t pos = rb * BM + BM / 2;
    if (pos >= n) pos = n - 1;
    rbc[rb] = label[perm[pos]];
  }
}

// Row c of the tile table: the first cap BN-column tiles of the stored order, each listed
// with the first cluster (in cluster c's order) whose stored range it overlaps.  One thread
// per cluster walks the order with a bitmap of the tiles already listed; err is set if a
// row does not list cap distinct tiles (cap = ntiles: every tile exactly once).
__global__ void k_tile_order(const int32_t* __restrict__ order, const int32_t* __restrict__ cl_start,
                             const int32_t* __restrict__ cl_end, int ncl, int BN, int64_t ntiles,
                             int64_t cap, int32_t* __restrict__ tile_order, int* __restrict__ err) {
  extern __shared__ uint32_t seen[];
  const int c = blockIdx.x;
  const int64_t words = (ntiles + 31) >> 5;
  for (int64_t w = threadIdx.x; w < words; w += blockDim.x) seen[w] = 0u;
  __syncthreads();
  if (threadIdx.x != 0) return;
  int32_t* out = tile_order + (int64_t)c * cap;
  int64_t k = 0;
  for (int oi = 0; oi < ncl && k < cap; ++oi) {
    const int cc = order[(int64_t)c * ncl + oi];
    const int64_t s = cl_start[cc], e = cl_end[cc];
    if (e <= s) continue;
    for (int64_t t = s / BN; t <= (e - 1) / BN && k < cap; ++t) {
      const uint32_t bit = 1u << (t & 31);
      if (seen[t >> 5] & bit) continue;
      seen[t >> 5] |= bit;
      out[k] = (int32_t)t;
      ++k;
    }
  }
  if (k != cap) atomicOr(err, 1);
}

bool knn_order_fits(int64_t n, int BN) {
  const int64_t ntiles = (n + BN - 1) / BN;
  return ((ntiles + 31) >> 5) * 4 <= 48 * 1024;
}

void knn_cluster_order(const float* X, int ld, int d, int64_t n, int BM, int BN, cudaStream_t st,
                       KnnOrder& o, int64_t walk, const float* x_norm) {
  SSG_REQUIRE(knn_order_fits(n, BN), SSG_EINTERNAL, "cluster order: too many column tiles");
  // A full walk only needs the near tiles first: about 4,096 rows per cluster, up to 512
  // clusters (1M x 128, K = 200: 341 ms for the kNN graph against 347 with 2,048 rows,
  // 344 with 8,192, and more the smaller the clusters: 504 ms with 256 rows).  A limited
  // walk (Alg. 4) takes its pools from the first tiles alone, so its clusters stay at about
  // 2,048 rows, up to 8,192 of them.
  const int ncl = (int)std::max<int64_t>(
      16, walk > 0 ? std::min<int64_t>(8192, n / 2048) : std::min<int64_t>(512, n / 4096));
  const int dc = (d + 3) & ~3;
  o.ncl = ncl;
  o.ntiles = (n + BN - 1) / BN;
  o.tstride = walk > 0 ? std::min<int64_t>(walk, o.ntiles) : o.ntiles;
  // Lloyd steps on an evenly spaced sample of about 64 rows per cluster, then one
  // assignment of every row.
  const int64_t m = std::min<int64_t>(n, (int64_t)ncl * 64);
  Scratch<float> C((size_t)ncl * dc, st), sums((size_t)ncl * dc, st);
  Scratch<int> counts((size_t)ncl, st);
  Scratch<int32_t> label((size_t)n, st);
  SSG_LAUNCH(k_init_centroids, ncl, 128, 0, st, X, ld, d, n, ncl, dc, C.p);
  const int grid = 8 * num_sms();
  Scratch<float> cn((size_t)ncl, st);
  for (int iter = 0; iter < 4; ++iter) {
    SSG_LAUNCH(k_centroid_norms, (unsigned)ceil_div(ncl, 128), 128, 0, st, C.p, ncl, dc, cn.p);
    SSG_LAUNCH(k_assign_tiled, (unsigned)ceil_div(m, AS_ROWS), 256, 0, st, X, ld, d, n, m, C.p,
               cn.p, ncl, dc, label.p, (int*)nullptr);
    SSG_CUDA(cudaMemsetAsync(sums.p, 0, sizeof(float) * ncl * dc, st));
    SSG_CUDA(cudaMemsetAsync(counts.p, 0, sizeof(int) * ncl, st));
    SSG_LAUNCH(k_accum, grid, 256, 0, st, X, ld, d, n, m, label.p, dc, sums.p, counts.p);
    SSG_LAUNCH(k_update, ncl, 128, 0, st, C.p, sums.p, counts.p, ncl, dc);
  }
  SSG_CUDA(cudaMemsetAsync(counts.p, 0, sizeof(int) * ncl, st));
  SSG_LAUNCH(k_centroid_norms, (unsigned)ceil_div(ncl, 128), 128, 0, st, C.p, ncl, dc, cn.p);
  if (x_norm && knn_tc_available(d) && ncl >= 1024) {
    // many centroids: the full assignment on the tensor cores, each row's nearest centroid
    // by bf16 distance (the order is a heuristic; any assignment keeps the kNN graph
    // exact).  With a few hundred centroids the per-row output of the top-K kernel costs
    // more than the tiled assignment saves.
    Scratch<float> d2((size_t)n, st);
    knn_exact_tc(X, n, ld, x_norm, C.p, ncl, dc, cn.p, d, 0, 1, label.p, d2.p, st, nullptr, 0,
                 true);
    SSG_LAUNCH(k_count_labels, grid, 256, 0, st, label.p, n, ncl, counts.p);
  } else {
    SSG_LAUNCH(k_assign_tiled, (unsigned)ceil_div(n, AS_ROWS), 256, 0, st, X, ld, d, n, n, C.p,
               cn.p, ncl, dc, label.p, counts.p);
  }
  std::vector<int> h((size_t)ncl);
  SSG_CUDA(cudaMemcpyAsync(h.data(), counts.p, sizeof(int) * ncl, cudaMemcpyDeviceToHost, st));
  SSG_CUDA(cudaStreamSynchronize(st));
  std::vector<int32_t> start((size_t)ncl), end((size_t)ncl);
  int64_t acc = 0;
  for (int c = 0; c < ncl; ++c) {
    start[c] = (int32_t)acc;
    acc += h[c];
    end[c] = (int32_t)acc;
  }
  SSG_REQUIRE(acc == n, SSG_EINTERNAL, "cluster order: sizes sum to %lld, not %lld",
              (long long)acc, (long long)n);
  Scratch<int32_t> cl_start((size_t)ncl, st), cl_end((size_t)ncl, st), order((size_t)ncl * ncl, st);
  Scratch<int> cursor((size_t)ncl, st), err(1, st);
  o.perm.alloc((size_t)n, st);
  o.inv.alloc((size_t)n, st);
  o.tile_order.alloc((size_t)ncl * o.tstride, st);
  const int64_t nrb = ceil_div(n, BM);
  o.rb_cluster.alloc((size_t)nrb, st);
  SSG_CUDA(cudaMemcpyAsync(cl_start.p, start.data(), sizeof(int32_t) * ncl, cudaMemcpyHostToDevice, st));
  SSG_CUDA(cudaMemcpyAsync(cl_end.p, end.data(), sizeof(int32_t) * ncl, cudaMemcpyHostToDevice, st));
  SSG_CUDA(cudaMemcpyAsync(cursor.p, start.data(), sizeof(int32_t) * ncl, cudaMemcpyHostToDevice, st));
  SSG_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), st));
  SSG_LAUNCH(k_scatter_perm, grid, 256, 0, st, label.p, n, cursor.p, o.perm.p, o.inv.p);
  const int p2 = next_pow2(ncl);
  ensure_smem((const void*)k_cluster_order, p2 * sizeof(uint64_t));
  SSG_LAUNCH(k_cluster_order, ncl, 256, p2 * sizeof(uint64_t), st, C.p, ncl, dc, p2, order.p);
  SSG_LAUNCH(k_tile_order, ncl, 256, (size_t)((o.ntiles + 31) >> 5) * 4, st, order.p, cl_start.p,
             cl_end.p, ncl, BN, o.ntiles, o.tstride, o.tile_order.p, err.p);
  SSG_LAUNCH(k_rb_cluster, (unsigned)ceil_div(nrb, 256), 256, 0, st, label.p, o.perm.p, n, BM, nrb,
             o.rb_cluster.p);
  int herr = 0;
  // the host vectors above are read by the copies before they go out of scope
  SSG_CUDA(cudaMemcpyAsync(&herr, err.p, sizeof(int), cudaMemcpyDeviceToHost, st));
  SSG_CUDA(cudaStreamSynchronize(st));
  SSG_REQUIRE(herr == 0, SSG_EINTERNAL, "cluster order: a tile list is incomplete");
}

}  // namespace ssg
