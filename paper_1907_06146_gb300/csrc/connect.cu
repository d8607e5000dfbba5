// Connectivity from the navigating nodes (Alg. 3: random navigating nodes NV, then
// "DFS-spanning" from each to strengthen connectivity; Sec. 4.1 defers the details to the
// NSG paper).
//
// Reading: for each root in the given order, mark everything reachable from it; while a
// node is unreached, take the smallest unreached id u, link u from the reached node v with
// a free slot (deg(v) < R) that minimises (d2(v, u), id), and mark everything reachable
// from u.  The reached set does not depend on the traversal order, so the GPU uses a
// level-synchronous frontier traversal (a visited bitmap with atomicOr) in place of a
// depth-first one and gets the same graph.  The argmin is taken in fp64 with the
// coordinate-order sum, so its ties resolve exactly as a sequential double loop would.
#include <climits>

#include "common.cuh"
#include "knn.cuh"

namespace ssg {

__global__ void k_mark(uint32_t* __restrict__ bm, int32_t* __restrict__ frontier,
                       int* __restrict__ fcount, int32_t root) {
  atomicOr(bm + (root >> 5), 1u << (root & 31));
  frontier[0] = root;
  *fcount = 1;
}

__global__ void k_bfs_level(const int32_t* __restrict__ adj, const int32_t* __restrict__ deg, int R,
                            uint32_t* __restrict__ bm, const int32_t* __restrict__ frontier,
                            const int* __restrict__ fcount, int32_t* __restrict__ next,
                            int* __restrict__ ncount) {
  const int lane = lane_id();
  const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
  const int fc = *fcount;
  for (int64_t w = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); w < fc;
       w += nwarps) {
    const int32_t node = frontier[w];
    const int dg = deg[node];
    for (int c = 0; c < dg; c += 32) {
      const int t = c + lane;
      bool fresh = false;
      int32_t v = 0;
      if (t < dg) {
        v = adj[(int64_t)node * R + t];
        const uint32_t bit = 1u << (v & 31);
        fresh = !(atomicOr(bm + (v >> 5), bit) & bit);
      }
      const unsigned bal = __ballot_sync(0xffffffffu, fresh);
      int basep = 0;
      if (lane == 0 && bal) basep = atomicAdd(ncount, __popc(bal));
      basep = __shfl_sync(0xffffffffu, basep, 0);
      if (fresh) next[basep + __popc(bal & lanemask_lt())] = v;
    }
  }
}

__global__ void k_first_unreached(const uint32_t* __restrict__ bm, int64_t nw, int64_t n,
                                  int64_t start_word, unsigned long long* __restrict__ out) {
  for (int64_t w = start_word + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < nw;
       w += (int64_t)gridDim.x * blockDim.x) {
    uint32_t word = bm[w];
    if (w == nw - 1 && (n & 31)) word |= ~((1u << (n & 31)) - 1u);
    if (word != 0xffffffffu) {
      const unsigned long long u = (unsigned long long)(w * 32 + __ffs(~word) - 1);
      atomicMin(out, u);
    }
  }
}

__global__ void k_repair_dist(const float* __restrict__ X, int ld, int d, int64_t n,
                              const uint32_t* __restrict__ bm, const int32_t* __restrict__ deg,
                              int R, int64_t u, double* __restrict__ dv,
                              unsigned long long* __restrict__ best_bits) {
  const float* xu = X + u * ld;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    const bool cand = ((bm[v >> 5] >> (v & 31)) & 1u) && deg[v] < R;
    double e = -1.0;
    if (cand) {
      e = dist2_f64(X + v * ld, xu, d);
      atomicMin(best_bits, (unsigned long long)__double_as_longlong(e));
    }
    dv[v] = e;
  }
}

__global__ void k_repair_pick(const double* __restrict__ dv, int64_t n,
                              const unsigned long long* __restrict__ best_bits,
                              int* __restrict__ best_id) {
  const unsigned long long b = *best_bits;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    const double e = dv[v];
    if (e >= 0.0 && (unsigned long long)__double_as_longlong(e) == b) atomicMin(best_id, (int)v);
  }
}

__global__ void k_add_edge(int32_t* __restrict__ adj, int32_t* __restrict__ deg, int R,
                           const int* __restrict__ best_id, int32_t u, uint32_t* __restrict__ bm,
                           int32_t* __restrict__ frontier, int* __restrict__ fcount) {
  const int v = *best_id;
  if (v == INT_MAX) return;
  adj[(int64_t)v * R + deg[v]] = u;
  deg[v] += 1;
  atomicOr(bm + (u >> 5), 1u << (u & 31));
  frontier[0] = u;
  *fcount = 1;
}

namespace {
struct Bfs {
  int32_t* f[2];
  int* cnt;  // [2]
};
}  // namespace

// Level-synchronous traversal from the frontier already in f[0] / cnt[0].
static void bfs_run(const int32_t* adj, const int32_t* deg, int R, uint32_t* bm, Bfs& b,
                    cudaStream_t st) {
  const int grid = 4 * num_sms();
  int cur = 0;
  for (;;) {
    SSG_CUDA(cudaMemsetAsync(b.cnt + (cur ^ 1), 0, sizeof(int), st));
    SSG_LAUNCH(k_bfs_level, grid, 256, 0, st, adj, deg, R, bm, b.f[cur], b.cnt + cur,
               b.f[cur ^ 1], b.cnt + (cur ^ 1));
    int h = 0;
    SSG_CUDA(cudaMemcpyAsync(&h, b.cnt + (cur ^ 1), sizeof(int), cudaMemcpyDeviceToHost, st));
    SSG_CUDA(cudaStreamSynchronize(st));
    cur ^= 1;
    if (h == 0) break;
  }
}

int64_t connect_run(const float* X, int ld, int d, int64_t n, int32_t* adj, int32_t* deg,
                    int R, const int32_t* nav_dev, const int32_t* nav_host, int n_nav,
                    cudaStream_t st) {
  (void)nav_dev;
  const int64_t nw = ceil_div(n, 32);
  Scratch<uint32_t> bm((size_t)nw, st);
  Scratch<int32_t> f0((size_t)n, st), f1((size_t)n, st);
  Scratch<int> cnt(4, st);
  Scratch<unsigned long long> ull(2, st);
  Scratch<double> dv((size_t)n, st);
  Bfs b{{f0.p, f1.p}, cnt.p};
  const int grid = 8 * num_sms();
  int64_t repairs = 0;
  for (int s = 0; s < n_nav; ++s) {
    SSG_CUDA(cudaMemsetAsync(bm.p, 0, sizeof(uint32_t) * nw, st));
    SSG_LAUNCH(k_mark, 1, 1, 0, st, bm.p, b.f[0], b.cnt, nav_host[s]);
    bfs_run(adj, deg, R, bm.p, b, st);
    int64_t start = 0;
    for (;;) {
      const unsigned long long init[2] = {(unsigned long long)n, ~0ull};
      SSG_CUDA(cudaMemcpyAsync(ull.p, init, sizeof(init), cudaMemcpyHostToDevice, st));
      SSG_LAUNCH(k_first_unreached, grid, 256, 0, st, bm.p, nw, n, start, ull.p);
      unsigned long long u = 0;
      SSG_CUDA(cudaMemcpyAsync(&u, ull.p, sizeof(u), cudaMemcpyDeviceToHost, st));
      SSG_CUDA(cudaStreamSynchronize(st));
      if ((int64_t)u >= n) break;
      start = (int64_t)u >> 5;
      const int imax = INT_MAX;
      SSG_CUDA(cudaMemcpyAsync(cnt.p + 2, &imax, sizeof(int), cudaMemcpyHostToDevice, st));
      SSG_LAUNCH(k_repair_dist, grid, 256, 0, st, X, ld, d, n, bm.p, deg, R, (int64_t)u, dv.p,
                 ull.p + 1);
      SSG_LAUNCH(k_repair_pick, grid, 256, 0, st, dv.p, n, ull.p + 1, cnt.p + 2);
      int best = 0;
      SSG_CUDA(cudaMemcpyAsync(&best, cnt.p + 2, sizeof(int), cudaMemcpyDeviceToHost, st));
      SSG_CUDA(cudaStreamSynchronize(st));
      SSG_REQUIRE(best != INT_MAX, SSG_EINTERNAL,
                  "connectivity: node %lld is unreached and no reached node has a free slot",
                  (long long)u);
      SSG_LAUNCH(k_add_edge, 1, 1, 0, st, adj, deg, R, cnt.p + 2, (int32_t)u, bm.p, b.f[0], b.cnt);
      bfs_run(adj, deg, R, bm.p, b, st);
      ++repairs;
    }
  }
  return repairs;
}

}  // namespace ssg
