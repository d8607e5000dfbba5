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
#include <mutex>
#include <new>
#include <vector>

#include "common.cuh"
#include "graph_dev.cuh"
#include "knn.cuh"

namespace ssg {

__global__ void k_mark(uint32_t* __restrict__ bm, int32_t* __restrict__ frontier,
                       int* __restrict__ fcount, int32_t root) {
  atomicOr(bm + (root >> 5), 1u << (root & 31));
  frontier[0] = root;
  *fcount = 1;
}

// Level l of the grid-wide traversal launched in batches (no host round trip per level):
// the frontier size is lvl[l % 3], the next one is counted in lvl[(l + 1) % 3], and
// lvl[(l + 2) % 3] (level l - 1's input, level l + 1's output) is cleared for the next
// launch.  A level whose frontier is empty does nothing.
__global__ void k_bfs_level_ring(const int32_t* __restrict__ adj, const int32_t* __restrict__ deg,
                                 int R, uint32_t* __restrict__ bm,
                                 const int32_t* __restrict__ frontier, int32_t* __restrict__ next,
                                 int* __restrict__ lvl, int l) {
  if (blockIdx.x == 0 && threadIdx.x == 0) lvl[(l + 2) % 3] = 0;
  const int lane = lane_id();
  const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
  const int fc = lvl[l % 3];
  int* ncount = lvl + (l + 1) % 3;
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

__global__ void k_ring_init(int* __restrict__ lvl, const int* __restrict__ fcount) {
  lvl[0] = *fcount;
  lvl[1] = 0;
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

// Exhaustive fp64 argmin (used only when the fp32 band below overflows its list).
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

__global__ void k_repair_pick_all(const double* __restrict__ dv, int64_t n,
                                  const unsigned long long* __restrict__ best_bits,
                                  int* __restrict__ best_id) {
  const unsigned long long b = *best_bits;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    const double e = dv[v];
    if (e >= 0.0 && (unsigned long long)__double_as_longlong(e) == b) atomicMin(best_id, (int)v);
  }
}

// Device-side state of one repair step.
struct RepairState {
  unsigned long long u;  // smallest unreached id (n if none)
  unsigned hi_bits;      // smallest fp32 upper bound of d2(v, u) over the candidates
  int band;              // candidates whose fp32 lower bound reaches that upper bound
  int best;              // chosen v (INT_MAX: none; -2: band overflow)
  int fcnt[2];           // frontier sizes
  int bfs_state;         // -1 traversal finished, else index of the frontier still to expand
  int lvl[3];            // frontier sizes of the batched traversal, by level mod 3
};

__global__ void k_repair_init(RepairState* __restrict__ s, int64_t n) {
  s->u = (unsigned long long)n;
  s->hi_bits = 0x7f800000u;
  s->band = 0;
  s->best = INT_MAX;
  s->fcnt[0] = 0;
}

// Pass 1: fp32 distance of every reached node with a free slot to u, by teams of 8 lanes;
// the smallest upper bound d32 (1 + 2 rel) over them.
__global__ void k_repair_fp32(const float* __restrict__ X, int ld, int64_t n,
                              const uint32_t* __restrict__ bm, const int32_t* __restrict__ deg,
                              int R, float rel, float* __restrict__ d32,
                              RepairState* __restrict__ s) {
  const int64_t u = (int64_t)s->u;
  if (u >= n) return;
  const int lane = lane_id(), team = lane >> 3, tl = lane & 7;
  const float* xu = X + u * ld;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
  float best = __int_as_float(0x7f800000);
  for (int64_t v0 = gw * 4; v0 < n; v0 += nwarp * 4) {
    const int64_t v = v0 + team;
    const bool cand = v < n && ((bm[v >> 5] >> (v & 31)) & 1u) && deg[v] < R;
    const float e = team8_dist(X + (cand ? v : 0) * ld, xu, ld >> 2, tl, cand);
    if (tl == 0 && v < n) d32[v] = cand ? e : -1.f;
    if (cand) best = fminf(best, e);
  }
  for (int o = 16; o > 0; o >>= 1) best = fminf(best, __shfl_xor_sync(0xffffffffu, best, o));
  if (lane == 0 && best < __int_as_float(0x7f800000))
    atomicMin(&s->hi_bits, __float_as_uint(best * (1.f + 2.f * rel) + 1e-30f));
}

// Pass 2: every candidate whose fp32 lower bound does not exceed that upper bound goes
// into a short list ...
__global__ void k_repair_band(const float* __restrict__ X, int ld, int d, int64_t n,
                              const float* __restrict__ d32, float rel, int cap,
                              int32_t* __restrict__ ids, double* __restrict__ dv,
                              RepairState* __restrict__ s) {
  const int64_t u = (int64_t)s->u;
  if (u >= n) return;
  const float hi = __uint_as_float(s->hi_bits);
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    const float e = d32[v];
    if (e >= 0.f && e * (1.f - 2.f * rel) <= hi) {
      const int p = atomicAdd(&s->band, 1);
      if (p < cap) ids[p] = (int32_t)v;
    }
  }
}

// ... whose fp64 distances to u are then summed, one list entry per warp
// (warp_dist2_f64; k_repair_pick re-takes near-equal ones in coordinate order).
__global__ void k_repair_band64(const float* __restrict__ X, int ld, int d, int64_t n,
                                int cap, const int32_t* __restrict__ ids, double* __restrict__ dv,
                                const RepairState* __restrict__ s) {
  const int64_t u = (int64_t)s->u;
  if (u >= n) return;
  const int m = min(s->band, cap);
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t p = gw; p < m; p += nwarp) {
    const double x = warp_dist2_f64(X + (int64_t)ids[p] * ld, X + u * ld, d);
    if (lane_id() == 0) dv[p] = x;
  }
}

// (d2, id)-smallest over the block (every thread returns it); bd / bi: 32 entries each.
__device__ __forceinline__ void block_argmin(double& best, int& bid, double* bd, int* bi) {
  for (int o = 16; o > 0; o >>= 1) {
    const double ob = __shfl_xor_sync(0xffffffffu, best, o);
    const int oi = __shfl_xor_sync(0xffffffffu, bid, o);
    if (ob < best || (ob == best && oi < bid)) {
      best = ob;
      bid = oi;
    }
  }
  const int w = threadIdx.x >> 5, lane = lane_id();
  __syncthreads();
  if (lane == 0) {
    bd[w] = best;
    bi[w] = bid;
  }
  __syncthreads();
  for (int t = 0; t < (int)(blockDim.x >> 5); ++t)
    if (bd[t] < best || (bd[t] == best && bi[t] < bid)) {
      best = bd[t];
      bid = bi[t];
    }
}

// Pass 3 (one block): the (d2, id)-smallest entry of the list; link it to u and make u the
// frontier of the next traversal.  Where other entries lie within fp64_order_rel of the
// smallest warp-summed value, those entries are re-taken in coordinate order, so the
// choice is the one the coordinate-order fp64 values give.
__global__ void k_repair_pick(const float* __restrict__ X, int ld, int d,
                              const int32_t* __restrict__ ids, const double* __restrict__ dv,
                              int cap, int32_t* __restrict__ adj, int32_t* __restrict__ deg, int R,
                              uint32_t* __restrict__ bm, int32_t* __restrict__ frontier,
                              int64_t n, RepairState* __restrict__ s) {
  __shared__ double bd[32];
  __shared__ int bi[32];
  __shared__ int nties;
  const int64_t u = (int64_t)s->u;
  if (u >= n) return;
  const int m = s->band;
  if (m > cap) {
    if (threadIdx.x == 0) s->best = -2;
    return;
  }
  const double INF = __longlong_as_double(0x7ff0000000000000ll);
  double best = INF;
  int bid = INT_MAX;
  for (int t = threadIdx.x; t < m; t += blockDim.x) {
    const double x = dv[t];
    const int v = ids[t];
    if (x < best || (x == best && v < bid)) {
      best = x;
      bid = v;
    }
  }
  if (threadIdx.x == 0) nties = 0;
  block_argmin(best, bid, bd, bi);
  const double lim = best + fp64_order_rel(d) * best;
  int mine = 0;
  for (int t = threadIdx.x; t < m; t += blockDim.x) mine += dv[t] <= lim;
  if (mine) atomicAdd(&nties, mine);
  __syncthreads();
  if (nties > 1) {
    double b2 = INF;
    int i2 = INT_MAX;
    for (int t = threadIdx.x; t < m; t += blockDim.x) {
      if (dv[t] > lim) continue;
      const int v = ids[t];
      const double x = dist2_f64(X + (int64_t)v * ld, X + u * ld, d);
      if (x < b2 || (x == b2 && v < i2)) {
        b2 = x;
        i2 = v;
      }
    }
    block_argmin(b2, i2, bd, bi);
    bid = i2;
  }
  if (threadIdx.x == 0) {
    s->best = bid;
    if (bid != INT_MAX) {
      adj[(int64_t)bid * R + deg[bid]] = (int32_t)u;
      deg[bid] += 1;
      atomicOr(bm + (u >> 5), 1u << (u & 31));
      frontier[0] = (int32_t)u;
      s->fcnt[0] = 1;
    }
  }
}

// Link v = *best (exhaustive path) and make u the next frontier.
__global__ void k_add_edge(int32_t* __restrict__ adj, int32_t* __restrict__ deg, int R,
                           const int* __restrict__ best_id, uint32_t* __restrict__ bm,
                           int32_t* __restrict__ frontier, RepairState* __restrict__ s) {
  const int v = *best_id;
  s->best = v;
  if (v == INT_MAX) return;
  const int64_t u = (int64_t)s->u;
  adj[(int64_t)v * R + deg[v]] = (int32_t)u;
  deg[v] += 1;
  atomicOr(bm + (u >> 5), 1u << (u & 31));
  frontier[0] = (int32_t)u;
  s->fcnt[0] = 1;
}

// Traversal by one block while the frontier stays small (no host round trip per level);
// leaves bfs_state = -1 when done, or the index of the frontier buffer still to expand.
__global__ void k_bfs_small(const int32_t* __restrict__ adj, const int32_t* __restrict__ deg, int R,
                            uint32_t* __restrict__ bm, int32_t* __restrict__ f0,
                            int32_t* __restrict__ f1, int limit, RepairState* __restrict__ s) {
  const int lane = lane_id();
  const int nwarps = blockDim.x >> 5;
  int cur = 0;
  for (;;) {
    __syncthreads();
    const int fc = s->fcnt[cur];
    if (fc == 0 || fc > limit) {
      if (threadIdx.x == 0) s->bfs_state = fc == 0 ? -1 : cur;
      return;
    }
    __syncthreads();
    if (threadIdx.x == 0) s->fcnt[cur ^ 1] = 0;
    __syncthreads();
    const int32_t* fr = cur ? f1 : f0;
    int32_t* nx = cur ? f0 : f1;
    for (int w = threadIdx.x >> 5; w < fc; w += nwarps) {
      const int32_t node = fr[w];
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
        if (lane == 0 && bal) basep = atomicAdd(&s->fcnt[cur ^ 1], __popc(bal));
        basep = __shfl_sync(0xffffffffu, basep, 0);
        if (fresh) nx[basep + __popc(bal & lanemask_lt())] = v;
      }
    }
    cur ^= 1;
  }
}

// Repairs that u's own kNN row settles, back to back in one block.  The row lists u's K
// nearest nodes in exact (d2, id) order, so when some of them is reached and has a free
// slot the first such one is the (d2, id)-smallest of all reached nodes with a free slot:
// the same choice as the exhaustive argmin, without a pass over all n nodes.  Each round:
// the smallest unreached u (from bitmap word `start` on), the link from the first
// qualifying row entry, and the traversal from u while its frontier stays within `limit`.
// Stops with s->u = n when every node is reached, with s->best = -3 when u's row has no
// qualifying node (the exhaustive path takes u), or with s->bfs_state set when a frontier
// outgrows the block (the grid-wide traversal finishes it).  *nrep += the repairs made.
__global__ void __launch_bounds__(1024)
    k_repair_knn(const int32_t* __restrict__ knn, int K, int32_t* __restrict__ adj,
                 int32_t* __restrict__ deg, int R, uint32_t* __restrict__ bm, int64_t nw,
                 int64_t n, int64_t start, int32_t* __restrict__ f0, int32_t* __restrict__ f1,
                 int limit, RepairState* __restrict__ s, unsigned long long* __restrict__ nrep) {
  __shared__ unsigned long long su;
  __shared__ int sv, sfc[2];
  const int tid = threadIdx.x, lane = lane_id(), warp = tid >> 5, nwarps = blockDim.x >> 5;
  unsigned long long made = 0;
  for (;;) {
    // the smallest unreached id from word `start` on
    for (;;) {
      if (tid == 0) su = (unsigned long long)n;
      __syncthreads();
      const int64_t w = start + tid;
      if (w < nw) {
        uint32_t word = bm[w];
        if (w == nw - 1 && (n & 31)) word |= ~((1u << (n & 31)) - 1u);
        if (word != 0xffffffffu) atomicMin(&su, (unsigned long long)(w * 32 + __ffs(~word) - 1));
      }
      __syncthreads();
      const bool stop = su < (unsigned long long)n || start + blockDim.x >= nw;
      __syncthreads();
      if (stop) break;
      start += blockDim.x;
    }
    const int64_t u = (int64_t)su;
    if (u >= n) {
      if (tid == 0) {
        s->u = (unsigned long long)n;
        s->best = INT_MAX;
        s->bfs_state = -1;
      }
      break;
    }
    if (warp == 0) {
      int found = -1;
      for (int c = 0; c < K; c += 32) {
        const int t = c + lane;
        int32_t v = -1;
        bool ok = false;
        if (t < K) {
          v = knn[u * K + t];
          ok = v >= 0 && ((bm[v >> 5] >> (v & 31)) & 1u) && deg[v] < R;
        }
        const unsigned bal = __ballot_sync(0xffffffffu, ok);
        if (bal) {
          found = __shfl_sync(0xffffffffu, v, __ffs(bal) - 1);
          break;
        }
      }
      if (lane == 0) sv = found;
    }
    __syncthreads();
    const int v = sv;
    if (v < 0) {
      if (tid == 0) {
        s->u = (unsigned long long)u;
        s->best = -3;
        s->bfs_state = -1;
      }
      break;
    }
    if (tid == 0) {
      adj[(int64_t)v * R + deg[v]] = (int32_t)u;
      deg[v] += 1;
      atomicOr(bm + (u >> 5), 1u << (u & 31));
      f0[0] = (int32_t)u;
      sfc[0] = 1;
      ++made;
    }
    __syncthreads();
    int cur = 0;
    bool big = false;
    for (;;) {
      const int fc = sfc[cur];
      if (fc == 0) break;
      if (fc > limit) {
        big = true;
        break;
      }
      __syncthreads();
      if (tid == 0) sfc[cur ^ 1] = 0;
      __syncthreads();
      const int32_t* fr = cur ? f1 : f0;
      int32_t* nx = cur ? f0 : f1;
      for (int w = warp; w < fc; w += nwarps) {
        const int32_t node = fr[w];
        const int dg = deg[node];
        for (int c = 0; c < dg; c += 32) {
          const int t = c + lane;
          bool fresh = false;
          int32_t x = 0;
          if (t < dg) {
            x = adj[(int64_t)node * R + t];
            const uint32_t bit = 1u << (x & 31);
            fresh = !(atomicOr(bm + (x >> 5), bit) & bit);
          }
          const unsigned bal = __ballot_sync(0xffffffffu, fresh);
          int basep = 0;
          if (lane == 0 && bal) basep = atomicAdd(&sfc[cur ^ 1], __popc(bal));
          basep = __shfl_sync(0xffffffffu, basep, 0);
          if (fresh) nx[basep + __popc(bal & lanemask_lt())] = x;
        }
      }
      __syncthreads();
      cur ^= 1;
    }
    if (big) {
      if (tid == 0) {
        s->u = (unsigned long long)u;
        s->best = v;
        s->fcnt[cur] = sfc[cur];
        s->bfs_state = cur;
      }
      break;
    }
    start = u >> 5;
    __syncthreads();
  }
  if (tid == 0 && made) atomicAdd(nrep, made);
}

// Level-synchronous traversal by the whole grid, starting from frontier buffer `cur`: the
// levels are launched in batches (4, 8, 16, then 32 at a time) and the host reads the
// next frontier's size once per batch.
static void bfs_levels(const int32_t* adj, const int32_t* deg, int R, uint32_t* bm, int32_t* f[2],
                       RepairState* s, int cur, cudaStream_t st) {
  const int grid = 4 * num_sms();
  SSG_LAUNCH(k_ring_init, 1, 1, 0, st, s->lvl, &s->fcnt[cur]);
  int l = 0, batch = 4;
  for (;;) {
    for (int b = 0; b < batch; ++b, ++l)
      SSG_LAUNCH(k_bfs_level_ring, grid, 256, 0, st, adj, deg, R, bm, f[(cur + l) & 1],
                 f[(cur + l + 1) & 1], s->lvl, l);
    int h = 0;
    SSG_CUDA(cudaMemcpyAsync(&h, &s->lvl[l % 3], sizeof(int), cudaMemcpyDeviceToHost, st));
    SSG_CUDA(cudaStreamSynchronize(st));
    if (h == 0) break;
    batch = std::min(2 * batch, 32);
  }
}

int64_t connect_run(const float* X, int ld, int d, int64_t n, int32_t* adj, int32_t* deg,
                    int R, const int32_t* nav_dev, const int32_t* nav_host, int n_nav,
                    cudaStream_t st, const int32_t* knn, int K, int64_t* knn_repairs) {
  (void)nav_dev;
  Scratch<unsigned long long> knn_rep;
  if (knn) {
    knn_rep.alloc(1, st);
    SSG_CUDA(cudaMemsetAsync(knn_rep.p, 0, sizeof(unsigned long long), st));
  }
  const int64_t nw = ceil_div(n, 32);
  const int cap = 1 << 16;
  Scratch<uint32_t> bm((size_t)nw, st);
  Scratch<int32_t> f0((size_t)n, st), f1((size_t)n, st), band_ids((size_t)cap, st);
  Scratch<double> band_d((size_t)cap, st);
  Scratch<float> d32((size_t)n, st);
  Scratch<RepairState> state(1, st);
  Scratch<unsigned long long> ull(1, st);
  Scratch<double> dv;
  int32_t* f[2] = {f0.p, f1.p};
  RepairState* S = state.p;
  const int grid = 8 * num_sms();
  const float rel = dist_rel_team8(ld);
  const int small_limit = 4096;
  int64_t repairs = 0;
  for (int r = 0; r < n_nav; ++r) {
    SSG_CUDA(cudaMemsetAsync(bm.p, 0, sizeof(uint32_t) * nw, st));
    SSG_LAUNCH(k_mark, 1, 1, 0, st, bm.p, f[0], &S->fcnt[0], nav_host[r]);
    int64_t start = 0;
    bool first = true;
    for (;;) {
      if (!first && knn) {
        // the repairs the kNN rows settle, in one launch; the rest below
        SSG_LAUNCH(k_repair_knn, 1, 1024, 0, st, knn, K, adj, deg, R, bm.p, nw, n, start, f[0], f[1],
                   small_limit, S, knn_rep.p);
        RepairState h;
        SSG_CUDA(cudaMemcpyAsync(&h, S, sizeof(h), cudaMemcpyDeviceToHost, st));
        SSG_CUDA(cudaStreamSynchronize(st));
        if ((int64_t)h.u >= n) break;
        start = (int64_t)h.u >> 5;
        if (h.best != -3) {
          // u is linked and its traversal outgrew the block: the grid finishes it
          if (h.bfs_state >= 0) bfs_levels(adj, deg, R, bm.p, f, S, h.bfs_state, st);
          continue;
        }
      }
      if (!first) {
        SSG_LAUNCH(k_repair_init, 1, 1, 0, st, S, n);
        SSG_LAUNCH(k_first_unreached, grid, 256, 0, st, bm.p, nw, n, start, &S->u);
        SSG_LAUNCH(k_repair_fp32, grid, 256, 0, st, X, ld, n, bm.p, deg, R, rel, d32.p, S);
        SSG_LAUNCH(k_repair_band, grid, 256, 0, st, X, ld, d, n, d32.p, rel, cap, band_ids.p,
                   band_d.p, S);
        SSG_LAUNCH(k_repair_band64, 2 * num_sms(), 256, 0, st, X, ld, d, n, cap, band_ids.p,
                   band_d.p, S);
        SSG_LAUNCH(k_repair_pick, 1, 256, 0, st, X, ld, d, band_ids.p, band_d.p, cap, adj, deg, R,
                   bm.p, f[0], n, S);
      }
      SSG_LAUNCH(k_bfs_small, 1, 1024, 0, st, adj, deg, R, bm.p, f[0], f[1], small_limit, S);
      RepairState h;
      SSG_CUDA(cudaMemcpyAsync(&h, S, sizeof(h), cudaMemcpyDeviceToHost, st));
      SSG_CUDA(cudaStreamSynchronize(st));
      if (!first) {
        if ((int64_t)h.u >= n) break;
        if (h.best == -2) {
          // the band list overflowed (many exact ties): exhaustive fp64 argmin instead
          if (!dv.p) dv.alloc((size_t)n, st);
          const unsigned long long init = ~0ull;
          const int imax = INT_MAX;
          SSG_CUDA(cudaMemcpyAsync(ull.p, &init, sizeof(init), cudaMemcpyHostToDevice, st));
          SSG_CUDA(cudaMemcpyAsync(&S->best, &imax, sizeof(int), cudaMemcpyHostToDevice, st));
          SSG_LAUNCH(k_repair_dist, grid, 256, 0, st, X, ld, d, n, bm.p, deg, R, (int64_t)h.u,
                     dv.p, ull.p);
          SSG_LAUNCH(k_repair_pick_all, grid, 256, 0, st, dv.p, n, ull.p, &S->best);
          SSG_LAUNCH(k_add_edge, 1, 1, 0, st, adj, deg, R, &S->best, bm.p, f[0], S);
          SSG_LAUNCH(k_bfs_small, 1, 1024, 0, st, adj, deg, R, bm.p, f[0], f[1], small_limit, S);
          SSG_CUDA(cudaMemcpyAsync(&h, S, sizeof(h), cudaMemcpyDeviceToHost, st));
          SSG_CUDA(cudaStreamSynchronize(st));
        }
        SSG_REQUIRE(h.best != INT_MAX, SSG_EINTERNAL,
                    "connectivity: node %lld is unreached and no reached node has a free slot",
                    (long long)h.u);
        start = (int64_t)h.u >> 5;
        ++repairs;
      }
      if (h.bfs_state >= 0) bfs_levels(adj, deg, R, bm.p, f, S, h.bfs_state, st);
      first = false;
    }
  }
  if (knn) {
    unsigned long long kr = 0;
    SSG_CUDA(cudaMemcpyAsync(&kr, knn_rep.p, sizeof(kr), cudaMemcpyDeviceToHost, st));
    SSG_CUDA(cudaStreamSynchronize(st));
    repairs += (int64_t)kr;
    if (knn_repairs) *knn_repairs = (int64_t)kr;
  }
  return repairs;
}

// ---------------------------------------------------------------------------------------
// Connectivity without device allocation (ssg_connect_noalloc).
//
// Some callers cannot allocate device memory while they run: serving loops that fix all
// their device memory before they take requests, or hosts that own a custom allocator and
// forbid the driver's.  For them the connectivity step also comes with its scratch in one
// fixed array that is part of the library's device image: the bitmap of reached nodes,
// two frontier buffers, the fp32 distance of every node and the short list of fp64
// re-tests, for graphs of up to NOALLOC_MAX_N nodes.  The same kernels run as in
// ssg_connect; only the scratch differs.  Like ssg_connect, the call reads the navigating
// ids and each repair's state back to the host, synchronising its stream each time.
// ---------------------------------------------------------------------------------------
namespace {
constexpr int64_t NOALLOC_MAX_N = 1 << 20;       // nodes
constexpr int NOALLOC_BAND = 1 << 14;            // fp64 re-tests per repair
constexpr size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }
constexpr size_t OFF_BM = 0;
constexpr size_t OFF_F0 = al256(OFF_BM + (size_t)(NOALLOC_MAX_N / 32) * 4);
constexpr size_t OFF_F1 = al256(OFF_F0 + (size_t)NOALLOC_MAX_N * 4);
constexpr size_t OFF_D32 = al256(OFF_F1 + (size_t)NOALLOC_MAX_N * 4);
constexpr size_t OFF_BAND_ID = al256(OFF_D32 + (size_t)NOALLOC_MAX_N * 4);
constexpr size_t OFF_BAND_D = al256(OFF_BAND_ID + (size_t)NOALLOC_BAND * 4);
constexpr size_t OFF_STATE = al256(OFF_BAND_D + (size_t)NOALLOC_BAND * 8);
constexpr size_t NOALLOC_BYTES = al256(OFF_STATE + sizeof(RepairState));
}  // namespace

// Held by every GPU that loads the library, until the process exits (about 12.3 MiB).
static __device__ __align__(256) unsigned char g_connect_scratch[NOALLOC_BYTES];

// Device address of g_connect_scratch on the current device, looked up once per device
// (host code cannot use the array's name as a device address).
static unsigned char* noalloc_scratch() {
  static std::mutex mu;
  static unsigned char* addr[64] = {};
  int dev = 0;
  SSG_CUDA(cudaGetDevice(&dev));
  SSG_REQUIRE(dev >= 0 && dev < 64, SSG_EINTERNAL, "device ordinal %d out of range", dev);
  std::lock_guard<std::mutex> lock(mu);
  if (!addr[dev]) {
    void* p = nullptr;
    SSG_CUDA(cudaGetSymbolAddress(&p, g_connect_scratch));
    addr[dev] = (unsigned char*)p;
  }
  return addr[dev];
}

static int64_t connect_run_noalloc(const float* X, int ld, int d, int64_t n, int32_t* adj,
                                   int32_t* deg, int R, const int32_t* nav_dev,
                                   const int32_t* nav_host, int n_nav, cudaStream_t st) {
  (void)nav_dev;
  unsigned char* base = noalloc_scratch();
  uint32_t* bm = (uint32_t*)(base + OFF_BM);
  int32_t* f[2] = {(int32_t*)(base + OFF_F0), (int32_t*)(base + OFF_F1)};
  float* d32 = (float*)(base + OFF_D32);
  int32_t* band_ids = (int32_t*)(base + OFF_BAND_ID);
  double* band_d = (double*)(base + OFF_BAND_D);
  RepairState* S = (RepairState*)(base + OFF_STATE);
  const int64_t nw = ceil_div(n, 32);
  const int grid = 8 * num_sms();
  const float rel = dist_rel_team8(ld);
  const int small_limit = 4096;
  int64_t repairs = 0;
  for (int r = 0; r < n_nav; ++r) {
    const int32_t root = nav_host[r];
    SSG_CUDA(cudaMemsetAsync(bm, 0, sizeof(uint32_t) * nw, st));
    SSG_LAUNCH(k_mark, 1, 1, 0, st, bm, f[0], &S->fcnt[0], root);
    int64_t start = 0;
    bool first = true;
    for (;;) {
      if (!first) {
        SSG_LAUNCH(k_repair_init, 1, 1, 0, st, S, n);
        SSG_LAUNCH(k_first_unreached, grid, 256, 0, st, bm, nw, n, start, &S->u);
        SSG_LAUNCH(k_repair_fp32, grid, 256, 0, st, X, ld, n, bm, deg, R, rel, d32, S);
        SSG_LAUNCH(k_repair_band, grid, 256, 0, st, X, ld, d, n, d32, rel, NOALLOC_BAND, band_ids,
                   band_d, S);
        SSG_LAUNCH(k_repair_band64, 2 * num_sms(), 256, 0, st, X, ld, d, n, NOALLOC_BAND, band_ids,
                   band_d, S);
        SSG_LAUNCH(k_repair_pick, 1, 256, 0, st, X, ld, d, band_ids, band_d, NOALLOC_BAND, adj, deg,
                   R, bm, f[0], n, S);
      }
      SSG_LAUNCH(k_bfs_small, 1, 1024, 0, st, adj, deg, R, bm, f[0], f[1], small_limit, S);
      RepairState h;
      SSG_CUDA(cudaMemcpyAsync(&h, S, sizeof(h), cudaMemcpyDeviceToHost, st));
      SSG_CUDA(cudaStreamSynchronize(st));
      if (!first) {
        if ((int64_t)h.u >= n) break;
        SSG_REQUIRE(h.best != -2, SSG_EINTERNAL,
                    "connectivity without allocation: more than %d nodes tie for the nearest "
                    "reached node of node %lld; use ssg_connect",
                    NOALLOC_BAND, (long long)h.u);
        SSG_REQUIRE(h.best != INT_MAX, SSG_EINTERNAL,
                    "connectivity: node %lld is unreached and no reached node has a free slot",
                    (long long)h.u);
        start = (int64_t)h.u >> 5;
        ++repairs;
      }
      if (h.bfs_state >= 0) bfs_levels(adj, deg, R, bm, f, S, h.bfs_state, st);
      first = false;
    }
  }
  return repairs;
}

}  // namespace ssg

extern "C" ssg_status ssg_connect_noalloc(const float* base, int64_t n, int32_t d, int32_t* adj,
                                          int32_t* deg, int32_t R, const int32_t* nav,
                                          int32_t n_nav, int64_t* n_repair_host,
                                          ssg_stream stream) {
  using namespace ssg;
  try {
    SSG_REQUIRE(base && adj && deg && nav, SSG_EINVAL, "null pointer");
    SSG_REQUIRE(n >= 1 && n <= NOALLOC_MAX_N, SSG_EINVAL,
                "connectivity without allocation handles 1 <= n <= %lld nodes, got %lld",
                (long long)NOALLOC_MAX_N, (long long)n);
    SSG_REQUIRE(d >= 1 && d % 4 == 0 && ((uintptr_t)base & 15) == 0, SSG_EINVAL,
                "connectivity without allocation needs d %% 4 == 0 and a 16-byte aligned base "
                "(no padded copy is made), got d = %d",
                d);
    SSG_REQUIRE(R >= 1 && n_nav >= 1, SSG_EINVAL, "need R >= 1 and n_nav >= 1");
    cudaStream_t st = (cudaStream_t)stream;
    // every navigating id is checked before the graph is touched (host memory only)
    std::vector<int32_t> h((size_t)n_nav);
    SSG_CUDA(cudaMemcpyAsync(h.data(), nav, sizeof(int32_t) * n_nav, cudaMemcpyDeviceToHost, st));
    SSG_CUDA(cudaStreamSynchronize(st));
    for (int t = 0; t < n_nav; ++t)
      SSG_REQUIRE(h[t] >= 0 && h[t] < n, SSG_EINVAL, "navigating node id %d out of range", h[t]);
    const int64_t rep = connect_run_noalloc(base, d, d, n, adj, deg, R, nav, h.data(), n_nav, st);
    if (n_repair_host) *n_repair_host = rep;
    return SSG_OK;
  } catch (const Fail& e) {
    return e.st;
  } catch (const std::bad_alloc&) {
    set_error("host allocation failed");
    return SSG_ENOMEM;
  } catch (...) {
    set_error("unexpected exception");
    return SSG_EINTERNAL;
  }
}
