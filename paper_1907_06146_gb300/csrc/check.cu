// Invariant checks of the build's intermediate and final arrays (ssg_build_opts.debug_checks,
// ssg_check_graph).  The checks only read the arrays within their declared shapes and
// compare ids; no id is ever dereferenced, so a corrupt array is reported, never followed.
// The first failing row (smallest index) and its failure code go to one 64-bit word:
// row << 8 | code.
#include "common.cuh"
#include "knn.cuh"

namespace ssg {

// Adjacency [n][R] (-1 padded) with degrees [n]: 0 <= deg <= R; every listed id in [0, n),
// not the row itself, listed once; every slot past deg -1.
__global__ void k_check_adj(const int32_t* __restrict__ adj, const int32_t* __restrict__ deg,
                            int64_t n, int R, unsigned long long* __restrict__ bad) {
  __shared__ int32_t ids[8][128];
  const int warp = threadIdx.x >> 5, lane = lane_id();
  for (int64_t i = (int64_t)blockIdx.x * 8 + warp; i < n; i += (int64_t)gridDim.x * 8) {
    const int dg = deg[i];
    int code = 0;
    if (dg < 0 || dg > R) code = CHECK_DEGREE;
    for (int t = lane; t < R; t += 32) {
      const int32_t v = adj[i * R + t];
      ids[warp][t] = v;
      if (code == 0) {
        if (t < dg) {
          if (v < 0 || v >= n) code = CHECK_RANGE;
          else if (v == (int32_t)i) code = CHECK_SELF;
        } else if (v != -1) {
          code = CHECK_PADDING;
        }
      }
    }
    __syncwarp();
    if (dg >= 0 && dg <= R) {
      for (int t = lane; t < dg && code == 0; t += 32)
        for (int u = t + 1; u < dg; ++u)
          if (ids[warp][u] == ids[warp][t]) {
            code = CHECK_DUPLICATE;
            break;
          }
    }
    if (code) atomicMin(bad, ((unsigned long long)i << 8) | (unsigned long long)code);
    __syncwarp();
  }
}

// Pools [n][L] with lengths [n]: 0 <= len <= L; ids in [0, n), not the node; slots past len
// -1; in order.  exact data: keys strictly increasing in (d2, id), so no id twice.  Other
// data: the pool is in exact (d2, id) order while the stored values are fp32, so each value
// may sit below its predecessor by the fp32 bound rel; an id twice would sit next to itself
// (same exact distance), so neighbours must differ.
__global__ void k_check_pool(const int32_t* __restrict__ pid, const float* __restrict__ pd2,
                             const int32_t* __restrict__ plen, int64_t n, int L, int exact,
                             float rel, unsigned long long* __restrict__ bad) {
  const int warp = threadIdx.x >> 5, lane = lane_id();
  for (int64_t i = (int64_t)blockIdx.x * 8 + warp; i < n; i += (int64_t)gridDim.x * 8) {
    const int len = plen[i];
    int code = 0;
    if (len < 0 || len > L) code = CHECK_DEGREE;
    for (int t = lane; t < L && code == 0; t += 32) {
      const int32_t v = pid[i * L + t];
      if (t < len) {
        if (v < 0 || v >= n) {
          code = CHECK_RANGE;
        } else if (v == (int32_t)i) {
          code = CHECK_SELF;
        } else if (t > 0) {
          const float pa = pd2[i * L + t - 1], pb = pd2[i * L + t];
          const int32_t ia = pid[i * L + t - 1];
          if (exact) {
            if (!(make_key(pa, ia) < make_key(pb, v))) code = CHECK_ORDER;
          } else if (ia == v) {
            code = CHECK_DUPLICATE;
          } else if (pa > pb + 2.f * rel * (pa + pb)) {
            code = CHECK_ORDER;
          }
        }
      } else if (v != -1) {
        code = CHECK_PADDING;
      }
    }
    if (code) atomicMin(bad, ((unsigned long long)i << 8) | (unsigned long long)code);
  }
}

static unsigned long long read_bad(Scratch<unsigned long long>& bad, cudaStream_t st) {
  unsigned long long h = ~0ull;
  SSG_CUDA(cudaMemcpyAsync(&h, bad.p, sizeof(h), cudaMemcpyDeviceToHost, st));
  SSG_CUDA(cudaStreamSynchronize(st));
  return h;
}

CheckResult check_adj(const int32_t* adj, const int32_t* deg, int64_t n, int R, cudaStream_t st) {
  Scratch<unsigned long long> bad(1, st);
  SSG_CUDA(cudaMemsetAsync(bad.p, 0xff, sizeof(unsigned long long), st));
  if (n > 0) {
    const int grid = (int)std::min<int64_t>(ceil_div(n, 8), 8 * num_sms());
    SSG_LAUNCH(k_check_adj, grid, 256, 0, st, adj, deg, n, R, bad.p);
  }
  const unsigned long long h = read_bad(bad, st);
  CheckResult r;
  if (h != ~0ull) {
    r.row = (int64_t)(h >> 8);
    r.code = (int)(h & 0xff);
  }
  return r;
}

CheckResult check_pool(const int32_t* pid, const float* pd2, const int32_t* plen, int64_t n, int L,
                       int exact, int d, cudaStream_t st) {
  Scratch<unsigned long long> bad(1, st);
  SSG_CUDA(cudaMemsetAsync(bad.p, 0xff, sizeof(unsigned long long), st));
  if (n > 0) {
    const int grid = (int)std::min<int64_t>(ceil_div(n, 8), 8 * num_sms());
    SSG_LAUNCH(k_check_pool, grid, 256, 0, st, pid, pd2, plen, n, L, exact, dist_rel_team8((d + 3) & ~3),
               bad.p);
  }
  const unsigned long long h = read_bad(bad, st);
  CheckResult r;
  if (h != ~0ull) {
    r.row = (int64_t)(h >> 8);
    r.code = (int)(h & 0xff);
  }
  return r;
}

const char* check_name(int code) {
  switch (code) {
    case CHECK_DEGREE: return "degree (or pool length) outside [0, cap]";
    case CHECK_RANGE: return "an id outside [0, n)";
    case CHECK_SELF: return "the node listed as its own neighbour";
    case CHECK_DUPLICATE: return "an id listed twice";
    case CHECK_PADDING: return "a slot past the degree that is not -1";
    case CHECK_ORDER: return "entries not strictly increasing in (d2, id)";
    default: return "none";
  }
}

}  // namespace ssg
