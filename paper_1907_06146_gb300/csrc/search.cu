// Search-on-Graph (Alg. 1) from the navigating node nearest the query (Sec. 4.1).
//
// One warp per query.  The candidate pool S (at most L_search entries, sorted by
// (d2, id), with a checked flag each) lives in shared memory; each round expands the
// first unchecked entry, gathers its adjacency row (coalesced), computes the distances
// of the neighbours not seen before with teams of 8 lanes, two rows per team at a time
// (all of both rows' float4 loads issued before the first multiply-add, so a warp keeps
// 8 row gathers in flight), sorts them with a warp bitonic sort and merges them into S
// with a rank-based parallel merge, cut at L_search.
//
// Rows: float32, or -- for data that are integers 0..255 -- a byte copy of the same
// values.  A byte row of 128 dimensions is one 128-byte line instead of four; every lane
// converts its bytes to the same float values and sums them in the same order as the
// float path, so the distances and results are bit for bit those of the float rows.
//
// Visited set: a direct-mapped cache of ids in shared memory.  Alg. 1 never re-adds a
// visited node; here a node that fell out of the cache may be met again and its distance
// recomputed, but the result is the same: a node that is still in S has the same key and
// is dropped by the duplicate check of the merge, and a node that left S (or never
// entered it) did so because S was full and its key was above the L_search-th key, which
// never increases once S is full, so it is cut again.  Before S first fills nothing has
// left it.  The cache only saves distance computations.
#include <type_traits>

#include "common.cuh"
#include "graph_dev.cuh"
#include "knn.cuh"

namespace ssg {

// Four consecutive values of a row as floats: one float4 load, or one 32-bit load of four
// bytes (each byte b becomes the float 2^23 + b by placing it under the exponent bits of
// 2^23, then b exactly by subtracting 2^23).
__device__ __forceinline__ float4 row_raw(const float* x, int f) {
  return __ldg((const float4*)x + f);
}
__device__ __forceinline__ uint32_t row_raw(const uint8_t* x, int f) {
  return __ldg((const unsigned int*)x + f);
}
__device__ __forceinline__ float4 raw_f4(float4 v) { return v; }
__device__ __forceinline__ float byte_f(uint32_t w, uint32_t sel) {
  return __uint_as_float(__byte_perm(w, 0x4B000000u, sel)) - 8388608.f;
}
__device__ __forceinline__ float4 raw_f4(uint32_t w) {
  return make_float4(byte_f(w, 0x7440), byte_f(w, 0x7441), byte_f(w, 0x7442), byte_f(w, 0x7443));
}
template <typename T>
struct RawOf;
template <>
struct RawOf<float> {
  using type = float4;
  static __device__ __forceinline__ float4 zero() { return make_float4(0.f, 0.f, 0.f, 0.f); }
};
template <>
struct RawOf<uint8_t> {
  using type = uint32_t;
  static __device__ __forceinline__ uint32_t zero() { return 0u; }
};

// x: a row of ld values (ld4 = ld / 4 groups of four)
template <typename T>
__device__ __forceinline__ float team8_dist_q(const float* __restrict__ qs,
                                              const T* __restrict__ x, int ld4, int tl,
                                              bool valid) {
  using Raw = typename RawOf<T>::type;
  float s = 0.f;
  if (valid) {
    const float4* q4 = (const float4*)qs;
    // the row's loads (up to four per lane per 128 values) are all issued before the first
    // multiply-add
    for (int f0 = tl; f0 < ld4; f0 += 32) {
      Raw b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int f = f0 + 8 * i;
        b[i] = f < ld4 ? row_raw(x, f) : RawOf<T>::zero();
      }
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int f = f0 + 8 * i;
        if (f < ld4) {
          const float4 a = q4[f];
          const float4 v = raw_f4(b[i]);
          float u;
          u = a.x - v.x;
          s = fmaf(u, u, s);
          u = a.y - v.y;
          s = fmaf(u, u, s);
          u = a.z - v.z;
          s = fmaf(u, u, s);
          u = a.w - v.w;
          s = fmaf(u, u, s);
        }
      }
    }
  }
  s += __shfl_xor_sync(0xffffffffu, s, 1);
  s += __shfl_xor_sync(0xffffffffu, s, 2);
  s += __shfl_xor_sync(0xffffffffu, s, 4);
  return s;
}

// NR rows per team at once (4 NR rows in flight per warp): the loads of all NR rows are
// issued before the first multiply-add.  Each row's sum runs in the same order as in
// team8_dist_q.  Rows are X + ids[r] * ld; rows with valid[r] false give 0.
template <typename T, int NR>
__device__ __forceinline__ void team8_distN_q(const float* __restrict__ qs,
                                              const T* __restrict__ X, int ld,
                                              const int32_t (&ids)[NR], const bool (&valid)[NR],
                                              int ld4, int tl, float (&out)[NR]) {
  using Raw = typename RawOf<T>::type;
  const float4* q4 = (const float4*)qs;
#pragma unroll
  for (int r = 0; r < NR; ++r) out[r] = 0.f;
  for (int f0 = tl; f0 < ld4; f0 += 32) {
    Raw raw[NR][4];
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      const T* x = X + (int64_t)ids[r] * ld;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int f = f0 + 8 * i;
        raw[r][i] = (valid[r] && f < ld4) ? row_raw(x, f) : RawOf<T>::zero();
      }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int f = f0 + 8 * i;
      if (f < ld4) {
        const float4 q = q4[f];
#pragma unroll
        for (int r = 0; r < NR; ++r) {
          const float4 v = raw_f4(raw[r][i]);
          float u;
          u = q.x - v.x; out[r] = fmaf(u, u, out[r]);
          u = q.y - v.y; out[r] = fmaf(u, u, out[r]);
          u = q.z - v.z; out[r] = fmaf(u, u, out[r]);
          u = q.w - v.w; out[r] = fmaf(u, u, out[r]);
        }
      }
    }
  }
#pragma unroll
  for (int o = 1; o < 8; o <<= 1) {
#pragma unroll
    for (int r = 0; r < NR; ++r) out[r] += __shfl_xor_sync(0xffffffffu, out[r], o);
  }
}

// Integer queries (every value an integer 0..255) against byte rows: with the query's bytes
// packed four to a word (qw) and q2 = |q|^2, d2 = q2 + |x|^2 - 2 q.x from byte dot products
// (dp4a), all in exact integer arithmetic.  Every value and partial sum of the float path
// is an integer below 2^24 in that case, so the float path's sums are exact too and the two
// give the same distances.
template <int NR>
__device__ __forceinline__ void team8_distN_qi(const uint32_t* __restrict__ qw,
                                               const uint8_t* __restrict__ X, int ld,
                                               const int32_t (&ids)[NR],
                                               const bool (&valid)[NR], int ld4, int tl, int q2,
                                               float (&out)[NR]) {
  unsigned dot[NR], xx[NR];
#pragma unroll
  for (int r = 0; r < NR; ++r) dot[r] = xx[r] = 0u;
  for (int f0 = tl; f0 < ld4; f0 += 32) {
    uint32_t raw[NR][4];
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      const uint8_t* x = X + (int64_t)ids[r] * ld;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int f = f0 + 8 * i;
        raw[r][i] = (valid[r] && f < ld4) ? row_raw(x, f) : 0u;
      }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int f = f0 + 8 * i;
      if (f < ld4) {
        const uint32_t q = qw[f];
#pragma unroll
        for (int r = 0; r < NR; ++r) {
          dot[r] = __dp4a(q, raw[r][i], dot[r]);
          xx[r] = __dp4a(raw[r][i], raw[r][i], xx[r]);
        }
      }
    }
  }
#pragma unroll
  for (int o = 1; o < 8; o <<= 1) {
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      dot[r] += __shfl_xor_sync(0xffffffffu, dot[r], o);
      xx[r] += __shfl_xor_sync(0xffffffffu, xx[r], o);
    }
  }
#pragma unroll
  for (int r = 0; r < NR; ++r) out[r] = (float)((int)q2 + (int)xx[r] - 2 * (int)dot[r]);
}

// Ascending bitonic sort of one key per lane across the warp (in registers).
__device__ __forceinline__ uint64_t warp_bitonic32(uint64_t b, int lane) {
#pragma unroll
  for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
    for (int j = k >> 1; j > 0; j >>= 1) {
      const uint64_t o = __shfl_xor_sync(0xffffffffu, b, j);
      const bool take_min = ((lane & j) == 0) == ((lane & k) == 0);
      b = take_min ? (o < b ? o : b) : (o > b ? o : b);
    }
  }
  return b;
}

// Same for two keys per lane (element e * 32 + lane in v[e]), 64 in all.
__device__ __forceinline__ void warp_bitonic64(uint64_t (&v)[2], int lane) {
#pragma unroll
  for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
    for (int j = k >> 1; j > 0; j >>= 1) {
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const uint64_t o = __shfl_xor_sync(0xffffffffu, v[e], j);
        const bool up = (((e << 5) | lane) & k) == 0;
        const bool take_min = ((lane & j) == 0) == up;
        v[e] = take_min ? (o < v[e] ? o : v[e]) : (o > v[e] ? o : v[e]);
      }
    }
  }
  // k = 64: the pair within a lane, then the halves
  if (v[1] < v[0]) {
    const uint64_t t = v[0];
    v[0] = v[1];
    v[1] = t;
  }
#pragma unroll
  for (int j = 16; j > 0; j >>= 1) {
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const uint64_t o = __shfl_xor_sync(0xffffffffu, v[e], j);
      const bool take_min = (lane & j) == 0;
      v[e] = take_min ? (o < v[e] ? o : v[e]) : (o > v[e] ? o : v[e]);
    }
  }
}

// number of entries of a[0, len) that are < x (a sorted ascending)
__device__ __forceinline__ int count_less(const uint64_t* a, int len, uint64_t x) {
  int lo = 0, hi = len;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (a[mid] < x)
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo;
}

struct SearchLayout {
  int Ls, RP, ld, log2h;
  __host__ __device__ size_t pool_bytes() const { return (size_t)Ls * 8; }
  __host__ __device__ size_t per_warp() const {
    size_t b = 2 * pool_bytes() + (((size_t)2 * Ls + 15) & ~(size_t)15) + (size_t)RP * 8 +
               (size_t)ld * 4 + ((size_t)4 << log2h) + (((size_t)ld + 15) & ~(size_t)15);
    return (b + 15) & ~(size_t)15;
  }
};

// Rows per team in the distance loop: a float row takes 16 registers per lane at d = 128,
// a byte row 4, so byte rows keep twice as many rows in flight at the same 24 warps per SM
// (measured on 1M x 128, L_search 40: 1.30 ms with 4 rows per team at 24 warps, 1.35 ms
// with 2 at 32 warps, 1.76 ms with 8 at 16 warps; float rows 1.45 ms).
template <typename T>
struct RowsPerTeam {
  static constexpr int value = 2;
};
template <>
struct RowsPerTeam<uint8_t> {
  static constexpr int value = 4;
};

template <typename T>
__global__ void __launch_bounds__(256, 3)
    k_search(const T* __restrict__ X, int ld, int d, const int32_t* __restrict__ adj,
                         const int32_t* __restrict__ deg, int R, const int32_t* __restrict__ nav,
                         int n_nav, const float* __restrict__ Q, int ldq, int64_t nq, int k,
                         const int32_t* __restrict__ qk, const int32_t* __restrict__ qls, int ldo,
                         SearchLayout lay, int32_t* __restrict__ out_ids,
                         float* __restrict__ out_d2, unsigned long long* __restrict__ work) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  const int wpb = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = lane_id();
  const int team = lane >> 3, tl = lane & 7;
  const int LsCap = lay.Ls;
  unsigned char* base = sm_raw + (size_t)warp * lay.per_warp();
  uint64_t* pA0 = (uint64_t*)base;
  uint64_t* pB0 = pA0 + LsCap;
  unsigned char* fA0 = (unsigned char*)(pB0 + LsCap);
  unsigned char* fB0 = fA0 + LsCap;
  uint64_t* newk = (uint64_t*)(base + 2 * lay.pool_bytes() + (((size_t)2 * LsCap + 15) & ~(size_t)15));
  float* qs = (float*)(newk + lay.RP);
  int32_t* cache = (int32_t*)(qs + ld);
  const int hcap = 1 << lay.log2h;
  uint32_t* qw = (uint32_t*)(cache + hcap);  // the query's bytes, when it is integer 0..255
  const int ld4 = ld >> 2;
  (void)d;

  for (int64_t qi = (int64_t)blockIdx.x * wpb + warp; qi < nq; qi += (int64_t)gridDim.x * wpb) {
    // per-query pool size and result count (a batch may mix them; the layout is sized for
    // the largest pool)
    const int Ls = qls ? qls[qi] : LsCap;
    const int kq = qk ? qk[qi] : k;
    uint64_t* pA = pA0;
    uint64_t* pB = pB0;
    unsigned char* fA = fA0;
    unsigned char* fB = fB0;
    const float* qg = Q + qi * ldq;
    for (int t = lane; t < ld; t += 32) qs[t] = t < d ? qg[t] : 0.f;
    for (int t = lane; t < hcap; t += 32) cache[t] = -1;
    __syncwarp();
    bool qint = false;
    int q2 = 0;
    if constexpr (std::is_same<T, uint8_t>::value) {
      bool ok = true;
      int sq = 0;
      for (int t = lane; t < ld; t += 32) {
        const float v = qs[t];
        ok = ok && v >= 0.f && v <= 255.f && v == rintf(v);
        const int iv = ok ? (int)v : 0;
        sq += iv * iv;
      }
      qint = __all_sync(0xffffffffu, ok);
      if (qint) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
        q2 = sq;
        for (int w = lane; w < ld4; w += 32)
          qw[w] = (uint32_t)qs[4 * w] | ((uint32_t)qs[4 * w + 1] << 8) |
                  ((uint32_t)qs[4 * w + 2] << 16) | ((uint32_t)qs[4 * w + 3] << 24);
        __syncwarp();
      }
    }

    // entry: the nearest navigating node by (d2, id)
    uint64_t best = KEY_NONE;
    for (int s0 = 0; s0 < n_nav; s0 += 4) {
      const int s = s0 + team;
      const bool valid = s < n_nav;
      const int32_t id = valid ? nav[s] : 0;
      const float dd = team8_dist_q(qs, X + (int64_t)id * ld, ld4, tl, valid);
      const uint64_t key = valid ? make_key(dd, id) : KEY_NONE;
      best = key < best ? key : best;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      uint64_t other = __shfl_xor_sync(0xffffffffu, best, o);
      best = other < best ? other : best;
    }
    if (lane == 0) {
      pA[0] = best;
      fA[0] = 0;
      const int32_t e = key_id(best);
      cache[((uint32_t)e * 2654435761u) >> (32 - lay.log2h)] = e;
    }
    int s = 1;
    unsigned long long w_exp = 0, w_dist = (unsigned long long)n_nav, w_adj = 0;
    __syncwarp();

    for (;;) {
      int p = -1;
      for (int c = 0; c < s; c += 32) {
        const int idx = c + lane;
        const unsigned bal = __ballot_sync(0xffffffffu, idx < s && !fA[idx]);
        if (bal) {
          p = c + __ffs(bal) - 1;
          break;
        }
      }
      if (p < 0) break;
      const int32_t node = key_id(pA[p]);
      __syncwarp();
      if (lane == 0) fA[p] = 1;
      const int dg = deg[node];
      int cnt = 0;
      for (int c = 0; c < dg; c += 32) {
        const int t = c + lane;
        bool fresh = false;
        int32_t id = -1;
        if (t < dg) {
          id = adj[(int64_t)node * R + t];
          const uint32_t slot = ((uint32_t)id * 2654435761u) >> (32 - lay.log2h);
          if (cache[slot] != id) {
            cache[slot] = id;
            fresh = true;
          }
        }
        const unsigned bal = __ballot_sync(0xffffffffu, fresh);
        if (fresh) newk[cnt + __popc(bal & lanemask_lt())] = (uint64_t)(uint32_t)id;
        cnt += __popc(bal);
      }
      ++w_exp;
      w_adj += (unsigned long long)dg;
      w_dist += (unsigned long long)cnt;
      __syncwarp();
      constexpr int NR = RowsPerTeam<T>::value;
      for (int t0 = 0; t0 < cnt; t0 += 4 * NR) {
        int32_t ir[NR];
        bool vr[NR];
        float dd[NR];
#pragma unroll
        for (int r = 0; r < NR; ++r) {
          const int t = t0 + 4 * r + team;
          vr[r] = t < cnt;
          ir[r] = vr[r] ? key_id(newk[t]) : 0;
        }
        if constexpr (std::is_same<T, uint8_t>::value) {
          if (qint)
            team8_distN_qi<NR>(qw, X, ld, ir, vr, ld4, tl, q2, dd);
          else
            team8_distN_q<T, NR>(qs, X, ld, ir, vr, ld4, tl, dd);
        } else {
          team8_distN_q<T, NR>(qs, X, ld, ir, vr, ld4, tl, dd);
        }
        __syncwarp();
        if (tl == 0) {
#pragma unroll
          for (int r = 0; r < NR; ++r)
            if (vr[r]) newk[t0 + 4 * r + team] = make_key(dd[r], ir[r]);
        }
      }
      __syncwarp();
      if (cnt <= 64) {
        // one or two new keys per lane (element e * 32 + lane), sorted in registers; one
        // binary search in S gives both the duplicate test and the key's place in the merge
        uint64_t b[2];
        b[0] = lane < cnt ? newk[lane] : KEY_NONE;
        b[1] = lane + 32 < cnt ? newk[lane + 32] : KEY_NONE;
        if (cnt <= 32)
          b[0] = warp_bitonic32(b[0], lane);
        else
          warp_bitonic64(b, lane);
        int r[2] = {0, 0}, j[2];
        bool keep[2] = {false, false};
        int kept = 0;
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          if (e * 32 + lane < cnt) {
            r[e] = count_less(pA, s, b[e]);
            keep[e] = !(r[e] < s && pA[r[e]] == b[e]);
          }
          const unsigned bal = __ballot_sync(0xffffffffu, keep[e]);
          j[e] = kept + __popc(bal & lanemask_lt());
          kept += __popc(bal);
        }
        __syncwarp();
#pragma unroll
        for (int e = 0; e < 2; ++e)
          if (keep[e]) newk[j[e]] = b[e];
        __syncwarp();
        for (int i = lane; i < s; i += 32) {
          const uint64_t a = pA[i];
          const int pos = i + count_less(newk, kept, a);
          if (pos < Ls) {
            pB[pos] = a;
            fB[pos] = fA[i];
          }
        }
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          if (keep[e] && j[e] + r[e] < Ls) {
            pB[j[e] + r[e]] = b[e];
            fB[j[e] + r[e]] = 0;
          }
        }
        s = s + kept < Ls ? s + kept : Ls;
        __syncwarp();
        uint64_t* tp = pA;
        pA = pB;
        pB = tp;
        unsigned char* tf = fA;
        fA = fB;
        fB = tf;
        continue;
      }
      int cp = 1;
      while (cp < cnt) cp <<= 1;
      for (int t = cnt + lane; t < cp; t += 32) newk[t] = KEY_NONE;
      __syncwarp();
      warp_sort_keys(newk, cp);
      // drop keys already in S (same id => same key), compacting in place
      int kept = 0;
      for (int c = 0; c < cnt; c += 32) {
        const int j = c + lane;
        uint64_t b = KEY_NONE;
        bool keep = false;
        if (j < cnt) {
          b = newk[j];
          const int r = count_less(pA, s, b);
          keep = !(r < s && pA[r] == b);
        }
        const unsigned bal = __ballot_sync(0xffffffffu, keep);
        __syncwarp();
        if (keep) newk[kept + __popc(bal & lanemask_lt())] = b;
        kept += __popc(bal);
        __syncwarp();
      }
      // merge S and the new keys into the other buffer, cut at Ls
      for (int i = lane; i < s; i += 32) {
        const uint64_t a = pA[i];
        const int pos = i + count_less(newk, kept, a);
        if (pos < Ls) {
          pB[pos] = a;
          fB[pos] = fA[i];
        }
      }
      for (int j = lane; j < kept; j += 32) {
        const uint64_t b = newk[j];
        const int pos = j + count_less(pA, s, b);
        if (pos < Ls) {
          pB[pos] = b;
          fB[pos] = 0;
        }
      }
      s = s + kept < Ls ? s + kept : Ls;
      __syncwarp();
      uint64_t* tp = pA;
      pA = pB;
      pB = tp;
      unsigned char* tf = fA;
      fA = fB;
      fB = tf;
    }
    for (int t = lane; t < ldo; t += 32) {
      const bool v = t < s && t < kq;
      out_ids[qi * ldo + t] = v ? key_id(pA[t]) : -1;
      if (out_d2) out_d2[qi * ldo + t] = v ? key_dist(pA[t]) : __int_as_float(0x7f800000);
    }
    if (work && lane == 0) {
      atomicAdd(work, w_exp);
      atomicAdd(work + 1, w_dist);
      atomicAdd(work + 2, w_adj);
    }
    __syncwarp();
  }
}

__global__ void k_rows_u8(const float* __restrict__ X, int ld, int d, int64_t n,
                          uint8_t* __restrict__ out) {
  const int64_t total = n * (int64_t)ld;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int t = (int)(e % ld);
    out[e] = t < d ? (uint8_t)__float2uint_rn(X[e]) : (uint8_t)0;
  }
}

void rows_to_u8(const float* X, int ld, int d, int64_t n, uint8_t* out, cudaStream_t st) {
  SSG_LAUNCH(k_rows_u8, 8 * num_sms(), 256, 0, st, X, ld, d, n, out);
}

template <typename T>
static void launch_search(const T* X, int ld, int d, const int32_t* adj, const int32_t* deg, int R,
                          const int32_t* nav, int n_nav, const float* Q, int ldq, int64_t nq, int k,
                          const int32_t* qk, const int32_t* qls, int ldo, SearchLayout lay, int wpb,
                          int32_t* out_ids, float* out_d2, unsigned long long* work,
                          cudaStream_t st) {
  while (lay.per_warp() * wpb > 200 * 1024 && lay.log2h > 8) --lay.log2h;
  const size_t smem = lay.per_warp() * wpb;
  SSG_REQUIRE(smem <= 220 * 1024, SSG_EINVAL, "search: L_search and d too large for shared memory");
  ensure_smem((const void*)k_search<T>, smem);
  int blocks_per_sm = 0;
  SSG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, k_search<T>, wpb * 32, smem));
  const int64_t want = ceil_div(nq, wpb);
  const int grid = (int)std::min<int64_t>(want, (int64_t)std::max(1, blocks_per_sm) * num_sms());
  SSG_LAUNCH(k_search<T>, grid, wpb * 32, smem, st, X, ld, d, adj, deg, R, nav, n_nav, Q, ldq, nq,
             k, qk, qls, ldo, lay, out_ids, out_d2, work);
}

void search_run_mixed(const float* X, const uint8_t* X8, int ld, int d, const int32_t* adj,
                      const int32_t* deg, int R, const int32_t* nav, int n_nav, const float* Q,
                      int ldq, int64_t nq, const int32_t* qk, const int32_t* qls, int ls_max,
                      int ldo, int32_t* out_ids, float* out_d2, cudaStream_t st) {
  if (nq == 0) return;
  SearchLayout lay;
  lay.Ls = ls_max;
  lay.RP = std::max(32, next_pow2(R));
  lay.ld = ld;
  // 8 warps per block and a 1,024-entry visited cache: 24 warps per SM (the register
  // limit) keep more row gathers in flight than a larger cache would save
  lay.log2h = 10;
  if (X8)
    launch_search(X8, ld, d, adj, deg, R, nav, n_nav, Q, ldq, nq, 0, qk, qls, ldo, lay, 8,
                  out_ids, out_d2, (unsigned long long*)nullptr, st);
  else
    launch_search(X, ld, d, adj, deg, R, nav, n_nav, Q, ldq, nq, 0, qk, qls, ldo, lay, 8, out_ids,
                  out_d2, (unsigned long long*)nullptr, st);
}

void search_run(const float* X, const uint8_t* X8, int ld, int d, int64_t n, const int32_t* adj,
                const int32_t* deg, int R, const int32_t* nav, int n_nav, const float* Q,
                int ldq, int64_t nq, int k, int Ls, int32_t* out_ids, float* out_d2,
                cudaStream_t st, unsigned long long* work) {
  (void)n;
  if (nq == 0) return;
  SearchLayout lay;
  lay.Ls = Ls;
  lay.RP = std::max(32, next_pow2(R));
  lay.ld = ld;
  // 8 warps per block and a 1,024-entry visited cache: 24 warps per SM (the register
  // limit) keep more row gathers in flight than a larger cache would save.  A call that
  // counts the work takes a 16,384-entry cache instead, so that its distance count is
  // Alg. 1's (each node once) and not inflated by recomputations after cache evictions.
  lay.log2h = work ? 14 : 10;
  const int wpb = work ? 2 : 8;
  if (X8)
    launch_search(X8, ld, d, adj, deg, R, nav, n_nav, Q, ldq, nq, k, (const int32_t*)nullptr,
                  (const int32_t*)nullptr, k, lay, wpb, out_ids, out_d2, work, st);
  else
    launch_search(X, ld, d, adj, deg, R, nav, n_nav, Q, ldq, nq, k, (const int32_t*)nullptr,
                  (const int32_t*)nullptr, k, lay, wpb, out_ids, out_d2, work, st);
}

}  // namespace ssg
