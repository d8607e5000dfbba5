// Warp-level building blocks shared by the pool, prune and reverse-merge kernels.
#pragma once

#include "common.cuh"

namespace ssg {

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// fp32 squared distance of two padded rows by a team of 8 lanes (float4 loads); every
// lane of the warp must call it (teams whose `valid` is false contribute nothing).
__device__ __forceinline__ float team8_dist(const float* __restrict__ a,
                                            const float* __restrict__ b, int ld4, int tl,
                                            bool valid) {
  float s = 0.f;
  if (valid) {
    const float4* a4 = (const float4*)a;
    const float4* b4 = (const float4*)b;
    for (int f = tl; f < ld4; f += 8) {
      float4 x = __ldg(a4 + f), y = __ldg(b4 + f);
      float u;
      u = x.x - y.x;
      s = fmaf(u, u, s);
      u = x.y - y.y;
      s = fmaf(u, u, s);
      u = x.z - y.z;
      s = fmaf(u, u, s);
      u = x.w - y.w;
      s = fmaf(u, u, s);
    }
  }
  s += __shfl_xor_sync(0xffffffffu, s, 1);
  s += __shfl_xor_sync(0xffffffffu, s, 2);
  s += __shfl_xor_sync(0xffffffffu, s, 4);
  return s;
}

// s + x with the rounding error of the sum added to c (Knuth's two-sum: s + x = t + err
// exactly).  The _rn intrinsics keep the compiler from fusing or reordering these steps.
__device__ __forceinline__ void two_sum_acc(float& s, float& c, float x) {
  const float t = __fadd_rn(s, x);
  const float z = __fsub_rn(t, s);
  c = __fadd_rn(c, __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(x, z)));
  s = t;
}

// Squared distances of a to two rows at once (b1 may be invalid) by a team of 8 lanes, with
// compensated sums: each rounded difference u is squared exactly (u*u = p + e with e from a
// fused multiply-add), the p are added with two-sum and every error term is kept in a
// second accumulator, also across the team's three shuffle levels.  The result lies within
// dist_rel_team8c(ld) of the exact squared distance (the rounding of the differences,
// then one rounding of the final sum), some forty times tighter than a plain fp32 sum of
// 960 terms, so that far fewer neighbouring distances need an fp64 re-sort.  On integer
// data below 2^24 every term and sum is exact and the value is that of a plain sum.
__device__ __forceinline__ void team8_dist2(const float* __restrict__ a,
                                            const float* __restrict__ b0,
                                            const float* __restrict__ b1, int ld4, int tl,
                                            bool v0, bool v1, float& r0, float& r1) {
  float s0 = 0.f, c0 = 0.f, s1 = 0.f, c1 = 0.f;
  if (v0) {
    const float4* a4 = (const float4*)a;
    const float4* p4 = (const float4*)b0;
    const float4* q4 = (const float4*)(v1 ? b1 : b0);
#pragma unroll 2
    for (int f = tl; f < ld4; f += 8) {
      const float4 x = __ldg(a4 + f), y = __ldg(p4 + f), z = __ldg(q4 + f);
      const float ux[4] = {__fsub_rn(x.x, y.x), __fsub_rn(x.y, y.y), __fsub_rn(x.z, y.z),
                           __fsub_rn(x.w, y.w)};
      const float uz[4] = {__fsub_rn(x.x, z.x), __fsub_rn(x.y, z.y), __fsub_rn(x.z, z.z),
                           __fsub_rn(x.w, z.w)};
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const float p = __fmul_rn(ux[e], ux[e]);
        c0 = __fadd_rn(c0, fmaf(ux[e], ux[e], -p));
        two_sum_acc(s0, c0, p);
        const float q = __fmul_rn(uz[e], uz[e]);
        c1 = __fadd_rn(c1, fmaf(uz[e], uz[e], -q));
        two_sum_acc(s1, c1, q);
      }
    }
    if (!v1) s1 = c1 = 0.f;
  }
#pragma unroll
  for (int o = 1; o < 8; o <<= 1) {
    const float os0 = __shfl_xor_sync(0xffffffffu, s0, o), oc0 = __shfl_xor_sync(0xffffffffu, c0, o);
    const float os1 = __shfl_xor_sync(0xffffffffu, s1, o), oc1 = __shfl_xor_sync(0xffffffffu, c1, o);
    c0 = __fadd_rn(c0, oc0);
    two_sum_acc(s0, c0, os0);
    c1 = __fadd_rn(c1, oc1);
    two_sum_acc(s1, c1, os1);
  }
  r0 = __fadd_rn(s0, c0);
  r1 = __fadd_rn(s1, c1);
}

// keys[t] holds a candidate id in its low 32 bits; replace the keys of steps t0 = first,
// first + stride, ... (eight keys t0 .. t0 + 7 per step, below m) by (fp32 d2(x_i,
// candidate), id).  xi points at node i's padded row.  Each team of 8 lanes takes two
// candidates per step (team8_dist2).
__device__ __forceinline__ void warp_fill_dist_keys_steps(uint64_t* keys, int m,
                                                          const float* __restrict__ X, int ld,
                                                          const float* __restrict__ xi,
                                                          int first, int stride) {
  const int lane = lane_id(), team = lane >> 3, tl = lane & 7;
  const int ld4 = ld >> 2;
  for (int t0 = first; t0 < m; t0 += stride) {
    const int t = t0 + team, t1 = t + 4;
    const bool v0 = t < m, v1 = t1 < m;
    const int32_t id0 = v0 ? key_id(keys[t]) : 0;
    const int32_t id1 = v1 ? key_id(keys[t1]) : 0;
    float d0, d1;
    team8_dist2(xi, X + (int64_t)id0 * ld, X + (int64_t)id1 * ld, ld4, tl, v0, v1, d0, d1);
    __syncwarp();
    if (tl == 0) {
      if (v0) keys[t] = make_key(d0, id0);
      if (v1) keys[t1] = make_key(d1, id1);
    }
  }
  __syncwarp();
}

// Every key in [0, m), by one warp.
__device__ __forceinline__ void warp_fill_dist_keys(uint64_t* keys, int m,
                                                    const float* __restrict__ X, int ld,
                                                    const float* __restrict__ xi) {
  warp_fill_dist_keys_steps(keys, m, X, ld, xi, 0, 8);
}

// Byte rows (integers 0..255, ld bytes per row, a multiple of 4): the squared distance of
// two rows by a team of 8 lanes in exact integer arithmetic, |a|^2 + |b|^2 - 2 a.b from
// byte dot products.  For such data every fp32 partial sum of team8_dist is an exact
// integer too, so the two functions return the same value.
__device__ __forceinline__ float team8_dist_u8(const uint8_t* __restrict__ a,
                                               const uint8_t* __restrict__ b, int ldw, int tl,
                                               bool valid) {
  unsigned aa = 0u, bb = 0u, ab = 0u;
  if (valid) {
    const unsigned int* a4 = (const unsigned int*)a;
    const unsigned int* b4 = (const unsigned int*)b;
    for (int f = tl; f < ldw; f += 8) {
      const unsigned x = __ldg(a4 + f), y = __ldg(b4 + f);
      aa = __dp4a(x, x, aa);
      bb = __dp4a(y, y, bb);
      ab = __dp4a(x, y, ab);
    }
  }
  int s = (int)aa + (int)bb - 2 * (int)ab;
  s += __shfl_xor_sync(0xffffffffu, s, 1);
  s += __shfl_xor_sync(0xffffffffu, s, 2);
  s += __shfl_xor_sync(0xffffffffu, s, 4);
  return (float)s;
}

// warp_fill_dist_keys from byte rows (X8 [n][ld] bytes, xi8 node i's row).  Rows of at
// most 128 bytes in 16-byte pieces (ld a multiple of 16) take one piece per team lane and
// four candidates per team at a time, so that a lane has four row loads in flight; other
// widths go a word at a time.  The sums are integers (exact in int32, and in fp32 below
// 2^24), so the order does not change the value.
__device__ __forceinline__ void warp_fill_dist_keys_u8(uint64_t* keys, int m,
                                                       const uint8_t* __restrict__ X8, int ld,
                                                       const uint8_t* __restrict__ xi8) {
  const int lane = lane_id(), team = lane >> 3, tl = lane & 7;
  if ((ld & 15) == 0 && ld <= 128) {
    const bool has = tl < (ld >> 4);
    const uint4 zero = make_uint4(0u, 0u, 0u, 0u);
    const uint4 a = has ? __ldg((const uint4*)xi8 + tl) : zero;
    const unsigned aa = __dp4a(a.w, a.w, __dp4a(a.z, a.z, __dp4a(a.y, a.y, __dp4a(a.x, a.x, 0u))));
    for (int t0 = 0; t0 < m; t0 += 16) {
      int id[4];
      bool val[4];
      uint4 y[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int t = t0 + u * 4 + team;
        val[u] = t < m;
        id[u] = val[u] ? key_id(keys[t]) : 0;
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
        y[u] = (val[u] && has) ? __ldg((const uint4*)(X8 + (int64_t)id[u] * ld) + tl) : zero;
      int s[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const unsigned bb = __dp4a(y[u].w, y[u].w, __dp4a(y[u].z, y[u].z,
                            __dp4a(y[u].y, y[u].y, __dp4a(y[u].x, y[u].x, 0u))));
        const unsigned ab = __dp4a(a.w, y[u].w, __dp4a(a.z, y[u].z,
                            __dp4a(a.y, y[u].y, __dp4a(a.x, y[u].x, 0u))));
        s[u] = (int)aa + (int)bb - 2 * (int)ab;
      }
#pragma unroll
      for (int o = 1; o < 8; o <<= 1)
#pragma unroll
        for (int u = 0; u < 4; ++u) s[u] += __shfl_xor_sync(0xffffffffu, s[u], o);
      __syncwarp();
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (val[u] && tl == 0) keys[t0 + u * 4 + team] = make_key((float)s[u], id[u]);
    }
    __syncwarp();
    return;
  }
  const int ldw = ld >> 2;
  for (int t0 = 0; t0 < m; t0 += 4) {
    const int t = t0 + team;
    const bool valid = t < m;
    const int32_t id = valid ? key_id(keys[t]) : 0;
    const float dd = team8_dist_u8(xi8, X8 + (int64_t)id * ld, ldw, tl, valid);
    __syncwarp();
    if (valid && tl == 0) keys[t] = make_key(dd, id);
  }
  __syncwarp();
}

// fp64 squared distance by all 32 lanes of a warp: lane l takes coordinates l, l + 32, ...;
// every term is rounded exactly as in dist2_f64 and only the order of the additions
// differs (a sum per lane, then a shuffle tree).  With non-negative terms both sums lie
// within (number of additions) x 2^-53 of the exact sum of the terms, so the two values
// differ by at most fp64_order_rel(d) / 2 relative; GB300's fp64 rate is low enough that
// the 32-fold shorter chain matters.  Every lane returns the same value.
__device__ __forceinline__ double warp_dist2_f64(const float* __restrict__ a,
                                                 const float* __restrict__ b, int d) {
  const int lane = lane_id();
  double s = 0.0;
  for (int t = lane; t < d; t += 32) {
    const double u = __dsub_rn((double)a[t], (double)b[t]);
    s = __dadd_rn(s, __dmul_rn(u, u));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s = __dadd_rn(s, __shfl_xor_sync(0xffffffffu, s, o));
  return s;
}

// Twice the largest relative gap between warp_dist2_f64 and dist2_f64 of the same pair.
__host__ __device__ inline double fp64_order_rel(int d) {
  return 2.0 * (d + (d + 31) / 32 + 6) * 1.1102230246251565e-16 * 1.01;
}

// Insertion sort of keys[s, e] (with their fp64 distances d64) by (d64, id); one lane.
__device__ __forceinline__ void sort_run_f64(uint64_t* keys, double* d64, int s, int e) {
  for (int t = s + 1; t <= e; ++t) {
    const uint64_t kk = keys[t];
    const double dv = d64[t];
    int u = t - 1;
    while (u >= s && (d64[u] > dv || (d64[u] == dv && (uint32_t)keys[u] > (uint32_t)kk))) {
      keys[u + 1] = keys[u];
      d64[u + 1] = d64[u];
      --u;
    }
    keys[u + 1] = kk;
    d64[u + 1] = dv;
  }
}

// keys[0, m) are sorted by their fp32 distances.  The fp32 value of a direct sum of d
// squared differences lies within a relative `rel` of the exact value, so two entries
// can be out of their true (d2, id) order only inside a run of neighbours whose fp32
// values are within that bound of each other.  Every such run that starts before
// `limit` is re-sorted by (fp64 d2, id): the warp computes each fp64 distance together
// (warp_dist2_f64), and where two of them are too close for that summation order to
// settle their order the way the coordinate-order sum does, those entries are re-taken in
// coordinate order (dist2_f64), so the order is always that of the coordinate-order fp64
// values.  d64 is scratch for m doubles.  Returns the number of runs re-sorted (in lane 0;
// the other lanes return 0, so a sum over lanes gives the total).
__device__ __forceinline__ int warp_fix_runs(uint64_t* keys, int m, int limit, double* d64,
                                             const float* __restrict__ X, int ld, int d,
                                             const float* __restrict__ xi, float rel) {
  const int lane = lane_id();
  auto close = [&](int p) -> bool {  // entries p and p + 1 are within the bound
    float a = key_dist(keys[p]), b = key_dist(keys[p + 1]);
    return (b - a) <= rel * (a + b);
  };
  const double trel = fp64_order_rel(d);
  int fixed = 0;
  const int smax = m - 1 < limit ? m - 1 : limit;
  for (int b0 = 0; b0 < smax; b0 += 32) {
    const int s = b0 + lane;
    const bool start = s < smax && close(s) && !(s > 0 && close(s - 1));
    unsigned bal = __ballot_sync(0xffffffffu, start);
    while (bal) {
      const int s0 = b0 + __ffs(bal) - 1;
      bal &= bal - 1;
      int e = s0 + 1;
      while (e + 1 < m && close(e)) ++e;
      for (int t = s0; t <= e; ++t) {
        const double v = warp_dist2_f64(xi, X + (int64_t)key_id(keys[t]) * ld, d);
        if (lane == 0) d64[t] = v;
      }
      __syncwarp();
      if (lane == 0) {
        sort_run_f64(keys, d64, s0, e);
        for (int t = s0; t < e;) {
          if (d64[t + 1] - d64[t] > trel * d64[t + 1]) {
            ++t;
            continue;
          }
          int u = t + 1;
          while (u < e && d64[u + 1] - d64[u] <= trel * d64[u + 1]) ++u;
          for (int q = t; q <= u; ++q) d64[q] = dist2_f64(xi, X + (int64_t)key_id(keys[q]) * ld, d);
          sort_run_f64(keys, d64, t, u);
          t = u + 1;
        }
        ++fixed;
      }
      __syncwarp();
    }
  }
  return fixed;
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(
                   (uint32_t)__cvta_generic_to_shared(smem)),
               "l"(gmem)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Candidate rows kept in flight by warp_prune_node (asynchronous copies into a ring).
constexpr int PRUNE_PREFETCH = 4;

// SSG prune of one node by one warp (Alg. 2 selection): cand[0, len) in (d2, id) order.
// Keeps cand[0]; keeps each later candidate unless its angle to a kept edge has
// cos > cos(alpha); stops at R kept.  The cosine comes from the centred dot products of
// the fp32 differences c - x_i held in shared memory (V: one row of D1 floats per kept
// edge plus one tentative row; D1 is a multiple of 4 with D1 % 32 == 4, so that the
// float4 reads of 8 lanes from 8 different rows fall in 8 different 16-byte bank groups).
// Candidate rows arrive through a ring of PRUNE_PREFETCH rows filled by cp.async ahead of
// use, so the global-memory latency of one row overlaps the work on earlier ones.
// A decision within `margin` of cos(alpha), or with a zero-length edge, is re-taken in
// fp64 from the original vectors; an fp64 cosine within `border` of cos(alpha) is counted
// in *nborder (the margin must cover border plus the fp32 error bound).  Rows are read
// up to d rounded to 4 (the padding of X is zero).  Shared memory per warp: prune_smem_floats(d, R) floats starting at V.
// Writes the kept ids to out[0, kept) (lane 0) and returns kept; *n64 += fp64 re-tests.
__device__ __forceinline__ int warp_prune_node(const float* __restrict__ X, int ld, int d,
                                               int64_t i, const int32_t* cand, int len, int R,
                                               float cosA32, double cosA64, float margin,
                                               float* V, int D1, float* xs, float* gkk,
                                               int32_t* out, unsigned long long* n64,
                                               double border, unsigned long long* nborder) {
  const int lane = lane_id();
  const float* xg = X + i * ld;
  const int d4 = (d + 3) & ~3;
  const int nq4 = d4 >> 2;
  float* ring = gkk + ((R + 1 + 3) & ~3);
  for (int t = lane; t < d4; t += 32) xs[t] = xg[t];
  auto prefetch = [&](int t) {
    if (t < len) {
      const float* src = X + (int64_t)cand[t] * ld;
      float* dst = ring + (t % PRUNE_PREFETCH) * D1;
      for (int f = lane; f < nq4; f += 32) cp_async16(dst + 4 * f, src + 4 * f);
    }
    cp_async_commit();
  };
  for (int t = 0; t < PRUNE_PREFETCH; ++t) prefetch(t);
  __syncwarp();
  int kept = 0;
  unsigned long long fp64_tests = 0, borderline = 0;
  for (int t = 0; t < len && kept < R; ++t) {
    const int32_t j = cand[t];
    cp_async_wait<PRUNE_PREFETCH - 1>();
    __syncwarp();
    const float* cs = ring + (t % PRUNE_PREFETCH) * D1;
    float* slot = V + kept * D1;
    float part = 0.f;
    for (int dd = lane; dd < d4; dd += 32) {
      float v = cs[dd] - xs[dd];
      slot[dd] = v;
      part = fmaf(v, v, part);
    }
    const float gjj = warp_sum(part);
    __syncwarp();
    prefetch(t + PRUNE_PREFETCH);
    bool definite = false;
    unsigned bmask = 0;
    for (int k = lane, r = 0; k < kept; k += 32, ++r) {
      const float4* vk = (const float4*)(V + k * D1);
      const float4* sl = (const float4*)slot;
      float g0 = 0.f, g1 = 0.f, g2 = 0.f, g3 = 0.f;
      for (int q = 0; q < nq4; ++q) {
        const float4 a = sl[q], b = vk[q];
        g0 = fmaf(a.x, b.x, g0);
        g1 = fmaf(a.y, b.y, g1);
        g2 = fmaf(a.z, b.z, g2);
        g3 = fmaf(a.w, b.w, g3);
      }
      const float g = (g0 + g1) + (g2 + g3);
      const float gk = gkk[k];
      if (gjj == 0.f || gk == 0.f) {
        bmask |= 1u << r;
      } else {
        const float c = g / (sqrtf(gjj) * sqrtf(gk));
        if (c > cosA32 + margin)
          definite = true;
        else if (c >= cosA32 - margin)
          bmask |= 1u << r;
      }
    }
    bool conflict = __any_sync(0xffffffffu, definite);
    if (!conflict && __any_sync(0xffffffffu, bmask != 0)) {
      bool c64 = false;
      const float* cj = X + (int64_t)j * ld;
      for (int r = 0; bmask >> r; ++r) {
        if (!((bmask >> r) & 1u)) continue;
        const int k = lane + 32 * r;
        const float* ck = X + (int64_t)out[k] * ld;
        const double gjk = centred_dot_f64(cj, ck, xg, d);
        const double g1 = centred_dot_f64(cj, cj, xg, d);
        const double g2 = centred_dot_f64(ck, ck, xg, d);
        const double c = cos_from_gram_f64(gjk, g1, g2);
        if (c > cosA64) c64 = true;
        if (fabs(c - cosA64) <= border) ++borderline;
        ++fp64_tests;
      }
      conflict = __any_sync(0xffffffffu, c64);
    }
    if (!conflict) {
      if (lane == 0) {
        out[kept] = j;
        gkk[kept] = gjj;
      }
      ++kept;
    }
    __syncwarp();
  }
  cp_async_wait<0>();
  __syncwarp();
  if (fp64_tests) atomicAdd(n64, fp64_tests);
  if (borderline) atomicAdd(nborder, borderline);
  return kept;
}

// Shared-memory layout of warp_prune_node for one warp, in floats: V [(R + 1) D1],
// xs [D1], gkk [R + 1 rounded to 4], ring [PRUNE_PREFETCH D1].
__host__ __device__ inline int prune_row_stride(int d) {
  int D1 = (d + 3) & ~3;
  while ((D1 & 31) != 4) D1 += 4;
  return D1;
}
__host__ __device__ inline size_t prune_smem_floats(int d, int R) {
  const int D1 = prune_row_stride(d);
  return (size_t)(R + 1) * D1 + (size_t)D1 + (size_t)((R + 1 + 3) & ~3) +
         (size_t)PRUNE_PREFETCH * D1;
}

// Rows too long for R + 1 of them to sit in shared memory (wide rows, e.g. d = 960):
// the kept centred vectors live in a global-memory slot of the warp, Vg [(R + 1)][d4],
// and each dot product is a warp-wide sum over coordinates (coalesced float4 reads).
// Same decisions and the same fp32 bound (any summation order), same fp64 re-test.
// Shared memory per warp: xs [d4], cs [d4], gkk [R + 1 rounded to 4].
__host__ __device__ inline size_t prune_wide_smem_floats(int d, int R) {
  const int d4 = (d + 3) & ~3;
  return 2 * (size_t)d4 + (size_t)((R + 1 + 3) & ~3);
}
__host__ __device__ inline bool prune_is_wide(int d, int R) {
  return prune_smem_floats(d, R) * sizeof(float) > 96 * 1024;
}

__device__ __forceinline__ int warp_prune_node_wide(const float* __restrict__ X, int ld, int d,
                                                    int64_t i, const int32_t* cand, int len,
                                                    int R, float cosA32, double cosA64,
                                                    float margin, float* __restrict__ Vg,
                                                    float* xs, float* cs, float* gkk,
                                                    int32_t* out, unsigned long long* n64,
                                                    double border,
                                                    unsigned long long* nborder) {
  const int lane = lane_id();
  const float* xg = X + i * ld;
  const int d4 = (d + 3) & ~3;
  const int nq4 = d4 >> 2;
  for (int t = lane; t < d4; t += 32) xs[t] = xg[t];
  __syncwarp();
  int kept = 0;
  unsigned long long fp64_tests = 0, borderline = 0;
  for (int t = 0; t < len && kept < R; ++t) {
    const int32_t j = cand[t];
    const float4* cj4 = (const float4*)(X + (int64_t)j * ld);
    float4* slot4 = (float4*)(Vg + (size_t)kept * d4);
    float part = 0.f;
    for (int f = lane; f < nq4; f += 32) {
      const float4 c = __ldg(cj4 + f);
      const float4 x = ((const float4*)xs)[f];
      const float4 v = make_float4(c.x - x.x, c.y - x.y, c.z - x.z, c.w - x.w);
      ((float4*)cs)[f] = v;
      slot4[f] = v;
      part = fmaf(v.x, v.x, part);
      part = fmaf(v.y, v.y, part);
      part = fmaf(v.z, v.z, part);
      part = fmaf(v.w, v.w, part);
    }
    const float gjj = warp_sum(part);
    __syncwarp();
    bool conflict = false;
    for (int k = 0; k < kept && !conflict; ++k) {
      const float4* vk = (const float4*)(Vg + (size_t)k * d4);
      float g = 0.f;
      for (int f = lane; f < nq4; f += 32) {
        const float4 a = ((const float4*)cs)[f], b = vk[f];
        g = fmaf(a.x, b.x, g);
        g = fmaf(a.y, b.y, g);
        g = fmaf(a.z, b.z, g);
        g = fmaf(a.w, b.w, g);
      }
      g = warp_sum(g);
      const float gk = gkk[k];
      bool near = gjj == 0.f || gk == 0.f;
      if (!near) {
        const float c = g / (sqrtf(gjj) * sqrtf(gk));
        if (c > cosA32 + margin)
          conflict = true;
        else if (c >= cosA32 - margin)
          near = true;
      }
      if (near) {
        // every lane takes the same fp64 decision from the same sequential sums
        const float* ck = X + (int64_t)out[k] * ld;
        const float* cjp = X + (int64_t)j * ld;
        const double gjk = centred_dot_f64(cjp, ck, xg, d);
        const double g1 = centred_dot_f64(cjp, cjp, xg, d);
        const double g2 = centred_dot_f64(ck, ck, xg, d);
        const double c = cos_from_gram_f64(gjk, g1, g2);
        conflict = c > cosA64;
        if (fabs(c - cosA64) <= border) ++borderline;
        ++fp64_tests;
      }
    }
    if (!conflict) {
      if (lane == 0) {
        out[kept] = j;
        gkk[kept] = gjj;
      }
      ++kept;
    }
    __syncwarp();
  }
  if (lane == 0 && fp64_tests) atomicAdd(n64, fp64_tests);
  if (lane == 0 && borderline) atomicAdd(nborder, borderline);
  return kept;
}

}  // namespace ssg
