// Streaming top-K selection helpers shared by the kNN kernels: per-row buffers of
// (distance, id) keys in global scratch, compacted by a warp-wide bitonic sort.
#pragma once

#include "common.cuh"

namespace ssg {

// Register bitonic sort of C keys held by a warp: element index e * 32 + lane.
template <int C>
__device__ __forceinline__ void warp_sort_regs(uint64_t (&v)[C / 32]) {
  constexpr int E = C / 32;
  const int lane = lane_id();
#pragma unroll
  for (int k = 2; k <= C; k <<= 1) {
#pragma unroll
    for (int j = k >> 1; j > 0; j >>= 1) {
      if (j >= 32) {
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const int p = e ^ (j >> 5);
          if (p > e) {
            const bool up = (((e << 5) | lane) & k) == 0;
            uint64_t a = v[e], b = v[p];
            if ((a > b) == up) {
              v[e] = b;
              v[p] = a;
            }
          }
        }
      } else {
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const int i = (e << 5) | lane;
          const bool up = (i & k) == 0;
          const bool lower = (lane & j) == 0;
          uint64_t o = __shfl_xor_sync(0xffffffffu, v[e], j);
          uint64_t mn = v[e] < o ? v[e] : o;
          uint64_t mx = v[e] < o ? o : v[e];
          v[e] = (lower == up) ? mn : mx;
        }
      }
    }
  }
}

// Compact one row's buffer: sort its cnt keys, keep the KS smallest at the front.
// Returns the new count; *tau receives the KS-th distance (or +inf while fewer).
// Not inlined: the unrolled sort is large and runs rarely, so one copy of it keeps the
// hot loops of the callers small in the instruction cache.
template <int C>
__device__ __noinline__ int compact_row(uint64_t* __restrict__ buf, int cnt, int KS,
                                        float* tau) {
  constexpr int E = C / 32;
  const int lane = lane_id();
  uint64_t v[E];
#pragma unroll
  for (int e = 0; e < E; ++e) {
    int i = (e << 5) | lane;
    v[e] = i < cnt ? buf[i] : KEY_NONE;
  }
  __syncwarp();
  warp_sort_regs<C>(v);
  const int keep = cnt < KS ? cnt : KS;
#pragma unroll
  for (int e = 0; e < E; ++e) {
    int i = (e << 5) | lane;
    if (i < keep) buf[i] = v[e];
  }
  uint64_t last = KEY_NONE;
  if (keep == KS) {
    const int ei = (KS - 1) >> 5;
#pragma unroll
    for (int e = 0; e < E; ++e)
      if (e == ei) last = v[e];
    last = __shfl_sync(0xffffffffu, last, (KS - 1) & 31);
  }
  __syncwarp();
  *tau = (keep == KS) ? key_dist(last) : __int_as_float(0x7f800000);
  return keep;
}

// Threshold step of a row's buffer without sorting: finds the KS-th smallest distance t
// by bisection over the 32-bit order keys (each step counts the entries at or below the
// midpoint), then keeps, unsorted and in their old relative order, every entry with a
// distance at most t (all ties at t stay).  The bisection stops early at a t with between
// KS and `good` entries at or below it (a looser t, still above every one of the KS
// smallest).  Returns the new count with *tau = t, or -1 with the buffer untouched when more
// than cap entries would stay.  Needs cnt >= KS.
template <int C>
__device__ __noinline__ int select_row(uint64_t* __restrict__ buf, int cnt, int KS, int good,
                                       int cap, float* tau) {
  constexpr int E = C / 32;
  const int lane = lane_id();
  uint32_t k[E];
  uint64_t v[E];
  uint32_t lo = 0xFFFFFFFFu, hi = 0u;
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int i = (e << 5) | lane;
    v[e] = i < cnt ? buf[i] : KEY_NONE;
    k[e] = (uint32_t)(v[e] >> 32);  // KEY_NONE: above every real key
    if (i < cnt) {
      lo = min(lo, k[e]);
      hi = max(hi, k[e]);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
  }
  // smallest t in [lo, hi] with at least KS keys <= t (hi qualifies: cnt >= KS)
  while (lo < hi) {
    const uint32_t mid = lo + ((hi - lo) >> 1);
    int c = 0;
#pragma unroll
    for (int e = 0; e < E; ++e) c += k[e] <= mid ? 1 : 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if (c >= KS) {
      hi = mid;
      if (c <= good) break;
    } else {
      lo = mid + 1;
    }
  }
  int n = 0;
#pragma unroll
  for (int e = 0; e < E; ++e) n += __popc(__ballot_sync(0xffffffffu, k[e] <= hi));
  if (n > cap) return -1;
  int base = 0;
  const unsigned lt = lanemask_lt();
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const unsigned b = __ballot_sync(0xffffffffu, k[e] <= hi);
    if (k[e] <= hi) buf[base + __popc(b & lt)] = v[e];
    base += __popc(b);
  }
  __syncwarp();
  *tau = order_bits_float(hi);
  return base;
}

}  // namespace ssg
