// Exact kNN graph on the 5th-generation tensor cores (tcgen05, sm_103a) for integer data
// that bf16 holds exactly (|x| <= 256, and the bounds of DataInfo::exact).
//
// The GEMM is augmented so that the accumulator already holds what the threshold test
// needs: A = [x | 1 1 1 1 0..], B = [y | -p1 -p2 -p3 -p4 0..] with p1 + .. + p4 = |y|^2 / 2
// (bf16 parts of an integer or half-integer below 2^23), so acc = x.y - |y|^2 / 2 and
// d2 = |x|^2 - 2 acc.  Every product and partial sum is a multiple of 1/2 below 2^23 in
// magnitude (2 d max|x|^2 <= 2^24 for non-negative data, 4 d max|x|^2 <= 2^24 otherwise),
// so the accumulation is exact in fp32 whatever its order, and so is d2.
//
// Persistent kernel, one CTA per SM, 10 warps:
//   warp 0      TMA producer: the CTA's 256 query rows (A, resident per row block) and a
//               pipeline of 128-column base tiles (B), bf16 with 128-byte swizzle, plus the
//               16-element augmentation rows with 32-byte swizzle;
//   warp 1      allocates 512 TMEM columns and issues tcgen05.mma: for every B tile two
//               128x128 accumulators (the two 128-row halves of A) into one of NBUF = 2
//               TMEM buffers, so the epilogue drains one buffer while the MMAs fill the
//               other;
//   warps 2..9  epilogue, one thread per query row (TMEM lane): tcgen05.ld 64 columns at
//               a time, their largest accumulator against the row's threshold (a tree of
//               three-input maxes), and only where some lane passes, the passing values go
//               to the row's buffer in global scratch (L2); a warp compacts a full buffer
//               with a bisection or a register bitonic sort (top-KS, new threshold).  The
//               row's own column (self) takes one extra slot and is dropped at output.
// Columns are visited in BN-wide tiles, in id order or (large self-joins) nearest cluster
// first; in id order "d2 < threshold" also settles equal distances by id, otherwise ties
// are admitted and settled by the compaction.  (64-column tiles with four TMEM buffers and
// twice the TMA stages were measured 1.65x slower: the MMAs then take about as long per
// instruction while doing half the work.)
// Every wait on an mbarrier is bounded (about 2 s); a wait that runs out sets an error
// word, tells the other roles to stop, and the CTA releases its TMEM and exits.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include "common.cuh"
#include "knn.cuh"
#include "knn_select.cuh"
#include "tc_common.cuh"

namespace ssg {
namespace {

using namespace tc;

constexpr int BM = 256;               // query rows per CTA (two UMMA_M = 128 halves)
constexpr int BN = 128;               // base columns per pipeline stage (UMMA_N)
constexpr int API_TILE = 128;         // tile limits are given in 128-point tiles
constexpr int NBUF = 2;               // TMEM accumulator buffers
constexpr uint32_t IDESC_N = idesc_bf16(BN);
constexpr int EPI_WARPS = 8;
constexpr int THREADS = 64 + EPI_WARPS * 32;
constexpr int TMEM_COLS = 512;        // 2 buffers x 2 halves x 128 fp32 columns
constexpr int MAX_STAGES = 6;
constexpr int AUG = 16;               // augmentation K-step (bf16 elements)
constexpr int AUG_BYTES = AUG * 2;    // one augmentation row: 32 bytes
struct TcArgs {
  const float* a_norm;  // |x|^2 of the stored query rows (exact integers)
  int64_t na;           // query rows
  int64_t nb;           // base rows: stored column positions >= nb are padding
  int64_t ntiles;       // BN-column tiles of the base
  int64_t tstride;      // length of each cluster's tile list
  int64_t nwalk;        // tiles each block of rows visits (ntiles, or fewer for Alg. 4)
  int kchunks;          // padded d / 64
  int stages;
  int self;
  int KS, K;
  int trig;             // a row buffer holding more than trig keys is compacted (<= C - BN)
  uint64_t* rowbuf;
  int32_t* out_id;
  float* out_d2;
  int* err;
  const int32_t* perm;        // stored position -> original id (null: the identity)
  const int32_t* inv;         // original id -> stored position
  const int32_t* tile_order;  // per cluster, its first tstride tile indices (null: in order)
  const int32_t* rb_cluster;  // cluster of each block of BM stored query rows
  float* out_thresh;          // nullable: per output row, the KS-th smallest distance kept
                              // (or, with fewer kept, the final admission bound)
  const int32_t* qid;         // nullable: query row r is base row qid[r] (the self column);
                              // outputs then go to row r
  const float* tau_in;        // nullable: per stored row, an upper bound of its KS-th
                              // distance to start the streaming threshold from
  float tau_relax;            // tau_in is widened by (|tau_in| + |x|^2) tau_relax (0: exact)
  float* tau_out;             // thresh_only: per stored row, the KS-th distance of its walk
  int thresh_only;            // 1: no output rows, only tau_out
};

__device__ __forceinline__ float fmax3(float a, float b, float c) {
  float d;
  asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
  return d;
}

// Largest of 32 accumulators: a depth-4 tree of three-input maxes.
__device__ __forceinline__ float max32(const uint32_t (&v)[32]) {
  float a[11];
#pragma unroll
  for (int i = 0; i < 10; ++i)
    a[i] = fmax3(__uint_as_float(v[3 * i]), __uint_as_float(v[3 * i + 1]),
                 __uint_as_float(v[3 * i + 2]));
  a[10] = fmaxf(__uint_as_float(v[30]), __uint_as_float(v[31]));
  const float b0 = fmax3(a[0], a[1], a[2]), b1 = fmax3(a[3], a[4], a[5]);
  const float b2 = fmax3(a[6], a[7], a[8]), b3 = fmaxf(a[9], a[10]);
  return fmaxf(fmax3(b0, b1, b2), b3);
}

// Parks 32 accumulators in a thread's stash: float4 slots XOR-swizzled by sw = lane & 7,
// so 8 lanes store to 8 different bank groups.
__device__ __forceinline__ void stash32(float* st, int sw, const uint32_t (&v)[32]) {
#pragma unroll
  for (int k = 0; k < 8; ++k)
    *(float4*)(st + ((k ^ sw) << 2)) =
        make_float4(__uint_as_float(v[4 * k]), __uint_as_float(v[4 * k + 1]),
                    __uint_as_float(v[4 * k + 2]), __uint_as_float(v[4 * k + 3]));
}

// Appends the parked accumulators above ts to a row's buffer as (|x|^2 - 2 acc, stored
// position) keys; column e of the chunk is stored position jc + e (padding from nb on).
// Out of line: once the threshold has settled it runs for few chunks, and one copy keeps
// the scan loop small in the instruction cache.
__device__ __noinline__ int append_stash(const float* st, int sw, float ts, float nx, int32_t jc,
                                         int64_t nb, uint64_t* buf, int cnt) {
  uint32_t m = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const float4 q = *(const float4*)(st + ((k ^ sw) << 2));
    m |= ((q.x > ts ? 1u : 0u) | (q.y > ts ? 2u : 0u) | (q.z > ts ? 4u : 0u) |
          (q.w > ts ? 8u : 0u))
         << (4 * k);
  }
  while (m) {
    const int e = __ffs(m) - 1;
    m &= m - 1;
    const int32_t j = jc + e;
    if (j >= nb) break;  // padding columns come last within a chunk
    const float acc = st[(((e >> 2) ^ sw) << 2) | (e & 3)];
    buf[cnt++] = make_key(fmaf(-2.f, acc, nx), j);
  }
  return cnt;
}

// Maps the ids of a row's first cnt keys through map (stored position -> original id, or
// back), warp-wide; a sort then settles equal distances by original id.  Without a map
// nothing changes.
__device__ __forceinline__ void map_key_ids(uint64_t* buf, int cnt, const int32_t* __restrict__ map) {
  if (!map) return;
  __syncwarp();
  for (int i = lane_id(); i < cnt; i += 32) {
    const uint64_t k = buf[i];
    buf[i] = (k & 0xFFFFFFFF00000000ull) | (uint32_t)map[(uint32_t)k];
  }
  __syncwarp();
}

// Cuts back the row buffers of a warp's 32 rows that the next tile could overflow (count
// above trig) to the entries at or below their KS-th smallest distance (a full sort only if
// ties would keep too many).  wbuf: the buffer of lane 0's row; lane l's is wbuf + l C.
template <int C>
__device__ __forceinline__ void compact_needed(const TcArgs& p, uint64_t* wbuf, int& cnt,
                                               float& tau) {
  unsigned need = __ballot_sync(0xffffffffu, cnt > p.trig);
  while (need) {
    const int l = __ffs(need) - 1;
    need &= need - 1;
    uint64_t* lb = wbuf + (size_t)l * C;
    const int cl = __shfl_sync(0xffffffffu, cnt, l);
    float t2;
    int c2 = select_row<C>(lb, cl, p.KS, (p.KS + p.trig) / 2, p.trig, &t2);
    if (c2 < 0) {
      // too many ties at the threshold: a sort settles them by original id, and the
      // kept keys go back to stored positions like the ones still to come
      map_key_ids(lb, cl, p.perm);
      c2 = compact_row<C>(lb, cl, p.KS, &t2);
      map_key_ids(lb, c2, p.inv);
    }
    if (lane_id() == l) {
      cnt = c2;
      tau = t2;
    }
  }
}

// Final compaction of a warp's 32 rows (stored rows r0 .. r0 + 31, buffers as for
// compact_needed), then their output: the first K keys after dropping the row itself (or,
// thresh_only, the KS-th distance), and the threshold when asked.
template <int C>
__device__ __forceinline__ void finish_rows(const TcArgs& p, uint64_t* wbuf, int64_t r0, int cnt,
                                            float tau) {
  const int lane = lane_id();
  const float INF = __int_as_float(0x7f800000);
  for (int l = 0; l < 32; ++l) {
    const int64_t r = r0 + l;
    uint64_t* lb = wbuf + (size_t)l * C;
    float t2;
    int cl = __shfl_sync(0xffffffffu, cnt, l);
    if (cl > 256 && cl > p.KS) {
      const int c1 = select_row<C>(lb, cl, p.KS, 256, 256, &t2);
      if (c1 >= 0) cl = c1;
    }
    if (p.thresh_only) {
      // the KS-th distance of this walk (the order of equal distances is irrelevant)
      if (cl <= 256)
        compact_row<256>(lb, cl, p.KS, &t2);
      else
        compact_row<C>(lb, cl, p.KS, &t2);
      if (r < p.na && lane == 0) p.tau_out[r] = t2;
      __syncwarp();
      continue;
    }
    map_key_ids(lb, cl, p.perm);
    const int c2 = cl <= 256 ? compact_row<256>(lb, cl, p.KS, &t2)
                             : compact_row<C>(lb, cl, p.KS, &t2);
    // the row's last admission bound: with fewer than KS kept (a bound from tau_in that
    // few columns meet) every column not kept lies above it
    const float taul = __shfl_sync(0xffffffffu, tau, l);
    if (r >= p.na) continue;
    // the output row, and the base id of the row itself (the self column)
    const int64_t ro = p.qid ? r : (p.perm ? (int64_t)p.perm[r] : r);
    const int32_t sid = p.qid ? p.qid[r] : (int32_t)ro;
    if (p.out_thresh && lane == 0) p.out_thresh[ro] = fminf(t2, taul);
    int selfpos = c2;
    if (p.self) {
      for (int e0 = 0; e0 < c2; e0 += 32) {
        const int e = e0 + lane;
        const unsigned m = __ballot_sync(0xffffffffu, e < c2 && key_id(lb[e]) == sid);
        if (m) {
          selfpos = e0 + __ffs(m) - 1;
          break;
        }
      }
    }
    for (int t = lane; t < p.K; t += 32) {
      const int src = t < selfpos ? t : t + 1;
      const uint64_t key = src < c2 ? lb[src] : KEY_NONE;
      p.out_id[ro * p.K + t] = key == KEY_NONE ? -1 : key_id(key);
      p.out_d2[ro * p.K + t] = key == KEY_NONE ? INF : key_dist(key);
    }
    __syncwarp();
  }
}

template <int C>
__global__ void __launch_bounds__(THREADS, 1)
k_knn_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
         const __grid_constant__ CUtensorMap tmAaug, const __grid_constant__ CUtensorMap tmBaug,
         TcArgs p) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* sm = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int S = p.stages;
  const uint32_t a_main = (uint32_t)p.kchunks * BM * 128;
  const uint32_t a_bytes = a_main + BM * AUG_BYTES;
  const uint32_t b_main = (uint32_t)p.kchunks * BN * 128;
  const uint32_t b_bytes = b_main + BN * AUG_BYTES;
  unsigned char* sA = sm;
  unsigned char* sB = sA + a_bytes;
  float* stash = (float*)(sB + (size_t)S * b_bytes);  // 32 floats per epilogue thread
  uint64_t* bars = (uint64_t*)(stash + EPI_WARPS * 32 * 32);
  uint64_t* a_full = bars;
  uint64_t* a_empty = bars + 1;
  uint64_t* b_full = bars + 2;
  uint64_t* b_empty = b_full + MAX_STAGES;
  uint64_t* t_full = b_empty + MAX_STAGES;
  uint64_t* t_empty = t_full + NBUF;
  uint32_t* tmem_slot = (uint32_t*)(t_empty + NBUF);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = lane_id();
  if (threadIdx.x == 0) {
    mbar_init(smem_u32(a_full), 1);
    mbar_init(smem_u32(a_empty), 1);
    for (int s = 0; s < S; ++s) {
      mbar_init(smem_u32(b_full + s), 1);
      mbar_init(smem_u32(b_empty + s), 1);
    }
    for (int b = 0; b < NBUF; ++b) {
      mbar_init(smem_u32(t_full + b), 1);
      mbar_init(smem_u32(t_empty + b), EPI_WARPS);
    }
    *abort_flag = 0;
    fence_barrier_init();
  }
  if (warp == 1) {
    tmem_alloc(smem_u32(tmem_slot), TMEM_COLS);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  const int64_t nrb = (p.na + BM - 1) / BM;
  const int64_t nwalk = p.nwalk;

  if (warp == 0) {
    // ---------------- TMA producer ----------------
    if (lane == 0) {
      int s = 0;         // B stage of the next tile
      uint32_t ph = 0;   // and the parity of its use
      int rbi = 0;
      bool ok = true;
      for (int64_t rb = blockIdx.x; rb < nrb && ok; rb += gridDim.x, ++rbi) {
        ok = mbar_wait(smem_u32(a_empty), (rbi & 1) ^ 1, abort_flag);
        if (!ok) break;
        mbar_expect_tx(smem_u32(a_full), a_bytes);
        for (int kc = 0; kc < p.kchunks; ++kc)
          tma_load_2d(smem_u32(sA + (size_t)kc * BM * 128), &tmA, smem_u32(a_full), kc * 64,
                      (int)(rb * BM));
        tma_load_2d(smem_u32(sA + a_main), &tmAaug, smem_u32(a_full), 0, 0);
        const int32_t* tl = p.tile_order ? p.tile_order + (int64_t)p.rb_cluster[rb] * p.tstride : nullptr;
        int64_t tn = tl ? tl[0] : 0;  // tile index, read one tile ahead
        for (int64_t i = 0; i < nwalk; ++i) {
          const int j0 = (int)(tn * BN);
          if (i + 1 < nwalk) tn = tl ? tl[i + 1] : i + 1;
          ok = mbar_wait(smem_u32(b_empty + s), ph ^ 1, abort_flag);
          if (!ok) break;
          mbar_expect_tx(smem_u32(b_full + s), b_bytes);
          unsigned char* dst = sB + (size_t)s * b_bytes;
          for (int kc = 0; kc < p.kchunks; ++kc)
            tma_load_2d(smem_u32(dst + (size_t)kc * BN * 128), &tmB, smem_u32(b_full + s), kc * 64,
                        j0);
          tma_load_2d(smem_u32(dst + b_main), &tmBaug, smem_u32(b_full + s), 0, j0);
          if (++s == S) {
            s = 0;
            ph ^= 1;
          }
        }
      }
      if (!ok) {
        atomicOr(p.err, 1);
        *abort_flag = 1;
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      int64_t it = 0;
      int s = 0;
      uint32_t ph = 0;
      int rbi = 0;
      bool ok = true;
      const uint64_t adesc0 = sdesc_sw128(smem_u32(sA));
      const uint64_t adesc_aug = sdesc_sw32(smem_u32(sA + a_main));
      for (int64_t rb = blockIdx.x; rb < nrb && ok; rb += gridDim.x, ++rbi) {
        ok = mbar_wait(smem_u32(a_full), rbi & 1, abort_flag);
        if (!ok) break;
        for (int64_t ct = 0; ct < nwalk; ++ct, ++it) {
          const int b = (int)(it % NBUF);
          const uint32_t tph = (uint32_t)((it / NBUF) & 1);
          ok = mbar_wait(smem_u32(t_empty + b), tph ^ 1, abort_flag) &&
               mbar_wait(smem_u32(b_full + s), ph, abort_flag);
          if (!ok) break;
          tc_fence_after();
          // descriptors of the K-steps: the 14-bit start-address field (bytes / 16) of the
          // base descriptor plus the step's offset; shared addresses stay below 256 KB, so
          // the sum never carries out of the field
          const uint32_t bst = smem_u32(sB + (size_t)s * b_bytes);
          const uint64_t bdesc0 = sdesc_sw128(bst);
          const uint64_t bdesc_aug = sdesc_sw32(bst + b_main);
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const uint32_t d_tmem = tmem_base + (uint32_t)((b * 2 + h) * BN);
            for (int kc = 0; kc < p.kchunks; ++kc) {
#pragma unroll
              for (int kk = 0; kk < 4; ++kk) {
                const uint64_t ad =
                    adesc0 + (uint64_t)((kc * BM * 128 + h * 128 * 128 + kk * 32) >> 4);
                const uint64_t bd = bdesc0 + (uint64_t)((kc * BN * 128 + kk * 32) >> 4);
                umma_bf16_id(d_tmem, ad, bd, IDESC_N, (kc | kk) ? 1u : 0u);
              }
            }
            umma_bf16_id(d_tmem, adesc_aug + (uint64_t)((h * 128 * AUG_BYTES) >> 4), bdesc_aug,
                         IDESC_N, 1u);
          }
          umma_commit(smem_u32(b_empty + s));
          umma_commit(smem_u32(t_full + b));
          if (++s == S) {
            s = 0;
            ph ^= 1;
          }
        }
        if (ok) umma_commit(smem_u32(a_empty));
      }
      if (!ok) {
        atomicOr(p.err, 2);
        *abort_flag = 1;
      }
    }
    __syncwarp();
  } else {
    // ---------------- epilogue: one thread per query row ----------------
    const int ew = warp - 2;
    const int h = ew >> 2;          // which 128-row half
    const int q = warp & 3;         // TMEM lane quadrant this warp may access
    const int row_in_cta = h * 128 + q * 32 + lane;
    float* st = stash + (size_t)(ew * 32 + lane) * 32;
    const int sw = lane & 7;
    const bool strict = p.tile_order == nullptr;
    int64_t it = 0;
    bool ok = true;
    const float INF = __int_as_float(0x7f800000);
    for (int64_t rb = blockIdx.x; rb < nrb && ok; rb += gridDim.x) {
      const int64_t row = rb * BM + row_in_cta;
      const float nx = row < p.na ? p.a_norm[row] : 0.f;
      float tau = INF;
      if (p.tau_in && row < p.na) {
        // a bound from a shorter walk over the same columns: every column at or below it
        // is admitted, so the KS smallest are all kept
        const float t0 = p.tau_in[row];
        tau = t0 + (fabsf(t0) + fabsf(nx)) * p.tau_relax;
      }
      int cnt = 0;
      uint64_t* buf = p.rowbuf + ((size_t)blockIdx.x * BM + row_in_cta) * C;
      const int32_t* tl = p.tile_order ? p.tile_order + (int64_t)p.rb_cluster[rb] * p.tstride : nullptr;
      int64_t tn = tl ? tl[0] : 0;  // tile index, read one tile ahead
      for (int64_t i = 0; i < nwalk; ++i, ++it) {
        const int32_t j0 = (int32_t)(tn * BN);
        if (i + 1 < nwalk) tn = tl ? tl[i + 1] : i + 1;
        const int b = (int)(it % NBUF);
        const uint32_t tph = (uint32_t)((it / NBUF) & 1);
        ok = mbar_wait(smem_u32(t_full + b), tph, abort_flag);
        if (!__all_sync(0xffffffffu, ok)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t taddr = tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)((b * 2 + h) * BN);
        // d2 < tau  <=>  acc > (|x|^2 - tau) / 2 (exact); ties admitted (ts just below the
        // bound) unless the columns arrive in id order.  tau = inf gives ts = -inf.
        const float thr = 0.5f * (nx - tau);
        const float ts = strict ? thr : nextafterf(thr, -INF);
        auto scan64 = [&](const uint32_t(&va)[32], const uint32_t(&vb)[32], int c) {
          const bool pa = max32(va) > ts;
          const bool pb = max32(vb) > ts;
          if (__any_sync(0xffffffffu, pa || pb)) {
            if (pa) {
              stash32(st, sw, va);
              cnt = append_stash(st, sw, ts, nx, j0 + c * 32, p.nb, buf, cnt);
            }
            if (pb) {
              stash32(st, sw, vb);
              cnt = append_stash(st, sw, ts, nx, j0 + c * 32 + 32, p.nb, buf, cnt);
            }
            __syncwarp();
          }
        };
        // two passes of 64 columns; the accumulator buffer goes back to the MMA warp as soon
        // as the second pass is in registers
        uint32_t v0[32], v1[32];
#pragma unroll 1
        for (int c = 0; c < BN / 32; c += 2) {
          tmem_ld32(taddr + (uint32_t)c * 32, v0);
          tmem_ld32(taddr + (uint32_t)c * 32 + 32, v1);
          tmem_wait_ld(v0);
          tmem_dep(v1);
          if (c + 2 == BN / 32) {
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(t_empty + b));
          }
          scan64(v0, v1, c);
        }
        // a buffer that the next tile could overflow drops to the entries at or below its
        // KS-th smallest distance
        compact_needed<C>(p, p.rowbuf + ((size_t)blockIdx.x * BM + h * 128 + q * 32) * C, cnt,
                          tau);
      }
      if (!ok) break;
      finish_rows<C>(p, p.rowbuf + ((size_t)blockIdx.x * BM + h * 128 + q * 32) * C,
                     rb * BM + h * 128 + q * 32, cnt, tau);
    }
    if (!ok && lane == 0) {
      atomicOr(p.err, 4);
      *abort_flag = 1;
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem_base, TMEM_COLS);
  }
}

// ---------------------------------------------------------------------------------------
// Rows wider than the resident pipeline holds (d > 128): the query rows are streamed with
// the base tiles, 64 values at a time.  A CTA owns BMW = 128 query rows and walks
// BNW = 256-column tiles; per tile and 64-wide chunk one stage holds the A chunk (16 KB)
// and the B chunk (32 KB), and the MMA thread issues four 128 x 256 x 16 MMAs into one of
// two 256-column TMEM buffers (N = 256: the wider instruction does twice the work of
// N = 128 for about the same issue time).  The augmentation step (-|y|^2/2 folded into the
// accumulator) comes last in each tile from a two-slot ring.  Four epilogue warps, one per
// TMEM lane quadrant, scan the tile's 256 columns of their 32 rows as the resident kernel
// does; a tile's MMAs take long enough that the handoff between the two buffers is cheap.
// ---------------------------------------------------------------------------------------
constexpr int BMW = 128;
constexpr int BNW = 256;
constexpr int EPI_W = 4;
constexpr int THREADS_W = 64 + EPI_W * 32;
constexpr int STAGES_W = 3;
constexpr uint32_t IDESC_W = idesc_bf16(BNW);
constexpr uint32_t A_CHUNK_W = BMW * 128;   // 16 KB
constexpr uint32_t B_CHUNK_W = BNW * 128;   // 32 KB
constexpr uint32_t STAGE_W = A_CHUNK_W + B_CHUNK_W;

size_t tcw_smem_bytes() {
  return 1024 + (size_t)STAGES_W * STAGE_W + 2 * (BNW * AUG_BYTES) + BMW * AUG_BYTES +
         EPI_W * 32 * 32 * sizeof(float) + sizeof(uint64_t) * (1 + 2 * STAGES_W + 4 + 4) + 16;
}

template <int C>
__global__ void __launch_bounds__(THREADS_W, 1)
k_knn_tc_wide(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
              const __grid_constant__ CUtensorMap tmAaug, const __grid_constant__ CUtensorMap tmBaug,
              TcArgs p) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* sm = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* sS = sm;                                        // STAGES_W x [A chunk | B chunk]
  unsigned char* sBaug = sS + (size_t)STAGES_W * STAGE_W;        // 2 x BNW rows x 32 B
  unsigned char* sAaug = sBaug + 2 * BNW * AUG_BYTES;            // BMW rows x 32 B
  float* stash = (float*)(sAaug + BMW * AUG_BYTES);              // 32 floats per epilogue thread
  uint64_t* bars = (uint64_t*)(stash + EPI_W * 32 * 32);
  uint64_t* aa_full = bars;
  uint64_t* s_full = bars + 1;
  uint64_t* s_empty = s_full + STAGES_W;
  uint64_t* g_full = s_empty + STAGES_W;   // augmentation ring
  uint64_t* g_empty = g_full + 2;
  uint64_t* t_full = g_empty + 2;
  uint64_t* t_empty = t_full + 2;
  uint32_t* tmem_slot = (uint32_t*)(t_empty + 2);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = lane_id();
  const int kc_n = p.kchunks;
  if (threadIdx.x == 0) {
    mbar_init(smem_u32(aa_full), 1);
    for (int s = 0; s < STAGES_W; ++s) {
      mbar_init(smem_u32(s_full + s), 1);
      mbar_init(smem_u32(s_empty + s), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(smem_u32(g_full + b), 1);
      mbar_init(smem_u32(g_empty + b), 1);
      mbar_init(smem_u32(t_full + b), 1);
      mbar_init(smem_u32(t_empty + b), EPI_W);
    }
    *abort_flag = 0;
    fence_barrier_init();
  }
  if (warp == 1) {
    tmem_alloc(smem_u32(tmem_slot), TMEM_COLS);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  const int64_t nrb = (p.na + BMW - 1) / BMW;
  const int64_t nwalk = p.nwalk;

  if (warp == 0) {
    // ---------------- TMA producer ----------------
    if (lane == 0) {
      bool ok = true;
      mbar_expect_tx(smem_u32(aa_full), BMW * AUG_BYTES);
      tma_load_2d(smem_u32(sAaug), &tmAaug, smem_u32(aa_full), 0, 0);
      int s = 0;
      uint32_t ph = 0;
      int64_t t = 0;  // tiles so far (augmentation slot t & 1)
      for (int64_t rb = blockIdx.x; rb < nrb && ok; rb += gridDim.x) {
        const int32_t* tl = p.tile_order ? p.tile_order + (int64_t)p.rb_cluster[rb] * p.tstride : nullptr;
        int64_t tn = tl ? tl[0] : 0;
        for (int64_t i = 0; i < nwalk && ok; ++i, ++t) {
          const int j0 = (int)(tn * BNW);
          if (i + 1 < nwalk) tn = tl ? tl[i + 1] : i + 1;
          const int g = (int)(t & 1);
          ok = mbar_wait(smem_u32(g_empty + g), (uint32_t)(((t >> 1) & 1) ^ 1), abort_flag);
          if (!ok) break;
          mbar_expect_tx(smem_u32(g_full + g), BNW * AUG_BYTES);
          tma_load_2d(smem_u32(sBaug + (size_t)g * BNW * AUG_BYTES), &tmBaug, smem_u32(g_full + g), 0,
                      j0);
          for (int kc = 0; kc < kc_n; ++kc) {
            ok = mbar_wait(smem_u32(s_empty + s), ph ^ 1, abort_flag);
            if (!ok) break;
            mbar_expect_tx(smem_u32(s_full + s), STAGE_W);
            unsigned char* dst = sS + (size_t)s * STAGE_W;
            tma_load_2d(smem_u32(dst), &tmA, smem_u32(s_full + s), kc * 64, (int)(rb * BMW));
            tma_load_2d(smem_u32(dst + A_CHUNK_W), &tmB, smem_u32(s_full + s), kc * 64, j0);
            if (++s == STAGES_W) {
              s = 0;
              ph ^= 1;
            }
          }
        }
      }
      if (!ok) {
        atomicOr(p.err, 1);
        *abort_flag = 1;
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      bool ok = mbar_wait(smem_u32(aa_full), 0, abort_flag);
      int s = 0;
      uint32_t ph = 0;
      int64_t t = 0;
      const uint64_t adesc_aug = sdesc_sw32(smem_u32(sAaug));
      for (int64_t rb = blockIdx.x; rb < nrb && ok; rb += gridDim.x) {
        for (int64_t i = 0; i < nwalk && ok; ++i, ++t) {
          const int b = (int)(t & 1);
          const uint32_t tph = (uint32_t)((t >> 1) & 1);
          ok = mbar_wait(smem_u32(t_empty + b), tph ^ 1, abort_flag);
          if (!ok) break;
          tc_fence_after();
          const uint32_t d_tmem = tmem_base + (uint32_t)(b * BNW);
          for (int kc = 0; kc < kc_n; ++kc) {
            ok = mbar_wait(smem_u32(s_full + s), ph, abort_flag);
            if (!ok) break;
            tc_fence_after();
            const uint32_t sa = smem_u32(sS + (size_t)s * STAGE_W);
            const uint64_t ad0 = sdesc_sw128(sa), bd0 = sdesc_sw128(sa + A_CHUNK_W);
#pragma unroll
            for (int kk = 0; kk < 4; ++kk)
              umma_bf16_id(d_tmem, ad0 + (uint64_t)((kk * 32) >> 4), bd0 + (uint64_t)((kk * 32) >> 4),
                           IDESC_W, (kc | kk) ? 1u : 0u);
            umma_commit(smem_u32(s_empty + s));
            if (++s == STAGES_W) {
              s = 0;
              ph ^= 1;
            }
          }
          if (!ok) break;
          const int g = (int)(t & 1);
          ok = mbar_wait(smem_u32(g_full + g), (uint32_t)((t >> 1) & 1), abort_flag);
          if (!ok) break;
          tc_fence_after();
          umma_bf16_id(d_tmem, adesc_aug,
                       sdesc_sw32(smem_u32(sBaug + (size_t)g * BNW * AUG_BYTES)), IDESC_W, 1u);
          umma_commit(smem_u32(g_empty + g));
          umma_commit(smem_u32(t_full + b));
        }
      }
      if (!ok) {
        atomicOr(p.err, 2);
        *abort_flag = 1;
      }
    }
    __syncwarp();
  } else {
    // ---------------- epilogue: one thread per query row ----------------
    const int ew = warp - 2;
    const int q = warp & 3;  // TMEM lane quadrant this warp may access
    const int row_in_cta = q * 32 + lane;
    float* st = stash + (size_t)(ew * 32 + lane) * 32;
    const int sw = lane & 7;
    const bool strict = p.tile_order == nullptr;
    int64_t t = 0;
    bool ok = true;
    const float INF = __int_as_float(0x7f800000);
    for (int64_t rb = blockIdx.x; rb < nrb && ok; rb += gridDim.x) {
      const int64_t row = rb * BMW + row_in_cta;
      const float nx = row < p.na ? p.a_norm[row] : 0.f;
      float tau = INF;
      if (p.tau_in && row < p.na) {
        const float t0 = p.tau_in[row];
        tau = t0 + (fabsf(t0) + fabsf(nx)) * p.tau_relax;
      }
      int cnt = 0;
      uint64_t* wbuf = p.rowbuf + ((size_t)blockIdx.x * BMW + q * 32) * C;
      uint64_t* buf = wbuf + (size_t)lane * C;
      const int32_t* tl = p.tile_order ? p.tile_order + (int64_t)p.rb_cluster[rb] * p.tstride : nullptr;
      int64_t tn = tl ? tl[0] : 0;
      for (int64_t i = 0; i < nwalk; ++i, ++t) {
        const int32_t j0 = (int32_t)(tn * BNW);
        if (i + 1 < nwalk) tn = tl ? tl[i + 1] : i + 1;
        const int b = (int)(t & 1);
        ok = mbar_wait(smem_u32(t_full + b), (uint32_t)((t >> 1) & 1), abort_flag);
        if (!__all_sync(0xffffffffu, ok)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t taddr = tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(b * BNW);
        const float thr = 0.5f * (nx - tau);
        const float ts = strict ? thr : nextafterf(thr, -INF);
        uint32_t v0[32], v1[32];
#pragma unroll 1
        for (int c = 0; c < BNW / 32; c += 2) {
          tmem_ld32(taddr + (uint32_t)c * 32, v0);
          tmem_ld32(taddr + (uint32_t)c * 32 + 32, v1);
          tmem_wait_ld(v0);
          tmem_dep(v1);
          if (c + 2 == BNW / 32) {
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(t_empty + b));
          }
          const bool pa = max32(v0) > ts;
          const bool pb = max32(v1) > ts;
          if (__any_sync(0xffffffffu, pa || pb)) {
            if (pa) {
              stash32(st, sw, v0);
              cnt = append_stash(st, sw, ts, nx, j0 + c * 32, p.nb, buf, cnt);
            }
            if (pb) {
              stash32(st, sw, v1);
              cnt = append_stash(st, sw, ts, nx, j0 + c * 32 + 32, p.nb, buf, cnt);
            }
            __syncwarp();
          }
        }
        compact_needed<C>(p, wbuf, cnt, tau);
      }
      if (!ok) break;
      finish_rows<C>(p, wbuf, rb * BMW + q * 32, cnt, tau);
    }
    if (!ok && lane == 0) {
      atomicOr(p.err, 4);
      *abort_flag = 1;
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem_base, TMEM_COLS);
  }
}

// bf16 copy with rows padded to dp; with perm, stored row r holds row perm[r] (and its norm);
// with mu, the rows are centred first (x - mu rounded to fp32, then to bf16).
// Rows of width dp (pairs = 0) or of three parts of width dp (pairs = 1: [hi | lo | hi],
// pairs = 2: [lo | hi | hi], hi = bf16(v), lo = bf16(v - hi), v the centred value), so
// that the accumulator takes the small products hi.lo and lo.hi before hi.hi.
__global__ void k_to_bf16(const float* __restrict__ X, int64_t n, int d, int ld,
                          __nv_bfloat16* __restrict__ Y, int dp, const int32_t* __restrict__ perm,
                          const float* __restrict__ norm_in, float* __restrict__ norm_out,
                          const float* __restrict__ mu, int pairs) {
  const int w = pairs ? 3 * dp : dp;
  const int64_t total = n * (int64_t)w;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / w;
    const int cw = (int)(i - r * w);
    const int part = cw / dp, c = cw - part * dp;
    const int64_t src = perm ? (int64_t)perm[r] : r;
    float v = c < d ? X[src * ld + c] : 0.f;
    if (mu && c < d) v = __fsub_rn(v, mu[c]);
    const __nv_bfloat16 hi = __float2bfloat16_rn(v);
    const bool low = (pairs == 1 && part == 1) || (pairs == 2 && part == 0);
    Y[i] = low ? __float2bfloat16_rn(__fsub_rn(v, __bfloat162float(hi))) : hi;
    if (norm_out && cw == 0) norm_out[r] = norm_in[src];
  }
}

// Augmentation rows of the base: -|y|^2 / 2 as four bf16 parts (each the bf16 rounding of
// what the previous ones leave), then zeros.  err is set if a row's parts do not add up
// to the value exactly.
__global__ void k_aug_rows(const float* __restrict__ norm, int64_t n, __nv_bfloat16* __restrict__ aug,
                           int* __restrict__ err, int approx) {
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n;
       r += (int64_t)gridDim.x * blockDim.x) {
    float rest = -0.5f * norm[r];
    __nv_bfloat16 part[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      part[k] = __float2bfloat16_rn(rest);
      rest -= __bfloat162float(part[k]);
    }
    if (rest != 0.f && !approx) atomicOr(err, 1);
    __nv_bfloat16* o = aug + r * AUG;
#pragma unroll
    for (int k = 0; k < AUG; ++k) o[k] = k < 4 ? part[k] : __float2bfloat16_rn(0.f);
  }
}

// Augmentation rows of the queries: four ones, then zeros (BM identical rows).
__global__ void k_aug_ones(__nv_bfloat16* __restrict__ aug) {
  for (int i = threadIdx.x; i < BM * AUG; i += blockDim.x)
    aug[i] = __float2bfloat16_rn((i % AUG) < 4 ? 1.f : 0.f);
}

size_t tc_smem_bytes(int kchunks, int stages) {
  return 1024 + (size_t)kchunks * BM * 128 + BM * AUG_BYTES +
         (size_t)stages * (kchunks * BN * 128 + BN * AUG_BYTES) +
         EPI_WARPS * 32 * 32 * sizeof(float) + sizeof(uint64_t) * (2 + 2 * MAX_STAGES + 2 * NBUF) +
         16;
}

struct TcMaps {
  CUtensorMap a, b, a_aug, b_aug;
};

template <int C>
void launch_tc(const TcMaps& m, TcArgs& a, int grid, size_t smem, cudaStream_t st, bool wide) {
  if (wide) {
    ensure_smem((const void*)k_knn_tc_wide<C>, smem);
    SSG_LAUNCH(k_knn_tc_wide<C>, grid, THREADS_W, smem, st, m.a, m.b, m.a_aug, m.b_aug, a);
  } else {
    ensure_smem((const void*)k_knn_tc<C>, smem);
    SSG_LAUNCH(k_knn_tc<C>, grid, THREADS, smem, st, m.a, m.b, m.a_aug, m.b_aug, a);
  }
}

constexpr int MAX_D_WIDE = 4096;  // rows of up to this many values take the streamed kernel

}  // namespace

bool knn_tc_available(int d) {
  static const int avail = [] {
    int dev = 0, major = 0, minor = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) == cudaSuccess)
      return (major == 10 && minor == 3 && encode_fn() != nullptr) ? 1 : 0;
    return 0;
  }();
  const int kchunks = ((d + 63) & ~63) / 64;
  if (avail != 1 || d < 1) return false;
  return tc_smem_bytes(kchunks, 2) <= 225 * 1024 ||
         (d <= MAX_D_WIDE && tcw_smem_bytes() <= 225 * 1024);
}

int knn_tc_max_k(int d, bool limited) {
  const int kchunks = ((d + 63) & ~63) / 64;
  const int bn = tc_smem_bytes(kchunks, 2) <= 225 * 1024 ? BN : BNW;
  // a row buffer holds 1024 keys: KS + bn (twice KS for a limited walk), KS = K + 1
  return limited ? (1024 - bn) / 2 - 1 : 1024 - bn - 1;
}

void knn_exact_tc(const float* A, int64_t na, int lda, const float* a_norm, const float* B,
                  int64_t nb, int ldb, const float* b_norm, int d, int self, int K,
                  int32_t* out_id, float* out_d2, cudaStream_t st, StageTimer* gemm_timer,
                  int max_tiles, bool approx, const TcExtra& ex) {
  const int dp = (d + 63) & ~63;
  const int dpe = ex.pairs ? 3 * dp : dp;  // row width the tensor cores see
  const int kchunks = dpe / 64;
  int stages = MAX_STAGES;
  while (stages > 2 && tc_smem_bytes(kchunks, stages) > 225 * 1024) --stages;
  // rows that do not fit the resident pipeline stream through the wide kernel
  const bool wide = tc_smem_bytes(kchunks, stages) > 225 * 1024 || ex.stream_rows;
  SSG_REQUIRE(!wide || (dpe <= MAX_D_WIDE && tcw_smem_bytes() <= 225 * 1024), SSG_EINVAL,
              "tensor-core kNN: d = %d is too large for the shared-memory pipeline", d);
  const int bm = wide ? BMW : BM, bn = wide ? BNW : BN;
  const int KS = self ? K + 1 : K;
  // Near-first column order for large self-joins with a deep top-K (where the streaming
  // threshold otherwise falls slowly and many candidates are appended).
  KnnOrder ord;
  Scratch<float> norm_p;
  // tile limits come in 128-point tiles; the walk counts bn-column tiles
  if (max_tiles > 0) max_tiles = (int)ceil_div((int64_t)max_tiles * API_TILE, bn);
  // same: the query rows are the base rows (a self-join); with ex.qid the query rows are a
  // gathered subset of the base and only the self column is excluded
  const bool same = self && !ex.qid;
  SSG_REQUIRE(max_tiles == 0 || (same && knn_order_fits(na, bn)), SSG_EINVAL,
              "a tile limit needs a self-join whose cluster order fits");
  // (not for the K-chunked kernel: its tiles are long enough that the appends a slowly
  // falling threshold costs matter less than L2 reuse, which needs every CTA to walk the
  // columns in the same order: 200,000 x 960 with bf16 pairs, 270 -> 227 ms, the
  // near-first walks kept DRAM 78% busy at a 34% L2 hit rate)
  const bool ordered =
      max_tiles > 0 || (!wide && same && na >= (1 << 16) && K >= 16 && knn_order_fits(na, bn));
  if (ordered) {
    knn_cluster_order(A, lda, d, na, bm, bn, st, ord, max_tiles,
                      ex.order_norm ? ex.order_norm : a_norm);
    norm_p.alloc((size_t)na, st);
  }
  Scratch<__nv_bfloat16> ab((size_t)na * dpe, st);
  Scratch<__nv_bfloat16> bb;
  const int cgrid = 8 * num_sms();
  SSG_LAUNCH(k_to_bf16, cgrid, 256, 0, st, A, na, d, lda, ab.p, dp,
             ordered ? (const int32_t*)ord.perm.p : nullptr, a_norm, ordered ? norm_p.p : nullptr,
             ex.mu, ex.pairs ? 1 : 0);
  if (ordered) a_norm = b_norm = norm_p.p;
  const __nv_bfloat16* bptr = ab.p;
  if (!same || ex.pairs) {
    // bf16 pairs: the base side has its own layout (in the self-join's stored order)
    bb.alloc((size_t)nb * dpe, st);
    SSG_LAUNCH(k_to_bf16, cgrid, 256, 0, st, B, nb, d, ldb, bb.p, dp,
               same && ordered ? (const int32_t*)ord.perm.p : nullptr, (const float*)nullptr,
               (float*)nullptr, ex.mu, ex.pairs ? 2 : 0);
    bptr = bb.p;
  }
  Scratch<__nv_bfloat16> aug_b((size_t)nb * AUG, st), aug_a((size_t)BM * AUG, st);
  Scratch<int> err(1, st);
  SSG_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), st));
  SSG_LAUNCH(k_aug_rows, (unsigned)std::min<int64_t>(ceil_div(nb, 256), cgrid), 256, 0, st, b_norm,
             nb, aug_b.p, err.p, approx ? 1 : 0);
  SSG_LAUNCH(k_aug_ones, 1, 256, 0, st, aug_a.p);
  TcMaps maps;
  maps.a = make_map(ab.p, na, dpe, 64, bm, CU_TENSOR_MAP_SWIZZLE_128B);
  maps.b = make_map(bptr, nb, dpe, 64, bn, CU_TENSOR_MAP_SWIZZLE_128B);
  maps.a_aug = make_map(aug_a.p, BM, AUG, AUG, bm, CU_TENSOR_MAP_SWIZZLE_32B);
  maps.b_aug = make_map(aug_b.p, nb, AUG, AUG, bn, CU_TENSOR_MAP_SWIZZLE_32B);
  const int64_t nrb = ceil_div(na, bm);
  const int grid = (int)std::min<int64_t>(nrb, num_sms());
  // A row buffer holds C keys and is compacted once a tile could overflow it.  A limited
  // walk spends most of its tiles while the threshold is still falling, so it gets room
  // for about KS more keys between compactions.
  const int need = max_tiles > 0 ? 2 * KS + bn : KS + bn;
  SSG_REQUIRE(need <= 1024, SSG_EINVAL, "tensor-core kNN: K = %d is too large for %d-column tiles",
              K, bn);
  const int C = need <= 256 ? 256 : (need <= 512 ? 512 : 1024);
  Scratch<uint64_t> rowbuf((size_t)grid * bm * C, st);
  TcArgs a{};
  a.a_norm = a_norm;
  a.na = na;
  a.nb = nb;
  a.ntiles = ceil_div(nb, bn);
  a.nwalk = max_tiles > 0 ? std::min<int64_t>(a.ntiles, max_tiles) : a.ntiles;
  a.tstride = ordered ? ord.tstride : a.ntiles;
  a.kchunks = kchunks;
  a.stages = stages;
  a.self = self;
  a.KS = KS;
  a.K = K;
  a.trig = C - bn;
  a.rowbuf = rowbuf.p;
  a.out_id = out_id;
  a.out_d2 = out_d2;
  a.err = err.p;
  a.out_thresh = ex.out_thresh;
  a.qid = ex.qid;
  a.tau_in = ex.tau_in;
  if (ordered) {
    a.perm = ord.perm.p;
    a.inv = ord.inv.p;
    a.tile_order = ord.tile_order.p;
    a.rb_cluster = ord.rb_cluster.p;
  }
  const size_t smem = wide ? tcw_smem_bytes() : tc_smem_bytes(kchunks, stages);
  auto launch = [&](TcArgs& args) {
    if (C == 256)
      launch_tc<256>(maps, args, grid, smem, st, wide);
    else if (C == 512)
      launch_tc<512>(maps, args, grid, smem, st, wide);
    else
      launch_tc<1024>(maps, args, grid, smem, st, wide);
  };
  // Near-first full walks: a first launch over each block's prepass_tiles nearest tiles
  // only records each row's KS-th distance there, an upper bound of its KS-th distance over
  // all columns (the same values: the MMAs are the same); the full walk then admits only
  // columns at or below that bound, so its appends and compactions are few from the start.
  Scratch<float> tau0;
  const int64_t pre_tiles = ceil_div((int64_t)ex.prepass_tiles * API_TILE, bn);
  const bool prepass = ordered && max_tiles == 0 && pre_tiles > 0 && a.ntiles > 2 * pre_tiles;
  if (gemm_timer) gemm_timer->start();
  if (prepass) {
    tau0.alloc((size_t)na, st);
    TcArgs a0 = a;
    a0.nwalk = pre_tiles;
    a0.thresh_only = 1;
    a0.tau_out = tau0.p;
    a0.out_thresh = nullptr;
    launch(a0);
    a.tau_in = tau0.p;
    // approximate data: widen by far more than the rounding of the threshold test
    a.tau_relax = approx ? 9.5367431640625e-07f : 0.f;  // 2^-20
  }
  launch(a);
  if (gemm_timer) gemm_timer->stop();
  int h = 0;
  SSG_CUDA(cudaMemcpyAsync(&h, err.p, sizeof(int), cudaMemcpyDeviceToHost, st));
  SSG_CUDA(cudaStreamSynchronize(st));
  if (h != 0) note_device_status(h == 1 ? SSG_EINTERNAL : SSG_ETIMEOUT);
  SSG_REQUIRE(h != 1, SSG_EINTERNAL, "tensor-core kNN: a squared norm is not split exactly");
  SSG_REQUIRE(h == 0, SSG_ETIMEOUT, "tensor-core kNN: a pipeline wait timed out (code %d)", h);
}

}  // namespace ssg
