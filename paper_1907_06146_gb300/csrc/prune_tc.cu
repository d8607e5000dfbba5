// SSG prune (Alg. 2 selection applied to every pool, Alg. 3) with the pool's Gram matrix
// on the 5th-generation tensor cores, for integer data that bf16 holds exactly.
//
// For node x with candidates c_1..c_m (m <= 127) the rows [x, c_1, .., c_m] are copied
// into shared memory in the tensor cores' operand layout (128-byte swizzle) and one
// 128x128xd UMMA gives H = C C^T in TMEM.  Every product and partial sum is an integer
// below 2^24, so H is exact, and so is every centred dot product the angle rule needs:
//     G_jk = (c_j - x).(c_k - x) = H_jk - H_j0 - H_k0 + H_00,   G_jj = d2(x, c_j).
// c_j and c_k conflict when cos(j, k) = G_jk / sqrt(G_jj G_kk) > cos(alpha); a zero-length
// edge conflicts with every other exactly when 0 > cos(alpha).  The fp32 cosine decides
// where it is more than 16 units of roundoff (plus the reporting band) from cos(alpha) (its
// inputs are exact, its error a few units); otherwise the test is taken in fp64 from the
// same exact integers with the operations of the definition, which reproduces the
// double-precision rule bit for bit.
//
// Only the tests the greedy selection needs are made (c_j against the candidates kept
// before it, in candidate order, until R are kept).  The lower triangle of H goes from TMEM
// to a shared-memory slot, row i at i(i+1)/2 (32 consecutive rows start in 32 different
// banks, so a column read across rows is conflict-free, as is a read along a row).  A
// selection warp then takes the candidates in blocks of 32, one per lane: each lane tests
// its candidate against the candidates kept in earlier blocks (a conflict with any of them
// rejects it, whatever the order); then each survivor is tested against the block's earlier
// survivors at once (a bitmask per lane), and the greedy runs over those bitmasks in rounds
// (a survivor is kept once every earlier survivor it conflicts with is rejected).
//
// Persistent kernel, one CTA per SM:
//   warps 0..2   load the rows of every third node into their tile (16-byte cp.async
//                copies);
//   warp 3       allocates 512 TMEM columns and issues the Gram UMMAs into one of 4 TMEM
//                buffers;
//   warps 4..7   copy the lower triangle of H into the node's slot, one TMEM lane quadrant
//                (32 rows) each;
//   warps 8..    select, one warp per slot, warp s taking every nsel-th node.
// Every wait is bounded (about 2 s); a wait that runs out sets an error word, tells the
// other roles to stop, and the CTA releases its TMEM and exits.
#include "common.cuh"
#include "knn.cuh"
#include "tc_common.cuh"

namespace ssg {
namespace {

using namespace tc;

constexpr int PT_ROWS = 128;                  // the node and up to 127 candidates
constexpr int GSLOTS = 3;                     // gather tiles, one loader warp each
constexpr int MMA_WARP = GSLOTS;
constexpr int COPY_WARPS = 4;                 // one per TMEM lane quadrant
constexpr int FIRST_COPY = MMA_WARP + 1;
constexpr int MAX_SEL = 8;                    // selection warps (and slots) at most
constexpr int FIRST_SEL = FIRST_COPY + COPY_WARPS;
constexpr int THREADS_MAX = (FIRST_SEL + MAX_SEL) * 32;
constexpr int TMEM_COLS_P = 512;              // 4 buffers of 128 fp32 columns
constexpr int SMEM_CAP = 227 * 1024;          // the opt-in limit of one CTA

struct PtArgs {
  const __nv_bfloat16* xb;      // the rows in bf16, dp = 64 kchunks values each
  const int32_t* pool_id;
  const int32_t* pool_len;
  const int32_t* items;         // nullable: the nodes to prune (else 0 .. n - 1)
  int64_t n;                    // nodes to prune (items' length)
  int L, R, kchunks;
  int nsel;                     // selection warps = slots
  int slot_floats;              // floats of one slot (the lower triangle of the longest pool)
  int sel_f4;                   // float4s per selection warp: the kept list (R) + a block's rows (32)
  float cosA32, margin;
  double cosA64;
  int32_t* adj;
  int32_t* deg;
  unsigned long long* n64;
  int* err;
  double border;                // fp64 cosines within this of cos(alpha) are counted
  unsigned long long* nborder;
};

// Offset of row i of a packed lower triangle.
__device__ __forceinline__ int tri(int i) { return (i * (i + 1)) >> 1; }

// The angle rule for a pair of candidates: g their exact centred dot product, dj and dk
// their exact squared lengths, rj and rk the reciprocal lengths (0 for a zero length).
struct AngleRule {
  float hi, lo;
  double cosA64, border;
  bool zc;                      // the rule for a zero-length edge
  unsigned long long n64, nb;

  // The fp32 decision; band: the cosine is too close to cos(alpha), the fp64 rule decides.
  __device__ __forceinline__ bool fast(float g, float dj, float dk, float rj, float rk,
                                       bool& band) const {
    const float cs = g * rj * rk;
    const bool zero = (dj == 0.f) | (dk == 0.f);
    band = !zero & (cs >= lo) & (cs <= hi);
    return zero ? zc : cs > hi;
  }
  // The double-precision rule on the same exact integers.
  __device__ __forceinline__ bool exact(float g, float dj, float dk) {
    const double c64 = cos_from_gram_f64((double)g, (double)dj, (double)dk);
    ++n64;
    if (fabs(c64 - cosA64) <= border) ++nb;
    return c64 > cosA64;
  }
};

__global__ void __launch_bounds__(THREADS_MAX, 1)
k_prune_tc(PtArgs p) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* sm = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const uint32_t g_bytes = (uint32_t)p.kchunks * PT_ROWS * 128;
  const int nsel = p.nsel;
  unsigned char* sG = sm;                                            // GSLOTS gather tiles
  float* sP = (float*)(sG + (size_t)GSLOTS * g_bytes);               // nsel slots
  float4* sK = (float4*)(sP + (size_t)nsel * p.slot_floats);          // nsel x sel_f4
  uint64_t* bars = (uint64_t*)(sK + (size_t)nsel * p.sel_f4);
  uint64_t* g_full = bars;
  uint64_t* g_empty = g_full + GSLOTS;
  uint64_t* t_full = g_empty + GSLOTS;
  uint64_t* t_empty = t_full + 4;
  uint64_t* d_full = t_empty + 4;
  uint64_t* d_empty = d_full + MAX_SEL;
  uint32_t* tmem_slot = (uint32_t*)(d_empty + MAX_SEL);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = lane_id();
  if (threadIdx.x == 0) {
    for (int s = 0; s < GSLOTS; ++s) {
      mbar_init(smem_u32(g_full + s), 1);
      mbar_init(smem_u32(g_empty + s), 1);
    }
    for (int b = 0; b < 4; ++b) {
      mbar_init(smem_u32(t_full + b), 1);
      mbar_init(smem_u32(t_empty + b), COPY_WARPS);
    }
    for (int s = 0; s < nsel; ++s) {
      mbar_init(smem_u32(d_full + s), COPY_WARPS);
      mbar_init(smem_u32(d_empty + s), 1);
    }
    *abort_flag = 0;
    fence_barrier_init();
  }
  if (warp == MMA_WARP) {
    tmem_alloc(smem_u32(tmem_slot), TMEM_COLS_P);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  const int64_t n = p.n;
  auto node = [&](int64_t t) -> int64_t { return p.items ? (int64_t)p.items[t] : t; };

  if (warp < GSLOTS) {
    // ---------------- loader of tile s = warp: every GSLOTS-th node ----------------
    // 16-byte cp.async copies straight into the UMMA operand layout (K-major, 128-byte
    // swizzle: row r of a 64-column chunk at (r / 8) 1024 + (r % 8) 128 bytes, its 16-byte
    // piece c at (c ^ (r % 8)) 16); the warp waits for its copies, makes them visible to
    // the tensor cores' proxy and signals the tile.  A node's length and candidate ids load
    // one node ahead.
    const int s = warp, L = p.L, dp = p.kchunks * 64;
    const int lpr = p.kchunks * 4;              // lanes per row, two 16-byte pieces each
    const int rpi = 32 / lpr;                   // rows per warp step
    const int sub = lane / lpr, v = (lane % lpr) * 2, kc = v >> 3, c = v & 7;
    unsigned char* tile = sG + (size_t)s * g_bytes + (size_t)kc * PT_ROWS * 128;
    const int64_t step = (int64_t)GSLOTS * gridDim.x;
    uint32_t ph = 0;
    bool ok = true;
    int64_t t = blockIdx.x + (int64_t)s * gridDim.x;
    int len = 0, ids[4];
    auto fetch = [&](int64_t tt) {
      const int64_t xx = node(tt);
      len = p.pool_len[xx];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int r = u * 32 + lane;            // row 0 is the node, row r the candidate r - 1
        ids[u] = (r >= 1 && r <= L) ? p.pool_id[xx * L + r - 1] : (int)xx;
      }
    };
    if (t < n) fetch(t);
    for (; t < n; t += step) {
      const int64_t x = node(t);
      const int lc = min(len, PT_ROWS - 1);
      int cur[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) cur[u] = u * 32 + lane > lc ? (int)x : ids[u];
      if (t + step < n) fetch(t + step);
      ok = mbar_wait(smem_u32(g_empty + s), ph ^ 1, abort_flag);
      if (!__all_sync(0xffffffffu, ok)) {
        ok = false;
        break;
      }
      ph ^= 1;
      const int nrows = lc + 1;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if (u * 32 >= nrows) break;
        for (int r0 = u * 32; r0 < min(nrows, u * 32 + 32); r0 += rpi) {
          const int r = r0 + sub;
          const int id = __shfl_sync(0xffffffffu, cur[u], r & 31);
          if (r < nrows) {
            const __nv_bfloat16* src = p.xb + (size_t)id * dp + kc * 64 + c * 8;
            const uint32_t dst = smem_u32(tile + (r >> 3) * 1024 + (r & 7) * 128);
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst + ((c ^ (r & 7)) << 4)),
                         "l"(src) : "memory");
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst + (((c + 1) ^ (r & 7)) << 4)),
                         "l"(src + 8) : "memory");
          }
        }
      }
      asm volatile("cp.async.wait_all;" ::: "memory");
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(g_full + s));
    }
    if (!ok && lane == 0) {
      atomicOr(p.err, 1);
      *abort_flag = 1;
    }
  } else if (warp == MMA_WARP) {
    // ---------------- Gram MMA issuer ----------------
    if (lane == 0) {
      int s = 0, b = 0;
      uint32_t ph = 0, tph = 0;
      bool ok = true;
      for (int64_t x = blockIdx.x; x < n; x += gridDim.x) {
        ok = mbar_wait(smem_u32(t_empty + b), tph ^ 1, abort_flag) &&
             mbar_wait(smem_u32(g_full + s), ph, abort_flag);
        if (!ok) break;
        tc_fence_after();
        const uint64_t desc0 = sdesc_sw128(smem_u32(sG + (size_t)s * g_bytes));
        const uint32_t d_tmem = tmem_base + (uint32_t)(b * 128);
        for (int kc = 0; kc < p.kchunks; ++kc) {
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {
            const uint64_t dsc = desc0 + (uint64_t)((kc * PT_ROWS * 128 + kk * 32) >> 4);
            umma_bf16(d_tmem, dsc, dsc, (kc | kk) ? 1u : 0u);
          }
        }
        umma_commit(smem_u32(g_empty + s));
        umma_commit(smem_u32(t_full + b));
        if (++s == GSLOTS) {
          s = 0;
          ph ^= 1;
        }
        if (++b == 4) {
          b = 0;
          tph ^= 1;
        }
      }
      if (!ok) {
        atomicOr(p.err, 2);
        *abort_flag = 1;
      }
    }
    __syncwarp();
  } else if (warp < FIRST_SEL) {
    // ---------------- TMEM -> packed lower triangle in the node's slot ----------------
    const int q = warp & 3;                  // TMEM lane quadrant
    const int i = q * 32 + lane;             // row: 0 the node, i the candidate i - 1
    int b = 0, s = 0;
    uint32_t tph = 0, sph = 0;
    bool ok = true;
    int len = blockIdx.x < n ? p.pool_len[node(blockIdx.x)] : 0;   // one node ahead
    for (int64_t t = blockIdx.x; t < n; t += gridDim.x) {
      const int nrows = min(len, PT_ROWS - 1) + 1;
      if (t + gridDim.x < n) len = p.pool_len[node(t + gridDim.x)];
      ok = mbar_wait(smem_u32(t_full + b), tph, abort_flag) &&
           mbar_wait(smem_u32(d_empty + s), sph ^ 1, abort_flag);
      if (!__all_sync(0xffffffffu, ok)) {
        ok = false;
        break;
      }
      tc_fence_after();
      if (q * 32 < nrows) {
        float* row = sP + (size_t)s * p.slot_floats + (i < nrows ? tri(i) : 0);
        const uint32_t taddr = tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(b * 128);
        for (int c = 0; c <= q; ++c) {
          uint32_t v[32];
          tmem_ld32(taddr + (uint32_t)(c * 32), v);
          tmem_wait_ld(v);
          if (i < nrows) {
#pragma unroll
            for (int e = 0; e < 32; ++e)
              if (c * 32 + e <= i) row[c * 32 + e] = __uint_as_float(v[e]);
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(smem_u32(t_empty + b));
        mbar_arrive(smem_u32(d_full + s));
      }
      if (++b == 4) {
        b = 0;
        tph ^= 1;
      }
      if (++s == nsel) {
        s = 0;
        sph ^= 1;
      }
    }
    if (!ok && lane == 0) {
      atomicOr(p.err, 4);
      *abort_flag = 1;
    }
  } else if (warp < FIRST_SEL + nsel) {
    // ---------------- selection in candidate order ----------------
    const int w = warp - FIRST_SEL;
    const float* P = sP + (size_t)w * p.slot_floats;
    float4* S = sK + (size_t)w * p.sel_f4;   // kept: H_k0, G_kk, 1/sqrt(G_kk), row k
    float4* T4 = S + p.R;                    // the block's rows: H_j0, G_jj, 1/sqrt(G_jj)
    AngleRule at{p.cosA32 + p.margin, p.cosA32 - p.margin, p.cosA64, p.border, 0.0 > p.cosA64,
                 0ull, 0ull};
    const int R = p.R, L = p.L;
    const unsigned lt = lanemask_lt();
    const int64_t step = (int64_t)nsel * gridDim.x;
    uint32_t ph = 0;
    bool ok = true;
    int64_t t = blockIdx.x + (int64_t)w * gridDim.x;
    int len = t < n ? p.pool_len[node(t)] : 0;   // one node ahead
    for (; t < n; t += step) {
      const int64_t x = node(t);
      const int nrows = min(len, PT_ROWS - 1) + 1;
      // the candidate ids (for the output) and the next length load during the wait
      const int32_t* cand = p.pool_id + x * L;
      int cid[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) cid[u] = u * 32 + lane < nrows - 1 ? cand[u * 32 + lane] : -1;
      if (t + step < n) len = p.pool_len[node(t + step)];
      ok = mbar_wait(smem_u32(d_full + w), ph, abort_flag);
      if (!__all_sync(0xffffffffu, ok)) {
        ok = false;
        break;
      }
      ph ^= 1;
      const float h00 = P[0];
      int kept = 0;
      for (int b0 = 0; b0 < nrows && kept < R; b0 += 32) {
        // lane: candidate j = b0 + lane
        const int j = b0 + lane;
        const bool valid = j >= 1 && j < nrows;
        const int jc = valid ? j : 0;          // last column of row j
        const int tj = tri(jc);
        const float aj = P[tj];                                  // H_j0
        const float dj = valid ? (P[tj + jc] - 2.f * aj) + h00 : 0.f;  // G_jj, exact
        const float rj = dj > 0.f ? __frsqrt_rn(dj) : 0.f;
        const float t0j = h00 - aj;
        // 1. against the candidates kept in earlier blocks (one conflict rejects)
        bool out = !valid;
        for (int m0 = 0; m0 < kept; m0 += 4) {
          if (!__any_sync(0xffffffffu, !out)) break;
          float4 s4[4];
          float h[4];
          bool bd[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) s4[u] = S[min(m0 + u, kept - 1)];
#pragma unroll
          for (int u = 0; u < 4; ++u) h[u] = P[tj + min(__float_as_int(s4[u].w), jc)];
          bool hit = false, band_any = false;
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const bool act = m0 + u < kept;
            const bool c = at.fast((h[u] - s4[u].x) + t0j, dj, s4[u].y, rj, s4[u].z, bd[u]);
            hit |= act & c;
            bd[u] &= act;
            band_any |= bd[u];
          }
          out |= hit;
          band_any &= !out;
          if (__any_sync(0xffffffffu, band_any) && band_any) {
#pragma unroll
            for (int u = 0; u < 4; ++u)
              if (bd[u] && !out) out = at.exact((h[u] - s4[u].x) + t0j, dj, s4[u].y);
          }
        }
        const uint32_t alive = __ballot_sync(0xffffffffu, !out);
        if (alive != 0u) {
          // 2. conflicts among the block's survivors: bit e of M (lane j) says survivor
          //    b0 + e (e < lane) conflicts with c_j
          T4[lane] = make_float4(aj, dj, rj, 0.f);
          __syncwarp();
          const bool me = !out;
          uint32_t M = 0, Mb = 0, rest = alive;
          while (rest != 0u) {
            int ee[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              ee[u] = rest ? __ffs(rest) - 1 : 31;
              rest &= rest - 1u;
            }
            float4 k4[4];
            float h[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) k4[u] = T4[ee[u]];
#pragma unroll
            for (int u = 0; u < 4; ++u) h[u] = P[tj + min(b0 + ee[u], jc)];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              bool band;
              const bool c = at.fast((h[u] - k4[u].x) + t0j, dj, k4[u].y, rj, k4[u].z, band);
              const bool act = me & (lane > ee[u]) & ((alive >> ee[u]) & 1u);
              M |= (act & c) ? 1u << ee[u] : 0u;
              Mb |= (act & band) ? 1u << ee[u] : 0u;
            }
          }
          if (__any_sync(0xffffffffu, Mb != 0u)) {
            while (Mb != 0u) {
              const int e = __ffs(Mb) - 1;
              Mb &= Mb - 1u;
              const float4 k4 = T4[e];
              if (at.exact((P[tj + b0 + e] - k4.x) + t0j, dj, k4.y)) M |= 1u << e;
            }
          }
          // 3. the greedy over the survivors in order, in rounds: a survivor whose earlier
          //    conflicting survivors are all rejected is kept, one with a kept one rejected
          uint32_t U = alive, K = 0;
          while (U != 0u) {
            const bool und = (U >> lane) & 1u;
            const uint32_t bk = __ballot_sync(0xffffffffu, und && (M & (K | U)) == 0u);
            const uint32_t br = __ballot_sync(0xffffffffu, und && (M & K) != 0u);
            K |= bk;
            U &= ~(bk | br);
          }
          // stop at R: the first R - kept of them in order
          while (__popc(K) > R - kept) K &= ~(1u << (31 - __clz(K)));
          // 4. the block's kept candidates join the kept list in order
          if ((K >> lane) & 1u) S[kept + __popc(K & lt)] = make_float4(aj, dj, rj, __int_as_float(j));
          kept += __popc(K);
        }
        __syncwarp();
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(d_empty + w));   // the slot is read
      int32_t* outp = p.adj + x * R;
      for (int m0 = 0; m0 < R; m0 += 32) {
        const int m = m0 + lane;
        const int r = m < kept ? __float_as_int(S[m].w) - 1 : 0;   // candidate r
        int v = -1;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int t = __shfl_sync(0xffffffffu, cid[u], r & 31);
          if ((r >> 5) == u) v = t;
        }
        if (m < R) outp[m] = m < kept ? v : -1;
      }
      if (lane == 0) p.deg[x] = kept;
      __syncwarp();
    }
    if (at.n64) atomicAdd(p.n64, at.n64);
    if (at.nb) atomicAdd(p.nborder, at.nb);
    if (!ok && lane == 0) {
      atomicOr(p.err, 8);
      *abort_flag = 1;
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == MMA_WARP) {
    tc_fence_after();
    tmem_dealloc(tmem_base, TMEM_COLS_P);
  }
}

// bf16 rows padded to dp (exact for the integer data this path takes).
__global__ void k_rows_bf16(const float* __restrict__ X, int64_t n, int d, int ld,
                            __nv_bfloat16* __restrict__ Y, int dp) {
  const int64_t total = n * (int64_t)dp;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / dp;
    const int c = (int)(i - r * dp);
    Y[i] = __float2bfloat16_rn(c < d ? X[r * ld + c] : 0.f);
  }
}

// Floats of one slot: the packed lower triangle of the longest pool's 1 + L rows.
int prune_tc_slot_floats(int L) {
  const int rows = std::min(L, PT_ROWS - 1) + 1;
  return ((rows * (rows + 1) / 2) + 3) & ~3;
}

size_t prune_tc_fixed_smem(int kchunks) {
  return 1024 + (size_t)GSLOTS * kchunks * PT_ROWS * 128 +
         sizeof(uint64_t) * (2 * GSLOTS + 8 + 2 * MAX_SEL) + 16;
}

// Selection warps (and slots) that fit beside the gather tiles, at most MAX_SEL.
int prune_tc_sel_f4(int R) { return R + 32; }

int prune_tc_nsel(int kchunks, int L, int R) {
  const size_t fixed = prune_tc_fixed_smem(kchunks);
  if (fixed >= (size_t)SMEM_CAP) return 0;
  const size_t per = (size_t)prune_tc_slot_floats(L) * sizeof(float) +
                     (size_t)prune_tc_sel_f4(R) * sizeof(float4);
  return (int)std::min<size_t>(MAX_SEL, ((size_t)SMEM_CAP - fixed) / per);
}

size_t prune_tc_smem(int kchunks, int L, int R, int nsel) {
  return prune_tc_fixed_smem(kchunks) +
         (size_t)nsel * ((size_t)prune_tc_slot_floats(L) * sizeof(float) +
                         (size_t)prune_tc_sel_f4(R) * sizeof(float4));
}

}  // namespace

bool prune_tc_available(int d, int L, int R) {
  const int kchunks = (d + 63) / 64;
  return knn_tc_available(d) && kchunks <= 2 && L >= 1 && L <= PT_ROWS - 1 && R >= 1 &&
         R <= PT_ROWS && prune_tc_nsel(kchunks, L, R) >= 2;
}

namespace {

// One launch over `items` (null: nodes 0 .. nitems - 1), slots sized for pools of up to
// Lrows candidates (pool rows L apart).
void launch_prune_tc(const __nv_bfloat16* xb, int kchunks, const int32_t* items, int64_t nitems,
                     const int32_t* pool_id, const int32_t* pool_len, int L, int Lrows, int R,
                     double cos_a, double border, int32_t* adj, int32_t* deg, Counters* dctr,
                     int* err, cudaStream_t st) {
  if (nitems <= 0) return;
  PtArgs a{};
  a.xb = xb;
  a.pool_id = pool_id;
  a.pool_len = pool_len;
  a.items = items;
  a.n = nitems;
  a.L = L;
  a.R = R;
  a.kchunks = kchunks;
  a.nsel = prune_tc_nsel(kchunks, Lrows, R);
  a.sel_f4 = prune_tc_sel_f4(R);
  a.slot_floats = prune_tc_slot_floats(Lrows);
  a.cosA32 = (float)cos_a;
  a.cosA64 = cos_a;
  a.margin = (float)(16.0 * U32 + border);
  a.adj = adj;
  a.deg = deg;
  a.n64 = &dctr->angle_fp64;
  a.border = border;
  a.nborder = &dctr->angle_border;
  a.err = err;
  SSG_REQUIRE(a.nsel >= 2 && a.nsel <= MAX_SEL, SSG_EINTERNAL,
              "tensor-core prune: %d selection slots for pools of %d", a.nsel, Lrows);
  const size_t smem = prune_tc_smem(kchunks, Lrows, R, a.nsel);
  ensure_smem((const void*)k_prune_tc, smem);
  const int grid = (int)std::min<int64_t>(nitems, num_sms());
  SSG_LAUNCH(k_prune_tc, grid, (FIRST_SEL + a.nsel) * 32, smem, st, a);
}

// Nodes with at most `thr` candidates to short_ids, the rest to long_ids (counts[0], [1]);
// a warp takes one slot per list with one atomic.
__global__ void k_split_by_len(const int32_t* __restrict__ len, int64_t n, int thr,
                               int32_t* __restrict__ short_ids, int32_t* __restrict__ long_ids,
                               int* __restrict__ counts) {
  const int lane = threadIdx.x & 31;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += stride) {
    const int64_t i = base + threadIdx.x;
    const bool in = i < n;
    const bool sh = in && len[i] <= thr;
    const unsigned bs = __ballot_sync(0xffffffffu, sh), bl = __ballot_sync(0xffffffffu, in && !sh);
    int s0 = 0, l0 = 0;
    if (lane == 0) {
      if (bs) s0 = atomicAdd(counts, __popc(bs));
      if (bl) l0 = atomicAdd(counts + 1, __popc(bl));
    }
    s0 = __shfl_sync(0xffffffffu, s0, 0);
    l0 = __shfl_sync(0xffffffffu, l0, 0);
    const unsigned lt = lanemask_lt();
    if (sh) short_ids[s0 + __popc(bs & lt)] = (int32_t)i;
    else if (in) long_ids[l0 + __popc(bl & lt)] = (int32_t)i;
  }
}

void check_prune_err(const int* err, cudaStream_t st) {
  int h = 0;
  SSG_CUDA(cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, st));
  SSG_CUDA(cudaStreamSynchronize(st));
  if (h != 0) note_device_status(SSG_ETIMEOUT);
  SSG_REQUIRE(h == 0, SSG_ETIMEOUT, "tensor-core prune: a pipeline wait timed out (code %d)", h);
}

}  // namespace

void prune_run_tc(const float* X, int ld, int d, int64_t n, const int32_t* pool_id,
                  const int32_t* pool_len, int L, int R, double cos_a, double border,
                  int32_t* adj, int32_t* deg, Counters* dctr, cudaStream_t st, bool split) {
  const int dp = (d + 63) & ~63;
  const int kchunks = dp / 64;
  Scratch<__nv_bfloat16> xb((size_t)n * dp, st);
  SSG_LAUNCH(k_rows_bf16, 8 * num_sms(), 256, 0, st, X, n, d, ld, xb.p, dp);
  Scratch<int> err(3, st);
  SSG_CUDA(cudaMemsetAsync(err.p, 0, 3 * sizeof(int), st));
  constexpr int SHORT = 63;   // pools of up to 63 candidates: slots a third the size
  if (!split || L <= SHORT) {
    launch_prune_tc(xb.p, kchunks, nullptr, n, pool_id, pool_len, L, L, R, cos_a, border, adj,
                    deg, dctr, err.p, st);
  } else {
    // short pools (most merged reverse lists) get small slots and more selection warps
    Scratch<int32_t> ids((size_t)2 * n, st);
    SSG_LAUNCH(k_split_by_len, 4 * num_sms(), 256, 0, st, pool_len, n, SHORT, ids.p, ids.p + n,
               err.p + 1);
    int cnt[2] = {0, 0};
    SSG_CUDA(cudaMemcpyAsync(cnt, err.p + 1, sizeof(cnt), cudaMemcpyDeviceToHost, st));
    SSG_CUDA(cudaStreamSynchronize(st));
    SSG_REQUIRE(cnt[0] >= 0 && cnt[1] >= 0 && (int64_t)cnt[0] + cnt[1] == n, SSG_EINTERNAL,
                "tensor-core prune: split %d + %d of %lld pools", cnt[0], cnt[1], (long long)n);
    launch_prune_tc(xb.p, kchunks, ids.p, cnt[0], pool_id, pool_len, L, SHORT, R, cos_a, border,
                    adj, deg, dctr, err.p, st);
    launch_prune_tc(xb.p, kchunks, ids.p + n, cnt[1], pool_id, pool_len, L, L, R, cos_a, border,
                    adj, deg, dctr, err.p, st);
  }
  check_prune_err(err.p, st);
}

}  // namespace ssg
