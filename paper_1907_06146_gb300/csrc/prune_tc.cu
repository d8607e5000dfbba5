// SSG prune (Alg. 2 selection applied to every pool, Alg. 3) with the pool's Gram matrix
// on the 5th-generation tensor cores, for integer data that bf16 holds exactly.
//
// For node x with candidates c_1..c_m (m <= 127) the 128 rows [x, c_1, .., c_m, ..] are
// gathered into shared memory (TMA gather4, 128-byte swizzle) and one 128x128xd UMMA gives
// H = C C^T in TMEM.  Every product and partial sum is an integer below 2^24, so H is
// exact, and so is every centred dot product the angle rule needs:
//     G_jk = (c_j - x).(c_k - x) = H_jk - H_j0 - H_k0 + H_00,   G_jj = d2(x, c_j).
// The selection then follows the rule in candidate order: keep c_j unless
// cos(j, k) = G_jk / sqrt(G_jj G_kk) > cos(alpha) for a kept c_k (0 for a zero-length
// edge).  The fp32 cosine decides where it is more than 16 units of roundoff from cos(alpha)
// (its inputs are exact, so its error is a few units); otherwise, and for zero-length
// edges, the decision is taken in fp64 from the same exact integers with the operations of
// the definition, which reproduces the double-precision rule bit for bit.
//
// Persistent kernel, one CTA per SM, 9 warps:
//   warp 0      gathers the node and candidate rows (gather4, 4 rows per TMA) into one of
//               GSLOTS shared-memory tiles;
//   warp 1      allocates 512 TMEM columns and issues the Gram UMMAs into one of 4 TMEM
//               buffers;
//   warps 2..5  (one per TMEM lane quadrant) turn H into the centred Gram's lower triangle
//               and diagonal (int32) in one of TSLOTS shared-memory slots;
//   warps 6..8  select: each takes every third node, lanes over the kept edges.
// Every wait is bounded (about 2 s); a wait that runs out sets an error word, tells the
// other roles to stop, and the CTA releases its TMEM and exits.
#include "common.cuh"
#include "knn.cuh"
#include "tc_common.cuh"

namespace ssg {
namespace {

using namespace tc;

constexpr int PT_ROWS = 128;                  // the node and up to 127 candidates
constexpr int GSLOTS = 3;                     // gather tiles
constexpr int TSLOTS = 3;                     // triangle slots, one per selection warp
constexpr int GRAM_WARPS = 4;
constexpr int THREADS_P = (2 + GRAM_WARPS + TSLOTS) * 32;
constexpr int TMEM_COLS_P = 512;              // 4 buffers of 128 fp32 columns
constexpr int TRI = 127 * 126 / 2;            // centred Gram entries (j, k), k < j < 127
constexpr int TSLOT_BYTES = 32768;            // TRI + 128 diagonal ints, rounded up

struct PtArgs {
  const int32_t* pool_id;
  const int32_t* pool_len;
  int64_t n;
  int L, R, kchunks;
  float cosA32, margin;
  double cosA64;
  int32_t* adj;
  int32_t* deg;
  unsigned long long* n64;
  int* err;
};

__device__ __forceinline__ int tri_row(int t) { return t * (t - 1) / 2; }

__global__ void __launch_bounds__(THREADS_P, 1)
k_prune_tc(const __grid_constant__ CUtensorMap tmX, PtArgs p) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* sm = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const uint32_t g_bytes = (uint32_t)p.kchunks * PT_ROWS * 128;
  unsigned char* sG = sm;                                       // GSLOTS gather tiles
  unsigned char* sT = sG + (size_t)GSLOTS * g_bytes;            // TSLOTS triangle slots
  int32_t* a_s = (int32_t*)(sT + (size_t)TSLOTS * TSLOT_BYTES);  // [2][128]: H_i0 per node
  uint64_t* bars = (uint64_t*)(a_s + 2 * PT_ROWS);
  uint64_t* g_full = bars;
  uint64_t* g_empty = g_full + GSLOTS;
  uint64_t* t_full = g_empty + GSLOTS;
  uint64_t* t_empty = t_full + 4;
  uint64_t* r_full = t_empty + 4;
  uint64_t* r_empty = r_full + TSLOTS;
  uint64_t* a_ready = r_empty + TSLOTS;
  uint32_t* tmem_slot = (uint32_t*)(a_ready + 2);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = lane_id();
  if (threadIdx.x == 0) {
    for (int s = 0; s < GSLOTS; ++s) {
      mbar_init(smem_u32(g_full + s), 1);
      mbar_init(smem_u32(g_empty + s), 1);
    }
    for (int b = 0; b < 4; ++b) {
      mbar_init(smem_u32(t_full + b), 1);
      mbar_init(smem_u32(t_empty + b), GRAM_WARPS);
    }
    for (int u = 0; u < TSLOTS; ++u) {
      mbar_init(smem_u32(r_full + u), GRAM_WARPS);
      mbar_init(smem_u32(r_empty + u), 1);
    }
    for (int k = 0; k < 2; ++k) mbar_init(smem_u32(a_ready + k), GRAM_WARPS);
    *abort_flag = 0;
    fence_barrier_init();
  }
  if (warp == 1) {
    tmem_alloc(smem_u32(tmem_slot), TMEM_COLS_P);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  const int64_t n = p.n;

  if (warp == 0) {
    // ---------------- gather producer ----------------
    int s = 0;
    uint32_t ph = 0;
    bool ok = true;
    for (int64_t x = blockIdx.x; x < n && ok; x += gridDim.x) {
      ok = mbar_wait(smem_u32(g_empty + s), ph ^ 1, abort_flag);
      if (!__all_sync(0xffffffffu, ok)) {
        ok = false;
        break;
      }
      const int len = min(p.pool_len[x], PT_ROWS - 1);
      const int ng4 = (len + 1 + 3) >> 2;
      if (lane == 0) mbar_expect_tx(smem_u32(g_full + s), (uint32_t)ng4 * 4 * 128 * p.kchunks);
      __syncwarp();
      if (lane < ng4) {
        int y[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int r = lane * 4 + e;  // row 0 is the node, row r the candidate r - 1
          y[e] = (r == 0 || r > len) ? (int)x : p.pool_id[x * p.L + r - 1];
        }
        unsigned char* dst = sG + (size_t)s * g_bytes + (size_t)lane * 4 * 128;
        for (int kc = 0; kc < p.kchunks; ++kc)
          tma_gather4(smem_u32(dst + (size_t)kc * PT_ROWS * 128), &tmX, smem_u32(g_full + s),
                      kc * 64, y[0], y[1], y[2], y[3]);
      }
      if (++s == GSLOTS) {
        s = 0;
        ph ^= 1;
      }
    }
    if (!ok && lane == 0) {
      atomicOr(p.err, 1);
      *abort_flag = 1;
    }
  } else if (warp == 1) {
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
  } else if (warp < 2 + GRAM_WARPS) {
    // ---------------- centred Gram: TMEM -> shared-memory triangle ----------------
    const int q = warp & 3;          // TMEM lane quadrant
    const int i = q * 32 + lane;     // row: 0 the node, i the candidate i - 1
    int b = 0, u = 0, k = 0;
    uint32_t tph = 0, uph = 0;
    bool ok = true;
    for (int64_t x = blockIdx.x; x < n; x += gridDim.x, ++k) {
      const int nrows = min(p.pool_len[x], PT_ROWS - 1) + 1;
      ok = mbar_wait(smem_u32(t_full + b), tph, abort_flag);
      if (!__all_sync(0xffffffffu, ok)) {
        ok = false;
        break;
      }
      tc_fence_after();
      const uint32_t taddr = tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(b * 128);
      int32_t* as = a_s + (k & 1) * PT_ROWS;
      uint32_t v[32];
      tmem_ld32(taddr, v);
      tmem_wait_ld(v);
      const int ai = __float2int_rn(__uint_as_float(v[0]));  // H_i0 = x.c
      as[i] = ai;
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(a_ready + (k & 1)));
      ok = mbar_wait(smem_u32(a_ready + (k & 1)), (uint32_t)((k >> 1) & 1), abort_flag) &&
           mbar_wait(smem_u32(r_empty + u), uph ^ 1, abort_flag);
      if (!__all_sync(0xffffffffu, ok)) {
        ok = false;
        break;
      }
      const int h00 = as[0];
      int32_t* tri = (int32_t*)(sT + (size_t)u * TSLOT_BYTES);
      int32_t* dg = tri + TRI;
      const bool row_ok = i >= 1 && i < nrows;
      const int toff = tri_row(i - 1) - 1;  // entry (i - 1, j - 1) at toff + j
      int hii = 0;
      for (int c = 0; c * 32 < nrows; ++c) {
        if (c > 0) {
          tmem_ld32(taddr + (uint32_t)(c * 32), v);
          tmem_wait_ld(v);
        }
#pragma unroll
        for (int e = 0; e < 32; ++e) {
          const int j = c * 32 + e;
          const int h = __float2int_rn(__uint_as_float(v[e]));
          if (j == i) hii = h;
          if (row_ok && j >= 1 && j < i) tri[toff + j] = h - ai - as[j] + h00;
        }
      }
      if (row_ok) dg[i - 1] = hii - 2 * ai + h00;
      tc_fence_before();
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(smem_u32(t_empty + b));
        mbar_arrive(smem_u32(r_full + u));
      }
      if (++b == 4) {
        b = 0;
        tph ^= 1;
      }
      if (++u == TSLOTS) {
        u = 0;
        uph ^= 1;
      }
    }
    if (!ok && lane == 0) {
      atomicOr(p.err, 4);
      *abort_flag = 1;
    }
  } else {
    // ---------------- selection: one warp per node, lanes over the kept edges ----------------
    const int u = warp - 2 - GRAM_WARPS;
    const int32_t* tri = (const int32_t*)(sT + (size_t)u * TSLOT_BYTES);
    const int32_t* dg = tri + TRI;
    uint32_t uph = 0;
    bool ok = true;
    unsigned long long fp64_tests = 0;
    const int R = p.R;
    for (int64_t x = blockIdx.x + (int64_t)u * gridDim.x; x < n; x += (int64_t)TSLOTS * gridDim.x) {
      ok = mbar_wait(smem_u32(r_full + u), uph, abort_flag);
      if (!__all_sync(0xffffffffu, ok)) {
        ok = false;
        break;
      }
      const int len = min(p.pool_len[x], PT_ROWS - 1);
      const int32_t* cand = p.pool_id + x * p.L;
      int kk[4], dk[4], gv[4];
      float sk[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        kk[r] = 0;
        dk[r] = 0;
        gv[r] = 0;
        sk[r] = 0.f;
      }
      int kept = 0;
      for (int t = 0; t < len && kept < R; ++t) {
        const int dgt = dg[t];
        const float st = sqrtf((float)dgt);
        const int32_t* trow = tri + tri_row(t);
        bool definite = false;
        unsigned border = 0;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          if (lane + 32 * r < kept) {
            const int g = trow[kk[r]];
            gv[r] = g;
            if (dgt == 0 || dk[r] == 0) {
              border |= 1u << r;
            } else {
              const float c = (float)g / (st * sk[r]);
              if (c > p.cosA32 + p.margin)
                definite = true;
              else if (c >= p.cosA32 - p.margin)
                border |= 1u << r;
            }
          }
        }
        bool conflict = __any_sync(0xffffffffu, definite);
        if (!conflict && __any_sync(0xffffffffu, border != 0)) {
          bool c64 = false;
#pragma unroll
          for (int r = 0; r < 4; ++r) {
            if ((border >> r) & 1u) {
              if (cos_from_gram_f64((double)gv[r], (double)dgt, (double)dk[r]) > p.cosA64)
                c64 = true;
              ++fp64_tests;
            }
          }
          conflict = __any_sync(0xffffffffu, c64);
        }
        if (!conflict) {
#pragma unroll
          for (int r = 0; r < 4; ++r) {
            if (r == (kept >> 5) && lane == (kept & 31)) {
              kk[r] = t;
              dk[r] = dgt;
              sk[r] = st;
            }
          }
          ++kept;
        }
      }
      int32_t* out = p.adj + x * R;
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int e = lane + 32 * r;
        if (e < R) out[e] = e < kept ? cand[kk[r]] : -1;
      }
      if (lane == 0) p.deg[x] = kept;
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(r_empty + u));
      uph ^= 1;
    }
    if (fp64_tests) atomicAdd(p.n64, fp64_tests);
    if (!ok && lane == 0) {
      atomicOr(p.err, 8);
      *abort_flag = 1;
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
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

size_t prune_tc_smem(int kchunks) {
  return 1024 + (size_t)GSLOTS * kchunks * PT_ROWS * 128 + (size_t)TSLOTS * TSLOT_BYTES +
         2 * PT_ROWS * sizeof(int32_t) +
         sizeof(uint64_t) * (2 * GSLOTS + 8 + 2 * TSLOTS + 2) + 16;
}

}  // namespace

bool prune_tc_available(int d, int L, int R) {
  const int kchunks = (d + 63) / 64;
  return knn_tc_available(d) && kchunks <= 2 && L >= 1 && L <= PT_ROWS - 1 && R >= 1 &&
         R <= 128 && prune_tc_smem(kchunks) <= 225 * 1024;
}

void prune_run_tc(const float* X, int ld, int d, int64_t n, const int32_t* pool_id,
                  const int32_t* pool_len, int L, int R, double cos_a, int32_t* adj,
                  int32_t* deg, Counters* dctr, cudaStream_t st) {
  const int dp = (d + 63) & ~63;
  const int kchunks = dp / 64;
  Scratch<__nv_bfloat16> xb((size_t)n * dp, st);
  SSG_LAUNCH(k_rows_bf16, 8 * num_sms(), 256, 0, st, X, n, d, ld, xb.p, dp);
  const CUtensorMap mx = make_map(xb.p, n, dp, 64, 1, CU_TENSOR_MAP_SWIZZLE_128B);
  Scratch<int> err(1, st);
  SSG_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), st));
  PtArgs a{};
  a.pool_id = pool_id;
  a.pool_len = pool_len;
  a.n = n;
  a.L = L;
  a.R = R;
  a.kchunks = kchunks;
  a.cosA32 = (float)cos_a;
  a.cosA64 = cos_a;
  a.margin = (float)(16.0 * U32);
  a.adj = adj;
  a.deg = deg;
  a.n64 = &dctr->angle_fp64;
  a.err = err.p;
  const size_t smem = prune_tc_smem(kchunks);
  static size_t attr = 0;
  if (smem > attr) {
    SSG_CUDA(cudaFuncSetAttribute(k_prune_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    attr = smem;
  }
  const int grid = (int)std::min<int64_t>(n, num_sms());
  SSG_LAUNCH(k_prune_tc, grid, THREADS_P, smem, st, mx, a);
  int h = 0;
  SSG_CUDA(cudaMemcpyAsync(&h, err.p, sizeof(int), cudaMemcpyDeviceToHost, st));
  SSG_CUDA(cudaStreamSynchronize(st));
  SSG_REQUIRE(h == 0, SSG_ETIMEOUT, "tensor-core prune: a pipeline wait timed out (code %d)", h);
}

}  // namespace ssg
