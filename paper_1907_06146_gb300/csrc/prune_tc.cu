// SSG prune (Alg. 2 selection applied to every pool, Alg. 3) with the pool's Gram matrix
// on the 5th-generation tensor cores, for integer data that bf16 holds exactly.
//
// For node x with candidates c_1..c_m (m <= 127) the 128 rows [x, c_1, .., c_m, ..] are
// gathered into shared memory (TMA gather4, 128-byte swizzle) and one 128x128xd UMMA gives
// H = C C^T in TMEM.  Every product and partial sum is an integer below 2^24, so H is
// exact, and so is every centred dot product the angle rule needs:
//     G_jk = (c_j - x).(c_k - x) = H_jk - H_j0 - H_k0 + H_00,   G_jj = d2(x, c_j).
// All pairs are tested at once: bit k of row j says whether cos(j, k) = G_jk / sqrt(G_jj
// G_kk) > cos(alpha) (0 for a zero-length edge).  The fp32 cosine decides where it is more
// than 16 units of roundoff (plus the reporting band) from cos(alpha) (its inputs are
// exact, its error a few units); otherwise the bit is taken in fp64 from the same exact integers with the operations of
// the definition, which reproduces the double-precision rule bit for bit.  The selection
// in candidate order (keep c_j unless it conflicts with a kept c_k, stop at R) is then a
// scan over these bit rows.
//
// Persistent kernel, one CTA per SM, 13 warps:
//   warp 0       gathers the node and candidate rows (gather4, 4 rows per TMA) into one
//                of GSLOTS shared-memory tiles;
//   warp 1       allocates 512 TMEM columns and issues the Gram UMMAs into one of 4 TMEM
//                buffers;
//   warps 2..9   conflict bits: two warps per TMEM lane quadrant (one row per lane), each
//                taking every other 32-column chunk left of the diagonal;
//   warps 10..12 select: each takes every third node.
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
constexpr int SEL_WARPS = 3;
constexpr int MSLOTS = 6;                     // conflict-bit slots (a multiple of SEL_WARPS)
constexpr int GRAM_WARPS = 8;
constexpr int THREADS_P = (2 + GRAM_WARPS + SEL_WARPS) * 32;
constexpr int TMEM_COLS_P = 512;              // 4 buffers of 128 fp32 columns
constexpr int MSLOT_BYTES = PT_ROWS * 4 * 4;  // 4 words of conflict bits per row
constexpr int XCH_FLOATS = 4 * PT_ROWS;       // per node: H_i0, H_ii, d2(x, c_i), 1/sqrt

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
  double border;                // fp64 cosines within this of cos(alpha) are counted
  unsigned long long* nborder;
};

__global__ void __launch_bounds__(THREADS_P, 1)
k_prune_tc(const __grid_constant__ CUtensorMap tmX, PtArgs p) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* sm = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const uint32_t g_bytes = (uint32_t)p.kchunks * PT_ROWS * 128;
  unsigned char* sG = sm;                                            // GSLOTS gather tiles
  uint32_t* sM = (uint32_t*)(sG + (size_t)GSLOTS * g_bytes);         // MSLOTS x [128][4] bits
  float* xch = (float*)(sM + (size_t)MSLOTS * PT_ROWS * 4);         // [2][4][128]
  uint32_t* xz = (uint32_t*)(xch + 2 * XCH_FLOATS);                  // [2][4] zero-edge bits
  float* stash = (float*)(xz + 8);                                   // 32 floats per thread
  uint64_t* bars = (uint64_t*)(stash + GRAM_WARPS * 32 * 32);
  uint64_t* g_full = bars;
  uint64_t* g_empty = g_full + GSLOTS;
  uint64_t* t_full = g_empty + GSLOTS;
  uint64_t* t_empty = t_full + 4;
  uint64_t* m_full = t_empty + 4;
  uint64_t* m_empty = m_full + MSLOTS;
  uint64_t* ex1 = m_empty + MSLOTS;
  uint64_t* ex2 = ex1 + 2;
  uint32_t* tmem_slot = (uint32_t*)(ex2 + 2);
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
    for (int u = 0; u < MSLOTS; ++u) {
      mbar_init(smem_u32(m_full + u), GRAM_WARPS);
      mbar_init(smem_u32(m_empty + u), 1);
    }
    for (int k = 0; k < 2; ++k) {
      mbar_init(smem_u32(ex1 + k), GRAM_WARPS);
      mbar_init(smem_u32(ex2 + k), GRAM_WARPS);
    }
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
    // ---------------- conflict bits: TMEM -> shared-memory bit rows ----------------
    const int q = warp & 3;                  // TMEM lane quadrant
    const int hh = (warp - 2) >> 2;          // which of the quadrant's two warps
    const int i = q * 32 + lane;             // row: 0 the node, i the candidate i - 1
    float* st = stash + (size_t)((warp - 2) * 32 + lane) * 32;
    const bool zc = 0.0 > p.cosA64;          // the rule for a zero-length edge
    const float hi = p.cosA32 + p.margin, lo = p.cosA32 - p.margin;
    int b = 0, u = 0, k = 0;
    uint32_t tph = 0, uph = 0;
    bool ok = true;
    unsigned long long fp64_tests = 0, borderline = 0;
    for (int64_t x = blockIdx.x; x < n; x += gridDim.x, ++k) {
      const int nrows = min(p.pool_len[x], PT_ROWS - 1) + 1;
      ok = mbar_wait(smem_u32(t_full + b), tph, abort_flag);
      if (!__all_sync(0xffffffffu, ok)) {
        ok = false;
        break;
      }
      tc_fence_after();
      const uint32_t taddr = tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(b * 128);
      float* xa = xch + (k & 1) * XCH_FLOATS;  // H_i0
      float* xh = xa + PT_ROWS;                // H_ii
      float* xd = xh + PT_ROWS;                // G_ii = d2(x, c_i)
      float* xr = xd + PT_ROWS;                // 1 / sqrt(G_ii)
      uint32_t* zq = xz + (k & 1) * 4;         // zero-length edges, one word per quadrant
      uint32_t v[32];
      tmem_ld32(taddr, v);
      tmem_wait_ld(v);
      const float ai = __uint_as_float(v[0]);
      if (q != 0) {
        tmem_ld32(taddr + (uint32_t)(q * 32), v);
        tmem_wait_ld(v);
      }
      float hii = 0.f;
#pragma unroll
      for (int e = 0; e < 32; ++e)
        if (e == lane) hii = __uint_as_float(v[e]);
      if (hh == 0) {
        xa[i] = ai;
        xh[i] = hii;
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(ex1 + (k & 1)));
      ok = mbar_wait(smem_u32(ex1 + (k & 1)), (uint32_t)((k >> 1) & 1), abort_flag);
      if (!__all_sync(0xffffffffu, ok)) {
        ok = false;
        break;
      }
      const float h00 = xa[0];
      const float dgi = (hii - 2.f * ai) + h00;  // exact: integers below 2^24
      const float ri = dgi > 0.f ? __frsqrt_rn(dgi) : 0.f;
      const uint32_t zb = __ballot_sync(0xffffffffu, dgi == 0.f);
      if (hh == 0) {
        xd[i] = dgi;
        xr[i] = ri;
        if (lane == 0) zq[q] = zb;
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(ex2 + (k & 1)));
      ok = mbar_wait(smem_u32(ex2 + (k & 1)), (uint32_t)((k >> 1) & 1), abort_flag) &&
           mbar_wait(smem_u32(m_empty + u), uph ^ 1, abort_flag);
      if (!__all_sync(0xffffffffu, ok)) {
        ok = false;
        break;
      }
      const float t2 = h00 - ai;
      const bool row_ok = i >= 1 && i < nrows;
      const bool zero_i = dgi == 0.f;
      uint32_t* mrow = sM + ((size_t)u * PT_ROWS + i) * 4;
      for (int c = hh; c <= q && c * 32 < nrows; c += 2) {
        tmem_ld32(taddr + (uint32_t)(c * 32), v);
        tmem_wait_ld(v);
        // columns j = 32c + e with 1 <= j < i
        const int lo_e = c == 0 ? 1 : 0;
        const int hi_e = i - c * 32;  // exclusive
        uint32_t valid = 0;
        if (row_ok && hi_e > lo_e)
          valid = (hi_e >= 32 ? 0xffffffffu : ((1u << hi_e) - 1u)) & ~((1u << lo_e) - 1u);
        uint32_t cf = 0, bd = 0;
#pragma unroll
        for (int e = 0; e < 32; ++e) {
          const int j = c * 32 + e;
          const float g = (__uint_as_float(v[e]) - xa[j]) + t2;  // exact centred dot product
          const float cs = g * ri * xr[j];
          cf |= (cs > hi ? 1u : 0u) << e;
          bd |= (cs >= lo && cs <= hi ? 1u : 0u) << e;
        }
        const uint32_t zcol = zq[c];
        if (zero_i) {
          cf = zc ? valid : 0u;
          bd = 0u;
        } else {
          cf = ((cf & ~zcol) | (zc ? zcol : 0u)) & valid;
          bd &= valid & ~zcol;
        }
        if (bd) {
          // near cos(alpha): the double-precision rule on the same exact integers
#pragma unroll
          for (int kq = 0; kq < 8; ++kq)
            *(float4*)(st + 4 * kq) = make_float4(__uint_as_float(v[4 * kq]), __uint_as_float(v[4 * kq + 1]),
                                                  __uint_as_float(v[4 * kq + 2]), __uint_as_float(v[4 * kq + 3]));
          while (bd) {
            const int e = __ffs(bd) - 1;
            bd &= bd - 1;
            const int j = c * 32 + e;
            const float g = (st[e] - xa[j]) + t2;
            const double c64 = cos_from_gram_f64((double)g, (double)dgi, (double)xd[j]);
            if (c64 > p.cosA64) cf |= 1u << e;
            if (fabs(c64 - p.cosA64) <= p.border) ++borderline;
            ++fp64_tests;
          }
        }
        mrow[c] = cf;
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(smem_u32(t_empty + b));
        mbar_arrive(smem_u32(m_full + u));
      }
      if (++b == 4) {
        b = 0;
        tph ^= 1;
      }
      if (++u == MSLOTS) {
        u = 0;
        uph ^= 1;
      }
    }
    if (fp64_tests) atomicAdd(p.n64, fp64_tests);
    if (borderline) atomicAdd(p.nborder, borderline);
    if (!ok && lane == 0) {
      atomicOr(p.err, 4);
      *abort_flag = 1;
    }
  } else {
    // ---------------- selection: candidate order over the bit rows ----------------
    const int sw = warp - 2 - GRAM_WARPS;
    int u = sw;
    uint32_t uph = 0;
    bool ok = true;
    const int R = p.R;
    for (int64_t x = blockIdx.x + (int64_t)sw * gridDim.x; x < n;
         x += (int64_t)SEL_WARPS * gridDim.x) {
      ok = mbar_wait(smem_u32(m_full + u), uph, abort_flag);
      if (!__all_sync(0xffffffffu, ok)) {
        ok = false;
        break;
      }
      const int nrows = min(p.pool_len[x], PT_ROWS - 1) + 1;
      const uint32_t* mrows = sM + (size_t)u * PT_ROWS * 4;
      // bit j of K: candidate j - 1 kept
      uint32_t K0 = 0, K1 = 0, K2 = 0, K3 = 0;
      int kept = 0;
      if (lane == 0) {
        for (int i = 1; i < nrows && kept < R; ++i) {
          const uint4 m = *(const uint4*)(mrows + (size_t)i * 4);
          if (((m.x & K0) | (m.y & K1) | (m.z & K2) | (m.w & K3)) == 0u) {
            const uint32_t bit = 1u << (i & 31);
            const int w = i >> 5;
            K0 |= w == 0 ? bit : 0u;
            K1 |= w == 1 ? bit : 0u;
            K2 |= w == 2 ? bit : 0u;
            K3 |= w == 3 ? bit : 0u;
            ++kept;
          }
        }
      }
      K0 = __shfl_sync(0xffffffffu, K0, 0);
      K1 = __shfl_sync(0xffffffffu, K1, 0);
      K2 = __shfl_sync(0xffffffffu, K2, 0);
      K3 = __shfl_sync(0xffffffffu, K3, 0);
      kept = __shfl_sync(0xffffffffu, kept, 0);
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(m_empty + u));
      const int32_t* cand = p.pool_id + x * p.L;
      int32_t* out = p.adj + x * R;
      const unsigned lt = lanemask_lt();
      const uint32_t Kw[4] = {K0, K1, K2, K3};
      int base = 0;
#pragma unroll
      for (int w = 0; w < 4; ++w) {
        if ((Kw[w] >> lane) & 1u) out[base + __popc(Kw[w] & lt)] = cand[w * 32 + lane - 1];
        base += __popc(Kw[w]);
      }
      for (int e = kept + lane; e < R; e += 32) out[e] = -1;
      if (lane == 0) p.deg[x] = kept;
      u += SEL_WARPS;
      if (u >= MSLOTS) {
        u -= MSLOTS;
        uph ^= 1;
      }
    }
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
  return 1024 + (size_t)GSLOTS * kchunks * PT_ROWS * 128 + (size_t)MSLOTS * MSLOT_BYTES +
         2 * XCH_FLOATS * sizeof(float) + 8 * sizeof(uint32_t) +
         (size_t)GRAM_WARPS * 32 * 32 * sizeof(float) +
         sizeof(uint64_t) * (2 * GSLOTS + 8 + 2 * MSLOTS + 4) + 16;
}

}  // namespace

bool prune_tc_available(int d, int L, int R) {
  const int kchunks = (d + 63) / 64;
  return knn_tc_available(d) && kchunks <= 2 && L >= 1 && L <= PT_ROWS - 1 && R >= 1 &&
         R <= 128 && prune_tc_smem(kchunks) <= 225 * 1024;
}

void prune_run_tc(const float* X, int ld, int d, int64_t n, const int32_t* pool_id,
                  const int32_t* pool_len, int L, int R, double cos_a, double border,
                  int32_t* adj, int32_t* deg, Counters* dctr, cudaStream_t st) {
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
  a.margin = (float)(16.0 * U32 + border);
  a.adj = adj;
  a.deg = deg;
  a.n64 = &dctr->angle_fp64;
  a.border = border;
  a.nborder = &dctr->angle_border;
  a.err = err.p;
  const size_t smem = prune_tc_smem(kchunks);
  ensure_smem((const void*)k_prune_tc, smem);
  const int grid = (int)std::min<int64_t>(n, num_sms());
  SSG_LAUNCH(k_prune_tc, grid, THREADS_P, smem, st, mx, a);
  int h = 0;
  SSG_CUDA(cudaMemcpyAsync(&h, err.p, sizeof(int), cudaMemcpyDeviceToHost, st));
  SSG_CUDA(cudaStreamSynchronize(st));
  if (h != 0) note_device_status(SSG_ETIMEOUT);
  SSG_REQUIRE(h == 0, SSG_ETIMEOUT, "tensor-core prune: a pipeline wait timed out (code %d)", h);
}

}  // namespace ssg
