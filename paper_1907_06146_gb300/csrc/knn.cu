// Exact k-nearest-neighbour graph and brute-force ground truth (sm_103a).
//
// Alg. 3 starts from a kNN graph; the graph built here is the exact one: for every row
// i, the K nearest rows j != i by (squared distance, id).  The same machinery serves
// the ground truth of Sec. 5.2 (queries against the base, no self exclusion).
//
// Pass 1 (k_knn_select_fp32): a single-precision SIMT distance GEMM,
//   d2(i, j) ~= |x_i|^2 + |y_j|^2 - 2 x_i . y_j,
// 128 x 128 tiles, fused with a streaming top-KS selection per row: each row keeps a
// threshold tau (the KS-th smallest value seen) and appends every value below tau to a
// per-row buffer in global scratch (L2 resident); a full buffer is compacted by a
// warp-wide bitonic sort in registers.  Columns are visited in increasing id order, so
// "value < tau" also resolves equal distances by id.
// When the data are small integers (every partial sum below 2^24) the pass is exact and
// KS = K.  Otherwise KS = K + slack, and
// Pass 2 (k_knn_rerank) recomputes the KS candidates in double precision, sorts them by
// (d2, id) and certifies the K-th against the pass-1 threshold minus a rigorous error
// bound of the single-precision GEMM form.  Rows that fail certification are recomputed
// exhaustively (k_knn_fallback).
#include "common.cuh"
#include "knn.cuh"
#include "knn_select.cuh"

namespace ssg {

// ---------------------------------------------------------------------------------------
// Ingest: row norms and facts about the data.
// ---------------------------------------------------------------------------------------
__global__ void k_row_stats(const float* __restrict__ X, int64_t n, int d, int ld,
                            float* __restrict__ norms, unsigned* __restrict__ max_norm_bits,
                            unsigned* __restrict__ max_abs_bits, int* __restrict__ non_integer,
                            int* __restrict__ negative) {
  int64_t row = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (row >= n) return;
  const int lane = lane_id();
  const float* x = X + row * ld;
  float s = 0.f, mx = 0.f;
  int bad = 0, neg = 0;
  for (int t = lane; t < d; t += 32) {
    float v = x[t];
    s = fmaf(v, v, s);
    mx = fmaxf(mx, fabsf(v));
    bad |= (v != rintf(v));
    neg |= (v < 0.f);
  }
  for (int o = 16; o > 0; o >>= 1) {
    s += __shfl_xor_sync(0xffffffffu, s, o);
    mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    bad |= __shfl_xor_sync(0xffffffffu, bad, o);
    neg |= __shfl_xor_sync(0xffffffffu, neg, o);
  }
  if (lane == 0) {
    if (norms) norms[row] = s;
    atomicMax(max_norm_bits, __float_as_uint(sqrtf(s)));
    atomicMax(max_abs_bits, __float_as_uint(mx));
    if (bad) atomicOr(non_integer, 1);
    if (neg) atomicOr(negative, 1);
  }
}

__global__ void k_pad_copy(const float* __restrict__ X, int64_t n, int d, float* __restrict__ Y,
                           int ld) {
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t total = n * ld;
  for (; idx < total; idx += (int64_t)gridDim.x * blockDim.x) {
    int64_t r = idx / ld;
    int c = (int)(idx - r * ld);
    Y[idx] = c < d ? X[r * d + c] : 0.f;
  }
}

// ---------------------------------------------------------------------------------------
// Pass 1: distance GEMM + streaming top-KS per row.
// ---------------------------------------------------------------------------------------
namespace {
constexpr int BM = 128, BN = 128, BK = 16;
constexpr int LDA_S = BM + 4;  // padded shared-memory row lengths (16-byte multiples)
constexpr int LDD_S = BN + 4;
constexpr int THREADS = 256;
constexpr int WARPS = THREADS / 32;
}  // namespace

size_t knn_select_smem_bytes() {
  return sizeof(float) * (2 * BK * LDA_S * 2 + BM * LDD_S + BN) + sizeof(float) * BM +
         sizeof(int) * BM;
}

template <int C>
__global__ void __launch_bounds__(THREADS, 2)
k_knn_select_fp32(const float* __restrict__ A, int64_t na, int lda,
                  const float* __restrict__ B, int64_t nb, int ldb, int d,
                  const float* __restrict__ a_norm, const float* __restrict__ b_norm,
                  int self_exclude, int KS, uint64_t* __restrict__ rowbuf,
                  int direct_K, int32_t* __restrict__ out_id, float* __restrict__ out_d2,
                  uint64_t* __restrict__ out_keys, float* __restrict__ out_thresh) {
  extern __shared__ __align__(16) float smem[];
  float* As = smem;                          // [2][BK][LDA_S]
  float* Bs = As + 2 * BK * LDA_S;           // [2][BK][LDA_S]
  float* Ds = Bs + 2 * BK * LDA_S;           // [BM][LDD_S]
  float* ny = Ds + BM * LDD_S;               // [BN]
  float* tau = ny + BN;                      // [BM]
  int* cnt = (int*)(tau + BM);               // [BM]

  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int warp = tid >> 5, lane = lane_id();
  uint64_t* mybuf = rowbuf + (size_t)blockIdx.x * BM * C;
  const int64_t nrb = (na + BM - 1) / BM, ncb = (nb + BN - 1) / BN;
  const int nk = (d + BK - 1) / BK;
  const float INF = __int_as_float(0x7f800000);

  for (int64_t rb = blockIdx.x; rb < nrb; rb += gridDim.x) {
    const int64_t i0 = rb * BM;
    for (int r = tid; r < BM; r += THREADS) {
      tau[r] = INF;
      cnt[r] = 0;
    }
    float nx[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      int64_t gi = i0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + i - 4);
      nx[i] = gi < na ? a_norm[gi] : 0.f;
    }
    __syncthreads();

    for (int64_t cb = 0; cb < ncb; ++cb) {
      const int64_t j0 = cb * BN;
      if (tid < BN) ny[tid] = (j0 + tid < nb) ? b_norm[j0 + tid] : 0.f;

      float acc[8][8];
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;

      float4 ra[2], rb4[2];
      auto load = [&](int k0) {
#pragma unroll
        for (int r = 0; r < 2; ++r) {
          int f = tid + THREADS * r;
          int row = f >> 2, kq = f & 3;
          int kk = k0 + kq * 4;
          int64_t gi = i0 + row, gj = j0 + row;
          ra[r] = (gi < na && kk < d) ? __ldg((const float4*)(A + gi * lda + kk))
                                      : make_float4(0.f, 0.f, 0.f, 0.f);
          rb4[r] = (gj < nb && kk < d) ? __ldg((const float4*)(B + gj * ldb + kk))
                                       : make_float4(0.f, 0.f, 0.f, 0.f);
        }
      };
      auto store = [&](int buf) {
        float* as = As + buf * BK * LDA_S;
        float* bs = Bs + buf * BK * LDA_S;
#pragma unroll
        for (int r = 0; r < 2; ++r) {
          int f = tid + THREADS * r;
          int row = f >> 2, kq = f & 3;
          as[(kq * 4 + 0) * LDA_S + row] = ra[r].x;
          as[(kq * 4 + 1) * LDA_S + row] = ra[r].y;
          as[(kq * 4 + 2) * LDA_S + row] = ra[r].z;
          as[(kq * 4 + 3) * LDA_S + row] = ra[r].w;
          bs[(kq * 4 + 0) * LDA_S + row] = rb4[r].x;
          bs[(kq * 4 + 1) * LDA_S + row] = rb4[r].y;
          bs[(kq * 4 + 2) * LDA_S + row] = rb4[r].z;
          bs[(kq * 4 + 3) * LDA_S + row] = rb4[r].w;
        }
      };

      load(0);
      store(0);
      __syncthreads();
      for (int kt = 0; kt < nk; ++kt) {
        if (kt + 1 < nk) load((kt + 1) * BK);
        const float* as = As + (kt & 1) * BK * LDA_S;
        const float* bs = Bs + (kt & 1) * BK * LDA_S;
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
          float4 a0 = *(const float4*)(as + kk * LDA_S + ty * 4);
          float4 a1 = *(const float4*)(as + kk * LDA_S + 64 + ty * 4);
          float4 b0 = *(const float4*)(bs + kk * LDA_S + tx * 4);
          float4 b1 = *(const float4*)(bs + kk * LDA_S + 64 + tx * 4);
          float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
          float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
          for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        if (kt + 1 < nk) store((kt + 1) & 1);
        __syncthreads();
      }

      // Epilogue: distances into the shared tile.
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int rr = i < 4 ? ty * 4 + i : 64 + ty * 4 + i - 4;
        const int64_t gi = i0 + rr;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          float o[4];
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const int cc = h * 64 + tx * 4 + j;
            const int64_t gj = j0 + cc;
            float v = fmaf(-2.f, acc[i][h * 4 + j], nx[i] + ny[cc]);
            if (gj >= nb || gi >= na || (self_exclude && gj == gi)) v = INF;
            o[j] = v;
          }
          *(float4*)(Ds + rr * LDD_S + h * 64 + tx * 4) = make_float4(o[0], o[1], o[2], o[3]);
        }
      }
      __syncthreads();

      // Selection: warp w owns rows w, w + 8, ...
      for (int rr = warp; rr < BM; rr += WARPS) {
        float t = tau[rr];
        int c0 = cnt[rr];
        uint64_t* buf = mybuf + (size_t)rr * C;
#pragma unroll
        for (int q = 0; q < BN / 32; ++q) {
          const int cc = q * 32 + lane;
          const float v = Ds[rr * LDD_S + cc];
          const bool pass = v < t;
          const unsigned m = __ballot_sync(0xffffffffu, pass);
          if (pass) buf[c0 + __popc(m & lanemask_lt())] = make_key(v, (int32_t)(j0 + cc));
          c0 += __popc(m);
        }
        if (c0 > C - BN) {
          __syncwarp();
          c0 = compact_row<C>(buf, c0, KS, &t);
        }
        if (lane == 0) {
          tau[rr] = t;
          cnt[rr] = c0;
        }
      }
      __syncthreads();
    }

    // Final compaction and output.
    for (int rr = warp; rr < BM; rr += WARPS) {
      const int64_t gi = i0 + rr;
      float t;
      uint64_t* buf = mybuf + (size_t)rr * C;
      __syncwarp();
      int c0 = compact_row<C>(buf, cnt[rr], KS, &t);
      if (gi < na) {
        if (direct_K > 0) {
          for (int e = lane; e < direct_K; e += 32) {
            uint64_t k = e < c0 ? buf[e] : KEY_NONE;
            out_id[gi * direct_K + e] = k == KEY_NONE ? -1 : key_id(k);
            out_d2[gi * direct_K + e] = k == KEY_NONE ? INF : key_dist(k);
          }
        } else {
          for (int e = lane; e < KS; e += 32) out_keys[gi * KS + e] = e < c0 ? buf[e] : KEY_NONE;
          if (lane == 0) out_thresh[gi] = t;
        }
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------------------
// Pass 2: double-precision re-rank and certification (single-precision GEMM form).
// ---------------------------------------------------------------------------------------
// Pairwise bitonic sort of (double d, int id) by one warp in shared memory.
__device__ __forceinline__ void warp_sort_pairs(double* dv, int32_t* iv, int m) {
  const int lane = lane_id();
  for (int k = 2; k <= m; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = lane; i < m; i += 32) {
        int p = i ^ j;
        if (p > i) {
          double a = dv[i], b = dv[p];
          int32_t ia = iv[i], ib = iv[p];
          bool gt = (a > b) || (a == b && (uint32_t)ia > (uint32_t)ib);
          bool up = (i & k) == 0;
          if (gt == up) {
            dv[i] = b;
            dv[p] = a;
            iv[i] = ib;
            iv[p] = ia;
          }
        }
      }
      __syncwarp();
    }
  }
}

__global__ void k_knn_rerank(const float* __restrict__ A, int lda, const float* __restrict__ B,
                             int ldb, int d, int64_t na, const uint64_t* __restrict__ keys,
                             const float* __restrict__ thresh, int KS, int K,
                             const float* __restrict__ a_norm, float b_max_norm,
                             int32_t* __restrict__ out_id, float* __restrict__ out_d2,
                             int32_t* __restrict__ fb_rows, double* __restrict__ fb_kth,
                             int* __restrict__ fb_count, int KSP, int certify) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  const int wpb = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = lane_id();
  double* dv = (double*)sm_raw + (size_t)warp * KSP;
  int32_t* iv = (int32_t*)((double*)sm_raw + (size_t)wpb * KSP) + (size_t)warp * KSP;
  const int64_t row = (int64_t)blockIdx.x * wpb + warp;
  if (row >= na) return;
  const float* a = A + row * lda;
  for (int e = lane; e < KSP; e += 32) {
    uint64_t k = e < KS ? keys[row * KS + e] : KEY_NONE;
    if (k == KEY_NONE) {
      dv[e] = __longlong_as_double(0x7ff0000000000000ll);
      iv[e] = -1;
    } else {
      int32_t j = key_id(k);
      dv[e] = dist2_f64(a, B + (int64_t)j * ldb, d);
      iv[e] = j;
    }
  }
  __syncwarp();
  warp_sort_pairs(dv, iv, KSP);
  for (int e = lane; e < K; e += 32) {
    out_id[row * K + e] = iv[e];
    out_d2[row * K + e] = (float)dv[e];
  }
  if (lane == 0) {
    const float t = thresh[row];
    if (certify && !isinf(t)) {
      // |d2_gemm - d2| <= (D + 4) u (|a| + |b|)^2 (with a 1% margin) for the
      // single-precision GEMM form with sequential fused multiply-adds.
      double an = sqrt((double)a_norm[row]);
      double e = (d + 4) * U32 * 1.01 * (an + (double)b_max_norm) * (an + (double)b_max_norm);
      e = e * 1.01 + 1e-30;
      if (!(dv[K - 1] < (double)t - e)) {
        int s = atomicAdd(fb_count, 1);
        fb_rows[s] = (int32_t)row;
        fb_kth[s] = dv[K - 1];
      }
    }
  }
}

// Exhaustive double-precision recomputation of flagged rows: every column whose
// single-precision direct distance could be <= the K-th re-ranked value is recomputed in
// double and collected; the collected set is sorted by (d2, id).
__global__ void k_knn_fallback(const float* __restrict__ A, int lda, const float* __restrict__ B,
                               int ldb, int d, int64_t nb, int self_exclude,
                               const int32_t* __restrict__ fb_rows,
                               const double* __restrict__ fb_kth, int K, int cap,
                               int32_t* __restrict__ out_id, float* __restrict__ out_d2,
                               int* __restrict__ overflow) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  double* dv = (double*)sm_raw;
  int32_t* iv = (int32_t*)(dv + cap);
  __shared__ int count;
  const int64_t row = fb_rows[blockIdx.x];
  const double bound = fb_kth[blockIdx.x];
  const float* a = A + row * lda;
  const double rel = (d + 4) * U32 * 1.01;
  if (threadIdx.x == 0) count = 0;
  __syncthreads();
  for (int64_t j = threadIdx.x; j < nb; j += blockDim.x) {
    if (self_exclude && j == row) continue;
    const float* b = B + j * ldb;
    float s = 0.f;
    for (int t = 0; t < d; ++t) {
      float u = a[t] - b[t];
      s = fmaf(u, u, s);
    }
    if ((double)s <= bound * (1.0 + rel) + 1e-30) {
      double e = dist2_f64(a, b, d);
      if (e <= bound) {
        int p = atomicAdd(&count, 1);
        if (p < cap) {
          dv[p] = e;
          iv[p] = (int32_t)j;
        }
      }
    }
  }
  __syncthreads();
  const int m = count < cap ? count : cap;
  if (count > cap && threadIdx.x == 0) atomicOr(overflow, 1);
  int mp = 1;
  while (mp < m) mp <<= 1;
  for (int i = m + threadIdx.x; i < mp; i += blockDim.x) {
    dv[i] = __longlong_as_double(0x7ff0000000000000ll);
    iv[i] = -1;
  }
  __syncthreads();
  for (int k = 2; k <= mp; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < mp; i += blockDim.x) {
        int p = i ^ j;
        if (p > i) {
          double x = dv[i], y = dv[p];
          int32_t ix = iv[i], iy = iv[p];
          bool gt = (x > y) || (x == y && (uint32_t)ix > (uint32_t)iy);
          bool up = (i & k) == 0;
          if (gt == up) {
            dv[i] = y;
            dv[p] = x;
            iv[i] = iy;
            iv[p] = ix;
          }
        }
      }
      __syncthreads();
    }
  }
  for (int e = threadIdx.x; e < K; e += blockDim.x) {
    out_id[row * K + e] = e < m ? iv[e] : -1;
    out_d2[row * K + e] = e < m ? (float)dv[e] : __int_as_float(0x7f800000);
  }
}

void knn_fallback_rows(const float* A, int lda, const float* B, int ldb, int d, int64_t nb,
                       int self, const int32_t* rows, const double* kth, int count, int K,
                       int32_t* out_id, float* out_d2, cudaStream_t st) {
  if (count <= 0) return;
  const int cap = 4096;
  const size_t smem_fb = (size_t)cap * (sizeof(double) + sizeof(int32_t));
  ensure_smem((const void*)k_knn_fallback, smem_fb);
  Scratch<int> ovf(1, st);
  SSG_CUDA(cudaMemsetAsync(ovf.p, 0, sizeof(int), st));
  SSG_LAUNCH(k_knn_fallback, count, 256, smem_fb, st, A, lda, B, ldb, d, nb, self, rows, kth, K, cap,
             out_id, out_d2, ovf.p);
  int h = 0;
  SSG_CUDA(cudaMemcpyAsync(&h, ovf.p, sizeof(int), cudaMemcpyDeviceToHost, st));
  SSG_CUDA(cudaStreamSynchronize(st));
  if (h) note_device_status(SSG_EINTERNAL);
  SSG_REQUIRE(h == 0, SSG_EINTERNAL,
              "kNN fallback: more than %d columns tie with a row's K-th distance", cap);
}

// ---------------------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------------------
void pad_rows(const float* X, int64_t n, int d, cudaStream_t st, PaddedRows& out) {
  out.ld = (d + 3) & ~3;
  const bool aligned = ((uintptr_t)X & 15) == 0;
  if (out.ld == d && aligned) {
    out.p = X;
  } else {
    out.own.alloc((size_t)n * out.ld, st);
    int64_t total = n * out.ld;
    int grid = (int)std::min<int64_t>(ceil_div(total, 256), 8 * num_sms());
    SSG_LAUNCH(k_pad_copy, grid, 256, 0, st, X, n, d, out.own.p, out.ld);
    out.p = out.own.p;
  }
}

void ingest(const float* X, int64_t n, int d, cudaStream_t st, PaddedRows& out, float* norms,
            DataInfo* info) {
  pad_rows(X, n, d, st, out);
  Scratch<unsigned> facts(4, st);
  SSG_CUDA(cudaMemsetAsync(facts.p, 0, 4 * sizeof(unsigned), st));
  SSG_LAUNCH(k_row_stats, (unsigned)ceil_div(n, 8), 256, 0, st, out.p, n, d, out.ld, norms,
             facts.p, facts.p + 1, (int*)facts.p + 2, (int*)facts.p + 3);
  unsigned h[4];
  SSG_CUDA(cudaMemcpyAsync(h, facts.p, sizeof(h), cudaMemcpyDeviceToHost, st));
  SSG_CUDA(cudaStreamSynchronize(st));
  float mn, ma;
  memcpy(&mn, &h[0], 4);
  memcpy(&ma, &h[1], 4);
  info->max_norm = mn;
  info->max_abs = ma;
  info->nonneg = h[3] == 0;
  info->exact = (h[2] == 0) && exact_bound(d, ma, info->nonneg);
  info->bf16_exact = info->exact && ma <= 256.f;
}

template <int C>
static void launch_select(const float* A, int64_t na, int lda, const float* B, int64_t nb,
                          int ldb, int d, const float* an, const float* bn, int self, int KS,
                          int direct_K, int32_t* out_id, float* out_d2, uint64_t* out_keys,
                          float* out_thresh, cudaStream_t st) {
  const size_t smem = knn_select_smem_bytes();
  ensure_smem((const void*)k_knn_select_fp32<C>, smem);
  const int64_t nrb = ceil_div(na, BM);
  const int grid = (int)std::min<int64_t>(nrb, 2 * num_sms());
  Scratch<uint64_t> rowbuf((size_t)grid * BM * C, st);
  SSG_LAUNCH(k_knn_select_fp32<C>, grid, THREADS, smem, st, A, na, lda, B, nb, ldb, d, an, bn,
             self, KS, rowbuf.p, direct_K, out_id, out_d2, out_keys, out_thresh);
}

static void select_dispatch(const float* A, int64_t na, int lda, const float* B, int64_t nb,
                            int ldb, int d, const float* an, const float* bn, int self, int KS,
                            int direct_K, int32_t* out_id, float* out_d2, uint64_t* out_keys,
                            float* out_thresh, cudaStream_t st) {
  if (KS + BN <= 256)
    launch_select<256>(A, na, lda, B, nb, ldb, d, an, bn, self, KS, direct_K, out_id, out_d2,
                       out_keys, out_thresh, st);
  else if (KS + BN <= 512)
    launch_select<512>(A, na, lda, B, nb, ldb, d, an, bn, self, KS, direct_K, out_id, out_d2,
                       out_keys, out_thresh, st);
  else
    launch_select<1024>(A, na, lda, B, nb, ldb, d, an, bn, self, KS, direct_K, out_id, out_d2,
                        out_keys, out_thresh, st);
}

KnnResult knn_exact(const float* A, int64_t na, int lda, const float* a_norm, const float* B,
                    int64_t nb, int ldb, const float* b_norm, int d, const DataInfo& info,
                    int self, int K, int32_t* out_id, float* out_d2, cudaStream_t st,
                    StageTimer* gemm_timer) {
  KnnResult res;
  if (info.exact) {
    if (gemm_timer) gemm_timer->start();
    select_dispatch(A, na, lda, B, nb, ldb, d, a_norm, b_norm, self, K, K, out_id, out_d2,
                    nullptr, nullptr, st);
    if (gemm_timer) gemm_timer->stop();
    return res;
  }
  // slack: enough room for near-boundary ties of the approximate values
  int64_t avail = self ? nb - 1 : nb;
  int KS = K + std::max(8, K / 4);
  KS = (int)std::min<int64_t>(KS, std::min<int64_t>(avail, 1024 - BN));
  if (KS < K) KS = K;
  Scratch<uint64_t> keys((size_t)na * KS, st);
  Scratch<float> thresh((size_t)na, st);
  if (gemm_timer) gemm_timer->start();
  select_dispatch(A, na, lda, B, nb, ldb, d, a_norm, b_norm, self, KS, 0, nullptr, nullptr,
                  keys.p, thresh.p, st);
  if (gemm_timer) gemm_timer->stop();
  Scratch<int32_t> fb_rows((size_t)na, st);
  Scratch<double> fb_kth((size_t)na, st);
  Scratch<int> fb_count(2, st);
  SSG_CUDA(cudaMemsetAsync(fb_count.p, 0, 2 * sizeof(int), st));
  const int KSP = next_pow2(KS);
  const int wpb = 4;
  const size_t smem = (size_t)wpb * KSP * (sizeof(double) + sizeof(int32_t));
  SSG_LAUNCH(k_knn_rerank, (unsigned)ceil_div(na, wpb), wpb * 32, smem, st, A, lda, B, ldb, d,
             na, keys.p, thresh.p, KS, K, a_norm, info.max_norm, out_id, out_d2, fb_rows.p,
             fb_kth.p, fb_count.p, KSP, (int)(KS < avail));
  int nfb = 0;
  SSG_CUDA(cudaMemcpyAsync(&nfb, fb_count.p, sizeof(int), cudaMemcpyDeviceToHost, st));
  SSG_CUDA(cudaStreamSynchronize(st));
  res.fallback_rows = nfb;
  if (nfb > 0) {
    const int cap = 4096;
    const size_t smem_fb = (size_t)cap * (sizeof(double) + sizeof(int32_t));
    ensure_smem((const void*)k_knn_fallback, smem_fb);
    SSG_LAUNCH(k_knn_fallback, nfb, 256, smem_fb, st, A, lda, B, ldb, d, nb, self, fb_rows.p,
               fb_kth.p, K, cap, out_id, out_d2, fb_count.p + 1);
    int ovf = 0;
    SSG_CUDA(cudaMemcpyAsync(&ovf, fb_count.p + 1, sizeof(int), cudaMemcpyDeviceToHost, st));
    SSG_CUDA(cudaStreamSynchronize(st));
    if (ovf) note_device_status(SSG_EINTERNAL);
    SSG_REQUIRE(ovf == 0, SSG_EINTERNAL,
                "kNN fallback: more than %d columns tie with a row's K-th distance", cap);
  }
  return res;
}

}  // namespace ssg
