// Exact kNN rows from the bf16 tensor cores on data that bf16 does not hold exactly
// (Alg. 3's kNN graph, and the serial-scan ground truth of Sec. 5.3, computed exactly).
//
// The rows are centred on the column mean mu before rounding (distances do not change
// under a translation, and centred rows have smaller norms, hence smaller rounding errors).
// The tensor-core kernel (knn_tc.cu) then keeps, per row, the KS columns with the smallest
// bf16 distance d2~ and the KS-th smallest value t.  For every column j,
//     |d2~(x, y_j) - d2(x, y_j)| <= E(x) = bf16_dist_bound(|x - mu|^2, max_j |y_j - mu|^2),
// (the rounding of both operands to bf16, the fp32 accumulation of the tensor cores, the
// fp32 norms and the centring; see the function), and a column that was not kept has
// d2~ >= t - s(x) (s: the rounding of the streaming threshold).  So the row is exact once
// the KS candidates are ordered exactly (fp32 distances from the original rows, runs of
// near-equal values re-sorted in fp64) and its K-th exact distance d2_(K) satisfies
//     d2_(K) < t - s(x) - E(x):
// no column outside the candidates can then be nearer than (or tie with) the K-th.
// Rows that fail take a second tensor-core pass with the largest candidate count, and
// the few that fail again the exact fp32 path.  KS itself only trades speed: it is sized
// from a seeded sample of rows (their exact K-th distance and the number of bf16
// distances below it plus the bound), so that a set fraction of rows certify.
#include <algorithm>
#include <cmath>
#include <vector>

#include <cuda_bf16.h>

#include "common.cuh"
#include "graph_dev.cuh"
#include "knn.cuh"

namespace ssg {

// Column sums in fp64: block (32, 8), column blockIdx.x * 32 + tx, rows strided over y.
__global__ void k_col_sum(const float* __restrict__ X, int64_t n, int d, int ld,
                          double* __restrict__ sum) {
  __shared__ double part[8][33];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int c = blockIdx.x * 32 + tx;
  double s = 0.0;
  if (c < d)
    for (int64_t r = (int64_t)blockIdx.y * 8 + ty; r < n; r += (int64_t)gridDim.y * 8)
      s += (double)X[r * ld + c];
  part[ty][tx] = s;
  __syncthreads();
  if (ty == 0 && c < d) {
    double t = 0.0;
    for (int k = 0; k < 8; ++k) t += part[k][tx];
    atomicAdd(sum + c, t);
  }
}

__global__ void k_col_mean(const double* __restrict__ sum, int d, int64_t n, float* __restrict__ mu) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < d) mu[c] = (float)(sum[c] / (double)n);
}

// Squared norms of the rows centred on mu (mu null: of the rows as given), with the same
// fp32 subtraction as the bf16 conversion; *max_bits receives the largest (as float bits).
__global__ void k_centred_norms(const float* __restrict__ X, int64_t n, int d, int ld,
                                const float* __restrict__ mu, float* __restrict__ norm,
                                unsigned* __restrict__ max_bits) {
  const int64_t row = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (row >= n) return;
  const int lane = lane_id();
  const float* x = X + row * ld;
  float s = 0.f;
  for (int t = lane; t < d; t += 32) {
    const float v = mu ? __fsub_rn(x[t], mu[t]) : x[t];
    s = fmaf(v, v, s);
  }
  s = warp_sum(s);
  if (lane == 0) {
    norm[row] = s;
    if (max_bits) atomicMax(max_bits, __float_as_uint(s));
  }
}

__global__ void k_gather_rows(const float* __restrict__ X, int ld, const int32_t* __restrict__ ids,
                              int64_t m, float* __restrict__ out) {
  const int64_t total = m * ld;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / ld;
    out[i] = X[(int64_t)ids[r] * ld + (i - r * ld)];
  }
}

__global__ void k_gather_vals(const float* __restrict__ v, const int32_t* __restrict__ ids, int64_t m,
                              float* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < m) out[i] = v[ids[i]];
}

// Upper bound on |d2~ - d2| for a row whose centred fp32 squared norm is nx, against any
// base row whose centred fp32 squared norm is at most ymax2 (d values, bf16 operands).
//  - bf16 rounding (8 significant bits, unit roundoff u = 2^-8) of both operands:
//    |x~ y~ - x y| <= (2u + u^2) |x y| per product, summed <= (2u + u^2) |x| |y|;
//  - the tensor cores' fp32 accumulation of the dp + 16 terms (the augmentation step adds
//    16, last): each added term charged at 2^-22 of the running sum's magnitude, four
//    times the error of a sequentially rounded fp32 sum and above any truncating alignment
//    of groups of 16 terms; the dp data terms run below (1 + u)^2 |x| |y|, the 16
//    augmentation terms below that plus (1 + 2u) |y|^2 / 2;
//  - the four bf16 parts of -|y|^2/2 (their sum misses it by at most 2^-28 |y|^2);
//  - the fp32 squared norms ((d + 2) u32 |.|^2 each) and |x|, |y| taken from them;
//  - the final fused multiply-add and the fp32 centring (x - mu rounded once per value):
//    4.2 u32 (|x| + |y|)^2 together.
// Every factor 2 on the dot product terms comes from d2 = |x|^2 + |y|^2 - 2 x.y.
// With bf16 pairs (pairs = 1: v = hi + lo + r, hi = bf16(v), lo = bf16(v - hi), so |r| <=
// u^2 |v| and |lo| <= u (1 + u) |v|) the products hi.hi + hi.lo + lo.hi miss x.y by at most
// (3u^2 + 2u^3 + 2u^4) |x| |y| (the product of the two pairs, less lo.lo).  The accumulation
// error is charged, as above, at 2^-22 of the running sum's magnitude per added term; the
// 2 dp cross terms come first (the MMAs run in K order), while that sum is below
// 2u (1 + u)^2 |x| |y|, so the 3 dp data terms together cost no more than dp terms at a
// running sum of (1 + u)^2 (1 + 6u) |x| |y|, as for a single bf16 with that magnitude.
__host__ __device__ inline double bf16_dist_bound(double nx, double ymax2, int d, int pairs) {
  const double u = 1.0 / 256.0, u32 = 5.9604644775390625e-08;
  const int dp = ((d + 63) / 64) * 64;
  const double g = 2.384185791015625e-07;  // 2^-22 per added term
  const double ax = sqrt(fmax(nx, 0.0) * (1.0 + (d + 2) * u32));
  const double ay = sqrt(fmax(ymax2, 0.0) * (1.0 + (d + 2) * u32));
  const double s = ax + ay;
  const double prod = pairs ? 3.0 * u * u + 2.0 * u * u * u + 2.0 * u * u * u * u : 2.0 * u + u * u;
  const double mag = pairs ? (1.0 + u) * (1.0 + u) * (1.0 + 6.0 * u) : (1.0 + u) * (1.0 + u);
  const double acc = g * ((dp + 16) * mag * ax * ay + 16.0 * 0.5 * (1.0 + 2.0 * u) * ay * ay);
  const double e = 2.0 * prod * ax * ay + 2.0 * acc + 4.0e-9 * ay * ay +
                   (d + 2) * u32 * (ax * ax + ay * ay) + 4.2 * u32 * s * s;
  return e * 1.05;
}

// How far below the final threshold t a column the kernel did not keep can lie: the
// streaming test compares acc with fp32 (|x|^2 - tau) / 2, rounded once.
__host__ __device__ inline double stream_slop(double nx, double t) {
  return 2.02 * 5.9604644775390625e-08 * (fabs(nx) + fabs(t)) + 1e-30;
}

// Calibration: for each sampled query row t, the number of base rows j (j != sid[t]) whose
// bf16 distance is at most lim[t].  One block of 256 threads walks tiles of CAL_TJ base
// rows; thread t owns sampled row t.  The dimensions go through in chunks of CAL_DC: the
// sampled rows' chunk (bf16 values, transposed) and the tile's chunk sit in shared memory
// (for rows of at most CAL_DC values the sample's chunk is loaded once).
constexpr int CAL_S = 256, CAL_TJ = 32, CAL_DC = 128;
// RAW: the centred values unrounded (fp32 distances; used to size KS for bf16 pairs, whose
// error is far below the band's width)
template <bool RAW>
__global__ void __launch_bounds__(CAL_S)
k_band_count(const float* __restrict__ As, int s, int lda, const float* __restrict__ B, int64_t nb,
             int ldb, int d, const float* __restrict__ mu, const float* __restrict__ nac,
             const float* __restrict__ nbc, const double* __restrict__ lim,
             const int32_t* __restrict__ sid, int* __restrict__ count) {
  extern __shared__ __align__(16) float csm[];
  float* Qt = csm;                        // [CAL_DC][CAL_S]
  float* Y = Qt + (size_t)CAL_DC * CAL_S; // [CAL_TJ][CAL_DC]
  const int t = threadIdx.x;
  const int nchunks = (d + CAL_DC - 1) / CAL_DC;
  auto load_q = [&](int c0) {
    for (int i = t; i < CAL_DC * CAL_S; i += CAL_S) {
      const int k = i / CAL_S, q = i - k * CAL_S;
      float v = 0.f;
      if (q < s && c0 + k < d) {
        v = __fsub_rn(As[(int64_t)q * lda + c0 + k], mu[c0 + k]);
        if (!RAW) v = __bfloat162float(__float2bfloat16_rn(v));
      }
      Qt[i] = v;
    }
  };
  if (nchunks == 1) load_q(0);
  const float nq = t < s ? nac[t] : 0.f;
  const double lq = t < s ? lim[t] : -1.0;
  const int32_t me = t < s && sid ? sid[t] : -1;
  int cnt = 0;
  for (int64_t j0 = (int64_t)blockIdx.x * CAL_TJ; j0 < nb; j0 += (int64_t)gridDim.x * CAL_TJ) {
    float acc[CAL_TJ];
#pragma unroll
    for (int r = 0; r < CAL_TJ; ++r) acc[r] = 0.f;
    for (int ch = 0; ch < nchunks; ++ch) {
      const int c0 = ch * CAL_DC;
      __syncthreads();
      if (nchunks > 1) load_q(c0);
      for (int i = t; i < CAL_TJ * CAL_DC; i += CAL_S) {
        const int r = i / CAL_DC, k = i - r * CAL_DC;
        const int64_t j = j0 + r;
        float v = 0.f;
        if (j < nb && c0 + k < d) {
          v = __fsub_rn(B[j * ldb + c0 + k], mu[c0 + k]);
          if (!RAW) v = __bfloat162float(__float2bfloat16_rn(v));
        }
        Y[i] = v;
      }
      __syncthreads();
      for (int k = 0; k < CAL_DC; k += 4) {
        const float q0 = Qt[(k + 0) * CAL_S + t], q1 = Qt[(k + 1) * CAL_S + t];
        const float q2 = Qt[(k + 2) * CAL_S + t], q3 = Qt[(k + 3) * CAL_S + t];
#pragma unroll
        for (int r = 0; r < CAL_TJ; ++r) {
          const float4 y = *(const float4*)(Y + r * CAL_DC + k);
          acc[r] = fmaf(q0, y.x, fmaf(q1, y.y, fmaf(q2, y.z, fmaf(q3, y.w, acc[r]))));
        }
      }
    }
    if (t < s) {
#pragma unroll
      for (int r = 0; r < CAL_TJ; ++r) {
        const int64_t j = j0 + r;
        if (j < nb && (int32_t)j != me && (double)nq + (double)nbc[j] - 2.0 * (double)acc[r] <= lq)
          ++cnt;
      }
    }
  }
  if (t < s && cnt) atomicAdd(count + t, cnt);
}

// lim[t] = the sampled row's exact K-th distance plus the bound (kth: [s][ld] rows of the
// exact kNN of the sample, the K-th distance in column col).
__global__ void k_band_limit(const float* __restrict__ d2, int ld, int col, int s,
                             const float* __restrict__ nac, double ymax2, int d, int pairs,
                             double widen, double* __restrict__ lim) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < s)
    lim[t] = (double)d2[(int64_t)t * ld + col] + widen * bf16_dist_bound(nac[t], ymax2, d, pairs);
}

// Exact order of each row's candidates and its certificate.  One warp per row r (rows:
// compact index -> row id, null = identity).  Of the candidates cand[r][0, KS) (-1
// padded) only those whose tensor-core distance cd2 lies within 2 E (plus the rounding of
// that value) of the K-th smallest one can be among the K nearest: K candidates lie at
// most at that K-th value plus E, any other candidate at least 2 E further minus E.  Those
// get fp32 distances from the original rows, are sorted by (d2, id), and runs of
// near-equal values up to position K are re-sorted in fp64; the first K go to row rows[r]
// of the output (d2 in fp64 rounded to float when exact_d2, else the fp32 value).  The row
// is certified when the K-th exact distance (bounded above through the fp32 value) lies
// below thr[r] - slop - E; otherwise it is listed in fb (with that bound) for another pass.
__global__ void k_knn_cert(const float* __restrict__ A, const float* __restrict__ B, int ld, int d,
                           const int32_t* __restrict__ rows, int64_t count,
                           const int32_t* __restrict__ cand, const float* __restrict__ cd2, int KS,
                           const float* __restrict__ thr,
                           const float* __restrict__ nac, double ymax2, int pairs, int K, int cap,
                           float rel, int exact_d2, int32_t* __restrict__ out_id,
                           float* __restrict__ out_d2,
                           int32_t* __restrict__ fb, double* __restrict__ fb_kth,
                           int* __restrict__ fb_count, unsigned long long* __restrict__ n_order) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  const int wpb = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = lane_id();
  uint64_t* keys = (uint64_t*)(sm_raw + (size_t)warp * cap * 16);
  double* d64 = (double*)(keys + cap);
  const int64_t r = (int64_t)blockIdx.x * wpb + warp;
  if (r >= count) return;
  const int64_t row = rows ? (int64_t)rows[r] : r;
  const float* xi = A + r * ld;
  int m = 0;
  for (int c = 0; c < KS; c += 32) {
    const int t = c + lane;
    const int32_t id = t < KS ? cand[r * KS + t] : -1;
    const bool v = id >= 0;
    const unsigned bal = __ballot_sync(0xffffffffu, v);
    if (v) keys[m + __popc(bal & lanemask_lt())] = make_key(cd2[r * KS + t], id);
    m += __popc(bal);
  }
  __syncwarp();
  int mp = 1;
  while (mp < m) mp <<= 1;
  for (int t = m + lane; t < mp; t += 32) keys[t] = KEY_NONE;
  __syncwarp();
  if (m > K) {
    // keep the candidates that can be among the K nearest (by their tensor-core distance)
    warp_sort_keys(keys, mp);
    const double nx = (double)nac[row];
    const double aK = (double)key_dist(keys[K - 1]);
    const double lim = aK + 2.0 * bf16_dist_bound(nx, ymax2, d, pairs) + stream_slop(nx, aK);
    int keep = K;
    for (int c = K; c < m; c += 32) {
      const int t = c + lane;
      const unsigned bal = __ballot_sync(0xffffffffu, t < m && (double)key_dist(keys[t]) <= lim);
      keep += __popc(bal);
      if (bal != 0xffffffffu) break;
    }
    m = keep;
  }
  for (int t = lane; t < m; t += 32) keys[t] = (uint64_t)(uint32_t)key_id(keys[t]);
  __syncwarp();
  warp_fill_dist_keys(keys, m, B, ld, xi);
  mp = 1;
  while (mp < m) mp <<= 1;
  for (int t = m + lane; t < mp; t += 32) keys[t] = KEY_NONE;
  __syncwarp();
  warp_sort_keys(keys, mp);
  if (m > 1) {
    int f = warp_fix_runs(keys, m, K, d64, B, ld, d, xi, rel);
    for (int o = 16; o > 0; o >>= 1) f += __shfl_xor_sync(0xffffffffu, f, o);
    if (lane == 0 && f) atomicAdd(n_order, (unsigned long long)f);
  }
  const float INF = __int_as_float(0x7f800000);
  for (int t = lane; t < K; t += 32) {
    const bool v = t < m;
    const int32_t id = v ? key_id(keys[t]) : -1;
    float dd = v ? key_dist(keys[t]) : INF;
    if (v && exact_d2) dd = (float)dist2_f64(xi, B + (int64_t)id * ld, d);
    out_id[row * K + t] = id;
    out_d2[row * K + t] = dd;
  }
  if (lane == 0) {
    const float t = thr[r];
    bool ok = m >= K && isinf(t) && t > 0.f;  // every column was a candidate
    double kth = INF;
    if (m >= K) {
      kth = (double)key_dist(keys[K - 1]) * (1.0 + 1.01 * (double)rel) + 1e-30;
      if (!ok) {
        const double nx = (double)nac[row];
        ok = kth < (double)t - stream_slop(nx, t) - bf16_dist_bound(nx, ymax2, d, pairs);
      }
    }
    if (!ok) {
      const int p = atomicAdd(fb_count, 1);
      fb[p] = (int32_t)row;
      fb_kth[p] = kth;
    }
  }
}

// Rows recomputed on the exact fp32 path as queries (no self exclusion) with K + 1
// neighbours: row r's own id is dropped (or the last entry, if its own id is not among
// them), the rest go to row rows[r] of the output.
__global__ void k_scatter_drop_self(const int32_t* __restrict__ ids, const float* __restrict__ d2,
                                    int K1, const int32_t* __restrict__ rows, int64_t count,
                                    int self, int32_t* __restrict__ out_id, float* __restrict__ out_d2) {
  const int64_t r = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (r >= count) return;
  const int lane = lane_id();
  const int32_t me = rows[r];
  const int K = self ? K1 - 1 : K1;
  int skip = K1;  // position dropped
  if (self) {
    skip = K1 - 1;
    for (int c = 0; c < K1; c += 32) {
      const unsigned m = __ballot_sync(0xffffffffu, c + lane < K1 && ids[r * K1 + c + lane] == me);
      if (m) {
        skip = c + __ffs(m) - 1;
        break;
      }
    }
  }
  for (int t = lane; t < K; t += 32) {
    const int src = t < skip ? t : t + 1;
    out_id[(int64_t)me * K + t] = ids[r * K1 + src];
    out_d2[(int64_t)me * K + t] = d2[r * K1 + src];
  }
}

// The second pass's admission bound of each failed row: its K-th exact distance so far
// (an upper bound of the true one) plus the bf16 bound, widened by three times the
// threshold rounding and four times the fp32 distance error (the K-th fp32 value of the new
// candidates may exceed the old one by up to twice that), so that every column that can be
// a true neighbour is admitted and a band that fits certifies against it.
__global__ void k_band_start(const double* __restrict__ kth, const float* __restrict__ nag, int m,
                             double ymax2, int d, int pairs, float* __restrict__ tau) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= m) return;
  const double nx = (double)nag[t];
  const double b = kth[t] + bf16_dist_bound(nx, ymax2, d, pairs);
  const double rel = (d + 4.0) * 5.9604644775390625e-08 * 1.01;
  const double v = b + 3.0 * stream_slop(nx, b) + 4.0 * rel * fabs(b) + 1e-30;
  tau[t] = isfinite(v) ? (float)v * (1.f + 1e-6f) : __int_as_float(0x7f800000);
}

static int read_count(const int* p, cudaStream_t st) {
  int h = 0;
  SSG_CUDA(cudaMemcpyAsync(&h, p, sizeof(int), cudaMemcpyDeviceToHost, st));
  SSG_CUDA(cudaStreamSynchronize(st));
  return h;
}

// One certification launch (k_knn_cert) over count rows; returns the rows that failed.
static int certify(const float* A, const float* B, int ld, int d, const int32_t* rows, int64_t count,
                   const int32_t* cand, const float* cd2, int KS, const float* thr, const float* nac, double ymax2,
                   int pairs, int K, bool exact_d2, int32_t* out_id, float* out_d2, int32_t* fb, double* fbk,
                   int* fbc, unsigned long long* n_order, cudaStream_t st) {
  SSG_CUDA(cudaMemsetAsync(fbc, 0, sizeof(int), st));
  if (count == 0) return 0;
  const int cap = next_pow2(std::max(KS, 32));
  const int wpb = 4;
  const size_t smem = (size_t)cap * 16 * wpb;
  ensure_smem((const void*)k_knn_cert, smem);
  SSG_LAUNCH(k_knn_cert, (unsigned)ceil_div(count, wpb), wpb * 32, smem, st, A, B, ld, d, rows, count,
             cand, cd2, KS, thr, nac, ymax2, pairs, K, cap, dist_rel_team8c(ld), exact_d2 ? 1 : 0, out_id,
             out_d2, fb,
             fbk, fbc, n_order);
  return read_count(fbc, st);
}

CertResult knn_bf16_certified(const float* A, int64_t na, int ld, const float* a_norm_raw,
                              const float* B, int64_t nb, const float* b_norm_raw, int d,
                              const DataInfo& info, int self, int K, int32_t* out_id, float* out_d2,
                              bool exact_d2, const KnnTune& tune, unsigned long long* n_order,
                              cudaStream_t st, StageTimer* gemm_timer) {
  CertResult res;
  SSG_REQUIRE(knn_tc_available(d), SSG_EINTERNAL,
              "certified bf16 kNN: the tensor-core path does not run for d = %d", d);
  const int grid = 8 * num_sms();
  // centre on the base's column mean; centred squared norms and their maximum
  Scratch<double> csum((size_t)d, st);
  SSG_CUDA(cudaMemsetAsync(csum.p, 0, sizeof(double) * d, st));
  const unsigned gy = (unsigned)std::min<int64_t>(ceil_div(nb, 8), 4 * num_sms());
  SSG_LAUNCH(k_col_sum, dim3((unsigned)ceil_div(d, 32), gy), dim3(32, 8), 0, st, B, nb, d, ld, csum.p);
  Scratch<float> mu((size_t)d, st);
  SSG_LAUNCH(k_col_mean, (unsigned)ceil_div(d, 128), 128, 0, st, csum.p, d, nb, mu.p);
  Scratch<float> nbc((size_t)nb, st), nac_own;
  Scratch<unsigned> mx(1, st);
  SSG_CUDA(cudaMemsetAsync(mx.p, 0, sizeof(unsigned), st));
  SSG_LAUNCH(k_centred_norms, (unsigned)ceil_div(nb, 8), 256, 0, st, B, nb, d, ld, mu.p, nbc.p, mx.p);
  const float* nac = nbc.p;
  if (!self) {
    nac_own.alloc((size_t)na, st);
    SSG_LAUNCH(k_centred_norms, (unsigned)ceil_div(na, 8), 256, 0, st, A, na, d, ld, mu.p,
               nac_own.p, (unsigned*)nullptr);
    nac = nac_own.p;
  }
  unsigned mbits = 0;
  SSG_CUDA(cudaMemcpyAsync(&mbits, mx.p, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
  SSG_CUDA(cudaStreamSynchronize(st));
  float ymax2f;
  memcpy(&ymax2f, &mbits, 4);
  const double ymax2 = (double)ymax2f;
  const int64_t avail = self ? nb - 1 : nb;
  const int dp = (d + 63) & ~63;
  // bf16 pairs triple the rows the tensor cores see; they run where that width fits
  const bool pairs_ok = knn_tc_available(3 * dp);
  int pairs = tune.bf16_pairs == 1 && pairs_ok ? 1 : 0;

  // KS: the tune.quantile point of the sampled rows' candidate needs, plus 5%
  int KS = std::min<int64_t>(avail, std::max(K + 8, 2 * K));
  const int s = (int)std::min<int64_t>(tune.sample_rows, na);
  if (s > 0 && avail > KS && K + (int)self <= (int)avail) {
    std::vector<int32_t> sid_h((size_t)s);
    for (int t = 0; t < s; ++t) sid_h[t] = (int32_t)(((int64_t)t * na) / s);
    Scratch<int32_t> sid((size_t)s, st);
    SSG_CUDA(cudaMemcpyAsync(sid.p, sid_h.data(), sizeof(int32_t) * s, cudaMemcpyHostToDevice, st));
    Scratch<float> As((size_t)s * ld, st), asn((size_t)s, st), asc((size_t)s, st);
    SSG_LAUNCH(k_gather_rows, grid, 256, 0, st, A, ld, sid.p, (int64_t)s, As.p);
    SSG_LAUNCH(k_centred_norms, (unsigned)ceil_div(s, 8), 256, 0, st, As.p, (int64_t)s, d, ld,
               (const float*)nullptr, asn.p, (unsigned*)nullptr);
    SSG_LAUNCH(k_gather_vals, (unsigned)ceil_div(s, 256), 256, 0, st, nac, sid.p, (int64_t)s, asc.p);
    // the sample's exact K-th distance (itself included as a column when self: K + 1),
    // through this same certified path with the sample as queries and no sizing of its own
    // (bf16 pairs where they run: their narrow band certifies most sample rows at once)
    const int Kq = K + self;
    Scratch<int32_t> sids((size_t)s * Kq, st);
    Scratch<float> sd2((size_t)s * Kq, st);
    KnnTune t0 = tune;
    t0.sample_rows = 0;
    t0.bf16_pairs = pairs_ok ? 1 : 0;
    knn_bf16_certified(As.p, s, ld, asn.p, B, nb, b_norm_raw, d, info, 0, Kq, sids.p, sd2.p, false,
                       t0, n_order, st, nullptr);
    Scratch<double> lim((size_t)s, st);
    Scratch<int> cnt((size_t)s, st);
    const size_t smem = sizeof(float) * ((size_t)CAL_DC * CAL_S + (size_t)CAL_TJ * CAL_DC);
    ensure_smem((const void*)k_band_count<false>, smem);
    ensure_smem((const void*)k_band_count<true>, smem);
    const unsigned cg = (unsigned)std::min<int64_t>(ceil_div(nb, CAL_TJ), num_sms());
    // columns a row's first pass must keep: single bf16, those whose bf16 distance lies
    // within the bound of the exact K-th; bf16 pairs (whose error is far below the band),
    // those whose fp32 distance lies within twice their bound
    auto need_for = [&](int pr) -> int {
      SSG_LAUNCH(k_band_limit, (unsigned)ceil_div(s, 128), 128, 0, st, sd2.p, Kq, Kq - 1, s, asc.p,
                 ymax2, d, pr, pr ? 2.0 : 1.0, lim.p);
      SSG_CUDA(cudaMemsetAsync(cnt.p, 0, sizeof(int) * s, st));
      const int32_t* me = self ? (const int32_t*)sid.p : nullptr;
      if (pr)
        SSG_LAUNCH(k_band_count<true>, cg, CAL_S, smem, st, As.p, s, ld, B, nb, ld, d, mu.p, asc.p,
                   nbc.p, lim.p, me, cnt.p);
      else
        SSG_LAUNCH(k_band_count<false>, cg, CAL_S, smem, st, As.p, s, ld, B, nb, ld, d, mu.p, asc.p,
                   nbc.p, lim.p, me, cnt.p);
      std::vector<int> h((size_t)s);
      SSG_CUDA(cudaMemcpyAsync(h.data(), cnt.p, sizeof(int) * s, cudaMemcpyDeviceToHost, st));
      SSG_CUDA(cudaStreamSynchronize(st));
      std::sort(h.begin(), h.end());
      const int qi = std::min(s - 1, (int)std::ceil(tune.slack_quantile * s) - 1);
      return (int)std::ceil(h[std::max(qi, 0)] * 1.05) + 8;
    };
    int need = need_for(pairs);
    // single bf16 too coarse for these data (its band would need more candidates than
    // PAIRS_AT, or than the kernel keeps): bf16 pairs, three products per coordinate
    constexpr int PAIRS_AT = 768;
    if (!pairs && pairs_ok && tune.bf16_pairs < 0 &&
        (need > PAIRS_AT || need > knn_tc_max_k(d, false))) {
      pairs = 1;
      need = need_for(1);
    }
    KS = (int)std::min<int64_t>(avail, std::max(K + 8, need));
  }
  const int KS_MAX = knn_tc_max_k(pairs ? 3 * dp : d, false);  // the largest top-K kept
  KS = std::min(KS, KS_MAX);
  res.candidates = KS;
  res.pairs = pairs;

  // pass 1: every row
  Scratch<int32_t> cid((size_t)na * KS, st);
  Scratch<float> cd2((size_t)na * KS, st), thr((size_t)na, st);
  TcExtra ex;
  ex.mu = mu.p;
  ex.out_thresh = thr.p;
  ex.order_norm = a_norm_raw;
  ex.prepass_tiles = tune.prepass_tiles;
  ex.stream_rows = tune.stream_rows;
  ex.pairs = pairs;
  knn_exact_tc(A, na, ld, nac, B, nb, ld, nbc.p, d, self, KS, cid.p, cd2.p, st, gemm_timer, 0, true,
               ex);
  Scratch<int32_t> fb((size_t)na, st), fb2((size_t)na, st);
  Scratch<double> fbk((size_t)na, st);
  Scratch<int> fbc(1, st);
  int nfb = certify(A, B, ld, d, nullptr, na, cid.p, cd2.p, KS, thr.p, nac, ymax2, pairs, K, exact_d2, out_id,
                    out_d2, fb.p, fbk.p, fbc.p, n_order, st);
  cid.release();
  cd2.release();
  res.fallback_rows = nfb;
  int nlast = nfb;
  const int32_t* last = fb.p;
  // pass 2: the failed rows again, admitting every column whose bf16 distance is at most
  // their K-th exact distance so far plus the bound (the band that can hold a true
  // neighbour), up to KS2 columns; a band that fits certifies the row
  if (nfb > 0 && KS < avail) {
    const int KS2 = (int)std::min<int64_t>(avail, std::min(KS_MAX, std::max(KS, 640)));
    Scratch<float> Ag((size_t)nfb * ld, st), nag((size_t)nfb, st), thr2((size_t)nfb, st),
        tau2((size_t)nfb, st);
    Scratch<int32_t> cid2((size_t)nfb * KS2, st);
    Scratch<float> cd22((size_t)nfb * KS2, st);
    SSG_LAUNCH(k_gather_rows, grid, 256, 0, st, A, ld, fb.p, (int64_t)nfb, Ag.p);
    SSG_LAUNCH(k_gather_vals, (unsigned)ceil_div(nfb, 256), 256, 0, st, nac, fb.p, (int64_t)nfb, nag.p);
    SSG_LAUNCH(k_band_start, (unsigned)ceil_div(nfb, 128), 128, 0, st, fbk.p, nag.p, nfb, ymax2, d,
               pairs, tau2.p);
    TcExtra ex2;
    ex2.mu = mu.p;
    ex2.out_thresh = thr2.p;
    ex2.qid = self ? fb.p : nullptr;
    ex2.tau_in = tau2.p;
    ex2.pairs = pairs;
    knn_exact_tc(Ag.p, nfb, ld, nag.p, B, nb, ld, nbc.p, d, self, KS2, cid2.p, cd22.p, st, nullptr, 0,
                 true, ex2);
    nlast = certify(Ag.p, B, ld, d, fb.p, nfb, cid2.p, cd22.p, KS2, thr2.p, nac, ymax2, pairs, K, exact_d2, out_id,
                    out_d2, fb2.p, fbk.p, fbc.p, n_order, st);
    last = fb2.p;
    res.pass2_rows = nfb;
  }
  // the rest: exhaustively (few rows), else the exact fp32 path as queries
  if (nlast > 0) {
    std::vector<double> kh((size_t)nlast);
    SSG_CUDA(cudaMemcpyAsync(kh.data(), fbk.p, sizeof(double) * nlast, cudaMemcpyDeviceToHost, st));
    SSG_CUDA(cudaStreamSynchronize(st));
    bool bounded = true;
    for (double v : kh) bounded = bounded && std::isfinite(v);
    if (bounded && (int64_t)nlast * nb <= (1ll << 28)) {
      knn_fallback_rows(A, ld, B, ld, d, nb, self, last, fbk.p, nlast, K, out_id, out_d2, st);
    } else {
      const int K1 = K + self;
      Scratch<float> Ag((size_t)nlast * ld, st), agn((size_t)nlast, st);
      SSG_LAUNCH(k_gather_rows, grid, 256, 0, st, A, ld, last, (int64_t)nlast, Ag.p);
      SSG_LAUNCH(k_centred_norms, (unsigned)ceil_div(nlast, 8), 256, 0, st, Ag.p, (int64_t)nlast, d,
                 ld, (const float*)nullptr, agn.p, (unsigned*)nullptr);
      Scratch<int32_t> ids((size_t)nlast * K1, st);
      Scratch<float> dd((size_t)nlast * K1, st);
      knn_exact(Ag.p, nlast, ld, agn.p, B, nb, ld, b_norm_raw, d, info, 0, K1, ids.p, dd.p, st,
                nullptr);
      SSG_LAUNCH(k_scatter_drop_self, (unsigned)ceil_div(nlast, 8), 256, 0, st, ids.p, dd.p, K1,
                 last, (int64_t)nlast, self, out_id, out_d2);
    }
    res.exact_rows = nlast;
  }
  return res;
}

}  // namespace ssg
