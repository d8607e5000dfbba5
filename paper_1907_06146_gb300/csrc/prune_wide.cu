// SSG prune (Alg. 2 selection applied to every pool, Alg. 3) of nodes whose rows are long
// (for example d = 960 with R = 70): one node per thread block.
//
// The warp prune keeps a node's kept centred vectors beside the warp, which rows this
// long do not fit, and a warp that then walks its kept vectors one dot product after
// another waits on memory for each of them.  Here:
//   * the block's shared memory holds the node's kept centred vectors c_k - x (the first
//     `cap` of them; the rest go to a device slot of the block, which stays in L2);
//   * candidate rows arrive through a ring of PF rows filled by asynchronous copies, PF
//     candidates ahead of the one being tested;
//   * every warp forms the candidate's centred vector c_j - x in its own registers (lane l
//     holds float4 columns l, l + 32, ...), so the eight warps test it against disjoint
//     subsets of the kept vectors at once (two at a time per warp) and stop as soon as one
//     of them finds a definite conflict; one barrier per candidate joins their verdicts.
// The decisions are those of the warp prune: the fp32 cosine decides outside a margin that
// bounds its rounding error for any summation order; the rest, and zero-length edges, are
// re-taken in fp64 from the original vectors.  Those fp64 dot products are summed by the
// 32 lanes of one warp; where the resulting cosine lies within 1e-10 of cos(alpha) --
// far more than the two summation orders can move it for any d up to 4,096 -- the three
// dot products are re-taken in coordinate order, so every decision is the one the
// coordinate-order fp64 rule takes.
#include "common.cuh"
#include "graph_dev.cuh"
#include "knn.cuh"

namespace ssg {
namespace {

constexpr int PW_WARPS = 8;
constexpr int PW_THREADS = PW_WARPS * 32;
constexpr int PW_PF = 4;                     // candidate rows in flight
constexpr double PW_TIE_COS = 1e-10;         // fp64 cosines this close to cos(alpha) are
                                             // re-taken in coordinate order

struct WideArgs {
  const float* X;
  int ld, d;
  int64_t n;
  const int32_t* cand;      // node i's candidates: cand[i * stride + t], t < len[i]
  const int32_t* len;
  int stride;
  int R;
  float cosA32, margin;
  double cosA64, border;
  int32_t* adj;             // [n][R]
  int32_t* deg;
  float* Vg;                // block b's kept vectors cap.. R: Vg + b * (R + 1 - cap) * d4
  int cap;                  // kept vectors held in shared memory
  unsigned long long* n64;
  unsigned long long* nborder;
};

// Byte offsets of the block's shared-memory regions (all multiples of 16).
struct WideLayout {
  size_t xs, ring, V, gkk, g64, kid, flags, nlist, total;
};
__host__ __device__ inline WideLayout wide_layout(int d, int R, int cap) {
  const size_t row = (size_t)((d + 3) & ~3) * 4;
  const size_t R1a = (size_t)((R + 1 + 3) & ~3);
  WideLayout L;
  L.xs = 0;
  L.ring = L.xs + row;
  L.V = L.ring + PW_PF * row;
  L.gkk = L.V + (size_t)cap * row;
  L.g64 = L.gkk + R1a * 4;
  L.kid = L.g64 + R1a * 8;
  L.flags = L.kid + R1a * 4;
  L.nlist = L.flags + 16 * 4;
  L.total = L.nlist + 3 * R1a * 4;
  return L;
}

// Centred fp64 dot product (a - o).(b - o) by the 32 lanes of a warp (see the header).
__device__ __forceinline__ double warp_cdot_f64(const float* __restrict__ a,
                                                const float* __restrict__ b,
                                                const float* __restrict__ o, int d) {
  const int lane = lane_id();
  double s = 0.0;
  for (int t = lane; t < d; t += 32) {
    const double u = __dsub_rn((double)a[t], (double)o[t]);
    const double v = __dsub_rn((double)b[t], (double)o[t]);
    s = __dadd_rn(s, __dmul_rn(u, v));
  }
#pragma unroll
  for (int o2 = 16; o2 > 0; o2 >>= 1) s = __dadd_rn(s, __shfl_xor_sync(0xffffffffu, s, o2));
  return s;
}

__device__ __forceinline__ float dot4(float4 a, float4 b, float s) {
  s = fmaf(a.x, b.x, s);
  s = fmaf(a.y, b.y, s);
  s = fmaf(a.z, b.z, s);
  return fmaf(a.w, b.w, s);
}

// NVR: float4 columns of the candidate vector each lane holds (rows of up to 128 NVR values).
template <int NVR>
__global__ void __launch_bounds__(PW_THREADS) k_prune_wide(WideArgs a) {
  extern __shared__ __align__(16) unsigned char smw[];
  const WideLayout Ly = wide_layout(a.d, a.R, a.cap);
  const int d4 = (a.d + 3) & ~3, nq4 = d4 >> 2;
  const int R1a = (a.R + 1 + 3) & ~3;
  float* xs = (float*)(smw + Ly.xs);
  float* ring = (float*)(smw + Ly.ring);
  float* V = (float*)(smw + Ly.V);
  float* gkk = (float*)(smw + Ly.gkk);
  double* g64 = (double*)(smw + Ly.g64);
  int32_t* kid = (int32_t*)(smw + Ly.kid);
  volatile int* conf = (volatile int*)(smw + Ly.flags);  // [3] by candidate index mod 3
  int* nnear = (int*)(smw + Ly.flags) + 4;               // [3]
  volatile int* dec = (volatile int*)(smw + Ly.flags) + 8;  // [3] fp64 verdicts
  int* nlist = (int*)(smw + Ly.nlist);                   // [3][R1a]
  float* spill = a.Vg ? a.Vg + (size_t)blockIdx.x * (a.R + 1 - a.cap) * d4 : nullptr;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  unsigned long long n64 = 0, nb = 0;

  for (int64_t i = blockIdx.x; i < a.n; i += gridDim.x) {
    const int len = a.len[i];
    const int32_t* cand = a.cand + i * a.stride;
    const float* xg = a.X + i * a.ld;
    int32_t* out = a.adj + i * a.R;
    __syncthreads();  // the previous node's readers are done with every buffer
    for (int f = tid; f < nq4; f += PW_THREADS) ((float4*)xs)[f] = __ldg((const float4*)xg + f);
    if (tid < 3) {
      conf[tid] = 0;
      nnear[tid] = 0;
    }
    auto prefetch = [&](int t) {
      if (t < len) {
        const float4* src = (const float4*)(a.X + (int64_t)cand[t] * a.ld);
        float* dst = ring + (size_t)(t % PW_PF) * d4;
        for (int f = tid; f < nq4; f += PW_THREADS) cp_async16(dst + 4 * f, src + f);
      }
      cp_async_commit();
    };
    for (int t = 0; t < PW_PF; ++t) prefetch(t);
    cp_async_wait<PW_PF - 1>();
    __syncthreads();  // xs, the flags and candidate 0's row in place

    int kept = 0;
    for (int t = 0; t < len && kept < a.R; ++t) {
      const int s3 = t % 3;
      const int32_t j = cand[t];
      const float4* cs4 = (const float4*)(ring + (size_t)(t % PW_PF) * d4);
      const float4* xs4 = (const float4*)xs;
      float4 v[NVR];
      float part = 0.f;
#pragma unroll
      for (int r = 0; r < NVR; ++r) {
        const int f = lane + 32 * r;
        if (f < nq4) {
          const float4 c = cs4[f], x = xs4[f];
          v[r] = make_float4(c.x - x.x, c.y - x.y, c.z - x.z, c.w - x.w);
        } else {
          v[r] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        part = dot4(v[r], v[r], part);
      }
      const float gjj = warp_sum(part);  // the same value in every warp
      if (warp == 0) {
        // the tentative kept row: used from the next candidate on if this one is kept
        float4* slot = (float4*)(kept < a.cap ? V + (size_t)kept * d4
                                              : spill + (size_t)(kept - a.cap) * d4);
#pragma unroll
        for (int r = 0; r < NVR; ++r) {
          const int f = lane + 32 * r;
          if (f < nq4) slot[f] = v[r];
        }
        if (lane == 0) {
          gkk[kept] = gjj;
          kid[kept] = j;
          g64[kept] = -1.0;  // fp64 norm not computed yet
          const int s1 = (t + 1) % 3;
          conf[s1] = 0;
          nnear[s1] = 0;
        }
      }
      // fp32 tests against the kept vectors k = warp, warp + 8, ... (two at a time)
      for (int k0 = warp; k0 < kept; k0 += 2 * PW_WARPS) {
        if (conf[s3]) break;
        const int k1 = k0 + PW_WARPS;
        const bool two = k1 < kept;
        const float4* v0 = (const float4*)(k0 < a.cap ? V + (size_t)k0 * d4
                                                      : spill + (size_t)(k0 - a.cap) * d4);
        const float4* v1 = !two ? v0
                                : (const float4*)(k1 < a.cap ? V + (size_t)k1 * d4
                                                             : spill + (size_t)(k1 - a.cap) * d4);
        float g0 = 0.f, g1 = 0.f;
#pragma unroll
        for (int r = 0; r < NVR; ++r) {
          const int f = lane + 32 * r;
          if (f < nq4) {
            g0 = dot4(v[r], v0[f], g0);
            g1 = dot4(v[r], v1[f], g1);
          }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          g0 += __shfl_xor_sync(0xffffffffu, g0, o);
          g1 += __shfl_xor_sync(0xffffffffu, g1, o);
        }
        bool definite = false;
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          if (q == 1 && !two) break;
          const int k = q ? k1 : k0;
          const float g = q ? g1 : g0;
          const float gk = gkk[k];
          bool near = gjj == 0.f || gk == 0.f;
          if (!near) {
            const float c = g / (sqrtf(gjj) * sqrtf(gk));
            if (c > a.cosA32 + a.margin)
              definite = true;
            else if (c >= a.cosA32 - a.margin)
              near = true;
          }
          if (near && lane == 0) nlist[s3 * R1a + atomicAdd(&nnear[s3], 1)] = k;
        }
        if (definite) {
          if (lane == 0) conf[s3] = 1;
          break;
        }
      }
      // the next candidate's row must be in place for every thread after the barrier
      cp_async_wait<PW_PF - 2>();
      __syncthreads();
      bool accept = !conf[s3];
      const int nn = *(volatile int*)&nnear[s3];
      if (accept && nn > 0) {
        if (warp == 0) {
          int* lst = nlist + s3 * R1a;
          if (lane == 0) {  // test in kept order, so the counts do not depend on timing
            for (int u = 1; u < nn; ++u) {
              const int x = lst[u];
              int w = u - 1;
              while (w >= 0 && lst[w] > x) {
                lst[w + 1] = lst[w];
                --w;
              }
              lst[w + 1] = x;
            }
          }
          __syncwarp();
          const float* cj = a.X + (int64_t)j * a.ld;
          const double gj = warp_cdot_f64(cj, cj, xg, a.d);
          bool c64 = false;
          for (int u = 0; u < nn && !c64; ++u) {
            const int k = lst[u];
            const float* ck = a.X + (int64_t)kid[k] * a.ld;
            double gk = g64[k];
            if (gk < 0.0) {
              gk = warp_cdot_f64(ck, ck, xg, a.d);
              __syncwarp();
              if (lane == 0) g64[k] = gk;
            }
            double c = cos_from_gram_f64(warp_cdot_f64(cj, ck, xg, a.d), gj, gk);
            if (fabs(c - a.cosA64) <= PW_TIE_COS)
              c = cos_from_gram_f64(centred_dot_f64(cj, ck, xg, a.d), centred_dot_f64(cj, cj, xg, a.d),
                                    centred_dot_f64(ck, ck, xg, a.d));
            if (fabs(c - a.cosA64) <= a.border) ++nb;
            ++n64;
            if (c > a.cosA64) c64 = true;
          }
          __syncwarp();
          if (lane == 0) {
            dec[s3] = c64 ? 1 : 0;
            if (!c64) g64[kept] = gj;
          }
        }
        __syncthreads();
        accept = !dec[s3];
      }
      if (accept) {
        if (tid == 0) out[kept] = j;
        ++kept;
      }
      prefetch(t + PW_PF);  // into the ring slot of candidate t, which every warp has read
    }
    cp_async_wait<0>();
    for (int t = kept + tid; t < a.R; t += PW_THREADS) out[t] = -1;
    if (tid == 0) a.deg[i] = kept;
  }
  if (lane == 0 && n64) atomicAdd(a.n64, n64);
  if (lane == 0 && nb) atomicAdd(a.nborder, nb);
}

}  // namespace

bool prune_wide_available(int d) { return ((d + 3) & ~3) <= 1024; }

void prune_run_wide(const float* X, int ld, int d, int64_t n, const int32_t* cand,
                    const int32_t* len, int stride, int R, double cos_a, double border,
                    int32_t* adj, int32_t* deg, Counters* dctr, cudaStream_t st, int blocks_per_sm) {
  SSG_REQUIRE(prune_wide_available(d), SSG_EINTERNAL, "wide prune: rows of %d values", d);
  const int d4 = (d + 3) & ~3;
  const size_t row = (size_t)d4 * 4;
  const int bps = blocks_per_sm > 0 ? blocks_per_sm : 2;
  const size_t budget = std::min<size_t>(225 * 1024, (226 * 1024) / bps - 1024);
  const size_t fixed = wide_layout(d, R, 0).total;
  SSG_REQUIRE(fixed + row <= budget, SSG_EINTERNAL, "wide prune: rows of %d values do not fit", d);
  const int cap = (int)std::min<size_t>((size_t)R + 1, (budget - fixed) / row);
  const size_t smem = wide_layout(d, R, cap).total;
  const void* fn = d4 <= 512 ? (const void*)k_prune_wide<4> : (const void*)k_prune_wide<8>;
  ensure_smem(fn, smem);
  int per_sm = 0;
  SSG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, PW_THREADS, smem));
  const int64_t grid = std::min<int64_t>(std::max<int64_t>(n, 1),
                                         (int64_t)std::max(1, per_sm) * num_sms());
  Scratch<float> Vg;
  if (cap < R + 1) Vg.alloc((size_t)grid * (R + 1 - cap) * d4, st);
  WideArgs a{X, ld, d, n, cand, len, stride, R, (float)cos_a,
             angle_margin_fp32(d) + (float)border, cos_a, border, adj, deg, Vg.p, cap,
             &dctr->angle_fp64, &dctr->angle_border};
  if (d4 <= 512)
    SSG_LAUNCH(k_prune_wide<4>, (unsigned)grid, PW_THREADS, smem, st, a);
  else
    SSG_LAUNCH(k_prune_wide<8>, (unsigned)grid, PW_THREADS, smem, st, a);
}

}  // namespace ssg
