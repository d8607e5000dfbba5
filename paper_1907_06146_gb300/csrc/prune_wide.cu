// SSG prune (Alg. 2 selection applied to every pool, Alg. 3) of nodes whose rows are long
// (for example d = 960 with R = 70): one node per thread block of eight warps.
//
// The warp prune keeps a node's kept centred vectors beside the warp, which rows this
// long do not fit, and a warp that then walks its kept vectors one dot product after
// another waits on memory for each of them.  Here the candidates are taken in windows of
// eight, one per warp:
//   1. every warp loads its candidate's row, forms the centred vector c_j - x in its
//      registers (lane l holds float4 columns l, l + 32, ...) and in the kept-vector slot
//      it would take if every candidate before it in the window were kept, and tests it
//      against the node's kept vectors as they stood when the window began (four dot
//      products at a time, stopping at the first definite conflict);
//   2. after one barrier, warp 0 settles the window in candidate order: a candidate that
//      passed step 1 is also tested against the candidates of this window kept before it,
//      then kept (its vector moved down to the next kept slot) or dropped, until R are
//      kept.
// The kept vectors sit in the block's shared memory (the first `cap` of them; the rest in
// a device slot of the block, which stays in L2).  So the eight warps run eight
// independent chains of dot products and meet twice per window, not once per candidate.
// The decisions are those of the warp prune: the fp32 cosine decides outside a margin that
// bounds its rounding error for any summation order; the rest, and zero-length edges, are
// re-taken in fp64 from the original vectors.  Those fp64 dot products are summed by the
// 32 lanes of warp 0; where the resulting cosine lies within 1e-10 of cos(alpha) -- far
// more than the two summation orders can move it for any d up to 4,096 -- the three dot
// products are re-taken in coordinate order, so every decision is the one the
// coordinate-order fp64 rule takes.
#include "common.cuh"
#include "graph_dev.cuh"
#include "knn.cuh"

namespace ssg {
namespace {

constexpr int PW_WARPS = 8;                  // = candidates per window
constexpr int PW_THREADS = PW_WARPS * 32;
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
  float* Vg;                // block b's kept vectors cap .. R + 7: Vg + b * (R + 8 - cap) * d4
  int cap;                  // kept vectors held in shared memory
  unsigned long long* n64;
  unsigned long long* nborder;
};

// Byte offsets of the block's shared-memory regions (all multiples of 16).
struct WideLayout {
  size_t xs, V, gkk, g64, kid, wmeta, nlist, total;
};
__host__ __device__ inline WideLayout wide_layout(int d, int R, int cap) {
  const size_t row = (size_t)((d + 3) & ~3) * 4;
  const size_t R1a = (size_t)((R + 1 + 3) & ~3);
  WideLayout L;
  L.xs = 0;
  L.V = L.xs + row;                          // cap kept vectors
  L.gkk = L.V + (size_t)cap * row;           // [R1a] fp32 |c_k - x|^2
  L.g64 = L.gkk + R1a * 4;                   // [R1a] fp64 |c_k - x|^2 (< 0: not computed)
  L.kid = L.g64 + R1a * 8;                   // [R1a] kept ids
  L.wmeta = L.kid + R1a * 4;                 // per window slot: |v|^2, id, verdict, near count
  L.nlist = L.wmeta + 4 * PW_WARPS * 4;      // [PW_WARPS][R1a] kept vectors to re-test in fp64
  L.total = L.nlist + PW_WARPS * R1a * 4;
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

// fp32 angle test of one pair from its centred dot product g and squared lengths:
// 2 = definite conflict, 1 = to be re-taken in fp64, 0 = no conflict.
__device__ __forceinline__ int angle_test32(float g, float gjj, float gk, float cosA32,
                                            float margin) {
  if (gjj == 0.f || gk == 0.f) return 1;
  const float c = g / (sqrtf(gjj) * sqrtf(gk));
  if (c > cosA32 + margin) return 2;
  return c >= cosA32 - margin ? 1 : 0;
}

// One node i of a (a.len, a.cand, ...) by the whole block.  NVR: float4 columns of the
// candidate vector each lane holds (rows of up to 128 NVR values).  spill: this block's
// device slot for kept vectors beyond a.cap.  n64 / nb: this thread's fp64 re-test counts.
template <int NVR>
__device__ __forceinline__ void block_prune_node(const WideArgs& a, int64_t i, unsigned char* smw,
                                                 float* spill, unsigned long long& n64,
                                                 unsigned long long& nb) {
  const WideLayout Ly = wide_layout(a.d, a.R, a.cap);
  const int d4 = (a.d + 3) & ~3, nq4 = d4 >> 2;
  const int R1a = (a.R + 1 + 3) & ~3;
  float* xs = (float*)(smw + Ly.xs);
  float* V = (float*)(smw + Ly.V);
  float* gkk = (float*)(smw + Ly.gkk);
  double* g64 = (double*)(smw + Ly.g64);
  int32_t* kid = (int32_t*)(smw + Ly.kid);
  float* wg = (float*)(smw + Ly.wmeta);                  // [8] |v|^2 of the window's vectors
  int32_t* wid = (int32_t*)(wg + PW_WARPS);              // [8] their ids
  int* wdead = (int*)(wid + PW_WARPS);                   // [8] definite conflict in step 1
  int* wnn = wdead + PW_WARPS;                           // [8] fp64 re-tests listed
  int* nlist = (int*)(smw + Ly.nlist);                   // [8][R1a]
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  auto kept_row = [&](int k) -> float* {
    return k < a.cap ? V + (size_t)k * d4 : spill + (size_t)(k - a.cap) * d4;
  };
  {
    const int len = a.len[i];
    const int32_t* cand = a.cand + i * a.stride;
    const float* xg = a.X + i * a.ld;
    int32_t* out = a.adj + i * a.R;
    __syncthreads();  // the previous node's readers are done with every buffer
    for (int f = tid; f < nq4; f += PW_THREADS) ((float4*)xs)[f] = __ldg((const float4*)xg + f);
    __syncthreads();
    int kept = 0;  // the same in every thread
    for (int t0 = 0; t0 < len && kept < a.R; t0 += PW_WARPS) {
      // ---- step 1: warp w takes candidate t0 + w against the kept vectors 0 .. kept-1
      const int t = t0 + warp;
      if (t < len) {
        const int32_t j = cand[t];
        const float4* c4 = (const float4*)(a.X + (int64_t)j * a.ld);
        const float4* xs4 = (const float4*)xs;
        float4 v[NVR];
#pragma unroll
        for (int r = 0; r < NVR; ++r) {
          const int f = lane + 32 * r;
          v[r] = f < nq4 ? __ldg(c4 + f) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        float part = 0.f;
        float4* slot = (float4*)kept_row(kept + warp);
#pragma unroll
        for (int r = 0; r < NVR; ++r) {
          const int f = lane + 32 * r;
          if (f < nq4) {
            const float4 x = xs4[f];
            v[r] = make_float4(v[r].x - x.x, v[r].y - x.y, v[r].z - x.z, v[r].w - x.w);
            slot[f] = v[r];
          }
          part = dot4(v[r], v[r], part);
        }
        const float gjj = warp_sum(part);
        int dead = 0, nn = 0;
        // four kept vectors per round; the four sums are reduced together (lanes 8u .. 8u+7
        // end up holding dot product u)
        const int mine = ((lane >> 4) & 1) * 2 + ((lane >> 3) & 1);
        for (int k0 = 0; k0 < kept && !dead; k0 += 4) {
          const int kn = min(4, kept - k0);
          const float4* w0 = (const float4*)kept_row(k0);
          const float4* w1 = kn > 1 ? (const float4*)kept_row(k0 + 1) : w0;
          const float4* w2 = kn > 2 ? (const float4*)kept_row(k0 + 2) : w0;
          const float4* w3 = kn > 3 ? (const float4*)kept_row(k0 + 3) : w0;
          float g0 = 0.f, g1 = 0.f, g2 = 0.f, g3 = 0.f;
#pragma unroll
          for (int r = 0; r < NVR; ++r) {
            const int f = lane + 32 * r;
            if (f < nq4) {
              g0 = dot4(v[r], w0[f], g0);
              g1 = dot4(v[r], w1[f], g1);
              g2 = dot4(v[r], w2[f], g2);
              g3 = dot4(v[r], w3[f], g3);
            }
          }
          const bool hi16 = (lane & 16) != 0, hi8 = (lane & 8) != 0;
          const float r0 = __shfl_xor_sync(0xffffffffu, hi16 ? g0 : g2, 16);
          const float r1 = __shfl_xor_sync(0xffffffffu, hi16 ? g1 : g3, 16);
          const float h0 = (hi16 ? g2 : g0) + r0, h1 = (hi16 ? g3 : g1) + r1;
          float g = (hi8 ? h1 : h0) + __shfl_xor_sync(0xffffffffu, hi8 ? h0 : h1, 8);
          g += __shfl_xor_sync(0xffffffffu, g, 4);
          g += __shfl_xor_sync(0xffffffffu, g, 2);
          g += __shfl_xor_sync(0xffffffffu, g, 1);
          const int res = mine < kn ? angle_test32(g, gjj, gkk[k0 + mine], a.cosA32, a.margin) : 0;
          if (__any_sync(0xffffffffu, res == 2)) {
            dead = 1;
          } else {
            const unsigned nb4 = __ballot_sync(0xffffffffu, res == 1 && (lane & 7) == 0);
            for (int u = 0; u < 4; ++u)
              if ((nb4 >> (8 * u)) & 1u) {
                if (lane == 0) nlist[warp * R1a + nn] = k0 + u;
                ++nn;
              }
          }
        }
        if (lane == 0) {
          wg[warp] = gjj;
          wid[warp] = j;
          wdead[warp] = dead;
          wnn[warp] = nn;
        }
      }
      __syncthreads();
      // ---- step 2: warp 0 settles the window in candidate order
      if (warp == 0) {
        const int kept0 = kept;
        const int wend = min(PW_WARPS, len - t0);
        for (int w = 0; w < wend && kept < a.R; ++w) {
          if (wdead[w]) continue;
          const float gjj = wg[w];
          const int32_t j = wid[w];
          const float4* vw = (const float4*)kept_row(kept0 + w);
          // against the vectors kept earlier in this window (their window slots)
          bool conflict = false;
          int wnear = 0;  // bit q: kept vector kept0 + q to re-take in fp64
          for (int q = 0; q < kept - kept0 && !conflict; ++q) {
            const float4* vu = (const float4*)kept_row(kept0 + q);
            float g = 0.f;
            for (int f = lane; f < nq4; f += 32) g = dot4(vw[f], vu[f], g);
            g = warp_sum(g);
            const int r = angle_test32(g, gjj, gkk[kept0 + q], a.cosA32, a.margin);
            if (r == 2) conflict = true;
            else if (r == 1) wnear |= 1 << q;
          }
          if (!conflict && (wnn[w] > 0 || wnear)) {
            // fp64 re-tests, kept order: first those listed in step 1, then this window's
            const float* cj = a.X + (int64_t)j * a.ld;
            const double gj = warp_cdot_f64(cj, cj, xg, a.d);
            const int nl = wnn[w];
            for (int u = 0; u < nl + PW_WARPS && !conflict; ++u) {
              int k;
              if (u < nl) {
                k = nlist[w * R1a + u];
              } else {
                if (!((wnear >> (u - nl)) & 1)) continue;
                k = kept0 + (u - nl);
              }
              const float* ck = a.X + (int64_t)kid[k] * a.ld;
              double gk = g64[k];
              if (gk < 0.0) {
                gk = warp_cdot_f64(ck, ck, xg, a.d);
                __syncwarp();
                if (lane == 0) g64[k] = gk;
              }
              double c = cos_from_gram_f64(warp_cdot_f64(cj, ck, xg, a.d), gj, gk);
              if (fabs(c - a.cosA64) <= PW_TIE_COS)
                c = cos_from_gram_f64(centred_dot_f64(cj, ck, xg, a.d),
                                      centred_dot_f64(cj, cj, xg, a.d),
                                      centred_dot_f64(ck, ck, xg, a.d));
              if (fabs(c - a.cosA64) <= a.border) ++nb;
              ++n64;
              if (c > a.cosA64) conflict = true;
            }
            if (!conflict && lane == 0) g64[kept] = gj;
          } else if (!conflict && lane == 0) {
            g64[kept] = -1.0;
          }
          if (!conflict) {
            if (kept != kept0 + w) {  // down to the next kept slot (a dropped one's)
              float4* dst = (float4*)kept_row(kept);
              for (int f = lane; f < nq4; f += 32) dst[f] = vw[f];
            }
            if (lane == 0) {
              gkk[kept] = gjj;
              kid[kept] = j;
              out[kept] = j;
            }
            ++kept;
          }
          __syncwarp();
        }
        if (lane == 0) wdead[0] = kept;  // hand the count to the other warps
      }
      __syncthreads();
      kept = wdead[0];
      __syncthreads();  // every warp has read the count before the next window writes it
    }
    for (int t = kept + tid; t < a.R; t += PW_THREADS) out[t] = -1;
    if (tid == 0) a.deg[i] = kept;
  }
}

template <int NVR>
__global__ void __launch_bounds__(PW_THREADS) k_prune_wide(WideArgs a) {
  extern __shared__ __align__(16) unsigned char smw[];
  const int d4 = (a.d + 3) & ~3;
  float* spill = a.Vg ? a.Vg + (size_t)blockIdx.x * (a.R + PW_WARPS - a.cap) * d4 : nullptr;
  unsigned long long n64 = 0, nb = 0;
  for (int64_t i = blockIdx.x; i < a.n; i += gridDim.x)
    block_prune_node<NVR>(a, i, smw, spill, n64, nb);
  if ((threadIdx.x & 31) == 0 && n64) atomicAdd(a.n64, n64);
  if ((threadIdx.x & 31) == 0 && nb) atomicAdd(a.nborder, nb);
}

// The same over the (index, node) work items of a batch, handed out from one counter in
// the order of items (longest pools first); each block's spill slot holds vg_stride floats.
template <int NVR>
__global__ void __launch_bounds__(PW_THREADS)
    k_prune_wide_batched(const WideArgs* __restrict__ jobs, const int2* __restrict__ items,
                         int64_t nitems, unsigned long long* __restrict__ next,
                         float* __restrict__ Vg, size_t vg_stride) {
  extern __shared__ __align__(16) unsigned char smw[];
  __shared__ unsigned long long s_it;
  float* spill = Vg ? Vg + (size_t)blockIdx.x * vg_stride : nullptr;
  for (;;) {
    __syncthreads();  // every thread has read the previous item
    if (threadIdx.x == 0) s_it = atomicAdd(next, 1ull);
    __syncthreads();
    const unsigned long long it = s_it;
    if (it >= (unsigned long long)nitems) break;
    const int2 w = items[it];
    const WideArgs a = jobs[w.x];
    unsigned long long n64 = 0, nb = 0;
    block_prune_node<NVR>(a, w.y, smw, spill, n64, nb);
    if ((threadIdx.x & 31) == 0 && n64) atomicAdd(a.n64, n64);
    if ((threadIdx.x & 31) == 0 && nb) atomicAdd(a.nborder, nb);
  }
}

}  // namespace

bool prune_wide_available(int d) { return ((d + 3) & ~3) <= 1024; }

bool prune_block_preferred(int d, int R) {
  return prune_wide_available(d) && (prune_is_wide(d, R) || ((d + 3) & ~3) >= 96);
}

// Shared memory a block of the block prune takes at blocks_per_sm blocks per SM.
static size_t wide_budget(int blocks_per_sm) {
  const int bps = blocks_per_sm > 0 ? blocks_per_sm : 2;
  return std::min<size_t>(225 * 1024, (226 * 1024) / bps - 1024);
}

void prune_wide_batched_prepare(const std::vector<PruneJob>& js, WideBatchPlan& plan,
                                cudaStream_t st) {
  const size_t budget = wide_budget(0);
  std::vector<WideArgs> h(js.size());
  int d4max = 4;
  for (size_t j = 0; j < js.size(); ++j) {
    const PruneJob& p = js[j];
    SSG_REQUIRE(prune_wide_available(p.d), SSG_EINTERNAL, "batched block prune: rows of %d values",
                p.d);
    const int d4 = (p.d + 3) & ~3;
    const size_t row = (size_t)d4 * 4, fixed = wide_layout(p.d, p.R, 0).total;
    SSG_REQUIRE(fixed + row <= budget, SSG_EINTERNAL, "batched block prune: rows of %d values",
                p.d);
    const int cap = (int)std::min<size_t>((size_t)p.R + PW_WARPS, (budget - fixed) / row);
    h[j] = WideArgs{p.X, p.ld, p.d, p.n, p.pool_id, p.pool_len, p.L, p.R, p.cosA32, p.margin,
                    p.cosA64, p.border, p.adj, p.deg, nullptr, cap, p.n64, p.nborder};
    plan.smem = std::max(plan.smem, wide_layout(p.d, p.R, cap).total);
    plan.vg_stride = std::max(plan.vg_stride, (size_t)(p.R + PW_WARPS - cap) * d4);
    d4max = std::max(d4max, d4);
  }
  plan.nvr = d4max <= 512 ? 4 : 8;
  const void* fn = plan.nvr == 4 ? (const void*)k_prune_wide_batched<4>
                                 : (const void*)k_prune_wide_batched<8>;
  ensure_smem(fn, plan.smem);
  int per_sm = 0;
  SSG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, PW_THREADS, plan.smem));
  plan.grid = std::max(1, per_sm) * num_sms();
  plan.jobs.alloc(sizeof(WideArgs) * h.size(), st);
  SSG_CUDA(cudaMemcpyAsync(plan.jobs.p, h.data(), sizeof(WideArgs) * h.size(),
                           cudaMemcpyHostToDevice, st));
  if (plan.vg_stride) plan.Vg.alloc((size_t)plan.grid * plan.vg_stride, st);
  SSG_CUDA(cudaStreamSynchronize(st));  // the host table is released on return
}

void prune_wide_batched_launch(const WideBatchPlan& plan, const int2* items, int64_t nitems,
                               unsigned long long* next, cudaStream_t st) {
  const WideArgs* jobs = (const WideArgs*)plan.jobs.p;
  if (plan.nvr == 4)
    SSG_LAUNCH(k_prune_wide_batched<4>, plan.grid, PW_THREADS, plan.smem, st, jobs, items, nitems,
               next, plan.Vg.p, plan.vg_stride);
  else
    SSG_LAUNCH(k_prune_wide_batched<8>, plan.grid, PW_THREADS, plan.smem, st, jobs, items, nitems,
               next, plan.Vg.p, plan.vg_stride);
}

void prune_run_wide(const float* X, int ld, int d, int64_t n, const int32_t* cand,
                    const int32_t* len, int stride, int R, double cos_a, double border,
                    int32_t* adj, int32_t* deg, Counters* dctr, cudaStream_t st, int blocks_per_sm) {
  SSG_REQUIRE(prune_wide_available(d), SSG_EINTERNAL, "wide prune: rows of %d values", d);
  const int d4 = (d + 3) & ~3;
  const size_t row = (size_t)d4 * 4;
  const size_t budget = wide_budget(blocks_per_sm);
  const size_t fixed = wide_layout(d, R, 0).total;
  SSG_REQUIRE(fixed + row <= budget, SSG_EINTERNAL, "wide prune: rows of %d values do not fit", d);
  const int cap = (int)std::min<size_t>((size_t)R + PW_WARPS, (budget - fixed) / row);
  const size_t smem = wide_layout(d, R, cap).total;
  const void* fn = d4 <= 512 ? (const void*)k_prune_wide<4> : (const void*)k_prune_wide<8>;
  ensure_smem(fn, smem);
  int per_sm = 0;
  SSG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, PW_THREADS, smem));
  const int64_t grid = std::min<int64_t>(std::max<int64_t>(n, 1),
                                         (int64_t)std::max(1, per_sm) * num_sms());
  Scratch<float> Vg;
  if (cap < R + PW_WARPS) Vg.alloc((size_t)grid * (R + PW_WARPS - cap) * d4, st);
  WideArgs a{X, ld, d, n, cand, len, stride, R, (float)cos_a,
             angle_margin_fp32(d) + (float)border, cos_a, border, adj, deg, Vg.p, cap,
             &dctr->angle_fp64, &dctr->angle_border};
  if (d4 <= 512)
    SSG_LAUNCH(k_prune_wide<4>, (unsigned)grid, PW_THREADS, smem, st, a);
  else
    SSG_LAUNCH(k_prune_wide<8>, (unsigned)grid, PW_THREADS, smem, st, a);
}

}  // namespace ssg
