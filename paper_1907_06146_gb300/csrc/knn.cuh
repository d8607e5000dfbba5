// Declarations shared by the library's translation units.
#pragma once

#include <vector>

#include "common.cuh"

namespace ssg {

// Rows with a 16-byte-aligned stride (ld % 4 == 0, zero padded beyond d).
struct PaddedRows {
  const float* p = nullptr;
  int ld = 0;
  Scratch<float> own;
};

struct KnnResult {
  int64_t fallback_rows = 0;
};

// Ingest (build step a0): padded view of X, fp32 squared norms (may be null), data facts.
void ingest(const float* X, int64_t n, int d, cudaStream_t st, PaddedRows& out, float* norms,
            DataInfo* info);

// Exact top-K by (d2, id) of every row of A against the rows of B (self = A is B and
// row i skips column i).  info describes A and B together.
KnnResult knn_exact(const float* A, int64_t na, int lda, const float* a_norm, const float* B,
                    int64_t nb, int ldb, const float* b_norm, int d, const DataInfo& info,
                    int self, int K, int32_t* out_id, float* out_d2, cudaStream_t st,
                    StageTimer* gemm_timer);

// Near-first column order: rows clustered and stored cluster by cluster (perm maps a
// stored position to the original row, inv the other way); for each cluster the ntiles BN-column tiles of the
// stored order, nearest cluster first (tile_order, ncl x ntiles); rb_cluster gives the
// cluster of each block of BM stored rows.
struct KnnOrder {
  int ncl = 0;
  int64_t ntiles = 0;
  int64_t tstride = 0;  // length of each cluster's tile list (ntiles, or the walk limit)
  Scratch<int32_t> perm, inv, tile_order, rb_cluster;
};
bool knn_order_fits(int64_t n, int BN);
// walk > 0: every block of rows visits only its first walk tiles (Alg. 4), so each
// cluster's list stops there and the clusters are kept small.
// x_norm (nullable): squared row norms; with them, large assignments run on the tensor
// cores.
void knn_cluster_order(const float* X, int ld, int d, int64_t n, int BM, int BN, cudaStream_t st,
                       KnnOrder& o, int64_t walk = 0, const float* x_norm = nullptr);

// bf16 tensor-core variant of the exact top-K (only for info.bf16_exact data).
// True on sm_103 for rows of up to 4,096 values: the resident pipeline holds d <= 128, wider
// rows stream through the K-chunked kernel.
bool knn_tc_available(int d);
// Largest K (self-joins; one less than the row buffer's room) the tensor-core kernel takes
// for rows of d values, for a full walk or a tile-limited one.
int knn_tc_max_k(int d, bool limited);
// Optional inputs and outputs of knn_exact_tc.
struct TcExtra {
  const float* mu = nullptr;          // centre every row on mu [d] before rounding to bf16
                                      // (a_norm / b_norm are then the centred rows' norms)
  float* out_thresh = nullptr;        // per output row: the KS-th smallest distance kept, or
                                      // the final admission bound if fewer were kept (every
                                      // column not returned is at least this far, up to the
                                      // rounding of the streaming threshold)
  const float* tau_in = nullptr;      // per query row: the admission bound to start from
                                      // (columns above it are never kept)
  const int32_t* qid = nullptr;       // self with A a gathered subset of B: query row r is
                                      // base row qid[r]; outputs go to row r
  const float* order_norm = nullptr;  // norms of A as given, for the cluster order
  int stream_rows = 0;                // 1: the K-chunked kernel (128 x 256 tiles, N = 256)
                                      // also for rows that fit the resident one
  int pairs = 0;                      // 1: each centred value v goes in as the bf16 pair
                                      // hi = bf16(v), lo = bf16(v - hi); A rows are laid out
                                      // [hi | lo | hi] and B rows [lo | hi | hi] (each part
                                      // padded to 64 values), so one accumulator sums
                                      // hi.lo + lo.hi, then hi.hi (K three times as long)
  int prepass_tiles = 0;              // near-first self-joins: a first walk over this many
                                      // tiles gives each row an upper bound of its KS-th
                                      // distance, from which the full walk starts (0: off;
                                      // measured slower at 4-16 tiles on the SIFT-shaped set)
};
// max_tiles > 0 (self-joins only): the columns are visited in the cluster order and each
// block of rows stops after its max_tiles nearest 128-column tiles, so the result is the
// top-K among those columns (Alg. 4's search-based pools).  approx: the data need not be
// exact in bf16 (the distances and the selection are then approximate).
void knn_exact_tc(const float* A, int64_t na, int lda, const float* a_norm, const float* B,
                  int64_t nb, int ldb, const float* b_norm, int d, int self, int K,
                  int32_t* out_id, float* out_d2, cudaStream_t st, StageTimer* gemm_timer,
                  int max_tiles = 0, bool approx = false, const TcExtra& ex = TcExtra());

// Launch parameters of the certified bf16 kNN (ssg_build_opts.tune_table).
struct KnnTune {
  int sample_rows = 256;        // rows sampled to size the candidate count KS
  double slack_quantile = 0.99; // fraction of sampled rows KS must certify
  int prepass_tiles = 0;        // TcExtra::prepass_tiles of the kNN graph
  int stream_rows = 0;          // TcExtra::stream_rows of the kNN graph
  int prune_warps = 0;          // PruneTune of a batched build
  int prune_bucket_width = 32;
  int prune_wide_blocks = 0;    // blocks per SM of the block prune of long rows (0: 2)
  int bf16_pairs = -1;          // certified kNN operands as bf16 pairs: 1 always, 0 never,
                                // -1 where the sized single-bf16 band is too wide
};
struct CertResult {
  int64_t fallback_rows = 0;  // rows not certified by the first pass
  int64_t pass2_rows = 0;     // rows that took the second tensor-core pass
  int64_t exact_rows = 0;     // rows recomputed on the exact fp32 path
  int candidates = 0;         // KS of the first pass
  int pairs = 0;              // 1: the operands went to the tensor cores as bf16 pairs
};

struct Counters {
  unsigned long long angle_fp64;
  unsigned long long order_fp64;
  int max_indeg;
  int status;
  unsigned long long angle_border;  // fp64 cosines within the reporting band of cos(alpha)
};

// Exhaustive exact rows (k_knn_fallback): row rows[t] of A gets the K nearest of B by
// (fp64 d2, id) among the columns whose fp64 d2 is at most kth[t] (an upper bound of the
// row's K-th distance); EINTERNAL if more than 4,096 columns lie within it.
void knn_fallback_rows(const float* A, int lda, const float* B, int ldb, int d, int64_t nb,
                       int self, const int32_t* rows, const double* kth, int count, int K,
                       int32_t* out_id, float* out_d2, cudaStream_t st);

// Exact kNN rows through the bf16 tensor cores for data that bf16 does not hold exactly
// (knn_cert.cu): A [na][ld] against B [nb][ld] (self: A is B, each row skips itself),
// both with their fp32 squared norms as given; out_id / out_d2 [na][K] sorted by (d2, id);
// d2 rounded from fp64 when exact_d2, else the fp32 direct value.  Needs
// knn_tc_available(d).
CertResult knn_bf16_certified(const float* A, int64_t na, int ld, const float* a_norm_raw,
                              const float* B, int64_t nb, const float* b_norm_raw, int d,
                              const DataInfo& info, int self, int K, int32_t* out_id, float* out_d2,
                              bool exact_d2, const KnnTune& tune, unsigned long long* n_order,
                              cudaStream_t st, StageTimer* gemm_timer);

// Pools (Alg. 3 neighbour / neighbour's-neighbour loop).  X8 (nullable): the rows as
// bytes (data integers 0..255, same stride), read instead of X for the distances.
// own_first: the node's own kNN row first, then its neighbours' rows (the alternative
// reading of the loop).
void pool_run(const float* X, const uint8_t* X8, int ld, int d, int64_t n, const int32_t* knn,
              int K, int L, int exact, int32_t* pool_id, float* pool_d2, int32_t* pool_len,
              Counters* dctr, cudaStream_t st, int own_first = 0);

// Pools from arbitrary candidate lists (cand [n][KS], -1 padded): the L nearest by
// (d2, id), ordered exactly as pool_run orders its pools.  X8 as for pool_run.
void pool_from_candidates(const float* X, const uint8_t* X8, int ld, int d, int64_t n,
                          const int32_t* cand, int KS, int L, int exact, int32_t* pool_id,
                          float* pool_d2, int32_t* pool_len, Counters* dctr, cudaStream_t st);

// SSG prune of each node's pool.  border: decisions whose fp32 cosine lies within the
// rigorous fp32 bound plus border of cos(alpha) are re-taken in fp64, and those whose fp64
// cosine lies within border are counted in dctr->angle_border.
void prune_run(const float* X, int ld, int d, int64_t n, const int32_t* pool_id,
               const int32_t* pool_len, int L, int R, double cos_a, double border, int32_t* adj,
               int32_t* deg, Counters* dctr, cudaStream_t st, int wide_blocks = 0);

// The same prune, one node per thread block, for rows too long for the warp prune to keep
// its vectors beside the warp (prune_is_wide) and of at most 1,024 values
// (prune_wide_available): node i's candidates are cand[i * stride + t], t < len[i].
// blocks_per_sm (0: 2) sets how much shared memory each block takes for kept vectors.
bool prune_wide_available(int d);
// Whether prune_run takes the block prune: rows too long for the warp prune, and rows of
// 96 or more values, where the block prune was measured faster (200,000 16-centre float
// points, L = 200, R = 32: d = 96 29.3 -> 27.0 ms, 128 45.9 -> 26.8, 256 131.4 -> 27.8;
// d = 64 19.8 -> 27.9 and d = 32 10.1 -> 29.6 stay with the warp prune).
bool prune_block_preferred(int d, int R);
void prune_run_wide(const float* X, int ld, int d, int64_t n, const int32_t* cand,
                    const int32_t* len, int stride, int R, double cos_a, double border,
                    int32_t* adj, int32_t* deg, Counters* dctr, cudaStream_t st,
                    int blocks_per_sm = 0);

// One index's share of a batched prune (prune_run_batched).
struct PruneJob {
  const float* X;
  const int32_t* pool_id;
  const int32_t* pool_len;
  int32_t* adj;
  int32_t* deg;
  unsigned long long* n64;
  unsigned long long* nborder;
  double cosA64, border;
  int64_t n;
  int ld, d, L, R;
  float cosA32, margin;
};
// Launch parameters of the batched prune: warps per block (0: the largest that fits 96 KB
// of shared memory, at most 8) and the width of the pool-length buckets.
struct PruneTune {
  int warps = 0;
  int bucket_width = 32;
};
// The prune of every job's nodes in one persistent launch per row shape class (recorded in
// a CUDA graph and launched once); returns its device time in ms.  Synchronises `st`.
double prune_run_batched(const std::vector<PruneJob>& jobs, const PruneTune& tune, cudaStream_t st);

// The block prune over the work items of jobs that prune_block_preferred picks: the job
// table (each job's kept-vector capacity in shared memory), the spill slots and the launch
// shape, prepared before a stream capture; the launch itself allocates nothing.
struct WideBatchPlan {
  Scratch<unsigned char> jobs;
  Scratch<float> Vg;
  size_t vg_stride = 0, smem = 0;
  int grid = 0, nvr = 8;
};
void prune_wide_batched_prepare(const std::vector<PruneJob>& js, WideBatchPlan& plan,
                                cudaStream_t st);
void prune_wide_batched_launch(const WideBatchPlan& plan, const int2* items, int64_t nitems,
                               unsigned long long* next, cudaStream_t st);

// The same prune with each pool's Gram matrix on the tensor cores (data exact in bf16,
// d <= 128, L <= 127, R <= 128; true where that path is available).  split: pools of up to
// 63 candidates go to a launch of their own with smaller slots (for pools whose lengths
// vary widely, like the reverse merge's lists).
bool prune_tc_available(int d, int L, int R);
void prune_run_tc(const float* X, int ld, int d, int64_t n, const int32_t* pool_id,
                  const int32_t* pool_len, int L, int R, double cos_a, double border,
                  int32_t* adj, int32_t* deg, Counters* dctr, cudaStream_t st, bool split = false);

// Reverse-neighbour merge; returns the largest in-degree.  tc: the prune of lists of up to
// 127 candidates on the tensor cores where the data allow it.  X8 as for pool_run.
int reverse_run(const float* X, const uint8_t* X8, int ld, int d, int64_t n,
                const int32_t* adj0, const int32_t* deg0, int R, double cos_a, double border,
                int exact, bool tc, int32_t* adj1, int32_t* deg1, Counters* dctr,
                cudaStream_t st, int wide_blocks = 0);

// Connectivity from navigating nodes; returns the number of repair edges.  knn (nullable):
// the exact kNN graph [n][K] in (d2, id) order, which settles most repairs without a pass
// over all nodes (same result).
int64_t connect_run(const float* X, int ld, int d, int64_t n, int32_t* adj, int32_t* deg,
                    int R, const int32_t* nav_dev, const int32_t* nav_host, int n_nav,
                    cudaStream_t st, const int32_t* knn = nullptr, int K = 0,
                    int64_t* knn_repairs = nullptr);

// Search-on-Graph.  X: float rows at stride ld; X8 (nullable): the same values as bytes
// (integers 0..255) at the same stride, read instead of X when given (same results).
// work (nullable, device): totals of expansions, distance evaluations, adjacency entries.
void search_run(const float* X, const uint8_t* X8, int ld, int d, int64_t n, const int32_t* adj,
                const int32_t* deg, int R, const int32_t* nav, int n_nav, const float* Q,
                int ldq, int64_t nq, int k, int Ls, int32_t* out_ids, float* out_d2,
                cudaStream_t st, unsigned long long* work = nullptr);

// Search with a per-query k (qk) and pool size (qls <= ls_max); results at stride ldo.
void search_run_mixed(const float* X, const uint8_t* X8, int ld, int d, const int32_t* adj,
                      const int32_t* deg, int R, const int32_t* nav, int n_nav, const float* Q,
                      int ldq, int64_t nq, const int32_t* qk, const int32_t* qls, int ls_max,
                      int ldo, int32_t* out_ids, float* out_d2, cudaStream_t st);

// Byte copy [n][ld] of rows that hold integers 0..255 (ld: the float rows' stride, a
// multiple of 4; padding bytes 0).
void rows_to_u8(const float* X, int ld, int d, int64_t n, uint8_t* out, cudaStream_t st);

// Invariant checks (csrc/check.cu).  row = -1: every row passed; else the smallest failing
// row and its code.
enum CheckCode { CHECK_DEGREE = 1, CHECK_RANGE, CHECK_SELF, CHECK_DUPLICATE, CHECK_PADDING,
                 CHECK_ORDER };
struct CheckResult {
  int64_t row = -1;
  int code = 0;
};
CheckResult check_adj(const int32_t* adj, const int32_t* deg, int64_t n, int R, cudaStream_t st);
CheckResult check_pool(const int32_t* pid, const float* pd2, const int32_t* plen, int64_t n, int L,
                       int exact, int d, cudaStream_t st);
const char* check_name(int code);

// Bounded-wait self-test (csrc/selftest.cu): mode 0 times out, 1 aborts, 2 succeeds.
void wait_selftest(int mode, int* ok_host, int* elapsed_ms_host, cudaStream_t st);

// Padded view of X only (no statistics, no synchronisation).
void pad_rows(const float* X, int64_t n, int d, cudaStream_t st, PaddedRows& out);

// Smallest margin (in cos units) beyond which the fp32 angle test is certain.
inline float angle_margin_fp32(int d) { return (float)((2.0 * d + 20.0) * U32 * 1.1); }
// Relative error bound of an fp32 squared distance summed directly from differences.
inline float dist_rel_fp32(int d) { return (float)((d + 4.0) * U32 * 1.01); }
// The same for distances summed by team8_dist over rows of stride ld: each lane adds
// m = 4 ceil(ld / 32) squares of rounded differences with fused multiply-adds (at most
// (m + 2) units of roundoff relative to the sum of the squares: one per addition, two for
// the rounded difference squared), then three pairwise additions join the 8 lanes.
inline float dist_rel_team8(int ld) {
  return (float)((4.0 * ((ld + 31) / 32) + 6.0) * U32 * 1.01);
}
// The same for the compensated sums of team8_dist2 (warp_fill_dist_keys): 2u + u^2 from
// the rounded differences, u from the final rounding, and second-order terms in the error
// accumulator, at most (4 m^2 + 8 m + 1) u^2 with m = 4 ceil(ld / 32) terms per lane.
inline float dist_rel_team8c(int ld) {
  const double m = 4.0 * ((ld + 31) / 32);
  return (float)((3.0 + (4.0 * m * m + 8.0 * m + 2.0) * U32) * U32 * 1.01);
}

}  // namespace ssg
