/*
 * ssg.h -- C ABI of the GB300 (sm_103a) NSSG library.
 *
 * NSSG = Navigating Satellite System Graph, from "High Dimensional Similarity Search
 * with Satellite System Graph" (Fu, Wang, Cai; arXiv 1907.06146).  The library builds
 * the graph index of Alg. 3 (exact kNN graph -> 2-hop candidate pools -> SSG angle
 * prune -> reverse-neighbour merge -> connectivity from navigating nodes) and runs
 * Search-on-Graph (Alg. 1) from the nearest navigating node (Sec. 4.1).
 *
 * Conventions shared by every entry point:
 *  - Array arguments are DEVICE pointers owned by the caller unless the name ends in
 *    _host.  Vectors are float32, row-major, one row of d values per point.  Ids are
 *    int32 (n < 2^31).  Adjacency rows are int32 [n][R], padded with -1 after deg[i].
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream).  Staged entry points
 *    enqueue their kernels on it and return; ssg_build and ssg_connect synchronise the
 *    stream at stage boundaries to read sizes.
 *  - Scratch memory is taken from the CUDA stream-ordered allocator on `stream` and
 *    released before the call returns (in stream order).  At its first scratch
 *    allocation on a device the library sets that device's default pool to keep up to
 *    an eighth of the device memory reserved across synchronisations (the pool's release
 *    threshold), so that the stages of a build do not map their scratch afresh each time.
 *  - Errors come back as an ssg_status; nothing is thrown across the ABI.  After a
 *    non-OK status, ssg_last_error() gives a message for the calling thread.  EINVAL
 *    means an argument is out of range and nothing was enqueued.
 *  - Orders: every list the library returns is sorted by (squared distance, id)
 *    ascending; squared Euclidean distance orders like the distance of Sec. 2.1.
 *  - Results are exact with respect to double-precision arithmetic on the float32
 *    inputs: fast single-precision (or tensor-core) results decide only where a
 *    rigorous error bound separates them from the decision boundary, and the rest is
 *    re-decided in double precision (counters in ssg_build_stats).
 */
#ifndef SSG_H
#define SSG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SSG_OK = 0,
  SSG_EINVAL = 1,     /* an argument is out of range; nothing was enqueued */
  SSG_ENOMEM = 2,     /* a device allocation failed */
  SSG_ECUDA = 3,      /* a CUDA runtime call or kernel launch failed */
  SSG_ETIMEOUT = 4,   /* a bounded device wait gave up (device status word set) */
  SSG_EINTERNAL = 5,  /* an internal capacity or invariant was exceeded */
  SSG_EIO = 6         /* ssg_save / ssg_load could not read or write the file */
} ssg_status;

/* Arithmetic of the kNN distance GEMM (ssg_build_opts.gemm_prec, ssg_knn, ssg_knn_query)
 * and of the prune's Gram matrix (ssg_build_opts.gram_prec).  Every precision gives the
 * same exact result (the precision changes the speed, not the graph): a low-precision value
 * decides only where a rigorous error bound separates it from the decision boundary, and
 * the rest is re-decided from the float32 inputs in fp32 / fp64.
 *
 * kNN GEMM:
 *   FP32  single-precision SIMT GEMM form, top-(K + slack) re-ranked in fp64, each row
 *         certified against the GEMM's error bound (uncertified rows recomputed exhaustively).
 *   BF16  bf16 tcgen05 GEMM with fp32 accumulation (sm_103, d <= 4096: rows of up to 128
 *         values stay resident in shared memory, wider rows stream in 64-value chunks
 *         through 128 x 256 tiles).  On integer data
 *         that bf16 holds exactly the GEMM itself is exact.  On other data the rows are
 *         centred on the column mean before rounding, each row keeps the KS nearest by bf16
 *         distance (KS sized from a seeded sample of rows so that about 99% of rows
 *         certify), the candidates are re-ranked in fp64, and a row is certified when its
 *         K-th exact distance lies below the KS-th bf16 distance minus the rigorous bound
 *         |d2_bf16 - d2| <= (2^-7 + ..) |x - mu| max_y |y - mu| + ..; every other row is
 *         recomputed exhaustively (counted in ssg_build_stats.n_knn_fallback_rows).  Where
 *         that band would need more than 768 candidates (high intrinsic dimension, as in
 *         the GIST-shaped data), every value goes in as a bf16 pair hi + lo (three products
 *         per coordinate, K three times as long, error about 3 * 2^-16 |x| |y| plus the
 *         fp32 accumulation), for rows of up to 1,344 values
 *         (ssg_build_stats.knn_bf16_pairs).
 *         EINVAL where the tensor-core path does not run.
 *   AUTO  BF16 where the tensor-core path runs, FP32 otherwise (the default).
 *   BF16_RERANK  the same as BF16 (an older name of the mode).
 *   FP8   e4m3 with per-vector scales: not built yet (EINVAL).
 * Prune Gram (gram_prec):
 *   FP32  one warp per node, fp32 centred dot products, fp64 near cos(alpha).
 *   BF16  the pool's Gram matrix from one tcgen05 MMA where the data are exact in bf16
 *         (d <= 128, L <= 127); the FP32 prune elsewhere.  AUTO = BF16.  FP8: EINVAL. */
typedef enum {
  SSG_PREC_FP32 = 0,
  SSG_PREC_BF16 = 1,
  SSG_PREC_AUTO = 2,
  SSG_PREC_BF16_RERANK = 3,
  SSG_PREC_FP8 = 4
} ssg_precision;

typedef void* ssg_stream; /* cudaStream_t */

/* Build options.  Initialise with ssg_default_opts(). */
typedef struct {
  ssg_precision gemm_prec;  /* precision of the kNN distance GEMM */
  int32_t n_nav;            /* navigating nodes s (Alg. 3 input; Sec. 5.3 uses 10) */
  const int32_t* nav_ids_host; /* optional: n_nav distinct ids in [0, n) (host memory);
                                  NULL = draw them with ssg_nav_ids(n, n_nav, seed) */
  uint64_t seed;            /* seed for the navigating-node draw */
  int32_t debug_checks;     /* nonzero: after the pools, the prune, the reverse merge and
                               connectivity, check their arrays' invariants on the device
                               (ids in range, no self loops or repeats, degrees within the
                               cap, -1 padding, pools in order); a failure stops the build
                               with SSG_EINTERNAL naming the stage, the row and the rule */
  int32_t pool_tiles;       /* 0: Alg. 3 pools (the exact kNN graph, neighbours and their
                               neighbours).  > 0: Alg. 4 pools without a stored kNN graph:
                               each node's L nearest among the points of the pool_tiles
                               128-point tiles nearest to it in the cluster order (an
                               IVF-style index over k-means clusters of the data, searched
                               nearest cluster first); needs sm_103 and d <= 4096 (EINVAL
                               otherwise).  On data exact in bf16 the selection is exact;
                               on other data the tensor cores select L + slack candidates
                               by bf16 distance and each pool is re-ranked exactly (so a
                               pool may miss a point that only the exact distance ranks in) */
  int32_t pool_own_row_first; /* 0: Alg. 3's pool loop as printed (for each neighbour n in
                               kNN order: n, then knn(n); stop once >= L ids).  1: the node's
                               own kNN row first, whole, then its neighbours' rows until >= L
                               ids (with K >= L the pool is the L nearest neighbours) */
  ssg_precision gram_prec;  /* arithmetic of the prune's Gram matrix (see ssg_precision);
                               the reverse merge's prune follows it */
  double cos_margin_fp64;   /* reporting band of the angle test (Alg. 2): every decision whose
                               fp32 cosine lies within the fp32 error bound plus this band of
                               cos(alpha) is re-taken in fp64, and those whose fp64 cosine
                               lies within the band are counted in
                               ssg_build_stats.n_angle_borderline (default 1e-5; >= 0) */
  const char* tune_table;   /* NULL: built-in launch parameters.  Otherwise the path of a
                               text file of "name = value" lines (# starts a comment) that
                               sets launch parameters; unknown names, bad values or an
                               unreadable file give EINVAL.  Names: knn_sample_rows (rows
                               sampled to size the bf16 candidate slack, 0..4096),
                               knn_slack_quantile (fraction of sampled rows the slack must
                               certify, 0.5..1), knn_prepass_tiles (tiles of the first,
                               threshold-only walk of the tensor-core kNN, 0..4096, 0 = none),
                               knn_stream_rows (1: rows of up to 128 values also take the
                               K-chunked 128 x 256-tile kernel), prune_warps (warps per
                               block of the batched prune, 0 = automatic, up to 16),
                               prune_bucket_width (pool lengths per bucket of the batched
                               prune's longest-first order, 1..1024), knn_bf16_pairs (the
                               certified bf16 kNN's operands as bf16 pairs: 1 always, 0
                               never, -1 = automatic: where the sized single-bf16 band
                               needs more than 768 candidates), prune_wide_blocks
                               (blocks per SM of the block prune of rows of 330 to 1,024
                               values, 0 = automatic (2), up to 4; fewer blocks hold more
                               kept vectors in shared memory) */
} ssg_build_opts;

/* Per-build measurements (all times from CUDA events on the build stream). */
typedef struct {
  double ms_ingest, ms_knn, ms_pool, ms_prune, ms_reverse, ms_connect, ms_total;
  int64_t n_repair;             /* edges added by the connectivity step */
  int64_t n_angle_fp64;         /* angle decisions re-tested in fp64 (|cos - cos a| small) */
  int64_t n_order_fp64;         /* near-tie orderings re-sorted in fp64 */
  int64_t n_knn_fallback_rows;  /* kNN rows recomputed exhaustively in fp64 */
  int32_t max_indegree;         /* largest in-degree seen by the reverse merge */
  int32_t exact_mode;           /* 1 if the inputs are small integers (all fp32 exact) */
  int64_t kernel_launches;      /* kernels this call launched */
  int32_t gemm_prec_used;       /* ssg_precision actually used for the kNN GEMM */
  double ms_knn_gemm;           /* time of the distance-GEMM + selection kernel alone */
  int32_t search_row_bytes;     /* bytes per value of the rows this graph's searches read:
                                   1 for data that are integers 0..255 (the graph keeps a byte
                                   copy of the rows, used when ssg_search is given the base it
                                   was built from), 4 otherwise */
  int32_t gram_prec_used;       /* ssg_precision of the first prune's Gram (BF16 or FP32) */
  int64_t n_angle_borderline;   /* angle decisions whose fp64 cosine lies within
                                   cos_margin_fp64 of cos(alpha) (decided exactly, counted) */
  int32_t knn_candidates;       /* candidates per row of a bf16 kNN on data not exact in bf16
                                   (the sized KS), 0 otherwise */
  double ms_knn_certify;        /* of ms_knn on the certified bf16 path: all but the first
                                   tensor-core pass (centring, sizing KS, re-rank and
                                   certification, the passes over rows that failed) */
  int64_t n_repair_knn_row;     /* of n_repair, the edges whose node was found in the
                                   unreached node's own kNN row (same choice as a scan of all
                                   reached nodes, made without one) */
  int32_t knn_bf16_pairs;       /* 1 if the certified bf16 kNN sent every value as a bf16
                                   pair (hi + lo, three products per coordinate) because a
                                   single bf16's error band was too wide for these data */
} ssg_build_stats;

typedef struct ssg_graph ssg_graph; /* opaque, owned by the library; ssg_free releases it */

/* ---- housekeeping -------------------------------------------------------------------- */
void ssg_default_opts(ssg_build_opts* opts);
const char* ssg_strerror(ssg_status s);
const char* ssg_last_error(void);        /* message of the last failure on this thread */
/* Status of the most recent failure that a kernel reported through its device status word
 * (a bounded wait that gave up: SSG_ETIMEOUT; a capacity a kernel found exceeded:
 * SSG_EINTERNAL), in any thread since the previous call; SSG_OK if none.  Reading it
 * clears it.  The call that launched the kernel has returned the same status. */
ssg_status ssg_last_device_status(void);
int64_t ssg_kernel_launch_count(void);   /* kernels launched by this process so far */

/* Fault injection for tests, on the host: the nth stream-ordered scratch allocation from
 * now on (counted over all calls and threads) fails as an out-of-memory would, so that call
 * returns SSG_ENOMEM after releasing what it holds; nth <= 0 switches it off.  No device
 * fault is involved. */
void ssg_debug_fail_alloc(int64_t nth);

/* Invariant check of an adjacency (device int32 adj [n][R] -1 padded, deg [n]; R <= 128):
 * 0 <= deg <= R, listed ids in [0, n), no self loop, no id twice, -1 past the degree.  The
 * check reads the arrays within those shapes and never follows an id.  *bad_row_host = -1
 * when every row passes, else the smallest failing row, with *bad_code_host = 1 degree,
 * 2 id range, 3 self loop, 4 repeated id, 5 padding.  EINVAL for null pointers or R
 * outside [1, 128]. */
ssg_status ssg_check_graph(const int32_t* adj, const int32_t* deg, int64_t n, int32_t R,
                           int64_t* bad_row_host, int32_t* bad_code_host, ssg_stream stream);

/* Failure-detection self-test of the bounded waits inside the tensor-core kernels: one
 * kernel waits, with the library's own bounded mbarrier wait, on a barrier that nothing
 * completes (mode 0: it gives up after its 2 s limit; mode 1: another warp raises the
 * abort flag after 20 ms; mode 2: the barrier completes first).  *ok_host = 1 if the wait
 * succeeded, *elapsed_ms_host = the wait's duration.  No mode faults or hangs the GPU; the
 * kernel always returns and the context stays usable.  EINVAL for another mode. */
ssg_status ssg_selftest_wait(int32_t mode, int32_t* ok_host, int32_t* elapsed_ms_host);

/* Navigating nodes (Alg. 3: "random select s points"): s distinct ids in [0, n), the
 * successive SplitMix64 outputs (Steele, Lea, Flood 2014) modulo n with repeats skipped.
 * Host only; out_host has room for s ids.  EINVAL if s < 1 or s > n. */
ssg_status ssg_nav_ids(int64_t n, int32_t s, uint64_t seed, int32_t* out_host);

/* ---- staged entry points (each step of Alg. 3 / Alg. 1 on its own) --------------------- */

/* Exact kNN graph (Alg. 3 line 1, computed exactly): for every i, the K nearest j != i
 * by (d2, id).  knn_id int32 [n][K], knn_d2 float32 [n][K] (d2 rounded to float32).
 * EINVAL if n < 2, d < 1, K < 1, K > n - 1 or K > 700. */
ssg_status ssg_knn(const float* base, int64_t n, int32_t d, int32_t K, ssg_precision prec,
                   int32_t* knn_id, float* knn_d2, ssg_stream stream);

/* Brute-force ground truth for unindexed queries (serial scan, Sec. 5.3 item 8): the k
 * base points nearest each query by (d2, id).  ids int32 [nq][k], d2 float32 [nq][k].
 * EINVAL if k < 1, k > n or k > 768. */
ssg_status ssg_knn_query(const float* base, int64_t n, int32_t d, const float* queries,
                         int64_t nq, int32_t k, ssg_precision prec, int32_t* ids, float* d2,
                         ssg_stream stream);

/* Candidate pools (Alg. 3, neighbours and neighbours' neighbours of each node): walk
 * knn(i) in order, adding n and then knn(n), skipping i and repeats, and stop after the
 * first n at which the pool holds >= L ids; sort by (d2(i, .), id) and keep the first L.
 * pool_id int32 [n][L] (-1 padded), pool_d2 float32 [n][L], pool_len int32 [n].
 * EINVAL if L < 1 or L + K > 1023. */
ssg_status ssg_pool(const float* base, int64_t n, int32_t d, const int32_t* knn_id, int32_t K,
                    int32_t L, int32_t* pool_id, float* pool_d2, int32_t* pool_len,
                    ssg_stream stream);

/* SSG prune (Alg. 2 selection, applied to each pool by Alg. 3): keep the first candidate;
 * keep each later one unless cos(angle j-i-k) > cos(alpha) for a kept k (cos from the
 * centred dot products, 0 for a zero-length edge); stop once R are kept.
 * pool_id [n][L] sorted as ssg_pool leaves it; adj int32 [n][R], deg int32 [n].
 * EINVAL if R < 1, R > 128, d > 8192 or alpha outside (0, 180).  Rows too long for R + 1
 * of them to fit in shared memory keep the kept vectors in device scratch instead. */
ssg_status ssg_prune(const float* base, int64_t n, int32_t d, const int32_t* pool_id,
                     const int32_t* pool_len, int32_t L, int32_t R, double alpha_deg,
                     int32_t* adj, int32_t* deg, ssg_stream stream);

/* Reverse-neighbour merge (Alg. 3, reverse neighbour checking; Sec. 4.1): every node j
 * re-prunes adj0[j] united with {i : j in adj0[i]}, sorted by (d2(j, .), id), with the
 * same rule and cap R.  adj0/adj1 int32 [n][R]; deg0/deg1 int32 [n].
 * EINTERNAL if some node has more than 16383 candidates (in-degree + R). */
ssg_status ssg_reverse(const float* base, int64_t n, int32_t d, const int32_t* adj0,
                       const int32_t* deg0, int32_t R, double alpha_deg, int32_t* adj1,
                       int32_t* deg1, ssg_stream stream);

/* Connectivity from navigating nodes (Alg. 3, DFS-spanning from each node of NV; details
 * in the NSG paper): for each root in order, while some node is unreachable from it,
 * link the smallest unreached id u from the reached node v with deg(v) < R that minimises
 * (d2(v, u), id) and mark all reachable from u.  adj/deg are updated in place; nav is a
 * device array of n_nav ids; *n_repair_host receives the number of added edges.
 * EINTERNAL if an unreached node remains and no reached node has a free slot. */
ssg_status ssg_connect(const float* base, int64_t n, int32_t d, int32_t* adj, int32_t* deg,
                       int32_t R, const int32_t* nav, int32_t n_nav, int64_t* n_repair_host,
                       ssg_stream stream);

/* ssg_connect for callers that cannot allocate device memory while they run: serving
 * loops whose device memory is fixed before requests arrive, or hosts that forbid
 * allocations outside their own allocator.  The paper has no counterpart; this is a
 * deployment variant of the connectivity step above, with the same arguments and the same
 * result (every navigating id is checked before the graph is modified).  Like ssg_connect
 * it reads the navigating ids and each repair's state back to the host, synchronising the
 * stream each time.
 * Its scratch (reached-node bitmap, two frontier buffers, per-node fp32 distances, the
 * list of fp64 re-tests) lives in one fixed array of about 12.3 MiB inside the library's
 * device image, which every GPU that loads the library holds until the process exits.
 * The call itself allocates nothing: no cudaMalloc, cudaFree or allocating library call.
 * Limits: 1 <= n <= 1,048,576 nodes; d % 4 == 0 and `base` 16-byte aligned (no padded
 * copy is made); at most 16,384 candidate nodes may tie for the nearest reached node of
 * one repair (EINTERNAL otherwise; ssg_connect has no such limit).  EINVAL beyond the
 * size limits.  The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress, once per device, with that device current); make that first call
 * before any stream capture.  All calls share the one array and each starts by clearing
 * what must start at zero, so calls whose work overlaps on the GPU (other streams, other
 * host threads) race on it and must be serialised by the caller. */
ssg_status ssg_connect_noalloc(const float* base, int64_t n, int32_t d, int32_t* adj,
                               int32_t* deg, int32_t R, const int32_t* nav, int32_t n_nav,
                               int64_t* n_repair_host, ssg_stream stream);

/* Search-on-Graph (Alg. 1) from the navigating node nearest each query (Sec. 4.1): a pool
 * of at most L_search entries sorted by (d2, id); expand the first unchecked entry, add
 * every neighbour not visited before, re-sort, cut to L_search; stop when all entries are
 * checked; return the first k (padded with -1 / +inf).  out_d2 may be NULL.
 * EINVAL if k < 1, k > L_search or L_search > 1024. */
ssg_status ssg_search_adj(const float* base, int64_t n, int32_t d, const int32_t* adj,
                          const int32_t* deg, int32_t R, const int32_t* nav, int32_t n_nav,
                          const float* queries, int64_t nq, int32_t k, int32_t L_search,
                          int32_t* out_ids, float* out_d2, ssg_stream stream);

/* ssg_search_adj plus the work it did, summed over the batch into work_host[3]:
 * expansions (pool entries checked), distance evaluations (navigating nodes included;
 * a node met again after leaving the visited cache counts again) and adjacency entries
 * read.  These give the search's algorithmic bytes.  Synchronises the stream. */
ssg_status ssg_search_work(const float* base, int64_t n, int32_t d, const int32_t* adj,
                           const int32_t* deg, int32_t R, const int32_t* nav, int32_t n_nav,
                           const float* queries, int64_t nq, int32_t k, int32_t L_search,
                           int32_t* out_ids, float* out_d2, int64_t* work_host,
                           ssg_stream stream);

/* Hits for precision(R) = |R n G| / |G| (Sec. 5.2): the number of (query, id) pairs where
 * id is among the first k of both found [nq][ld_found] and truth [nq][ld_truth].
 * *hits_host receives the count (the call synchronises the stream). */
ssg_status ssg_recall_hits(const int32_t* found, int32_t ld_found, const int32_t* truth,
                           int32_t ld_truth, int64_t nq, int32_t k, int64_t* hits_host,
                           ssg_stream stream);

/* ---- whole build and search ---------------------------------------------------------- */

/* NSSGIndexing (Alg. 3) end to end on device-resident base vectors.  `base` must stay
 * alive and unchanged while the graph is searched.  *out receives a graph owned by the
 * library.  stats may be NULL.  When every value is an integer 0..255 the graph also
 * holds a byte copy of the rows (n x round_up(d, 4) bytes), which the build's pool and
 * reverse-merge distances and later searches given this same `base` read instead of the
 * float rows (same results). */
ssg_status ssg_build(const float* base, int64_t n, int32_t d, int32_t K, int32_t L, int32_t R,
                     double alpha_deg, const ssg_build_opts* opts, ssg_stream stream,
                     ssg_graph** out, ssg_build_stats* stats);

/* Same as ssg_build from HOST base vectors: the library copies them to a device buffer
 * that the graph owns, builds, and (when adj_host/deg_host are not NULL) copies the
 * adjacency [n][R] and degrees [n] back to host memory.  Pinned host memory is fastest. */
ssg_status ssg_build_host(const float* base_host, int64_t n, int32_t d, int32_t K, int32_t L,
                          int32_t R, double alpha_deg, const ssg_build_opts* opts,
                          ssg_stream stream, ssg_graph** out, int32_t* adj_host,
                          int32_t* deg_host, ssg_build_stats* stats);

/* Many independent indices at once (the multi-tenant case): index i is built from the
 * device array bases[i] (float32 [n[i]][d[i]]) with K[i], L[i], R[i], alpha_deg[i] and the
 * shared opts (its navigating nodes drawn from opts->seed; opts->nav_ids_host must be
 * NULL), into graphs[i].  Three phases: (1) every index's kNN graph and pools, on
 * n_streams (1..64) internal streams, each driven by its own host thread, the indices
 * dealt out largest first (n^2 d) to the least loaded stream; (2) one persistent prune
 * launch per row shape class over the (index, node) work items of every index (indices
 * whose data take the tensor-core Gram prune it in phase 1), the items bucketed by pool
 * length and handed out longest first, the launches recorded once into a CUDA graph and
 * replayed; (3) every index's reverse merge and connectivity, as in (1).  Launch
 * parameters come from opts->tune_table (see ssg_autotune_batched).  Each graph equals
 * what ssg_build returns for the same input, bit for bit.  stats (NULL or count entries)
 * gets each build's stats (ms_prune: the shared phase-2 time).  The call returns when every
 * build has finished; on failure it returns the first failing status, ssg_last_error()
 * names the index, and graphs[] holds no graph (all NULL). */
ssg_status ssg_build_batched(int32_t count, const float* const* bases, const int64_t* n,
                             const int32_t* d, const int32_t* K, const int32_t* L,
                             const int32_t* R, const double* alpha_deg,
                             const ssg_build_opts* opts, int32_t n_streams, ssg_graph** graphs,
                             ssg_build_stats* stats);

/* Autotuner of ssg_build_batched's launch parameters (no paper counterpart): on the four
 * largest indices of the batch (same arguments as ssg_build_batched) it times the batched
 * prune for 2, 4 and 8 warps per block and pool-length buckets 16, 64 and 1,024 wide, and
 * the resident (256 x 128 tiles) against the streamed (128 x 256 tiles) kNN kernel for
 * rows of up to 128 values, then writes the fastest choice as a tune_table file at path_out
 * (prune_warps, prune_bucket_width, knn_stream_rows).  best_ms_host (nullable, 2 entries)
 * receives the best batched-prune and kNN times.  EIO if the file cannot be written. */
ssg_status ssg_autotune_batched(int32_t count, const float* const* bases, const int64_t* n,
                                const int32_t* d, const int32_t* K, const int32_t* L,
                                const int32_t* R, const double* alpha_deg,
                                const ssg_build_opts* opts, const char* path_out,
                                double* best_ms_host);

/* Device views of a graph (no copies).  Any output pointer may be NULL. */
ssg_status ssg_graph_view(const ssg_graph* g, const int32_t** adj, const int32_t** deg,
                          const int32_t** nav, int32_t* n_nav, int32_t* R, int64_t* n,
                          int32_t* d);

/* Alg. 1 on a built graph.  `base` is the device array the graph was built from (NULL
 * for a graph from ssg_build_host, which owns its copy). */
ssg_status ssg_search(const ssg_graph* g, const float* base, const float* queries, int64_t nq,
                      int32_t k, int32_t L_search, int32_t* out_ids, float* out_d2,
                      ssg_stream stream);

/* Alg. 1 with HOST queries and results (copies inside; synchronises the stream).  Needs a
 * graph from ssg_build_host (which owns its device copy of the base); EINVAL otherwise. */
ssg_status ssg_search_host(const ssg_graph* g, const float* queries_host, int64_t nq, int32_t k,
                           int32_t L_search, int32_t* out_ids_host, float* out_d2_host,
                           ssg_stream stream);

/* ---- serving: continuous batching of searches -------------------------------------------
 * A server owns a scheduler thread and n_streams batch slots (CUDA streams with their own
 * pinned and device buffers).  Requests (a block of queries with one k and one L_search)
 * are submitted from any host thread and waited for by ticket.  Whenever a slot is free the
 * scheduler admits waiting requests first come, first served, while the batch stays within
 * max_batch queries and the device bytes of everything in flight (per query: the query row,
 * two parameters, k ids and k distances) stay within mem_budget_bytes; it then copies the
 * batch in, runs Alg. 1 for every query with its own k and L_search, and copies the results
 * out on that slot's stream.  Batches on different slots overlap on the device; requests
 * arriving meanwhile join the next free slot.  A query's result does not depend on the rest
 * of its batch.  The graph and `base` must outlive the server. */
typedef struct ssg_server ssg_server;
typedef struct {
  int32_t n_streams;        /* batch slots in flight (default 4) */
  int32_t max_batch;        /* queries per batch (default 8192); larger requests: EINVAL */
  int64_t mem_budget_bytes; /* device bytes of all queries in flight (default 256 MiB) */
  int32_t max_k;            /* largest k of a request (default 128) */
  int32_t max_L_search;     /* largest L_search of a request (default 1024) */
} ssg_server_opts;
typedef struct {
  int64_t requests_done, queries_done, batches;
  int64_t max_batches_in_flight;  /* most slots busy at once */
  int64_t max_queries_in_flight;  /* most queries on the device at once */
  double busy_ms;                 /* wall time with at least one batch in flight */
} ssg_server_stats;

void ssg_server_default_opts(ssg_server_opts* opts);
/* `base` = the device array the graph was built from (NULL for a graph from
 * ssg_build_host). */
ssg_status ssg_server_create(const ssg_graph* g, const float* base, const ssg_server_opts* opts,
                             ssg_server** out);
/* Copies the nq x d host queries; returns at once with a ticket. */
ssg_status ssg_server_submit(ssg_server* s, const float* queries_host, int64_t nq, int32_t k,
                             int32_t L_search, uint64_t* ticket);
ssg_status ssg_server_poll(ssg_server* s, uint64_t ticket, int32_t* done);
/* Blocks until the request is done; writes ids [nq][k] (and d2, nullable) to host memory,
 * the submit-to-done latency in ms (nullable), and forgets the ticket. */
ssg_status ssg_server_wait(ssg_server* s, uint64_t ticket, int32_t* ids_host, float* d2_host,
                           double* latency_ms);
ssg_status ssg_server_get_stats(ssg_server* s, ssg_server_stats* out);
/* Finishes every submitted request, then releases the server. */
void ssg_server_destroy(ssg_server* s);

/* Graph file: header (magic, version, n, d, R, n_nav, alpha) + nav + deg + adj. */
ssg_status ssg_save(const ssg_graph* g, const char* path);
ssg_status ssg_load(const char* path, ssg_graph** out);
void ssg_free(ssg_graph* g);

#ifdef __cplusplus
}
#endif

#endif /* SSG_H */
