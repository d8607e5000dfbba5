// C ABI entry points of the NSSG library (declared in include/ssg.h).
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <memory>
#include <new>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "common.cuh"
#include "graph.cuh"
#include "graph_dev.cuh"
#include "knn.cuh"

namespace ssg {

std::atomic<int64_t> g_launches{0};
std::atomic<int64_t> g_fail_alloc{0};
static std::atomic<int> g_dev_status{0};

void note_device_status(ssg_status s) { g_dev_status.store((int)s); }
thread_local int64_t t_launches = 0;
static thread_local char g_err[1024] = "";

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

double cos_alpha_of(double a) {
  if (a == 0.0) return 1.0;
  if (a == 60.0) return 0.5;
  if (a == 90.0) return 0.0;
  if (a == 120.0) return -0.5;
  if (a == 180.0) return -1.0;
  return std::cos(a * 3.14159265358979323846 / 180.0);
}

template <class F>
static ssg_status guard(F&& f) {
  try {
    f();
    return SSG_OK;
  } catch (const Fail& e) {
    return e.st;
  } catch (const std::bad_alloc&) {
    set_error("host allocation failed");
    return SSG_ENOMEM;
  } catch (...) {
    set_error("unexpected exception");
    return SSG_EINTERNAL;
  }
}

// Kernel that counts, per query, the ids found among the first k of both lists.
__global__ void k_recall_hits(const int32_t* __restrict__ found, int ldf,
                              const int32_t* __restrict__ truth, int ldt, int64_t nq, int k,
                              unsigned long long* __restrict__ hits) {
  const int64_t q = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (q >= nq) return;
  const int lane = lane_id();
  unsigned c = 0;
  for (int t = lane; t < k; t += 32) {
    const int32_t id = found[q * ldf + t];
    if (id < 0) continue;
    for (int u = 0; u < k; ++u)
      if (truth[q * ldt + u] == id) {
        ++c;
        break;
      }
  }
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if (lane == 0 && c) atomicAdd(hits, (unsigned long long)c);
}

static void check_alpha(double a) {
  SSG_REQUIRE(a > 0.0 && a < 180.0, SSG_EINVAL, "alpha must lie in (0, 180) degrees, got %g", a);
}
static void check_prune_fit(int d, int R) {
  SSG_REQUIRE(R >= 1 && R <= 128, SSG_EINVAL, "R must lie in [1, 128], got %d", R);
  SSG_REQUIRE(d >= 1 && d <= 8192, SSG_EINVAL, "d must lie in [1, 8192], got %d", d);
}

struct Ingested {
  PaddedRows rows;
  Scratch<float> norms;
  DataInfo info{};
};

// Length of each id row (the valid entries come first, -1 after them).
__global__ void k_pool_len_from_ids(const int32_t* __restrict__ ids, int64_t n, int L,
                                    int32_t* __restrict__ len) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int m = 0;
  while (m < L && ids[i * L + m] >= 0) ++m;
  len[i] = m;
}

// The prune on the tensor cores where the data are exact in bf16 (and the pool and degree
// fit its tile), the fp32 warp prune otherwise; both take the same decisions.  Returns the
// precision used.
static ssg_precision prune_dispatch(bool tc_ok, const float* X, int ld, int d, int64_t n,
                                    const int32_t* pool_id, const int32_t* pool_len, int L, int R,
                                    double cos_a, double border, int32_t* adj, int32_t* deg,
                                    Counters* ctr, cudaStream_t st, int wide_blocks = 0) {
  if (tc_ok && prune_tc_available(d, L, R)) {
    prune_run_tc(X, ld, d, n, pool_id, pool_len, L, R, cos_a, border, adj, deg, ctr, st);
    return SSG_PREC_BF16;
  }
  prune_run(X, ld, d, n, pool_id, pool_len, L, R, cos_a, border, adj, deg, ctr, st, wide_blocks);
  return SSG_PREC_FP32;
}

static void check_prec(ssg_precision p, const char* what) {
  SSG_REQUIRE((int)p >= 0 && (int)p <= 4, SSG_EINVAL, "%s: unknown precision %d", what, (int)p);
  SSG_REQUIRE(p != SSG_PREC_FP8, SSG_EINVAL,
              "%s: FP8 (e4m3 with per-vector scales) is not built; use BF16, FP32 or AUTO", what);
}

// The kNN GEMM a precision request takes on given data: 1 the bf16 tensor cores on data they
// hold exactly, 2 the certified bf16 path on other data, 0 the fp32 path.
static int knn_path(ssg_precision p, const DataInfo& info, int d) {
  if (p == SSG_PREC_FP32 || !knn_tc_available(d)) return 0;
  return info.bf16_exact ? 1 : 2;
}

// "name = value" lines of a launch-parameter file (ssg_build_opts.tune_table).
static KnnTune read_tune_table(const char* path) {
  KnnTune t;
  if (!path) return t;
  FILE* f = fopen(path, "r");
  SSG_REQUIRE(f, SSG_EINVAL, "tune_table: cannot open %s", path);
  std::unique_ptr<FILE, int (*)(FILE*)> fc(f, fclose);
  char line[512];
  int ln = 0;
  while (fgets(line, sizeof(line), f)) {
    ++ln;
    char* h = strchr(line, '#');
    if (h) *h = 0;
    char name[128];
    double v = 0.0;
    char tail[8];
    const int got = sscanf(line, " %127[A-Za-z0-9_] = %lf %7s", name, &v, tail);
    if (got <= 0) {
      char rest[8];
      SSG_REQUIRE(sscanf(line, " %7s", rest) <= 0, SSG_EINVAL, "tune_table %s:%d: cannot parse",
                  path, ln);
      continue;
    }
    SSG_REQUIRE(got == 2, SSG_EINVAL, "tune_table %s:%d: expected \"name = value\"", path, ln);
    if (!strcmp(name, "knn_sample_rows")) {
      SSG_REQUIRE(v >= 0 && v <= 4096 && v == std::floor(v), SSG_EINVAL,
                  "tune_table %s:%d: knn_sample_rows must be an integer in [0, 4096]", path, ln);
      t.sample_rows = (int)v;
    } else if (!strcmp(name, "knn_prepass_tiles")) {
      SSG_REQUIRE(v >= 0 && v <= 4096 && v == std::floor(v), SSG_EINVAL,
                  "tune_table %s:%d: knn_prepass_tiles must be an integer in [0, 4096]", path, ln);
      t.prepass_tiles = (int)v;
    } else if (!strcmp(name, "prune_warps")) {
      SSG_REQUIRE(v >= 0 && v <= 16 && v == std::floor(v), SSG_EINVAL,
                  "tune_table %s:%d: prune_warps must be an integer in [0, 16]", path, ln);
      t.prune_warps = (int)v;
    } else if (!strcmp(name, "prune_bucket_width")) {
      SSG_REQUIRE(v >= 1 && v <= 1024 && v == std::floor(v), SSG_EINVAL,
                  "tune_table %s:%d: prune_bucket_width must be an integer in [1, 1024]", path,
                  ln);
      t.prune_bucket_width = (int)v;
    } else if (!strcmp(name, "knn_bf16_pairs")) {
      SSG_REQUIRE(v >= -1 && v <= 1 && v == std::floor(v), SSG_EINVAL,
                  "tune_table %s:%d: knn_bf16_pairs must be -1, 0 or 1", path, ln);
      t.bf16_pairs = (int)v;
    } else if (!strcmp(name, "prune_wide_blocks")) {
      SSG_REQUIRE(v >= 0 && v <= 4 && v == std::floor(v), SSG_EINVAL,
                  "tune_table %s:%d: prune_wide_blocks must be an integer in [0, 4]", path, ln);
      t.prune_wide_blocks = (int)v;
    } else if (!strcmp(name, "knn_stream_rows")) {
      SSG_REQUIRE(v == 0 || v == 1, SSG_EINVAL, "tune_table %s:%d: knn_stream_rows must be 0 or 1",
                  path, ln);
      t.stream_rows = (int)v;
    } else if (!strcmp(name, "knn_slack_quantile")) {
      SSG_REQUIRE(v >= 0.5 && v <= 1.0, SSG_EINVAL,
                  "tune_table %s:%d: knn_slack_quantile must lie in [0.5, 1]", path, ln);
      t.slack_quantile = v;
    } else {
      SSG_REQUIRE(false, SSG_EINVAL, "tune_table %s:%d: unknown name %s", path, ln, name);
    }
  }
  return t;
}

static void ingest_all(const float* X, int64_t n, int d, cudaStream_t st, Ingested& g,
                       bool want_norms) {
  if (want_norms) g.norms.alloc((size_t)n, st);
  ingest(X, n, d, st, g.rows, want_norms ? g.norms.p : nullptr, &g.info);
}

}  // namespace ssg

using namespace ssg;

static const char* const kStatusNames[] = {"ok", "invalid argument", "out of device memory",
                                           "CUDA error", "device wait timed out",
                                           "internal capacity exceeded", "file I/O error"};

extern "C" {

void ssg_default_opts(ssg_build_opts* o) {
  if (!o) return;
  o->gemm_prec = SSG_PREC_AUTO;
  o->n_nav = 10;
  o->nav_ids_host = nullptr;
  o->seed = 190706145ull;
  o->debug_checks = 0;
  o->pool_tiles = 0;
  o->pool_own_row_first = 0;
  o->gram_prec = SSG_PREC_AUTO;
  o->cos_margin_fp64 = 1e-5;
  o->tune_table = nullptr;
}

const char* ssg_strerror(ssg_status s) {
  if ((int)s < 0 || (int)s > 6) return "unknown status";
  return kStatusNames[s];
}

const char* ssg_last_error(void) { return g_err; }

ssg_status ssg_last_device_status(void) { return (ssg_status)g_dev_status.exchange(0); }

int64_t ssg_kernel_launch_count(void) { return g_launches.load(); }

void ssg_debug_fail_alloc(int64_t nth) { g_fail_alloc.store(nth > 0 ? nth : 0); }

ssg_status ssg_check_graph(const int32_t* adj, const int32_t* deg, int64_t n, int32_t R,
                           int64_t* bad_row_host, int32_t* bad_code_host, ssg_stream stream) {
  return guard([&] {
    SSG_REQUIRE(adj && deg && bad_row_host && bad_code_host, SSG_EINVAL, "null pointer");
    SSG_REQUIRE(n >= 0 && R >= 1 && R <= 128, SSG_EINVAL, "need n >= 0 and 1 <= R <= 128");
    const CheckResult r = check_adj(adj, deg, n, R, (cudaStream_t)stream);
    *bad_row_host = r.row;
    *bad_code_host = r.code;
  });
}

ssg_status ssg_selftest_wait(int32_t mode, int32_t* ok_host, int32_t* elapsed_ms_host) {
  return guard([&] {
    SSG_REQUIRE(ok_host && elapsed_ms_host, SSG_EINVAL, "null pointer");
    SSG_REQUIRE(mode >= 0 && mode <= 2, SSG_EINVAL, "mode must be 0, 1 or 2");
    int ok = 0, ms = 0;
    wait_selftest(mode, &ok, &ms, (cudaStream_t)0);
    *ok_host = ok;
    *elapsed_ms_host = ms;
  });
}

ssg_status ssg_nav_ids(int64_t n, int32_t s, uint64_t seed, int32_t* out) {
  return guard([&] {
    SSG_REQUIRE(out && s >= 1 && s <= n, SSG_EINVAL, "need 1 <= s <= n (s=%d, n=%lld)", s,
                (long long)n);
    uint64_t state = seed;
    int got = 0;
    std::vector<char> seen;
    while (got < s) {
      state += 0x9E3779B97F4A7C15ull;
      uint64_t z = state;
      z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
      z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
      z ^= z >> 31;
      const int32_t v = (int32_t)(z % (uint64_t)n);
      bool dup = false;
      for (int t = 0; t < got; ++t) dup |= out[t] == v;
      if (!dup) out[got++] = v;
    }
  });
}

// The kNN rows of A against B (self: A is B) on the path the precision request and the
// data select: the exact bf16 tensor cores, the certified bf16 path, or the fp32 path.
static KnnResult knn_any(const Ingested& a, int64_t na, const Ingested& b, int64_t nb, int d,
                         const DataInfo& info, int self, int K, ssg_precision prec, int32_t* ids,
                         float* d2, bool exact_d2, const KnnTune& tune, Counters* ctr,
                         cudaStream_t st, StageTimer* t_gemm, CertResult* cr) {
  const int path = knn_path(prec, info, d);
  SSG_REQUIRE(prec != SSG_PREC_BF16 || path != 0, SSG_EINVAL,
              "bf16 distance GEMM needs sm_103 and d <= 4096");
  KnnResult kr;
  if (path == 1) {
    TcExtra ex;
    ex.prepass_tiles = tune.prepass_tiles;
    ex.stream_rows = tune.stream_rows;
    knn_exact_tc(a.rows.p, na, a.rows.ld, a.norms.p, b.rows.p, nb, b.rows.ld, b.norms.p, d, self, K,
                 ids, d2, st, t_gemm, 0, false, ex);
  } else if (path == 2) {
    const CertResult c = knn_bf16_certified(a.rows.p, na, a.rows.ld, a.norms.p, b.rows.p, nb,
                                            b.norms.p, d, info, self, K, ids, d2, exact_d2, tune,
                                            &ctr->order_fp64, st, t_gemm);
    kr.fallback_rows = c.fallback_rows;
    if (cr) *cr = c;
  } else {
    kr = knn_exact(a.rows.p, na, a.rows.ld, a.norms.p, b.rows.p, nb, b.rows.ld, b.norms.p, d, info,
                   self, K, ids, d2, st, t_gemm);
  }
  return kr;
}

ssg_status ssg_knn(const float* base, int64_t n, int32_t d, int32_t K, ssg_precision prec,
                   int32_t* knn_id, float* knn_d2, ssg_stream stream) {
  return guard([&] {
    SSG_REQUIRE(base && knn_id && knn_d2, SSG_EINVAL, "null pointer");
    SSG_REQUIRE(n >= 2 && n < (1ll << 31) && d >= 1, SSG_EINVAL, "need 2 <= n < 2^31 and d >= 1");
    SSG_REQUIRE(K >= 1 && K <= n - 1 && K <= 700, SSG_EINVAL, "need 1 <= K <= min(n - 1, 700)");
    check_prec(prec, "ssg_knn");
    cudaStream_t st = (cudaStream_t)stream;
    Ingested g;
    ingest_all(base, n, d, st, g, true);
    Scratch<Counters> ctr(1, st);
    SSG_CUDA(cudaMemsetAsync(ctr.p, 0, sizeof(Counters), st));
    knn_any(g, n, g, n, d, g.info, 1, K, prec, knn_id, knn_d2, true, KnnTune(), ctr.p, st, nullptr,
            nullptr);
  });
}

ssg_status ssg_knn_query(const float* base, int64_t n, int32_t d, const float* queries,
                         int64_t nq, int32_t k, ssg_precision prec, int32_t* ids, float* d2,
                         ssg_stream stream) {
  return guard([&] {
    SSG_REQUIRE(base && queries && ids && d2, SSG_EINVAL, "null pointer");
    SSG_REQUIRE(n >= 1 && n < (1ll << 31) && d >= 1 && nq >= 0, SSG_EINVAL, "bad sizes");
    SSG_REQUIRE(k >= 1 && k <= n && k <= 700, SSG_EINVAL, "need 1 <= k <= min(n, 700)");
    check_prec(prec, "ssg_knn_query");
    if (nq == 0) return;
    cudaStream_t st = (cudaStream_t)stream;
    Ingested gb, gq;
    ingest_all(base, n, d, st, gb, true);
    ingest_all(queries, nq, d, st, gq, true);
    DataInfo info;
    const float ma = std::max(gb.info.max_abs, gq.info.max_abs);
    info.nonneg = gb.info.nonneg && gq.info.nonneg;
    info.exact = gb.info.exact && gq.info.exact && exact_bound(d, ma, info.nonneg);
    info.bf16_exact = info.exact && ma <= 256.f;
    info.max_norm = gb.info.max_norm;
    info.max_abs = ma;
    Scratch<Counters> ctr(1, st);
    SSG_CUDA(cudaMemsetAsync(ctr.p, 0, sizeof(Counters), st));
    knn_any(gq, nq, gb, n, d, info, 0, k, prec, ids, d2, true, KnnTune(), ctr.p, st, nullptr,
            nullptr);
  });
}

ssg_status ssg_pool(const float* base, int64_t n, int32_t d, const int32_t* knn_id, int32_t K,
                    int32_t L, int32_t* pool_id, float* pool_d2, int32_t* pool_len,
                    ssg_stream stream) {
  return guard([&] {
    SSG_REQUIRE(base && knn_id && pool_id && pool_d2 && pool_len, SSG_EINVAL, "null pointer");
    SSG_REQUIRE(n >= 2 && d >= 1 && K >= 1 && K <= n - 1, SSG_EINVAL, "bad sizes");
    SSG_REQUIRE(L >= 1 && L + K <= 1023, SSG_EINVAL, "need L >= 1 and L + K <= 1023");
    cudaStream_t st = (cudaStream_t)stream;
    Ingested g;
    ingest_all(base, n, d, st, g, false);
    Scratch<Counters> ctr(1, st);
    SSG_CUDA(cudaMemsetAsync(ctr.p, 0, sizeof(Counters), st));
    pool_run(g.rows.p, nullptr, g.rows.ld, d, n, knn_id, K, L, g.info.exact, pool_id, pool_d2,
             pool_len,
             ctr.p, st);
  });
}

ssg_status ssg_prune(const float* base, int64_t n, int32_t d, const int32_t* pool_id,
                     const int32_t* pool_len, int32_t L, int32_t R, double alpha_deg,
                     int32_t* adj, int32_t* deg, ssg_stream stream) {
  return guard([&] {
    SSG_REQUIRE(base && pool_id && pool_len && adj && deg, SSG_EINVAL, "null pointer");
    SSG_REQUIRE(n >= 1 && d >= 1 && L >= 1, SSG_EINVAL, "bad sizes");
    check_alpha(alpha_deg);
    check_prune_fit(d, R);
    cudaStream_t st = (cudaStream_t)stream;
    Ingested g;
    ingest_all(base, n, d, st, g, false);
    Scratch<Counters> ctr(1, st);
    SSG_CUDA(cudaMemsetAsync(ctr.p, 0, sizeof(Counters), st));
    prune_dispatch(g.info.bf16_exact != 0, g.rows.p, g.rows.ld, d, n, pool_id, pool_len, L, R,
                   cos_alpha_of(alpha_deg), 1e-5, adj, deg, ctr.p, st);
  });
}

ssg_status ssg_reverse(const float* base, int64_t n, int32_t d, const int32_t* adj0,
                       const int32_t* deg0, int32_t R, double alpha_deg, int32_t* adj1,
                       int32_t* deg1, ssg_stream stream) {
  return guard([&] {
    SSG_REQUIRE(base && adj0 && deg0 && adj1 && deg1, SSG_EINVAL, "null pointer");
    SSG_REQUIRE(n >= 1 && d >= 1, SSG_EINVAL, "bad sizes");
    check_alpha(alpha_deg);
    check_prune_fit(d, R);
    cudaStream_t st = (cudaStream_t)stream;
    Ingested g;
    ingest_all(base, n, d, st, g, false);
    Scratch<Counters> ctr(1, st);
    SSG_CUDA(cudaMemsetAsync(ctr.p, 0, sizeof(Counters), st));
    reverse_run(g.rows.p, nullptr, g.rows.ld, d, n, adj0, deg0, R, cos_alpha_of(alpha_deg), 1e-5,
                g.info.exact, g.info.bf16_exact != 0, adj1, deg1, ctr.p, st);
  });
}

ssg_status ssg_connect(const float* base, int64_t n, int32_t d, int32_t* adj, int32_t* deg,
                       int32_t R, const int32_t* nav, int32_t n_nav, int64_t* n_repair_host,
                       ssg_stream stream) {
  return guard([&] {
    SSG_REQUIRE(base && adj && deg && nav, SSG_EINVAL, "null pointer");
    SSG_REQUIRE(n >= 1 && d >= 1 && R >= 1 && n_nav >= 1, SSG_EINVAL, "bad sizes");
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<int32_t> h((size_t)n_nav);
    SSG_CUDA(cudaMemcpyAsync(h.data(), nav, sizeof(int32_t) * n_nav, cudaMemcpyDeviceToHost, st));
    SSG_CUDA(cudaStreamSynchronize(st));
    for (int t = 0; t < n_nav; ++t)
      SSG_REQUIRE(h[t] >= 0 && h[t] < n, SSG_EINVAL, "navigating node id %d out of range", h[t]);
    Ingested g;
    ingest_all(base, n, d, st, g, false);
    const int64_t rep = connect_run(g.rows.p, g.rows.ld, d, n, adj, deg, R, nav, h.data(), n_nav, st);
    if (n_repair_host) *n_repair_host = rep;
  });
}

ssg_status ssg_search_adj(const float* base, int64_t n, int32_t d, const int32_t* adj,
                          const int32_t* deg, int32_t R, const int32_t* nav, int32_t n_nav,
                          const float* queries, int64_t nq, int32_t k, int32_t L_search,
                          int32_t* out_ids, float* out_d2, ssg_stream stream) {
  return guard([&] {
    SSG_REQUIRE(base && adj && deg && nav && queries && out_ids, SSG_EINVAL, "null pointer");
    SSG_REQUIRE(n >= 1 && d >= 1 && R >= 1 && R <= 128 && n_nav >= 1 && nq >= 0, SSG_EINVAL,
                "bad sizes");
    SSG_REQUIRE(k >= 1 && k <= L_search && L_search <= 1024, SSG_EINVAL,
                "need 1 <= k <= L_search <= 1024");
    if (nq == 0) return;
    cudaStream_t st = (cudaStream_t)stream;
    PaddedRows b, q;
    pad_rows(base, n, d, st, b);
    pad_rows(queries, nq, d, st, q);
    search_run(b.p, nullptr, b.ld, d, n, adj, deg, R, nav, n_nav, q.p, q.ld, nq, k, L_search,
               out_ids, out_d2, st);
  });
}

ssg_status ssg_search_work(const float* base, int64_t n, int32_t d, const int32_t* adj,
                           const int32_t* deg, int32_t R, const int32_t* nav, int32_t n_nav,
                           const float* queries, int64_t nq, int32_t k, int32_t L_search,
                           int32_t* out_ids, float* out_d2, int64_t* work_host,
                           ssg_stream stream) {
  return guard([&] {
    SSG_REQUIRE(base && adj && deg && nav && queries && out_ids && work_host, SSG_EINVAL,
                "null pointer");
    SSG_REQUIRE(n >= 1 && d >= 1 && R >= 1 && R <= 128 && n_nav >= 1 && nq >= 0, SSG_EINVAL,
                "bad sizes");
    SSG_REQUIRE(k >= 1 && k <= L_search && L_search <= 1024, SSG_EINVAL,
                "need 1 <= k <= L_search <= 1024");
    cudaStream_t st = (cudaStream_t)stream;
    Scratch<unsigned long long> w(3, st);
    SSG_CUDA(cudaMemsetAsync(w.p, 0, 3 * sizeof(unsigned long long), st));
    if (nq > 0) {
      PaddedRows b, q;
      pad_rows(base, n, d, st, b);
      pad_rows(queries, nq, d, st, q);
      search_run(b.p, nullptr, b.ld, d, n, adj, deg, R, nav, n_nav, q.p, q.ld, nq, k, L_search,
                 out_ids, out_d2, st, w.p);
    }
    unsigned long long h[3];
    SSG_CUDA(cudaMemcpyAsync(h, w.p, sizeof(h), cudaMemcpyDeviceToHost, st));
    SSG_CUDA(cudaStreamSynchronize(st));
    for (int t = 0; t < 3; ++t) work_host[t] = (int64_t)h[t];
  });
}

ssg_status ssg_recall_hits(const int32_t* found, int32_t ld_found, const int32_t* truth,
                           int32_t ld_truth, int64_t nq, int32_t k, int64_t* hits_host,
                           ssg_stream stream) {
  return guard([&] {
    SSG_REQUIRE(found && truth && hits_host, SSG_EINVAL, "null pointer");
    SSG_REQUIRE(k >= 1 && k <= ld_found && k <= ld_truth && nq >= 0, SSG_EINVAL, "bad sizes");
    cudaStream_t st = (cudaStream_t)stream;
    Scratch<unsigned long long> h(1, st);
    SSG_CUDA(cudaMemsetAsync(h.p, 0, sizeof(unsigned long long), st));
    if (nq > 0)
      SSG_LAUNCH(k_recall_hits, (unsigned)ceil_div(nq, 8), 256, 0, st, found, ld_found, truth,
                 ld_truth, nq, k, h.p);
    unsigned long long v = 0;
    SSG_CUDA(cudaMemcpyAsync(&v, h.p, sizeof(v), cudaMemcpyDeviceToHost, st));
    SSG_CUDA(cudaStreamSynchronize(st));
    *hits_host = (int64_t)v;
  });
}

// ---- the build in stages (Alg. 3) --------------------------------------------------------
// front: ingest, kNN graph (or Alg. 4's search-based pools) and pools; prune: the first SSG
// prune; back: reverse merge, connectivity and the stats.  ssg_build runs them in a row; a
// batch of indices runs every front, then one persistent prune over all of them, then every
// back.
struct BuildCtx {
  const float* base = nullptr;
  int64_t n = 0;
  int d = 0, K = 0, L = 0, R = 0;
  double alpha = 0.0;
  ssg_build_opts opts{};
  KnnTune tune;
  cudaStream_t st = nullptr;
  std::vector<int32_t> nav;
  std::unique_ptr<ssg_graph> g;
  Ingested in;
  Scratch<Counters> ctr;
  double cos_a = 0.0;
  int kpath = 0;
  bool gram_tc = false;
  CertResult cert;
  KnnResult kr;
  Scratch<int32_t> pool_id, pool_len, adj0, deg0;
  Scratch<int32_t> knn_id;  // the exact kNN graph, kept for the connectivity repairs
  Scratch<float> pool_d2;
  ssg_precision gram_used = SSG_PREC_FP32;
  int64_t launches = 0;  // kernels launched for this build, over the threads that ran it
  double prune_ms = -1.0;  // the shared batched prune's time (batched builds)
  int64_t n_repair = 0, n_repair_knn = 0;
  int max_indeg = 0;
  Counters hc{};
  std::unique_ptr<StageTimer> t_all, t_ing, t_knn, t_gemm, t_pool, t_prune, t_rev, t_con;
};

// Checks the arguments, draws the navigating nodes and allocates the graph (host work only
// until the graph's device arrays).
static void build_setup(BuildCtx& c, const float* base, int64_t n, int32_t d, int32_t K,
                        int32_t L, int32_t R, double alpha_deg, const ssg_build_opts* opts_in,
                        cudaStream_t st) {
  SSG_REQUIRE(base, SSG_EINVAL, "null pointer");
  ssg_default_opts(&c.opts);
  if (opts_in) c.opts = *opts_in;
  const ssg_build_opts& opts = c.opts;
  SSG_REQUIRE(n >= 2 && n < (1ll << 31) && d >= 1, SSG_EINVAL, "need 2 <= n < 2^31 and d >= 1");
  SSG_REQUIRE(K >= 1 && K <= n - 1 && K <= 700, SSG_EINVAL, "need 1 <= K <= min(n - 1, 700)");
  SSG_REQUIRE(L >= 1 && L + K <= 1023, SSG_EINVAL, "need L >= 1 and L + K <= 1023");
  check_alpha(alpha_deg);
  check_prune_fit(d, R);
  check_prec(opts.gemm_prec, "gemm_prec");
  check_prec(opts.gram_prec, "gram_prec");
  SSG_REQUIRE(opts.cos_margin_fp64 >= 0.0 && opts.cos_margin_fp64 <= 0.5, SSG_EINVAL,
              "cos_margin_fp64 must lie in [0, 0.5], got %g", opts.cos_margin_fp64);
  c.tune = read_tune_table(opts.tune_table);
  SSG_REQUIRE(opts.n_nav >= 1 && opts.n_nav <= n && opts.n_nav <= 4096, SSG_EINVAL,
              "need 1 <= n_nav <= min(n, 4096)");
  c.nav.resize((size_t)opts.n_nav);
  if (opts.nav_ids_host) {
    for (int t = 0; t < opts.n_nav; ++t) {
      c.nav[t] = opts.nav_ids_host[t];
      SSG_REQUIRE(c.nav[t] >= 0 && c.nav[t] < n, SSG_EINVAL, "navigating node %d out of range",
                  c.nav[t]);
      for (int u = 0; u < t; ++u)
        SSG_REQUIRE(c.nav[u] != c.nav[t], SSG_EINVAL, "navigating nodes must be distinct");
    }
  } else {
    ssg_status s = ssg_nav_ids(n, opts.n_nav, opts.seed, c.nav.data());
    if (s != SSG_OK) throw Fail{s};
  }
  c.base = base;
  c.n = n;
  c.d = d;
  c.K = K;
  c.L = L;
  c.R = R;
  c.alpha = alpha_deg;
  c.st = st;
  c.t_all.reset(new StageTimer(st, "ssg_build"));
  c.t_ing.reset(new StageTimer(st, "ingest"));
  c.t_knn.reset(new StageTimer(st, "knn graph"));
  c.t_gemm.reset(new StageTimer(st, "knn kernel"));
  c.t_pool.reset(new StageTimer(st, "pools"));
  c.t_prune.reset(new StageTimer(st, "prune"));
  c.t_rev.reset(new StageTimer(st, "reverse merge"));
  c.t_con.reset(new StageTimer(st, "connectivity"));
  c.g.reset(new ssg_graph());
  ssg_graph* g = c.g.get();
  g->n = n;
  g->d = d;
  g->R = R;
  g->n_nav = opts.n_nav;
  g->alpha = alpha_deg;
  g->nav_host = c.nav;
}

static void build_front(BuildCtx& c) {
  const int64_t l0 = t_launches;
  const int64_t n = c.n;
  const int d = c.d, K = c.K, L = c.L;
  const ssg_build_opts& opts = c.opts;
  cudaStream_t st = c.st;
  ssg_graph* g = c.g.get();
  c.t_all->start();
  SSG_CUDA(cudaMalloc(&g->adj, sizeof(int32_t) * n * c.R));
  SSG_CUDA(cudaMalloc(&g->deg, sizeof(int32_t) * n));
  SSG_CUDA(cudaMalloc(&g->nav_dev, sizeof(int32_t) * opts.n_nav));
  SSG_CUDA(cudaMemcpyAsync(g->nav_dev, c.nav.data(), sizeof(int32_t) * opts.n_nav,
                           cudaMemcpyHostToDevice, st));

  c.t_ing->start();
  ingest_all(c.base, n, d, st, c.in, true);
  Ingested& in = c.in;
  // integers 0..255: a byte copy of the rows (a quarter of the bytes, the same distances)
  // for the pool, reverse-merge and search distances
  if (in.info.exact && in.info.nonneg && in.info.max_abs <= 255.f) {
    SSG_CUDA(cudaMalloc(&g->rows_u8, (size_t)n * in.rows.ld));
    g->rows_ld = in.rows.ld;
    g->rows_src = c.base;
    rows_to_u8(in.rows.p, in.rows.ld, d, n, g->rows_u8, st);
  }
  c.t_ing->stop();
  c.ctr.alloc(1, st);
  SSG_CUDA(cudaMemsetAsync(c.ctr.p, 0, sizeof(Counters), st));
  c.cos_a = cos_alpha_of(c.alpha);

  const uint8_t* X8 = g->rows_u8;
  c.kpath = knn_path(opts.gemm_prec, in.info, d);
  const bool tc = c.kpath == 1;
  c.gram_tc = opts.gram_prec != SSG_PREC_FP32 && in.info.bf16_exact;
  SSG_REQUIRE(opts.gemm_prec != SSG_PREC_BF16 || c.kpath != 0, SSG_EINVAL,
              "bf16 distance GEMM needs sm_103 and d <= 4096");
  c.pool_id.alloc((size_t)n * L, st);
  c.pool_len.alloc((size_t)n, st);
  c.pool_d2.alloc((size_t)n * L, st);
  if (opts.pool_tiles > 0) {
    // a1 + a2 of Alg. 4: no kNN graph; each node's L nearest among the points of its
    // nearest pool_tiles tiles in the cluster order (the index searched on the fly)
    const bool tc_any = opts.gemm_prec != SSG_PREC_FP32 && knn_tc_available(d);
    SSG_REQUIRE(tc_any, SSG_EINVAL,
                "search-based pools (pool_tiles > 0) need the bf16 tensor-core path: sm_103 "
                "and d <= 4096");
    SSG_REQUIRE(knn_order_fits(n, 128), SSG_EINVAL, "search-based pools: n too large");
    const int lmax = knn_tc_max_k(d, true);
    SSG_REQUIRE(L <= lmax, SSG_EINVAL, "search-based pools: need L <= %d for d = %d", lmax, d);
    c.t_knn->start();
    if (tc) {
      // data exact in bf16: the selection itself is exact
      knn_exact_tc(in.rows.p, n, in.rows.ld, in.norms.p, in.rows.p, n, in.rows.ld, in.norms.p, d, 1,
                   L, c.pool_id.p, c.pool_d2.p, st, c.t_gemm.get(), opts.pool_tiles);
      c.t_knn->stop();
      in.norms.release();
      c.t_pool->start();
      SSG_LAUNCH(k_pool_len_from_ids, (unsigned)ceil_div(n, 256), 256, 0, st, c.pool_id.p, n, L,
                 c.pool_len.p);
      c.t_pool->stop();
    } else {
      // other data: a bf16 selection of L + slack candidates (approximate distances), then
      // each pool ordered from the original vectors as Alg. 3's pools are and cut to L
      const int Lp = (int)std::min<int64_t>(
          std::min(L + std::max(8, L / 4), knn_tc_max_k(d, true)), n - 1);
      Scratch<int32_t> cid((size_t)n * Lp, st);
      Scratch<float> cd2((size_t)n * Lp, st);
      knn_exact_tc(in.rows.p, n, in.rows.ld, in.norms.p, in.rows.p, n, in.rows.ld, in.norms.p, d, 1,
                   Lp, cid.p, cd2.p, st, c.t_gemm.get(), opts.pool_tiles, true);
      c.t_knn->stop();
      in.norms.release();
      c.t_pool->start();
      pool_from_candidates(in.rows.p, X8, in.rows.ld, d, n, cid.p, Lp, L, in.info.exact, c.pool_id.p,
                           c.pool_d2.p, c.pool_len.p, c.ctr.p, st);
      c.t_pool->stop();
    }
  } else {
    // a1: exact kNN graph
    c.knn_id.alloc((size_t)n * K, st);
    Scratch<int32_t>& knn_id = c.knn_id;
    Scratch<float> knn_d2((size_t)n * K, st);
    c.t_knn->start();
    c.kr = knn_any(in, n, in, n, d, in.info, 1, K, opts.gemm_prec, knn_id.p, knn_d2.p, false, c.tune,
                   c.ctr.p, st, c.t_gemm.get(), &c.cert);
    c.t_knn->stop();
    in.norms.release();

    // a2: candidate pools
    c.t_pool->start();
    pool_run(in.rows.p, X8, in.rows.ld, d, n, knn_id.p, K, L, in.info.exact, c.pool_id.p,
             c.pool_d2.p, c.pool_len.p, c.ctr.p, st, opts.pool_own_row_first);
    c.t_pool->stop();
  }
  if (opts.debug_checks) {
    const CheckResult r = check_pool(c.pool_id.p, c.pool_d2.p, c.pool_len.p, n, L, in.info.exact, d, st);
    SSG_REQUIRE(r.row < 0, SSG_EINTERNAL, "debug check after the pools: row %lld: %s",
                (long long)r.row, check_name(r.code));
  }
  c.adj0.alloc((size_t)n * c.R, st);
  c.deg0.alloc((size_t)n, st);
  c.launches += t_launches - l0;
}

// a3, one index at a time (a batch prunes on the warps in one persistent launch instead)
static void build_prune(BuildCtx& c) {
  const int64_t l0 = t_launches;
  c.t_prune->start();
  c.gram_used = prune_dispatch(c.gram_tc, c.in.rows.p, c.in.rows.ld, c.d, c.n, c.pool_id.p,
                               c.pool_len.p, c.L, c.R, c.cos_a, c.opts.cos_margin_fp64, c.adj0.p,
                               c.deg0.p, c.ctr.p, c.st, c.tune.prune_wide_blocks);
  c.t_prune->stop();
  c.launches += t_launches - l0;
}

static void build_back(BuildCtx& c) {
  const int64_t l0 = t_launches;
  const int64_t n = c.n;
  const int d = c.d, R = c.R;
  cudaStream_t st = c.st;
  ssg_graph* g = c.g.get();
  Ingested& in = c.in;
  auto debug_check = [&](const CheckResult& r, const char* stage) {
    SSG_REQUIRE(r.row < 0, SSG_EINTERNAL, "debug check after %s: row %lld: %s", stage,
                (long long)r.row, check_name(r.code));
  };
  if (c.opts.debug_checks) debug_check(check_adj(c.adj0.p, c.deg0.p, n, R, st), "the prune");
  c.pool_id.release();
  c.pool_d2.release();
  c.pool_len.release();

  // a4: reverse-neighbour merge
  c.t_rev->start();
  c.max_indeg = reverse_run(in.rows.p, g->rows_u8, in.rows.ld, d, n, c.adj0.p, c.deg0.p, R,
                                c.cos_a, c.opts.cos_margin_fp64, in.info.exact, c.gram_tc, g->adj,
                                g->deg, c.ctr.p, st, c.tune.prune_wide_blocks);
  c.t_rev->stop();
  if (c.opts.debug_checks) debug_check(check_adj(g->adj, g->deg, n, R, st), "the reverse merge");
  c.adj0.release();
  c.deg0.release();

  // a5: connectivity from the navigating nodes
  c.t_con->start();
  c.n_repair = connect_run(in.rows.p, in.rows.ld, d, n, g->adj, g->deg, R, g->nav_dev,
                           c.nav.data(), c.opts.n_nav, st, c.knn_id.p, c.knn_id.p ? c.K : 0, &c.n_repair_knn);
  c.knn_id.release();
  c.t_con->stop();
  if (c.opts.debug_checks) debug_check(check_adj(g->adj, g->deg, n, R, st), "connectivity");
  c.t_all->stop();

  SSG_CUDA(cudaMemcpyAsync(&c.hc, c.ctr.p, sizeof(c.hc), cudaMemcpyDeviceToHost, st));
  SSG_CUDA(cudaStreamSynchronize(st));
  c.launches += t_launches - l0;
}

// The per-build measurements of a finished build.
static void build_stats(BuildCtx& c, ssg_build_stats* stats) {
  const Counters& hc = c.hc;
  ssg_build_stats S{};
  S.ms_ingest = c.t_ing->ms();
  S.ms_knn = c.t_knn->ms();
  S.ms_knn_gemm = c.t_gemm->ms();
  S.ms_pool = c.t_pool->ms();
  S.ms_prune = c.prune_ms >= 0.0 ? c.prune_ms : c.t_prune->ms();
  S.ms_reverse = c.t_rev->ms();
  S.ms_connect = c.t_con->ms();
  S.ms_total = c.t_all->ms();
  S.n_repair = c.n_repair;
  S.n_repair_knn_row = c.n_repair_knn;
  S.knn_bf16_pairs = c.cert.pairs;
  S.n_angle_fp64 = (int64_t)hc.angle_fp64;
  S.n_order_fp64 = (int64_t)hc.order_fp64;
  S.n_knn_fallback_rows = c.kr.fallback_rows;
  S.max_indegree = c.max_indeg;
  S.exact_mode = c.in.info.exact;
  S.gemm_prec_used = c.kpath == 0 ? SSG_PREC_FP32 : SSG_PREC_BF16;
  S.gram_prec_used = c.gram_used;
  S.n_angle_borderline = (int64_t)hc.angle_border;
  S.knn_candidates = c.cert.candidates;
  S.ms_knn_certify = c.kpath == 2 && c.opts.pool_tiles == 0 ? S.ms_knn - S.ms_knn_gemm : 0.0;
  S.kernel_launches = c.launches;
  S.search_row_bytes = c.g->rows_u8 ? 1 : 4;
  *stats = S;
}

ssg_status ssg_build(const float* base, int64_t n, int32_t d, int32_t K, int32_t L, int32_t R,
                     double alpha_deg, const ssg_build_opts* opts_in, ssg_stream stream,
                     ssg_graph** out, ssg_build_stats* stats) {
  return guard([&] {
    SSG_REQUIRE(out, SSG_EINVAL, "null pointer");
    *out = nullptr;
    BuildCtx c;
    build_setup(c, base, n, d, K, L, R, alpha_deg, opts_in, (cudaStream_t)stream);
    build_front(c);
    build_prune(c);
    build_back(c);
    if (stats) build_stats(c, stats);
    *out = c.g.release();
  });
}

ssg_status ssg_build_batched(int32_t count, const float* const* bases, const int64_t* n,
                             const int32_t* d, const int32_t* K, const int32_t* L,
                             const int32_t* R, const double* alpha_deg,
                             const ssg_build_opts* opts, int32_t n_streams, ssg_graph** graphs,
                             ssg_build_stats* stats) {
  return guard([&] {
    SSG_REQUIRE(count >= 0, SSG_EINVAL, "count must be >= 0");
    if (count == 0) return;
    SSG_REQUIRE(bases && n && d && K && L && R && alpha_deg && graphs, SSG_EINVAL, "null pointer");
    SSG_REQUIRE(n_streams >= 1 && n_streams <= 64, SSG_EINVAL, "need 1 <= n_streams <= 64");
    SSG_REQUIRE(!opts || !opts->nav_ids_host, SSG_EINVAL,
                "batched builds draw navigating nodes from the seed (nav_ids_host must be NULL)");
    for (int32_t i = 0; i < count; ++i) graphs[i] = nullptr;
    int dev = 0;
    SSG_CUDA(cudaGetDevice(&dev));
    const int nt = std::min<int32_t>(n_streams, count);
    std::vector<cudaStream_t> streams((size_t)nt + 1, nullptr);
    struct StreamsGuard {
      std::vector<cudaStream_t>& v;
      ~StreamsGuard() {
        for (cudaStream_t s : v)
          if (s) cudaStreamDestroy(s);
      }
    } sg{streams};
    for (int t = 0; t <= nt; ++t)
      SSG_CUDA(cudaStreamCreateWithFlags(&streams[t], cudaStreamNonBlocking));
    // every index checked and set up first (host work), so that no build starts on a batch
    // with a bad member
    std::vector<std::unique_ptr<BuildCtx>> ctx((size_t)count);
    for (int32_t i = 0; i < count; ++i) {
      ctx[i].reset(new BuildCtx());
      try {
        build_setup(*ctx[i], bases[i], n[i], d[i], K[i], L[i], R[i], alpha_deg[i], opts, nullptr);
      } catch (const Fail& e) {
        const std::string m = ssg_last_error();
        set_error("index %d: %s", i, m.c_str());
        throw;
      }
    }
    // the largest work (n^2 d: the kNN graph dominates) first, each index to the least
    // loaded stream, so every stream's share ends at about the same time
    std::vector<int32_t> order((size_t)count);
    for (int32_t i = 0; i < count; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
      return (double)n[a] * n[a] * d[a] > (double)n[b] * n[b] * d[b];
    });
    std::vector<std::vector<int32_t>> share((size_t)nt);
    std::vector<double> load((size_t)nt, 0.0);
    for (int32_t i : order) {
      const int t = (int)(std::min_element(load.begin(), load.end()) - load.begin());
      share[t].push_back(i);
      load[t] += (double)n[i] * n[i] * d[i];
      ctx[i]->st = streams[t];
    }
    // rebuild the stage timers on the index's stream
    for (int32_t i = 0; i < count; ++i) {
      BuildCtx& c = *ctx[i];
      c.t_all.reset(new StageTimer(c.st, "ssg_build"));
      c.t_ing.reset(new StageTimer(c.st, "ingest"));
      c.t_knn.reset(new StageTimer(c.st, "knn graph"));
      c.t_gemm.reset(new StageTimer(c.st, "knn kernel"));
      c.t_pool.reset(new StageTimer(c.st, "pools"));
      c.t_prune.reset(new StageTimer(c.st, "prune"));
      c.t_rev.reset(new StageTimer(c.st, "reverse merge"));
      c.t_con.reset(new StageTimer(c.st, "connectivity"));
    }
    std::mutex mu;
    ssg_status first = SSG_OK;
    std::string first_msg;
    auto fail = [&](int32_t i, ssg_status s) {
      std::lock_guard<std::mutex> lk(mu);
      if (first == SSG_OK) {
        first = s;
        first_msg = "index " + std::to_string(i) + ": " + ssg_last_error();
      }
    };
    auto run_phase = [&](auto&& body) {
      std::vector<std::thread> pool;
      for (int t = 0; t < nt; ++t)
        pool.emplace_back([&, t] {
          cudaSetDevice(dev);
          for (int32_t i : share[t]) {
            {
              std::lock_guard<std::mutex> lk(mu);
              if (first != SSG_OK) break;
            }
            const ssg_status s = guard([&] { body(*ctx[i]); });
            if (s != SSG_OK) fail(i, s);
          }
          cudaStreamSynchronize(streams[t]);
        });
      for (auto& th : pool) th.join();
    };
    // 1: every index's kNN graph and pools (indices whose data allow the tensor-core Gram
    // prune it right away)
    run_phase([&](BuildCtx& c) {
      build_front(c);
      if (c.gram_tc) build_prune(c);
    });
    SSG_REQUIRE(first == SSG_OK, first, "%s", first_msg.c_str());
    // 2: every other index's prune in one persistent launch over (index, node) items
    std::vector<PruneJob> jobs;
    std::vector<int32_t> jobs_of;
    for (int32_t i = 0; i < count; ++i) {
      BuildCtx& c = *ctx[i];
      if (c.gram_tc) continue;
      PruneJob j{};
      j.X = c.in.rows.p;
      j.pool_id = c.pool_id.p;
      j.pool_len = c.pool_len.p;
      j.adj = c.adj0.p;
      j.deg = c.deg0.p;
      j.n64 = &c.ctr.p->angle_fp64;
      j.nborder = &c.ctr.p->angle_border;
      j.cosA64 = c.cos_a;
      j.border = c.opts.cos_margin_fp64;
      j.n = c.n;
      j.ld = c.in.rows.ld;
      j.d = c.d;
      j.L = c.L;
      j.R = c.R;
      j.cosA32 = (float)c.cos_a;
      j.margin = angle_margin_fp32(c.d) + (float)c.opts.cos_margin_fp64;
      jobs.push_back(j);
      jobs_of.push_back(i);
    }
    if (!jobs.empty()) {
      PruneTune pt;
      pt.warps = ctx[0]->tune.prune_warps;
      pt.bucket_width = ctx[0]->tune.prune_bucket_width;
      const double ms = prune_run_batched(jobs, pt, streams[nt]);
      for (int32_t i : jobs_of) {
        ctx[i]->gram_used = SSG_PREC_FP32;
        ctx[i]->prune_ms = ms;
      }
    }
    // 3: every index's reverse merge and connectivity
    run_phase([&](BuildCtx& c) { build_back(c); });
    SSG_REQUIRE(first == SSG_OK, first, "%s", first_msg.c_str());
    for (int32_t i = 0; i < count; ++i) {
      if (stats) build_stats(*ctx[i], &stats[i]);
      graphs[i] = ctx[i]->g.release();
    }
  });
}

ssg_status ssg_autotune_batched(int32_t count, const float* const* bases, const int64_t* n,
                               const int32_t* d, const int32_t* K, const int32_t* L,
                               const int32_t* R, const double* alpha_deg,
                               const ssg_build_opts* opts, const char* path_out,
                               double* best_ms_host) {
  return guard([&] {
    SSG_REQUIRE(count >= 1 && bases && n && d && K && L && R && alpha_deg && path_out, SSG_EINVAL,
                "need count >= 1 and non-null arrays and path");
    SSG_REQUIRE(!opts || !opts->nav_ids_host, SSG_EINVAL, "nav_ids_host must be NULL");
    cudaStream_t st = nullptr;
    SSG_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    struct SG {
      cudaStream_t s;
      ~SG() { cudaStreamDestroy(s); }
    } sg{st};
    // the sample: the four largest indices (by n^2 d), with the kNN graphs and pools the
    // batched build would compute
    std::vector<int32_t> order((size_t)count);
    for (int32_t i = 0; i < count; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
      return (double)n[a] * n[a] * d[a] > (double)n[b] * n[b] * d[b];
    });
    order.resize((size_t)std::min<int32_t>(count, 4));
    std::vector<std::unique_ptr<BuildCtx>> ctx;
    double knn_ms[2] = {0.0, 0.0};
    for (int32_t i : order) {
      ctx.emplace_back(new BuildCtx());
      BuildCtx& c = *ctx.back();
      build_setup(c, bases[i], n[i], d[i], K[i], L[i], R[i], alpha_deg[i], opts, st);
      if (knn_tc_available(d[i]) && d[i] <= 128 && c.opts.gemm_prec != SSG_PREC_FP32 &&
          c.opts.pool_tiles == 0) {
        // the kNN kernel: resident 256 x 128 tiles against streamed 128 x 256 tiles
        for (int w = 0; w < 2; ++w) {
          Ingested in;
          ingest_all(bases[i], n[i], d[i], st, in, true);
          Scratch<int32_t> ids((size_t)n[i] * K[i], st);
          Scratch<float> dd((size_t)n[i] * K[i], st);
          Scratch<Counters> ct(1, st);
          SSG_CUDA(cudaMemsetAsync(ct.p, 0, sizeof(Counters), st));
          KnnTune t = c.tune;
          t.stream_rows = w;
          StageTimer tm(st);
          tm.start();
          knn_any(in, n[i], in, n[i], d[i], in.info, 1, K[i], c.opts.gemm_prec, ids.p, dd.p, false, t,
                  ct.p, st, nullptr, nullptr);
          tm.stop();
          knn_ms[w] += tm.ms();
        }
      }
      build_front(c);
    }
    std::vector<PruneJob> jobs;
    for (auto& cp : ctx) {
      BuildCtx& c = *cp;
      PruneJob j{};
      j.X = c.in.rows.p;
      j.pool_id = c.pool_id.p;
      j.pool_len = c.pool_len.p;
      j.adj = c.adj0.p;
      j.deg = c.deg0.p;
      j.n64 = &c.ctr.p->angle_fp64;
      j.nborder = &c.ctr.p->angle_border;
      j.cosA64 = c.cos_a;
      j.border = c.opts.cos_margin_fp64;
      j.n = c.n;
      j.ld = c.in.rows.ld;
      j.d = c.d;
      j.L = c.L;
      j.R = c.R;
      j.cosA32 = (float)c.cos_a;
      j.margin = angle_margin_fp32(c.d) + (float)c.opts.cos_margin_fp64;
      jobs.push_back(j);
    }
    // the batched prune: warps per block x pool-length bucket width, best of two runs each
    PruneTune best;
    double best_ms = 1e300;
    for (int warps : {2, 4, 8})
      for (int width : {16, 64, 1024}) {
        PruneTune t;
        t.warps = warps;
        t.bucket_width = width;
        double ms = 1e300;
        try {
          for (int r = 0; r < 2; ++r) ms = std::min(ms, prune_run_batched(jobs, t, st));
        } catch (const Fail&) {
          continue;  // this many warps do not fit shared memory for these rows
        }
        if (ms < best_ms) {
          best_ms = ms;
          best = t;
        }
      }
    SSG_REQUIRE(best_ms < 1e300, SSG_EINTERNAL, "autotune: no batched prune configuration ran");
    const int stream_rows = knn_ms[0] > 0.0 && knn_ms[1] < knn_ms[0] ? 1 : 0;
    FILE* f = fopen(path_out, "w");
    SSG_REQUIRE(f, SSG_EIO, "cannot open %s for writing", path_out);
    const bool ok =
        fprintf(f,
                "# launch parameters chosen by ssg_autotune_batched on the %d largest of %d "
                "indices\n# batched prune %.3f ms; kNN kernel resident %.3f ms, streamed %.3f ms\n"
                "prune_warps = %d\nprune_bucket_width = %d\nknn_stream_rows = %d\n",
                (int)order.size(), count, best_ms, knn_ms[0], knn_ms[1], best.warps,
                best.bucket_width, stream_rows) > 0;
    SSG_REQUIRE(fclose(f) == 0 && ok, SSG_EIO, "short write to %s", path_out);
    if (best_ms_host) {
      best_ms_host[0] = best_ms;
      best_ms_host[1] = std::min(knn_ms[0], knn_ms[1] > 0.0 ? knn_ms[1] : knn_ms[0]);
    }
  });
}

ssg_status ssg_build_host(const float* base_host, int64_t n, int32_t d, int32_t K, int32_t L,
                          int32_t R, double alpha_deg, const ssg_build_opts* opts,
                          ssg_stream stream, ssg_graph** out, int32_t* adj_host, int32_t* deg_host,
                          ssg_build_stats* stats) {
  float* dev = nullptr;
  ssg_status s = guard([&] {
    SSG_REQUIRE(base_host && out && n >= 2 && d >= 1, SSG_EINVAL, "bad arguments");
    cudaStream_t st = (cudaStream_t)stream;
    SSG_CUDA(cudaMalloc(&dev, sizeof(float) * n * d));
    SSG_CUDA(cudaMemcpyAsync(dev, base_host, sizeof(float) * n * d, cudaMemcpyHostToDevice, st));
  });
  if (s != SSG_OK) {
    if (dev) cudaFree(dev);
    return s;
  }
  s = ssg_build(dev, n, d, K, L, R, alpha_deg, opts, stream, out, stats);
  if (s != SSG_OK) {
    cudaFree(dev);
    return s;
  }
  (*out)->base_owned = dev;
  return guard([&] {
    cudaStream_t st = (cudaStream_t)stream;
    if (adj_host)
      SSG_CUDA(cudaMemcpyAsync(adj_host, (*out)->adj, sizeof(int32_t) * n * R,
                               cudaMemcpyDeviceToHost, st));
    if (deg_host)
      SSG_CUDA(cudaMemcpyAsync(deg_host, (*out)->deg, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, st));
    SSG_CUDA(cudaStreamSynchronize(st));
  });
}

ssg_status ssg_graph_view(const ssg_graph* g, const int32_t** adj, const int32_t** deg,
                          const int32_t** nav, int32_t* n_nav, int32_t* R, int64_t* n, int32_t* d) {
  if (!g) {
    set_error("null graph");
    return SSG_EINVAL;
  }
  if (adj) *adj = g->adj;
  if (deg) *deg = g->deg;
  if (nav) *nav = g->nav_dev;
  if (n_nav) *n_nav = g->n_nav;
  if (R) *R = g->R;
  if (n) *n = g->n;
  if (d) *d = g->d;
  return SSG_OK;
}

ssg_status ssg_search(const ssg_graph* g, const float* base, const float* queries, int64_t nq,
                      int32_t k, int32_t L_search, int32_t* out_ids, float* out_d2,
                      ssg_stream stream) {
  if (!g) {
    set_error("null graph");
    return SSG_EINVAL;
  }
  const float* b = base ? base : g->base_owned;
  if (!b) {
    set_error("no base vectors: pass the device array the graph was built from");
    return SSG_EINVAL;
  }
  if (!(g->rows_u8 && b == g->rows_src))
    return ssg_search_adj(b, g->n, g->d, g->adj, g->deg, g->R, g->nav_dev, g->n_nav, queries, nq,
                          k, L_search, out_ids, out_d2, stream);
  // the base the graph was built from, held as bytes: search the byte rows
  return guard([&] {
    SSG_REQUIRE(queries && out_ids, SSG_EINVAL, "null pointer");
    SSG_REQUIRE(k >= 1 && k <= L_search && L_search <= 1024, SSG_EINVAL,
                "need 1 <= k <= L_search <= 1024");
    SSG_REQUIRE(nq >= 0, SSG_EINVAL, "bad sizes");
    if (nq == 0) return;
    cudaStream_t st = (cudaStream_t)stream;
    PaddedRows q;
    pad_rows(queries, nq, g->d, st, q);
    SSG_REQUIRE(q.ld == g->rows_ld, SSG_EINTERNAL, "byte rows: stride %d, queries %d", g->rows_ld,
                q.ld);
    search_run(b, g->rows_u8, g->rows_ld, g->d, g->n, g->adj, g->deg, g->R, g->nav_dev, g->n_nav,
               q.p, q.ld, nq, k, L_search, out_ids, out_d2, st);
  });
}

ssg_status ssg_search_host(const ssg_graph* g, const float* queries_host, int64_t nq, int32_t k,
                           int32_t L_search, int32_t* out_ids_host, float* out_d2_host,
                           ssg_stream stream) {
  return guard([&] {
    SSG_REQUIRE(g && g->base_owned, SSG_EINVAL, "ssg_search_host needs a graph from ssg_build_host");
    SSG_REQUIRE(queries_host && out_ids_host && nq >= 0, SSG_EINVAL, "bad arguments");
    if (nq == 0) return;
    cudaStream_t st = (cudaStream_t)stream;
    Scratch<float> q((size_t)nq * g->d, st);
    Scratch<int32_t> ids((size_t)nq * k, st);
    Scratch<float> dd((size_t)nq * k, st);
    SSG_CUDA(cudaMemcpyAsync(q.p, queries_host, sizeof(float) * nq * g->d, cudaMemcpyHostToDevice, st));
    ssg_status s = ssg_search(g, nullptr, q.p, nq, k, L_search, ids.p, dd.p, stream);
    if (s != SSG_OK) throw Fail{s};
    SSG_CUDA(cudaMemcpyAsync(out_ids_host, ids.p, sizeof(int32_t) * nq * k, cudaMemcpyDeviceToHost, st));
    if (out_d2_host)
      SSG_CUDA(cudaMemcpyAsync(out_d2_host, dd.p, sizeof(float) * nq * k, cudaMemcpyDeviceToHost, st));
    SSG_CUDA(cudaStreamSynchronize(st));
  });
}

static const char kMagic[8] = {'N', 'S', 'S', 'G', 'r', 'a', 'p', 'h'};

ssg_status ssg_save(const ssg_graph* g, const char* path) {
  return guard([&] {
    SSG_REQUIRE(g && path, SSG_EINVAL, "null argument");
    std::vector<int32_t> adj((size_t)g->n * g->R), deg((size_t)g->n);
    SSG_CUDA(cudaDeviceSynchronize());
    SSG_CUDA(cudaMemcpy(adj.data(), g->adj, sizeof(int32_t) * adj.size(), cudaMemcpyDeviceToHost));
    SSG_CUDA(cudaMemcpy(deg.data(), g->deg, sizeof(int32_t) * deg.size(), cudaMemcpyDeviceToHost));
    FILE* f = fopen(path, "wb");
    SSG_REQUIRE(f, SSG_EIO, "cannot open %s for writing", path);
    const uint32_t version = 1;
    bool ok = fwrite(kMagic, 1, 8, f) == 8 && fwrite(&version, 4, 1, f) == 1 &&
              fwrite(&g->n, 8, 1, f) == 1 && fwrite(&g->d, 4, 1, f) == 1 &&
              fwrite(&g->R, 4, 1, f) == 1 && fwrite(&g->n_nav, 4, 1, f) == 1 &&
              fwrite(&g->alpha, 8, 1, f) == 1 &&
              fwrite(g->nav_host.data(), 4, g->nav_host.size(), f) == g->nav_host.size() &&
              fwrite(deg.data(), 4, deg.size(), f) == deg.size() &&
              fwrite(adj.data(), 4, adj.size(), f) == adj.size();
    ok = (fclose(f) == 0) && ok;
    SSG_REQUIRE(ok, SSG_EIO, "short write to %s", path);
  });
}

ssg_status ssg_load(const char* path, ssg_graph** out) {
  return guard([&] {
    SSG_REQUIRE(path && out, SSG_EINVAL, "null argument");
    *out = nullptr;
    FILE* f = fopen(path, "rb");
    SSG_REQUIRE(f, SSG_EIO, "cannot open %s", path);
    std::unique_ptr<FILE, int (*)(FILE*)> fc(f, fclose);
    char magic[8];
    uint32_t version = 0;
    std::unique_ptr<ssg_graph> g(new ssg_graph());
    bool ok = fread(magic, 1, 8, f) == 8 && memcmp(magic, kMagic, 8) == 0 &&
              fread(&version, 4, 1, f) == 1 && version == 1 && fread(&g->n, 8, 1, f) == 1 &&
              fread(&g->d, 4, 1, f) == 1 && fread(&g->R, 4, 1, f) == 1 &&
              fread(&g->n_nav, 4, 1, f) == 1 && fread(&g->alpha, 8, 1, f) == 1;
    SSG_REQUIRE(ok && g->n >= 1 && g->R >= 1 && g->n_nav >= 1 && g->n_nav <= g->n, SSG_EIO,
                "%s is not a graph file of this library", path);
    g->nav_host.resize(g->n_nav);
    std::vector<int32_t> adj((size_t)g->n * g->R), deg((size_t)g->n);
    ok = fread(g->nav_host.data(), 4, g->n_nav, f) == (size_t)g->n_nav &&
         fread(deg.data(), 4, deg.size(), f) == deg.size() &&
         fread(adj.data(), 4, adj.size(), f) == adj.size();
    SSG_REQUIRE(ok, SSG_EIO, "%s is truncated", path);
    SSG_CUDA(cudaMalloc(&g->adj, sizeof(int32_t) * adj.size()));
    SSG_CUDA(cudaMalloc(&g->deg, sizeof(int32_t) * deg.size()));
    SSG_CUDA(cudaMalloc(&g->nav_dev, sizeof(int32_t) * g->n_nav));
    SSG_CUDA(cudaMemcpy(g->adj, adj.data(), sizeof(int32_t) * adj.size(), cudaMemcpyHostToDevice));
    SSG_CUDA(cudaMemcpy(g->deg, deg.data(), sizeof(int32_t) * deg.size(), cudaMemcpyHostToDevice));
    SSG_CUDA(cudaMemcpy(g->nav_dev, g->nav_host.data(), sizeof(int32_t) * g->n_nav,
                        cudaMemcpyHostToDevice));
    *out = g.release();
  });
}

void ssg_free(ssg_graph* g) { delete g; }

}  // extern "C"
