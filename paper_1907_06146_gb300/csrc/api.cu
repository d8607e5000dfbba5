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
                                    Counters* ctr, cudaStream_t st) {
  if (tc_ok && prune_tc_available(d, L, R)) {
    prune_run_tc(X, ld, d, n, pool_id, pool_len, L, R, cos_a, border, adj, deg, ctr, st);
    return SSG_PREC_BF16;
  }
  prune_run(X, ld, d, n, pool_id, pool_len, L, R, cos_a, border, adj, deg, ctr, st);
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

ssg_status ssg_build(const float* base, int64_t n, int32_t d, int32_t K, int32_t L, int32_t R,
                     double alpha_deg, const ssg_build_opts* opts_in, ssg_stream stream,
                     ssg_graph** out, ssg_build_stats* stats) {
  return guard([&] {
    SSG_REQUIRE(base && out, SSG_EINVAL, "null pointer");
    *out = nullptr;
    ssg_build_opts opts;
    ssg_default_opts(&opts);
    if (opts_in) opts = *opts_in;
    SSG_REQUIRE(n >= 2 && n < (1ll << 31) && d >= 1, SSG_EINVAL, "need 2 <= n < 2^31 and d >= 1");
    SSG_REQUIRE(K >= 1 && K <= n - 1 && K <= 700, SSG_EINVAL, "need 1 <= K <= min(n - 1, 700)");
    SSG_REQUIRE(L >= 1 && L + K <= 1023, SSG_EINVAL, "need L >= 1 and L + K <= 1023");
    check_alpha(alpha_deg);
    check_prune_fit(d, R);
    check_prec(opts.gemm_prec, "gemm_prec");
    check_prec(opts.gram_prec, "gram_prec");
    SSG_REQUIRE(opts.cos_margin_fp64 >= 0.0 && opts.cos_margin_fp64 <= 0.5, SSG_EINVAL,
                "cos_margin_fp64 must lie in [0, 0.5], got %g", opts.cos_margin_fp64);
    const KnnTune tune = read_tune_table(opts.tune_table);
    SSG_REQUIRE(opts.n_nav >= 1 && opts.n_nav <= n && opts.n_nav <= 4096, SSG_EINVAL,
                "need 1 <= n_nav <= min(n, 4096)");
    std::vector<int32_t> nav((size_t)opts.n_nav);
    if (opts.nav_ids_host) {
      for (int t = 0; t < opts.n_nav; ++t) {
        nav[t] = opts.nav_ids_host[t];
        SSG_REQUIRE(nav[t] >= 0 && nav[t] < n, SSG_EINVAL, "navigating node %d out of range", nav[t]);
        for (int u = 0; u < t; ++u)
          SSG_REQUIRE(nav[u] != nav[t], SSG_EINVAL, "navigating nodes must be distinct");
      }
    } else {
      ssg_status s = ssg_nav_ids(n, opts.n_nav, opts.seed, nav.data());
      if (s != SSG_OK) throw Fail{s};
    }
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t launches0 = t_launches;
    ssg_build_stats S{};
    StageTimer t_all(st, "ssg_build"), t_ing(st, "ingest"), t_knn(st, "knn graph"),
        t_gemm(st, "knn kernel"), t_pool(st, "pools"), t_prune(st, "prune"),
        t_rev(st, "reverse merge"), t_con(st, "connectivity");
    t_all.start();

    ssg_graph* g = new ssg_graph();
    std::unique_ptr<ssg_graph> gp(g);
    g->n = n;
    g->d = d;
    g->R = R;
    g->n_nav = opts.n_nav;
    g->alpha = alpha_deg;
    g->nav_host = nav;
    SSG_CUDA(cudaMalloc(&g->adj, sizeof(int32_t) * n * R));
    SSG_CUDA(cudaMalloc(&g->deg, sizeof(int32_t) * n));
    SSG_CUDA(cudaMalloc(&g->nav_dev, sizeof(int32_t) * opts.n_nav));
    SSG_CUDA(cudaMemcpyAsync(g->nav_dev, nav.data(), sizeof(int32_t) * opts.n_nav,
                             cudaMemcpyHostToDevice, st));

    t_ing.start();
    Ingested in;
    ingest_all(base, n, d, st, in, true);
    // integers 0..255: a byte copy of the rows (a quarter of the bytes, the same distances)
    // for the pool, reverse-merge and search distances
    if (in.info.exact && in.info.nonneg && in.info.max_abs <= 255.f) {
      SSG_CUDA(cudaMalloc(&g->rows_u8, (size_t)n * in.rows.ld));
      g->rows_ld = in.rows.ld;
      g->rows_src = base;
      rows_to_u8(in.rows.p, in.rows.ld, d, n, g->rows_u8, st);
    }
    t_ing.stop();
    Scratch<Counters> ctr(1, st);
    SSG_CUDA(cudaMemsetAsync(ctr.p, 0, sizeof(Counters), st));
    const double cos_a = cos_alpha_of(alpha_deg);

    const uint8_t* X8 = g->rows_u8;
    const int kpath = knn_path(opts.gemm_prec, in.info, d);
    const bool tc = kpath == 1;
    const double border = opts.cos_margin_fp64;
    const bool gram_tc = opts.gram_prec != SSG_PREC_FP32 && in.info.bf16_exact;
    SSG_REQUIRE(opts.gemm_prec != SSG_PREC_BF16 || kpath != 0, SSG_EINVAL,
                "bf16 distance GEMM needs sm_103 and d <= 4096");
    CertResult cert;
    Scratch<int32_t> pool_id((size_t)n * L, st), pool_len((size_t)n, st);
    Scratch<float> pool_d2((size_t)n * L, st);
    KnnResult kr;
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
      t_knn.start();
      if (tc) {
        // data exact in bf16: the selection itself is exact
        knn_exact_tc(in.rows.p, n, in.rows.ld, in.norms.p, in.rows.p, n, in.rows.ld, in.norms.p,
                     d, 1, L, pool_id.p, pool_d2.p, st, &t_gemm, opts.pool_tiles);
        t_knn.stop();
        in.norms.release();
        t_pool.start();
        SSG_LAUNCH(k_pool_len_from_ids, (unsigned)ceil_div(n, 256), 256, 0, st, pool_id.p, n, L,
                   pool_len.p);
        t_pool.stop();
      } else {
        // other data: a bf16 selection of L + slack candidates (approximate distances), then
        // each pool ordered from the original vectors as Alg. 3's pools are and cut to L
        const int Lp = (int)std::min<int64_t>(
            std::min(L + std::max(8, L / 4), knn_tc_max_k(d, true)), n - 1);
        Scratch<int32_t> cid((size_t)n * Lp, st);
        Scratch<float> cd2((size_t)n * Lp, st);
        knn_exact_tc(in.rows.p, n, in.rows.ld, in.norms.p, in.rows.p, n, in.rows.ld, in.norms.p,
                     d, 1, Lp, cid.p, cd2.p, st, &t_gemm, opts.pool_tiles, true);
        t_knn.stop();
        in.norms.release();
        t_pool.start();
        pool_from_candidates(in.rows.p, X8, in.rows.ld, d, n, cid.p, Lp, L, in.info.exact, pool_id.p,
                             pool_d2.p, pool_len.p, ctr.p, st);
        t_pool.stop();
      }
    } else {
      // a1: exact kNN graph
      Scratch<int32_t> knn_id((size_t)n * K, st);
      Scratch<float> knn_d2((size_t)n * K, st);
      t_knn.start();
      kr = knn_any(in, n, in, n, d, in.info, 1, K, opts.gemm_prec, knn_id.p, knn_d2.p, false, tune,
                   ctr.p, st, &t_gemm, &cert);
      t_knn.stop();
      in.norms.release();

      // a2: candidate pools
      t_pool.start();
      pool_run(in.rows.p, X8, in.rows.ld, d, n, knn_id.p, K, L, in.info.exact, pool_id.p, pool_d2.p,
               pool_len.p, ctr.p, st, opts.pool_own_row_first);
      t_pool.stop();
    }

    auto debug_check = [&](const CheckResult& r, const char* stage) {
      SSG_REQUIRE(r.row < 0, SSG_EINTERNAL, "debug check after %s: row %lld: %s", stage,
                  (long long)r.row, check_name(r.code));
    };
    if (opts.debug_checks)
      debug_check(check_pool(pool_id.p, pool_d2.p, pool_len.p, n, L, in.info.exact, d, st),
                  "the pools");

    // a3: SSG prune
    Scratch<int32_t> adj0((size_t)n * R, st), deg0((size_t)n, st);
    t_prune.start();
    const ssg_precision gram_used =
        prune_dispatch(gram_tc, in.rows.p, in.rows.ld, d, n, pool_id.p, pool_len.p, L, R, cos_a,
                       border, adj0.p, deg0.p, ctr.p, st);
    t_prune.stop();
    if (opts.debug_checks) debug_check(check_adj(adj0.p, deg0.p, n, R, st), "the prune");
    pool_id.release();
    pool_d2.release();
    pool_len.release();

    // a4: reverse-neighbour merge
    t_rev.start();
    const int maxin = reverse_run(in.rows.p, X8, in.rows.ld, d, n, adj0.p, deg0.p, R, cos_a, border,
                                  in.info.exact, gram_tc, g->adj, g->deg, ctr.p, st);
    t_rev.stop();
    if (opts.debug_checks) debug_check(check_adj(g->adj, g->deg, n, R, st), "the reverse merge");
    adj0.release();
    deg0.release();

    // a5: connectivity from the navigating nodes
    t_con.start();
    const int64_t rep = connect_run(in.rows.p, in.rows.ld, d, n, g->adj, g->deg, R, g->nav_dev,
                                    nav.data(), opts.n_nav, st);
    t_con.stop();
    if (opts.debug_checks) debug_check(check_adj(g->adj, g->deg, n, R, st), "connectivity");
    t_all.stop();

    Counters hc;
    SSG_CUDA(cudaMemcpyAsync(&hc, ctr.p, sizeof(hc), cudaMemcpyDeviceToHost, st));
    SSG_CUDA(cudaStreamSynchronize(st));
    S.ms_ingest = t_ing.ms();
    S.ms_knn = t_knn.ms();
    S.ms_knn_gemm = t_gemm.ms();
    S.ms_pool = t_pool.ms();
    S.ms_prune = t_prune.ms();
    S.ms_reverse = t_rev.ms();
    S.ms_connect = t_con.ms();
    S.ms_total = t_all.ms();
    S.n_repair = rep;
    S.n_angle_fp64 = (int64_t)hc.angle_fp64;
    S.n_order_fp64 = (int64_t)hc.order_fp64;
    S.n_knn_fallback_rows = kr.fallback_rows;
    S.max_indegree = maxin;
    S.exact_mode = in.info.exact;
    S.gemm_prec_used = kpath == 0 ? SSG_PREC_FP32 : SSG_PREC_BF16;
    S.gram_prec_used = gram_used;
    S.n_angle_borderline = (int64_t)hc.angle_border;
    S.knn_candidates = cert.candidates;
    S.ms_knn_certify = kpath == 2 && opts.pool_tiles == 0 ? S.ms_knn - S.ms_knn_gemm : 0.0;
    S.kernel_launches = t_launches - launches0;
    S.search_row_bytes = g->rows_u8 ? 1 : 4;
    if (stats) *stats = S;
    *out = gp.release();
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
    // largest work first (n^2 d: the kNN graph dominates), so the tail is short
    std::vector<int32_t> order((size_t)count);
    for (int32_t i = 0; i < count; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
      return (double)n[a] * n[a] * d[a] > (double)n[b] * n[b] * d[b];
    });
    int dev = 0;
    SSG_CUDA(cudaGetDevice(&dev));
    const int nt = std::min<int32_t>(n_streams, count);
    std::vector<cudaStream_t> streams((size_t)nt, nullptr);
    for (int t = 0; t < nt; ++t)
      SSG_CUDA(cudaStreamCreateWithFlags(&streams[t], cudaStreamNonBlocking));
    std::atomic<int32_t> next{0};
    std::mutex mu;
    ssg_status first = SSG_OK;
    std::string first_msg;
    auto worker = [&](int t) {
      cudaSetDevice(dev);
      for (;;) {
        const int32_t k = next.fetch_add(1);
        if (k >= count) break;
        const int32_t i = order[k];
        const ssg_status s = ssg_build(bases[i], n[i], d[i], K[i], L[i], R[i], alpha_deg[i], opts,
                                       (ssg_stream)streams[t], &graphs[i],
                                       stats ? &stats[i] : nullptr);
        if (s != SSG_OK) {
          std::lock_guard<std::mutex> lk(mu);
          if (first == SSG_OK) {
            first = s;
            first_msg = "index " + std::to_string(i) + ": " + ssg_last_error();
          }
        }
      }
      cudaStreamSynchronize(streams[t]);
    };
    std::vector<std::thread> pool;
    for (int t = 0; t < nt; ++t) pool.emplace_back(worker, t);
    for (auto& th : pool) th.join();
    for (int t = 0; t < nt; ++t) cudaStreamDestroy(streams[t]);
    SSG_REQUIRE(first == SSG_OK, first, "%s", first_msg.c_str());
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
