/* Runs every oracle entry point on small seeded inputs (float data, and integer data full
 * of ties and duplicates) so that tests/test_oracle_sanitized.py can execute the oracle
 * under AddressSanitizer and UndefinedBehaviorSanitizer.  Exit status 0: every call
 * returned its success code; the sanitizers report anything else on stderr. */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

int or_knn_rows(const float* base, int64_t n, int d, const int64_t* rows, int64_t nrows, int k,
                int32_t* ids, double* d2);
int or_knn_queries(const float* base, int64_t n, int d, const float* q, int64_t nq, int k,
                   int32_t* ids, double* d2);
int or_pool2(const float* base, int64_t n, int d, const int32_t* knn, int K, int L,
             const int64_t* rows, int64_t nrows, int own_first, int32_t* pool_ids,
             double* pool_d2, int32_t* pool_len);
int or_prune(const float* base, int64_t n, int d, const int64_t* nodes, int64_t nrows,
             const int32_t* cand, const int32_t* cand_len, int stride, int R, double cos_alpha,
             int32_t* adj, int32_t* deg);
int or_reverse(const float* base, int64_t n, int d, const int32_t* adj0, const int32_t* deg0,
               int R, double cos_alpha, int32_t* adj1, int32_t* deg1);
int or_connect(const float* base, int64_t n, int d, int32_t* adj, int32_t* deg, int R,
               const int32_t* nav, int n_nav, int64_t* n_repair);
int or_search(const float* base, int64_t n, int d, const int32_t* adj, const int32_t* deg, int R,
              const int32_t* nav, int n_nav, const float* queries, int64_t nq, int k, int Ls,
              int32_t* out_ids, double* out_d2, int64_t* n_dist, int64_t* n_hops);
void or_dist2_pairs(const float* base, int d, const int64_t* a, const int64_t* b, int64_t m,
                    double* out);
void or_cos_triples(const float* base, int d, const int64_t* i, const int64_t* j,
                    const int64_t* k, int64_t m, double* out);

static uint64_t rng_state = 88172645463325252ull;
static double rnd(void) {
  rng_state ^= rng_state << 13;
  rng_state ^= rng_state >> 7;
  rng_state ^= rng_state << 17;
  return (double)(rng_state >> 11) / 9007199254740992.0;
}

#define CHECK(x)                                                \
  do {                                                          \
    if ((x) != 0) {                                             \
      fprintf(stderr, "call failed: %s (line %d)\n", #x, __LINE__); \
      return 1;                                                 \
    }                                                           \
  } while (0)

static int run(int64_t n, int d, int integer, int own_first) {
  const int K = 12, L = 30, R = 10, nq = 25, k = 5, Ls = 24, n_nav = 3;
  const double cos_a = 0.5;
  float* x = malloc(sizeof(float) * (size_t)n * d);
  float* q = malloc(sizeof(float) * (size_t)nq * d);
  for (int64_t t = 0; t < n * d; ++t)
    x[t] = integer ? (float)(int)(rnd() * 4.0) : (float)(rnd() * 2.0 - 1.0);
  for (int64_t t = 0; t < (int64_t)nq * d; ++t) q[t] = (float)(rnd() * 2.0 - 1.0);
  int64_t* rows = malloc(sizeof(int64_t) * (size_t)n);
  for (int64_t i = 0; i < n; ++i) rows[i] = i;
  int32_t* knn = malloc(sizeof(int32_t) * (size_t)n * K);
  double* kd = malloc(sizeof(double) * (size_t)n * K);
  CHECK(or_knn_rows(x, n, d, rows, n, K, knn, kd));
  int32_t* pid = malloc(sizeof(int32_t) * (size_t)n * L);
  double* pd = malloc(sizeof(double) * (size_t)n * L);
  int32_t* plen = malloc(sizeof(int32_t) * (size_t)n);
  CHECK(or_pool2(x, n, d, knn, K, L, rows, n, own_first, pid, pd, plen));
  int32_t* adj0 = malloc(sizeof(int32_t) * (size_t)n * R);
  int32_t* deg0 = malloc(sizeof(int32_t) * (size_t)n);
  CHECK(or_prune(x, n, d, rows, n, pid, plen, L, R, cos_a, adj0, deg0));
  int32_t* adj1 = malloc(sizeof(int32_t) * (size_t)n * R);
  int32_t* deg1 = malloc(sizeof(int32_t) * (size_t)n);
  CHECK(or_reverse(x, n, d, adj0, deg0, R, cos_a, adj1, deg1));
  int32_t nav[3] = {0, (int32_t)(n / 2), (int32_t)(n - 1)};
  int64_t rep = 0;
  CHECK(or_connect(x, n, d, adj1, deg1, R, nav, n_nav, &rep));
  int32_t* ids = malloc(sizeof(int32_t) * (size_t)nq * k);
  double* dd = malloc(sizeof(double) * (size_t)nq * k);
  int64_t* nd = malloc(sizeof(int64_t) * (size_t)nq);
  int64_t* nh = malloc(sizeof(int64_t) * (size_t)nq);
  CHECK(or_search(x, n, d, adj1, deg1, R, nav, n_nav, q, nq, k, Ls, ids, dd, nd, nh));
  int32_t* gt = malloc(sizeof(int32_t) * (size_t)nq * k);
  double* gd = malloc(sizeof(double) * (size_t)nq * k);
  CHECK(or_knn_queries(x, n, d, q, nq, k, gt, gd));
  int64_t a[4] = {0, 1, 2, n - 1}, b[4] = {n - 1, 0, 1, 2}, c[4] = {1, 2, 0, 0};
  double out[4];
  or_dist2_pairs(x, d, a, b, 4, out);
  or_cos_triples(x, d, a, b, c, 4, out);
  free(x); free(q); free(rows); free(knn); free(kd); free(pid); free(pd); free(plen);
  free(adj0); free(deg0); free(adj1); free(deg1); free(ids); free(dd); free(nd); free(nh);
  free(gt); free(gd);
  return 0;
}

int main(void) {
  if (run(257, 7, 0, 0)) return 1;
  if (run(257, 7, 0, 1)) return 1;
  if (run(180, 5, 1, 0)) return 1; /* many ties and duplicate points */
  if (run(180, 5, 1, 1)) return 1;
  printf("oracle sanitized run ok\n");
  return 0;
}
