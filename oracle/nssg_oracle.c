/*
 * CPU oracle for the NSSG hot path -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow, obviously correct C: every distance and every angle is computed in
 * double precision from the float32 inputs (float -> double is exact), sums run
 * sequentially over the coordinates, and the build compiles with
 * -ffp-contract=off so that no multiply-add is fused.  Parallelism is only over
 * independent rows / nodes / queries (OpenMP), which changes no arithmetic.
 *
 * Only the tests, the smoke check and the benchmark's CPU-baseline leg may load
 * this library.  It shares no source with the CUDA library.
 *
 * Paper: "High Dimensional Similarity Search with Satellite System Graph"
 * (Fu, Wang, Cai, arXiv 1907.06146).  Each function names the passage it follows.
 * Readings where the paper is silent or garbled (numbered R1..R13) are stated
 * where they apply.
 *
 * Orders: every sort in this file is by (squared distance, id) ascending.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
  double d2;
  int32_t id;
} or_pair;

static int cmp_pair(const void* a, const void* b) {
  const or_pair* x = (const or_pair*)a;
  const or_pair* y = (const or_pair*)b;
  if (x->d2 < y->d2) return -1;
  if (x->d2 > y->d2) return 1;
  return (x->id > y->id) - (x->id < y->id);
}

/* Squared Euclidean distance (Sec. 2.1: delta is Euclidean; ordering by the square is
 * equivalent and avoids the root).  Sequential double-precision sum. */
static double dist2(const float* a, const float* b, int d) {
  double s = 0.0;
  for (int t = 0; t < d; ++t) {
    double diff = (double)a[t] - (double)b[t];
    s = s + diff * diff;
  }
  return s;
}

/* Dot product of the centred vectors (a - o) and (b - o). */
static double centred_dot(const float* a, const float* b, const float* o, int d) {
  double s = 0.0;
  for (int t = 0; t < d; ++t) {
    double u = (double)a[t] - (double)o[t];
    double v = (double)b[t] - (double)o[t];
    s = s + u * v;
  }
  return s;
}

int or_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void or_set_threads(int t) {
#ifdef _OPENMP
  if (t > 0) omp_set_num_threads(t);
#else
  (void)t;
#endif
}

/*
 * Exact k nearest neighbours of selected base rows (Alg. 3 line 1 builds a kNN graph;
 * the exact graph is its brute-force definition).  For row i = rows[r]: every j != i
 * gets d2(i, j); all are sorted by (d2, id); the first k are written.  Duplicate
 * vectors are distinct ids at distance 0 and are kept.
 * ids/d2: [nrows][k].  Returns 0, or -1 if k > n - 1.
 */
int or_knn_rows(const float* base, int64_t n, int d, const int64_t* rows, int64_t nrows,
                int k, int32_t* ids, double* d2) {
  if (k > n - 1) return -1;
  int64_t r;
#pragma omp parallel for schedule(dynamic, 1)
  for (r = 0; r < nrows; ++r) {
    int64_t i = rows[r];
    or_pair* all = (or_pair*)malloc(sizeof(or_pair) * (size_t)n);
    int64_t m = 0;
    for (int64_t j = 0; j < n; ++j) {
      if (j == i) continue;
      all[m].d2 = dist2(base + i * d, base + j * d, d);
      all[m].id = (int32_t)j;
      ++m;
    }
    qsort(all, (size_t)m, sizeof(or_pair), cmp_pair);
    for (int t = 0; t < k; ++t) {
      ids[r * k + t] = all[t].id;
      d2[r * k + t] = all[t].d2;
    }
    free(all);
  }
  return 0;
}

/*
 * Ground truth for unindexed queries (serial scan, Sec. 5.3 item 8; precision in
 * Sec. 5.2): the k base points nearest each query, by (d2, id).
 */
int or_knn_queries(const float* base, int64_t n, int d, const float* q, int64_t nq, int k,
                   int32_t* ids, double* d2) {
  if (k > n) return -1;
  int64_t r;
#pragma omp parallel for schedule(dynamic, 1)
  for (r = 0; r < nq; ++r) {
    or_pair* all = (or_pair*)malloc(sizeof(or_pair) * (size_t)n);
    for (int64_t j = 0; j < n; ++j) {
      all[j].d2 = dist2(q + r * d, base + j * d, d);
      all[j].id = (int32_t)j;
    }
    qsort(all, (size_t)n, sizeof(or_pair), cmp_pair);
    for (int t = 0; t < k; ++t) {
      ids[r * k + t] = all[t].id;
      d2[r * k + t] = all[t].d2;
    }
    free(all);
  }
  return 0;
}

static int in_list(const int32_t* a, int m, int32_t x) {
  for (int t = 0; t < m; ++t)
    if (a[t] == x) return 1;
  return 0;
}

/*
 * Candidate pool (Alg. 3, the loop over neighbours n of node i and their neighbours n').
 * For n in knn(i) in kNN order: add n, then every n' in knn(n) in kNN order; repeats
 * are dropped (the set P); after the whole of knn(n) has been added, stop if |P| >= L.
 * R1: node i itself is never a candidate.  R2: the collected set is sorted by
 * (d2(i, .), id) and the L closest are kept.
 * knn: [n][K] for all nodes.  Outputs for each selected node r: pool_ids/pool_d2
 * [nrows][L] (padded with -1 / INFINITY), pool_len[nrows].
 */
/*
 * own_first = 1: the "own row first" reading of the same loop (the alternative to R2):
 * the node's whole kNN row enters the pool first, then the rows of its neighbours, whole
 * and in kNN order, until the pool holds >= L ids; sorted and cut to L as above.  With
 * K >= L the pool is the node's L nearest neighbours.
 */
int or_pool2(const float* base, int64_t n, int d, const int32_t* knn, int K, int L,
             const int64_t* rows, int64_t nrows, int own_first, int32_t* pool_ids,
             double* pool_d2, int32_t* pool_len) {
  (void)n;
  int64_t r;
#pragma omp parallel for schedule(dynamic, 16)
  for (r = 0; r < nrows; ++r) {
    int64_t i = rows[r];
    int cap = L + 2 * K + 1;
    int32_t* P = (int32_t*)malloc(sizeof(int32_t) * (size_t)cap);
    int m = 0;
    if (own_first) {
      for (int t = 0; t < K; ++t) {
        int32_t nb = knn[i * K + t];
        if (nb != i && !in_list(P, m, nb)) P[m++] = nb;
      }
      for (int t = 0; t < K && m < L; ++t) {
        int32_t nb = knn[i * K + t];
        for (int t2 = 0; t2 < K; ++t2) {
          int32_t nb2 = knn[(int64_t)nb * K + t2];
          if (nb2 != i && !in_list(P, m, nb2)) P[m++] = nb2;
        }
      }
    } else {
      for (int t = 0; t < K; ++t) {
        int32_t nb = knn[i * K + t];
        if (nb != i && !in_list(P, m, nb)) P[m++] = nb;
        for (int t2 = 0; t2 < K; ++t2) {
          int32_t nb2 = knn[(int64_t)nb * K + t2];
          if (nb2 != i && !in_list(P, m, nb2)) P[m++] = nb2;
        }
        if (m >= L) break;
      }
    }
    or_pair* pr = (or_pair*)malloc(sizeof(or_pair) * (size_t)(m > 0 ? m : 1));
    for (int t = 0; t < m; ++t) {
      pr[t].d2 = dist2(base + i * d, base + (int64_t)P[t] * d, d);
      pr[t].id = P[t];
    }
    qsort(pr, (size_t)m, sizeof(or_pair), cmp_pair);
    int keep = m < L ? m : L;
    for (int t = 0; t < L; ++t) {
      pool_ids[r * L + t] = t < keep ? pr[t].id : -1;
      pool_d2[r * L + t] = t < keep ? pr[t].d2 : INFINITY;
    }
    pool_len[r] = keep;
    free(pr);
    free(P);
  }
  return 0;
}

int or_pool(const float* base, int64_t n, int d, const int32_t* knn, int K, int L,
            const int64_t* rows, int64_t nrows, int32_t* pool_ids, double* pool_d2,
            int32_t* pool_len) {
  return or_pool2(base, n, d, knn, K, L, rows, nrows, 0, pool_ids, pool_d2, pool_len);
}

/*
 * The SSG angle test between two candidate edges i->j and i->k (Alg. 2, the inner
 * test on cos of angle d_j d_i d_k against cos a).  cos is taken from the centred
 * dot products g_jk = (c_j - x_i).(c_k - x_i): cos = g_jk / sqrt(g_jj * g_kk).
 * R5: a zero-length edge (a duplicate of node i) has no direction; its cosine is 0.
 * Returns 1 when the two edges conflict (cos > cos_alpha, strict: R10).
 */
static int conflicts(const float* base, int d, int64_t i, int32_t j, int32_t k,
                     double cos_alpha) {
  const float* xi = base + i * d;
  const float* cj = base + (int64_t)j * d;
  const float* ck = base + (int64_t)k * d;
  double gjj = centred_dot(cj, cj, xi, d);
  double gkk = centred_dot(ck, ck, xi, d);
  double gjk = centred_dot(cj, ck, xi, d);
  double c = 0.0;
  if (gjj != 0.0 && gkk != 0.0) c = gjk / sqrt(gjj * gkk);
  return c > cos_alpha;
}

/* One node's prune: cand[0..len) is already in (d2, id) order.  Keep cand[0]; walk on,
 * keeping a candidate when it conflicts with no kept edge; stop once R are kept (R3). */
static int prune_one(const float* base, int d, int64_t i, const int32_t* cand, int len,
                     int R, double cos_alpha, int32_t* out) {
  int kept = 0;
  for (int t = 0; t < len && kept < R; ++t) {
    int32_t j = cand[t];
    int ok = 1;
    for (int u = 0; u < kept && ok; ++u)
      if (conflicts(base, d, i, j, out[u], cos_alpha)) ok = 0;
    if (ok) out[kept++] = j;
  }
  return kept;
}

/*
 * SSG prune of given candidate lists (Alg. 2 selection; Alg. 3 applies it to each
 * pool).  nodes[r] is the node whose candidates are cand[r*stride .. + cand_len[r]),
 * already sorted by (d2, id).  adj: [nrows][R] padded with -1; deg: [nrows].
 * With R >= n - 1 and full candidate lists this is SSG-Build (Alg. 2) itself.
 */
int or_prune(const float* base, int64_t n, int d, const int64_t* nodes, int64_t nrows,
             const int32_t* cand, const int32_t* cand_len, int stride, int R,
             double cos_alpha, int32_t* adj, int32_t* deg) {
  (void)n;
  int64_t r;
#pragma omp parallel for schedule(dynamic, 16)
  for (r = 0; r < nrows; ++r) {
    int32_t* out = adj + r * R;
    int k = prune_one(base, d, nodes[r], cand + r * stride, cand_len[r], R, cos_alpha, out);
    for (int t = k; t < R; ++t) out[t] = -1;
    deg[r] = k;
  }
  return 0;
}

/*
 * Reverse-neighbour checking (Alg. 3, the loop that tries to add i to the neighbours
 * of each j in G[i]; Sec. 4.1 motivates it).  R4, the order-free reading: from the
 * graph adj0 as a whole, every node j gets the candidate set adj0[j] united with
 * {i : j in adj0[i]}, sorted by (d2(j, .), id), and the same prune with the same cap R
 * is run on it.  adj0/adj1: [n][R] padded with -1.
 */
int or_reverse(const float* base, int64_t n, int d, const int32_t* adj0, const int32_t* deg0,
               int R, double cos_alpha, int32_t* adj1, int32_t* deg1) {
  int32_t* indeg = (int32_t*)calloc((size_t)n, sizeof(int32_t));
  int64_t* off = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
  for (int64_t i = 0; i < n; ++i)
    for (int t = 0; t < deg0[i]; ++t) indeg[adj0[i * R + t]]++;
  off[0] = 0;
  for (int64_t j = 0; j < n; ++j) off[j + 1] = off[j] + indeg[j];
  int32_t* rev = (int32_t*)malloc(sizeof(int32_t) * (size_t)(off[n] > 0 ? off[n] : 1));
  int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
  for (int64_t j = 0; j < n; ++j) fill[j] = off[j];
  for (int64_t i = 0; i < n; ++i)
    for (int t = 0; t < deg0[i]; ++t) rev[fill[adj0[i * R + t]]++] = (int32_t)i;
  int64_t j;
#pragma omp parallel for schedule(dynamic, 16)
  for (j = 0; j < n; ++j) {
    int cap = deg0[j] + indeg[j];
    int32_t* c = (int32_t*)malloc(sizeof(int32_t) * (size_t)(cap > 0 ? cap : 1));
    int m = 0;
    for (int t = 0; t < deg0[j]; ++t) c[m++] = adj0[j * R + t];
    for (int64_t t = off[j]; t < off[j + 1]; ++t)
      if (!in_list(c, m, rev[t])) c[m++] = rev[t];
    or_pair* pr = (or_pair*)malloc(sizeof(or_pair) * (size_t)(m > 0 ? m : 1));
    for (int t = 0; t < m; ++t) {
      pr[t].d2 = dist2(base + j * d, base + (int64_t)c[t] * d, d);
      pr[t].id = c[t];
    }
    qsort(pr, (size_t)m, sizeof(or_pair), cmp_pair);
    for (int t = 0; t < m; ++t) c[t] = pr[t].id;
    int32_t* out = adj1 + j * R;
    int k = prune_one(base, d, j, c, m, R, cos_alpha, out);
    for (int t = k; t < R; ++t) out[t] = -1;
    deg1[j] = k;
    free(pr);
    free(c);
  }
  free(fill);
  free(rev);
  free(off);
  free(indeg);
  return 0;
}

/* Mark everything reachable from src that is not yet marked (iterative traversal). */
static void reach_from(const int32_t* adj, const int32_t* deg, int R, int64_t n, int64_t src,
                       unsigned char* reached, int32_t* stack) {
  (void)n;
  if (reached[src]) return;
  int64_t top = 0;
  reached[src] = 1;
  stack[top++] = (int32_t)src;
  while (top > 0) {
    int32_t v = stack[--top];
    for (int t = 0; t < deg[v]; ++t) {
      int32_t w = adj[(int64_t)v * R + t];
      if (!reached[w]) {
        reached[w] = 1;
        stack[top++] = w;
      }
    }
  }
}

/*
 * Connectivity from the navigating nodes (Alg. 3, the DFS-spanning loop over NV; Sec. 4.1
 * defers its details to the NSG paper).  R7: for each root in the given order, mark
 * the set reachable from it; while some node is unreached, take the smallest unreached
 * id u, link to it from the reached node v with deg(v) < R that minimises
 * (d2(v, u), id), and mark everything reachable from u.  The reached set does not depend
 * on the traversal order, so any traversal gives the same graph.
 * adj/deg are updated in place.  *n_repair counts the added edges.
 * Returns 0, or -2 if an unreached node exists but no reached node has a free slot.
 */
int or_connect(const float* base, int64_t n, int d, int32_t* adj, int32_t* deg, int R,
               const int32_t* nav, int n_nav, int64_t* n_repair) {
  unsigned char* reached = (unsigned char*)malloc((size_t)n);
  int32_t* stack = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  int64_t repairs = 0;
  int rc = 0;
  for (int s = 0; s < n_nav && rc == 0; ++s) {
    memset(reached, 0, (size_t)n);
    reach_from(adj, deg, R, n, nav[s], reached, stack);
    int64_t u = 0;
    for (;;) {
      while (u < n && reached[u]) ++u;
      if (u >= n) break;
      int64_t best = -1;
      double bd = 0.0;
      for (int64_t v = 0; v < n; ++v) {
        if (!reached[v] || deg[v] >= R) continue;
        double dv = dist2(base + v * d, base + u * d, d);
        if (best < 0 || dv < bd) {  /* v ascends, so a tie keeps the smaller id */
          best = v;
          bd = dv;
        }
      }
      if (best < 0) {
        rc = -2;
        break;
      }
      adj[best * R + deg[best]] = (int32_t)u;
      deg[best]++;
      repairs++;
      reach_from(adj, deg, R, n, u, reached, stack);
    }
  }
  free(stack);
  free(reached);
  *n_repair = repairs;
  return rc;
}

/*
 * Search-on-Graph (Alg. 1) with the NSSG start rule (Sec. 4.1: start from the navigating
 * node nearest to the query).  R8: the pool S holds at most Ls entries sorted by
 * (d2, id); each round expands the first unchecked entry, adds every neighbour not
 * visited before (visited marks survive truncation), re-sorts and truncates; the search
 * ends when every entry of S is checked.  The first k entries are returned, padded
 * with -1 / INFINITY when S holds fewer.
 * Counters per query: n_dist = distances evaluated (including the navigating nodes),
 * n_hops = expansions.
 */
int or_search(const float* base, int64_t n, int d, const int32_t* adj, const int32_t* deg,
              int R, const int32_t* nav, int n_nav, const float* queries, int64_t nq, int k,
              int Ls, int32_t* out_ids, double* out_d2, int64_t* n_dist, int64_t* n_hops) {
  if (k > Ls || n_nav < 1) return -1;
  int64_t qi;
#pragma omp parallel for schedule(dynamic, 4)
  for (qi = 0; qi < nq; ++qi) {
    const float* q = queries + qi * d;
    unsigned char* visited = (unsigned char*)calloc((size_t)n, 1);
    or_pair* S = (or_pair*)malloc(sizeof(or_pair) * (size_t)(Ls + R + 1));
    unsigned char* checked = (unsigned char*)malloc((size_t)(Ls + R + 1));
    or_pair* tmp = (or_pair*)malloc(sizeof(or_pair) * (size_t)(Ls + R + 1));
    unsigned char* tmpc = (unsigned char*)malloc((size_t)(Ls + R + 1));
    int64_t nd = 0, nh = 0;
    /* entry: nearest navigating node by (d2, id) */
    int32_t entry = -1;
    double ed = 0.0;
    for (int s = 0; s < n_nav; ++s) {
      double dv = dist2(q, base + (int64_t)nav[s] * d, d);
      nd++;
      if (entry < 0 || dv < ed || (dv == ed && nav[s] < entry)) {
        entry = nav[s];
        ed = dv;
      }
    }
    int m = 1;
    S[0].d2 = ed;
    S[0].id = entry;
    checked[0] = 0;
    visited[entry] = 1;
    for (;;) {
      int p = -1;
      for (int t = 0; t < m; ++t)
        if (!checked[t]) {
          p = t;
          break;
        }
      if (p < 0) break;
      checked[p] = 1;
      nh++;
      int32_t node = S[p].id;
      for (int t = 0; t < deg[node]; ++t) {
        int32_t nb = adj[(int64_t)node * R + t];
        if (visited[nb]) continue;
        visited[nb] = 1;
        S[m].d2 = dist2(q, base + (int64_t)nb * d, d);
        S[m].id = nb;
        checked[m] = 0;
        nd++;
        m++;
      }
      /* sort S (ids are distinct, so the order is total) carrying the checked flags:
         insertion sort keeps this obviously correct */
      for (int t = 0; t < m; ++t) {
        tmp[t] = S[t];
        tmpc[t] = checked[t];
      }
      for (int t = 1; t < m; ++t) {
        or_pair key = tmp[t];
        unsigned char kc = tmpc[t];
        int u = t - 1;
        while (u >= 0 && cmp_pair(&tmp[u], &key) > 0) {
          tmp[u + 1] = tmp[u];
          tmpc[u + 1] = tmpc[u];
          --u;
        }
        tmp[u + 1] = key;
        tmpc[u + 1] = kc;
      }
      if (m > Ls) m = Ls;
      for (int t = 0; t < m; ++t) {
        S[t] = tmp[t];
        checked[t] = tmpc[t];
      }
    }
    for (int t = 0; t < k; ++t) {
      out_ids[qi * k + t] = t < m ? S[t].id : -1;
      out_d2[qi * k + t] = t < m ? S[t].d2 : INFINITY;
    }
    if (n_dist) n_dist[qi] = nd;
    if (n_hops) n_hops[qi] = nh;
    free(tmpc);
    free(tmp);
    free(checked);
    free(S);
    free(visited);
  }
  return 0;
}

/* Pairwise squared distances of selected rows to selected columns (used by the tests to
 * classify near-tie orderings). */
void or_dist2_pairs(const float* base, int d, const int64_t* a, const int64_t* b, int64_t m,
                    double* out) {
  for (int64_t t = 0; t < m; ++t) out[t] = dist2(base + a[t] * d, base + b[t] * d, d);
}

/* cos of the angle j-i-k (centred form used by the prune) for a list of triples. */
void or_cos_triples(const float* base, int d, const int64_t* i, const int64_t* j,
                    const int64_t* k, int64_t m, double* out) {
  for (int64_t t = 0; t < m; ++t) {
    const float* xi = base + i[t] * d;
    const float* cj = base + j[t] * d;
    const float* ck = base + k[t] * d;
    double gjj = centred_dot(cj, cj, xi, d);
    double gkk = centred_dot(ck, ck, xi, d);
    double gjk = centred_dot(cj, ck, xi, d);
    out[t] = (gjj != 0.0 && gkk != 0.0) ? gjk / sqrt(gjj * gkk) : 0.0;
  }
}
