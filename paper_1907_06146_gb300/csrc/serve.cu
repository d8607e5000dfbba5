// Serving loop: continuous batching of Search-on-Graph (Alg. 1) requests against a
// device-resident NSSG index.
//
// Callers submit requests (a block of queries with its own k and L_search) from any host
// thread and wait for them by ticket.  One scheduler thread owns the GPU side.  Whenever a
// batch slot is free it packs waiting requests first come, first served, into one batch,
// as long as the batch stays within max_batch queries and the device bytes of all queries
// in flight (queries, per-query parameters, results) stay within the memory budget; the
// batch is copied in, searched (one kernel, each query with its own k and L_search) and
// copied out on the slot's own CUDA stream, and a host callback on that stream tells the
// scheduler that the slot is free.  Batches on different streams overlap on the device, and
// requests that arrive meanwhile are admitted as soon as a slot and memory free up.
//
// The search of one query does not depend on the other queries of its batch (one warp
// per query, private shared memory), so a result is the same alone and in any mix.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "common.cuh"
#include "graph.cuh"
#include "knn.cuh"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  uint64_t ticket = 0;
  std::vector<float> q;  // nq x d, as submitted
  int64_t nq = 0;
  int32_t k = 0, ls = 0;
  std::vector<int32_t> ids;  // nq x k
  std::vector<float> d2;
  bool done = false;
  ssg_status status = SSG_OK;
  Clock::time_point t_submit, t_done;
  size_t bytes = 0;  // device bytes while in flight
};

struct Member {
  Request* r;
  int64_t offset;  // first row of the batch
};

struct Slot {
  ssg_server* srv = nullptr;
  cudaStream_t st = nullptr;
  float* h_q = nullptr;
  int32_t* h_par = nullptr;  // k then L_search, per query
  int32_t* h_ids = nullptr;
  float* h_d2 = nullptr;
  float* d_q = nullptr;
  int32_t* d_par = nullptr;
  int32_t* d_ids = nullptr;
  float* d_d2 = nullptr;
  bool busy = false, ready = false;
  ssg_status launch_status = SSG_OK;
  std::vector<Member> members;
  int64_t nq = 0;
  int ldo = 0;
  size_t bytes = 0;
  Clock::time_point t_launch;
};

}  // namespace

struct ssg_server {
  const ssg_graph* g = nullptr;
  int dev = 0;
  int d = 0, ld = 0;
  const float* base = nullptr;
  const uint8_t* rows_u8 = nullptr;  // the graph's byte rows when they are of this base
  ssg::Scratch<float> base_pad;
  ssg_server_opts opts{};
  std::vector<std::unique_ptr<Slot>> slots;
  std::deque<Request*> pending;
  std::unordered_map<uint64_t, std::unique_ptr<Request>> reqs;
  uint64_t next_ticket = 1;
  std::mutex mu;
  std::condition_variable cv;
  std::thread worker;
  bool stop = false;
  size_t mem_in_use = 0;
  ssg_server_stats stats{};
  Clock::time_point t_busy_start;
  int busy_slots = 0;
};

namespace {

void CUDART_CB on_slot_done(void* p) {
  Slot* s = (Slot*)p;
  ssg_server* srv = s->srv;
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    s->ready = true;
  }
  srv->cv.notify_all();
}

size_t request_bytes(const ssg_server* s, int64_t nq, int k) {
  return (size_t)nq * ((size_t)s->ld * 4 + 8 + (size_t)k * 8);
}

// Copy a finished slot's results into its requests (mutex held).
void finish_slot(ssg_server* s, Slot& sl) {
  const auto now = Clock::now();
  for (const Member& m : sl.members) {
    Request* r = m.r;
    r->ids.resize((size_t)r->nq * r->k);
    r->d2.resize((size_t)r->nq * r->k);
    for (int64_t i = 0; i < r->nq; ++i) {
      memcpy(&r->ids[i * r->k], sl.h_ids + (m.offset + i) * sl.ldo, sizeof(int32_t) * r->k);
      memcpy(&r->d2[i * r->k], sl.h_d2 + (m.offset + i) * sl.ldo, sizeof(float) * r->k);
    }
    r->status = sl.launch_status;
    r->done = true;
    r->t_done = now;
    s->stats.requests_done += 1;
    s->stats.queries_done += r->nq;
  }
  s->mem_in_use -= sl.bytes;
  sl.members.clear();
  sl.busy = sl.ready = false;
  if (--s->busy_slots == 0)
    s->stats.busy_ms +=
        std::chrono::duration<double, std::milli>(now - s->t_busy_start).count();
}

// Pack waiting requests into a free slot and launch it (mutex held).  Returns false if
// nothing could be admitted.
bool launch_batch(ssg_server* s, Slot& sl) {
  int64_t nq = 0;
  int kmax = 1, lsmax = 1;
  size_t bytes = 0;
  while (!s->pending.empty()) {
    Request* r = s->pending.front();
    const size_t b = request_bytes(s, r->nq, r->k);
    if (nq + r->nq > s->opts.max_batch || s->mem_in_use + bytes + b > (size_t)s->opts.mem_budget_bytes)
      break;
    s->pending.pop_front();
    sl.members.push_back({r, nq});
    for (int64_t i = 0; i < r->nq; ++i) {
      float* dst = sl.h_q + (nq + i) * s->ld;
      memcpy(dst, &r->q[i * s->d], sizeof(float) * s->d);
      for (int t = s->d; t < s->ld; ++t) dst[t] = 0.f;
      sl.h_par[nq + i] = r->k;
      sl.h_par[s->opts.max_batch + nq + i] = r->ls;
    }
    nq += r->nq;
    bytes += b;
    kmax = std::max(kmax, r->k);
    lsmax = std::max(lsmax, r->ls);
  }
  if (nq == 0) return false;
  sl.nq = nq;
  sl.ldo = kmax;
  sl.bytes = bytes;
  sl.busy = true;
  sl.ready = false;
  sl.launch_status = SSG_OK;
  sl.t_launch = Clock::now();
  s->mem_in_use += bytes;
  if (s->busy_slots++ == 0) s->t_busy_start = sl.t_launch;
  s->stats.batches += 1;
  s->stats.max_batches_in_flight = std::max<int64_t>(s->stats.max_batches_in_flight, s->busy_slots);
  int64_t inflight_q = 0;
  for (auto& o : s->slots)
    if (o->busy) inflight_q += o->nq;
  s->stats.max_queries_in_flight = std::max<int64_t>(s->stats.max_queries_in_flight, inflight_q);
  try {
    const ssg_graph* g = s->g;
    SSG_CUDA(cudaMemcpyAsync(sl.d_q, sl.h_q, sizeof(float) * nq * s->ld, cudaMemcpyHostToDevice, sl.st));
    SSG_CUDA(cudaMemcpyAsync(sl.d_par, sl.h_par, sizeof(int32_t) * nq, cudaMemcpyHostToDevice, sl.st));
    SSG_CUDA(cudaMemcpyAsync(sl.d_par + s->opts.max_batch, sl.h_par + s->opts.max_batch,
                             sizeof(int32_t) * nq, cudaMemcpyHostToDevice, sl.st));
    ssg::search_run_mixed(s->base, s->rows_u8, s->ld, s->d, g->adj, g->deg, g->R, g->nav_dev, g->n_nav, sl.d_q,
                          s->ld, nq, sl.d_par, sl.d_par + s->opts.max_batch, lsmax, kmax, sl.d_ids,
                          sl.d_d2, sl.st);
    SSG_CUDA(cudaMemcpyAsync(sl.h_ids, sl.d_ids, sizeof(int32_t) * nq * kmax, cudaMemcpyDeviceToHost,
                             sl.st));
    SSG_CUDA(cudaMemcpyAsync(sl.h_d2, sl.d_d2, sizeof(float) * nq * kmax, cudaMemcpyDeviceToHost, sl.st));
    SSG_CUDA(cudaLaunchHostFunc(sl.st, on_slot_done, &sl));
  } catch (const ssg::Fail& e) {
    sl.launch_status = e.st;
    sl.ready = true;  // finish it with the error status on the next pass
  }
  return true;
}

void scheduler(ssg_server* s) {
  cudaSetDevice(s->dev);
  std::unique_lock<std::mutex> lk(s->mu);
  for (;;) {
    for (auto& sl : s->slots)
      if (sl->busy && sl->ready) finish_slot(s, *sl);
    bool launched = false;
    for (auto& sl : s->slots) {
      if (s->pending.empty()) break;
      if (!sl->busy && launch_batch(s, *sl)) launched = true;
    }
    if (launched) continue;
    if (s->stop && s->pending.empty() && s->busy_slots == 0) break;
    s->cv.notify_all();  // waiters may have results
    s->cv.wait(lk);
  }
  s->cv.notify_all();
}

}  // namespace

using namespace ssg;

extern "C" {

void ssg_server_default_opts(ssg_server_opts* o) {
  if (!o) return;
  o->n_streams = 4;
  o->max_batch = 8192;
  o->mem_budget_bytes = 256ll << 20;
  o->max_k = 128;
  o->max_L_search = 1024;
}

ssg_status ssg_server_create(const ssg_graph* g, const float* base, const ssg_server_opts* opts_in,
                             ssg_server** out) {
  std::unique_ptr<ssg_server> s(new ssg_server());
  try {
    SSG_REQUIRE(g && out, SSG_EINVAL, "null argument");
    *out = nullptr;
    ssg_server_opts o;
    ssg_server_default_opts(&o);
    if (opts_in) o = *opts_in;
    SSG_REQUIRE(o.n_streams >= 1 && o.n_streams <= 64 && o.max_batch >= 1 && o.max_k >= 1 &&
                    o.max_L_search >= o.max_k && o.max_L_search <= 1024 && o.mem_budget_bytes > 0,
                SSG_EINVAL, "bad server options");
    const float* b = base ? base : g->base_owned;
    SSG_REQUIRE(b, SSG_EINVAL, "no base vectors: pass the device array the graph was built from");
    s->g = g;
    s->opts = o;
    s->d = g->d;
    SSG_CUDA(cudaGetDevice(&s->dev));
    for (int i = 0; i < o.n_streams; ++i) {
      std::unique_ptr<Slot> sl(new Slot());
      sl->srv = s.get();
      SSG_CUDA(cudaStreamCreateWithFlags(&sl->st, cudaStreamNonBlocking));
      s->slots.push_back(std::move(sl));
    }
    PaddedRows pr;
    pad_rows(b, g->n, g->d, s->slots[0]->st, pr);
    s->ld = pr.ld;
    if (pr.own.p) {
      s->base_pad.p = pr.own.p;  // keep the padded copy for the server's lifetime
      s->base_pad.s = pr.own.s;
      s->base_pad.count = pr.own.count;
      pr.own.p = nullptr;
    }
    s->base = s->base_pad.p ? s->base_pad.p : b;
    if (g->rows_u8 && b == g->rows_src && g->rows_ld == s->ld) s->rows_u8 = g->rows_u8;
    SSG_CUDA(cudaStreamSynchronize(s->slots[0]->st));
    const size_t mb = (size_t)o.max_batch;
    for (auto& sl : s->slots) {
      SSG_CUDA(cudaHostAlloc((void**)&sl->h_q, sizeof(float) * mb * s->ld, cudaHostAllocDefault));
      SSG_CUDA(cudaHostAlloc((void**)&sl->h_par, sizeof(int32_t) * 2 * mb, cudaHostAllocDefault));
      SSG_CUDA(cudaHostAlloc((void**)&sl->h_ids, sizeof(int32_t) * mb * o.max_k, cudaHostAllocDefault));
      SSG_CUDA(cudaHostAlloc((void**)&sl->h_d2, sizeof(float) * mb * o.max_k, cudaHostAllocDefault));
      SSG_CUDA(cudaMalloc(&sl->d_q, sizeof(float) * mb * s->ld));
      SSG_CUDA(cudaMalloc(&sl->d_par, sizeof(int32_t) * 2 * mb));
      SSG_CUDA(cudaMalloc(&sl->d_ids, sizeof(int32_t) * mb * o.max_k));
      SSG_CUDA(cudaMalloc(&sl->d_d2, sizeof(float) * mb * o.max_k));
    }
    s->worker = std::thread(scheduler, s.get());
    *out = s.release();
    return SSG_OK;
  } catch (const Fail& e) {
    ssg_server_destroy(s.release());
    return e.st;
  } catch (...) {
    set_error("unexpected exception");
    ssg_server_destroy(s.release());
    return SSG_EINTERNAL;
  }
}

ssg_status ssg_server_submit(ssg_server* s, const float* queries_host, int64_t nq, int32_t k,
                             int32_t L_search, uint64_t* ticket) {
  try {
    SSG_REQUIRE(s && queries_host && ticket && nq >= 1, SSG_EINVAL, "bad arguments");
    SSG_REQUIRE(k >= 1 && k <= s->opts.max_k && k <= L_search && L_search <= s->opts.max_L_search,
                SSG_EINVAL, "need 1 <= k <= min(L_search, max_k) and L_search <= max_L_search");
    SSG_REQUIRE(nq <= s->opts.max_batch, SSG_EINVAL, "a request may hold at most max_batch = %d queries",
                s->opts.max_batch);
    SSG_REQUIRE(request_bytes(s, nq, k) <= (size_t)s->opts.mem_budget_bytes, SSG_EINVAL,
                "the request needs more device memory than the whole budget");
    std::unique_ptr<Request> r(new Request());
    r->q.assign(queries_host, queries_host + (size_t)nq * s->d);
    r->nq = nq;
    r->k = k;
    r->ls = L_search;
    r->t_submit = Clock::now();
    {
      std::lock_guard<std::mutex> lk(s->mu);
      SSG_REQUIRE(!s->stop, SSG_EINVAL, "server is shutting down");
      r->ticket = s->next_ticket++;
      *ticket = r->ticket;
      s->pending.push_back(r.get());
      s->reqs[r->ticket] = std::move(r);
    }
    s->cv.notify_all();
    return SSG_OK;
  } catch (const Fail& e) {
    return e.st;
  } catch (...) {
    set_error("unexpected exception");
    return SSG_EINTERNAL;
  }
}

ssg_status ssg_server_poll(ssg_server* s, uint64_t ticket, int32_t* done) {
  if (!s || !done) {
    set_error("null argument");
    return SSG_EINVAL;
  }
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) {
    set_error("unknown ticket %llu", (unsigned long long)ticket);
    return SSG_EINVAL;
  }
  *done = it->second->done ? 1 : 0;
  return SSG_OK;
}

ssg_status ssg_server_wait(ssg_server* s, uint64_t ticket, int32_t* ids_host, float* d2_host,
                           double* latency_ms) {
  if (!s || !ids_host) {
    set_error("null argument");
    return SSG_EINVAL;
  }
  std::unique_ptr<Request> r;
  {
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) {
      set_error("unknown ticket %llu", (unsigned long long)ticket);
      return SSG_EINVAL;
    }
    Request* rp = it->second.get();
    s->cv.wait(lk, [&] { return rp->done; });
    r = std::move(it->second);
    s->reqs.erase(it);
  }
  if (r->status != SSG_OK) return r->status;
  memcpy(ids_host, r->ids.data(), sizeof(int32_t) * r->ids.size());
  if (d2_host) memcpy(d2_host, r->d2.data(), sizeof(float) * r->d2.size());
  if (latency_ms) *latency_ms = std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count();
  return SSG_OK;
}

ssg_status ssg_server_get_stats(ssg_server* s, ssg_server_stats* out) {
  if (!s || !out) {
    set_error("null argument");
    return SSG_EINVAL;
  }
  std::lock_guard<std::mutex> lk(s->mu);
  *out = s->stats;
  return SSG_OK;
}

void ssg_server_destroy(ssg_server* s) {
  if (!s) return;
  if (s->worker.joinable()) {
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->stop = true;
    }
    s->cv.notify_all();
    s->worker.join();
  }
  for (auto& sl : s->slots) {
    if (sl->st) cudaStreamSynchronize(sl->st);
    if (sl->h_q) cudaFreeHost(sl->h_q);
    if (sl->h_par) cudaFreeHost(sl->h_par);
    if (sl->h_ids) cudaFreeHost(sl->h_ids);
    if (sl->h_d2) cudaFreeHost(sl->h_d2);
    if (sl->d_q) cudaFree(sl->d_q);
    if (sl->d_par) cudaFree(sl->d_par);
    if (sl->d_ids) cudaFree(sl->d_ids);
    if (sl->d_d2) cudaFree(sl->d_d2);
  }
  s->base_pad.release();
  if (!s->slots.empty() && s->slots[0]->st) cudaStreamSynchronize(s->slots[0]->st);
  for (auto& sl : s->slots)
    if (sl->st) cudaStreamDestroy(sl->st);
  delete s;
}

}  // extern "C"
