// Serving: many problems (k, n) behind one submit / poll interface (include/hh.h,
// hh_server_*).  Host code only, layered on the handle API.
//
// * Factor cache.  One handle per (k, n, strips, dirs), kept resident (strip factors, sweep
//   workspaces, Krylov block pool) and reused by later requests for the same problem.
// * Admission by device memory.  A request whose problem is not cached needs a new handle;
//   its device bytes are estimated (factor store, its tensor-core copies, sweep arrays,
//   Krylov state for the handle's slots) and admitted against the budget, evicting idle
//   handles least recently used first.  A request that cannot be admitted yet stays queued
//   until running requests release memory.
// * Overlap.  Every handle has its own stream and request loop (continuous batching of its
//   requests), so the solves of different problems and the setup of a new one run on the
//   device at the same time.
// * Latency.  A completion thread polls the running requests and stamps their completion
//   time; hh_server_poll reports submit-to-completion time in t_solve_ms.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <tuple>
#include <unordered_map>
#include <vector>

#include "../../include/hh.h"
#include "engine.h"

namespace hh {
void set_error(const std::string& msg);
}

namespace {

using Clock = std::chrono::steady_clock;
using Key = std::tuple<double, int, int, uint32_t>;

struct Entry {
  hh_handle* h = nullptr;
  size_t bytes = 0;
  int inflight = 0;
  uint64_t last_use = 0;
};

struct SReq {
  hh_ticket id = 0;
  Key key;
  std::vector<double> src;  // nsrc rows of (x0, y0, sigma, re, im)
  double* x = nullptr;
  double tol = 0;
  size_t rhs_bytes = 0;
  void* rhs = nullptr;  // assembled load vector on the device
  Entry* e = nullptr;
  hh_ticket inner = 0;
  int state = 0;  // 0 queued, 1 running, 2 done
  hh_result res{};
  Clock::time_point t_submit, t_done;
};

int popcount4(uint32_t d) { return (d & 1) + ((d >> 1) & 1) + ((d >> 2) & 1) + ((d >> 3) & 1); }

}  // namespace

struct hh_server {
  hh_opts opts{};
  size_t budget = 0, used = 0;
  int device = 0;
  std::mutex mu;
  std::condition_variable cv;
  std::map<Key, Entry*> cache;
  std::deque<SReq*> queue;
  std::vector<SReq*> running;
  std::unordered_map<hh_ticket, SReq*> all;
  std::multimap<size_t, void*> rhs_pool;  // free device buffers by size
  std::thread dispatcher, reaper;
  bool stopping = false;
  uint64_t use_clock = 0, next_ticket = 1;
  int64_t setups = 0, hits = 0, evictions = 0, completed = 0;
  double setup_ms = 0;

  // Device bytes a handle for this problem can hold once warm (the estimate admission uses):
  // its factor store (every block of its sweep form and cyclic-reduction depths, with the
  // tensor cores' hi and lo copies), sweep workspaces, and per slot the Krylov state of a solve
  // that runs to the iteration cap opts.maxit (basis and search directions of t columns per
  // iteration), so that no admitted request can outgrow the budget.
  size_t estimate(const Key& k) const {
    const int n = std::get<1>(k), N = std::get<2>(k);
    const int t = popcount4(std::get<3>(k));
    const size_t m = (size_t)n + 1, R = (size_t)n / N, ldf = (m + 3) & ~(size_t)3;
    const size_t elem = opts.precision != HH_PREC_FP64 ? 8 : 16;
    const size_t copies = (opts.precision != HH_PREC_FP64 && opts.tensor_cores) ? 4 : 1;
    unsigned depths = 0;
    if (opts.bcr_depth > 0) depths = 1u << opts.bcr_depth;
    else if (opts.bcr_depth < 0)
      for (int d = 1; d <= hh::max_bcr_depth((int)R); ++d) depths |= 1u << d;
    const bool twisted =
        opts.twisted != 0 && opts.bcr_depth <= 0 && opts.precision == HH_PREC_FP32 && opts.tensor_cores;
    const size_t blocks = (size_t)hh::block_directory((int)R, N, opts.interface_form, depths, twisted).total;
    const size_t factors = copies * blocks * m * ldf * elem;
    const size_t C = (size_t)t * opts.serve_slots;
    const size_t sweep = 3 * (R + 1) * m * N * C * elem + 10 * m * N * C * elem;
    const size_t D = m * m;
    // per slot: t-column W and its three planes, b, staging x, and 2 t basis / search vectors
    // per iteration up to the cap; with the tensor-core Gram-Schmidt no planes, but 64 bytes
    // per node for every basis vector's slice images
    const size_t iters = (size_t)opts.maxit * t;
    const size_t krylov =
        opts.gs_tensor ? (size_t)opts.serve_slots * (D * 8 * (2 * t + 4 + 4 * iters) + 64 * D * (1 + iters))
                       : (size_t)opts.serve_slots * D * 8 * (2 * t + 3 * t + 4 + 4 * iters);
    return factors + sweep + krylov + (64u << 20);
  }

  void* take_rhs(size_t bytes) {
    auto it = rhs_pool.find(bytes);
    if (it != rhs_pool.end()) {
      void* p = it->second;
      rhs_pool.erase(it);
      return p;
    }
    void* p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    return p;
  }

  // Evicts the least recently used idle handle (lock held on entry, released while the handle
  // is destroyed).  Returns false if no handle is idle.
  bool evict_one(std::unique_lock<std::mutex>& lk) {
    auto victim = cache.end();
    for (auto it = cache.begin(); it != cache.end(); ++it)
      if (it->second->inflight == 0 && (victim == cache.end() || it->second->last_use < victim->second->last_use))
        victim = it;
    if (victim == cache.end()) return false;
    Entry* e = victim->second;
    cache.erase(victim);
    used -= e->bytes;
    ++evictions;
    lk.unlock();
    hh_destroy(e->h);
    delete e;
    lk.lock();
    return true;
  }

  void fail(SReq* q, hh_status st) {
    std::memset(&q->res, 0, sizeof(q->res));
    q->res.status = st;
    q->state = 2;
    q->t_done = Clock::now();
  }

  void dispatch_loop() {
    cudaSetDevice(device);
    std::unique_lock<std::mutex> lk(mu);
    for (;;) {
      cv.wait(lk, [&] { return stopping || !queue.empty(); });
      if (stopping) return;
      SReq* q = queue.front();
      Entry* e = nullptr;
      auto it = cache.find(q->key);
      if (it != cache.end()) {
        e = it->second;
        ++hits;
      } else {
        const size_t need = estimate(q->key);
        while (used + need > budget && evict_one(lk)) {
        }
        if (stopping) return;
        if (queue.empty() || queue.front() != q) continue;
        if (used + need > budget) {
          if (running.empty()) {  // nothing will ever free memory for it
            queue.pop_front();
            fail(q, HH_ENOMEM);
            continue;
          }
          cv.wait_for(lk, std::chrono::milliseconds(2));  // a completion may free memory
          continue;
        }
        used += need;  // reserved while the handle is built
        lk.unlock();
        hh_opts o = opts;
        o.stream = nullptr;
        hh_handle* h = nullptr;
        const auto t0 = Clock::now();
        const hh_status st = hh_setup(std::get<0>(q->key), std::get<1>(q->key), std::get<2>(q->key),
                                      std::get<3>(q->key), &o, &h);
        const double ms = std::chrono::duration<double, std::milli>(Clock::now() - t0).count();
        lk.lock();
        if (stopping) {  // the queue was failed and cleared meanwhile; hand the handle to the cache
          if (st == HH_OK) {
            e = new Entry();
            e->h = h;
            e->bytes = need;
            cache[q->key] = e;
          }
          return;
        }
        if (st != HH_OK) {
          used -= need;
          queue.pop_front();
          fail(q, st);
          continue;
        }
        e = new Entry();
        e->h = h;
        e->bytes = need;
        cache[q->key] = e;
        ++setups;
        setup_ms += ms;
      }
      queue.pop_front();
      e->inflight++;
      e->last_use = ++use_clock;
      q->e = e;
      q->rhs = take_rhs(q->rhs_bytes);
      lk.unlock();
      hh_status st = q->rhs ? HH_OK : HH_ENOMEM;
      if (st == HH_OK)
        st = hh_assemble_rhs(e->h, (int)(q->src.size() / 5), q->src.data(), reinterpret_cast<double*>(q->rhs));
      if (st == HH_OK) st = hh_submit(e->h, reinterpret_cast<const double*>(q->rhs), q->x, q->tol, &q->inner);
      lk.lock();
      if (st != HH_OK) {
        e->inflight--;
        if (q->rhs) rhs_pool.emplace(q->rhs_bytes, q->rhs);
        q->rhs = nullptr;
        fail(q, st);
        continue;
      }
      q->state = 1;
      running.push_back(q);
    }
  }

  void reap_loop() {
    cudaSetDevice(device);
    std::unique_lock<std::mutex> lk(mu);
    while (!stopping || !running.empty()) {
      for (size_t i = 0; i < running.size();) {
        SReq* q = running[i];
        hh_result r{};
        const hh_status st = hh_poll(q->inner, &r);
        if (st == HH_EPENDING) {
          ++i;
          continue;
        }
        q->t_done = Clock::now();
        q->res = r;
        q->res.status = st;
        q->state = 2;
        q->e->inflight--;
        rhs_pool.emplace(q->rhs_bytes, q->rhs);
        q->rhs = nullptr;
        ++completed;
        running[i] = running.back();
        running.pop_back();
        cv.notify_all();
      }
      cv.wait_for(lk, std::chrono::microseconds(300));
    }
  }
};

extern "C" {

hh_status hh_server_create(const hh_opts* opts, size_t mem_budget, hh_server** out) {
  if (!out) return (hh::set_error("out must be non-NULL"), HH_EINVAL);
  *out = nullptr;
  auto* s = new hh_server();
  hh_default_opts(&s->opts);
  if (opts) s->opts = *opts;
  if (s->opts.serve_slots < 1 || s->opts.serve_slots > 256 || s->opts.maxit < 1 ||
      s->opts.discretization != HH_DISC_P1) {
    delete s;
    return (hh::set_error("invalid options"), HH_EINVAL);
  }
  cudaGetDevice(&s->device);
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
    cudaGetLastError();
    delete s;
    return (hh::set_error("cudaMemGetInfo failed"), HH_ECUDA);
  }
  s->budget = mem_budget ? mem_budget : (size_t)(0.85 * (double)free_b);
  s->dispatcher = std::thread([s] { s->dispatch_loop(); });
  s->reaper = std::thread([s] { s->reap_loop(); });
  *out = s;
  return HH_OK;
}

hh_status hh_server_submit(hh_server* s, double k, int n, int strips, uint32_t dirs, int nsrc, const double* src,
                           double* x, double tol, hh_ticket* ticket) {
  if (!s || !x || !ticket || nsrc < 1 || !src) return (hh::set_error("bad arguments"), HH_EINVAL);
  if (!(k > 0) || n < 2 || strips < 1 || n % strips || n / strips < 2 || dirs == 0 || (dirs & ~15u) || !(tol > 0))
    return (hh::set_error("bad problem (k, n, strips, dirs, tol)"), HH_EINVAL);
  auto* q = new SReq();
  q->key = Key(k, n, strips, dirs);
  q->src.assign(src, src + 5 * (size_t)nsrc);
  q->x = x;
  q->tol = tol;
  q->rhs_bytes = (size_t)(n + 1) * (n + 1) * 16;
  q->t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stopping) {
      delete q;
      return (hh::set_error("server is shutting down"), HH_EINVAL);
    }
    q->id = s->next_ticket++;
    s->all[q->id] = q;
    s->queue.push_back(q);
  }
  s->cv.notify_all();
  *ticket = q->id;
  return HH_OK;
}

hh_status hh_server_poll(hh_server* s, hh_ticket ticket, hh_result* res) {
  if (!s) return (hh::set_error("server is NULL"), HH_EINVAL);
  SReq* q = nullptr;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->all.find(ticket);
    if (it == s->all.end()) return (hh::set_error("unknown ticket"), HH_EINVAL);
    q = it->second;
    if (q->state != 2) return HH_EPENDING;
    s->all.erase(it);
  }
  hh_result r = q->res;
  r.t_solve_ms = std::chrono::duration<double, std::milli>(q->t_done - q->t_submit).count();
  if (res) *res = r;
  const hh_status st = r.status;
  delete q;
  return st;
}

hh_status hh_server_get_stats(hh_server* s, hh_server_stats* st) {
  if (!s || !st) return (hh::set_error("bad arguments"), HH_EINVAL);
  std::lock_guard<std::mutex> lk(s->mu);
  std::memset(st, 0, sizeof(*st));
  st->handles = (int64_t)s->cache.size();
  st->bytes_reserved = (int64_t)s->used;
  st->budget = (int64_t)s->budget;
  st->setups = s->setups;
  st->cache_hits = s->hits;
  st->evictions = s->evictions;
  st->completed = s->completed;
  st->queued = (int64_t)s->queue.size();
  st->running = (int64_t)s->running.size();
  st->setup_ms = s->setup_ms;
  return HH_OK;
}

void hh_server_destroy(hh_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stopping = true;
    for (SReq* q : s->queue) s->fail(q, HH_EINVAL);
    s->queue.clear();
  }
  s->cv.notify_all();
  if (s->dispatcher.joinable()) s->dispatcher.join();
  if (s->reaper.joinable()) s->reaper.join();  // waits for the running requests
  for (auto& kv : s->cache) {
    hh_destroy(kv.second->h);
    delete kv.second;
  }
  for (auto& kv : s->rhs_pool) cudaFree(kv.second);
  for (auto& kv : s->all) delete kv.second;
  delete s;
}

}  // extern "C"
