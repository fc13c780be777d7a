// Serving layer of libgdwd: a slot scheduler for many independent problems.
//
// Each of `slots` host worker threads owns one CUDA stream and runs one
// problem at a time through the public entry points (gdwd_create on its stream
// with grid = sms / slots, gdwd_solve, gdwd_free), so the persistent kernels of
// different slots run side by side on disjoint SM shares.  Requests are served
// in arrival order as slots free up (continuous batching); a request is
// admitted only while the summed device footprint of the problems in flight
// stays within the HBM budget.  Cooperative launches of different slots never
// wait on one another: their grids add up to at most the SM count.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/gdwd.h"
#include <cuda_runtime.h>

namespace gdwd {
void set_thread_error(const std::string& m);
}

namespace {

using clk = std::chrono::steady_clock;

struct Pending {
  gdwd_request r;
  uint64_t ticket;
  clk::time_point t_submit;
};

struct Finished {
  gdwd_result res;
  gdwd_status st;
  double latency_ms;
  std::string msg;
};

// device bytes of one problem: stored Z, G and G^{-1} (8 n^2 each), set-up
// temporaries (Gram partials, Cholesky work: up to ~6 x 8 n^2), state vectors
uint64_t footprint(const gdwd_request& r) {
  const int st = r.opts.store;
  const uint64_t es = st == GDWD_F64 ? 8 : st == GDWD_F32 ? 4 : st == GDWD_E4M3 ? 1 : 2;
  const uint64_t d = (uint64_t)r.d, n = (uint64_t)r.n;
  if (r.opts.solver == 1)   // direct solver: Z^T plus a transposed copy at set-up, d x d matrices, n-vectors
    return 2 * (n + 4096) * d * es + 64ull * d * d + 96ull * n + 4096ull * d + (8ull << 20);
  const uint64_t kern = r.opts.kernelized ? 8ull * n * (n + 1) : 0;   // K as double-float
  return (d + 4096) * n * es + 64ull * n * n + kern + 160ull * (d + 4096) + 4096ull * n + (8ull << 20);
}

}  // namespace

struct gdwd_server {
  int slots = 1;
  int device = 0;
  int share = 1;
  uint64_t budget = 0;
  uint64_t used = 0;
  int inflight = 0;
  bool stop = false;
  uint64_t next = 1;
  std::mutex m;
  std::condition_variable cv_work, cv_done, cv_mem;
  std::deque<Pending> queue;
  std::unordered_map<uint64_t, Finished> done;
  std::vector<std::thread> workers;
  std::vector<cudaStream_t> streams;
  uint64_t outstanding = 0;
};

static void worker_main(gdwd_server* s, int k) {
  cudaSetDevice(s->device);
  for (;;) {
    Pending p;
    uint64_t bytes = 0;
    {
      std::unique_lock<std::mutex> lk(s->m);
      s->cv_work.wait(lk, [&] { return s->stop || !s->queue.empty(); });
      if (s->queue.empty()) return;
      p = s->queue.front();
      s->queue.pop_front();
      bytes = footprint(p.r);
      // admission by HBM footprint; a request that alone exceeds the budget runs by itself
      s->cv_mem.wait(lk, [&] { return s->used + bytes <= s->budget || s->inflight == 0; });
      s->used += bytes;
      s->inflight += 1;
    }
    gdwd_request r = p.r;
    r.opts.stream = (void*)s->streams[k];
    r.opts.grid = s->share;
    gdwd_result res;
    std::memset(&res, 0, sizeof(res));
    gdwd_handle* h = nullptr;
    std::string msg;
    gdwd_status st = gdwd_create(r.Z, r.zdt, r.d, r.n, r.ldz, r.z_on_device, r.y, r.q, r.C, &r.opts, &h);
    if (st == GDWD_OK) {
      st = gdwd_solve(h, nullptr, 0, r.w, 0, r.alpha, &res);
      if (st != GDWD_OK) msg = gdwd_last_error(h);
      gdwd_free(h);
    } else {
      res.status = st;
      msg = gdwd_last_error(nullptr);
    }
    const double lat = std::chrono::duration<double, std::milli>(clk::now() - p.t_submit).count();
    {
      std::lock_guard<std::mutex> lk(s->m);
      s->used -= bytes;
      s->inflight -= 1;
      s->done[p.ticket] = Finished{res, st, lat, msg};
      s->outstanding -= 1;
    }
    s->cv_mem.notify_all();
    s->cv_done.notify_all();
  }
}

extern "C" gdwd_status gdwd_server_create(int32_t slots, uint64_t hbm_budget, gdwd_server** out) {
  if (!out || slots < 1 || slots > 64) return GDWD_EINVAL;
  *out = nullptr;
  gdwd_server* s = new gdwd_server();
  s->slots = slots;
  if (cudaGetDevice(&s->device) != cudaSuccess) {
    delete s;
    return GDWD_ECUDA;
  }
  int sms = 1;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s->device);
  s->share = std::max(1, sms / slots);
  if (hbm_budget == 0) {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
      delete s;
      return GDWD_ECUDA;
    }
    hbm_budget = (uint64_t)(0.8 * (double)fr);
  }
  s->budget = hbm_budget;
  s->streams.resize(slots);
  for (int k = 0; k < slots; ++k) {
    if (cudaStreamCreateWithFlags(&s->streams[k], cudaStreamNonBlocking) != cudaSuccess) {
      for (int j = 0; j < k; ++j) cudaStreamDestroy(s->streams[j]);
      delete s;
      return GDWD_ECUDA;
    }
  }
  for (int k = 0; k < slots; ++k) s->workers.emplace_back(worker_main, s, k);
  *out = s;
  return GDWD_OK;
}

extern "C" gdwd_status gdwd_server_submit(gdwd_server* s, const gdwd_request* r, uint64_t* ticket) {
  if (!s || !r || !ticket || !r->Z || !r->y) return GDWD_EINVAL;
  std::lock_guard<std::mutex> lk(s->m);
  if (s->stop) return GDWD_EINVAL;
  Pending p{*r, s->next++, clk::now()};
  *ticket = p.ticket;
  s->queue.push_back(p);
  s->outstanding += 1;
  s->cv_work.notify_one();
  return GDWD_OK;
}

extern "C" gdwd_status gdwd_server_poll(gdwd_server* s, uint64_t ticket, int32_t wait, gdwd_result* res,
                                        double* latency_ms) {
  if (!s || !res) return GDWD_EINVAL;
  std::unique_lock<std::mutex> lk(s->m);
  if (ticket == 0 || ticket >= s->next) return GDWD_EINVAL;
  auto it = s->done.find(ticket);
  if (it == s->done.end()) {
    if (!wait) return GDWD_EAGAIN;
    s->cv_done.wait(lk, [&] { return s->done.count(ticket) > 0; });
    it = s->done.find(ticket);
  }
  *res = it->second.res;
  if (latency_ms) *latency_ms = it->second.latency_ms;
  const gdwd_status st = it->second.st;
  if (st != GDWD_OK) gdwd::set_thread_error(it->second.msg);
  s->done.erase(it);
  return st;
}

extern "C" gdwd_status gdwd_server_destroy(gdwd_server* s) {
  if (!s) return GDWD_OK;
  {
    std::unique_lock<std::mutex> lk(s->m);
    s->cv_done.wait(lk, [&] { return s->outstanding == 0; });
    s->stop = true;
  }
  s->cv_work.notify_all();
  s->cv_mem.notify_all();
  for (auto& t : s->workers) t.join();
  for (auto st : s->streams) cudaStreamDestroy(st);
  delete s;
  return GDWD_OK;
}

extern "C" gdwd_status gdwd_solve_batch(const gdwd_request* reqs, int32_t nreq, int32_t slots, gdwd_result* res,
                                        double* latency_ms) {
  if (nreq < 0 || (nreq > 0 && (!reqs || !res))) return GDWD_EINVAL;
  if (nreq == 0) return GDWD_OK;
  gdwd_server* s = nullptr;
  gdwd_status st = gdwd_server_create(std::max(1, std::min(slots, nreq)), 0, &s);
  if (st != GDWD_OK) return st;
  std::vector<uint64_t> tickets(nreq);
  gdwd_status worst = GDWD_OK;
  for (int i = 0; i < nreq; ++i) {
    st = gdwd_server_submit(s, &reqs[i], &tickets[i]);
    if (st != GDWD_OK) {
      worst = st;
      tickets[i] = 0;
    }
  }
  for (int i = 0; i < nreq; ++i) {
    if (!tickets[i]) continue;
    double lat = 0.0;
    st = gdwd_server_poll(s, tickets[i], 1, &res[i], &lat);
    if (latency_ms) latency_ms[i] = lat;
    if (st != GDWD_OK && (worst == GDWD_OK || worst == GDWD_EMAXITER)) worst = st;
  }
  gdwd_server_destroy(s);
  return worst;
}
