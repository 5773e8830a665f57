// parem_server.cpp -- request server: continuous batching of independent match requests.
//
// Each request is one instance of the matching problem (a DFA, a text); Algorithm 1 runs on
// it unchanged inside the batch kernels, so a response equals parem_match on that request
// alone.  What the server adds is the choice of which requests share a launch:
//
//   submit -> pending (arrival order) --dispatcher--> batch in a free arena --stream-->
//   completion thread (whichever batch finished) -> responses (poll queue, or a replay sink)
//
// * Arenas: each holds one batch's device scratch, device descriptors, the pinned host image
//   of the descriptors and the pinned result words, plus its own stream and event.  They are
//   allocated once; a batch is planned into a free arena (memory admission: requests are
//   taken in arrival order while the count, byte and arena limits hold; a plan that does not
//   fit is halved and the rest goes back to the head of the queue).
// * With several arenas the next batches are launched while earlier ones run: their thread
//   blocks start as soon as blocks of the running batches retire, so new arrivals do not
//   wait for the slowest request of a batch ahead of them (256 arenas by default: with 2, a
//   long request held the GPU's throughput to a third of the offered load, and with 32 the
//   arenas held by long requests made new arrivals queue for half of their p50 latency).
// * FIFO mode serves one request at a time with parem_match (the plain comparison).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "../../include/parem.h"
#include "parem_batch_impl.h"
#include "parem_internal.h"
#include "parem_launch.h"

using namespace parem;

namespace {

int64_t now_ns() {
  return std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

struct ReplaySink {
  parem_response* out = nullptr;
  uint32_t n = 0;
  uint32_t done = 0;
};

struct Req {
  parem_request r;
  ReplaySink* sink = nullptr;
};

struct Arena {
  BatchArena a;
  cudaEvent_t done = nullptr;
};

struct Round {
  int arena = -1;
  parem_batch* batch = nullptr;
  std::vector<Req> reqs;  // in the batch's given order
  int64_t launch_ns = 0;
  std::vector<uint8_t> answered;  // per sorted position: answered early
  uint32_t n_answered = 0;
};

}  // namespace

struct parem_server {
  int device = 0;
  std::vector<parem_dfa*> dfas;
  parem_server_opts opts{};
  std::vector<Arena> arenas;
  cudaStream_t fifo_stream = nullptr;

  std::mutex mu;
  std::condition_variable cv_dispatch;  // pending work and a free arena, or stop
  std::condition_variable cv_done;      // a round in flight, or stop
  std::condition_variable cv_answer;    // responses delivered
  std::deque<Req> pending;
  std::deque<Round> inflight;
  std::vector<int> free_arenas;
  std::deque<parem_response> completed;
  bool stop = false;
  bool dispatcher_done = false;
  parem_server_stats stats{};

  std::thread dispatcher, completer;
};

namespace {

// Deliver responses (server mutex held).
void deliver(parem_server* s, const std::vector<Req>& reqs, const std::vector<parem_response>& resp) {
  for (size_t i = 0; i < reqs.size(); ++i) {
    if (reqs[i].sink) {
      ReplaySink* k = reqs[i].sink;
      k->out[resp[i].tag] = resp[i];
      k->done++;
    } else {
      s->completed.push_back(resp[i]);
    }
  }
  s->stats.answered += reqs.size();
  s->cv_answer.notify_all();
}

parem_response make_response(const Req& q, int status, uint32_t batch_size, const parem_result& res,
                             int64_t launch_ns, int64_t done_ns) {
  parem_response o;
  std::memset(&o, 0, sizeof(o));
  o.tag = q.r.tag;
  o.status = status;
  o.batch_size = batch_size;
  o.result = res;
  o.arrival_ns = q.r.arrival_ns;
  o.launch_ns = launch_ns;
  o.done_ns = done_ns;
  return o;
}

// Plan and launch one batch into arena `ai`.  Requests that do not fit go back to the head of
// the queue; a single request that does not fit an empty arena is answered TOO_LARGE.
void launch_round(parem_server* s, int ai, std::vector<Req>& take, std::unique_lock<std::mutex>& lk) {
  NvtxRange range("parem_server launch");
  Arena& A = s->arenas[ai];
  for (;;) {
    std::vector<parem_batch_item> items(take.size());
    std::vector<uint64_t> seg(take.size());
    for (size_t i = 0; i < take.size(); ++i) {
      const parem_request& r = take[i].r;
      items[i].dfa = s->dfas[r.dfa_index];
      items[i].text = r.text;
      items[i].len = r.len;
      items[i].positions = r.positions;
      items[i].capacity = r.capacity;
      seg[i] = batch_default_segment(items[i].dfa);
    }
    parem_batch* b = nullptr;
    int rc = batch_create_in(items.data(), (uint32_t)items.size(), seg, &A.a, &b);
    if (rc == PAREM_ERR_TOO_LARGE && take.size() > 1) {
      const size_t keep = take.size() / 2;
      lk.lock();
      for (size_t i = take.size(); i-- > keep;) s->pending.push_front(take[i]);
      lk.unlock();
      take.resize(keep);
      continue;
    }
    const int64_t t = now_ns();
    if (rc == PAREM_OK) rc = batch_enqueue(b, A.a.stream);
    if (rc == PAREM_OK && cudaEventRecord(A.done, A.a.stream) != cudaSuccess) rc = PAREM_ERR_CUDA;
    if (rc != PAREM_OK) {
      if (b) {
        cudaStreamSynchronize(A.a.stream);
        batch_release(b);
      }
      parem_result none;
      std::memset(&none, 0, sizeof(none));
      std::vector<parem_response> resp;
      for (const Req& q : take) resp.push_back(make_response(q, rc, (uint32_t)take.size(), none, t, now_ns()));
      lk.lock();
      deliver(s, take, resp);
      s->free_arenas.push_back(ai);
      return;
    }
    Round round;
    round.arena = ai;
    round.batch = b;
    round.reqs = std::move(take);
    round.launch_ns = t;
    round.answered.assign(batch_size(b), 0);
    const uint32_t nk = batch_kernels(b);
    lk.lock();
    s->stats.batches++;
    s->stats.kernels += nk;
    s->stats.max_batch = std::max<uint64_t>(s->stats.max_batch, round.reqs.size());
    s->inflight.push_back(std::move(round));
    s->cv_done.notify_one();
    return;
  }
}

void dispatch_batches(parem_server* s) {
  cudaSetDevice(s->device);
  const uint32_t max_items = s->opts.max_items ? s->opts.max_items : 4096;
  const uint64_t max_bytes = s->opts.max_batch_bytes ? s->opts.max_batch_bytes : (1ull << 30);
  std::unique_lock<std::mutex> lk(s->mu);
  for (;;) {
    s->cv_dispatch.wait(lk, [&] { return s->stop || (!s->pending.empty() && !s->free_arenas.empty()); });
    if (s->pending.empty() || s->free_arenas.empty()) {
      if (s->stop) break;
      continue;
    }
    const int ai = s->free_arenas.back();
    s->free_arenas.pop_back();
    std::vector<Req> take;
    uint64_t bytes = 0;
    while (!s->pending.empty() && take.size() < max_items) {
      const Req& q = s->pending.front();
      if (!take.empty() && bytes + q.r.len > max_bytes) break;
      bytes += q.r.len;
      take.push_back(q);
      s->pending.pop_front();
    }
    lk.unlock();
    launch_round(s, ai, take, lk);  // returns with the lock held
  }
  s->dispatcher_done = true;
  s->cv_done.notify_all();
}

void dispatch_fifo(parem_server* s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  for (;;) {
    s->cv_dispatch.wait(lk, [&] { return s->stop || !s->pending.empty(); });
    if (s->pending.empty()) {
      if (s->stop) break;
      continue;
    }
    Req q = s->pending.front();
    s->pending.pop_front();
    lk.unlock();
    parem_result res;
    const int64_t t = now_ns();
    const int rc = parem_match(s->dfas[q.r.dfa_index], q.r.text, q.r.len, q.r.positions, q.r.capacity,
                               s->fifo_stream, &res);
    if (rc != PAREM_OK && rc != PAREM_ERR_CAPACITY) std::memset(&res, 0, sizeof(res));
    std::vector<parem_response> resp{make_response(q, rc, 1, res, t, now_ns())};
    std::vector<Req> one{q};
    parem_stats ps;
    const uint32_t nk = parem_last_stats(s->fifo_stream, &ps) == PAREM_OK ? ps.kernels : 0u;
    lk.lock();
    s->stats.batches++;
    s->stats.kernels += nk;
    s->stats.max_batch = std::max<uint64_t>(s->stats.max_batch, 1);
    deliver(s, one, resp);
  }
  s->dispatcher_done = true;
}

void complete_batches(parem_server* s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  for (;;) {
    s->cv_done.wait(lk, [&] { return s->dispatcher_done || !s->inflight.empty(); });
    if (s->inflight.empty()) break;  // the dispatcher has stopped and nothing is left
    // Rounds finish out of launch order (a batch holding one long request runs for long
    // after later, short batches are done): answer whichever round has finished, so that
    // short requests are not held behind a long one and its arena is free again at once.
    size_t ready = s->inflight.size();
    for (size_t k = 0; k < s->inflight.size(); ++k) {
      const cudaError_t q = cudaEventQuery(s->arenas[s->inflight[k].arena].done);
      if (q != cudaErrorNotReady) {
        ready = k;
        break;
      }
    }
    // requests whose results their kernels have already published (count-only requests):
    // answered now, before the rest of their batch
    bool early = false;
    if (ready == s->inflight.size()) {
      const int64_t t = now_ns();
      for (Round& r : s->inflight) {
        if (r.n_answered == r.answered.size()) continue;
        std::vector<Req> reqs;
        std::vector<parem_response> resp;
        const uint32_t n = batch_size(r.batch);
        for (uint32_t k = 0; k < n; ++k) {
          if (r.answered[k]) continue;
          parem_result res;
          if (!batch_early_result(r.batch, k, &res)) continue;
          const uint32_t i = batch_order(r.batch, k);
          r.answered[k] = 1;
          r.n_answered++;
          reqs.push_back(r.reqs[i]);
          resp.push_back(make_response(r.reqs[i], PAREM_OK, n, res, r.launch_ns, t));
        }
        if (!reqs.empty()) {
          deliver(s, reqs, resp);
          early = true;
        }
      }
    }
    if (early) continue;
    if (ready == s->inflight.size()) {
      // nothing finished: poll again shortly (early results arrive while batches run)
      lk.unlock();
      std::this_thread::sleep_for(std::chrono::microseconds(20));
      lk.lock();
      continue;
    }
    Round r = std::move(s->inflight[ready]);
    s->inflight.erase(s->inflight.begin() + (std::ptrdiff_t)ready);
    const int ai = r.arena;
    parem_batch* b = r.batch;
    const int64_t launch = r.launch_ns;
    lk.unlock();
    const bool ok = cudaEventSynchronize(s->arenas[ai].done) == cudaSuccess;
    const int64_t t = now_ns();
    const uint32_t n = batch_size(b);
    std::vector<Req> reqs;
    std::vector<parem_response> resp;
    for (uint32_t k = 0; k < n; ++k) {
      const uint32_t i = batch_order(b, k);
      parem_result res;
      // the final result also teaches the DFA's convergence hints, answered early or not
      int rc = ok ? batch_sorted_result(b, k, &res) : PAREM_ERR_CUDA;
      if (r.answered[k]) continue;
      if (rc != PAREM_OK && rc != PAREM_ERR_CAPACITY) std::memset(&res, 0, sizeof(res));
      reqs.push_back(r.reqs[i]);
      resp.push_back(make_response(r.reqs[i], rc, n, res, launch, t));
    }
    batch_release(b);
    lk.lock();
    s->free_arenas.push_back(ai);
    deliver(s, reqs, resp);
    s->cv_dispatch.notify_one();
  }
}

void destroy(parem_server* s) {
  for (Arena& A : s->arenas) {
    if (A.done) cudaEventDestroy(A.done);
    if (A.a.stream) cudaStreamDestroy(A.a.stream);
    if (A.a.scratch) cudaFree(A.a.scratch);
    if (A.a.desc) cudaFree(A.a.desc);
    if (A.a.host_desc) cudaFreeHost(A.a.host_desc);
    if (A.a.host_res) cudaFreeHost(A.a.host_res);
    if (A.a.host_early) cudaFreeHost(A.a.host_early);
  }
  if (s->fifo_stream) cudaStreamDestroy(s->fifo_stream);
  delete s;
}

bool valid(const parem_server* s, const parem_request* reqs, uint32_t n) {
  if (n && !reqs) return false;
  for (uint32_t i = 0; i < n; ++i) {
    const parem_request& r = reqs[i];
    if (r.dfa_index >= s->dfas.size() || (r.len && !r.text) || r.len > kMaxText) return false;
  }
  return true;
}

// Queue requests.  For a replay sink, request i gets tag first + i (its index in the trace)
// and the given arrival time.
void submit_internal(parem_server* s, const parem_request* reqs, uint32_t n, ReplaySink* sink, uint32_t first,
                     const int64_t* arrival) {
  const int64_t t = now_ns();
  std::lock_guard<std::mutex> g(s->mu);
  for (uint32_t i = 0; i < n; ++i) {
    Req q;
    q.r = reqs[i];
    q.sink = sink;
    if (sink) q.r.tag = first + i;
    if (arrival) q.r.arrival_ns = arrival[i];
    else if (q.r.arrival_ns == 0) q.r.arrival_ns = t;
    s->pending.push_back(q);
    s->stats.bytes += q.r.len;
  }
  s->stats.submitted += n;
  s->cv_dispatch.notify_one();
}

}  // namespace

extern "C" int64_t parem_clock_ns(void) { return now_ns(); }

extern "C" int parem_server_create(parem_dfa* const* dfas, uint32_t n_dfas, const parem_server_opts* opts,
                                   parem_server** out) {
  if (!out) return PAREM_ERR_INVALID_ARG;
  *out = nullptr;
  if (!dfas || n_dfas == 0) return PAREM_ERR_INVALID_ARG;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return PAREM_ERR_CUDA;
  for (uint32_t i = 0; i < n_dfas; ++i)
    if (!dfas[i] || dfas[i]->device != dev) return PAREM_ERR_INVALID_ARG;
  if (opts && opts->mode > PAREM_SERVE_FIFO) return PAREM_ERR_INVALID_ARG;
  parem_server* s = new (std::nothrow) parem_server();
  if (!s) return PAREM_ERR_OOM;
  s->device = dev;
  s->dfas.assign(dfas, dfas + n_dfas);
  if (opts) s->opts = *opts;
  const bool fifo = s->opts.mode == PAREM_SERVE_FIFO;
  if (fifo) {
    if (cudaStreamCreateWithFlags(&s->fifo_stream, cudaStreamNonBlocking) != cudaSuccess) {
      destroy(s);
      return PAREM_ERR_CUDA;
    }
  } else {
    for (parem_dfa* d : s->dfas) {
      const int rc = batch_prepare_dfa(d);
      if (rc != PAREM_OK) {
        destroy(s);
        return rc;
      }
    }
    const uint32_t n_arenas = s->opts.arenas ? s->opts.arenas : 256;
    const uint32_t max_items = s->opts.max_items ? s->opts.max_items : 4096;
    const uint64_t scratch = s->opts.arena_scratch_bytes ? s->opts.arena_scratch_bytes : (128ull << 20);
    // descriptors: per item its scan parameters and tensor map, per slot its record, the CTA
    // assignment and the emit block lists
    const uint64_t desc = (uint64_t)max_items * (sizeof(BatchItem) + 64) + (scratch / 64) + (1u << 20);
    s->arenas.resize(n_arenas);
    for (uint32_t i = 0; i < n_arenas; ++i) {
      Arena& A = s->arenas[i];
      A.a.scratch_cap = scratch;
      A.a.desc_cap = desc;
      A.a.res_cap = max_items;
      bool ok = cudaMalloc(&A.a.scratch, scratch) == cudaSuccess &&
                cudaMalloc(&A.a.desc, desc) == cudaSuccess &&
                cudaMallocHost(&A.a.host_desc, desc) == cudaSuccess &&
                cudaMallocHost(&A.a.host_res, sizeof(DevResult) * max_items) == cudaSuccess &&
                cudaHostAlloc(&A.a.host_early, sizeof(EarlyResult) * max_items, cudaHostAllocMapped) == cudaSuccess &&
                cudaHostGetDevicePointer(reinterpret_cast<void**>(&A.a.dev_early), A.a.host_early, 0) == cudaSuccess;
      if (!ok) {
        destroy(s);
        return PAREM_ERR_OOM;
      }
      if (cudaStreamCreateWithFlags(&A.a.stream, cudaStreamNonBlocking) != cudaSuccess ||
          cudaEventCreateWithFlags(&A.done, cudaEventDisableTiming) != cudaSuccess) {
        destroy(s);
        return PAREM_ERR_CUDA;
      }
      s->free_arenas.push_back((int)(n_arenas - 1 - i));
    }
  }
  try {
    if (fifo) {
      s->dispatcher = std::thread(dispatch_fifo, s);
    } else {
      s->dispatcher = std::thread(dispatch_batches, s);
      s->completer = std::thread(complete_batches, s);
    }
  } catch (...) {
    {
      std::lock_guard<std::mutex> g(s->mu);
      s->stop = true;
      s->dispatcher_done = true;
    }
    s->cv_dispatch.notify_all();
    s->cv_done.notify_all();
    if (s->dispatcher.joinable()) s->dispatcher.join();
    if (s->completer.joinable()) s->completer.join();
    destroy(s);
    return PAREM_ERR_OOM;
  }
  *out = s;
  return PAREM_OK;
}

extern "C" int parem_server_submit(parem_server* srv, const parem_request* reqs, uint32_t n) {
  if (!srv || !valid(srv, reqs, n)) return PAREM_ERR_INVALID_ARG;
  submit_internal(srv, reqs, n, nullptr, 0, nullptr);
  return PAREM_OK;
}

extern "C" int parem_server_poll(parem_server* srv, parem_response* out, uint32_t max, uint32_t* n_out,
                                 int64_t wait_ns) {
  if (!srv || !n_out || (max && !out)) return PAREM_ERR_INVALID_ARG;
  *n_out = 0;
  std::unique_lock<std::mutex> lk(srv->mu);
  if (srv->completed.empty() && wait_ns > 0)
    srv->cv_answer.wait_for(lk, std::chrono::nanoseconds(wait_ns), [&] { return !srv->completed.empty(); });
  uint32_t k = 0;
  while (k < max && !srv->completed.empty()) {
    out[k++] = srv->completed.front();
    srv->completed.pop_front();
  }
  *n_out = k;
  return PAREM_OK;
}

extern "C" int parem_server_drain(parem_server* srv) {
  if (!srv) return PAREM_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(srv->mu);
  srv->cv_answer.wait(lk, [&] { return srv->stats.answered == srv->stats.submitted; });
  return PAREM_OK;
}

extern "C" int parem_server_replay(parem_server* srv, const parem_request* reqs, uint32_t n, parem_response* out) {
  if (!srv || (n && !out) || !valid(srv, reqs, n)) return PAREM_ERR_INVALID_ARG;
  for (uint32_t i = 1; i < n; ++i)
    if (reqs[i].arrival_ns < reqs[i - 1].arrival_ns) return PAREM_ERR_INVALID_ARG;
  if (n == 0) return PAREM_OK;
  ReplaySink sink;
  sink.out = out;
  sink.n = n;
  const int64_t t0 = now_ns();
  // feeder: submits every request whose arrival time has come, sleeping while the next one is
  // far away and spinning when it is close
  std::thread feeder([&] {
    std::vector<int64_t> when;
    uint32_t i = 0;
    while (i < n) {
      int64_t t = now_ns();
      const int64_t next = t0 + reqs[i].arrival_ns;
      if (next > t + 200000) {
        std::this_thread::sleep_for(std::chrono::nanoseconds(next - t - 100000));
        continue;
      }
      if (next > t) continue;
      uint32_t j = i;
      when.clear();
      while (j < n && t0 + reqs[j].arrival_ns <= t) {
        when.push_back(t0 + reqs[j].arrival_ns);
        ++j;
      }
      submit_internal(srv, reqs + i, j - i, &sink, i, when.data());
      i = j;
    }
  });
  {
    std::unique_lock<std::mutex> lk(srv->mu);
    srv->cv_answer.wait(lk, [&] { return sink.done == sink.n; });
  }
  feeder.join();
  return PAREM_OK;
}

extern "C" int parem_server_get_stats(const parem_server* srv, parem_server_stats* out) {
  if (!srv || !out) return PAREM_ERR_INVALID_ARG;
  parem_server* s = const_cast<parem_server*>(srv);
  std::lock_guard<std::mutex> g(s->mu);
  *out = s->stats;
  return PAREM_OK;
}

extern "C" void parem_server_free(parem_server* srv) {
  if (!srv) return;
  parem_server_drain(srv);
  {
    std::lock_guard<std::mutex> g(srv->mu);
    srv->stop = true;
  }
  srv->cv_dispatch.notify_all();
  if (srv->dispatcher.joinable()) srv->dispatcher.join();
  {
    std::lock_guard<std::mutex> g(srv->mu);
    srv->dispatcher_done = true;
  }
  srv->cv_done.notify_all();
  if (srv->completer.joinable()) srv->completer.join();
  destroy(srv);
}
