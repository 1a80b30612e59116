// Request loop of the C ABI (ts_submit / ts_poll): continuous batching of
// state solves on one GPU.
//
// A user context owns a FIFO of requests and `slots` worker threads.  A worker
// takes the oldest queued request whose handle is idle (one request per handle
// at a time, in submission order: the handle holds that design's PCG state)
// and whose extra device memory fits, runs it on the handle's own streams and
// marks it finished.  Requests of other handles run at the same time on other
// workers, so their kernels overlap on the device, and a request that arrives
// while others run is admitted as soon as a slot and the memory it needs are
// free.  A request may carry new densities (one optimisation step, Eq. 4 with
// the next design): the design is then rebuilt before the solve, which needs a
// second copy of the handle's buffers while the new one is built.
#include <chrono>
#include <condition_variable>
#include <deque>
#include <memory>
#include <thread>
#include <unordered_map>
#include <unordered_set>

#include "ts_internal.cuh"

namespace {

struct Request {
  ts_ticket id = 0;
  ts_handle h = nullptr;
  const double* rho = nullptr;  // new densities, or nullptr
  const double* f = nullptr;
  double* u = nullptr;
  int nrhs = 1;
  double rtol = 1e-8;
  int64_t need = 0;             // extra device bytes while it runs (a rebuild)
  cudaEvent_t ready = nullptr;  // recorded on the caller's stream at submission
  bool finished = false;
  ts_status st = TS_PENDING;
  std::string err;
  std::vector<ts_stats> stats;
};

// device memory kept free beside the requests' own needs
constexpr int64_t kMemMargin = 256ll << 20;

}  // namespace

struct Server {
  ts_ctx ctx = nullptr;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<std::shared_ptr<Request>> queue;                    // waiting, FIFO
  std::unordered_map<ts_ticket, std::shared_ptr<Request>> reqs;  // not yet polled
  std::unordered_map<ts_handle, int> held;                       // queued + running, per handle
  std::unordered_set<ts_handle> busy;                            // running
  int64_t reserved = 0;                                          // bytes of running rebuilds
  std::vector<std::thread> workers;
  bool stop = false;
  ts_ticket next = 1;
};

namespace {

std::mutex g_server_create_mu;

// The oldest admissible queued request (caller holds S->mu): its handle is
// idle, no earlier request of the same handle waits, and its extra memory
// fits in what is free (or nothing else runs, so waiting cannot help).
std::deque<std::shared_ptr<Request>>::iterator pick(Server* S) {
  std::unordered_set<ts_handle> seen;
  size_t fr = 0, tot = 0;
  bool mem_known = false;
  for (auto it = S->queue.begin(); it != S->queue.end(); ++it) {
    Request& r = **it;
    if (S->busy.count(r.h) || seen.count(r.h)) {
      seen.insert(r.h);
      continue;
    }
    if (r.need > 0 && !S->busy.empty()) {
      if (!mem_known) {
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
          cudaGetLastError();
          fr = 0;
        }
        fr += (size_t)ts_scratch_pool_idle(S->ctx->device);  // held by the scratch pool, reusable
        mem_known = true;
      }
      if ((int64_t)fr - S->reserved - kMemMargin < r.need) {
        seen.insert(r.h);
        continue;
      }
    }
    return it;
  }
  return S->queue.end();
}

void worker_main(Server* S) {
  cudaSetDevice(S->ctx->device);
  std::unique_lock<std::mutex> lk(S->mu);
  for (;;) {
    auto it = pick(S);
    if (it == S->queue.end()) {
      if (S->stop) return;
      // woken by a submission or a finished request; the timeout re-checks
      // device memory freed outside the loop
      S->cv.wait_for(lk, std::chrono::milliseconds(20));
      continue;
    }
    std::shared_ptr<Request> r = *it;
    S->queue.erase(it);
    S->busy.insert(r->h);
    S->reserved += r->need;
    lk.unlock();
    ts_status st = TS_OK;
    std::string err;
    try {
      if (r->rho) {
        TS_CUDA(cudaStreamWaitEvent(r->h->ctx->stream, r->ready, 0));
        ts_update_by_policy(r->h, r->rho);
      }
      st = ts_solve_impl(r->h, r->f, r->u, r->nrhs, r->rtol, r->stats.data(), r->ready);
      if (st != TS_OK) {
        std::lock_guard<std::mutex> g(r->h->ctx->err_mu);
        err = r->h->ctx->err;
      }
    } catch (const TsError& e) {
      st = e.st;
      err = e.msg;
    } catch (const std::exception& e) {
      st = TS_ERR_INVALID;
      err = e.what();
    }
    lk.lock();
    r->st = st;
    r->err = err;
    r->finished = true;
    S->busy.erase(r->h);
    S->reserved -= r->need;
    if (--S->held[r->h] == 0) S->held.erase(r->h);
    S->cv.notify_all();
  }
}

Server* ensure_server(ts_ctx ctx) {
  std::lock_guard<std::mutex> g(g_server_create_mu);
  if (ctx->server) return ctx->server;
  Server* S = new Server();
  S->ctx = ctx;
  for (int i = 0; i < ctx->slots; ++i) S->workers.emplace_back(worker_main, S);
  ctx->server = S;
  return S;
}

ts_status submit(ts_ctx ctx, ts_handle h, const double* rho, const double* f, double* u, int nrhs, double rtol,
                 ts_ticket* ticket) {
  if (!ctx || ctx->parent) return TS_ERR_INVALID;
  if (!h || h->root != ctx || !f || !u || !ticket || nrhs < 1 || !(rtol > 0.0)) {
    ts_set_error(ctx, "ts_submit: bad arguments (the handle must come from this context)");
    return TS_ERR_INVALID;
  }
  auto r = std::make_shared<Request>();
  r->h = h;
  r->rho = rho;
  r->f = f;
  r->u = u;
  r->nrhs = nrhs;
  r->rtol = rtol;
  r->stats.resize(nrhs);
  if (rho) {
    r->need = h->bytes + h->scratch_peak;  // the new design beside the old, and its setup scratch
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
      cudaGetLastError();
      ts_set_error(ctx, "ts_submit: cudaMemGetInfo failed");
      return TS_ERR_CUDA;
    }
    if (r->need + kMemMargin > (int64_t)tot) {
      ts_set_error(ctx, "ts_submit: the rebuild needs more than the device's memory");
      return TS_ERR_BUSY;
    }
  }
  cudaError_t e = cudaEventCreateWithFlags(&r->ready, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventRecord(r->ready, ctx->user_stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    if (r->ready) cudaEventDestroy(r->ready);
    ts_set_error(ctx, std::string("ts_submit: ") + cudaGetErrorString(e));
    return TS_ERR_CUDA;
  }
  Server* S = ensure_server(ctx);
  std::lock_guard<std::mutex> lk(S->mu);
  if (S->stop) {
    cudaEventDestroy(r->ready);
    return TS_ERR_INVALID;
  }
  r->id = S->next++;
  S->queue.push_back(r);
  S->reqs[r->id] = r;
  S->held[h]++;
  *ticket = r->id;
  S->cv.notify_all();
  return TS_OK;
}

}  // namespace

void stop_server(ts_ctx ctx) {
  if (!ctx || !ctx->server) return;
  Server* S = ctx->server;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
    for (auto& r : S->queue) {
      r->finished = true;
      r->st = TS_ERR_INVALID;
      r->err = "context destroyed before the request ran";
    }
    S->queue.clear();
    S->cv.notify_all();
  }
  for (auto& t : S->workers) t.join();
  for (auto& kv : S->reqs)
    if (kv.second->ready) cudaEventDestroy(kv.second->ready);
  ctx->server = nullptr;
  delete S;
}

bool server_holds(ts_ctx ctx, ts_handle h) {
  if (!ctx || !ctx->server) return false;
  std::lock_guard<std::mutex> lk(ctx->server->mu);
  return ctx->server->held.count(h) != 0;
}

extern "C" {

ts_status ts_ctx_set_slots(ts_ctx ctx, int slots) {
  if (!ctx || ctx->parent || slots < 1 || slots > 64) return TS_ERR_INVALID;
  std::lock_guard<std::mutex> g(g_server_create_mu);
  if (ctx->server) {
    ts_set_error(ctx, "ts_ctx_set_slots: the request loop is already running");
    return TS_ERR_BUSY;
  }
  ctx->slots = slots;
  return TS_OK;
}

ts_status ts_submit(ts_ctx ctx, ts_handle h, const double* f, double* u, int nrhs, double rtol, ts_ticket* ticket) {
  return submit(ctx, h, nullptr, f, u, nrhs, rtol, ticket);
}

ts_status ts_submit_update(ts_ctx ctx, ts_handle h, const double* rho, const double* f, double* u, int nrhs,
                           double rtol, ts_ticket* ticket) {
  if (!rho) return TS_ERR_INVALID;
  return submit(ctx, h, rho, f, u, nrhs, rtol, ticket);
}

ts_status ts_poll(ts_ctx ctx, ts_ticket ticket, ts_stats* stats) {
  if (!ctx || ctx->parent || !ctx->server) return TS_ERR_INVALID;
  Server* S = ctx->server;
  std::shared_ptr<Request> r;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return TS_ERR_INVALID;
    if (!it->second->finished) return TS_PENDING;
    r = it->second;
    S->reqs.erase(it);
  }
  if (stats)
    for (int k = 0; k < r->nrhs; ++k) stats[k] = r->stats[k];
  if (!r->err.empty()) ts_set_error(ctx, r->err);
  cudaEventDestroy(r->ready);
  return r->st;
}

}  // extern "C"
