// Serving loop: many independent interior eigenproblems on one GPU, with
// continuous batching.
//
// Requests (a Hermitian matrix in host CSR plus solver parameters) are queued
// in arrival order.  One engine thread runs every admitted request's Alg. 4
// and batches their filter steps: each launch of the batched Clenshaw step
// (spmm_multi.cuh) carries the next step (Alg. 2) of every request that is in
// the filter phase of its current outer iteration, real and complex problems
// in one launch each.  A request whose recurrence ends queues its
// orthogonalisation, Rayleigh-Ritz and residual steps on its own CUDA stream
// (they overlap with the batched launches and with the other requests' dense
// work) and rejoins the launches with its next iteration as soon as its
// checks are done, so no request waits for another's iteration.  The head of
// the queue is admitted between launches when a slot is free and its
// estimated device footprint fits in what the running solves leave of the HBM
// budget (or when nothing runs).  Each request's state (subspace, locked
// vectors, filter buffers) stays on the device from admission to completion.
// The arithmetic of a request does not depend on the other requests, so its
// result is the same alone and in a mix (and the same as apf_solve's).
//
// The result of a request owns that request's context; apf_result_destroy
// releases both.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "engine.h"
#include "solver.h"

namespace {
using Clock = std::chrono::steady_clock;

struct Request {
  int64_t ticket = 0;
  int64_t n = 0, nnz = 0;
  int32_t dtype = APF_R64;
  std::vector<int64_t> rowptr;
  std::vector<int32_t> colidx;
  std::vector<unsigned char> vals;
  apf_params prm{};
  int64_t footprint = 0;
  Clock::time_point t_submit, t_start, t_end;
  int32_t worker = -1;
  apf_status status = APF_OK;
  apf_result* result = nullptr;
  bool done = false;
  bool claimed = false;  // a thread waits for it (a ticket can be waited for once)
};

// An admitted request: its context (own stream), matrix and solve, and where
// it stands in its current outer iteration.
struct Active {
  enum Phase { kFilter, kDense };
  Request* r = nullptr;
  apf_ctx* ctx = nullptr;
  apf_matrix* A = nullptr;
  std::unique_ptr<apf::EngineSolve> solve;
  Phase phase = kDense;
  int next_step = -1;             // next Clenshaw step (kFilter), counting down to 0
  cudaEvent_t ready = nullptr;    // the request's filter inputs are on its stream
  cudaEvent_t dense = nullptr;    // its orthogonalisation / Rayleigh-Ritz are done
  apf_status fail = APF_OK;
};

double ms_between(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}
}  // namespace

struct apf_server {
  int device = 0;
  int64_t budget = 0;
  std::mutex mu;
  std::condition_variable cv_queue, cv_done;
  std::deque<Request*> queue;
  std::map<int64_t, std::unique_ptr<Request>> reqs;
  int64_t next_ticket = 1;
  int64_t in_flight = 0;  // footprint of the running requests
  int32_t running = 0;
  int32_t peak_running = 0;
  int64_t peak_in_flight = 0;
  int64_t completed = 0;
  int32_t max_active = 1;
  int64_t batched_launches = 0;  // batched Clenshaw-step launches
  int32_t widest_batch = 0;      // most requests in one of them
  bool stop = false;
  std::thread engine;
  // set-up of admitted requests runs on threads of its own; the engine
  // thread picks the requests up when they are ready
  std::vector<std::thread> setups;
  std::vector<std::unique_ptr<Active>> ready;
  int32_t pending_setup = 0;
};

namespace {

// Device bytes of one solve, estimated from the sizes: the matrix in CSR
// (FP64 values), its FP32 scaled copy and SELL-8 copies (padding allowance
// included), five n x p blocks of the subspace state, three FP32 recurrence
// blocks, the result and its residual check, the bf16 slices of two operands
// of a tensor-core Gram product when those are on (7 slices per real part),
// and 64 MiB of small buffers.  p = 0 (estimated size) counts as min(n, 256).
int64_t footprint(int64_t n, int64_t nnz, int32_t dtype, int64_t p, bool gram_tc) {
  const int64_t s = dtype == APF_C128 ? 16 : 8, sl = s / 2;
  const int64_t parts = dtype == APF_C128 ? 2 : 1;
  const int64_t pp = p > 0 ? p : std::min<int64_t>(n, 256);
  const int64_t ld = apf::round_up(pp, 8);
  const int64_t mat = nnz * (s + 4) + (n + 1) * 8 + 4 * nnz * (sl + 8);
  const int64_t blocks = 8 * n * ld * s + 3 * n * ld * sl;
  const int64_t slices = gram_tc ? 2 * 7 * parts * apf::round_up(n, 64) * apf::round_up(pp, 32) * 2 : 0;
  return mat + blocks + slices + (64ll << 20);
}

bool admissible(const apf_server* s, const Request* r) {
  return s->running == 0 || s->in_flight + r->footprint <= s->budget;
}

void release_host_copies(Request* r) {
  std::vector<int64_t>().swap(r->rowptr);
  std::vector<int32_t>().swap(r->colidx);
  std::vector<unsigned char>().swap(r->vals);
}

// Ends a request: its result (or its failure) goes to the waiter.
void finish(apf_server* s, Active& a, apf_status st, apf_result* res) {
  if (a.ready) cudaEventDestroy(a.ready);
  if (a.dense) cudaEventDestroy(a.dense);
  a.ready = a.dense = nullptr;
  if (a.A) apf_matrix_destroy(a.A);
  a.A = nullptr;
  a.solve.reset();
  if (res) {
    res->owns_ctx = true;
    a.r->result = res;
  } else if (a.ctx) {
    apf_destroy(a.ctx);
  }
  a.ctx = nullptr;
  a.r->status = st;
  release_host_copies(a.r);
  {
    std::lock_guard<std::mutex> lk(s->mu);
    a.r->t_end = Clock::now();
    s->in_flight -= a.r->footprint;
    s->running -= 1;
    s->completed += 1;
    a.r->done = true;
  }
  s->cv_done.notify_all();
}

template <class F>
apf_status guarded(F&& f) {
  try {
    f();
  } catch (const ApfError& e) {
    return e.status;
  } catch (...) {
    return APF_ERR_CUDA;
  }
  return APF_OK;
}

// Opens an outer iteration: the filter inputs on the request's stream; with
// batched steps to run, the engine stream will wait for them; without (FP64
// filter, no SELL copy, degree 0 or 1) the rest of the iteration is queued now.
void open_iteration(apf_ctx* ectx, Active& a) {
  a.fail = guarded([&] {
    a.solve->begin_iteration();
    if (a.solve->batched() && a.solve->steps() > 0) {
      APF_CUDA(cudaEventRecord(a.ready, a.ctx->stream));
      APF_CUDA(cudaStreamWaitEvent(ectx->stream, a.ready, 0));
      a.phase = Active::kFilter;
      a.next_step = a.solve->steps() - 1;
    } else {
      a.solve->end_iteration();
      APF_CUDA(cudaEventRecord(a.dense, a.ctx->stream));
      a.phase = Active::kDense;
    }
  });
}

// Set-up of an admitted request (ingest, bounds, coefficients, subspace size,
// initial block) on a thread of its own, so that the engine keeps launching
// the running requests' steps meanwhile; the request then waits in `ready`.
void setup_job(apf_server* s, Active* a) {
  cudaSetDevice(s->device);
  apf_status st = apf_create(&a->ctx, s->device, nullptr);
  if (st == APF_OK)
    st = apf_matrix_create_csr(a->ctx, a->r->n, a->r->nnz, a->r->rowptr.data(), a->r->colidx.data(),
                               a->r->vals.data(), a->r->dtype, 0, &a->A);
  if (st == APF_OK)
    st = guarded([&] {
      APF_CUDA(cudaEventCreateWithFlags(&a->ready, cudaEventDisableTiming));
      APF_CUDA(cudaEventCreateWithFlags(&a->dense, cudaEventDisableTiming));
      a->solve = apf::engine_start(a->ctx, a->A, &a->r->prm);
    });
  std::unique_ptr<Active> own(a);
  if (st != APF_OK) {
    finish(s, *a, st, nullptr);
    std::lock_guard<std::mutex> lk(s->mu);
    s->pending_setup -= 1;
  } else {
    std::lock_guard<std::mutex> lk(s->mu);
    s->ready.push_back(std::move(own));
    s->pending_setup -= 1;
  }
  s->cv_queue.notify_all();
}

// One batched launch per problem type: the next Clenshaw step of every request
// in its filter phase (at most kMaxBatch per launch).  A request whose
// recurrence ends with this launch queues the rest of its iteration on its own
// stream, after the launch.
void tick(apf_server* s, apf_ctx* ectx, std::vector<Active>& act, cudaEvent_t step_done) {
  int64_t launches = 0;
  int32_t widest = 0;
  for (int cplx = 0; cplx < 2; ++cplx) {
    apf::MultiArgs ma{};
    std::vector<size_t> members;
    auto launch = [&]() {
      const apf_status st = guarded([&] { apf::engine_step_launch(ectx, cplx == 1, ma); });
      if (st != APF_OK)
        for (size_t m : members) act[m].fail = st;
      launches += 1;
      widest = std::max(widest, (int32_t)ma.nreq);
      ma = apf::MultiArgs{};
      members.clear();
    };
    for (size_t i = 0; i < act.size(); ++i) {
      Active& a = act[i];
      if (a.fail != APF_OK || a.phase != Active::kFilter || a.solve->is_complex() != (cplx == 1)) continue;
      if (ma.nreq == apf::kMaxBatch) launch();
      a.solve->step_desc(a.next_step, &ma.d[ma.nreq++]);
      a.next_step -= 1;
      members.push_back(i);
    }
    if (ma.nreq) launch();
  }
  bool ended = false;
  for (auto& a : act) ended = ended || (a.fail == APF_OK && a.phase == Active::kFilter && a.next_step < 0);
  if (ended) {
    const apf_status st = guarded([&] { APF_CUDA(cudaEventRecord(step_done, ectx->stream)); });
    for (auto& a : act) {
      if (a.fail != APF_OK || a.phase != Active::kFilter || a.next_step >= 0) continue;
      a.fail = st != APF_OK ? st : guarded([&] {
        APF_CUDA(cudaStreamWaitEvent(a.ctx->stream, step_done, 0));
        a.solve->end_iteration();
        APF_CUDA(cudaEventRecord(a.dense, a.ctx->stream));
      });
      a.phase = Active::kDense;
    }
  }
  std::lock_guard<std::mutex> lk(s->mu);
  s->batched_launches += launches;
  s->widest_batch = std::max(s->widest_batch, widest);
}

// The engine: admission between steps, one batched launch per tick for the
// requests in their filter phase, and the requests whose dense work is done
// moved on to their next iteration (or finished).
void engine_main(apf_server* s) {
  cudaSetDevice(s->device);
  apf_ctx* ectx = nullptr;
  const apf_status est = apf_create(&ectx, s->device, nullptr);
  cudaEvent_t step_done = nullptr;
  if (est == APF_OK && cudaEventCreateWithFlags(&step_done, cudaEventDisableTiming) != cudaSuccess) step_done = nullptr;
  std::vector<Active> act;
  int32_t slot = 0;
  int64_t ticks = 0;
  for (;;) {
    std::vector<std::unique_ptr<Active>> picked;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      auto in_flight = [&] { return (int32_t)act.size() + s->pending_setup + (int32_t)s->ready.size(); };
      auto can_admit = [&] {
        return !s->queue.empty() && in_flight() < s->max_active && admissible(s, s->queue.front());
      };
      if (act.empty())
        s->cv_queue.wait(lk, [&] {
          return !s->ready.empty() || can_admit() || (s->stop && s->queue.empty() && s->pending_setup == 0);
        });
      while (can_admit() && est == APF_OK && step_done) {
        Request* r = s->queue.front();
        s->queue.pop_front();
        s->in_flight += r->footprint;
        s->running += 1;
        s->peak_running = std::max(s->peak_running, s->running);
        s->peak_in_flight = std::max(s->peak_in_flight, s->in_flight);
        r->worker = slot++;
        r->t_start = Clock::now();
        auto* a = new Active();
        a->r = r;
        s->pending_setup += 1;
        s->setups.emplace_back(setup_job, s, a);
      }
      picked.swap(s->ready);
      if (act.empty() && picked.empty() && s->pending_setup == 0 && s->stop && s->queue.empty()) break;
      if (est != APF_OK || !step_done) {  // no engine: fail what is queued
        while (!s->queue.empty()) {
          Request* r = s->queue.front();
          s->queue.pop_front();
          s->in_flight += r->footprint;
          s->running += 1;
          Active a;
          a.r = r;
          lk.unlock();
          finish(s, a, est != APF_OK ? est : APF_ERR_CUDA, nullptr);
          lk.lock();
        }
      }
    }
    for (auto& p : picked) {
      open_iteration(ectx, *p);
      act.push_back(std::move(*p));
    }
    if (act.empty()) continue;
    // a few batched steps between looks at the dense phases
    bool filtering = false;
    for (int t = 0; t < 8; ++t) {
      filtering = false;
      for (auto& a : act) filtering = filtering || (a.fail == APF_OK && a.phase == Active::kFilter);
      if (!filtering) break;
      tick(s, ectx, act, step_done);
      ++ticks;
    }
    // a kernel of the batched launches that gave up on a wait fails the requests it served
    if (!filtering || ticks % 256 == 0) {
      int derr = 0;
      const apf_status st = guarded([&] { derr = apf::fetch_device_error(ectx); });
      if (st != APF_OK || derr != 0)
        for (auto& a : act)
          if (a.fail == APF_OK) a.fail = st != APF_OK ? st : APF_ERR_TIMEOUT;
    }
    bool progressed = false;
    for (auto& a : act) {
      if (a.fail != APF_OK || a.phase != Active::kDense) continue;
      const cudaError_t q = cudaEventQuery(a.dense);
      if (q == cudaErrorNotReady) continue;
      progressed = true;
      if (q != cudaSuccess) {
        cudaGetLastError();
        a.fail = APF_ERR_CUDA;
        continue;
      }
      a.fail = guarded([&] { a.solve->check(); });
      if (a.fail == APF_OK && !a.solve->finished()) open_iteration(ectx, a);
    }
    if (!filtering && !progressed) {  // nothing to launch: wait for a dense phase instead of spinning
      for (auto& a : act)
        if (a.fail == APF_OK && a.phase == Active::kDense) {
          cudaEventSynchronize(a.dense);
          break;
        }
    }
    std::vector<Active> keep;
    for (auto& a : act) {
      if (a.fail != APF_OK) {
        finish(s, a, a.fail, nullptr);
      } else if (a.phase == Active::kDense && a.solve->finished()) {
        apf_status st = APF_OK;
        apf_result* res = nullptr;
        const apf_status g = guarded([&] { res = a.solve->take_result(&st); });
        finish(s, a, g != APF_OK ? g : st, res);
      } else {
        keep.push_back(std::move(a));
      }
    }
    act.swap(keep);
  }
  for (auto& t : s->setups)
    if (t.joinable()) t.join();
  if (step_done) cudaEventDestroy(step_done);
  if (ectx) apf_destroy(ectx);
}
}  // namespace

extern "C" {

apf_status apf_server_create(apf_server** out, int32_t device, int32_t max_concurrent, int64_t hbm_budget_bytes) {
  if (!out || max_concurrent < 1 || max_concurrent > 64 || hbm_budget_bytes < 0) return APF_ERR_ARG;
  // active requests of one batch: up to kMaxBatch descriptors per launch and type
  if (max_concurrent > 2 * apf::kMaxBatch) max_concurrent = 2 * apf::kMaxBatch;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess) {
    cudaGetLastError();
    return APF_ERR_CUDA;
  }
  if (device < 0 || device >= ndev) return APF_ERR_ARG;
  int64_t budget = hbm_budget_bytes;
  if (budget == 0) {  // 90 % of what is free now
    size_t freeb = 0, total = 0;
    if (cudaSetDevice(device) != cudaSuccess || cudaMemGetInfo(&freeb, &total) != cudaSuccess) {
      cudaGetLastError();
      return APF_ERR_CUDA;
    }
    budget = (int64_t)(0.9 * (double)freeb);
  }
  apf_server* s = new apf_server();
  s->device = device;
  s->budget = budget;
  s->max_active = max_concurrent;
  try {
    s->engine = std::thread(engine_main, s);
  } catch (...) {
    delete s;
    return APF_ERR_OOM;
  }
  *out = s;
  return APF_OK;
}

apf_status apf_server_submit(apf_server* s, int64_t n, int64_t nnz, const int64_t* rowptr, const int32_t* colidx,
                             const void* vals, int32_t dtype, const apf_params* params, int64_t* ticket) {
  if (!s || !ticket || !params || n < 1 || nnz < 0 || !rowptr || (nnz > 0 && (!colidx || !vals))) return APF_ERR_ARG;
  if (dtype != APF_R64 && dtype != APF_C128) return APF_ERR_ARG;
  if (params->init_block != nullptr) return APF_ERR_ARG;  // caller buffers are not kept
  if (rowptr[0] != 0 || rowptr[n] != nnz) return APF_ERR_ARG;
  auto r = std::make_unique<Request>();
  r->n = n;
  r->nnz = nnz;
  r->dtype = dtype;
  r->prm = *params;
  r->footprint = footprint(n, nnz, dtype, params->p, params->gram_tensor_cores != 0);
  if (r->footprint > s->budget) return APF_ERR_OOM;
  const size_t vs = dtype == APF_C128 ? 16 : 8;
  r->rowptr.assign(rowptr, rowptr + n + 1);
  r->colidx.assign(colidx, colidx + nnz);
  r->vals.resize((size_t)nnz * vs);
  if (nnz) memcpy(r->vals.data(), vals, (size_t)nnz * vs);
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) return APF_ERR_ARG;
    r->ticket = s->next_ticket++;
    r->t_submit = Clock::now();
    *ticket = r->ticket;
    s->queue.push_back(r.get());
    s->reqs[r->ticket] = std::move(r);
  }
  s->cv_queue.notify_all();
  return APF_OK;
}

apf_status apf_server_wait(apf_server* s, int64_t ticket, apf_result** out, apf_request_info* info) {
  if (!s || !out) return APF_ERR_ARG;
  std::unique_ptr<Request> r;
  {
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return APF_ERR_ARG;
    Request* rp = it->second.get();
    if (rp->claimed) return APF_ERR_ARG;  // another thread already waits for it
    rp->claimed = true;
    s->cv_done.wait(lk, [&] { return rp->done; });
    // the entry stays in the map while claimed: look it up again after the wait
    it = s->reqs.find(ticket);
    r = std::move(it->second);
    s->reqs.erase(it);
  }
  *out = r->result;
  if (info) {
    info->status = r->status;
    info->worker = r->worker;
    info->queue_ms = ms_between(r->t_submit, r->t_start);
    info->run_ms = ms_between(r->t_start, r->t_end);
    info->latency_ms = ms_between(r->t_submit, r->t_end);
    info->footprint_bytes = r->footprint;
  }
  return r->status;
}

apf_status apf_server_state(apf_server* s, apf_server_info* out) {
  if (!s || !out) return APF_ERR_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  out->queued = (int32_t)s->queue.size();
  out->running = s->running;
  out->peak_running = s->peak_running;
  out->workers = s->max_active;
  out->in_flight_bytes = s->in_flight;
  out->peak_in_flight_bytes = s->peak_in_flight;
  out->budget_bytes = s->budget;
  out->completed = s->completed;
  out->batched_launches = s->batched_launches;
  out->widest_batch = s->widest_batch;
  return APF_OK;
}

apf_status apf_server_destroy(apf_server* s) {
  if (!s) return APF_OK;
  {
    std::unique_lock<std::mutex> lk(s->mu);
    s->cv_done.wait(lk, [&] { return s->queue.empty() && s->running == 0; });
    s->stop = true;
  }
  s->cv_queue.notify_all();
  if (s->engine.joinable()) s->engine.join();
  for (auto& kv : s->reqs)  // results nobody waited for
    if (kv.second->result) apf_result_destroy(kv.second->result);
  delete s;
  return APF_OK;
}

}  // extern "C"
