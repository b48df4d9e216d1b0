// Serving loop: many independent interior eigenproblems on one GPU.
//
// Requests (a Hermitian matrix in host CSR plus solver parameters) are queued
// in arrival order.  A fixed pool of worker threads takes them off the queue;
// the head of the queue is admitted when its estimated device footprint fits
// in what the running solves leave of the HBM budget (or when nothing runs).
// Each admitted request gets its own context, hence its own CUDA stream, so
// the Clenshaw steps and dense steps of the running solves interleave on the
// GPU.  The kernels' arithmetic does not depend on what else runs: a request
// returns the same result alone and in a mix.
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
  bool stop = false;
  std::vector<std::thread> workers;
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

void run_request(apf_server* s, Request* r) {
  apf_ctx* ctx = nullptr;
  apf_status st = apf_create(&ctx, s->device, nullptr);
  if (st != APF_OK) {
    r->status = st;
    return;
  }
  apf_matrix* A = nullptr;
  st = apf_matrix_create_csr(ctx, r->n, r->nnz, r->rowptr.data(), r->colidx.data(), r->vals.data(), r->dtype, 0, &A);
  apf_result* res = nullptr;
  if (st == APF_OK) {
    st = apf_solve(ctx, A, &r->prm, &res);
    apf_matrix_destroy(A);
  }
  cudaSetDevice(s->device);
  cudaStreamSynchronize(ctx->stream);
  if (res) {
    res->owns_ctx = true;
    r->result = res;
  } else {
    apf_destroy(ctx);
  }
  r->status = st;
  // the host copies are no longer needed
  std::vector<int64_t>().swap(r->rowptr);
  std::vector<int32_t>().swap(r->colidx);
  std::vector<unsigned char>().swap(r->vals);
}

void worker_main(apf_server* s, int32_t w) {
  cudaSetDevice(s->device);
  for (;;) {
    Request* r = nullptr;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv_queue.wait(lk, [&] { return s->stop || (!s->queue.empty() && admissible(s, s->queue.front())); });
      if (s->queue.empty() || !admissible(s, s->queue.front())) {
        if (s->stop) return;
        continue;
      }
      r = s->queue.front();
      s->queue.pop_front();
      s->in_flight += r->footprint;
      s->running += 1;
      s->peak_running = std::max(s->peak_running, s->running);
      s->peak_in_flight = std::max(s->peak_in_flight, s->in_flight);
      r->worker = w;
      r->t_start = Clock::now();
    }
    run_request(s, r);
    {
      std::lock_guard<std::mutex> lk(s->mu);
      r->t_end = Clock::now();
      s->in_flight -= r->footprint;
      s->running -= 1;
      s->completed += 1;
      r->done = true;
    }
    s->cv_done.notify_all();
    s->cv_queue.notify_all();
  }
}

}  // namespace

extern "C" {

apf_status apf_server_create(apf_server** out, int32_t device, int32_t max_concurrent, int64_t hbm_budget_bytes) {
  if (!out || max_concurrent < 1 || max_concurrent > 64 || hbm_budget_bytes < 0) return APF_ERR_ARG;
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
  try {
    for (int32_t w = 0; w < max_concurrent; ++w) s->workers.emplace_back(worker_main, s, w);
  } catch (...) {
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->stop = true;
    }
    s->cv_queue.notify_all();
    for (auto& t : s->workers) t.join();
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
  out->workers = (int32_t)s->workers.size();
  out->in_flight_bytes = s->in_flight;
  out->peak_in_flight_bytes = s->peak_in_flight;
  out->budget_bytes = s->budget;
  out->completed = s->completed;
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
  for (auto& t : s->workers) t.join();
  for (auto& kv : s->reqs)  // results nobody waited for
    if (kv.second->result) apf_result_destroy(kv.second->result);
  delete s;
  return APF_OK;
}

}  // extern "C"
