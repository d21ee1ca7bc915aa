// Serving loop: continuous batching of applies on resident operators (the paper has
// no counterpart).  A worker thread owns the CUDA work; mbf_submit / mbf_poll only
// touch the queue under the server's mutex.
//
// Per batch: the oldest queued request whose operator is idle, plus the queued
// requests on the same operator in FIFO order up to max_batch_rhs RHS.  One request
// runs in place; several are gathered into a staging panel (device-to-device copies),
// applied once, and scattered back.  With use_graphs the batch's copies and kernels
// are captured into one CUDA graph; an executable graph is kept per batch shape
// (operator, request RHS counts, SM share) and updated in place for new buffers.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <set>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "op_internal.hpp"

namespace {

using mbf::Error;
using mbf::fail;

void cuda_ok(cudaError_t e, const char* what) {
  if (e != cudaSuccess) fail(MBF_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

struct Request {
  mbf_op_s* op = nullptr;
  const void* g = nullptr;
  void* u = nullptr;
  int64_t nrhs = 0;
  int64_t reserved = 0;   // staging bytes held until completion
  mbf_request_status_t st{};
};

struct Batch {
  int slot = -1;
  mbf_op_s* op = nullptr;
  std::vector<mbf_ticket_t> ids;
  int64_t rhs = 0;
  void* stage = nullptr;   // [rhs][n_in] then [rhs][n_out]
  cudaEvent_t done = nullptr;
};

struct GraphEntry {
  cudaGraphExec_t exec = nullptr;
  uint64_t last_use = 0;
};

}  // namespace

struct mbf_server_s {
  mbf_server_opts_t opts{};
  int device = 0, sms = 0;
  std::chrono::steady_clock::time_point t0;
  std::mutex mu;
  std::condition_variable cv_work, cv_idle;
  std::deque<mbf_ticket_t> queue;
  std::unordered_map<mbf_ticket_t, Request> reqs;
  mbf_ticket_t next_id = 1;
  int64_t reserved = 0;
  bool stop = false;
  std::vector<cudaStream_t> streams;
  std::vector<int*> status_host;   // pinned: copy of the operator's status word per slot
  std::vector<Batch> slots;        // slot i busy iff slots[i].op != nullptr
  std::set<mbf_op_s*> busy_ops;
  std::map<std::string, GraphEntry> graphs;
  uint64_t use_clock = 0;
  mbf_server_stats_t stats{};
  int64_t graph_launches = 0, graph_insts = 0;   // worker-only; copied into stats under the lock
  std::thread worker;

  double now() const {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  int inflight() const {
    int n = 0;
    for (const auto& b : slots) n += b.op != nullptr;
    return n;
  }

  // Copies, apply and scatter of one batch on stream st (captured or not).
  void enqueue_batch(const Batch& b, const std::vector<Request*>& rq, int grid, cudaStream_t st) {
    mbf_op_s* op = b.op;
    if (rq.size() == 1) {
      mbf::apply_dev(op, rq[0]->g, rq[0]->u, rq[0]->nrhs, MBF_PREC_AUTO, st, false, grid);
      return;
    }
    auto* in = static_cast<float2*>(b.stage);
    float2* out = in + b.rhs * op->n_in;
    int64_t r0 = 0;
    for (Request* r : rq) {
      cuda_ok(cudaMemcpyAsync(in + r0 * op->n_in, r->g, size_t(r->nrhs * op->n_in) * sizeof(float2),
                              cudaMemcpyDeviceToDevice, st),
              "gather copy");
      r0 += r->nrhs;
    }
    mbf::apply_dev(op, in, out, b.rhs, MBF_PREC_AUTO, st, false, grid);
    r0 = 0;
    for (Request* r : rq) {
      cuda_ok(cudaMemcpyAsync(r->u, out + r0 * op->n_out, size_t(r->nrhs * op->n_out) * sizeof(float2),
                              cudaMemcpyDeviceToDevice, st),
              "scatter copy");
      r0 += r->nrhs;
    }
  }

  // Launch a batch on its slot (worker thread, lock not held).
  void launch(Batch& b, const std::vector<Request*>& rq, int grid) {
    cudaStream_t st = streams[size_t(b.slot)];
    mbf_op_s* op = b.op;
    if (mbf::uses_tensor(op, b.rhs, MBF_PREC_AUTO, false)) mbf::tc_prepare(op);   // no allocation in capture
    if (rq.size() > 1)
      cuda_ok(cudaMallocAsync(&b.stage, size_t(b.rhs * (op->n_in + op->n_out)) * sizeof(float2), st),
              "staging allocation");
    if (opts.use_graphs) {
      std::string key = std::to_string(reinterpret_cast<uintptr_t>(op)) + "/" + std::to_string(grid);
      for (Request* r : rq) key += "/" + std::to_string(r->nrhs);
      cuda_ok(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal), "begin capture");
      cudaGraph_t graph = nullptr;
      try {
        enqueue_batch(b, rq, grid, st);
      } catch (...) {
        cudaStreamEndCapture(st, &graph);
        if (graph) cudaGraphDestroy(graph);
        throw;
      }
      cuda_ok(cudaStreamEndCapture(st, &graph), "end capture");
      GraphEntry& ge = graphs[key];
      bool ok = false;
      if (ge.exec) {
        cudaGraphExecUpdateResultInfo info{};
        ok = cudaGraphExecUpdate(ge.exec, graph, &info) == cudaSuccess;
        if (!ok) {
          cudaGetLastError();
          cudaGraphExecDestroy(ge.exec);
          ge.exec = nullptr;
        }
      }
      if (!ok) {
        const cudaError_t e = cudaGraphInstantiate(&ge.exec, graph, 0);
        if (e != cudaSuccess) {
          cudaGraphDestroy(graph);
          graphs.erase(key);
          cuda_ok(e, "graph instantiate");
        }
        ++graph_insts;
      }
      cudaGraphDestroy(graph);
      ge.last_use = ++use_clock;
      cuda_ok(cudaGraphLaunch(ge.exec, st), "graph launch");
      ++graph_launches;
      if (graphs.size() > 256) {   // drop the least recently used executable graph
        auto lru = graphs.begin();
        for (auto it = graphs.begin(); it != graphs.end(); ++it)
          if (it->second.last_use < lru->second.last_use) lru = it;
        cudaGraphExecDestroy(lru->second.exec);
        graphs.erase(lru);
      }
    } else {
      enqueue_batch(b, rq, grid, st);
    }
    if (b.stage) cuda_ok(cudaFreeAsync(b.stage, st), "staging free");
    b.stage = nullptr;
    cuda_ok(cudaMemcpyAsync(status_host[size_t(b.slot)], op->d_status, sizeof(int), cudaMemcpyDeviceToHost, st),
            "status copy");
    cuda_ok(cudaEventRecord(b.done, st), "event record");
  }

  // Worker: retire finished batches, start new ones, sleep briefly while work is out.
  void run() {
    cudaSetDevice(device);
    std::unique_lock<std::mutex> lk(mu);
    for (;;) {
      bool progress = false;
      // 1. completions
      for (size_t i = 0; i < slots.size(); ++i) {
        Batch& b = slots[i];
        if (!b.op) continue;
        const cudaError_t q = cudaEventQuery(b.done);
        if (q == cudaErrorNotReady) continue;
        int dev_status = *status_host[i];
        int32_t err = MBF_OK;
        if (q != cudaSuccess) {
          err = MBF_ERR_CUDA;
          mbf::set_last_error(std::string("batch failed: ") + cudaGetErrorString(q));
        } else if (dev_status != 0) {
          err = MBF_ERR_TIMEOUT;
          cudaMemsetAsync(b.op->d_status, 0, sizeof(int), streams[i]);
          cudaStreamSynchronize(streams[i]);
        }
        const double t = now();
        for (mbf_ticket_t id : b.ids) {
          auto it = reqs.find(id);
          if (it == reqs.end()) continue;
          Request& r = it->second;
          r.st.state = err == MBF_OK ? MBF_REQ_DONE : MBF_REQ_ERROR;
          r.st.error = err;
          r.st.t_done = t;
          reserved -= r.reserved;
          r.reserved = 0;
          if (err == MBF_OK) ++stats.completed;
          else ++stats.failed;
        }
        busy_ops.erase(b.op);
        b.op = nullptr;
        b.ids.clear();
        progress = true;
      }
      // 2. dispatch
      for (size_t i = 0; i < slots.size(); ++i) {
        if (slots[i].op) continue;
        auto qi = queue.begin();
        while (qi != queue.end() && busy_ops.count(reqs[*qi].op)) ++qi;
        if (qi == queue.end()) break;
        mbf_op_s* op = reqs[*qi].op;
        Batch& b = slots[i];
        b.slot = int(i);
        b.op = op;
        b.rhs = 0;
        std::vector<Request*> rq;
        for (auto it = qi; it != queue.end();) {
          Request& r = reqs[*it];
          if (r.op == op && (rq.empty() || b.rhs + r.nrhs <= opts.max_batch_rhs)) {
            b.ids.push_back(*it);
            rq.push_back(&r);
            b.rhs += r.nrhs;
            it = queue.erase(it);
          } else {
            ++it;
          }
        }
        busy_ops.insert(op);
        const double t = now();
        for (Request* r : rq) {
          r->st.state = MBF_REQ_RUNNING;
          r->st.t_start = t;
          r->st.batch_requests = int32_t(rq.size());
          r->st.batch_rhs = int32_t(b.rhs);
        }
        ++stats.batches;
        if (rq.size() > 1) stats.coalesced_requests += int64_t(rq.size());
        stats.max_batch_requests = std::max(stats.max_batch_requests, int32_t(rq.size()));
        stats.max_concurrent_batches = std::max(stats.max_concurrent_batches, int32_t(inflight()));
        // SM share: the whole GPU when this batch runs alone, 1 / max_inflight otherwise
        const bool shared = inflight() > 1 || !queue.empty();
        const int grid = shared ? std::max(1, sms / opts.max_inflight) : 0;
        lk.unlock();
        int32_t err = MBF_OK;
        std::string msg;
        try {
          launch(b, rq, grid);
        } catch (const Error& e) {
          err = e.code;
          msg = e.what();
        } catch (const std::exception& e) {
          err = MBF_ERR_INVALID;
          msg = e.what();
        }
        lk.lock();
        stats.graph_launches = graph_launches;
        stats.graph_instantiations = graph_insts;
        if (err != MBF_OK) {
          // nothing (more) runs for this batch: fail its requests now
          cudaStreamSynchronize(streams[i]);
          cudaGetLastError();
          mbf::set_last_error(msg);
          const double t2 = now();
          for (mbf_ticket_t id : b.ids) {
            Request& r = reqs[id];
            r.st.state = MBF_REQ_ERROR;
            r.st.error = err;
            r.st.t_done = t2;
            reserved -= r.reserved;
            r.reserved = 0;
            ++stats.failed;
          }
          busy_ops.erase(op);
          b.op = nullptr;
          b.ids.clear();
        }
        progress = true;
      }
      if (queue.empty() && inflight() == 0) {
        cv_idle.notify_all();
        if (stop) break;
        cv_work.wait(lk, [&] { return stop || !queue.empty(); });
        continue;
      }
      if (!progress) {
        // work is on the device: poll its events again shortly (new submissions wake us)
        cv_work.wait_for(lk, std::chrono::microseconds(20));
      }
    }
  }
};

namespace {

template <class F>
mbf_status sguard(F&& fn) {
  try {
    fn();
    mbf::set_last_error("");
    return MBF_OK;
  } catch (const Error& e) {
    mbf::set_last_error(e.what());
    return e.code;
  } catch (const std::bad_alloc&) {
    mbf::set_last_error("host allocation failed");
    return MBF_ERR_OOM;
  } catch (const std::exception& e) {
    mbf::set_last_error(e.what());
    return MBF_ERR_INVALID;
  }
}

void server_free(mbf_server_s* s) {
  if (!s) return;
  if (s->worker.joinable()) {
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->stop = true;
    }
    s->cv_work.notify_all();
    s->worker.join();
  }
  for (auto& kv : s->graphs) cudaGraphExecDestroy(kv.second.exec);
  for (auto& b : s->slots)
    if (b.done) cudaEventDestroy(b.done);
  for (int* p : s->status_host) cudaFreeHost(p);
  for (cudaStream_t st : s->streams) cudaStreamDestroy(st);
  delete s;
}

}  // namespace

extern "C" {

mbf_status mbf_server_create(const mbf_server_opts_t* opts, mbf_server_t* out) {
  return sguard([&] {
    if (!out) fail(MBF_ERR_INVALID, "NULL argument");
    auto* s = new mbf_server_s();
    try {
      if (opts) s->opts = *opts;
      if (s->opts.staging_budget_bytes <= 0) s->opts.staging_budget_bytes = int64_t(1) << 30;
      if (s->opts.max_inflight <= 0) s->opts.max_inflight = 4;
      if (s->opts.max_inflight > 16) fail(MBF_ERR_INVALID, "max_inflight > 16");
      if (s->opts.max_batch_rhs <= 0) s->opts.max_batch_rhs = 64;
      if (s->opts.max_queue <= 0) s->opts.max_queue = 4096;
      cuda_ok(cudaGetDevice(&s->device), "cudaGetDevice");
      cuda_ok(cudaDeviceGetAttribute(&s->sms, cudaDevAttrMultiProcessorCount, s->device), "attr");
      s->t0 = std::chrono::steady_clock::now();
      s->slots.resize(size_t(s->opts.max_inflight));
      for (int i = 0; i < s->opts.max_inflight; ++i) {
        cudaStream_t st = nullptr;
        cuda_ok(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking), "stream");
        s->streams.push_back(st);
        int* p = nullptr;
        cuda_ok(cudaMallocHost(&p, sizeof(int)), "pinned status");
        *p = 0;
        s->status_host.push_back(p);
        cuda_ok(cudaEventCreateWithFlags(&s->slots[size_t(i)].done, cudaEventDisableTiming), "event");
      }
      s->worker = std::thread([s] { s->run(); });
    } catch (...) {
      server_free(s);
      throw;
    }
    *out = s;
  });
}

mbf_status mbf_submit(mbf_server_t s, mbf_op_t op, const void* g, void* u, int64_t nrhs, mbf_ticket_t* ticket) {
  return sguard([&] {
    if (!s || !op || !g || !u || !ticket) fail(MBF_ERR_INVALID, "NULL argument");
    if (nrhs <= 0 || nrhs > (int64_t(1) << 24)) fail(MBF_ERR_INVALID, "nrhs out of range");
    if (op->device != s->device) fail(MBF_ERR_INVALID, "operator lives on another device");
    const int64_t need = 2 * nrhs * std::max(op->n_in, op->n_out) * int64_t(sizeof(float2));
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) fail(MBF_ERR_INVALID, "server is shutting down");
    if (int64_t(s->queue.size()) >= s->opts.max_queue || s->reserved + need > s->opts.staging_budget_bytes) {
      ++s->stats.rejected_busy;
      fail(MBF_ERR_BUSY, "server busy: queue or staging budget full");
    }
    const mbf_ticket_t id = s->next_id++;
    Request& r = s->reqs[id];
    r.op = op;
    r.g = g;
    r.u = u;
    r.nrhs = nrhs;
    r.reserved = need;
    r.st.state = MBF_REQ_QUEUED;
    r.st.t_submit = s->now();
    s->reserved += need;
    s->queue.push_back(id);
    ++s->stats.submitted;
    *ticket = id;
    s->cv_work.notify_one();
  });
}

mbf_status mbf_poll(mbf_server_t s, mbf_ticket_t ticket, mbf_request_status_t* status) {
  return sguard([&] {
    if (!s || !status) fail(MBF_ERR_INVALID, "NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) fail(MBF_ERR_NOT_FOUND, "unknown ticket");
    *status = it->second.st;
    if (status->state == MBF_REQ_DONE || status->state == MBF_REQ_ERROR) s->reqs.erase(it);
  });
}

mbf_status mbf_server_drain(mbf_server_t s, double timeout_s) {
  return sguard([&] {
    if (!s) fail(MBF_ERR_INVALID, "NULL argument");
    std::unique_lock<std::mutex> lk(s->mu);
    s->cv_work.notify_all();
    const bool ok = s->cv_idle.wait_for(lk, std::chrono::duration<double>(std::max(0.0, timeout_s)),
                                        [&] { return s->queue.empty() && s->inflight() == 0; });
    if (!ok) fail(MBF_ERR_TIMEOUT, "requests still queued or running");
  });
}

mbf_status mbf_server_stats(mbf_server_t s, mbf_server_stats_t* out) {
  return sguard([&] {
    if (!s || !out) fail(MBF_ERR_INVALID, "NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    *out = s->stats;
  });
}

mbf_status mbf_server_destroy(mbf_server_t s) {
  return sguard([&] { server_free(s); });
}

}  // extern "C"
