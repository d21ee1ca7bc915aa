// Serving loop: continuous batching of applies on resident operators (the paper has
// no counterpart).  A worker thread owns the CUDA work; mbf_submit / mbf_poll only
// touch the queue under the server's mutex.
//
// Per batch (one slot = one stream): the oldest queued request and the queued requests
// on its operator in FIFO order up to max_batch_rhs RHS form the batch's first group;
// when requests back up and more operators are queued than slots are free, the oldest
// requests on other operators add further groups the same way, up to max_batch_ops
// operators of at most mix_work_pct percent of the first group's factor traffic.  A
// group's requests are applied at once in place: the kernels read and write the
// requests' own rows through a table of row addresses (up to 64 RHS); a larger group
// is gathered into a staging panel (device-to-device copies) and scattered back.
// Each group borrows a workspace of its operator for the batch (the operator's own one
// when free, else one of its pool, allocated once and kept by the operator), so batches
// of one operator in different slots run at the same time.  With use_graphs the whole batch --
// every group's copies and kernels, in parallel branches -- is captured into one CUDA
// graph and started by one graph launch; an executable graph is kept per batch shape
// (operators, request RHS counts, SM shares) and updated in place for new buffers.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <deque>
#include <functional>
#include <map>
#include <mutex>
#include <set>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "apply.hpp"
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

// One operator's share of a batch.
struct Group {
  mbf_op_s* op = nullptr;
  std::vector<mbf_ticket_t> ids;
  std::vector<Request*> rq;
  int64_t rhs = 0;
  void* stage = nullptr;       // [rhs][n_in] then [rhs][n_out]
  mbf::Workspace* ws = nullptr;   // borrowed from the operator for the batch
};

constexpr int kMaxGroups = 8;   // operators per batch at most

struct Batch {
  int slot = -1;
  std::vector<Group> groups;   // empty: the slot is free
  cudaEvent_t done = nullptr;
};

struct GraphEntry {
  cudaGraphExec_t exec = nullptr;
  uint64_t last_use = 0;
};

// The server options with the defaults of their zero fields applied; invalid ones fail.
mbf_server_opts_t with_defaults(const mbf_server_opts_t* in) {
  mbf_server_opts_t o{};
  if (in) o = *in;
  if (o.staging_budget_bytes <= 0) o.staging_budget_bytes = int64_t(1) << 30;
  if (o.max_inflight <= 0) o.max_inflight = 4;
  if (o.max_inflight > 16) fail(MBF_ERR_INVALID, "max_inflight > 16");
  if (o.max_batch_rhs <= 0) o.max_batch_rhs = 64;
  if (o.max_queue <= 0) o.max_queue = 4096;
  if (o.max_batch_ops <= 0) o.max_batch_ops = 4;
  if (o.max_batch_ops > kMaxGroups) fail(MBF_ERR_INVALID, "max_batch_ops > 8");
  if (o.mix_work_pct < 0) fail(MBF_ERR_INVALID, "mix_work_pct < 0");
  if (o.mix_work_pct == 0) o.mix_work_pct = 25;
  return o;
}

// One queued request as the batch rule sees it: its operator (an index) and RHS count.
struct QueuedReq {
  int32_t op;
  int64_t nrhs;
};

// The batch rule: which queued requests (oldest first) form the next batch on a slot
// while `free_slots` slots are free.  groups[k] lists the queue positions of group k's
// requests in FIFO order.  One operator per batch unless requests back up (more queued
// than max_inflight * max_batch_ops) and the free slots cannot take every queued
// operator on its own; then the queued operators are spread over the free slots, up to
// max_batch_ops per batch.  The oldest request on an operator not yet in (or passed over
// for) the batch opens a group, and that operator's queued requests join it while they
// fit max_batch_rhs; a further group joins only if its factor traffic work(op, rhs) is at
// most mix_work_pct percent of the first group's (the batch ends with its longest group).
std::vector<std::vector<size_t>> form_batch(const std::vector<QueuedReq>& q, int free_slots,
                                            const mbf_server_opts_t& o,
                                            const std::function<double(int32_t, int64_t)>& work) {
  std::vector<std::vector<size_t>> groups;
  if (q.empty()) return groups;
  std::set<int32_t> qops;
  for (const QueuedReq& r : q) qops.insert(r.op);
  const bool backlog = int64_t(q.size()) > int64_t(o.max_inflight) * o.max_batch_ops;
  const int want = backlog ? (int(qops.size()) + free_slots - 1) / std::max(1, free_slots) : 1;
  const int max_ops = std::min({kMaxGroups, std::max(1, o.max_batch_ops), std::max(1, want)});
  std::set<int32_t> in_batch, passed;
  double work0 = 0;
  while (int(groups.size()) < max_ops) {
    size_t qo = 0;
    while (qo < q.size() && (in_batch.count(q[qo].op) || passed.count(q[qo].op))) ++qo;
    if (qo == q.size()) break;
    const int32_t op = q[qo].op;
    std::vector<size_t> take;
    int64_t rhs = 0;
    for (size_t i = qo; i < q.size(); ++i)
      if (q[i].op == op && (take.empty() || rhs + q[i].nrhs <= o.max_batch_rhs)) {
        take.push_back(i);
        rhs += q[i].nrhs;
      }
    const double wk = work(op, rhs);
    if (groups.empty()) {
      work0 = wk;
    } else if (wk * 100.0 > double(o.mix_work_pct) * work0) {
      passed.insert(op);
      continue;
    }
    in_batch.insert(op);
    groups.push_back(std::move(take));
  }
  return groups;
}

// SMs of each group of a batch: `share` split in proportion to the groups' factor
// traffic (work > 0), at least one each, the rounding remainder to the group of most
// work (the first of equal ones), so that the groups finish together.  The shares sum
// to `share` when it is at least the number of groups; with fewer SMs than groups every
// group still gets one (the groups then share SMs).
std::vector<int> split_share(const std::vector<double>& work, int share) {
  const size_t ng = work.size();
  if (ng == 0) return {};
  if (ng == 1) return {share};
  double sum = 0;
  for (double w : work) sum += w;
  std::vector<int> g(ng);
  int used = 0;
  size_t big = 0;
  for (size_t k = 0; k < ng; ++k) {
    g[k] = std::max(1, int(double(share) * work[k] / sum));
    used += g[k];
    if (work[k] > work[big]) big = k;
  }
  g[big] = std::max(1, g[big] + share - used);
  return g;
}

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
  std::vector<cudaStream_t> streams;                 // per slot
  std::vector<std::vector<cudaStream_t>> aux;        // per slot: branch streams of a batch
  std::vector<cudaEvent_t> fork_ev;                  // per slot
  std::vector<std::vector<cudaEvent_t>> join_ev;     // per slot and branch
  std::vector<int*> status_host;   // pinned: [slot][group] copies of the groups' status words
  std::vector<Batch> slots;

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
    for (const auto& b : slots) n += !b.groups.empty();
    return n;
  }

  // Copies and apply of one group on stream st (captured or not).
  void enqueue_group(const Group& gr, int grid, cudaStream_t st) {
    mbf_op_s* op = gr.op;
    if (gr.rq.size() == 1) {
      mbf::apply_dev(op, gr.rq[0]->g, gr.rq[0]->u, gr.rq[0]->nrhs, MBF_PREC_AUTO, st, false, grid, false, gr.ws);
      return;
    }
    if (!gr.stage) {   // up to kRowTab RHS: applied in place through a table of the requests' rows
      mbf::RowTable rows{};
      int64_t r0 = 0;
      for (Request* r : gr.rq)
        for (int64_t k = 0; k < r->nrhs; ++k, ++r0) {
          rows.in[r0] = static_cast<const float2*>(r->g) + k * op->n_in;
          rows.out[r0] = static_cast<float2*>(r->u) + k * op->n_out;
        }
      mbf::apply_dev(op, nullptr, nullptr, gr.rhs, MBF_PREC_AUTO, st, false, grid, false, gr.ws, &rows);
      return;
    }
    auto* in = static_cast<float2*>(gr.stage);
    float2* out = in + gr.rhs * op->n_in;
    int64_t r0 = 0;
    for (Request* r : gr.rq) {
      cuda_ok(cudaMemcpyAsync(in + r0 * op->n_in, r->g, size_t(r->nrhs * op->n_in) * sizeof(float2),
                              cudaMemcpyDeviceToDevice, st),
              "gather copy");
      r0 += r->nrhs;
    }
    mbf::apply_dev(op, in, out, gr.rhs, MBF_PREC_AUTO, st, false, grid, false, gr.ws);
    r0 = 0;
    for (Request* r : gr.rq) {
      cuda_ok(cudaMemcpyAsync(r->u, out + r0 * op->n_out, size_t(r->nrhs * op->n_out) * sizeof(float2),
                              cudaMemcpyDeviceToDevice, st),
              "scatter copy");
      r0 += r->nrhs;
    }
  }

  // Factor bytes a group streams: the operator's factors once per pass (a 64-RHS panel
  // on the tensor cores, up to 4 RHS on the SIMT kernel).  The apply is bound by this
  // traffic, so it sets the group's share of the batch's SMs.
  static double group_work(const mbf_op_s* op, int64_t rhs) {
    if (mbf::uses_tensor(op, rhs, MBF_PREC_AUTO, false))
      return double(std::max<int64_t>(op->tc_bytes, 1)) * double((rhs + 63) / 64);
    return 8.0 * double(std::max<int64_t>(op->nnz, 1)) * double((rhs + 3) / 4);
  }

  // SMs of each group: the batch's share (grid, or the whole GPU when 0) split by the
  // groups' factor traffic (split_share).  A batch of one group keeps `grid` as it is.
  std::vector<int> group_grids(const Batch& b, int grid) const {
    if (b.groups.size() == 1) return {grid};
    std::vector<double> w;
    for (const Group& gr : b.groups) w.push_back(group_work(gr.op, gr.rhs));
    return split_share(w, grid > 0 ? grid : sms);
  }

  // All groups of a batch: group 0 on the slot's stream, the others on branch streams
  // forked from it and joined back into it.
  void enqueue_batch(const Batch& b, int grid, cudaStream_t st) {
    const size_t ng = b.groups.size();
    const std::vector<int> gg = group_grids(b, grid);
    if (ng > 1) cuda_ok(cudaEventRecord(fork_ev[size_t(b.slot)], st), "fork");
    for (size_t k = 1; k < ng; ++k) {
      cudaStream_t as = aux[size_t(b.slot)][k - 1];
      cuda_ok(cudaStreamWaitEvent(as, fork_ev[size_t(b.slot)], 0), "fork wait");
      enqueue_group(b.groups[k], gg[k], as);
      cuda_ok(cudaEventRecord(join_ev[size_t(b.slot)][k - 1], as), "join");
    }
    enqueue_group(b.groups[0], gg[0], st);
    for (size_t k = 1; k < ng; ++k) cuda_ok(cudaStreamWaitEvent(st, join_ev[size_t(b.slot)][k - 1], 0), "join wait");
  }

  // Launch a batch on its slot (worker thread, lock not held).
  void launch(Batch& b, int grid) {
    cudaStream_t st = streams[size_t(b.slot)];
    std::string key = std::to_string(grid);
    for (Group& gr : b.groups) {
      // no allocation inside the capture: workspaces and staging first
      gr.ws = mbf::ws_acquire(gr.op, mbf::uses_tensor(gr.op, gr.rhs, MBF_PREC_AUTO, false));
      if (gr.rq.size() > 1 && gr.rhs > mbf::kRowTab)   // beyond a row table: through a staging panel
        cuda_ok(cudaMallocAsync(&gr.stage, size_t(gr.rhs * (gr.op->n_in + gr.op->n_out)) * sizeof(float2), st),
                "staging allocation");
      key += "|" + std::to_string(gr.op->serial);
      for (Request* r : gr.rq) key += "/" + std::to_string(r->nrhs);
    }
    if (opts.use_graphs) {
      cuda_ok(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal), "begin capture");
      cudaGraph_t graph = nullptr;
      try {
        enqueue_batch(b, grid, st);
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
      enqueue_batch(b, grid, st);
    }
    for (size_t k = 0; k < b.groups.size(); ++k) {
      Group& gr = b.groups[k];
      if (gr.stage) cuda_ok(cudaFreeAsync(gr.stage, st), "staging free");
      gr.stage = nullptr;
      cuda_ok(cudaMemcpyAsync(status_host[size_t(b.slot)] + k, gr.ws->status, sizeof(int), cudaMemcpyDeviceToHost, st),
              "status copy");
    }
    cuda_ok(cudaEventRecord(b.done, st), "event record");
  }

  // Fail every request of group gr with err at time t (lock held).
  void fail_group(Group& gr, int32_t err, double t) {
    for (mbf_ticket_t id : gr.ids) {
      auto it = reqs.find(id);
      if (it == reqs.end()) continue;
      Request& r = it->second;
      r.st.state = MBF_REQ_ERROR;
      r.st.error = err;
      r.st.t_done = t;
      reserved -= r.reserved;
      r.reserved = 0;
      ++stats.failed;
    }
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
        if (b.groups.empty()) continue;
        const cudaError_t q = cudaEventQuery(b.done);
        if (q == cudaErrorNotReady) continue;
        const double t = now();
        for (size_t k = 0; k < b.groups.size(); ++k) {
          Group& gr = b.groups[k];
          int32_t err = MBF_OK;
          if (q != cudaSuccess) {
            err = MBF_ERR_CUDA;
            mbf::set_last_error(std::string("batch failed: ") + cudaGetErrorString(q));
          } else if (status_host[i][k] != 0) {
            // a device wait of this group's apply gave up: its requests fail, its
            // workspace's status word is cleared for the next batch
            err = MBF_ERR_TIMEOUT;
            cudaMemsetAsync(gr.ws->status, 0, sizeof(int), streams[i]);
            cudaStreamSynchronize(streams[i]);
            status_host[i][k] = 0;
          }
          if (err != MBF_OK) {
            mbf::ws_release(gr.op, gr.ws);
            fail_group(gr, err, t);
            continue;
          }
          mbf::ws_release(gr.op, gr.ws);
          for (mbf_ticket_t id : gr.ids) {
            auto it = reqs.find(id);
            if (it == reqs.end()) continue;
            Request& r = it->second;
            r.st.state = MBF_REQ_DONE;
            r.st.error = MBF_OK;
            r.st.t_done = t;
            reserved -= r.reserved;
            r.reserved = 0;
            ++stats.completed;
          }
        }
        b.groups.clear();
        progress = true;
      }
      // 2. dispatch
      for (size_t i = 0; i < slots.size(); ++i) {
        if (!slots[i].groups.empty() || queue.empty()) continue;
        Batch& b = slots[i];
        b.slot = int(i);
        int free_slots = 0;
        for (const auto& x : slots) free_slots += x.groups.empty();
        // the batch rule on the queue, operators numbered in order of appearance
        std::vector<QueuedReq> qv;
        std::vector<mbf_op_s*> opv;
        std::unordered_map<mbf_op_s*, int32_t> opi;
        qv.reserve(queue.size());
        for (mbf_ticket_t id : queue) {
          mbf_op_s* op = reqs[id].op;
          auto it = opi.find(op);
          const int32_t k = it != opi.end() ? it->second : int32_t(opv.size());
          if (it == opi.end()) {
            opi.emplace(op, k);
            opv.push_back(op);
          }
          qv.push_back({k, reqs[id].nrhs});
        }
        const auto gl = form_batch(qv, free_slots, opts,
                                   [&](int32_t k, int64_t rhs) { return group_work(opv[size_t(k)], rhs); });
        int64_t nreq = 0, nrhs_all = 0;
        std::vector<size_t> taken;
        for (const auto& gpos : gl) {
          Group gr;
          gr.op = opv[size_t(qv[gpos[0]].op)];
          for (size_t pos : gpos) {
            const mbf_ticket_t id = queue[pos];
            Request& r = reqs[id];
            gr.ids.push_back(id);
            gr.rq.push_back(&r);
            gr.rhs += r.nrhs;
            taken.push_back(pos);
          }
          nreq += int64_t(gr.rq.size());
          nrhs_all += gr.rhs;
          b.groups.push_back(std::move(gr));
        }
        std::sort(taken.begin(), taken.end());
        for (auto t = taken.rbegin(); t != taken.rend(); ++t) queue.erase(queue.begin() + std::ptrdiff_t(*t));
        const double t = now();
        for (Group& gr : b.groups)
          for (Request* r : gr.rq) {
            r->st.state = MBF_REQ_RUNNING;
            r->st.t_start = t;
            r->st.batch_requests = int32_t(nreq);
            r->st.batch_rhs = int32_t(nrhs_all);
          }
        ++stats.batches;
        if (nreq > 1) stats.coalesced_requests += nreq;
        if (b.groups.size() > 1) ++stats.mixed_batches;
        stats.max_batch_requests = std::max(stats.max_batch_requests, int32_t(nreq));
        stats.max_batch_ops = std::max(stats.max_batch_ops, int32_t(b.groups.size()));
        stats.max_concurrent_batches = std::max(stats.max_concurrent_batches, int32_t(inflight()));
        // SM share: the whole GPU when this batch runs alone, 1 / max_inflight otherwise
        // (split among the batch's groups in proportion to their factor traffic)
        const bool shared = inflight() > 1 || !queue.empty();
        const int grid = shared ? std::max(1, sms / opts.max_inflight) : 0;
        lk.unlock();
        int32_t err = MBF_OK;
        std::string msg;
        try {
          launch(b, grid);
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
          for (auto& as : aux[i]) cudaStreamSynchronize(as);
          cudaGetLastError();
          mbf::set_last_error(msg);
          const double t2 = now();
          for (Group& gr : b.groups) {
            if (gr.ws) mbf::ws_release(gr.op, gr.ws);
            fail_group(gr, err, t2);
          }
          b.groups.clear();
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
  for (auto& v : s->aux)
    for (cudaStream_t st : v) cudaStreamDestroy(st);
  for (cudaEvent_t e : s->fork_ev) cudaEventDestroy(e);
  for (auto& v : s->join_ev)
    for (cudaEvent_t e : v) cudaEventDestroy(e);
  delete s;
}

}  // namespace

extern "C" {

mbf_status mbf_server_create(const mbf_server_opts_t* opts, mbf_server_t* out) {
  return mbf::abi_guard([&] {
    if (!out) fail(MBF_ERR_INVALID, "NULL argument");
    auto* s = new mbf_server_s();
    try {
      s->opts = with_defaults(opts);
      cuda_ok(cudaGetDevice(&s->device), "cudaGetDevice");
      cuda_ok(cudaDeviceGetAttribute(&s->sms, cudaDevAttrMultiProcessorCount, s->device), "attr");
      s->t0 = std::chrono::steady_clock::now();
      s->slots.resize(size_t(s->opts.max_inflight));
      s->aux.resize(size_t(s->opts.max_inflight));
      s->join_ev.resize(size_t(s->opts.max_inflight));
      for (int i = 0; i < s->opts.max_inflight; ++i) {
        cudaStream_t st = nullptr;
        cuda_ok(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking), "stream");
        s->streams.push_back(st);
        int* p = nullptr;
        cuda_ok(cudaMallocHost(&p, sizeof(int) * kMaxGroups), "pinned status");
        for (int k = 0; k < kMaxGroups; ++k) p[k] = 0;
        s->status_host.push_back(p);
        cuda_ok(cudaEventCreateWithFlags(&s->slots[size_t(i)].done, cudaEventDisableTiming), "event");
        cudaEvent_t fe = nullptr;
        cuda_ok(cudaEventCreateWithFlags(&fe, cudaEventDisableTiming), "event");
        s->fork_ev.push_back(fe);
        for (int k = 1; k < s->opts.max_batch_ops; ++k) {
          cudaStream_t as = nullptr;
          cuda_ok(cudaStreamCreateWithFlags(&as, cudaStreamNonBlocking), "stream");
          s->aux[size_t(i)].push_back(as);
          cudaEvent_t je = nullptr;
          cuda_ok(cudaEventCreateWithFlags(&je, cudaEventDisableTiming), "event");
          s->join_ev[size_t(i)].push_back(je);
        }
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
  return mbf::abi_guard([&] {
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
  return mbf::abi_guard([&] {
    if (!s || !status) fail(MBF_ERR_INVALID, "NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) fail(MBF_ERR_NOT_FOUND, "unknown ticket");
    *status = it->second.st;
    if (status->state == MBF_REQ_DONE || status->state == MBF_REQ_ERROR) s->reqs.erase(it);
  });
}

mbf_status mbf_server_drain(mbf_server_t s, double timeout_s) {
  return mbf::abi_guard([&] {
    if (!s) fail(MBF_ERR_INVALID, "NULL argument");
    std::unique_lock<std::mutex> lk(s->mu);
    s->cv_work.notify_all();
    const bool ok = s->cv_idle.wait_for(lk, std::chrono::duration<double>(std::max(0.0, timeout_s)),
                                        [&] { return s->queue.empty() && s->inflight() == 0; });
    if (!ok) fail(MBF_ERR_TIMEOUT, "requests still queued or running");
  });
}

mbf_status mbf_server_stats(mbf_server_t s, mbf_server_stats_t* out) {
  return mbf::abi_guard([&] {
    if (!s || !out) fail(MBF_ERR_INVALID, "NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    *out = s->stats;
  });
}

mbf_status mbf_server_destroy(mbf_server_t s) {
  return mbf::abi_guard([&] { server_free(s); });
}

mbf_status mbf_debug_split_sms(const double* work, int32_t n, int32_t share, int32_t* sms_out) {
  return mbf::abi_guard([&] {
    if (n < 0 || (n > 0 && (!work || !sms_out))) fail(MBF_ERR_INVALID, "NULL argument or negative count");
    if (share < 1) fail(MBF_ERR_INVALID, "share < 1");
    std::vector<double> w(static_cast<size_t>(n));
    for (int32_t k = 0; k < n; ++k) {
      if (!(work[k] > 0.0) || !std::isfinite(work[k])) fail(MBF_ERR_INVALID, "work must be positive and finite");
      w[size_t(k)] = work[k];
    }
    const std::vector<int> g = split_share(w, share);
    for (int32_t k = 0; k < n; ++k) sms_out[k] = g[size_t(k)];
  });
}

mbf_status mbf_debug_form_batch(const int32_t* ops, const int64_t* nrhs, int64_t n, const double* op_work,
                                int32_t n_ops, int32_t free_slots, const mbf_server_opts_t* opts,
                                int32_t* group_of) {
  return mbf::abi_guard([&] {
    if (n < 0 || n_ops < 0 || (n > 0 && (!ops || !nrhs || !group_of)) || (n_ops > 0 && !op_work))
      fail(MBF_ERR_INVALID, "NULL argument or negative count");
    if (free_slots < 1) fail(MBF_ERR_INVALID, "free_slots < 1");
    const mbf_server_opts_t o = with_defaults(opts);
    std::vector<QueuedReq> q(static_cast<size_t>(n));
    for (int64_t i = 0; i < n; ++i) {
      if (ops[i] < 0 || ops[i] >= n_ops) fail(MBF_ERR_INVALID, "operator index out of range");
      if (nrhs[i] <= 0) fail(MBF_ERR_INVALID, "nrhs <= 0");
      q[size_t(i)] = {ops[i], nrhs[i]};
    }
    const auto gl = form_batch(q, free_slots, o, [&](int32_t k, int64_t rhs) { return op_work[k] * double(rhs); });
    for (int64_t i = 0; i < n; ++i) group_of[i] = -1;
    for (size_t k = 0; k < gl.size(); ++k)
      for (size_t pos : gl[k]) group_of[pos] = int32_t(k);
  });
}

}  // extern "C"
