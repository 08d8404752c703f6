// lq_serve.cpp -- continuous-batching request server over the lq kernels.
//
// A server owns a caller-provided device arena (the library still allocates
// no device memory) and `slots` worker threads, each with its own CUDA stream.
// Requests (a circuit, its parameters, a Pauli sum, energy only or energy and
// gradient) are queued on submit.  A worker admits the oldest request whose
// footprint fits in the arena's free space (first-fit placement; a request
// that has been bypassed `kMaxBypass` times blocks younger ones, so large
// requests cannot starve), runs it on its stream and frees its memory; the
// next admission happens as soon as memory and a slot free up, so work of
// different requests overlaps on the device.  Energy-only requests of at most
// kSmallQubits qubits waiting together are merged into one persistent batch
// launch (lq_batch_param_shift).  Gradients use the adjoint method.  Every
// request records submit/start/done times (monotonic seconds) for latency
// percentiles.  Results do not depend on what else is in flight: each request
// runs the same kernels with the same fixed-order reductions alone or mixed.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/lq.h"
#include "lq_internal.h"

namespace lq {

static double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

static constexpr int kSmallQubits = 12;
static constexpr int kMaxBatch = 64;
static constexpr int kMaxBypass = 16;

static inline std::size_t al(std::size_t b) { return (b + 255) & ~(std::size_t)255; }

struct SReq {
  int64_t id = 0;
  int n = 0, np = 0, nt = 0, want_grad = 0;
  std::vector<lq_gate> gates;
  std::vector<double> params;
  std::vector<lq_pauli_term> terms;
  std::size_t footprint = 0;
  double t_submit = 0, t_start = 0, t_done = 0;
  int status = -1;
  double energy = 0;
  std::vector<double> grad;
  std::string error;
  bool done = false;
  int bypassed = 0;
};

// First-fit allocator over [0, size) of the arena.
class Arena {
 public:
  void init(std::size_t size) {
    free_.clear();
    if (size) free_[0] = size;
  }
  bool alloc(std::size_t bytes, std::size_t* off) {
    bytes = al(bytes);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        *off = it->first;
        std::size_t rest = it->second - bytes, start = it->first + bytes;
        free_.erase(it);
        if (rest) free_[start] = rest;
        return true;
      }
    }
    return false;
  }
  void release(std::size_t off, std::size_t bytes) {
    bytes = al(bytes);
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }

 private:
  std::map<std::size_t, std::size_t> free_;
};

struct Server {
  char* arena = nullptr;
  std::size_t arena_bytes = 0;
  int device = 0;
  Arena alloc;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<std::shared_ptr<SReq>> queue;
  std::unordered_map<int64_t, std::shared_ptr<SReq>> reqs;
  std::vector<std::thread> workers;
  std::vector<cudaStream_t> streams;
  bool stop = false;
  int64_t next_id = 1;

  void run_single(SReq& r, char* ws, std::size_t ws_bytes, cudaStream_t s) {
    lq_status st;
    if (r.want_grad) {
      r.grad.assign((std::size_t)r.np, 0.0);
      st = lq_adjoint_grad(r.n, r.gates.data(), (int)r.gates.size(), r.params.data(), r.np,
                           r.terms.data(), r.nt, &r.energy, r.grad.data(), ws, ws_bytes,
                           (lq_stream)s);
    } else {
      std::size_t sb = al(sizeof(double) * 2 << r.n);
      st = lq_state_init(ws, r.n, 0, (lq_stream)s);
      if (!st)
        st = lq_apply_circuit(ws, r.n, r.gates.data(), (int)r.gates.size(), r.params.data(), r.np,
                              (lq_stream)s);
      if (!st)
        st = lq_expval_pauli_sum(ws, r.n, r.terms.data(), r.nt, &r.energy, ws + sb,
                                 ws_bytes - sb, (lq_stream)s);
    }
    r.status = st;
    if (st) r.error = lq_last_error();
  }

  void run_batch(std::vector<std::shared_ptr<SReq>>& group, char* ws, std::size_t ws_bytes,
                 cudaStream_t s) {
    std::vector<lq_problem> pb(group.size());
    for (std::size_t i = 0; i < group.size(); i++) {
      SReq& r = *group[i];
      lq_problem& q = pb[i];
      std::memset(&q, 0, sizeof q);
      q.n = r.n;
      q.ng = (int)r.gates.size();
      q.np = r.np;
      q.nt = r.nt;
      q.want_grad = 0;
      q.gates = r.gates.data();
      q.params = r.params.data();
      q.terms = r.terms.data();
      q.energy = &r.energy;
      q.grad = nullptr;
    }
    lq_status st = lq_batch_param_shift(pb.data(), (int)pb.size(), ws, ws_bytes, (lq_stream)s);
    std::string msg = st ? lq_last_error() : "";
    for (auto& r : group) {
      r->status = st;
      r->error = msg;
    }
  }

  // Footprint of a single request in the arena.
  static std::size_t footprint(const SReq& r) {
    if (r.want_grad)
      return lq_adjoint_workspace_size(r.n, (int)r.gates.size(), r.np, r.nt);
    return al(sizeof(double) * 2 << r.n) + lq_expval_workspace_size(r.n, r.nt);
  }

  static std::size_t batch_footprint(const std::vector<std::shared_ptr<SReq>>& g) {
    std::vector<lq_problem> pb(g.size());
    for (std::size_t i = 0; i < g.size(); i++) {
      const SReq& r = *g[i];
      lq_problem& q = pb[i];
      std::memset(&q, 0, sizeof q);
      q.n = r.n;
      q.ng = (int)r.gates.size();
      q.np = r.np;
      q.nt = r.nt;
      q.gates = r.gates.data();
      q.params = r.params.data();
      q.terms = r.terms.data();
    }
    return lq_batch_workspace_size(pb.data(), (int)pb.size());
  }

  void worker(int w) {
    cudaSetDevice(device);
    cudaStream_t s = streams[w];
    std::unique_lock<std::mutex> lock(mu);
    for (;;) {
      std::vector<std::shared_ptr<SReq>> group;
      std::size_t off = 0, bytes = 0;
      for (;;) {
        if (stop) return;
        // admission: oldest request that fits; an old request that keeps
        // being bypassed blocks the younger ones
        for (std::size_t qi = 0; qi < queue.size(); qi++) {
          std::shared_ptr<SReq> r = queue[qi];
          bool small = !r->want_grad && r->n <= kSmallQubits;
          std::vector<std::shared_ptr<SReq>> g{r};
          if (small) {
            for (std::size_t qj = qi + 1; qj < queue.size() && (int)g.size() < kMaxBatch; qj++)
              if (!queue[qj]->want_grad && queue[qj]->n <= kSmallQubits) g.push_back(queue[qj]);
          }
          std::size_t need = small && g.size() > 1 ? batch_footprint(g) : r->footprint;
          if (need > 0 && alloc.alloc(need, &off)) {
            group = g;
            bytes = need;
            break;
          }
          if (g.size() > 1 && alloc.alloc(r->footprint, &off)) {  // the batch does not fit
            group = {r};
            bytes = r->footprint;
            break;
          }
          if (qi == 0 && ++queue[0]->bypassed > kMaxBypass) break;
        }
        if (!group.empty()) break;
        cv_work.wait(lock);
      }
      for (auto& r : group) {
        queue.erase(std::find(queue.begin(), queue.end(), r));
        r->t_start = now_s();
      }
      lock.unlock();
      if (group.size() == 1)
        run_single(*group[0], arena + off, bytes, s);
      else
        run_batch(group, arena + off, bytes, s);
      double t = now_s();
      lock.lock();
      alloc.release(off, bytes);
      for (auto& r : group) {
        r->t_done = t;
        r->done = true;
      }
      cv_done.notify_all();
      cv_work.notify_all();
    }
  }
};

}  // namespace lq

using namespace lq;

struct lq_server {
  Server s;
};

extern "C" {

size_t lq_server_footprint(int n, int want_grad, int ng, int np, int nt) {
  if (n < 1 || n > 34) return 0;
  if (want_grad) return lq_adjoint_workspace_size(n, ng, np, nt);
  return al(sizeof(double) * 2 << n) + lq_expval_workspace_size(n, nt);
}

lq_status lq_server_create(void* arena, size_t arena_bytes, int slots, lq_server** out) {
  if (!arena || !out || arena_bytes == 0) return fail(LQ_ERR_INVALID_ARG, "NULL arena or out");
  if (slots < 1 || slots > 64) return fail(LQ_ERR_INVALID_ARG, "slots must be in [1, 64]");
  lq_server* h = new lq_server;
  Server& S = h->s;
  S.arena = (char*)arena;
  S.arena_bytes = arena_bytes;
  S.alloc.init(arena_bytes);
  cudaGetDevice(&S.device);
  for (int i = 0; i < slots; i++) {
    cudaStream_t st;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
      (void)cudaGetLastError();
      for (auto x : S.streams) cudaStreamDestroy(x);
      delete h;
      return fail(LQ_ERR_CUDA, "cudaStreamCreate failed");
    }
    S.streams.push_back(st);
  }
  for (int i = 0; i < slots; i++) S.workers.emplace_back(&Server::worker, &S, i);
  *out = h;
  return LQ_OK;
}

lq_status lq_server_submit(lq_server* h, const lq_request* q, int64_t* id) {
  if (!h || !q || !id) return fail(LQ_ERR_INVALID_ARG, "NULL argument");
  lq_status st = check_n(q->n);
  if (st) return st;
  st = check_gates(q->n, q->gates, q->ng, q->params, q->np);
  if (st) return st;
  st = check_terms(q->n, q->terms, q->nt);
  if (st) return st;
  auto r = std::make_shared<SReq>();
  r->n = q->n;
  r->np = q->np;
  r->nt = q->nt;
  r->want_grad = q->want_grad != 0;
  r->gates.assign(q->gates, q->gates + q->ng);
  r->params.assign(q->params, q->params + q->np);
  r->terms.assign(q->terms, q->terms + q->nt);
  r->footprint = Server::footprint(*r);
  Server& S = h->s;
  if (r->footprint > S.arena_bytes)
    return fail(LQ_ERR_OOM, "request needs %zu bytes, arena holds %zu", r->footprint,
                S.arena_bytes);
  std::lock_guard<std::mutex> lock(S.mu);
  r->id = S.next_id++;
  r->t_submit = now_s();
  S.reqs[r->id] = r;
  S.queue.push_back(r);
  *id = r->id;
  S.cv_work.notify_one();
  return LQ_OK;
}

lq_status lq_server_wait(lq_server* h, int64_t id, double timeout_s, lq_result* res,
                         double* grad) {
  if (!h || !res) return fail(LQ_ERR_INVALID_ARG, "NULL argument");
  Server& S = h->s;
  std::unique_lock<std::mutex> lock(S.mu);
  auto it = S.reqs.find(id);
  if (it == S.reqs.end()) return fail(LQ_ERR_INVALID_ARG, "unknown request %lld", (long long)id);
  std::shared_ptr<SReq> r = it->second;
  bool ok = S.cv_done.wait_for(lock, std::chrono::duration<double>(timeout_s),
                               [&] { return r->done; });
  if (!ok) return fail(LQ_ERR_TIMEOUT, "request %lld not done", (long long)id);
  res->id = r->id;
  res->status = r->status;
  res->np = r->np;
  res->energy = r->energy;
  res->t_submit = r->t_submit;
  res->t_start = r->t_start;
  res->t_done = r->t_done;
  if (grad && r->want_grad && r->status == LQ_OK)
    for (int i = 0; i < r->np; i++) grad[i] = r->grad[i];
  S.reqs.erase(it);
  if (r->status != LQ_OK) return fail((lq_status)r->status, "request failed: %s", r->error.c_str());
  return LQ_OK;
}

lq_status lq_server_destroy(lq_server* h) {
  if (!h) return LQ_OK;
  Server& S = h->s;
  {
    std::lock_guard<std::mutex> lock(S.mu);
    S.stop = true;
  }
  S.cv_work.notify_all();
  for (auto& t : S.workers) t.join();
  for (auto x : S.streams) cudaStreamDestroy(x);
  delete h;
  return LQ_OK;
}

}  // extern "C"
