// Serving: continuous batching of independent rotation problems on one GPU.
//
// Requests queue on the host. Worker threads, each owning a CUDA stream, a device input
// arena and (through solve()) a device workspace, repeatedly take every request that fits
// the device-memory budget from the front of the queue (admission; a batch holds at most
// kServerBatchPairs pairs), copy their inputs to the device and solve them together with one
// launch sequence. While one worker's batch is on the GPU another admits the requests that
// arrived meanwhile and launches them on its own stream, so consecutive batches overlap. Each
// request completes on its own (a waiter is woken per request), and its result depends only on
// its own inputs: instances share no accumulator and no floating-point reduction.
#include <chrono>
#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "sprot_internal.h"

using namespace sprot;

namespace {

using Clock = std::chrono::steady_clock;

// Worker threads (each its own stream and workspace) and the pairs one batch may hold: small
// batches and several in flight keep a request's wait short when large requests arrive in a
// row, at loads well below the device's throughput.
constexpr int kServerWorkers = 12;
constexpr int64_t kServerBatchPairs = 2 << 20;
// initial input arena of a worker: a full batch of pairs (P and Q, 12 bytes each per pair)
constexpr size_t kServerArenaBytes = (size_t)kServerBatchPairs * 24 + (64u << 10);

struct Req {
  uint64_t ticket;
  sprot_request r;
  size_t bytes;
  double t_submit = 0, t_admit = 0, t_done = 0;
  bool done = false;
  sprot_result res;
};

}  // namespace

struct sprot_server {
  sprot_server_cfg cfg;
  Clock::time_point t0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  bool stopping = false;
  uint64_t next_ticket = 1;
  std::deque<std::shared_ptr<Req>> queue;
  std::unordered_map<uint64_t, std::shared_ptr<Req>> reqs;
  size_t in_use = 0;
  std::vector<std::thread> workers;
  int init_status = SPROT_OK;

  double now_ms() const {
    return std::chrono::duration<double, std::milli>(Clock::now() - t0).count();
  }
  void worker_main(int idx);
};

namespace {

size_t request_bytes(const sprot_request& r, int dev) {
  int G = r.params.grid ? r.params.grid : sprot_autotune_grid(r.n);
  return (size_t)r.n * 24 + problem_footprint(r.n, G, r.params.angle_bins, r.params.k, dev);
}

bool request_valid(const sprot_request& r) {
  const sprot_params& p = r.params;
  const int G = p.grid ? p.grid : sprot_autotune_grid(r.n);
  return r.P && r.Q && r.n >= 1 && !(G & (G - 1)) && G >= SPROT_MIN_GRID && G <= SPROT_MAX_GRID &&
         p.angle_bins >= 2 && p.angle_bins <= SPROT_MAX_ANGLE_BINS && p.k >= 1 && p.k <= SPROT_MAX_K &&
         p.tau > 0.0 && p.gate_window >= -1 && p.angle_window >= 0 && p.nms_deg >= 0.f;
}

}  // namespace

void sprot_server::worker_main(int idx) {
  cudaSetDevice(cfg.device);
  cudaStream_t st = nullptr;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
    std::lock_guard<std::mutex> g(mu);
    init_status = SPROT_E_CUDA;
    stopping = true;
    cv_work.notify_all();
    cv_done.notify_all();
    return;
  }
  char* arena = nullptr;
  size_t arena_cap = 0;
  (void)idx;
  for (;;) {
    std::vector<std::shared_ptr<Req>> batch;
    {
      std::unique_lock<std::mutex> lk(mu);
      cv_work.wait(lk, [&] {
        return (!queue.empty() && in_use + queue.front()->bytes <= cfg.device_budget_bytes) ||
               (stopping && queue.empty());
      });
      if (queue.empty()) break;  // stopping and drained
      double t = now_ms();
      int64_t pairs = 0;
      while (!queue.empty() && (int)batch.size() < cfg.max_batch &&
             in_use + queue.front()->bytes <= cfg.device_budget_bytes &&
             (batch.empty() || pairs + queue.front()->r.n <= kServerBatchPairs)) {
        auto r = queue.front();
        pairs += r->r.n;
        queue.pop_front();
        in_use += r->bytes;
        r->t_admit = t;
        batch.push_back(r);
      }
    }
    // inputs -> device arena (grown geometrically, in stream order: a synchronous free would
    // wait for the other workers' batches)
    size_t need = 0;
    for (auto& r : batch) need += ((size_t)r->r.n * 12 + 255) / 256 * 256 * 2;
    int status = SPROT_OK;
    if (need > arena_cap) {
      const size_t want = std::max(need, std::max<size_t>(arena_cap * 2, kServerArenaBytes));
      if (arena && cudaFreeAsync(arena, st) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(arena);
      }
      arena = nullptr;
      arena_cap = 0;
      if (cudaMallocAsync(reinterpret_cast<void**>(&arena), want, st) == cudaSuccess) {
        arena_cap = want;
      } else {
        cudaGetLastError();
        arena = nullptr;
        status = SPROT_E_NOMEM;
      }
    }
    std::vector<Problem> probs;
    std::vector<int32_t> nfound(batch.size(), 0);
    if (status == SPROT_OK) {
      size_t off = 0;
      for (size_t i = 0; i < batch.size(); ++i) {
        const sprot_request& q = batch[i]->r;
        size_t bytes = (size_t)q.n * 12;
        float* dP = reinterpret_cast<float*>(arena + off);
        off += (bytes + 255) / 256 * 256;
        float* dQ = reinterpret_cast<float*>(arena + off);
        off += (bytes + 255) / 256 * 256;
        if (cudaMemcpyAsync(dP, q.P, bytes, cudaMemcpyHostToDevice, st) != cudaSuccess ||
            cudaMemcpyAsync(dQ, q.Q, bytes, cudaMemcpyHostToDevice, st) != cudaSuccess) {
          status = SPROT_E_CUDA;
          break;
        }
        sprot_params p = q.params;
        p.flags &= ~SPROT_HOST_PTRS;
        if (p.grid == 0) p.grid = sprot_autotune_grid(q.n);
        probs.push_back(Problem{dP, dQ, q.n, p, p.k, false, batch[i]->res.rot, &nfound[i], nullptr,
                                nullptr, nullptr});
      }
    }
    // mixed batches rarely repeat a shape: no graph capture on the serving path
    if (status == SPROT_OK) status = solve(probs, st, false);
    {
      std::lock_guard<std::mutex> g(mu);
      double t = now_ms();
      for (size_t i = 0; i < batch.size(); ++i) {
        auto& r = batch[i];
        r->res.status = status;
        r->res.n_found = status == SPROT_OK ? nfound[i] : 0;
        if (status == SPROT_OK && nfound[i] == 0) r->res.status = SPROT_E_NOAXIS;
        r->res.t_submit_ms = r->t_submit;
        r->res.t_admit_ms = r->t_admit;
        r->res.t_done_ms = t;
        r->done = true;
        in_use -= r->bytes;
      }
    }
    cv_done.notify_all();
    cv_work.notify_all();
  }
  if (arena) cudaFreeAsync(arena, st);
  cudaStreamSynchronize(st);
  release_workspace(st);  // the worker's workspace goes with its stream
  cudaStreamDestroy(st);
}

extern "C" {

int sprot_server_create(const sprot_server_cfg* cfg, sprot_server** out) {
  if (!cfg || !out || cfg->device_budget_bytes == 0) return SPROT_E_INVAL;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || cfg->device < 0 || cfg->device >= ndev)
    return SPROT_E_CUDA;
  sprot_server* s = new (std::nothrow) sprot_server();
  if (!s) return SPROT_E_NOMEM;
  s->cfg = *cfg;
  if (s->cfg.max_batch <= 0) s->cfg.max_batch = 256;
  if (s->cfg.max_queue <= 0) s->cfg.max_queue = 65536;
  s->t0 = Clock::now();
  for (int i = 0; i < kServerWorkers; ++i) s->workers.emplace_back(&sprot_server::worker_main, s, i);
  *out = s;
  return SPROT_OK;
}

size_t sprot_server_request_bytes(const sprot_server_cfg* cfg, const sprot_request* req) {
  if (!cfg || !req || !request_valid(*req)) return 0;
  return request_bytes(*req, cfg->device);
}

int sprot_server_submit(sprot_server* s, const sprot_request* req, uint64_t* ticket) {
  if (!s || !req || !ticket || !request_valid(*req)) return SPROT_E_INVAL;
  auto r = std::make_shared<Req>();
  r->r = *req;
  r->bytes = request_bytes(*req, s->cfg.device);
  std::lock_guard<std::mutex> g(s->mu);
  if (s->init_status != SPROT_OK) return s->init_status;
  if (r->bytes > s->cfg.device_budget_bytes) return SPROT_E_NOMEM;
  if (s->stopping || (int)s->queue.size() >= s->cfg.max_queue) return SPROT_E_BUSY;
  r->ticket = s->next_ticket++;
  r->t_submit = s->now_ms();
  s->reqs[r->ticket] = r;
  s->queue.push_back(r);
  *ticket = r->ticket;
  s->cv_work.notify_one();
  return SPROT_OK;
}

int sprot_server_wait(sprot_server* s, uint64_t ticket, int32_t timeout_ms, sprot_result* res) {
  if (!s || !res) return SPROT_E_INVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return SPROT_E_INVAL;
  std::shared_ptr<Req> r = it->second;
  auto pred = [&] { return r->done || s->init_status != SPROT_OK; };
  if (timeout_ms < 0)
    s->cv_done.wait(lk, pred);
  else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), pred))
    return SPROT_E_TIMEOUT;
  if (!r->done) return s->init_status;
  *res = r->res;
  s->reqs.erase(ticket);
  return SPROT_OK;
}

int sprot_server_destroy(sprot_server* s) {
  if (!s) return SPROT_E_INVAL;
  {
    std::lock_guard<std::mutex> g(s->mu);
    s->stopping = true;
  }
  s->cv_work.notify_all();
  for (auto& t : s->workers) t.join();
  delete s;
  return SPROT_OK;
}

}  // extern "C"
