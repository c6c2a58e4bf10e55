// Host runtime of libsprot: validation, planning, device workspaces and the launch sequence
// behind the C ABI of include/sprot.h.
//
// A call (single problem or batch) is planned on the host: each instance gets its accumulator
// side G, row bands that fit the 227 KB shared-memory tile and carry equal expected vote
// work, circle slices, and per-pair work items. The plan becomes three work tables and an
// instance table, copied to the device in one transfer; the kernels then run on the caller's
// stream in a fixed order with no host round trip until the final results copy.
#include <algorithm>
#include <array>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <map>
#include <optional>
#include <memory>
#include <mutex>
#include <vector>

#include "sprot_internal.h"

namespace sprot {

static std::atomic<uint64_t> g_launches{0};
uint64_t launches_add(uint64_t k) { return g_launches.fetch_add(k) + k; }

void ensure_dynamic_smem(const void* func, int bytes) {
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, int> done;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> g(mu);
  int& cur = done[{dev, func}];
  if (bytes > cur) {
    if (cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) == cudaSuccess)
      cur = bytes;
    else
      cudaGetLastError();  // the launch reports the failure
  }
}

// Axis-vote kernel timing (measurement only): events around each launch, read after the
// launching call has synchronised its stream.
static std::atomic<int> g_timing{0};
static std::mutex g_timing_mu;
static double g_vote_ms = 0.0;
static uint64_t g_vote_launches = 0;

struct VoteTimer {
  cudaEvent_t a = nullptr, b = nullptr;
  explicit VoteTimer(cudaStream_t st) {
    if (!g_timing.load()) return;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
      a = b = nullptr;
      return;
    }
    cudaEventRecord(a, st);
  }
  void stop(cudaStream_t st) {
    if (a) cudaEventRecord(b, st);
  }
  // call after the stream has been synchronised
  void collect() {
    if (!a) return;
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, a, b) == cudaSuccess) {
      std::lock_guard<std::mutex> g(g_timing_mu);
      g_vote_ms += ms;
      g_vote_launches += 1;
    } else {
      cudaGetLastError();
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    a = b = nullptr;
  }
  ~VoteTimer() { collect(); }
};

namespace {

constexpr size_t kAlign = 256;
inline size_t align_up(size_t x, size_t a = kAlign) { return (x + a - 1) / a * a; }

int sm_count(int dev) {
  static std::mutex mu;
  static std::map<int, int> cache;
  std::lock_guard<std::mutex> g(mu);
  auto it = cache.find(dev);
  if (it != cache.end()) return it->second;
  int v = 0;
  cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
  if (v <= 0) v = 1;
  cache[dev] = v;
  return v;
}

bool is_pow2(int x) { return x > 0 && (x & (x - 1)) == 0; }

// The device address of a host buffer of `bytes` bytes when all of it lies in one pinned,
// device-mapped allocation (cudaHostAlloc / cudaMallocHost / cudaHostRegister); else null.
// True when [p, p + bytes) lies in one pinned host allocation (cudaHostAlloc, cudaMallocHost or
// cudaHostRegister): a copy from it may be captured in a CUDA graph.
bool pinned_host(const void* p, size_t bytes) {
  cudaPointerAttributes a{}, b{};
  const char* last = static_cast<const char*>(p) + bytes - 1;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess || cudaPointerGetAttributes(&b, last) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (a.type != cudaMemoryTypeHost || b.type != cudaMemoryTypeHost || !a.devicePointer || !b.devicePointer)
    return false;
  // one contiguous mapping
  return static_cast<const char*>(b.devicePointer) - static_cast<const char*>(a.devicePointer) == (ptrdiff_t)(bytes - 1);
}

int validate(const float* P, const float* Q, int64_t n, const sprot_params* p, int k) {
  if (!P || !Q || !p) return SPROT_E_INVAL;
  if (n < 1 || n > (int64_t)1 << 31) return SPROT_E_INVAL;
  int G = p->grid;
  if (G != 0 && (!is_pow2(G) || G < SPROT_MIN_GRID || G > SPROT_MAX_GRID)) return SPROT_E_INVAL;
  if (p->angle_bins < 2 || p->angle_bins > SPROT_MAX_ANGLE_BINS) return SPROT_E_INVAL;
  if (k < 1 || k > SPROT_MAX_K) return SPROT_E_INVAL;
  if (!(p->tau > 0.0) || !std::isfinite(p->tau)) return SPROT_E_INVAL;
  if (!(p->nms_deg >= 0.f) || !std::isfinite(p->nms_deg)) return SPROT_E_INVAL;
  if (p->gate_window < -1 || p->angle_window < 0) return SPROT_E_INVAL;
  if (p->flags & ~(SPROT_HOST_PTRS | SPROT_SUBCELL_AXIS)) return SPROT_E_INVAL;
  return SPROT_OK;
}

// Bands of a G x G accumulator (of rows; the curve vote cuts its columns at the same edges).
// Each band must fit the shared tile (row_bytes per row beside table_bytes of per-warp tables,
// smem_bytes in all); band edges are multiples of 8 (the curve vote's tiles pack two rows or
// two columns per word and write them with 16-byte stores) and split the expected work evenly:
// random great circles cross the plane with density proportional to 2 / (1 + u^2 + v^2) (the
// stereographic length element over the uniform density of the sphere), whose integral across a
// row is (4 / a) atan(1 / a), a = sqrt(1 + v^2).
void plan_bands_uncached(int G, int smem_bytes, int row_bytes, int table_bytes, int* n_bands, int32_t* row0) {
  constexpr int U = 8;  // rows per planning unit
  const int cap = (smem_bytes - table_bytes) / row_bytes;
  const int P = G / U, capp = cap / U;  // units in all, per band
  std::vector<double> cum(P + 1, 0.0);
  for (int r = 0; r < G; ++r) {
    double v = -1.0 + (2.0 * r + 1.0) / G, a = std::sqrt(1.0 + v * v);
    cum[r / U + 1] += 4.0 / a * std::atan(1.0 / a);
  }
  for (int q = 0; q < P; ++q) cum[q + 1] += cum[q];
  for (int T = (P + capp - 1) / capp; T <= kMaxBands; ++T) {
    std::vector<int32_t> e(T + 1);
    e[0] = 0;
    e[T] = P;
    for (int b = 1; b < T; ++b) {
      double target = cum[P] * b / T;
      int r = (int)(std::lower_bound(cum.begin(), cum.end(), target) - cum.begin());
      int lo = std::max(e[b - 1] + 1, P - (T - b) * capp);  // the rest must still fit
      int hi = std::min(e[b - 1] + capp, P - (T - b));
      e[b] = std::min(std::max(r, lo), hi);
    }
    bool fits = true;
    for (int b = 0; b < T; ++b) fits &= (e[b + 1] - e[b]) <= capp && e[b + 1] > e[b];
    if (fits) {
      *n_bands = T;
      for (int b = 0; b <= T; ++b) row0[b] = U * e[b];
      return;
    }
  }
  // unreachable for G <= 2048 (cap >= 88 rows)
  *n_bands = 0;
}

// The band plan depends only on its four arguments and is needed once per instance of every
// call (thousands in a batch): computed once per thread and key.
void plan_bands(int G, int smem_bytes, int row_bytes, int table_bytes, int* n_bands, int32_t* row0) {
  struct Entry {
    int T;
    std::vector<int32_t> row0;
  };
  thread_local std::map<std::array<int, 4>, Entry> cache;
  const std::array<int, 4> key{G, smem_bytes, row_bytes, table_bytes};
  auto it = cache.find(key);
  if (it == cache.end()) {
    Entry e;
    e.row0.assign(kMaxBands + 1, 0);
    plan_bands_uncached(G, smem_bytes, row_bytes, table_bytes, &e.T, e.row0.data());
    it = cache.emplace(key, std::move(e)).first;
  }
  *n_bands = it->second.T;
  for (int b = 0; b <= it->second.T; ++b) row0[b] = it->second.row0[b];
}

// Shared bytes per accumulator row (or column) of a band: the curve vote's tile holds G + 4
// words per row pair of a row band (two rows share a word; 4 words of padding) and G + 1
// half-words per column of a column band (two columns share a word; one row of padding);
// the eps-band vote's tile G/2 words per row.
inline int vote_row_bytes(int G) { return 2 * G + 8; }
inline int eps_row_bytes(int G) { return 2 * G; }

struct InstPlan {
  int64_t n;
  int G, J, k, w, window;
  float tau;
  double cos_nms;
  int T, S;  // row bands and circle slices of the axis vote
  int32_t row0[kMaxBands + 1];
  int chunk, n_items, item0;
  // arena offsets
  size_t o_partial, o_grid, o_bins, o_msum, o_labels, o_vote_set, o_P, o_Q, o_mask;
  size_t o_peak, o_hist, o_ndeg, o_done;  // zero region
  int n_ritems = 0;
  size_t o_nfound, o_rot;          // result region
};

// An instantiated CUDA graph of one solve's launch sequence and the number of kernels in it
// (exec = nullptr: the shape could not be captured and runs directly).
struct GraphEntry {
  cudaGraphExec_t exec = nullptr;
  uint64_t kernels = 0;
  int uses = 0;            // calls seen with this shape
  bool capturable = true;  // false after a failed capture
};

struct Workspace {
  std::mutex mu;
  int device = 0;
  cudaStream_t stream = nullptr;  // the stream the workspace serves
  char* dev = nullptr;
  size_t dev_cap = 0;
  char* host = nullptr;  // pinned
  size_t host_cap = 0;
  // Graphs keyed by everything a captured sequence bakes in: workspace addresses, copy sizes,
  // grid sizes and item counts (the tables themselves are re-uploaded by the graph).
  std::map<std::vector<uint64_t>, GraphEntry> graphs;
  // events recorded around the vote kernel inside every captured sequence (solves on a
  // workspace are serialised and synchronised, so one pair serves all its graphs)
  cudaEvent_t tv0 = nullptr, tv1 = nullptr;
  // second stream for the second half of a host problem's input copy (under the first half's
  // vote), with its fork and join events
  cudaStream_t aux = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
  bool aux_stream() {
    if (!aux && cudaStreamCreateWithFlags(&aux, cudaStreamNonBlocking) != cudaSuccess) aux = nullptr;
    if (!fork && cudaEventCreateWithFlags(&fork, cudaEventDisableTiming) != cudaSuccess) fork = nullptr;
    if (!join && cudaEventCreateWithFlags(&join, cudaEventDisableTiming) != cudaSuccess) join = nullptr;
    if (!(aux && fork && join)) cudaGetLastError();
    return aux && fork && join;
  }
  // the stream a solve runs on when the caller passed the legacy default stream (which cannot
  // be captured in a graph), ordered after the caller's work by an event
  cudaStream_t own = nullptr;
  cudaEvent_t own_in = nullptr;
  bool own_stream() {
    if (!own && cudaStreamCreateWithFlags(&own, cudaStreamNonBlocking) != cudaSuccess) own = nullptr;
    if (!own_in && cudaEventCreateWithFlags(&own_in, cudaEventDisableTiming) != cudaSuccess) own_in = nullptr;
    if (!(own && own_in)) cudaGetLastError();
    return own && own_in;
  }
  bool timing_events() {
    if (!tv0 && cudaEventCreate(&tv0) != cudaSuccess) tv0 = nullptr;
    if (!tv1 && cudaEventCreate(&tv1) != cudaSuccess) tv1 = nullptr;
    return tv0 && tv1;
  }
  void drop_graphs() {
    for (auto& kv : graphs)
      if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    graphs.clear();
  }
  ~Workspace() {
    drop_graphs();
    if (tv0) cudaEventDestroy(tv0);
    if (tv1) cudaEventDestroy(tv1);
    if (fork) cudaEventDestroy(fork);
    if (join) cudaEventDestroy(join);
    if (own_in) cudaEventDestroy(own_in);
    if (own) cudaStreamDestroy(own);
    if (aux) cudaStreamDestroy(aux);
    if (dev) cudaFree(dev);
    if (host) cudaFreeHost(host);
  }
  // Device memory grows geometrically and is allocated and freed in stream order
  // (cudaMallocAsync / cudaFreeAsync): a synchronous cudaFree would wait for the whole device,
  // stalling the other workspaces' streams (e.g. concurrent server batches). `use` is the
  // caller's stream: the allocation is ordered before the call's work on it (a solve moved to
  // the workspace's own stream waits on an event recorded after it); every call synchronises
  // the stream it ran on before it returns, so no earlier work still reads a freed buffer.
  int reserve(size_t dbytes, size_t hbytes, cudaStream_t use) {
    if (dbytes > dev_cap || hbytes > host_cap) drop_graphs();  // their addresses are about to change
    if (dbytes > dev_cap) {
      size_t want = std::max(dbytes, dev_cap + dev_cap / 2);
      if (dev && cudaFreeAsync(dev, use) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(dev);
      }
      dev = nullptr;
      dev_cap = 0;
      auto alloc = [&](size_t b) {
        if (cudaMallocAsync(reinterpret_cast<void**>(&dev), b, use) == cudaSuccess) return true;
        cudaGetLastError();
        dev = nullptr;
        if (cudaMalloc(&dev, b) == cudaSuccess) return true;
        cudaGetLastError();
        dev = nullptr;
        return false;
      };
      if (!alloc(want)) {
        if (!alloc(dbytes)) return SPROT_E_NOMEM;
        want = dbytes;
      }
      dev_cap = want;
    }
    if (hbytes > host_cap) {
      hbytes = std::max<size_t>(hbytes, std::max<size_t>(4u << 20, host_cap * 2));  // rare regrowth
      if (host) cudaFreeHost(host);
      host = nullptr;
      host_cap = 0;
      if (cudaMallocHost(&host, hbytes) != cudaSuccess) {
        cudaGetLastError();
        host = nullptr;
        return SPROT_E_NOMEM;
      }
      host_cap = hbytes;
    }
    return SPROT_OK;
  }
};

std::mutex g_ws_mu;
// Workspaces are shared: a call holds its own reference for its whole duration, so releasing
// the cache (sprot_release_workspaces / sprot_release_stream_workspace) while a call runs on
// another host thread frees that workspace only when the call returns.
std::map<std::pair<int, cudaStream_t>, std::shared_ptr<Workspace>> g_ws;

std::shared_ptr<Workspace> workspace_for(cudaStream_t st, int* status) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    *status = SPROT_E_CUDA;
    return nullptr;
  }
  std::lock_guard<std::mutex> g(g_ws_mu);
  auto& slot = g_ws[{dev, st}];
  if (!slot) {
    slot.reset(new Workspace());
    slot->device = dev;
    slot->stream = st;
  }
  *status = SPROT_OK;
  return slot;
}


// The plan's knobs (the autotuner's search space); the defaults are the untuned plan.
sprot_plan_knobs default_knobs() { return sprot_plan_knobs{1, 600, 32768, 1200, 0.0, 0.0}; }

// Pairs per work item of the per-pair kernels. One problem: about `div` items (600 by
// default), so that the problem alone fills the GPU. A batch: sized from the batch's total (the
// instances provide the parallelism), so that small instances do not pay a block's fixed cost
// per few hundred pairs. At least 256 pairs an item.
int stream_chunk(int64_t n, int div = 600) {
  int64_t c = (n + div - 1) / div;
  c = (c + 255) / 256 * 256;
  return (int)std::min<int64_t>(std::max<int64_t>(c, 256), kStreamChunk);
}

int batch_chunk(int64_t total, int div = 1200) {
  int64_t c = (total + div - 1) / div;
  c = (c + 255) / 256 * 256;
  return (int)std::min<int64_t>(std::max<int64_t>(c, 256), kStreamChunk);
}

// Vote layout of one instance: row bands that fit the shared tile, and circle slices (at most
// 65535 circles each, so the 16-bit counters cannot overflow). A single problem is spread
// over every SM, its items filling `rounds` rounds of the SMs; in a batch each instance gets
// slices of batch_slice circles.
void plan_vote(InstPlan& ip, int64_t n, bool single, int nsm, bool eps = false,
               int64_t max_slices = INT64_MAX, int rounds = 1, int batch_slice = 32768) {
  if (eps)
    plan_bands(ip.G, kMaxSmemBytes, eps_row_bytes(ip.G), 0, &ip.T, ip.row0);
  else
    plan_bands(ip.G, kRunSmemBytes, vote_row_bytes(ip.G), vote_run_table_bytes(), &ip.T, ip.row0);
  const int64_t s_min = (n + kMaxSliceCircles - 1) / kMaxSliceCircles;
  // the curve vote has 2 T items per slice (row bands and column bands), the eps-band vote T
  const int per_slice = (eps ? 1 : 2) * std::max(ip.T, 1);
  int64_t s;
  if (single) {
    // k rounds of the SMs, at least as many as the counters force (k nsm >= s_min per_slice),
    // so that no round runs with most SMs idle: the most slices whose items fit them
    const int64_t k = std::max<int64_t>(rounds, (s_min * per_slice + nsm - 1) / nsm);
    s = std::max<int64_t>(1, k * nsm / per_slice);
  } else {
    s = (n + batch_slice - 1) / batch_slice;
  }
  s = std::min<int64_t>(s, std::max<int64_t>(1, (n + 511) / 512));
  s = std::min<int64_t>(s, max_slices);
  ip.S = (int)std::max(s, s_min);
}

// Tuned knobs, per class: {device, 0, bit length of n, G} for one problem, {device, 1, bit
// length of the mean n, 0} for a batch.
using TuneKey = std::array<int64_t, 4>;
std::mutex g_tune_mu;
std::map<TuneKey, sprot_plan_knobs> g_tuned;

int bit_length(int64_t x) {
  int b = 0;
  for (; x > 0; x >>= 1) ++b;
  return b;
}
TuneKey tune_key(int dev, bool batched, int64_t n, int G) {
  return TuneKey{dev, batched ? 1 : 0, bit_length(n), batched ? 0 : G};
}
bool tuned_lookup(const TuneKey& key, sprot_plan_knobs* kn) {
  std::lock_guard<std::mutex> g(g_tune_mu);
  auto it = g_tuned.find(key);
  if (it == g_tuned.end()) return false;
  *kn = it->second;
  return true;
}

int tile_bytes(const InstPlan& ip, bool eps = false) {
  int rows = 0;
  for (int b = 0; b < ip.T; ++b) rows = std::max(rows, ip.row0[b + 1] - ip.row0[b]);
  return rows * (eps ? eps_row_bytes(ip.G) : vote_row_bytes(ip.G));
}

}  // namespace

bool single_vote_plan(int64_t n, int G, int dev, int* T, int32_t* row0, int* S, int* tile, int* nsm,
                      int64_t max_slices) {
  InstPlan ip{};
  ip.G = G;
  *nsm = sm_count(dev);
  plan_vote(ip, n, true, *nsm, false, max_slices);
  if (ip.T <= 0) return false;
  *T = ip.T;
  for (int b = 0; b <= ip.T; ++b) row0[b] = ip.row0[b];
  *S = ip.S;
  *tile = tile_bytes(ip);
  return true;
}

// Frees the workspace of stream st on the current device (its buffers, graphs, events and
// second stream), for callers that destroy st; a later stream reusing the handle starts anew.
void release_workspace(cudaStream_t st) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return;
  std::shared_ptr<Workspace> w;
  {
    std::lock_guard<std::mutex> g(g_ws_mu);
    auto it = g_ws.find({dev, st});
    if (it == g_ws.end()) return;
    w = std::move(it->second);
    g_ws.erase(it);
  }
  // destroyed here, outside the lock, unless a call in flight still holds it (then when that
  // call returns)
}

size_t problem_footprint(int64_t n, int G, int J, int k, int dev) {
  // the most slices any plan within the knobs' ranges gives the problem: alone (three rounds of
  // the SMs) or in a batch (slices of 16384 circles); at most one per-pair item per 256 pairs
  InstPlan ip{};
  ip.G = G;
  plan_vote(ip, n, true, sm_count(dev), false, INT64_MAX, 3);
  const int64_t S = std::max<int64_t>(ip.S, (n + 16383) / 16384);
  const int64_t items = (n + 255) / 256;
  return align_up((size_t)2 * S * G * (G / 2) * 4) + align_up((size_t)G * G * 4) +
         align_up((size_t)k * n * 2) + align_up((size_t)2 * items * k * 80) + align_up((size_t)n * 4) +
         align_up((size_t)k * J * 4) + align_up(sizeof(DevRot) * k) + 4096;
}

// Runs `enqueue` (which issues one solve's asynchronous work on st) through the graph cached
// under `key`. A shape is captured when it is seen for the second time (shapes that never
// repeat, as in a server's mixed batches, are not worth a capture and instantiation); a shape
// that cannot be captured runs directly from then on. Returns enqueue's success (or the graph
// launch's).
template <class F>
bool run_graph(Workspace* ws, const std::vector<uint64_t>& key, cudaStream_t st, F&& enqueue) {
  auto it = ws->graphs.find(key);
  if (it == ws->graphs.end()) {
    if (ws->graphs.size() >= 64) ws->drop_graphs();
    ws->graphs[key].uses = 1;
    return enqueue();
  }
  GraphEntry& ge = it->second;
  if (ge.exec) {
    if (cudaGraphLaunch(ge.exec, st) != cudaSuccess) return false;
    launches_add(ge.kernels);
    return true;
  }
  if (!ge.capturable || ++ge.uses < 2) return enqueue();
  const uint64_t l0 = launches_add(0);
  if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    ge.capturable = false;
    return enqueue();
  }
  const bool ok = enqueue();
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(st, &g);
  const uint64_t kernels = launches_add(0) - l0;
  cudaGraphExec_t ex = nullptr;
  if (!ok || e != cudaSuccess || !g || cudaGraphInstantiate(&ex, g, 0) != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    launches_add(0 - kernels);  // captured launches that never ran
    ge.capturable = false;
    return enqueue();
  }
  cudaGraphDestroy(g);
  ge.exec = ex;
  ge.kernels = kernels;
  // the captured launches were counted once: they stand for this first execution
  return cudaGraphLaunch(ex, st) == cudaSuccess;
}

// Solves a batch of problems on stream st. Every Problem must be validated already.
int solve(std::vector<Problem>& probs, cudaStream_t st, bool graphs, const sprot_plan_knobs* force) {
  const int m = (int)probs.size();
  int status = SPROT_OK;
  std::shared_ptr<Workspace> ws = workspace_for(st, &status);
  if (!ws) return status;
  std::lock_guard<std::mutex> lock(ws->mu);
  const int nsm = sm_count(ws->device);

  // ---- plan ---------------------------------------------------------------------------
  std::vector<InstPlan> plan(m);
  int64_t total_n = 0;
  for (int i = 0; i < m; ++i) total_n += probs[i].n;
  sprot_plan_knobs kn = default_knobs();
  if (force)
    kn = *force;
  else
    tuned_lookup(tune_key(ws->device, m > 1, m > 1 ? total_n / m : probs[0].n,
                          probs[0].prm.grid ? probs[0].prm.grid : sprot_autotune_grid(probs[0].n)),
                 &kn);
  // One large problem from host buffers: its input copy is split in two, the vote's items of
  // the first half of the slices run as soon as the first half is copied, and the second half
  // is copied under them (two rounds of items at least, so that each half fills the SMs).
  const bool split = m == 1 && probs[0].host_io && probs[0].n >= (1 << 18) && ws->aux_stream();
  if (split) kn.vote_rounds = std::max(kn.vote_rounds, 2);
  // slice-reduction items: 512 words (one 16-byte column per thread) for one problem; in a
  // batch about 64 x 512 word-slices per item (an item reads every slice of its words), between
  // 512 and 8192 words
  std::vector<VoteItem> vitems;
  int vote_tile = 0;
  std::vector<ReduceItem> ritems;
  std::vector<StreamItem> sitems;
  int max_k = 1, max_J = 2;
  for (int i = 0; i < m; ++i) {
    const Problem& pb = probs[i];
    InstPlan& ip = plan[i];
    ip.n = pb.n;
    ip.G = pb.prm.grid ? pb.prm.grid : sprot_autotune_grid(pb.n);
    ip.J = pb.prm.angle_bins;
    ip.k = pb.k;
    ip.w = pb.prm.gate_window;
    ip.window = pb.prm.angle_window;
    ip.tau = (float)pb.prm.tau;
    ip.cos_nms = std::cos((double)pb.prm.nms_deg * 3.14159265358979323846 / 180.0);
    plan_vote(ip, pb.n, m == 1, nsm, false, INT64_MAX, kn.vote_rounds, kn.batch_slice);
    if (ip.T <= 0) return SPROT_E_INVAL;
    vote_tile = std::max(vote_tile, tile_bytes(ip));
    for (int sl = 0; sl < ip.S; ++sl) {
      int64_t c0 = pb.n * sl / ip.S, c1 = pb.n * (sl + 1) / ip.S;
      for (int b = 0; b < ip.T; ++b) {
        vitems.push_back(VoteItem{i, b, sl, 0, c0, c1});         // row caps -> partial sl
        vitems.push_back(VoteItem{i, b, ip.S + sl, 1, c0, c1});  // column caps -> partial S + sl
      }
    }
    int64_t words = (int64_t)ip.G * (ip.G / 2);
    const int64_t red_words =
        m == 1 ? kReduceWords
               : kReduceWords * std::min<int64_t>(64, std::max<int64_t>(1, 256 / std::max(ip.S, 1)));
    const size_t r0 = ritems.size();
    for (int64_t w0 = 0; w0 < words; w0 += red_words)
      ritems.push_back(ReduceItem{i, 0, w0, std::min<int64_t>(w0 + red_words, words)});
    ip.n_ritems = (int)(ritems.size() - r0);
    ip.chunk = m == 1 ? stream_chunk(pb.n, kn.chunk_div) : batch_chunk(total_n, kn.batch_div);
    ip.item0 = (int)sitems.size();
    for (int64_t a = 0; a < pb.n; a += ip.chunk)
      sitems.push_back(StreamItem{i, 0, a, std::min<int64_t>(a + ip.chunk, pb.n)});
    ip.n_items = (int)sitems.size() - ip.item0;
    max_k = std::max(max_k, ip.k);
    max_J = std::max(max_J, ip.J);
  }
  // Longest vote items first (the persistent CTAs then finish together).
  // (one problem: items stay in slice order, which the split copy relies on)
  if (m > 1)
    std::stable_sort(vitems.begin(), vitems.end(), [&](const VoteItem& a, const VoteItem& b) {
      double wa = (double)(a.c1 - a.c0) * plan[a.inst].G / plan[a.inst].T;
      double wb = (double)(b.c1 - b.c0) * plan[b.inst].G / plan[b.inst].T;
      return wa > wb;
    });
  // split copy: the items of the first half of the slices, and the pairs they read
  int n_first = (int)vitems.size();
  int64_t pairs_first = total_n;
  if (split) {
    const int half = plan[0].S / 2;
    n_first = 0;
    while (n_first < (int)vitems.size() && vitems[n_first].slice % plan[0].S < half) ++n_first;
    pairs_first = n_first > 0 ? vitems[n_first - 1].c1 : 0;
  }

  // ---- layout -------------------------------------------------------------------------
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off = align_up(off + std::max<size_t>(bytes, 1));
    return o;
  };
  const size_t o_inst = take(sizeof(InstDev) * m);
  const size_t o_vit = take(sizeof(VoteItem) * vitems.size());
  const size_t o_rit = take(sizeof(ReduceItem) * ritems.size());
  const size_t o_sit = take(sizeof(StreamItem) * sitems.size());
  const size_t header_end = off;
  const size_t o_zero = off;
  const size_t o_counter = take(2 * sizeof(int));  // the vote's item counters (two with a split copy)
  for (auto& ip : plan) {
    ip.o_peak = take(sizeof(unsigned long long) * ip.k);
    ip.o_hist = take(sizeof(uint32_t) * ip.k * ip.J);
    ip.o_ndeg = take(sizeof(uint32_t));
    ip.o_done = take(sizeof(uint32_t) * 4);
  }
  const size_t zero_end = off;
  const size_t o_res = off;
  for (auto& ip : plan) {
    ip.o_nfound = take(sizeof(int32_t));
    ip.o_rot = take(sizeof(DevRot) * ip.k);
  }
  const size_t res_end = off;
  for (int i = 0; i < m; ++i) {
    InstPlan& ip = plan[i];
    const Problem& pb = probs[i];
    ip.o_partial = take((size_t)2 * ip.S * ip.G * (ip.G / 2) * 4);
    ip.o_grid = take((size_t)ip.G * ip.G * 4);
    ip.o_bins = take((size_t)ip.k * ip.n * 2);
    ip.o_msum = take((size_t)2 * ip.n_items * ip.k * 10 * 8);
    ip.o_labels = (pb.labels && !pb.host_io) ? 0 : take((size_t)ip.n * 4);
    ip.o_vote_set = 0;
    ip.o_P = pb.host_io ? take((size_t)ip.n * 12) : 0;
    ip.o_Q = pb.host_io ? take((size_t)ip.n * 12) : 0;
    ip.o_mask = (pb.host_io && pb.mask) ? take((size_t)ip.n) : 0;
  }
  const size_t dev_bytes = off;
  const size_t host_bytes = align_up(header_end) + (res_end - o_res);
  status = ws->reserve(dev_bytes, host_bytes, st);
  if (status != SPROT_OK) return status;
  char* D = ws->dev;
  char* H = ws->host;

  // Host inputs are copied to the workspace at the start of the launch sequence. Copies from
  // pinned host memory can be captured in the sequence's graph (keyed by the host addresses);
  // pageable ones run directly. (The vote reads every pair once per band and orientation, so
  // it reads the device copy: reading pinned memory over the host link made it 65% slower.)
  std::vector<bool> pinned(m, false);
  for (int i = 0; i < m; ++i) {
    const Problem& pb = probs[i];
    if (pb.host_io)
      pinned[i] = pinned_host(pb.P, (size_t)pb.n * 12) && pinned_host(pb.Q, (size_t)pb.n * 12);
  }

  // ---- tables -------------------------------------------------------------------------
  InstDev* hid = reinterpret_cast<InstDev*>(H + o_inst);
  for (int i = 0; i < m; ++i) {
    const InstPlan& ip = plan[i];
    const Problem& pb = probs[i];
    InstDev& d = hid[i];
    std::memset(&d, 0, sizeof(d));
    d.P = pb.host_io ? reinterpret_cast<const float*>(D + ip.o_P) : pb.P;
    d.Q = pb.host_io ? reinterpret_cast<const float*>(D + ip.o_Q) : pb.Q;
    d.n = ip.n;
    d.G = ip.G;
    d.J = ip.J;
    d.k = ip.k;
    d.w = ip.w;
    d.window = ip.window;
    d.n_bands = ip.T;
    d.S = 2 * ip.S;  // partials: the row caps' and the column caps' of every slice
    d.subcell = (pb.prm.flags & SPROT_SUBCELL_AXIS) ? 1 : 0;
    d.tau = ip.tau;
    d.cos_nms = ip.cos_nms;
    for (int b = 0; b <= ip.T; ++b) d.band_row0[b] = ip.row0[b];
    d.partial = reinterpret_cast<uint32_t*>(D + ip.o_partial);
    d.grid = (pb.dbg && pb.dbg->grid) ? pb.dbg->grid : reinterpret_cast<uint32_t*>(D + ip.o_grid);
    d.peak_key = reinterpret_cast<unsigned long long*>(D + ip.o_peak);
    d.hist = (pb.dbg && pb.dbg->hist) ? nullptr : reinterpret_cast<uint32_t*>(D + ip.o_hist);
    d.bins = (pb.dbg && pb.dbg->bins) ? pb.dbg->bins : reinterpret_cast<int16_t*>(D + ip.o_bins);
    d.msum = reinterpret_cast<float2*>(D + ip.o_msum);
    d.item0 = ip.item0;
    d.n_items = ip.n_items;
    d.n_found = reinterpret_cast<int32_t*>(D + ip.o_nfound);
    d.n_deg = reinterpret_cast<uint32_t*>(D + ip.o_ndeg);
    d.done = reinterpret_cast<uint32_t*>(D + ip.o_done);
    d.n_ritems = ip.n_ritems;
    d.rot = reinterpret_cast<DevRot*>(D + ip.o_rot);
    d.labels = (pb.labels && !pb.host_io) ? pb.labels : reinterpret_cast<int32_t*>(D + ip.o_labels);
    d.vote_set = pb.dbg ? pb.dbg->vote_set : nullptr;
    d.mask = pb.mask ? (pb.host_io ? reinterpret_cast<uint8_t*>(D + ip.o_mask) : pb.mask) : nullptr;
  }
  // A caller-supplied histogram buffer is zeroed and used in place.
  for (int i = 0; i < m; ++i)
    if (probs[i].dbg && probs[i].dbg->hist) hid[i].hist = probs[i].dbg->hist;
  std::memcpy(H + o_vit, vitems.data(), sizeof(VoteItem) * vitems.size());
  std::memcpy(H + o_rit, ritems.data(), sizeof(ReduceItem) * ritems.size());
  std::memcpy(H + o_sit, sitems.data(), sizeof(StreamItem) * sitems.size());

  // ---- launches (replayed from a cached CUDA graph when the shape repeats) ----------------
  auto ck = [](cudaError_t e) { return e == cudaSuccess; };
  const InstDev* dinst = reinterpret_cast<const InstDev*>(D + o_inst);
  const VoteItem* dvit = reinterpret_cast<const VoteItem*>(D + o_vit);
  const ReduceItem* drit = reinterpret_cast<const ReduceItem*>(D + o_rit);
  const StreamItem* dsit = reinterpret_cast<const StreamItem*>(D + o_sit);
  int* dcounter = reinterpret_cast<int*>(D + o_counter);
  char* Hres = H + align_up(header_end);
  // Caller pointers outside the workspace are baked into a graph. Debug exports and pageable
  // host inputs run directly; pinned host inputs (and outputs) are part of the graph's key.
  bool direct_only = !graphs || !ws->timing_events();
  for (int i = 0; i < m; ++i) direct_only |= probs[i].dbg != nullptr || (probs[i].host_io && !pinned[i]);
  std::optional<VoteTimer> vt;
  auto enqueue = [&](bool direct) -> bool {
    bool ok = true;
    cudaGetLastError();  // an earlier call's error, not this solve's (sticky errors stay)
    ok &= ck(cudaMemcpyAsync(D, H, header_end, cudaMemcpyHostToDevice, st));
    ok &= ck(cudaMemsetAsync(D + o_zero, 0, zero_end - o_zero, st));
    for (int i = 0; i < m; ++i) {
      const Problem& pb = probs[i];
      if (pb.dbg && pb.dbg->hist)
        ok &= ck(cudaMemsetAsync(pb.dbg->hist, 0, sizeof(uint32_t) * plan[i].k * plan[i].J, st));
      if (pb.host_io) {
        const size_t b0 = (size_t)(split ? pairs_first : pb.n) * 12;  // the first (or only) part
        ok &= ck(cudaMemcpyAsync(D + plan[i].o_P, pb.P, b0, cudaMemcpyHostToDevice, st));
        ok &= ck(cudaMemcpyAsync(D + plan[i].o_Q, pb.Q, b0, cudaMemcpyHostToDevice, st));
      }
    }
    if (!ok) return false;
    if (split) ok &= ck(cudaEventRecord(ws->fork, st));  // the first part is on the device
    // The vote's timing events: while the stream is captured they are recorded as external
    // events, which become event record nodes that time every replay (the flag is refused
    // outside a capture).
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (!direct) ok &= ck(cudaStreamIsCapturing(st, &cs));
    const unsigned tv_flags = cs == cudaStreamCaptureStatusActive ? cudaEventRecordExternal : cudaEventRecordDefault;
    if (direct)
      vt.emplace(st);
    else
      ok &= ck(cudaEventRecordWithFlags(ws->tv0, st, tv_flags));
    launch_axis_vote_runs(dvit, n_first, dinst, dcounter, std::min(n_first, nsm), vote_tile, st);
    if (split) {
      // the second part, copied under the first items' vote (after the first part, so that the
      // two copies do not share the link)
      const Problem& pb = probs[0];
      const size_t b0 = (size_t)pairs_first * 12, b1 = (size_t)(pb.n - pairs_first) * 12;
      ok &= ck(cudaStreamWaitEvent(ws->aux, ws->fork, 0));
      ok &= ck(cudaMemcpyAsync(D + plan[0].o_P + b0, reinterpret_cast<const char*>(pb.P) + b0, b1,
                               cudaMemcpyHostToDevice, ws->aux));
      ok &= ck(cudaMemcpyAsync(D + plan[0].o_Q + b0, reinterpret_cast<const char*>(pb.Q) + b0, b1,
                               cudaMemcpyHostToDevice, ws->aux));
      ok &= ck(cudaEventRecord(ws->join, ws->aux));
      ok &= ck(cudaStreamWaitEvent(st, ws->join, 0));
      const int n_second = (int)vitems.size() - n_first;
      launch_axis_vote_runs(dvit + n_first, n_second, dinst, dcounter + 1, std::min(n_second, nsm), vote_tile, st);
    }
    if (direct)
      vt->stop(st);
    else
      ok &= ck(cudaEventRecordWithFlags(ws->tv1, st, tv_flags));
    // each kernel's last block per instance finishes that instance's stage (peaks; angle peak
    // and Rodrigues; the two Kabsch solves)
    launch_grid_reduce(drit, (int)ritems.size(), dinst, st);
    for (int r = 1; r < max_k; ++r) launch_nms_round(drit, (int)ritems.size(), dinst, r, st);
    launch_angle_vote(dsit, (int)sitems.size(), dinst, max_k, max_J, st);
    launch_vote_set_sum(dsit, (int)sitems.size(), dinst, max_k, st);
    launch_label_sum(dsit, (int)sitems.size(), dinst, max_k, st);
    if (!ck(cudaGetLastError())) return false;
    ok &= ck(cudaMemcpyAsync(Hres, D + o_res, res_end - o_res, cudaMemcpyDeviceToHost, st));
    for (int i = 0; i < m; ++i) {
      const Problem& pb = probs[i];
      if (!pb.host_io) continue;
      if (pb.labels)
        ok &= ck(cudaMemcpyAsync(pb.labels, D + plan[i].o_labels, (size_t)pb.n * 4,
                                 cudaMemcpyDeviceToHost, st));
      if (pb.mask)
        ok &= ck(cudaMemcpyAsync(pb.mask, D + plan[i].o_mask, (size_t)pb.n, cudaMemcpyDeviceToHost, st));
    }
    return ok;
  };
  bool ok;
  if (direct_only) {
    ok = enqueue(true);
  } else {
    const std::vector<uint64_t> key = {
        (uint64_t)(uintptr_t)D, (uint64_t)(uintptr_t)H, header_end, o_zero, zero_end, o_res, res_end,
        vitems.size(), ritems.size(), sitems.size(), (uint64_t)m, (uint64_t)max_k, (uint64_t)max_J,
        (uint64_t)vote_tile, (uint64_t)nsm, (uint64_t)split, (uint64_t)pairs_first};
    std::vector<uint64_t> k2 = key;
    for (int i = 0; i < m; ++i) {
      if (!probs[i].host_io) continue;
      // the host buffers the graph copies from and to, the copy sizes and staging offsets
      for (const void* q : {(const void*)probs[i].P, (const void*)probs[i].Q, (const void*)probs[i].mask,
                            (const void*)probs[i].labels})
        k2.push_back((uint64_t)(uintptr_t)q);
      for (uint64_t v : {(uint64_t)probs[i].n, (uint64_t)plan[i].o_P, (uint64_t)plan[i].o_Q,
                         (uint64_t)plan[i].o_mask, (uint64_t)plan[i].o_labels})
        k2.push_back(v);
    }
    // The legacy default stream cannot be captured: a solve whose graph is captured or
    // replayed now runs on the workspace's own stream instead, after everything the caller
    // ordered before it, the workspace's allocation included (the solve waits for its results
    // before returning, so the caller's later work follows it). Shapes seen for the first time
    // run directly on the caller's stream.
    auto ge = ws->graphs.find(k2);
    if ((st == nullptr || st == cudaStreamLegacy) && ge != ws->graphs.end() &&
        (ge->second.exec || ge->second.capturable) && ws->own_stream()) {
      if (!ck(cudaEventRecord(ws->own_in, st)) || !ck(cudaStreamWaitEvent(ws->own, ws->own_in, 0))) return SPROT_E_CUDA;
      st = ws->own;
    }
    ok = run_graph(ws.get(), k2, st, [&] { return enqueue(false); });
  }
  if (!ok || !ck(cudaStreamSynchronize(st))) return SPROT_E_CUDA;
  if (vt) {
    vt->collect();
  } else if (g_timing.load()) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, ws->tv0, ws->tv1) == cudaSuccess) {
      std::lock_guard<std::mutex> g(g_timing_mu);
      g_vote_ms += ms;
      g_vote_launches += 1;
    } else {
      cudaGetLastError();
    }
  }
  int worst = SPROT_OK;
  for (int i = 0; i < m; ++i) {
    const InstPlan& ip = plan[i];
    const Problem& pb = probs[i];
    int32_t nf = *reinterpret_cast<int32_t*>(Hres + (ip.o_nfound - o_res));
    const DevRot* dr = reinterpret_cast<const DevRot*>(Hres + (ip.o_rot - o_res));
    if (pb.n_found) *pb.n_found = nf;
    for (int a = 0; a < nf; ++a) {
      sprot_rotation& o = pb.out[a];
      const DevRot& r = dr[a];
      std::memcpy(o.R, r.R, sizeof(o.R));
      std::memcpy(o.R_init, r.R_init, sizeof(o.R_init));
      std::memcpy(o.R_vote, r.R_vote, sizeof(o.R_vote));
      std::memcpy(o.axis, r.axis, sizeof(o.axis));
      o.theta = r.theta;
      o.cell_row = r.cell_row;
      o.cell_col = r.cell_col;
      o.angle_bin = r.angle_bin;
      o.axis_votes = r.axis_votes;
      o.angle_votes = r.angle_votes;
      o.n_vote_set = r.n_vote_set;
      o.n_inliers = r.n_inliers;
      o.n_degenerate = r.n_degenerate;
      o.cell_offset[0] = r.cell_offset[0];
      o.cell_offset[1] = r.cell_offset[1];
    }
    if (nf == 0) worst = SPROT_E_NOAXIS;
    probs[i].prm.grid = ip.G;
  }
  return m == 1 ? worst : SPROT_OK;
}

// Accumulator only (stage entry points): the curve vote (eps < 0) or the eps-band vote of
// Eq. 9 (eps >= 0), then the slice reduction into a caller grid.
int axis_vote_only(const float* P, const float* Q, int64_t n, int G, uint32_t* grid,
                   cudaStream_t st, float eps) {
  int status = SPROT_OK;
  std::shared_ptr<Workspace> ws = workspace_for(st, &status);
  if (!ws) return status;
  std::lock_guard<std::mutex> lock(ws->mu);
  const int nsm = sm_count(ws->device);
  InstPlan ip{};
  ip.G = G;
  plan_vote(ip, n, true, nsm, eps >= 0.f);
  if (ip.T <= 0) return SPROT_E_INVAL;
  const int smem = tile_bytes(ip, eps >= 0.f);
  // the curve vote votes every slice twice (row bands: partial sl; column bands: partial S + sl)
  const int kinds = eps >= 0.f ? 1 : 2;
  std::vector<VoteItem> vit;
  for (int sl = 0; sl < ip.S; ++sl)
    for (int b = 0; b < ip.T; ++b)
      for (int kd = 0; kd < kinds; ++kd)
        vit.push_back(VoteItem{0, b, kd * ip.S + sl, kd, n * sl / ip.S, n * (sl + 1) / ip.S});
  std::vector<ReduceItem> rit;
  int64_t words = (int64_t)G * (G / 2);
  for (int64_t w0 = 0; w0 < words; w0 += kReduceWords) rit.push_back(ReduceItem{0, 0, w0, std::min<int64_t>(w0 + kReduceWords, words)});
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off = align_up(off + std::max<size_t>(bytes, 1)); return o; };
  size_t o_inst = take(sizeof(InstDev)), o_vit = take(sizeof(VoteItem) * vit.size()),
         o_rit = take(sizeof(ReduceItem) * rit.size());
  size_t hdr = off;
  size_t o_zero = take(sizeof(int)), o_peak = take(8);
  size_t zend = off;
  size_t o_part = take((size_t)kinds * ip.S * G * (G / 2) * 4);
  status = ws->reserve(off, hdr, st);
  if (status != SPROT_OK) return status;
  char* D = ws->dev;
  char* H = ws->host;
  InstDev& d = *reinterpret_cast<InstDev*>(H + o_inst);
  std::memset(&d, 0, sizeof(d));
  d.P = P;
  d.Q = Q;
  d.n = n;
  d.G = G;
  d.k = 1;
  d.n_bands = ip.T;
  d.S = kinds * ip.S;
  for (int b = 0; b <= ip.T; ++b) d.band_row0[b] = ip.row0[b];
  d.partial = reinterpret_cast<uint32_t*>(D + o_part);
  d.grid = grid;
  d.peak_key = reinterpret_cast<unsigned long long*>(D + o_peak);
  std::memcpy(H + o_vit, vit.data(), sizeof(VoteItem) * vit.size());
  std::memcpy(H + o_rit, rit.data(), sizeof(ReduceItem) * rit.size());
  if (cudaMemcpyAsync(D, H, hdr, cudaMemcpyHostToDevice, st) != cudaSuccess) return SPROT_E_CUDA;
  if (cudaMemsetAsync(D + o_zero, 0, zend - o_zero, st) != cudaSuccess) return SPROT_E_CUDA;
  const VoteItem* dv = reinterpret_cast<VoteItem*>(D + o_vit);
  const InstDev* di = reinterpret_cast<InstDev*>(D + o_inst);
  int* dc = reinterpret_cast<int*>(D + o_zero);
  const int nit = (int)vit.size();
  std::optional<VoteTimer> vt;
  if (eps < 0.f) {
    vt.emplace(st);
    launch_axis_vote_runs(dv, nit, di, dc, std::min(nit, nsm), smem, st);
    vt->stop(st);
  } else {
    launch_axis_vote_eps(dv, nit, di, dc, std::min(nit, nsm), smem, eps, st);
  }
  launch_grid_reduce(reinterpret_cast<ReduceItem*>(D + o_rit), (int)rit.size(), di, st);
  if (cudaGetLastError() != cudaSuccess) return SPROT_E_CUDA;
  // the host staging is reused by the next call: wait for the copy to have been consumed
  if (cudaStreamSynchronize(st) != cudaSuccess) return SPROT_E_CUDA;
  return SPROT_OK;
}

// Greedy top-k with suppression on a caller grid (stage entry point).
int select_peaks(const uint32_t* grid, int G, int k, float nms_deg, int32_t* cells,
                 uint32_t* counts, int32_t* n_found, cudaStream_t st) {
  int status = SPROT_OK;
  std::shared_ptr<Workspace> ws = workspace_for(st, &status);
  if (!ws) return status;
  std::lock_guard<std::mutex> lock(ws->mu);
  std::vector<ReduceItem> rit;
  int64_t words = (int64_t)G * (G / 2);
  for (int64_t w0 = 0; w0 < words; w0 += kReduceWords) rit.push_back(ReduceItem{0, 0, w0, std::min<int64_t>(w0 + kReduceWords, words)});
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off = align_up(off + std::max<size_t>(bytes, 1)); return o; };
  size_t o_inst = take(sizeof(InstDev)), o_rit = take(sizeof(ReduceItem) * rit.size());
  size_t hdr = off;
  size_t o_peak = take(8 * (size_t)k);
  status = ws->reserve(off, hdr, st);
  if (status != SPROT_OK) return status;
  char* D = ws->dev;
  char* H = ws->host;
  InstDev& d = *reinterpret_cast<InstDev*>(H + o_inst);
  std::memset(&d, 0, sizeof(d));
  d.G = G;
  d.k = k;
  d.cos_nms = std::cos((double)nms_deg * 3.14159265358979323846 / 180.0);
  d.grid = const_cast<uint32_t*>(grid);
  d.peak_key = reinterpret_cast<unsigned long long*>(D + o_peak);
  std::memcpy(H + o_rit, rit.data(), sizeof(ReduceItem) * rit.size());
  if (cudaMemcpyAsync(D, H, hdr, cudaMemcpyHostToDevice, st) != cudaSuccess) return SPROT_E_CUDA;
  if (cudaMemsetAsync(D + o_peak, 0, 8 * (size_t)k, st) != cudaSuccess) return SPROT_E_CUDA;
  const InstDev* di = reinterpret_cast<const InstDev*>(D + o_inst);
  for (int r = 0; r < k; ++r)
    launch_nms_round(reinterpret_cast<const ReduceItem*>(D + o_rit), (int)rit.size(), di, r, st);
  launch_write_peaks(di, cells, counts, n_found, st);
  if (cudaGetLastError() != cudaSuccess) return SPROT_E_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return SPROT_E_CUDA;
  return SPROT_OK;
}

}  // namespace sprot

using namespace sprot;

extern "C" {

void sprot_default_params(sprot_params* p) {
  if (!p) return;
  p->grid = 256;
  p->angle_bins = 360;
  p->k = 1;
  p->nms_deg = 2.0f;
  p->gate_window = 1;
  p->angle_window = 1;
  p->tau = 0.05;
  p->flags = 0;
}

const char* sprot_status_string(int s) {
  switch (s) {
    case SPROT_OK: return "ok";
    case SPROT_E_INVAL: return "invalid argument";
    case SPROT_E_NOMEM: return "out of memory or over budget";
    case SPROT_E_CUDA: return "CUDA error";
    case SPROT_E_TIMEOUT: return "timed out";
    case SPROT_E_NOAXIS: return "no axis: every accumulator cell is zero";
    case SPROT_E_UNIMPL: return "not implemented";
    case SPROT_E_BUSY: return "server busy or stopping";
    default: return "unknown status";
  }
}

int32_t sprot_autotune_grid(int64_t n) {
  if (n < 3000) return 128;
  if (n < 300000) return 256;
  return 512;
}

int sprot_estimate_rotations_ex(const float* P, const float* Q, int64_t n, const sprot_params* params,
                                sprot_rotation* out, int32_t* n_found, int32_t* labels,
                                const sprot_debug* dbg, void* stream) {
  if (!params || !out) return SPROT_E_INVAL;
  int st = validate(P, Q, n, params, params->k);
  if (st != SPROT_OK) return st;
  bool host = (params->flags & SPROT_HOST_PTRS) != 0;
  if (host && dbg) return SPROT_E_INVAL;
  std::vector<Problem> pb(1);
  pb[0] = Problem{P, Q, n, *params, params->k, host, out, n_found, labels, nullptr, dbg};
  if (pb[0].prm.grid == 0) pb[0].prm.grid = sprot_autotune_grid(n);
  return solve(pb, reinterpret_cast<cudaStream_t>(stream));
}

int sprot_estimate_rotations_k(const float* P, const float* Q, int64_t n, const sprot_params* params,
                               sprot_rotation* out, int32_t* n_found, int32_t* labels, void* stream) {
  return sprot_estimate_rotations_ex(P, Q, n, params, out, n_found, labels, nullptr, stream);
}

int sprot_estimate_rotation(const float* P, const float* Q, int64_t n, const sprot_params* params,
                            sprot_rotation* out, uint8_t* inlier_mask, void* stream) {
  if (!params || !out) return SPROT_E_INVAL;
  sprot_params p1 = *params;
  p1.k = 1;
  int st = validate(P, Q, n, &p1, 1);
  if (st != SPROT_OK) return st;
  bool host = (p1.flags & SPROT_HOST_PTRS) != 0;
  int32_t nf = 0;
  std::vector<Problem> pb(1);
  pb[0] = Problem{P, Q, n, p1, 1, host, out, &nf, nullptr, inlier_mask, nullptr};
  if (pb[0].prm.grid == 0) pb[0].prm.grid = sprot_autotune_grid(n);
  return solve(pb, reinterpret_cast<cudaStream_t>(stream));
}

int sprot_axis_vote(const float* P, const float* Q, int64_t n, int32_t G, uint32_t* grid, void* stream) {
  if (!P || !Q || !grid || n < 1 || !is_pow2(G) || G < SPROT_MIN_GRID || G > SPROT_MAX_GRID)
    return SPROT_E_INVAL;
  return axis_vote_only(P, Q, n, G, grid, reinterpret_cast<cudaStream_t>(stream), -1.f);
}

namespace {
bool vote_plan_args_ok(int64_t n, int32_t G, const int32_t* n_bands, const int32_t* band_row0,
                       const int32_t* slices) {
  return n_bands && band_row0 && slices && n >= 1 && n <= (int64_t)1 << 31 && is_pow2(G) &&
         G >= SPROT_MIN_GRID && G <= SPROT_MAX_GRID;
}
}  // namespace

int sprot_vote_plan_sm(int64_t n, int32_t G, int32_t batched, int32_t n_sm, int32_t* n_bands,
                       int32_t* band_row0, int32_t* slices) {
  if (!vote_plan_args_ok(n, G, n_bands, band_row0, slices) || n_sm < 1 || n_sm > 4096) return SPROT_E_INVAL;
  InstPlan ip{};
  ip.G = G;
  plan_vote(ip, n, batched == 0, n_sm);
  if (ip.T <= 0) return SPROT_E_INVAL;
  *n_bands = ip.T;
  for (int b = 0; b <= ip.T; ++b) band_row0[b] = ip.row0[b];
  *slices = ip.S;
  return SPROT_OK;
}

int sprot_vote_plan(int64_t n, int32_t G, int32_t batched, int32_t* n_bands, int32_t* band_row0,
                    int32_t* slices) {
  if (!vote_plan_args_ok(n, G, n_bands, band_row0, slices)) return SPROT_E_INVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return SPROT_E_CUDA;
  }
  return sprot_vote_plan_sm(n, G, batched, sm_count(dev), n_bands, band_row0, slices);
}

int sprot_axis_vote_eps(const float* P, const float* Q, int64_t n, int32_t G, float eps, uint32_t* grid,
                        void* stream) {
  if (!P || !Q || !grid || n < 1 || n > (int64_t)1 << 31 || !is_pow2(G) || G < SPROT_MIN_GRID ||
      G > SPROT_MAX_GRID || !(eps >= 0.f && eps < 1.f))
    return SPROT_E_INVAL;
  return axis_vote_only(P, Q, n, G, grid, reinterpret_cast<cudaStream_t>(stream), eps);
}

int sprot_refine_axis(const float* P, const float* Q, int64_t n, const int32_t* labels, int32_t label,
                      const double* hint, double* axis, double* lambda_min, int64_t* count, void* stream) {
  if (!P || !Q || !axis || n < 1 || n > (int64_t)1 << 31) return SPROT_E_INVAL;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  int status = SPROT_OK;
  std::shared_ptr<Workspace> ws = workspace_for(st, &status);
  if (!ws) return status;
  std::lock_guard<std::mutex> lock(ws->mu);
  const int chunk = kStreamChunk;
  const int nb = (int)((n + chunk - 1) / chunk);
  const size_t part_bytes = align_up(sizeof(double) * 8 * (size_t)nb);
  status = ws->reserve(part_bytes + align_up(sizeof(double) * 8), align_up(sizeof(double) * 8), st);
  if (status != SPROT_OK) return status;
  double* dpart = reinterpret_cast<double*>(ws->dev);
  double* dout = reinterpret_cast<double*>(ws->dev + part_bytes);
  double* hout = reinterpret_cast<double*>(ws->host);
  launch_axis_ls(P, Q, n, labels, label, chunk, nb, dpart, hint, dout, st);
  if (cudaGetLastError() != cudaSuccess) return SPROT_E_CUDA;
  if (cudaMemcpyAsync(hout, dout, sizeof(double) * 6, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return SPROT_E_CUDA;
  const int res = (int)hout[5];
  if (res != SPROT_OK) return res;
  for (int t = 0; t < 3; ++t) axis[t] = hout[t];
  if (lambda_min) *lambda_min = hout[3];
  if (count) *count = (int64_t)hout[4];
  return SPROT_OK;
}

int sprot_axis_vote_sampled(const float* P, const float* Q, int64_t n, int32_t G, int32_t J,
                            uint32_t* grid, void* stream) {
  if (!P || !Q || !grid || n < 1 || n > (int64_t)1 << 31 || !is_pow2(G) || G < SPROT_MIN_GRID ||
      G > SPROT_MAX_GRID || J < 1 || J > SPROT_MAX_SAMPLES)
    return SPROT_E_INVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return SPROT_E_CUDA;
  return launch_axis_vote_sampled(P, Q, n, G, J, grid, sm_count(dev), reinterpret_cast<cudaStream_t>(stream));
}

int sprot_select_peaks(const uint32_t* grid, int32_t G, int32_t k, float nms_deg, int32_t* cells,
                       uint32_t* counts, int32_t* n_found, void* stream) {
  if (!grid || !cells || !counts || !n_found || !is_pow2(G) || G < SPROT_MIN_GRID ||
      G > SPROT_MAX_GRID || k < 1 || k > SPROT_MAX_K || !(nms_deg >= 0.f))
    return SPROT_E_INVAL;
  return select_peaks(grid, G, k, nms_deg, cells, counts, n_found, reinterpret_cast<cudaStream_t>(stream));
}

int sprot_estimate_batch(sprot_instance* inst, int64_t m, void* stream) {
  if (!inst || m < 1) return SPROT_E_INVAL;
  std::vector<Problem> pb((size_t)m);
  for (int64_t i = 0; i < m; ++i) {
    const sprot_instance& x = inst[i];
    int st = validate(x.P, x.Q, x.n, &x.params, x.params.k);
    if (st != SPROT_OK || !x.out || (x.params.flags & SPROT_HOST_PTRS)) return SPROT_E_INVAL;
    pb[i] = Problem{x.P, x.Q, x.n, x.params, x.params.k, false, x.out, x.n_found, x.labels, nullptr, nullptr};
    if (pb[i].prm.grid == 0) pb[i].prm.grid = sprot_autotune_grid(x.n);
  }
  int st = solve(pb, reinterpret_cast<cudaStream_t>(stream));
  if (st == SPROT_OK)
    for (int64_t i = 0; i < m; ++i) inst[i].params.grid = pb[i].prm.grid;
  return st;
}

namespace sprot {
namespace {

// Median wall time (ms) of `reps` solves of probs under knobs kn, after two untimed runs (the
// second captures the launch graph that the timed runs replay). status: the first failure
// other than E_NOAXIS.
double time_plan(std::vector<Problem>& probs, cudaStream_t st, const sprot_plan_knobs& kn, int reps,
                 int* status) {
  auto run = [&]() {
    const int r = solve(probs, st, true, &kn);
    if (r != SPROT_OK && r != SPROT_E_NOAXIS && *status == SPROT_OK) *status = r;
  };
  run();
  run();
  std::vector<double> t;
  for (int r = 0; r < reps && *status == SPROT_OK; ++r) {
    const auto t0 = std::chrono::steady_clock::now();
    run();
    t.push_back(std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count());
  }
  if (t.empty()) return 0.0;
  std::sort(t.begin(), t.end());
  return t[t.size() / 2];
}

// Times every candidate (the defaults first), stores the fastest under key and returns it.
int tune(std::vector<Problem>& probs, cudaStream_t st, const std::vector<sprot_plan_knobs>& cands, int reps,
         const TuneKey& key, sprot_plan_knobs* out) {
  int status = SPROT_OK;
  sprot_plan_knobs best = cands[0];
  double best_ms = 0.0, default_ms = 0.0;
  for (size_t c = 0; c < cands.size(); ++c) {
    const double ms = time_plan(probs, st, cands[c], reps, &status);
    if (status != SPROT_OK) return status;
    if (c == 0) default_ms = ms;
    if (c == 0 || ms < best_ms) {
      best_ms = ms;
      best = cands[c];
    }
  }
  // the outputs end with the winner's results
  time_plan(probs, st, best, 1, &status);
  if (status != SPROT_OK) return status;
  best.ms_tuned = best_ms;
  best.ms_default = default_ms;
  {
    std::lock_guard<std::mutex> g(g_tune_mu);
    g_tuned[key] = best;
  }
  if (out) *out = best;
  return SPROT_OK;
}

}  // namespace
}  // namespace sprot

void sprot_default_knobs(sprot_plan_knobs* k) {
  if (k) *k = default_knobs();
}

int sprot_autotune_plan(const float* P, const float* Q, int64_t n, const sprot_params* params, int32_t reps,
                        sprot_plan_knobs* out, void* stream) {
  if (!params || reps < 1 || reps > 15) return SPROT_E_INVAL;
  int st = validate(P, Q, n, params, params->k);
  if (st != SPROT_OK) return st;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return SPROT_E_CUDA;
  std::vector<sprot_rotation> rot(std::max(params->k, 1));
  int32_t nf = 0;
  std::vector<Problem> pb(1);
  pb[0] = Problem{P, Q, n, *params, params->k, (params->flags & SPROT_HOST_PTRS) != 0, rot.data(), &nf,
                  nullptr, nullptr, nullptr};
  if (pb[0].prm.grid == 0) pb[0].prm.grid = sprot_autotune_grid(n);
  std::vector<sprot_plan_knobs> cands;
  cands.push_back(default_knobs());
  for (int r = 1; r <= 3; ++r)
    for (int d : {600, 300, 1200}) {
      sprot_plan_knobs k = default_knobs();
      k.vote_rounds = r;
      k.chunk_div = d;
      if (r != 1 || d != 600) cands.push_back(k);
    }
  return tune(pb, reinterpret_cast<cudaStream_t>(stream), cands, reps, tune_key(dev, false, n, pb[0].prm.grid), out);
}

int sprot_autotune_batch(sprot_instance* inst, int64_t m, int32_t reps, sprot_plan_knobs* out, void* stream) {
  if (!inst || m < 2 || reps < 1 || reps > 15) return SPROT_E_INVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return SPROT_E_CUDA;
  std::vector<Problem> pb((size_t)m);
  int64_t total = 0;
  for (int64_t i = 0; i < m; ++i) {
    const sprot_instance& x = inst[i];
    int st = validate(x.P, x.Q, x.n, &x.params, x.params.k);
    if (st != SPROT_OK || !x.out || (x.params.flags & SPROT_HOST_PTRS)) return SPROT_E_INVAL;
    pb[i] = Problem{x.P, x.Q, x.n, x.params, x.params.k, false, x.out, x.n_found, x.labels, nullptr, nullptr};
    if (pb[i].prm.grid == 0) pb[i].prm.grid = sprot_autotune_grid(x.n);
    total += x.n;
  }
  std::vector<sprot_plan_knobs> cands;
  cands.push_back(default_knobs());
  for (int sl : {32768, 16384, 65535})
    for (int d : {1200, 600, 2400}) {
      sprot_plan_knobs k = default_knobs();
      k.batch_slice = sl;
      k.batch_div = d;
      if (sl != 32768 || d != 1200) cands.push_back(k);
    }
  const int st = tune(pb, reinterpret_cast<cudaStream_t>(stream), cands, reps, tune_key(dev, true, total / m, 0), out);
  if (st == SPROT_OK)
    for (int64_t i = 0; i < m; ++i) inst[i].params.grid = pb[i].prm.grid;
  return st;
}

int32_t sprot_tuned_plan(int64_t n, int32_t G, int32_t batched, sprot_plan_knobs* out) {
  sprot_plan_knobs k = default_knobs();
  int dev = 0;
  bool found = false;
  if (cudaGetDevice(&dev) == cudaSuccess) {
    cudaGetLastError();
    found = tuned_lookup(tune_key(dev, batched != 0, n, G ? G : sprot_autotune_grid(n)), &k);
  } else {
    cudaGetLastError();
  }
  if (out) *out = k;
  return found ? 1 : 0;
}

int sprot_set_tuned_plan(int64_t n, int32_t G, int32_t batched, const sprot_plan_knobs* k) {
  if (!k || n < 1 || !(k->vote_rounds >= 1 && k->vote_rounds <= 3 && k->chunk_div >= 100 && k->chunk_div <= 2400 &&
                       k->batch_slice >= 16384 && k->batch_slice <= kMaxSliceCircles && k->batch_div >= 300 &&
                       k->batch_div <= 4800))
    return SPROT_E_INVAL;
  if (!batched && G != 0 && (!is_pow2(G) || G < SPROT_MIN_GRID || G > SPROT_MAX_GRID)) return SPROT_E_INVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return SPROT_E_CUDA;
  }
  std::lock_guard<std::mutex> g(g_tune_mu);
  g_tuned[tune_key(dev, batched != 0, n, G ? G : sprot_autotune_grid(n))] = *k;
  return SPROT_OK;
}

void sprot_autotune_reset(void) {
  std::lock_guard<std::mutex> g(g_tune_mu);
  g_tuned.clear();
}

void sprot_release_stream_workspace(void* stream) { release_workspace(reinterpret_cast<cudaStream_t>(stream)); }

void sprot_release_workspaces(void) {
  std::map<std::pair<int, cudaStream_t>, std::shared_ptr<Workspace>> gone;
  {
    std::lock_guard<std::mutex> g(g_ws_mu);
    gone.swap(g_ws);
  }
  // freed here, outside the lock (a workspace still held by a call in flight: when it returns)
}

uint64_t sprot_kernel_launch_count(void) { return g_launches.load(); }

void sprot_kernel_timing(int enable) {
  std::lock_guard<std::mutex> g(g_timing_mu);
  g_timing.store(enable ? 1 : 0);
  if (enable) {
    g_vote_ms = 0.0;
    g_vote_launches = 0;
  }
}

void sprot_kernel_timing_read(double* vote_ms, uint64_t* vote_launches) {
  std::lock_guard<std::mutex> g(g_timing_mu);
  if (vote_ms) *vote_ms = g_vote_ms;
  if (vote_launches) *vote_launches = g_vote_launches;
}

int sprot_probe_smem_atomic_rate(int32_t iters, double* rate, void* stream) {
  if (!rate || iters < 1) return SPROT_E_INVAL;
  double r = probe_smem_atomics(iters, reinterpret_cast<cudaStream_t>(stream));
  if (r <= 0) return SPROT_E_CUDA;
  *rate = r;
  return SPROT_OK;
}

}  // extern "C"
