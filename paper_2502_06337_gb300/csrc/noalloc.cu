// The axis vote (the accumulator of Algorithm 1) for callers that cannot allocate device
// memory: sprot_axis_vote_noalloc.
//
// Some callers cannot call cudaMalloc or any routine that allocates. Code that runs while
// another component owns the device heap (a host framework with its own caching allocator and
// a hard memory cap), a plug-in loaded into a process whose allocations are budgeted by the
// host, and code on a real-time path where an allocation may block on the driver all need a
// call whose device memory is fixed in advance. This entry point keeps every byte of scratch
// it needs -- the instance record, the work tables, the queue counter, the peak key and the
// per-slice partial accumulators -- in one file-scope __device__ array of
// SPROT_NOALLOC_SCRATCH_BYTES, which every GPU that loads the library holds until the process
// exits. The caller passes the inputs and the output grid. The work tables are written on the
// device by a small set-up kernel, so no host staging buffer is needed either.
//
// The launches are the ones sprot_axis_vote makes, with the same plan (bands, slices, items),
// so the grid equals sprot_axis_vote's.
#include <algorithm>
#include <mutex>

#include "sprot_internal.h"

namespace sprot {

namespace {

// The shared scratch. Host code must not use this name as an address: on the host it denotes
// a host-side stand-in, so its device address is looked up once per device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[SPROT_NOALLOC_SCRATCH_BYTES];

constexpr size_t kAlignNA = 256;
inline size_t align_na(size_t x) { return (x + kAlignNA - 1) / kAlignNA * kAlignNA; }

// Everything the set-up kernel needs, by value.
struct NoallocSetup {
  InstDev inst;  // complete except for the table pointers, which the host fills in too
  int64_t n;
  int32_t T, S, n_items, n_ritems;
  int64_t words;
  VoteItem* items;
  ReduceItem* ritems;
  InstDev* inst_dev;
  int* counter;
  unsigned long long* peak;
};

// Writes the instance record and the vote and reduction items (the same order and ranges as
// the allocating path) and zeroes the queue counter and the peak key.
__global__ void k_noalloc_setup(const NoallocSetup s) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t == 0) {
    *s.inst_dev = s.inst;
    *s.counter = 0;
    *s.peak = 0ull;
  }
  if (t < s.n_items) {
    // slice sl, band b, kind kd (0: the row caps -> partial sl, 1: the column caps -> S + sl)
    const int sl = t / (2 * s.T), r = t - sl * 2 * s.T, b = r >> 1, kd = r & 1;
    s.items[t] = VoteItem{0, b, kd * s.S + sl, kd, s.n * sl / s.S, s.n * (sl + 1) / s.S};
  }
  if (t < s.n_ritems) {
    const int64_t w0 = (int64_t)t * kReduceWords;
    s.ritems[t] = ReduceItem{0, 0, w0, w0 + kReduceWords < s.words ? w0 + kReduceWords : s.words};
  }
}

std::mutex g_na_mu;
void* g_na_ptr[64] = {};

}  // namespace

}  // namespace sprot

using namespace sprot;

extern "C" int sprot_axis_vote_noalloc(const float* P, const float* Q, int64_t n, int32_t G, uint32_t* grid,
                                       void* stream) {
  if (!P || !Q || !grid || n < 1 || n > (int64_t)1 << 31 || G < SPROT_MIN_GRID || G > SPROT_MAX_GRID ||
      (G & (G - 1)) != 0)
    return SPROT_E_INVAL;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return SPROT_E_CUDA;
  int T = 0, S = 0, tile = 0, nsm = 0;
  NoallocSetup s{};
  // at most the slices whose partials (4 G^2 bytes a slice) fit the scratch beside 2 MB of tables
  const int64_t cap = ((int64_t)SPROT_NOALLOC_SCRATCH_BYTES - (2 << 20)) / (4 * (int64_t)G * G);
  if (!single_vote_plan(n, G, dev, &T, s.inst.band_row0, &S, &tile, &nsm, std::max<int64_t>(cap, 1)))
    return SPROT_E_INVAL;
  const int n_items = 2 * T * S;
  const int64_t words = (int64_t)G * (G / 2);
  const int n_ritems = (int)((words + kReduceWords - 1) / kReduceWords);
  // layout of the scratch
  size_t off = 0;
  const size_t o_inst = off;
  off = align_na(off + sizeof(InstDev));
  const size_t o_items = off;
  off = align_na(off + sizeof(VoteItem) * n_items);
  const size_t o_ritems = off;
  off = align_na(off + sizeof(ReduceItem) * n_ritems);
  const size_t o_counter = off;
  off = align_na(off + sizeof(int));
  const size_t o_peak = off;
  off = align_na(off + sizeof(unsigned long long));
  const size_t o_partial = off;
  off = align_na(off + (size_t)2 * S * words * 4);
  if (off > (size_t)SPROT_NOALLOC_SCRATCH_BYTES) return SPROT_E_INVAL;  // beyond the fixed scratch
  // the scratch's device address on this device (looked up once per device)
  char* base = nullptr;
  {
    std::lock_guard<std::mutex> g(g_na_mu);
    if (!g_na_ptr[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
        cudaGetLastError();
        return SPROT_E_CUDA;
      }
      g_na_ptr[dev] = p;
    }
    base = static_cast<char*>(g_na_ptr[dev]);
  }
  InstDev& d = s.inst;
  d.P = P;
  d.Q = Q;
  d.n = n;
  d.G = G;
  d.k = 1;
  d.n_bands = T;
  d.S = 2 * S;  // partials: the row caps' and the column caps' of every slice
  d.partial = reinterpret_cast<uint32_t*>(base + o_partial);
  d.grid = grid;
  d.peak_key = reinterpret_cast<unsigned long long*>(base + o_peak);
  d.done = nullptr;  // no fused epilogue: the reduction writes the grid and the peak key only
  s.n = n;
  s.T = T;
  s.S = S;
  s.n_items = n_items;
  s.n_ritems = n_ritems;
  s.words = words;
  s.items = reinterpret_cast<VoteItem*>(base + o_items);
  s.ritems = reinterpret_cast<ReduceItem*>(base + o_ritems);
  s.inst_dev = reinterpret_cast<InstDev*>(base + o_inst);
  s.counter = reinterpret_cast<int*>(base + o_counter);
  s.peak = reinterpret_cast<unsigned long long*>(base + o_peak);
  const int threads = 256, blocks = (std::max(n_items, n_ritems) + threads - 1) / threads;
  k_noalloc_setup<<<blocks, threads, 0, st>>>(s);
  launches_add(1);
  launch_axis_vote_runs(s.items, n_items, s.inst_dev, s.counter, std::min(n_items, nsm), tile, st);
  launch_grid_reduce(s.ritems, n_ritems, s.inst_dev, st);
  if (cudaGetLastError() != cudaSuccess) return SPROT_E_CUDA;
  return SPROT_OK;
}
