// Internal structures shared by the CUDA translation units of libsprot (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/sprot.h"

namespace sprot {

constexpr int kMaxK = SPROT_MAX_K;
constexpr int kMaxBands = SPROT_MAX_BANDS;  // row bands of one accumulator (G = 2048 needs 94)
constexpr int kStreamThreads = 256;  // threads of the per-pair kernels
constexpr int kStreamChunk = 8192;   // pairs per per-pair work item
constexpr int kReduceWords = 128;   // accumulator words per slice-reduction item (32 x uint4)
constexpr int kMaxSmemBytes = 227 * 1024 - 1024;  // tile; leaves room for static shared
constexpr int kRunSmemBytes = 227 * 1024 - 64;    // the curve vote's tiles and tables (16 B static)
constexpr int kMaxSliceCircles = 65535;  // u16 tile counters: at most this many circles/slice

// Device-side result of one rotation; mirrors sprot_rotation plus internals.
struct DevRot {
  double R[9];
  double R_init[9];
  double R_vote[9];
  double axis[3];
  double theta;
  float r_cell[3];   // canonical (r_z <= 0) cell axis in float32, used by the angle vote
  float R_init_f[9]; // R_init rounded to float32, used by the residual labels
  int32_t cell_row, cell_col, angle_bin;
  uint32_t axis_votes, angle_votes, n_vote_set, n_inliers, n_degenerate;
  double cell_offset[2];  // sub-cell peak offset (u, v) in cells
  float q_init[4];        // unit quaternion of R_init (w, x, y, z): the start of the second solve
};

// 2^-e for the binary exponent e of a finite m > 0 (from the exponent field ex: 2^(127 - ex),
// clamped to a normal number), so that m * inv_pow2_of(m) lies in [1, 2). A subnormal m
// (ex = 0) gets 2^127, which brings it into the normal range. Multiplying by it is exact, so
// every later float32 decision on the scaled values is the one on the unscaled values.
__device__ __forceinline__ float inv_pow2_of(float m) {
  const int ex = min((__float_as_int(m) >> 23) & 0xff, 253);
  return __int_as_float((254 - ex) << 23);
}

// One problem of a (possibly single-element) batch, as the kernels see it.
struct InstDev {
  const float* P;  // device memory (the caller's, or the workspace copy of host inputs)
  const float* Q;
  int64_t n;
  int32_t G, J, k, w, window;
  int32_t n_bands, S;            // bands and partial slices of the axis vote (the curve vote
                                 // writes two partials per slice of circles: rows, columns)
  int32_t subcell;               // axis at the sub-cell peak (SPROT_SUBCELL_AXIS)
  float tau;
  double cos_nms;                // cosine of the suppression radius between axis lines
  int32_t band_row0[kMaxBands + 1];
  // workspace
  uint32_t* partial;             // [S][G][G/2] u16 pairs (columns 2j and 2j+1 share a word)
  uint32_t* grid;                // [G][G]
  unsigned long long* peak_key;  // [k] packed (count, ~index) maxima
  uint32_t* hist;                // [k][J]
  int16_t* bins;                 // [k][n]
  float2* msum;                  // [2][n_items][k][10]: 9 sums of q p^T and a count, each a
                                 // float-float (hi, lo)
  int32_t item0, n_items;        // this instance's per-pair work items
  int32_t* n_found;              // device int
  uint32_t* n_deg;               // device count of degenerate pairs
  DevRot* rot;                   // [k]
  int32_t* labels;               // [n] (caller or workspace)
  uint8_t* vote_set;             // [k][n] or null
  uint8_t* mask;                 // [n] 1 = labelled inlier, or null
  // per-stage arrival counters (zeroed per solve; null: no fused epilogues): [0] slice
  // reduction and suppression rounds, [1] angle vote, [2] vote-set sums, [3] label sums
  uint32_t* done;
  int32_t n_ritems;              // this instance's slice-reduction items
};

struct VoteItem {
  int32_t inst, band, slice;
  int32_t kind;    // curve vote: 0 the row caps of band `band` of rows, 1 the column caps of band
                   // `band` of columns (the same band edges); the eps-band vote: 0
  int64_t c0, c1;  // circle range [c0, c1)
};

struct StreamItem {
  int32_t inst, pad;
  int64_t i0, i1;
};

struct ReduceItem {
  int32_t inst, pad;
  int64_t w0, w1;  // packed-word range of the grid
};

// One problem of a solve() call. Pointers are device pointers unless host_io is set.
struct Problem {
  const float* P;
  const float* Q;
  int64_t n;
  sprot_params prm;
  int k;
  bool host_io;
  sprot_rotation* out;    // host, k entries
  int32_t* n_found;       // host
  int32_t* labels;        // per-pair labels (device, or host if host_io), may be null
  uint8_t* mask;          // per-pair inlier mask (device, or host if host_io), may be null
  const sprot_debug* dbg; // device debug outputs, may be null
};

// Solves the problems (validated by the caller) with one launch sequence on st and waits for
// the results. Returns SPROT_OK, or for a single problem SPROT_E_NOAXIS when it has no peak.
// graphs: replay the launch sequence from a CUDA graph when its shape repeats (see runtime.cu).
// force: plan knobs to use (the autotuner's trials); null: the tuned knobs of the call's class,
// else the defaults.
int solve(std::vector<Problem>& probs, cudaStream_t st, bool graphs = true,
          const sprot_plan_knobs* force = nullptr);

// The axis-vote plan of a single solve of n pairs on a G x G grid on device dev: T row bands
// (row0[T + 1]), S circle slices, the largest band tile in bytes and the device's SM count.
bool single_vote_plan(int64_t n, int G, int dev, int* T, int32_t* row0, int* S, int* tile, int* nsm,
                      int64_t max_slices = INT64_MAX);

// Frees the solve() workspace of stream st (call before destroying st).
void release_workspace(cudaStream_t st);

// Device bytes one problem may occupy in a solve() workspace on device dev (inputs excluded):
// the most that any plan within the autotuner's knob ranges takes, alone or in a batch.
size_t problem_footprint(int64_t n, int G, int J, int k, int dev);

// ---- launchers -------------------------------------------------------------------------
// Axis vote (vote_runs.cu). tile_bytes: the largest band's two tiles (4 G bytes per row); the
// kernel adds its per-warp circle tables and per-lane dummy vote words (vote_run_table_bytes())
// to the dynamic shared memory.
int vote_run_table_bytes();
void launch_axis_vote_runs(const VoteItem* items, int n_items, const InstDev* insts, int* counter,
                           int grid_ctas, int tile_bytes, cudaStream_t st);
// eps-band accumulator of Eq. 9 (vote_eps.cu): same items, tiles and partials as the curve vote.
void launch_axis_vote_eps(const VoteItem* items, int n_items, const InstDev* insts, int* counter, int grid_ctas,
                          int tile_bytes, float eps, cudaStream_t st);
// Least-squares axis (post_kernels.cu): FP64 sums of z z^T over the selected pairs in nb chunks
// of `chunk` pairs into partial[nb][8], then out[6] = axis[3], lambda_min, count, status.
// hint: host double[3] or NULL.
void launch_axis_ls(const float* P, const float* Q, int64_t n, const int32_t* labels, int label, int chunk,
                    int nb, double* partial, const double* hint, double* out, cudaStream_t st);
// Algorithm 1's sampled accumulator (vote_sampled.cu): zeroes grid[G*G] and adds one per drawn
// point of every circle, J points per circle.
int launch_axis_vote_sampled(const float* P, const float* Q, int64_t n, int G, int J, uint32_t* grid,
                             int n_sm, cudaStream_t st);
// The slice reduction, suppression rounds, angle vote and FP64 sums finish each instance in the
// last block to arrive (peaks, angle peak and Rodrigues, Kabsch) when InstDev::done is set.
void launch_grid_reduce(const ReduceItem* items, int n_items, const InstDev* insts,
                        cudaStream_t st);
void launch_nms_round(const ReduceItem* items, int n_items, const InstDev* insts, int round,
                      cudaStream_t st);
void launch_write_peaks(const InstDev* insts, int32_t* cells, uint32_t* counts, int32_t* n_found,
                        cudaStream_t st);
void launch_angle_vote(const StreamItem* items, int n_items, const InstDev* insts, int max_k,
                       int max_J, cudaStream_t st);
void launch_vote_set_sum(const StreamItem* items, int n_items, const InstDev* insts, int max_k,
                         cudaStream_t st);
void launch_label_sum(const StreamItem* items, int n_items, const InstDev* insts, int max_k,
                      cudaStream_t st);
double probe_smem_atomics(int iters, cudaStream_t st);

uint64_t launches_add(uint64_t k);
// Raises `func`'s dynamic shared-memory limit to at least `bytes` on the current device, once
// per (device, function, size) and thread-safely (the launchers are called from several host
// threads).
void ensure_dynamic_smem(const void* func, int bytes);

}  // namespace sprot
