/*
 * sprot.h -- C ABI of the GB300-native stereographic-projection rotation vote.
 *
 * Method: "Accelerating Outlier-robust Rotation Estimation by Stereographic Projection"
 * (arXiv 2502.06337). Given point sets P = {p_i}, Q = {q_i} and n correspondences with
 * q_i = R p_i + noise for the inliers (Eq. 1), the estimator
 *   1. maps every correspondence to the great circle of admissible rotation axes
 *      {r : r . (p_i - q_i) = 0} (Eqs. 5-8), and that circle by stereographic projection
 *      from the pole (0,0,1) to a plane circle (Eqs. 11-13);
 *   2. counts, in a G x G accumulator over the square [-1,1]^2 of the plane, the circles that
 *      pass through every cell (Algorithm 1; Sec. IV-A), and takes the peak cell -- or the k
 *      best cells with non-maximum suppression for several rotations (Sec. IV-D) -- whose
 *      centre, back-projected by Eq. 12, is the axis;
 *   3. votes the per-pair rotation angle about that axis into J bins over [-pi, pi]
 *      (Algorithm 1; Sec. IV-B, Eq. 15) and takes the peak bin;
 *   4. builds R_vote by Rodrigues' formula (Eq. 2; Sec. IV-C), then refines it in FP64 by
 *      least squares on the inliers (two Kabsch/Horn solves; not part of the paper).
 *
 * Conventions shared by every entry point
 *   - P and Q are n x 3 row-major float32 arrays (x, y, z of each point). They are device
 *     pointers unless the call's flags contain SPROT_HOST_PTRS, in which case they (and the
 *     per-pair output arrays) are host pointers, copied to the device at the start of the
 *     solve. Calls with inputs in pinned host memory (cudaHostAlloc, cudaMallocHost,
 *     cudaHostRegister) are replayed from a CUDA graph keyed by the host addresses when they
 *     repeat; pageable inputs run directly. The library reads P and Q only; the caller owns
 *     them and every output buffer.
 *   - Grid cell (row, col) spans u in [-1 + 2 col/G, -1 + 2 (col+1)/G] and v likewise for
 *     row; cells are closed, so a circle on a shared edge counts in both cells. Grids are
 *     row-major uint32 [row][col].
 *   - Every call is ordered on the CUDA stream it is given (a cudaStream_t passed as void*,
 *     NULL = the legacy default stream). Calls that return results in host structs
 *     synchronise that stream before returning. (The legacy default stream cannot be
 *     captured in a CUDA graph, so a solve given it whose launch sequence is captured or
 *     replayed, a shape seen before, runs on a stream the library owns, after the work
 *     already ordered on the default stream.) Calls on one stream must not be issued
 *     concurrently from several host threads; calls on different streams may be.
 *   - Return value: SPROT_OK (0) or a negative status; sprot_status_string() describes it.
 *     On error nothing is written to the outputs except where stated.
 *   - The library allocates its own device workspace (cached per device and stream, grown on
 *     demand); sprot_release_workspaces() frees all of them, and
 *     sprot_release_stream_workspace() the one of a stream that is about to be destroyed.
 */
#ifndef SPROT_H
#define SPROT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------------------------- */
#define SPROT_OK 0
#define SPROT_E_INVAL (-1)   /* bad argument (see each entry point) */
#define SPROT_E_NOMEM (-2)   /* device or host allocation failed, or over a server budget */
#define SPROT_E_CUDA (-3)    /* a CUDA runtime call failed */
#define SPROT_E_TIMEOUT (-4) /* a bounded wait expired */
#define SPROT_E_NOAXIS (-5)  /* every accumulator cell is zero: no axis can be voted */
#define SPROT_E_UNIMPL (-6)  /* not implemented */
#define SPROT_E_BUSY (-7)    /* server queue full or shutting down */

/* ---- flags ------------------------------------------------------------------------------ */
#define SPROT_HOST_PTRS 0x1u /* P, Q and per-pair outputs are host pointers */
/* The axis of each peak is taken at its sub-cell position instead of the cell centre: along
 * each grid axis, the vertex of the parabola through the counts of the peak cell and its two
 * edge neighbours, clamped to the cell (offset 0 where the parabola does not open downwards
 * or a neighbour is off the grid). The angle vote, R_vote and the reported axis use it; the
 * gate still uses the peak's cells. The paper back-projects the cell centre (Algorithm 1,
 * Eq. 12); the offsets are reported in sprot_rotation.cell_offset with or without the flag. */
#define SPROT_SUBCELL_AXIS 0x2u

/* ---- limits ----------------------------------------------------------------------------- */
#define SPROT_MAX_K 8          /* rotations per problem */
#define SPROT_MIN_GRID 16      /* G is a power of two in [16, 2048] */
#define SPROT_MAX_GRID 2048
#define SPROT_MAX_ANGLE_BINS 4096
#define SPROT_MAX_SAMPLES 4096     /* points per circle of the sampled accumulator */
#define SPROT_MAX_BANDS 96         /* row bands of one accumulator in the axis vote */
#define SPROT_NOALLOC_SCRATCH_BYTES (40u << 20) /* fixed scratch of sprot_axis_vote_noalloc */

/* Solver parameters. The paper fixes none of them; the defaults are those of
 * sprot_default_params(). */
typedef struct sprot_params {
  int32_t grid;         /* G: accumulator side, a power of two in [16, 2048] (default 256) */
  int32_t angle_bins;   /* J: bins over [-pi, pi] (Algorithm 1), 2..4096 (default 360) */
  int32_t k;            /* rotations sought, 1..SPROT_MAX_K (default 1) */
  float nms_deg;        /* peaks closer than this (degrees, as axis lines) are suppressed */
  int32_t gate_window;  /* w: a pair votes an angle only if its circle meets the
                           (2w+1)^2 cells around the peak; -1 = every pair votes
                           (Algorithm 1 as printed). Default 1. */
  int32_t angle_window; /* a: the vote set is the voters within a bins of the peak bin
                           (circularly). Default 1. */
  double tau;           /* inlier residual threshold ||q - R p|| <= tau: the "noise level"
                           input of Algorithm 1 (default 0.05) */
  uint32_t flags;       /* SPROT_HOST_PTRS | SPROT_SUBCELL_AXIS; other bits: E_INVAL */
} sprot_params;

/* One estimated rotation. Axis/angle/R_vote are the paper's estimate (Sec. IV-C); R_init and
 * R are the FP64 least-squares refinements (first on the angle-vote set, then on the
 * residual inliers). */
typedef struct sprot_rotation {
  double R[9];          /* refined rotation, row-major */
  double R_init[9];     /* Kabsch over the angle-vote set */
  double R_vote[9];     /* Rodrigues(axis, theta) */
  double axis[3];       /* unit axis (cell centre by Eq. 12, or the sub-cell point with
                           SPROT_SUBCELL_AXIS), sign chosen so theta in [0,pi] */
  double theta;         /* bin-centre angle, radians, in [0, pi] */
  int32_t cell_row, cell_col; /* peak cell */
  int32_t angle_bin;    /* peak bin of the histogram about the canonical (r_z <= 0) axis */
  uint32_t axis_votes;  /* count of the peak cell */
  uint32_t angle_votes; /* count of the peak bin */
  uint32_t n_vote_set;  /* pairs in the angle-vote set used for R_init */
  uint32_t n_inliers;   /* pairs labelled with this rotation */
  uint32_t n_degenerate;/* pairs with p_i == q_i exactly (no circle) */
  double cell_offset[2]; /* sub-cell peak position relative to the cell centre, in cells,
                           along u (columns) and v (rows); each in [-1/2, 1/2] */
} sprot_rotation;

/* Fills the defaults listed in sprot_params. */
void sprot_default_params(sprot_params* p);

/* Text of a status code (static storage). */
const char* sprot_status_string(int status);

/* ---- whole-problem solves ----------------------------------------------------------------- */

/* Every whole-problem solve issues its copies and launches on `stream` as one sequence. With
 * device pointers (no SPROT_HOST_PTRS, no sprot_debug export) the sequence is captured once
 * per shape (sizes, item counts, workspace) as a CUDA graph and replayed on later calls. */

/* Single rotation (Algorithm 1 end to end plus refinement).
 *   P, Q         n x 3 float32 (device, or host with SPROT_HOST_PTRS)
 *   n            number of correspondences, >= 1
 *   params       non-NULL; params->k is ignored (treated as 1)
 *   out          host struct, written on success
 *   inlier_mask  n bytes (device, or host with SPROT_HOST_PTRS), 1 = inlier; may be NULL
 *   stream       cudaStream_t; synchronised before return
 * Errors: E_INVAL (NULL pointer, n < 1, bad G/J/tau), E_NOAXIS (all pairs degenerate),
 *         E_NOMEM, E_CUDA. */
int sprot_estimate_rotation(const float* P, const float* Q, int64_t n, const sprot_params* params,
                            sprot_rotation* out, uint8_t* inlier_mask, void* stream);

/* Up to params->k rotations from one accumulator (Sec. IV-D).
 *   out      host array of params->k structs; the first *n_found are written
 *   n_found  host int; number of peaks found (peaks with zero votes are not reported)
 *   labels   n int32 (device, or host with SPROT_HOST_PTRS): rotation index of each pair
 *            (smallest residual among those <= tau), -1 for outliers; may be NULL
 * Errors as sprot_estimate_rotation; also E_INVAL for k outside 1..SPROT_MAX_K. */
int sprot_estimate_rotations_k(const float* P, const float* Q, int64_t n,
                               const sprot_params* params, sprot_rotation* out, int32_t* n_found,
                               int32_t* labels, void* stream);

/* Optional intermediate outputs of a solve, for inspection and testing. Every pointer is a
 * DEVICE pointer or NULL (not written). */
typedef struct sprot_debug {
  uint32_t* grid;       /* G*G accumulator, row-major [row][col] */
  uint32_t* hist;       /* k*J angle histograms (rotation-major), about the canonical axis */
  int16_t* bins;        /* k*n: bin of each pair about each axis, -1 if it did not vote */
  uint8_t* vote_set;    /* k*n: 1 if the pair is in that rotation's angle-vote set */
} sprot_debug;

/* sprot_estimate_rotations_k plus intermediate outputs (dbg may be NULL). */
int sprot_estimate_rotations_ex(const float* P, const float* Q, int64_t n,
                                const sprot_params* params, sprot_rotation* out,
                                int32_t* n_found, int32_t* labels, const sprot_debug* dbg,
                                void* stream);

/* ---- stage entry points (device pointers only; asynchronous on the stream) -------------- */

/* Step 2, the accumulator only: grid[G*G] (device uint32) = number of circles of the
 * non-degenerate pairs passing through each closed cell (Algorithm 1; Fig. 3c). The grid is
 * overwritten, not accumulated. Errors: E_INVAL (NULL, n < 1, bad G), E_NOMEM, E_CUDA. */
int sprot_axis_vote(const float* P, const float* Q, int64_t n, int32_t grid_size,
                    uint32_t* grid, void* stream);

/* sprot_axis_vote without any allocation. The paper has no counterpart: this is a service
 * for callers that cannot allocate device memory -- code running under a host framework that
 * owns the device heap (its caching allocator, a hard memory cap), a plug-in whose memory is
 * budgeted by its host process, or a latency-critical path where an allocation may block on
 * the driver. It computes the same grid as sprot_axis_vote (the same launches and plan) but
 * takes all its scratch (work tables, queue counter, peak key and the slices' partial
 * accumulators, 2 x S x G x G/2 x 4 bytes for S slices) from one file-scope device array of
 * SPROT_NOALLOC_SCRATCH_BYTES (40 MB) that every GPU loading the library holds until the
 * process exits. It calls no cudaMalloc, cudaFree or other allocating routine. The caller
 * passes P, Q (device, n x 3 float32) and grid (device uint32[G*G], overwritten).
 * - Limit: a problem whose plan needs more scratch than the array holds is rejected with
 *   E_INVAL before anything runs. On a 152-SM GPU every n <= 2,555,865 fits for G <= 512,
 *   n <= 589,815 for G = 1024 and n <= 131,070 for G = 2048.
 * - Set-up: the first call on a device looks up the array's device address
 *   (cudaGetSymbolAddress) with that device current; make that first call before any stream
 *   capture on the device.
 * - Sharing: every call on a device uses the same array and leaves the last call's contents
 *   there; each call clears what must start at zero itself (on the device, in stream order).
 *   Calls whose work overlaps on the GPU -- on different streams or from different host
 *   threads without ordering between them -- race on the array and give wrong grids.
 * Asynchronous on the stream. Errors: E_INVAL (NULL, n < 1, bad G, plan beyond the scratch),
 * E_CUDA. */
int sprot_axis_vote_noalloc(const float* P, const float* Q, int64_t n, int32_t grid_size,
                            uint32_t* grid, void* stream);

/* The work split of the axis vote (Algorithm 1's accumulator) for n pairs on a G x G grid on
 * the current device, as a single solve (batched = 0) or a batch instance (batched = 1) would
 * use it: the pairs are cut into *slices consecutive slices of at most 65535 circles, and each
 * slice is voted band by band: *n_bands bands, band b covering rows (for the curve's caps that
 * are walked along rows) and columns (for those walked along columns) [band_row0[b],
 * band_row0[b+1]) (band_row0: host int32[SPROT_MAX_BANDS + 1]). Host-only; for tests and
 * tuning. Errors: E_INVAL (NULL, n < 1, bad G), E_CUDA (no device). */
int sprot_vote_plan(int64_t n, int32_t grid_size, int32_t batched, int32_t* n_bands,
                    int32_t* band_row0, int32_t* slices);

/* sprot_vote_plan for a device with n_sm streaming multiprocessors (1 <= n_sm <= 4096), given
 * instead of read from the current device: the same split that device would get. Pure host
 * code; makes no CUDA call, so it runs without a GPU. Errors: E_INVAL (as sprot_vote_plan, or
 * n_sm out of range). */
int sprot_vote_plan_sm(int64_t n, int32_t grid_size, int32_t batched, int32_t n_sm,
                       int32_t* n_bands, int32_t* band_row0, int32_t* slices);

/* The consensus accumulator of Eq. 9 at cell resolution: grid[G*G] (device uint32) = the
 * number of non-degenerate pairs for which some axis r of the closed cell has
 * |r . z_i| < eps, z_i = (p_i - q_i)/|p_i - q_i| (the cells within angular distance asin(eps)
 * of the pair's great circle). 0 <= eps < 1; eps = 0 gives the cells the curve crosses
 * (open test). Overwritten, not accumulated. Errors: E_INVAL (NULL, n < 1, bad G or eps),
 * E_NOMEM, E_CUDA. */
int sprot_axis_vote_eps(const float* P, const float* Q, int64_t n, int32_t grid_size, float eps,
                        uint32_t* grid, void* stream);

/* Least-squares rotation axis of a set of pairs (Eq. 10): the unit r minimising
 * sum_i (z_i . r)^2 over the non-degenerate pairs with labels[i] == label (every pair when
 * labels is NULL), z_i = (p_i - q_i)/|p_i - q_i| -- the eigenvector of S = sum_i z_i z_i^T for
 * its smallest eigenvalue. S is summed in FP64 on the device (z_i in float32) and the
 * eigenvector found by power iteration on adj(S). Used after the vote on its inliers, it
 * refines the cell-resolution axis. P, Q, labels: device pointers. hint: host double[3] or
 * NULL; r is signed so that r . hint >= 0, else r_z <= 0. axis: host double[3];
 * lambda_min (the smallest eigenvalue, the residual sum of squares) and count (pairs used):
 * host, may be NULL. Nothing is written on error. Synchronous. Errors: E_INVAL, E_NOAXIS (fewer than two independent
 * directions: the axis is not determined), E_NOMEM, E_CUDA. */
int sprot_refine_axis(const float* P, const float* Q, int64_t n, const int32_t* labels,
                      int32_t label, const double* hint, double* axis, double* lambda_min,
                      int64_t* count, void* stream);

/* Algorithm 1's accumulator taken literally (its first loop): for every non-degenerate pair
 * the great circle of z = (p - q)/|p - q| is drawn as J points alpha1 cos(t_j) +
 * alpha2 sin(t_j), t_j = -pi + 2 pi j / J (the printed second cosine read as a sine), with
 * alpha1 = the normalised component of alpha0 orthogonal to z (alpha0 = e3, or e1 when
 * p - q has zero first and second components) and alpha2 = alpha1 x z. Each point is
 * projected by Eq. 11 and, if inside the square [-1,1]^2, adds one to its cell of
 * grid[G*G] (device uint32, row = v, col = u; overwritten, not accumulated). A circle can
 * vote a cell several times and may miss a cell it only grazes. J <= SPROT_MAX_SAMPLES.
 * Errors: E_INVAL (NULL, n < 1, bad G or J), E_CUDA. */
int sprot_axis_vote_sampled(const float* P, const float* Q, int64_t n, int32_t grid_size,
                            int32_t samples, uint32_t* grid, void* stream);

/* Greedy top-k of a grid with non-maximum suppression (Sec. IV-D), on the device:
 * cells[2*i] = row, cells[2*i+1] = col, counts[i] = votes of peak i, for i < *n_found
 * (n_found a device int32). Ties go to the smallest row-major index. */
int sprot_select_peaks(const uint32_t* grid, int32_t grid_size, int32_t k, float nms_deg,
                       int32_t* cells, uint32_t* counts, int32_t* n_found, void* stream);

/* ---- batched solve ------------------------------------------------------------------------ */

/* One independent problem of a batch. P, Q, labels are device pointers. */
typedef struct sprot_instance {
  const float* P;
  const float* Q;
  int64_t n;
  sprot_params params;  /* params.grid may be 0: the autotuner picks G from n */
  sprot_rotation* out;  /* HOST array of params.k entries */
  int32_t* n_found;     /* HOST int */
  int32_t* labels;      /* device n int32, or NULL */
} sprot_instance;

/* Solves m independent problems with one set of launches over a segmented work queue
 * (persistent axis-vote kernel, per-instance accumulators), replayed from a cached CUDA
 * graph when the batch shape repeats. Results equal those of solving each instance alone
 * with the same parameters. The chosen G is written back into inst[i].params.grid when it
 * was 0 (so callers can replay an instance alone).
 * Errors: E_INVAL (m < 1 or any instance invalid; nothing is solved), E_NOMEM, E_CUDA. */
int sprot_estimate_batch(sprot_instance* inst, int64_t m, void* stream);

/* Accumulator side the autotuner picks for n pairs (used when params.grid == 0). */
int32_t sprot_autotune_grid(int64_t n);

/* ---- plan autotuning ---------------------------------------------------------------------
 * The grid side G above is chosen for accuracy (Sec. IV-A: the accumulator's resolution).
 * The knobs below change only how the work is cut, never a result's integer parts: the
 * accumulator is an exact count whatever the slicing, and the FP64 sums differ only in their
 * summation order (results within 1e-9 of the default plan's). The paper has no counterpart;
 * it is this library's speed tuning.
 *
 * sprot_autotune_plan / sprot_autotune_batch time a small candidate set of knobs on the
 * caller's own inputs on the current device and store the fastest for the input's class in a
 * process-wide table; every later solve of that class on that device (sprot_estimate_*,
 * sprot_estimate_batch and the server's batches) then uses it. Classes: one problem, by
 * (device, bit length of n, G); a batch of m instances, by (device, bit length of the mean n). */
typedef struct sprot_plan_knobs {
  int32_t vote_rounds; /* one problem: the vote's (slice x band) items fill this many rounds of
                          the SMs, 1-3 (more slices than the 16-bit counters need balance
                          uneven items; each slice costs a partial accumulator) (default 1) */
  int32_t chunk_div;   /* one problem: the per-pair passes cut the n pairs into about this many
                          items, 100-2400 (default 600) */
  int32_t batch_slice; /* batch: circles per vote slice of an instance, 16384-65535 (32768) */
  int32_t batch_div;   /* batch: the per-pair passes cut the batch's pairs into about this many
                          items, 300-4800 (default 1200) */
  double ms_tuned;     /* set by the tuner: median solve time of the winner (ms, wall clock) */
  double ms_default;   /* set by the tuner: median solve time of the default knobs (ms) */
} sprot_plan_knobs;

/* The default (untuned) knobs; ms fields 0. */
void sprot_default_knobs(sprot_plan_knobs* k);

/* Times the single solve of (P, Q, n, params) -- the arguments of sprot_estimate_rotations_k,
 * HOST_PTRS allowed -- under each candidate (vote_rounds 1-3 x chunk_div 300/600/1200: two
 * untimed runs, then the median of `reps` timed runs, reps 1-15) and stores the fastest for
 * the class of (n, G) on the current device (G: params->grid, or sprot_autotune_grid(n)).
 * *out receives the winner with both times. Errors: E_INVAL (bad arguments), E_NOMEM,
 * E_CUDA; E_NOAXIS from a solve does not stop the tuning. */
int sprot_autotune_plan(const float* P, const float* Q, int64_t n, const sprot_params* params,
                        int32_t reps, sprot_plan_knobs* out, void* stream);

/* As sprot_autotune_plan for a batch (the arguments of sprot_estimate_batch; candidates
 * batch_slice 16384/32768/65535 x batch_div 600/1200/2400), stored for the class of the
 * batch's mean n. The instances' outputs hold the last timed run's results (the winner's
 * plan, equal to any other plan's up to FP64 summation order). */
int sprot_autotune_batch(sprot_instance* inst, int64_t m, int32_t reps, sprot_plan_knobs* out, void* stream);

/* The knobs a solve on the current device would use: for one problem of n pairs on G x G
 * (batched = 0), or for a batch whose mean instance has n pairs (batched = 1, G ignored).
 * Returns 1 and the stored knobs when that class was tuned, else 0 and the defaults. */
int32_t sprot_tuned_plan(int64_t n, int32_t grid_size, int32_t batched, sprot_plan_knobs* out);

/* Stores knobs for a class on the current device, as a tuner would (for example knobs saved
 * from an earlier process's tuning). Errors: E_INVAL when a knob is outside its range above,
 * E_CUDA when there is no current device. */
int sprot_set_tuned_plan(int64_t n, int32_t grid_size, int32_t batched, const sprot_plan_knobs* k);

/* Forgets every tuned class (later solves use the defaults). */
void sprot_autotune_reset(void);

/* ---- serving ------------------------------------------------------------------------------ */

typedef struct sprot_server sprot_server;

typedef struct sprot_server_cfg {
  size_t device_budget_bytes; /* admission budget for resident request buffers (e.g. 40 GB) */
  int32_t max_batch;          /* most requests launched together (default 256) */
  int32_t max_queue;          /* most requests waiting for admission (default 65536) */
  int32_t device;             /* CUDA device ordinal */
} sprot_server_cfg;

typedef struct sprot_request {
  const float* P;       /* HOST n x 3; must stay valid until the request completes */
  const float* Q;
  int64_t n;
  sprot_params params;  /* params.grid may be 0 (autotuned) */
} sprot_request;

typedef struct sprot_result {
  int32_t status;       /* SPROT_OK or the request's error */
  int32_t n_found;
  sprot_rotation rot[SPROT_MAX_K];
  double t_submit_ms, t_admit_ms, t_done_ms; /* server clock, for latency accounting */
} sprot_result;

/* Starts a server thread that admits requests while their device buffers fit in the
 * budget, launches every admitted request together (continuous batching: requests that
 * arrive while a batch runs join the next one, which overlaps it on a second stream), and
 * completes each request independently. Errors: E_INVAL, E_NOMEM, E_CUDA. */
int sprot_server_create(const sprot_server_cfg* cfg, sprot_server** out);

/* Device bytes the server's admission counts for a request against device_budget_bytes: its
 * inputs (24 bytes a pair) and the largest workspace any plan within the autotuner's knob
 * ranges gives it, solved alone or in a batch (cfg is read for its device). 0 for a request
 * the server would reject as invalid. */
size_t sprot_server_request_bytes(const sprot_server_cfg* cfg, const sprot_request* req);

/* Queues a request; *ticket identifies it. E_NOMEM if the request alone exceeds the budget;
 * E_BUSY if the queue is full or the server is stopping; E_INVAL for bad parameters. */
int sprot_server_submit(sprot_server* s, const sprot_request* req, uint64_t* ticket);

/* Waits up to timeout_ms (-1 = forever) for a request; on completion copies its result and
 * forgets the ticket. E_TIMEOUT if not done in time (the ticket stays valid); E_INVAL for an
 * unknown ticket. */
int sprot_server_wait(sprot_server* s, uint64_t ticket, int32_t timeout_ms, sprot_result* res);

/* Drains the queue (every queued request completes), stops the thread and frees all
 * resources. */
int sprot_server_destroy(sprot_server* s);

/* ---- housekeeping and measurement ----------------------------------------------------------- */

/* Frees every cached device workspace of the calling process (device memory returned). A
 * workspace that a call on another host thread is using at that moment stays alive until that
 * call returns, and is freed then; the next call on that stream starts a new workspace. */
void sprot_release_workspaces(void);

/* Frees the cached workspace of one stream on the current device (its buffers, captured
 * graphs and events), waiting for the work it holds. Call it before destroying a stream that
 * was passed to the library; a later stream that reuses the handle starts afresh. No effect
 * when the stream has no workspace. A call still running on the stream in another host
 * thread keeps the workspace until it returns. */
void sprot_release_stream_workspace(void* stream);

/* Number of kernels this library has launched in the process (monotone counter). */
uint64_t sprot_kernel_launch_count(void);

/* Kernel timing for measurement: while enabled, CUDA events recorded on the launching stream
 * bracket every axis-vote kernel launch, and their elapsed times are accumulated (the events
 * are read when the call that launched the kernel synchronises). enable = 1 turns it on and
 * clears the totals, 0 turns it off. */
void sprot_kernel_timing(int enable);

/* Accumulated axis-vote kernel time (ms) and launch count since timing was enabled. */
void sprot_kernel_timing_read(double* vote_ms, uint64_t* vote_launches);

/* Shared-memory atomic throughput probe: every CTA of a full-chip launch performs
 * iters rounds of conflict-free 32-bit shared atomic adds (one per thread per round).
 * Writes the measured atomics per second to *rate (host double). Used to state the roofline
 * of the axis vote. Synchronises the stream. */
int sprot_probe_smem_atomic_rate(int32_t iters, double* rate, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* SPROT_H */
