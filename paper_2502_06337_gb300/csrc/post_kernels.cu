// Kernels after the axis vote: slice reduction and peak search (Sec. IV-A, IV-D), the angle
// vote (Algorithm 1 second loop; Sec. IV-B), Rodrigues (Eq. 2) and the FP64 least-squares
// refinement with labels.
#include <math_constants.h>

#include "pdl.cuh"
#include "sprot_internal.h"

namespace sprot {

namespace {

constexpr unsigned kFull = 0xffffffffu;

// (count, index) packed so that the maximum key is the largest count, then smallest index.
__device__ __forceinline__ unsigned long long peak_key(uint32_t count, uint32_t index) {
  return count ? ((unsigned long long)count << 32) | (0xffffffffu - index) : 0ull;
}

__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    unsigned long long w = __shfl_xor_sync(kFull, v, o);
    v = w > v ? w : v;
  }
  return v;
}

__device__ unsigned long long block_max_u64(unsigned long long v) {
  __shared__ unsigned long long s[32];
  v = warp_max_u64(v);
  int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) s[w] = v;
  __syncthreads();
  unsigned long long r = 0;
  if (w == 0) {
    r = l < (int)(blockDim.x >> 5) ? s[l] : 0ull;
    r = warp_max_u64(r);
  }
  __syncthreads();
  return r;  // valid in thread 0
}

// Exact axis-line geometry of a cell centre: with a = 2 col + 1 - G and b = 2 row + 1 - G the
// centre is (a, b)/G, and Eq. 12 gives r = w / N with w = (2aG, 2bG, a^2 + b^2 - G^2) and
// N = |w| = G^2 + a^2 + b^2 (all integers, exact in double for G <= 2048).
struct CellAxis {
  double w0, w1, w2, N;
};
// Eq. 12 at the plane point (a, b) / G, unnormalised: w / N is the unit axis.
__device__ __forceinline__ CellAxis axis_at(double a, double b, double g) {
  CellAxis c;
  c.w0 = 2.0 * a * g;
  c.w1 = 2.0 * b * g;
  c.w2 = a * a + b * b - g * g;
  c.N = g * g + a * a + b * b;
  return c;
}
// The axis of a cell's centre (u, v) = ((2 col + 1 - G) / G, (2 row + 1 - G) / G).
__device__ __forceinline__ CellAxis cell_axis(int G, int row, int col) {
  return axis_at(2.0 * col + 1.0 - G, 2.0 * row + 1.0 - G, (double)G);
}

// Sub-cell peak along one grid axis: the vertex of the parabola through the counts cm, c0, cp
// at offsets -1, 0, +1, i.e. (cm - cp) / (2 (cm - 2 c0 + cp)), clamped to the cell; 0 when the
// parabola does not open downwards. Integer counts make every step but the quotient exact.
__device__ __forceinline__ double parabola_vertex(uint32_t cm, uint32_t c0, uint32_t cp) {
  const double den = (double)cm - 2.0 * (double)c0 + (double)cp;
  if (!(den < 0.0)) return 0.0;
  return fmin(0.5, fmax(-0.5, 0.5 * ((double)cm - (double)cp) / den));
}

// Axis lines of two cells within the suppression radius: |r1 . r2| >= cos(radius).
__device__ __forceinline__ bool suppressed(const CellAxis& c, const CellAxis& p, double cosr) {
  double dot = fabs(c.w0 * p.w0 + c.w1 * p.w1 + c.w2 * p.w2);
  return dot >= cosr * (c.N * p.N);
}

// Sum of the slice partials of an item of accumulator words: one 16-byte column (4 words,
// 8 cells) per thread and pass, the S slices loaded several at a time, then the grid and the
// largest peak key of the item.
// Last-block election on a per-instance stage counter: every thread of the block calls it
// after its own writes (each thread fences them); the block whose arrival completes `target`
// gets true in all its threads and may then read every other block's results. No block waits
// on another: the last one to arrive does the instance's remaining work.
__device__ __forceinline__ bool last_block(uint32_t* counter, uint32_t target) {
  __shared__ uint32_t s_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(counter, 1u) + 1u == target ? 1u : 0u;
  __syncthreads();
  const bool last = s_last != 0u;
  if (last) __threadfence();
  return last;
}

// The instance's peaks (thread 0): axes by Eq. 12 at the cell centres (exact integer
// geometry), canonical r_z <= 0, and the number found.
__device__ void finalize_instance(const InstDev& D) {
  int found = 0;
  for (int a = 0; a < D.k; ++a) {
    const unsigned long long key = __ldcg(D.peak_key + a);
    if (!key) break;
    const uint32_t idx = 0xffffffffu - (uint32_t)(key & 0xffffffffu);
    const int G = D.G, row = idx / G, col = idx % G;
    DevRot& R = D.rot[a];
    // sub-cell offsets from the edge neighbours (none along an axis at the grid border)
    const uint32_t c0 = (uint32_t)(key >> 32);
    const uint32_t* g = D.grid + (int64_t)row * G + col;
    const double du = (col > 0 && col < G - 1) ? parabola_vertex(__ldcg(g - 1), c0, __ldcg(g + 1)) : 0.0;
    const double dv = (row > 0 && row < G - 1) ? parabola_vertex(__ldcg(g - G), c0, __ldcg(g + G)) : 0.0;
    R.cell_offset[0] = du;
    R.cell_offset[1] = dv;
    const CellAxis c = D.subcell ? axis_at(2.0 * col + 1.0 + 2.0 * du - G, 2.0 * row + 1.0 + 2.0 * dv - G, (double)G)
                                 : cell_axis(G, row, col);
    const double sgn = c.w2 > 0 ? -1.0 : 1.0;  // canonical: southern hemisphere, r_z <= 0
    const double r0 = sgn * c.w0 / c.N, r1 = sgn * c.w1 / c.N, r2 = sgn * c.w2 / c.N;
    R.axis[0] = r0;
    R.axis[1] = r1;
    R.axis[2] = r2;
    R.r_cell[0] = (float)r0;
    R.r_cell[1] = (float)r1;
    R.r_cell[2] = (float)r2;
    R.cell_row = row;
    R.cell_col = col;
    R.axis_votes = (uint32_t)(key >> 32);
    ++found;
  }
  *D.n_found = found;
}

// Sum of the slice partials over an item of accumulator words, 128 words (256 cells) at a time:
// the block's 8 warps take every 8th slice, each lane one 16-byte column of 4 words (the loads
// of a lane's slices are independent and issued together), then each thread adds one cell over
// the 8 warps' sums, writes it to the grid and keeps the largest peak key.
constexpr int kReduceThreads = 256;
constexpr int kReduceGroups = kReduceThreads / 32;
__global__ void __launch_bounds__(kReduceThreads)
    k_grid_reduce(const ReduceItem* __restrict__ items, const InstDev* __restrict__ insts) {
  __shared__ uint32_t part[kReduceGroups][256];
  pdl_launch_dependents();
  const ReduceItem I = items[blockIdx.x];
  const InstDev& D = insts[I.inst];
  const int G = D.G, W = G >> 1, S = D.S;
  pdl_wait();  // the partials
  const int64_t stride = (int64_t)G * W / 4;  // uint4 per slice
  const int lane = threadIdx.x & 31, grp = threadIdx.x >> 5;
  unsigned long long best = 0;
  for (int64_t w0 = I.w0; w0 < I.w1; w0 += 128) {
    const int64_t w = w0 + 4 * lane;  // words w .. w+3 (W % 4 == 0: one row)
    uint32_t c[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    if (w < I.w1) {
      const uint4* p = reinterpret_cast<const uint4*>(D.partial + w);
      int s = grp;
      for (; s + 3 * kReduceGroups < S; s += 4 * kReduceGroups) {
        uint4 v[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) v[t] = __ldcs(p + (s + t * kReduceGroups) * stride);
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          c[0] += v[t].x & 0xffffu;
          c[1] += v[t].x >> 16;
          c[2] += v[t].y & 0xffffu;
          c[3] += v[t].y >> 16;
          c[4] += v[t].z & 0xffffu;
          c[5] += v[t].z >> 16;
          c[6] += v[t].w & 0xffffu;
          c[7] += v[t].w >> 16;
        }
      }
      for (; s < S; s += kReduceGroups) {
        const uint4 v = __ldcs(p + s * stride);
        c[0] += v.x & 0xffffu;
        c[1] += v.x >> 16;
        c[2] += v.y & 0xffffu;
        c[3] += v.y >> 16;
        c[4] += v.z & 0xffffu;
        c[5] += v.z >> 16;
        c[6] += v.w & 0xffffu;
        c[7] += v.w >> 16;
      }
    }
#pragma unroll
    for (int t = 0; t < 8; ++t) part[grp][8 * lane + t] = c[t];
    __syncthreads();
    // cell t of the chunk: word w0 + t/2, column half t&1
    const int t = threadIdx.x;
    const int64_t wc = w0 + (t >> 1);
    if (wc < I.w1) {
      uint32_t v = 0;
#pragma unroll
      for (int g = 0; g < kReduceGroups; ++g) v += part[g][t];
      const int row = (int)(wc / W), col = 2 * (int)(wc - (int64_t)row * W) + (t & 1);
      D.grid[(int64_t)row * G + col] = v;
      const unsigned long long k = peak_key(v, (uint32_t)(row * G + col));
      best = k > best ? k : best;
    }
    __syncthreads();
  }
  best = block_max_u64(best);
  if (threadIdx.x == 0 && best) atomicMax(&D.peak_key[0], best);
  // the last item of the instance (of the last suppression round when k > 1) finalises
  if (D.done && last_block(&D.done[0], (uint32_t)(D.n_ritems * D.k)) && threadIdx.x == 0)
    finalize_instance(D);
}

// A peak of the accumulator (Sec. IV-D; Fig. 3d-f): no cell of the 8-neighbourhood (inside
// the grid) has a larger key, i.e. more votes, or as many at a smaller row-major index.
__device__ __forceinline__ bool is_peak(const uint32_t* __restrict__ grid, int G, int row, int col,
                                        unsigned long long key) {
  for (int dr = -1; dr <= 1; ++dr) {
    const int rr = row + dr;
    if (rr < 0 || rr >= G) continue;
    for (int dc = -1; dc <= 1; ++dc) {
      const int cc = col + dc;
      if ((dr == 0 && dc == 0) || cc < 0 || cc >= G) continue;
      if (peak_key(grid[(int64_t)rr * G + cc], (uint32_t)(rr * G + cc)) > key) return false;
    }
  }
  return true;
}

// Round `round` of the greedy top-k: the largest peak whose axis line is farther than the
// suppression radius from every axis taken in the earlier rounds.
__global__ void __launch_bounds__(256)
    k_nms_round(const ReduceItem* __restrict__ items, const InstDev* __restrict__ insts, int round) {
  pdl_launch_dependents();
  pdl_wait();  // the grid and the peak keys
  const ReduceItem I = items[blockIdx.x];
  const InstDev& D = insts[I.inst];
  if (round >= D.k) return;
  __shared__ CellAxis taken[kMaxK];
  const int G = D.G, W = G >> 1;
  if (round > 0 && D.peak_key[round - 1] == 0) {  // fewer peaks than asked for
    if (D.done && last_block(&D.done[0], (uint32_t)(D.n_ritems * D.k)) && threadIdx.x == 0)
      finalize_instance(D);
    return;
  }
  if (threadIdx.x < round) {
    unsigned long long key = D.peak_key[threadIdx.x];
    uint32_t idx = 0xffffffffu - (uint32_t)(key & 0xffffffffu);
    taken[threadIdx.x] = cell_axis(G, idx / G, idx % G);
  }
  __syncthreads();
  unsigned long long best = 0;
  // w indexes packed words; each covers cells (row, 2j) and (row, 2j + 1).
  for (int64_t w = I.w0 + threadIdx.x; w < I.w1; w += blockDim.x) {
    int row = (int)(w / W), c0 = 2 * (int)(w - (int64_t)row * W);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      int col = c0 + h;
      uint32_t cnt = D.grid[(int64_t)row * G + col];
      if (!cnt) continue;
      unsigned long long key = peak_key(cnt, (uint32_t)(row * G + col));
      if (key <= best) continue;
      CellAxis ca = cell_axis(G, row, col);
      bool sup = false;
      for (int t = 0; t < round; ++t) sup |= suppressed(ca, taken[t], D.cos_nms);
      if (!sup && is_peak(D.grid, G, row, col, key)) best = key;
    }
  }
  best = block_max_u64(best);
  if (threadIdx.x == 0 && best) atomicMax(&D.peak_key[round], best);
  if (D.done && last_block(&D.done[0], (uint32_t)(D.n_ritems * D.k)) && threadIdx.x == 0)
    finalize_instance(D);
}

// Peak bin of the histogram of rotation a, the bin-centre angle and R_vote by Rodrigues
// (Eq. 2). Called by a whole block.
__device__ void angle_peak_block(const InstDev& D, int a) {
  const int J = D.J;
  const uint32_t* h = D.hist + (int64_t)a * J;
  unsigned long long best = 0;
  for (int b = threadIdx.x; b < J; b += blockDim.x) {
    unsigned long long key = ((unsigned long long)__ldcg(h + b) << 32) | (0xffffffffu - (uint32_t)b);
    best = key > best ? key : best;
  }
  best = block_max_u64(best);
  if (threadIdx.x != 0) return;
  DevRot& R = D.rot[a];
  int b = (int)(0xffffffffu - (uint32_t)(best & 0xffffffffu));
  R.angle_bin = b;
  R.angle_votes = (uint32_t)(best >> 32);
  double th = -CUDART_PI + (b + 0.5) * (2.0 * CUDART_PI / J);
  double r0 = R.axis[0], r1 = R.axis[1], r2 = R.axis[2];
  if (th < 0) {
    th = -th;
    r0 = -r0;
    r1 = -r1;
    r2 = -r2;
  }
  R.axis[0] = r0;
  R.axis[1] = r1;
  R.axis[2] = r2;
  R.theta = th;
  double s = sin(th), c1 = 1.0 - cos(th);
  // K = [r]_x ; R = I + s K + (1 - cos) K^2, K^2 = r r^T - I
  double K[9] = {0, -r2, r1, r2, 0, -r0, -r1, r0, 0};
  double rr[3] = {r0, r1, r2};
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      R.R_vote[3 * i + j] = (i == j ? 1.0 : 0.0) + s * K[3 * i + j] +
                            c1 * (rr[i] * rr[j] - (i == j ? 1.0 : 0.0));
}

// ---- angle vote ------------------------------------------------------------------------

struct PairGeom {
  float p0, p1, p2, q0, q1, q2;
  float d1, d2, d3;  // scaled p - q
  bool deg;
};

// Raw p and q of pair i (six loads, independent of one another).
__device__ __forceinline__ void load_raw(const float* __restrict__ P, const float* __restrict__ Q, int64_t i,
                                         float* r) {
  const float* p = P + 3 * i;
  const float* q = Q + 3 * i;
  r[0] = __ldg(p);
  r[1] = __ldg(p + 1);
  r[2] = __ldg(p + 2);
  r[3] = __ldg(q);
  r[4] = __ldg(q + 1);
  r[5] = __ldg(q + 2);
}

// The pair's points and its scaled difference p - q.
__device__ __forceinline__ void pair_geom(const float* r, PairGeom& g) {
  g.p0 = r[0];
  g.p1 = r[1];
  g.p2 = r[2];
  g.q0 = r[3];
  g.q1 = r[4];
  g.q2 = r[5];
  float d1 = g.p0 - g.q0, d2 = g.p1 - g.q1, d3 = g.p2 - g.q2;
  float m = fmaxf(fabsf(d1), fmaxf(fabsf(d2), fabsf(d3)));
  g.deg = (m == 0.f);
  const float sc = inv_pow2_of(m);
  g.d1 = d1 * sc;
  g.d2 = d2 * sc;
  g.d3 = d3 * sc;
}

// min / max of c2 x^2 + c1 x over [lo, hi].
__device__ __forceinline__ void quad_range(float c2, float c1, float lo, float hi, float& mn,
                                           float& mx) {
  float flo = fmaf(c2, lo * lo, c1 * lo);
  float fhi = fmaf(c2, hi * hi, c1 * hi);
  mn = fminf(flo, fhi);
  mx = fmaxf(flo, fhi);
  // vertex -c1 / (2 c2) inside [lo, hi]: sign tests on 2 c2 x + c1 at the ends
  float sl = fmaf(2.f * c2, lo, c1), sh = fmaf(2.f * c2, hi, c1);
  if (c2 != 0.f && ((sl <= 0.f && sh >= 0.f) || (sl >= 0.f && sh <= 0.f))) {
    float fv = -0.25f * c1 * c1 / c2;
    mn = fminf(mn, fv);
    mx = fmaxf(mx, fv);
  }
}

struct Window {
  float u0, u1, v0, v1;
  float r0, r1, r2;
};

__global__ void __launch_bounds__(kStreamThreads)
    k_angle_vote(const StreamItem* __restrict__ items, const InstDev* __restrict__ insts, int J_max) {
  extern __shared__ uint32_t shist[];  // [k_found][J]
  __shared__ Window win[kMaxK];
  __shared__ int s_found;
  __shared__ unsigned s_deg;
  pdl_launch_dependents();
  const StreamItem I = items[blockIdx.x];
  const InstDev& D = insts[I.inst];
  const int J = D.J;
  // the first pair's loads (the inputs) go out before the wait for the peaks
  // the instance's fields the pair loop uses, held in registers (the loop's stores to the bins
  // would otherwise make every iteration reload them)
  const float* __restrict__ const Pp = D.P;
  const float* __restrict__ const Qp = D.Q;
  int16_t* __restrict__ const bins = D.bins;
  const int64_t nn = D.n;
  const int gw = D.w;
  float nx[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  if (I.i0 + threadIdx.x < I.i1) load_raw(Pp, Qp, I.i0 + threadIdx.x, nx);
  pdl_wait();
  if (threadIdx.x == 0) {
    s_found = *D.n_found;
    s_deg = 0;
  }
  __syncthreads();
  const int kf = s_found;
  if (threadIdx.x < kf) {
    const DevRot& R = D.rot[threadIdx.x];
    float step = 2.0f / (float)D.G;
    int w = D.w < 0 ? 0 : D.w;
    int r0 = max(R.cell_row - w, 0), r1 = min(R.cell_row + w, D.G - 1);
    int c0 = max(R.cell_col - w, 0), c1 = min(R.cell_col + w, D.G - 1);
    Window& W = win[threadIdx.x];
    W.u0 = fmaf((float)c0, step, -1.f);
    W.u1 = fmaf((float)(c1 + 1), step, -1.f);
    W.v0 = fmaf((float)r0, step, -1.f);
    W.v1 = fmaf((float)(r1 + 1), step, -1.f);
    W.r0 = R.r_cell[0];
    W.r1 = R.r_cell[1];
    W.r2 = R.r_cell[2];
  }
  for (int t = threadIdx.x; t < kf * J; t += blockDim.x) shist[t] = 0;
  __syncthreads();
  const float two_pi = 6.283185307179586f;
  const float scale = (float)J / two_pi;
  const float pi_f = 3.14159265358979f;
  unsigned ndeg = 0;
  // each thread's pairs i, i + blockDim, ...: the next pair's loads are issued before the
  // current pair is processed
  for (int64_t i = I.i0 + threadIdx.x; i < I.i1; i += blockDim.x) {
    float cur[6];
#pragma unroll
    for (int t = 0; t < 6; ++t) cur[t] = nx[t];
    if (i + blockDim.x < I.i1) load_raw(Pp, Qp, i + blockDim.x, nx);
    PairGeom g;
    pair_geom(cur, g);
    ndeg += g.deg;
    float pp = fmaf(g.p0, g.p0, fmaf(g.p1, g.p1, g.p2 * g.p2));
    float qq = fmaf(g.q0, g.q0, fmaf(g.q1, g.q1, g.q2 * g.q2));
    for (int a = 0; a < kf; ++a) {
      const Window& W = win[a];
      int bin = -1;
      if (!g.deg) {
        bool gate = true;
        if (gw >= 0) {
          float gmin, gmax, hmin, hmax;
          quad_range(g.d3, 2.f * g.d1, W.u0, W.u1, gmin, gmax);
          quad_range(g.d3, 2.f * g.d2, W.v0, W.v1, hmin, hmax);
          gate = (gmin + hmin - g.d3 <= 0.f) && (gmax + hmax - g.d3 >= 0.f);
        }
        if (gate) {
          // beta = r x p, gamma = r x q (Algorithm 1)
          float b0 = W.r1 * g.p2 - W.r2 * g.p1, b1 = W.r2 * g.p0 - W.r0 * g.p2,
                b2 = W.r0 * g.p1 - W.r1 * g.p0;
          float c0 = W.r1 * g.q2 - W.r2 * g.q1, c1 = W.r2 * g.q0 - W.r0 * g.q2,
                c2 = W.r0 * g.q1 - W.r1 * g.q0;
          float bb = fmaf(b0, b0, fmaf(b1, b1, b2 * b2));
          float cc = fmaf(c0, c0, fmaf(c1, c1, c2 * c2));
          if (bb > 1e-6f * pp && cc > 1e-6f * qq) {
            // signed angle: atan2(r . (beta x gamma), beta . gamma)
            float x0 = b1 * c2 - b2 * c1, x1 = b2 * c0 - b0 * c2, x2 = b0 * c1 - b1 * c0;
            float sn = fmaf(W.r0, x0, fmaf(W.r1, x1, W.r2 * x2));
            float cs = fmaf(b0, c0, fmaf(b1, c1, b2 * c2));
            float th = atan2f(sn, cs);
            int b = (int)floorf((th + pi_f) * scale);
            if (b >= J) b -= J;
            if (b < 0) b += J;
            bin = b;
            atomicAdd(&shist[a * J + b], 1u);
          }
        }
      }
      bins[(int64_t)a * nn + i] = (int16_t)bin;
    }
  }
  atomicAdd(&s_deg, ndeg);
  __syncthreads();
  for (int t = threadIdx.x; t < kf * J; t += blockDim.x) {
    uint32_t v = shist[t];
    if (v) atomicAdd(&D.hist[t], v);
  }
  if (threadIdx.x == 0 && s_deg) atomicAdd(D.n_deg, s_deg);
  // the last item of the instance takes the peak bins
  if (D.done && last_block(&D.done[1], (uint32_t)D.n_items)) {
    for (int a = 0; a < kf; ++a) {
      angle_peak_block(D, a);
      __syncthreads();
    }
  }
}

__device__ __noinline__ void kabsch_all(const InstDev& D, int kf, int phase);

// ---- FP64 sums of q p^T ----------------------------------------------------------------

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

// Warp sums of 16 per-lane doubles by recursive halving: at each level a lane keeps half of
// its values and adds the partner lane's copies of them, so the 16 sums cost 8 + 4 + 2 + 1 + 1
// FP64 additions per lane instead of 5 per value (FP64 instructions are scarce on this part:
// about two lanes per clock per SM). Lane l returns the total of value (l >> 1) & 15.
__device__ __forceinline__ double warp_sum16(const double (&v)[16], int lane) {
  double a8[8], a4[4], a2[2];
  const bool h16 = lane & 16, h8 = lane & 8, h4 = lane & 4, h2 = lane & 2;
#pragma unroll
  for (int j = 0; j < 8; ++j)
    a8[j] = (h16 ? v[8 + j] : v[j]) + __shfl_xor_sync(kFull, h16 ? v[j] : v[8 + j], 16);
#pragma unroll
  for (int j = 0; j < 4; ++j)
    a4[j] = (h8 ? a8[4 + j] : a8[j]) + __shfl_xor_sync(kFull, h8 ? a8[j] : a8[4 + j], 8);
#pragma unroll
  for (int j = 0; j < 2; ++j)
    a2[j] = (h4 ? a4[2 + j] : a4[j]) + __shfl_xor_sync(kFull, h4 ? a4[j] : a4[2 + j], 4);
  double a1 = (h2 ? a2[1] : a2[0]) + __shfl_xor_sync(kFull, h2 ? a2[0] : a2[1], 2);
  return a1 + __shfl_xor_sync(kFull, a1, 1);
}

// ---- float-float sums of q p^T ---------------------------------------------------------
//
// FP64 instructions run on GB300 at about two lanes per clock per SM, so the per-pair sums of
// the rotation passes are carried as unevaluated pairs of float32 (hi + lo, about 48
// significant bits), on the FP32 pipes: a product of two float32 values splits exactly into
// hi = fl(a b) and lo = a b - hi (one FMA), and two pairs add by Knuth's two-sum of the high
// parts with the low parts folded into its error term, then renormalised (Dekker's
// double-length addition). The explicitly rounded intrinsics keep the compiler from fusing or
// reassociating these steps. Only the last block's solve converts the totals to FP64.
struct FF {
  float hi, lo;
};

__device__ __forceinline__ FF ff_add(FF a, FF b) {
  const float s = __fadd_rn(a.hi, b.hi);
  const float v = __fsub_rn(s, a.hi);
  const float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, v)), __fsub_rn(b.hi, v));
  const float t = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  const float hi = __fadd_rn(s, t);
  return FF{hi, __fsub_rn(t, __fsub_rn(hi, s))};
}

__device__ __forceinline__ FF ff_prod(float a, float b) {
  const float h = __fmul_rn(a, b);
  return FF{h, fmaf(a, b, -h)};
}

__device__ __forceinline__ FF ff_shfl_xor(FF v, int o) {
  return FF{__shfl_xor_sync(kFull, v.hi, o), __shfl_xor_sync(kFull, v.lo, o)};
}

__device__ __forceinline__ double ff_to_double(FF v) { return (double)v.hi + (double)v.lo; }

// Warp sums of 16 per-lane float-float values by recursive halving (as warp_sum16). Lane l
// returns the total of value (l >> 1) & 15.
__device__ __forceinline__ FF warp_sum16_ff(const FF (&v)[16], int lane) {
  FF a8[8], a4[4], a2[2];
  const bool h16 = lane & 16, h8 = lane & 8, h4 = lane & 4, h2 = lane & 2;
#pragma unroll
  for (int j = 0; j < 8; ++j) a8[j] = ff_add(h16 ? v[8 + j] : v[j], ff_shfl_xor(h16 ? v[j] : v[8 + j], 16));
#pragma unroll
  for (int j = 0; j < 4; ++j) a4[j] = ff_add(h8 ? a8[4 + j] : a8[j], ff_shfl_xor(h8 ? a8[j] : a8[4 + j], 8));
#pragma unroll
  for (int j = 0; j < 2; ++j) a2[j] = ff_add(h4 ? a4[2 + j] : a4[j], ff_shfl_xor(h4 ? a4[j] : a4[2 + j], 4));
  const FF a1 = ff_add(h2 ? a2[1] : a2[0], ff_shfl_xor(h2 ? a2[0] : a2[1], 2));
  return ff_add(a1, ff_shfl_xor(a1, 1));
}

// Block sum of acc[K][10] into out[kf][10] (fixed order: warps in index order). All threads
// call; the rotation loop is unrolled so that acc stays in registers.
template <int K>
__device__ __forceinline__ void block_sums(FF (&acc)[K][10], int kf, float2* out) {
  __shared__ FF s[kStreamThreads / 32][10];
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
#pragma unroll
  for (int a = 0; a < K; ++a) {
    if (a >= kf) break;
    FF v16[16];
#pragma unroll
    for (int t = 0; t < 16; ++t) v16[t] = t < 10 ? acc[a][t] : FF{0.f, 0.f};
    const FF tot = warp_sum16_ff(v16, l);
    if ((l & 1) == 0 && (l >> 1) < 10) s[w][l >> 1] = tot;
    __syncthreads();
    if (threadIdx.x < 10) {
      FF v{0.f, 0.f};
      for (int i = 0; i < (int)(blockDim.x >> 5); ++i) v = ff_add(v, s[i][threadIdx.x]);
      out[a * 10 + threadIdx.x] = make_float2(v.hi, v.lo);
    }
    __syncthreads();
  }
}

// q p^T of pair i added to acc[0..8] (each float32 product split exactly into hi + lo).
__device__ __forceinline__ void add_qpT(FF* acc, const float* __restrict__ P, const float* __restrict__ Q,
                                        int64_t i) {
  const float p[3] = {__ldg(P + 3 * i), __ldg(P + 3 * i + 1), __ldg(P + 3 * i + 2)};
  const float q[3] = {__ldg(Q + 3 * i), __ldg(Q + 3 * i + 1), __ldg(Q + 3 * i + 2)};
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) acc[3 * r + c] = ff_add(acc[3 * r + c], ff_prod(q[r], p[c]));
}

// Per-warp queues of selected pairs, one per rotation: a pair is queued (as its offset in the
// work item) when selected, and each time a queue holds 32 pairs the whole warp adds them, so
// that the sums run over full warps.
template <int K>
struct PairQueues {
  FF acc[K][10];
  int len[K];    // warp-uniform queue lengths
  int total[K];  // warp-uniform counts of selected pairs
  int* q;        // this warp's queues: [K][64] in shared memory

  __device__ __forceinline__ void init(int* warp_q) {
    q = warp_q;
#pragma unroll
    for (int a = 0; a < K; ++a) {
      len[a] = total[a] = 0;
#pragma unroll
      for (int t = 0; t < 10; ++t) acc[a][t] = FF{0.f, 0.f};
    }
  }
  // Queue pair i0 + off for rotation a if sel (called by the whole warp with a uniform a).
  __device__ __forceinline__ void push(int A, bool sel, int off, const float* __restrict__ P,
                                      const float* __restrict__ Q, int64_t i0, int lane) {
    const unsigned bal = __ballot_sync(kFull, sel);
    if (!bal) return;
    const int pos = len[A] + __popc(bal & ((1u << lane) - 1u));
    if (sel) q[A * 64 + pos] = off;
    len[A] += __popc(bal);
    total[A] += __popc(bal);
    if (len[A] >= 32) {
      __syncwarp();
      add_qpT(acc[A], P, Q, i0 + q[A * 64 + lane]);
      const int rest = len[A] - 32;
      const int moved = lane < rest ? q[A * 64 + 32 + lane] : 0;
      __syncwarp();
      if (lane < rest) q[A * 64 + lane] = moved;
      __syncwarp();
      len[A] = rest;
    }
  }
  __device__ __forceinline__ void flush(const float* __restrict__ P, const float* __restrict__ Q, int64_t i0,
                                       int lane) {
    __syncwarp();
#pragma unroll
    for (int a = 0; a < K; ++a)
      if (lane < len[a]) add_qpT(acc[a], P, Q, i0 + q[a * 64 + lane]);
    // the pair count travels in slot 9, once per warp (exact in float32: at most an item's pairs)
#pragma unroll
    for (int a = 0; a < K; ++a) acc[a][9] = FF{lane == 0 ? (float)total[a] : 0.f, 0.f};
  }
};

// four blocks per SM: the once-per-instance Kabsch epilogue may spill, the pair loop does not
template <int K>
__global__ void __launch_bounds__(kStreamThreads, 4)
    k_vote_set_sum(const StreamItem* __restrict__ items, const InstDev* __restrict__ insts) {
  pdl_launch_dependents();
  pdl_wait();  // the angle peaks and the pairs' bins
  const StreamItem I = items[blockIdx.x];
  const InstDev& D = insts[I.inst];
  __shared__ int bhat[kMaxK];
  __shared__ int s_found;
  __shared__ int queues[kStreamThreads / 32][K * 64];
  if (threadIdx.x == 0) s_found = *D.n_found;
  __syncthreads();
  const int kf = s_found;
  if (threadIdx.x < kf) bhat[threadIdx.x] = D.rot[threadIdx.x].angle_bin;
  __syncthreads();
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  PairQueues<K> pq;
  pq.init(queues[wp]);
  const int J = D.J, window = D.window;
  // the instance's fields the pair loop uses, held in registers (the loop's stores would
  // otherwise make every iteration reload them)
  const float* __restrict__ const Pp = D.P;
  const float* __restrict__ const Qp = D.Q;
  const int16_t* __restrict__ const bins = D.bins;
  uint8_t* __restrict__ const vset = D.vote_set;
  const int64_t nn = D.n;
  // each warp takes 32 consecutive pairs per iteration; the next iteration's bins are loaded
  // before the current ones are used
  int nb[K];
#pragma unroll
  for (int a = 0; a < K; ++a) nb[a] = (a < kf && I.i0 + 32 * wp + lane < I.i1) ? bins[(int64_t)a * nn + I.i0 + 32 * wp + lane] : -1;
  for (int64_t base = I.i0 + 32 * wp; base < I.i1; base += blockDim.x) {
    const int64_t i = base + lane;
    const bool valid = i < I.i1;
    int cb[K];
#pragma unroll
    for (int a = 0; a < K; ++a) {
      cb[a] = nb[a];
      nb[a] = (a < kf && i + blockDim.x < I.i1) ? bins[(int64_t)a * nn + i + blockDim.x] : -1;
    }
#pragma unroll
    for (int a = 0; a < K; ++a) {
      if (a >= kf) break;
      bool in = false;
      if (valid) {
        const int b = cb[a];
        if (b >= 0) {
          int dd = b - bhat[a];
          if (dd < 0) dd = -dd;
          dd = min(dd, J - dd);
          in = dd <= window;
        }
        if (vset) vset[(int64_t)a * nn + i] = in;
      }
      pq.push(a, in, (int)(i - I.i0), Pp, Qp, I.i0, lane);
    }
  }
  pq.flush(Pp, Qp, I.i0, lane);
  block_sums(pq.acc, kf, D.msum + ((int64_t)(blockIdx.x - D.item0) * D.k) * 10);
  // the last item of the instance solves the vote-set rotations
  if (D.done && last_block(&D.done[2], (uint32_t)D.n_items))
    kabsch_all(D, kf, 0);
}

// Residual labels against every R_init (float32 test of ||q - R p||^2 <= tau^2) and the
// FP64 sums of each label class.
template <int K>
__global__ void __launch_bounds__(kStreamThreads, 4)
    k_label_sum(const StreamItem* __restrict__ items, const InstDev* __restrict__ insts) {
  pdl_launch_dependents();
  const StreamItem I = items[blockIdx.x];
  const InstDev& D = insts[I.inst];
  __shared__ float Rf[kMaxK][9];
  __shared__ int s_found;
  __shared__ int queues[kStreamThreads / 32][K * 64];
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  // each warp takes 32 consecutive pairs per iteration; the next iteration's loads are issued
  // before the current pairs are processed (the first before the wait for R_init)
  // the instance's fields the pair loop uses, held in registers (the loop's stores would
  // otherwise make every iteration reload them)
  const float* __restrict__ const Pp = D.P;
  const float* __restrict__ const Qp = D.Q;
  int32_t* __restrict__ const labels = D.labels;
  uint8_t* __restrict__ const mask = D.mask;
  float nx[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  if (I.i0 + 32 * wp + lane < I.i1) load_raw(Pp, Qp, I.i0 + 32 * wp + lane, nx);
  pdl_wait();
  if (threadIdx.x == 0) s_found = *D.n_found;
  __syncthreads();
  const int kf = s_found;
  if (threadIdx.x < kf * 9) Rf[threadIdx.x / 9][threadIdx.x % 9] = D.rot[threadIdx.x / 9].R_init_f[threadIdx.x % 9];
  __syncthreads();
  PairQueues<K> pq;
  pq.init(queues[wp]);
  const float tau2 = D.tau * D.tau;
  for (int64_t base = I.i0 + 32 * wp; base < I.i1; base += blockDim.x) {
    const int64_t i = base + lane;
    const bool valid = i < I.i1;
    float cur[6];
#pragma unroll
    for (int t = 0; t < 6; ++t) cur[t] = nx[t];
    if (i + blockDim.x < I.i1) load_raw(Pp, Qp, i + blockDim.x, nx);
    int lab = -1;
    if (valid) {
      const float p0 = cur[0], p1 = cur[1], p2 = cur[2];
      const float q0 = cur[3], q1 = cur[4], q2 = cur[5];
      float best = CUDART_INF_F;
      for (int a = 0; a < kf; ++a) {
        const float* R = Rf[a];
        const float e0 = q0 - fmaf(R[0], p0, fmaf(R[1], p1, R[2] * p2));
        const float e1 = q1 - fmaf(R[3], p0, fmaf(R[4], p1, R[5] * p2));
        const float e2 = q2 - fmaf(R[6], p0, fmaf(R[7], p1, R[8] * p2));
        const float r2 = fmaf(e0, e0, fmaf(e1, e1, e2 * e2));
        if (r2 <= tau2 && r2 < best) {
          best = r2;
          lab = a;
        }
      }
      if (labels) labels[i] = lab;
      if (mask) mask[i] = lab >= 0;
    }
#pragma unroll
    for (int a = 0; a < K; ++a) {
      if (a >= kf) break;
      pq.push(a, lab == a, (int)(i - I.i0), Pp, Qp, I.i0, lane);
    }
  }
  pq.flush(Pp, Qp, I.i0, lane);
  block_sums(pq.acc, kf, D.msum + ((int64_t)D.n_items + (blockIdx.x - D.item0)) * D.k * 10);
  // the last item of the instance solves the refined rotations
  if (D.done && last_block(&D.done[3], (uint32_t)D.n_items))
    kabsch_all(D, kf, 1);
}

// ---- FP64 rotation from the sums (Horn's unit-quaternion method) --------------------------

// Eigen-decomposition of a symmetric N x N matrix by cyclic Jacobi rotations (each rotation
// zeroes one off-diagonal entry; the sweeps converge quadratically). On return A is diagonal
// to working precision (the eigenvalues on the diagonal) and the columns of V are the unit
// eigenvectors.
template <int N>
__device__ void jacobi_sym(double (&A)[N][N], double (&V)[N][N]) {
  for (int i = 0; i < N; ++i)
    for (int j = 0; j < N; ++j) V[i][j] = (i == j) ? 1.0 : 0.0;
  for (int sweep = 0; sweep < 24; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int i = 0; i < N; ++i)
      for (int j = 0; j < N; ++j) {
        tot += A[i][j] * A[i][j];
        if (i != j) off += A[i][j] * A[i][j];
      }
    if (off <= 1e-28 * tot || off == 0.0) break;
    for (int p = 0; p < N - 1; ++p)
      for (int q = p + 1; q < N; ++q) {
        double apq = A[p][q];
        if (apq == 0.0) continue;
        double theta = (A[q][q] - A[p][p]) / (2.0 * apq);
        double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
        double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < N; ++k) {  // A <- A J
          double akp = A[k][p], akq = A[k][q];
          A[k][p] = c * akp - s * akq;
          A[k][q] = s * akp + c * akq;
        }
        for (int k = 0; k < N; ++k) {  // A <- J^T A
          double apk = A[p][k], aqk = A[q][k];
          A[p][k] = c * apk - s * aqk;
          A[q][k] = s * apk + c * aqk;
        }
        for (int k = 0; k < N; ++k) {
          double vkp = V[k][p], vkq = V[k][q];
          V[k][p] = c * vkp - s * vkq;
          V[k][q] = s * vkp + c * vkq;
        }
      }
  }
}

// The unit eigenvector of the largest eigenvalue of a symmetric 4x4 matrix.
__device__ void jacobi4_top(double A[4][4], double v[4]) {
  double M[4][4], V[4][4];
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) M[i][j] = A[i][j];
  jacobi_sym<4>(M, V);
  int best = 0;
  for (int i = 1; i < 4; ++i)
    if (M[i][i] > M[best][best]) best = i;
  double n = 0.0;
  for (int i = 0; i < 4; ++i) n += V[i][best] * V[i][best];
  n = sqrt(n);
  for (int i = 0; i < 4; ++i) v[i] = V[i][best] / n;
}

// Rotation maximising tr(R^T M) for M = sum q p^T: Horn's 4x4 matrix of S = M^T (S_ab =
// sum p_a q_b), whose top eigenvector is the unit quaternion of the rotation p -> q.
__device__ void horn_rotation(const double* M, double* R) {
  double Sxx = M[0], Sxy = M[3], Sxz = M[6];
  double Syx = M[1], Syy = M[4], Syz = M[7];
  double Szx = M[2], Szy = M[5], Szz = M[8];
  double N[4][4] = {
      {Sxx + Syy + Szz, Syz - Szy, Szx - Sxz, Sxy - Syx},
      {Syz - Szy, Sxx - Syy - Szz, Sxy + Syx, Szx + Sxz},
      {Szx - Sxz, Sxy + Syx, -Sxx + Syy - Szz, Syz + Szy},
      {Sxy - Syx, Szx + Sxz, Syz + Szy, -Sxx - Syy + Szz}};
  double q[4];
  jacobi4_top(N, q);
  double w = q[0], x = q[1], y = q[2], z = q[3];
  R[0] = w * w + x * x - y * y - z * z;
  R[1] = 2 * (x * y - w * z);
  R[2] = 2 * (x * z + w * y);
  R[3] = 2 * (x * y + w * z);
  R[4] = w * w - x * x + y * y - z * z;
  R[5] = 2 * (y * z - w * x);
  R[6] = 2 * (x * z - w * y);
  R[7] = 2 * (y * z + w * x);
  R[8] = w * w - x * x - y * y + z * z;
}

// Rotation maximising tr(R^T M) when det M > 0: the orthogonal polar factor of M (M = U S V^T
// gives U V^T, which is Kabsch's solution with no reflection to correct). Scaled Newton
// iteration X <- (g X + X^{-T} / g) / 2 with g = sqrt(|X^{-1}|_F / |X|_F) (Higham), converging
// quadratically; X^{-T} is the cofactor matrix over the determinant. Returns false (R not
// written) when M is singular or reflecting to working precision.
__device__ bool polar_rotation(const double* M, double* R) {
  double X[9];
  double n2 = 0.0;
  for (int t = 0; t < 9; ++t) n2 += M[t] * M[t];
  if (!(n2 > 0.0)) return false;
  const double inv = 1.0 / sqrt(n2);
  for (int t = 0; t < 9; ++t) X[t] = M[t] * inv;
  for (int it = 0; it < 40; ++it) {
    const double C[9] = {X[4] * X[8] - X[5] * X[7], X[5] * X[6] - X[3] * X[8], X[3] * X[7] - X[4] * X[6],
                         X[2] * X[7] - X[1] * X[8], X[0] * X[8] - X[2] * X[6], X[1] * X[6] - X[0] * X[7],
                         X[1] * X[5] - X[2] * X[4], X[2] * X[3] - X[0] * X[5], X[0] * X[4] - X[1] * X[3]};
    const double det = X[0] * C[0] + X[1] * C[1] + X[2] * C[2];
    double xn = 0.0, cn = 0.0;
    for (int t = 0; t < 9; ++t) {
      xn += X[t] * X[t];
      cn += C[t] * C[t];
    }
    if (it == 0 && !(det > 1e-9 * xn * sqrt(xn))) return false;  // singular or reflecting
    const double g = sqrt(sqrt(cn / xn) / fabs(det));
    const double a = 0.5 * g, b = 0.5 / (g * det);
    double diff = 0.0;
    for (int t = 0; t < 9; ++t) {
      const double y = a * X[t] + b * C[t];
      diff += (y - X[t]) * (y - X[t]);
      X[t] = y;
    }
    if (diff < 1e-30) break;
  }
  for (int t = 0; t < 9; ++t) R[t] = X[t];
  return true;
}

// Rotation matrix of a unit quaternion (w, x, y, z), row-major.
__device__ __forceinline__ void quat_to_rot(const double* q, double* R) {
  const double w = q[0], x = q[1], y = q[2], z = q[3];
  R[0] = w * w + x * x - y * y - z * z;
  R[1] = 2 * (x * y - w * z);
  R[2] = 2 * (x * z + w * y);
  R[3] = 2 * (x * y + w * z);
  R[4] = w * w - x * x + y * y - z * z;
  R[5] = 2 * (y * z - w * x);
  R[6] = 2 * (x * z - w * y);
  R[7] = 2 * (y * z + w * x);
  R[8] = w * w - x * x - y * y + z * z;
}

// Start value of the polar factor: scaled Newton iteration in float32 on X (|X|_F = 1,
// det X > 0), then Shepperd's quaternion of the result (largest of the trace and the diagonal
// chooses the stable formula). Returns false if float32 cannot carry the iteration.
__device__ bool polar_start_f32(const double* Xd, double* q) {
  float X[9];
  for (int t = 0; t < 9; ++t) X[t] = (float)Xd[t];
  for (int it = 0; it < 30; ++it) {
    const float C[9] = {X[4] * X[8] - X[5] * X[7], X[5] * X[6] - X[3] * X[8], X[3] * X[7] - X[4] * X[6],
                        X[2] * X[7] - X[1] * X[8], X[0] * X[8] - X[2] * X[6], X[1] * X[6] - X[0] * X[7],
                        X[1] * X[5] - X[2] * X[4], X[2] * X[3] - X[0] * X[5], X[0] * X[4] - X[1] * X[3]};
    const float det = X[0] * C[0] + X[1] * C[1] + X[2] * C[2];
    float xn = 0.f, cn = 0.f;
    for (int t = 0; t < 9; ++t) {
      xn += X[t] * X[t];
      cn += C[t] * C[t];
    }
    if (!(det > 0.f) || !(xn > 0.f)) return false;
    const float g = sqrtf(sqrtf(cn / xn) / det);
    const float a = 0.5f * g, b = 0.5f / (g * det);
    float diff = 0.f;
    for (int t = 0; t < 9; ++t) {
      const float y = fmaf(a, X[t], b * C[t]);
      diff += (y - X[t]) * (y - X[t]);
      X[t] = y;
    }
    if (diff < 1e-12f) break;
  }
  const float tr = X[0] + X[4] + X[8];
  float w, x, y, z;
  if (tr >= X[0] && tr >= X[4] && tr >= X[8]) {
    w = 0.5f * sqrtf(fmaxf(1.f + tr, 0.f));
    const float f = 0.25f / w;
    x = (X[7] - X[5]) * f;
    y = (X[2] - X[6]) * f;
    z = (X[3] - X[1]) * f;
  } else if (X[0] >= X[4] && X[0] >= X[8]) {
    x = 0.5f * sqrtf(fmaxf(1.f + X[0] - X[4] - X[8], 0.f));
    const float f = 0.25f / x;
    w = (X[7] - X[5]) * f;
    y = (X[1] + X[3]) * f;
    z = (X[2] + X[6]) * f;
  } else if (X[4] >= X[8]) {
    y = 0.5f * sqrtf(fmaxf(1.f - X[0] + X[4] - X[8], 0.f));
    const float f = 0.25f / y;
    w = (X[2] - X[6]) * f;
    x = (X[1] + X[3]) * f;
    z = (X[5] + X[7]) * f;
  } else {
    z = 0.5f * sqrtf(fmaxf(1.f - X[0] - X[4] + X[8], 0.f));
    const float f = 0.25f / z;
    w = (X[3] - X[1]) * f;
    x = (X[2] + X[6]) * f;
    y = (X[5] + X[7]) * f;
  }
  const double qn = sqrt((double)w * w + (double)x * x + (double)y * y + (double)z * z);
  if (!(qn > 0.5)) return false;
  q[0] = w / qn;
  q[1] = x / qn;
  q[2] = y / qn;
  q[3] = z / qn;
  return true;
}

// Polar factor of X (det X > 0, entries of order 1) from the unit quaternion q0 of a nearby
// rotation, in float32: the Cayley steps of the FP64 refinement below (the symmetric part H of
// U^T X, the solve (tr(H) I - H) w = v for the antisymmetric residual v, q <- q (1, w/2)) carried
// out entirely in float32. Each step squares the error until float32 rounding (about 1e-7)
// limits it; from a start within a few degrees three steps reach it. Returns false (q not
// written) if the system is not positive definite or the steps do not settle.
__device__ bool polar_cayley_f32(const double* Xd, const float* q0, double* q) {
  float X[9];
  for (int t = 0; t < 9; ++t) X[t] = (float)Xd[t];
  float a = q0[0], b = q0[1], c = q0[2], d = q0[3];
  float n2 = 1.f;
  int it = 0;
  for (; it < 8 && n2 >= 1e-13f; ++it) {
    // U = |q|^2 x the rotation of q
    const float U[9] = {a * a + b * b - c * c - d * d, 2.f * (b * c - a * d), 2.f * (b * d + a * c),
                        2.f * (b * c + a * d), a * a - b * b + c * c - d * d, 2.f * (c * d - a * b),
                        2.f * (b * d - a * c), 2.f * (c * d + a * b), a * a - b * b - c * c + d * d};
    float Y[9];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) Y[3 * i + j] = fmaf(U[i], X[j], fmaf(U[3 + i], X[3 + j], U[6 + i] * X[6 + j]));
    const float v0 = Y[7] - Y[5], v1 = Y[2] - Y[6], v2 = Y[3] - Y[1];
    const float a00 = Y[4] + Y[8], a11 = Y[0] + Y[8], a22 = Y[0] + Y[4];
    const float a01 = -0.5f * (Y[1] + Y[3]), a02 = -0.5f * (Y[2] + Y[6]), a12 = -0.5f * (Y[5] + Y[7]);
    const float c00 = a11 * a22 - a12 * a12, c11 = a00 * a22 - a02 * a02, c22 = a00 * a11 - a01 * a01;
    const float c01 = a02 * a12 - a01 * a22, c02 = a01 * a12 - a02 * a11, c12 = a01 * a02 - a00 * a12;
    const float det = a00 * c00 + a01 * c01 + a02 * c02;
    if (!(det > 0.f) || !(a00 > 0.f)) return false;
    const float inv = 0.5f * __frcp_rn(det);  // half of w: the Cayley vector
    const float w0 = (c00 * v0 + c01 * v1 + c02 * v2) * inv;
    const float w1 = (c01 * v0 + c11 * v1 + c12 * v2) * inv;
    const float w2 = (c02 * v0 + c12 * v1 + c22 * v2) * inv;
    n2 = w0 * w0 + w1 * w1 + w2 * w2;
    const float na = a - b * w0 - c * w1 - d * w2, nb = a * w0 + b + c * w2 - d * w1;
    const float nc = a * w1 - b * w2 + c + d * w0, nd = a * w2 + b * w1 - c * w0 + d;
    // renormalise (the step scales |q| by sqrt(1 + |w|^2))
    const float rn = rsqrtf(na * na + nb * nb + nc * nc + nd * nd);
    a = na * rn;
    b = nb * rn;
    c = nc * rn;
    d = nd * rn;
  }
  if (!(n2 < 1e-10f)) return false;
  q[0] = a;
  q[1] = b;
  q[2] = c;
  q[3] = d;
  return true;
}

// Polar factor of X (det X > 0) refined from the quaternion q of a nearby rotation U. The
// polar factor is the rotation U with U^T X symmetric. Writing the correction as U exp([w]x)
// and keeping first-order terms, with Y = U^T X and H its symmetric part,
// [w]x H + H [w]x = [(tr(H) I - H) w]x gives (tr(H) I - H) w = v, v = (Y21 - Y12, Y02 - Y20,
// Y10 - Y01). The step is applied as the Cayley rotation of w: q <- q (1, w/2). Only v (the
// residual that the iteration drives to zero) and the quaternion are carried in FP64; H and
// the 3 x 3 solve need no more than float32, whose relative error in w only adds a factor
// 1 + 1e-7 cond to the quadratic convergence. q is left unnormalised until the end (a scale
// of U scales v and H alike and leaves w unchanged). The loop ends after the step whose
// correction has |w|^2 < 1e-13: the error left is then of the order of |w|^2 + 1e-7 cond |w|,
// about 1e-13 rad, four orders below the 1e-9 to which the rotations are held. From a
// float32-accurate start (|w| about 1e-7) that is the first step; each FP64 instruction of a
// single thread costs tens of cycles on this part, so the step that would only confirm it is
// not taken. Returns false if the system is not positive definite or no step settled within
// four.
__device__ bool polar_refine_f64(const double* X, double* q, double* R) {
  float Xf[9];
  for (int t = 0; t < 9; ++t) Xf[t] = (float)X[t];
  float n2 = 1.f;
  for (int it = 0; it < 4 && n2 >= 1e-13f; ++it) {
    quat_to_rot(q, R);  // |q|^2 times a rotation
    // v in FP64
    const double v0 = (R[2] * X[1] + R[5] * X[4] + R[8] * X[7]) - (R[1] * X[2] + R[4] * X[5] + R[7] * X[8]);
    const double v1 = (R[0] * X[2] + R[3] * X[5] + R[6] * X[8]) - (R[2] * X[0] + R[5] * X[3] + R[8] * X[6]);
    const double v2 = (R[1] * X[0] + R[4] * X[3] + R[7] * X[6]) - (R[0] * X[1] + R[3] * X[4] + R[6] * X[7]);
    // H and the solve in float32
    float Rf[9], Yf[9];
    for (int t = 0; t < 9; ++t) Rf[t] = (float)R[t];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j)
        Yf[3 * i + j] = fmaf(Rf[i], Xf[j], fmaf(Rf[3 + i], Xf[3 + j], Rf[6 + i] * Xf[6 + j]));
    const float a00 = Yf[4] + Yf[8], a11 = Yf[0] + Yf[8], a22 = Yf[0] + Yf[4];
    const float a01 = -0.5f * (Yf[1] + Yf[3]), a02 = -0.5f * (Yf[2] + Yf[6]), a12 = -0.5f * (Yf[5] + Yf[7]);
    const float c00 = a11 * a22 - a12 * a12, c11 = a00 * a22 - a02 * a02, c22 = a00 * a11 - a01 * a01;
    const float c01 = a02 * a12 - a01 * a22, c02 = a01 * a12 - a02 * a11, c12 = a01 * a02 - a00 * a12;
    const float det = a00 * c00 + a01 * c01 + a02 * c02;
    if (!(det > 0.f) || !(a00 > 0.f)) return false;
    const float inv = 0.5f / det;  // half of w: the Cayley vector
    const float fv0 = (float)v0, fv1 = (float)v1, fv2 = (float)v2;
    const float w0 = (c00 * fv0 + c01 * fv1 + c02 * fv2) * inv;
    const float w1 = (c01 * fv0 + c11 * fv1 + c12 * fv2) * inv;
    const float w2 = (c02 * fv0 + c12 * fv1 + c22 * fv2) * inv;
    n2 = w0 * w0 + w1 * w1 + w2 * w2;
    // q <- q (1, w) in FP64
    const double a = q[0], b = q[1], c = q[2], d = q[3];
    const double x0 = w0, x1 = w1, x2 = w2;
    q[0] = a - b * x0 - c * x1 - d * x2;
    q[1] = a * x0 + b + c * x2 - d * x1;
    q[2] = a * x1 - b * x2 + c + d * x0;
    q[3] = a * x2 + b * x1 - c * x0 + d;
  }
  const double rn = 1.0 / sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  for (int t = 0; t < 4; ++t) q[t] *= rn;
  quat_to_rot(q, R);
  return n2 < 1e-13f;
}

// phase 0: R_init from the vote-set sums; phase 1: R from the label sums, for rotation a of
// the instance. Called by a whole block (the last block of the sum kernel). The item partials
// are summed in a fixed order: thread t adds items t, t + blockDim, ...; then each warp adds
// some of the ten quantities over the threads; thread 0 solves for the rotation. A dependent
// FP64 operation costs tens of cycles on this part, so the chains are kept short: the
// singularity test needs no square root and X is M scaled by a power of two (the polar factor
// does not depend on the scale).
// Unit quaternion (w, x, y, z) of a rotation matrix, row-major, by Shepperd's method (the
// largest of the trace and the diagonal picks the stable formula); float32 output.
__device__ void rot_to_quat(const double* M, float* q) {
  const double tr = M[0] + M[4] + M[8];
  double w, x, y, z;
  if (tr >= M[0] && tr >= M[4] && tr >= M[8]) {
    w = 0.5 * sqrt(fmax(1.0 + tr, 0.0));
    const double f = 0.25 / w;
    x = (M[7] - M[5]) * f;
    y = (M[2] - M[6]) * f;
    z = (M[3] - M[1]) * f;
  } else if (M[0] >= M[4] && M[0] >= M[8]) {
    x = 0.5 * sqrt(fmax(1.0 + M[0] - M[4] - M[8], 0.0));
    const double f = 0.25 / x;
    w = (M[7] - M[5]) * f;
    y = (M[1] + M[3]) * f;
    z = (M[2] + M[6]) * f;
  } else if (M[4] >= M[8]) {
    y = 0.5 * sqrt(fmax(1.0 - M[0] + M[4] - M[8], 0.0));
    const double f = 0.25 / y;
    w = (M[2] - M[6]) * f;
    x = (M[1] + M[3]) * f;
    z = (M[5] + M[7]) * f;
  } else {
    z = 0.5 * sqrt(fmax(1.0 - M[0] - M[4] + M[8], 0.0));
    const double f = 0.25 / z;
    w = (M[3] - M[1]) * f;
    x = (M[2] + M[6]) * f;
    y = (M[5] + M[7]) * f;
  }
  q[0] = (float)w;
  q[1] = (float)x;
  q[2] = (float)y;
  q[3] = (float)z;
}

// The FP64 rotation of rotation a from its ten sums (M = sum q p^T and the count): the polar
// factor of M (float32 start, FP64 refinement), with the Jacobi fallbacks for reflecting or
// rank-deficient sums. One thread.
__device__ void solve_rotation(const InstDev& D, int a, int phase, const double* tot) {
  double s[10];
#pragma unroll
  for (int t = 0; t < 10; ++t) s[t] = tot[t];
  DevRot& R = D.rot[a];
  double out[9];
  bool q_set = false;  // R.q_init written from the refined quaternion
  const uint32_t cnt = (uint32_t)s[9];
  if (cnt == 0) {
    const double* fb = phase == 0 ? R.R_vote : R.R_init;
    for (int t = 0; t < 9; ++t) out[t] = fb[t];
  } else {
    // det M > 1e-9 |M|_F^3 (polar path) tested as det > 0 and det^2 > 1e-18 (|M|_F^2)^3
    const double c0 = s[4] * s[8] - s[5] * s[7], c1 = s[5] * s[6] - s[3] * s[8], c2 = s[3] * s[7] - s[4] * s[6];
    const double det = s[0] * c0 + s[1] * c1 + s[2] * c2;
    const double n2 = (s[0] * s[0] + s[1] * s[1] + s[2] * s[2]) + (s[3] * s[3] + s[4] * s[4] + s[5] * s[5]) +
                      (s[6] * s[6] + s[7] * s[7] + s[8] * s[8]);
    // X = M 2^-e with the largest |entry| in [1, 2), exact, by integer arithmetic on the
    // exponent fields (entries that would fall below the normal range become 0)
    int emax = 0;
    for (int t = 0; t < 9; ++t) emax = max(emax, (int)((__double_as_longlong(s[t]) >> 52) & 0x7ff));
    const int e = emax - 1023;
    double X[9];
    for (int t = 0; t < 9; ++t) {
      const long long b = __double_as_longlong(s[t]);
      X[t] = (int)((b >> 52) & 0x7ff) - e > 0 ? __longlong_as_double(b - ((long long)e << 52)) : 0.0;
    }
    double q[4];
    // the start: the nearby rotation the previous stage found (R_vote for the vote set, R_init for
    // the inliers), carried to float32 precision by float32 Cayley steps; the scaled Newton
    // iteration when those do not settle
    float q0[4];
    if (phase == 0) {
      float sh, ch;
      sincosf(0.5f * (float)R.theta, &sh, &ch);
      q0[0] = ch;
      q0[1] = sh * (float)R.axis[0];
      q0[2] = sh * (float)R.axis[1];
      q0[3] = sh * (float)R.axis[2];
    } else {
      for (int t = 0; t < 4; ++t) q0[t] = R.q_init[t];
    }
    const bool ok = det > 0.0 && det * det > 1e-18 * (n2 * n2 * n2) && e > -1000 && e < 1000 &&
                    (polar_cayley_f32(X, q0, q) || polar_start_f32(X, q)) && polar_refine_f64(X, q, out);
    if (ok && phase == 0) {
      for (int t = 0; t < 4; ++t) R.q_init[t] = (float)q[t];
      q_set = true;
    }
    if (!ok && !polar_rotation(s, out)) horn_rotation(s, out);  // reflecting or rank-deficient sums
  }
  if (phase == 0) {
    for (int t = 0; t < 9; ++t) {
      R.R_init[t] = out[t];
      R.R_init_f[t] = (float)out[t];
    }
    R.n_vote_set = cnt;
    if (!q_set) rot_to_quat(out, R.q_init);
  } else {
    for (int t = 0; t < 9; ++t) R.R[t] = out[t];
    R.n_inliers = cnt;
    R.n_degenerate = *D.n_deg;
  }
}

// The sums of every rotation of an instance are reduced in turn by the whole block (a fixed
// order); then the rotations' polar solves, each a single-thread FP64 dependency chain, run
// concurrently, rotation a on lane 0 of warp a.
static_assert(kStreamThreads / 32 >= kMaxK, "one warp per rotation");
__device__ __noinline__ void kabsch_all(const InstDev& D, int kf, int phase) {
  __shared__ FF part[kStreamThreads][10];
  __shared__ double tot[kMaxK][10];
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int a = 0; a < kf; ++a) {
    FF v[10];
#pragma unroll
    for (int t = 0; t < 10; ++t) v[t] = FF{0.f, 0.f};
    const float2* base = D.msum + ((int64_t)phase * D.n_items * D.k + a) * 10;
    for (int it = threadIdx.x; it < D.n_items; it += blockDim.x) {
      const float2* src = base + (int64_t)it * D.k * 10;
#pragma unroll
      for (int t = 0; t < 10; ++t) {
        const float2 x = __ldcg(src + t);
        v[t] = ff_add(v[t], FF{x.x, x.y});
      }
    }
#pragma unroll
    for (int t = 0; t < 10; ++t) part[threadIdx.x][t] = v[t];
    __syncthreads();
    for (int col = w; col < 10; col += nw) {
      FF x{0.f, 0.f};
      for (int i = l; i < (int)blockDim.x; i += 32) x = ff_add(x, part[i][col]);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) x = ff_add(x, ff_shfl_xor(x, o));
      if (l == 0) tot[a][col] = ff_to_double(x);
    }
    __syncthreads();
  }
  if (l == 0 && w < kf) solve_rotation(D, w, phase, tot[w]);
  __syncthreads();
}

// ---- least-squares axis of a set of pairs (Eq. 10) ---------------------------------------

constexpr int kAxisThreads = 256;

// S = sum z z^T (6 distinct entries, FP64) over the selected non-degenerate pairs of one chunk,
// z = (p - q)/|p - q| in float32 (its products are exact in FP64). Pairs are queued per warp
// and summed over full warps only, as in the rotation sums. partial[block] = 6 sums + count.
__global__ void __launch_bounds__(kAxisThreads)
    k_axis_sums(const float* __restrict__ P, const float* __restrict__ Q, int64_t n,
                const int32_t* __restrict__ labels, int label, int chunk, double* __restrict__ partial) {
  __shared__ int queue[kAxisThreads / 32][64];
  __shared__ double red[kAxisThreads / 32][7];
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  const int64_t i0 = (int64_t)blockIdx.x * chunk, i1 = n < i0 + chunk ? n : i0 + chunk;
  double acc[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  int len = 0, total = 0;
  auto add = [&](int64_t i) {
    float d1 = __ldg(P + 3 * i) - __ldg(Q + 3 * i);
    float d2 = __ldg(P + 3 * i + 1) - __ldg(Q + 3 * i + 1);
    float d3 = __ldg(P + 3 * i + 2) - __ldg(Q + 3 * i + 2);
    const float sc = inv_pow2_of(fmaxf(fabsf(d1), fmaxf(fabsf(d2), fabsf(d3))));
    d1 *= sc;
    d2 *= sc;
    d3 *= sc;
    const float r = rsqrtf(fmaf(d1, d1, fmaf(d2, d2, d3 * d3)));
    const double z1 = d1 * r, z2 = d2 * r, z3 = d3 * r;
    acc[0] = fma(z1, z1, acc[0]);
    acc[1] = fma(z1, z2, acc[1]);
    acc[2] = fma(z1, z3, acc[2]);
    acc[3] = fma(z2, z2, acc[3]);
    acc[4] = fma(z2, z3, acc[4]);
    acc[5] = fma(z3, z3, acc[5]);
  };
  for (int64_t base = i0 + 32 * wp; base < i1; base += blockDim.x) {
    const int64_t i = base + lane;
    bool sel = false;
    if (i < i1 && (!labels || labels[i] == label)) {
      sel = __ldg(P + 3 * i) != __ldg(Q + 3 * i) || __ldg(P + 3 * i + 1) != __ldg(Q + 3 * i + 1) ||
            __ldg(P + 3 * i + 2) != __ldg(Q + 3 * i + 2);
    }
    const unsigned bal = __ballot_sync(kFull, sel);
    if (!bal) continue;
    const int pos = len + __popc(bal & ((1u << lane) - 1u));
    if (sel) queue[wp][pos] = (int)(i - i0);
    len += __popc(bal);
    total += __popc(bal);
    if (len >= 32) {
      __syncwarp();
      add(i0 + queue[wp][lane]);
      const int rest = len - 32;
      const int moved = lane < rest ? queue[wp][32 + lane] : 0;
      __syncwarp();
      if (lane < rest) queue[wp][lane] = moved;
      __syncwarp();
      len = rest;
    }
  }
  __syncwarp();
  if (lane < len) add(i0 + queue[wp][lane]);
  double v16[16];
#pragma unroll
  for (int t = 0; t < 16; ++t) v16[t] = t < 6 ? acc[t] : 0.0;
  const double tot = warp_sum16(v16, lane);
  if ((lane & 1) == 0 && (lane >> 1) < 6) red[wp][lane >> 1] = tot;
  if (lane == 0) red[wp][6] = (double)total;
  __syncthreads();
  if (threadIdx.x < 7) {
    double v = 0.0;
    for (int w = 0; w < kAxisThreads / 32; ++w) v += red[w][threadIdx.x];
    partial[(int64_t)blockIdx.x * 8 + threadIdx.x] = v;
  }
}

// Sum of the partials (fixed order) and the eigenvector of S for its smallest eigenvalue, by
// cyclic Jacobi rotations in FP64 (converged to working precision whatever the eigen-gap).
// The axis is undetermined when S has rank <= 1 (adj(S) vanishes relative to trace(S)^2).
// out = axis[3], lambda_min, count, status.
__global__ void __launch_bounds__(kAxisThreads)
    k_axis_eig(const double* __restrict__ partial, int nb, double h0, double h1, double h2, int has_hint,
               double* __restrict__ out) {
  __shared__ double part[kAxisThreads][7];
  __shared__ double tot[7];
  {
    double v[7] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    for (int b = threadIdx.x; b < nb; b += blockDim.x)
#pragma unroll
      for (int t = 0; t < 7; ++t) v[t] += partial[(int64_t)b * 8 + t];
#pragma unroll
    for (int t = 0; t < 7; ++t) part[threadIdx.x][t] = v[t];
  }
  __syncthreads();
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (w < 7) {
    double v = 0.0;
    for (int i = l; i < kAxisThreads; i += 32) v += part[i][w];
    v = warp_sum_d(v);
    if (l == 0) tot[w] = v;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  const double s00 = tot[0], s01 = tot[1], s02 = tot[2], s11 = tot[3], s12 = tot[4], s22 = tot[5];
  out[4] = tot[6];
  const double A[9] = {s11 * s22 - s12 * s12, s02 * s12 - s01 * s22, s01 * s12 - s02 * s11,
                       s02 * s12 - s01 * s22, s00 * s22 - s02 * s02, s01 * s02 - s00 * s12,
                       s01 * s12 - s02 * s11, s01 * s02 - s00 * s12, s00 * s11 - s01 * s01};
  double best = 0.0;
  for (int k = 0; k < 3; ++k) best = fmax(best, A[k] * A[k] + A[3 + k] * A[3 + k] + A[6 + k] * A[6 + k]);
  const double tr = s00 + s11 + s22;
  // fewer than two independent directions: adj(S) vanishes (relative to trace(S)^2)
  if (!(best > 1e-24 * (tr * tr) * (tr * tr))) {
    out[5] = (double)SPROT_E_NOAXIS;
    return;
  }
  double E[3][3] = {{s00, s01, s02}, {s01, s11, s12}, {s02, s12, s22}}, V[3][3];
  jacobi_sym<3>(E, V);
  int lo = 0;
  for (int k = 1; k < 3; ++k)
    if (E[k][k] < E[lo][lo]) lo = k;
  const double rn = 1.0 / sqrt(V[0][lo] * V[0][lo] + V[1][lo] * V[1][lo] + V[2][lo] * V[2][lo]);
  double r0 = V[0][lo] * rn, r1 = V[1][lo] * rn, r2 = V[2][lo] * rn;
  bool flip;
  if (has_hint) {
    flip = r0 * h0 + r1 * h1 + r2 * h2 < 0.0;
  } else {  // r_z <= 0 (then r_y, r_x for ties at zero)
    flip = r2 != 0.0 ? r2 > 0.0 : (r1 != 0.0 ? r1 > 0.0 : r0 > 0.0);
  }
  if (flip) {
    r0 = -r0;
    r1 = -r1;
    r2 = -r2;
  }
  out[0] = r0;
  out[1] = r1;
  out[2] = r2;
  // Rayleigh quotient: the smallest eigenvalue
  out[3] = r0 * (s00 * r0 + s01 * r1 + s02 * r2) + r1 * (s01 * r0 + s11 * r1 + s12 * r2) +
           r2 * (s02 * r0 + s12 * r1 + s22 * r2);
  out[5] = (double)SPROT_OK;
}

// Peaks of a caller grid as (row, col) pairs and counts (stage entry point).
__global__ void k_write_peaks(const InstDev* __restrict__ insts, int32_t* cells, uint32_t* counts,
                              int32_t* n_found) {
  const InstDev& D = insts[0];
  int found = 0;
  for (int a = 0; a < D.k; ++a) {
    unsigned long long key = D.peak_key[a];
    if (!key) break;
    uint32_t idx = 0xffffffffu - (uint32_t)(key & 0xffffffffu);
    cells[2 * a] = idx / D.G;
    cells[2 * a + 1] = idx % D.G;
    counts[a] = (uint32_t)(key >> 32);
    ++found;
  }
  *n_found = found;
}

}  // namespace

void launch_write_peaks(const InstDev* insts, int32_t* cells, uint32_t* counts, int32_t* n_found,
                        cudaStream_t st) {
  k_write_peaks<<<1, 1, 0, st>>>(insts, cells, counts, n_found);
  launches_add(1);
}

void launch_grid_reduce(const ReduceItem* items, int n_items, const InstDev* insts,
                        cudaStream_t st) {
  launch_dependent(k_grid_reduce, n_items, kReduceThreads, 0, st, items, insts);
  launches_add(1);
}

void launch_nms_round(const ReduceItem* items, int n_items, const InstDev* insts, int round,
                      cudaStream_t st) {
  launch_dependent(k_nms_round, n_items, 256, 0, st, items, insts, round);
  launches_add(1);
}

void launch_angle_vote(const StreamItem* items, int n_items, const InstDev* insts, int max_k,
                       int max_J, cudaStream_t st) {
  size_t smem = (size_t)max_k * max_J * sizeof(uint32_t);
  if (smem > 48 * 1024) ensure_dynamic_smem(reinterpret_cast<const void*>(k_angle_vote), (int)smem);
  launch_dependent(k_angle_vote, n_items, kStreamThreads, smem, st, items, insts, max_J);
  launches_add(1);
}

void launch_vote_set_sum(const StreamItem* items, int n_items, const InstDev* insts, int max_k,
                         cudaStream_t st) {
  if (max_k <= 1)
    launch_dependent(k_vote_set_sum<1>, n_items, kStreamThreads, 0, st, items, insts);
  else if (max_k <= 2)
    launch_dependent(k_vote_set_sum<2>, n_items, kStreamThreads, 0, st, items, insts);
  else if (max_k <= 4)
    launch_dependent(k_vote_set_sum<4>, n_items, kStreamThreads, 0, st, items, insts);
  else
    launch_dependent(k_vote_set_sum<kMaxK>, n_items, kStreamThreads, 0, st, items, insts);
  launches_add(1);
}

void launch_label_sum(const StreamItem* items, int n_items, const InstDev* insts, int max_k,
                      cudaStream_t st) {
  if (max_k <= 1)
    launch_dependent(k_label_sum<1>, n_items, kStreamThreads, 0, st, items, insts);
  else if (max_k <= 2)
    launch_dependent(k_label_sum<2>, n_items, kStreamThreads, 0, st, items, insts);
  else if (max_k <= 4)
    launch_dependent(k_label_sum<4>, n_items, kStreamThreads, 0, st, items, insts);
  else
    launch_dependent(k_label_sum<kMaxK>, n_items, kStreamThreads, 0, st, items, insts);
  launches_add(1);
}

void launch_axis_ls(const float* P, const float* Q, int64_t n, const int32_t* labels, int label, int chunk,
                    int nb, double* partial, const double* hint, double* out, cudaStream_t st) {
  k_axis_sums<<<nb, kAxisThreads, 0, st>>>(P, Q, n, labels, label, chunk, partial);
  k_axis_eig<<<1, kAxisThreads, 0, st>>>(partial, nb, hint ? hint[0] : 0.0, hint ? hint[1] : 0.0,
                                         hint ? hint[2] : 0.0, hint ? 1 : 0, out);
  launches_add(2);
}

}  // namespace sprot
