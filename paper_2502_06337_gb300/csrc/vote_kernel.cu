// Axis vote: the 2-D accumulator of Algorithm 1 (Sec. IV-A), rasterised exactly.
//
// Every correspondence i gives d = p_i - q_i; its admissible rotation axes form the great
// circle r . d = 0 (Eqs. 5-8), whose stereographic image (Eqs. 11-13, D = 0) is the zero set
// of F(u, v) = 2 d1 u + 2 d2 v + d3 (u^2 + v^2 - 1). A cell is voted when that curve meets
// the closed cell. For d3 > 0 the curve is a circle of centre (-d1, -d2)/d3 and radius
// |d|/d3 >= 1; for d3 = 0 it is a line through the origin.
//
// Rasterisation. The circle is cut at its four 45-degree points into two x-major arcs (top,
// bottom: |slope| <= 1) and two y-major arcs (left, right). Columns whose both edge lines lie
// within the x-major span are handled column by column: each lane takes one vertical grid
// line, solves F = 0 on it for the two crossings (a quadratic, in the cancellation-free
// form), and the cells of column j are the rows between the crossings on lines j and j+1
// (plus the top or bottom point of the circle in the column that holds it). The remaining
// columns are handled row by row in the same way with horizontal lines. Every column is
// owned by exactly one of the two passes, so no cell is counted twice, and each lane
// touches only one or two cells. Row/column indices are fixed up against the exact grid
// edges, so the only error is that of the crossing itself, which for these well-separated
// roots is a few float32 ulps of |d| in F.
//
// Privatisation. A CTA owns one row band of the accumulator in shared memory as 16-bit
// counters packed in pairs (columns c and c + G/2 share a 32-bit word, incremented by 1 or
// 1 << 16 with red.shared.add.u32). Rows are XOR-swizzled so that both lanes-along-columns
// and lanes-along-rows hit distinct banks. A CTA processes at most 65535 circles per item,
// so no counter overflows, then writes its band to a per-slice partial in global memory;
// the reduce kernel sums slices. Items (instance, band, slice) are taken from a global
// queue by persistent CTAs, which also serves batches of many instances.
#include "sprot_internal.h"

namespace sprot {

namespace {

constexpr unsigned kFull = 0xffffffffu;

struct Band {
  uint32_t sbase;  // shared-window address of the tile
  int G, W, swz, R0, R1;
  float step, half;
};

__device__ __forceinline__ float edgef(int k, float step) { return fmaf((float)k, step, -1.0f); }

// Roots of c3 y^2 + 2 b y + kk = 0 (c3 >= 0), lo <= hi, without cancellation: one root from
// |b| + sqrt(disc), the other from the product of the roots. c3 == 0 (inv3 = +inf) leaves
// the linear root finite and the other infinite. Returns false when there is no real root.
__device__ __forceinline__ bool qroots(float c3, float inv3, float b, float kk, float& lo,
                                       float& hi) {
  float disc = fmaf(-c3, kk, b * b);
  if (!(disc >= 0.f)) {
    lo = hi = 0.f;
    return false;
  }
  float t = fabsf(b) + sqrtf(disc);
  if (t == 0.f) {
    lo = hi = 0.f;
    return true;
  }
  float far = t * inv3;
  float nr = __fdiv_rn(kk, t);
  if (b >= 0.f) {
    lo = -far;
    hi = -nr;
  } else {
    hi = far;
    lo = nr;
  }
  return true;
}

__device__ __forceinline__ int floor_index(float y, float half, int G) {
  float s = fminf(fmaxf(fmaf(y, half, half), -4.f), (float)(G + 4));
  return (int)floorf(s);
}

// Cells k whose closed interval [e_k, e_k+1] meets [ymin, ymax].
__device__ __forceinline__ int2 cell_span(float ymin, float ymax, float half, float step, int G) {
  float s0 = fminf(fmaxf(fmaf(ymin, half, half), -4.f), (float)(G + 4));
  float s1 = fminf(fmaxf(fmaf(ymax, half, half), -4.f), (float)(G + 4));
  int a = (int)ceilf(s0) - 1;
  if (edgef(a + 1, step) < ymin) ++a;
  int b = (int)floorf(s1);
  if (edgef(b, step) > ymax) --b;
  return make_int2(a, b);
}

__device__ __forceinline__ void vote(const Band& B, int r, int c) {
  int rr = r - B.R0;
  uint32_t word = (uint32_t)(rr * B.W + ((c & (B.W - 1)) ^ (rr & B.swz)));
  uint32_t inc = c >= B.W ? 0x10000u : 1u;
  asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(B.sbase + 4u * word), "r"(inc) : "memory");
}

// Column-by-column pass over columns [j0, j1] for one x-major arc (top: upper crossing).
// jc is the column holding the circle centre, where the arc reaches yext (top or bottom).
__device__ __forceinline__ void x_pass(const Band& B, float d1x2, float d2, float d3, float inv3,
                                      int j0, int j1, bool top, int jc, float yext, int lane) {
  for (int base = j0; base <= j1; base += 31) {
    int l = base + lane;
    float x = edgef(l, B.step);
    float kk = fmaf(d3, fmaf(x, x, -1.f), d1x2 * x);
    float lo, hi;
    bool ok = qroots(d3, inv3, d2, kk, lo, hi);
    float y = top ? hi : lo;
    float yn = __shfl_down_sync(kFull, y, 1);
    bool okn = __shfl_down_sync(kFull, ok, 1);
    if (lane < 31 && l <= j1 && ok && okn) {
      float ymin = fminf(y, yn), ymax = fmaxf(y, yn);
      if (l == jc) {
        if (top)
          ymax = fmaxf(ymax, yext);
        else
          ymin = fminf(ymin, yext);
      }
      int2 rg = cell_span(ymin, ymax, B.half, B.step, B.G);
      int ra = max(rg.x, B.R0), rb = min(rg.y, B.R1 - 1);
      for (int r = ra; r <= rb; ++r) vote(B, r, l);
    }
  }
}

__device__ __forceinline__ void vote_row_piece(const Band& B, int r, int2 cg, int jA, int jB) {
  int a = max(cg.x, 0), b = min(cg.y, jA);
  for (int c = a; c <= b; ++c) vote(B, r, c);
  a = max(cg.x, jB);
  b = min(cg.y, B.G - 1);
  for (int c = a; c <= b; ++c) vote(B, r, c);
}

// Row-by-row pass over rows [i0, i1], voting only columns <= jA or >= jB (the y-major
// part). ic is the row holding the circle centre, where the arcs reach uL / uR.
__device__ __forceinline__ void y_pass(const Band& B, float d1, float d2x2, float d3, float inv3,
                                      int i0, int i1, int ic, float uL, float uR, int jA, int jB,
                                      int lane) {
  for (int base = i0; base <= i1; base += 31) {
    int l = base + lane;
    float x = edgef(l, B.step);
    float kk = fmaf(d3, fmaf(x, x, -1.f), d2x2 * x);
    float lo, hi;
    bool ok = qroots(d3, inv3, d1, kk, lo, hi);
    float lon = __shfl_down_sync(kFull, lo, 1);
    float hin = __shfl_down_sync(kFull, hi, 1);
    bool okn = __shfl_down_sync(kFull, ok, 1);
    if (lane < 31 && l <= i1 && ok && okn) {
      float umin = fminf(lo, lon), umax = fmaxf(lo, lon);
      if (l == ic) umin = fminf(umin, uL);
      vote_row_piece(B, l, cell_span(umin, umax, B.half, B.step, B.G), jA, jB);
      umin = fminf(hi, hin);
      umax = fmaxf(hi, hin);
      if (l == ic) umax = fmaxf(umax, uR);
      vote_row_piece(B, l, cell_span(umin, umax, B.half, B.step, B.G), jA, jB);
    }
  }
}

// One column interval [lo, hi] (plane coordinates, possibly infinite) of an x-major arc,
// widened by one column and clipped to [xj0, xj1].
__device__ __forceinline__ int2 col_interval(float lo, float hi, const Band& B, int xj0, int xj1) {
  if (!(lo <= hi)) return make_int2(1, 0);
  int a = floor_index(lo, B.half, B.G) - 1;
  int b = floor_index(hi, B.half, B.G) + 1;
  return make_int2(max(a, xj0), min(b, xj1));
}

// The x-major arc's columns inside the band: A \ B with A = [ap, aq], B = (br, bs); up to two
// intervals, merged when the widened pieces touch so no column is visited twice.
__device__ __forceinline__ void arc_columns(const Band& B, float ap, float aq, float br, float bs,
                                            int xj0, int xj1, int2& i1, int2& i2) {
  i1 = col_interval(ap, fminf(aq, br), B, xj0, xj1);
  i2 = col_interval(fmaxf(ap, bs), aq, B, xj0, xj1);
  if (i1.x <= i1.y && i2.x <= i2.y && i2.x <= i1.y + 1) {
    i1 = make_int2(min(i1.x, i2.x), max(i1.y, i2.y));
    i2 = make_int2(1, 0);
  }
}

__device__ void rasterise(const Band& B, float d1, float d2, float d3, int lane) {
  const int G = B.G;
  const float INF = __int_as_float(0x7f800000);
  float nd = sqrtf(fmaf(d1, d1, fmaf(d2, d2, d3 * d3)));
  float d1x2 = 2.f * d1, d2x2 = 2.f * d2;
  if (d3 <= 1e-8f * nd) {
    // A line through the origin (d3 = 0 up to a change of F below 2e-8 |d|).
    if (fabsf(d2) >= fabsf(d1)) {
      x_pass(B, d1x2, d2, 0.f, INF, 0, G - 1, true, -100, 0.f, lane);
      x_pass(B, d1x2, d2, 0.f, INF, 0, G - 1, false, -100, 0.f, lane);
    } else {
      y_pass(B, d1, d2x2, 0.f, INF, B.R0, B.R1 - 1, -100, 0.f, 0.f, G - 1, G, lane);
    }
    return;
  }
  const float inv3 = __frcp_rn(d3);
  const float s = 0.70710678f;
  // 45-degree points cx -/+ rho/sqrt(2), in cancellation-free form.
  float q1 = fmaf(d2, d2, d3 * d3) - d1 * d1;
  float uA = d1 >= 0.f ? -(d1 + s * nd) * inv3 : -0.5f * q1 / ((s * nd - d1) * d3);
  float uB = d1 <= 0.f ? (s * nd - d1) * inv3 : 0.5f * q1 / ((s * nd + d1) * d3);
  int jA = min(max(floor_index(uA, B.half, G), -1), G - 1);
  int jB = min(max(floor_index(uB, B.half, G), 0), G);
  int xj0 = max(jA + 1, 0), xj1 = min(jB - 1, G - 1);
  float cx = -d1 * inv3, cy = -d2 * inv3;
  int jc = floor_index(cx, B.half, G);
  int ic = floor_index(cy, B.half, G);
  float ybot, ytop, uL, uR;
  qroots(d3, inv3, d2, -fmaf(d1, d1, d3 * d3) * inv3, ybot, ytop);
  qroots(d3, inv3, d1, -fmaf(d2, d2, d3 * d3) * inv3, uL, uR);

  // y-major part: rows spanned by the circle left of line jA+1 and right of line jB.
  int yr0 = 1 << 30, yr1 = -(1 << 30);
  if (jA >= 0) {
    float x = edgef(jA + 1, B.step), lo, hi;
    if (qroots(d3, inv3, d2, fmaf(d3, fmaf(x, x, -1.f), d1x2 * x), lo, hi)) {
      yr0 = min(yr0, floor_index(lo, B.half, G) - 1);
      yr1 = max(yr1, floor_index(hi, B.half, G) + 1);
    }
  }
  if (jB <= G - 1) {
    float x = edgef(jB, B.step), lo, hi;
    if (qroots(d3, inv3, d2, fmaf(d3, fmaf(x, x, -1.f), d1x2 * x), lo, hi)) {
      yr0 = min(yr0, floor_index(lo, B.half, G) - 1);
      yr1 = max(yr1, floor_index(hi, B.half, G) + 1);
    }
  }
  yr0 = max(yr0, B.R0);
  yr1 = min(yr1, B.R1 - 1);
  if (yr0 <= yr1) y_pass(B, d1, d2x2, d3, inv3, yr0, yr1, ic, uL, uR, jA, jB, lane);

  // x-major part, restricted to the columns where each arc is inside the band [V0, V1].
  if (xj0 <= xj1) {
    float V0 = edgef(B.R0, B.step), V1 = edgef(B.R1, B.step);
    float a0, b0, a1, b1;
    bool ok0 = qroots(d3, inv3, d1, fmaf(d3, fmaf(V0, V0, -1.f), d2x2 * V0), a0, b0);
    bool ok1 = qroots(d3, inv3, d1, fmaf(d3, fmaf(V1, V1, -1.f), d2x2 * V1), a1, b1);
    // top arc: {u : top(u) >= V0} minus {u : top(u) > V1}
    float ap, aq, br, bs;
    if (V0 <= cy) { ap = -INF; aq = INF; }
    else if (ok0) { ap = a0; aq = b0; }
    else { ap = INF; aq = -INF; }
    if (V1 < cy) { br = -INF; bs = INF; }
    else if (ok1) { br = a1; bs = b1; }
    else { br = INF; bs = INF; }
    int2 i1, i2;
    arc_columns(B, ap, aq, br, bs, xj0, xj1, i1, i2);
    if (i1.x <= i1.y) x_pass(B, d1x2, d2, d3, inv3, i1.x, i1.y, true, jc, ytop, lane);
    if (i2.x <= i2.y) x_pass(B, d1x2, d2, d3, inv3, i2.x, i2.y, true, jc, ytop, lane);
    // bottom arc: {u : bottom(u) <= V1} minus {u : bottom(u) < V0}
    if (V1 >= cy) { ap = -INF; aq = INF; }
    else if (ok1) { ap = a1; aq = b1; }
    else { ap = INF; aq = -INF; }
    if (V0 > cy) { br = -INF; bs = INF; }
    else if (ok0) { br = a0; bs = b0; }
    else { br = INF; bs = INF; }
    arc_columns(B, ap, aq, br, bs, xj0, xj1, i1, i2);
    if (i1.x <= i1.y) x_pass(B, d1x2, d2, d3, inv3, i1.x, i1.y, false, jc, ybot, lane);
    if (i2.x <= i2.y) x_pass(B, d1x2, d2, d3, inv3, i2.x, i2.y, false, jc, ybot, lane);
  }
}

// p - q scaled by a power of two (exact) so that max |d_k| is in [1, 2), and sign-normalised
// to d3 >= 0 (F and -F have the same zero set). Returns false for p == q.
__device__ __forceinline__ bool circle_of(const float* P, const float* Q, int64_t i, float& d1,
                                          float& d2, float& d3) {
  d1 = P[3 * i] - Q[3 * i];
  d2 = P[3 * i + 1] - Q[3 * i + 1];
  d3 = P[3 * i + 2] - Q[3 * i + 2];
  float m = fmaxf(fabsf(d1), fmaxf(fabsf(d2), fabsf(d3)));
  if (m == 0.f) return false;
  int e = ilogbf(m);
  d1 = scalbnf(d1, -e);
  d2 = scalbnf(d2, -e);
  d3 = scalbnf(d3, -e);
  if (d3 < 0.f) {
    d1 = -d1;
    d2 = -d2;
    d3 = -d3;
  }
  return true;
}

__global__ void __launch_bounds__(kVoteThreads, 1)
    k_axis_vote(const VoteItem* __restrict__ items, int n_items, const InstDev* __restrict__ insts,
                int* __restrict__ counter) {
  extern __shared__ __align__(16) uint32_t tile[];
  __shared__ int s_item;
  __shared__ int s_next;
  const int lane = threadIdx.x & 31;
  for (;;) {
    if (threadIdx.x == 0) {
      s_item = atomicAdd(counter, 1);
      s_next = 0;
    }
    __syncthreads();
    const int it = s_item;
    if (it >= n_items) break;
    const VoteItem I = items[it];
    const InstDev& D = insts[I.inst];
    Band B;
    B.G = D.G;
    B.W = D.G >> 1;
    B.swz = min(B.W, 32) - 1;
    B.R0 = D.band_row0[I.band];
    B.R1 = D.band_row0[I.band + 1];
    B.step = 2.0f / (float)D.G;
    B.half = 0.5f * (float)D.G;
    B.sbase = (uint32_t)__cvta_generic_to_shared(tile);
    const int words = (B.R1 - B.R0) * B.W;
    uint4* t4 = reinterpret_cast<uint4*>(tile);
    for (int w = threadIdx.x; w < (words >> 2); w += blockDim.x) t4[w] = make_uint4(0, 0, 0, 0);
    __syncthreads();

    const float* __restrict__ P = D.P;
    const float* __restrict__ Q = D.Q;
    const int64_t count = I.c1 - I.c0;
    for (;;) {
      int base = 0;
      if (lane == 0) base = atomicAdd(&s_next, 32);
      base = __shfl_sync(kFull, base, 0);
      if (base >= count) break;
      float e1 = 0.f, e2 = 0.f, e3 = 0.f;
      bool live = false;
      if (base + lane < count) live = circle_of(P, Q, I.c0 + base + lane, e1, e2, e3);
      unsigned mask = __ballot_sync(kFull, live);
      while (mask) {
        int src = __ffs(mask) - 1;
        mask &= mask - 1;
        float d1 = __shfl_sync(kFull, e1, src);
        float d2 = __shfl_sync(kFull, e2, src);
        float d3 = __shfl_sync(kFull, e3, src);
        rasterise(B, d1, d2, d3, lane);
      }
    }
    __syncthreads();

    // Write the band to this slice's partial, undoing the row swizzle (4 words at a time).
    uint32_t* out = D.partial + ((int64_t)I.slice * D.G + B.R0) * B.W;
    const int groups = words >> 2;
    for (int g = threadIdx.x; g < groups; g += blockDim.x) {
      int rr = (g * 4) / B.W;
      int wp = (g * 4) - rr * B.W;
      int x = rr & B.swz;
      uint4 v = t4[g];
      uint32_t e[4] = {v.x, v.y, v.z, v.w};
      int lb = wp ^ (x & ~3);
      int p = x & 3;
      uint4 o;
      o.x = e[0 ^ p];
      o.y = e[1 ^ p];
      o.z = e[2 ^ p];
      o.w = e[3 ^ p];
      *reinterpret_cast<uint4*>(out + (int64_t)rr * B.W + lb) = o;
    }
    __syncthreads();
  }
}

// Shared-atomic throughput probe: conflict-free red.shared.add.u32, one per thread per
// round, on every SM.
__global__ void __launch_bounds__(1024) k_probe_atomics(int iters, uint32_t* sink) {
  __shared__ uint32_t buf[1024];
  buf[threadIdx.x] = 0;
  __syncthreads();
  uint32_t addr = (uint32_t)__cvta_generic_to_shared(buf + threadIdx.x);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 16; ++u)
      asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(addr), "r"(1u) : "memory");
  }
  __syncthreads();
  if (buf[threadIdx.x] != (uint32_t)iters * 16u) atomicAdd(sink, 1u);
}

}  // namespace

void launch_axis_vote(const VoteItem* items, int n_items, const InstDev* insts, int* counter,
                      int grid_ctas, int smem_bytes, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_axis_vote, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmemBytes);
    attr = true;
  }
  k_axis_vote<<<grid_ctas, kVoteThreads, smem_bytes, st>>>(items, n_items, insts, counter);
  launches_add(1);
}

double probe_smem_atomics(int iters, cudaStream_t st) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  uint32_t* sink = nullptr;
  if (cudaMalloc(&sink, 4) != cudaSuccess) return -1.0;
  cudaMemsetAsync(sink, 0, 4, st);
  int ctas = sms * 2;
  k_probe_atomics<<<ctas, 1024, 0, st>>>(4, sink);  // warm-up
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  cudaEventRecord(a, st);
  k_probe_atomics<<<ctas, 1024, 0, st>>>(iters, sink);
  cudaEventRecord(b, st);
  launches_add(2);
  cudaEventSynchronize(b);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, a, b);
  uint32_t bad = 0;
  cudaMemcpy(&bad, sink, 4, cudaMemcpyDeviceToHost);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaFree(sink);
  if (bad != 0 || ms <= 0.f) return -1.0;
  return (double)ctas * 1024.0 * iters * 16.0 / (ms * 1e-3);
}

}  // namespace sprot
