// Axis vote: the 2-D accumulator of Algorithm 1 (Sec. IV-A), rasterised exactly as runs of cells.
//
// Every correspondence i gives d = p_i - q_i; its admissible rotation axes form the great
// circle r . d = 0 (Eqs. 5-8), whose stereographic image (Eqs. 11-13, D = 0) is the zero set of
//     F(u, v) = 2 d1 u + 2 d2 v + d3 (u^2 + v^2 - 1) = f(u) + h(v) - d3,
// f(u) = d3 u^2 + 2 d1 u, h(v) = d3 v^2 + 2 d2 v. After scaling d by a power of two and choosing
// its sign so that d3 >= 0, the curve is a circle of centre (-d1, -d2)/d3 and radius |d|/d3 >= 1,
// or for d3 = 0 a line through the origin. A cell is voted when the curve meets the closed cell.
//
// Runs. Take a row strip [v_m, v_m+1] of the grid. Because F is separable, the cells of the
// strip that the curve meets are those that meet the disc {F <= 0} along the strip's wider
// chord minus those lying inside the disc along its narrower chord (the chord is the disc's
// intersection with a lattice line; the wider one is on the side of the circle's centre). With
// the wider chord [lo_w, hi_w] and the narrower one [lo_n, hi_n] (cells of the quadratic's roots
// f(u) = d3 - h(v) on the two lattice lines, taken without cancellation), the strip's cells are
// the two runs [lo_w, lo_n] and [hi_n, hi_w] -- one run [lo_w, hi_w] when the narrower line misses
// the circle, and merged when the two touch. Each run is voted as a difference: +1 at its first
// column and -1 after its last, so a row of the curve costs one quadratic and four atomics
// whatever its length. Columns are walked the same way with u and v exchanged.
//
// Which cells each orientation votes. Runs are long where the curve is flat in the walked
// direction. For a circle whose centre lies near the grid, with (ic, jc) the cell of its centre
// and M = floor(R / sqrt 2) in cells, the rows vote every cell of the rows |i - ic| >= M (the top
// and bottom caps, where the curve is flatter than 45 degrees) and the columns every cell of the
// other rows (the left and right caps): a split on integer row indices, so the orientations
// never both vote a cell. Circles whose centre lies far outside the grid (and lines) are nearly
// straight over the grid and are voted in one orientation, chosen by the direction of their
// normal. Every walk steps from the wider chord toward the narrower one (toward the cap's
// extreme), so the chord computed on the next line is always the narrower one of the strip.
//
// Work split. A work item is one slice of circles in one orientation and band: the row caps
// voted into a band of rows, or the column caps voted into a band of columns with the same
// edges. A persistent CTA takes items from a queue; for each it zeroes a shared tile of
// differences (two rows' 16-bit counters per 32-bit word for a row band, two columns' for a
// column band; one pad column or row takes the -1 of a run that ends on the grid's last cell),
// incremented with red.shared.add.u32. A warp loads 32 circles (the next 32 are loaded before
// these are walked); in phase A each lane prepares its circle for the item (the caps of the
// item's orientation, culled to where the curve crosses the band and the grid) and stores it in
// a per-warp table. In phase B the units (one strip each) of those caps are cut into segments
// of at most kSeg and dealt out in rounds, kWalkers segments per lane, walked in lock step.
// After the slice, prefix sums along the rows (or down the columns) turn the differences into
// counts, and the tile is written to the item's partial of the accumulator. The words are summed
// modulo 2^32: every count of a slice is at most its 65535 circles, so each prefix sum yields the
// exact pair of 16-bit counts.
//
// Decisions. A crossing's cell is the floor of a float32 root computed with hardware square root
// and reciprocal approximations (a few ulp). The cell differs from the exact test only when the
// root lies within rounding of a lattice line, where F at that lattice corner is within a few
// float32 roundings of zero: inside the band in which the closed-cell test may go either way.
#include <stdint.h>

#include "pdl.cuh"
#include "row_tiles.cuh"
#include "sprot_internal.h"

namespace sprot {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kRunThreads = 768;  // 24 warps
constexpr int kRunWarps = kRunThreads / 32;
constexpr int kSeg = 12;          // units per segment of phase B
constexpr int kWalkers = 1;       // walkers per lane (more lengthen each deal's longest segment)

// Per-warp circle table in shared memory, one column per lane (structure of arrays): 0 d1, 1 d2,
// 2 d3, 3-6 the unit ranges of the caps (lo | hi << 16: 0 top rows, walked up; 1 bottom rows,
// walked down; 2 left columns, walked left; 3 right columns, walked right), 7 the rows the
// column caps vote (lo | hi << 16), 8 the circle's first segment in the current deal.
constexpr int kRec = 9;
constexpr int kTab = kRec * 32;

// The work item's part of the grid: rows [R0, R1) x columns [C0, C1) (a band of rows for the
// row caps, a band of columns for the column caps) and its shared tile at byte address tb: for
// rows, (R1 - R0)/2 x RS words, RS = G + 4 (word (i, j) holds rows R0 + 2i and R0 + 2i + 1 of
// column j); for columns, (G + 1) x W words with W = (C1 - C0)/2 (word (i, j) holds columns
// C0 + 2j and C0 + 2j + 1 of row i). The extra column of a row tile and the extra row of a
// column tile take the -1 of a run that ends on the grid's last cell, so no vote tests for it;
// they are never read.
struct Band {
  int G, R0, R1, C0, C1, W;
  int RS;  // words per row pair of a row tile (G plus a pad of 4 that takes a run's end beyond the grid)
  float step, half;
  uint32_t tb;
};

__device__ __forceinline__ uint32_t range16(int lo, int hi) {  // [lo, hi) or empty
  return hi > lo ? ((uint32_t)lo | ((uint32_t)hi << 16)) : 0u;
}

__device__ __forceinline__ void red_add(uint32_t addr, uint32_t v) {
  asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}

// Hardware approximations (flush to zero): reciprocal square root and reciprocal.
__device__ __forceinline__ float rsqrt_approx(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ int cellf(float x, float half) { return __float2int_rd(fmaf(x, half, half)); }

struct Prepared {
  float d1, d2, d3;
  uint32_t cap[4], clip;
};

// Roots of C y^2 + 2 b y - T = 0 at a bounding line, the root nearer the origin and whether one
// exists (C >= 0, invC = 1/C or +inf). Cancellation-free (the far root from |b| + sqrt(disc),
// the near one from the product of the roots).
__device__ __forceinline__ bool near_root(float C, float invC, float b, float T, float& r) {
  const float disc = fmaf(C, T, b * b);
  const float t = fabsf(b) + (disc > 0.f ? disc * rsqrtf(disc) : 0.f);
  const float fr = t * invC;
  const float nr = t > 0.f ? __fdividef(T, t) : 0.f;
  const float lo = b >= 0.f ? -fr : -nr, hi = b >= 0.f ? nr : fr;
  r = fabsf(lo) < fabsf(hi) ? lo : hi;
  return disc >= 0.f;
}

// The extent [lo, hi] of w = sqrt(R^2 - x^2) for x between dmin and dmax: the offsets from the
// centre, along one axis, of the circle's points whose other coordinate lies at those distances.
__device__ __forceinline__ bool wrange(float R2, float dmin, float dmax, float& lo, float& hi) {
  if (dmin * dmin > R2) return false;
  hi = sqrtf(fmaxf(R2 - dmin * dmin, 0.f));
  lo = dmax * dmax < R2 ? sqrtf(fmaxf(R2 - dmax * dmax, 0.f)) : 0.f;
  return true;
}

// Geometry shared by the two orientations (so that they agree on which one votes each cell): a
// circle whose centre lies near the grid has its centre cell (ic, jc) and the 45-degree split
// M = floor(R / sqrt 2) in cells (rows |i - ic| >= M belong to the row caps); any other curve is
// voted by rows when |d2| >= |d1| and by columns otherwise.
struct Geo {
  float nd, invC, cu, cv, R;
  int ic, jc, M;
  bool nearc;
};

__device__ __forceinline__ Geo geo_of(float d1, float d2, float d3, float half) {
  Geo g;
  g.nd = sqrtf(fmaf(d1, d1, fmaf(d2, d2, d3 * d3)));
  g.invC = d3 > 0.f ? __frcp_rn(d3) : __int_as_float(0x7f800000);
  g.cu = g.cv = g.R = 0.f;
  g.ic = g.jc = g.M = 0;
  g.nearc = false;
  if (d3 > 0.f) {
    g.cu = -d1 * g.invC;
    g.cv = -d2 * g.invC;
    g.nearc = fabsf(g.cu) <= 4.f && fabsf(g.cv) <= 4.f;
  }
  if (g.nearc) {
    g.R = g.nd * g.invC;
    g.ic = cellf(g.cv, half);
    g.jc = cellf(g.cu, half);
    g.M = max(1, __float2int_rd(g.R * half * 0.70710678f));
  }
  return g;
}

// Phase A (one lane, one circle): the caps of its curve that this item votes (ROWS: the top and
// bottom caps within the item's rows; else the left and right caps within its columns), culled
// to where the curve crosses the item's part of the grid, with a margin of mg cells for the
// float32 error of the bounds. Exact horizontal and vertical lines (through the origin, hence
// along the grid's middle lattice lines) are voted here directly.
template <bool ROWS>
__device__ __forceinline__ void prepare(const Band& B, float d1, float d2, float d3, Prepared& S) {
  const int G = B.G;
  const float half = B.half, step = B.step;
  const int mg = 2 + (G >> 9);
#pragma unroll
  for (int c = 0; c < 4; ++c) S.cap[c] = 0u;
  S.clip = 0u;
  {
    const float nd = sqrtf(fmaf(d1, d1, fmaf(d2, d2, d3 * d3)));
    if (d3 <= 1e-8f * nd) d3 = 0.f;  // a line through the origin (F changes by under 2e-8 |d|)
  }
  S.d1 = d1;
  S.d2 = d2;
  S.d3 = d3;
  if (d3 == 0.f && (d1 == 0.f || d2 == 0.f)) {
    if (ROWS && d1 == 0.f) {  // F = 2 d2 v: the rows on both sides of v = 0, whole
      for (int r = G / 2 - 1; r <= G / 2; ++r)
        if (r >= B.R0 && r < B.R1)
          red_add(B.tb + 4u * (uint32_t)(((r - B.R0) >> 1) * B.RS), ((r - B.R0) & 1) ? 0x10000u : 1u);
    }
    if (!ROWS && d2 == 0.f) {  // F = 2 d1 u: the columns on both sides of u = 0, whole
      for (int c = G / 2 - 1; c <= G / 2; ++c)
        if (c >= B.C0 && c < B.C1) red_add(B.tb + 4u * (uint32_t)((c - B.C0) >> 1), (c & 1) ? 0x10000u : 1u);
    }
    return;
  }
  const Geo g = geo_of(d1, d2, d3, half);
  if (g.nearc) {
    const float R2 = g.R * g.R, cu = g.cu, cv = g.cv;
    float lo, hi;
    if (ROWS) {
      // the top and bottom arcs within the grid's columns u in [-1, 1]
      if (wrange(R2, fmaxf(fmaxf(-1.f - cu, cu - 1.f), 0.f), fmaxf(fabsf(-1.f - cu), fabsf(1.f - cu)), lo, hi)) {
        const int t0 = max(max(cellf(cv + lo, half) - mg, g.ic + g.M), B.R0);
        const int t1 = min(cellf(cv + hi, half) + mg, B.R1 - 1);
        const int b0 = max(cellf(cv - hi, half) - mg, B.R0);
        const int b1 = min(min(cellf(cv - lo, half) + mg, g.ic - g.M), B.R1 - 1);
        S.cap[0] = range16(t0, t1 + 1);
        S.cap[1] = range16(b0, b1 + 1);
      }
    } else {
      // the left and right arcs within the rows they vote and the item's columns
      const int clo = max(0, g.ic - g.M + 1), chi = min(G - 1, g.ic + g.M - 1);
      if (clo <= chi) {
        S.clip = (uint32_t)clo | ((uint32_t)chi << 16);
        const float Va = fmaf((float)clo, step, -1.f), Vb = fmaf((float)(chi + 1), step, -1.f);
        if (wrange(R2, fmaxf(fmaxf(Va - cv, cv - Vb), 0.f), fmaxf(fabsf(Va - cv), fabsf(Vb - cv)), lo, hi)) {
          S.cap[2] = range16(max(cellf(cu - hi, half) - mg, B.C0), min(cellf(cu - lo, half) + mg, B.C1 - 1) + 1);
          S.cap[3] = range16(max(cellf(cu + lo, half) - mg, B.C0), min(cellf(cu + hi, half) + mg, B.C1 - 1) + 1);
        }
      }
    }
    return;
  }
  // A far circle or a line: nearly straight over the grid, voted in one orientation and walked
  // toward its extreme (the near arc of a circle whose centre lies below the grid is walked up).
  // The walked range is the arc's extent between the grid's two bounding lines of the other
  // axis, from its crossings with them and its extreme point when that lies between them;
  // without both crossings it is not culled.
  const bool rows = fabsf(d2) >= fabsf(d1);
  if (rows != ROWS) return;
  const float a = ROWS ? d1 : d2;   // coefficient of the run axis
  const float bw = ROWS ? d2 : d1;  // coefficient of the walked axis
  // crossings with the bounding lines x = -1 and x = 1 of the run axis: roots in the walked axis
  // of C y^2 + 2 bw y - T(x), T(x) = C - x (C x + 2 a)
  const float L0 = -1.f, L1 = 1.f;
  float e0, e1;
  const bool k0 = near_root(d3, g.invC, bw, fmaf(-L0, fmaf(d3, L0, 2.f * a), d3), e0);
  const bool k1 = near_root(d3, g.invC, bw, fmaf(-L1, fmaf(d3, L1, 2.f * a), d3), e1);
  const int lim0 = ROWS ? B.R0 : B.C0, lim1 = ROWS ? B.R1 - 1 : B.C1 - 1;
  int w0 = lim0, w1 = lim1;
  if (k0 && k1) {
    float lo = fminf(e0, e1), hi = fmaxf(e0, e1);
    const float ca = -a * g.invC;  // the extreme point's run coordinate (inf for a line)
    if (d3 > 0.f && ca >= L0 && ca <= L1) {
      // the extreme's walked coordinate on the near arc, cancellation-free
      const float ext = copysignf(fmaf(a, a, d3 * d3) / (d3 * (g.nd + fabsf(bw))), bw);
      lo = fminf(lo, ext);
      hi = fmaxf(hi, ext);
    }
    w0 = max(cellf(fmaxf(lo, -2.f), half) - mg, lim0);
    w1 = min(cellf(fminf(hi, 2.f), half) + mg, lim1);
  }
  const uint32_t wr = range16(w0, w1 + 1);
  if (ROWS) {
    S.cap[0] = bw > 0.f ? wr : 0u;
    S.cap[1] = bw > 0.f ? 0u : wr;
  } else {
    S.cap[2] = bw > 0.f ? 0u : wr;
    S.cap[3] = bw > 0.f ? wr : 0u;
    S.clip = (uint32_t)(G - 1) << 16;
  }
}

// Raw p and q of pair i.
__device__ __forceinline__ void load_pair(const float* __restrict__ P, const float* __restrict__ Q,
                                          int64_t i, float* r) {
  r[0] = __ldg(P + 3 * i);
  r[1] = __ldg(P + 3 * i + 1);
  r[2] = __ldg(P + 3 * i + 2);
  r[3] = __ldg(Q + 3 * i);
  r[4] = __ldg(Q + 3 * i + 1);
  r[5] = __ldg(Q + 3 * i + 2);
}

// p - q from raw values, scaled by a power of two so that max |d_k| is in [1, 2), signed so
// d3 >= 0; false for a degenerate pair.
__device__ __forceinline__ bool circle_from(const float* r, float& d1, float& d2, float& d3) {
  d1 = r[0] - r[3];
  d2 = r[1] - r[4];
  d3 = r[2] - r[5];
  const float m = fmaxf(fabsf(d1), fmaxf(fabsf(d2), fabsf(d3)));
  if (m == 0.f) return false;
  const float sc = inv_pow2_of(m);
  d1 *= sc;
  d2 *= sc;
  d3 *= sc;
  if (d3 < 0.f) {
    d1 = -d1;
    d2 = -d2;
    d3 = -d3;
  }
  return true;
}

__device__ __forceinline__ int segments_of(uint32_t pk) {
  const int l = (int)(pk >> 16) - (int)(pk & 0xffffu);
  return l > 0 ? (l + kSeg - 1) / kSeg : 0;
}

__device__ __forceinline__ void store_rec(uint32_t* tab, int lane, const Prepared& S) {
  tab[0 * 32 + lane] = __float_as_uint(S.d1);
  tab[1 * 32 + lane] = __float_as_uint(S.d2);
  tab[2 * 32 + lane] = __float_as_uint(S.d3);
#pragma unroll
  for (int c = 0; c < 4; ++c) tab[(3 + c) * 32 + lane] = S.cap[c];
  tab[7 * 32 + lane] = S.clip;
}

// One walker: a segment of one cap of one circle, the cap's units (strips) visited from its
// wider chord toward its extreme. It holds the cells of both crossings of the curve with the
// strip's wider line and computes those of the narrower line per step (the narrower line of one
// strip is the wider line of the next). Rows walk the run axis u; columns walk v.
struct Walker {
  int len;                        // units of the segment (0: idle)
  float C, a2, absa, bT;
  float kfl, knl, kfh, knh;       // cell coordinates (root + 1) G/2 of the lower root
                                  // kfl t + knl T/t + G/2 and of the upper kfh t + knh T/t + G/2
  float y, dy;                    // the next (narrower) line and its step
  int lw, hw;                     // cells of the crossings with the wider line
  bool ew;                        // the curve reaches the wider line
  int cl, cr;                     // the run axis's cells this walk may vote
  uint32_t ub, inc, trig;         // address base of the unit, its increment (1 or 0x10000), and
  int pstep;                      // the increment value at which the base moves by pstep
};

// Cells of the lower and upper crossing of lattice line y with the curve; false if none.
__device__ __forceinline__ bool line_cells(const Walker& w, float y, float half, int& lo, int& hi) {
  const float T = fmaf(-y, fmaf(w.C, y, w.bT), w.C);
  const float disc = fmaf(w.C, T, w.a2);
  const float s = disc * rsqrt_approx(fmaxf(disc, 1e-30f));
  const float t = w.absa + s;  // > 0: absa carries a tiny offset
  const float nr = T * rcp_approx(t);
  lo = __float2int_rd(fmaf(w.kfl, t, fmaf(w.knl, nr, half)));
  hi = __float2int_rd(fmaf(w.kfh, t, fmaf(w.knh, nr, half)));
  return disc >= 0.f;
}

// Decodes segment sid of the current deal (the row caps 0-1 when ROWS, else the column caps 2-3)
// and places the walker on its first unit (len = 0 if none); with nparts > 1 the walker takes
// part `part` of nparts consecutive parts of the segment.
template <bool ROWS>
__device__ __forceinline__ void start_walker(const Band& B, const uint32_t* tab, int total_segs, int sid,
                                             int part, int nparts, Walker& w) {
  w.len = 0;
  if (sid >= total_segs) {
    w.C = w.a2 = w.absa = w.bT = w.kfl = w.knl = w.kfh = w.knh = w.y = w.dy = 0.f;
    w.lw = w.hw = w.cl = w.cr = w.pstep = 0;
    w.ew = false;
    w.ub = w.trig = 0u;
    w.inc = 1u;
    return;
  }
  int k = 0;
#pragma unroll
  for (int s = 16; s > 0; s >>= 1)
    if ((int)tab[8 * 32 + k + s] <= sid) k += s;
  const int loc = sid - (int)tab[8 * 32 + k];
  const uint32_t c0 = tab[(ROWS ? 3 : 5) * 32 + k], c1 = tab[(ROWS ? 4 : 6) * 32 + k];
  const int s0 = segments_of(c0);
  const bool second = loc >= s0;  // cap 1 (bottom) / 3 (right)
  const uint32_t pk = second ? c1 : c0;
  const int seg = second ? loc - s0 : loc;
  const int lo = (int)(pk & 0xffffu), hi = (int)(pk >> 16);
  // walk direction: rows up (cap 0) or down (cap 1); columns left (cap 2) or right (cap 3)
  const int dm = ROWS ? (second ? -1 : 1) : (second ? 1 : -1);
  int off = seg * kSeg;
  int len = min(kSeg, hi - lo - off);
  if (nparts > 1) {
    const int sub = nparts == 2 ? (len + 1) >> 1 : (len + 2) / 3;
    off += part * sub;
    len = max(0, min(sub, len - part * sub));
  }
  const int m = dm > 0 ? lo + off : hi - 1 - off;  // first unit
  const float d1 = __uint_as_float(tab[0 * 32 + k]), d2 = __uint_as_float(tab[1 * 32 + k]);
  const float C = __uint_as_float(tab[2 * 32 + k]);
  const float a = ROWS ? d1 : d2, bw = ROWS ? d2 : d1;
  const int G = B.G;
  w.len = len;
  w.C = C;
  w.a2 = a * a;
  w.absa = fabsf(a) + 1e-30f;
  w.bT = 2.f * bw;
  // roots of C x^2 + 2 a x - T: lower -t/C and upper T/t for a >= 0, else -T/t and t/C, in
  // cells (scaled by G/2, a power of two); 1/C by the hardware approximation, like 1/t
  const float invC = C > 0.f ? rcp_approx(C) : __int_as_float(0x7f800000);
  const bool apos = a >= 0.f;
  const float hs = B.half;
  w.kfl = apos ? -invC * hs : 0.f;
  w.knl = apos ? 0.f : -hs;
  w.kfh = apos ? 0.f : invC * hs;
  w.knh = apos ? hs : 0.f;
  w.dy = dm > 0 ? B.step : -B.step;
  const float yw = fmaf((float)(dm > 0 ? m : m + 1), B.step, -1.f);  // the first unit's wider line
  w.y = yw + w.dy;
  if (ROWS) {
    w.cl = 0;
    w.cr = G - 1;
    w.ub = B.tb + 4u * (uint32_t)(((m - B.R0) >> 1) * B.RS);
    w.inc = ((m - B.R0) & 1) ? 0x10000u : 1u;
    w.pstep = dm > 0 ? 4 * B.RS : -4 * B.RS;
  } else {
    const uint32_t clip = tab[7 * 32 + k];
    w.cl = (int)(clip & 0xffffu);
    w.cr = (int)(clip >> 16);
    w.ub = B.tb + 4u * (uint32_t)((m - B.C0) >> 1);
    w.inc = ((m - B.C0) & 1) ? 0x10000u : 1u;
    w.pstep = dm > 0 ? 4 : -4;
  }
  w.trig = dm > 0 ? 1u : 0x10000u;
  w.ew = line_cells(w, yw, B.half, w.lw, w.hw);
}

// One unit: the crossings with the strip's narrower line, the strip's two runs (lower and upper
// crossings, or one run when the narrower line misses the curve, merged where they touch),
// clipped to the walk's cells, each voted as +inc at its first cell and -inc after its last. A
// vote that fails its test goes to the lane's dummy word, so every vote is one unconditional
// atomic.
template <bool ROWS>
__device__ __forceinline__ void step_walker(Walker& w, int i, const Band& B, uint32_t dummy) {
  int ln, hn;
  const bool en = line_cells(w, w.y, B.half, ln, hn);
  const uint32_t xs = ROWS ? 4u : 4u * (uint32_t)B.W;
  const int b1 = en ? min(ln, max(hn, -(1 << 30)) - 1) : w.hw;
  const int a2 = en ? hn : (1 << 30);
  const int x1 = max(w.lw, w.cl), y1 = min(b1, w.cr);
  const int x2 = max(a2, w.cl), y2 = min(w.hw, w.cr);
  const bool act = (i < w.len) && w.ew;
  const bool v1 = act && x1 <= y1, v2 = act && x2 <= y2;
  const uint32_t ninc = 0u - w.inc;
  // a run ending on the grid's last cell puts its -inc in the tile's pad (y + 1 = G)
  red_add(v1 ? w.ub + (uint32_t)x1 * xs : dummy, w.inc);
  red_add(v1 ? w.ub + (uint32_t)(y1 + 1) * xs : dummy, ninc);
  red_add(v2 ? w.ub + (uint32_t)x2 * xs : dummy, w.inc);
  red_add(v2 ? w.ub + (uint32_t)(y2 + 1) * xs : dummy, ninc);
  w.lw = ln;
  w.hw = hn;
  w.ew = en;
  w.y += w.dy;
  w.inc ^= 0x10001u;
  w.ub += w.inc == w.trig ? (uint32_t)w.pstep : 0u;
}

// Phase B (the whole warp) for one deal of its batch: segments dealt out in rounds, kWalkers per
// lane; when at most half the walkers of the deal's last round would get a segment, each
// remaining segment is cut into two or three parts so that the deal takes fewer rounds.
template <bool ROWS>
__device__ __forceinline__ void walk_deal(const Band& B, const uint32_t* tab, int total_segs, int lane,
                                          uint32_t dummy) {
  for (int base = 0; base < total_segs; base += 32 * kWalkers) {
    const int rem = total_segs - base;
    const int nparts = rem > 16 * kWalkers ? 1 : (rem > 32 * kWalkers / 3 ? 2 : 3);
    Walker w[kWalkers];
    int longest = 0;
#pragma unroll
    for (int j = 0; j < kWalkers; ++j) {
      const int t = 32 * j + lane;
      const int q = nparts == 1 ? t : (nparts == 2 ? t >> 1 : t / 3);
      start_walker<ROWS>(B, tab, total_segs, base + q, t - q * nparts, nparts, w[j]);
      longest = max(longest, w[j].len);
    }
    const int rounds = __reduce_max_sync(kFull, (unsigned)longest);
    for (int i = 0; i < rounds; ++i) {
#pragma unroll
      for (int j = 0; j < kWalkers; ++j) step_walker<ROWS>(w[j], i, B, dummy);
    }
  }
}

// The segments of this lane's circle in the deal (row caps or column caps), the circle's first
// segment stored in its table record; returns the deal's total.
__device__ __forceinline__ int deal_offsets(uint32_t* tab, int lane, bool live, bool rows) {
  int segs = 0;
  if (live) segs = segments_of(tab[(rows ? 3 : 5) * 32 + lane]) + segments_of(tab[(rows ? 4 : 6) * 32 + lane]);
  int incl = segs;
#pragma unroll
  for (int s = 1; s < 32; s <<= 1) {
    const int v = __shfl_up_sync(kFull, incl, s);
    if (lane >= s) incl += v;
  }
  tab[8 * 32 + lane] = (uint32_t)(incl - segs);
  __syncwarp();
  return __shfl_sync(kFull, incl, 31);
}

// One work item: the pairs c0..c1 of a slice voted into the item's tile (ROWS: the row caps of
// a band of rows; else the column caps of a band of columns), the differences turned into
// counts and the tile written to the slice's partial of the accumulator (columns 2j and 2j + 1
// of a row share a word).
template <bool ROWS>
__device__ __forceinline__ void vote_item(const VoteItem& I, const InstDev& D, uint32_t* smem, int tile_words,
                                          int* s_next) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t* tab = smem + tile_words + warp * kTab;
  const uint32_t dummy = (uint32_t)__cvta_generic_to_shared(smem + tile_words + kRunWarps * kTab + lane);
  Band B;
  B.G = D.G;
  const int G = B.G, W2 = G >> 1;
  const int e0 = D.band_row0[I.band], e1 = D.band_row0[I.band + 1];
  B.R0 = ROWS ? e0 : 0;
  B.R1 = ROWS ? e1 : G;
  B.C0 = ROWS ? 0 : e0;
  B.C1 = ROWS ? G : e1;
  B.W = (B.C1 - B.C0) >> 1;
  B.step = 2.0f / (float)G;
  B.half = 0.5f * (float)G;
  uint32_t* tile = smem;
  B.tb = (uint32_t)__cvta_generic_to_shared(tile);
  B.RS = G + 4;
  const int words = ROWS ? ((B.R1 - B.R0) >> 1) * B.RS : G * B.W;
  uint4* t4 = reinterpret_cast<uint4*>(tile);
  for (int x = threadIdx.x; x < (words >> 2); x += blockDim.x) t4[x] = make_uint4(0, 0, 0, 0);
  __syncthreads();

  const float* __restrict__ P = D.P;
  const float* __restrict__ Q = D.Q;
  const int64_t count = I.c1 - I.c0;
  int base = 0;
  if (lane == 0) base = atomicAdd(s_next, 32);
  base = __shfl_sync(kFull, base, 0);
  float r[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  if (base + lane < count) load_pair(P, Q, I.c0 + base + lane, r);
  for (;;) {
    if (base >= count) break;
    float d1 = 0.f, d2 = 0.f, d3 = 0.f;
    const bool live = base + lane < count && circle_from(r, d1, d2, d3);
    int nbase = 0;
    if (lane == 0) nbase = atomicAdd(s_next, 32);
    nbase = __shfl_sync(kFull, nbase, 0);
    if (nbase + lane < count) load_pair(P, Q, I.c0 + nbase + lane, r);
    Prepared S;
    if (live) {
      prepare<ROWS>(B, d1, d2, d3, S);
      store_rec(tab, lane, S);
    } else {
#pragma unroll
      for (int c = 0; c < 4; ++c) tab[(3 + c) * 32 + lane] = 0u;
    }
    __syncwarp();
    const int total = deal_offsets(tab, lane, live, ROWS);
    if (total > 0) walk_deal<ROWS>(B, tab, total, lane, dummy);
    __syncwarp();
    base = nbase;
  }
  __syncthreads();

  uint32_t* out = D.partial + (int64_t)I.slice * G * W2;
  if (ROWS) {
    flush_row_pair_tile(tile, G, B.RS, B.R0, B.R1, out);
  } else {
    // prefix sums down each word column in chunks of rows (a thread per column and chunk), the
    // chunks' carries, then the rows
    const int W = B.W;
    const int nch = max(1, min((int)blockDim.x / W, G / 8));
    const int rpc = (G + nch - 1) / nch;
    if ((int)threadIdx.x < W * nch) {
      const int c2 = threadIdx.x % W, ch = threadIdx.x / W;
      const int r1 = min(G, (ch + 1) * rpc);
      uint32_t acc = 0;
      for (int rr = ch * rpc; rr < r1; ++rr) {
        acc += tile[rr * W + c2];
        tile[rr * W + c2] = acc;
      }
    }
    __syncthreads();
    uint32_t* carry = smem + tile_words;  // the tables' space, free after the walk
    if ((int)threadIdx.x < W * nch) {
      const int c2 = threadIdx.x % W, ch = threadIdx.x / W;
      uint32_t c = 0;
      for (int k = 0; k < ch; ++k) c += tile[(min(G, (k + 1) * rpc) - 1) * W + c2];
      carry[ch * W + c2] = c;
    }
    __syncthreads();
    for (int g = threadIdx.x; g < ((G * W) >> 2); g += blockDim.x) {
      const int rr = (4 * g) / W, c2 = 4 * g - rr * W;
      const uint4 v = reinterpret_cast<const uint4*>(tile)[g];
      const uint4 c = *reinterpret_cast<const uint4*>(carry + (rr / rpc) * W + c2);
      reinterpret_cast<uint4*>(out)[(rr * W2 + (B.C0 >> 1) + c2) >> 2] = make_uint4(v.x + c.x, v.y + c.y, v.z + c.z, v.w + c.w);
    }
  }
  __syncthreads();
}

__global__ void __launch_bounds__(kRunThreads, 1)
    k_axis_vote_runs(const VoteItem* __restrict__ items, int n_items, const InstDev* __restrict__ insts,
                     int* __restrict__ counter, int tile_words) {
  extern __shared__ __align__(16) uint32_t smem[];
  __shared__ int s_item, s_next;
  pdl_launch_dependents();  // the slice reduction may be scheduled on the SMs this grid frees
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
    if (I.kind == 0)
      vote_item<true>(I, D, smem, tile_words, &s_next);
    else
      vote_item<false>(I, D, smem, tile_words, &s_next);
  }
}

// Shared-atomic throughput probe: conflict-free red.shared.add.u32, one per thread per
// round, on every SM.
__global__ void __launch_bounds__(1024) k_probe_atomics(int iters, uint32_t* sink) {
  __shared__ uint32_t buf[1024];
  buf[threadIdx.x] = 0;
  __syncthreads();
  const uint32_t addr = (uint32_t)__cvta_generic_to_shared(buf + threadIdx.x);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 16; ++u)
      asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(addr), "r"(1u) : "memory");
  }
  __syncthreads();
  if (buf[threadIdx.x] != (uint32_t)iters * 16u) atomicAdd(sink, 1u);
}

}  // namespace

int vote_run_table_bytes() { return kRunWarps * kTab * 4 + 32 * 4; }  // tables + dummy words

void launch_axis_vote_runs(const VoteItem* items, int n_items, const InstDev* insts, int* counter,
                           int grid_ctas, int tile_bytes, cudaStream_t st) {
  ensure_dynamic_smem(reinterpret_cast<const void*>(k_axis_vote_runs), kRunSmemBytes);
  k_axis_vote_runs<<<grid_ctas, kRunThreads, tile_bytes + vote_run_table_bytes(), st>>>(
      items, n_items, insts, counter, tile_bytes / 4);
  launches_add(1);
}

double probe_smem_atomics(int iters, cudaStream_t st) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  uint32_t* sink = nullptr;
  if (cudaMalloc(&sink, 4) != cudaSuccess) return -1.0;
  cudaMemsetAsync(sink, 0, 4, st);
  const int ctas = sms * 2;
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
