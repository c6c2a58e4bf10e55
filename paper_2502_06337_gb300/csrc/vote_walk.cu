// Axis vote: the 2-D accumulator of Algorithm 1 (Sec. IV-A), rasterised exactly by walking
// the projected circles cell by cell.
//
// Every correspondence i gives d = p_i - q_i; its admissible rotation axes form the great
// circle r . d = 0 (Eqs. 5-8), whose stereographic image (Eqs. 11-13, D = 0) is the zero set of
//     F(u, v) = 2 d1 u + 2 d2 v + d3 (u^2 + v^2 - 1).
// After scaling d by a power of two and choosing its sign so that d3 >= 0, the curve is a
// circle of centre (-d1, -d2)/d3 and radius |d|/d3 >= 1, or for d3 = 0 a line through the
// origin. A cell is voted when the curve meets the closed cell.
//
// The circle is split at its four extreme points and four 45-degree points into eight
// monotone pieces: four x-major pieces (|slope| <= 1), walked column by column, and four
// y-major pieces, walked row by row (the same code with u and v exchanged). Walking a piece
// along its major axis, the crossing moves by at most about one cell per step; whether it
// passes the next lattice edge is the sign of F at the lattice corner (exact grid
// coordinates, three roundings). The two cells of extreme points are voted directly.
//
// Work split. A CTA owns one row band of the accumulator as 16-bit counters in shared
// memory (columns 2j and 2j+1 share a 32-bit word), incremented with red.shared.add.u32
// (unconditionally: a vote that fails its test is sent to a per-lane dummy word). A
// warp loads 32 circles; in phase A each lane prepares its own circle for the band (piece
// ranges culled to the band and the grid, extreme cells voted) and stores it in a per-warp
// table. In phase B the pieces of all 32 circles are cut into segments of at most kSeg major
// steps, dealt out in rounds of kWalkers segments per lane; a walker starts a segment with
// one quadratic solve and walks it in lock step with the warp. One step of a walker votes
// one cell and then either crosses one lattice edge of the minor axis -- when the piece is
// beyond that edge at the exit line, i.e. when F at the lattice corner has the sign of
// "beyond" -- or advances one major step. F is
// evaluated as g(x) + h(y) with g, h updated only when x or y changes, three roundings in
// all. Decisions whose F is within a few float32 roundings of zero lie inside the band
// where the closed-cell test may go either way; all others match the exact test.
#include <stdint.h>

#include "sprot_internal.h"

namespace sprot {

namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ float edgef(int k, float step) { return fmaf((float)k, step, -1.0f); }

// Roots lo <= hi of c3 y^2 + 2 b y + kk = 0 (c3 >= 0, inv3 = 1/c3, +inf for c3 = 0), one from
// |b| + sqrt(disc) and the other from the product of the roots. Returns false (roots NaN)
// when the quadratic has no real root. The square root and quotient are the hardware
// approximations (a few ulp): a root only places a start cell or a piece boundary, and a
// start cell is wrong only when the root lies within rounding of a cell edge, where F at that
// edge is within the boundary band.
__device__ __forceinline__ bool qroots(float c3, float inv3, float b, float kk, float& lo,
                                       float& hi) {
  const float disc = fmaf(-c3, kk, b * b);
  const float t = fabsf(b) + (disc > 0.f ? disc * rsqrtf(disc) : sqrtf(disc));
  const float far = t * inv3;
  const float nr = t > 0.f ? __fdividef(kk, t) : 0.f;  // t = 0: b = 0, double root at 0
  lo = b >= 0.f ? -far : nr;
  hi = b >= 0.f ? -nr : far;
  return disc >= 0.f;
}

// Cell of coordinate y clamped to [lo, hi] (NaN -> lo).
__device__ __forceinline__ int cell_clamped(float y, float half, int lo, int hi) {
  return __float2int_rd(fminf(fmaxf(fmaf(y, half, half), (float)lo), (float)hi));
}

struct Band {
  uint32_t sbase;
  int G, W, R0, R1;
  float step, half, Gf;

  __device__ __forceinline__ void vote(int r, int c) const {
    const uint32_t word = (uint32_t)((r - R0) * W + (c >> 1));
    asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(sbase + 4u * word),
                 "r"((c & 1) ? 0x10000u : 1u)
                 : "memory");
  }
  __device__ __forceinline__ int cell(float y) const { return cell_clamped(y, half, -1, G); }
  __device__ __forceinline__ int index(float y) const { return cell_clamped(y, half, -4, G + 4); }
};

// Piece p: 0-3 x-major (top-left, top-right, bottom-left, bottom-right), 4-7 y-major
// (left-lower, left-upper, right-lower, right-upper). The branch is the upper root along the
// minor axis for pieces 0, 1, 6, 7. kDirUp: pieces whose minor coordinate grows along the
// major axis. For every piece, (direction) x (sign of dF/d(minor) on its branch) is +1 for
// even p and -1 for odd p; even pieces walk toward the circle's centre, odd ones away.
constexpr uint32_t kDirUp = 0x69u;

struct Prepared {
  float d1, d2, d3, inv3;
  uint32_t piece[8];  // major range [lo, hi) packed lo | hi << 16
  uint32_t jAB;       // y-major column windows: jA + 1 | jB << 16 (left <= jA, right >= jB)
};

__device__ __forceinline__ uint32_t pack(int lo, int hi) {
  return hi > lo ? ((uint32_t)lo | ((uint32_t)hi << 16)) : 0u;
}

// Phase A (one lane, one circle): piece ranges for this band; extreme-point cells voted.
__device__ void prepare(const Band& B, float d1, float d2, float d3, Prepared& S) {
  const int G = B.G;
  const float step = B.step;
  const float V0 = edgef(B.R0, step), V1 = edgef(B.R1, step);
  const float nd = sqrtf(fmaf(d1, d1, fmaf(d2, d2, d3 * d3)));
  const float d1x2 = 2.f * d1, d2x2 = 2.f * d2;
#pragma unroll
  for (int p = 0; p < 8; ++p) S.piece[p] = 0u;
  S.d1 = d1;
  S.d2 = d2;
  if (d3 <= 1e-8f * nd) {
    // a line through the origin (d3 = 0 up to a change of F below 2e-8 |d|)
    S.d3 = 0.f;
    S.inv3 = __int_as_float(0x7f800000);
    const bool rise = d1 * d2 <= 0.f;
    if (fabsf(d2) >= fabsf(d1)) {
      const bool up = d2 >= 0.f;
      const int p = up ? (rise ? 0 : 1) : (rise ? 3 : 2);
      S.piece[p] = pack(0, G);
      S.jAB = 0u | ((uint32_t)G << 16);
    } else {
      const bool up = d1 >= 0.f;
      const int p = up ? (rise ? 6 : 7) : (rise ? 5 : 4);
      S.piece[p] = pack(B.R0, B.R1);
      S.jAB = (uint32_t)G | (0u << 16);  // both windows are the whole row
    }
    return;
  }
  S.d3 = d3;
  const float inv3 = __frcp_rn(d3);
  S.inv3 = inv3;
  const float s = 0.70710678f;
  // 45-degree points cx -/+ rho/sqrt(2), without cancellation
  const float q1 = fmaf(d2, d2, d3 * d3) - d1 * d1;
  const float uA = d1 >= 0.f ? -(d1 + s * nd) * inv3 : __fdividef(-0.5f * q1, (s * nd - d1) * d3);
  const float uB = d1 <= 0.f ? (s * nd - d1) * inv3 : __fdividef(0.5f * q1, (s * nd + d1) * d3);
  const int jA = min(max(cell_clamped(uA, B.half, -2, G + 2), -1), G - 1);
  const int jB = min(max(cell_clamped(uB, B.half, -2, G + 2), 0), G);
  S.jAB = (uint32_t)(jA + 1) | ((uint32_t)jB << 16);
  const int xj0 = max(jA + 1, 0), xj1 = min(jB - 1, G - 1);
  const float cx = -d1 * inv3, cy = -d2 * inv3;
  const int jc = B.index(cx), ic = B.index(cy);
  float lo, hi, lo1, hi1;

  // the column holding the top and bottom points
  if (jc >= xj0 && jc <= xj1) {
    float yb, yt;
    qroots(d3, inv3, d2, -fmaf(d1, d1, d3 * d3) * inv3, yb, yt);
    float x = edgef(jc, step);
    qroots(d3, inv3, d2, fmaf(d3, fmaf(x, x, -1.f), d1x2 * x), lo, hi);
    x = edgef(jc + 1, step);
    qroots(d3, inv3, d2, fmaf(d3, fmaf(x, x, -1.f), d1x2 * x), lo1, hi1);
    int a = max(min(B.cell(hi), B.cell(hi1)), B.R0), b = min(B.cell(yt), B.R1 - 1);
    for (int r = a; r <= b; ++r) B.vote(r, jc);
    a = max(B.cell(yb), B.R0);
    b = min(max(B.cell(lo), B.cell(lo1)), B.R1 - 1);
    for (int r = a; r <= b; ++r) B.vote(r, jc);
  }

  // x-major pieces, culled to the columns where they are inside the band [V0, V1]
  {
    float a0, b0, a1, b1;
    const bool ok0 = qroots(d3, inv3, d1, fmaf(d3, fmaf(V0, V0, -1.f), d2x2 * V0), a0, b0);
    const bool ok1 = qroots(d3, inv3, d1, fmaf(d3, fmaf(V1, V1, -1.f), d2x2 * V1), a1, b1);
    const int L0 = xj0, L1 = min(jc, xj1 + 1), Rr0 = max(jc + 1, xj0), Rr1 = xj1 + 1;
    // bounds: 'lo' restricts the first column, 'hi' the last; k = 0 none, 1 value, 2 empty
    auto clip = [&](int a, int b, int klo, float ulo, int khi, float uhi) -> uint32_t {
      if (klo == 2 || khi == 2) return 0u;
      if (klo == 1) a = max(a, B.index(ulo) - 1);
      if (khi == 1) b = min(b, B.index(uhi) + 2);
      return pack(a, b);
    };
    // top-left: v >= V0 <=> u >= a0 ; v <= V1 <=> u <= a1
    S.piece[0] = clip(L0, L1, V0 <= cy ? 0 : (ok0 ? 1 : 2), a0, V1 < cy ? 2 : (ok1 ? 1 : 0), a1);
    // top-right: v >= V0 <=> u <= b0 ; v <= V1 <=> u >= b1
    S.piece[1] = clip(Rr0, Rr1, V1 < cy ? 2 : (ok1 ? 1 : 0), b1, V0 <= cy ? 0 : (ok0 ? 1 : 2), b0);
    // bottom-left: v <= V1 <=> u >= a1 ; v >= V0 <=> u <= a0
    S.piece[2] = clip(L0, L1, V1 >= cy ? 0 : (ok1 ? 1 : 2), a1, V0 > cy ? 2 : (ok0 ? 1 : 0), a0);
    // bottom-right: v >= V0 <=> u >= b0 ; v <= V1 <=> u <= b1
    S.piece[3] = clip(Rr0, Rr1, V0 > cy ? 2 : (ok0 ? 1 : 0), b0, V1 >= cy ? 0 : (ok1 ? 1 : 2), b1);
  }

  // y-major pieces: rows of the chord at the split line, within the band and the grid
#pragma unroll
  for (int side = 0; side < 2; ++side) {
    if (side == 0 ? jA < 0 : jB > G - 1) continue;
    float x = edgef(side == 0 ? jA + 1 : jB, step);
    qroots(d3, inv3, d2, fmaf(d3, fmaf(x, x, -1.f), d1x2 * x), lo, hi);
    const int y0 = max(B.index(lo) - 1, B.R0), y1 = min(B.index(hi) + 1, B.R1 - 1);
    // rows where the arc is beyond u = -1 (left) or u = +1 (right) are outside the grid
    x = side == 0 ? -1.f : 1.f;
    const bool okg = qroots(d3, inv3, d2, fmaf(d3, fmaf(x, x, -1.f), d1x2 * x), lo, hi);
    const int lower_end = okg ? min(ic, B.index(lo) + 2) : ic;
    const int upper_beg = okg ? max(ic + 1, B.index(hi) - 1) : ic + 1;
    S.piece[side == 0 ? 4 : 6] = pack(y0, min(lower_end, y1 + 1));
    S.piece[side == 0 ? 5 : 7] = pack(max(upper_beg, y0), y1 + 1);
    // the row holding the leftmost (rightmost) point
    if (ic >= y0 && ic <= y1) {
      float ul, ur;
      qroots(d3, inv3, d1, -fmaf(d2, d2, d3 * d3) * inv3, ul, ur);
      x = edgef(ic, step);
      qroots(d3, inv3, d1, fmaf(d3, fmaf(x, x, -1.f), d2x2 * x), lo, hi);
      x = edgef(ic + 1, step);
      qroots(d3, inv3, d1, fmaf(d3, fmaf(x, x, -1.f), d2x2 * x), lo1, hi1);
      if (side == 0) {
        const int a = max(B.cell(ul), 0), b = min(max(B.cell(lo), B.cell(lo1)), jA);
        for (int c = a; c <= b; ++c) B.vote(ic, c);
      } else {
        const int a = max(min(B.cell(hi), B.cell(hi1)), jB), b = min(B.cell(ur), G - 1);
        for (int c = a; c <= b; ++c) B.vote(ic, c);
      }
    }
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
  const int e = ilogbf(m);
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

// Segment length of phase B: every piece is cut into segments of at most kSeg major steps.
constexpr int kSeg = 24;
constexpr int kWalkers = 2;  // independent walkers per lane (instruction-level parallelism)

__device__ __forceinline__ int segments_of(uint32_t pk) {
  const int l = (int)(pk >> 16) - (int)(pk & 0xffffu);
  return l > 0 ? (l + kSeg - 1) / kSeg : 0;
}

// Per-warp circle table in shared memory, one column per lane (structure of arrays):
// d1 d2 d3 inv3 jAB piece[0..7] offset, where offset is the circle's first segment in the
// batch.
constexpr int kRecWords = 18;  // 14 words of structure of arrays + 4 words of cumulative counts
constexpr int kTabWords = kRecWords * 32;
constexpr int kWalkThreads = 512;  // 16 warps: room for the tables beside the tile
constexpr int kWalkWarps = kWalkThreads / 32;

__device__ __forceinline__ void store_rec(uint32_t* tab, int lane, const Prepared& S, int off) {
  tab[0 * 32 + lane] = __float_as_uint(S.d1);
  tab[1 * 32 + lane] = __float_as_uint(S.d2);
  tab[2 * 32 + lane] = __float_as_uint(S.d3);
  tab[3 * 32 + lane] = __float_as_uint(S.inv3);
  tab[4 * 32 + lane] = S.jAB;
#pragma unroll
  for (int p = 0; p < 8; ++p) tab[(5 + p) * 32 + lane] = S.piece[p];
  tab[13 * 32 + lane] = (uint32_t)off;
  // inclusive prefix counts of the pieces' segments, packed as u16 pairs (array of structures:
  // one 16-byte record per circle)
  uint32_t cum[4];
  int acc = 0;
#pragma unroll
  for (int p = 0; p < 8; ++p) {
    acc += segments_of(S.piece[p]);
    if (p & 1)
      cum[p >> 1] |= (uint32_t)acc << 16;
    else
      cum[p >> 1] = (uint32_t)acc;
  }
  *reinterpret_cast<uint4*>(tab + 14 * 32 + 4 * lane) = make_uint4(cum[0], cum[1], cum[2], cum[3]);
}


// One walker: a segment of one piece, advanced one major step per iteration. The cell is
// tracked as the shared-memory byte address hb of its 16-bit counter (two counters per word,
// so the word's address is hb & ~3) with the increment inc = 1 or 0x10000 for its half, and
// as its minor coordinate rel relative to the piece's window. The state changes of a step
// are multiply-adds by the 0/1 move flag rather than selects (they leave the integer ALU
// pipe, the kernel's busiest, for the FMA pipe). The crossing
// test is gx < -h (F < 0) for every piece: the coefficients of odd pieces are negated, which
// negates F exactly, and without flush to zero the sign of a rounded sum is the sign of the
// exact one.
struct Walker {
  int len, hb, rel, span, rlim, dmaj, dmin, dir;
  uint32_t inc, fmaj;  // fmaj: the flip of inc on a major step (the minor flip is its complement)
  int tog;             // 1 if a minor step changes the column (swaps the half of inc)
  bool in;             // the current cell lies in the piece's window (a major step keeps it)
  float d3, dM2, dN2, xe, gx, yb, h, dys;
};

// A vote whose condition fails goes to the lane's own dummy word (32 words behind the warp
// tables, never read), so every vote is one unconditional atomic: no predicate is formed
// from the condition, and lanes never diverge around the atomics. The dummy words of the
// 32 lanes lie in 32 distinct banks.
__device__ __forceinline__ void vote_if(bool cond, int hb, uint32_t inc, uint32_t dummy) {
  const uint32_t addr = dummy + (uint32_t)cond * (((uint32_t)hb & ~3u) - dummy);  // cond ? word : dummy
  asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(addr), "r"(inc) : "memory");
}

// Decodes segment sid of the batch and places the walker on its first cell (len = 0 if none);
// with nparts > 1 the walker takes part `part` of nparts consecutive parts of the segment.
__device__ __forceinline__ void start_walker(const Band& B, const uint32_t* tab, int total_segs,
                                             int sid, int part, int nparts, Walker& w) {
  const int G = B.G;
  const float step = B.step;
  w.len = 0;
  w.hb = 0;
  w.rel = -1;
  w.span = -1;
  w.rlim = 0;
  w.dmaj = w.dmin = 0;
  w.dir = 1;
  w.inc = 1u;
  w.fmaj = 0u;
  w.tog = 0;
  w.in = false;
  w.d3 = w.dM2 = w.dN2 = w.xe = w.gx = w.yb = w.h = w.dys = 0.f;
  if (sid >= total_segs) return;
  // the circle: the largest k with first_segment[k] <= sid
  int k = 0;
#pragma unroll
  for (int s = 16; s > 0; s >>= 1)
    if ((int)tab[13 * 32 + k + s] <= sid) k += s;
  const int loc = sid - (int)tab[13 * 32 + k];
  // the piece: the number of pieces whose inclusive segment count is <= loc; the segment
  // within it: loc minus the largest such count
  const uint4 cw = *reinterpret_cast<const uint4*>(tab + 14 * 32 + 4 * k);
  const uint32_t cv[8] = {cw.x & 0xffffu, cw.x >> 16, cw.y & 0xffffu, cw.y >> 16,
                          cw.z & 0xffffu, cw.z >> 16, cw.w & 0xffffu, cw.w >> 16};
  int p = 0;
  uint32_t before = 0;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const bool done = cv[q] <= (uint32_t)loc;
    p += done;
    before = done ? cv[q] : before;
  }
  const int seg = loc - (int)before;
  const uint32_t pk = tab[(5 + p) * 32 + k];
  const int lo = (int)(pk & 0xffffu);
  const int plen = (int)(pk >> 16) - lo;
  int c = lo + seg * kSeg;
  int len = min(kSeg, plen - seg * kSeg);
  if (nparts > 1) {  // part `part` of nparts consecutive parts of the segment
    const int sub = nparts == 2 ? (len + 1) >> 1 : (len + 2) / 3;
    c += part * sub;
    len = max(0, min(sub, len - part * sub));
  }
  const float d1 = __uint_as_float(tab[0 * 32 + k]), d2 = __uint_as_float(tab[1 * 32 + k]);
  const float inv3 = __uint_as_float(tab[3 * 32 + k]);
  const float d3 = __uint_as_float(tab[2 * 32 + k]);
  const uint32_t jAB = tab[4 * 32 + k];
  const bool tr = p >= 4;
  const bool up = p < 2 || p >= 6;
  const int dir = ((kDirUp >> p) & 1u) ? 1 : -1;
  const bool flip = (p & 1) != 0;  // "beyond" is F < 0 for even pieces and F > 0 for odd ones
  const float dM2 = 2.f * (tr ? d2 : d1);
  const float dN = tr ? d1 : d2;
  const float dN2 = 2.f * dN;
  const int jA = (int)(jAB & 0xffffu) - 1, jB = (int)(jAB >> 16);
  const int wlo = tr ? (p < 6 ? 0 : jB) : B.R0;
  w.span = (tr ? (p < 6 ? jA : G - 1) : B.R1 - 1) - wlo;
  // start: the crossing of this piece's branch with the major line c
  const float x = edgef(c, step);
  float rlo, rhi;
  int r;
  if (qroots(d3, inv3, dN, fmaf(d3, fmaf(x, x, -1.f), dM2 * x), rlo, rhi)) {
    r = B.cell(up ? rhi : rlo);
  } else if (!flip) {
    // The start line misses the circle (a margin row of a y-major piece): even pieces walk
    // toward the centre, so start at the centre's column, which lies inside every chord of
    // the circle and outside the piece's column window. If the next line meets the circle,
    // the walk sweeps from there to the branch, voting exactly the cells of the cap in this
    // row; if it does not, nothing moves.
    r = B.cell(-dN * inv3);
  } else {
    r = 0;
    len = 0;  // odd pieces walk away from the centre: the rest lies beyond the circle
  }
  w.len = len;
  w.dir = dir;
  w.rel = r - wlo;
  w.in = (unsigned)w.rel <= (unsigned)w.span;
  w.rlim = (dir > 0 ? G : -1) - wlo;  // the rare-crossing loop stops at the grid edge
  const int W2 = 2 * B.W;              // half-words per tile row
  const int row = tr ? c : r, col = tr ? r : c;
  w.hb = 2 * ((row - B.R0) * W2 + col) + (int)B.sbase;
  w.inc = (col & 1) ? 0x10000u : 1u;
  w.fmaj = tr ? 0u : 0x10001u;
  w.tog = tr ? 1 : 0;
  w.dmaj = tr ? 2 * W2 : 2;
  w.dmin = tr ? 2 * dir : 2 * dir * W2;
  const float sg = flip ? -1.f : 1.f;
  w.d3 = sg * d3;
  w.dM2 = sg * dM2;
  w.dN2 = sg * dN2;
  w.dys = dir > 0 ? step : -step;
  w.xe = x + step;  // exit line of column c
  w.gx = w.xe * fmaf(w.d3, w.xe, w.dM2);
  w.yb = edgef(r + (dir > 0 ? 1 : 0), step);  // next minor edge in the walking direction
  w.h = fmaf(w.yb, fmaf(w.d3, w.yb, w.dN2), -w.d3);
}

// One major step of a walker, straight-line: vote the cell, cross the next minor edge if the
// piece is beyond it at the exit line (voting that cell), step on. Returns whether the piece
// is still beyond the following edge (a second crossing in the same step, which is rare).
// A walker that leaves the grid never returns (each piece is monotone along its minor axis)
// and its votes are masked by the window test, so the common step does not stop at the edge.
__device__ __forceinline__ bool step_walker(Walker& w, int i, uint32_t dummy) {
  const bool act = i < w.len;
  vote_if(act && w.in, w.hb, w.inc, dummy);
  const bool mv = act && w.gx < -w.h;
  const int m = (int)mv;
  w.rel += m * w.dir;
  w.hb += m * w.dmin;
  // a column change swaps the half: 1 <-> 0x10000, i.e. inc -> 0x10001 - inc
  w.inc += (uint32_t)(m * w.tog) * (0x10001u - 2u * w.inc);
  w.yb += mv ? w.dys : 0.f;
  w.h = fmaf(w.yb, fmaf(w.d3, w.yb, w.dN2), -w.d3);
  w.in = (unsigned)w.rel <= (unsigned)w.span;
  vote_if(mv && w.in, w.hb, w.inc, dummy);
  return mv && w.gx < -w.h;
}

// Remaining crossings of a step (slopes above one cell per step; rare). Bounded by the
// grid edge.
__device__ __forceinline__ void more_crossings(Walker& w) {
  while (w.gx < -w.h && (w.dir > 0 ? w.rel < w.rlim : w.rel > w.rlim)) {
    w.rel += w.dir;
    w.hb += w.dmin;
    w.inc ^= w.fmaj ^ 0x10001u;
    w.yb += w.dys;
    w.h = fmaf(w.yb, fmaf(w.d3, w.yb, w.dN2), -w.d3);
    w.in = (unsigned)w.rel <= (unsigned)w.span;
    if (w.in)  // the rare loop keeps a plain branch
      asm volatile("red.shared.add.u32 [%0], %1;" ::"r"((uint32_t)w.hb & ~3u), "r"(w.inc) : "memory");
  }
}

__device__ __forceinline__ void advance(Walker& w, float step) {
  w.hb += w.dmaj;
  w.inc ^= w.fmaj;
  w.xe += step;
  w.gx = w.xe * fmaf(w.d3, w.xe, w.dM2);
}

// Phase B (the whole warp, its batch of circles). The pieces of all circles are cut into
// segments of at most kSeg major steps and dealt out in rounds, kWalkers segments per lane,
// so that every lane decodes its segments and solves their start quadratics at the same time
// and walks independent segments in lock step.
__device__ __forceinline__ void walk_batch(const Band& B, const uint32_t* tab, int total_segs,
                                           int lane, uint32_t dummy) {
  for (int base = 0; base < total_segs; base += 32 * kWalkers) {
    // The last deal of a batch: when at most half the walkers would get a segment, each
    // remaining segment is cut into two or three consecutive parts, so that more walkers
    // share it and the deal takes fewer rounds.
    const int rem = total_segs - base;
    const int nparts = rem > 16 * kWalkers ? 1 : (rem > 32 * kWalkers / 3 ? 2 : 3);
    Walker w[kWalkers];
    int longest = 0;
#pragma unroll
    for (int j = 0; j < kWalkers; ++j) {
      const int t = 32 * j + lane;
      const int q = nparts == 1 ? t : (nparts == 2 ? t >> 1 : t / 3);
      start_walker(B, tab, total_segs, base + q, t - q * nparts, nparts, w[j]);
      longest = max(longest, w[j].len);
    }
    const int rounds = __reduce_max_sync(kFull, (unsigned)longest);
    for (int i = 0; i < rounds; ++i) {
      bool more[kWalkers], any = false;
#pragma unroll
      for (int j = 0; j < kWalkers; ++j) {
        more[j] = step_walker(w[j], i, dummy);
        any |= more[j];
      }
      if (__any_sync(kFull, any)) {
#pragma unroll
        for (int j = 0; j < kWalkers; ++j)
          if (more[j]) more_crossings(w[j]);
      }
#pragma unroll
      for (int j = 0; j < kWalkers; ++j) advance(w[j], B.step);
    }
  }
}

__global__ void __launch_bounds__(kWalkThreads, 1)
    k_axis_vote_walk(const VoteItem* __restrict__ items, int n_items,
                     const InstDev* __restrict__ insts, int* __restrict__ counter, int tile_words) {
  extern __shared__ __align__(16) uint32_t smem[];
  uint32_t* tile = smem;
  __shared__ int s_item, s_next;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t* tab = smem + tile_words + warp * kTabWords;
  // this lane's dummy word for votes that fail their test
  const uint32_t dummy = (uint32_t)__cvta_generic_to_shared(smem + tile_words + kWalkWarps * kTabWords + lane);
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
    B.R0 = D.band_row0[I.band];
    B.R1 = D.band_row0[I.band + 1];
    B.Gf = (float)D.G;
    B.step = 2.0f / B.Gf;
    B.half = 0.5f * B.Gf;
    B.sbase = (uint32_t)__cvta_generic_to_shared(tile);
    const int words = (B.R1 - B.R0) * B.W;
    uint4* t4 = reinterpret_cast<uint4*>(tile);
    for (int w = threadIdx.x; w < (words >> 2); w += blockDim.x) t4[w] = make_uint4(0, 0, 0, 0);
    __syncthreads();

    const float* __restrict__ P = D.Pv;  // device memory, or pinned host memory (see InstDev)
    const float* __restrict__ Q = D.Qv;
    const int64_t count = I.c1 - I.c0;
    // the warp's batches of 32 circles; the next batch's pairs are loaded while this one is
    // walked
    int base = 0;
    if (lane == 0) base = atomicAdd(&s_next, 32);
    base = __shfl_sync(kFull, base, 0);
    float r[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (base + lane < count) load_pair(P, Q, I.c0 + base + lane, r);
    for (;;) {
      if (base >= count) break;
      float e1 = 0.f, e2 = 0.f, e3 = 0.f;
      const bool live = base + lane < count && circle_from(r, e1, e2, e3);
      int nbase = 0;
      if (lane == 0) nbase = atomicAdd(&s_next, 32);
      nbase = __shfl_sync(kFull, nbase, 0);
      if (nbase + lane < count) load_pair(P, Q, I.c0 + nbase + lane, r);
      // phase A: this lane's circle
      Prepared S;
      int steps = 0;  // segments of this circle
      if (live) {
        prepare(B, e1, e2, e3, S);
#pragma unroll
        for (int p = 0; p < 8; ++p) steps += segments_of(S.piece[p]);
      }
      int incl = steps;
#pragma unroll
      for (int s = 1; s < 32; s <<= 1) {
        const int v = __shfl_up_sync(kFull, incl, s);
        if (lane >= s) incl += v;
      }
      const int total = __shfl_sync(kFull, incl, 31);
      if (live) {
        store_rec(tab, lane, S, incl - steps);
      } else {
#pragma unroll
        for (int p = 0; p < 8; ++p) tab[(5 + p) * 32 + lane] = 0u;
        tab[13 * 32 + lane] = (uint32_t)(incl - steps);
        *reinterpret_cast<uint4*>(tab + 14 * 32 + 4 * lane) = make_uint4(0u, 0u, 0u, 0u);
      }
      __syncwarp();
      // phase B: the whole batch
      if (total > 0) walk_batch(B, tab, total, lane, dummy);
      __syncwarp();
      base = nbase;
    }
    __syncthreads();

    // the band -> this slice's partial
    uint4* out = reinterpret_cast<uint4*>(D.partial + ((int64_t)I.slice * D.G + B.R0) * B.W);
    for (int g = threadIdx.x; g < (words >> 2); g += blockDim.x) out[g] = t4[g];
    __syncthreads();
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

int vote_table_bytes() { return kWalkWarps * kTabWords * 4 + 32 * 4; }  // tables + dummy words

void launch_axis_vote_walk(const VoteItem* items, int n_items, const InstDev* insts, int* counter,
                           int grid_ctas, int tile_bytes, cudaStream_t st) {
  ensure_dynamic_smem(reinterpret_cast<const void*>(k_axis_vote_walk), kMaxSmemBytes);
  k_axis_vote_walk<<<grid_ctas, kWalkThreads, tile_bytes + vote_table_bytes(), st>>>(
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
