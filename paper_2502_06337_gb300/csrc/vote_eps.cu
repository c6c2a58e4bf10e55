// The consensus accumulator of Eq. 9 at cell resolution: circle i counts in cell c when some
// axis r of the cell has |r . z_i| < eps. With F(u, v) = 2 d1 u + 2 d2 v + d3 (u^2 + v^2 - 1)
// and F / (1 + u^2 + v^2) = d . r (Eq. 12, 13), the band is F_minus < 0 < F_plus with
// F_minus/plus = F -/+ eps |d| (1 + u^2 + v^2); both are separable quadratics, and a
// connected cell meets the band iff min_cell F_minus < 0 and max_cell F_plus > 0.
//
// Scanline form: for a row strip [v0, v1] the v parts reduce to their extremes over the strip
// (m = min of the F_minus part, M = max of the F_plus part), and the cell of column c meets
// the band iff [u_c, u_c+1] meets S1 = {u : Cm u^2 + 2 d1 u + m < 0} and meets
// S2 = {u : Cp u^2 + 2 d1 u + M > 0}, Cm/Cp = d3 -/+ eps |d|. Each set is at most two open
// intervals, so a row votes at most four disjoint column ranges.
//
// Work split. One warp takes one circle; its lanes take consecutive rows of the band, limited to
// the rows of the disc {F_minus < 0} when that set is a disc (d scaled by a power of two and
// signed so that d3 >= 0; then F_plus's quadratic term d3 + eps |d| is positive and
// {F_plus > 0} is the outside of a disc or a half-plane, met on every row). A row's ranges are
// entered as differences (+1 at a range's first column, -1 after its last) into a shared tile of
// row pairs, so a row costs its quadratics and at most eight atomics however long its ranges
// are. After the slice, prefix sums along the rows turn the tile into counts, which go to the
// slice's partial of the accumulator; the reduction of the curve vote sums the slices.
#include "row_tiles.cuh"
#include "sprot_internal.h"

namespace sprot {

namespace {

constexpr int kEpsThreads = 1024;

struct Ranges {
  int a[2], b[2];  // closed column ranges, sorted and disjoint; empty when a > b
  int n;
};

// Columns whose closed cell [u_c, u_c+1] meets the open interval (lo, hi): u_c+1 > lo and
// u_c < hi, i.e. floor((lo + 1) G/2) <= c <= ceil((hi + 1) G/2) - 1, clipped to the grid.
__device__ __forceinline__ void cols_meeting(float lo, float hi, float half, int G, int& a, int& b) {
  const float fa = floorf(fmaf(lo, half, half));
  const float fb = ceilf(fmaf(hi, half, half)) - 1.f;
  a = (int)fminf(fmaxf(fa, 0.f), (float)G);
  b = (int)fminf(fmaxf(fb, -1.f), (float)(G - 1));
}

// Roots r1 <= r2 of c u^2 + 2 b u + k (c != 0 with inv_c = 1/c, disc = b^2 - c k > 0),
// cancellation-free; quotients by correctly rounded reciprocals.
__device__ __forceinline__ void roots2(float inv_c, float b, float k, float disc, float& r1, float& r2) {
  const float q = -(b + copysignf(sqrtf(disc), b));
  const float x = q * inv_c, y = k * __frcp_rn(q);
  r1 = fminf(x, y);
  r2 = fmaxf(x, y);
}

// Hardware approximations (flush to zero): reciprocal square root and reciprocal, a few ulp.
__device__ __forceinline__ float rsqrt_apx(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rcp_apx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ int clampi(int x, int G) { return min(max(x, 0), G); }

// roots2 through the approximations, for disc > 1e-30 (so that the square root is a normal
// number and q cannot vanish).
__device__ __forceinline__ void roots2_apx(float inv_c, float b, float k, float disc, float& r1, float& r2) {
  const float q = -(b + copysignf(disc * rsqrt_apx(disc), b));
  const float x = q * inv_c, y = k * rcp_apx(q);
  r1 = fminf(x, y);
  r2 = fmaxf(x, y);
}

// Column ranges of the cells meeting {u : sgn * (c u^2 + 2 b u + k) < 0} (sgn = +1 for S1,
// -1 for S2).
__device__ __forceinline__ Ranges cell_ranges(float c, float inv_c, float b, float k, float sgn, float half,
                                               int G) {
  Ranges R;
  R.n = 0;
  const float inf = __int_as_float(0x7f800000);
  float lo0 = 0.f, hi0 = 0.f, lo1 = 0.f, hi1 = 0.f;
  int parts = 0;  // 0: empty, 1: (lo0, hi0), 2: (lo0, hi0) u (lo1, hi1), 3: everything
  if (c != 0.f) {
    const float disc = fmaf(-c, k, b * b);
    const bool up = sgn * c > 0.f;  // sgn q opens upwards: negative between the roots
    if (disc > 0.f) {
      float r1, r2;
      roots2(inv_c, b, k, disc, r1, r2);
      if (up) {
        lo0 = r1;
        hi0 = r2;
        parts = 1;
      } else {
        lo0 = -inf;
        hi0 = r1;
        lo1 = r2;
        hi1 = inf;
        parts = 2;
      }
    } else {
      parts = up ? 0 : 3;  // no sign change: sgn q >= 0 (up) or <= 0 (down) everywhere
    }
  } else {
    // linear: sgn (2 b u + k) < 0
    const float bb = sgn * b, kk = sgn * k;
    if (bb > 0.f) {
      lo0 = -inf;
      hi0 = -kk * __frcp_rn(2.f * bb);
      parts = 1;
    } else if (bb < 0.f) {
      lo0 = -kk * __frcp_rn(2.f * bb);
      hi0 = inf;
      parts = 1;
    } else {
      parts = kk < 0.f ? 3 : 0;
    }
  }
  if (parts == 3) {
    R.a[0] = 0;
    R.b[0] = G - 1;
    R.n = 1;
    return R;
  }
  if (parts >= 1) {
    cols_meeting(lo0, hi0, half, G, R.a[0], R.b[0]);
    R.n = 1;
  }
  if (parts == 2) {
    int a1, b1;
    cols_meeting(lo1, hi1, half, G, a1, b1);
    if (R.a[0] > R.b[0]) {  // first part empty
      R.a[0] = a1;
      R.b[0] = b1;
    } else if (a1 <= b1) {
      if (a1 <= R.b[0] + 1) {
        R.b[0] = max(R.b[0], b1);  // overlapping or adjacent: one range
      } else {
        R.a[1] = a1;
        R.b[1] = b1;
        R.n = 2;
      }
    }
  }
  return R;
}

// Enters the run of columns [a, b] of one row as a difference at the row's tile address
// rowbase (inc = 1 for the first row of a pair, 2^16 for the second).
__device__ __forceinline__ void vote_run(uint32_t rowbase, uint32_t inc, int G, int a, int b) {
  if (a > b) return;
  asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(rowbase + 4u * (uint32_t)a), "r"(inc) : "memory");
  if (b + 1 < G)
    asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(rowbase + 4u * (uint32_t)(b + 1)), "r"(0u - inc) : "memory");
}

// min (lo) or max (!lo) of c v^2 + 2 b v over [v0, v1] (inv_c = 1/c): the ends, and the
// vertex value -b^2/c when the derivative 2 (c v + b) changes sign inside.
__device__ __forceinline__ float quad_extreme(float c, float inv_c, float b, float v0, float v1, bool lo) {
  const float s0 = fmaf(c, v0, b), s1 = fmaf(c, v1, b);
  const float f0 = v0 * (s0 + b), f1 = v1 * (s1 + b);
  float r = lo ? fminf(f0, f1) : fmaxf(f0, f1);
  if (c != 0.f && ((s0 < 0.f && s1 > 0.f) || (s0 > 0.f && s1 < 0.f))) {
    const float fv = -b * b * inv_c;
    r = lo ? fminf(r, fv) : fmaxf(r, fv);
  }
  return r;
}

__global__ void __launch_bounds__(kEpsThreads, 1)
    k_axis_vote_eps(const VoteItem* __restrict__ items, int n_items, const InstDev* __restrict__ insts,
                    int* __restrict__ counter, float eps) {
  extern __shared__ __align__(16) uint32_t tile[];
  __shared__ int s_item;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
    __syncthreads();
    const int it = s_item;
    if (it >= n_items) break;
    const VoteItem I = items[it];
    const InstDev& D = insts[I.inst];
    const int G = D.G;
    const int R0 = D.band_row0[I.band], R1 = D.band_row0[I.band + 1];
    const float step = 2.0f / (float)G, half = 0.5f * (float)G;
    const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(tile);
    const int words = ((R1 - R0) >> 1) * G;
    uint4* t4 = reinterpret_cast<uint4*>(tile);
    for (int w = threadIdx.x; w < (words >> 2); w += blockDim.x) t4[w] = make_uint4(0, 0, 0, 0);
    __syncthreads();
    for (int64_t i = I.c0 + warp; i < I.c1; i += nwarps) {
      float d1 = __ldg(D.P + 3 * i) - __ldg(D.Q + 3 * i);
      float d2 = __ldg(D.P + 3 * i + 1) - __ldg(D.Q + 3 * i + 1);
      float d3 = __ldg(D.P + 3 * i + 2) - __ldg(D.Q + 3 * i + 2);
      const float m = fmaxf(fabsf(d1), fmaxf(fabsf(d2), fabsf(d3)));
      if (m == 0.f) continue;  // degenerate: no circle
      // scaled to max |d_k| in [1, 2) and signed so that d3 >= 0 (-d gives the same band: F_minus
      // and F_plus exchange and change sign)
      const float sc = (d3 < 0.f ? -1.f : 1.f) * inv_pow2_of(m);
      d1 *= sc;
      d2 *= sc;
      d3 *= sc;
      const float ed = eps * sqrtf(fmaf(d1, d1, fmaf(d2, d2, d3 * d3)));
      const float Cm = d3 - ed, Cp = d3 + ed;
      const float iCm = Cm != 0.f ? __frcp_rn(Cm) : 0.f, iCp = Cp != 0.f ? __frcp_rn(Cp) : 0.f;
      if (Cm > 1e-20f) {
        // Cm > 0 (below 1e-20 the general rows below: a disc far beyond the grid's reach of
        // float32). {F_minus < 0} is the disc of centre -(d1, d2)/Cm and radius sqrt(d1^2 + d2^2 + Cm Cp)/Cm:
        // rows beyond its extent (with a margin for the float32 error of the bounds) have
        // min F_minus > 0 well outside the decision band
        const float vc = -d2 * iCm, rad = sqrtf(fmaf(d1, d1, fmaf(d2, d2, Cm * Cp))) * iCm;
        const float mg = 2.f + 1e-5f * (fabsf(vc) + rad) * half;
        const float flo = fmaf(vc - rad, half, half) - mg, fhi = fmaf(vc + rad, half, half) + mg;
        const int r_lo = max(R0, (int)floorf(fminf(fmaxf(flo, -1.f), (float)G)));
        const int r_hi = min(R1 - 1, (int)fminf(fmaxf(fhi, -1.f), (float)G));
        // S1 is one interval (the disc's chord) or empty, S2 the outside of one interval or
        // everything, so a row votes at most two runs. A discriminant at most 1e-30 leaves a
        // sliver of S1 (no cell) or of S2's complement (no cell inside it) whose cells have |F|
        // below 1e-10: inside the decision band.
        //
        // The v parts Cm v^2 + 2 d2 v and Cp v^2 + 2 d2 v are convex: the maximum of the second
        // over a strip is at one of its lines, and so is the minimum of the first except in the
        // strip holding its vertex vc, where it is -d2^2/Cm. (A vertex within rounding of a line
        // gives the two strips beside it minima that differ by a square of that rounding.)
        const int rv = __float2int_rd(fmaf(vc, half, half));
        const float hvert = -d2 * d2 * iCm, d2x2 = d2 + d2;
        for (int r = r_lo + lane; r <= r_hi; r += 32) {
          const float v0 = fmaf((float)r, step, -1.f), v1 = v0 + step;
          float hm = fminf(v0 * fmaf(Cm, v0, d2x2), v1 * fmaf(Cm, v1, d2x2));
          if (r == rv) hm = fminf(hm, hvert);
          const float mr = hm - Cp;
          const float discA = fmaf(-Cm, mr, d1 * d1);
          if (!(discA > 1e-30f)) continue;
          float r1, r2;
          roots2_apx(iCm, d1, mr, discA, r1, r2);
          // cells meeting (r1, r2): columns floor((r1 + 1) G/2) .. ceil((r2 + 1) G/2) - 1, the
          // saturated conversions clamped to [0, G] before the subtraction
          const int a0 = clampi(__float2int_rd(fmaf(r1, half, half)), G);
          const int a1 = clampi(__float2int_ru(fmaf(r2, half, half)), G) - 1;
          const float Mr = fmaxf(v0 * fmaf(Cp, v0, d2x2), v1 * fmaf(Cp, v1, d2x2)) - Cm;
          const float discB = fmaf(-Cp, Mr, d1 * d1);
          int x1 = G - 1, x2 = G;  // S2's columns: [0, x1] and [x2, G - 1]
          if (discB > 1e-30f) {
            float s1, s2;
            roots2_apx(iCp, d1, Mr, discB, s1, s2);
            x1 = clampi(__float2int_ru(fmaf(s1, half, half)), G) - 1;
            x2 = clampi(__float2int_rd(fmaf(s2, half, half)), G);
          }
          const uint32_t rowbase = sbase + 4u * (uint32_t)(((r - R0) >> 1) * G);
          const uint32_t inc = ((r - R0) & 1) ? 0x10000u : 1u;
          if (x2 <= x1 + 1) {
            vote_run(rowbase, inc, G, a0, a1);
          } else {
            vote_run(rowbase, inc, G, a0, min(a1, x1));
            vote_run(rowbase, inc, G, max(a0, x2), a1);
          }
        }
        continue;
      }
      for (int r = R0 + lane; r < R1; r += 32) {  // Cm <= 0 (about 0.2% of the headline's circles)
        const float v0 = fmaf((float)r, step, -1.f), v1 = fmaf((float)(r + 1), step, -1.f);
        // F_minus = Cm (u^2 + v^2) + 2 d1 u + 2 d2 v - Cp ; F_plus = Cp (u^2 + v^2) + 2 d1 u + 2 d2 v - Cm
        const float mr = quad_extreme(Cm, iCm, d2, v0, v1, true) - Cp;
        const float Mr = quad_extreme(Cp, iCp, d2, v0, v1, false) - Cm;
        const Ranges A = cell_ranges(Cm, iCm, d1, mr, 1.f, half, G);   // Cm u^2 + 2 d1 u + mr < 0
        const Ranges B = cell_ranges(Cp, iCp, d1, Mr, -1.f, half, G);  // Cp u^2 + 2 d1 u + Mr > 0
        const uint32_t rowbase = sbase + 4u * (uint32_t)(((r - R0) >> 1) * G);
        const uint32_t inc = ((r - R0) & 1) ? 0x10000u : 1u;
        for (int x = 0; x < A.n; ++x)
          for (int y = 0; y < B.n; ++y) vote_run(rowbase, inc, G, max(A.a[x], B.a[y]), min(A.b[x], B.b[y]));
      }
    }
    __syncthreads();
    flush_row_pair_tile(tile, G, G, R0, R1, D.partial + (int64_t)I.slice * G * (G >> 1));
    __syncthreads();
  }
}

}  // namespace

void launch_axis_vote_eps(const VoteItem* items, int n_items, const InstDev* insts, int* counter, int grid_ctas,
                          int tile_bytes, float eps, cudaStream_t st) {
  ensure_dynamic_smem(reinterpret_cast<const void*>(k_axis_vote_eps), tile_bytes);
  k_axis_vote_eps<<<grid_ctas, kEpsThreads, tile_bytes, st>>>(items, n_items, insts, counter, eps);
  launches_add(1);
}

}  // namespace sprot
