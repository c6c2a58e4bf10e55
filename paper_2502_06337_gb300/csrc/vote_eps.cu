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
// intervals, so a row votes at most four disjoint column ranges. One warp takes one circle;
// its lanes take consecutive rows of the band (neighbouring rows have similar spans). Votes go
// to the same shared band tiles (two u16 counters per word) and slice partials as the curve
// vote, and the same reduction sums them.
#include "sprot_internal.h"

namespace sprot {

namespace {

constexpr int kEpsThreads = 512;

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

// Adds one to the cells of row `row` (relative to the tile) in columns [a, b]; two adjacent
// columns share a word (low half even, high half odd).
__device__ __forceinline__ void vote_span(uint32_t sbase, int W, int row, int a, int b) {
  if (a > b) return;
  uint32_t addr = sbase + 4u * (uint32_t)(row * W + (a >> 1));
  int c = a;
  if (c & 1) {
    asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(addr), "r"(0x10000u) : "memory");
    addr += 4;
    ++c;
  }
  for (; c + 1 <= b; c += 2, addr += 4)
    asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(addr), "r"(0x10001u) : "memory");
  if (c == b) asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(addr), "r"(1u) : "memory");
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
    const int G = D.G, W = G >> 1;
    const int R0 = D.band_row0[I.band], R1 = D.band_row0[I.band + 1];
    const float step = 2.0f / (float)G, half = 0.5f * (float)G;
    const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(tile);
    const int words = (R1 - R0) * W;
    uint4* t4 = reinterpret_cast<uint4*>(tile);
    for (int w = threadIdx.x; w < (words >> 2); w += blockDim.x) t4[w] = make_uint4(0, 0, 0, 0);
    __syncthreads();
    for (int64_t i = I.c0 + warp; i < I.c1; i += nwarps) {
      float d1 = __ldg(D.P + 3 * i) - __ldg(D.Q + 3 * i);
      float d2 = __ldg(D.P + 3 * i + 1) - __ldg(D.Q + 3 * i + 1);
      float d3 = __ldg(D.P + 3 * i + 2) - __ldg(D.Q + 3 * i + 2);
      const float m = fmaxf(fabsf(d1), fmaxf(fabsf(d2), fabsf(d3)));
      if (m == 0.f) continue;  // degenerate: no circle
      const int e = ilogbf(m);
      d1 = scalbnf(d1, -e);
      d2 = scalbnf(d2, -e);
      d3 = scalbnf(d3, -e);
      const float ed = eps * sqrtf(fmaf(d1, d1, fmaf(d2, d2, d3 * d3)));
      const float Cm = d3 - ed, Cp = d3 + ed;
      const float iCm = Cm != 0.f ? __frcp_rn(Cm) : 0.f, iCp = Cp != 0.f ? __frcp_rn(Cp) : 0.f;
      for (int r = R0 + lane; r < R1; r += 32) {
        const float v0 = fmaf((float)r, step, -1.f), v1 = fmaf((float)(r + 1), step, -1.f);
        // F_minus = Cm (u^2 + v^2) + 2 d1 u + 2 d2 v - Cp ; F_plus = Cp (u^2 + v^2) + 2 d1 u + 2 d2 v - Cm
        const float mr = quad_extreme(Cm, iCm, d2, v0, v1, true) - Cp;
        const float Mr = quad_extreme(Cp, iCp, d2, v0, v1, false) - Cm;
        const Ranges A = cell_ranges(Cm, iCm, d1, mr, 1.f, half, G);   // Cm u^2 + 2 d1 u + mr < 0
        const Ranges B = cell_ranges(Cp, iCp, d1, Mr, -1.f, half, G);  // Cp u^2 + 2 d1 u + Mr > 0
        for (int x = 0; x < A.n; ++x)
          for (int y = 0; y < B.n; ++y)
            vote_span(sbase, W, r - R0, max(A.a[x], B.a[y]), min(A.b[x], B.b[y]));
      }
    }
    __syncthreads();
    uint4* out = reinterpret_cast<uint4*>(D.partial + ((int64_t)I.slice * G + R0) * W);
    for (int g = threadIdx.x; g < (words >> 2); g += blockDim.x) out[g] = t4[g];
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
