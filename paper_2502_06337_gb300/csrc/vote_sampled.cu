// Algorithm 1's accumulator taken literally: every great circle is drawn as J points
// alpha1 cos(t_j) + alpha2 sin(t_j), t_j = -pi + 2 pi j / J, each projected by Eq. 11, and
// every point inside the square [-1, 1]^2 adds one to its cell (a cell can receive several
// votes from one circle, and a cell the circle only grazes may receive none).
//
// One warp draws one circle: all lanes build the basis (broadcast loads of the pair), and
// lane l takes the points j = l, l + 32, ... The angles' cosines and sines are tabulated
// once per block in shared memory. Votes go to the caller's grid in global memory with
// red.global.add (the grid lives in L2: 1 MB at G = 512).
#include <algorithm>

#include "sprot_internal.h"

namespace sprot {

namespace {

constexpr int kSampledThreads = 256;

__global__ void __launch_bounds__(kSampledThreads)
    k_axis_vote_sampled(const float* __restrict__ P, const float* __restrict__ Q, int64_t n, int G,
                        int J, uint32_t* __restrict__ grid) {
  extern __shared__ float2 cs[];  // (cos t_j, sin t_j)
  for (int j = threadIdx.x; j < J; j += blockDim.x) {
    float s, c;
    // t_j / pi = -1 + 2 j / J
    sincospif(fmaf(2.0f / (float)J, (float)j, -1.0f), &s, &c);
    cs[j] = make_float2(c, s);
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  const float half = 0.5f * (float)G;
  for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < n; i += warps) {
    const float d1 = __ldg(P + 3 * i) - __ldg(Q + 3 * i);
    const float d2 = __ldg(P + 3 * i + 1) - __ldg(Q + 3 * i + 1);
    const float d3 = __ldg(P + 3 * i + 2) - __ldg(Q + 3 * i + 2);
    if (d1 == 0.f && d2 == 0.f && d3 == 0.f) continue;  // degenerate: no circle
    // z = d / |d| (scaled first so that the squares cannot overflow or underflow)
    const float m = fmaxf(fabsf(d1), fmaxf(fabsf(d2), fabsf(d3)));
    const int e = ilogbf(m);
    const float s1 = scalbnf(d1, -e), s2 = scalbnf(d2, -e), s3 = scalbnf(d3, -e);
    const float inv = rsqrtf(fmaf(s1, s1, fmaf(s2, s2, s3 * s3)));
    const float z1 = s1 * inv, z2 = s2 * inv, z3 = s3 * inv;
    // alpha1 = normalised alpha0 - (alpha0 . z) z with alpha0 = e3, i.e.
    // (-z3 z1, -z3 z2, z1^2 + z2^2) / sqrt(z1^2 + z2^2) without cancellation; alpha0 = e1
    // when d1 = d2 = 0 (z = +-e3), where alpha1 = e1.
    float a1x, a1y, a1z;
    if (d1 == 0.f && d2 == 0.f) {
      a1x = 1.f;
      a1y = 0.f;
      a1z = 0.f;
    } else {
      const float na = sqrtf(fmaf(z1, z1, z2 * z2));
      const float r = 1.0f / na;
      a1x = -z3 * z1 * r;
      a1y = -z3 * z2 * r;
      a1z = na;
    }
    // alpha2 = alpha1 x z
    const float a2x = a1y * z3 - a1z * z2;
    const float a2y = a1z * z1 - a1x * z3;
    const float a2z = a1x * z2 - a1y * z1;
    for (int j = lane; j < J; j += 32) {
      const float2 t = cs[j];
      const float X = fmaf(a1x, t.x, a2x * t.y);
      const float Y = fmaf(a1y, t.x, a2y * t.y);
      const float W = 1.0f - fmaf(a1z, t.x, a2z * t.y);
      // A point of the square has u^2 + v^2 = (2 - W)/W <= 2, i.e. W >= 2/3; W <= 1/2 is
      // outside. The bound also drops the pole itself (W = 0 exactly), which float32 can see
      // as a tiny positive W with X = Y = 0 and would otherwise vote the centre cell.
      if (!(W > 0.5f)) continue;
      const float rw = 1.0f / W;
      const float u = X * rw, v = Y * rw;
      if (!(fabsf(u) < 1.f && fabsf(v) < 1.f)) continue;
      const int col = min(max((int)floorf(fmaf(u, half, half)), 0), G - 1);
      const int row = min(max((int)floorf(fmaf(v, half, half)), 0), G - 1);
      atomicAdd(grid + (int64_t)row * G + col, 1u);
    }
  }
}

}  // namespace

int launch_axis_vote_sampled(const float* P, const float* Q, int64_t n, int G, int J, uint32_t* grid,
                             int n_sm, cudaStream_t st) {
  if (cudaMemsetAsync(grid, 0, sizeof(uint32_t) * (size_t)G * G, st) != cudaSuccess) return SPROT_E_CUDA;
  const int64_t warps_needed = n;
  const int per_block = kSampledThreads / 32;
  const int64_t blocks = std::min<int64_t>((warps_needed + per_block - 1) / per_block, (int64_t)n_sm * 8);
  k_axis_vote_sampled<<<(int)std::max<int64_t>(blocks, 1), kSampledThreads, sizeof(float2) * J, st>>>(
      P, Q, n, G, J, grid);
  launches_add(1);
  return cudaGetLastError() == cudaSuccess ? SPROT_OK : SPROT_E_CUDA;
}

}  // namespace sprot
