// Axis vote with the whole accumulator in the distributed shared memory of a thread-block
// cluster (Algorithm 1; Sec. IV-A).
//
// A cluster of C CTAs holds one G x G accumulator as 16-bit counters, CTA r owning rows
// [r G/C, (r+1) G/C) (128 KB per CTA for G = 256, C = 1; G = 512, C = 4; G = 1024, C = 16).
// Every circle of a work item is rasterised once by one warp of the cluster, and each voted
// cell is incremented in the owning CTA's shared memory with red.shared::cluster.add (a plain
// red.shared.add when C = 1). The cluster then writes its accumulator to a per-slice partial
// that the reduce kernel sums.
//
// Rasterisation. d = p - q (scaled by a power of two, sign chosen so d3 >= 0) defines
// F(u, v) = 2 d1 u + 2 d2 v + d3 (u^2 + v^2 - 1), whose zero set is the projected great circle
// (Eq. 13, D = 0). The circle is cut at its 45-degree points: columns between them are
// x-major (each vertical grid line meets the circle twice, in the top and bottom arcs), the
// other columns are y-major and are handled row by row. One lane takes one grid line and
// solves F = 0 on it for both crossings (one quadratic, in the form free of cancellation); the
// cells of a column are the rows between the crossings on its two lines, for each arc, plus
// the top or bottom point of the circle in the column that holds the centre. A crossing is
// turned into a row by a plain floor: a crossing within rounding of a grid edge puts the
// corner of the cell within ~1e-7 |d| of the curve, inside the band where the closed-cell test
// may go either way.
#include <stdint.h>

#include "sprot_internal.h"

namespace sprot {

namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ float edgef(int k, float step) { return fmaf((float)k, step, -1.0f); }

// Both roots of c3 y^2 + 2 b y + kk = 0, c3 >= 0, lo <= hi; inv3 = 1 / c3 (+inf for c3 = 0).
// Callers guarantee disc > 0 except on lines they skip (then the roots are NaN).
__device__ __forceinline__ void roots(float c3, float inv3, float b, float kk, float& lo,
                                      float& hi) {
  float disc = fmaf(-c3, kk, b * b);
  float t = fabsf(b) + sqrtf(disc);
  float far = t * inv3;
  float nr = kk * __frcp_rn(t);
  lo = b >= 0.f ? -far : nr;
  hi = b >= 0.f ? -nr : far;
}

// Cell index of plane coordinate y, clamped to [-1, G] (NaN -> -1).
__device__ __forceinline__ int cell_of(float y, float half, float Gf) {
  float s = fminf(fmaxf(fmaf(y, half, half), -1.f), Gf);
  return __float2int_rd(s);
}

template <int C>
struct ClusterTile {
  uint32_t sbase;  // this CTA's tile, shared::cta address
  int G, W, swz, rc_shift, rc_mask;

  __device__ __forceinline__ void vote(int r, int c) const {
    int lr = r & rc_mask;
    uint32_t word = (uint32_t)(lr * W + ((c & (W - 1)) ^ (lr & swz)));
    uint32_t inc = c >= W ? 0x10000u : 1u;
    uint32_t a = sbase + 4u * word;
    if (C == 1) {
      asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(a), "r"(inc) : "memory");
    } else {
      uint32_t owner = (uint32_t)(r >> rc_shift), ra;
      asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(a), "r"(owner));
      asm volatile("red.shared::cluster.add.u32 [%0], %1;" ::"r"(ra), "r"(inc) : "memory");
    }
  }
};

__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::
                   : "memory");
}

template <int C>
__device__ __forceinline__ void rasterise(const ClusterTile<C>& T, float d1, float d2, float d3,
                                          int lane) {
  const int G = T.G;
  const float Gf = (float)G, step = 2.0f / Gf, half = 0.5f * Gf;
  const float INF = __int_as_float(0x7f800000);
  const float nd = sqrtf(fmaf(d1, d1, fmaf(d2, d2, d3 * d3)));
  const float d1x2 = 2.f * d1, d2x2 = 2.f * d2;
  float inv3;
  int jA, jB, jc, ic, Rtop = 0, Rbot = 0, Cl = 0, Cr = 0, yr0, yr1;
  if (d3 <= 1e-8f * nd) {
    // a line through the origin (d3 = 0 up to a change of F below 2e-8 |d|)
    d3 = 0.f;
    inv3 = INF;
    jc = ic = -100;
    if (fabsf(d2) >= fabsf(d1)) {
      jA = -1;
      jB = G;
      yr0 = 1;
      yr1 = 0;
    } else {
      jA = G - 1;
      jB = G;
      yr0 = 0;
      yr1 = G - 1;
    }
  } else {
    inv3 = __frcp_rn(d3);
    const float s = 0.70710678f;
    // 45-degree points cx -/+ rho/sqrt(2) without cancellation
    float q1 = fmaf(d2, d2, d3 * d3) - d1 * d1;
    float uA = d1 >= 0.f ? -(d1 + s * nd) * inv3 : -0.5f * q1 / ((s * nd - d1) * d3);
    float uB = d1 <= 0.f ? (s * nd - d1) * inv3 : 0.5f * q1 / ((s * nd + d1) * d3);
    jA = min(max(__float2int_rd(fminf(fmaxf(fmaf(uA, half, half), -2.f), Gf + 2.f)), -1), G - 1);
    jB = min(max(__float2int_rd(fminf(fmaxf(fmaf(uB, half, half), -2.f), Gf + 2.f)), 0), G);
    jc = __float2int_rd(fminf(fmaxf(fmaf(-d1 * inv3, half, half), -4.f), Gf + 4.f));
    ic = __float2int_rd(fminf(fmaxf(fmaf(-d2 * inv3, half, half), -4.f), Gf + 4.f));
    float lo, hi;
    roots(d3, inv3, d2, -fmaf(d1, d1, d3 * d3) * inv3, lo, hi);
    Rbot = cell_of(lo, half, Gf);
    Rtop = cell_of(hi, half, Gf);
    roots(d3, inv3, d1, -fmaf(d2, d2, d3 * d3) * inv3, lo, hi);
    Cl = cell_of(lo, half, Gf);
    Cr = cell_of(hi, half, Gf);
    // rows holding the y-major parts: within the chords at lines jA + 1 and jB
    yr0 = 1 << 30;
    yr1 = -(1 << 30);
    if (jA >= 0) {
      float x = edgef(jA + 1, step);
      roots(d3, inv3, d2, fmaf(d3, fmaf(x, x, -1.f), d1x2 * x), lo, hi);
      yr0 = min(yr0, cell_of(lo, half, Gf) - 1);
      yr1 = max(yr1, cell_of(hi, half, Gf) + 1);
    }
    if (jB <= G - 1) {
      float x = edgef(jB, step);
      roots(d3, inv3, d2, fmaf(d3, fmaf(x, x, -1.f), d1x2 * x), lo, hi);
      yr0 = min(yr0, cell_of(lo, half, Gf) - 1);
      yr1 = max(yr1, cell_of(hi, half, Gf) + 1);
    }
    yr0 = max(yr0, 0);
    yr1 = min(yr1, G - 1);
  }

  // x-major columns [xj0, xj1]: lane l takes vertical line xj0 + l; column j uses lines j, j+1
  const int xj0 = max(jA + 1, 0), xj1 = min(jB - 1, G - 1);
  for (int base = xj0; base <= xj1; base += 31) {
    const int l = base + lane;
    const float x = edgef(l, step);
    float lo, hi;
    roots(d3, inv3, d2, fmaf(d3, fmaf(x, x, -1.f), d1x2 * x), lo, hi);
    const int Rl = cell_of(lo, half, Gf), Rh = cell_of(hi, half, Gf);
    const int Rln = __shfl_down_sync(kFull, Rl, 1), Rhn = __shfl_down_sync(kFull, Rh, 1);
    if (lane < 31 && l <= xj1) {
      int a = max(min(Rh, Rhn), 0), b = max(Rh, Rhn);
      if (l == jc) b = max(b, Rtop);
      b = min(b, G - 1);
      for (int r = a; r <= b; ++r) T.vote(r, l);
      a = min(Rl, Rln);
      b = min(max(Rl, Rln), G - 1);
      if (l == jc) a = min(a, Rbot);
      a = max(a, 0);
      for (int r = a; r <= b; ++r) T.vote(r, l);
    }
  }
  // y-major part: lane l takes horizontal line yr0 + l; only columns <= jA or >= jB
  for (int base = yr0; base <= yr1; base += 31) {
    const int l = base + lane;
    const float x = edgef(l, step);
    float lo, hi;
    const float kk = fmaf(d3, fmaf(x, x, -1.f), d2x2 * x);
    const bool ok = fmaf(-d3, kk, d1 * d1) >= 0.f;  // the line meets the circle
    roots(d3, inv3, d1, kk, lo, hi);
    const int Cl0 = cell_of(lo, half, Gf), Ch0 = cell_of(hi, half, Gf);
    const int Cln = __shfl_down_sync(kFull, Cl0, 1), Chn = __shfl_down_sync(kFull, Ch0, 1);
    const bool okn = __shfl_down_sync(kFull, ok, 1);
    if (lane < 31 && l <= yr1 && ok && okn) {
      int a = min(Cl0, Cln), b = max(Cl0, Cln);
      if (l == ic) a = min(a, Cl);
      for (int c = max(a, 0); c <= min(b, jA); ++c) T.vote(l, c);
      for (int c = max(a, jB); c <= min(b, G - 1); ++c) T.vote(l, c);
      a = min(Ch0, Chn);
      b = max(Ch0, Chn);
      if (l == ic) b = max(b, Cr);
      for (int c = max(a, 0); c <= min(b, jA); ++c) T.vote(l, c);
      for (int c = max(a, jB); c <= min(b, G - 1); ++c) T.vote(l, c);
    }
  }
}

// p - q scaled by a power of two so that max |d_k| is in [1, 2), signed so d3 >= 0.
__device__ __forceinline__ bool circle_of(const float* __restrict__ P, const float* __restrict__ Q,
                                          int64_t i, float& d1, float& d2, float& d3) {
  d1 = __ldg(P + 3 * i) - __ldg(Q + 3 * i);
  d2 = __ldg(P + 3 * i + 1) - __ldg(Q + 3 * i + 1);
  d3 = __ldg(P + 3 * i + 2) - __ldg(Q + 3 * i + 2);
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

template <int C>
__global__ void __launch_bounds__(kVoteThreads, 1)
    k_axis_vote_cluster(const VoteItem* __restrict__ items, int n_items,
                        const InstDev* __restrict__ insts, int* __restrict__ counter) {
  extern __shared__ __align__(16) uint32_t tile[];
  __shared__ int s_next, s_item;
  const int lane = threadIdx.x & 31;
  uint32_t rank = 0, cid = blockIdx.x, ncl = gridDim.x;
  if (C > 1) {
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(rank));
    asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(cid));
    asm volatile("mov.u32 %0, %%nclusterid.x;" : "=r"(ncl));
  }
  int it = (int)cid;
  for (;;) {
    if (C == 1) {  // one CTA per accumulator: take items from a global queue
      if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
      __syncthreads();
      it = s_item;
    }
    if (it >= n_items) break;
    const VoteItem I = items[it];
    const InstDev& D = insts[I.inst];
    ClusterTile<C> T;
    T.G = D.G;
    T.W = D.G >> 1;
    T.swz = min(T.W, 32) - 1;
    const int rc = D.G / C;  // rows owned by each CTA
    T.rc_shift = __ffs(rc) - 1;
    T.rc_mask = rc - 1;
    T.sbase = (uint32_t)__cvta_generic_to_shared(tile);
    const int words = rc * T.W;
    uint4* t4 = reinterpret_cast<uint4*>(tile);
    for (int w = threadIdx.x; w < (words >> 2); w += blockDim.x) t4[w] = make_uint4(0, 0, 0, 0);
    if (threadIdx.x == 0) s_next = 0;
    if (C > 1)
      cluster_sync();
    else
      __syncthreads();

    const float* __restrict__ P = D.P;
    const float* __restrict__ Q = D.Q;
    const int64_t span = I.c1 - I.c0;
    const int64_t m0 = I.c0 + span * rank / C, m1 = I.c0 + span * (rank + 1) / C;
    const int64_t count = m1 - m0;
    for (;;) {
      int base = 0;
      if (lane == 0) base = atomicAdd(&s_next, 32);
      base = __shfl_sync(kFull, base, 0);
      if (base >= count) break;
      float e1 = 0.f, e2 = 0.f, e3 = 0.f;
      bool live = false;
      if (base + lane < count) live = circle_of(P, Q, m0 + base + lane, e1, e2, e3);
      unsigned mask = __ballot_sync(kFull, live);
      while (mask) {
        const int src = __ffs(mask) - 1;
        mask &= mask - 1;
        const float d1 = __shfl_sync(kFull, e1, src);
        const float d2 = __shfl_sync(kFull, e2, src);
        const float d3 = __shfl_sync(kFull, e3, src);
        rasterise<C>(T, d1, d2, d3, lane);
      }
    }
    if (C > 1)
      cluster_sync();
    else
      __syncthreads();

    // this CTA's rows -> the item's partial, undoing the row swizzle four words at a time
    uint32_t* out = D.partial + ((int64_t)I.slice * D.G + (int64_t)rank * rc) * T.W;
    for (int g = threadIdx.x; g < (words >> 2); g += blockDim.x) {
      const int rr = (g * 4) / T.W;
      const int wp = g * 4 - rr * T.W;
      const int x = rr & T.swz;
      const uint4 v = t4[g];
      const uint32_t e[4] = {v.x, v.y, v.z, v.w};
      const int p = x & 3;
      uint4 o;
      o.x = e[0 ^ p];
      o.y = e[1 ^ p];
      o.z = e[2 ^ p];
      o.w = e[3 ^ p];
      *reinterpret_cast<uint4*>(out + (int64_t)rr * T.W + (wp ^ (x & ~3))) = o;
    }
    __syncthreads();
    if (C > 1) it += (int)ncl;
  }
}

template <int C>
cudaError_t launch_c(const VoteItem* items, int n_items, const InstDev* insts, int* counter,
                     int n_ctas, int smem, cudaStream_t st) {
  auto kern = k_axis_vote_cluster<C>;
  static bool init = false;
  if (!init) {
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmemBytes);
    if (C > 8) cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    init = true;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(n_ctas, 1, 1);
  cfg.blockDim = dim3(kVoteThreads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = C > 1 ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kern, items, n_items, insts, counter);
}

template <int C>
int max_clusters_c(int smem) {
  auto kern = k_axis_vote_cluster<C>;
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmemBytes);
  if (C > 8) cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(C * 64, 1, 1);
  cfg.blockDim = dim3(kVoteThreads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, kern, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

}  // namespace

int cluster_size_for(int G) {
  long long bytes = (long long)G * G * 2;  // 16-bit counters
  long long per = 128 * 1024;
  int C = (int)((bytes + per - 1) / per);
  if (C <= 1) return 1;
  if (C <= 2) return 2;
  if (C <= 4) return 4;
  if (C <= 8) return 8;
  if (C <= 16) return 16;
  return 0;  // does not fit a cluster: banded kernel
}

int max_active_clusters(int C, int smem) {
  switch (C) {
    case 1: return 0;
    case 2: return max_clusters_c<2>(smem);
    case 4: return max_clusters_c<4>(smem);
    case 8: return max_clusters_c<8>(smem);
    case 16: return max_clusters_c<16>(smem);
  }
  return 0;
}

void launch_axis_vote_cluster(int C, const VoteItem* items, int n_items, const InstDev* insts,
                              int* counter, int n_ctas, int smem, cudaStream_t st) {
  switch (C) {
    case 1: launch_c<1>(items, n_items, insts, counter, n_ctas, smem, st); break;
    case 2: launch_c<2>(items, n_items, insts, counter, n_ctas, smem, st); break;
    case 4: launch_c<4>(items, n_items, insts, counter, n_ctas, smem, st); break;
    case 8: launch_c<8>(items, n_items, insts, counter, n_ctas, smem, st); break;
    case 16: launch_c<16>(items, n_items, insts, counter, n_ctas, smem, st); break;
  }
  launches_add(1);
}

}  // namespace sprot
