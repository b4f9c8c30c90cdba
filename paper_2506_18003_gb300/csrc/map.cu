// K5: (f, alpha) maps.
//
// Both maps are injective (no two estimator cells land on one grid point), so they are
// written as gathers: every grid point works out which cell, if any, lands on it and
// stores |S|^power or 0.  One write per grid point, no memset, no atomics.
//
// FAM (Algorithm 1 `FFT2` keeps the central band; Sec. II-B-2 gives f and alpha): cell
// (k, l, q), q in [-Q, Q) with Q = P L / Np, lands on fh = k + l + Np,
// ah = (k - l) Q + q + P L.  Inverse: s = fh - Np; d = k - l has the parity of s and
// q = (ah - P L) - d Q in [-Q, Q), so d = 2 floor((ah - P L - (s&1) Q + Q) / (2Q)) + (s&1).
// SSCA (Sec. II-C; Sec. III-B-1's mapping): cell (k, q) lands on ah = k N/Np + q + N,
// fh = floor((k N/Np - q + N) Np / (2N)).  Inverse: c = ah - N, k = fh - floor((N - c) Np / (2N)),
// q = c - k N/Np.
#include "fft.cuh"
#include "internal.h"

namespace scd {
namespace {

__device__ __forceinline__ float magp(float2 v, int power) {
  const float m2 = fmaf(v.x, v.x, v.y * v.y);
  return power == 2 ? m2 : sqrtf(m2);
}

// All extents are powers of two, so every division below is an exact shift (arithmetic
// shifts of negative values round toward minus infinity, i.e. floor).  Each thread writes
// 4 consecutive grid points of one row with a single 16-byte store.
__global__ void __launch_bounds__(256)
k_fam_map(const float2* __restrict__ S, int Np, int lnp, int P, int lw /*log2 2PL*/, int lq /*log2 Q*/,
          int power, float* __restrict__ map) {
  const int PL = 1 << (lw - 1), Q = 1 << lq;
  const int total4 = (2 * Np) << (lw - 2);
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < total4; g += gridDim.x * blockDim.x) {
    const int e = g << 2;
    const int fh = e >> lw;
    const int s = fh - Np;
    const int par = s & 1;
    float out[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int ah = (e + u) & ((1 << lw) - 1);
      const int t = (ah - PL - par * Q + Q) >> (lq + 1);
      const int d = 2 * t + par;
      const int q = ah - PL - d * Q;
      const int k = (s + d) >> 1, l = (s - d) >> 1;
      float val = 0.f;
      if (k >= -Np / 2 && k < Np / 2 && l >= -Np / 2 && l < Np / 2)
        val = magp(__ldg(S + ((((k + Np / 2) << lnp) + l + Np / 2) * (int64_t)P) + q + P / 2), power);
      out[u] = val;
    }
    *reinterpret_cast<float4*>(map + e) = make_float4(out[0], out[1], out[2], out[3]);
  }
}

// Runs of constant k are 2N/Np points long but start one point after a multiple of
// 2N/Np, so each of the 4 points of a group is resolved on its own.
__global__ void __launch_bounds__(256)
k_ssca_map(const float2* __restrict__ S, int ln /*log2 N*/, int lnp, int power, float* __restrict__ map) {
  const int N = 1 << ln, Np = 1 << lnp, D = 1 << (ln - lnp);
  const int total4 = Np << (ln + 1 - 2);
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < total4; g += gridDim.x * blockDim.x) {
    const int e = g << 2;
    const int fh = e >> (ln + 1);
    float out[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int ah = (e + u) & ((2 << ln) - 1);
      const int c = ah - N;
      const int k = fh - ((N - c) >> (ln + 1 - lnp));          // N - c > 0
      const int q = c - k * D;
      float val = 0.f;
      if (k >= -Np / 2 && k < Np / 2 && q >= -N / 2 && q < N / 2)
        val = magp(__ldg(S + ((int64_t)(k + Np / 2) << ln) + q + N / 2), power);
      out[u] = val;
    }
    *reinterpret_cast<float4*>(map + e) = make_float4(out[0], out[1], out[2], out[3]);
  }
}

int grid_cap(int64_t total) {
  int64_t g = (total + 255) / 256;
  return (int)(g < 152 * 16 ? g : 152 * 16);
}

}  // namespace

cudaError_t fam_map(const float2* S, int Np, int L, int P, int power, float* map, cudaStream_t st) {
  const int64_t PL = (int64_t)P * L;
  const int Q = (int)(PL / Np);
  if (!is_pow2(PL) || !is_pow2(Q) || 4 * (int64_t)Np * PL >= (int64_t(1) << 31)) return cudaErrorInvalidValue;
  const int64_t total4 = (int64_t)Np * PL;                      // 2Np x 2PL grid points / 4
  count_launches(1);
  k_fam_map<<<grid_cap(total4), 256, 0, st>>>(S, Np, ilog2(Np), P, ilog2(2 * PL), ilog2(Q), power, map);
  return cudaGetLastError();
}

cudaError_t ssca_map(const float2* S, int64_t N, int Np, int power, float* map, cudaStream_t st) {
  const int64_t total4 = (int64_t)Np * N / 2;                   // Np x 2N grid points / 4
  count_launches(1);
  k_ssca_map<<<grid_cap(total4), 256, 0, st>>>(S, ilog2(N), ilog2(Np), power, map);
  return cudaGetLastError();
}

}  // namespace scd
