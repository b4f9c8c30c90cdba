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

__device__ __forceinline__ int64_t floordiv(int64_t a, int64_t b) {   // b > 0
  const int64_t q = a / b;
  return (a % b != 0 && a < 0) ? q - 1 : q;
}

__device__ __forceinline__ float magp(float2 v, int power) {
  const float m2 = fmaf(v.x, v.x, v.y * v.y);
  return power == 2 ? m2 : sqrtf(m2);
}

__global__ void k_fam_map(const float2* __restrict__ S, int Np, int P, int64_t PL, int Q, int power,
                          float* __restrict__ map) {
  const int64_t W = 2 * PL;
  const int64_t total = 2 * (int64_t)Np * W;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t fh = e / W, ah = e % W;
    const int64_t s = fh - Np;
    const int64_t par = s & 1;
    const int64_t t = floordiv(ah - PL - par * Q + Q, 2 * (int64_t)Q);
    const int64_t d = 2 * t + par;
    const int64_t q = ah - PL - d * Q;
    const int64_t k = (s + d) / 2, l = (s - d) / 2;   // s + d is even
    float val = 0.f;
    if (k >= -Np / 2 && k < Np / 2 && l >= -Np / 2 && l < Np / 2) {
      const int64_t kh = k + Np / 2, lh = l + Np / 2;
      val = magp(__ldg(S + (kh * Np + lh) * P + q + P / 2), power);
    }
    map[e] = val;
  }
}

__global__ void k_ssca_map(const float2* __restrict__ S, int64_t N, int Np, int power, float* __restrict__ map) {
  const int64_t W = 2 * N;
  const int64_t D = N / Np;
  const int64_t total = (int64_t)Np * W;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t fh = e / W, ah = e % W;
    const int64_t c = ah - N;
    const int64_t k = fh - ((N - c) * Np) / (2 * N);   // N - c > 0
    const int64_t q = c - k * D;
    float val = 0.f;
    if (k >= -Np / 2 && k < Np / 2 && q >= -N / 2 && q < N / 2)
      val = magp(__ldg(S + (k + Np / 2) * N + q + N / 2), power);
    map[e] = val;
  }
}

int grid_cap(int64_t total) {
  int64_t g = (total + 255) / 256;
  return (int)(g < 152 * 64 ? g : 152 * 64);
}

}  // namespace

cudaError_t fam_map(const float2* S, int Np, int L, int P, int power, float* map, cudaStream_t st) {
  const int64_t PL = (int64_t)P * L;
  const int Q = (int)(PL / Np);
  const int64_t total = 2 * (int64_t)Np * 2 * PL;
  count_launches(1);
  k_fam_map<<<grid_cap(total), 256, 0, st>>>(S, Np, P, PL, Q, power, map);
  return cudaGetLastError();
}

cudaError_t ssca_map(const float2* S, int64_t N, int Np, int power, float* map, cudaStream_t st) {
  const int64_t total = (int64_t)Np * 2 * N;
  count_launches(1);
  k_ssca_map<<<grid_cap(total), 256, 0, st>>>(S, N, Np, power, map);
  return cudaGetLastError();
}

}  // namespace scd
