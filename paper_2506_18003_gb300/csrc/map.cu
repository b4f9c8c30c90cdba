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
// The conjugate FAM estimate (X(p,k) Y(p,l)) has f = (f_k - f_l)/2, alpha = f_k + f_l +
// q/(P L): fh = k - l + Np, ah = (k + l) Q + q + P L, the same inverse with the roles of
// s = k + l and d = k - l exchanged.
// SSCA (Sec. II-C; Sec. III-B-1's mapping): cell (k, q) lands on ah = k N/Np + q + N,
// fh = floor((k N/Np - q + N) Np / (2N)).  Inverse: c = ah - N, k = fh - floor((N - c) Np / (2N)),
// q = c - k N/Np.
//
// Alpha profiles: profile[ah] = max over the cells of column ah of |S|^power.  A gather per
// column again: FAM column c = ah - P L holds the cells with k - l (k + l for the conjugate
// estimate) equal to v in {t - 1, t}, t = floor((c + Q)/Q), at q = c - v Q; SSCA column c
// holds channel k at q = c - k N/Np for the k with q in [-N/2, N/2).  Consecutive columns
// read consecutive q of one channel row, so the warps' loads are contiguous; the maximum of
// |S|^2 is taken first and the square root (monotone) applied once.
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
          int power, int conj, float* __restrict__ map) {
  const int PL = 1 << (lw - 1), Q = 1 << lq;
  const int total4 = (2 * Np) << (lw - 2);
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < total4; g += gridDim.x * blockDim.x) {
    const int e = g << 2;
    const int fh = e >> lw;
    const int s = fh - Np;                                      // k + l (conjugate: k - l)
    const int par = s & 1;
    float out[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int ah = (e + u) & ((1 << lw) - 1);
      const int t = (ah - PL - par * Q + Q) >> (lq + 1);
      const int d = 2 * t + par;                                // k - l (conjugate: k + l)
      const int q = ah - PL - d * Q;
      const int k = (s + d) >> 1, l = conj ? (d - s) >> 1 : (s - d) >> 1;
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

__device__ __forceinline__ float mag2(float2 v) { return fmaf(v.x, v.x, v.y * v.y); }

__global__ void __launch_bounds__(256)
k_fam_profile(const float2* __restrict__ S, int Np, int lnp, int P, int lw /*log2 2PL*/, int lq /*log2 Q*/,
              int power, int conj, float* __restrict__ prof) {
  const int PL = 1 << (lw - 1), Q = 1 << lq, H = Np / 2;
  for (int ah = blockIdx.x * blockDim.x + threadIdx.x; ah < (1 << lw); ah += gridDim.x * blockDim.x) {
    const int c = ah - PL;
    const int t = (c + Q) >> lq;                                // floor((c + Q) / Q)
    float best = 0.f;
    for (int v = t - 1; v <= t; ++v) {                          // k - l (conjugate: k + l)
      const int qh = c - v * Q + P / 2;
      // channels k whose partner l = k - v (conjugate: v - k) lies in [-Np/2, Np/2)
      const int k0 = conj ? max(-H, v - H + 1) : max(-H, v - H);
      const int k1 = conj ? min(H - 1, v + H) : min(H - 1, v + H - 1);
#pragma unroll 4
      for (int k = k0; k <= k1; ++k) {
        const int l = conj ? v - k : k - v;
        best = fmaxf(best, mag2(__ldg(S + ((((int64_t)(k + H) << lnp) + l + H) * P) + qh)));
      }
    }
    prof[ah] = power == 2 ? best : sqrtf(best);
  }
}

__global__ void __launch_bounds__(256)
k_ssca_profile(const float2* __restrict__ S, int ln /*log2 N*/, int lnp, int power, float* __restrict__ prof) {
  const int N = 1 << ln, H = 1 << (lnp - 1), ld = ln - lnp;   // D = N / Np = 2^ld
  for (int ah = blockIdx.x * blockDim.x + threadIdx.x; ah < 2 * N; ah += gridDim.x * blockDim.x) {
    const int c = ah - N;
    // q = c - k D in [-N/2, N/2)  <=>  floor((c - N/2) / D) < k <= floor((c + N/2) / D)
    const int k0 = max(-H, ((c - N / 2) >> ld) + 1);
    const int k1 = min(H - 1, (c + N / 2) >> ld);
    float best = 0.f;
#pragma unroll 4
    for (int k = k0; k <= k1; ++k)
      best = fmaxf(best, mag2(__ldg(S + ((int64_t)(k + H) << ln) + (c - (k << ld)) + N / 2)));
    prof[ah] = power == 2 ? best : sqrtf(best);
  }
}

int grid_cap(int64_t total) {
  int64_t g = (total + 255) / 256;
  return (int)(g < 152 * 16 ? g : 152 * 16);
}

}  // namespace

cudaError_t fam_map(const float2* S, int Np, int L, int P, int power, bool conj, float* map, cudaStream_t st) {
  const int64_t PL = (int64_t)P * L;
  const int Q = (int)(PL / Np);
  if (!is_pow2(PL) || !is_pow2(Q) || 4 * (int64_t)Np * PL >= (int64_t(1) << 31)) return cudaErrorInvalidValue;
  const int64_t total4 = (int64_t)Np * PL;                      // 2Np x 2PL grid points / 4
  count_launches(1);
  k_fam_map<<<grid_cap(total4), 256, 0, st>>>(S, Np, ilog2(Np), P, ilog2(2 * PL), ilog2(Q), power, conj ? 1 : 0,
                                               map);
  return cudaGetLastError();
}

cudaError_t fam_alpha_profile(const float2* S, int Np, int L, int P, int power, bool conj, float* prof,
                              cudaStream_t st) {
  const int64_t PL = (int64_t)P * L;
  const int Q = (int)(PL / Np);
  if (!is_pow2(PL) || !is_pow2(Q) || 4 * (int64_t)Np * PL >= (int64_t(1) << 31)) return cudaErrorInvalidValue;
  count_launches(1);
  k_fam_profile<<<(unsigned)((2 * PL + 255) / 256), 256, 0, st>>>(S, Np, ilog2(Np), P, ilog2(2 * PL), ilog2(Q),
                                                                   power, conj ? 1 : 0, prof);
  return cudaGetLastError();
}

cudaError_t ssca_alpha_profile(const float2* S, int64_t N, int Np, int power, float* prof, cudaStream_t st) {
  count_launches(1);
  k_ssca_profile<<<(unsigned)((2 * N + 255) / 256), 256, 0, st>>>(S, ilog2(N), ilog2(Np), power, prof);
  return cudaGetLastError();
}

cudaError_t ssca_map(const float2* S, int64_t N, int Np, int power, float* map, cudaStream_t st) {
  const int64_t total4 = (int64_t)Np * N / 2;                   // Np x 2N grid points / 4
  count_launches(1);
  k_ssca_map<<<grid_cap(total4), 256, 0, st>>>(S, ilog2(N), ilog2(Np), power, map);
  return cudaGetLastError();
}

}  // namespace scd
