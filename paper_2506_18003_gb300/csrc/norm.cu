// Input normalisation (Algorithm 1, `Framing`: the norm kernel normalises the input before
// decimation, Sec. III-A).  The estimates are bilinear in the input, so instead of writing a
// scaled copy of x the scale is folded into the window the channeliser already multiplies by:
// FAM uses the window once per factor (a' = a s), SSCA once in X_T and not in the CDP factor
// x[n] (a' = a s^2).  Two small kernels: a grid reduction of the consumed samples (sum of
// |x|^2 in FP64, maximum of |x|^2 as ordered float bits) and the window scaling (factor in FP64,
// rounded once).
#include "internal.h"

namespace scd {
namespace {

__global__ void __launch_bounds__(256) k_norm_reduce(const float2* __restrict__ x, int64_t n, double* sum,
                                                     unsigned* mx) {
  __shared__ double ssum[256];
  __shared__ float smax[256];
  double acc = 0.0;
  float m = 0.f;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float2 v = __ldg(x + i);
    const float p = fmaf(v.x, v.x, v.y * v.y);
    acc += (double)v.x * v.x + (double)v.y * v.y;
    m = fmaxf(m, p);
  }
  ssum[threadIdx.x] = acc;
  smax[threadIdx.x] = m;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) {
      ssum[threadIdx.x] += ssum[threadIdx.x + s];
      smax[threadIdx.x] = fmaxf(smax[threadIdx.x], smax[threadIdx.x + s]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    atomicAdd(sum, ssum[0]);
    atomicMax(mx, __float_as_uint(smax[0]));          // non-negative floats order like their bits
  }
}

__global__ void k_norm_window(const float* __restrict__ a, int Np, int64_t n, int mode, int power,
                              const double* __restrict__ sum, const unsigned* __restrict__ mx, float* out) {
  const double p = mode == 1 ? *sum / (double)n : (double)__uint_as_float(*mx);   // mean or peak of |x|^2
  const double s = p > 0.0 ? 1.0 / sqrt(p) : 1.0;                                 // input factor
  const double f = power == 2 ? s * s : s;
  for (int r = threadIdx.x; r < Np; r += blockDim.x) out[r] = (float)((double)__ldg(a + r) * f);
}

}  // namespace

size_t norm_workspace_bytes() { return 2048; }

cudaError_t normalised_window(const float2* x, int64_t n, const float* a, int Np, int mode, int power, void* area,
                              const float** window_out, cudaStream_t st) {
  double* sum = reinterpret_cast<double*>(area);
  unsigned* mx = reinterpret_cast<unsigned*>(static_cast<char*>(area) + 8);
  float* w = reinterpret_cast<float*>(static_cast<char*>(area) + 256);
  cudaError_t e = cudaMemsetAsync(area, 0, 16, st);
  if (e != cudaSuccess) return e;
  count_launches(2);
  const int64_t blocks = (n + 255) / 256;
  k_norm_reduce<<<(unsigned)(blocks < 152 * 4 ? blocks : 152 * 4), 256, 0, st>>>(x, n, sum, mx);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_norm_window<<<1, 256, 0, st>>>(a, Np, n, mode, power, sum, mx, w);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  *window_out = w;
  return cudaSuccess;
}

}  // namespace scd
