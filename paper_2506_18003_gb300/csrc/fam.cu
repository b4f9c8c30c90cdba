// FAM kernels (FP32 form): K1 channeliser and K2 conjugate-product + P-point FFT.
//
// K1 implements Eq. II.B-complex_demodulate_final with the block framing of Algorithm 1
// (`Framing`, `Demodulate`): window, Np-point FFT, down-conversion W_Np^{(k p L) mod Np}
// fused into the FFT's output stage.  It writes X[kh][p] (P contiguous per channel), the
// layout the pair stage reads rows from.
//
// K2 implements Eq. II.B-SCD_function_FAM (Algorithm 1, `FFT2`): for every channel pair the
// conjugate product z(p) = X(p,k) conj(X(p,l)) is formed inside the FFT's first pass (no
// product array ever exists in memory), then the P-point FFT, and the fftshifted bins go
// straight to out[kh][lh][qh].  X (Np*P*8 bytes, 2 MiB at Np=256, P=1024) stays in L2, so
// the kernel's DRAM traffic is essentially the 8 Np^2 P output bytes.
#include "fft.cuh"
#include "internal.h"

namespace scd {
namespace {

template <int NP, int C>
__global__ void __launch_bounds__(C * PlanInfo<NP>::T)
k_fam_channelise(const float2* __restrict__ x, int L, int P, const float* __restrict__ a,
                 const float2* __restrict__ wnp, const float2* __restrict__ tw, float2* __restrict__ X) {
  extern __shared__ float2 sm[];
  const int p0 = blockIdx.x * C;
  auto src = [&](int c, int n) -> float2 {
    const int p = p0 + c;
    if (p >= P) return make_float2(0.f, 0.f);
    return cscale(__ldg(x + (int64_t)p * L + n), __ldg(a + n));
  };
  auto dst = [&](int c, int f, float2 v) {
    const int p = p0 + c;
    if (p >= P) return;
    const int pl = (int)(((int64_t)p * L) & (NP - 1));          // (p L) mod Np
    const int kh = (f + NP / 2) & (NP - 1);
    X[(int64_t)kh * P + p] = cmul(v, __ldg(wnp + ((f * pl) & (NP - 1))));
  };
  fft_batch<NP, C, true, false>(sm, tw, src, dst);
}

template <int PP, int C>
__global__ void __launch_bounds__(C * PlanInfo<PP>::T)
k_fam_pairs(const float2* __restrict__ X, int Np, float2* __restrict__ out, const float2* __restrict__ tw) {
  extern __shared__ float2 sm[];
  const int64_t pair0 = (int64_t)blockIdx.x * C;
  const int64_t npairs = (int64_t)Np * Np;
  auto src = [&](int c, int p) -> float2 {
    const int64_t pair = pair0 + c;
    if (pair >= npairs) return make_float2(0.f, 0.f);
    const int kh = (int)(pair / Np), lh = (int)(pair % Np);
    return cmulc(__ldg(X + (int64_t)kh * PP + p), __ldg(X + (int64_t)lh * PP + p));
  };
  auto dst = [&](int c, int f, float2 v) {
    const int64_t pair = pair0 + c;
    if (pair >= npairs) return;
    out[pair * PP + ((f + PP / 2) & (PP - 1))] = v;
  };
  fft_batch<PP, C, false, false>(sm, tw, src, dst);
}

template <int M> constexpr int smem_bytes(int C) { return PlanInfo<M>::n == 1 ? 0 : C * PlanInfo<M>::stride() * (int)sizeof(float2); }

template <class K>
cudaError_t set_smem(K kernel, int bytes) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

}  // namespace

cudaError_t fam_channelise(const float2* x, int Np, int L, int P, const float* window, float2* X, cudaStream_t st) {
  cudaError_t err;
  const float2* wnp = table_roots(Np, &err);
  if (!wnp) return err;
  const float2* tw = table_pass(Np, &err);
  if (!tw) return err;
  count_launches(1);
#define SCD_K1(NPV)                                                                        \
  {                                                                                        \
    constexpr int T = PlanInfo<NPV>::T;                                                    \
    constexpr int C = (256 / T) < 1 ? 1 : 256 / T;                                         \
    const int sm = smem_bytes<NPV>(C);                                                     \
    if ((err = set_smem(k_fam_channelise<NPV, C>, sm)) != cudaSuccess) return err;         \
    k_fam_channelise<NPV, C><<<(P + C - 1) / C, C * T, sm, st>>>((const float2*)x, L, P, window, wnp, tw, X); \
  }
  switch (Np) {
    case 16: SCD_K1(16); break;
    case 32: SCD_K1(32); break;
    case 64: SCD_K1(64); break;
    case 128: SCD_K1(128); break;
    case 256: SCD_K1(256); break;
    default: return cudaErrorInvalidValue;
  }
#undef SCD_K1
  return cudaGetLastError();
}

cudaError_t fam_pair_fft(const float2* X, int Np, int P, float2* out, cudaStream_t st) {
  cudaError_t err;
  const float2* tw = table_pass(P, &err);
  if (!tw) return err;
  const int64_t npairs = (int64_t)Np * Np;
  count_launches(1);
#define SCD_K2(PV)                                                                         \
  {                                                                                        \
    constexpr int T = PlanInfo<PV>::T;                                                     \
    constexpr int C = (256 / T) < 1 ? 1 : 256 / T;                                         \
    const int sm = smem_bytes<PV>(C);                                                      \
    if ((err = set_smem(k_fam_pairs<PV, C>, sm)) != cudaSuccess) return err;               \
    k_fam_pairs<PV, C><<<(unsigned)((npairs + C - 1) / C), C * T, sm, st>>>(X, Np, out, tw); \
  }
  switch (P) {
    case 2: SCD_K2(2); break;
    case 4: SCD_K2(4); break;
    case 8: SCD_K2(8); break;
    case 16: SCD_K2(16); break;
    case 32: SCD_K2(32); break;
    case 64: SCD_K2(64); break;
    case 128: SCD_K2(128); break;
    case 256: SCD_K2(256); break;
    case 512: SCD_K2(512); break;
    case 1024: SCD_K2(1024); break;
    case 2048: SCD_K2(2048); break;
    case 4096: SCD_K2(4096); break;
    case 8192: SCD_K2(8192); break;
    case 16384: SCD_K2(16384); break;
    default: return cudaErrorInvalidValue;
  }
#undef SCD_K2
  return cudaGetLastError();
}

cudaError_t fam_channelise_with(const float2* x, int Np, int L, int P, const float* window, float2* X,
                                const float2* wnp, const float2* tw, cudaStream_t st) {
  cudaError_t err;
  count_launches(1);
#define SCD_K1W(NPV)                                                                       \
  {                                                                                        \
    constexpr int T = PlanInfo<NPV>::T;                                                    \
    constexpr int C = (256 / T) < 1 ? 1 : 256 / T;                                         \
    const int sm = smem_bytes<NPV>(C);                                                     \
    if ((err = set_smem(k_fam_channelise<NPV, C>, sm)) != cudaSuccess) return err;         \
    k_fam_channelise<NPV, C><<<(P + C - 1) / C, C * T, sm, st>>>(x, L, P, window, wnp, tw, X); \
  }
  switch (Np) {
    case 16: SCD_K1W(16); break;
    case 32: SCD_K1W(32); break;
    case 64: SCD_K1W(64); break;
    case 128: SCD_K1W(128); break;
    case 256: SCD_K1W(256); break;
    default: return cudaErrorInvalidValue;
  }
#undef SCD_K1W
  return cudaGetLastError();
}

cudaError_t fam_pair_fft_with(const float2* X, int Np, int P, float2* out, const float2* tw, cudaStream_t st) {
  cudaError_t err;
  const int64_t npairs = (int64_t)Np * Np;
  count_launches(1);
#define SCD_K2W(PV)                                                                        \
  {                                                                                        \
    constexpr int T = PlanInfo<PV>::T;                                                     \
    constexpr int C = (256 / T) < 1 ? 1 : 256 / T;                                         \
    const int sm = smem_bytes<PV>(C);                                                      \
    if ((err = set_smem(k_fam_pairs<PV, C>, sm)) != cudaSuccess) return err;               \
    k_fam_pairs<PV, C><<<(unsigned)((npairs + C - 1) / C), C * T, sm, st>>>(X, Np, out, tw); \
  }
  switch (P) {
    case 2: SCD_K2W(2); break;
    case 4: SCD_K2W(4); break;
    case 8: SCD_K2W(8); break;
    case 16: SCD_K2W(16); break;
    case 32: SCD_K2W(32); break;
    case 64: SCD_K2W(64); break;
    case 128: SCD_K2W(128); break;
    case 256: SCD_K2W(256); break;
    case 512: SCD_K2W(512); break;
    case 1024: SCD_K2W(1024); break;
    case 2048: SCD_K2W(2048); break;
    case 4096: SCD_K2W(4096); break;
    case 8192: SCD_K2W(8192); break;
    case 16384: SCD_K2W(16384); break;
    default: return cudaErrorInvalidValue;
  }
#undef SCD_K2W
  return cudaGetLastError();
}

}  // namespace scd
