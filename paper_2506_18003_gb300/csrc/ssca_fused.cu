// SSCA, fused schedule (FP32 form): tile A (hop-1 channeliser + channel-data product + the
// strip transform's M1-point pass over m1 and rotate factor) and tile B (M2-point pass over m2,
// fftshifted output), one kernel each.  The tiles and the split are described in
// ssca_fused.cuh.
#include "internal.h"
#include "ssca_fused.cuh"

namespace scd {
namespace {

template <int NP, int M1, int Q>
__global__ void __cluster_dims__(Q, 1, 1) __launch_bounds__(256, 2)
k_sf_chancol(const float2* __restrict__ x, const float2* __restrict__ y, int conj, int N, int M2,
             const float* __restrict__ a, const float2* __restrict__ tw_np, const float2* __restrict__ tw_m1,
             const float2* __restrict__ wN, float2* __restrict__ Y) {
  extern __shared__ __align__(128) float2 sm[];
  const int m2 = (int)blockIdx.x / Q, q = (int)blockIdx.x % Q;
  ssca_chancol_tile<NP, M1, Q>(sm, x, y, conj != 0, N, M2, a, tw_np, tw_m1, wN, Y, m2, q);
}

// three CTAs per SM below M2 = 1024 (80 registers without spills); two at 1024; one of 1024
// threads at 2048
template <int M2>
__global__ void __launch_bounds__(rowsf_threads(M2), M2 >= 2048 ? 1 : (M2 >= 1024 ? 2 : 3))
k_sf_rows(const float2* __restrict__ Y, int N, int M1, const float2* __restrict__ tw, float2* __restrict__ out) {
  extern __shared__ __align__(128) float2 sm[];
  const int64_t kh = blockIdx.y;
  ssca_rowsf_tile<M2>(sm, Y + kh * N, out + kh * N, M1, tw, (int)blockIdx.x * rowsf_c(M2));
}

template <class K>
cudaError_t set_smem(K kernel, int bytes) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

template <int NP, int M1, int Q>
cudaError_t launch_chancol_t(const float2* x, const float2* y, int conj, int N, int M2, const float* a, float2* Y,
                             cudaStream_t st) {
  using Lay = ChanColSmem<NP, M1, Q>;
  cudaError_t e;
  const float2 *tw_np, *tw_m1, *wN;
  if (!(tw_np = table_pass(NP, &e)) || !(tw_m1 = table_pass(M1, &e)) || !(wN = table_roots(N, &e))) return e;
  if ((e = set_smem(k_sf_chancol<NP, M1, Q>, Lay::total)) != cudaSuccess) return e;
  k_sf_chancol<NP, M1, Q><<<M2 * Q, 256, Lay::total, st>>>(x, y, conj, N, M2, a, tw_np, tw_m1, wN, Y);
  return cudaGetLastError();
}

template <int M2>
cudaError_t launch_rowsf_t(const float2* Y, int N, int Np, int M1, float2* out, cudaStream_t st) {
  using S = TileShape<M2, rowsf_threads(M2)>;
  constexpr int smem = FftSmem<M2, S::C, S::NT, false>::total;
  cudaError_t e;
  const float2* tw = table_pass(M2, &e);
  if (!tw) return e;
  if ((e = set_smem(k_sf_rows<M2>, smem)) != cudaSuccess) return e;
  k_sf_rows<M2><<<dim3(M1 / S::C, Np), S::NT, smem, st>>>(Y, N, M1, tw, out);
  return cudaGetLastError();
}

}  // namespace

bool ssca_fused_supported(int64_t N, int Np, int precision) {
  FusedSplit s;
  return precision == SCD_FP32 && fused_split(N, Np, &s);
}

cudaError_t ssca_fused_chancol(const float2* x, const float2* y, bool conj, int64_t N, int Np, const float* window,
                               float2* ws, cudaStream_t st) {
  FusedSplit s;
  if (!fused_split(N, Np, &s)) return cudaErrorInvalidValue;
  count_launches(1);
  const int n = (int)N, cj = conj ? 1 : 0;
#define SCD_SF(NPV, M1V, QV)                                                   \
  if (Np == NPV && s.M1 == M1V && s.Q == QV)                                   \
    return launch_chancol_t<NPV, M1V, QV>(x, y, cj, n, s.M2, window, ws, st);
  SCD_SF(64, 64, 1) SCD_SF(64, 128, 1) SCD_SF(64, 256, 2)
  SCD_SF(128, 64, 1) SCD_SF(128, 128, 2) SCD_SF(128, 256, 4)
  SCD_SF(256, 64, 2) SCD_SF(256, 128, 4)
#undef SCD_SF
  return cudaErrorInvalidValue;
}

cudaError_t ssca_fused_rows(const float2* ws, int64_t N, int Np, float2* out, cudaStream_t st) {
  FusedSplit s;
  if (!fused_split(N, Np, &s)) return cudaErrorInvalidValue;
  count_launches(1);
  switch (s.M2) {
    case 64: return launch_rowsf_t<64>(ws, (int)N, Np, s.M1, out, st);
    case 128: return launch_rowsf_t<128>(ws, (int)N, Np, s.M1, out, st);
    case 256: return launch_rowsf_t<256>(ws, (int)N, Np, s.M1, out, st);
    case 512: return launch_rowsf_t<512>(ws, (int)N, Np, s.M1, out, st);
    case 1024: return launch_rowsf_t<1024>(ws, (int)N, Np, s.M1, out, st);
    case 2048: return launch_rowsf_t<2048>(ws, (int)N, Np, s.M1, out, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace scd
