// SSCA kernels (FP32 form): K3 hop-1 channeliser + channel-data product, K4a column pass
// and K4b row pass of the decomposed N-point strip FFT.
//
// K3: Sec. II-C with the complex demodulate of Sec. II-A (Eq. II.A-complex demodulate)
//     centred on n: window, Np-point FFT, down-conversion W_Np^{(k s) mod Np} and the
//     product with conj(x[n]) (Eq. Xg), all in the FFT's output stage.  Writes
//     X_g[kh][n] (channel-major, n contiguous).
// K4a: Stage 1 of Sec. III-B-1 (Eq. Chap4_2DFFT, "M1-point DFT on the m2-th column" times
//     the rotate factor W_N^{(m2 m1') mod N}), in place on X_g viewed as [kh][m1][m2] with
//     n = m1 M2 + m2.  A CTA owns C1 consecutive columns m2, so every global access is a
//     run of C1 contiguous complex values.
// K4b: Stage 2 (M2-point DFT along the contiguous rows m2), output bin q_nat = m1' + M1 m2'
//     stored fftshifted at sh = (q_nat + N/2) mod N = m1' + M1 ((m2' + M2/2) mod M2).  A CTA
//     owns C2 consecutive rows m1' and transposes through shared memory so the strided
//     output is written as runs of C2 contiguous values.
#include "fft_tc.cuh"
#include "internal.h"

namespace scd {
namespace {

constexpr int kC2 = 8;   // rows per CTA in the row pass (FP32 form)

// Transforms per CTA: the FP32 form uses C_FP32; the tensor-core form needs a multiple of
// 128 threads.
template <int M, int C_FP32, bool TC>
struct Batch {
  static constexpr int T = PlanInfo<M>::T;
  static constexpr int C = (TC && C_FP32 * T < 128) ? 128 / T : C_FP32;
  static constexpr int THREADS = C * T;
};

template <int NP, int C, bool TC>
__global__ void __launch_bounds__(C * PlanInfo<NP>::T)
k_ssca_cdp(const float2* __restrict__ x, int N, const float* __restrict__ a, const float2* __restrict__ wnp,
           const float2* __restrict__ tw, float2* __restrict__ Xg, const unsigned char* __restrict__ bmats,
           unsigned* err) {
  extern __shared__ __align__(128) float2 sm[];
  const int n0 = blockIdx.x * C;
  auto src = [&](int c, int r) -> float2 {
    const int m = n0 + c - NP / 2 + r;
    if (m < 0 || m >= N) return make_float2(0.f, 0.f);
    return cscale(__ldg(x + m), __ldg(a + r));
  };
  auto dst = [&](int c, int f, float2 v) {
    const int n = n0 + c;
    const int s = (n - NP / 2) & (NP - 1);                        // s mod Np (s may be < 0)
    const int kh = (f + NP / 2) & (NP - 1);
    const float2 y = cmul(v, __ldg(wnp + ((f * s) & (NP - 1))));
    Xg[(int64_t)kh * N + n] = cmulc(y, __ldg(x + n));
  };
  fft_run<NP, C, true, false, C * PlanInfo<NP>::T, TC, 0>(sm, tw, bmats, err, src, dst);
}

template <int M1, int C, bool TC>
__global__ void __launch_bounds__(C * PlanInfo<M1>::T)
k_ssca_cols(float2* __restrict__ Y, int N, int M2, const float2* __restrict__ wN, const float2* __restrict__ cols,
            const float2* __restrict__ tw, const unsigned char* __restrict__ bmats, unsigned* err) {
  extern __shared__ __align__(128) float2 sm[];
  const int m20 = blockIdx.x * C;
  float2* __restrict__ row = Y + (int64_t)blockIdx.y * N + m20;
  auto src = [&](int c, int m1) -> float2 { return row[(int64_t)m1 * M2 + c]; };
  auto dst = [&](int c, int f, float2 v) {
    const float2 w = cmul(__ldg(wN + ((m20 * f) & (N - 1))), __ldg(cols + f * C + c));  // W_N^{(m20+c) f}
    row[(int64_t)f * M2 + c] = cmul(v, w);
  };
  fft_run<M1, C, true, false, C * PlanInfo<M1>::T, TC, 0>(sm, tw, bmats, err, src, dst);
}

template <int M2, int C, bool TC>
__global__ void __launch_bounds__(C * PlanInfo<M2>::T)
k_ssca_rows(const float2* __restrict__ Y, int N, int M1, const float2* __restrict__ tw, float2* __restrict__ out,
            const unsigned char* __restrict__ bmats, unsigned* err) {
  extern __shared__ __align__(128) float2 sm[];
  const int r0 = blockIdx.x * C;
  const float2* __restrict__ in = Y + (int64_t)blockIdx.y * N + (int64_t)r0 * M2;
  auto src = [&](int c, int m2) -> float2 { return in[c * M2 + m2]; };
  auto dst = [&](int c, int f, float2 v) { sm[f * (C + 1) + c] = v; };
  fft_run<M2, C, false, true, C * PlanInfo<M2>::T, TC, M2 * (C + 1) * 8>(sm, tw, bmats, err, src, dst);
  __syncthreads();
  float2* __restrict__ o = out + (int64_t)blockIdx.y * N + r0;
  for (int e = threadIdx.x; e < C * M2; e += blockDim.x) {
    const int c = e % C, f = e / C;
    o[c + (int64_t)M1 * ((f + M2 / 2) & (M2 - 1))] = sm[f * (C + 1) + c];
  }
}

template <class K>
cudaError_t set_smem(K kernel, int bytes) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

struct TcArgs {
  const unsigned char* bm = nullptr;
  unsigned* err = nullptr;
};

cudaError_t tc_args(bool tc, int M, TcArgs* a) {
  if (!tc) return cudaSuccess;
  cudaError_t err;
  int bytes = 0;
  if (!(a->bm = table_tc_bmats(M, &bytes, &err))) return err;
  if (!(a->err = device_error_word(&err))) return err;
  return cudaSuccess;
}

template <int NPV, bool TC>
cudaError_t launch_cdp_t(const float2* x, int N, const float* a, const float2* wnp, const float2* tw, float2* Xg,
                         TcArgs t, cudaStream_t st) {
  constexpr int T = PlanInfo<NPV>::T;
  constexpr int C = (256 / T) < 16 ? 16 : 256 / T;
  constexpr int sm = FftSmem<NPV, C, C * T, TC>::total;
  cudaError_t e = set_smem(k_ssca_cdp<NPV, C, TC>, sm);
  if (e != cudaSuccess) return e;
  k_ssca_cdp<NPV, C, TC><<<N / C, C * T, sm, st>>>(x, N, a, wnp, tw, Xg, t.bm, t.err);
  return cudaGetLastError();
}

template <int MV, bool TC>
cudaError_t launch_cols_t(float2* Y, int N, int Np, int M1, int M2, TcArgs t, cudaStream_t st) {
  using B = Batch<MV, kSscaCols, TC>;
  cudaError_t err;
  const float2* wN = table_roots(N, &err);
  if (!wN) return err;
  const float2* cols = table_cols(N, M1, B::C, &err);
  if (!cols) return err;
  const float2* tw = table_pass(M1, &err);
  if (!tw) return err;
  constexpr int sm = FftSmem<MV, B::C, B::THREADS, TC>::total;
  if ((err = set_smem(k_ssca_cols<MV, B::C, TC>, sm)) != cudaSuccess) return err;
  k_ssca_cols<MV, B::C, TC><<<dim3(M2 / B::C, Np), B::THREADS, sm, st>>>(Y, N, M2, wN, cols, tw, t.bm, t.err);
  return cudaGetLastError();
}

template <int MV, bool TC>
cudaError_t launch_rows_t(const float2* Y, int N, int Np, int M1, int M2, float2* out, TcArgs t, cudaStream_t st) {
  using B = Batch<MV, kC2, TC>;
  cudaError_t err;
  const float2* tw = table_pass(M2, &err);
  if (!tw) return err;
  constexpr int sm = FftSmem<MV, B::C, B::THREADS, TC, MV * (B::C + 1) * 8>::total;
  if ((err = set_smem(k_ssca_rows<MV, B::C, TC>, sm)) != cudaSuccess) return err;
  k_ssca_rows<MV, B::C, TC><<<dim3(M1 / B::C, Np), B::THREADS, sm, st>>>(Y, N, M1, tw, out, t.bm, t.err);
  return cudaGetLastError();
}

cudaError_t launch_cdp(const float2* x, int N, int Np, const float* a, float2* Xg, bool tc, cudaStream_t st) {
  cudaError_t err;
  const float2* wnp = table_roots(Np, &err);
  if (!wnp) return err;
  const float2* tw = table_pass(Np, &err);
  if (!tw) return err;
  TcArgs t;
  if ((err = tc_args(tc, Np, &t)) != cudaSuccess) return err;
#define SCD_K3(NPV) return tc ? launch_cdp_t<NPV, true>(x, N, a, wnp, tw, Xg, t, st) \
                              : launch_cdp_t<NPV, false>(x, N, a, wnp, tw, Xg, t, st)
  switch (Np) {
    case 16: SCD_K3(16);
    case 32: SCD_K3(32);
    case 64: SCD_K3(64);
    case 128: SCD_K3(128);
    case 256: SCD_K3(256);
    default: return cudaErrorInvalidValue;
  }
#undef SCD_K3
}

cudaError_t launch_cols(float2* Y, int N, int Np, int M1, int M2, bool tc, cudaStream_t st) {
  TcArgs t;
  cudaError_t err = tc_args(tc, M1, &t);
  if (err != cudaSuccess) return err;
#define SCD_K4A(MV) return tc ? launch_cols_t<MV, true>(Y, N, Np, M1, M2, t, st) \
                              : launch_cols_t<MV, false>(Y, N, Np, M1, M2, t, st)
  switch (M1) {
    case 64: SCD_K4A(64);
    case 128: SCD_K4A(128);
    case 256: SCD_K4A(256);
    case 512: SCD_K4A(512);
    case 1024: SCD_K4A(1024);
    default: return cudaErrorInvalidValue;
  }
#undef SCD_K4A
}

cudaError_t launch_rows(const float2* Y, int N, int Np, int M1, int M2, float2* out, bool tc, cudaStream_t st) {
  TcArgs t;
  cudaError_t err = tc_args(tc, M2, &t);
  if (err != cudaSuccess) return err;
#define SCD_K4B(MV) return tc ? launch_rows_t<MV, true>(Y, N, Np, M1, M2, out, t, st) \
                              : launch_rows_t<MV, false>(Y, N, Np, M1, M2, out, t, st)
  switch (M2) {
    case 64: SCD_K4B(64);
    case 128: SCD_K4B(128);
    case 256: SCD_K4B(256);
    case 512: SCD_K4B(512);
    case 1024: SCD_K4B(1024);
    default: return cudaErrorInvalidValue;
  }
#undef SCD_K4B
}

}  // namespace

void ssca_split(int64_t N, int* M1, int* M2) {
  const int e = ilog2(N);
  *M1 = 1 << ((e + 1) / 2);
  *M2 = 1 << (e / 2);
}

cudaError_t ssca_cdp(const float2* x, int64_t N, int Np, const float* window, float2* ws, cudaStream_t st,
                     int precision) {
  count_launches(1);
  return launch_cdp(x, (int)N, Np, window, ws, precision == SCD_SPLIT_BF16, st);
}

cudaError_t ssca_cols(float2* ws, int64_t N, int Np, cudaStream_t st, int precision) {
  int M1, M2;
  ssca_split(N, &M1, &M2);
  count_launches(1);
  return launch_cols(ws, (int)N, Np, M1, M2, precision == SCD_SPLIT_BF16, st);
}

cudaError_t ssca_rows(const float2* ws, int64_t N, int Np, float2* out, cudaStream_t st, int precision) {
  int M1, M2;
  ssca_split(N, &M1, &M2);
  count_launches(1);
  return launch_rows(ws, (int)N, Np, M1, M2, out, precision == SCD_SPLIT_BF16, st);
}

}  // namespace scd
