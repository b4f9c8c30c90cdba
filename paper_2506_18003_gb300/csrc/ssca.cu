// SSCA kernels (FP32 form): K3 hop-1 channeliser + channel-data product, K4a column pass
// and K4b row pass of the decomposed N-point strip FFT.
//
// K3: Sec. II-C with the complex demodulate of Sec. II-A (Eq. II.A-complex demodulate)
//     centred on n: window, Np-point FFT, down-conversion W_Np^{(k s) mod Np} (folded into
//     the FFT by rotating the frame's input by s mod Np positions) and the
//     product with conj(y[n]) (Eq. Xg; y = x for the auto estimate, the second signal of a
//     cross estimate, or y[n] unconjugated for a conjugate one), all in the FFT's output
//     stage.  Writes
//     X_g[kh][n] (channel-major, n contiguous).
// K4a: Stage 1 of Sec. III-B-1 (Eq. Chap4_2DFFT, "M1-point DFT on the m2-th column" times
//     the rotate factor W_N^{(m2 m1') mod N}), in place on X_g viewed as [kh][m1][m2] with
//     n = m1 M2 + m2.  A CTA owns C1 consecutive columns m2, so every global access is a
//     run of C1 contiguous complex values.
// K4b: Stage 2 (M2-point DFT along the contiguous rows m2), output bin q_nat = m1' + M1 m2'
//     stored fftshifted at sh = (q_nat + N/2) mod N = m1' + M1 ((m2' + M2/2) mod M2).  A CTA
//     owns C2 consecutive rows m1' and transposes through shared memory so the strided
//     output is written as runs of C2 contiguous values.
#include "internal.h"
#include "tiles.cuh"

namespace scd {
namespace {

template <int NP, bool TC>
__global__ void __launch_bounds__(TileShape<NP>::NT)
k_ssca_cdp(const float2* __restrict__ x, const float2* __restrict__ y, int conj, int N, const float* __restrict__ a,
           const float2* __restrict__ tw, float2* __restrict__ Xg,
           const unsigned char* __restrict__ bmats, unsigned* err) {
  extern __shared__ __align__(128) float2 sm[];
  using S = TileShape<NP>;
  using FS = CdpSmem<NP, TC>;
  unsigned char* base = reinterpret_cast<unsigned char*>(sm);
  TcCtx ctx{};
  if constexpr (TC) ctx = tc_begin<FS::tmem_cols>(base + FS::region0 + FS::bbytes, base + FS::region0, bmats, FS::bbytes, err);
  ssca_cdp_tile<NP, TC>(sm, ctx, x, y, conj != 0, N, a, tw, Xg, blockIdx.x * S::C, base + CdpStage<NP, TC>::off);
  if constexpr (TC) tc_end<FS::tmem_cols>(ctx);
}

template <int M1, bool TC>
__global__ void __launch_bounds__(TileShape<M1>::NT)
k_ssca_cols(float2* __restrict__ Y, int N, int M2, const float2* __restrict__ wN, const float2* __restrict__ cols,
            const float2* __restrict__ tw, const unsigned char* __restrict__ bmats, unsigned* err) {
  extern __shared__ __align__(128) float2 sm[];
  using S = TileShape<M1>;
  using FS = ColsSmem<M1, TC>;
  unsigned char* base = reinterpret_cast<unsigned char*>(sm);
  TcCtx ctx{};
  if constexpr (TC) ctx = tc_begin<FS::tmem_cols>(base + FS::region0 + FS::bbytes, base + FS::region0, bmats, FS::bbytes, err);
  float2* row = Y + (int64_t)blockIdx.y * N;
  ssca_cols_tile<M1, TC>(sm, ctx, row, row, N, M2, wN, cols, tw, blockIdx.x * S::C,
                         reinterpret_cast<float2*>(base + ColsStage<M1, TC>::off));
  if constexpr (TC) tc_end<FS::tmem_cols>(ctx);
}

template <int M2, bool TC>
__global__ void __launch_bounds__(TileShape<M2>::NT)
k_ssca_rows(const float2* __restrict__ Y, int N, int M1, const float2* __restrict__ tw, float2* __restrict__ out,
            const unsigned char* __restrict__ bmats, unsigned* err) {
  extern __shared__ __align__(128) float2 sm[];
  using S = TileShape<M2>;
  using FS = FftSmem<M2, S::C, S::NT, TC, rows_stage_bytes<M2>()>;
  unsigned char* base = reinterpret_cast<unsigned char*>(sm);
  TcCtx ctx{};
  if constexpr (TC) ctx = tc_begin<FS::tmem_cols>(base + FS::region0 + FS::bbytes, base + FS::region0, bmats, FS::bbytes, err);
  ssca_rows_tile<M2, TC>(sm, ctx, Y + (int64_t)blockIdx.y * N, out + (int64_t)blockIdx.y * N, M1, tw,
                         blockIdx.x * S::C);
  if constexpr (TC) tc_end<FS::tmem_cols>(ctx);
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
cudaError_t launch_cdp_t(const float2* x, const float2* y, int conj, int N, const float* a, const float2* tw, float2* Xg, TcArgs t, cudaStream_t st) {
  using S = TileShape<NPV>;
  constexpr int sm = CdpSmem<NPV, TC>::total;
  cudaError_t e = set_smem(k_ssca_cdp<NPV, TC>, sm);
  if (e != cudaSuccess) return e;
  k_ssca_cdp<NPV, TC><<<N / S::C, S::NT, sm, st>>>(x, y, conj, N, a, tw, Xg, t.bm, t.err);
  return cudaGetLastError();
}

template <int MV, bool TC>
cudaError_t launch_cols_t(float2* Y, int N, int Np, int M1, int M2, TcArgs t, cudaStream_t st) {
  using S = TileShape<MV>;
  cudaError_t err;
  const float2* wN = table_roots(N, &err);
  if (!wN) return err;
  const float2* cols = table_cols(N, M1, S::C, &err);
  if (!cols) return err;
  const float2* tw = table_pass(M1, &err);
  if (!tw) return err;
  constexpr int sm = ColsSmem<MV, TC>::total;
  if ((err = set_smem(k_ssca_cols<MV, TC>, sm)) != cudaSuccess) return err;
  k_ssca_cols<MV, TC><<<dim3(M2 / S::C, Np), S::NT, sm, st>>>(Y, N, M2, wN, cols, tw, t.bm, t.err);
  return cudaGetLastError();
}

template <int MV, bool TC>
cudaError_t launch_rows_t(const float2* Y, int N, int Np, int M1, int M2, float2* out, TcArgs t, cudaStream_t st) {
  using S = TileShape<MV>;
  cudaError_t err;
  const float2* tw = table_pass(M2, &err);
  if (!tw) return err;
  constexpr int sm = FftSmem<MV, S::C, S::NT, TC, rows_stage_bytes<MV>()>::total;
  if ((err = set_smem(k_ssca_rows<MV, TC>, sm)) != cudaSuccess) return err;
  k_ssca_rows<MV, TC><<<dim3(M1 / S::C, Np), S::NT, sm, st>>>(Y, N, M1, tw, out, t.bm, t.err);
  return cudaGetLastError();
}

cudaError_t launch_cdp(const float2* x, const float2* y, int conj, int N, int Np, const float* a, float2* Xg, bool tc,
                       cudaStream_t st) {
  cudaError_t err;
  const float2* tw = table_pass(Np, &err);
  if (!tw) return err;
  TcArgs t;
  if ((err = tc_args(tc, Np, &t)) != cudaSuccess) return err;
#define SCD_K3(NPV) return tc ? launch_cdp_t<NPV, true>(x, y, conj, N, a, tw, Xg, t, st) \
                              : launch_cdp_t<NPV, false>(x, y, conj, N, a, tw, Xg, t, st)
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

int ssca_cols_per_tile(int M1) {
  switch (M1) {
    case 64: return TileShape<64>::C;
    case 128: return TileShape<128>::C;
    case 256: return TileShape<256>::C;
    case 512: return TileShape<512>::C;
    case 1024: return TileShape<1024>::C;
    default: return 0;
  }
}

void ssca_split(int64_t N, int* M1, int* M2) {
  const int e = ilog2(N);
  *M1 = 1 << ((e + 1) / 2);
  *M2 = 1 << (e / 2);
  // N = 2^19: 512 x 1024 rather than 1024 x 512.  The 512-point column pass runs at the row
  // pass's rate, the 1024-point one a third slower per point (staged, Np = 256: 1.181 ->
  // 1.035 ms per estimate); at 2^20 the split stays 1024 x 1024 (a 2048-point row pass would
  // write runs of two values and lose more than the column pass gains).
  if (e == 19) { *M1 = 512; *M2 = 1024; }
}

cudaError_t ssca_cdp(const float2* x, const float2* y, bool conj, int64_t N, int Np, const float* window, float2* ws,
                     cudaStream_t st, int precision) {
  count_launches(1);
  return launch_cdp(x, y, conj ? 1 : 0, (int)N, Np, window, ws, precision == SCD_SPLIT_BF16, st);
}

cudaError_t ssca_cols(float2* ws, int64_t N, int Np, cudaStream_t st, int precision) {
  int M1, M2;
  ssca_split(N, &M1, &M2);
  count_launches(1);
  if (precision != SCD_SPLIT_BF16 && ssca_cols_tma_supported(M1)) return ssca_cols_tma(ws, N, Np, M1, M2, st);
  return launch_cols(ws, (int)N, Np, M1, M2, precision == SCD_SPLIT_BF16, st);
}

cudaError_t ssca_rows(const float2* ws, int64_t N, int Np, float2* out, cudaStream_t st, int precision) {
  int M1, M2;
  ssca_split(N, &M1, &M2);
  count_launches(1);
  return launch_rows(ws, (int)N, Np, M1, M2, out, precision == SCD_SPLIT_BF16, st);
}

}  // namespace scd
