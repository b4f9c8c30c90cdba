// FAM kernels: K1 channeliser and K2 conjugate-product + P-point FFT, each in the FP32 form
// (CUDA-core radix butterflies) and the split-precision form (radix DFTs as bf16 hi/lo
// tensor-core GEMMs with FP32 accumulation, fft_tc.cuh).
//
// K1 implements Eq. II.B-complex_demodulate_final with the block framing of Algorithm 1
// (`Framing`, `Demodulate`): window, Np-point FFT and the down-conversion W_Np^{(k p L) mod Np},
// which is folded into the FFT by rotating each frame's input by (p L) mod Np positions.  It writes X[kh][p] (P contiguous per channel), the
// layout the pair stage reads rows from.
//
// K2 implements Eq. II.B-SCD_function_FAM (Algorithm 1, `FFT2`): for every channel pair the
// conjugate product z(p) = X(p,k) conj(Y(p,l)) (Y = X for the auto estimate, the second
// signal's channeliser output for a cross estimate, Eq. II.A-SCD function, and that output
// conjugated for a conjugate estimate) is formed inside the FFT's first pass (no
// product array ever exists in memory), then the P-point FFT, and the fftshifted bins go
// straight to out[kh][lh][qh].  X (Np*P*8 bytes, 2 MiB at Np=256, P=1024) stays in L2, so
// the kernel's DRAM traffic is essentially the 8 Np^2 P output bytes.
#include "internal.h"
#include "tiles.cuh"

namespace scd {
namespace {

template <int NP, bool TC>
__global__ void __launch_bounds__(TileShape<NP>::NT)
k_fam_channelise(const float2* __restrict__ x, int L, int P, const float* __restrict__ a,
                 const float2* __restrict__ tw, float2* __restrict__ X,
                 const unsigned char* __restrict__ bmats, unsigned* err, int conj_out) {
  extern __shared__ __align__(128) float2 sm[];
  using S = TileShape<NP>;
  using FS = FftSmem<NP, S::C, S::NT, TC>;
  unsigned char* base = reinterpret_cast<unsigned char*>(sm);
  TcCtx ctx{};
  if constexpr (TC) ctx = tc_begin<FS::tmem_cols>(base + FS::region0 + FS::bbytes, base + FS::region0, bmats, FS::bbytes, err);
  fam_channelise_tile<NP, TC>(sm, ctx, x, L, P, a, tw, X, blockIdx.x * S::C, conj_out != 0);
  if constexpr (TC) tc_end<FS::tmem_cols>(ctx);
}

// SYM: the auto estimate (Y = X): only the pairs kh <= lh are transformed, each writing both
// rows (fam_pairs_tile)
template <int PP, bool TC, bool SYM>
__device__ __forceinline__ void fam_pairs_cta(const float2* __restrict__ X, const float2* __restrict__ Y, int Np,
                                              float2* __restrict__ out, const float2* __restrict__ tw,
                                              const unsigned char* __restrict__ bmats, unsigned* err) {
  extern __shared__ __align__(128) float2 sm[];
  using S = TileShape<PP>;
  using FS = FftSmem<PP, S::C, S::NT, TC>;
  unsigned char* base = reinterpret_cast<unsigned char*>(sm);
  TcCtx ctx{};
  if constexpr (TC) ctx = tc_begin<FS::tmem_cols>(base + FS::region0 + FS::bbytes, base + FS::region0, bmats, FS::bbytes, err);
  fam_pairs_tile<PP, TC, false, SYM>(sm, ctx, X, Y, Np, out, tw, (int64_t)blockIdx.x * S::C);
  if constexpr (TC) tc_end<FS::tmem_cols>(ctx);
}

template <int PP, bool TC, bool SYM>
__global__ void __launch_bounds__(TileShape<PP>::NT)
k_fam_pairs(const float2* __restrict__ X, const float2* __restrict__ Y, int Np, float2* __restrict__ out,
            const float2* __restrict__ tw, const unsigned char* __restrict__ bmats, unsigned* err) {
  fam_pairs_cta<PP, TC, SYM>(X, Y, Np, out, tw, bmats, err);
}

// The same kernel with its registers capped so that MINB CTAs share an SM.
template <int PP, bool TC, bool SYM, int MINB>
__global__ void __launch_bounds__(TileShape<PP>::NT, MINB)
k_fam_pairs_capped(const float2* __restrict__ X, const float2* __restrict__ Y, int Np, float2* __restrict__ out,
                   const float2* __restrict__ tw, const unsigned char* __restrict__ bmats, unsigned* err) {
  fam_pairs_cta<PP, TC, SYM>(X, Y, Np, out, tw, bmats, err);
}

template <class K>
cudaError_t set_smem(K kernel, int bytes) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

template <int NPV, bool TC>
cudaError_t launch_k1(const float2* x, int L, int P, const float* window, const float2* tw,
                      float2* X, const unsigned char* bm, unsigned* err, int conj_out, cudaStream_t st) {
  using S = TileShape<NPV>;
  constexpr int sm = FftSmem<NPV, S::C, S::NT, TC>::total;
  cudaError_t e = set_smem(k_fam_channelise<NPV, TC>, sm);
  if (e != cudaSuccess) return e;
  k_fam_channelise<NPV, TC><<<(P + S::C - 1) / S::C, S::NT, sm, st>>>(x, L, P, window, tw, X, bm, err, conj_out);
  return cudaGetLastError();
}

// CTAs per SM that the FP32 pair kernel's registers are capped for (0: as the compiler picks).
// Measured at Np = 256 (pair stage, GB300): P = 512 0.074 -> 0.068 ms (3 CTAs, 80 registers),
// 1024 0.144 -> 0.140 (3), 2048 0.341 -> 0.328 (4, 64 registers), 4096 0.732 -> 0.703 (4),
// 8192 1.95 -> 1.57 (2, 128 registers: the compiler's 155 left one CTA per SM).
template <int PV, bool TC>
struct FamPairsBlocks { static constexpr int value = 0; };
template <> struct FamPairsBlocks<512, false> { static constexpr int value = 3; };
template <> struct FamPairsBlocks<1024, false> { static constexpr int value = 3; };
template <> struct FamPairsBlocks<2048, false> { static constexpr int value = 4; };
template <> struct FamPairsBlocks<4096, false> { static constexpr int value = 4; };
template <> struct FamPairsBlocks<8192, false> { static constexpr int value = 2; };

template <int PV, bool TC, bool SYM>
auto fam_pairs_kernel() {
  if constexpr (FamPairsBlocks<PV, TC>::value > 0) return k_fam_pairs_capped<PV, TC, SYM, FamPairsBlocks<PV, TC>::value>;
  else return k_fam_pairs<PV, TC, SYM>;
}

template <int PV, bool TC, bool SYM>
cudaError_t launch_k2_t(const float2* X, const float2* Y, int Np, float2* out, const float2* tw,
                        const unsigned char* bm, unsigned* err, cudaStream_t st) {
  using S = TileShape<PV>;
  constexpr int sm = FftSmem<PV, S::C, S::NT, TC>::total;
  auto kernel = fam_pairs_kernel<PV, TC, SYM>();
  cudaError_t e = set_smem(kernel, sm);
  if (e != cudaSuccess) return e;
  const int64_t npairs = fam_pair_count<PV>(Np, SYM);
  kernel<<<(unsigned)((npairs + S::C - 1) / S::C), S::NT, sm, st>>>(X, Y, Np, out, tw, bm, err);
  return cudaGetLastError();
}

// The auto estimate (Y is X) transforms the pairs kh <= lh only.
template <int PV, bool TC>
cudaError_t launch_k2(const float2* X, const float2* Y, int Np, float2* out, const float2* tw, const unsigned char* bm,
                      unsigned* err, cudaStream_t st) {
  return X == Y ? launch_k2_t<PV, TC, true>(X, Y, Np, out, tw, bm, err, st)
                : launch_k2_t<PV, TC, false>(X, Y, Np, out, tw, bm, err, st);
}

template <bool TC>
cudaError_t dispatch_k1(int Np, const float2* x, int L, int P, const float* window, const float2* tw, float2* X, const unsigned char* bm, unsigned* err, int conj_out,
                        cudaStream_t st) {
  switch (Np) {
    case 16: return launch_k1<16, TC>(x, L, P, window, tw, X, bm, err, conj_out, st);
    case 32: return launch_k1<32, TC>(x, L, P, window, tw, X, bm, err, conj_out, st);
    case 64: return launch_k1<64, TC>(x, L, P, window, tw, X, bm, err, conj_out, st);
    case 128: return launch_k1<128, TC>(x, L, P, window, tw, X, bm, err, conj_out, st);
    case 256: return launch_k1<256, TC>(x, L, P, window, tw, X, bm, err, conj_out, st);
    default: return cudaErrorInvalidValue;
  }
}

template <bool TC>
cudaError_t dispatch_k2(int P, const float2* X, const float2* Y, int Np, float2* out, const float2* tw,
                        const unsigned char* bm, unsigned* err, cudaStream_t st) {
  switch (P) {
    case 2: return launch_k2<2, TC>(X, Y, Np, out, tw, bm, err, st);
    case 4: return launch_k2<4, TC>(X, Y, Np, out, tw, bm, err, st);
    case 8: return launch_k2<8, TC>(X, Y, Np, out, tw, bm, err, st);
    case 16: return launch_k2<16, TC>(X, Y, Np, out, tw, bm, err, st);
    case 32: return launch_k2<32, TC>(X, Y, Np, out, tw, bm, err, st);
    case 64: return launch_k2<64, TC>(X, Y, Np, out, tw, bm, err, st);
    case 128: return launch_k2<128, TC>(X, Y, Np, out, tw, bm, err, st);
    case 256: return launch_k2<256, TC>(X, Y, Np, out, tw, bm, err, st);
    case 512: return launch_k2<512, TC>(X, Y, Np, out, tw, bm, err, st);
    case 1024: return launch_k2<1024, TC>(X, Y, Np, out, tw, bm, err, st);
    case 2048: return launch_k2<2048, TC>(X, Y, Np, out, tw, bm, err, st);
    case 4096: return launch_k2<4096, TC>(X, Y, Np, out, tw, bm, err, st);
    case 8192: return launch_k2<8192, TC>(X, Y, Np, out, tw, bm, err, st);
    case 16384: return launch_k2<16384, TC>(X, Y, Np, out, tw, bm, err, st);
    default: return cudaErrorInvalidValue;
  }
}

// Tables of the split form for a size-M transform.
cudaError_t tc_tables(int M, const unsigned char** bm, unsigned** ew) {
  cudaError_t err;
  int bytes = 0;
  if (!(*bm = table_tc_bmats(M, &bytes, &err))) return err;
  if (!(*ew = device_error_word(&err))) return err;
  return cudaSuccess;
}

}  // namespace

cudaError_t fam_channelise(const float2* x, int Np, int L, int P, const float* window, float2* X, cudaStream_t st,
                           int precision, bool conj_out) {
  cudaError_t err;
  const float2* tw = table_pass(Np, &err);
  if (!tw) return err;
  count_launches(1);
  if (precision == SCD_SPLIT_BF16) {
    const unsigned char* bm;
    unsigned* ew;
    if ((err = tc_tables(Np, &bm, &ew)) != cudaSuccess) return err;
    return dispatch_k1<true>(Np, x, L, P, window, tw, X, bm, ew, conj_out, st);
  }
  return dispatch_k1<false>(Np, x, L, P, window, tw, X, nullptr, nullptr, conj_out, st);
}

cudaError_t fam_pair_fft(const float2* X, const float2* Y, int Np, int P, float2* out, cudaStream_t st, int precision) {
  cudaError_t err;
  const float2* tw = table_pass(P, &err);
  if (!tw) return err;
  count_launches(1);
  if (precision == SCD_SPLIT_BF16) {
    const unsigned char* bm;
    unsigned* ew;
    if ((err = tc_tables(P, &bm, &ew)) != cudaSuccess) return err;
    return dispatch_k2<true>(P, X, Y, Np, out, tw, bm, ew, st);
  }
  return dispatch_k2<false>(P, X, Y, Np, out, tw, nullptr, nullptr, st);
}

cudaError_t fam_channelise_with(const float2* x, int Np, int L, int P, const float* window, float2* X,
                                const float2* tw, cudaStream_t st) {
  count_launches(1);
  return dispatch_k1<false>(Np, x, L, P, window, tw, X, nullptr, nullptr, 0, st);
}

cudaError_t fam_pair_fft_with(const float2* X, int Np, int P, float2* out, const float2* tw, cudaStream_t st) {
  count_launches(1);
  return dispatch_k2<false>(P, X, X, Np, out, tw, nullptr, nullptr, st);
}

}  // namespace scd
