// Kernels of the any-length DFTs (bluestein.cuh): the FAM pair stage for any P and the SSCA
// strip transform for any N, in the FP32 form and the split-precision tensor-core form.
//
// FAM (Eq. II.B-SCD_function_FAM with P not a power of two): one CTA runs C pairs; each pair's
// conjugate product times the chirp goes through a size-MM FFT, the product with the kernel
// spectrum stays in the transform's shared-memory region, a second FFT and the chirp give the
// P bins, stored fftshifted.  X and Y (Np P values each) stay in L2 as in the power-of-two
// pair kernel, so DRAM traffic is again about the 8 Np^2 P output bytes; the arithmetic grows
// to two transforms of size MM in [2P - 1, 4P - 3].
//
// SSCA (Eq. II.B-SSCA_auto with N not a power of two), three stages:
//   0. the inputs padded with zeros to a multiple of the channeliser tile and the chirp folded
//      into the second factor (k_bl_prep), then the power-of-two K3 (channeliser + CDP):
//      X_g(n, k) c[n] for n < N, zero beyond, rows of Npad values;
//   1. the first size-M transform's column pass (reading the short rows, zero beyond), then the
//      fused middle pass (row DFT, times Bh and conjugated, the second transform's row DFT);
//   2. the second transform's column pass, c[j] conj(G[j]) for j < N stored fftshifted.
// Workspace: [x padded | y' padded | W1 (Np M) | W2 (Np M)]; X_g lives in W2 (row stride
// Npad) until the middle pass overwrites it.
#include <algorithm>

#include "bluestein.cuh"
#include "internal.h"

namespace scd {
namespace {

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

// ---------------------------------------------------------------- FAM
template <int MM, bool TC>
__device__ __forceinline__ void fam_pairs_any_cta(const float2* __restrict__ X, const float2* __restrict__ Y, int Np,
                                                  int P, float2* __restrict__ out, const float2* __restrict__ tw,
                                                  const float2* __restrict__ chirp, const float2* __restrict__ bh,
                                                  const unsigned char* __restrict__ bmats, unsigned* err) {
  extern __shared__ __align__(128) float2 sm[];
  using S = TileShape<MM>;
  using FS = ResidentSmem<MM, TC>;
  unsigned char* base = reinterpret_cast<unsigned char*>(sm);
  TcCtx ctx{};
  if constexpr (TC) ctx = tc_begin<FS::tmem_cols>(base + FS::region0 + FS::bbytes, base + FS::region0, bmats, FS::bbytes, err);
  // the auto estimate (Y is X): the pairs kh <= lh, both rows from each
  if (X == Y) fam_pairs_any_tile<MM, TC, true>(sm, ctx, X, Y, Np, P, out, tw, chirp, bh, (int64_t)blockIdx.x * S::C);
  else fam_pairs_any_tile<MM, TC, false>(sm, ctx, X, Y, Np, P, out, tw, chirp, bh, (int64_t)blockIdx.x * S::C);
  if constexpr (TC) tc_end<FS::tmem_cols>(ctx);
}

template <int MM, bool TC>
__global__ void __launch_bounds__(TileShape<MM>::NT)
k_fam_pairs_any(const float2* __restrict__ X, const float2* __restrict__ Y, int Np, int P, float2* __restrict__ out,
                const float2* __restrict__ tw, const float2* __restrict__ chirp, const float2* __restrict__ bh,
                const unsigned char* __restrict__ bmats, unsigned* err) {
  fam_pairs_any_cta<MM, TC>(X, Y, Np, P, out, tw, chirp, bh, bmats, err);
}

// The same kernel held to 128 registers per thread, so that two 256-thread CTAs share an SM.
template <int MM, bool TC>
__global__ void __launch_bounds__(TileShape<MM>::NT, 2)
k_fam_pairs_any_2cta(const float2* __restrict__ X, const float2* __restrict__ Y, int Np, int P,
                     float2* __restrict__ out, const float2* __restrict__ tw, const float2* __restrict__ chirp,
                     const float2* __restrict__ bh, const unsigned char* __restrict__ bmats, unsigned* err) {
  fam_pairs_any_cta<MM, TC>(X, Y, Np, P, out, tw, chirp, bh, bmats, err);
}

template <class K>
cudaError_t launch_fam_any_k(K kernel, int smem, int NT, int C, const float2* X, const float2* Y, int Np, int P,
                             float2* out, const float2* tw, const float2* chirp, const float2* bh, TcArgs t,
                             cudaStream_t st) {
  cudaError_t e = set_smem(kernel, smem);
  if (e != cudaSuccess) return e;
  const int64_t npairs = X == Y ? (int64_t)Np * (Np + 1) / 2 : (int64_t)Np * Np;     // auto estimate: kh <= lh
  kernel<<<(unsigned)((npairs + C - 1) / C), NT, smem, st>>>(X, Y, Np, P, out, tw, chirp, bh, t.bm, t.err);
  return cudaGetLastError();
}

// The FP32 form from MM = 2048 runs two CTAs per SM (Np = 256, P = 1000: 0.86 -> 0.64 ms;
// Np = 64, P = 4000: 0.24 -> 0.21 ms); below MM = 2048 the register cap spills, and the
// tensor-core form lost time under it.
template <int MM, bool TC>
cudaError_t launch_fam_any(const float2* X, const float2* Y, int Np, int P, float2* out, const float2* tw,
                           const float2* chirp, const float2* bh, TcArgs t, cudaStream_t st) {
  using S = TileShape<MM>;
  constexpr int sm = ResidentSmem<MM, TC>::total;
  if constexpr (!TC && MM >= 2048 && S::NT <= 256)
    return launch_fam_any_k(k_fam_pairs_any_2cta<MM, TC>, sm, S::NT, S::C, X, Y, Np, P, out, tw, chirp, bh, t, st);
  else
    return launch_fam_any_k(k_fam_pairs_any<MM, TC>, sm, S::NT, S::C, X, Y, Np, P, out, tw, chirp, bh, t, st);
}

// ---------------------------------------------------------------- SSCA
// xp[n] = x[n], yp[n] = y[n] conj(c[n]) (conj: y[n] c[n]) for n < N, both 0 for N <= n < Npad.
// The channeliser's product X_T conj(yp) (X_T yp) is then X_g(n, k) c[n].
__global__ void __launch_bounds__(256)
k_bl_prep(const float2* __restrict__ x, const float2* __restrict__ y, int conj, int64_t N, int64_t Npad,
          const float2* __restrict__ chirp, float2* __restrict__ xp, float2* __restrict__ yp) {
  for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < Npad; n += (int64_t)gridDim.x * blockDim.x) {
    float2 a = make_float2(0.f, 0.f), b = make_float2(0.f, 0.f);
    if (n < N) {
      a = __ldg(x + n);
      const float2 yn = __ldg(y + n), cn = __ldg(chirp + n);
      b = conj ? cmul(yn, cn) : cmulc(yn, cn);
    }
    xp[n] = a;
    yp[n] = b;
  }
}

template <int M1, bool TC, bool FINAL>
__global__ void __launch_bounds__(TileShape<M1>::NT)
k_bl_cols(const float2* __restrict__ in, int64_t ld, int64_t nvalid, float2* __restrict__ out, int64_t ldo, int64_t M,
          int M2, int64_t N, const float2* __restrict__ wM, const float2* __restrict__ cols,
          const float2* __restrict__ chirp, const float2* __restrict__ tw, const unsigned char* __restrict__ bmats,
          unsigned* err) {
  extern __shared__ __align__(128) float2 sm[];
  using S = TileShape<M1>;
  using FS = FftSmem<M1, S::C, S::NT, TC>;
  unsigned char* base = reinterpret_cast<unsigned char*>(sm);
  TcCtx ctx{};
  if constexpr (TC) ctx = tc_begin<FS::tmem_cols>(base + FS::region0 + FS::bbytes, base + FS::region0, bmats, FS::bbytes, err);
  bl_cols_tile<M1, TC, FINAL>(sm, ctx, in + (int64_t)blockIdx.y * ld, nvalid, out + (int64_t)blockIdx.y * ldo, M, M2, N,
                              wM, cols, chirp, tw, blockIdx.x * S::C);
  if constexpr (TC) tc_end<FS::tmem_cols>(ctx);
}

template <int M2, bool TC>
__device__ __forceinline__ void bl_mid_cta(const float2* __restrict__ in, float2* __restrict__ out, int64_t M,
                                           const float2* __restrict__ tw, const float2* __restrict__ bhr,
                                           const unsigned char* __restrict__ bmats, unsigned* err) {
  extern __shared__ __align__(128) float2 sm[];
  using S = TileShape<M2>;
  using FS = ResidentSmem<M2, TC>;
  unsigned char* base = reinterpret_cast<unsigned char*>(sm);
  TcCtx ctx{};
  if constexpr (TC) ctx = tc_begin<FS::tmem_cols>(base + FS::region0 + FS::bbytes, base + FS::region0, bmats, FS::bbytes, err);
  bl_mid_tile<M2, TC>(sm, ctx, in + (int64_t)blockIdx.y * M, out + (int64_t)blockIdx.y * M, tw, bhr, blockIdx.x * S::C);
  if constexpr (TC) tc_end<FS::tmem_cols>(ctx);
}

// Tensor-core form: registers as the compiler picks them.
template <int M2>
__global__ void __launch_bounds__(TileShape<M2>::NT)
k_bl_mid_tc(const float2* __restrict__ in, float2* __restrict__ out, int64_t M, const float2* __restrict__ tw,
            const float2* __restrict__ bhr, const unsigned char* __restrict__ bmats, unsigned* err) {
  bl_mid_cta<M2, true>(in, out, M, tw, bhr, bmats, err);
}

// FP32 form: two CTAs per SM (N = 500,000, Np = 256: 3.81 -> 3.52 ms per estimate).
template <int M2>
__global__ void __launch_bounds__(TileShape<M2>::NT, 2)
k_bl_mid_f32(const float2* __restrict__ in, float2* __restrict__ out, int64_t M, const float2* __restrict__ tw,
             const float2* __restrict__ bhr, const unsigned char* __restrict__ bmats, unsigned* err) {
  bl_mid_cta<M2, false>(in, out, M, tw, bhr, bmats, err);
}

// Column pass of either transform over Np channel rows: in rows of stride ld (first nvalid
// values given), out rows of stride ldo.
template <int MV, bool TC, bool FINAL>
cudaError_t launch_cols_t(const float2* in, int64_t ld, int64_t nvalid, float2* out, int64_t ldo, int64_t M, int64_t N,
                          int Np, int M1, int M2, const float2* chirp, cudaStream_t st) {
  using S = TileShape<MV>;
  cudaError_t err;
  TcArgs t;
  if ((err = tc_args(TC, M1, &t)) != cudaSuccess) return err;
  const float2* wM = table_roots((int)M, &err);
  if (!wM) return err;
  const float2* cols = table_cols((int)M, M1, S::C, &err);
  if (!cols) return err;
  const float2* tw = table_pass(M1, &err);
  if (!tw) return err;
  constexpr int sm = FftSmem<MV, S::C, S::NT, TC>::total;
  if ((err = set_smem(k_bl_cols<MV, TC, FINAL>, sm)) != cudaSuccess) return err;
  k_bl_cols<MV, TC, FINAL><<<dim3(M2 / S::C, Np), S::NT, sm, st>>>(in, ld, nvalid, out, ldo, M, M2, N, wM, cols, chirp,
                                                                   tw, t.bm, t.err);
  return cudaGetLastError();
}

template <int MV, bool TC>
cudaError_t launch_mid_t(const float2* in, float2* out, int64_t M, int64_t N, int Np, int M1, int M2,
                         cudaStream_t st) {
  using S = TileShape<MV>;
  cudaError_t err;
  TcArgs t;
  if ((err = tc_args(TC, M2, &t)) != cudaSuccess) return err;
  const float2* tw = table_pass(M2, &err);
  if (!tw) return err;
  const float2* bhr = table_bluestein_rows(N, M, M1, &err);
  if (!bhr) return err;
  constexpr int sm = ResidentSmem<MV, TC>::total;
  auto kernel = TC ? k_bl_mid_tc<MV> : k_bl_mid_f32<MV>;
  if ((err = set_smem(kernel, sm)) != cudaSuccess) return err;
  kernel<<<dim3(M1 / S::C, Np), S::NT, sm, st>>>(in, out, M, tw, bhr, t.bm, t.err);
  return cudaGetLastError();
}

template <bool TC, bool FINAL>
cudaError_t launch_cols(const float2* in, int64_t ld, int64_t nvalid, float2* out, int64_t ldo, int64_t M, int64_t N,
                        int Np, int M1, int M2, const float2* chirp, cudaStream_t st) {
  switch (M1) {
#define SCD_BC(MV) case MV: return launch_cols_t<MV, TC, FINAL>(in, ld, nvalid, out, ldo, M, N, Np, M1, M2, chirp, st);
    SCD_BC(64) SCD_BC(128) SCD_BC(256) SCD_BC(512) SCD_BC(1024)
#undef SCD_BC
    default: return cudaErrorInvalidValue;
  }
}

template <bool TC>
cudaError_t launch_mid(const float2* in, float2* out, int64_t M, int64_t N, int Np, int M1, int M2, cudaStream_t st) {
  switch (M2) {
#define SCD_BM(MV) case MV: return launch_mid_t<MV, TC>(in, out, M, N, Np, M1, M2, st);
    SCD_BM(64) SCD_BM(128) SCD_BM(256) SCD_BM(512) SCD_BM(1024)
#undef SCD_BM
    default: return cudaErrorInvalidValue;
  }
}

int cdp_tile(int Np) {                      // time points per K3 tile
  switch (Np) {
    case 16: return TileShape<16>::C;
    case 32: return TileShape<32>::C;
    case 64: return TileShape<64>::C;
    case 128: return TileShape<128>::C;
    case 256: return TileShape<256>::C;
    default: return 0;
  }
}

size_t up256(size_t v) { return (v + 255) / 256 * 256; }

struct AnyLayout {
  int64_t Npad, M;
  int M1, M2;
  float2 *xp, *yp, *w1, *w2;
};

AnyLayout any_layout(int64_t N, int Np, void* ws) {
  AnyLayout a;
  const int64_t c = cdp_tile(Np);
  a.Npad = c > 0 ? (N + c - 1) / c * c : N;
  a.M = bluestein_len(N);
  ssca_split(a.M, &a.M1, &a.M2);
  char* p = (char*)ws;
  a.xp = (float2*)p;  p += up256(8 * (size_t)a.Npad);
  a.yp = (float2*)p;  p += up256(8 * (size_t)a.Npad);
  a.w1 = (float2*)p;  p += up256(8 * (size_t)Np * a.M);
  a.w2 = (float2*)p;
  return a;
}

}  // namespace

cudaError_t fam_pair_fft_any(const float2* X, const float2* Y, int Np, int P, float2* out, cudaStream_t st,
                             int precision) {
  const int64_t MM = bluestein_len(P);
  cudaError_t err;
  const float2* tw = table_pass((int)MM, &err);
  if (!tw) return err;
  const float2* chirp = table_chirp(P, &err);
  if (!chirp) return err;
  const float2* bh = table_bluestein(P, MM, &err);
  if (!bh) return err;
  const bool tc = precision == SCD_SPLIT_BF16;
  TcArgs t;
  if ((err = tc_args(tc, (int)MM, &t)) != cudaSuccess) return err;
  count_launches(1);
#define SCD_FA(MV) return tc ? launch_fam_any<MV, true>(X, Y, Np, P, out, tw, chirp, bh, t, st) \
                             : launch_fam_any<MV, false>(X, Y, Np, P, out, tw, chirp, bh, t, st)
  switch (MM) {
    case 8: SCD_FA(8);
    case 16: SCD_FA(16);
    case 32: SCD_FA(32);
    case 64: SCD_FA(64);
    case 128: SCD_FA(128);
    case 256: SCD_FA(256);
    case 512: SCD_FA(512);
    case 1024: SCD_FA(1024);
    case 2048: SCD_FA(2048);
    case 4096: SCD_FA(4096);
    case 8192: SCD_FA(8192);
    case 16384: SCD_FA(16384);
    default: return cudaErrorInvalidValue;
  }
#undef SCD_FA
}

size_t ssca_any_workspace(int64_t N, int Np) {
  const AnyLayout a = any_layout(N, Np, nullptr);
  return 2 * up256(8 * (size_t)a.Npad) + 2 * up256(8 * (size_t)Np * a.M);
}

cudaError_t ssca_any_cdp(const float2* x, const float2* y, bool conj, int64_t N, int Np, const float* window,
                         void* ws, cudaStream_t st, int precision) {
  const AnyLayout a = any_layout(N, Np, ws);
  cudaError_t err;
  const float2* chirp = table_chirp(N, &err);
  if (!chirp) return err;
  count_launches(1);
  k_bl_prep<<<(unsigned)std::min<int64_t>((a.Npad + 255) / 256, 152 * 8), 256, 0, st>>>(x, y, conj ? 1 : 0, N, a.Npad,
                                                                                      chirp, a.xp, a.yp);
  if ((err = cudaGetLastError()) != cudaSuccess) return err;
  return ssca_cdp(a.xp, a.yp, conj, a.Npad, Np, window, a.w2, st, precision);
}

cudaError_t ssca_any_first(int64_t N, int Np, void* ws, cudaStream_t st, int precision) {
  const AnyLayout a = any_layout(N, Np, ws);
  const bool tc = precision == SCD_SPLIT_BF16;
  count_launches(2);
  // first transform's column pass: X_g (rows of Npad values) -> W1; fused middle: W1 -> W2
  cudaError_t err = tc ? launch_cols<true, false>(a.w2, a.Npad, a.Npad, a.w1, a.M, a.M, N, Np, a.M1, a.M2, nullptr, st)
                       : launch_cols<false, false>(a.w2, a.Npad, a.Npad, a.w1, a.M, a.M, N, Np, a.M1, a.M2, nullptr, st);
  if (err != cudaSuccess) return err;
  return tc ? launch_mid<true>(a.w1, a.w2, a.M, N, Np, a.M1, a.M2, st)
            : launch_mid<false>(a.w1, a.w2, a.M, N, Np, a.M1, a.M2, st);
}

cudaError_t ssca_any_second(int64_t N, int Np, void* ws, float2* out, cudaStream_t st, int precision) {
  const AnyLayout a = any_layout(N, Np, ws);
  cudaError_t err;
  const float2* chirp = table_chirp(N, &err);
  if (!chirp) return err;
  const bool tc = precision == SCD_SPLIT_BF16;
  count_launches(1);
  // second transform's column pass: W2 -> the fftshifted output (rows of N values)
  return tc ? launch_cols<true, true>(a.w2, a.M, a.M, out, N, a.M, N, Np, a.M1, a.M2, chirp, st)
            : launch_cols<false, true>(a.w2, a.M, a.M, out, N, a.M, N, Np, a.M1, a.M2, chirp, st);
}

}  // namespace scd
