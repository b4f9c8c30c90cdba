// Exact-length batch plans (every sample of every signal: FAM P_i = (len_i - Np)//L + 1,
// SSCA N_i = len_i), run like the staged schedule: one launch per stage and transform size
// over every signal of the plan, captured in the plan's CUDA graph.  The sizes that are not
// powers of two go through Bluestein's identity (bluestein.cuh) with per-signal chirp and
// kernel-spectrum tables; the power-of-two ones through the staged kernels (batch_staged.cu).
//
// SSCA, per signal i (N_i samples, cyclic length M_i = bluestein_len(N_i) = M1 M2,
// Npad_i = N_i rounded up to the channeliser tile):
//   kind 10  xp = x, yp = conj(c) y (c the chirp of N_i), zero from N_i to Npad_i;
//   kind 0   the staged channeliser + CDP on (xp, yp): X_g(n, k) c[n] into the signal's
//            workspace rows of M_i values (first Npad_i of each row written);
//   kind 11  the first size-M_i transform's column pass, in place (rows read up to Npad_i);
//   kind 12  the fused middle pass (row DFT, times Bh, conjugated, second row DFT), in place;
//   kind 13  the second transform's column pass: c[j] conj(G[j]) for j < N_i into the output,
//            fftshifted.
// One launch of kinds 10 and 0 covers every signal; kinds 11..13 run once per cyclic length.
// FAM: the staged channeliser over every signal (kind 3), then per size class the staged pair
// kernel (kind 4, P_i a power of two) or kind 14 (any P_i: both size-MM transforms in one CTA).
#include "batch_kernel.cuh"
#include "bluestein.cuh"

namespace scd {
namespace bk {
namespace {

// kind 10: 1024 values of one signal per CTA
constexpr int kPrepPerTile = 1024;

__global__ void __launch_bounds__(kThreads) k_ex_prep(BatchArgs A, const Task* __restrict__ tl, int nt, int64_t total) {
  const int64_t tile = blockIdx.x;
  const Task& t = tl[find_task(tl, nt, tile)];
  const int64_t base = (tile - t.first) * kPrepPerTile;
  const int64_t npad = t.P;                                     // the padded length Npad_i
  const float2* __restrict__ x = A.x + t.x_off;
  const float2* __restrict__ y = A.y + t.x_off;
  float2* __restrict__ xp = A.ws + t.xp_off;
  float2* __restrict__ yp = A.ws + t.yp_off;
  for (int i = threadIdx.x; i < kPrepPerTile; i += kThreads) {
    const int64_t n = base + i;
    if (n >= npad) break;
    float2 a = make_float2(0.f, 0.f), b = make_float2(0.f, 0.f);
    if (n < t.N) {
      a = __ldg(x + n);
      const float2 yn = __ldg(y + n), cn = __ldg(t.chirp + n);
      b = A.conj ? cmul(yn, cn) : cmulc(yn, cn);
    }
    xp[n] = a;
    yp[n] = b;
  }
}

// kinds 11 / 13: column passes of one cyclic length (tile = C columns of one channel row)
template <int M1, bool TC, bool FINAL>
__global__ void __launch_bounds__(kThreads) k_ex_cols(BatchArgs A, const Task* __restrict__ tl, int nt, int64_t total) {
  extern __shared__ __align__(128) float2 sm[];
  using S = TileShape<M1>;
  using FS = FftSmem<M1, S::C, S::NT, TC>;
  unsigned char* base = reinterpret_cast<unsigned char*>(sm);
  TcCtx ctx{};
  if constexpr (TC) ctx = tc_begin<FS::tmem_cols>(base + FS::region0 + FS::bbytes, base + FS::region0, tl[0].bmats, FS::bbytes, A.err);
  {
    const int64_t tile = blockIdx.x;
    const Task& t = tl[find_task(tl, nt, tile)];
    const int64_t local = tile - t.first;
    const int per = t.M2 / S::C;
    const int64_t kh = local / per;
    const int64_t M = (int64_t)t.M1 * t.M2;
    float2* row = A.ws + t.ws_off + kh * M;
    if constexpr (FINAL) {
      bl_cols_tile<M1, TC, true>(sm, ctx, row, M, A.out + t.out_off + kh * t.N, M, t.M2, t.N, t.wN, t.cols, t.chirp,
                                 t.tw, (int)(local % per) * S::C);
    } else {
      // in place (every read of the tile's columns precedes the transform's first barrier); the
      // rows hold Npad_i (t.P) channeliser values, zero beyond
      bl_cols_tile<M1, TC, false>(sm, ctx, row, t.P, row, M, t.M2, t.N, t.wN, t.cols, nullptr, t.tw,
                                  (int)(local % per) * S::C);
    }
  }
  if constexpr (TC) tc_end<FS::tmem_cols>(ctx);
}

// kind 12: the fused middle pass of one cyclic length, in place (tile = C rows of one channel)
template <int M2, bool TC>
__device__ __forceinline__ void ex_mid_cta(const BatchArgs& A, const Task* __restrict__ tl, int nt) {
  extern __shared__ __align__(128) float2 sm[];
  using S = TileShape<M2>;
  using FS = ResidentSmem<M2, TC>;
  unsigned char* base = reinterpret_cast<unsigned char*>(sm);
  TcCtx ctx{};
  if constexpr (TC) ctx = tc_begin<FS::tmem_cols>(base + FS::region0 + FS::bbytes, base + FS::region0, tl[0].bmats, FS::bbytes, A.err);
  {
    const int64_t tile = blockIdx.x;
    const Task& t = tl[find_task(tl, nt, tile)];
    const int64_t local = tile - t.first;
    const int per = t.M1 / S::C;
    const int64_t kh = local / per;
    float2* row = A.ws + t.ws_off + kh * (int64_t)t.M1 * t.M2;
    bl_mid_tile<M2, TC>(sm, ctx, row, row, t.tw, t.bh, (int)(local % per) * S::C);
  }
  if constexpr (TC) tc_end<FS::tmem_cols>(ctx);
}
template <int M2>
__global__ void __launch_bounds__(kThreads) k_ex_mid_tc(BatchArgs A, const Task* __restrict__ tl, int nt, int64_t total) {
  ex_mid_cta<M2, true>(A, tl, nt);
}
// FP32 form: two CTAs per SM, as the single-estimate middle pass
template <int M2>
__global__ void __launch_bounds__(kThreads, 2) k_ex_mid_f32(BatchArgs A, const Task* __restrict__ tl, int nt, int64_t total) {
  ex_mid_cta<M2, false>(A, tl, nt);
}

// kind 14: FAM pair transforms of any P sharing the cyclic length MM
template <int MM, bool TC>
__device__ __forceinline__ void ex_fpairs_cta(const BatchArgs& A, const Task* __restrict__ tl, int nt) {
  extern __shared__ __align__(128) float2 sm[];
  using S = TileShape<MM>;
  using FS = ResidentSmem<MM, TC>;
  unsigned char* base = reinterpret_cast<unsigned char*>(sm);
  TcCtx ctx{};
  if constexpr (TC) ctx = tc_begin<FS::tmem_cols>(base + FS::region0 + FS::bbytes, base + FS::region0, tl[0].bmats, FS::bbytes, A.err);
  {
    const int64_t tile = blockIdx.x;
    const Task& t = tl[find_task(tl, nt, tile)];
    const float2* X = A.ws + t.ws_off;
    fam_pairs_any_tile<MM, TC, true>(sm, ctx, X, X, A.Np, t.P, A.out + t.out_off, t.tw, t.chirp, t.bh,
                                     (tile - t.first) * S::C);
  }
  if constexpr (TC) tc_end<FS::tmem_cols>(ctx);
}
template <int MM, bool TC>
__global__ void __launch_bounds__(TileShape<MM>::NT) k_ex_fpairs(BatchArgs A, const Task* __restrict__ tl, int nt,
                                                                int64_t total) {
  ex_fpairs_cta<MM, TC>(A, tl, nt);
}
// FP32 form from MM = 2048: two CTAs per SM, as the single-estimate kernel
template <int MM>
__global__ void __launch_bounds__(TileShape<MM>::NT, 2) k_ex_fpairs_2cta(BatchArgs A, const Task* __restrict__ tl,
                                                                        int nt, int64_t total) {
  ex_fpairs_cta<MM, false>(A, tl, nt);
}

template <class K>
cudaError_t prepare_k(K kernel, int smem, bool tc, int* smem_out, int* per_sm, int threads) {
  *smem_out = smem;
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, kernel, threads, smem);
  if (tc && *per_sm < 2) *per_sm = 2;
  return e;
}

template <int M, bool TC>
cudaError_t prep_ex(int kind, int* smem, int* per_sm) {
  if constexpr (M >= 64 && M <= 1024) {
    if (kind == 11)
      return prepare_k(k_ex_cols<M, TC, false>, FftSmem<M, TileShape<M>::C, TileShape<M>::NT, TC>::total, TC, smem,
                       per_sm, kThreads);
    if (kind == 13)
      return prepare_k(k_ex_cols<M, TC, true>, FftSmem<M, TileShape<M>::C, TileShape<M>::NT, TC>::total, TC, smem,
                       per_sm, kThreads);
    if (kind == 12) {
      if constexpr (TC) return prepare_k(k_ex_mid_tc<M>, ResidentSmem<M, true>::total, true, smem, per_sm, kThreads);
      else return prepare_k(k_ex_mid_f32<M>, ResidentSmem<M, false>::total, false, smem, per_sm, kThreads);
    }
  }
  if constexpr (M >= 8 && M <= 16384) {
    if (kind == 14) {
      if constexpr (!TC && M >= 2048 && TileShape<M>::NT <= 256)
        return prepare_k(k_ex_fpairs_2cta<M>, ResidentSmem<M, false>::total, false, smem, per_sm, TileShape<M>::NT);
      else
        return prepare_k(k_ex_fpairs<M, TC>, ResidentSmem<M, TC>::total, TC, smem, per_sm, TileShape<M>::NT);
    }
  }
  return cudaErrorInvalidValue;
}

template <int M, bool TC>
void launch_ex(int kind, int grid, int smem, const BatchArgs& A, const Task* tl, int nt, int64_t total,
               cudaStream_t st) {
  if constexpr (M >= 64 && M <= 1024) {
    if (kind == 11) k_ex_cols<M, TC, false><<<grid, kThreads, smem, st>>>(A, tl, nt, total);
    if (kind == 13) k_ex_cols<M, TC, true><<<grid, kThreads, smem, st>>>(A, tl, nt, total);
    if (kind == 12) {
      if constexpr (TC) k_ex_mid_tc<M><<<grid, kThreads, smem, st>>>(A, tl, nt, total);
      else k_ex_mid_f32<M><<<grid, kThreads, smem, st>>>(A, tl, nt, total);
    }
  }
  if constexpr (M >= 8 && M <= 16384) {
    if (kind == 14) {
      if constexpr (!TC && M >= 2048 && TileShape<M>::NT <= 256)
        k_ex_fpairs_2cta<M><<<grid, TileShape<M>::NT, smem, st>>>(A, tl, nt, total);
      else
        k_ex_fpairs<M, TC><<<grid, TileShape<M>::NT, smem, st>>>(A, tl, nt, total);
    }
  }
}

bool valid_ex(int kind, int M) {
  const bool pow2 = M >= 2 && (M & (M - 1)) == 0;
  if (kind == 10) return true;
  if (kind >= 11 && kind <= 13) return pow2 && M >= 64 && M <= 1024;
  if (kind == 14) return pow2 && M >= 8 && M <= 16384;
  return false;
}

}  // namespace

int exact_prep_per_tile() { return kPrepPerTile; }

cudaError_t exact_prepare(int kind, int M, int Np, bool tc, int* smem, int* per_sm) {
  (void)Np;
  if (!valid_ex(kind, M)) return cudaErrorInvalidValue;
  if (kind == 10) return prepare_k(k_ex_prep, 0, false, smem, per_sm, kThreads);
#define SCD_EP(MV) case MV: return tc ? prep_ex<MV, true>(kind, smem, per_sm) : prep_ex<MV, false>(kind, smem, per_sm);
  switch (M) {
    SCD_EP(8) SCD_EP(16) SCD_EP(32) SCD_EP(64) SCD_EP(128) SCD_EP(256) SCD_EP(512) SCD_EP(1024) SCD_EP(2048)
    SCD_EP(4096) SCD_EP(8192) SCD_EP(16384)
    default: return cudaErrorInvalidValue;
  }
#undef SCD_EP
}

cudaError_t exact_launch(int kind, int M, int Np, bool tc, int grid, int smem, const BatchArgs& A, const Task* tl,
                         int nt, int64_t total, cudaStream_t st) {
  (void)Np;
  if (!valid_ex(kind, M)) return cudaErrorInvalidValue;
  if (kind == 10) {
    k_ex_prep<<<grid, kThreads, 0, st>>>(A, tl, nt, total);
    return cudaGetLastError();
  }
#define SCD_EL(MV) case MV: if (tc) launch_ex<MV, true>(kind, grid, smem, A, tl, nt, total, st); \
                            else launch_ex<MV, false>(kind, grid, smem, A, tl, nt, total, st); break;
  switch (M) {
    SCD_EL(8) SCD_EL(16) SCD_EL(32) SCD_EL(64) SCD_EL(128) SCD_EL(256) SCD_EL(512) SCD_EL(1024) SCD_EL(2048)
    SCD_EL(4096) SCD_EL(8192) SCD_EL(16384)
    default: return cudaErrorInvalidValue;
  }
#undef SCD_EL
  return cudaGetLastError();
}

}  // namespace bk
}  // namespace scd
