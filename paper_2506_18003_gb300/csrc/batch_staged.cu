// Staged schedule of a batch plan: instead of one persistent launch with a device work queue,
// one launch per stage and transform size over every signal of the plan, in stream order (no
// device-side waits).  SSCA: the channeliser + CDP of all signals, then per size class the
// column passes (in place on each signal's X_g) and the row passes (to the output arena).
// FAM: the channelisers of all signals, then per size class P the pair transforms.
// Each kernel has only its own tile's registers and shared memory, so it runs at the
// occupancy of the standalone kernels (the column pass's registers capped for 2 CTAs per SM
// at M1 >= 512, 3 at 128 and 256, 4 below); the price is the X_g round trip through HBM that the
// persistent schedule's rotating slots avoid.  The autotuner picks the faster of the two.
//
// Every kernel runs one CTA tile per CTA (grid = the launch's tiles); task i covers the tiles
// [first_i, first_i + subtiles_i) and a CTA finds its task by binary search.  (A persistent
// walk over the tiles kept more state live and spilled in the column pass.)
#include "batch_kernel.cuh"
#include "ssca_fused.cuh"

namespace scd {
namespace bk {
namespace {

template <int NP, bool TC>
__device__ __forceinline__ void st_cdp_cta(const BatchArgs& A, const Task* __restrict__ tl, int nt) {
  extern __shared__ __align__(128) float2 sm[];
  using FS = CdpSmem<NP, TC>;
  static_assert(TileShape<NP>::NT == kThreads, "one tile per CTA");
  unsigned char* base = reinterpret_cast<unsigned char*>(sm);
  TcCtx ctx{};
  if constexpr (TC) ctx = tc_begin<FS::tmem_cols>(base + FS::region0 + FS::bbytes, base + FS::region0, A.bmats_np, FS::bbytes, A.err);
  {
    const int64_t tile = blockIdx.x;
    const Task& t = tl[find_task(tl, nt, tile)];
    const int64_t local = tile - t.first;
    // exact-length plans: the zero-padded inputs with the chirp folded in sit in the workspace
    const float2* xb = t.in_ws ? A.ws + t.xp_off : A.x + t.x_off;
    const float2* yb = t.in_ws ? A.ws + t.yp_off : A.y + t.x_off;
    ssca_cdp_tile<NP, TC>(sm, ctx, xb, yb, A.conj != 0, t.N, A.window, A.tw_np, A.ws + t.ws_off,
                          (int)local * TileShape<NP>::C, base + CdpStage<NP, TC>::off, t.ld);
  }
  if constexpr (TC) tc_end<FS::tmem_cols>(ctx);
}

template <int NP, bool TC>
__global__ void __launch_bounds__(kThreads) k_st_cdp(BatchArgs A, const Task* __restrict__ tl, int nt, int64_t total) {
  st_cdp_cta<NP, TC>(A, tl, nt);
}

// The FP32 channeliser at Np >= 64 held to 48 registers: five CTAs per SM, as its shared memory
// allows (batch SSCA 23.42 -> 23.12 ms; the split form, capped for three, lost 35.8 -> 37.2 ms).
template <int NP>
__global__ void __launch_bounds__(kThreads, 5) k_st_cdp5(BatchArgs A, const Task* __restrict__ tl, int nt, int64_t total) {
  st_cdp_cta<NP, false>(A, tl, nt);
}
template <int NP, bool TC>
constexpr bool cdp_capped() { return !TC && NP >= 64; }

// Column passes of one size class (all tasks share N, M1, M2 and the tables).
template <int M1, bool TC>
__global__ void __launch_bounds__(kThreads, M1 >= 512 ? 2 : (M1 >= 128 ? 3 : 4)) k_st_cols(BatchArgs A, const Task* __restrict__ tl, int nt, int64_t total) {
  extern __shared__ __align__(128) float2 sm[];
  using S = TileShape<M1>;
  using FS = ColsSmem<M1, TC>;
  unsigned char* base = reinterpret_cast<unsigned char*>(sm);
  TcCtx ctx{};
  if constexpr (TC) ctx = tc_begin<FS::tmem_cols>(base + FS::region0 + FS::bbytes, base + FS::region0, tl[0].bmats, FS::bbytes, A.err);
  {
    const int64_t tile = blockIdx.x;
    const Task& t = tl[find_task(tl, nt, tile)];
    const int64_t local = tile - t.first;
    const int per = t.M2 / S::C;
    const int64_t kh = local / per;
    float2* row = A.ws + t.ws_off + kh * t.N;
    ssca_cols_tile<M1, TC>(sm, ctx, row, row, t.N, t.M2, t.wN, t.cols, t.tw, (int)(local % per) * S::C,
                           reinterpret_cast<float2*>(base + ColsStage<M1, TC>::off));
  }
  if constexpr (TC) tc_end<FS::tmem_cols>(ctx);
}

// Row passes of one size class; PROF: each bin reduced into the signal's alpha profile
// (out arena of float32 profiles) instead of stored.
template <int M2, bool TC, bool PROF>
__global__ void __launch_bounds__(kThreads) k_st_rows(BatchArgs A, const Task* __restrict__ tl, int nt, int64_t total) {
  extern __shared__ __align__(128) float2 sm[];
  using S = TileShape<M2>;
  using FS = FftSmem<M2, S::C, S::NT, TC, rows_stage_bytes<M2>()>;
  unsigned char* base = reinterpret_cast<unsigned char*>(sm);
  TcCtx ctx{};
  if constexpr (TC) ctx = tc_begin<FS::tmem_cols>(base + FS::region0 + FS::bbytes, base + FS::region0, tl[0].bmats, FS::bbytes, A.err);
  {
    const int64_t tile = blockIdx.x;
    const Task& t = tl[find_task(tl, nt, tile)];
    const int64_t local = tile - t.first;
    const int per = t.M1 / S::C;
    const int64_t kh = local / per;
    if constexpr (PROF) {
      // alpha column of stored bin sh of channel k: ah = sh + k N/Np + N/2
      const int ah_off = (int)(kh - A.Np / 2) * (t.N / A.Np) + t.N / 2;
      ssca_rows_tile<M2, TC, false, true>(sm, ctx, A.ws + t.ws_off + kh * t.N, nullptr, t.M1, t.tw,
                                          (int)(local % per) * S::C, reinterpret_cast<float*>(A.out) + t.out_off,
                                          ah_off, A.prof_power);
    } else {
      ssca_rows_tile<M2, TC>(sm, ctx, A.ws + t.ws_off + kh * t.N, A.out + t.out_off + kh * t.N, t.M1, t.tw,
                             (int)(local % per) * S::C);
    }
  }
  if constexpr (TC) tc_end<FS::tmem_cols>(ctx);
}

// Fused SSCA (ssca_fused.cuh), one launch per size class N: tile A = channeliser + CDP + the
// M1-point pass over m1 of column m2, clusters of Q CTAs (a task's tiles are m2 Q + q, and
// every task's first tile is a multiple of Q, so a cluster never straddles two signals) ...
template <int NP, int M1, int Q>
__global__ void __cluster_dims__(Q, 1, 1) __launch_bounds__(kThreads, 2)
    k_st_sfa(BatchArgs A, const Task* __restrict__ tl, int nt, int64_t total) {
  extern __shared__ __align__(128) float2 sm[];
  const int64_t tile = blockIdx.x;
  const Task& t = tl[find_task(tl, nt, tile)];
  const int local = (int)(tile - t.first);
  ssca_chancol_tile<NP, M1, Q>(sm, A.x + t.x_off, A.y + t.x_off, A.conj != 0, t.N, t.M2, A.window, A.tw_np, t.tw,
                               t.wN, A.ws + t.ws_off, local / Q, local % Q);
}

// ... and tile B = the M2-point pass over m2 for C consecutive q1 of one channel; PROF: each
// bin reduced into the signal's alpha profile instead of stored.
template <int M2, bool PROF>
__global__ void __launch_bounds__(rowsf_threads(M2), M2 >= 2048 ? 1 : (M2 >= 1024 ? 2 : 3))
    k_st_sfb(BatchArgs A, const Task* __restrict__ tl, int nt, int64_t total) {
  extern __shared__ __align__(128) float2 sm[];
  constexpr int C = rowsf_c(M2);
  const int64_t tile = blockIdx.x;
  const Task& t = tl[find_task(tl, nt, tile)];
  const int64_t local = tile - t.first;
  const int per = t.M1 / C;
  const int64_t kh = local / per;
  const int q10 = (int)(local % per) * C;
  const float2* Yk = A.ws + t.ws_off + kh * t.N;
  if constexpr (PROF) {
    const int ah_off = (int)(kh - A.Np / 2) * (t.N / A.Np) + t.N / 2;
    ssca_rowsf_tile<M2, true>(sm, Yk, nullptr, t.M1, t.tw, q10, reinterpret_cast<float*>(A.out) + t.out_off, ah_off,
                              A.prof_power);
  } else {
    ssca_rowsf_tile<M2, false>(sm, Yk, A.out + t.out_off + kh * t.N, t.M1, t.tw, q10);
  }
}

// FAM channelisers of all signals (X[kh][p] of signal i at ws + ws_off_i).
template <int NP, bool TC>
__global__ void __launch_bounds__(kThreads) k_st_fchan(BatchArgs A, const Task* __restrict__ tl, int nt, int64_t total) {
  extern __shared__ __align__(128) float2 sm[];
  using S = TileShape<NP>;
  using FS = FftSmem<NP, S::C, S::NT, TC>;
  unsigned char* base = reinterpret_cast<unsigned char*>(sm);
  TcCtx ctx{};
  if constexpr (TC) ctx = tc_begin<FS::tmem_cols>(base + FS::region0 + FS::bbytes, base + FS::region0, A.bmats_np, FS::bbytes, A.err);
  {
    const int64_t tile = blockIdx.x;
    const Task& t = tl[find_task(tl, nt, tile)];
    fam_channelise_tile<NP, TC>(sm, ctx, A.x + t.x_off, A.L, t.P, A.window, A.tw_np, A.ws + t.ws_off,
                                (int)(tile - t.first) * S::C);
  }
  if constexpr (TC) tc_end<FS::tmem_cols>(ctx);
}

// FAM pair transforms of one size class P, the FP32 form's registers capped for 2 CTAs per SM at
// P = 512 and 1024 (128 registers; 3 at 80 measured 0.3% slower on the FAM batch), 4 at 2048 and
// 4096, 3 at 8192 (80 registers, 44 bytes of spills: the FAM batch 11.03 -> 10.60 ms against 2
// CTAs of 128 registers) except in the profile mode, whose reduction needs more registers there
// (2); the split form at 2 CTAs per SM (128 registers instead of up to 221: its staged FAM batch
// 23.97 -> 19.87 ms).
template <int PP, bool TC, bool PROF>
__host__ __device__ constexpr int fpairs_minb() {
  return TC ? 2 : (PP == 8192 ? (PROF ? 2 : 3) : (PP >= 2048 ? 4 : (PP >= 512 ? 2 : 1)));
}
template <int PP, bool TC, bool PROF>
__global__ void __launch_bounds__(kThreads, fpairs_minb<PP, TC, PROF>()) k_st_fpairs(BatchArgs A, const Task* __restrict__ tl,
                                                                              int nt, int64_t total) {
  extern __shared__ __align__(128) float2 sm[];
  using S = TileShape<PP>;
  using FS = FftSmem<PP, S::C, S::NT, TC>;
  unsigned char* base = reinterpret_cast<unsigned char*>(sm);
  TcCtx ctx{};
  if constexpr (TC) ctx = tc_begin<FS::tmem_cols>(base + FS::region0 + FS::bbytes, base + FS::region0, tl[0].bmats, FS::bbytes, A.err);
  {
    const int64_t tile = blockIdx.x;
    const Task& t = tl[find_task(tl, nt, tile)];
    const float2* X = A.ws + t.ws_off;
    if constexpr (PROF) {
      const int PL = t.P * A.L;
      fam_pairs_tile<PP, TC, true, true>(sm, ctx, X, X, A.Np, nullptr, t.tw, (tile - t.first) * S::C,
                                   reinterpret_cast<float*>(A.out) + t.out_off, PL, PL / A.Np, A.prof_power);
    } else {
      fam_pairs_tile<PP, TC, false, true>(sm, ctx, X, X, A.Np, A.out + t.out_off, t.tw, (tile - t.first) * S::C);
    }
  }
  if constexpr (TC) tc_end<FS::tmem_cols>(ctx);
}

template <class K>
cudaError_t prepare_t(K kernel, int smem, bool tc, int* smem_out, int* per_sm) {
  *smem_out = smem;
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, kernel, kThreads, smem);
  // the query answers one for kernels that allocate tensor memory; two CTAs of at most 128
  // TMEM columns always fit (as for the persistent kernel)
  if (tc && *per_sm < 2) *per_sm = 2;
  return e;
}

// Fused tile A of the size class N at Np channels (kind 7).
template <int NP, int M1, int Q>
cudaError_t prep_sfa(int* smem, int* per_sm) {
  return prepare_t(k_st_sfa<NP, M1, Q>, ChanColSmem<NP, M1, Q>::total, false, smem, per_sm);
}
template <int NP, int M1, int Q>
void launch_sfa(int grid, int smem, const BatchArgs& A, const Task* tl, int nt, int64_t total, cudaStream_t st) {
  k_st_sfa<NP, M1, Q><<<grid, kThreads, smem, st>>>(A, tl, nt, total);
}
#define SCD_SFA_SHAPES(X) \
  X(64, 64, 1) X(64, 128, 1) X(64, 256, 2) X(128, 64, 1) X(128, 128, 2) X(128, 256, 4) X(256, 64, 2) X(256, 128, 4)

template <int M, bool TC>
cudaError_t prep_m(int kind, int* smem, int* per_sm) {
  using S = TileShape<M>;
  if constexpr (M >= 16 && M <= 256) {
    if (kind == 0) {
      if constexpr (cdp_capped<M, TC>()) return prepare_t(k_st_cdp5<M>, CdpSmem<M, TC>::total, TC, smem, per_sm);
      else return prepare_t(k_st_cdp<M, TC>, CdpSmem<M, TC>::total, TC, smem, per_sm);
    }
    if (kind == 3) return prepare_t(k_st_fchan<M, TC>, FftSmem<M, S::C, S::NT, TC>::total, TC, smem, per_sm);
  }
  if constexpr (M <= 8192) {
    if (kind == 4) return prepare_t(k_st_fpairs<M, TC, false>, FftSmem<M, S::C, S::NT, TC>::total, TC, smem, per_sm);
    if (kind == 6) return prepare_t(k_st_fpairs<M, TC, true>, FftSmem<M, S::C, S::NT, TC>::total, TC, smem, per_sm);
  }
  if constexpr (M >= 64 && M <= 2048 && !TC) {
    using SB = TileShape<M, rowsf_threads(M)>;
    if (kind == 8) return prepare_t(k_st_sfb<M, false>, FftSmem<M, SB::C, SB::NT, false>::total, false, smem, per_sm);
    if (kind == 9) return prepare_t(k_st_sfb<M, true>, FftSmem<M, SB::C, SB::NT, false>::total, false, smem, per_sm);
  }
  if constexpr (M >= 64 && M <= 1024) {
    if (kind == 1) return prepare_t(k_st_cols<M, TC>, ColsSmem<M, TC>::total, TC, smem, per_sm);
    if (kind == 2)
      return prepare_t(k_st_rows<M, TC, false>, FftSmem<M, S::C, S::NT, TC, rows_stage_bytes<M>()>::total, TC, smem,
                       per_sm);
    if (kind == 5)
      return prepare_t(k_st_rows<M, TC, true>, FftSmem<M, S::C, S::NT, TC, rows_stage_bytes<M>()>::total, TC, smem,
                       per_sm);
  }
  return cudaErrorInvalidValue;
}

template <int M, bool TC>
void launch_m(int kind, int grid, int smem, const BatchArgs& A, const Task* tl, int nt, int64_t total, cudaStream_t st) {
  if constexpr (M >= 16 && M <= 256) {
    if (kind == 0) {
      if constexpr (cdp_capped<M, TC>()) k_st_cdp5<M><<<grid, kThreads, smem, st>>>(A, tl, nt, total);
      else k_st_cdp<M, TC><<<grid, kThreads, smem, st>>>(A, tl, nt, total);
    }
    if (kind == 3) k_st_fchan<M, TC><<<grid, kThreads, smem, st>>>(A, tl, nt, total);
  }
  if constexpr (M <= 8192) {
    if (kind == 4) k_st_fpairs<M, TC, false><<<grid, kThreads, smem, st>>>(A, tl, nt, total);
    if (kind == 6) k_st_fpairs<M, TC, true><<<grid, kThreads, smem, st>>>(A, tl, nt, total);
  }
  if constexpr (M >= 64 && M <= 2048 && !TC) {
    if (kind == 8) k_st_sfb<M, false><<<grid, rowsf_threads(M), smem, st>>>(A, tl, nt, total);
    if (kind == 9) k_st_sfb<M, true><<<grid, rowsf_threads(M), smem, st>>>(A, tl, nt, total);
  }
  if constexpr (M >= 64 && M <= 1024) {
    if (kind == 1) k_st_cols<M, TC><<<grid, kThreads, smem, st>>>(A, tl, nt, total);
    if (kind == 2) k_st_rows<M, TC, false><<<grid, kThreads, smem, st>>>(A, tl, nt, total);
    if (kind == 5) k_st_rows<M, TC, true><<<grid, kThreads, smem, st>>>(A, tl, nt, total);
  }
}

// kinds: SSCA 0 channeliser + CDP (M = Np in 16..256), 1 column pass (M = M1), 2 row pass
// (M = M2), M1 and M2 in 64..1024; FAM 3 channeliser (M = Np), 4 pair transforms (M = P in
// 2..8192); 5 and 6: kinds 2 and 4 reducing into alpha profiles; fused SSCA (FP32 form):
// 7 tile A (M = N, the split from fused_split(N, Np)), 8 tile B (M = M2 in 64..1024), 9 tile B
// reducing into alpha profiles
bool valid(int kind, int M, bool tc) {
  const bool pow2 = M >= 2 && (M & (M - 1)) == 0;
  if (kind == 0 || kind == 3) return pow2 && M >= 16 && M <= 256;
  if (kind == 4 || kind == 6) return pow2 && M <= 8192;
  if (kind == 7) return !tc;
  if (kind == 8 || kind == 9) return !tc && pow2 && M >= 64 && M <= 2048;
  return pow2 && M >= 64 && M <= 1024 && kind >= 1 && kind <= 5;
}

}  // namespace

cudaError_t staged_prepare(int kind, int M, int Np, bool tc, int* smem, int* per_sm) {
  if (kind >= 10) return exact_prepare(kind, M, Np, tc, smem, per_sm);
  if (!valid(kind, M, tc)) return cudaErrorInvalidValue;
  if (kind == 7) {
    FusedSplit fs;
    if (!fused_split(M, Np, &fs)) return cudaErrorInvalidValue;
#define SCD_SFA_P(NPV, M1V, QV) \
    if (Np == NPV && fs.M1 == M1V && fs.Q == QV) return prep_sfa<NPV, M1V, QV>(smem, per_sm);
    SCD_SFA_SHAPES(SCD_SFA_P)
#undef SCD_SFA_P
    return cudaErrorInvalidValue;
  }
#define SCD_SP(MV) case MV: return tc ? prep_m<MV, true>(kind, smem, per_sm) : prep_m<MV, false>(kind, smem, per_sm);
  switch (M) {
    SCD_SP(2) SCD_SP(4) SCD_SP(8) SCD_SP(16) SCD_SP(32) SCD_SP(64) SCD_SP(128) SCD_SP(256) SCD_SP(512)
    SCD_SP(1024) SCD_SP(2048) SCD_SP(4096) SCD_SP(8192)
    default: return cudaErrorInvalidValue;
  }
#undef SCD_SP
}

cudaError_t staged_launch(int kind, int M, int Np, bool tc, int grid, int smem, const BatchArgs& A, const Task* tl,
                          int nt, int64_t total, cudaStream_t st) {
  if (kind >= 10) return exact_launch(kind, M, Np, tc, grid, smem, A, tl, nt, total, st);
  if (!valid(kind, M, tc)) return cudaErrorInvalidValue;
  if (kind == 7) {
    FusedSplit fs;
    if (!fused_split(M, Np, &fs)) return cudaErrorInvalidValue;
#define SCD_SFA_L(NPV, M1V, QV)                                                      \
    if (Np == NPV && fs.M1 == M1V && fs.Q == QV) {                                   \
      launch_sfa<NPV, M1V, QV>(grid, smem, A, tl, nt, total, st);                    \
      return cudaGetLastError();                                                     \
    }
    SCD_SFA_SHAPES(SCD_SFA_L)
#undef SCD_SFA_L
    return cudaErrorInvalidValue;
  }
#define SCD_SL(MV) case MV: if (tc) launch_m<MV, true>(kind, grid, smem, A, tl, nt, total, st); else launch_m<MV, false>(kind, grid, smem, A, tl, nt, total, st); break;
  switch (M) {
    SCD_SL(2) SCD_SL(4) SCD_SL(8) SCD_SL(16) SCD_SL(32) SCD_SL(64) SCD_SL(128) SCD_SL(256) SCD_SL(512)
    SCD_SL(1024) SCD_SL(2048) SCD_SL(4096) SCD_SL(8192)
    default: return cudaErrorInvalidValue;
  }
#undef SCD_SL
  return cudaGetLastError();
}

}  // namespace bk
}  // namespace scd
