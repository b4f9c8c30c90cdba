// The persistent batch kernel, shared by batch.cu (full estimates) and batch_profile.cu
// (alpha profiles fused into the last stage): the task list, the kernel's arguments, its
// shared-memory layout and the kernel itself.  The scheduling is described in batch.cu.
#pragma once
#include "internal.h"
#include "tiles.cuh"

namespace scd {
namespace bk {

enum Op : int32_t { OP_FAM_CHAN = 0, OP_FAM_PAIRS = 1, OP_SSCA_CDP = 2, OP_SSCA_COLS = 3, OP_SSCA_ROWS = 4 };

struct Task {
  int32_t op, size, dep, bbytes;          // op, transform size, prerequisite task (-1), B bytes
  int32_t dep2, ch0;                      // second prerequisite (-1); SSCA: first channel of the unit
  int64_t first, tiles;                   // queue items [first, first + tiles)
  int64_t subtiles;                       // CTA tiles of the task; one queue item covers `per_item`
  int32_t per_item;
  int32_t in_ws;                          // exact-length SSCA: channeliser inputs at xp_off / yp_off of ws
  int64_t x_off, out_off, ws_off;         // element offsets into the arenas
  int64_t mid_off;                        // SSCA: workspace offset of the unit's column-pass slot
  int32_t N, P, M1, M2;                   // the signal's sizes
  const float2* tw;                       // pass twiddles of this task's transform size
  const float2* wN;                       // SSCA column pass: W_N^j
  const float2* cols;                     // SSCA column pass: W_N^{c m1'} at [m1'][c]
  const unsigned char* bmats;             // split form: B matrices of this size
  // exact-length plans (batch_exact.cu)
  int64_t xp_off, yp_off;                 // workspace offsets of the zero-padded channeliser inputs
  int64_t ld;                             // row stride of the channeliser's output (0: N)
                                          // (exact-length SSCA: t.P holds the padded length Npad_i)
  const float2* chirp;                    // Bluestein chirp c[j] of the signal's length
  const float2* bh;                       // Bluestein kernel spectrum (FAM: Bh; SSCA: row-ordered Bh)
};

struct BatchArgs {
  const Task* tasks;
  int32_t ntasks, Np, L;
  int32_t prof_power;                     // alpha-profile output (1: |S|, 2: |S|^2); 0: full estimates
  int32_t drop_task;                      // test-time fault injection: never publish this task (-1)
  int64_t total;                          // tiles in the whole plan
  unsigned* counters;                     // [0]: next tile, [1 + t]: tiles of task t done
  const float2* x;                        // x arena
  const float2* y;                        // SSCA: second factor's arena (x for the auto estimate)
  int32_t conj, pad_;                     // SSCA: 1 = conjugate estimate (y unconjugated)
  float2* out;                            // output arena
  float2* ws;                             // workspace arena
  const float* window;
  const float2* tw_np;                    // pass twiddles of size Np
  const unsigned char* bmats_np;          // split form: B matrices of size Np
  int32_t bbytes_np;
  unsigned* err;
};

constexpr int kThreads = 256;
constexpr int kSlots = 3;                                  // rotating column-pass slots (SSCA)
constexpr int64_t kSlotBytes = 16ll << 20;                 // target bytes of one slot
constexpr int64_t kItemBytes = 128ll << 10;                // output bytes per queue item (target)
constexpr int64_t kSlotBytesMax = 64ll << 20;              // largest slot the autotuner tries

// Channels per SSCA unit: the largest power of two G <= Np with G N 8 <= slot bytes.
inline int64_t slot_group(int Np, int64_t N, int64_t slot_bytes) {
  int64_t G = Np;
  while (G > 1 && G * N * 8 > slot_bytes) G >>= 1;
  return G;
}
constexpr unsigned long long kWaitNs = 2000000000ull;   // bound on any dependency wait

__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Shared-memory layout of the batch kernel: region 0 (largest over every size the estimator
// may meet), then (split form) the largest B-matrix set, the tensor-core slot and slack.
template <bool FAM, bool TC>
struct BatchSmem {
  template <int M, int EXTRA = 0>
  using FS = FftSmem<M, TileShape<M>::C, TileShape<M>::NT, TC, EXTRA>;
  static constexpr int mx(int a, int b) { return a > b ? a : b; }
  static constexpr int fam_r0() {
    return mx(mx(mx(FS<16>::region0, FS<32>::region0), mx(FS<64>::region0, FS<128>::region0)),
              mx(mx(FS<256>::region0, FS<512>::region0),
                 mx(mx(FS<1024>::region0, FS<2048>::region0), mx(FS<4096>::region0, FS<8192>::region0))));
  }
  static constexpr int fam_b() {
    return mx(mx(mx(FS<16>::bbytes, FS<32>::bbytes), mx(FS<64>::bbytes, FS<128>::bbytes)),
              mx(mx(FS<256>::bbytes, FS<512>::bbytes),
                 mx(mx(FS<1024>::bbytes, FS<2048>::bbytes), mx(FS<4096>::bbytes, FS<8192>::bbytes))));
  }
  static constexpr int cdp_r0() {
    return mx(mx(mx(CdpSmem<16, TC>::region0, CdpSmem<32, TC>::region0),
                 mx(mx(CdpSmem<64, TC>::region0, CdpSmem<128, TC>::region0), CdpSmem<256, TC>::region0)),
              mx(mx(mx(ColsSmem<64, TC>::region0, ColsSmem<128, TC>::region0), ColsSmem<256, TC>::region0),
                 mx(ColsSmem<512, TC>::region0, ColsSmem<1024, TC>::region0)));
  }
  static constexpr int ssca_r0() {
    return mx(cdp_r0(), mx(mx(mx(FS<16>::region0, FS<32>::region0), mx(FS<64>::region0, FS<128>::region0)),
              mx(mx(FS<256>::region0, FS<512>::region0),
                 mx(mx(FS<1024>::region0, FS<64, rows_stage_bytes<64>()>::region0),
                    mx(mx(FS<128, rows_stage_bytes<128>()>::region0, FS<256, rows_stage_bytes<256>()>::region0),
                       mx(FS<512, rows_stage_bytes<512>()>::region0, FS<1024, rows_stage_bytes<1024>()>::region0))))));
  }
  static constexpr int ssca_b() {
    return mx(mx(mx(FS<16>::bbytes, FS<32>::bbytes), mx(FS<64>::bbytes, FS<128>::bbytes)),
              mx(mx(FS<256>::bbytes, FS<512>::bbytes), FS<1024>::bbytes));
  }
  static constexpr int region0 = FAM ? fam_r0() : ssca_r0();
  static constexpr int bbytes = TC ? (FAM ? fam_b() : ssca_b()) : 0;
  static constexpr int total = TC ? region0 + bbytes + 16 + 4096 : region0;
  // TMEM columns: 256 threads, at most 32 values per thread, 2 fp32 columns per value
  static constexpr int tmem_cols = 128;
};

template <bool TC>
__device__ __forceinline__ void load_b(TcCtx& ctx, unsigned char* bsm, const unsigned char* bm, int bytes,
                                       const unsigned char*& loaded) {
  if constexpr (TC) {
    if (loaded != bm) {
      tc_load_b(ctx, bsm, bm, bytes);
      loaded = bm;
    }
  }
}

template <bool TC, bool PROF>
__device__ __forceinline__ void fam_tile(const BatchArgs& A, const Task& t, int64_t tile, float2* sm, TcCtx& ctx, unsigned char* bsm,
                         const unsigned char*& loaded) {
  const float2* x = A.x + t.x_off;
  float2* X = A.ws + t.ws_off;
  if (t.op == OP_FAM_CHAN) {
    load_b<TC>(ctx, bsm, A.bmats_np, A.bbytes_np, loaded);
    switch (A.Np) {
#define SCD_CH(NPV) case NPV: fam_channelise_tile<NPV, TC>(sm, ctx, x, A.L, t.P, A.window, A.tw_np, X, (int)tile * TileShape<NPV>::C); break;
      SCD_CH(16) SCD_CH(32) SCD_CH(64) SCD_CH(128) SCD_CH(256)
#undef SCD_CH
    }
  } else {
    load_b<TC>(ctx, bsm, t.bmats, t.bbytes, loaded);
    float2* out = PROF ? nullptr : A.out + t.out_off;
    float* prof = PROF ? reinterpret_cast<float*>(A.out) + t.out_off : nullptr;
    const int PL = t.P * A.L, Q = PL / A.Np;
    switch (t.P) {
#define SCD_PR(PV) case PV: fam_pairs_tile<PV, TC, PROF, true>(sm, ctx, X, X, A.Np, out, t.tw, tile * TileShape<PV>::C, prof, PL, Q, A.prof_power); break;
      SCD_PR(2) SCD_PR(4) SCD_PR(8) SCD_PR(16) SCD_PR(32) SCD_PR(64) SCD_PR(128) SCD_PR(256) SCD_PR(512)
      SCD_PR(1024) SCD_PR(2048) SCD_PR(4096) SCD_PR(8192)
#undef SCD_PR
    }
  }
}

template <bool TC, bool PROF>
__device__ __forceinline__ void ssca_tile(const BatchArgs& A, const Task& t, int64_t tile, float2* sm, TcCtx& ctx, unsigned char* bsm,
                          const unsigned char*& loaded) {
  const float2* x = A.x + t.x_off;
  float2* ws = A.ws + t.ws_off;
  if (t.op == OP_SSCA_CDP) {
    load_b<TC>(ctx, bsm, A.bmats_np, A.bbytes_np, loaded);
    switch (A.Np) {
#define SCD_CD(NPV) case NPV: ssca_cdp_tile<NPV, TC>(sm, ctx, x, A.y + t.x_off, A.conj != 0, t.N, A.window, A.tw_np, ws, (int)tile * TileShape<NPV>::C, reinterpret_cast<unsigned char*>(sm) + CdpStage<NPV, TC>::off); break;
      SCD_CD(16) SCD_CD(32) SCD_CD(64) SCD_CD(128) SCD_CD(256)
#undef SCD_CD
    }
  } else if (t.op == OP_SSCA_COLS) {
    // unit of channels [ch0, ch0 + G): X_g rows of the signal -> the unit's slot
    load_b<TC>(ctx, bsm, t.bmats, t.bbytes, loaded);
    switch (t.M1) {
#define SCD_CO(MV)                                                                          \
  case MV: {                                                                                \
    constexpr int C = TileShape<MV>::C;                                                     \
    const int per = t.M2 / C;                                                               \
    const int64_t kh = tile / per;                                                          \
    ssca_cols_tile<MV, TC, true>(sm, ctx, ws + (t.ch0 + kh) * t.N, A.ws + t.mid_off + kh * t.N, t.N, t.M2, t.wN, \
                           t.cols, t.tw, (int)(tile % per) * C,                             \
                           reinterpret_cast<float2*>(reinterpret_cast<unsigned char*>(sm) + ColsStage<MV, TC>::off)); \
  } break;
      SCD_CO(64) SCD_CO(128) SCD_CO(256) SCD_CO(512) SCD_CO(1024)
#undef SCD_CO
    }
  } else {
    load_b<TC>(ctx, bsm, t.bmats, t.bbytes, loaded);
    float2* out = PROF ? nullptr : A.out + t.out_off;
    float* prof = PROF ? reinterpret_cast<float*>(A.out) + t.out_off : nullptr;
    switch (t.M2) {
#define SCD_RO(MV)                                                                          \
  case MV: {                                                                                \
    constexpr int C = TileShape<MV>::C;                                                     \
    const int per = t.M1 / C;                                                               \
    const int64_t kh = tile / per;                                                          \
    /* alpha column of stored bin sh of channel k: ah = sh + k N/Np + N/2 */                \
    const int ah_off = (int)(t.ch0 + kh - A.Np / 2) * (t.N / A.Np) + t.N / 2;               \
    ssca_rows_tile<MV, TC, true, PROF>(sm, ctx, A.ws + t.mid_off + kh * t.N,                \
                                       PROF ? nullptr : out + (t.ch0 + kh) * t.N, t.M1, t.tw, \
                                       (int)(tile % per) * C, prof, ah_off, A.prof_power);  \
  } break;
      SCD_RO(64) SCD_RO(128) SCD_RO(256) SCD_RO(512) SCD_RO(1024)
#undef SCD_RO
    }
  }
}

template <bool FAM, bool TC, bool PROF>
__global__ void __launch_bounds__(kThreads, 2) k_batch(BatchArgs A) {
  extern __shared__ __align__(128) float2 sm[];
  __shared__ int64_t s_tile;
  __shared__ int s_task;
  __shared__ int s_skip;
  using BS = BatchSmem<FAM, TC>;
  unsigned char* base = reinterpret_cast<unsigned char*>(sm);
  TcCtx ctx{};
  unsigned char* bsm = base + BS::region0;
  if constexpr (TC) ctx = tc_open<BS::tmem_cols>(base + BS::region0 + BS::bbytes, A.err);
  const unsigned char* loaded = nullptr;
  // Scheduling state, kept by thread 0: the next tile index is claimed one tile ahead so the
  // atomic's latency overlaps the current tile; a CTA's tiles only increase, so the task is
  // found by scanning forward; a satisfied dependency is remembered per task.
  int64_t next = 0;
  int cur = 0, dep_ok_task = -1;
  if (threadIdx.x == 0) next = (int64_t)atomicAdd(A.counters, 1u);
  for (;;) {
    __syncthreads();                                         // previous tile fully done with smem
    if (threadIdx.x == 0) {
      const int64_t tile = next;
      s_tile = tile;
      int skip = 0;
      if (tile < A.total) {
        next = (int64_t)atomicAdd(A.counters, 1u);           // claim the following tile now
        while (cur + 1 < A.ntasks && __ldg(&A.tasks[cur + 1].first) <= tile) ++cur;
        if (dep_ok_task != cur) {
          const int deps[2] = {__ldg(&A.tasks[cur].dep), __ldg(&A.tasks[cur].dep2)};
          const unsigned long long t0 = globaltimer();
          for (int d = 0; d < 2 && !skip; ++d) {
            if (deps[d] < 0) continue;
            const unsigned need = (unsigned)__ldg(&A.tasks[deps[d]].tiles);
            while (ld_acquire(A.counters + 1 + deps[d]) < need) {
              if (globaltimer() - t0 > kWaitNs) {
                atomicOr(A.err, 2u);
                skip = 1;
                break;
              }
              __nanosleep(128);
            }
          }
          if (!skip) dep_ok_task = cur;
        }
      }
      s_task = cur;
      s_skip = skip;
    }
    __syncthreads();
    const int64_t tile = s_tile;
    if (tile >= A.total) break;
    const Task& t = A.tasks[s_task];
    if (!s_skip) {
      const int64_t s0 = (tile - t.first) * t.per_item;
      const int64_t s1 = s0 + t.per_item < t.subtiles ? s0 + t.per_item : t.subtiles;
      for (int64_t st = s0; st < s1; ++st) {
        if (st > s0) __syncthreads();                        // shared memory reused by the next tile
        if constexpr (FAM) fam_tile<TC, PROF>(A, t, st, sm, ctx, bsm, loaded);
        else ssca_tile<TC, PROF>(A, t, st, sm, ctx, bsm, loaded);
      }
    }
    __syncthreads();
    if (threadIdx.x == 0 && s_task != A.drop_task) {
      __threadfence();
      atomicAdd(A.counters + 1 + s_task, 1u);
    }
  }
  if constexpr (TC) tc_end<BS::tmem_cols>(ctx);
}

// Launchers: the full-estimate kernels (batch.cu) and the alpha-profile kernels
// (batch_profile.cu), each instantiated in its own translation unit.
int smem_of(bool fam, bool tc);
cudaError_t prepare_kernel(bool fam, bool tc, bool prof, int smem, int* blocks_per_sm);
cudaError_t launch_batch(bool fam, bool tc, bool prof, int grid, int smem, const BatchArgs& A, cudaStream_t st);
cudaError_t prepare_kernel_profile(bool fam, bool tc, int smem, int* blocks_per_sm);
cudaError_t launch_batch_profile(bool fam, bool tc, int grid, int smem, const BatchArgs& A, cudaStream_t st);
// Staged schedule (batch_staged.cu): kinds SSCA 0 channeliser + CDP (M = Np), 1 column pass
// (M = M1), 2 row pass (M = M2); FAM 3 channeliser (M = Np), 4 pair transforms (M = P); 5 / 6
// the row pass / pair transforms reducing into alpha profiles.  Each launch runs a task list
// whose tasks hold `first` and `subtiles` in CTA tiles; lists of kinds 1, 2, 4, 5 and 6 hold one
// size class.
// The task of CTA tile `tile` in a launch's task list: the last task whose first tile is <=
// tile (binary search; one CTA tile per CTA).
__device__ __forceinline__ int find_task(const Task* __restrict__ tl, int nt, int64_t tile) {
  int lo = 0, hi = nt - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(&tl[mid].first) <= tile) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

cudaError_t staged_prepare(int kind, int M, int Np, bool tc, int* smem, int* per_sm);
cudaError_t staged_launch(int kind, int M, int Np, bool tc, int grid, int smem, const BatchArgs& A, const Task* tl,
                          int nt, int64_t total, cudaStream_t st);
// The exact-length plans' own launch kinds (batch_exact.cu): 10 input preparation (chirp folded
// into the channel-data product's second factor, zero padding), 11 / 13 the two Bluestein
// column passes (M = M1), 12 the fused middle pass (M = M2), 14 the FAM pair transform of any
// P (M = the cyclic length MM).
cudaError_t exact_prepare(int kind, int M, int Np, bool tc, int* smem, int* per_sm);
int exact_prep_per_tile();                                   // values of one signal per kind-10 CTA
cudaError_t exact_launch(int kind, int M, int Np, bool tc, int grid, int smem, const BatchArgs& A, const Task* tl,
                         int nt, int64_t total, cudaStream_t st);

}  // namespace bk
}  // namespace scd
