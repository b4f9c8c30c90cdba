// Split-precision tensor-core form of the batched FFT (fft.cuh): every radix-R DFT of every
// Stockham pass is a complex-as-real GEMM on the 5th-generation tensor cores,
//     [Yr Yi](row) = [Xr Xi](row) * B_R,   B_R[2j + c'][2r + c] from W_R^{j r},
// with rows = butterflies (one per thread per butterfly), K = N = 2R (padded to >= 16).
// Operands are split into bf16 hi = rn(v) and lo = rn(v - hi); the FP32 accumulator in TMEM
// receives A_hi B_hi + A_hi B_lo + A_lo B_hi.  Twiddles between passes, the producers and the
// consumers stay in FP32 on the CUDA cores exactly as in the FP32 form.
//
// Per pass: threads gather and twiddle their butterflies' inputs, write their rows of the
// A tiles (hi and lo) to shared memory in the canonical K-major layout (aliasing the exchange
// buffer, whose reads are complete by then), one thread issues the MMAs (M = 128 rows per
// tile, tiles side by side in TMEM columns) and commits them to an mbarrier, every thread
// waits (bounded) and reads its rows back from TMEM.
#pragma once
#include "fft.cuh"
#include "umma.cuh"

namespace scd {

__host__ __device__ constexpr int tc_kp(int R) { return 2 * R < 16 ? 16 : 2 * R; }
// bytes of one DFT matrix (hi or lo) for radix R
__host__ __device__ constexpr int tc_bmat_bytes(int R) { return tc_kp(R) * tc_kp(R) * 2; }

template <int M, int THREADS>
struct TcPlan {
  using PI = PlanInfo<M>;
  static_assert(THREADS % 128 == 0, "tensor-core FFT needs a multiple of 128 threads");
  // TMEM columns and A-tile bytes of pass s
  static constexpr int tiles(int s) { return THREADS * (PI::E / PI::R(s)) / 128; }
  static constexpr int cols(int s) { return tiles(s) * tc_kp(PI::R(s)); }
  static constexpr int abytes(int s) { return tiles(s) * 2 * 128 * tc_kp(PI::R(s)) * 2; }
  static constexpr int max3(int a, int b, int c) { return a > b ? (a > c ? a : c) : (b > c ? b : c); }
  static constexpr int max_cols() {
    return max3(cols(0), PI::n > 1 ? cols(1) : 0, PI::n > 2 ? cols(2) : 0);
  }
  static constexpr int tmem_cols() {
    int c = 32;
    while (c < max_cols()) c <<= 1;
    return c;
  }
  static constexpr int max_abytes() {
    return max3(abytes(0), PI::n > 1 ? abytes(1) : 0, PI::n > 2 ? abytes(2) : 0);
  }
  // B-matrix slot of pass s: passes with the same radix share one (slot 0 = radix r0)
  static constexpr int bslot(int s) {
    return s == 0 ? 0 : (s == 1 ? (PI::r1 == PI::r0 ? 0 : 1)
                                : (PI::r2 == PI::r0 ? 0 : (PI::r2 == PI::r1 ? bslot(1) : 2)));
  }
  static constexpr int slot_bytes(int R) { return 2 * tc_bmat_bytes(R); }      // hi + lo
  static constexpr int boff(int slot) {
    return slot == 0 ? 0 : (slot == 1 ? slot_bytes(PI::r0) : slot_bytes(PI::r0) + (PI::n > 1 && bslot(1) == 1 ? slot_bytes(PI::r1) : 0));
  }
  static constexpr int bmat_bytes_total() {
    return slot_bytes(PI::r0) + (PI::n > 1 && bslot(1) == 1 ? slot_bytes(PI::r1) : 0) +
           (PI::n > 2 && bslot(2) == 2 ? slot_bytes(PI::r2) : 0);
  }
};

// Per-CTA tensor-core state (lives in registers; the pointed-to words live in shared memory).
struct TcCtx {
  uint64_t* mbar;
  uint32_t tmem;          // TMEM base address (lane 0, first allocated column)
  uint32_t phase;         // parity of the mbarrier phase to wait for next
  unsigned* err;          // device error word (set on a wait that timed out)
  const unsigned char* bsm;  // B matrices in shared memory
  bool ok;
};

constexpr uint32_t kMbarPollLimit = 1u << 24;

// Kernel prologue: mbarrier init and TMEM allocation (warp 0).  `slot` points at 16 bytes
// of shared memory (mbarrier + TMEM address word).
template <int NCOLS>
__device__ __forceinline__ TcCtx tc_open(unsigned char* slot, unsigned* err) {
  uint64_t* mbar = reinterpret_cast<uint64_t*>(slot);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(slot + 8);
  if (threadIdx.x == 0) umma::mbar_init(mbar, 1);
  if (threadIdx.x < 32) {
    umma::tmem_alloc(tslot, NCOLS);
    umma::tmem_relinquish();
  }
  umma::fence_before_sync();
  __syncthreads();
  umma::fence_after_sync();
  TcCtx c;
  c.mbar = mbar;
  c.tmem = *tslot;
  c.phase = 0;
  c.err = err;
  c.bsm = nullptr;
  c.ok = true;
  return c;
}

// Copies the B matrices of the transform size about to run into shared memory.
__device__ __forceinline__ void tc_load_b(TcCtx& c, unsigned char* bsm, const unsigned char* bglobal, int bbytes) {
  __syncthreads();                                             // no MMA of the previous tile reads bsm
  for (int i = threadIdx.x * 16; i < bbytes; i += blockDim.x * 16)
    *reinterpret_cast<uint4*>(bsm + i) = *reinterpret_cast<const uint4*>(bglobal + i);
  umma::fence_proxy_async();
  __syncthreads();
  c.bsm = bsm;
}

template <int NCOLS>
__device__ __forceinline__ TcCtx tc_begin(unsigned char* slot, unsigned char* bsm, const unsigned char* bglobal,
                                          int bbytes, unsigned* err) {
  TcCtx c = tc_open<NCOLS>(slot, err);
  tc_load_b(c, bsm, bglobal, bbytes);
  return c;
}

template <int NCOLS>
__device__ __forceinline__ void tc_end(TcCtx& c) {
  umma::fence_before_sync();
  __syncthreads();
  if (threadIdx.x < 32) {
    umma::fence_after_sync();
    umma::tmem_dealloc(c.tmem, NCOLS);
  }
  if (threadIdx.x == 0) umma::mbar_inval(c.mbar);
}

// One tensor-core DFT step for the B = E/R butterflies each thread holds in v[b*R + r]:
// rows (b * THREADS + tid) of tiles in `abuf`, result back into v.
template <int R, int E, int THREADS>
__device__ __forceinline__ void tc_dft(float2* v, unsigned char* abuf, const unsigned char* bmat, TcCtx& c) {
  constexpr int Kp = tc_kp(R), B = E / R;
  constexpr int TILE = 2 * 128 * Kp * 2;                      // hi + lo bytes of a 128-row tile
  constexpr int TILES = THREADS * B / 128;
  const int tid = threadIdx.x;
  // ---- rows of A (hi, lo)
#pragma unroll
  for (int b = 0; b < B; ++b) {
    const int row = b * THREADS + tid;
    unsigned char* hi = abuf + (row >> 7) * TILE;
    unsigned char* lo = hi + TILE / 2;
    const int m = row & 127;
#pragma unroll
    for (int kc = 0; kc < Kp / 8; ++kc) {                    // 16-byte chunks of 4 complex values
      uint32_t h[4], l[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int r = kc * 4 + q;
        if (r < R) umma::split2(v[b * R + r].x, v[b * R + r].y, h[q], l[q]);
        else { h[q] = 0u; l[q] = 0u; }
      }
      const uint32_t off = umma::kmajor_offset(m, kc * 8, Kp);
      *reinterpret_cast<uint4*>(hi + off) = make_uint4(h[0], h[1], h[2], h[3]);
      *reinterpret_cast<uint4*>(lo + off) = make_uint4(l[0], l[1], l[2], l[3]);
    }
  }
  umma::fence_proxy_async();
  umma::fence_before_sync();
  __syncthreads();
  // ---- MMAs (one thread)
  if (tid == 0) {
    umma::fence_after_sync();
    constexpr uint32_t idesc = umma::idesc_bf16_f32(128, Kp);
    const uint32_t sbo = Kp * 16;
    const uint32_t bhi = umma::smem_u32(bmat), blo = bhi + Kp * Kp * 2;
#pragma unroll
    for (int t = 0; t < TILES; ++t) {
      const uint32_t ahi = umma::smem_u32(abuf + t * TILE), alo = ahi + TILE / 2;
      const uint32_t d = c.tmem + t * Kp;
#pragma unroll
      for (int ks = 0; ks < Kp / 16; ++ks) {
        const uint32_t ko = ks * 256;                          // two core matrices along K
        umma::mma_bf16(d, umma::smem_desc(ahi + ko, 128, sbo), umma::smem_desc(bhi + ko, 128, sbo), idesc, ks > 0);
        umma::mma_bf16(d, umma::smem_desc(ahi + ko, 128, sbo), umma::smem_desc(blo + ko, 128, sbo), idesc, true);
        umma::mma_bf16(d, umma::smem_desc(alo + ko, 128, sbo), umma::smem_desc(bhi + ko, 128, sbo), idesc, true);
      }
    }
    umma::mma_commit(c.mbar);
  }
  // ---- wait (bounded) and read the rows back
  if (!umma::mbar_wait_bounded(c.mbar, c.phase, kMbarPollLimit)) {
    if (c.err) atomicOr(c.err, 1u);
    c.ok = false;
    umma::mbar_wait_bounded(c.mbar, c.phase, kMbarPollLimit);  // let the MMAs drain before going on
  }
  c.phase ^= 1u;
  umma::fence_after_sync();
  const uint32_t lane_base = (uint32_t)(32 * ((tid >> 5) & 3)) << 16;
#pragma unroll
  for (int b = 0; b < B; ++b) {
    const int row = b * THREADS + tid;
    const uint32_t taddr = c.tmem + lane_base + (row >> 7) * Kp;
#pragma unroll
    for (int j0 = 0; j0 < 2 * R; j0 += 16) {
      float f[16];
      umma::tmem_ld<16>(taddr + j0, f);
      umma::tmem_ld_wait();
#pragma unroll
      for (int q = 0; q < 8; ++q)
        if (j0 / 2 + q < R) v[b * R + j0 / 2 + q] = make_float2(f[2 * q], f[2 * q + 1]);
    }
  }
  umma::fence_before_sync();
}

// Same contract as fft_batch (fft.cuh) with THREADS == blockDim.x, plus the tensor-core
// context; `sm` must hold max(C * stride(C) * 8, TcPlan::max_abytes()) bytes.
template <int M, int C, bool CFAST, bool SYNC_DST, int THREADS, class Src, class Dst>
__device__ __forceinline__ void fft_batch_tc(float2* __restrict__ sm, const float2* __restrict__ tw, Src& src,
                                             Dst& dst, TcCtx& ctx) {
  using PI = PlanInfo<M>;
  using F = FftPieces<M>;
  using TP = TcPlan<M, THREADS>;
  constexpr int E = PI::E, T = PI::T;
  static_assert(C * T == THREADS, "block shape");
  const int tid = threadIdx.x;
  const int c = CFAST ? (tid % C) : (tid / T);
  const int t = CFAST ? (tid / C) : (tid % T);
  float2* reg = sm + c * PI::stride(C);
  unsigned char* abuf = reinterpret_cast<unsigned char*>(sm);
  float2 v[E];
  // pass 0: inputs straight from the producer
#pragma unroll
  for (int r = 0; r < PI::r0; ++r) v[r] = src(c, t + r * (M / PI::r0));
  __syncthreads();                                             // earlier users of sm are done
  tc_dft<PI::r0, E, THREADS>(v, abuf, ctx.bsm + TP::boff(TP::bslot(0)), ctx);
  if constexpr (PI::n == 1) {
    if constexpr (SYNC_DST) __syncthreads();
    F::template pass_out<0>(c, t, dst, v);
  } else {
    F::pass0_store(t, reg, v);
    __syncthreads();
    // pass 1: gather + twiddle exactly as the FP32 form, DFT on the tensor cores
    {
      constexpr int R = PI::r1, p = PI::p(1), B = E / R;
#pragma unroll
      for (int b = 0; b < B; ++b) {
        const int i = t + b * T;
        const int k = i & (p - 1);
#pragma unroll
        for (int r = 0; r < R; ++r) {
          float2 x = reg[PI::pad(i + r * (M / R))];
          if (r > 0) x = cmul(x, SCD_LDG(tw + PI::off(1) + r * p + k));
          v[b * R + r] = x;
        }
      }
    }
    __syncthreads();                                           // exchange reads done before A writes
    tc_dft<PI::r1, E, THREADS>(v, abuf, ctx.bsm + TP::boff(TP::bslot(1)), ctx);
    if constexpr (PI::n == 2) {
      if constexpr (SYNC_DST) __syncthreads();
      F::template pass_out<1>(c, t, dst, v);
    } else {
      __syncthreads();
      F::template pass_store<1>(t, reg, v);
      __syncthreads();
      {
        constexpr int R = PI::r2, p = PI::p(2), B = E / R;
#pragma unroll
        for (int b = 0; b < B; ++b) {
          const int i = t + b * T;
          const int k = i & (p - 1);
#pragma unroll
          for (int r = 0; r < R; ++r) {
            float2 x = reg[PI::pad(i + r * (M / R))];
            if (r > 0) x = cmul(x, SCD_LDG(tw + PI::off(2) + r * p + k));
            v[b * R + r] = x;
          }
        }
      }
      __syncthreads();
      tc_dft<PI::r2, E, THREADS>(v, abuf, ctx.bsm + TP::boff(TP::bslot(2)), ctx);
      if constexpr (SYNC_DST) __syncthreads();
      F::template pass_out<2>(c, t, dst, v);
    }
  }
}

// Shared-memory layout of a kernel that runs either form: region 0 (exchange buffer, A tiles
// of the tensor-core form, any staging of the consumer), then the B matrices, then 16 bytes
// for the mbarrier and the TMEM address.
template <int M, int THREADS, bool TC>
struct TcSizes {                                   // FP32 form: no tensor-core state
  static constexpr int abytes = 0, bbytes = 0, tmem_cols = 0;
};
template <int M, int THREADS>
struct TcSizes<M, THREADS, true> {
  static constexpr int abytes = TcPlan<M, THREADS>::max_abytes();
  static constexpr int bbytes = TcPlan<M, THREADS>::bmat_bytes_total();
  static constexpr int tmem_cols = TcPlan<M, THREADS>::tmem_cols();
};

template <int M, int C, int THREADS, bool TC, int EXTRA = 0>
struct FftSmem {
  static constexpr int up128(int v) { return (v + 127) / 128 * 128; }
  static constexpr int mx(int a, int b) { return a > b ? a : b; }
  static constexpr int exch = PlanInfo<M>::n == 1 ? 0 : C * PlanInfo<M>::stride(C) * 8;
  static constexpr int region0 = up128(mx(mx(exch, EXTRA), TcSizes<M, THREADS, TC>::abytes));
  static constexpr int bbytes = TcSizes<M, THREADS, TC>::bbytes;
  // (tensor-core form: 4 KB of slack after the descriptors' farthest reach)
  static constexpr int total = TC ? region0 + bbytes + 16 + 4096 : region0;
  static constexpr int tmem_cols = TcSizes<M, THREADS, TC>::tmem_cols;
};

// Runs one batch of C transforms in the form selected by TC (FP32 CUDA cores, or split bf16
// tensor cores with `bmats` (global, FftSmem::bbytes bytes) and the device error word).
template <int M, int C, bool CFAST, bool SYNC_DST, int THREADS, bool TC, int EXTRA, class Src, class Dst>
__device__ __forceinline__ void fft_run(float2* sm, const float2* __restrict__ tw, const unsigned char* bmats,
                                        unsigned* err, Src& src, Dst& dst) {
  if constexpr (TC) {
    using S = FftSmem<M, C, THREADS, true, EXTRA>;
    unsigned char* base = reinterpret_cast<unsigned char*>(sm);
    TcCtx ctx = tc_begin<S::tmem_cols>(base + S::region0 + S::bbytes, base + S::region0, bmats, S::bbytes, err);
    fft_batch_tc<M, C, CFAST, SYNC_DST, THREADS>(sm, tw, src, dst, ctx);
    tc_end<S::tmem_cols>(ctx);
  } else {
    fft_batch<M, C, CFAST, SYNC_DST>(sm, tw, src, dst);
  }
}

}  // namespace scd
