// DFTs of any length on the power-of-two transforms: Bluestein's chirp-z identity
// (L. I. Bluestein, "A linear filtering approach to the computation of the discrete Fourier
// transform", 1970).  With qn = (q^2 + n^2 - (q - n)^2) / 2,
//     sum_{n<N} z[n] W_N^{q n} = c[q] sum_{n<N} (z[n] c[n]) conj(c[q - n]),   c[j] = W_{2N}^{j^2},
// a linear convolution of a = z c with conj(c) over lags (-N, N).  It is evaluated as a cyclic
// convolution of length M (a power of two, M >= 2N - 1) on the tensor-core / CUDA-core FFTs of
// fft.cuh and fft_tc.cuh:
//     G = FFT_M( conj( FFT_M(a) * Bh ) ),   Bh = FFT_M(bt) / M,
//     bt[j] = conj(c[j]) for j < N, conj(c[M - j]) for M - j < N, 0 otherwise,
//     sum_n z[n] W_N^{q n} = c[q] conj(G[q])          (q < N)
// (the inverse transform as the conjugate of a forward one).  c and Bh are tables built once in
// FP64 (tables.cu) and rounded to float.
//
// Two users: the FAM pair transform for any P (both FFTs inside one CTA, the intermediate in the
// transform's own shared-memory exchange region), and the SSCA strip transform for any N (two
// four-step FFTs of size M = M1 M2 through global memory whose row passes are fused).
#pragma once
#include "tiles.cuh"

namespace scd {

// Smallest power of two >= 2n - 1: the cyclic length that carries a length-n DFT.
__host__ __device__ inline int64_t bluestein_len(int64_t n) {
  int64_t m = 1;
  while (m < 2 * n - 1) m <<= 1;
  return m;
}

// A batch of C transforms of size M whose inputs already sit in each transform's shared-memory
// exchange region (element idx at PlanInfo<M>::pad(idx) of region c): every thread loads its
// pass-0 inputs before any thread of the transform overwrites the region.  t-fast layout
// (c = tid / T), as fft_batch with CFAST = false.
template <int M, int C, int THREADS, bool TC, class Dst>
__device__ __forceinline__ void fft_resident(float2* sm, const float2* __restrict__ tw, TcCtx& ctx, Dst& dst) {
  using PI = PlanInfo<M>;
  using F = FftPieces<M>;
  constexpr int E = PI::E, T = PI::T;
  const int c = (int)threadIdx.x / T, t = (int)threadIdx.x % T;
  float2* reg = sm + c * PI::stride(C);
  auto src = [&](int, int j) -> float2 { return reg[PI::pad(j)]; };
  if constexpr (TC) {
    // the tensor-core form reads every input into registers and passes a CTA barrier before
    // its first shared-memory write
    fft_batch_tc<M, C, false, false, THREADS>(sm, tw, src, dst, ctx);
  } else {
    float2 v[E];
    F::pass0_load(c, t, src, v);
    if constexpr (PI::n == 1) {
      F::template pass_out<0>(c, t, dst, v);
    } else {
      team_sync<T, false>();                                 // every load precedes the stores
      F::pass0_store(t, reg, v);
      team_sync<T, false>();
      F::template pass_load<1>(t, reg, tw, v);
      if constexpr (PI::n == 2) {
        F::template pass_out<1>(c, t, dst, v);
      } else {
        team_sync<T, false>();
        F::template pass_store<1>(t, reg, v);
        team_sync<T, false>();
        F::template pass_load<2>(t, reg, tw, v);
        F::template pass_out<2>(c, t, dst, v);
      }
    }
  }
}

// Shared-memory layout of a kernel running size-M transforms with the intermediate kept in
// the exchange regions (which therefore exist even for single-pass plans).
template <int M, bool TC>
using ResidentSmem = FftSmem<M, TileShape<M>::C, TileShape<M>::NT, TC, TileShape<M>::C * PlanInfo<M>::stride(TileShape<M>::C) * 8>;

// ---------------------------------------------------------------- FAM pair transform, any P
// pairs pair0 .. pair0 + C - 1 (pair = kh Np + lh), P < MM <= 2P - 1 rounded up to a power of 2:
//   out[kh][lh][qh] = sum_{p<P} X[kh][p] conj(Y[lh][p]) W_P^{(q p) mod P},  qh = (q + P/2) mod P
// (q in natural order; for odd P the zero bin is stored at floor(P/2)).  X and Y rows are P long.
// SYM (auto estimate, Y = X): the pairs kh <= lh only, each writing its row and the mirrored row
// S(l, k, -q) = conj S(k, l, q), as fam_pairs_tile (tiles.cuh).
template <int MM, bool TC, bool SYM = false>
__device__ __forceinline__ void fam_pairs_any_tile(float2* sm, TcCtx& ctx, const float2* __restrict__ X,
                                                   const float2* __restrict__ Y, int Np, int P,
                                                   float2* __restrict__ out, const float2* __restrict__ tw,
                                                   const float2* __restrict__ chirp, const float2* __restrict__ bh,
                                                   int64_t pair0) {
  using S = TileShape<MM>;
  using PI = PlanInfo<MM>;
  const int c = (int)threadIdx.x / S::T;
  const int64_t pair = pair0 + c;
  const bool valid = pair < (SYM ? (int64_t)Np * (Np + 1) / 2 : (int64_t)Np * Np);
  int kh = 0, lh = 0;
  if (valid) {
    if constexpr (SYM) {
      const int r = (int)(pair / (Np + 1)), cc = (int)(pair % (Np + 1));
      if (cc < Np - r) { kh = r; lh = r + cc; }
      else { kh = Np - 1 - r; lh = cc - 1; }
    } else {
      kh = (int)(pair / Np);
      lh = (int)(pair % Np);
    }
  }
  const bool mirror = SYM && valid && kh != lh;
  const float2* __restrict__ xk = X + (int64_t)kh * P;
  const float2* __restrict__ xl = Y + (int64_t)lh * P;
  float2* __restrict__ o = out + ((int64_t)kh * Np + lh) * P;
  float2* __restrict__ om = out + ((int64_t)lh * Np + kh) * P;
  float2* reg = sm + c * PI::stride(S::C);
  auto src1 = [&](int, int p) -> float2 {
    return (valid && p < P) ? cmul(cmulc(__ldg(xk + p), __ldg(xl + p)), __ldg(chirp + p)) : make_float2(0.f, 0.f);
  };
  auto dst1 = [&](int, int f, float2 v) { reg[PI::pad(f)] = cconj(cmul(v, __ldg(bh + f))); };
  tile_fft<MM, S::C, false, true, S::NT, TC>(sm, tw, ctx, src1, dst1);
  __syncthreads();
  const int half = P / 2;
  auto dst2 = [&](int, int f, float2 v) {
    if (valid && f < P) {
      const float2 s = cmulc(__ldg(chirp + f), v);
      const int qh = f + half < P ? f + half : f + half - P;
      o[qh] = s;
      if (mirror) {                                      // bin -q of the mirrored pair
        const int fm = f == 0 ? 0 : P - f;
        om[fm + half < P ? fm + half : fm + half - P] = cconj(s);
      }
    }
  };
  fft_resident<MM, S::C, S::NT, TC>(sm, tw, ctx, dst2);
}

// ---------------------------------------------------------------- SSCA strip transform, any N
// The cyclic convolution runs as two size-M four-step transforms (M = M1 M2) sharing their
// middle: with n = m1 M2 + m2, q = q1 + M1 q2 and j = j2 + M2 j1,
//   A[q1 + M1 q2] = sum_{m2} W_M2^{q2 m2} W_M^{q1 m2} sum_{m1} W_M1^{q1 m1} a[m1 M2 + m2]
//   G[j2 + M2 j1] = sum_{q1} W_M1^{j1 q1} W_M^{j2 q1} sum_{q2} W_M2^{j2 q2} B[q1 + M1 q2]
// so the first transform's row DFT (over m2 -> q2 in row q1), the product B = conj(A Bh) and
// the second transform's row DFT (over q2 -> j2 in the same row q1) all touch one row: they
// run as one pass, and the data crosses HBM three times instead of four.
//
// Column passes (interleaved columns m2 = m20 + c of one channel row, M1-point DFT over m1):
//   FINAL = false:  in = the X_g row, first `nvalid` values given (zero beyond);
//                   out[m1' M2 + m2] = W_M^{m2 m1'} DFT(...)[m1']
//   FINAL = true:   in = the middle pass's rows, input m1 taken times W_M^{m2 m1};
//                   G[j] at j = m2 + M2 m1' for j < N: out[(j + N/2) mod N] = c[j] conj(G[j])
// wM = W_M^j, cols = W_M^{c m1} at [m1][c], chirp = c[j].
template <int M1, bool TC, bool FINAL>
__device__ __forceinline__ void bl_cols_tile(float2* sm, TcCtx& ctx, const float2* __restrict__ in, int64_t nvalid,
                                             float2* __restrict__ out, int64_t M, int M2, int64_t N,
                                             const float2* __restrict__ wM, const float2* __restrict__ cols,
                                             const float2* __restrict__ chirp, const float2* __restrict__ tw,
                                             int m20) {
  using S = TileShape<M1>;
  constexpr int C = S::C;
  const int c = (int)threadIdx.x % C;                            // interleaved columns: c = tid % C
  const int m2 = m20 + c;
  const float2* __restrict__ colc = cols + c;
  // W_M^{(m20 + c) m1} = W_M^{m20 m1} W_M^{c m1}
  auto rot = [&](int m1) { return cmul(__ldg(wM + (((int64_t)m20 * m1) & (M - 1))), __ldg(colc + m1 * C)); };
  if constexpr (!FINAL) {
    float2* ob = out + m2;
    auto src = [&](int, int m1) -> float2 {
      const int64_t n = (int64_t)m1 * M2 + m2;
      return n < nvalid ? __ldg(in + n) : make_float2(0.f, 0.f);
    };
    auto dst = [&](int, int f, float2 v) { ob[(int64_t)f * M2] = cmul(v, rot(f)); };
    tile_fft<M1, C, true, false, S::NT, TC>(sm, tw, ctx, src, dst);
  } else {
    const int64_t half = N / 2;
    auto src = [&](int, int m1) -> float2 { return cmul(__ldg(in + (int64_t)m1 * M2 + m2), rot(m1)); };
    auto dst = [&](int, int f, float2 v) {
      const int64_t j = m2 + (int64_t)M2 * f;
      if (j < N) out[j + half < N ? j + half : j + half - N] = cmulc(__ldg(chirp + j), v);
    };
    tile_fft<M1, C, true, false, S::NT, TC>(sm, tw, ctx, src, dst);
  }
}

// Middle pass: rows r0 .. r0 + C - 1 of one channel (row q1 of [q1][m2], t-fast): M2-point
// DFT over m2 -> q2, times bhr[q1][q2] = Bh[q1 + M1 q2] and conjugated in the transform's
// shared-memory region, M2-point DFT over q2 -> j2, written back as row q1 of `out`.
template <int M2, bool TC>
__device__ __forceinline__ void bl_mid_tile(float2* sm, TcCtx& ctx, const float2* __restrict__ in,
                                            float2* __restrict__ out, const float2* __restrict__ tw,
                                            const float2* __restrict__ bhr, int r0) {
  using S = TileShape<M2>;
  using PI = PlanInfo<M2>;
  const int c = (int)threadIdx.x / S::T;
  const int64_t row = (int64_t)(r0 + c) * M2;
  const float2* __restrict__ rowp = in + row;
  const float2* __restrict__ bhp = bhr + row;
  float2* reg = sm + c * PI::stride(S::C);
  auto src1 = [&](int, int m2) -> float2 { return __ldg(rowp + m2); };
  auto dst1 = [&](int, int f, float2 v) { reg[PI::pad(f)] = cconj(cmul(v, __ldg(bhp + f))); };
  tile_fft<M2, S::C, false, true, S::NT, TC>(sm, tw, ctx, src1, dst1);
  __syncthreads();
  float2* __restrict__ orow = out + row;
  auto dst2 = [&](int, int f, float2 v) { orow[f] = v; };
  fft_resident<M2, S::C, S::NT, TC>(sm, tw, ctx, dst2);
}

}  // namespace scd
