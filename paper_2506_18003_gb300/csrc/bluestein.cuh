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
// four-step FFTs of size M = M1 M2 through global memory, as the power-of-two strip transform).
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
template <int MM, bool TC>
__device__ __forceinline__ void fam_pairs_any_tile(float2* sm, TcCtx& ctx, const float2* __restrict__ X,
                                                   const float2* __restrict__ Y, int Np, int P,
                                                   float2* __restrict__ out, const float2* __restrict__ tw,
                                                   const float2* __restrict__ chirp, const float2* __restrict__ bh,
                                                   int64_t pair0) {
  using S = TileShape<MM>;
  using PI = PlanInfo<MM>;
  const int c = (int)threadIdx.x / S::T;
  const int64_t pair = pair0 + c;
  const bool valid = pair < (int64_t)Np * Np;
  const int kh = valid ? (int)(pair / Np) : 0, lh = valid ? (int)(pair % Np) : 0;
  const float2* __restrict__ xk = X + (int64_t)kh * P;
  const float2* __restrict__ xl = Y + (int64_t)lh * P;
  float2* __restrict__ o = out + pair * P;
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
      const int qh = f + half < P ? f + half : f + half - P;
      o[qh] = cmulc(__ldg(chirp + f), v);
    }
  };
  fft_resident<MM, S::C, S::NT, TC>(sm, tw, ctx, dst2);
}

// ---------------------------------------------------------------- SSCA strip transform, any N
// Column pass of a size-M = M1 M2 four-step transform (n = m1 M2 + m2) over one channel row
// `in` whose first `nvalid` values are given (row stride >= nvalid; zero beyond): M1-point DFT
// over m1 for the tile's columns m20 .. m20 + C - 1, times W_M^{(m2 m1') mod M}, to `out` at
// [m1'][m2] (row of M values).  wM = W_M^j, cols = W_M^{c m1'} at [m1'][c].
template <int M1, bool TC>
__device__ __forceinline__ void bl_cols_tile(float2* sm, TcCtx& ctx, const float2* __restrict__ in, int64_t nvalid,
                                             float2* __restrict__ out, int M, int M2, const float2* __restrict__ wM,
                                             const float2* __restrict__ cols, const float2* __restrict__ tw, int m20) {
  using S = TileShape<M1>;
  constexpr int C = S::C;
  const int c = (int)threadIdx.x % C;                            // interleaved columns: c = tid % C
  const int m2 = m20 + c;
  float2* ob = out + m2;
  const float2* __restrict__ colc = cols + c;
  auto src = [&](int, int m1) -> float2 {
    const int64_t n = (int64_t)m1 * M2 + m2;
    return n < nvalid ? __ldg(in + n) : make_float2(0.f, 0.f);
  };
  auto dst = [&](int, int f, float2 v) {
    const float2 w = cmul(__ldg(wM + ((m20 * f) & (M - 1))), __ldg(colc + f * C));   // W_M^{(m20+c) f}
    ob[(int64_t)f * M2] = cmul(v, w);
  };
  tile_fft<M1, C, true, false, S::NT, TC>(sm, tw, ctx, src, dst);
}

// Row pass of the same transform: rows r0 .. r0 + C - 1 of `in` ([m1'][m2]), M2-point DFT over
// m2, bin q = m1' + M1 m2' (natural order), transposed through shared memory so that the C
// rows' results leave as runs of C consecutive bins.
//   FINAL = false: out[q] = conj(G[q] Bh[q])                  (q < M, the first transform)
//   FINAL = true:  out[(q + N/2) mod N] = c[q] conj(G[q])     (q < N, the strip transform's bins)
template <int M2, bool TC, bool FINAL>
__device__ __forceinline__ void bl_rows_tile(float2* sm, TcCtx& ctx, const float2* __restrict__ in,
                                             float2* __restrict__ out, int M1, int64_t N,
                                             const float2* __restrict__ tw, const float2* __restrict__ lut, int r0) {
  using S = TileShape<M2>;
  constexpr int C = S::C;
  const float2* __restrict__ rowp = in + (int64_t)(r0 + (int)threadIdx.x / S::T) * M2;   // t-fast
  auto src = [&](int, int m2) -> float2 { return __ldg(rowp + m2); };
  auto dst = [&](int c, int f, float2 v) { sm[f * (C + 1) + c] = v; };
  tile_fft<M2, C, false, true, S::NT, TC>(sm, tw, ctx, src, dst);
  __syncthreads();
  const int64_t half = N / 2;
  for (int e = threadIdx.x; e < C * M2; e += blockDim.x) {
    const int c = e % C, f = e / C;
    const int64_t q = r0 + c + (int64_t)M1 * f;
    const float2 g = sm[f * (C + 1) + c];
    if constexpr (FINAL) {
      if (q < N) {
        const int64_t sh = q + half < N ? q + half : q + half - N;
        out[sh] = cmulc(__ldg(lut + q), g);
      }
    } else {
      out[q] = cconj(cmul(g, __ldg(lut + q)));
    }
  }
}

}  // namespace scd
