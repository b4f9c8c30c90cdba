// Tile functions: one CTA's share of each stage of the estimators, callable from the
// standalone kernels (one tile per CTA) and from the persistent batch kernel (tiles pulled
// from a device work queue).  Every tile function runs with THREADS = blockDim.x threads
// and C = THREADS / T transforms, in the FP32 form or (TC) the split tensor-core form.
#pragma once
#include "fft_tc.cuh"

namespace scd {

// Transforms of size M handled by one CTA of THREADS threads.
template <int M, int THREADS = 256>
struct TileShape {
  static constexpr int T = PlanInfo<M>::T;
  static constexpr int C = T >= THREADS ? 1 : THREADS / T;
  static constexpr int NT = C * T;                      // threads actually used
};

// prof[i] = max(prof[i], v) for a non-negative float given by its bits (non-negative floats
// order like their bit patterns); a fire-and-forget reduction in L2.  (Reading the current
// value first and skipping the atomic when v cannot raise it measured slower: the dependent
// load sits on every thread's path.)
__device__ __forceinline__ void profile_max(unsigned* p, unsigned v) { atomicMax(p, v); }

// Runs the C transforms of one tile in the requested form; for TC the caller has opened the
// tensor-core context and loaded the B matrices of size M into ctx.bsm.
template <int M, int C, bool CFAST, bool SYNC_DST, int THREADS, bool TC, bool PK = false, class Src, class Dst>
__device__ __forceinline__ void tile_fft(float2* sm, const float2* __restrict__ tw, TcCtx& ctx, Src& src, Dst& dst) {
  if constexpr (TC) fft_batch_tc<M, C, CFAST, SYNC_DST, THREADS>(sm, tw, src, dst, ctx);
  else fft_batch<M, C, CFAST, SYNC_DST, PK>(sm, tw, src, dst);
}

// ---------------------------------------------------------------- FAM channeliser (K1)
// frames p0 .. p0 + C - 1:  X[kh][p] = W_Np^{(k p L) mod Np} sum_n a[n] x[pL+n] W_Np^{(k n) mod Np}
// The down-conversion costs nothing: the windowed sample a[n] x[pL+n] is placed at FFT input
// position (pL + n) mod Np, so the transform itself produces sum_n a[n] x[pL+n] W_Np^{k (pL+n)}.
// (conj_out: conj(X) is stored instead, the second operand of a conjugate estimate)
template <int NP, bool TC>
__device__ __forceinline__ void fam_channelise_tile(float2* sm, TcCtx& ctx, const float2* __restrict__ x, int L, int P,
                                                    const float* __restrict__ a, const float2* __restrict__ tw,
                                                    float2* __restrict__ X, int p0, bool conj_out = false) {
  using S = TileShape<NP>;
  auto src = [&](int c, int j) -> float2 {
    const int p = p0 + c;
    if (p >= P) return make_float2(0.f, 0.f);
    const int n = (j - (int)(((int64_t)p * L) & (NP - 1))) & (NP - 1);    // j = (pL + n) mod Np
    return cscale(__ldg(x + (int64_t)p * L + n), __ldg(a + n));
  };
  auto dst = [&](int c, int f, float2 v) {
    const int p = p0 + c;
    if (p >= P) return;
    if (conj_out) v.y = -v.y;
    X[(int64_t)((f + NP / 2) & (NP - 1)) * P + p] = v;
  };
  tile_fft<NP, S::C, true, false, S::NT, TC>(sm, tw, ctx, src, dst);
}

// ---------------------------------------------------------------- FAM pair FFT (K2)
// pairs pair0 .. pair0 + C - 1 (pair = kh Np + lh):
//   out[kh][lh][qh] = sum_p X[kh][p] conj(Y[lh][p]) W_P^{(q p) mod P}
// Y = X for the auto estimate, the partner's channeliser output for a cross estimate, and
// the conjugated one for a conjugate estimate.
// SYM (auto estimate, Y = X): the pair products are conjugate-symmetric, z_lk(p) = conj(z_kl(p)),
// so S(l, k, -q) = conj(S(k, l, q)) exactly; only the Np (Np + 1) / 2 pairs with kh <= lh are
// transformed and each writes both rows (the mirrored one at qh' = (P/2 - f) mod P for natural
// bin f).  The pairs are enumerated over a folded triangle: pair = r (Np + 1) + c, r < Np/2, is
// (r, r + c) for c < Np - r and (Np - 1 - r, c - 1) otherwise (rows r and Np - 1 - r of the
// triangle together hold Np + 1 pairs).
// PROF: instead of storing S, every kept bin (q in [-Q, Q)) is reduced into the alpha profile
// prof[ah], ah = (k - l) Q + q + P L, by profile_max of |S|^power.
template <int PP>
__host__ __device__ inline int64_t fam_pair_count(int Np, bool sym) {
  return sym ? (int64_t)Np * (Np + 1) / 2 : (int64_t)Np * Np;
}

template <int PP, bool TC, bool PROF = false, bool SYM = false>
__device__ __forceinline__ void fam_pairs_tile(float2* sm, TcCtx& ctx, const float2* __restrict__ X,
                                               const float2* __restrict__ Y, int Np, float2* __restrict__ out,
                                               const float2* __restrict__ tw, int64_t pair0, float* prof = nullptr,
                                               int PL = 0, int Q = 0, int power = 1) {
  using S = TileShape<PP>;
  // this thread's pair (transforms are t-fast: c = tid / T), resolved once
  const int64_t pair = pair0 + (int)threadIdx.x / S::T;
  const bool valid = pair < fam_pair_count<PP>(Np, SYM);
  int kh = 0, lh = 0;
  if (valid) {
    if constexpr (SYM) {
      const int r = (int)(pair / (Np + 1)), c = (int)(pair % (Np + 1));
      if (c < Np - r) { kh = r; lh = r + c; }
      else { kh = Np - 1 - r; lh = c - 1; }
    } else {
      kh = (int)(pair / Np);
      lh = (int)(pair % Np);
    }
  }
  const bool mirror = SYM && kh != lh;
  const float2* __restrict__ xk = X + (int64_t)kh * PP;
  const float2* __restrict__ xl = Y + (int64_t)lh * PP;
  float2* __restrict__ o = PROF ? nullptr : out + ((int64_t)kh * Np + lh) * PP;
  float2* __restrict__ om = PROF ? nullptr : out + ((int64_t)lh * Np + kh) * PP;
  auto src = [&](int, int p) -> float2 {
    return valid ? cmulc(__ldg(xk + p), __ldg(xl + p)) : make_float2(0.f, 0.f);
  };
  auto dst = [&](int, int f, float2 v) {
    if constexpr (PROF) {
      const int q = ((f + PP / 2) & (PP - 1)) - PP / 2;
      const float m2 = fmaf(v.x, v.x, v.y * v.y);
      const unsigned val = __float_as_uint(power == 2 ? m2 : sqrtf(m2));
      if (valid && q >= -Q && q < Q)
        profile_max(reinterpret_cast<unsigned*>(prof) + ((kh - lh) * Q + q + PL), val);
      if (mirror && -q >= -Q && -q < Q)                  // S(l, k, -q): the same magnitude
        profile_max(reinterpret_cast<unsigned*>(prof) + ((lh - kh) * Q - q + PL), val);
    } else {
      if (valid) o[(f + PP / 2) & (PP - 1)] = v;
      if (mirror) om[(PP / 2 - f) & (PP - 1)] = cconj(v);
    }
  };
  tile_fft<PP, S::C, false, false, S::NT, TC, true>(sm, tw, ctx, src, dst);   // packed sums (FP32 form)
}

// ---------------------------------------------------------------- SSCA channeliser + CDP (K3)
// time points n0 .. n0 + C - 1:  X_g[kh][n] = W_Np^{(k s) mod Np} DFT_Np(a x[s ..])[k] conj(y[n])
// (y = x for the auto estimate; conj: y[n] itself, the conjugate estimate).  As in K1 the
// down-conversion is the placement of a[r] x[s+r] at FFT input position (s + r) mod Np.
// The tile's C + Np - 1 input samples (zero outside [0, N)) and the window are staged in
// shared memory first (`stage`, cdp_stage_bytes<NP>() bytes, disjoint from the FFT's
// exchange and tensor-core buffers): the C transforms read the same samples at shifted
// window positions, so every lane of a half-warp then reads one broadcast word.
template <int NP>
__host__ __device__ constexpr int cdp_stage_bytes() { return (TileShape<NP>::C + NP) * 8 + NP * 4; }

// Layout of a CTA running K3 tiles: the FFT's exchange / tensor-core buffers, then the
// staging area at `off`, all inside region 0 (the split form's B matrices follow region 0).
template <int NP, bool TC>
struct CdpStage {
  static constexpr int off = FftSmem<NP, TileShape<NP>::C, TileShape<NP>::NT, TC>::region0;
  static constexpr int end = off + cdp_stage_bytes<NP>();
};
template <int NP, bool TC>
using CdpSmem = FftSmem<NP, TileShape<NP>::C, TileShape<NP>::NT, TC, CdpStage<NP, TC>::end>;

// ld: row stride of X_g (0: N; exact-length plans lay X_g out in rows of the cyclic length)
template <int NP, bool TC>
__device__ __forceinline__ void ssca_cdp_tile(float2* sm, TcCtx& ctx, const float2* __restrict__ x,
                                              const float2* __restrict__ y, bool conj, int N,
                                              const float* __restrict__ a, const float2* __restrict__ tw,
                                              float2* __restrict__ Xg, int n0, unsigned char* stage,
                                              int64_t ld = 0) {
  using S = TileShape<NP>;
  float2* xs = reinterpret_cast<float2*>(stage);
  float* as = reinterpret_cast<float*>(stage + (S::C + NP) * 8);
  for (int i = threadIdx.x; i < S::C + NP; i += blockDim.x) {
    const int m = n0 - NP / 2 + i;
    xs[i] = (m >= 0 && m < N) ? __ldg(x + m) : make_float2(0.f, 0.f);
  }
  for (int i = threadIdx.x; i < NP; i += blockDim.x) as[i] = __ldg(a + i);
  // this thread's time point (transforms interleaved: c = tid % C), resolved once
  const int c = (int)threadIdx.x % S::C;
  const int n = n0 + c;
  const int smod = (n - NP / 2) & (NP - 1);                         // window start mod Np
  float2 xn = __ldg(y + n);                                         // the factor is conj(xn)
  if (conj) xn.y = -xn.y;
  float2* __restrict__ o = Xg + n;
  __syncthreads();                                                  // staged samples visible
  auto src = [&](int, int j) -> float2 {
    const int r = (j - smod) & (NP - 1);                            // j = (s + r) mod Np
    return cscale(xs[c + r], as[r]);
  };
  const int64_t row = ld ? ld : N;
  auto dst = [&](int, int f, float2 v) { o[(int64_t)((f + NP / 2) & (NP - 1)) * row] = cmulc(v, xn); };
  tile_fft<NP, S::C, true, false, S::NT, TC>(sm, tw, ctx, src, dst);
}

// ---------------------------------------------------------------- SSCA column pass (K4a)
// channel row `in` (N values, viewed [m1][m2], n = m1 M2 + m2), columns m20 .. m20 + C - 1:
// M1-point DFT over m1, times the rotate factor W_N^{(m2 m1') mod N}, to `out` (may equal in)
// at [m1'][m2].  wN = W_N^j table, cols = W_N^{c m1'} at [m1'][c].
// DISCARD: the input (X_g) is dead once this tile has read it and `out` is another buffer:
// the tile's whole L2 lines of it are discarded so that they are never written back.
// FP32 form: the last pass hands thread (c, t) the bins f = i + p j (p = r0, the first radix;
// i in [0, p) one of the thread's B = r0/r1 residues, j < r1), so the rotate factor splits as
//     W_N^{(m20 + c) f} = W_N^{(m20 + c) i} * W_N^{(m20 + c) p j}:
// the first factor is gathered from the W_N table per thread (B values), the second is shared
// by the tile's C columns and r1 values of j (C r1 = 256, one per thread), gathered into shared
// memory (`stage`, [j][c], disjoint from the FFT's buffers) before the transform, whose
// barriers order it before the last pass reads it.  No per-bin table read remains.  The split
// form reads W_N^{m20 f} and W_N^{c f} from the tables directly: its larger layout would
// otherwise outgrow the shared-memory carveout that leaves two CTAs per SM a useful L1.
template <int M1, bool TC>
struct ColsStage {
  static constexpr int off = FftSmem<M1, TileShape<M1>::C, TileShape<M1>::NT, TC>::region0;
  static constexpr int end = off + (TC ? 0 : TileShape<M1>::C * PlanInfo<M1>::r1 * 8);
};
template <int M1, bool TC>
using ColsSmem = FftSmem<M1, TileShape<M1>::C, TileShape<M1>::NT, TC, ColsStage<M1, TC>::end>;

template <int M1, bool TC, bool DISCARD = false>
__device__ __forceinline__ void ssca_cols_tile(float2* sm, TcCtx& ctx, const float2* in, float2* out, int N, int M2,
                                               const float2* __restrict__ wN, const float2* __restrict__ cols,
                                               const float2* __restrict__ tw, int m20, float2* stage) {
  using S = TileShape<M1>;
  using PI = PlanInfo<M1>;
  constexpr int C = S::C;
  static_assert(PI::n == 2, "the staged factors rely on the transform's barrier; f = i + r0 j");
  const int c = (int)threadIdx.x % C;                             // interleaved columns: c = tid % C
  const float2* ib = in + m20 + c;
  float2* ob = out + m20 + c;
  auto src = [&](int, int m1) -> float2 { return ib[(int64_t)m1 * M2]; };
  if constexpr (TC) {
    const float2* __restrict__ colc = cols + c;
    auto dst = [&](int, int f, float2 v) {
      const float2 w = cmul(__ldg(wN + ((m20 * f) & (N - 1))), __ldg(colc + f * C));   // W_N^{(m20+c) f}
      ob[(int64_t)f * M2] = cmul(v, w);
    };
    tile_fft<M1, C, true, false, S::NT, TC>(sm, tw, ctx, src, dst);
  } else {
    constexpr int p = PI::r0, T = PI::T;
    static_assert(C * PI::r1 == S::NT && (p == T || p == 2 * T), "one staged factor per thread, B <= 2");
    const int64_t col = m20 + c;
    {                                                             // stage[j C + cc] = W_N^{(m20 + cc) p j}
      const int jj = (int)threadIdx.x / C, cc = (int)threadIdx.x % C;
      stage[threadIdx.x] = __ldg(wN + (((int64_t)(m20 + cc) * p * jj) & (N - 1)));
    }
    const int t = (int)threadIdx.x / C;
    const float2 a0 = __ldg(wN + ((col * t) & (N - 1)));          // W_N^{(m20 + c) i}, i = t, t + T
    const float2 a1 = p == 2 * T ? __ldg(wN + ((col * (t + T)) & (N - 1))) : a0;
    auto dst = [&](int, int f, float2 v) {
      const int i = f & (p - 1), j = f / p;
      const float2 w = cmul(i < T ? a0 : a1, stage[j * C + c]);   // W_N^{(m20+c) f}
      ob[(int64_t)f * M2] = cmul(v, w);
    };
    tile_fft<M1, C, true, false, S::NT, TC>(sm, tw, ctx, src, dst);
  }
  if constexpr (DISCARD && C * 8 % 128 == 0) {                   // the tile owns whole lines of each row
    __syncthreads();                                            // every read of the input is done
    constexpr int LPR = C * 8 / 128;                            // lines per row
    for (int l = threadIdx.x; l < M1 * LPR; l += blockDim.x) {
      const char* p = reinterpret_cast<const char*>(in + (int64_t)(l / LPR) * M2 + m20) + (l % LPR) * 128;
      asm volatile("discard.global.L2 [%0], 128;" :: "l"(p) : "memory");
    }
  }
}

// ---------------------------------------------------------------- SSCA row pass (K4b)
// rows r0 .. r0 + C - 1 of one channel (`in` = [m1'][m2]): M2-point DFT over m2, output bin
// q_nat = m1' + M1 m2' stored fftshifted at m1' + M1 ((m2' + M2/2) mod M2) of `out`; the
// strided output is transposed through shared memory into runs of C contiguous values.
template <int M2>
__host__ __device__ constexpr int rows_stage_bytes() { return M2 * (TileShape<M2>::C + 1) * 8; }

// SLOT: the input rows are a rotating slot of the persistent schedule, dead once read: their
// L2 lines are discarded (never written back), and the output is stored with the streaming
// hint so that it does not push the live slots out of L2.
// PROF: instead of storing S, every bin is reduced into the alpha profile prof[sh + ah_off]
// (ah_off = k N/Np + N/2 for channel k) by profile_max of |S|^power; the transposed order
// makes each warp's reads and reductions hit consecutive words.
template <int M2, bool TC, bool SLOT = false, bool PROF = false>
__device__ __forceinline__ void ssca_rows_tile(float2* sm, TcCtx& ctx, const float2* in, float2* __restrict__ out,
                                               int M1, const float2* __restrict__ tw, int r0, float* prof = nullptr,
                                               int ah_off = 0, int power = 1) {
  using S = TileShape<M2>;
  constexpr int C = S::C;
  const float2* __restrict__ rowp = in + (int64_t)(r0 + (int)threadIdx.x / S::T) * M2;   // t-fast: c = tid / T
  auto src = [&](int, int m2) -> float2 { return rowp[m2]; };
  auto dst = [&](int c, int f, float2 v) { sm[f * (C + 1) + c] = v; };
  tile_fft<M2, C, false, true, S::NT, TC>(sm, tw, ctx, src, dst);
  __syncthreads();
  if constexpr (SLOT) {                                        // C rows of M2 values, 128-byte aligned
    const char* base = reinterpret_cast<const char*>(in + (int64_t)r0 * M2);
    for (int l = threadIdx.x; l < C * M2 * 8 / 128; l += blockDim.x)
      asm volatile("discard.global.L2 [%0], 128;" :: "l"(base + (int64_t)l * 128) : "memory");
  }
  if constexpr (PROF) {
    unsigned* __restrict__ pr = reinterpret_cast<unsigned*>(prof) + ah_off + r0;
    for (int e = threadIdx.x; e < C * M2; e += blockDim.x) {
      const int c = e % C, f = e / C;
      const float2 v = sm[f * (C + 1) + c];
      const float m2 = fmaf(v.x, v.x, v.y * v.y);
      profile_max(pr + c + M1 * ((f + M2 / 2) & (M2 - 1)), __float_as_uint(power == 2 ? m2 : sqrtf(m2)));
    }
    return;
  }
  float2* __restrict__ o = out + r0;
  for (int e = threadIdx.x; e < C * M2; e += blockDim.x) {
    const int c = e % C, f = e / C;
    float2* dstp = o + c + (int64_t)M1 * ((f + M2 / 2) & (M2 - 1));
    if constexpr (SLOT) __stcs(dstp, sm[f * (C + 1) + c]);
    else *dstp = sm[f * (C + 1) + c];
  }
}

}  // namespace scd
