// SSCA with the channel-data product formed on chip: the hop-1 channeliser, the product with
// conj(y[n]) (Sec. II-C, Eq. Xg) and the first pass of the strip transform (Sec. III-B-1,
// Stage 1) run in one tile, so X_g never goes to global memory.
//
// The strip transform is the four-step split of Eq. II.B-SSCA_auto with N = M1 M2,
// n = m1 M2 + m2 and q = q1 + M1 q2:
//     S(k, q) = sum_{m2} W_M2^{q2 m2} [ W_N^{q1 m2} sum_{m1} X_g(m1 M2 + m2, k) W_M1^{q1 m1} ].
// Tile A (ssca_chancol_tile) owns one column m2: the M1 time points n = m1 M2 + m2 (their
// windows lie M2 >= Np samples apart) and all Np channels.  The block X_g(m1 M2 + m2, k) of
// Np x M1 values is held in shared memory, split over a cluster of Q CTAs: CTA q channelises the
// time points m1 in [q M1/Q, (q + 1) M1/Q) (full Np-point transforms), multiplies by conj(y[n])
// and stores each channel's value into the shared memory of the CTA that owns that channel
// (kh in [q' Np/Q, (q' + 1) Np/Q), distributed shared memory); after a cluster barrier every CTA
// runs the M1-point DFTs over m1 of its own channels, multiplies by the rotate factor
// W_N^{q1 m2} and writes Y.  A channel row of Y holds N values in blocks of C = the second
// pass's transforms per tile: Y[kh][q1 / C][m2][q1 mod C] (yf_index), so tile A writes runs of C
// values and tile B reads one contiguous block.
// Tile B (ssca_rowsf_tile) runs the M2-point DFTs over m2 for the C consecutive q1 of one block
// of one channel (consecutive lanes on consecutive q1: every warp load is a contiguous run) and
// stores bin q = q1 + M1 q2 fftshifted at sh = q1 + M1 ((q2 + M2/2) mod M2) (runs of C values).
// Global traffic: x (L2-resident) in, Y out and back, S out: 3 x 8 Np N bytes instead of the
// 5 x 8 Np N of the three-stage schedule (X_g written, column pass in place, row pass).
#pragma once
#include <cooperative_groups.h>

#include "tiles.cuh"

namespace scd {

// The fused split of an SSCA strip transform, or false where the tiles do not fit:
// M1 = max(64, N / 2048) (so M2 <= 2048 fits the second pass's tile: 1024 threads, 8 columns, at
// M2 = 2048), Q = Np M1 / 8192 CTAs per cluster (the block X_g(., k) takes 64 KB of shared memory
// per CTA, two CTAs per SM), and the windows of one tile >= Np samples apart (M2 >= Np: every
// time point of the tile then sees the same rotation s mod Np).  Tile shapes (Np, M1, Q):
// (64, 64..128, 1), (64, 256, 2), (128, 64, 1), (128, 128, 2), (128, 256, 4), (256, 64, 2),
// (256, 128, 4).  (M1 = 64 up to N = 2^17: the 64-point column pass costs less per point than a
// 128-point one in a cluster, batch SSCA 20.80 -> 20.39 ms against M2 <= 1024.)
struct FusedSplit {
  int M1, M2, Q;
};
inline bool fused_split(int64_t N, int Np, FusedSplit* s) {
  if (N < 4096 || N > (int64_t(1) << 20) || (N & (N - 1))) return false;
  if (Np != 64 && Np != 128 && Np != 256) return false;
  int64_t M1 = N / 2048 > 64 ? N / 2048 : 64;
  if (M1 > 256) return false;
  const int64_t Q = Np * M1 / 8192 > 1 ? Np * M1 / 8192 : 1;
  if (Q > 4) return false;
  const int64_t M2 = N / M1;
  if (M2 < Np || M2 > 2048) return false;
  s->M1 = (int)M1;
  s->M2 = (int)M2;
  s->Q = (int)Q;
  return true;
}

// Position of (m2, q1) in a channel row of Y: blocks of C consecutive q1, C = TileShape<M2>::C.
__host__ __device__ __forceinline__ int64_t yf_index(int m2, int q1, int M2, int C) {
  return (int64_t)(q1 / C) * M2 * C + (int64_t)m2 * C + (q1 % C);
}
// threads of a second-pass CTA (1024 at M2 = 2048, one CTA per SM, so that a tile still holds 8
// columns: tile A then writes Y in 64-byte runs, tile B writes S in 64-byte runs; 4 columns on
// 512 threads measured 1.1% slower on the batch SSCA) and transforms per tile for a runtime M2
__host__ __device__ constexpr int rowsf_threads(int M2) { return M2 >= 2048 ? 1024 : 256; }
__host__ __device__ constexpr int rowsf_c(int M2) {
  return M2 >= 1024 ? 8 : (M2 >= 256 ? 16 : 32);
}

// t-fast transforms (a transform's threads consecutive, at most 32 of them): exchange stride
// M + M / r0 per transform (fft_batch_from)
template <int M>
__host__ __device__ constexpr int tfast_stride() { return M + M / PlanInfo<M>::r0; }

// Shared-memory layout of tile A: the FFT exchange area (shared by the channeliser's and the
// column pass's transforms, which run one after the other), the CTA's X_g block Xs[kappa][m1]
// (G = Np / Q channels; row stride M1 + 8 and an XOR swizzle of m1, so that both the
// channeliser's stores and the column pass's loads are free of bank conflicts), and the
// tile's M1 rotate factors.
template <int NP, int M1, int Q>
struct ChanColSmem {
  static constexpr int G = NP / Q;
  static constexpr int up128(int v) { return (v + 127) / 128 * 128; }
  static constexpr int mx(int a, int b) { return a > b ? a : b; }
  static constexpr int exch =
      up128(mx(TileShape<NP>::C * tfast_stride<NP>() * 8, TileShape<M1>::C * tfast_stride<M1>() * 8));
  static constexpr int SX = M1 + 8;
  static constexpr int xs_off = exch;
  static constexpr int rot_off = xs_off + up128(G * SX * 8);
  // the tile's rotated window, and the pass twiddles of both transform sizes, staged once
  static constexpr int win_off = rot_off + up128(M1 * 8);
  static constexpr int twn_off = win_off + up128(NP * 4);
  static constexpr int twm_off = twn_off + up128(PlanInfo<NP>::tw_len() * 8);
  static constexpr int total = twm_off + up128(PlanInfo<M1>::tw_len() * 8);
};

// Position of X_g(m1, channel kappa) in a CTA's block.  The swizzle depends on how many threads
// carry one channeliser transform (8: Np <= 128, 16: Np = 256), whose last pass stores
// consecutive channels from consecutive threads.
template <int TG>
__device__ __forceinline__ int xs_pos(int kappa, int m1, int SX) {
  return kappa * SX + (m1 ^ (TG == 8 ? ((kappa >> 1) & 3) << 1 : (kappa >> 1) & 7));
}

__device__ __forceinline__ void cluster_arrive_relaxed() {
  asm volatile("barrier.cluster.arrive.relaxed.aligned;" ::: "memory");
}
__device__ __forceinline__ void cluster_arrive_release() {
  asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
}
__device__ __forceinline__ void cluster_wait_acquire() {
  asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// Tile A: column m2, one signal; this CTA is rank q of a cluster of Q.
//   x, y, conj : the signal and the channel-data product's second factor (as ssca_cdp_tile)
//   a          : window, Np floats;  tw_np, tw_m1: pass twiddles of sizes Np and M1
//   wN         : W_N^j (j < N)
//   Y          : the signal's Np x N intermediate, channel rows of N values
template <int NP, int M1, int Q>
__device__ __forceinline__ void ssca_chancol_tile(float2* sm, const float2* __restrict__ x, const float2* __restrict__ y,
                                                  bool conj, int N, int M2, const float* __restrict__ a,
                                                  const float2* __restrict__ tw_np, const float2* __restrict__ tw_m1,
                                                  const float2* __restrict__ wN, float2* __restrict__ Y, int m2, int q) {
  using Lay = ChanColSmem<NP, M1, Q>;
  constexpr int G = Lay::G, MQ = M1 / Q;
  using PG = PlanInfo<NP>;
  using PM = PlanInfo<M1>;
  constexpr int CA = TileShape<NP>::C, CB = TileShape<M1>::C;
  constexpr int EG = PG::E, TG = PG::T, TM = PM::T;
  static_assert(CA * TG == 256 && CB * TM == 256 && MQ % CA == 0 && G % CB == 0, "tile shape");
  static_assert(TG <= 32 && TM <= 32, "transforms synchronise within their warp");
  unsigned char* base = reinterpret_cast<unsigned char*>(sm);
  float2* xs = reinterpret_cast<float2*>(base + Lay::xs_off);
  float2* rot = reinterpret_cast<float2*>(base + Lay::rot_off);
  float* win = reinterpret_cast<float*>(base + Lay::win_off);
  float2* twn = reinterpret_cast<float2*>(base + Lay::twn_off);
  float2* twm = reinterpret_cast<float2*>(base + Lay::twm_off);
  const int tid = threadIdx.x;
  const int CY = rowsf_c(M2);                           // Y's column blocks (yf_index)
  const int lcy = CY == 4 ? 2 : (CY == 8 ? 3 : (CY == 16 ? 4 : 5));
  const int smod = (m2 - NP / 2) & (NP - 1);            // s mod Np for every m1 (Np divides M2)
  if constexpr (Q > 1) cluster_arrive_relaxed();        // every CTA of the cluster has started ...
  for (int i = tid; i < M1; i += 256) rot[i] = __ldg(wN + (((int64_t)i * m2) & (N - 1)));   // W_N^{q1 m2}
  for (int j = tid; j < NP; j += 256) win[j] = __ldg(a + ((j - smod) & (NP - 1)));         // a[rho] at input j
  for (int i = tid; i < PlanInfo<NP>::tw_len(); i += 256) twn[i] = __ldg(tw_np + i);
  for (int i = tid; i < PlanInfo<M1>::tw_len(); i += 256) twm[i] = __ldg(tw_m1 + i);
  __syncthreads();

  // ---- channeliser + CDP: batches of CA time points (transforms t-fast: c = tid / TG); the
  // samples of the next batch are loaded while this batch is transformed
  {
    const int c = tid / TG, t = tid % TG;
    constexpr int NB = MQ / CA;
    // FFT input j = t + i TG takes the sample rho - Np/2 after n, rho = (j - smod) mod Np
    auto load = [&](int bt, float2 (&xv)[EG]) {
      const int m1 = q * MQ + bt * CA + c;
      const int n = m1 * M2 + m2;
      // only the first and the last time point of a column have window samples outside [0, N)
      const bool edge = m1 == 0 || m1 == M1 - 1;
#pragma unroll
      for (int i = 0; i < EG; ++i) {
        const int idx = n + ((t + i * TG - smod) & (NP - 1)) - NP / 2;
        xv[i] = (!edge || (idx >= 0 && idx < N)) ? __ldg(x + (edge ? max(0, min(idx, N - 1)) : idx))
                                                 : make_float2(0.f, 0.f);
      }
    };
    float2 xnext[EG];
    load(0, xnext);
    if constexpr (Q > 1) cluster_wait_acquire();       // ... before any store into a peer's block
#pragma unroll 1
    for (int bt = 0; bt < NB; ++bt) {
      const int m1 = q * MQ + bt * CA + c;
      const int n = m1 * M2 + m2;
      float2 v[EG];
#pragma unroll
      for (int i = 0; i < EG; ++i) v[i] = cscale(xnext[i], win[t + i * TG]);
      float2 yn = __ldg(y + n);                         // the factor is conj(yn)
      if (bt + 1 < NB) load(bt + 1, xnext);
      if (conj) yn.y = -yn.y;
      auto dst = [&](int, int f, float2 val) {
        const int kh = (f + NP / 2) & (NP - 1);
        float2* p = xs + xs_pos<TG>(kh % G, m1, Lay::SX);
        if constexpr (Q > 1) p = cooperative_groups::this_cluster().map_shared_rank(p, (unsigned)(kh / G));
        *p = cmulc(val, yn);
      };
      fft_batch_from<NP, CA, false, false, tfast_stride<NP>(), true>(sm, twn, v, dst);
      __syncwarp();                                     // this warp's exchange reads precede the next batch's writes
    }
  }
  if constexpr (Q > 1) {
    cluster_arrive_release();                           // the cluster's blocks and rotate factors are complete
    cluster_wait_acquire();
  } else {
    __syncthreads();
  }

  // ---- column pass: M1-point DFTs over m1 of this CTA's G channels, times W_N^{q1 m2}
  {
    const int c = tid / TM, t = tid % TM;
    for (int bt = 0; bt < G / CB; ++bt) {
      const int kappa = bt * CB + c;
      const int kh = q * G + kappa;
      float2* __restrict__ yo = Y + (int64_t)kh * N + (int64_t)m2 * CY;
      float2 v[PM::E];
#pragma unroll
      for (int i = 0; i < PM::E; ++i) v[i] = xs[xs_pos<TG>(kappa, t + i * TM, Lay::SX)];
      auto dst = [&](int, int q1, float2 val) { yo[(int64_t)(q1 >> lcy) * M2 * CY + (q1 & (CY - 1))] = cmul(val, rot[q1]); };
      fft_batch_from<M1, CB, false, false, tfast_stride<M1>(), true>(sm, twm, v, dst);
      __syncwarp();
    }
  }
}

// Tile B: the q1 in [q10, q10 + C) of one channel, q10 a multiple of C: Yk = that channel's
// row of Y (yf_index), outk = its output row (N values, fftshifted).
// PROF: instead of storing S, every bin is reduced into the alpha profile prof[ah_off + sh]
// (ah_off = k N/Np + N/2 for channel k) by profile_max of |S|^power (as ssca_rows_tile).
template <int M2, bool PROF = false>
__device__ __forceinline__ void ssca_rowsf_tile(float2* sm, const float2* __restrict__ Yk, float2* __restrict__ outk,
                                                int M1, const float2* __restrict__ tw_m2, int q10,
                                                float* prof = nullptr, int ah_off = 0, int power = 1) {
  using S = TileShape<M2, rowsf_threads(M2)>;
  constexpr int C = S::C;
  static_assert(C == rowsf_c(M2), "Y's column blocks are the second pass's tiles");
  const int c = (int)threadIdx.x % C;                   // interleaved: consecutive lanes, consecutive q1
  const float2* __restrict__ ib = Yk + (int64_t)q10 * M2 + c;
  auto src = [&](int, int m2) -> float2 { return ib[m2 * C]; };
  if constexpr (PROF) {
    unsigned* __restrict__ pr = reinterpret_cast<unsigned*>(prof) + ah_off + q10 + c;
    auto dst = [&](int, int q2, float2 v) {
      const float m2 = fmaf(v.x, v.x, v.y * v.y);
      profile_max(pr + M1 * ((q2 + M2 / 2) & (M2 - 1)), __float_as_uint(power == 2 ? m2 : sqrtf(m2)));
    };
    fft_batch<M2, C, true, false>(sm, tw_m2, src, dst);
  } else {
    float2* __restrict__ ob = outk + q10 + c;
    auto dst = [&](int, int q2, float2 v) { ob[(int64_t)M1 * ((q2 + M2 / 2) & (M2 - 1))] = v; };
    fft_batch<M2, C, true, false>(sm, tw_m2, src, dst);
  }
}

}  // namespace scd
