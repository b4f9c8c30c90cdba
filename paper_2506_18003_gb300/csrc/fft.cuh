// Batched power-of-two FFT building blocks for the SCD kernels (sm_103a).
//
// Every DFT on the hot path is a forward transform, X[f] = sum_n x[n] W_M^{f n} with
// W_M = exp(-i 2 pi / M).  A size-M transform is carried by a team of T threads that each
// hold E = M/T complex values in registers.  It runs as a short sequence of Stockham
// radix-R passes (R in {2..32}); the first pass reads straight from the producer (global
// memory or an on-the-fly product), the last pass hands each output straight to the
// consumer, and only the passes in between go through shared memory.
//
// Stockham recurrence used by every pass (decimation in time).  With p the product of the
// radices already applied, the array holds A_p[s, k] = sum_{t<p} x[s + t M/p] W_p^{k t} at
// index k + s p.  One radix-R pass turns A_p into A_{pR}:
//     A_{pR}[s, k + p j] = sum_{r<R} W_R^{j r} ( W_{pR}^{k r} A_p[s + r M/(pR), k] ),
// so butterfly i = k + s p (i < M/R) reads indices i + r M/R, scales them by W_{pR}^{k r},
// runs an R-point DFT and writes output j to index (i - k) R + k + p j.  After the last
// pass (pR = M) the output index is the natural frequency index.
//
// Twiddles W_{pR}^{k r} come from per-size tables built once in FP64 from exact integer
// indices (tables.cu); the radix-R butterflies use compile-time constants.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace scd {

// ----------------------------------------------------------------------------- complex
__host__ __device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
// The same sums with the packed two-lane FP32 instructions (add / sub .rn.f32x2): one
// instruction for both components, each lane rounded exactly like the scalar add, so the results
// are bit-identical.  Transforms opt in per call site (PK): it pays where the butterflies' adds
// bound the kernel (the FAM pair transform: batch 17.19 -> 16.68 ms) and costs where the
// register pairs it needs raise pressure (the fused SSCA's 1024-point second pass: +6%).
#if defined(__CUDA_ARCH__)
__device__ __forceinline__ unsigned long long f2_bits(float2 a) {
  return (unsigned long long)__float_as_uint(a.x) | ((unsigned long long)__float_as_uint(a.y) << 32);
}
__device__ __forceinline__ float2 f2_from(unsigned long long r) {
  return make_float2(__uint_as_float((unsigned)r), __uint_as_float((unsigned)(r >> 32)));
}
#endif
__host__ __device__ __forceinline__ float2 cadd_pk(float2 a, float2 b) {
#if defined(__CUDA_ARCH__)
  unsigned long long r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(f2_bits(a)), "l"(f2_bits(b)));
  return f2_from(r);
#else
  return cadd(a, b);
#endif
}
__host__ __device__ __forceinline__ float2 csub_pk(float2 a, float2 b) {
#if defined(__CUDA_ARCH__)
  unsigned long long r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(f2_bits(a)), "l"(f2_bits(b)));
  return f2_from(r);
#else
  return csub(a, b);
#endif
}
__host__ __device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// a * conj(b)
__host__ __device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
__host__ __device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__host__ __device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }

// ----------------------------------------------------------------------------- radix plans
// Radices of the Stockham passes for a size-M transform; the largest radix comes first,
// so p jumps from 1 straight to >= 8 and the shared-memory writes stay bank-friendly.
template <int M> struct Plan;
template <> struct Plan<2>     { static constexpr int n = 1; static constexpr int r[3] = {2, 0, 0}; };
template <> struct Plan<4>     { static constexpr int n = 1; static constexpr int r[3] = {4, 0, 0}; };
template <> struct Plan<8>     { static constexpr int n = 1; static constexpr int r[3] = {8, 0, 0}; };
template <> struct Plan<16>    { static constexpr int n = 1; static constexpr int r[3] = {16, 0, 0}; };
template <> struct Plan<32>    { static constexpr int n = 1; static constexpr int r[3] = {32, 0, 0}; };
template <> struct Plan<64>    { static constexpr int n = 2; static constexpr int r[3] = {8, 8, 0}; };
template <> struct Plan<128>   { static constexpr int n = 2; static constexpr int r[3] = {16, 8, 0}; };
template <> struct Plan<256>   { static constexpr int n = 2; static constexpr int r[3] = {16, 16, 0}; };
template <> struct Plan<512>   { static constexpr int n = 2; static constexpr int r[3] = {32, 16, 0}; };
template <> struct Plan<1024>  { static constexpr int n = 2; static constexpr int r[3] = {32, 32, 0}; };
template <> struct Plan<2048>  { static constexpr int n = 3; static constexpr int r[3] = {16, 16, 8}; };
template <> struct Plan<4096>  { static constexpr int n = 3; static constexpr int r[3] = {16, 16, 16}; };
template <> struct Plan<8192>  { static constexpr int n = 3; static constexpr int r[3] = {32, 16, 16}; };
template <> struct Plan<16384> { static constexpr int n = 3; static constexpr int r[3] = {32, 32, 16}; };

template <int M> struct PlanInfo {
  static constexpr int n = Plan<M>::n;
  static constexpr int r0 = Plan<M>::r[0], r1 = Plan<M>::r[1], r2 = Plan<M>::r[2];
  static constexpr int E = r0;            // values per thread (largest radix first)
  static constexpr int T = M / E;         // threads per transform
  // product of radices before pass s
  static constexpr int p(int s) { return s == 0 ? 1 : (s == 1 ? r0 : r0 * r1); }
  static constexpr int R(int s) { return s == 0 ? r0 : (s == 1 ? r1 : r2); }
  // offset of pass s (s >= 1) in the concatenated pass-twiddle table; entry (r, k) of pass
  // s sits at off(s) + r p(s) + k and holds W_{p R}^{k r}
  static constexpr int off(int s) { return s <= 1 ? 0 : r0 * r1; }
  static constexpr int tw_len() { return n == 1 ? 1 : (n == 2 ? r0 * r1 : r0 * r1 + r0 * r1 * r2); }
  // shared-memory position of exchange index i: one pad element after every r0 elements, so
  // that the 16 threads of a half-warp storing their r0 pass-0 outputs (index t r0 + j) hit
  // 16 different banks (odd stride r0 + 1), and consecutive indices stay consecutive
  static constexpr int lr0 = r0 >= 32 ? 5 : (r0 >= 16 ? 4 : (r0 >= 8 ? 3 : (r0 >= 4 ? 2 : 1)));
  __host__ __device__ static constexpr int pad(int i) { return i + (i >> lr0); }
  // shared-memory stride (complex elements) of one of C transforms laid side by side: the
  // 16 lanes of a half-warp touch min(C, 16) transforms at 16 / min(C, 16) consecutive
  // positions each, so the stride is 1 mod 16 for C >= 16 and 16 / C mod 16 below (M + M/r0 is
  // a multiple of 16 whenever C < 16), which puts every lane in its own bank
  static constexpr int stride(int C) { return M + M / r0 + (C >= 16 ? 1 : 16 / C); }
};

// ----------------------------------------------------------------------------- radix-R DFT
// W_32^j for j < 16 (cos, -sin), double literals rounded to float at compile time.
struct W32 {
  static constexpr float c[16] = {1.0f, 0.98078528040323043f, 0.92387953251128674f, 0.83146961230254524f, 0.70710678118654757f, 0.55557023301960229f, 0.38268343236508984f, 0.19509032201612833f, 0.0f, -0.19509032201612819f, -0.38268343236508973f, -0.55557023301960196f, -0.70710678118654746f, -0.83146961230254535f, -0.92387953251128674f, -0.98078528040323043f};
  static constexpr float s[16] = {0.0f, -0.19509032201612825f, -0.38268343236508978f, -0.55557023301960218f, -0.70710678118654746f, -0.83146961230254524f, -0.92387953251128674f, -0.98078528040323043f, -1.0f, -0.98078528040323043f, -0.92387953251128674f, -0.83146961230254546f, -0.70710678118654757f, -0.55557023301960218f, -0.38268343236508989f, -0.19509032201612861f};
};

// d * W_{L}^{j}, L <= 32, with the trivial factors (1, -i, (+-1 - i)/sqrt2) special-cased
template <int L, int J>
__host__ __device__ __forceinline__ float2 twc(float2 d) {
  constexpr int q = J * (32 / L);          // W_L^J = W_32^q, q < 16
  if constexpr (q == 0) {
    return d;
  } else if constexpr (q == 8) {           // -i
    return make_float2(d.y, -d.x);
  } else if constexpr (q == 4) {           // (1 - i)/sqrt2
    constexpr float h = 0.70710678118654752f;
    return make_float2((d.x + d.y) * h, (d.y - d.x) * h);
  } else if constexpr (q == 12) {          // (-1 - i)/sqrt2
    constexpr float h = 0.70710678118654752f;
    return make_float2((d.y - d.x) * h, -(d.x + d.y) * h);
  } else {
    constexpr float c = W32::c[q], s = W32::s[q];
    return make_float2(fmaf(d.x, c, -d.y * s), fmaf(d.x, s, d.y * c));
  }
}

template <int R, int SPAN, int START, int J, bool PK>
__host__ __device__ __forceinline__ void dif_bfly(float2* v) {
  if constexpr (J < SPAN) {
    float2 a = v[START + J], b = v[START + J + SPAN];
    v[START + J] = PK ? cadd_pk(a, b) : cadd(a, b);
    v[START + J + SPAN] = twc<2 * SPAN, J>(PK ? csub_pk(a, b) : csub(a, b));
    dif_bfly<R, SPAN, START, J + 1, PK>(v);
  }
}
template <int R, int SPAN, int START, bool PK>
__host__ __device__ __forceinline__ void dif_stage(float2* v) {
  if constexpr (START < R) {
    dif_bfly<R, SPAN, START, 0, PK>(v);
    dif_stage<R, SPAN, START + 2 * SPAN, PK>(v);
  }
}
template <int R, int SPAN, bool PK>
__host__ __device__ __forceinline__ void dif_all(float2* v) {
  if constexpr (SPAN >= 1) {
    dif_stage<R, SPAN, 0, PK>(v);
    dif_all<R, SPAN / 2, PK>(v);
  }
}
__host__ __device__ constexpr int bitrev(int i, int R) {
  int r = 0;
  for (int b = 1; b < R; b <<= 1) { r = (r << 1) | (i & 1); i >>= 1; }
  return r;
}
template <int R, int I>
__host__ __device__ __forceinline__ void unscramble(float2* v) {
  if constexpr (I < R) {
    constexpr int J = bitrev(I, R);
    if constexpr (J > I) { float2 t = v[I]; v[I] = v[J]; v[J] = t; }
    unscramble<R, I + 1>(v);
  }
}
// In-register R-point forward DFT, natural order in and out (radix-2 DIF network).
template <int R, bool PK = false>
__host__ __device__ __forceinline__ void dft(float2* v) {
  if constexpr (R > 1) {
    dif_all<R, R / 2, PK>(v);
    unscramble<R, 0>(v);
  }
}

// ----------------------------------------------------------------------------- pass pieces
#ifdef __CUDA_ARCH__
#define SCD_LDG(p) __ldg(p)
#else
#define SCD_LDG(p) (*(p))
#endif

// Index of entry e of the concatenated pass-twiddle table of a size-M plan with radices
// (r0, r1, r2): entry off(s) + r p + k holds W_M^{k r M/(p R)} (k < p, r < R).
__host__ __device__ inline int64_t pass_twiddle_exponent(int e, int M, int r0, int r1, int r2) {
  const int n1 = r0 * r1;
  int p, R, loc;
  if (e < n1) { p = r0; R = r1; loc = e; }
  else        { p = r0 * r1; R = r2; loc = e - n1; }
  const int r = loc / p, k = loc % p;
  return (int64_t)k * r * (M / (p * R));
}

// Per-thread pieces of the batched transform; registers v[] persist between pieces and
// the caller separates the pieces that touch shared memory with barriers.  PK: the radix DFTs'
// complex sums with the packed two-lane instructions (bit-identical results).
template <int M, bool PK = false>
struct FftPieces {
  using PI = PlanInfo<M>;
  static constexpr int E = PI::E, T = PI::T;

  // pass 0: E inputs of thread t straight from the producer, then an R0-point DFT
  template <class Src>
  __host__ __device__ __forceinline__ static void pass0_load(int c, int t, Src& src, float2* v) {
    constexpr int R = PI::r0;
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = src(c, t + r * (M / R));
    dft<R, PK>(v);
  }
  // pass 0 outputs of thread t to shared memory (A_{r0}[t, j] at j + t r0)
  __host__ __device__ __forceinline__ static void pass0_store(int t, float2* reg, const float2* v) {
    constexpr int R = PI::r0;
#pragma unroll
    for (int j = 0; j < R; ++j) reg[PI::pad(t * R + j)] = v[j];
  }
  // pass S >= 1: load from shared memory with twiddles and run the DFTs (TWS: the twiddle
  // table is a copy in shared memory, read with plain loads instead of the read-only path)
  template <int S, bool TWS = false>
  __host__ __device__ __forceinline__ static void pass_load(int t, const float2* reg, const float2* tw, float2* v) {
    constexpr int R = PI::R(S), p = PI::p(S), B = E / R;
#pragma unroll
    for (int b = 0; b < B; ++b) {
      const int i = t + b * T;
      const int k = i & (p - 1);
#pragma unroll
      for (int r = 0; r < R; ++r) {
        float2 x = reg[PI::pad(i + r * (M / R))];
        if (r > 0) x = cmul(x, TWS ? tw[PI::off(S) + r * p + k] : SCD_LDG(tw + PI::off(S) + r * p + k));
        v[b * R + r] = x;
      }
      dft<R, PK>(v + b * R);
    }
  }
  // pass S outputs to shared memory (not the last pass)
  template <int S>
  __host__ __device__ __forceinline__ static void pass_store(int t, float2* reg, const float2* v) {
    constexpr int R = PI::R(S), p = PI::p(S), B = E / R;
#pragma unroll
    for (int b = 0; b < B; ++b) {
      const int i = t + b * T;
      const int k = i & (p - 1);
#pragma unroll
      for (int j = 0; j < R; ++j) reg[PI::pad((i - k) * R + k + p * j)] = v[b * R + j];
    }
  }
  // outputs of the last pass S to the consumer (bin f in natural order)
  template <int S, class Dst>
  __host__ __device__ __forceinline__ static void pass_out(int c, int t, Dst& dst, const float2* v) {
    constexpr int R = PI::R(S), p = PI::p(S), B = E / R;
#pragma unroll
    for (int b = 0; b < B; ++b) {
      const int i = t + b * T;
      const int k = i & (p - 1);
#pragma unroll
      for (int j = 0; j < R; ++j) dst(c, (i - k) * R + k + p * j, v[b * R + j]);
    }
  }
};

// ----------------------------------------------------------------------------- team barrier
// Barrier among the T threads of one transform.  With consecutive threads per transform
// (!CFAST) a transform of at most 32 threads lives inside one warp (__syncwarp), a larger one
// occupies whole warps and uses its own named barrier (1 + team index; 0 is __syncthreads),
// so transforms of one CTA do not wait for each other.  Interleaved transforms (CFAST) span
// every warp and use the CTA barrier.
template <int T, bool CFAST>
__device__ __forceinline__ void team_sync() {
  if constexpr (CFAST) {
    __syncthreads();
  } else if constexpr (T <= 32) {
    __syncwarp();
  } else {
    if (T >= (int)blockDim.x) {
      __syncthreads();
    } else {
      asm volatile("bar.sync %0, %1;" :: "r"(1 + (int)threadIdx.x / T), "r"(T) : "memory");
    }
  }
}

// ----------------------------------------------------------------------------- batched FFT
// C transforms of size M per CTA, T = M/E threads each (blockDim.x == C*T).
// CFAST: thread tid works on transform c = tid % C (transforms interleaved across lanes,
// good when consecutive transforms touch consecutive addresses); otherwise c = tid / T
// (a transform's threads are consecutive).  `sm` holds C regions of PlanInfo<M>::stride(C)
// complex values; `tw` is the concatenated pass-twiddle table for size M.
//   src(c, idx)      -> float2   input idx of transform c (idx in [0, M))
//   dst(c, f, value)             output bin f (natural order) of transform c
// SYNC_DST: put a CTA barrier between the last pass's shared-memory reads and the dst
// calls, for consumers that stage outputs in the same shared memory.  Callers that loop
// over several batches must also barrier between batches.
template <int M, int C, bool CFAST, bool SYNC_DST, bool PK = false, class Src, class Dst>
__device__ __forceinline__ void fft_batch(float2* __restrict__ sm, const float2* __restrict__ tw,
                                          Src& src, Dst& dst) {
  using PI = PlanInfo<M>;
  using F = FftPieces<M, PK>;
  constexpr int E = PI::E, T = PI::T;
  const int tid = threadIdx.x;
  const int c = CFAST ? (tid % C) : (tid / T);
  const int t = CFAST ? (tid / C) : (tid % T);
  float2* reg = sm + c * PI::stride(C);
  float2 v[E];
  F::pass0_load(c, t, src, v);
  if constexpr (PI::n == 1) {
    F::template pass_out<0>(c, t, dst, v);
  } else {
    F::pass0_store(t, reg, v);
    team_sync<T, CFAST>();
    F::template pass_load<1>(t, reg, tw, v);
    if constexpr (PI::n == 2) {
      if constexpr (SYNC_DST) __syncthreads();
      F::template pass_out<1>(c, t, dst, v);
    } else {
      team_sync<T, CFAST>();               // every read of pass 1 precedes its writes
      F::template pass_store<1>(t, reg, v);
      team_sync<T, CFAST>();
      F::template pass_load<2>(t, reg, tw, v);
      if constexpr (SYNC_DST) __syncthreads();
      F::template pass_out<2>(c, t, dst, v);
    }
  }
}

// fft_batch with the pass-0 inputs already in registers: v[r] holds input t + r (M / r0) of
// this thread's transform (the layout pass0_load gathers), for producers whose per-thread state
// (coefficients held across several batches) does not fit the src(c, idx) form.  Same barriers
// and dst contract as fft_batch; XSTRIDE > 0 sets the exchange stride of one transform (complex
// values), otherwise PlanInfo<M>::stride(C).  With t-fast transforms of 8 threads (4 per warp)
// the conflict-free stride is M + M / r0 (8 mod 16: the two transforms of a half-warp then fill
// complementary banks in both the pass-0 stores and the pass-1 loads), where stride(C) costs two
// wavefronts per access.
template <int M, int C, bool CFAST, bool SYNC_DST, int XSTRIDE = 0, bool TWS = false, class Dst>
__device__ __forceinline__ void fft_batch_from(float2* __restrict__ sm, const float2* __restrict__ tw,
                                               float2 (&v)[PlanInfo<M>::E], Dst& dst) {
  using PI = PlanInfo<M>;
  using F = FftPieces<M>;
  constexpr int T = PI::T;
  const int tid = threadIdx.x;
  const int c = CFAST ? (tid % C) : (tid / T);
  const int t = CFAST ? (tid / C) : (tid % T);
  float2* reg = sm + c * (XSTRIDE > 0 ? XSTRIDE : PI::stride(C));
  dft<PI::r0>(v);
  if constexpr (PI::n == 1) {
    F::template pass_out<0>(c, t, dst, v);
  } else {
    F::pass0_store(t, reg, v);
    team_sync<T, CFAST>();
    F::template pass_load<1, TWS>(t, reg, tw, v);
    if constexpr (PI::n == 2) {
      if constexpr (SYNC_DST) __syncthreads();
      F::template pass_out<1>(c, t, dst, v);
    } else {
      team_sync<T, CFAST>();
      F::template pass_store<1>(t, reg, v);
      team_sync<T, CFAST>();
      F::template pass_load<2, TWS>(t, reg, tw, v);
      if constexpr (SYNC_DST) __syncthreads();
      F::template pass_out<2>(c, t, dst, v);
    }
  }
}

// Invokes F::template run<M>() for a runtime power-of-two M in [2, 16384].
#define SCD_DISPATCH_POW2(M_RUNTIME, CALL)                     \
  switch (M_RUNTIME) {                                          \
    case 2: CALL(2); break;                                     \
    case 4: CALL(4); break;                                     \
    case 8: CALL(8); break;                                     \
    case 16: CALL(16); break;                                   \
    case 32: CALL(32); break;                                   \
    case 64: CALL(64); break;                                   \
    case 128: CALL(128); break;                                 \
    case 256: CALL(256); break;                                 \
    case 512: CALL(512); break;                                 \
    case 1024: CALL(1024); break;                               \
    case 2048: CALL(2048); break;                               \
    case 4096: CALL(4096); break;                               \
    case 8192: CALL(8192); break;                               \
    case 16384: CALL(16384); break;                             \
    default: return SCD_ERR_UNSUPPORTED;                        \
  }

}  // namespace scd
