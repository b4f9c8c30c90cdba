// SSCA column pass (K4a, Stage 1 of Sec. III-B-1, Eq. Chap4_2DFFT) with its input staged
// through TMA: the FP32 form for M1 = 1024 (the N = 2^20 strip transform).
//
// At M1 = 1024 a CTA's tile is C = 8 columns x 1024 rows, and with per-thread loads every warp
// load instruction touches four 64-byte pieces of four rows; the plain kernel waits on those
// loads (ncu: long-scoreboard stalls 4.0 per issued instruction, LSU throttling) and reaches
// 61% of the copy bandwidth.  Here two persistent CTAs per SM walk the tiles b, b + grid, ...;
// the tensor memory accelerator moves a tile (cp.async.bulk.tensor.3d over X_g viewed as
// [Np][M1][M2], four boxes of 8 columns x 256 rows, completion counted on an mbarrier) into a
// shared-memory buffer that, once every thread has read its pass-0 inputs, serves as the
// transform's exchange area; the next tile's load is issued as soon as the exchange reads of
// pass 1 are done, so it overlaps the last pass and the stores.  Measured (N = 2^20, staged):
// Np = 256 1.048 -> 1.000 ms, Np = 128 0.532 -> 0.496 ms.  At M1 = 512 (128-byte pieces) the
// plain kernel is faster (2^18: 0.203 against 0.223 ms), and two buffers per CTA (the next
// load in flight for a whole tile) leave room for one CTA per SM only, which is slower still.
//
// Per tile (columns m2 = m20 + c of channel kh): M1-point DFT over m1, times the rotate factor
// W_N^{(m2 m1') mod N} (split as in ssca_cols_tile), written in place to Y[kh][m1'][m2] (the
// tile's own input, already in shared memory).
#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "internal.h"
#include "tiles.cuh"

namespace scd {
namespace {

// Bounded waits: every poll loop gives up after this many polls.
constexpr uint32_t kTmaPollLimit = kMbarPollLimit;

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_expect_tx(uint64_t* mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(su32(mbar)), "r"(bytes) : "memory");
}

// One box of the 3-D tensor map into shared memory; x is the innermost coordinate (m2).
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* tm, int x, int y, int z, uint64_t* mbar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
      :: "r"(su32(dst)), "l"(reinterpret_cast<uint64_t>(tm)), "r"(x), "r"(y), "r"(z), "r"(su32(mbar))
      : "memory");
}

template <int M1>
struct ColsTma {
  using PI = PlanInfo<M1>;
  using S = TileShape<M1>;
  static constexpr int C = S::C;
  static constexpr int ROWS = M1 < 256 ? M1 : 256;                     // box height (at most 256)
  static constexpr int BOXES = M1 / ROWS;
  static constexpr int TILE_BYTES = M1 * C * 8;                        // dense landing area
  static constexpr int EXCH_BYTES = C * PI::stride(C) * 8;             // padded exchange area
  static constexpr int BUF = ((TILE_BYTES > EXCH_BYTES ? TILE_BYTES : EXCH_BYTES) + 127) / 128 * 128;
  static constexpr int STAGE_OFF = BUF;                                // 256 shared rotate factors
  static constexpr int MBAR_OFF = STAGE_OFF + 256 * 8;
  static constexpr int SMEM = MBAR_OFF + 16;
  static_assert(PI::n == 2 && PI::r0 == PI::T, "two-pass plans, one residue per thread");
  static_assert(C * PI::r1 == 256, "one staged factor per thread");
  static_assert(C * 8 % 16 == 0, "TMA boxes need 16-byte rows");
};

template <int M1>
__global__ void __launch_bounds__(256, 2)
k_ssca_cols_tma(const __grid_constant__ CUtensorMap tm, float2* __restrict__ Y, int N, int M2, int Np,
                const float2* __restrict__ wN, const float2* __restrict__ tw, unsigned* err) {
  using K = ColsTma<M1>;
  using PI = PlanInfo<M1>;
  using F = FftPieces<M1>;
  constexpr int C = K::C, E = PI::E, T = PI::T;
  static_assert(C * T == 256, "block shape");
  extern __shared__ __align__(128) unsigned char smem[];
  float2* buf = reinterpret_cast<float2*>(smem);
  float2* stage = reinterpret_cast<float2*>(smem + K::STAGE_OFF);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + K::MBAR_OFF);
  const int tid = threadIdx.x;
  const int c = tid % C, t = tid / C;                                  // interleaved columns
  const int per_row = M2 / C;
  const int64_t ntiles = (int64_t)Np * per_row;

  auto issue = [&](int64_t tile) {                                     // thread 0 only
    const int kh = (int)(tile / per_row), m20 = (int)(tile % per_row) * C;
    mbar_expect_tx(mbar, (uint32_t)K::TILE_BYTES);
#pragma unroll
    for (int q = 0; q < K::BOXES; ++q)
      tma_load_3d(reinterpret_cast<unsigned char*>(buf) + q * K::ROWS * C * 8, &tm, m20, q * K::ROWS, kh, mbar);
  };
  if (tid == 0) {
    umma::mbar_init(mbar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (tid == 0 && (int64_t)blockIdx.x < ntiles) issue(blockIdx.x);
  uint32_t phase = 0u;
  bool ok = true;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int kh = (int)(tile / per_row), m20 = (int)(tile % per_row) * C;
    __syncthreads();                                                   // previous tile's stage reads done
    // rotate factor of bin f = t + p j (p = r0 = T): W_N^{(m20 + c) t} W_N^{(m20 + c) p j}, the
    // second staged as [j][c] (one per thread)
    stage[tid] = __ldg(wN + (((int64_t)(m20 + tid % C) * PI::r0 * (tid / C)) & (N - 1)));
    const float2 a0 = __ldg(wN + (((int64_t)(m20 + c) * t) & (N - 1)));
    const bool got = umma::mbar_wait_bounded(mbar, phase, kTmaPollLimit);
    if (__syncthreads_or(!got)) { ok = false; break; }                 // one decision for the whole CTA
    phase ^= 1u;
    float2* reg = buf + c * PI::stride(C);
    float2 v[E];
    {                                                                  // pass 0 from the landing area
      constexpr int R = PI::r0;
#pragma unroll
      for (int r = 0; r < R; ++r) v[r] = buf[(t + r * (M1 / R)) * C + c];
      dft<R>(v);
    }
    __syncthreads();                                                   // every dense read precedes the stores
    F::pass0_store(t, reg, v);
    __syncthreads();
    F::template pass_load<1>(t, reg, tw, v);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");       // generic accesses before the next TMA write
    __syncthreads();                                                   // every exchange read is done: buffer free
    if (tid == 0 && tile + (int64_t)gridDim.x < ntiles) issue(tile + (int64_t)gridDim.x);
    float2* ob = Y + (int64_t)kh * N + m20 + c;
    auto dst = [&](int, int f, float2 val) {
      const float2 w = cmul(a0, stage[(f / PI::r0) * C + c]);         // W_N^{(m20 + c) f}, f = t + r0 j
      ob[(int64_t)f * M2] = cmul(val, w);
    };
    F::template pass_out<1>(c, t, dst, v);
  }
  if (!ok) {
    if (tid == 0) atomicOr(err, 4u);
    umma::mbar_wait_bounded(mbar, phase, kTmaPollLimit);              // the copy in flight, if any
  }
  __syncthreads();
  if (tid == 0) umma::mbar_inval(mbar);
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn(cudaError_t* err) {
  static std::once_flag once;
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static cudaError_t status = cudaSuccess;
  std::call_once(once, [] {
    cudaDriverEntryPointQueryResult q;
    void* p = nullptr;
    status = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q);
    if (status == cudaSuccess && q != cudaDriverEntryPointSuccess) status = cudaErrorSymbolNotFound;
    if (status == cudaSuccess) fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  *err = status;
  return fn;
}

template <int M1>
cudaError_t launch_t(float2* Y, int N, int Np, int M2, cudaStream_t st) {
  using K = ColsTma<M1>;
  cudaError_t e;
  PFN_cuTensorMapEncodeTiled_v12000 encode = encode_fn(&e);
  if (!encode) return e;
  const float2* wN = table_roots(N, &e);
  if (!wN) return e;
  const float2* tw = table_pass(M1, &e);
  if (!tw) return e;
  unsigned* errw = device_error_word(&e);
  if (!errw) return e;
  // X_g as [Np][M1][M2] 8-byte elements (complex64 moved as raw 64-bit words)
  CUtensorMap tm;
  const cuuint64_t dims[3] = {(cuuint64_t)M2, (cuuint64_t)M1, (cuuint64_t)Np};
  const cuuint64_t strides[2] = {(cuuint64_t)M2 * 8, (cuuint64_t)M1 * M2 * 8};
  const cuuint32_t box[3] = {(cuuint32_t)K::C, (cuuint32_t)K::ROWS, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  if (encode(&tm, CU_TENSOR_MAP_DATA_TYPE_UINT64, 3, Y, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return cudaErrorInvalidValue;
  if ((e = cudaFuncSetAttribute(k_ssca_cols_tma<M1>, cudaFuncAttributeMaxDynamicSharedMemorySize, K::SMEM)) !=
      cudaSuccess)
    return e;
  int dev = 0, sms = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  const int64_t ntiles = (int64_t)Np * (M2 / K::C);
  const int grid = (int)(ntiles < 2 * sms ? ntiles : 2 * sms);         // two persistent CTAs per SM
  k_ssca_cols_tma<M1><<<grid, 256, K::SMEM, st>>>(tm, Y, N, M2, Np, wN, tw, errw);
  return cudaGetLastError();
}

}  // namespace

bool ssca_cols_tma_supported(int M1) { return M1 == 1024; }

cudaError_t ssca_cols_tma(float2* Y, int64_t N, int Np, int M1, int M2, cudaStream_t st) {
  if (((uintptr_t)Y % 16) != 0) return cudaErrorInvalidValue;         // TMA global address alignment
  switch (M1) {
    case 1024: return launch_t<1024>(Y, (int)N, Np, M2, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace scd
