// scd_fam_noalloc: the FAM estimator for callers that cannot allocate device memory.
//
// The paper has no counterpart to this entry point; it exists for callers of this library
// that are not allowed to call cudaMalloc (or any allocating routine) at the point where
// they run an estimate: for example a real-time receive loop that forbids allocation after
// start-up because an allocation can synchronise the device and stall the sample stream, or
// a plug-in that only receives device pointers for inputs and outputs from a host framework
// that owns all memory.  Instead of a caller workspace and the library's cached tables, it
// uses one file-scope __device__ array of fixed size.
//
// Limits and behaviour:
//  * the scratch holds X (Np x P complex64) plus the FP64-built tables of this call:
//    Np * P <= kNoallocMaxX (= 2^18, i.e. Np=256 with P<=1024, Np=64 with P<=4096, ...);
//    larger sizes are rejected with SCD_ERR_UNSUPPORTED before anything is enqueued, and
//    scd_last_error() then names the limit;
//  * every GPU that loads the library holds the array (about 2.25 MB) until the process exits;
//  * all calls share the array and it keeps the last call's contents: each call rebuilds the
//    tables it uses and overwrites every element of X it reads, so nothing needs to start at
//    zero; calls whose executions overlap on the GPU (different streams, or devices sharing
//    nothing but this code) race on the array on the same device and must be serialised;
//  * the first call on a device resolves the array's device address with
//    cudaGetSymbolAddress (a set-up step per device, guarded by a mutex); make that first
//    call before any stream capture on that device.
// It calls no cudaMalloc, cudaFree or allocating library routine.
#include <stdio.h>

#include <mutex>

#include "fft.cuh"
#include "internal.h"

namespace {

constexpr int64_t kNoallocMaxX = 1 << 18;                  // complex elements of X
// table region: pass table of Np (<= 256), pass table of P (<= 17408), Hamming window
// (256 float = 128 float2)
constexpr int64_t kTabPassNp = 0, kTabPassP = 256, kTabWindow = 256 + 17408;
constexpr int64_t kTabLen = kTabWindow + 128;
constexpr int64_t kScratchLen = kNoallocMaxX + kTabLen;     // float2 elements

__device__ __align__(256) float2 g_noalloc_scratch[kScratchLen];

std::mutex g_noalloc_mu;
constexpr int kMaxDevices = 64;
float2* g_noalloc_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device (resolved once per device).
cudaError_t scratch_address(float2** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_noalloc_addr[dev] = (float2*)p;
  }
  *out = g_noalloc_addr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" {

scd_status scd_fam_noalloc(const void* x, int64_t N, int32_t Np, int32_t L, int32_t P, const float* window,
                           void* out, const scd_opts* opts) {
  if (!x || !out || ((uintptr_t)x % 8) || ((uintptr_t)out % 16) || (window && ((uintptr_t)window % 4)))
    return SCD_ERR_ARG;
  if (L < 1 || N < 1) return SCD_ERR_ARG;
  if (Np < 16 || Np > 256 || !scd::is_pow2(Np) || P < 2 || P > 16384 || !scd::is_pow2(P))
    return SCD_ERR_UNSUPPORTED;
  if ((int64_t)(P - 1) * L + Np > N) return SCD_ERR_ARG;
  if ((int64_t)Np * P > kNoallocMaxX) {
    char msg[160];
    snprintf(msg, sizeof msg, "scd_fam_noalloc: Np*P = %lld exceeds the fixed scratch limit of %lld",
             (long long)Np * P, (long long)kNoallocMaxX);
    scd::set_last_error(msg);
    return SCD_ERR_UNSUPPORTED;
  }
  if (opts && opts->precision != SCD_FP32) return SCD_ERR_UNSUPPORTED;
  if (opts && (opts->y || opts->conjugate || opts->normalise)) return SCD_ERR_UNSUPPORTED;   // plain auto estimate only
  cudaStream_t st = opts ? (cudaStream_t)opts->stream : nullptr;
  float2* base = nullptr;
  cudaError_t e = scratch_address(&base);
  if (e == cudaSuccess) {
    float2* tab = base + kNoallocMaxX;
    float2* tw_np = tab + kTabPassNp;
    float2* tw_p = tab + kTabPassP;
    if (!window) {
      float* w = (float*)(tab + kTabWindow);
      if ((e = scd::build_hamming_into(w, Np, st)) == cudaSuccess) window = w;
    }
    if (e == cudaSuccess) e = scd::build_pass_into(tw_np, Np, st);
    if (e == cudaSuccess) e = scd::build_pass_into(tw_p, P, st);
    if (e == cudaSuccess)
      e = scd::fam_channelise_with((const float2*)x, Np, L, P, window, base, tw_np, st);
    if (e == cudaSuccess) e = scd::fam_pair_fft_with(base, Np, P, (float2*)out, tw_p, st);
  }
  if (e != cudaSuccess) {
    char msg[160];
    snprintf(msg, sizeof msg, "%s: %s", cudaGetErrorName(e), cudaGetErrorString(e));
    scd::set_last_error(msg);
    return SCD_ERR_CUDA;
  }
  return SCD_OK;
}

}  // extern "C"
