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
//  * FP32 form, auto estimate only, no per-stage timing events;
//  * every GPU that loads the library holds the array (about 2.25 MB) until the process exits;
//  * all calls share the array and it keeps the last call's contents: each call rebuilds the
//    tables it uses and overwrites every element of X it reads, so nothing needs to start at
//    zero; calls that overlap on the same device (on different streams, or issued from
//    different host threads) race on that device's array and must be serialised by the
//    caller; calls on different devices are independent (each device has its own copy);
//  * the first call in a device context resolves the array's device address with
//    cudaGetSymbolAddress (a set-up step guarded by a mutex, cached per device and keyed by
//    the context's ID, so that a context created again after cudaDeviceReset resolves it
//    again); make that first call before any stream capture on that device, and again after
//    a device reset.
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

// The current context's unique ID (driver API, reached through the runtime's entry-point
// query so that the library needs no link to libcuda); 0 when it cannot be read.
using CtxGetCurrentFn = int (*)(void** ctx);
using CtxGetIdFn = int (*)(void* ctx, unsigned long long* id);

unsigned long long current_context_id() {
  static CtxGetCurrentFn get_current = nullptr;
  static CtxGetIdFn get_id = nullptr;
  static bool looked_up = false;
  if (!looked_up) {
    looked_up = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<CtxGetCurrentFn>(p);
    p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<CtxGetIdFn>(p);
  }
  if (!get_current || !get_id) return 0;
  void* ctx = nullptr;
  unsigned long long id = 0;
  if (get_current(&ctx) != 0 || !ctx || get_id(ctx, &id) != 0) return 0;
  return id;
}

std::mutex g_noalloc_mu;
constexpr int kMaxDevices = 64;
struct Resolved {
  unsigned long long ctx_id;   // context the address belongs to (0: unknown, resolve every call)
  float2* addr;
};
Resolved g_noalloc_addr[kMaxDevices] = {};

// Device address of the scratch array in the current device's context.
cudaError_t scratch_address(float2** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  Resolved& r = g_noalloc_addr[dev];
  const unsigned long long id = current_context_id();
  if (!r.addr || id == 0 || r.ctx_id != id) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);       // also makes the primary context current
    if (e != cudaSuccess) return e;
    r.addr = (float2*)p;
    r.ctx_id = current_context_id();
  }
  *out = r.addr;
  return cudaSuccess;
}

scd_status reject(scd_status s, const char* why) {
  char msg[200];
  snprintf(msg, sizeof msg, "scd_fam_noalloc: %s", why);
  scd::set_last_error(msg);
  return s;
}

}  // namespace

extern "C" {

scd_status scd_fam_noalloc(const void* x, int64_t N, int32_t Np, int32_t L, int32_t P, const float* window,
                           void* out, const scd_opts* opts) {
  scd_status s = scd::check_fam_args(x, N, Np, L, P, window, out);
  if (s != SCD_OK) return reject(s, "arguments rejected by scd_fam's checks");
  if (!scd::is_pow2(P)) return reject(SCD_ERR_UNSUPPORTED, "P must be a power of two");
  if ((int64_t)Np * P > kNoallocMaxX) {
    char msg[160];
    snprintf(msg, sizeof msg, "Np*P = %lld exceeds the fixed scratch limit of %lld", (long long)Np * P,
             (long long)kNoallocMaxX);
    return reject(SCD_ERR_UNSUPPORTED, msg);
  }
  if (opts && opts->precision != SCD_FP32) return reject(SCD_ERR_UNSUPPORTED, "only the FP32 form (SCD_FP32)");
  if (opts && (opts->y || opts->conjugate || opts->normalise))
    return reject(SCD_ERR_UNSUPPORTED, "only the auto estimate without normalisation");
  if (opts && opts->stage_events) return reject(SCD_ERR_UNSUPPORTED, "stage_events are not recorded");
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
