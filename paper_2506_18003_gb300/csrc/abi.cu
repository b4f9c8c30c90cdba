// C-ABI entry points of libscd.so (declared in include/scd.h): argument validation,
// workspace carving and kernel dispatch.  No entry point allocates caller-visible memory
// and none falls back to anything but the CUDA kernels of this library.
#include <stdio.h>
#include <string.h>

#include <atomic>

#include "internal.h"

namespace scd {
std::atomic<uint64_t> g_launches{0};
void count_launches(int n) { g_launches.fetch_add((uint64_t)n, std::memory_order_relaxed); }
}  // namespace scd

namespace {

thread_local char g_last_error[256] = "";

scd_status cuda_fail(cudaError_t e) {
  snprintf(g_last_error, sizeof g_last_error, "%s: %s", cudaGetErrorName(e), cudaGetErrorString(e));
  return SCD_ERR_CUDA;
}

bool aligned(const void* p, size_t a) { return ((uintptr_t)p % a) == 0; }

const scd_opts kDefaultOpts = {nullptr, SCD_FP32, 1, nullptr, 0, nullptr, 0, SCD_SCHEDULE_AUTO, nullptr, 0, 0};

// Records opts.stage_events[i] (when the caller asked for at least `needed` events).
struct StageMarks {
  const scd_opts& o;
  int needed;
  cudaError_t mark(int i, cudaStream_t st) const {
    if (!o.stage_events || o.n_stage_events < needed || i >= o.n_stage_events) return cudaSuccess;
    return cudaEventRecord((cudaEvent_t)o.stage_events[i], st);
  }
};

const scd_opts& opts_or_default(const scd_opts* o) { return o ? *o : kDefaultOpts; }

bool np_ok(int32_t Np) { return Np >= 16 && Np <= 256 && scd::is_pow2(Np); }

// Sizes that are not powers of two run on Bluestein's identity with transforms of size
// M >= 2n - 1: FAM pairs in one CTA (M <= 16384), SSCA four-step transforms (M <= 2^20).
constexpr int32_t kMaxAnyP = 8192;
constexpr int64_t kMaxAnyN = int64_t(1) << 19;

scd_status check_fam(const void* x, int64_t N, int32_t Np, int32_t L, int32_t P, const float* window,
                     const void* out) {
  if (!x || !out) return SCD_ERR_ARG;
  if (!aligned(x, 8) || !aligned(out, 16) || (window && !aligned(window, 4))) return SCD_ERR_ARG;
  if (L < 1 || Np < 1 || P < 1 || N < 1) return SCD_ERR_ARG;
  if (!np_ok(Np)) return SCD_ERR_UNSUPPORTED;
  if (P < 2 || P > 16384 || (!scd::is_pow2(P) && P > kMaxAnyP)) return SCD_ERR_UNSUPPORTED;
  if ((int64_t)(P - 1) * L + Np > N) return SCD_ERR_ARG;
  if ((int64_t)(P - 1) * L + Np > (int64_t(1) << 31)) return SCD_ERR_UNSUPPORTED;
  return SCD_OK;
}

scd_status check_ssca(const void* x, int64_t N, int32_t Np, const float* window, const void* out) {
  if (!x || !out) return SCD_ERR_ARG;
  if (!aligned(x, 8) || !aligned(out, 16) || (window && !aligned(window, 4))) return SCD_ERR_ARG;
  if (N < 1 || Np < 1) return SCD_ERR_ARG;
  if (!np_ok(Np)) return SCD_ERR_UNSUPPORTED;
  if (N < 4096 || N > (1 << 20) || (!scd::is_pow2(N) && N > kMaxAnyN)) return SCD_ERR_UNSUPPORTED;
  return SCD_OK;
}

size_t round_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// The variant fields: y (when given) a complex64 device array aligned like x; conjugate 0 / 1.
bool variant_ok(const scd_opts& o) {
  return (!o.y || aligned(o.y, 8)) && (o.conjugate == 0 || o.conjugate == 1) && o.normalise >= 0 &&
         o.normalise <= 2;
}

}  // namespace

namespace scd {
void set_last_error(const char* msg) { snprintf(g_last_error, sizeof g_last_error, "%s", msg); }
scd_status check_fam_args(const void* x, int64_t N, int32_t Np, int32_t L, int32_t P, const float* window,
                          const void* out) {
  return check_fam(x, N, Np, L, P, window, out);
}
}  // namespace scd

extern "C" {

size_t scd_fam_workspace_bytes(int64_t N, int32_t Np, int32_t L, int32_t P, int32_t precision) {
  (void)N; (void)L; (void)precision;
  if (Np < 1 || P < 1) return 0;
  // X[kh][p], Y[lh][p], then the input-normalisation area
  return 2 * round_up(sizeof(float) * 2 * (size_t)Np * (size_t)P, 256) + scd::norm_workspace_bytes();
}

size_t scd_ssca_workspace_bytes(int64_t N, int32_t Np, int32_t precision) {
  (void)precision;
  if (Np < 1 || N < 1) return 0;
  if (!scd::is_pow2(N)) return scd::ssca_any_workspace(N, Np) + scd::norm_workspace_bytes();
  // the persistent schedule's X_g + rotating slots + counters cover the staged schedule's X_g;
  // the input-normalisation area follows
  return scd::ssca_persistent_workspace(N, Np) + scd::norm_workspace_bytes();
}

scd_status scd_fam(const void* x, int64_t N, int32_t Np, int32_t L, int32_t P, const float* window, void* out,
                   const scd_opts* opts) {
  scd::NvtxRange range("scd_fam");
  scd_status s = check_fam(x, N, Np, L, P, window, out);
  if (s != SCD_OK) return s;
  const scd_opts& o = opts_or_default(opts);
  if (o.precision != SCD_FP32 && o.precision != SCD_SPLIT_BF16) return SCD_ERR_UNSUPPORTED;
  if (!variant_ok(o)) return SCD_ERR_ARG;
  const size_t need = scd_fam_workspace_bytes(N, Np, L, P, o.precision);
  if (!o.workspace || o.workspace_bytes < need) return SCD_ERR_WORKSPACE;
  if (!aligned(o.workspace, 16)) return SCD_ERR_ARG;
  if (scd::fault_host("fam")) return SCD_ERR_CUDA;
  if (o.normalise && o.y) return SCD_ERR_UNSUPPORTED;
  cudaStream_t st = (cudaStream_t)o.stream;
  cudaError_t e;
  if (!window) {
    window = scd::table_hamming(Np, &e);
    if (!window) return cuda_fail(e);
  }
  if (o.normalise) {
    void* area = (char*)o.workspace + need - scd::norm_workspace_bytes();
    if ((e = scd::normalised_window((const float2*)x, (int64_t)(P - 1) * L + Np, window, Np, o.normalise, 1, area,
                                    &window, st)) != cudaSuccess)
      return cuda_fail(e);
  }
  float2* X = (float2*)o.workspace;
  const bool partner = o.y || o.conjugate;
  StageMarks m{o, partner ? 4 : 3};
  int mk = 0;
  if ((e = m.mark(mk++, st)) != cudaSuccess) return cuda_fail(e);
  if ((e = scd::fam_channelise((const float2*)x, Np, L, P, window, X, st, o.precision)) != cudaSuccess) return cuda_fail(e);
  const float2* Y = X;
  if (partner) {
    // the second operand: y's (or x's) demodulates, conjugated for the conjugate estimate so
    // that the pair kernel's X conj(Y) becomes X Y
    float2* Z = (float2*)((char*)o.workspace + scd_fam_workspace_bytes(N, Np, L, P, o.precision) / 2);
    if ((e = m.mark(mk++, st)) != cudaSuccess) return cuda_fail(e);
    if ((e = scd::fam_channelise((const float2*)(o.y ? o.y : x), Np, L, P, window, Z, st, o.precision,
                                 o.conjugate != 0)) != cudaSuccess)
      return cuda_fail(e);
    Y = Z;
  }
  if ((e = m.mark(mk++, st)) != cudaSuccess) return cuda_fail(e);
  e = scd::is_pow2(P) ? scd::fam_pair_fft(X, Y, Np, P, (float2*)out, st, o.precision)
                      : scd::fam_pair_fft_any(X, Y, Np, P, (float2*)out, st, o.precision);
  if (e != cudaSuccess) return cuda_fail(e);
  if ((e = m.mark(mk++, st)) != cudaSuccess) return cuda_fail(e);
  return SCD_OK;
}

scd_status scd_ssca(const void* x, int64_t N, int32_t Np, const float* window, void* out, const scd_opts* opts) {
  scd::NvtxRange range("scd_ssca");
  scd_status s = check_ssca(x, N, Np, window, out);
  if (s != SCD_OK) return s;
  const scd_opts& o = opts_or_default(opts);
  if (o.precision != SCD_FP32 && o.precision != SCD_SPLIT_BF16) return SCD_ERR_UNSUPPORTED;
  if (!variant_ok(o)) return SCD_ERR_ARG;
  const float2* y = (const float2*)(o.y ? o.y : x);
  const bool conj = o.conjugate != 0;
  const size_t need = scd_ssca_workspace_bytes(N, Np, o.precision);
  if (!o.workspace || o.workspace_bytes < need) return SCD_ERR_WORKSPACE;
  if (!aligned(o.workspace, 16)) return SCD_ERR_ARG;
  if (scd::fault_host("ssca")) return SCD_ERR_CUDA;
  if (o.normalise && o.y) return SCD_ERR_UNSUPPORTED;
  cudaStream_t st = (cudaStream_t)o.stream;
  cudaError_t e;
  if (!window) {
    window = scd::table_hamming(Np, &e);
    if (!window) return cuda_fail(e);
  }
  if (o.normalise) {
    void* area = (char*)o.workspace + need - scd::norm_workspace_bytes();
    if ((e = scd::normalised_window((const float2*)x, N, window, Np, o.normalise, 2, area, &window, st)) !=
        cudaSuccess)
      return cuda_fail(e);
  }
  float2* ws = (float2*)o.workspace;
  if (!scd::is_pow2(N)) {
    // any N: the strip transform on Bluestein's identity (staged kernels only)
    if (o.schedule == SCD_SCHEDULE_PERSISTENT) return SCD_ERR_UNSUPPORTED;
    if (o.schedule != SCD_SCHEDULE_AUTO && o.schedule != SCD_SCHEDULE_STAGES && o.schedule != SCD_SCHEDULE_FUSED)
      return SCD_ERR_ARG;
    StageMarks m{o, 4};
    if ((e = m.mark(0, st)) != cudaSuccess) return cuda_fail(e);
    if ((e = scd::ssca_any_cdp((const float2*)x, y, conj, N, Np, window, ws, st, o.precision)) != cudaSuccess)
      return cuda_fail(e);
    if ((e = m.mark(1, st)) != cudaSuccess) return cuda_fail(e);
    if ((e = scd::ssca_any_first(N, Np, ws, st, o.precision)) != cudaSuccess) return cuda_fail(e);
    if ((e = m.mark(2, st)) != cudaSuccess) return cuda_fail(e);
    if ((e = scd::ssca_any_second(N, Np, ws, (float2*)out, st, o.precision)) != cudaSuccess) return cuda_fail(e);
    if ((e = m.mark(3, st)) != cudaSuccess) return cuda_fail(e);
    return SCD_OK;
  }
  scd::TuneEntry choice{o.schedule, 0, 0, 0.0};
  if (o.schedule == SCD_SCHEDULE_AUTO) choice = scd::ssca_auto_choice(N, Np, o.precision);
  if (choice.schedule != SCD_SCHEDULE_STAGES && choice.schedule != SCD_SCHEDULE_PERSISTENT &&
      choice.schedule != SCD_SCHEDULE_FUSED)
    return SCD_ERR_ARG;
  if (choice.schedule == SCD_SCHEDULE_FUSED && scd::ssca_fused_supported(N, Np, o.precision)) {
    StageMarks m{o, 3};
    if ((e = m.mark(0, st)) != cudaSuccess) return cuda_fail(e);
    if ((e = scd::ssca_fused_chancol((const float2*)x, y, conj, N, Np, window, ws, st)) != cudaSuccess)
      return cuda_fail(e);
    if ((e = m.mark(1, st)) != cudaSuccess) return cuda_fail(e);
    if ((e = scd::ssca_fused_rows(ws, N, Np, (float2*)out, st)) != cudaSuccess) return cuda_fail(e);
    if ((e = m.mark(2, st)) != cudaSuccess) return cuda_fail(e);
    return SCD_OK;
  }
  if (choice.schedule == SCD_SCHEDULE_PERSISTENT) {
    StageMarks m{o, 2};
    if ((e = m.mark(0, st)) != cudaSuccess) return cuda_fail(e);
    scd_status r = choice.item_bytes
                       ? scd::ssca_persistent_tuned((const float2*)x, y, conj, N, Np, window, (float2*)out, o.workspace,
                                                    o.workspace_bytes, st, o.precision, choice.item_bytes,
                                                    choice.slot_bytes)
                       : scd::ssca_persistent((const float2*)x, y, conj, N, Np, window, (float2*)out, o.workspace,
                                              o.workspace_bytes, st, o.precision);
    if (r != SCD_OK) return r;
    if ((e = m.mark(1, st)) != cudaSuccess) return cuda_fail(e);
    return SCD_OK;
  }
  StageMarks m{o, 4};
  if ((e = m.mark(0, st)) != cudaSuccess) return cuda_fail(e);
  if ((e = scd::ssca_cdp((const float2*)x, y, conj, N, Np, window, ws, st, o.precision)) != cudaSuccess)
    return cuda_fail(e);
  if ((e = m.mark(1, st)) != cudaSuccess) return cuda_fail(e);
  if ((e = scd::ssca_cols(ws, N, Np, st, o.precision)) != cudaSuccess) return cuda_fail(e);
  if ((e = m.mark(2, st)) != cudaSuccess) return cuda_fail(e);
  if ((e = scd::ssca_rows(ws, N, Np, (float2*)out, st, o.precision)) != cudaSuccess) return cuda_fail(e);
  if ((e = m.mark(3, st)) != cudaSuccess) return cuda_fail(e);
  return SCD_OK;
}

}  // extern "C"

namespace {
scd_status check_fam_grid(const void* S, int32_t Np, int32_t L, int32_t P, const float* dst) {
  if (!S || !dst || !aligned(S, 16) || !aligned(dst, 16)) return SCD_ERR_ARG;
  if (L < 1) return SCD_ERR_ARG;
  if (!np_ok(Np) || P < 2 || P > 16384 || !scd::is_pow2(P)) return SCD_ERR_UNSUPPORTED;
  if (((int64_t)P * L) % Np != 0 || 2 * (int64_t)L > Np) return SCD_ERR_UNSUPPORTED;
  if (4 * (int64_t)Np * P * L >= (int64_t(1) << 31)) return SCD_ERR_UNSUPPORTED;
  return SCD_OK;
}

scd_status check_ssca_grid(const void* S, int64_t N, int32_t Np, const float* dst) {
  if (!S || !dst || !aligned(S, 16) || !aligned(dst, 16)) return SCD_ERR_ARG;
  if (!np_ok(Np) || N < 4096 || N > (1 << 20) || !scd::is_pow2(N)) return SCD_ERR_UNSUPPORTED;
  return SCD_OK;
}

// Runs one map / profile kernel between stage marks 0 and 1.
template <class Launch>
scd_status run_one(const scd_opts& o, Launch launch) {
  if (o.map_power != 1 && o.map_power != 2) return SCD_ERR_ARG;
  StageMarks m{o, 2};
  cudaStream_t st = (cudaStream_t)o.stream;
  cudaError_t e;
  if ((e = m.mark(0, st)) != cudaSuccess) return cuda_fail(e);
  if ((e = launch(st)) != cudaSuccess) return cuda_fail(e);
  if ((e = m.mark(1, st)) != cudaSuccess) return cuda_fail(e);
  return SCD_OK;
}
}  // namespace

extern "C" {

scd_status scd_fam_map(const void* S, int32_t Np, int32_t L, int32_t P, float* map, const scd_opts* opts) {
  scd::NvtxRange range("scd_fam_map");
  scd_status s = check_fam_grid(S, Np, L, P, map);
  if (s != SCD_OK) return s;
  if (scd::fault_host("fam_map")) return SCD_ERR_CUDA;
  const scd_opts& o = opts_or_default(opts);
  return run_one(o, [&](cudaStream_t st) {
    return scd::fam_map((const float2*)S, Np, L, P, o.map_power, o.conjugate != 0, map, st);
  });
}

scd_status scd_fam_alpha_profile(const void* S, int32_t Np, int32_t L, int32_t P, float* profile,
                                 const scd_opts* opts) {
  scd_status s = check_fam_grid(S, Np, L, P, profile);
  if (s != SCD_OK) return s;
  const scd_opts& o = opts_or_default(opts);
  return run_one(o, [&](cudaStream_t st) {
    return scd::fam_alpha_profile((const float2*)S, Np, L, P, o.map_power, o.conjugate != 0, profile, st);
  });
}

scd_status scd_ssca_alpha_profile(const void* S, int64_t N, int32_t Np, float* profile, const scd_opts* opts) {
  scd_status s = check_ssca_grid(S, N, Np, profile);
  if (s != SCD_OK) return s;
  const scd_opts& o = opts_or_default(opts);
  return run_one(o, [&](cudaStream_t st) {
    return scd::ssca_alpha_profile((const float2*)S, N, Np, o.map_power, profile, st);
  });
}

scd_status scd_ssca_map(const void* S, int64_t N, int32_t Np, float* map, const scd_opts* opts) {
  scd::NvtxRange range("scd_ssca_map");
  scd_status s = check_ssca_grid(S, N, Np, map);
  if (s != SCD_OK) return s;
  if (scd::fault_host("ssca_map")) return SCD_ERR_CUDA;
  const scd_opts& o = opts_or_default(opts);
  return run_one(o, [&](cudaStream_t st) { return scd::ssca_map((const float2*)S, N, Np, o.map_power, map, st); });
}

scd_status scd_chebyshev_window(int32_t Np, double atten_db, float* window, void* stream) {
  if (!window || !aligned(window, 4) || Np < 2 || Np > 256) return SCD_ERR_ARG;
  if (!(atten_db > 0.0 && atten_db <= 300.0)) return SCD_ERR_ARG;   // also rejects NaN
  scd::count_launches(1);
  cudaError_t e = scd::build_chebyshev_into(window, Np, atten_db, (cudaStream_t)stream);
  return e == cudaSuccess ? SCD_OK : cuda_fail(e);
}

scd_status scd_prepare(int32_t estimator, int64_t N, int32_t Np, int32_t P) {
  if (!np_ok(Np)) return SCD_ERR_UNSUPPORTED;
  cudaError_t e;
  if (!scd::table_hamming(Np, &e) || !scd::table_roots(Np, &e) || !scd::table_pass(Np, &e)) return cuda_fail(e);
  if (estimator == 0) {
    if (P < 2 || P > 16384 || (!scd::is_pow2(P) && P > kMaxAnyP)) return SCD_ERR_UNSUPPORTED;
    if (scd::is_pow2(P)) return scd::table_pass(P, &e) ? SCD_OK : cuda_fail(e);
    const int64_t M = scd::bluestein_len_host(P);
    if (!scd::table_pass((int)M, &e) || !scd::table_chirp(P, &e) || !scd::table_bluestein(P, M, &e))
      return cuda_fail(e);
    return SCD_OK;
  }
  if (estimator == 1) {
    if (N < 4096 || N > (1 << 20) || (!scd::is_pow2(N) && N > kMaxAnyN)) return SCD_ERR_UNSUPPORTED;
    const int64_t M = scd::is_pow2(N) ? N : scd::bluestein_len_host(N);
    int M1, M2;
    scd::ssca_split(M, &M1, &M2);
    if (!scd::table_roots((int)M, &e) || !scd::table_pass(M1, &e) || !scd::table_pass(M2, &e) ||
        !scd::table_cols((int)M, M1, scd::ssca_cols_per_tile(M1), &e) || !scd::device_error_word(&e))
      return cuda_fail(e);
    if (!scd::is_pow2(N) && (!scd::table_chirp(N, &e) || !scd::table_bluestein_rows(N, M, M1, &e)))
      return cuda_fail(e);
    return SCD_OK;
  }
  return SCD_ERR_ARG;
}

// ------------------------------------------------------------------------- host buffers
size_t scd_fam_host_workspace_bytes(int64_t N, int32_t Np, int32_t L, int32_t P, int32_t precision) {
  if (Np < 1 || P < 1 || N < 1) return 0;
  return round_up(8 * (size_t)N, 256) + round_up(4 * (size_t)Np, 256) + round_up(8 * (size_t)Np * Np * P, 256) +
         scd_fam_workspace_bytes(N, Np, L, P, precision);
}

size_t scd_ssca_host_workspace_bytes(int64_t N, int32_t Np, int32_t precision) {
  if (Np < 1 || N < 1) return 0;
  return round_up(8 * (size_t)N, 256) + round_up(4 * (size_t)Np, 256) + round_up(8 * (size_t)Np * N, 256) +
         scd_ssca_workspace_bytes(N, Np, precision);
}

}  // extern "C"

namespace {
// Carves [x | window | out | estimator workspace] from the caller's device workspace,
// copies the inputs in, runs `run(dev_x, dev_window, dev_out, inner_opts)`, copies the
// estimate out and synchronises.
template <class Run>
scd_status run_host(const void* x_host, int64_t N, int32_t Np, const float* window_host, void* out_host,
                    size_t out_bytes, size_t need, const scd_opts* opts, Run run) {
  if (!x_host || !out_host) return SCD_ERR_ARG;
  const scd_opts& o = opts_or_default(opts);
  if (o.y) return SCD_ERR_ARG;                                 // no host form of the cross estimate
  if (!o.workspace || o.workspace_bytes < need) return SCD_ERR_WORKSPACE;
  if (!aligned(o.workspace, 256)) return SCD_ERR_ARG;
  char* base = (char*)o.workspace;
  char* dx = base;
  char* dw = dx + round_up(8 * (size_t)N, 256);
  char* dout = dw + round_up(4 * (size_t)Np, 256);
  char* dws = dout + round_up(out_bytes, 256);
  scd_opts inner = o;
  inner.workspace = dws;
  inner.workspace_bytes = o.workspace_bytes - (size_t)(dws - base);
  cudaStream_t st = (cudaStream_t)o.stream;
  cudaError_t e;
  if ((e = cudaMemcpyAsync(dx, x_host, 8 * (size_t)N, cudaMemcpyHostToDevice, st)) != cudaSuccess) return cuda_fail(e);
  if (window_host &&
      (e = cudaMemcpyAsync(dw, window_host, 4 * (size_t)Np, cudaMemcpyHostToDevice, st)) != cudaSuccess)
    return cuda_fail(e);
  scd_status s = run((const void*)dx, window_host ? (const float*)dw : nullptr, (void*)dout, &inner);
  if (s != SCD_OK) return s;
  if ((e = cudaMemcpyAsync(out_host, dout, out_bytes, cudaMemcpyDeviceToHost, st)) != cudaSuccess) return cuda_fail(e);
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(e);
  return SCD_OK;
}
}  // namespace

extern "C" {

scd_status scd_fam_host(const void* x_host, int64_t N, int32_t Np, int32_t L, int32_t P, const float* window_host,
                        void* out_host, const scd_opts* opts) {
  scd_status s = check_fam((const void*)16, N, Np, L, P, nullptr, (const void*)16);
  if (s != SCD_OK) return s;
  const scd_opts& o = opts_or_default(opts);
  const size_t need = scd_fam_host_workspace_bytes(N, Np, L, P, o.precision);
  return run_host(x_host, N, Np, window_host, out_host, 8 * (size_t)Np * Np * P, need, opts,
                  [&](const void* dx, const float* dw, void* dout, const scd_opts* in) {
                    return scd_fam(dx, N, Np, L, P, dw, dout, in);
                  });
}

scd_status scd_ssca_host(const void* x_host, int64_t N, int32_t Np, const float* window_host, void* out_host,
                         const scd_opts* opts) {
  scd_status s = check_ssca((const void*)16, N, Np, nullptr, (const void*)16);
  if (s != SCD_OK) return s;
  const scd_opts& o = opts_or_default(opts);
  const size_t need = scd_ssca_host_workspace_bytes(N, Np, o.precision);
  return run_host(x_host, N, Np, window_host, out_host, 8 * (size_t)Np * N, need, opts,
                  [&](const void* dx, const float* dw, void* dout, const scd_opts* in) {
                    return scd_ssca(dx, N, Np, dw, dout, in);
                  });
}

// ------------------------------------------------------------------------- timing
scd_status scd_events_create(int32_t n, void** events) {
  if (n < 0 || (n > 0 && !events)) return SCD_ERR_ARG;
  for (int i = 0; i < n; ++i) {
    cudaEvent_t ev;
    cudaError_t e = cudaEventCreate(&ev);
    if (e != cudaSuccess) {
      for (int j = 0; j < i; ++j) cudaEventDestroy((cudaEvent_t)events[j]);
      return cuda_fail(e);
    }
    events[i] = (void*)ev;
  }
  return SCD_OK;
}

scd_status scd_events_destroy(int32_t n, void** events) {
  if (n < 0 || (n > 0 && !events)) return SCD_ERR_ARG;
  for (int i = 0; i < n; ++i)
    if (events[i]) cudaEventDestroy((cudaEvent_t)events[i]);
  return SCD_OK;
}

scd_status scd_event_elapsed_ms(void* start, void* end, float* ms) {
  if (!start || !end || !ms) return SCD_ERR_ARG;
  cudaError_t e = cudaEventSynchronize((cudaEvent_t)end);
  if (e == cudaSuccess) e = cudaEventElapsedTime(ms, (cudaEvent_t)start, (cudaEvent_t)end);
  return e == cudaSuccess ? SCD_OK : cuda_fail(e);
}

scd_status scd_event_record(void* event, void* stream) {
  if (!event) return SCD_ERR_ARG;
  cudaError_t e = cudaEventRecord((cudaEvent_t)event, (cudaStream_t)stream);
  return e == cudaSuccess ? SCD_OK : cuda_fail(e);
}

scd_status scd_check_device(void* stream) {
  cudaError_t e;
  unsigned* w = scd::device_error_word(&e);
  if (!w) return cuda_fail(e);
  if ((e = cudaStreamSynchronize((cudaStream_t)stream)) != cudaSuccess) return cuda_fail(e);
  unsigned h = 0;
  if ((e = cudaMemcpy(&h, w, sizeof h, cudaMemcpyDeviceToHost)) != cudaSuccess) return cuda_fail(e);
  if (h == 0) return SCD_OK;
  if ((e = cudaMemset(w, 0, sizeof h)) != cudaSuccess) return cuda_fail(e);
  scd::set_last_error("a bounded device-side wait expired");
  return SCD_ERR_TIMEOUT;
}

uint64_t scd_launch_count(void) { return scd::g_launches.load(std::memory_order_relaxed); }

void scd_release_cache(void) {
  scd::release_single_plans();
  scd::release_tables();
}

const char* scd_status_string(scd_status s) {
  switch (s) {
    case SCD_OK: return "ok";
    case SCD_ERR_ARG: return "invalid argument";
    case SCD_ERR_UNSUPPORTED: return "unsupported size or option";
    case SCD_ERR_CUDA: return "CUDA error";
    case SCD_ERR_WORKSPACE: return "workspace missing or too small";
    case SCD_ERR_TIMEOUT: return "device-side wait timed out";
    case SCD_ERR_INTERNAL: return "internal error";
  }
  return "unknown status";
}

const char* scd_last_error(void) { return g_last_error; }

int32_t scd_version(void) { return 200; }

}  // extern "C"
