// Internal interfaces between the C-ABI layer and the kernels (not exported).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/scd.h"

namespace scd {

// ---------------------------------------------------------------- phase tables (tables.cu)
// Every table is built once per device on first use, in FP64 from exact integer indices,
// rounded to float2 (and, for the split form, to bf16 hi/lo), and cached until
// scd_release_cache() or process exit.  The returned pointers are device pointers valid
// on every stream of that device.  Building allocates device memory and synchronises, so
// the first call for a size must not happen inside a stream capture.
const float2* table_roots(int M, cudaError_t* err);        // W_M^j, j in [0, M)
const float2* table_pass(int M, cudaError_t* err);         // Stockham pass twiddles of a size-M FFT
const float2* table_cols(int N, int M1, int C, cudaError_t* err);  // W_N^{c m1'}, [m1'][c], c < C
const float* table_hamming(int Np, cudaError_t* err);      // default window, float32
// Bluestein tables of a length-N DFT carried by size-M transforms (M a power of two >= 2N - 1):
// chirp c[j] = W_{2N}^{(j^2) mod 2N} (j < N) and Bh = FFT_M(bt) / M (bluestein.cuh)
const float2* table_chirp(int64_t N, cudaError_t* err);
const float2* table_bluestein(int64_t N, int64_t M, cudaError_t* err);
// Bh in row order of the size-M four-step split M = M1 M2: [q1][q2] = Bh[q1 + M1 q2]
const float2* table_bluestein_rows(int64_t N, int64_t M, int M1, cudaError_t* err);
// bf16 hi/lo complex-as-real DFT matrices of the radices of a size-M plan (tensor-core form)
const unsigned char* table_tc_bmats(int M, int* bytes, cudaError_t* err);
// one word per device, set by kernels whose bounded device-side waits expired
unsigned* device_error_word(cudaError_t* err);
void release_tables();
// The same FP64 builders, writing into memory the caller provides (no allocation, no
// synchronisation; enqueued on st).
cudaError_t build_pass_into(float2* out, int M, cudaStream_t st);   // PlanInfo<M>::tw_len() entries
cudaError_t build_hamming_into(float* out, int Np, cudaStream_t st);
cudaError_t build_chebyshev_into(float* out, int Np, double atten_db, cudaStream_t st);   // Np <= 256

// ---------------------------------------------------------------- FAM (fam.cu)
// X[kh][p] = W_Np^{(k p L) mod Np} sum_n a[n] x[pL + n] W_Np^{(k n) mod Np}  (conj(X) if conj_out)
// precision: SCD_FP32 or SCD_SPLIT_BF16 (radix DFTs as bf16 hi/lo tensor-core GEMMs)
cudaError_t fam_channelise(const float2* x, int Np, int L, int P, const float* window, float2* X,
                           cudaStream_t st, int precision, bool conj_out = false);
// out[kh][lh][qh] = sum_p X[kh][p] conj(Y[lh][p]) W_P^{(q p) mod P}   (Y = X: auto estimate)
cudaError_t fam_pair_fft(const float2* X, const float2* Y, int Np, int P, float2* out, cudaStream_t st,
                         int precision);
// The same two kernels with caller-provided tables (pass twiddles of size Np and of size P)
// instead of the cached ones.
cudaError_t fam_channelise_with(const float2* x, int Np, int L, int P, const float* window, float2* X,
                                const float2* tw_np, cudaStream_t st);
cudaError_t fam_pair_fft_with(const float2* X, int Np, int P, float2* out, const float2* tw_p, cudaStream_t st);

// ---------------------------------------------------------------- SSCA (ssca.cu)
void ssca_split(int64_t N, int* M1, int* M2);
int ssca_cols_per_tile(int M1);    // columns m2 per CTA of the column pass (256 threads)
// Stage 0: channeliser + CDP, X_g into ws[kh][n]: X_T(n,k) conj(y[n]) (y[n] if conj)
cudaError_t ssca_cdp(const float2* x, const float2* y, bool conj, int64_t N, int Np, const float* window, float2* ws,
                     cudaStream_t st, int precision);
// Stage 1: M1-point column FFTs times the rotate factor, in place on ws
cudaError_t ssca_cols(float2* ws, int64_t N, int Np, cudaStream_t st, int precision);
// The FP32 column pass with its input staged through TMA (cols_tma.cu), for the M1 where it
// is the faster one; ws 16-byte aligned, rows of N = M1 M2 values.
bool ssca_cols_tma_supported(int M1);
cudaError_t ssca_cols_tma(float2* ws, int64_t N, int Np, int M1, int M2, cudaStream_t st);
// Stage 2: M2-point row FFTs, fftshifted into out[kh][sh]
cudaError_t ssca_rows(const float2* ws, int64_t N, int Np, float2* out, cudaStream_t st, int precision);

// Fused schedule (ssca_fused.cu): tile A = channeliser + CDP + the M1-point pass over m1 and the
// rotate factor, Y[kh][m2][q1] into ws; tile B = the M2-point pass over m2 into out[kh][sh].
// Supported where fused_split (ssca_fused.cuh) fits the tiles, FP32 form.
bool ssca_fused_supported(int64_t N, int Np, int precision);
cudaError_t ssca_fused_chancol(const float2* x, const float2* y, bool conj, int64_t N, int Np, const float* window,
                               float2* ws, cudaStream_t st);
cudaError_t ssca_fused_rows(const float2* ws, int64_t N, int Np, float2* out, cudaStream_t st);

// Default schedule of scd_ssca: one persistent launch (batch.cu) over a cached one-signal plan.
size_t ssca_persistent_workspace(int64_t N, int Np);
// y, conj: the channel-data product's second factor, as ssca_cdp
scd_status ssca_persistent(const float2* x, const float2* y, bool conj, int64_t N, int Np, const float* window,
                           float2* out, void* ws, size_t ws_bytes, cudaStream_t st, int precision);
void release_single_plans();

// ---------------------------------------------------------------- any-length DFTs (bluestein.cu)
// FAM pair stage for a P that is not a power of two (3 <= P <= 8192), same contract as
// fam_pair_fft.
cudaError_t fam_pair_fft_any(const float2* X, const float2* Y, int Np, int P, float2* out, cudaStream_t st,
                             int precision);
// SSCA for an N that is not a power of two (4096 <= N <= 2^19): the strip transform of length N
// as Bluestein's cyclic convolution of length M = bluestein_len(N), in three stages on the
// workspace ws (ssca_any_workspace bytes): channeliser + CDP with the chirp folded into the
// second factor; the first size-M transform times the kernel spectrum; the second transform
// into the fftshifted output.
size_t ssca_any_workspace(int64_t N, int Np);
cudaError_t ssca_any_cdp(const float2* x, const float2* y, bool conj, int64_t N, int Np, const float* window,
                         void* ws, cudaStream_t st, int precision);
cudaError_t ssca_any_first(int64_t N, int Np, void* ws, cudaStream_t st, int precision);
cudaError_t ssca_any_second(int64_t N, int Np, void* ws, float2* out, cudaStream_t st, int precision);

// ---------------------------------------------------------------- maps (map.cu)
cudaError_t fam_map(const float2* S, int Np, int L, int P, int power, bool conj, float* map, cudaStream_t st);
cudaError_t ssca_map(const float2* S, int64_t N, int Np, int power, float* map, cudaStream_t st);
// alpha profiles: the largest |S|^power over f of every alpha column of the maps above
cudaError_t fam_alpha_profile(const float2* S, int Np, int L, int P, int power, bool conj, float* prof,
                              cudaStream_t st);
cudaError_t ssca_alpha_profile(const float2* S, int64_t N, int Np, int power, float* prof, cudaStream_t st);

// ---------------------------------------------------------------- autotuner cache (tune.cu)
struct TuneEntry {
  int schedule;           // scd_schedule for single SSCA calls; batch plans: 1 = the SSCA
                          // staged schedule (batch_staged.cu), else 0
  int64_t item_bytes;     // output bytes per persistent-queue item
  int64_t slot_bytes;     // bytes of one SSCA column-pass slot
  double ms;              // measured time of the choice
};
std::string device_key();                                    // "<GPU name>/sm<cc>"
bool tune_lookup(const std::string& key, TuneEntry* out);
void tune_store(const std::string& key, const TuneEntry& e);
// scd_ssca under SCD_SCHEDULE_AUTO: the tuned choice, else the default (STAGES)
TuneEntry ssca_auto_choice(int64_t N, int Np, int precision);
scd_status ssca_persistent_tuned(const float2* x, const float2* y, bool conj, int64_t N, int Np, const float* window,
                                 float2* out, void* ws, size_t ws_bytes, cudaStream_t st, int precision,
                                 int64_t item_bytes, int64_t slot_bytes);

// ---------------------------------------------------------------- input normalisation (norm.cu)
// Window a scaled for the input normalisation of the first n samples of x (mode 1: mean power
// 1, mode 2: peak magnitude 1; `power` 1 for FAM, 2 for SSCA), written into `area`
// (norm_workspace_bytes() bytes of device workspace); *window_out points into it.
size_t norm_workspace_bytes();
cudaError_t normalised_window(const float2* x, int64_t n, const float* a, int Np, int mode, int power, void* area,
                              const float** window_out, cudaStream_t st);

// ---------------------------------------------------------------- diagnostics (diag.cu)
// Fault injection for tests, from the environment variable SCD_FAULT_INJECT (read on every
// call, so a test can set and clear it):
//   "host:<site>"     the entry point <site> (fam, ssca, fam_map, ssca_map, batch_run) fails
//                     with SCD_ERR_CUDA and scd_last_error() "injected fault at <site>" after
//                     its argument checks and before it touches the GPU;
//   "batch_drop:<t>"  batch runs never publish the completion of task t (0 = the first
//                     signal's first stage), so the tasks that depend on it give up their
//                     bounded waits and scd_check_device() reports SCD_ERR_TIMEOUT.
bool fault_host(const char* site);
int fault_batch_drop();
// NVTX range around an entry point (visible to Nsight tools; no cost without one attached).
struct NvtxRange {
  explicit NvtxRange(const char* name);
  ~NvtxRange();
};

// ---------------------------------------------------------------- launch accounting
void count_launches(int n);
// Sets the text scd_last_error() returns on this thread.
void set_last_error(const char* msg);
// scd_fam's argument checks (pointers, alignment, Np, P, N >= (P - 1) L + Np), shared by the
// entry points that take scd_fam's arguments.
scd_status check_fam_args(const void* x, int64_t N, int32_t Np, int32_t L, int32_t P, const float* window,
                          const void* out);

// ---------------------------------------------------------------- helpers
inline bool is_pow2(int64_t v) { return v > 0 && (v & (v - 1)) == 0; }
inline int ilog2(int64_t v) { int r = 0; while ((int64_t(1) << r) < v) ++r; return r; }
// smallest power of two >= 2n - 1 (the cyclic length of a length-n Bluestein DFT)
inline int64_t bluestein_len_host(int64_t n) { int64_t m = 1; while (m < 2 * n - 1) m <<= 1; return m; }

}  // namespace scd
