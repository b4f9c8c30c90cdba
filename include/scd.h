/* scd.h -- C ABI of libscd.so: spectral correlation density (SCD) estimation on one
 * NVIDIA GB300 (sm_103a) by the FFT accumulation method (FAM) and the strip spectral
 * correlation analyser (SSCA), after Li, Wu and Leong, "AMD Versal Implementations of FAM
 * and SSCA Estimators" (arXiv 2506.18003).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Sample rate fs = 1.  Complex values are complex64: interleaved (re, im) float32 pairs.
 *  - Channel k in [-Np/2, Np/2) (centre frequency k/Np) is stored at kh = k + Np/2.
 *    FAM bin q in [-P/2, P/2) is stored at qh = q + P/2; SSCA bin q in [-N/2, N/2) at
 *    sh = q + N/2 ("fftshifted" axes).
 *  - W_M^j = exp(-i 2 pi j / M).  Phase indices are exact integer products reduced mod M;
 *    all phase and twiddle tables are built once in FP64 and rounded.
 *  - No 1/N or 1/P normalisation (raw sums).  The SCD low-pass windows g and g_d of
 *    Sec. II are rectangular.
 *  - Pointers: every data pointer is a DEVICE pointer of the current CUDA device, aligned
 *    to 16 bytes (8 bytes for float arrays), unless an entry point says otherwise.  The
 *    caller owns all of them; the library never frees or retains them after the call.
 *    The library owns only its cached phase tables (released by scd_release_cache()).
 *  - Asynchrony: work is enqueued on opts->stream (a cudaStream_t; NULL = legacy default
 *    stream) and the call returns after enqueueing.  Argument errors are returned
 *    synchronously and enqueue nothing.  SCD_ERR_CUDA means a CUDA launch or runtime
 *    error; scd_last_error() gives its text.
 *  - First use of a size builds cached tables (device allocation plus a synchronisation);
 *    make that first call, or scd_prepare(), outside any stream capture.
 *  - window == NULL selects the symmetric Hamming window a[n] = 0.54 - 0.46 cos(2 pi n /
 *    (Np - 1)), computed in FP64 and rounded to float32.
 */
#ifndef SCD_H_
#define SCD_H_

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define SCD_API __attribute__((visibility("default")))
#else
#define SCD_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SCD_OK = 0,
  SCD_ERR_ARG = 1,          /* invalid argument (NULL pointer, bad size, misalignment) */
  SCD_ERR_UNSUPPORTED = 2,  /* valid but outside the supported sizes */
  SCD_ERR_CUDA = 3,         /* CUDA runtime or launch error */
  SCD_ERR_WORKSPACE = 4,    /* workspace missing or smaller than the query */
  SCD_ERR_TIMEOUT = 5,      /* a bounded device-side wait expired (batched runs) */
  SCD_ERR_INTERNAL = 6
} scd_status;

typedef enum { SCD_FP32 = 0, SCD_SPLIT_BF16 = 1 } scd_precision;

/* How scd_ssca schedules its stages.
 * STAGES: one kernel per stage (channeliser + CDP, column pass, row pass).
 * PERSISTENT: one persistent launch that runs the channeliser + CDP and then the column and
 *   row passes channel group by channel group through small rotating slots (so each group's
 *   intermediate is read back from L2).
 * FUSED: two kernels: the channeliser, the channel-data product and the strip transform's
 *   first pass in one (the product X_g never leaves the chip), the second pass in the other.
 *   Where its tiles do not fit the sizes (FP32 form; Np in {64, 128, 256}, N = M1 M2 with
 *   M1 = 64, 128 or 256, Np <= M2 <= 2048: N = 2^12..2^19 at Np = 64, 2^13..2^19 at
 *   Np = 128, 2^14..2^18 at Np = 256), the call runs the STAGES kernels instead.
 * AUTO: the choice scd_ssca_tune measured fastest for (N, Np, precision) on this GPU model
 *   (in this process, or from the SCD_TUNE_CACHE file); if never tuned, FUSED where it fits,
 *   else STAGES. */
typedef enum {
  SCD_SCHEDULE_AUTO = 0,
  SCD_SCHEDULE_STAGES = 1,
  SCD_SCHEDULE_PERSISTENT = 2,
  SCD_SCHEDULE_FUSED = 3
} scd_schedule;

/* Options.  Pass NULL for defaults: legacy default stream, FP32, no workspace, |S|,
 * no stage events, auto estimate.  Zero-initialise the struct before filling it. */
typedef struct {
  void* stream;             /* cudaStream_t to enqueue on */
  int32_t precision;        /* scd_precision */
  int32_t map_power;        /* maps only: 1 -> |S|, 2 -> |S|^2 */
  void* workspace;          /* device scratch owned by the caller (may be NULL if 0 needed) */
  size_t workspace_bytes;   /* its size */
  /* Optional per-kernel timing: when stage_events is non-NULL and n_stage_events is at
   * least (kernels launched by the call) + 1, event i (a cudaEvent_t, see
   * scd_events_create) is recorded on the stream just before the call's i-th kernel and
   * the next one after its last kernel.  scd_fam launches 2 kernels (channeliser, pair
   * FFT; 3 for a cross or conjugate estimate: channeliser of x, of y, pair FFT); scd_ssca 3
   * with the STAGES schedule (channeliser + CDP, column pass, row pass), 2 with FUSED
   * (channeliser + CDP + first pass, second pass) or 1 with PERSISTENT (AUTO resolves to
   * one of these); each map and profile 1. */
  void** stage_events;
  int32_t n_stage_events;
  int32_t schedule;         /* scd_ssca only: scd_schedule */
  /* Second signal of a cross estimate (Sec. II-A, Eq. II.A-SCD function correlates the
   * demodulates of x and y): complex64[N] device pointer, the same length as x, used by
   * scd_fam and scd_ssca in place of x wherever the estimate conjugates (FAM: the second
   * channeliser output; SSCA: the factor y[n] of the channel-data product, as Sec. II-C
   * describes).  NULL = the auto estimate (y = x).  Host-buffer variants: must be NULL. */
  const void* y;
  /* 1 = conjugate estimate: the second factor is not conjugated (FAM: X(p,k) Y(p,l); SSCA:
   * X_T(n,k) y[n]); it correlates x near f1 with y near f2 at alpha = f1 + f2.  Used by
   * scd_fam, scd_ssca, scd_fam_map and scd_fam_alpha_profile; 0 = the paper's estimate. */
  int32_t conjugate;
  /* Input normalisation (Algorithm 1's Framing stage normalises the input before
   * decimation; the paper does not say how): 0 = none, 1 = the consumed samples scaled to
   * mean power 1, 2 = scaled to peak magnitude 1 (an all-zero input is left as it is).  The
   * estimates are bilinear in x, so this equals S / (mean |x|^2) or S / max |x|^2; it is
   * applied by scaling the window (two small kernels before the first stage event).  scd_fam
   * and scd_ssca, auto estimate only (with opts->y: SCD_ERR_UNSUPPORTED). */
  int32_t normalise;
} scd_opts;

/* ------------------------------------------------------------------------------ FAM
 * scd_fam: FFT accumulation method, Sec. II-B (Eq. II.B-complex_demodulate_final and
 * Eq. II.B-SCD_function_FAM), framing as in Algorithm 1 (block p = x[pL .. pL+Np-1]):
 *   X(p,k)   = W_Np^{(k p L) mod Np} * sum_{n<Np} a[n] x[pL+n] W_Np^{(k n) mod Np}
 *   S(k,l,q) = sum_{p<P} X(p,k) conj(X(p,l)) W_P^{(q p) mod P}
 * alpha = (k - l)/Np + q/(P L), f = (k + l)/(2 Np).
 * Cross estimate (opts->y): X(p,l) in the product is replaced by the same demodulate of y.
 * Conjugate estimate (opts->conjugate): S(k,l,q) = sum_p X(p,k) Y(p,l) W_P^{(q p) mod P}
 * with Y = X or y's demodulate; alpha = (k + l)/Np + q/(P L), f = (k - l)/(2 Np).
 *   x       complex64[N], N >= (P-1) L + Np (later samples are ignored)
 *   Np      channels, power of two in [16, 256] (the paper's range 2^4..2^8)
 *   L       hop between blocks, 1 <= L
 *   P       blocks in [2, 16384]: a power of two, or any P <= 8192 (evaluated by Bluestein's
 *           identity: the P-point DFT as a cyclic convolution of power-of-two length
 *           M >= 2P - 1, both size-M transforms inside one CTA per channel pair)
 *   window  float32[Np] or NULL (Hamming)
 *   out     complex64[Np][Np][P], out[kh][lh][qh] = S(k, l, q), qh = q + floor(P/2) with
 *           q in [-floor(P/2), P - floor(P/2)) (for odd P the zero bin sits at (P-1)/2)
 *   opts    workspace >= scd_fam_workspace_bytes(...) bytes (covers every variant and option)
 * Errors: SCD_ERR_ARG (NULL/misaligned pointers, N too short, L < 1),
 *         SCD_ERR_UNSUPPORTED (Np or P out of range / not a power of two, precision),
 *         SCD_ERR_WORKSPACE, SCD_ERR_CUDA. */
SCD_API scd_status scd_fam(const void* x, int64_t N, int32_t Np, int32_t L, int32_t P, const float* window,
                   void* out, const scd_opts* opts);
SCD_API size_t scd_fam_workspace_bytes(int64_t N, int32_t Np, int32_t L, int32_t P, int32_t precision);

/* ------------------------------------------------------------------------------ SSCA
 * scd_ssca: strip spectral correlation analyser, Sec. II-C (Eq. Xg and
 * Eq. II.B-SSCA_auto) with the hop-1 complex demodulate of Sec. II-A
 * (Eq. II.A-complex demodulate) centred on n, x taken as 0 outside [0, N):
 *   X_T(n,k) = W_Np^{(k s) mod Np} sum_{r<Np} a[r] x[s+r] W_Np^{(k r) mod Np},  s = n - Np/2
 *   X_g(n,k) = X_T(n,k) conj(x[n])
 *   S(k,q)   = sum_{n<N} X_g(n,k) W_N^{(q n) mod N}
 * alpha = k/Np + q/N, f = (k/Np - q/N)/2.  Cross estimate (opts->y): conj(y[n]) replaces
 * conj(x[n]); conjugate estimate (opts->conjugate): y[n] (or x[n]) unconjugated, with the
 * same alpha and f (x near f_k paired with y near q/N: alpha = f_k + q/N).  The N-point transform is the decomposed
 * (four-step) FFT of Sec. III-B-1 (Eq. Chap4_2DFFT) with N = M1 M2.
 *   x       complex64[N], N in [2^12, 2^20] (Sec. III-B-2's range): a power of two, or any
 *           N <= 2^19, whose N-point transform runs by Bluestein's identity as two four-step
 *           transforms of power-of-two length M >= 2N - 1 (staged kernels only: with
 *           opts->schedule = SCD_SCHEDULE_PERSISTENT such an N gives SCD_ERR_UNSUPPORTED)
 *   Np      power of two in [16, 256]
 *   window  float32[Np] or NULL (Hamming)
 *   out     complex64[Np][N], out[kh][sh] = S(k, q), sh = q + floor(N/2) with
 *           q in [-floor(N/2), N - floor(N/2))
 *   opts    workspace >= scd_ssca_workspace_bytes(...) bytes
 * Errors as scd_fam. */
SCD_API scd_status scd_ssca(const void* x, int64_t N, int32_t Np, const float* window, void* out,
                    const scd_opts* opts);
SCD_API size_t scd_ssca_workspace_bytes(int64_t N, int32_t Np, int32_t precision);

/* ------------------------------------------------------------------------------ maps
 * scd_fam_map: places |S|^map_power of the kept FAM cells on the (f, alpha) grid.
 * Algorithm 1 (`FFT2`) keeps only the central half of every P-point output; the kept band
 * is q in [-Q, Q), Q = P L / Np (= [-P/4, P/4) at L = Np/4).  Cell (k, l, q) goes to
 *   fh = k + l + Np            (f = (fh - Np)/(2 Np))
 *   ah = (k - l) Q + q + P L   (alpha = (ah - P L)/(P L))
 * No two cells share a grid point; grid points no cell reaches are written as 0.
 * With opts->conjugate (the output of a conjugate scd_fam): fh = k - l + Np,
 * ah = (k + l) Q + q + P L; the cells with alpha < -1 (k = l = -Np/2, q < 0) are not kept.
 *   S    complex64[Np][Np][P] (scd_fam's output)
 *   map  float32[2 Np][2 P L], 16-byte aligned, fully overwritten
 * Needs P a power of two, P L divisible by Np and 2 L <= Np (else SCD_ERR_UNSUPPORTED). */
SCD_API scd_status scd_fam_map(const void* S, int32_t Np, int32_t L, int32_t P, float* map, const scd_opts* opts);

/* scd_ssca_map: places |S|^map_power of every SSCA cell on the (f, alpha) grid
 * (Sec. II-C; Sec. III-B-1's SSCA_2DFFT mapping with stored index M1 m2' + m1' = sh):
 *   ah = k N/Np + q + N                          (alpha = (ah - N)/N)
 *   fh = floor((k N/Np - q + N) / (2 N / Np))     (f = fh/Np - 1/2, bin width 1/Np)
 *   S    complex64[Np][N] (scd_ssca's output)
 *   map  float32[Np][2 N], 16-byte aligned, fully overwritten (unreached points are 0)
 * Needs N a power of two (the grid steps by N/Np per channel; else SCD_ERR_UNSUPPORTED). */
SCD_API scd_status scd_ssca_map(const void* S, int64_t N, int32_t Np, float* map, const scd_opts* opts);

/* ------------------------------------------------------------------------------ alpha profiles
 * Cycle-frequency profile: for every alpha column ah of the map above, the largest
 * |S|^map_power over f (0 where no cell lands), the feature vector that the paper's RFML
 * motivation (Sec. I) draws from the SCD.  Computed straight from S (the map itself is not
 * formed); deterministic (a max, no atomics).
 *   scd_fam_alpha_profile   S complex64[Np][Np][P]; profile float32[2 P L]; limits and
 *                           opts->conjugate as scd_fam_map
 *   scd_ssca_alpha_profile  S complex64[Np][N]; profile float32[2 N]
 * profile is a device pointer, 16-byte aligned, fully overwritten. */
SCD_API scd_status scd_fam_alpha_profile(const void* S, int32_t Np, int32_t L, int32_t P, float* profile,
                                         const scd_opts* opts);
SCD_API scd_status scd_ssca_alpha_profile(const void* S, int64_t N, int32_t Np, float* profile, const scd_opts* opts);

/* ------------------------------------------------------------------------------ batches
 * Batched form: nsig signals of uneven lengths through ONE persistent kernel launch (a
 * device work queue of per-signal stage tiles with bounded dependency waits), or the staged
 * schedule (one launch per stage and transform size over all signals; the default for SSCA
 * full estimates, see scd_batch_plan_set_schedule), captured in a CUDA graph that later runs
 * with the same buffers and stream replay.
 *   estimator  0 = FAM (Np, L), 1 = SSCA (Np; L ignored)
 *   lengths    HOST array of nsig signal lengths (samples)
 *   Np         power of two in [16, 256]; precision: scd_precision
 * Per-signal transform sizes: FAM P_i = largest power of two with (P_i - 1) L + Np <= len_i
 * (at most 8192); SSCA N_i = largest power of two <= len_i (in [2^12, 2^20]); the samples
 * beyond are not used.  A signal too short for the smallest size gives SCD_ERR_ARG.
 * The plan owns its task list and counters (device memory allocated here, freed by
 * scd_batch_plan_destroy); the caller owns the arenas. */
typedef struct scd_batch_plan scd_batch_plan;
SCD_API scd_status scd_batch_plan_create(int32_t estimator, int32_t nsig, const int64_t* lengths, int32_t Np,
                                         int32_t L, int32_t precision, scd_batch_plan** out);
/* Exact-length plan: no sample is dropped.  Per-signal sizes FAM P_i = floor((len_i - Np)/L) + 1
 * (>= 2; at most 8192 unless a power of two <= 16384) and SSCA N_i = len_i (>= 4096; at most 2^19
 * unless a power of two <= 2^20); sizes that are not powers of two run by Bluestein's identity
 * (as scd_fam / scd_ssca).  scd_batch_run then runs each signal's estimate with the
 * single-estimate kernels, one signal after the other on the stream (plain launches, no graph;
 * the workspace is the largest single estimate's, from scd_batch_query).  Full estimates only:
 * scd_batch_plan_set_output(plan, 1 or 2) and scd_batch_plan_set_schedule(plan, STAGES or
 * PERSISTENT) give SCD_ERR_UNSUPPORTED; scd_batch_tune runs once.  The tables of every size
 * are built here, so runs allocate nothing.  Errors as scd_batch_plan_create, and
 * SCD_ERR_UNSUPPORTED for sizes outside the limits above. */
SCD_API scd_status scd_batch_plan_create_exact(int32_t estimator, int32_t nsig, const int64_t* lengths, int32_t Np,
                                               int32_t L, int32_t precision, scd_batch_plan** out);
/* Layout of the arenas (any output pointer may be NULL):
 *   x_offsets[nsig+1]    signal i starts at x_arena[x_offsets[i]] (batches: it is
 *                        x_arena[x_offsets[i] .. x_offsets[i+1]); streaming windows overlap);
 *                        x_offsets[nsig] is the arena's length in samples
 *   out_offsets[nsig+1]  its estimate starts at out_arena + out_offsets[i] (complex64 elements):
 *                        FAM [Np][Np][P_i], SSCA [Np][N_i], as scd_fam / scd_ssca lay them out
 *   sizes[nsig]          P_i (FAM) or N_i (SSCA);  used_len[nsig]  samples consumed
 *   workspace_bytes      device workspace scd_batch_run needs */
SCD_API scd_status scd_batch_query(const scd_batch_plan* plan, int64_t* x_offsets, int64_t* out_offsets,
                                   int64_t* sizes, int64_t* used_len, size_t* workspace_bytes);
/* Enqueues the whole batch on `stream` (a cudaStream_t; with NULL the kernel is launched
 * directly instead of through a graph).  x_arena complex64[x_offsets[nsig]], out_arena
 * complex64[out_offsets[nsig]], window float32[Np] or NULL (Hamming), workspace as queried.
 * Runs of one plan must not overlap in time (they share the plan's counters).  A dependency
 * wait that gives up (bounded at 2 s) sets the device error word: scd_check_device() then
 * returns SCD_ERR_TIMEOUT. */
SCD_API scd_status scd_batch_run(scd_batch_plan* plan, const void* x_arena, const float* window, void* out_arena,
                                 void* workspace, void* stream);
SCD_API void scd_batch_plan_destroy(scd_batch_plan* plan);
/* A run on host buffers, for batches that arrive from and return to host memory (the paper's
 * setting of a front end that streams samples in and reads estimates out, Sec. I).  Copies the
 * input arena from host memory x_host into the device arena x_dev (x_host NULL: x_dev already
 * holds it), enqueues the run exactly as scd_batch_run (x_dev, window, out_dev, workspace, on
 * `stream`), then copies out_dev into host memory out_host (the out arena's bytes: complex64, or
 * float32 in an alpha-profile output mode) on the plan's own copy stream once the run is done.
 * Asynchronous: returns when all of it is enqueued, so a following call with another out_dev
 * computes while this call's results travel to the host; a call whose out_dev an earlier call
 * used first waits (on the device) for that call's copy.  Successive calls must use the same
 * `stream` (runs of one plan must not overlap).  scd_batch_host_wait blocks until every copy
 * this plan queued has reached host memory.  Host buffers should be page-locked
 * (scd_host_alloc) for full link bandwidth; pageable memory works but copies slower.  x_dev,
 * out_dev, out_host and x_host must stay valid until the copies are done (scd_batch_host_wait),
 * as for any asynchronous call.  The plan keeps one event per distinct out_dev (freed by
 * scd_batch_plan_destroy, which first waits for the plan's copies).  Errors as scd_batch_run
 * (its argument checks come first, so an argument error enqueues nothing); SCD_ERR_ARG for a
 * NULL x_dev, out_dev or out_host; SCD_ERR_CUDA if a copy or event call fails (message in
 * scd_last_error). */
SCD_API scd_status scd_batch_run_host(scd_batch_plan* plan, const void* x_host, void* x_dev, const float* window,
                                      void* out_dev, void* out_host, void* workspace, void* stream);
SCD_API scd_status scd_batch_host_wait(scd_batch_plan* plan);
/* Page-locked host memory (cudaHostAlloc) of `bytes` bytes, and its release; the caller owns it.
 * SCD_ERR_ARG for bytes == 0 or a NULL ptr; SCD_ERR_CUDA if the allocation is refused (message
 * in scd_last_error). */
SCD_API scd_status scd_host_alloc(size_t bytes, void** ptr);
SCD_API scd_status scd_host_free(void* ptr);
/* Output of the plan's runs: mode 0 = the estimates (default); 1 / 2 = only each signal's
 * alpha profile of |S| / |S|^2 (scd_fam_alpha_profile / scd_ssca_alpha_profile of its
 * estimate, bit for bit), reduced inside the last stage so the estimate is never written
 * (the output shrinks from Np^2 P_i or Np N_i complex values to 2 P_i L or 2 N_i floats).
 * Changes the layout: scd_batch_query then gives out_offsets in float32 elements and the
 * out arena is float32[out_offsets[nsig]], zeroed by every run.  FAM needs 2 L <= Np and
 * P_i L divisible by Np for every signal (else SCD_ERR_UNSUPPORTED). */
SCD_API scd_status scd_batch_plan_set_output(scd_batch_plan* plan, int32_t mode);
/* Schedule of a plan's full estimates (scd_schedule): SCD_SCHEDULE_PERSISTENT = the one
 * persistent launch (SSCA: column-pass output in rotating L2-sized slots);
 * SCD_SCHEDULE_STAGES = one launch per stage and transform size over all signals (the
 * channelisers, then per size class the SSCA column passes in place on the workspace and row
 * passes, or the FAM pair transforms; same workspace, no device-side waits);
 * SCD_SCHEDULE_AUTO = the autotuner's choice for this workload, else the default of new plans
 * (STAGES for SSCA, PERSISTENT for FAM).  Both schedules serve both output modes. */
SCD_API scd_status scd_batch_plan_set_schedule(scd_batch_plan* plan, int32_t schedule);

/* ------------------------------------------------------------------------------ streaming
 * Successive windows of one continuous signal (the real-time use the paper targets, Sec. I):
 * a plan over nwin windows of window_len samples, window i starting at sample i * hop of the
 * x arena (x_offsets[i] = i * hop; the arena holds span = (nwin - 1) hop + window_len
 * samples).  It is a batch plan in every other respect: scd_batch_query / run / tune /
 * destroy apply, and the run replays one captured graph as long as the buffers and stream
 * stay the same.  The windows' sizes follow the batch rules (FAM P from window_len and L,
 * SSCA N = largest power of two <= window_len).  Needs nwin * hop >= window_len - hop.
 *
 * scd_stream_advance slides the arena to the next group of nwin windows: it moves the last
 * keep = max(window_len - hop, 0) samples to the front (they belong to the next group's
 * first windows) and copies span - keep samples from `samples` behind them; both copies are
 * enqueued on `stream`.  `samples` (HOST memory if samples_on_host, else device memory)
 * holds the nwin * hop stream samples that follow the kept ones: for group k >= 1 they
 * start at stream sample k * nwin * hop + keep.  Start a stream by filling x_arena[0, span)
 * with its first span samples.  After k advances the arena holds stream samples
 * [k nwin hop, k nwin hop + span), so window i of group k is stream window k * nwin + i. */
SCD_API scd_status scd_stream_plan_create(int32_t estimator, int64_t window_len, int64_t hop, int32_t nwin,
                                          int32_t Np, int32_t L, int32_t precision, scd_batch_plan** out);
SCD_API scd_status scd_stream_advance(scd_batch_plan* plan, void* x_arena, const void* samples,
                                      int32_t samples_on_host, void* stream);

/* ------------------------------------------------------------------------------ autotuner
 * The persistent schedule has two sizing knobs: how much output one queue item covers (the
 * scheduling cost is paid once per item) and, for SSCA, how many channels one unit of the
 * column/row passes covers (the size of its rotating slot, which decides whether the
 * intermediate can stay in L2).  The autotuner times candidate settings on the caller's
 * buffers and keeps the fastest; it records the choice per (GPU model, workload) in this
 * process and, when the environment variable SCD_TUNE_CACHE names a file, in that JSON file,
 * from which later processes start.  Both calls enqueue and time real runs on `stream`
 * (the outputs hold a valid estimate afterwards) and synchronise it.
 *
 * scd_batch_tune: items of 32..512 KiB, SSCA slots of 8..64 MiB, and for full estimates the
 *   staged schedule; re-plans `plan` with the fastest setting (plans created later for the
 *   same workload start from it).
 * scd_ssca_tune: the STAGES schedule and the PERSISTENT one with the same knobs, for
 *   (N, Np, opts->precision); later SCD_SCHEDULE_AUTO calls use the fastest.  Arguments as
 *   scd_ssca (opts->workspace at least scd_ssca_workspace_bytes). */
SCD_API scd_status scd_batch_tune(scd_batch_plan* plan, const void* x_arena, const float* window, void* out_arena,
                                  void* workspace, void* stream, int32_t reps);
SCD_API scd_status scd_ssca_tune(const void* x, int64_t N, int32_t Np, const float* window, void* out,
                                 const scd_opts* opts, int32_t reps);

/* ------------------------------------------------------------------------------ host buffers
 * scd_fam_host / scd_ssca_host: the same estimates for HOST input and output buffers
 * (pinned memory gives full copy bandwidth; pageable memory works).  The call copies x
 * (and the window, if given) to the device, runs the estimator, copies the estimate
 * back and returns only when out_host holds it (the stream is synchronised).  The
 * device staging area is the caller's workspace: opts->workspace must be a device buffer
 * of at least scd_*_host_workspace_bytes(...) bytes.  Window, x and out are host
 * pointers here; errors as for the device entry points. */
SCD_API scd_status scd_fam_host(const void* x_host, int64_t N, int32_t Np, int32_t L, int32_t P,
                                const float* window_host, void* out_host, const scd_opts* opts);
SCD_API size_t scd_fam_host_workspace_bytes(int64_t N, int32_t Np, int32_t L, int32_t P, int32_t precision);
SCD_API scd_status scd_ssca_host(const void* x_host, int64_t N, int32_t Np, const float* window_host,
                                 void* out_host, const scd_opts* opts);
SCD_API size_t scd_ssca_host_workspace_bytes(int64_t N, int32_t Np, int32_t precision);

/* ------------------------------------------------------------------------------ no allocation
 * scd_fam_noalloc: scd_fam for callers that cannot allocate device memory when they run an
 * estimate (for example a real-time receive loop that forbids allocation after start-up,
 * because an allocation can synchronise the device and stall the sample stream, or a
 * plug-in that is handed device pointers for its inputs and outputs and owns no memory).
 * The paper has no counterpart to this entry point.
 * Instead of a caller workspace and the library's cached tables it uses one fixed
 * __device__ scratch array inside the library (about 2.25 MB, held by every GPU that loads
 * the library until the process exits), and calls no cudaMalloc, cudaFree or allocating
 * library routine.  Arguments, output and results are those of scd_fam (opts->workspace is
 * ignored; the same argument checks), restricted to: the FP32 form (opts->precision =
 * SCD_SPLIT_BF16 returns SCD_ERR_UNSUPPORTED); the auto estimate without normalisation
 * (opts->y, opts->conjugate or opts->normalise set: SCD_ERR_UNSUPPORTED); no per-stage timing
 * (opts->stage_events non-NULL: SCD_ERR_UNSUPPORTED); P a power of two; and Np * P <= 262144
 * (e.g. Np = 256 with P <= 1024, Np = 16 with P <= 16384).  Every rejection sets the text of
 * scd_last_error(); a size beyond the scratch names the limit.
 * All calls share the scratch array, which keeps the last call's contents (each call
 * rewrites everything it reads, so nothing has to start at zero).  Calls that overlap on the
 * same device (on different streams, or from different host threads) race on that device's
 * array and must be serialised by the caller; calls on different devices are independent.
 * The first call in a device's context resolves the array's device address (a set-up step,
 * cached per device and context); make that first call before any stream capture on that
 * device, and again after a device reset (cudaDeviceReset), which creates a new context. */
SCD_API scd_status scd_fam_noalloc(const void* x, int64_t N, int32_t Np, int32_t L, int32_t P,
                                   const float* window, void* out, const scd_opts* opts);

/* ------------------------------------------------------------------------------ timing
 * Helpers for opts->stage_events: create / destroy n CUDA events (with timing) on the
 * current device, and read the time between two recorded events (blocks until `end`
 * has completed). */
SCD_API scd_status scd_events_create(int32_t n, void** events);
SCD_API scd_status scd_events_destroy(int32_t n, void** events);
SCD_API scd_status scd_event_elapsed_ms(void* start, void* end, float* ms);
/* Records one of those events on `stream` (a cudaStream_t). */
SCD_API scd_status scd_event_record(void* event, void* stream);
/* Synchronises `stream` and reports whether a kernel of this library on the current
 * device gave up a bounded device-side wait since the last call (SCD_ERR_TIMEOUT; the
 * affected estimate is invalid); clears the record.  SCD_OK otherwise. */
SCD_API scd_status scd_check_device(void* stream);
/* Number of kernels this library has launched in this process (all devices). */
SCD_API uint64_t scd_launch_count(void);

/* ------------------------------------------------------------------------------ windows
 * scd_chebyshev_window: the Dolph-Chebyshev window that Algorithms 1 and 2 apply to the
 * channeliser input (`chebwin[Np]`), for passing as `window` to the estimators: sidelobes
 * atten_db below the main lobe (the paper gives no value; 100 dB is the customary default),
 * symmetric about (Np - 1)/2, peak 1.  Computed on the device in FP64 from the definition
 * (spectrum samples T_{Np-1}(x0 cos(pi k/Np)), x0 = cosh(acosh(10^{atten/20})/(Np-1)),
 * inverted by a cosine sum) and rounded to float32 once.
 *   Np      2 .. 256;  atten_db in (0, 300]
 *   window  float32[Np] device pointer (4-byte aligned), fully overwritten
 *   stream  cudaStream_t to enqueue on
 * Errors: SCD_ERR_ARG (NULL/misaligned window, Np or atten_db out of range), SCD_ERR_CUDA. */
SCD_API scd_status scd_chebyshev_window(int32_t Np, double atten_db, float* window, void* stream);

/* ------------------------------------------------------------------------------ misc */
/* Builds the cached tables the given sizes need (estimator 0 = FAM with (Np, P), 1 =
 * SSCA with (Np, N)), so that later calls may be captured in a CUDA graph. */
SCD_API scd_status scd_prepare(int32_t estimator, int64_t N, int32_t Np, int32_t P);
/* Frees every cached table on every device (no call may be in flight). */
SCD_API void scd_release_cache(void);
SCD_API const char* scd_status_string(scd_status s);
/* Text of the last CUDA error seen by this thread ("" if none). */
SCD_API const char* scd_last_error(void);
/* Library version as major*10000 + minor*100 + patch. */
SCD_API int32_t scd_version(void);

#ifdef __cplusplus
}
#endif

#endif /* SCD_H_ */
