// Batched form: hundreds of signals of uneven lengths through one CUDA graph per estimator,
// holding either ONE persistent launch (below) or the staged schedule's launches (one per
// stage and size class, batch_staged.cu; the SSCA default).
//
// A batch plan lists tasks (one stage of one signal: FAM channeliser / pair FFT, SSCA
// channeliser+CDP / column pass / row pass), each a range of tiles (one tile = one CTA's
// share, the same tile functions the standalone kernels run).  The persistent kernel's CTAs
// pull tile indices from a device counter in increasing order; a tile whose task depends on
// an earlier task (same signal, previous stage) first waits until every tile of that task
// has been published.  Dependencies always point to lower tile indices, and a tile is only
// pulled by a running CTA, so the schedule cannot deadlock; every wait is still bounded (2 s
// of device time), after which the tile is skipped and the device error word is set
// (scd_batch_run then returns SCD_ERR_TIMEOUT).
//
// Per-signal sizes (uneven lengths, Sec. II with power-of-two transforms):
//   FAM:  P_i = largest power of two with (P_i - 1) L + Np <= len_i, at most 8192;
//   SSCA: N_i = largest power of two <= len_i, in [2^12, 2^20];
// samples beyond those are not used.
#include <stdio.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "batch_kernel.cuh"
#include "ssca_fused.cuh"

namespace scd {
namespace bk {
int smem_of(bool fam, bool tc) {
  if (fam) return tc ? BatchSmem<true, true>::total : BatchSmem<true, false>::total;
  return tc ? BatchSmem<false, true>::total : BatchSmem<false, false>::total;
}

namespace {
template <bool FAM, bool TC>
cudaError_t prepare_one(int smem, int* blocks_per_sm) {
  cudaError_t e = cudaFuncSetAttribute(k_batch<FAM, TC, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_batch<FAM, TC, false>, kThreads, smem);
}
}  // namespace

cudaError_t prepare_kernel(bool fam, bool tc, bool prof, int smem, int* blocks_per_sm) {
  if (prof) return prepare_kernel_profile(fam, tc, smem, blocks_per_sm);
  if (fam) return tc ? prepare_one<true, true>(smem, blocks_per_sm) : prepare_one<true, false>(smem, blocks_per_sm);
  return tc ? prepare_one<false, true>(smem, blocks_per_sm) : prepare_one<false, false>(smem, blocks_per_sm);
}

cudaError_t launch_batch(bool fam, bool tc, bool prof, int grid, int smem, const BatchArgs& A, cudaStream_t st) {
  if (prof) return launch_batch_profile(fam, tc, grid, smem, A, st);
  if (fam) {
    if (tc) k_batch<true, true, false><<<grid, kThreads, smem, st>>>(A);
    else k_batch<true, false, false><<<grid, kThreads, smem, st>>>(A);
  } else {
    if (tc) k_batch<false, true, false><<<grid, kThreads, smem, st>>>(A);
    else k_batch<false, false, false><<<grid, kThreads, smem, st>>>(A);
  }
  return cudaGetLastError();
}
}  // namespace bk

using namespace bk;

namespace {

int tile_c(int M) {                       // transforms per tile for size M (256 threads)
  switch (M) {
    case 2: return TileShape<2>::C;       case 4: return TileShape<4>::C;
    case 8: return TileShape<8>::C;       case 16: return TileShape<16>::C;
    case 32: return TileShape<32>::C;     case 64: return TileShape<64>::C;
    case 128: return TileShape<128>::C;   case 256: return TileShape<256>::C;
    case 512: return TileShape<512>::C;   case 1024: return TileShape<1024>::C;
    case 2048: return TileShape<2048>::C; case 4096: return TileShape<4096>::C;
    case 8192: return TileShape<8192>::C; case 16384: return TileShape<16384>::C;
    default: return 0;
  }
}

}  // namespace
}  // namespace scd

struct scd_batch_plan {
  int estimator = 0, nsig = 0, Np = 0, L = 0, precision = 0, device = 0;
  int64_t item_bytes = scd::bk::kItemBytes;   // tunables (autotuner): output bytes per queue item,
  int64_t slot_bytes = scd::bk::kSlotBytes;   // bytes of one SSCA column-pass slot
  int staged = 0;                         // 1 = staged schedule (batch_staged.cu)
  int exact = 0;                          // 1 = exact-length plan: every sample, per-signal launches
  uint64_t signature = 0;                 // hash of (estimator, Np, L, precision, lengths)
  std::vector<int64_t> x_off, out_off, ws_off, sizes, used;
  std::vector<scd::bk::Task> tasks;
  scd::bk::Task* d_tasks = nullptr;
  // staged schedule: one task list per launch, concatenated
  struct StageLaunch { int kind, M; int first, count; int64_t total; int grid, smem; };
  std::vector<scd::bk::Task> st_tasks;
  std::vector<StageLaunch> st_launches;
  scd::bk::Task* d_st = nullptr;
  unsigned* d_counters = nullptr;
  int64_t total = 0;
  size_t ws_bytes = 0;
  int grid = 0, smem = 0;
  const float2* tw_np = nullptr;
  const unsigned char* bm_np = nullptr;
  int bbytes_np = 0;
  const float* hamming = nullptr;
  unsigned* err = nullptr;
  // cached graphs of the last two (x, window, out, workspace, stream) combinations (two, so that
  // runs alternating between two output buffers replay their graphs)
  struct Graph {
    cudaGraphExec_t exec = nullptr;
    const void* x = nullptr;
    const void* w = nullptr;
    const void* out = nullptr;
    const void* ws = nullptr;
    void* stream = nullptr;
    int drop = -1;
  };
  Graph graphs[2];
  int graph_next = 0;                     // the entry the next capture replaces
  // streaming plans (scd_stream_plan_create): window length and hop; 0 for batches
  int64_t stream_window = 0, stream_hop = 0;
  // output mode (scd_batch_plan_set_output): 0 full estimates, 1 / 2 alpha profiles of |S|^1 / |S|^2
  int prof_power = 0;
  int grid_prof = 0;                      // grid of the profile kernel (0: not prepared yet)
  // runs on host buffers (scd_batch_run_host): the device-to-host copies run on the plan's own
  // stream after the estimate; one event per output buffer marks the end of its last copy
  cudaStream_t copy_st = nullptr;
  cudaEvent_t computed = nullptr;
  std::vector<std::pair<const void*, cudaEvent_t>> copied;
};

namespace {

void drop_graphs(scd_batch_plan* p) {
  for (auto& g : p->graphs) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    g = scd_batch_plan::Graph();
  }
}

void free_plan(scd_batch_plan* p) {
  if (!p) return;
  if (p->copy_st) cudaStreamSynchronize(p->copy_st);          // copies still reading the plan's buffers
  for (auto& c : p->copied) cudaEventDestroy(c.second);
  if (p->computed) cudaEventDestroy(p->computed);
  if (p->copy_st) cudaStreamDestroy(p->copy_st);
  drop_graphs(p);
  if (p->d_tasks) cudaFree(p->d_tasks);
  if (p->d_st) cudaFree(p->d_st);
  if (p->d_counters) cudaFree(p->d_counters);
  delete p;
}

scd_status cuda_status(cudaError_t e) {
  char msg[160];
  snprintf(msg, sizeof msg, "%s: %s", cudaGetErrorName(e), cudaGetErrorString(e));
  scd::set_last_error(msg);
  return SCD_ERR_CUDA;
}

// Schedule of a new plan's full estimates (the plan's `staged`: 0 persistent, 1 staged, 2 staged
// with the fused SSCA kernels where their tiles fit): SSCA defaults to the staged schedule
// (measured faster on every batch tried: 512 signals of 2^12..2^18 samples, Np = 128: 29.0 ->
// 23.5 ms FP32, 42.0 -> 35.9 ms split), fused in the FP32 form; FAM to the persistent one.
int default_staged(int estimator, int precision) {
  return estimator == 1 ? (precision == SCD_FP32 ? 2 : 1) : 0;
}

// Output arena layout of the plan's mode: full estimates (complex64 elements: FAM Np^2 P_i,
// SSCA Np N_i per signal) or alpha profiles (float32 elements: FAM 2 P_i L, SSCA 2 N_i).
void layout_outputs(scd_batch_plan* p) {
  const bool fam = p->estimator == 0;
  const int64_t Np = p->Np;
  for (int i = 0; i < p->nsig; ++i) {
    const int64_t sz = p->sizes[i];
    const int64_t n = p->prof_power ? (fam ? 2 * sz * p->L : 2 * sz) : (fam ? Np * Np * sz : Np * sz);
    p->out_off[i + 1] = p->out_off[i] + n;
  }
}

// (Re)builds the plan's task list with its current tunables and uploads it.
scd_status build_tasks(scd_batch_plan* p) {
  using namespace scd;
  const int nsig = p->nsig, Np = p->Np;
  const bool fam = p->estimator == 0, tc = p->precision == SCD_SPLIT_BF16;
  cudaError_t e = cudaSuccess;
  p->tasks.clear();
  p->ws_bytes = sizeof(float2) * (size_t)p->ws_off[nsig];
  // Task order.  FAM: every channeliser task (tiny), then every pair task.  SSCA: software-
  // pipelined by signal (cdp_s, cols_{s-1}, rows_{s-2}, ...), so a signal's intermediate is
  // consumed soon after it is produced (small signals stay in L2) and every dependency has
  // another task queued between it and its consumer.
  const int cnp = tile_c(Np);
  std::vector<Task>& T = p->tasks;
  int64_t first = 0;
  // One queue item covers enough CTA tiles (of one task) for about kItemBytes of output, so
  // the scheduling cost (one atomic, a barrier) is spread over several tiles.
  auto add = [&](Task t) {
    const int64_t out_per_tile = t.op == OP_FAM_CHAN || t.op == OP_SSCA_CDP
                                     ? (int64_t)tile_c(Np) * Np * 8
                                     : (int64_t)tile_c(t.size) * t.size * 8;
    t.subtiles = t.tiles;
    t.per_item = (int32_t)std::max<int64_t>(1, p->item_bytes / std::max<int64_t>(1, out_per_tile));
    t.tiles = (t.subtiles + t.per_item - 1) / t.per_item;
    t.first = first;
    first += t.tiles;
    T.push_back(t);
    return (int)T.size() - 1;
  };
  auto stage0_task = [&](int i) {
    Task t{};
    t.op = fam ? OP_FAM_CHAN : OP_SSCA_CDP;
    t.size = Np;
    t.dep = -1;
    t.dep2 = -1;
    t.x_off = p->x_off[i]; t.out_off = p->out_off[i]; t.ws_off = p->ws_off[i];
    if (fam) { t.P = (int)p->sizes[i]; t.tiles = (t.P + cnp - 1) / cnp; }
    else { t.N = (int)p->sizes[i]; t.tiles = t.N / cnp; }
    return t;
  };
  std::vector<int> stage0(nsig, -1), cols_idx(nsig, -1);
  if (fam) {
    for (int i = 0; i < nsig; ++i) stage0[i] = add(stage0_task(i));
    for (int i = 0; i < nsig; ++i) {
      const int64_t sz = p->sizes[i];
      Task t = T[stage0[i]];
      t.op = OP_FAM_PAIRS; t.size = (int)sz; t.dep = stage0[i];
      const int c = tile_c((int)sz);
      t.tiles = (fam_pair_count<0>(Np, true) + c - 1) / c;      // the pairs kh <= lh (auto estimate)
      if (!(t.tw = table_pass((int)sz, &e))) { return cuda_status(e); }
      if (tc && !(t.bmats = table_tc_bmats((int)sz, &t.bbytes, &e))) { return cuda_status(e); }
      add(t);
    }
  } else {
    // SSCA: the column and row passes run per unit of G channels of one signal; a unit's
    // column-pass output goes to one of kSlots rotating slots of G*N values and is read by
    // the unit's row pass right away, so it can stay in L2.  Order: cdp_0, then per signal s:
    // cdp_{s+1}, then (cols_u, rows_u) for the units of s.  cols_u waits for the signal's cdp
    // and for rows_{u - kSlots} (the previous user of its slot).
    std::vector<int> rows_task;                                 // per unit, in order
    auto units_of = [&](int64_t N) {
      int G = Np;
      while (G > 1 && (int64_t)G * N * 8 > p->slot_bytes) G >>= 1;
      return G;
    };
    int64_t slot_elems = 0;                                     // sized for the largest tunable slot
    for (int i = 0; i < nsig; ++i) slot_elems = std::max<int64_t>(slot_elems, slot_group(Np, p->sizes[i], kSlotBytesMax) * p->sizes[i]);
    const int64_t slots_off = p->ws_off[nsig];
    p->ws_bytes = sizeof(float2) * (size_t)(slots_off + kSlots * slot_elems);
    // units in signal order; rows passes lag the column passes by one unit so that no row
    // pass is queued right behind the column pass it waits for
    struct Unit { int sig, ch0, G; };
    std::vector<Unit> units;
    for (int i = 0; i < nsig; ++i) {
      const int G = units_of(p->sizes[i]);
      for (int g = 0; g < Np / G; ++g) units.push_back({i, g * G, G});
    }
    const int U = (int)units.size();
    std::vector<Task> cols_t(U), rows_t(U);
    std::vector<int> cols_idx(U, -1);
    rows_task.assign(U, -1);
    for (int u = 0; u < U; ++u) {
      const int i = units[u].sig, G = units[u].G;
      const int64_t sz = p->sizes[i];
      int M1, M2;
      ssca_split(sz, &M1, &M2);
      Task c1 = stage0_task(i);
      c1.op = OP_SSCA_COLS; c1.size = M1; c1.M1 = M1; c1.M2 = M2; c1.ch0 = units[u].ch0;
      c1.tiles = (int64_t)G * (M2 / tile_c(M1));
      c1.mid_off = slots_off + (int64_t)(u % kSlots) * slot_elems;
      if (!(c1.tw = table_pass(M1, &e)) || !(c1.wN = table_roots((int)sz, &e)) ||
          !(c1.cols = table_cols((int)sz, M1, tile_c(M1), &e)))
        return cuda_status(e);
      if (tc && !(c1.bmats = table_tc_bmats(M1, &c1.bbytes, &e))) { return cuda_status(e); }
      Task r = c1;
      r.op = OP_SSCA_ROWS; r.size = M2;
      r.tiles = (int64_t)G * (M1 / tile_c(M2));
      r.wN = nullptr; r.cols = nullptr; r.bmats = nullptr; r.bbytes = 0;
      if (!(r.tw = table_pass(M2, &e))) { return cuda_status(e); }
      if (tc && !(r.bmats = table_tc_bmats(M2, &r.bbytes, &e))) { return cuda_status(e); }
      cols_t[u] = c1;
      rows_t[u] = r;
    }
    int next_cdp = 0;
    auto emit_cdp = [&]() { stage0[next_cdp] = add(stage0_task(next_cdp)); ++next_cdp; };
    if (nsig > 0) emit_cdp();
    for (int j = 0; j <= U; ++j) {
      if (j < U) {
        const int i = units[j].sig;
        if (next_cdp == i + 1 && next_cdp < nsig) emit_cdp();     // one signal's channeliser ahead
        Task c1 = cols_t[j];
        c1.dep = stage0[i];
        c1.dep2 = j >= kSlots ? rows_task[j - kSlots] : -1;    // previous user of the slot
        cols_idx[j] = add(c1);
      }
      if (j >= 1) {
        Task r = rows_t[j - 1];
        r.dep = cols_idx[j - 1];
        r.dep2 = -1;
        rows_task[j - 1] = add(r);
      }
    }
  }
  p->total = first;
  if (p->total >= (int64_t)0xFFFFFFF0u) return SCD_ERR_UNSUPPORTED;
  drop_graphs(p);
  if (p->d_st) { cudaFree(p->d_st); p->d_st = nullptr; }
  p->st_tasks.clear();
  p->st_launches.clear();
  if (p->staged) {
    // staged schedule: every signal's channeliser, then per size class (ascending N or P) the
    // SSCA column passes and row passes, or the FAM pair transforms, of its signals
    int sms = 0;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device)) != cudaSuccess)
      return cuda_status(e);
    auto launch_of = [&](int kind, int M, int first_task) -> scd_status {
      scd_batch_plan::StageLaunch L{kind, M, first_task, (int)p->st_tasks.size() - first_task, 0, 0, 0};
      if (L.count == 0) return SCD_OK;
      int64_t tiles = 0;
      for (int i = first_task; i < (int)p->st_tasks.size(); ++i) {
        p->st_tasks[i].first = tiles;
        tiles += p->st_tasks[i].subtiles;
      }
      L.total = tiles;
      int per_sm = 0;
      cudaError_t ee = staged_prepare(kind, M, Np, tc, &L.smem, &per_sm);
      if (ee != cudaSuccess) return cuda_status(ee);
      if (tiles >= (int64_t)0x7FFFFFFF) return SCD_ERR_UNSUPPORTED;
      L.grid = (int)tiles;                                      // one CTA per tile
      p->st_launches.push_back(L);
      return SCD_OK;
    };
    // fused SSCA kernels (staged == 2, FP32 form) for the size classes their tiles fit
    const bool fused = !fam && !tc && p->staged == 2;
    auto fused_n = [&](int64_t N, FusedSplit* fs) { return fused && fused_split(N, Np, fs); };
    int f0 = 0;
    for (int i = 0; i < nsig; ++i) {
      FusedSplit fs;
      if (fused_n(p->sizes[i], &fs)) continue;                  // its channeliser runs inside tile A
      Task t = stage0_task(i);
      t.subtiles = t.tiles;
      p->st_tasks.push_back(t);
    }
    scd_status ls = launch_of(fam ? 3 : 0, Np, f0);
    if (ls != SCD_OK) return ls;
    std::vector<int64_t> classes(p->sizes.begin(), p->sizes.end());
    std::sort(classes.begin(), classes.end());
    classes.erase(std::unique(classes.begin(), classes.end()), classes.end());
    for (int64_t P : fam ? classes : std::vector<int64_t>()) {
      f0 = (int)p->st_tasks.size();
      for (int i = 0; i < nsig; ++i) {
        if (p->sizes[i] != P) continue;
        Task t = stage0_task(i);
        t.size = (int)P;
        t.subtiles = (fam_pair_count<0>(Np, true) + tile_c((int)P) - 1) / tile_c((int)P);   // pairs kh <= lh
        if (!(t.tw = table_pass((int)P, &e))) return cuda_status(e);
        if (tc && !(t.bmats = table_tc_bmats((int)P, &t.bbytes, &e))) return cuda_status(e);
        p->st_tasks.push_back(t);
      }
      if ((ls = launch_of(p->prof_power ? 6 : 4, (int)P, f0)) != SCD_OK) return ls;
    }
    for (int64_t N : fam ? std::vector<int64_t>() : classes) {
      FusedSplit fs;
      if (fused_n(N, &fs)) {
        // tile A (kind 7, clusters of fs.Q CTAs), then tile B (kind 8; 9 reduces into profiles)
        for (int kind = 7; kind <= 8; ++kind) {
          f0 = (int)p->st_tasks.size();
          for (int i = 0; i < nsig; ++i) {
            if (p->sizes[i] != N) continue;
            Task t = stage0_task(i);
            t.M1 = fs.M1; t.M2 = fs.M2;
            t.size = kind == 7 ? fs.M1 : fs.M2;
            t.subtiles = kind == 7 ? (int64_t)fs.M2 * fs.Q : (int64_t)Np * (fs.M1 / rowsf_c(fs.M2));
            if (!(t.tw = table_pass(t.size, &e))) return cuda_status(e);
            if (kind == 7 && !(t.wN = table_roots((int)N, &e))) return cuda_status(e);
            p->st_tasks.push_back(t);
          }
          if ((ls = launch_of(kind == 8 && p->prof_power ? 9 : kind, kind == 7 ? (int)N : fs.M2, f0)) != SCD_OK)
            return ls;
        }
        continue;
      }
      int M1, M2;
      ssca_split(N, &M1, &M2);
      for (int kind = 1; kind <= 2; ++kind) {
        const int M = kind == 1 ? M1 : M2;
        f0 = (int)p->st_tasks.size();
        for (int i = 0; i < nsig; ++i) {
          if (p->sizes[i] != N) continue;
          Task t = stage0_task(i);
          t.M1 = M1; t.M2 = M2; t.size = M;
          t.subtiles = kind == 1 ? (int64_t)Np * (M2 / tile_c(M1)) : (int64_t)Np * (M1 / tile_c(M2));
          if (!(t.tw = table_pass(M, &e))) return cuda_status(e);
          if (kind == 1 && (!(t.wN = table_roots((int)N, &e)) || !(t.cols = table_cols((int)N, M1, tile_c(M1), &e))))
            return cuda_status(e);
          if (tc && !(t.bmats = table_tc_bmats(M, &t.bbytes, &e))) return cuda_status(e);
          p->st_tasks.push_back(t);
        }
        if ((ls = launch_of(kind == 2 && p->prof_power ? 5 : kind, M, f0)) != SCD_OK) return ls;
      }
    }
    if ((e = cudaMalloc(&p->d_st, sizeof(Task) * p->st_tasks.size())) != cudaSuccess ||
        (e = cudaMemcpy(p->d_st, p->st_tasks.data(), sizeof(Task) * p->st_tasks.size(), cudaMemcpyHostToDevice)) !=
            cudaSuccess)
      return cuda_status(e);
  }
  if (p->d_tasks) { cudaFree(p->d_tasks); p->d_tasks = nullptr; }
  if (p->d_counters) { cudaFree(p->d_counters); p->d_counters = nullptr; }
  if ((e = cudaMalloc(&p->d_tasks, sizeof(Task) * T.size())) != cudaSuccess ||
      (e = cudaMemcpy(p->d_tasks, T.data(), sizeof(Task) * T.size(), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMalloc(&p->d_counters, sizeof(unsigned) * (T.size() + 1))) != cudaSuccess)
    return cuda_status(e);
  return SCD_OK;
}

std::string batch_key(const scd_batch_plan* p) {
  char buf[128];
  snprintf(buf, sizeof buf, "|batch|est=%d|Np=%d|L=%d|p=%d|n=%d|h=%016llx", p->estimator, p->Np, p->L, p->precision,
           p->nsig, (unsigned long long)p->signature);
  return scd::device_key() + buf;
}

// Times `run` (already enqueued work of one candidate) on the stream: one warm-up, then reps.
template <class Run>
scd_status time_candidate(cudaStream_t st, int reps, Run run, float* ms) {
  cudaEvent_t a, b;
  cudaError_t e;
  if ((e = cudaEventCreate(&a)) != cudaSuccess) return cuda_status(e);
  if ((e = cudaEventCreate(&b)) != cudaSuccess) { cudaEventDestroy(a); return cuda_status(e); }
  scd_status s = run();
  if (s == SCD_OK) {
    cudaEventRecord(a, st);
    for (int r = 0; r < reps && s == SCD_OK; ++r) s = run();
    cudaEventRecord(b, st);
    if ((e = cudaEventSynchronize(b)) != cudaSuccess) s = cuda_status(e);
    else if ((e = cudaEventElapsedTime(ms, a, b)) != cudaSuccess) s = cuda_status(e);
    else *ms /= reps;
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return s;
}

// Plan over nsig signals: signal i has lengths[i] samples starting at starts[i] of the x arena
// (starts == nullptr: packed back to back); the arena holds `span` samples (0: the sum).
scd_status plan_create(int32_t estimator, int32_t nsig, const int64_t* lengths, const int64_t* starts, int64_t span,
                       int32_t Np, int32_t L, int32_t precision, scd_batch_plan** out) {
  using namespace scd;
  if (!out || !lengths || nsig < 1 || (estimator != 0 && estimator != 1)) return SCD_ERR_ARG;
  *out = nullptr;
  if (Np < 16 || Np > 256 || !is_pow2(Np)) return SCD_ERR_UNSUPPORTED;
  if (estimator == 0 && L < 1) return SCD_ERR_ARG;
  if (precision != SCD_FP32 && precision != SCD_SPLIT_BF16) return SCD_ERR_UNSUPPORTED;
  const bool fam = estimator == 0, tc = precision == SCD_SPLIT_BF16;
  scd_batch_plan* p = new scd_batch_plan();
  p->estimator = estimator; p->nsig = nsig; p->Np = Np; p->L = L; p->precision = precision;
  p->staged = default_staged(estimator, precision);
  cudaError_t e = cudaGetDevice(&p->device);
  if (e != cudaSuccess) { free_plan(p); return cuda_status(e); }
  p->x_off.assign(nsig + 1, 0); p->out_off.assign(nsig + 1, 0); p->ws_off.assign(nsig + 1, 0);
  p->sizes.assign(nsig, 0); p->used.assign(nsig, 0);
  for (int i = 0; i < nsig; ++i) {
    const int64_t len = lengths[i];
    if (len < 1) { free_plan(p); return SCD_ERR_ARG; }
    int64_t sz = 0, used = 0;
    if (fam) {
      for (int64_t P = 8192; P >= 2; P >>= 1)
        if ((P - 1) * L + Np <= len) { sz = P; break; }
      used = (sz - 1) * L + Np;
    } else {
      for (int64_t n = 1 << 20; n >= 4096; n >>= 1)
        if (n <= len) { sz = n; break; }
      used = sz;
    }
    if (!sz) { free_plan(p); return SCD_ERR_ARG; }               // signal too short
    p->sizes[i] = sz;
    p->used[i] = used;
    if (starts) p->x_off[i] = starts[i];
    p->x_off[i + 1] = starts ? span : p->x_off[i] + len;
    p->ws_off[i + 1] = p->ws_off[i] + (int64_t)Np * sz;
  }
  layout_outputs(p);
  // tables
  if (!(p->tw_np = table_pass(Np, &e)) || !(p->hamming = table_hamming(Np, &e)) ||
      !(p->err = device_error_word(&e))) {
    free_plan(p);
    return cuda_status(e);
  }
  if (tc && !(p->bm_np = table_tc_bmats(Np, &p->bbytes_np, &e))) { free_plan(p); return cuda_status(e); }
  {
    uint64_t h = 1469598103934665603ull;                       // FNV-1a over the workload
    auto mix = [&](int64_t v) { for (int b = 0; b < 8; ++b) { h ^= (uint64_t)((v >> (8 * b)) & 0xFF); h *= 1099511628211ull; } };
    mix(estimator); mix(Np); mix(L); mix(precision); mix(nsig);
    for (int i = 0; i < nsig; ++i) mix(lengths[i]);
    if (starts) { mix(span); for (int i = 0; i < nsig; ++i) mix(starts[i]); }
    p->signature = h;
    TuneEntry te;
    if (tune_lookup(batch_key(p), &te)) {
      p->item_bytes = te.item_bytes;
      p->slot_bytes = te.slot_bytes;
      p->staged = te.schedule;
    }
    scd_status bs = build_tasks(p);
    if (bs != SCD_OK) { free_plan(p); return bs; }
  }
  p->smem = smem_of(fam, tc);
  int per_sm = 0;
  e = prepare_kernel(fam, tc, false, p->smem, &per_sm);
  if (e != cudaSuccess) { free_plan(p); return cuda_status(e); }
  int sms = 0;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device)) != cudaSuccess) {
    free_plan(p);
    return cuda_status(e);
  }
  if (tc && per_sm > 4) per_sm = 4;                              // 4 x 128 TMEM columns per SM
  // The occupancy query answers one CTA per SM for the kernels that allocate tensor memory,
  // whatever their size; registers (128 x 256) and shared memory allow two, two CTAs of 128
  // TMEM columns each fit in the SM's 512, and measured they do run two per SM (the split
  // batch runs 1.5x faster).  A CTA that is not resident claims no work, so launching more
  // CTAs than fit can never stall the queue.
  if (tc && per_sm < 2) per_sm = 2;
  p->grid = sms * (per_sm > 0 ? per_sm : 1);
  *out = p;
  return SCD_OK;
}
// Task lists and launches of an exact-length plan (batch_exact.cu describes the stages).
scd_status build_exact(scd_batch_plan* p) {
  using namespace scd;
  const int nsig = p->nsig, Np = p->Np;
  const bool fam = p->estimator == 0, tc = p->precision == SCD_SPLIT_BF16;
  cudaError_t e;
  p->st_tasks.clear();
  p->st_launches.clear();
  auto launch_of = [&](int kind, int M, int first_task) -> scd_status {
    scd_batch_plan::StageLaunch L{kind, M, first_task, (int)p->st_tasks.size() - first_task, 0, 0, 0};
    if (L.count == 0) return SCD_OK;
    int64_t tiles = 0;
    for (int i = first_task; i < (int)p->st_tasks.size(); ++i) {
      p->st_tasks[i].first = tiles;
      tiles += p->st_tasks[i].subtiles;
    }
    L.total = tiles;
    int per_sm = 0;
    cudaError_t ee = staged_prepare(kind, M, Np, tc, &L.smem, &per_sm);
    if (ee != cudaSuccess) return cuda_status(ee);
    if (tiles < 1) return SCD_ERR_INTERNAL;
    if (tiles >= (int64_t)0x7FFFFFFF) return SCD_ERR_UNSUPPORTED;
    L.grid = (int)tiles;
    p->st_launches.push_back(L);
    return SCD_OK;
  };
  auto base_task = [&](int i) {
    Task t{};
    t.dep = -1;
    t.dep2 = -1;
    t.x_off = p->x_off[i];
    t.out_off = p->out_off[i];
    return t;
  };
  const int cnp = tile_c(Np);
  int64_t off = 0;                                              // workspace elements
  auto take = [&](int64_t n) { const int64_t o = off; off += (n + 31) / 32 * 32; return o; };
  std::vector<int64_t> ws(nsig), xp(nsig), padded(nsig), cyc(nsig);
  scd_status ls;
  if (fam) {
    // channelisers of every signal (X_i: Np x P_i), then per size class the pair transforms
    int f0 = 0;
    for (int i = 0; i < nsig; ++i) {
      Task t = base_task(i);
      t.P = (int)p->sizes[i];
      t.ws_off = ws[i] = take((int64_t)Np * t.P);
      t.subtiles = (t.P + cnp - 1) / cnp;
      p->st_tasks.push_back(t);
    }
    if ((ls = launch_of(3, Np, f0)) != SCD_OK) return ls;
    std::vector<int64_t> classes;
    for (int i = 0; i < nsig; ++i) classes.push_back(is_pow2(p->sizes[i]) ? p->sizes[i] : -bluestein_len_host(p->sizes[i]));
    std::sort(classes.begin(), classes.end());
    classes.erase(std::unique(classes.begin(), classes.end()), classes.end());
    for (int64_t cls : classes) {                                 // > 0: power of two P; < 0: cyclic length
      const int M = (int)(cls > 0 ? cls : -cls);
      f0 = (int)p->st_tasks.size();
      for (int i = 0; i < nsig; ++i) {
        const int64_t P = p->sizes[i];
        const bool mine = cls > 0 ? P == cls : (!is_pow2(P) && bluestein_len_host(P) == M);
        if (!mine) continue;
        Task t = base_task(i);
        t.P = (int)P;
        t.size = M;
        t.ws_off = ws[i];
        t.subtiles = (fam_pair_count<0>(Np, true) + tile_c(M) - 1) / tile_c(M);   // pairs kh <= lh
        if (!(t.tw = table_pass(M, &e))) return cuda_status(e);
        if (cls < 0 && (!(t.chirp = table_chirp(P, &e)) || !(t.bh = table_bluestein(P, M, &e)))) return cuda_status(e);
        if (tc && !(t.bmats = table_tc_bmats(M, &t.bbytes, &e))) return cuda_status(e);
        p->st_tasks.push_back(t);
      }
      if ((ls = launch_of(cls > 0 ? 4 : 14, M, f0)) != SCD_OK) return ls;
    }
  } else {
    for (int i = 0; i < nsig; ++i) {
      const int64_t N = p->sizes[i];
      if (is_pow2(N)) {
        padded[i] = N;
        cyc[i] = N;
        xp[i] = -1;
        ws[i] = take((int64_t)Np * N);
      } else {
        padded[i] = (N + cnp - 1) / cnp * cnp;
        cyc[i] = bluestein_len_host(N);
        xp[i] = take(2 * padded[i]);                            // xp then yp, padded[i] apart
        ws[i] = take((int64_t)Np * cyc[i]);
      }
    }
    // kind 10: padded inputs with the chirp folded into the second factor
    int f0 = (int)p->st_tasks.size();
    for (int i = 0; i < nsig; ++i) {
      if (xp[i] < 0) continue;
      Task t = base_task(i);
      t.N = (int)p->sizes[i];
      t.P = (int)padded[i];
      t.xp_off = xp[i];
      t.yp_off = xp[i] + padded[i];
      t.subtiles = (padded[i] + exact_prep_per_tile() - 1) / exact_prep_per_tile();
      if (!(t.chirp = table_chirp(t.N, &e))) return cuda_status(e);
      p->st_tasks.push_back(t);
    }
    if ((ls = launch_of(10, 0, f0)) != SCD_OK) return ls;
    // kind 0: every signal's channeliser + CDP (rows of the cyclic length for Bluestein signals)
    f0 = (int)p->st_tasks.size();
    for (int i = 0; i < nsig; ++i) {
      Task t = base_task(i);
      t.N = (int)padded[i];
      t.ws_off = ws[i];
      if (xp[i] >= 0) {
        t.in_ws = 1;
        t.xp_off = xp[i];
        t.yp_off = xp[i] + padded[i];
        t.ld = cyc[i];
      }
      t.subtiles = padded[i] / cnp;
      p->st_tasks.push_back(t);
    }
    if ((ls = launch_of(0, Np, f0)) != SCD_OK) return ls;
    // per transform size: the staged column and row passes (powers of two) or the three
    // Bluestein passes (cyclic lengths)
    std::vector<int64_t> classes;
    for (int i = 0; i < nsig; ++i) classes.push_back(xp[i] < 0 ? p->sizes[i] : -cyc[i]);
    std::sort(classes.begin(), classes.end());
    classes.erase(std::unique(classes.begin(), classes.end()), classes.end());
    for (int64_t cls : classes) {
      const int64_t M = cls > 0 ? cls : -cls;
      int M1, M2;
      ssca_split(M, &M1, &M2);
      const int kinds_pow2[] = {1, 2}, kinds_bl[] = {11, 12, 13};
      const int* kinds = cls > 0 ? kinds_pow2 : kinds_bl;
      const int nk = cls > 0 ? 2 : 3;
      for (int ki = 0; ki < nk; ++ki) {
        const int kind = kinds[ki];
        const int size = (kind == 2 || kind == 12) ? M2 : M1;
        f0 = (int)p->st_tasks.size();
        for (int i = 0; i < nsig; ++i) {
          const bool mine = cls > 0 ? (xp[i] < 0 && p->sizes[i] == cls) : (xp[i] >= 0 && cyc[i] == M);
          if (!mine) continue;
          Task t = base_task(i);
          t.N = (int)p->sizes[i];
          t.P = (int)padded[i];
          t.M1 = M1; t.M2 = M2; t.size = size;
          t.ws_off = ws[i];
          t.subtiles = (kind == 2 || kind == 12) ? (int64_t)Np * (M1 / tile_c(M2)) : (int64_t)Np * (M2 / tile_c(M1));
          if (!(t.tw = table_pass(size, &e))) return cuda_status(e);
          if ((kind == 1 || kind == 11 || kind == 13) &&
              (!(t.wN = table_roots((int)M, &e)) || !(t.cols = table_cols((int)M, M1, tile_c(M1), &e))))
            return cuda_status(e);
          if (kind == 12 && !(t.bh = table_bluestein_rows(t.N, M, M1, &e))) return cuda_status(e);
          if (kind == 13 && !(t.chirp = table_chirp(t.N, &e))) return cuda_status(e);
          if (tc && !(t.bmats = table_tc_bmats(size, &t.bbytes, &e))) return cuda_status(e);
          p->st_tasks.push_back(t);
        }
        if ((ls = launch_of(kind, size, f0)) != SCD_OK) return ls;
      }
    }
  }
  p->ws_bytes = sizeof(float2) * (size_t)off;
  if ((e = cudaMalloc(&p->d_st, sizeof(Task) * p->st_tasks.size())) != cudaSuccess ||
      (e = cudaMemcpy(p->d_st, p->st_tasks.data(), sizeof(Task) * p->st_tasks.size(), cudaMemcpyHostToDevice)) !=
          cudaSuccess)
    return cuda_status(e);
  if ((e = cudaMalloc(&p->d_counters, sizeof(unsigned))) != cudaSuccess) return cuda_status(e);
  return SCD_OK;
}

// Exact-length plan: every signal's estimate at the sizes its length gives (FAM P_i =
// floor((len_i - Np)/L) + 1, SSCA N_i = len_i), run with the single-estimate kernels (Bluestein's
// identity for the sizes that are not powers of two) one signal after the other on the stream.
scd_status plan_create_exact(int32_t estimator, int32_t nsig, const int64_t* lengths, int32_t Np, int32_t L,
                             int32_t precision, scd_batch_plan** out) {
  using namespace scd;
  if (!out || !lengths || nsig < 1 || (estimator != 0 && estimator != 1)) return SCD_ERR_ARG;
  *out = nullptr;
  if (Np < 16 || Np > 256 || !is_pow2(Np)) return SCD_ERR_UNSUPPORTED;
  if (estimator == 0 && L < 1) return SCD_ERR_ARG;
  if (precision != SCD_FP32 && precision != SCD_SPLIT_BF16) return SCD_ERR_UNSUPPORTED;
  const bool fam = estimator == 0;
  scd_batch_plan* p = new scd_batch_plan();
  p->estimator = estimator; p->nsig = nsig; p->Np = Np; p->L = L; p->precision = precision;
  p->exact = 1;
  cudaError_t e = cudaGetDevice(&p->device);
  if (e != cudaSuccess) { free_plan(p); return cuda_status(e); }
  p->x_off.assign(nsig + 1, 0); p->out_off.assign(nsig + 1, 0); p->ws_off.assign(nsig + 1, 0);
  p->sizes.assign(nsig, 0); p->used.assign(nsig, 0);
  for (int i = 0; i < nsig; ++i) {
    const int64_t len = lengths[i];
    if (len < 1) { free_plan(p); return SCD_ERR_ARG; }
    int64_t sz;
    if (fam) {
      if (len < Np + L) { free_plan(p); return SCD_ERR_ARG; }   // at least two blocks
      sz = (len - Np) / L + 1;
      if (sz > 16384 || (!is_pow2(sz) && sz > 8192)) { free_plan(p); return SCD_ERR_UNSUPPORTED; }
      p->used[i] = (sz - 1) * L + Np;
    } else {
      sz = len;
      if (sz < 4096) { free_plan(p); return SCD_ERR_ARG; }
      if (sz > (1 << 20) || (!is_pow2(sz) && sz > (1 << 19))) { free_plan(p); return SCD_ERR_UNSUPPORTED; }
      p->used[i] = sz;
    }
    p->sizes[i] = sz;
    p->x_off[i + 1] = p->x_off[i] + len;
    // the tables of this size, built now (runs then allocate nothing)
    const scd_status ps = scd_prepare(estimator, sz, Np, fam ? (int32_t)sz : 0);
    if (ps != SCD_OK) { free_plan(p); return ps; }
  }
  layout_outputs(p);
  if (!(p->hamming = table_hamming(Np, &e)) || !(p->err = device_error_word(&e)) ||
      !(p->tw_np = table_pass(Np, &e))) {
    free_plan(p);
    return cuda_status(e);
  }
  if (precision == SCD_SPLIT_BF16 && !(p->bm_np = table_tc_bmats(Np, &p->bbytes_np, &e))) {
    free_plan(p);
    return cuda_status(e);
  }
  const scd_status bs = build_exact(p);
  if (bs != SCD_OK) { free_plan(p); return bs; }
  *out = p;
  return SCD_OK;
}

}  // namespace

extern "C" {

scd_status scd_batch_plan_create_exact(int32_t estimator, int32_t nsig, const int64_t* lengths, int32_t Np,
                                       int32_t L, int32_t precision, scd_batch_plan** out) {
  return plan_create_exact(estimator, nsig, lengths, Np, L, precision, out);
}

scd_status scd_batch_plan_create(int32_t estimator, int32_t nsig, const int64_t* lengths, int32_t Np, int32_t L,
                                 int32_t precision, scd_batch_plan** out) {
  return plan_create(estimator, nsig, lengths, nullptr, 0, Np, L, precision, out);
}

scd_status scd_stream_plan_create(int32_t estimator, int64_t window_len, int64_t hop, int32_t nwin, int32_t Np,
                                  int32_t L, int32_t precision, scd_batch_plan** out) {
  if (!out || window_len < 1 || hop < 1 || nwin < 1) return SCD_ERR_ARG;
  // the overlap kept between groups must not overlap the part it is copied from
  if (window_len > hop && (int64_t)nwin * hop < window_len - hop) return SCD_ERR_ARG;
  std::vector<int64_t> lengths((size_t)nwin, window_len), starts((size_t)nwin);
  for (int i = 0; i < nwin; ++i) starts[i] = (int64_t)i * hop;
  const int64_t span = (int64_t)(nwin - 1) * hop + window_len;
  scd_status s = plan_create(estimator, nwin, lengths.data(), starts.data(), span, Np, L, precision, out);
  if (s == SCD_OK) {
    (*out)->stream_window = window_len;
    (*out)->stream_hop = hop;
  }
  return s;
}

scd_status scd_stream_advance(scd_batch_plan* p, void* x_arena, const void* samples, int32_t samples_on_host,
                              void* stream) {
  using namespace scd;
  if (!p || !x_arena || !samples || !p->stream_hop || ((uintptr_t)x_arena % 8)) return SCD_ERR_ARG;
  const int64_t W = p->stream_window, H = p->stream_hop, span = p->x_off[p->nsig];
  const int64_t keep = W > H ? W - H : 0;                       // samples shared with the next group
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e;
  float2* xa = (float2*)x_arena;
  if (keep && (e = cudaMemcpyAsync(xa, xa + (span - keep), sizeof(float2) * (size_t)keep, cudaMemcpyDeviceToDevice,
                                   st)) != cudaSuccess)
    return cuda_status(e);
  e = cudaMemcpyAsync(xa + keep, samples, sizeof(float2) * (size_t)(span - keep),
                      samples_on_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, st);
  return e == cudaSuccess ? SCD_OK : cuda_status(e);
}

scd_status scd_batch_query(const scd_batch_plan* p, int64_t* x_offsets, int64_t* out_offsets, int64_t* sizes,
                           int64_t* used_len, size_t* workspace_bytes) {
  if (!p) return SCD_ERR_ARG;
  for (int i = 0; i <= p->nsig; ++i) {
    if (x_offsets) x_offsets[i] = p->x_off[i];
    if (out_offsets) out_offsets[i] = p->out_off[i];
    if (i < p->nsig) {
      if (sizes) sizes[i] = p->sizes[i];
      if (used_len) used_len[i] = p->used[i];
    }
  }
  if (workspace_bytes) *workspace_bytes = p->ws_bytes;
  return SCD_OK;
}

scd_status scd_batch_run(scd_batch_plan* p, const void* x_arena, const float* window, void* out_arena, void* workspace,
                         void* stream) {
  using namespace scd;
  NvtxRange range("scd_batch_run");
  if (!p || !x_arena || !out_arena || !workspace) return SCD_ERR_ARG;
  if (((uintptr_t)x_arena % 8) || ((uintptr_t)out_arena % 16) || ((uintptr_t)workspace % 16) ||
      (window && ((uintptr_t)window % 4)))
    return SCD_ERR_ARG;
  if (fault_host("batch_run")) return SCD_ERR_CUDA;
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_status(e);
  if (dev != p->device) return SCD_ERR_ARG;
  const float* w = window ? window : p->hamming;
  cudaStream_t st = (cudaStream_t)stream;
  BatchArgs A;
  A.tasks = p->d_tasks; A.ntasks = (int)p->tasks.size(); A.Np = p->Np; A.L = p->L; A.total = p->total;
  A.counters = p->d_counters; A.x = (const float2*)x_arena; A.y = A.x; A.conj = 0; A.pad_ = 0;
  A.out = (float2*)out_arena; A.ws = (float2*)workspace;
  A.window = w; A.tw_np = p->tw_np; A.bmats_np = p->bm_np; A.bbytes_np = p->bbytes_np; A.err = p->err;
  A.prof_power = p->prof_power;
  A.drop_task = fault_batch_drop();
  const bool fam = p->estimator == 0, tc = p->precision == SCD_SPLIT_BF16, prof = p->prof_power != 0;
  const int grid = prof ? p->grid_prof : p->grid;
  const size_t cbytes = sizeof(unsigned) * (p->tasks.size() + 1);
  // profiles are maxima of non-negative values: they start from 0 on every run
  const size_t pbytes = prof ? sizeof(float) * (size_t)p->out_off[p->nsig] : 0;
  const bool staged = !p->st_launches.empty();
  auto launch_all = [&]() -> cudaError_t {
    if (!staged) return launch_batch(fam, tc, prof, grid, p->smem, A, st);
    for (const auto& L : p->st_launches) {
      cudaError_t el =
          staged_launch(L.kind, L.M, p->Np, tc, L.grid, L.smem, A, p->d_st + L.first, L.count, L.total, st);
      if (el != cudaSuccess) return el;
    }
    return cudaSuccess;
  };
  count_launches(staged ? (int)p->st_launches.size() : 1);
  if (!st) {                                                    // legacy stream: no capture, plain launch
    if ((e = cudaMemsetAsync(p->d_counters, 0, cbytes, st)) != cudaSuccess) return cuda_status(e);
    if (prof && (e = cudaMemsetAsync(out_arena, 0, pbytes, st)) != cudaSuccess) return cuda_status(e);
    e = launch_all();
    return e == cudaSuccess ? SCD_OK : cuda_status(e);
  }
  scd_batch_plan::Graph* gr = nullptr;
  for (auto& c : p->graphs)
    if (c.exec && c.x == x_arena && c.w == (const void*)w && c.out == out_arena && c.ws == workspace &&
        c.stream == stream && c.drop == A.drop_task)
      gr = &c;
  if (!gr) {
    gr = &p->graphs[p->graph_next];
    p->graph_next ^= 1;
    if (gr->exec) { cudaGraphExecDestroy(gr->exec); *gr = scd_batch_plan::Graph(); }
    cudaGraph_t g = nullptr;
    if ((e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) return cuda_status(e);
    cudaError_t e1 = cudaMemsetAsync(p->d_counters, 0, cbytes, st);
    if (e1 == cudaSuccess && prof) e1 = cudaMemsetAsync(out_arena, 0, pbytes, st);
    cudaError_t e2 = e1 == cudaSuccess ? launch_all() : cudaSuccess;
    e = cudaStreamEndCapture(st, &g);
    if (e1 != cudaSuccess) e = e1;
    if (e2 != cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&gr->exec, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) { gr->exec = nullptr; return cuda_status(e); }
    gr->x = x_arena; gr->w = w; gr->out = out_arena; gr->ws = workspace; gr->stream = stream;
    gr->drop = A.drop_task;
  }
  e = cudaGraphLaunch(gr->exec, st);
  return e == cudaSuccess ? SCD_OK : cuda_status(e);
}

void scd_batch_plan_destroy(scd_batch_plan* p) { free_plan(p); }

scd_status scd_batch_run_host(scd_batch_plan* p, const void* x_host, void* x_dev, const float* window, void* out_dev,
                              void* out_host, void* workspace, void* stream) {
  using namespace scd;
  NvtxRange range("scd_batch_run_host");
  if (!p || !x_dev || !out_dev || !out_host || !workspace) return SCD_ERR_ARG;
  // the argument checks of scd_batch_run, before anything is enqueued or created
  if (((uintptr_t)x_dev % 8) || ((uintptr_t)out_dev % 16) || ((uintptr_t)workspace % 16) ||
      (window && ((uintptr_t)window % 4)))
    return SCD_ERR_ARG;
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_status(e);
  if (dev != p->device) return SCD_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  if (!p->copy_st && (e = cudaStreamCreateWithFlags(&p->copy_st, cudaStreamNonBlocking)) != cudaSuccess) {
    p->copy_st = nullptr;
    return cuda_status(e);
  }
  if (!p->computed && (e = cudaEventCreateWithFlags(&p->computed, cudaEventDisableTiming)) != cudaSuccess) {
    p->computed = nullptr;
    return cuda_status(e);
  }
  cudaEvent_t done = nullptr;
  for (auto& c : p->copied)
    if (c.first == out_dev) done = c.second;
  if (done) {
    // the previous copy out of this buffer ends before the estimate overwrites it
    if ((e = cudaStreamWaitEvent(st, done, 0)) != cudaSuccess) return cuda_status(e);
  } else {
    if ((e = cudaEventCreateWithFlags(&done, cudaEventDisableTiming)) != cudaSuccess) return cuda_status(e);
    p->copied.emplace_back(out_dev, done);           // (waited on only once a copy has been recorded)
  }
  const size_t xbytes = sizeof(float2) * (size_t)p->x_off[p->nsig];
  const size_t obytes = (p->prof_power ? sizeof(float) : sizeof(float2)) * (size_t)p->out_off[p->nsig];
  if (x_host && (e = cudaMemcpyAsync(x_dev, x_host, xbytes, cudaMemcpyHostToDevice, st)) != cudaSuccess)
    return cuda_status(e);
  const scd_status s = scd_batch_run(p, x_dev, window, out_dev, workspace, stream);
  if (s != SCD_OK) return s;
  if ((e = cudaEventRecord(p->computed, st)) != cudaSuccess || (e = cudaStreamWaitEvent(p->copy_st, p->computed, 0)) != cudaSuccess ||
      (e = cudaMemcpyAsync(out_host, out_dev, obytes, cudaMemcpyDeviceToHost, p->copy_st)) != cudaSuccess ||
      (e = cudaEventRecord(done, p->copy_st)) != cudaSuccess)
    return cuda_status(e);
  return SCD_OK;
}

scd_status scd_batch_host_wait(scd_batch_plan* p) {
  if (!p) return SCD_ERR_ARG;
  if (!p->copy_st) return SCD_OK;
  const cudaError_t e = cudaStreamSynchronize(p->copy_st);
  return e == cudaSuccess ? SCD_OK : cuda_status(e);
}

// Page-locked host memory for the copies of scd_batch_run_host.  (Measured with a GB300 and its
// Grace host: device-to-host copies into page-locked buffers ran between 38 and 193 GB/s
// depending on the buffer, whether it came from cudaHostAlloc or from huge-page memory
// registered with cudaHostRegister; the rate follows where the host pages land, not how they
// were allocated, so the plain call stays.)
scd_status scd_host_alloc(size_t bytes, void** ptr) {
  if (!ptr || bytes == 0) return SCD_ERR_ARG;
  *ptr = nullptr;
  const cudaError_t e = cudaHostAlloc(ptr, bytes, cudaHostAllocDefault);
  return e == cudaSuccess ? SCD_OK : cuda_status(e);
}

scd_status scd_host_free(void* ptr) {
  if (!ptr) return SCD_OK;
  const cudaError_t e = cudaFreeHost(ptr);
  return e == cudaSuccess ? SCD_OK : cuda_status(e);
}

scd_status scd_batch_plan_set_output(scd_batch_plan* p, int32_t mode) {
  using namespace scd;
  if (!p || mode < 0 || mode > 2) return SCD_ERR_ARG;
  if (p->exact) return mode ? SCD_ERR_UNSUPPORTED : SCD_OK;
  const bool fam = p->estimator == 0, tc = p->precision == SCD_SPLIT_BF16;
  if (mode && fam) {                                            // the FAM map's band must tile alpha
    if (2 * (int64_t)p->L > p->Np) return SCD_ERR_UNSUPPORTED;
    for (int i = 0; i < p->nsig; ++i)
      if ((p->sizes[i] * p->L) % p->Np) return SCD_ERR_UNSUPPORTED;
  }
  if (mode && !p->grid_prof) {
    int per_sm = 0, sms = 0;
    cudaError_t e = prepare_kernel(fam, tc, true, p->smem, &per_sm);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device);
    if (e != cudaSuccess) return cuda_status(e);
    if (tc && per_sm > 4) per_sm = 4;
    p->grid_prof = sms * (per_sm > 0 ? per_sm : 1);
  }
  p->prof_power = mode;
  layout_outputs(p);
  drop_graphs(p);
  return build_tasks(p);
}

scd_status scd_batch_plan_set_schedule(scd_batch_plan* p, int32_t schedule) {
  using namespace scd;
  if (!p || schedule < SCD_SCHEDULE_AUTO || schedule > SCD_SCHEDULE_FUSED) return SCD_ERR_ARG;
  if (p->exact) return schedule == SCD_SCHEDULE_AUTO ? SCD_OK : SCD_ERR_UNSUPPORTED;
  int staged = 0;
  if (schedule == SCD_SCHEDULE_STAGES) {
    staged = 1;
  } else if (schedule == SCD_SCHEDULE_FUSED) {
    staged = 2;                                                 // falls back to 1 where it does not apply
  } else if (schedule == SCD_SCHEDULE_AUTO) {
    TuneEntry te;
    staged = tune_lookup(batch_key(p), &te) ? te.schedule : default_staged(p->estimator, p->precision);
  }
  if (staged == p->staged) return SCD_OK;
  p->staged = staged;
  return build_tasks(p);
}

scd_status scd_batch_tune(scd_batch_plan* p, const void* x_arena, const float* window, void* out_arena,
                          void* workspace, void* stream, int32_t reps) {
  using namespace scd;
  if (!p || reps < 1) return SCD_ERR_ARG;
  if (p->exact) {                                               // nothing to tune: one run
    scd_status s = scd_batch_run(p, x_arena, window, out_arena, workspace, stream);
    if (s != SCD_OK) return s;
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    return e == cudaSuccess ? SCD_OK : cuda_status(e);
  }
  const int64_t items[] = {32ll << 10, 64ll << 10, 128ll << 10, 256ll << 10, 512ll << 10};
  const int64_t slots[] = {8ll << 20, 16ll << 20, 32ll << 20, 64ll << 20};
  const int nslots = p->estimator == 0 ? 1 : 4;
  cudaStream_t st = (cudaStream_t)stream;
  float best = 3.4e38f;
  int64_t best_item = p->item_bytes, best_slot = p->slot_bytes;
  int best_staged = 0;
  auto try_one = [&](int staged, int64_t item, int64_t slot) -> scd_status {
    p->staged = staged;
    p->item_bytes = item;
    p->slot_bytes = slot;
    scd_status s = build_tasks(p);
    if (s != SCD_OK) return s;
    float ms = 0.f;
    s = time_candidate(st, reps, [&]() { return scd_batch_run(p, x_arena, window, out_arena, workspace, stream); }, &ms);
    if (s != SCD_OK) return s;
    if (ms < best) { best = ms; best_item = item; best_slot = slot; best_staged = staged; }
    return SCD_OK;
  };
  for (int64_t item : items)
    for (int k = 0; k < nslots; ++k) {
      scd_status s = try_one(0, item, p->estimator == 1 ? slots[k] : p->slot_bytes);
      if (s != SCD_OK) return s;
    }
  {                                                             // the staged schedule
    scd_status s = try_one(1, p->item_bytes, p->slot_bytes);
    if (s != SCD_OK) return s;
  }
  if (p->estimator == 1 && p->precision == SCD_FP32) {          // ... with the fused SSCA kernels
    scd_status s = try_one(2, p->item_bytes, p->slot_bytes);
    if (s != SCD_OK) return s;
  }
  p->staged = best_staged;
  p->item_bytes = best_item;
  p->slot_bytes = best_slot;
  scd_status s = build_tasks(p);
  if (s != SCD_OK) return s;
  tune_store(batch_key(p), TuneEntry{best_staged, best_item, best_slot, best});
  s = scd_batch_run(p, x_arena, window, out_arena, workspace, stream);   // leave a valid estimate
  if (s != SCD_OK) return s;
  cudaError_t e = cudaStreamSynchronize(st);
  return e == cudaSuccess ? SCD_OK : cuda_status(e);
}

}  // extern "C"

// ----------------------------------------------------------------------------- single SSCA
// scd_ssca's default schedule: the whole estimate (channeliser + CDP, then the column and row
// passes unit by unit through rotating slots) in one persistent launch of the same kernel,
// from a one-signal plan cached per (device, N, Np, precision).  The tile counters live in
// the caller's workspace, so concurrent calls with different workspaces do not interfere.
namespace scd {
namespace {
std::mutex g_plan_mu;
std::map<std::tuple<int, int64_t, int, int, int64_t, int64_t>, scd_batch_plan*> g_plans;

scd_batch_plan* single_plan(int64_t N, int Np, int precision, int64_t item, int64_t slot, cudaError_t* err,
                            scd_status* st) {
  int dev = 0;
  if ((*err = cudaGetDevice(&dev)) != cudaSuccess) { *st = SCD_ERR_CUDA; return nullptr; }
  std::lock_guard<std::mutex> lock(g_plan_mu);
  auto key = std::make_tuple(dev, N, Np, precision, item, slot);
  auto it = g_plans.find(key);
  if (it != g_plans.end()) return it->second;
  scd_batch_plan* p = nullptr;
  const int64_t len = N;
  *st = scd_batch_plan_create(1, 1, &len, Np, 1, precision, &p);
  if (*st != SCD_OK) return nullptr;
  if (p->item_bytes != item || p->slot_bytes != slot || p->staged) {
    p->item_bytes = item;
    p->slot_bytes = slot;
    p->staged = 0;                                              // this path is the persistent launch
    if ((*st = build_tasks(p)) != SCD_OK) { free_plan(p); return nullptr; }
  }
  g_plans[key] = p;
  return p;
}

size_t up256(size_t v) { return (v + 255) / 256 * 256; }

std::string ssca_key(int64_t N, int Np, int precision) {
  char buf[96];
  snprintf(buf, sizeof buf, "|ssca|N=%lld|Np=%d|p=%d", (long long)N, Np, precision);
  return device_key() + buf;
}
}  // namespace

size_t ssca_persistent_workspace(int64_t N, int Np) {
  const int64_t Gmax = slot_group(Np, N, kSlotBytesMax);
  const size_t data = sizeof(float2) * (size_t)(Np * N + kSlots * Gmax * N);
  const size_t ntasks = 1 + 2 * (size_t)Np;                    // at most Np units
  return up256(data) + up256(sizeof(unsigned) * (ntasks + 1));
}

scd_status ssca_persistent_tuned(const float2* x, const float2* y, bool conj, int64_t N, int Np, const float* window,
                                 float2* out, void* ws, size_t ws_bytes, cudaStream_t st, int precision,
                                 int64_t item_bytes, int64_t slot_bytes) {
  cudaError_t e = cudaSuccess;
  scd_status s = SCD_OK;
  scd_batch_plan* p = single_plan(N, Np, precision, item_bytes, slot_bytes, &e, &s);
  if (!p) {
    if (s == SCD_ERR_CUDA) return cuda_status(e);
    return s;
  }
  const size_t data = up256(p->ws_bytes);
  const size_t cbytes = sizeof(unsigned) * (p->tasks.size() + 1);
  if (ws_bytes < data + up256(cbytes)) return SCD_ERR_WORKSPACE;
  unsigned* counters = (unsigned*)((char*)ws + data);
  BatchArgs A;
  A.tasks = p->d_tasks; A.ntasks = (int)p->tasks.size(); A.Np = Np; A.L = 1; A.total = p->total;
  A.counters = counters; A.x = x; A.y = y ? y : x; A.conj = conj ? 1 : 0; A.pad_ = 0;
  A.prof_power = 0;
  A.drop_task = -1;
  A.out = out; A.ws = (float2*)ws;
  A.window = window ? window : p->hamming; A.tw_np = p->tw_np; A.bmats_np = p->bm_np;
  A.bbytes_np = p->bbytes_np; A.err = p->err;
  count_launches(1);
  if ((e = cudaMemsetAsync(counters, 0, cbytes, st)) != cudaSuccess) return cuda_status(e);
  e = launch_batch(false, precision == SCD_SPLIT_BF16, false, p->grid, p->smem, A, st);
  return e == cudaSuccess ? SCD_OK : cuda_status(e);
}

scd_status ssca_persistent(const float2* x, const float2* y, bool conj, int64_t N, int Np, const float* window,
                           float2* out, void* ws, size_t ws_bytes, cudaStream_t st, int precision) {
  return ssca_persistent_tuned(x, y, conj, N, Np, window, out, ws, ws_bytes, st, precision, kItemBytes, kSlotBytes);
}

TuneEntry ssca_auto_choice(int64_t N, int Np, int precision) {
  TuneEntry e;
  if (tune_lookup(ssca_key(N, Np, precision), &e)) return e;
  return TuneEntry{ssca_fused_supported(N, Np, precision) ? SCD_SCHEDULE_FUSED : SCD_SCHEDULE_STAGES, kItemBytes,
                   kSlotBytes, 0.0};
}

void release_single_plans() {
  std::lock_guard<std::mutex> lock(g_plan_mu);
  for (auto& kv : g_plans) free_plan(kv.second);
  g_plans.clear();
}

}  // namespace scd

extern "C" scd_status scd_ssca_tune(const void* x, int64_t N, int32_t Np, const float* window, void* out,
                                    const scd_opts* opts, int32_t reps) {
  using namespace scd;
  if (!opts || reps < 1) return SCD_ERR_ARG;
  scd_opts o = *opts;
  o.stage_events = nullptr;
  o.n_stage_events = 0;
  cudaStream_t st = (cudaStream_t)o.stream;
  TuneEntry best{SCD_SCHEDULE_STAGES, kItemBytes, kSlotBytes, 3.4e38};
  o.schedule = SCD_SCHEDULE_STAGES;
  float ms = 0.f;
  scd_status s = time_candidate(st, reps, [&]() { return scd_ssca(x, N, Np, window, out, &o); }, &ms);
  if (s != SCD_OK) return s;
  best.ms = ms;
  if (ssca_fused_supported(N, Np, o.precision)) {
    o.schedule = SCD_SCHEDULE_FUSED;
    s = time_candidate(st, reps, [&]() { return scd_ssca(x, N, Np, window, out, &o); }, &ms);
    if (s != SCD_OK) return s;
    if (ms < best.ms) best = TuneEntry{SCD_SCHEDULE_FUSED, kItemBytes, kSlotBytes, ms};
  }
  const int64_t items[] = {64ll << 10, 128ll << 10, 256ll << 10};
  const int64_t slots[] = {8ll << 20, 16ll << 20, 32ll << 20, 64ll << 20};
  for (int64_t item : items)
    for (int64_t slot : slots) {
      s = time_candidate(st, reps, [&]() {
        return ssca_persistent_tuned((const float2*)x, (const float2*)o.y, o.conjugate != 0, N, Np, window,
                                     (float2*)out, o.workspace, o.workspace_bytes, st, o.precision, item, slot);
      }, &ms);
      if (s != SCD_OK) return s;
      if (ms < best.ms) best = TuneEntry{SCD_SCHEDULE_PERSISTENT, item, slot, ms};
    }
  tune_store(ssca_key(N, Np, o.precision), best);
  return SCD_OK;
}
