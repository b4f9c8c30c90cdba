// Autotuner result cache: the best measured schedule / tile sizing per workload signature,
// kept in-process and, when the environment variable SCD_TUNE_CACHE names a file, persisted
// there as JSON (one entry per line) so later processes start from the tuned choice.
//
// Entry format:
//   {"key": "<gpu>|<workload>", "schedule": S, "item_kib": I, "slot_kib": K, "ms": T}
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <map>
#include <mutex>
#include <string>

#include "internal.h"

namespace scd {
namespace {

std::mutex g_mu;
std::map<std::string, TuneEntry> g_cache;
bool g_loaded = false;

const char* cache_path() {
  const char* p = getenv("SCD_TUNE_CACHE");
  return (p && *p) ? p : nullptr;
}

void load_locked() {
  if (g_loaded) return;
  g_loaded = true;
  const char* path = cache_path();
  if (!path) return;
  FILE* f = fopen(path, "r");
  if (!f) return;
  char line[1024];
  while (fgets(line, sizeof line, f)) {
    const char* k = strstr(line, "\"key\": \"");
    if (!k) continue;
    k += 8;
    const char* end = strchr(k, '"');
    if (!end) continue;
    std::string key(k, (size_t)(end - k));
    TuneEntry e{};
    long long item = 0, slot = 0;
    if (sscanf(end, "\", \"schedule\": %d, \"item_kib\": %lld, \"slot_kib\": %lld, \"ms\": %lf", &e.schedule, &item,
               &slot, &e.ms) == 4) {
      e.item_bytes = item << 10;
      e.slot_bytes = slot << 10;
      g_cache[key] = e;
    }
  }
  fclose(f);
}

void save_locked() {
  const char* path = cache_path();
  if (!path) return;
  const std::string tmp = std::string(path) + ".tmp";
  FILE* f = fopen(tmp.c_str(), "w");
  if (!f) return;
  fprintf(f, "{\"scd_tune_version\": 1, \"entries\": [\n");
  size_t i = 0;
  for (const auto& kv : g_cache) {
    fprintf(f, "{\"key\": \"%s\", \"schedule\": %d, \"item_kib\": %lld, \"slot_kib\": %lld, \"ms\": %.6f}%s\n",
            kv.first.c_str(), kv.second.schedule, (long long)(kv.second.item_bytes >> 10),
            (long long)(kv.second.slot_bytes >> 10), kv.second.ms, ++i < g_cache.size() ? "," : "");
  }
  fprintf(f, "]}\n");
  fclose(f);
  rename(tmp.c_str(), path);
}

}  // namespace

std::string device_key() {
  int dev = 0;
  cudaDeviceProp prop;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return "unknown";
  std::string name = prop.name;
  for (char& c : name)
    if (c == '"' || c == '|') c = '_';
  return name + "/sm" + std::to_string(prop.major * 10 + prop.minor);
}

bool tune_lookup(const std::string& key, TuneEntry* out) {
  std::lock_guard<std::mutex> lock(g_mu);
  load_locked();
  auto it = g_cache.find(key);
  if (it == g_cache.end()) return false;
  *out = it->second;
  return true;
}

void tune_store(const std::string& key, const TuneEntry& e) {
  std::lock_guard<std::mutex> lock(g_mu);
  load_locked();
  g_cache[key] = e;
  save_locked();
}

}  // namespace scd
