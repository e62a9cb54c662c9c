// Launch-shape autotuner.
//
// A launcher that has several correct launch shapes for one problem (for
// example how many slices the points of a kernel-matrix product are split
// into) names the problem by a key and asks tune_pick() for a shape.  The
// first time a key is seen, each candidate runs once to warm up and twice
// under CUDA events on the caller's stream; the fastest is kept for the rest
// of the process and, when NYS_TUNE_CACHE names a file, written there as a
// flat JSON object {"key": choice, ...} that later processes read back
// before they time anything.  With tuning off (NYS_TUNE=0 or
// nys_autotune(0)), or on a stream that is being captured into a graph
// (nothing can be timed there), an uncached key gets the launcher's own rule
// and nothing is stored.
//
// The candidates of one key compute the same mathematical result; shapes
// that split a sum differ in the rounding of its last bits only.

#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <map>
#include <mutex>
#include <string>

#include <unistd.h>

#include "common.cuh"
#include "internal.h"

namespace nys {

namespace {

std::mutex g_mu;
std::map<std::string, int> g_cache;
bool g_loaded = false;
std::atomic<int> g_on{-1};
std::atomic<unsigned long long> g_timed{0};

const char* cache_path() {
  const char* p = getenv("NYS_TUNE_CACHE");
  return (p && p[0]) ? p : nullptr;
}

// Reads {"key": int, ...}; anything it does not understand ends the parse.
void load_locked() {
  if (g_loaded) return;
  g_loaded = true;
  const char* path = cache_path();
  if (!path) return;
  FILE* f = fopen(path, "rb");
  if (!f) return;
  std::string txt;
  char buf[4096];
  size_t k;
  while ((k = fread(buf, 1, sizeof(buf), f)) > 0) txt.append(buf, k);
  fclose(f);
  size_t i = 0;
  while (true) {
    const size_t q0 = txt.find('"', i);
    if (q0 == std::string::npos) break;
    const size_t q1 = txt.find('"', q0 + 1);
    if (q1 == std::string::npos) break;
    const size_t c = txt.find(':', q1 + 1);
    if (c == std::string::npos) break;
    char* end = nullptr;
    const long v = strtol(txt.c_str() + c + 1, &end, 10);
    if (end == txt.c_str() + c + 1) break;
    g_cache[txt.substr(q0 + 1, q1 - q0 - 1)] = (int)v;
    i = (size_t)(end - txt.c_str());
  }
}

void save_locked() {
  const char* path = cache_path();
  if (!path) return;
  // one temporary per process: ranks sharing a cache file each write their
  // own and rename it into place (the last rename wins, whole)
  const std::string tmp = std::string(path) + ".tmp." + std::to_string((long)getpid());
  FILE* f = fopen(tmp.c_str(), "wb");
  if (!f) return;
  fputs("{\n", f);
  size_t k = 0;
  for (const auto& kv : g_cache)
    fprintf(f, "  \"%s\": %d%s\n", kv.first.c_str(), kv.second, ++k < g_cache.size() ? "," : "");
  fputs("}\n", f);
  fclose(f);
  rename(tmp.c_str(), path);
}

}  // namespace

bool tune_enabled() {
  int v = g_on.load(std::memory_order_relaxed);
  if (v < 0) {
    const char* e = getenv("NYS_TUNE");
    int want = (e && e[0] == '0') ? 0 : 1;
    g_on.compare_exchange_strong(v, want);
    v = g_on.load(std::memory_order_relaxed);
  }
  return v == 1;
}

int32_t tune_switch(int32_t on) {
  const int32_t prev = tune_enabled() ? 1 : 0;
  if (on == 0 || on == 1) g_on.store(on, std::memory_order_relaxed);
  return prev;
}

bool tune_cached(const std::string& key, int* choice) {
  std::lock_guard<std::mutex> lk(g_mu);
  load_locked();
  auto it = g_cache.find(key);
  if (it == g_cache.end()) return false;
  if (choice) *choice = it->second;
  return true;
}

int32_t tune_pick(const std::string& key, const std::vector<int>& cands, int fallback,
                  const std::function<int32_t(int)>& run, cudaStream_t s, int* choice) {
  *choice = fallback;
  if (cands.size() < 2) {
    if (cands.size() == 1) *choice = cands[0];
    return NYS_OK;
  }
  int c = 0;
  if (tune_cached(key, &c)) {
    for (int k : cands)
      if (k == c) {
        *choice = c;
        return NYS_OK;
      }
    // a stale entry names no current candidate: time again
  }
  if (!tune_enabled()) return NYS_OK;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  NYS_CUDA_TRY(cudaStreamIsCapturing(s, &cs));
  if (cs != cudaStreamCaptureStatusNone) return NYS_OK;
  cudaEvent_t e0, e1;
  NYS_CUDA_TRY(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return NYS_ERR_CUDA;
  }
  int32_t st = NYS_OK;
  float best = 0.f;
  int pick = fallback;
  bool have = false;
  for (int k : cands) {
    st = run(k);  // warm-up
    if (st != NYS_OK) break;
    if (cudaEventRecord(e0, s) != cudaSuccess) { st = NYS_ERR_CUDA; break; }
    for (int r = 0; r < 2 && st == NYS_OK; ++r) st = run(k);
    if (st != NYS_OK) break;
    float ms = 0.f;
    if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
      st = NYS_ERR_CUDA;
      break;
    }
    if (!have || ms < best) {
      best = ms;
      pick = k;
      have = true;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != NYS_OK) return st;
  *choice = pick;
  g_timed.fetch_add(1, std::memory_order_relaxed);
  std::lock_guard<std::mutex> lk(g_mu);
  g_cache[key] = pick;
  save_locked();
  return NYS_OK;
}

int64_t tune_dump(char* buf, int64_t cap) {
  std::lock_guard<std::mutex> lk(g_mu);
  load_locked();
  std::string out = "{";
  size_t k = 0;
  for (const auto& kv : g_cache) {
    out += "\"" + kv.first + "\": " + std::to_string(kv.second);
    if (++k < g_cache.size()) out += ", ";
  }
  out += "}";
  if (buf && cap > 0) {
    const size_t m = std::min<size_t>(out.size(), (size_t)cap - 1);
    memcpy(buf, out.data(), m);
    buf[m] = '\0';
  }
  return (int64_t)out.size();
}

void tune_clear() {
  std::lock_guard<std::mutex> lk(g_mu);
  g_cache.clear();
  g_loaded = true;  // the file is not read again
}

int32_t tune_set(const char* key, int32_t choice) {
  if (!key || !key[0]) return NYS_ERR_ARG;
  std::lock_guard<std::mutex> lk(g_mu);
  load_locked();
  g_cache[key] = choice;
  save_locked();
  return NYS_OK;
}

unsigned long long tune_timed() { return g_timed.load(std::memory_order_relaxed); }

}  // namespace nys
