// Launch autotuner (see tune.cuh) and the C entry point that reports its decisions.
#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <sstream>

#include "common.cuh"
#include "tune.cuh"

namespace coarse {
namespace {

struct Entry {
  TuneChoice choice;
  float us = 0.f;           // time of the chosen configuration (0: read from the cache file)
  std::string tried;        // "a,b,c:us ..." of every candidate timed
};

std::mutex g_mu;
std::map<std::string, Entry> g_table;
bool g_loaded = false;

const char* cache_path() {
  const char* p = getenv("COARSE_AUTOTUNE_CACHE");
  return (p && *p) ? p : nullptr;
}

// cache file: one decision per line, "key a b c us"
void load_cache() {
  if (g_loaded) return;
  g_loaded = true;
  const char* path = cache_path();
  if (!path) return;
  FILE* f = fopen(path, "r");
  if (!f) return;
  char key[256];
  Entry e;
  while (fscanf(f, "%255s %d %d %d %f", key, &e.choice.a, &e.choice.b, &e.choice.c, &e.us) == 5) g_table[key] = e;
  fclose(f);
}

void append_cache(const std::string& key, const Entry& e) {
  const char* path = cache_path();
  if (!path) return;
  FILE* f = fopen(path, "a");
  if (!f) return;
  fprintf(f, "%s %d %d %d %.3f\n", key.c_str(), e.choice.a, e.choice.b, e.choice.c, e.us);
  fclose(f);
}

constexpr int kFastDevices = 64;
std::atomic<int> g_fast[kFastDevices][2][3][3][32];
std::once_flag g_fast_once;
std::string g_model[kFastDevices];

void fast_clear() {
  for (auto& d : g_fast)
    for (auto& f : d)
      for (auto& p : f)
        for (auto& n : p)
          for (auto& v : n) v.store(-1, std::memory_order_relaxed);
}

int current_device() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  return (dev >= 0 && dev < kFastDevices) ? dev : -1;
}

// "@sm<major><minor>x<SMs>" of the current device (under g_mu)
const std::string& model_suffix() {
  static const std::string none;
  const int dev = current_device();
  if (dev < 0) return none;
  if (g_model[dev].empty()) {
    int maj = 0, mnr = 0, sms = 0;
    cudaDeviceGetAttribute(&maj, cudaDevAttrComputeCapabilityMajor, dev);
    cudaDeviceGetAttribute(&mnr, cudaDevAttrComputeCapabilityMinor, dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaGetLastError();
    char buf[48];
    snprintf(buf, sizeof(buf), "@sm%d%dx%d", maj, mnr, sms);
    g_model[dev] = buf;
  }
  return g_model[dev];
}

}  // namespace

int tune_fast_get(int family, int prec, int ni, int vb) {
  std::call_once(g_fast_once, fast_clear);
  const int dev = current_device();
  if (dev < 0 || family < 0 || family > 1 || prec < 0 || prec > 2 || ni < 0 || ni > 2 || vb < 0 || vb > 31) return -1;
  return g_fast[dev][family][prec][ni][vb].load(std::memory_order_acquire);
}

void tune_fast_put(int family, int prec, int ni, int vb, int choice) {
  std::call_once(g_fast_once, fast_clear);
  const int dev = current_device();
  if (dev < 0 || family < 0 || family > 1 || prec < 0 || prec > 2 || ni < 0 || ni > 2 || vb < 0 || vb > 31) return;
  g_fast[dev][family][prec][ni][vb].store(choice, std::memory_order_release);
}

int tune_bucket(long long v) {
  int b = 0;
  while (v > 1) { v >>= 1; ++b; }
  return b;
}

int tune_pick(const std::string& key, const std::vector<TuneChoice>& cands,
              const std::function<int(const TuneChoice&)>& run, cudaStream_t s, TuneChoice* out) {
  std::string mkey;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    load_cache();
    mkey = key + model_suffix();
    auto it = g_table.find(mkey);
    if (it == g_table.end()) it = g_table.find(key);  // a model-independent entry (cache file, set)
    if (it != g_table.end()) {
      *out = it->second.choice;
      return COARSE_OK;
    }
  }
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  COARSE_CUDA(cudaStreamIsCapturing(s, &cap));
  if (cap != cudaStreamCaptureStatusNone || cands.size() == 1) {
    *out = cands[0];
    return COARSE_OK;
  }
  cudaEvent_t e0, e1;
  COARSE_CUDA(cudaEventCreate(&e0));
  COARSE_CUDA(cudaEventCreate(&e1));
  Entry best;
  best.us = -1.f;
  std::ostringstream tried;
  int rc_last = COARSE_OK;
  for (const TuneChoice& c : cands) {
    int rc = run(c);  // warm-up (and the check that this configuration launches at all)
    if (rc != COARSE_OK) {
      rc_last = rc;
      continue;
    }
    float t_best = 1e30f;
    for (int rep = 0; rep < 3 && rc == COARSE_OK; ++rep) {
      cudaEventRecord(e0, s);
      rc = run(c);
      cudaEventRecord(e1, s);
      if (cudaEventSynchronize(e1) != cudaSuccess) rc = cuda_fail(cudaGetLastError(), "autotune timing");
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      t_best = std::min(t_best, ms * 1e3f);
    }
    if (rc != COARSE_OK) {
      rc_last = rc;
      continue;
    }
    tried << c.a << "," << c.b << "," << c.c << ":" << t_best << " ";
    if (best.us < 0.f || t_best < best.us) {
      best.us = t_best;
      best.choice = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (best.us < 0.f) return rc_last != COARSE_OK ? rc_last : COARSE_ERR_INVALID_ARG;
  best.tried = tried.str();
  {
    std::lock_guard<std::mutex> lk(g_mu);
    g_table[mkey] = best;
    append_cache(mkey, best);
  }
  *out = best.choice;
  return COARSE_OK;
}

}  // namespace coarse

// Text table of the autotuner's decisions, one line per key:
//   "<key> -> <a> <b> <c> <us> | <candidates timed>".
extern "C" int coarse_autotune_report(char* buf, long long len) {
  using namespace coarse;
  if (!buf || len < 1) {
    set_error("coarse_autotune_report: need a buffer");
    return COARSE_ERR_INVALID_ARG;
  }
  std::ostringstream os;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    for (const auto& kv : g_table)
      os << kv.first << " -> " << kv.second.choice.a << " " << kv.second.choice.b << " " << kv.second.choice.c << " "
         << kv.second.us << " | " << kv.second.tried << "\n";
  }
  const std::string s = os.str();
  const size_t n = std::min<size_t>(s.size(), (size_t)len - 1);
  memcpy(buf, s.data(), n);
  buf[n] = '\0';
  return COARSE_OK;
}

// Fixes the decision for `key` (a key as coarse_autotune_report prints it, with or without the
// model suffix) for every later launch in this process.
extern "C" int coarse_autotune_set(const char* key, int a, int b, int c) {
  using namespace coarse;
  if (!key || !*key) {
    set_error("coarse_autotune_set: empty key");
    return COARSE_ERR_INVALID_ARG;
  }
  {
    std::lock_guard<std::mutex> lk(g_mu);
    load_cache();
    const std::string k(key);
    if (a >= 0) {
      Entry e;
      e.choice = TuneChoice{a, b, c};
      e.tried = "set";
      g_table[k] = e;
    } else {
      g_table.erase(k);  // a < 0: forget the decision; the next launch times the candidates again
    }
    // a plain key overrides (or, with a < 0, forgets) every model-specific decision of that shape
    if (k.find('@') == std::string::npos) {
      for (auto it = g_table.begin(); it != g_table.end();) {
        if (it->first.size() > k.size() && it->first.compare(0, k.size(), k) == 0 && it->first[k.size()] == '@')
          it = g_table.erase(it);
        else
          ++it;
      }
    }
  }
  std::call_once(g_fast_once, fast_clear);
  fast_clear();
  return COARSE_OK;
}
