// Autotuner cache: the batching choice of a plan (execution mode, resident
// blocks per SM, child staging, section order) keyed by the plan's shape, so
// that a plan whose shape was tuned before is configured without timing.
// The choice is how uneven boards and sections are assigned to the device
// (the role the paper's pseudorandom placement of uneven lines plays in
// "Data layout and distribution"); the values computed never depend on it.
#include <cuda_runtime.h>
#include <unistd.h>

#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>

#include "pp_internal.h"

namespace pp {
namespace {

std::mutex g_tune_mutex;
std::map<std::string, pp_batch_opts> g_tune;
int g_hits = 0, g_misses = 0;
bool g_env_read = false;

const char* env_path() {
  const char* p = std::getenv("PP_AUTOTUNE_CACHE");
  return p && *p ? p : nullptr;
}

int err(int code, const char* fmt, const char* a, int b = 0) {
  char buf[512];
  std::snprintf(buf, sizeof buf, fmt, a, b);
  return report_error(code, buf);
}

// "<key>\t<persistent> <threads_per_block> <ctas_per_sm> <stage_children> <largest_first>"
bool parse(const char* line, std::string* key, pp_batch_opts* o) {
  const char* tab = std::strchr(line, '\t');
  if (!tab || tab == line) return false;
  int v[5];
  char extra;
  if (std::sscanf(tab + 1, "%d %d %d %d %d %c", &v[0], &v[1], &v[2], &v[3], &v[4], &extra) != 5) return false;
  if (v[0] < 0 || v[0] > 3 || (v[1] != 0 && v[1] != 256) || v[2] < 0 || v[2] > 32 || v[3] < 0 || v[3] > 2 ||
      v[4] < 0 || v[4] > 1)
    return false;
  key->assign(line, tab - line);
  *o = pp_batch_opts{v[0], v[1], v[2], v[3], v[4]};
  return true;
}

// All lines parse or nothing is merged; entries read replace those of the
// same key.
int load_locked(const char* path, int* entries) {
  FILE* f = std::fopen(path, "r");
  if (!f) return err(PP_EIO, "cannot read autotune cache %s", path);
  std::map<std::string, pp_batch_opts> add;
  char buf[1024];
  int lineno = 0;
  while (std::fgets(buf, sizeof buf, f)) {
    lineno++;
    size_t len = std::strlen(buf);
    if (len == sizeof buf - 1 && buf[len - 1] != '\n') {
      std::fclose(f);
      return err(PP_EINVAL, "autotune cache %s: line %d too long", path, lineno);
    }
    while (len && (buf[len - 1] == '\n' || buf[len - 1] == '\r')) buf[--len] = 0;
    if (!len || buf[0] == '#') continue;
    std::string key;
    pp_batch_opts o;
    if (!parse(buf, &key, &o)) {
      std::fclose(f);
      return err(PP_EINVAL, "autotune cache %s: line %d malformed", path, lineno);
    }
    add[key] = o;
  }
  const bool bad = std::ferror(f);
  std::fclose(f);
  if (bad) return err(PP_EIO, "error reading autotune cache %s", path);
  for (auto& kv : add) g_tune[kv.first] = kv.second;
  if (entries) *entries = (int)add.size();
  return PP_OK;
}

// Written to a temporary file beside the target and renamed over it, so a
// reader never sees half a file.
int save_locked(const char* path) {
  std::string tmp = std::string(path) + ".tmp." + std::to_string((long)getpid());
  FILE* f = std::fopen(tmp.c_str(), "w");
  if (!f) return err(PP_EIO, "cannot write autotune cache %s", path);
  std::fprintf(f, "# key\tpersistent threads_per_block ctas_per_sm stage_children largest_first\n");
  for (auto& kv : g_tune) {
    const pp_batch_opts& o = kv.second;
    std::fprintf(f, "%s\t%d %d %d %d %d\n", kv.first.c_str(), o.persistent, o.threads_per_block, o.ctas_per_sm,
                 o.stage_children, o.largest_first);
  }
  const bool bad = std::ferror(f);
  if (std::fclose(f) || bad || std::rename(tmp.c_str(), path)) {
    std::remove(tmp.c_str());
    return err(PP_EIO, "cannot write autotune cache %s", path);
  }
  return PP_OK;
}

}  // namespace

std::string tune_device_tag() {
  int dev = 0, sms = 0, major = 0, minor = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
  return "sm_" + std::to_string(major) + std::to_string(minor) + "x" + std::to_string(sms);
}

namespace {

bool find_locked(const std::string& key, pp_batch_opts* o) {
  if (!g_env_read) {  // a missing or malformed file only means nothing is cached yet
    g_env_read = true;
    if (const char* p = env_path()) load_locked(p, nullptr);
  }
  auto it = g_tune.find(key);
  if (it == g_tune.end()) return false;
  *o = it->second;
  return true;
}

}  // namespace

bool tune_lookup(const std::string& key, pp_batch_opts* o) {
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  const bool hit = find_locked(key, o);
  (hit ? g_hits : g_misses)++;
  return hit;
}

bool tune_peek(const std::string& key, pp_batch_opts* o) {
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  return find_locked(key, o);
}

void tune_record(const std::string& key, const pp_batch_opts& o) {
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  g_tune[key] = o;
  if (const char* p = env_path()) save_locked(p);  // the choice stands even if the file cannot be written
}

}  // namespace pp

extern "C" {

int pp_autotune_cache_load(const char* path, int* entries) {
  if (!path) return pp::report_error(PP_EINVAL, "null path");
  std::lock_guard<std::mutex> lock(pp::g_tune_mutex);
  return pp::load_locked(path, entries);
}

int pp_autotune_cache_save(const char* path) {
  if (!path) return pp::report_error(PP_EINVAL, "null path");
  std::lock_guard<std::mutex> lock(pp::g_tune_mutex);
  return pp::save_locked(path);
}

int pp_autotune_cache_clear(void) {
  std::lock_guard<std::mutex> lock(pp::g_tune_mutex);
  pp::g_tune.clear();
  pp::g_hits = pp::g_misses = 0;
  pp::g_env_read = true;  // cleared means empty: the file is not read again
  return PP_OK;
}

int pp_autotune_cache_stats(int* entries, int* hits, int* misses) {
  std::lock_guard<std::mutex> lock(pp::g_tune_mutex);
  if (entries) *entries = (int)pp::g_tune.size();
  if (hits) *hits = pp::g_hits;
  if (misses) *misses = pp::g_misses;
  return PP_OK;
}

}  // extern "C"
