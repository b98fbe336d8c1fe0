// The autotuner's cache of plan schedules: an in-memory table keyed by the
// device name and the plan's shape class, which can be written to and read
// back from a JSON file (cg_tune_cache_save / cg_tune_cache_load). When the
// environment names a file (CGMIMO_TUNE_CACHE), the first lookup reads it
// and every new entry rewrites it, so a schedule tuned once is reused by
// later processes. Host code only.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>

#include "cgmimo.h"
#include "tune.h"

namespace cgm {

namespace {

std::mutex g_mu;
std::map<std::string, TuneEntry> g_table;
bool g_env_loaded = false;

// JSON string escaping for the characters a key can hold.
std::string escape(const std::string& s) {
  std::string o;
  for (char c : s) {
    if (c == '"' || c == '\\') o += '\\';
    if (static_cast<unsigned char>(c) < 0x20) continue;
    o += c;
  }
  return o;
}

// Value of number field `name` in one JSON object line, or false.
bool field_num(const char* line, const char* name, double* out) {
  char pat[64];
  std::snprintf(pat, sizeof(pat), "\"%s\":", name);
  const char* p = std::strstr(line, pat);
  if (p == nullptr) return false;
  p += std::strlen(pat);
  char* end = nullptr;
  const double v = std::strtod(p, &end);
  if (end == p) return false;
  *out = v;
  return true;
}

// The "key" string of one JSON object line (unescaped), or false.
bool field_key(const char* line, std::string* out) {
  const char* p = std::strstr(line, "\"key\":");
  if (p == nullptr) return false;
  p = std::strchr(p + 6, '"');
  if (p == nullptr) return false;
  std::string k;
  for (++p; *p && *p != '"'; ++p) {
    if (*p == '\\' && p[1]) ++p;
    k += *p;
  }
  if (*p != '"') return false;
  *out = k;
  return true;
}

bool valid(const TuneEntry& e) {
  return (e.precision == CG_PREC_FP16X3 || e.precision == CG_PREC_BF16X3 ||
          e.precision == CG_PREC_FP16 || e.precision == CG_PREC_BF16) &&
         (e.order == 0 || e.order == 1) && (e.concurrent == 0 || e.concurrent == 1) &&
         e.grid_pct >= 1 && e.grid_pct <= 100;
}

// Merges the entries of a file written by save_locked (one object per line);
// a file with any malformed entry merges nothing.
int load_locked(const char* path) {
  FILE* f = std::fopen(path, "r");
  if (f == nullptr) return CG_EINVAL;
  char line[4096];
  int n = 0, bad = 0;
  std::map<std::string, TuneEntry> add;
  while (std::fgets(line, sizeof(line), f)) {
    if (std::strchr(line, '{') == nullptr) continue;  // the array brackets
    std::string key;
    double pr, od, cc, gp, ms = 0.0;
    if (!field_key(line, &key) || !field_num(line, "precision", &pr) ||
        !field_num(line, "order", &od) || !field_num(line, "concurrent", &cc) ||
        !field_num(line, "grid_pct", &gp)) {
      ++bad;
      continue;
    }
    field_num(line, "ms", &ms);
    const TuneEntry e{int32_t(pr), int32_t(od), int32_t(cc), int32_t(gp), float(ms)};
    if (!valid(e)) {
      ++bad;
      continue;
    }
    add[key] = e;
    ++n;
  }
  std::fclose(f);
  if (bad) return CG_EINVAL;
  for (auto& kv : add) g_table[kv.first] = kv.second;
  return n;
}

int save_locked(const char* path) {
  const std::string tmp = std::string(path) + ".tmp";
  FILE* f = std::fopen(tmp.c_str(), "w");
  if (f == nullptr) return CG_EINVAL;
  std::fprintf(f, "[\n");
  size_t i = 0;
  for (const auto& kv : g_table) {
    const TuneEntry& e = kv.second;
    std::fprintf(f,
                 "{\"key\": \"%s\", \"precision\": %d, \"order\": %d, \"concurrent\": %d, "
                 "\"grid_pct\": %d, \"ms\": %.6f}%s\n",
                 escape(kv.first).c_str(), e.precision, e.order, e.concurrent, e.grid_pct,
                 double(e.ms), ++i < g_table.size() ? "," : "");
  }
  std::fprintf(f, "]\n");
  const bool ok = std::fclose(f) == 0;
  if (!ok || std::rename(tmp.c_str(), path) != 0) return CG_EINVAL;
  return int(g_table.size());
}

void env_load_locked() {
  if (g_env_loaded) return;
  g_env_loaded = true;
  const char* path = std::getenv("CGMIMO_TUNE_CACHE");
  if (path && *path) load_locked(path);  // a missing or malformed file leaves the table as is
}

}  // namespace

bool tune_lookup(const std::string& key, TuneEntry* out) {
  std::lock_guard<std::mutex> lk(g_mu);
  env_load_locked();
  auto it = g_table.find(key);
  if (it == g_table.end()) return false;
  *out = it->second;
  return true;
}

void tune_store(const std::string& key, const TuneEntry& e) {
  std::lock_guard<std::mutex> lk(g_mu);
  env_load_locked();
  g_table[key] = e;
  const char* path = std::getenv("CGMIMO_TUNE_CACHE");
  if (path && *path) save_locked(path);
}

}  // namespace cgm

extern "C" {

int cg_tune_cache_load(const char* path) {
  if (path == nullptr) return CG_EINVAL;
  std::lock_guard<std::mutex> lk(cgm::g_mu);
  return cgm::load_locked(path);
}

int cg_tune_cache_save(const char* path) {
  if (path == nullptr) return CG_EINVAL;
  std::lock_guard<std::mutex> lk(cgm::g_mu);
  return cgm::save_locked(path);
}

int cg_tune_cache_size(void) {
  std::lock_guard<std::mutex> lk(cgm::g_mu);
  return int(cgm::g_table.size());
}

}  // extern "C"
