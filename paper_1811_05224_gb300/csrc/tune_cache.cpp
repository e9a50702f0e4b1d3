// Tuned-parameter cache: an in-process map guarded by a mutex, mirrored to a
// text file of "key<TAB>value" lines after a header line.  The file is
// rewritten whole on every store (temporary file + rename), so a reader never
// sees a half-written file; lines that do not parse are skipped.
#include "tune_cache.h"

#include <cuda_runtime.h>

#include <cstdio>
#include <cstdlib>
#include <fstream>
#include <map>
#include <mutex>
#include <sstream>

namespace stbem {
namespace {

const char* kHeader = "# stbem tuned launch parameters v1";

struct Cache {
  std::mutex mu;
  std::map<std::string, std::string> table;
  std::string path;
  bool env_checked = false;
};

Cache& cache() {
  static Cache c;
  return c;
}

bool load_file(const std::string& path, std::map<std::string, std::string>* into) {
  std::ifstream in(path);
  if (!in.good()) {
    // a missing file is an empty cache; an unreadable existing one is an error
    FILE* f = std::fopen(path.c_str(), "r");
    if (f) {
      std::fclose(f);
      return false;
    }
    return true;
  }
  std::string line;
  while (std::getline(in, line)) {
    if (line.empty() || line[0] == '#') continue;
    const size_t tab = line.find('\t');
    if (tab == std::string::npos || tab == 0 || tab + 1 >= line.size()) continue;
    (*into)[line.substr(0, tab)] = line.substr(tab + 1);
  }
  return true;
}

bool write_file(const std::string& path, const std::map<std::string, std::string>& table) {
  const std::string tmp = path + ".tmp";
  {
    std::ofstream out(tmp, std::ios::trunc);
    if (!out.good()) return false;
    out << kHeader << "\n";
    for (const auto& kv : table) out << kv.first << "\t" << kv.second << "\n";
    out.flush();
    if (!out.good()) return false;
  }
  return std::rename(tmp.c_str(), path.c_str()) == 0;
}

// the STBEM_TUNE_CACHE environment variable names the default file
void check_env(Cache& c) {
  if (c.env_checked) return;
  c.env_checked = true;
  const char* p = std::getenv("STBEM_TUNE_CACHE");
  if (p && *p) {
    c.path = p;
    load_file(c.path, &c.table);
  }
}

}  // namespace

bool tune_cache_token_ok(const std::string& s) {
  if (s.empty()) return false;
  for (char ch : s)
    if (ch == '\t' || ch == '\n' || ch == '\r') return false;
  return true;
}

bool tune_cache_set_path(const char* path) {
  Cache& c = cache();
  std::lock_guard<std::mutex> lock(c.mu);
  c.env_checked = true;
  c.path = path ? path : "";
  if (c.path.empty()) return true;
  return load_file(c.path, &c.table);
}

std::string tune_cache_path() {
  Cache& c = cache();
  std::lock_guard<std::mutex> lock(c.mu);
  check_env(c);
  return c.path;
}

bool tune_cache_get(const std::string& key, std::string* value) {
  Cache& c = cache();
  std::lock_guard<std::mutex> lock(c.mu);
  check_env(c);
  auto it = c.table.find(key);
  if (it == c.table.end()) return false;
  if (value) *value = it->second;
  return true;
}

bool tune_cache_put(const std::string& key, const std::string& value) {
  Cache& c = cache();
  std::lock_guard<std::mutex> lock(c.mu);
  check_env(c);
  c.table[key] = value;
  if (c.path.empty()) return true;
  // merge entries another process may have written meanwhile, then rewrite
  std::map<std::string, std::string> disk;
  load_file(c.path, &disk);
  for (const auto& kv : c.table) disk[kv.first] = kv.second;
  return write_file(c.path, disk);
}

void tune_cache_clear() {
  Cache& c = cache();
  std::lock_guard<std::mutex> lock(c.mu);
  c.table.clear();
}

std::string tune_device_key(int device) {
  static std::mutex mu;
  static std::map<int, std::string> keys;
  {
    std::lock_guard<std::mutex> lock(mu);
    auto it = keys.find(device);
    if (it != keys.end()) return it->second;
  }
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return "";
  std::ostringstream os;
  std::string name = prop.name;
  for (char& ch : name)
    if (ch == '\t' || ch == '\n' || ch == '\r' || ch == '|') ch = ' ';
  os << name << "|sm" << prop.multiProcessorCount << "|cc" << prop.major << "." << prop.minor;
  std::lock_guard<std::mutex> lock(mu);
  keys[device] = os.str();
  return os.str();
}

}  // namespace stbem
