// Process-wide cache of tuned launch parameters (tile shapes, lag-chunk
// lengths), optionally backed by a text file so that a later process reuses
// what an earlier one measured.  Keys name the device, the kernel family and
// the problem shape; values are short "name=value" lists.  Host-only.
#pragma once
#include <string>

namespace stbem {

// Sets the backing file (nullptr or "": memory only) and merges its entries
// into the in-process table.  Returns false if an existing file cannot be read.
bool tune_cache_set_path(const char* path);
// The backing file in use ("" if none).
std::string tune_cache_path();
bool tune_cache_get(const std::string& key, std::string* value);
// Stores in memory and, with a backing file, rewrites the file (write to a
// temporary name, then rename).  Returns false if the file cannot be written.
bool tune_cache_put(const std::string& key, const std::string& value);
// Drops every in-process entry (the file is left as it is).
void tune_cache_clear();
// "name|sm<count>|cc<major>.<minor>" of a CUDA device (empty on error);
// queried once per device and kept.
std::string tune_device_key(int device);
// A key or value may not hold tabs or line breaks.
bool tune_cache_token_ok(const std::string& s);

}  // namespace stbem
