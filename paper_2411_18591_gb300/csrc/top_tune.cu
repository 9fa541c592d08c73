// The autotune table: per line length M (half a padded size), the pass variants measured fastest
// by top_autotune (TOP_TUNE_* flags), with a text file format that carries a checksum.
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "top_internal.h"

namespace top {

namespace {

std::mutex g_tune_mutex;
std::map<int, uint32_t> g_tune;

constexpr const char* kTuneHeader = "top-autotune 1";
constexpr uint32_t kTuneMask = 0xfffu;  // every defined flag bit

// FNV-1a, 64 bits
uint64_t fnv1a(const char* p, size_t n) {
  uint64_t h = 1469598103934665603ull;
  for (size_t i = 0; i < n; ++i) {
    h ^= (unsigned char)p[i];
    h *= 1099511628211ull;
  }
  return h;
}

}  // namespace

uint32_t tune_flags(int M) {
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  auto it = g_tune.find(M);
  return it == g_tune.end() ? 0u : it->second;
}

bool tune_flags_valid(uint32_t flags) { return (flags & ~kTuneMask) == 0 && ((flags >> 8) & 7u) <= 4u; }

void tune_set(int M, uint32_t flags) {
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  g_tune[M] = flags;
}

void tune_clear() {
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  g_tune.clear();
}

bool tune_save(const char* path, std::string* err) {
  std::string text = std::string(kTuneHeader) + "\n";
  {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    char line[64];
    for (const auto& kv : g_tune) {
      std::snprintf(line, sizeof line, "%d %x\n", kv.first, kv.second);
      text += line;
    }
  }
  char tail[64];
  std::snprintf(tail, sizeof tail, "checksum %016llx\n", (unsigned long long)fnv1a(text.data(), text.size()));
  text += tail;
  FILE* f = std::fopen(path, "wb");
  if (!f) {
    *err = "cannot open for writing";
    return false;
  }
  const bool ok = std::fwrite(text.data(), 1, text.size(), f) == text.size();
  if (std::fclose(f) != 0 || !ok) {
    *err = "write failed";
    return false;
  }
  return true;
}

bool tune_load(const char* path, std::string* err) {
  FILE* f = std::fopen(path, "rb");
  if (!f) {
    *err = "cannot open";
    return false;
  }
  std::string text;
  char buf[4096];
  size_t n;
  while ((n = std::fread(buf, 1, sizeof buf, f)) > 0) {
    text.append(buf, n);
    if (text.size() > (1u << 20)) {
      std::fclose(f);
      *err = "larger than 1 MiB";
      return false;
    }
  }
  std::fclose(f);
  // the checksum line covers every byte before it
  const size_t cpos = text.rfind("checksum ");
  if (cpos == std::string::npos || (cpos > 0 && text[cpos - 1] != '\n')) {
    *err = "no checksum line";
    return false;
  }
  unsigned long long want = 0;
  char rest = 0;
  if (std::sscanf(text.c_str() + cpos, "checksum %llx%c", &want, &rest) != 2 || rest != '\n' ||
      text.size() != cpos + std::strlen("checksum ") + 16 + 1) {
    *err = "malformed checksum line";
    return false;
  }
  if (fnv1a(text.data(), cpos) != want) {
    *err = "checksum mismatch";
    return false;
  }
  std::map<int, uint32_t> table;
  size_t pos = 0;
  bool header = true;
  while (pos < cpos) {
    const size_t eol = text.find('\n', pos);
    if (eol == std::string::npos || eol > cpos) {
      *err = "unterminated line";
      return false;
    }
    const std::string line = text.substr(pos, eol - pos);
    pos = eol + 1;
    if (header) {
      if (line != kTuneHeader) {
        *err = "unknown header";
        return false;
      }
      header = false;
      continue;
    }
    int M = 0;
    unsigned flags = 0;
    char extra = 0;
    if (std::sscanf(line.c_str(), "%d %x %c", &M, &flags, &extra) != 2 || M < 1 || M > (1 << 20) ||
        !tune_flags_valid(flags)) {
      *err = "bad entry '" + line + "'";
      return false;
    }
    table[M] = flags;
  }
  if (header) {
    *err = "empty file";
    return false;
  }
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  g_tune = table;
  return true;
}

}  // namespace top
