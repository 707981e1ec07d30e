// JSON cache of the product autotuner (the search itself runs in capi.cu, where the
// handle's buffers are).  File layout:
//   {"format": "...", "devices": {"<name>/<SMs>": {"dense/bf16/n8192/N64":
//       {"splits": 2, "stages": 3, "per_sm": 2, "bn": 64, "ms": 0.0441}, ...}, ...}}
// The reader accepts any JSON of that shape (objects, strings, numbers, true/false/null);
// unknown keys are ignored.  Entries of other devices are kept when the file is rewritten.
#include <cuda_runtime.h>

#include <cctype>
#include <cstdio>
#include <cstdlib>
#include <fstream>
#include <map>
#include <mutex>
#include <sstream>
#include <string>

#include "tune.cuh"

namespace snmf {

namespace {

using Table = std::map<std::string, std::map<std::string, TuneEntry>>;

std::mutex g_mu;
Table g_mem;  // in-process cache (also holds what was read from files)

struct Parser {
  const std::string& t;
  size_t i = 0;
  bool ok = true;
  explicit Parser(const std::string& s) : t(s) {}
  void ws() {
    while (i < t.size() && std::isspace((unsigned char)t[i])) ++i;
  }
  bool eat(char c) {
    ws();
    if (i < t.size() && t[i] == c) { ++i; return true; }
    return false;
  }
  std::string str() {
    ws();
    std::string out;
    if (i >= t.size() || t[i] != '"') { ok = false; return out; }
    ++i;
    while (i < t.size() && t[i] != '"') {
      if (t[i] == '\\' && i + 1 < t.size()) ++i;
      out += t[i++];
    }
    if (i >= t.size()) { ok = false; return out; }
    ++i;
    return out;
  }
  double num() {
    ws();
    const char* b = t.c_str() + i;
    char* e = nullptr;
    const double v = std::strtod(b, &e);
    if (e == b) { ok = false; return 0.0; }
    i += (size_t)(e - b);
    return v;
  }
  // skips any value
  void skip() {
    ws();
    if (i >= t.size()) { ok = false; return; }
    if (t[i] == '"') { str(); return; }
    if (t[i] == '{') {
      ++i;
      if (eat('}')) return;
      do { str(); if (!eat(':')) { ok = false; return; } skip(); } while (ok && eat(','));
      if (!eat('}')) ok = false;
      return;
    }
    if (t[i] == '[') {
      ++i;
      if (eat(']')) return;
      do { skip(); } while (ok && eat(','));
      if (!eat(']')) ok = false;
      return;
    }
    if (t.compare(i, 4, "true") == 0 || t.compare(i, 4, "null") == 0) { i += 4; return; }
    if (t.compare(i, 5, "false") == 0) { i += 5; return; }
    num();
  }
  // {"splits": .., "stages": .., "per_sm": .., "ms": ..}
  TuneEntry entry() {
    TuneEntry e;
    if (!eat('{')) { ok = false; return e; }
    if (eat('}')) return e;
    do {
      const std::string k = str();
      if (!eat(':')) { ok = false; return e; }
      ws();
      if (k == "splits") e.cfg.splits = (int)num();
      else if (k == "stages") e.cfg.stages = (int)num();
      else if (k == "per_sm") e.cfg.per_sm = (int)num();
      else if (k == "bn") e.cfg.bn = (int)num();
      else if (k == "row_bm") e.cfg.row_bm = (int)num();
      else if (k == "row_tc") e.cfg.row_tc = (int)num();
      else if (k == "ms") e.ms = num();
      else skip();
    } while (ok && eat(','));
    if (!eat('}')) ok = false;
    return e;
  }
  void file(Table* out) {
    if (!eat('{')) { ok = false; return; }
    if (eat('}')) return;
    do {
      const std::string k = str();
      if (!eat(':')) { ok = false; return; }
      if (k != "devices") { skip(); continue; }
      if (!eat('{')) { ok = false; return; }
      if (eat('}')) continue;
      do {
        const std::string dev = str();
        if (!eat(':') || !eat('{')) { ok = false; return; }
        if (eat('}')) continue;
        do {
          const std::string key = str();
          if (!eat(':')) { ok = false; return; }
          const TuneEntry e = entry();
          if (ok) (*out)[dev][key] = e;
        } while (ok && eat(','));
        if (!eat('}')) ok = false;
      } while (ok && eat(','));
      if (!eat('}')) ok = false;
    } while (ok && eat(','));
  }
};

bool read_file(const char* path, Table* out) {
  std::ifstream f(path);
  if (!f) return false;
  std::stringstream ss;
  ss << f.rdbuf();
  const std::string text = ss.str();
  Parser p(text);
  Table t;
  p.file(&t);
  if (!p.ok) return false;
  for (auto& d : t)
    for (auto& e : d.second) (*out)[d.first][e.first] = e.second;
  return true;
}

std::string quoted(const std::string& s) {
  std::string o = "\"";
  for (char c : s) {
    if (c == '"' || c == '\\') o += '\\';
    o += c;
  }
  return o + "\"";
}

bool write_file(const char* path, const Table& t) {
  const std::string tmp = std::string(path) + ".tmp";
  FILE* f = std::fopen(tmp.c_str(), "w");
  if (!f) return false;
  std::fprintf(f, "{\n  \"format\": \"snmf_gb300 product tuning cache, v1\",\n  \"devices\": {");
  bool first_dev = true;
  for (const auto& d : t) {
    std::fprintf(f, "%s\n    %s: {", first_dev ? "" : ",", quoted(d.first).c_str());
    first_dev = false;
    bool first = true;
    for (const auto& e : d.second) {
      std::fprintf(f,
                   "%s\n      %s: {\"splits\": %d, \"stages\": %d, \"per_sm\": %d, \"bn\": %d, \"row_bm\": %d, "
                   "\"row_tc\": %d, \"ms\": %.6g}",
                   first ? "" : ",", quoted(e.first).c_str(), e.second.cfg.splits, e.second.cfg.stages,
                   e.second.cfg.per_sm, e.second.cfg.bn, e.second.cfg.row_bm, e.second.cfg.row_tc, e.second.ms);
      first = false;
    }
    std::fprintf(f, "\n    }");
  }
  std::fprintf(f, "\n  }\n}\n");
  const bool ok = std::fclose(f) == 0;
  return ok && std::rename(tmp.c_str(), path) == 0;
}

}  // namespace

std::string tune_device_key() {
  int dev = 0;
  cudaDeviceProp p{};
  if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&p, dev) != cudaSuccess) return "";
  return std::string(p.name) + "/" + std::to_string(p.multiProcessorCount);
}

bool tune_lookup(const char* path, const std::string& dev, const std::string& key, TuneEntry* out) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (path && *path) read_file(path, &g_mem);
  auto d = g_mem.find(dev);
  if (d == g_mem.end()) return false;
  auto e = d->second.find(key);
  if (e == d->second.end()) return false;
  *out = e->second;
  return true;
}

bool tune_store(const char* path, const std::string& dev, const std::string& key, const TuneEntry& e) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_mem[dev][key] = e;
  if (!(path && *path)) return true;
  Table t;
  read_file(path, &t);  // keep what other processes / devices wrote
  t[dev][key] = e;
  for (auto& d : g_mem)
    for (auto& x : d.second)
      if (!t[d.first].count(x.first)) t[d.first][x.first] = x.second;
  return write_file(path, t);
}

}  // namespace snmf
