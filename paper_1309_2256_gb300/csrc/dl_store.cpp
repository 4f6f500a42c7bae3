// Base-2 storage of per-noise loop arrays (App. A, "Binary storage system",
// Fig. St).
//
// Each noise vector's loops are an array of n_values doubles.  Sources are
// numbered from 0 in the order they are added.  The file of weight w = 2^k holds
// the elementwise sum of the arrays of sources w-1 .. 2w-2 (weight 1: source 0,
// weight 2: sources 1-2, weight 4: sources 3-6, ...).  With K complete files the
// sum over a set of any n < 2^K sources is the sum of the files whose weights are
// the set bits of n, so N sources need O(log2 N) files instead of N.
//
// File "<prefix>.<w>" (and "<prefix>.partial" for an incomplete group), all
// integers little-endian:
//   0  char[8]  "DLLOOPB2"
//   8  u32      format version (1)
//  12  u32      0
//  16  u64      weight w of the group
//  24  u64      sources summed (w for a complete file, 1 .. w-1 for .partial)
//  32  u64      index of the group's first source (w - 1)
//  40  u64      n_values
//  48  u64      FNV-1a 64 of the payload bytes
//  56  f64[n_values]  the sum, IEEE binary64 little-endian
// Host code only: it works on loop arrays the caller has copied to host memory.
#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <memory>
#include <new>
#include <string>
#include <vector>

#include "discloop.h"

struct dl_store {
  std::string prefix;
  int64_t n_values = 0;
  uint64_t weight = 1;    // weight of the group being filled
  uint64_t in_group = 0;  // sources of that group added so far
  uint64_t total = 0;     // sources added, complete groups included
  std::vector<double> acc;
};

namespace {

thread_local std::string g_err;

dl_status fail(dl_status st, const std::string& msg) {
  g_err = msg;
  return st;
}

const unsigned char kMagic[8] = {'D', 'L', 'L', 'O', 'O', 'P', 'B', '2'};
const uint32_t kVersion = 1;
const size_t kHeader = 56;
const int kMaxLog = 62;                      // weights up to 2^62
const int64_t kMaxValues = int64_t(1) << 40;  // 8 TiB of payload per file

void put_u64(unsigned char* p, uint64_t v) {
  for (int i = 0; i < 8; ++i) p[i] = (unsigned char)(v >> (8 * i));
}
uint64_t get_u64(const unsigned char* p) {
  uint64_t v = 0;
  for (int i = 0; i < 8; ++i) v |= (uint64_t)p[i] << (8 * i);
  return v;
}
void put_u32(unsigned char* p, uint32_t v) {
  for (int i = 0; i < 4; ++i) p[i] = (unsigned char)(v >> (8 * i));
}
uint32_t get_u32(const unsigned char* p) {
  uint32_t v = 0;
  for (int i = 0; i < 4; ++i) v |= (uint32_t)p[i] << (8 * i);
  return v;
}

// FNV-1a, 64-bit (Fowler, Noll, Vo): offset basis and prime of the published definition.
uint64_t fnv1a64(const unsigned char* p, size_t n) {
  uint64_t h = 14695981039346656037ull;
  for (size_t i = 0; i < n; ++i) {
    h ^= p[i];
    h *= 1099511628211ull;
  }
  return h;
}

std::string group_path(const std::string& prefix, uint64_t w) { return prefix + "." + std::to_string(w); }
std::string partial_path(const std::string& prefix) { return prefix + ".partial"; }

bool file_exists(const std::string& path) {
  FILE* f = std::fopen(path.c_str(), "rb");
  if (!f) return false;
  std::fclose(f);
  return true;
}

struct Header {
  uint64_t weight, count, first, n_values, checksum;
};

dl_status write_group(const std::string& path, uint64_t weight, uint64_t count, const std::vector<double>& sum) {
  const size_t n = sum.size();
  std::vector<unsigned char> buf(kHeader + 8 * n);
  unsigned char* pay = buf.data() + kHeader;
  for (size_t i = 0; i < n; ++i) {
    uint64_t bits;
    std::memcpy(&bits, &sum[i], 8);
    put_u64(pay + 8 * i, bits);
  }
  std::memcpy(buf.data(), kMagic, 8);
  put_u32(buf.data() + 8, kVersion);
  put_u32(buf.data() + 12, 0);
  put_u64(buf.data() + 16, weight);
  put_u64(buf.data() + 24, count);
  put_u64(buf.data() + 32, weight - 1);
  put_u64(buf.data() + 40, (uint64_t)n);
  put_u64(buf.data() + 48, fnv1a64(pay, 8 * n));
  // write beside the target and rename, so that a reader never sees half a file
  const std::string tmp = path + ".tmp";
  FILE* f = std::fopen(tmp.c_str(), "wb");
  if (!f) return fail(DL_ERR_IO, "cannot create " + tmp);
  const bool ok = std::fwrite(buf.data(), 1, buf.size(), f) == buf.size();
  const bool closed = std::fclose(f) == 0;
  if (!ok || !closed) {
    std::remove(tmp.c_str());
    return fail(DL_ERR_IO, "cannot write " + tmp);
  }
  if (std::rename(tmp.c_str(), path.c_str()) != 0) {
    std::remove(tmp.c_str());
    return fail(DL_ERR_IO, "cannot rename " + tmp + " to " + path);
  }
  return DL_OK;
}

// Reads and checks one file; payload (if not NULL) receives n_values doubles.
dl_status read_group(const std::string& path, int64_t n_values, Header* h, std::vector<double>* payload) {
  FILE* f = std::fopen(path.c_str(), "rb");
  if (!f) return fail(DL_ERR_IO, "missing " + path);
  unsigned char head[kHeader];
  if (std::fread(head, 1, kHeader, f) != kHeader) {
    std::fclose(f);
    return fail(DL_ERR_IO, path + ": truncated header");
  }
  if (std::memcmp(head, kMagic, 8) != 0 || get_u32(head + 8) != kVersion) {
    std::fclose(f);
    return fail(DL_ERR_IO, path + ": not a loop store file of version 1");
  }
  h->weight = get_u64(head + 16);
  h->count = get_u64(head + 24);
  h->first = get_u64(head + 32);
  h->n_values = get_u64(head + 40);
  h->checksum = get_u64(head + 48);
  if (h->n_values != (uint64_t)n_values) {
    std::fclose(f);
    return fail(DL_ERR_IO, path + ": holds " + std::to_string(h->n_values) + " values, expected " +
                               std::to_string(n_values));
  }
  std::vector<unsigned char> pay((size_t)n_values * 8);
  const bool ok = std::fread(pay.data(), 1, pay.size(), f) == pay.size();
  const bool at_end = ok && std::fgetc(f) == EOF;
  std::fclose(f);
  if (!ok) return fail(DL_ERR_IO, path + ": truncated payload");
  if (!at_end) return fail(DL_ERR_IO, path + ": trailing bytes after the payload");
  if (fnv1a64(pay.data(), pay.size()) != h->checksum) return fail(DL_ERR_IO, path + ": checksum mismatch");
  if (payload) {
    payload->resize((size_t)n_values);
    for (int64_t i = 0; i < n_values; ++i) {
      const uint64_t bits = get_u64(pay.data() + 8 * i);
      std::memcpy(&(*payload)[(size_t)i], &bits, 8);
    }
  }
  return DL_OK;
}

bool is_group_header(const Header& h, uint64_t w) { return h.weight == w && h.first == w - 1; }

// Writes the current group once it is complete and starts the next one.
dl_status flush_complete(dl_store* s) {
  if (s->in_group < s->weight) return DL_OK;
  dl_status st = write_group(group_path(s->prefix, s->weight), s->weight, s->weight, s->acc);
  if (st != DL_OK) return st;
  std::remove(partial_path(s->prefix).c_str());  // an earlier snapshot of this group, if any
  std::fill(s->acc.begin(), s->acc.end(), 0.0);
  s->in_group = 0;
  s->weight <<= 1;
  return DL_OK;
}

// Runs f; host allocation failures and any other exception become status codes
// (nothing is thrown across the C boundary).
template <class F>
dl_status guarded(const char* name, F&& f) {
  try {
    return f();
  } catch (const std::bad_alloc&) {
    return fail(DL_ERR_OOM, std::string(name) + ": host allocation failed");
  } catch (...) {
    return fail(DL_ERR_IO, std::string(name) + ": unexpected host error");
  }
}

dl_status open_store(dl_store** out, const char* prefix, int64_t n_values, int resume) {
  std::unique_ptr<dl_store> s(new dl_store);
  s->prefix = prefix;
  s->n_values = n_values;
  s->acc.assign((size_t)n_values, 0.0);
  if (!resume) {
    std::vector<std::string> names{partial_path(s->prefix)};
    for (int k = 0; k <= kMaxLog; ++k) names.push_back(group_path(s->prefix, uint64_t(1) << k));
    for (const std::string& p : names)
      if (file_exists(p))
        return fail(DL_ERR_STATE, "dl_store_open: " + p + " exists (resume, or remove the earlier store)");
    *out = s.release();
    return DL_OK;
  }
  // resume: the complete files 1, 2, 4, ... without a gap, then the partial group
  Header h;
  int k = 0;
  for (; k <= kMaxLog; ++k) {
    const uint64_t w = uint64_t(1) << k;
    const std::string p = group_path(s->prefix, w);
    if (!file_exists(p)) break;
    dl_status st = read_group(p, n_values, &h, nullptr);
    if (st != DL_OK) return st;
    if (!is_group_header(h, w) || h.count != w)
      return fail(DL_ERR_IO, p + ": header does not describe the group of weight " + std::to_string(w));
    s->total += w;
    s->weight = w << 1;
  }
  for (int j = k + 1; j <= kMaxLog; ++j) {
    const std::string p = group_path(s->prefix, uint64_t(1) << j);
    if (file_exists(p)) return fail(DL_ERR_IO, "dl_store_open: " + p + " exists but a lighter group file is missing");
  }
  const std::string pp = partial_path(s->prefix);
  if (file_exists(pp)) {
    dl_status st = read_group(pp, n_values, &h, &s->acc);
    if (st != DL_OK) return st;
    if (!is_group_header(h, s->weight) || h.count == 0 || h.count >= s->weight)
      return fail(DL_ERR_IO, pp + ": does not continue the complete files");
    s->in_group = h.count;
    s->total += h.count;
  }
  *out = s.release();
  return DL_OK;
}

dl_status add_sources(dl_store* s, const double* values, int64_t n_sources) {
  // a group completed by an earlier call whose write failed goes out first
  dl_status st = flush_complete(s);
  if (st != DL_OK) return st;
  const size_t nv = (size_t)s->n_values;
  for (int64_t r = 0; r < n_sources; ++r) {
    if (s->weight > (uint64_t(1) << kMaxLog)) return fail(DL_ERR_ARG, "dl_store_add: more than 2^63 - 1 sources");
    const double* v = values + (size_t)r * nv;
    double* a = s->acc.data();
    for (size_t i = 0; i < nv; ++i) a[i] += v[i];
    ++s->in_group;
    ++s->total;
    st = flush_complete(s);
    if (st != DL_OK) return st;
  }
  return DL_OK;
}

dl_status close_store(dl_store* s) {
  dl_status st = flush_complete(s);
  if (st != DL_OK) return st;
  if (s->in_group > 0) return write_group(partial_path(s->prefix), s->weight, s->in_group, s->acc);
  std::remove(partial_path(s->prefix).c_str());
  return DL_OK;
}

dl_status load_sum(const char* prefix, int64_t n_values, int64_t n, double* out) {
  std::vector<double> sum((size_t)n_values, 0.0), file;
  Header h;
  for (int k = 0; k <= kMaxLog; ++k) {
    const uint64_t w = uint64_t(1) << k;
    if (!((uint64_t)n & w)) continue;
    const std::string p = group_path(prefix, w);
    dl_status st = read_group(p, n_values, &h, &file);
    if (st != DL_OK) return st;
    if (!is_group_header(h, w) || h.count != w)
      return fail(DL_ERR_IO, p + ": header does not describe the group of weight " + std::to_string(w));
    for (int64_t i = 0; i < n_values; ++i) sum[(size_t)i] += file[(size_t)i];
  }
  std::memcpy(out, sum.data(), sizeof(double) * (size_t)n_values);
  return DL_OK;
}

}  // namespace

extern "C" {

const char* dl_store_last_error(void) { return g_err.c_str(); }

dl_status dl_store_open(dl_store** out, const char* prefix, int64_t n_values, int resume) {
  if (!out) return fail(DL_ERR_ARG, "dl_store_open: out is NULL");
  *out = nullptr;
  if (!prefix || !*prefix) return fail(DL_ERR_ARG, "dl_store_open: empty prefix");
  if (n_values < 1 || n_values > kMaxValues) return fail(DL_ERR_ARG, "dl_store_open: n_values out of range");
  if (resume != 0 && resume != 1) return fail(DL_ERR_ARG, "dl_store_open: resume must be 0 or 1");
  return guarded("dl_store_open", [&] { return open_store(out, prefix, n_values, resume); });
}

dl_status dl_store_add(dl_store* s, const double* values, int64_t n_sources) {
  if (!s) return fail(DL_ERR_ARG, "dl_store_add: store is NULL");
  if (n_sources < 0 || (n_sources > 0 && !values)) return fail(DL_ERR_ARG, "dl_store_add: bad sources");
  return guarded("dl_store_add", [&] { return add_sources(s, values, n_sources); });
}

dl_status dl_store_count(const dl_store* s, int64_t* total) {
  if (!s || !total) return fail(DL_ERR_ARG, "dl_store_count: NULL argument");
  *total = (int64_t)s->total;
  return DL_OK;
}

dl_status dl_store_close(dl_store* s) {
  if (!s) return DL_OK;
  std::unique_ptr<dl_store> owned(s);
  return guarded("dl_store_close", [&] { return close_store(s); });
}

dl_status dl_store_load(const char* prefix, int64_t n_values, int64_t n, double* out) {
  if (!prefix || !*prefix) return fail(DL_ERR_ARG, "dl_store_load: empty prefix");
  if (n_values < 1 || n_values > kMaxValues || n < 0 || !out) return fail(DL_ERR_ARG, "dl_store_load: bad arguments");
  return guarded("dl_store_load", [&] { return load_sum(prefix, n_values, n, out); });
}

dl_status dl_store_sources(int64_t n, int64_t* list) {
  if (n < 0) return fail(DL_ERR_ARG, "dl_store_sources: n < 0");
  if (!list) return DL_OK;
  int64_t j = 0;
  for (int k = 0; k <= kMaxLog; ++k) {
    const uint64_t w = uint64_t(1) << k;
    if (!((uint64_t)n & w)) continue;
    for (uint64_t i = 0; i < w; ++i) list[j++] = (int64_t)(w - 1 + i);
  }
  return DL_OK;
}

}  // extern "C"
