// Launch-shape tuning: a process-wide table of knob values, keyed by knob name,
// point dimension and problem-size bucket (floor(log2(N M))), that the shape
// functions of the sweeps consult.  Every knob has a fixed set of allowed
// values (each one a shape the kernels are compiled for), so a tuned shape is
// always a valid launch; a value of 0 clears an entry.  The table is filled by
// uot_tune_set or uot_tune_load (a JSON file written by the autotuner of the
// Python package, which measures the candidates on the device it runs on);
// plans load the file named by UOT_TUNE_FILE once, at their first creation.
#include <cuda_runtime.h>

#include <cstdarg>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "uot_internal.cuh"

namespace uot {
namespace {

uot_status fail(uot_status s, const char* fmt, ...) __attribute__((format(printf, 2, 3)));
uot_status fail(uot_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  set_last_error(buf);
  return s;
}

struct Knob {
  const char* name;
  long long allowed[6];  // 0-terminated
};

// rows per thread of the tiled sweep; its per-CTA fixed cost (tenths of a tile)
// in the choice of key chunks; the fewest waves of CTAs it may choose; rows per thread of the direct sweep (dim <= 3);
// resident CTAs per SM the direct sweep's chunking aims at; columns per CTA of
// the dense row sweep; CTAs per SM of the dense column sweep; CTAs per SM of
// the batched solver's persistent grid
const Knob kKnobs[] = {
    {"tile.rows", {2, 4, 0}},
    {"tile.cta_cost", {5, 10, 15, 25, 40, 0}},
    {"tile.waves", {1, 2, 3, 4, 0}},
    {"points.rows", {1, 2, 4, 0}},
    {"points.resident", {2, 3, 4, 6, 0}},
    {"dense.row_chunk", {2048, 4096, 8192, 0}},
    {"dense.col_ctas", {2, 4, 8, 0}},
    {"batch.ctas_per_sm", {1, 2, 3, 4, 0}},
};

struct Entry {
  std::string knob;
  int dim, bucket;
  long long value;
};

std::mutex g_mu;
std::vector<Entry> g_tab;
// values fixed for this thread by a TuneScope (workspace sizing)
thread_local std::vector<TuneFix> t_fix;

const Knob* find_knob(const char* name) {
  if (!name) return nullptr;
  for (const Knob& k : kKnobs)
    if (std::strcmp(k.name, name) == 0) return &k;
  return nullptr;
}

bool allowed(const Knob& k, long long v) {
  for (int i = 0; i < 6 && k.allowed[i] != 0; ++i)
    if (k.allowed[i] == v) return true;
  return false;
}

uot_status set_entry(const char* knob, int dim, int bucket, long long value) {
  const Knob* k = find_knob(knob);
  if (!k) return fail(UOT_ERR_INVALID_ARG, "unknown tuning knob '%s'", knob ? knob : "(null)");
  if (dim < -1 || dim > 64 || bucket < -1 || bucket > 126)
    return fail(UOT_ERR_INVALID_ARG, "tuning key out of range (dim %d, bucket %d)", dim, bucket);
  if (value != 0 && !allowed(*k, value))
    return fail(UOT_ERR_INVALID_ARG, "value %lld not allowed for knob '%s'", value, knob);
  std::lock_guard<std::mutex> lk(g_mu);
  for (size_t i = 0; i < g_tab.size(); ++i) {
    Entry& e = g_tab[i];
    if (e.knob == knob && e.dim == dim && e.bucket == bucket) {
      if (value == 0) g_tab.erase(g_tab.begin() + (long)i);
      else e.value = value;
      return UOT_OK;
    }
  }
  if (value != 0) g_tab.push_back(Entry{knob, dim, bucket, value});
  return UOT_OK;
}

// ---- the cache file: {"entries": [{"knob": "...", "dim": d, "bucket": b, "value": v}, ...]}
// (other keys are ignored).  A minimal reader for exactly this layout.
struct Reader {
  const char* s;
  size_t i, n;
  void ws() {
    while (i < n && (s[i] == ' ' || s[i] == '\n' || s[i] == '\r' || s[i] == '\t')) ++i;
  }
  bool lit(char c) {
    ws();
    if (i < n && s[i] == c) { ++i; return true; }
    return false;
  }
  bool str(std::string& out) {
    ws();
    if (i >= n || s[i] != '"') return false;
    ++i;
    out.clear();
    while (i < n && s[i] != '"') {
      if (s[i] == '\\' && i + 1 < n) ++i;
      out.push_back(s[i++]);
    }
    if (i >= n) return false;
    ++i;
    return true;
  }
  bool num(double& v) {
    ws();
    char* end = nullptr;
    v = std::strtod(s + i, &end);
    if (end == s + i) return false;
    i = (size_t)(end - s);
    return true;
  }
  // skips one value of any kind
  bool skip() {
    ws();
    if (i >= n) return false;
    if (s[i] == '"') { std::string t; return str(t); }
    if (s[i] == '{' || s[i] == '[') {
      const char open = s[i], close = open == '{' ? '}' : ']';
      int depth = 0;
      bool in_str = false;
      for (; i < n; ++i) {
        const char c = s[i];
        if (in_str) {
          if (c == '\\') ++i;
          else if (c == '"') in_str = false;
        } else if (c == '"') in_str = true;
        else if (c == open) ++depth;
        else if (c == close && --depth == 0) { ++i; return true; }
      }
      return false;
    }
    while (i < n && s[i] != ',' && s[i] != '}' && s[i] != ']') ++i;
    return true;
  }
};

bool parse_entry(Reader& r, std::vector<Entry>& out) {
  if (!r.lit('{')) return false;
  Entry e{"", -1, -1, 0};
  bool have_knob = false, have_value = false;
  if (r.lit('}')) return false;
  do {
    std::string key;
    if (!r.str(key) || !r.lit(':')) return false;
    double v = 0.0;
    if (key == "knob") {
      if (!r.str(e.knob)) return false;
      have_knob = true;
    } else if (key == "dim" || key == "bucket" || key == "value") {
      if (!r.num(v)) return false;
      if (key == "dim") e.dim = (int)v;
      else if (key == "bucket") e.bucket = (int)v;
      else { e.value = (long long)v; have_value = true; }
    } else if (!r.skip()) {
      return false;
    }
  } while (r.lit(','));
  if (!r.lit('}') || !have_knob || !have_value) return false;
  out.push_back(e);
  return true;
}

bool parse_cache(const std::string& text, std::vector<Entry>& out) {
  Reader r{text.c_str(), 0, text.size()};
  if (!r.lit('{')) return false;
  if (r.lit('}')) return true;
  do {
    std::string key;
    if (!r.str(key) || !r.lit(':')) return false;
    if (key == "entries") {
      if (!r.lit('[')) return false;
      if (!r.lit(']')) {
        do {
          if (!parse_entry(r, out)) return false;
        } while (r.lit(','));
        if (!r.lit(']')) return false;
      }
    } else if (!r.skip()) {
      return false;
    }
  } while (r.lit(','));
  return r.lit('}');
}

uot_status load_file(const char* path) {
  if (!path) return fail(UOT_ERR_INVALID_ARG, "path is NULL");
  FILE* fp = std::fopen(path, "rb");
  if (!fp) return fail(UOT_ERR_INVALID_ARG, "cannot open tuning file '%s'", path);
  std::string text;
  char buf[4096];
  size_t got;
  while ((got = std::fread(buf, 1, sizeof(buf), fp)) > 0) text.append(buf, got);
  std::fclose(fp);
  std::vector<Entry> es;
  if (!parse_cache(text, es)) return fail(UOT_ERR_INVALID_ARG, "tuning file '%s' is not a tuning cache", path);
  // validate everything before changing the table
  for (const Entry& e : es) {
    const Knob* k = find_knob(e.knob.c_str());
    if (!k || (e.value != 0 && !allowed(*k, e.value)) || e.dim < -1 || e.dim > 64 || e.bucket < -1 ||
        e.bucket > 126)
      return fail(UOT_ERR_INVALID_ARG, "tuning file '%s': bad entry for knob '%s'", path, e.knob.c_str());
  }
  for (const Entry& e : es) set_entry(e.knob.c_str(), e.dim, e.bucket, e.value);
  return UOT_OK;
}

}  // namespace

int tune_bucket(long long entries) {
  if (entries <= 1) return 0;
  int b = 0;
  while (b < 126 && (entries >> (b + 1)) > 0) ++b;
  return b;
}

TuneScope::TuneScope(const TuneFix* f, int n) : n_(n) {
  for (int i = 0; i < n; ++i) t_fix.push_back(f[i]);
}
TuneScope::~TuneScope() { t_fix.resize(t_fix.size() - (size_t)n_); }

std::vector<long long> tune_allowed(const char* knob) {
  std::vector<long long> v;
  if (const Knob* k = find_knob(knob))
    for (int i = 0; i < 6 && k->allowed[i] != 0; ++i) v.push_back(k->allowed[i]);
  return v;
}

long long tune_value(const char* knob, int dim, long long entries, long long dflt) {
  for (size_t i = t_fix.size(); i-- > 0;)
    if (std::strcmp(t_fix[i].knob, knob) == 0) return t_fix[i].value;
  const int bucket = entries > 0 ? tune_bucket(entries) : -1;
  std::lock_guard<std::mutex> lk(g_mu);
  if (g_tab.empty()) return dflt;
  // most specific match first: (dim, bucket), (dim, any), (any, bucket), (any, any)
  const int keys[4][2] = {{dim, bucket}, {dim, -1}, {-1, bucket}, {-1, -1}};
  for (const auto& k : keys) {
    if ((k[0] != -1 && dim < 0) || (k[1] != -1 && bucket < 0)) continue;
    for (const Entry& e : g_tab)
      if (e.dim == k[0] && e.bucket == k[1] && e.knob == knob) return e.value;
  }
  return dflt;
}

void tune_autoload() {
  static std::once_flag once;
  std::call_once(once, [] {
    const char* path = std::getenv("UOT_TUNE_FILE");
    if (path && *path) load_file(path);  // a bad file leaves the defaults (uot_tune_load reports why)
  });
}

}  // namespace uot

using namespace uot;

extern "C" uot_status uot_tune_set(const char* knob, int32_t dim, int32_t bucket, int64_t value) {
  return set_entry(knob, dim, bucket, value);
}

extern "C" uot_status uot_tune_get(const char* knob, int32_t dim, int64_t entries, int64_t* value) {
  if (!value) return fail(UOT_ERR_INVALID_ARG, "value is NULL");
  if (!find_knob(knob)) return fail(UOT_ERR_INVALID_ARG, "unknown tuning knob '%s'", knob ? knob : "(null)");
  *value = tune_value(knob, dim, entries, 0);
  return UOT_OK;
}

extern "C" int32_t uot_tune_bucket(int64_t entries) { return tune_bucket(entries); }

extern "C" uot_status uot_tune_clear(void) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_tab.clear();
  return UOT_OK;
}

extern "C" uot_status uot_tune_load(const char* path) { return load_file(path); }
