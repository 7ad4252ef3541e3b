// Host-only part of the autotuner: the tuning's JSON form, the batch
// signature that keys the tuning cache, and the cache file itself. Nothing
// here touches the device.
//
// Tuning JSON (every key optional; missing keys keep their defaults):
//   {"blur_tile_rows": [[r_1, ..., r_{S+2}], ...],   one list per octave (or a
//                                                    flat list: octave 0)
//    "blur_ctas_per_sm": [c_0, c_1, ...],            per octave
//    "extrema_ctas_per_sm": c, "orientation_ctas_per_sm": c,
//    "descriptor_ctas_per_sm": c, "compaction_ctas_per_sm": c, "batch_lanes": 1 .. 4}
// r is 32 or 64; c is 0 (the occupancy maximum) or 1..64 (capped by the
// occupancy maximum at launch).
//
// Cache file: {"version": 1, "entries": {"<signature>": <tuning JSON>, ...}}.
#include <cerrno>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <utility>
#include <vector>

#include <algorithm>
#include <fstream>
#include <sstream>
#include <unistd.h>

#include "engine.h"

namespace sift {
namespace {

// A cursor over a NUL-terminated JSON text (the subset the tuning and the
// cache use: objects, arrays, strings without escapes beyond \" and \\,
// integers; other scalars are skipped but not interpreted).
struct Cur {
  const char *p;
  void ws() {
    while (*p == ' ' || *p == '\n' || *p == '\t' || *p == '\r') p++;
  }
  bool eat(char c) {
    ws();
    if (*p != c) return false;
    p++;
    return true;
  }
  bool at(char c) {
    ws();
    return *p == c;
  }
  bool str(std::string *out) {
    ws();
    if (*p != '"') return false;
    p++;
    std::string s;
    while (*p && *p != '"') {
      if (*p == '\\') {
        p++;
        if (!*p) return false;
      }
      s += *p++;
    }
    if (*p != '"') return false;
    p++;
    if (out) *out = s;
    return true;
  }
  bool integer(long *v) {
    ws();
    char *end = nullptr;
    errno = 0;
    const long x = std::strtol(p, &end, 10);
    if (end == p || errno != 0) return false;
    if (*end == '.' || *end == 'e' || *end == 'E') return false;  // integers only
    p = end;
    *v = x;
    return true;
  }
  // Skip one value of any kind; false if malformed or nested too deeply.
  bool skip(int depth = 0) {
    if (depth > 32) return false;
    ws();
    if (*p == '{') {
      p++;
      if (eat('}')) return true;
      do {
        if (!str(nullptr) || !eat(':') || !skip(depth + 1)) return false;
      } while (eat(','));
      return eat('}');
    }
    if (*p == '[') {
      p++;
      if (eat(']')) return true;
      do {
        if (!skip(depth + 1)) return false;
      } while (eat(','));
      return eat(']');
    }
    if (*p == '"') return str(nullptr);
    const char *q = p;
    while ((*p >= '0' && *p <= '9') || (*p >= 'a' && *p <= 'z') || *p == '-' || *p == '+' ||
           *p == '.' || *p == 'E')
      p++;
    return p != q;
  }
};

bool int_list(Cur &c, std::vector<long> *out) {
  if (!c.eat('[')) return false;
  out->clear();
  if (c.eat(']')) return true;
  do {
    long v;
    if (!c.integer(&v)) return false;
    out->push_back(v);
  } while (c.eat(','));
  return c.eat(']');
}

bool ctas_ok(long v) { return v >= 0 && v <= 64; }

}  // namespace

Tuning default_tuning() {
  Tuning t{};
  for (int o = 0; o < kMaxOct; o++) {
    for (int l = 0; l < kMaxLevels; l++) t.lvl_kind[o][l] = TK_BLUR32;
    t.blur_ctas[o] = 0;
  }
  t.ext_ctas = t.ori_ctas = t.desc_ctas = t.cmp_ctas = 0;
  t.batch_lanes = 2;
  return t;
}

std::string tuning_json(const Tuning &t, int S) {
  // Octaves are written up to the last one that differs from the default
  // (octave 0 always), so the common case stays one short line.
  int last_rows = 0, last_ctas = 0;
  for (int o = 0; o < kMaxOct; o++) {
    for (int l = 1; l <= S + 2; l++)
      if (t.lvl_kind[o][l] != TK_BLUR32) last_rows = o;
    if (t.blur_ctas[o] != 0) last_ctas = o;
  }
  std::string s = "{\"blur_tile_rows\": [";
  for (int o = 0; o <= last_rows; o++) {
    s += o ? ", [" : "[";
    for (int l = 1; l <= S + 2; l++) {
      s += std::to_string(t.lvl_kind[o][l] == TK_BLUR64 ? 64 : 32);
      if (l < S + 2) s += ", ";
    }
    s += "]";
  }
  s += "], \"blur_ctas_per_sm\": [";
  for (int o = 0; o <= last_ctas; o++) {
    s += std::to_string(t.blur_ctas[o]);
    if (o < last_ctas) s += ", ";
  }
  s += "], \"extrema_ctas_per_sm\": " + std::to_string(t.ext_ctas) +
       ", \"orientation_ctas_per_sm\": " + std::to_string(t.ori_ctas) +
       ", \"descriptor_ctas_per_sm\": " + std::to_string(t.desc_ctas) +
       ", \"compaction_ctas_per_sm\": " + std::to_string(t.cmp_ctas) +
       ", \"batch_lanes\": " + std::to_string(t.batch_lanes) + "}";
  return s;
}

bool parse_tuning(const char *json, int S, const Tuning &base, Tuning *out, std::string *why) {
  Tuning t = base;
  Cur c{json};
  auto bad = [&](const std::string &m) {
    if (why) *why = m;
    return false;
  };
  if (!c.eat('{')) return bad("tuning: expected a JSON object");
  if (!c.eat('}')) {
    do {
      std::string key;
      if (!c.str(&key) || !c.eat(':')) return bad("tuning: expected \"key\": value");
      if (key == "blur_tile_rows") {
        // A flat list (octave 0) or a list of per-octave lists.
        if (!c.eat('[')) return bad("tuning: blur_tile_rows must be a list");
        const bool nested = c.at('[');
        std::vector<std::vector<long>> rows;
        if (nested) {
          do {
            std::vector<long> r;
            if (!int_list(c, &r)) return bad("tuning: blur_tile_rows: expected lists of integers");
            rows.push_back(r);
          } while (c.eat(','));
        } else if (!c.at(']')) {
          std::vector<long> r;
          do {
            long v;
            if (!c.integer(&v)) return bad("tuning: blur_tile_rows: expected integers");
            r.push_back(v);
          } while (c.eat(','));
          rows.push_back(r);
        }
        if (!c.eat(']')) return bad("tuning: blur_tile_rows: unterminated list");
        if ((int)rows.size() > kMaxOct) return bad("tuning: blur_tile_rows: too many octaves");
        for (size_t o = 0; o < rows.size(); o++) {
          if ((int)rows[o].size() != S + 2)
            return bad("tuning: blur_tile_rows: each octave needs n_scales + 2 entries");
          for (int l = 1; l <= S + 2; l++) {
            const long v = rows[o][l - 1];
            if (v != 32 && v != 64) return bad("tuning: tile rows must be 32 or 64");
            t.lvl_kind[o][l] = v == 64 ? TK_BLUR64 : TK_BLUR32;
          }
        }
      } else if (key == "blur_ctas_per_sm") {
        std::vector<long> v;
        if (!int_list(c, &v)) return bad("tuning: blur_ctas_per_sm must be a list of integers");
        if ((int)v.size() > kMaxOct) return bad("tuning: blur_ctas_per_sm: too many octaves");
        for (size_t o = 0; o < v.size(); o++) {
          if (!ctas_ok(v[o])) return bad("tuning: CTAs per SM must be 0..64");
          t.blur_ctas[o] = (int)v[o];
        }
      } else if (key == "extrema_ctas_per_sm" || key == "orientation_ctas_per_sm" ||
                 key == "descriptor_ctas_per_sm" || key == "compaction_ctas_per_sm") {
        long v;
        if (!c.integer(&v) || !ctas_ok(v)) return bad("tuning: " + key + " must be 0..64");
        (key[0] == 'e'   ? t.ext_ctas
         : key[0] == 'o' ? t.ori_ctas
         : key[0] == 'd' ? t.desc_ctas
                         : t.cmp_ctas) = (int)v;
      } else if (key == "batch_lanes") {
        long v;
        if (!c.integer(&v) || v < 1 || v > kMaxLanes) return bad("tuning: batch_lanes must be 1 to 4");
        t.batch_lanes = (int)v;
      } else {
        return bad("tuning: unknown key \"" + key + "\"");
      }
    } while (c.eat(','));
    if (!c.eat('}')) return bad("tuning: expected '}'");
  }
  c.ws();
  if (*c.p) return bad("tuning: trailing characters");
  *out = t;
  return true;
}

std::string batch_signature(const sift_params &p, int n, const int *H, const int *W) {
  // Every parameter that changes the work, the image count, and the multiset
  // of image shapes (sorted, so a reordered batch has the same signature):
  // readable totals plus a 64-bit FNV-1a hash of the sorted shapes.
  std::vector<std::pair<int, int>> sh(n);
  long long px = 0;
  int side = 0;
  for (int i = 0; i < n; i++) {
    sh[i] = {H[i], W[i]};
    px += (long long)H[i] * W[i];
    side = std::max(side, std::max(H[i], W[i]));
  }
  std::sort(sh.begin(), sh.end());
  uint64_t h = 1469598103934665603ull;
  auto mix = [&](uint32_t v) {
    for (int k = 0; k < 4; k++) {
      h ^= (v >> (8 * k)) & 0xffu;
      h *= 1099511628211ull;
    }
  };
  for (auto &s : sh) {
    mix((uint32_t)s.first);
    mix((uint32_t)s.second);
  }
  char buf[512];
  std::snprintf(buf, sizeof buf,
                "S%d,s%.7g,b%.7g,up%d,umax%d,mos%d,ct%.7g,er%.7g,bd%d,it%d,pf%.7g,pk%.7g,cap%d,"
                "ur%d,dsp%d,rs%d,h%d;n%d;px%lld;side%d;shapes%016llx",
                p.n_scales, p.sigma0, p.init_blur, p.upsample, p.upsample_max_px,
                p.min_octave_side, p.contrast_thr, p.edge_ratio, p.border, p.max_refine_iter,
                p.prefilter_ratio, p.ori_peak_ratio, p.max_kpts, p.upright, p.dsp, p.rootsift,
                p.fp16_pyramid, n, px, side, (unsigned long long)h);
  return buf;
}

namespace {

bool key_ok(const char *k) {
  if (!k || !*k || std::strlen(k) > 1024) return false;
  for (const char *q = k; *q; q++)
    if (*q == '"' || *q == '\\' || (unsigned char)*q < 0x20) return false;
  return true;
}

bool read_file(const char *path, std::string *out) {
  std::ifstream f(path, std::ios::binary);
  if (!f) return false;
  std::ostringstream ss;
  ss << f.rdbuf();
  *out = ss.str();
  return true;
}

// Entries of a cache text, in file order, as (signature, raw JSON value).
bool parse_cache(const std::string &text, std::vector<std::pair<std::string, std::string>> *ents) {
  Cur c{text.c_str()};
  if (!c.eat('{')) return false;
  bool version_ok = false;
  if (!c.eat('}')) {
    do {
      std::string key;
      if (!c.str(&key) || !c.eat(':')) return false;
      if (key == "version") {
        long v;
        if (!c.integer(&v) || v != 1) return false;
        version_ok = true;
      } else if (key == "entries") {
        if (!c.eat('{')) return false;
        if (!c.eat('}')) {
          do {
            std::string sig;
            if (!c.str(&sig) || !c.eat(':')) return false;
            c.ws();
            const char *b = c.p;
            if (!c.skip()) return false;
            ents->emplace_back(sig, std::string(b, c.p));
          } while (c.eat(','));
          if (!c.eat('}')) return false;
        }
      } else if (!c.skip()) {
        return false;
      }
    } while (c.eat(','));
    if (!c.eat('}')) return false;
  }
  c.ws();
  return version_ok && *c.p == 0;
}

}  // namespace

sift_status cache_get(const char *path, const char *sig, std::string *json) {
  if (!path || !*path || !key_ok(sig)) return SIFT_E_INVALID;
  std::string text;
  if (!read_file(path, &text)) return SIFT_E_NOTFOUND;
  std::vector<std::pair<std::string, std::string>> ents;
  if (!parse_cache(text, &ents)) return SIFT_E_INVALID;
  for (auto &e : ents)
    if (e.first == sig) {
      *json = e.second;
      return SIFT_OK;
    }
  return SIFT_E_NOTFOUND;
}

sift_status cache_put(const char *path, const char *sig, const char *json) {
  if (!path || !*path || !key_ok(sig) || !json) return SIFT_E_INVALID;
  {
    Cur c{json};
    if (!c.at('{') || !c.skip()) return SIFT_E_INVALID;
    c.ws();
    if (*c.p) return SIFT_E_INVALID;
  }
  std::vector<std::pair<std::string, std::string>> ents;
  std::string text;
  if (read_file(path, &text) && !parse_cache(text, &ents))
    return SIFT_E_INVALID;  // an unreadable cache is left as it is, not overwritten
  bool found = false;
  for (auto &e : ents)
    if (e.first == sig) {
      e.second = json;
      found = true;
    }
  if (!found) ents.emplace_back(sig, json);
  std::string out = "{\"version\": 1, \"entries\": {";
  for (size_t i = 0; i < ents.size(); i++) {
    out += i ? ",\n  \"" : "\n  \"";
    out += ents[i].first + "\": " + ents[i].second;
  }
  out += "\n}}\n";
  // Written beside the target and renamed over it, so a reader sees either
  // the old file or the new one. Concurrent writers: the last rename wins.
  const std::string tmp = std::string(path) + ".tmp." + std::to_string((long)getpid());
  {
    std::ofstream f(tmp, std::ios::binary | std::ios::trunc);
    if (!f) return SIFT_E_INVALID;
    f << out;
    f.flush();
    if (!f) {
      std::remove(tmp.c_str());
      return SIFT_E_INVALID;
    }
  }
  if (std::rename(tmp.c_str(), path) != 0) {
    std::remove(tmp.c_str());
    return SIFT_E_INVALID;
  }
  return SIFT_OK;
}

}  // namespace sift

extern "C" {

sift_status sift_batch_signature(const sift_params *p, int n, const int *H, const int *W,
                                 char *out, size_t len) {
  if (!p || n < 1 || !H || !W || !out || len == 0) return SIFT_E_INVALID;
  std::string why;
  if (sift::validate_params(*p, &why) != SIFT_OK) return SIFT_E_INVALID;
  for (int i = 0; i < n; i++)
    if (H[i] < 1 || W[i] < 1) return SIFT_E_INVALID;
  const std::string s = sift::batch_signature(*p, n, H, W);
  if (s.size() + 1 > len) return SIFT_E_INVALID;
  std::memcpy(out, s.c_str(), s.size() + 1);
  return SIFT_OK;
}

sift_status sift_tuning_cache_get(const char *path, const char *signature, char *json, size_t len) {
  if (!json || len == 0) return SIFT_E_INVALID;
  std::string s;
  const sift_status st = sift::cache_get(path, signature, &s);
  if (st != SIFT_OK) return st;
  if (s.size() + 1 > len) return SIFT_E_INVALID;
  std::memcpy(json, s.c_str(), s.size() + 1);
  return SIFT_OK;
}

sift_status sift_tuning_cache_put(const char *path, const char *signature, const char *json) {
  return sift::cache_put(path, signature, json);
}

}  // extern "C"
