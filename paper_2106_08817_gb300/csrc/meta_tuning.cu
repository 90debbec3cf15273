// Tile-shape table on disk: a JSON file of tuned tile shapes per problem shape
// (ndim, extents, batch, sigma), written and read by meta_tuning_save /
// meta_tuning_load, and the cache that meta_autotune consults and extends
// once meta_tuning_cache names a file.  Host code only: a small JSON reader
// (objects, arrays, numbers, strings, true / false / null) and writer for
// this one format.  The tile shapes change no result (every output is summed
// in the same order whatever the tiles), so a stale or foreign file can only
// cost time; a malformed one is refused as a whole.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include <unistd.h>

#include "meta.h"
#include "meta_kernels.h"

namespace meta {
namespace {

// ------------------------------------------------------------------ reader

struct JVal {
    enum Kind { NUL, BOOL, NUM, STR, ARR, OBJ } kind = NUL;
    double num = 0.0;
    bool b = false;
    std::string str;
    std::vector<JVal> arr;
    std::vector<std::pair<std::string, JVal>> obj;
    const JVal* get(const char* key) const {
        if (kind != OBJ) return nullptr;
        for (const auto& kv : obj)
            if (kv.first == key) return &kv.second;
        return nullptr;
    }
};

class JReader {
  public:
    JReader(const char* p, const char* e) : p_(p), e_(e) {}
    bool parse(JVal* out) {
        if (!value(out, 0)) return false;
        ws();
        return p_ == e_;  // nothing but white space after the value
    }

  private:
    const char* p_;
    const char* e_;
    static constexpr int kMaxDepth = 32;

    void ws() {
        while (p_ < e_ && (*p_ == ' ' || *p_ == '\t' || *p_ == '\n' || *p_ == '\r')) ++p_;
    }
    bool lit(const char* w) {
        const size_t n = std::strlen(w);
        if ((size_t)(e_ - p_) < n || std::memcmp(p_, w, n) != 0) return false;
        p_ += n;
        return true;
    }
    static bool digit(char c) { return c >= '0' && c <= '9'; }
    bool number(double* v) {
        const char* s = p_;
        if (p_ < e_ && *p_ == '-') ++p_;
        if (p_ >= e_ || !digit(*p_)) return false;
        if (*p_ == '0') {
            ++p_;
        } else {
            while (p_ < e_ && digit(*p_)) ++p_;
        }
        if (p_ < e_ && *p_ == '.') {
            ++p_;
            if (p_ >= e_ || !digit(*p_)) return false;
            while (p_ < e_ && digit(*p_)) ++p_;
        }
        if (p_ < e_ && (*p_ == 'e' || *p_ == 'E')) {
            ++p_;
            if (p_ < e_ && (*p_ == '+' || *p_ == '-')) ++p_;
            if (p_ >= e_ || !digit(*p_)) return false;
            while (p_ < e_ && digit(*p_)) ++p_;
        }
        const std::string tok(s, p_);
        char* end = nullptr;
        *v = std::strtod(tok.c_str(), &end);
        return end == tok.c_str() + tok.size() && std::isfinite(*v);
    }
    static int hexval(char c) {
        if (c >= '0' && c <= '9') return c - '0';
        if (c >= 'a' && c <= 'f') return c - 'a' + 10;
        if (c >= 'A' && c <= 'F') return c - 'A' + 10;
        return -1;
    }
    bool string(std::string* out) {
        if (p_ >= e_ || *p_ != '"') return false;
        ++p_;
        out->clear();
        while (p_ < e_ && *p_ != '"') {
            const unsigned char c = (unsigned char)*p_++;
            if (c < 0x20) return false;  // control characters must be escaped
            if (c != '\\') {
                out->push_back((char)c);
                continue;
            }
            if (p_ >= e_) return false;
            const char esc = *p_++;
            switch (esc) {
                case '"': out->push_back('"'); break;
                case '\\': out->push_back('\\'); break;
                case '/': out->push_back('/'); break;
                case 'b': out->push_back('\b'); break;
                case 'f': out->push_back('\f'); break;
                case 'n': out->push_back('\n'); break;
                case 'r': out->push_back('\r'); break;
                case 't': out->push_back('\t'); break;
                case 'u': {
                    if (e_ - p_ < 4) return false;
                    unsigned cp = 0;
                    for (int i = 0; i < 4; ++i) {
                        const int h = hexval(p_[i]);
                        if (h < 0) return false;
                        cp = cp * 16 + (unsigned)h;
                    }
                    p_ += 4;
                    if (cp >= 0xD800 && cp <= 0xDFFF) return false;  // no surrogate pairs here
                    if (cp < 0x80) {
                        out->push_back((char)cp);
                    } else if (cp < 0x800) {
                        out->push_back((char)(0xC0 | (cp >> 6)));
                        out->push_back((char)(0x80 | (cp & 0x3F)));
                    } else {
                        out->push_back((char)(0xE0 | (cp >> 12)));
                        out->push_back((char)(0x80 | ((cp >> 6) & 0x3F)));
                        out->push_back((char)(0x80 | (cp & 0x3F)));
                    }
                    break;
                }
                default: return false;
            }
        }
        if (p_ >= e_) return false;
        ++p_;  // closing quote
        return true;
    }
    bool value(JVal* v, int depth) {
        if (depth > kMaxDepth) return false;
        ws();
        if (p_ >= e_) return false;
        const char c = *p_;
        if (c == '{') {
            ++p_;
            v->kind = JVal::OBJ;
            ws();
            if (p_ < e_ && *p_ == '}') {
                ++p_;
                return true;
            }
            for (;;) {
                ws();
                std::pair<std::string, JVal> kv;
                if (!string(&kv.first)) return false;
                ws();
                if (p_ >= e_ || *p_ != ':') return false;
                ++p_;
                if (!value(&kv.second, depth + 1)) return false;
                v->obj.push_back(std::move(kv));
                ws();
                if (p_ < e_ && *p_ == ',') {
                    ++p_;
                    continue;
                }
                if (p_ < e_ && *p_ == '}') {
                    ++p_;
                    return true;
                }
                return false;
            }
        }
        if (c == '[') {
            ++p_;
            v->kind = JVal::ARR;
            ws();
            if (p_ < e_ && *p_ == ']') {
                ++p_;
                return true;
            }
            for (;;) {
                JVal item;
                if (!value(&item, depth + 1)) return false;
                v->arr.push_back(std::move(item));
                ws();
                if (p_ < e_ && *p_ == ',') {
                    ++p_;
                    continue;
                }
                if (p_ < e_ && *p_ == ']') {
                    ++p_;
                    return true;
                }
                return false;
            }
        }
        if (c == '"') {
            v->kind = JVal::STR;
            return string(&v->str);
        }
        if (lit("true")) {
            v->kind = JVal::BOOL;
            v->b = true;
            return true;
        }
        if (lit("false")) {
            v->kind = JVal::BOOL;
            return true;
        }
        if (lit("null")) {
            v->kind = JVal::NUL;
            return true;
        }
        v->kind = JVal::NUM;
        return number(&v->num);
    }
};

// ------------------------------------------------------------ the format

constexpr const char* kFormat = "meta-tuning";
constexpr int kVersion = 1;
constexpr long kMaxFile = 64l << 20;  // bytes

bool as_int(const JVal* v, int* out) {
    if (!v || v->kind != JVal::NUM || v->num != std::floor(v->num) || v->num < -2147483648.0 ||
        v->num > 2147483647.0)
        return false;
    *out = (int)v->num;
    return true;
}

// One entry: {"ndim", "dims", "batch", "sigma", "sigma_bits" (optional, the
// FP32 bit pattern, which wins over "sigma"), "zc_transport", "zc_advect", "ly",
// "lz", "txw", "split"}.  The problem shape is checked like any call's and the
// tile shapes like meta_tuning_set's.
bool entry_of(const JVal& e, TuneEntry* out) {
    if (e.kind != JVal::OBJ) return false;
    std::memset(out, 0, sizeof(*out));
    meta_problem& p = out->prob;
    const JVal* dims = e.get("dims");
    if (!as_int(e.get("ndim"), &p.ndim) || (p.ndim != 2 && p.ndim != 3)) return false;
    if (!dims || dims->kind != JVal::ARR || (int)dims->arr.size() != p.ndim) return false;
    for (int a = 0; a < p.ndim; ++a)
        if (!as_int(&dims->arr[a], &p.dims[a])) return false;
    if (!as_int(e.get("batch"), &p.batch)) return false;
    const JVal* sb = e.get("sigma_bits");
    if (sb) {
        if (sb->kind != JVal::NUM || sb->num < 0 || sb->num > 4294967295.0 ||
            sb->num != std::floor(sb->num))
            return false;
        const uint32_t bits = (uint32_t)sb->num;
        std::memcpy(&p.sigma, &bits, 4);
    } else {
        const JVal* sg = e.get("sigma");
        if (!sg || sg->kind != JVal::NUM) return false;
        p.sigma = (float)sg->num;
    }
    p.T = 1;
    meta_tuning& t = out->tun;
    if (!as_int(e.get("zc_transport"), &t.zc_transport) ||
        !as_int(e.get("zc_advect"), &t.zc_advect) || !as_int(e.get("ly"), &t.ly) ||
        !as_int(e.get("lz"), &t.lz) || !as_int(e.get("txw"), &t.txw) ||
        !as_int(e.get("split"), &t.split))
        return false;
    return tuning_check(&p, &t) == META_OK;
}

// The whole file, or META_ERR_IO / META_ERR_FORMAT; nothing is applied here.
meta_status read_entries(const char* path, std::vector<TuneEntry>* out) {
    out->clear();
    FILE* f = std::fopen(path, "rb");
    if (!f) return META_ERR_IO;
    std::string text;
    char buf[65536];
    size_t n;
    while ((n = std::fread(buf, 1, sizeof(buf), f)) > 0) {
        text.append(buf, n);
        if ((long)text.size() > kMaxFile) {
            std::fclose(f);
            return META_ERR_FORMAT;
        }
    }
    const bool err = std::ferror(f) != 0;
    std::fclose(f);
    if (err) return META_ERR_IO;
    JVal root;
    JReader rd(text.data(), text.data() + text.size());
    if (!rd.parse(&root) || root.kind != JVal::OBJ) return META_ERR_FORMAT;
    const JVal* fmt = root.get("format");
    int ver = 0;
    if (!fmt || fmt->kind != JVal::STR || fmt->str != kFormat) return META_ERR_FORMAT;
    if (!as_int(root.get("version"), &ver) || ver != kVersion) return META_ERR_FORMAT;
    const JVal* ents = root.get("entries");
    if (!ents || ents->kind != JVal::ARR) return META_ERR_FORMAT;
    for (const JVal& e : ents->arr) {
        TuneEntry te;
        if (!entry_of(e, &te)) return META_ERR_FORMAT;
        out->push_back(te);
    }
    return META_OK;
}

// Written to `path`.tmp.<pid> and renamed over `path`, so that a reader never
// sees half a file.
meta_status write_entries(const char* path, const std::vector<TuneEntry>& ents) {
    const std::string tmp = std::string(path) + ".tmp." + std::to_string((long)getpid());
    FILE* f = std::fopen(tmp.c_str(), "wb");
    if (!f) return META_ERR_IO;
    bool ok = std::fprintf(f, "{\"format\": \"%s\", \"version\": %d, \"arch\": \"sm_103a\",\n"
                              " \"entries\": [", kFormat, kVersion) > 0;
    for (size_t i = 0; i < ents.size() && ok; ++i) {
        const meta_problem& p = ents[i].prob;
        const meta_tuning& t = ents[i].tun;
        uint32_t bits;
        std::memcpy(&bits, &p.sigma, 4);
        char dims[64];
        if (p.ndim == 3)
            std::snprintf(dims, sizeof(dims), "[%d, %d, %d]", p.dims[0], p.dims[1], p.dims[2]);
        else
            std::snprintf(dims, sizeof(dims), "[%d, %d]", p.dims[0], p.dims[1]);
        ok = std::fprintf(f,
                          "%s\n  {\"ndim\": %d, \"dims\": %s, \"batch\": %d, \"sigma\": %.9g, "
                          "\"sigma_bits\": %u, \"zc_transport\": %d, \"zc_advect\": %d, "
                          "\"ly\": %d, \"lz\": %d, \"txw\": %d, \"split\": %d}",
                          i ? "," : "", p.ndim, dims, p.batch, (double)p.sigma, bits,
                          t.zc_transport, t.zc_advect, t.ly, t.lz, t.txw, t.split) > 0;
    }
    ok = ok && std::fprintf(f, "\n ]}\n") > 0;
    ok = (std::fclose(f) == 0) && ok;
    if (!ok || std::rename(tmp.c_str(), path) != 0) {
        std::remove(tmp.c_str());
        return META_ERR_IO;
    }
    return META_OK;
}

bool same_key(const meta_problem& a, const meta_problem& b) {
    if (a.ndim != b.ndim || a.batch != b.batch || std::memcmp(&a.sigma, &b.sigma, 4) != 0)
        return false;
    for (int k = 0; k < a.ndim; ++k)
        if (a.dims[k] != b.dims[k]) return false;
    return true;
}

// Later entries for the same shape replace earlier ones.
void merge(std::vector<TuneEntry>* into, const TuneEntry& e) {
    for (auto& x : *into)
        if (same_key(x.prob, e.prob)) {
            x.tun = e.tun;
            return;
        }
    into->push_back(e);
}

// The cache named by meta_tuning_cache and the entries read from it.
std::mutex g_cache_mu;
std::string g_cache_path;
std::vector<TuneEntry> g_cache;

}  // namespace

bool tuning_cache_lookup(const meta_problem* prob, meta_tuning* tun) {
    std::lock_guard<std::mutex> lk(g_cache_mu);
    if (g_cache_path.empty()) return false;
    for (const auto& e : g_cache)
        if (same_key(e.prob, *prob)) {
            *tun = e.tun;
            return true;
        }
    return false;
}

meta_status tuning_cache_note(const meta_problem* prob, const meta_tuning& tun) {
    std::lock_guard<std::mutex> lk(g_cache_mu);
    if (g_cache_path.empty()) return META_OK;
    TuneEntry e;
    std::memset(&e, 0, sizeof(e));
    e.prob.ndim = prob->ndim;
    for (int a = 0; a < prob->ndim; ++a) e.prob.dims[a] = prob->dims[a];
    e.prob.batch = prob->batch;
    e.prob.sigma = prob->sigma;
    e.prob.T = 1;
    e.tun = tun;
    // entries another process added since the file was read are kept
    std::vector<TuneEntry> disk;
    if (read_entries(g_cache_path.c_str(), &disk) != META_OK) disk.clear();
    for (const auto& x : g_cache) merge(&disk, x);
    merge(&disk, e);
    merge(&g_cache, e);
    return write_entries(g_cache_path.c_str(), disk);
}

}  // namespace meta

using namespace meta;

extern "C" {

meta_status meta_tuning_save(const char* path) {
    if (!path || !*path) return META_ERR_INVALID_ARG;
    std::vector<TuneEntry> ents;
    tuning_snapshot(&ents);
    return write_entries(path, ents);
}

meta_status meta_tuning_load(const char* path, int* entries) {
    if (!path || !*path) return META_ERR_INVALID_ARG;
    std::vector<TuneEntry> ents;
    const meta_status s = read_entries(path, &ents);
    if (s != META_OK) return s;
    for (const auto& e : ents) {
        const meta_status r = meta_tuning_set(&e.prob, &e.tun);  // checked when read
        if (r != META_OK) return r;
    }
    if (entries) *entries = (int)ents.size();
    return META_OK;
}

meta_status meta_tuning_cache(const char* path, int* entries) {
    std::vector<TuneEntry> ents;
    if (path && *path) {
        const meta_status s = read_entries(path, &ents);
        if (s == META_ERR_FORMAT) return s;
        if (s == META_ERR_IO) {  // no such file yet: an empty cache, if it can be made
            FILE* f = std::fopen(path, "rb");
            if (f) {
                std::fclose(f);
                return META_ERR_IO;  // it exists but could not be read
            }
            ents.clear();
        }
    }
    for (const auto& e : ents) {
        const meta_status r = meta_tuning_set(&e.prob, &e.tun);
        if (r != META_OK) return r;
    }
    std::lock_guard<std::mutex> lk(g_cache_mu);
    g_cache_path = path ? path : "";
    g_cache = ents;
    if (entries) *entries = (int)ents.size();
    return META_OK;
}

}  // extern "C"
