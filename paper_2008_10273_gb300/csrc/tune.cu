// Persistent table of the autotuner's choices (host code only).
//
// The library tunes schedule parameters that change speed but never a
// result: the red-black sweep kernel's region tiling (k_intra.cu) and the
// number of CTAs per SM of the persistent coefficient kernel (k_block.cu).
// A choice is keyed by the GPU's name and the shape it was made for (plane
// sizes, block counts), kept in memory for the process and in a small JSON
// file (one flat object of "key": integer) so that later processes on the
// same kind of GPU skip the timing runs.  The file is the path in the
// environment variable HIVC_TUNE_CACHE, else $XDG_CACHE_HOME/hivc/tune.json,
// else $HOME/.cache/hivc/tune.json; an unreadable or malformed file counts as
// empty, and a failed write only costs the next process its timing runs.
#include <cerrno>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>

#include <sys/stat.h>
#include <unistd.h>

#include "hivc_internal.cuh"

namespace hivc {
namespace {

std::mutex g_mu;
bool g_loaded = false;
std::map<std::string, int> g_table;

std::string cache_path()
{
    if (const char *p = std::getenv("HIVC_TUNE_CACHE")) return p;
    std::string base;
    if (const char *x = std::getenv("XDG_CACHE_HOME")) base = x;
    else if (const char *h = std::getenv("HOME")) base = std::string(h) + "/.cache";
    else return std::string();
    return base + "/hivc/tune.json";
}

// the flat JSON object {"key": int, ...}; returns false on a syntax error
bool parse(const std::string &t, std::map<std::string, int> &out)
{
    size_t i = 0;
    auto ws = [&]() {
        while (i < t.size() && (t[i] == ' ' || t[i] == '\n' || t[i] == '\r' || t[i] == '\t')) ++i;
    };
    ws();
    if (i >= t.size() || t[i] != '{') return false;
    ++i;
    ws();
    if (i < t.size() && t[i] == '}') return true;
    for (;;) {
        ws();
        if (i >= t.size() || t[i] != '"') return false;
        ++i;
        std::string key;
        while (i < t.size() && t[i] != '"') {
            if (t[i] == '\\' && i + 1 < t.size()) ++i;
            key += t[i++];
        }
        if (i >= t.size()) return false;
        ++i;
        ws();
        if (i >= t.size() || t[i] != ':') return false;
        ++i;
        ws();
        char *end = nullptr;
        const long v = std::strtol(t.c_str() + i, &end, 10);
        if (end == t.c_str() + i) return false;
        i = (size_t)(end - t.c_str());
        out[key] = (int)v;
        ws();
        if (i < t.size() && t[i] == ',') {
            ++i;
            continue;
        }
        return i < t.size() && t[i] == '}';
    }
}

void load_locked()
{
    if (g_loaded) return;
    g_loaded = true;
    const std::string path = cache_path();
    if (path.empty()) return;
    FILE *f = std::fopen(path.c_str(), "rb");
    if (!f) return;
    std::string text;
    char buf[4096];
    size_t n;
    while ((n = std::fread(buf, 1, sizeof buf, f)) > 0 && text.size() < (1u << 20)) text.append(buf, n);
    std::fclose(f);
    std::map<std::string, int> t;
    if (parse(text, t)) g_table.insert(t.begin(), t.end());
}

void mkdirs(const std::string &dir)
{
    for (size_t p = 1; p <= dir.size(); ++p)
        if (p == dir.size() || dir[p] == '/') mkdir(dir.substr(0, p).c_str(), 0755);
}

// rewrites the file with the table merged into what is there (another
// process may have added keys); written to a temporary file and renamed
void save_locked()
{
    const std::string path = cache_path();
    if (path.empty()) return;
    const size_t slash = path.rfind('/');
    if (slash != std::string::npos) mkdirs(path.substr(0, slash));
    std::map<std::string, int> merged;
    if (FILE *f = std::fopen(path.c_str(), "rb")) {
        std::string text;
        char buf[4096];
        size_t n;
        while ((n = std::fread(buf, 1, sizeof buf, f)) > 0 && text.size() < (1u << 20)) text.append(buf, n);
        std::fclose(f);
        parse(text, merged);
    }
    for (const auto &kv : g_table) merged[kv.first] = kv.second;
    const std::string tmp = path + "." + std::to_string((long)getpid()) + ".tmp";
    FILE *f = std::fopen(tmp.c_str(), "wb");
    if (!f) return;
    std::fputs("{\n", f);
    size_t k = 0;
    for (const auto &kv : merged) {
        std::string key;
        for (char c : kv.first) {
            if (c == '"' || c == '\\') key += '\\';
            key += c;
        }
        std::fprintf(f, "  \"%s\": %d%s\n", key.c_str(), kv.second, ++k < merged.size() ? "," : "");
    }
    std::fputs("}\n", f);
    const bool ok = std::fclose(f) == 0;
    if (ok) std::rename(tmp.c_str(), path.c_str());
    else std::remove(tmp.c_str());
}

}  // namespace

std::string gpu_name()
{
    static std::mutex mu;
    static std::string names[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return "unknown";
    std::lock_guard<std::mutex> lk(mu);
    if (names[dev].empty()) {
        cudaDeviceProp prop;
        names[dev] = cudaGetDeviceProperties(&prop, dev) == cudaSuccess ? std::string(prop.name) : "unknown";
    }
    return names[dev];
}

int tune_lookup(const std::string &key)
{
    std::lock_guard<std::mutex> lk(g_mu);
    load_locked();
    const auto it = g_table.find(key);
    return it == g_table.end() ? -1 : it->second;
}

void tune_store(const std::string &key, int value)
{
    std::lock_guard<std::mutex> lk(g_mu);
    load_locked();
    g_table[key] = value;
    save_locked();
}

}  // namespace hivc

extern "C" int32_t hivc_tune_lookup(const char *key)
{
    return key ? hivc::tune_lookup(key) : -1;
}

extern "C" hivc_status hivc_tune_record(const char *key, int32_t value)
{
    if (!key || !*key || value < 0) return HIVC_E_INVALID;
    hivc::tune_store(key, value);
    return HIVC_OK;
}
