// tune.cu -- the autotuner's cache: choices keyed by a text signature
// (architecture + shapes), kept in memory and, when the environment variable
// GF2_TUNE_CACHE names a file, loaded from and saved to it as a flat JSON
// object {"signature": "choice", ...}.
#include "common.cuh"

#include <cstdio>
#include <cstdlib>
#include <map>
#include <mutex>
#include <string>

namespace gf2 {
namespace {

std::mutex g_mu;
std::map<std::string, std::string> g_cache;
bool g_loaded = false;

void load_locked()
{
    if (g_loaded) return;
    g_loaded = true;
    const char *path = getenv("GF2_TUNE_CACHE");
    if (!path || !*path) return;
    FILE *f = fopen(path, "r");
    if (!f) return;
    char line[512];
    while (fgets(line, sizeof line, f)) {
        char k[256], v[128];
        if (sscanf(line, " \"%255[^\"]\" : \"%127[^\"]\"", k, v) == 2) g_cache[k] = v;
    }
    fclose(f);
}

void save_locked()
{
    const char *path = getenv("GF2_TUNE_CACHE");
    if (!path || !*path) return;
    const std::string tmp = std::string(path) + ".tmp";
    FILE *f = fopen(tmp.c_str(), "w");
    if (!f) return;
    fprintf(f, "{\n");
    size_t i = 0;
    for (const auto &kv : g_cache)
        fprintf(f, "  \"%s\": \"%s\"%s\n", kv.first.c_str(), kv.second.c_str(), ++i < g_cache.size() ? "," : "");
    fprintf(f, "}\n");
    fclose(f);
    rename(tmp.c_str(), path);
}

}  // namespace

bool tune_get(const std::string &key, std::string *value)
{
    std::lock_guard<std::mutex> lk(g_mu);
    load_locked();
    auto it = g_cache.find(key);
    if (it == g_cache.end()) return false;
    *value = it->second;
    return true;
}

void tune_put(const std::string &key, const std::string &value)
{
    std::lock_guard<std::mutex> lk(g_mu);
    load_locked();
    g_cache[key] = value;
    save_locked();
}

std::string arch_tag()
{
    int dev = 0, major = 0, minor = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess) {
        cudaGetLastError();
        return "sm?";
    }
    char b[32];
    snprintf(b, sizeof b, "sm%d%d", major, minor);
    return b;
}

}  // namespace gf2
