// Optional persistent autotuning decisions.  With CTM_AUTOTUNE_CACHE=<file> in the
// environment, the contraction and QR autotuners first look their shape up in that
// file (read once per process) and append every new decision to it, one line
// "<tag> <key ints> : <value ints>".  A later process -- a profiler run, a
// production job -- then runs the same plans without timing them again.
#include <cstdio>
#include <cstdlib>
#include <map>
#include <mutex>
#include <sstream>
#include <string>
#include <vector>

#include "ctm_internal.h"

namespace {
std::mutex g_mu;
bool g_loaded = false;
std::map<std::string, std::vector<int>> g_entries;

std::string key_of(const char *tag, const int *key, int nkey)
{
    std::ostringstream os;
    os << tag;
    for (int i = 0; i < nkey; ++i) os << ' ' << key[i];
    return os.str();
}

void load_locked()
{
    if (g_loaded) return;
    g_loaded = true;
    const char *path = std::getenv("CTM_AUTOTUNE_CACHE");
    if (!path || !*path) return;
    FILE *f = std::fopen(path, "r");
    if (!f) return;
    char line[512];
    while (std::fgets(line, sizeof(line), f)) {
        std::string s(line);
        const size_t colon = s.find(':');
        if (colon == std::string::npos) continue;
        std::string k = s.substr(0, colon);
        while (!k.empty() && k.back() == ' ') k.pop_back();
        std::istringstream vs(s.substr(colon + 1));
        std::vector<int> v;
        int x;
        while (vs >> x) v.push_back(x);
        if (!k.empty() && !v.empty()) g_entries[k] = v;
    }
    std::fclose(f);
}
}  // namespace

bool tune_cache_lookup(const char *tag, const int *key, int nkey, int *val, int nval)
{
    std::lock_guard<std::mutex> lk(g_mu);
    load_locked();
    auto it = g_entries.find(key_of(tag, key, nkey));
    if (it == g_entries.end() || (int)it->second.size() != nval) return false;
    for (int i = 0; i < nval; ++i) val[i] = it->second[i];
    return true;
}

void tune_cache_store(const char *tag, const int *key, int nkey, const int *val, int nval)
{
    std::lock_guard<std::mutex> lk(g_mu);
    load_locked();
    const std::string k = key_of(tag, key, nkey);
    g_entries[k] = std::vector<int>(val, val + nval);
    const char *path = std::getenv("CTM_AUTOTUNE_CACHE");
    if (!path || !*path) return;
    FILE *f = std::fopen(path, "a");
    if (!f) return;
    std::fprintf(f, "%s :", k.c_str());
    for (int i = 0; i < nval; ++i) std::fprintf(f, " %d", val[i]);
    std::fprintf(f, "\n");
    std::fclose(f);
}
