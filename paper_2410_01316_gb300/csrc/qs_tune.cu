// Autotune cache: tuned launch choices keyed by the problem's shape class
// (d bucket, N_ft, P bucket, projection form, window width), written by the
// tuners (qs_plan_autotune, qs_plan_autotune_gemm) and read by plan creation,
// so later plans of the same class start with the tuned choices.  The cache
// is process-wide, guarded by a mutex, and can be saved to and loaded from a
// text file (one entry per line: dbits n_ft pbits proj W spread_variant
// gemm_pair, -1 where a choice was not tuned).
#include <stdio.h>

#include <mutex>
#include <vector>

#include "qs_internal.cuh"

namespace {

struct TuneEntry {
    int dbits, n_ft, pbits, proj, W;
    int spread_variant;  // -1: not tuned
    int gemm_pair;       // -1: not tuned
};

std::mutex g_tune_mutex;
std::vector<TuneEntry> g_tune;

int ceil_log2(int v)
{
    int b = 0;
    while ((1 << b) < v && b < 30) ++b;
    return b;
}

TuneEntry key_of(const qs_plan_s* p)
{
    TuneEntry k;
    k.dbits = ceil_log2(p->desc.d);
    k.n_ft = p->desc.n_ft;
    k.pbits = ceil_log2(p->desc.P);
    k.proj = (int)p->proj;
    k.W = p->W;
    k.spread_variant = -1;
    k.gemm_pair = -1;
    return k;
}

bool same_key(const TuneEntry& a, const TuneEntry& b)
{
    return a.dbits == b.dbits && a.n_ft == b.n_ft && a.pbits == b.pbits && a.proj == b.proj && a.W == b.W;
}

TuneEntry* find_locked(const TuneEntry& k)
{
    for (auto& e : g_tune)
        if (same_key(e, k)) return &e;
    return nullptr;
}

}  // namespace

bool qs_tune_lookup(const qs_plan_s* p, int* spread_variant, int* gemm_pair)
{
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    const TuneEntry* e = find_locked(key_of(p));
    if (!e) return false;
    *spread_variant = e->spread_variant;
    *gemm_pair = e->gemm_pair;
    return true;
}

void qs_tune_store(const qs_plan_s* p, int spread_variant, int gemm_pair)
{
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    const TuneEntry k = key_of(p);
    TuneEntry* e = find_locked(k);
    if (!e) {
        g_tune.push_back(k);
        e = &g_tune.back();
    }
    if (spread_variant >= 0) e->spread_variant = spread_variant;
    if (gemm_pair >= 0) e->gemm_pair = gemm_pair;
}

extern "C" qs_status qs_tune_cache_save(const char* path)
{
    if (!path) return QS_ERR_ARG;
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    FILE* f = fopen(path, "w");
    if (!f) {
        qs_set_error_message("qs_tune_cache_save: cannot open the file for writing");
        return QS_ERR_ARG;
    }
    fprintf(f, "# qmcslice autotune cache: dbits n_ft pbits proj W spread_variant gemm_pair\n");
    for (const auto& e : g_tune)
        fprintf(f, "%d %d %d %d %d %d %d\n", e.dbits, e.n_ft, e.pbits, e.proj, e.W, e.spread_variant, e.gemm_pair);
    const bool ok = fclose(f) == 0;
    if (!ok) qs_set_error_message("qs_tune_cache_save: write failed");
    return ok ? QS_OK : QS_ERR_ARG;
}

extern "C" qs_status qs_tune_cache_load(const char* path)
{
    if (!path) return QS_ERR_ARG;
    FILE* f = fopen(path, "r");
    if (!f) {
        qs_set_error_message("qs_tune_cache_load: cannot open the file");
        return QS_ERR_ARG;
    }
    std::vector<TuneEntry> got;
    char line[256];
    bool bad = false;
    while (fgets(line, sizeof(line), f)) {
        if (line[0] == '#' || line[0] == '\n') continue;
        TuneEntry e;
        if (sscanf(line, "%d %d %d %d %d %d %d", &e.dbits, &e.n_ft, &e.pbits, &e.proj, &e.W, &e.spread_variant,
                   &e.gemm_pair) != 7 ||
            e.spread_variant < -1 || e.spread_variant >= QS_SPREAD_NVARIANTS || e.gemm_pair < -1 || e.gemm_pair > 1) {
            bad = true;
            break;
        }
        got.push_back(e);
    }
    fclose(f);
    if (bad) {
        qs_set_error_message("qs_tune_cache_load: malformed line");
        return QS_ERR_ARG;
    }
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    for (const auto& e : got) {
        TuneEntry* have = find_locked(e);
        if (have) *have = e;
        else g_tune.push_back(e);
    }
    return QS_OK;
}

extern "C" qs_status qs_tune_cache_clear(void)
{
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    g_tune.clear();
    return QS_OK;
}

extern "C" int qs_tune_cache_size(void)
{
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    return (int)g_tune.size();
}
