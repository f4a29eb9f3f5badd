// Tuned launch parameters of the filtration, per workload bucket.
//
// Two parameters change the speed of a filtration but not its results (every
// value and source is bitwise the same for any choice, since each pair
// distance depends only on the sample, the point and the sample's coarse
// cube): the edge of the grid cells, as a multiple of the FPS covering radius
// (the search radius of a sample scales with the size of its simplex, which
// FPS spacing sets), and the shell count from which a sample group is run by
// a whole CTA instead of a warp. The best values depend on the cloud's shape
// and size and on the GPU, so they are measured (paper_2509_22432_b300.tune
// sweeps them) and kept in a table keyed by (SM count, log2 points, log2
// landmarks, m). A lookup takes the entry of the nearest bucket on a GPU with
// the same SM count, else the defaults. The table lives in the process and
// can be loaded from and written to a text file; FLOOD_TUNE_CACHE names a
// file loaded at the first lookup.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include <mutex>
#include <vector>

#include "common.cuh"

namespace flood {
namespace {

constexpr float kDefaultCellFactor = 0.5f;
constexpr int kDefaultHeavyShells = 9;

std::mutex g_mu;
std::vector<flood_tuning_entry> g_table;
bool g_env_loaded = false;

int log2_bucket(int64_t v) { return v <= 1 ? 0 : static_cast<int>(lround(log2(static_cast<double>(v)))); }

bool entry_ok(const flood_tuning_entry& e) {
    return e.sm_count >= 1 && e.log2_points >= 0 && e.log2_points <= 40 && e.log2_landmarks >= 0 &&
           e.log2_landmarks <= 40 && e.m >= 1 && e.m <= FLOOD_MAX_M && e.cell_factor > 0.0f &&
           e.cell_factor <= 64.0f && e.heavy_shells >= 1 && e.heavy_shells <= 63;
}

void put_locked(const flood_tuning_entry& e) {
    for (flood_tuning_entry& x : g_table)
        if (x.sm_count == e.sm_count && x.log2_points == e.log2_points && x.log2_landmarks == e.log2_landmarks &&
            x.m == e.m) {
            x = e;
            return;
        }
    g_table.push_back(e);
}

// Lines "sm_count log2_points log2_landmarks m cell_factor heavy_shells";
// blank lines and lines starting with '#' are skipped.
int load_locked(const char* path, int32_t* n_loaded) {
    FILE* f = fopen(path, "r");
    if (!f) {
        set_error("flood_tuning_load: cannot open %s", path);
        return FLOOD_EINVAL;
    }
    char line[256];
    int n = 0, lineno = 0, rc = FLOOD_OK;
    while (fgets(line, sizeof(line), f)) {
        ++lineno;
        const char* p = line;
        while (*p == ' ' || *p == '\t') ++p;
        if (*p == '#' || *p == '\n' || *p == '\r' || *p == '\0') continue;
        flood_tuning_entry e{};
        if (sscanf(p, "%d %d %d %d %f %d", &e.sm_count, &e.log2_points, &e.log2_landmarks, &e.m, &e.cell_factor,
                   &e.heavy_shells) != 6 ||
            !entry_ok(e)) {
            set_error("flood_tuning_load: %s line %d is not a valid entry", path, lineno);
            rc = FLOOD_EINVAL;
            break;
        }
        put_locked(e);
        ++n;
    }
    fclose(f);
    if (n_loaded) *n_loaded = n;
    return rc;
}

void env_load_locked() {
    if (g_env_loaded) return;
    g_env_loaded = true;
    const char* p = getenv("FLOOD_TUNE_CACHE");
    if (p && *p) {
        FILE* f = fopen(p, "r");
        if (f) {
            fclose(f);
            load_locked(p, nullptr);  // a bad file leaves the entries before the bad line
        }
    }
}

}  // namespace

flood_tuning tuning_for(int64_t n_points, int32_t n_landmarks, int32_t m) {
    flood_tuning out{kDefaultCellFactor, kDefaultHeavyShells, 0};
    const int sms = device_sm_count();
    const int ln = log2_bucket(n_points), ll = log2_bucket(n_landmarks);
    std::lock_guard<std::mutex> lock(g_mu);
    env_load_locked();
    double best = 1e30;
    for (const flood_tuning_entry& e : g_table) {
        if (e.sm_count != sms) continue;
        const double d = abs(e.log2_points - ln) + abs(e.log2_landmarks - ll) + 0.25 * abs(e.m - m);
        if (d < best) {
            best = d;
            out.cell_factor = e.cell_factor;
            out.heavy_shells = e.heavy_shells;
            out.tuned = 1;
        }
    }
    return out;
}

}  // namespace flood

using namespace flood;

extern "C" int flood_tuning_lookup(int64_t n_points, int32_t n_landmarks, int32_t m, flood_tuning* out) {
    if (!out || n_points < 1 || n_landmarks < 1 || m < 1) {
        set_error("flood_tuning_lookup: need out != NULL, n_points >= 1, n_landmarks >= 1, m >= 1");
        return FLOOD_EINVAL;
    }
    *out = tuning_for(n_points, n_landmarks, m);
    return FLOOD_OK;
}

extern "C" int flood_tuning_set(const flood_tuning_entry* e) {
    if (!e || !entry_ok(*e)) {
        set_error("flood_tuning_set: entry out of range (sm_count >= 1, 0 < cell_factor <= 64, "
                  "1 <= heavy_shells <= 63, 1 <= m <= %d)", FLOOD_MAX_M);
        return FLOOD_EINVAL;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    env_load_locked();
    put_locked(*e);
    return FLOOD_OK;
}

extern "C" int flood_tuning_load(const char* path, int32_t* n_loaded) {
    if (!path) {
        set_error("flood_tuning_load: path is NULL");
        return FLOOD_EINVAL;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    env_load_locked();
    return load_locked(path, n_loaded);
}

extern "C" int flood_tuning_entries(flood_tuning_entry* out, int32_t capacity, int32_t* n_entries) {
    if (!n_entries || capacity < 0 || (capacity > 0 && !out)) {
        set_error("flood_tuning_entries: need n_entries != NULL and out for capacity > 0");
        return FLOOD_EINVAL;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    env_load_locked();
    *n_entries = static_cast<int32_t>(g_table.size());
    for (int32_t i = 0; i < capacity && i < static_cast<int32_t>(g_table.size()); ++i) out[i] = g_table[i];
    return FLOOD_OK;
}

extern "C" int flood_tuning_clear(void) {
    std::lock_guard<std::mutex> lock(g_mu);
    g_env_loaded = true;  // an explicit clear also drops the FLOOD_TUNE_CACHE file
    g_table.clear();
    return FLOOD_OK;
}
