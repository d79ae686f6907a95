// Autotuner of the per-plan launch configuration: the spreading / force-interpolation tile edge (8^3 or 16^3
// mesh points) and CTA size (128 or 256 threads). Both leave every result bit-identical (the charge mesh is
// an exact integer sum and each atom's force sums its support in a fixed order whatever tile holds it), so
// the choice is a pure speed decision, which the tuner makes by timing the candidates on the caller's own
// atoms; it also checks the bit-identity and rejects any candidate that differs. Choices are kept per plan
// and, when a cache file is set, persisted as JSON keyed by (device, mesh, order, atoms-per-tile class).
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <mutex>
#include <string>
#include <vector>

#include "../../include/pme.h"
#include "host_tables.h"
#include "kernels.h"
#include "plan_internal.h"

namespace pme {

struct TuneEntry {
    std::string device;
    int K[3] = {0, 0, 0};
    int p = 0, apt = 0, tile_edge = 0, tile_threads = 0;
    double us = 0.0;
};

static std::mutex g_tune_mu;
static std::string g_cache_path;         // "" = no file
static bool g_cache_loaded = false;
static std::vector<TuneEntry> g_entries;

// ---- minimal JSON reading and writing for the cache's own format -------------------------------------

static const char *skip_ws(const char *s) {
    while (*s == ' ' || *s == '\n' || *s == '\r' || *s == '\t') ++s;
    return s;
}
// position just after "key": inside [b, e), or nullptr
static const char *find_key(const char *b, const char *e, const char *key) {
    const std::string pat = std::string("\"") + key + "\"";
    for (const char *s = b; s + pat.size() <= e; ++s) {
        if (strncmp(s, pat.c_str(), pat.size()) == 0) {
            const char *t = skip_ws(s + pat.size());
            if (*t == ':') return skip_ws(t + 1);
        }
    }
    return nullptr;
}
static bool get_num(const char *b, const char *e, const char *key, double *v) {
    const char *s = find_key(b, e, key);
    if (!s) return false;
    char *end = nullptr;
    *v = strtod(s, &end);
    return end != s;
}
static bool get_str(const char *b, const char *e, const char *key, std::string *v) {
    const char *s = find_key(b, e, key);
    if (!s || *s != '"') return false;
    const char *t = strchr(s + 1, '"');
    if (!t || t > e) return false;
    v->assign(s + 1, t);
    return true;
}
static bool get_int3(const char *b, const char *e, const char *key, int out[3]) {
    const char *s = find_key(b, e, key);
    if (!s || *s != '[') return false;
    ++s;
    for (int i = 0; i < 3; ++i) {
        char *end = nullptr;
        out[i] = (int)strtol(skip_ws(s), &end, 10);
        if (end == s) return false;
        s = skip_ws(end);
        if (i < 2) {
            if (*s != ',') return false;
            ++s;
        }
    }
    return true;
}

static void load_cache_locked() {
    if (g_cache_loaded) return;
    g_cache_loaded = true;
    g_entries.clear();
    if (g_cache_path.empty()) return;
    FILE *f = fopen(g_cache_path.c_str(), "rb");
    if (!f) return;
    std::string text;
    char buf[4096];
    size_t got;
    while ((got = fread(buf, 1, sizeof(buf), f)) > 0) text.append(buf, got);
    fclose(f);
    const char *s = strstr(text.c_str(), "\"entries\"");
    if (!s) return;
    s = strchr(s, '[');
    while (s && (s = strchr(s, '{')) != nullptr) {
        const char *e = strchr(s, '}');
        if (!e) break;
        TuneEntry t;
        double p, apt, te, tt, us;
        if (get_str(s, e, "device", &t.device) && get_int3(s, e, "K", t.K) && get_num(s, e, "p", &p) &&
            get_num(s, e, "apt", &apt) && get_num(s, e, "tile_edge", &te) && get_num(s, e, "tile_threads", &tt) &&
            get_num(s, e, "us", &us)) {
            t.p = (int)p;
            t.apt = (int)apt;
            t.tile_edge = (int)te;
            t.tile_threads = (int)tt;
            t.us = us;
            if ((t.tile_edge == 8 || t.tile_edge == 16) &&
                (t.tile_threads == 0 || t.tile_threads == 128 || t.tile_threads == 256 ||
                 (t.tile_threads == 512 && t.tile_edge == 16)))
                g_entries.push_back(t);
        }
        s = e + 1;
    }
}

static bool save_cache_locked() {
    if (g_cache_path.empty()) return true;
    const std::string tmp = g_cache_path + ".tmp";
    FILE *f = fopen(tmp.c_str(), "wb");
    if (!f) return false;
    fprintf(f, "{\"pme_tune_cache\": 1, \"entries\": [\n");
    for (size_t i = 0; i < g_entries.size(); ++i) {
        const TuneEntry &t = g_entries[i];
        fprintf(f,
                "  {\"device\": \"%s\", \"K\": [%d, %d, %d], \"p\": %d, \"apt\": %d, \"tile_edge\": %d, "
                "\"tile_threads\": %d, \"us\": %.3f}%s\n",
                t.device.c_str(), t.K[0], t.K[1], t.K[2], t.p, t.apt, t.tile_edge, t.tile_threads, t.us,
                i + 1 < g_entries.size() ? "," : "");
    }
    fprintf(f, "]}\n");
    const bool ok = fclose(f) == 0;
    return ok && rename(tmp.c_str(), g_cache_path.c_str()) == 0;
}

// Atoms-per-tile class: round(2 log2(n / number of 8^3 tiles)), half-octave steps.
static int apt_class(const int K[3], int64_t n) {
    const double tiles = (double)((K[0] + 7) / 8) * ((K[1] + 7) / 8) * ((K[2] + 7) / 8);
    const double a = (double)(n > 0 ? n : 1) / tiles;
    return (int)lround(2.0 * log2(a));
}

static std::string device_name(int dev) {
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return "unknown";
    std::string s(prop.name);
    for (char &c : s)
        if (c == '"' || c == '\\') c = '_';
    return s;
}

// Switch a plan to tile edge 2^tlog and CTA size nt (0: density rule), reallocating the per-atom buckets
// for n atoms when the tiling changes.
pme_status plan_retile(pme_plan *pl, int tlog, int nt, int64_t n) {
    const bool changed = pl->d.tlog != tlog || pl->tile_log_set != tlog;
    pl->tile_log_set = tlog;
    pl->d.nt_tile = nt;
    ++pl->gen;  // recorded graphs of synchronous calls hold the old launch configuration
    if (!changed && pl->atom_mem) return plan_reserve(pl, n);
    cudaError_t e = cudaStreamSynchronize(pl->stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    const int64_t keep = pl->n_cap > n ? pl->n_cap : n;
    if (pl->atom_mem) cudaFree(pl->atom_mem);
    pl->atom_mem = nullptr;
    pl->atom_bytes = 0;
    pl->n_cap = 0;
    return plan_reserve(pl, keep);
}

// One evaluation's outputs on the host, for the bit-identity check.
static pme_status eval_bits(pme_plan *pl, const float *pos, const float *q, int64_t n, float *forces,
                            std::vector<float> &F, double ev[7]) {
    const SysDev d = plan_descriptor(pl, pos, q, n, forces, nullptr);
    cudaError_t e = launch_pipeline(d, pl->stream);
    if (e == cudaSuccess && n > 0)
        e = cudaMemcpyAsync(F.data(), forces, (size_t)n * 12, cudaMemcpyDeviceToHost, pl->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(ev, pl->d.ctl->ev, 7 * sizeof(double), cudaMemcpyDeviceToHost, pl->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(pl->stream);
    if (e != cudaSuccess) return cuda_fail(e, "tuning evaluation");
    return PME_OK;
}

static pme_status time_evals(pme_plan *pl, const float *pos, const float *q, int64_t n, float *forces, int reps,
                             double *us) {
    const SysDev d = plan_descriptor(pl, pos, q, n, forces, nullptr);
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < 2 && e == cudaSuccess; ++i) e = launch_pipeline(d, pl->stream);
    if (e == cudaSuccess) e = cudaEventRecord(a, pl->stream);
    for (int i = 0; i < reps && e == cudaSuccess; ++i) e = launch_pipeline(d, pl->stream);
    if (e == cudaSuccess) e = cudaEventRecord(b, pl->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(b);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (e != cudaSuccess) return cuda_fail(e, "tuning timing");
    *us = 1000.0 * ms / reps;
    return PME_OK;
}

// Apply a cached choice for this plan and n if there is one; true when applied.
bool tune_apply_cached(pme_plan *pl, int64_t n, pme_status *st) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    load_cache_locked();
    const std::string dev = device_name(pl->dev);
    const int apt = apt_class(pl->K, n);
    for (const TuneEntry &t : g_entries)
        if (t.device == dev && t.K[0] == pl->K[0] && t.K[1] == pl->K[1] && t.K[2] == pl->K[2] && t.p == pl->p &&
            t.apt == apt) {
            *st = plan_retile(pl, t.tile_edge == 16 ? 4 : 3, t.tile_threads, n);
            pl->tuned_apt = apt;
            return true;
        }
    return false;
}

void tune_record(const pme_plan *pl, int64_t n, int tlog, int nt, double us) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    load_cache_locked();
    TuneEntry t;
    t.device = device_name(pl->dev);
    memcpy(t.K, pl->K, sizeof(t.K));
    t.p = pl->p;
    t.apt = apt_class(pl->K, n);
    t.tile_edge = 1 << tlog;
    t.tile_threads = nt;
    t.us = us;
    bool replaced = false;
    for (TuneEntry &o : g_entries)
        if (o.device == t.device && o.K[0] == t.K[0] && o.K[1] == t.K[1] && o.K[2] == t.K[2] && o.p == t.p &&
            o.apt == t.apt) {
            o = t;
            replaced = true;
        }
    if (!replaced) g_entries.push_back(t);
    save_cache_locked();
}

}  // namespace pme

using namespace pme;

extern "C" {

pme_status pme_tune_cache(const char *path) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_cache_path = path ? path : "";
    g_cache_loaded = false;
    return PME_OK;
}

pme_status pme_plan_set_tiling(pme_plan *pl, int tile_edge, int tile_threads) {
    if (!pl) return fail(PME_EINVAL, "plan is NULL");
    if (tile_edge != 0 && tile_edge != 8 && tile_edge != 16) return fail(PME_EINVAL, "tile_edge must be 0, 8 or 16");
    if (tile_threads != 0 && tile_threads != 128 && tile_threads != 256 && !(tile_threads == 512 && tile_edge == 16))
        return fail(PME_EINVAL, "tile_threads must be 0, 128 or 256 (or 512 with tile_edge 16)");
    DeviceGuard g(pl->dev);
    const int tlog = tile_edge == 16 ? 4 : (tile_edge == 8 ? 3 : 0);
    return plan_retile(pl, tlog, tile_threads, pl->n_cap);
}

pme_status pme_plan_get_tiling(const pme_plan *pl, int *tile_edge, int *tile_threads) {
    if (!pl) return fail(PME_EINVAL, "plan is NULL");
    if (tile_edge) *tile_edge = 1 << pl->d.tlog;
    if (tile_threads) *tile_threads = pl->d.nt_tile;  // 0: the per-stage default sizes
    return PME_OK;
}

pme_status pme_autotune(pme_plan *pl, const float *pos, const float *q, int64_t n, float *forces, int reps, int flags,
                        pme_tune_result *out) {
    pme_status st = check_atoms(pl, pos, q, n, forces);
    if (st) return st;
    if (reps < 1 || reps > 100000) return fail(PME_EINVAL, "reps must be in [1, 100000]");
    DeviceGuard g(pl->dev);
    pme_tune_result res;
    memset(&res, 0, sizeof(res));
    if (!(flags & PME_TUNE_FORCE) && tune_apply_cached(pl, n, &st)) {
        if (st != PME_OK) return st;
        res.tile_edge = 1 << pl->d.tlog;
        res.tile_threads = pl->d.nt_tile;
        res.from_cache = 1;
        if (out) *out = res;
        return PME_OK;
    }
    // candidates: the default first (its results are the reference bits), then every other combination
    const int tdef = pl->tile_log_set ? pl->tile_log_set : choose_tile_log(n > 0 ? n : 1, pl->K, pl->sms);
    if ((st = plan_retile(pl, tdef, 0, n)) != PME_OK) return st;
    // the default sizes (nt = 0): spreading and force interpolation take different CTA sizes
    const int ntdef = 0;
    struct Cand { int tlog, nt; double us; bool same; };
    std::vector<Cand> cands = {{tdef, ntdef, 0.0, true}};
    for (int tlog : {3, 4})
        for (int nt : {tlog == 3 ? 128 : NT_TILE, tlog == 3 ? NT_TILE : NT_TILE16})
            if (!(tlog == tdef && nt == ntdef)) cands.push_back({tlog, nt, 0.0, false});
    std::vector<float> F0((size_t)(n > 0 ? n : 1) * 3), F1(F0.size());
    double ev0[7], ev1[7];
    for (size_t c = 0; c < cands.size(); ++c) {
        if ((st = plan_retile(pl, cands[c].tlog, cands[c].nt, n)) != PME_OK) return st;
        if ((st = eval_bits(pl, pos, q, n, forces, c == 0 ? F0 : F1, c == 0 ? ev0 : ev1)) != PME_OK) return st;
        if (c > 0)
            cands[c].same = memcmp(F0.data(), F1.data(), (size_t)n * 12) == 0 && memcmp(ev0, ev1, sizeof(ev0)) == 0;
        if (cands[c].same && (st = time_evals(pl, pos, q, n, forces, reps, &cands[c].us)) != PME_OK) return st;
        ++res.candidates;
        if (!cands[c].same) ++res.rejected;
    }
    size_t best = 0;
    for (size_t c = 1; c < cands.size(); ++c)
        if (cands[c].same && cands[c].us < cands[best].us) best = c;
    if ((st = plan_retile(pl, cands[best].tlog, cands[best].nt, n)) != PME_OK) return st;
    pl->tuned_apt = apt_class(pl->K, n);
    tune_record(pl, n, cands[best].tlog, cands[best].nt, cands[best].us);
    res.tile_edge = 1 << cands[best].tlog;
    res.tile_threads = cands[best].nt;
    res.us_per_eval = cands[best].us;
    res.default_us = cands[0].us;
    if (out) *out = res;
    return collect_status(pl, false);
}

}  // extern "C"
