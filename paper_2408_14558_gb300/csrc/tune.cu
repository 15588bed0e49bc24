// Autotuner: times candidate configurations on the caller's own inputs and
// keeps the fastest, cached in a small JSON file keyed by the device name and
// a signature of the workload (log2 buckets of its sizes).
//   batched path: task size (columns per queue task) and CTA shape (warps)
//   plain path:   light-bin threshold (largest per-column bound handled by the
//                 warp hash bins) and heavy base-slab rows
// The cache file is a flat JSON object of objects with numeric fields; the
// tuner reads it, adds its entry and rewrites it.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "spg_internal.cuh"

namespace spg {
const char *last_error_str();
void clear_error();
}  // namespace spg

using namespace spg;

namespace {

using Entry = std::map<std::string, double>;
using Cache = std::map<std::string, Entry>;

// Parser for the flat format this file writes: {"key": {"name": number, ...}, ...}
bool read_cache(const char *path, Cache &out) {
    FILE *f = fopen(path, "rb");
    if (!f) return false;
    std::string s;
    char buf[4096];
    size_t r;
    while ((r = fread(buf, 1, sizeof buf, f)) > 0) s.append(buf, r);
    fclose(f);
    size_t i = 0;
    auto skip = [&]() {
        while (i < s.size() && (s[i] == ' ' || s[i] == '\n' || s[i] == '\r' || s[i] == '\t' || s[i] == ',')) i++;
    };
    auto str = [&](std::string &o) {
        skip();
        if (i >= s.size() || s[i] != '"') return false;
        size_t j = s.find('"', i + 1);
        if (j == std::string::npos) return false;
        o = s.substr(i + 1, j - i - 1);
        i = j + 1;
        return true;
    };
    auto expect = [&](char c) {
        skip();
        if (i < s.size() && s[i] == c) {
            i++;
            return true;
        }
        return false;
    };
    if (!expect('{')) return false;
    while (true) {
        skip();
        if (i < s.size() && s[i] == '}') break;
        std::string key;
        if (!str(key) || !expect(':') || !expect('{')) return false;
        Entry e;
        while (true) {
            skip();
            if (i < s.size() && s[i] == '}') {
                i++;
                break;
            }
            std::string name;
            if (!str(name) || !expect(':')) return false;
            skip();
            char *end = nullptr;
            double v = strtod(s.c_str() + i, &end);
            if (end == s.c_str() + i) return false;
            i = end - s.c_str();
            e[name] = v;
        }
        out[key] = e;
    }
    return true;
}

bool write_cache(const char *path, const Cache &c) {
    std::string tmp = std::string(path) + ".tmp";
    FILE *f = fopen(tmp.c_str(), "wb");
    if (!f) return false;
    fprintf(f, "{\n");
    size_t k = 0;
    for (auto &kv : c) {
        fprintf(f, "  \"%s\": {", kv.first.c_str());
        size_t m = 0;
        for (auto &nv : kv.second) fprintf(f, "%s\"%s\": %.6g", m++ ? ", " : "", nv.first.c_str(), nv.second);
        fprintf(f, "}%s\n", ++k < c.size() ? "," : "");
    }
    fprintf(f, "}\n");
    bool ok = fclose(f) == 0;
    return ok && rename(tmp.c_str(), path) == 0;
}

std::string device_name() {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceProp p;
    if (cudaGetDeviceProperties(&p, dev) != cudaSuccess) return "gpu";
    std::string n = p.name;
    for (char &ch : n)
        if (ch == '"' || ch == ' ') ch = '_';
    return n;
}

int lg(double x) { return x < 1 ? 0 : (int)std::floor(std::log2(x)); }

}  // namespace

extern "C" spg_status spgemm_batch_autotune(int32_t count, const spg_csc *A, const spg_csc *B, int32_t sample,
                                            const char *cache_path, spg_batch_options *best, double *best_ms) {
    clear_error();
    if (count < 1 || !A || !B || !best) {
        set_error("bad autotune arguments");
        return SPG_INVALID_ARGUMENT;
    }
    spgemm_batch_default_options(best);
    double cols = 0, nnzb = 0;
    for (int i = 0; i < count; i++) {
        cols += (double)B[i].ncols;
        nnzb += (double)B[i].nnz;
    }
    char sig[256];
    snprintf(sig, sizeof sig, "%s|batch|c%d|n%d|d%d|%s", device_name().c_str(), lg(count), lg(cols / count),
             lg(cols > 0 ? nnzb / cols : 0), A[0].val_type == SPG_VAL_F64 ? "f64" : "int");
    Cache cache;
    if (cache_path && read_cache(cache_path, cache)) {
        auto it = cache.find(sig);
        if (it != cache.end() && it->second.count("task_cols") && it->second.count("warps_per_cta")) {
            best->task_cols = (int32_t)it->second["task_cols"];
            best->warps_per_cta = (int32_t)it->second["warps_per_cta"];
            if (best_ms) *best_ms = it->second.count("ms") ? it->second["ms"] : -1;
            return SPG_OK;
        }
    }
    const int ns = sample > 0 && sample < count ? sample : count;
    const int task_opts[] = {16, 64, 256};
    const int warp_opts[] = {4, 8};
    double bms = 1e300;
    cudaStream_t st;
    spg_status s = cuda_check(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking), "stream");
    if (s) return s;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    for (int tc : task_opts) {
        for (int w : warp_opts) {
            spg_batch_options o;
            spgemm_batch_default_options(&o);
            o.task_cols = tc;
            o.warps_per_cta = w;
            spg_batch *b = nullptr;
            s = spgemm_batch_create(ns, A, B, &o, &b);
            if (s == SPG_UNSUPPORTED) continue;
            if (s) break;
            float total = 0;
            for (int r = 0; r < 4 && !s; r++) {
                cudaEventRecord(e0, st);
                s = spgemm_batch_execute(b, st);
                cudaEventRecord(e1, st);
                if (!s) s = spgemm_batch_status(b, st);
                float ms = 0;
                cudaEventElapsedTime(&ms, e0, e1);
                if (r > 0) total += ms;  // the first run warms up
            }
            spgemm_batch_destroy(b);
            if (s) break;
            const double ms = total / 3.0;
            if (ms < bms) {
                bms = ms;
                best->task_cols = tc;
                best->warps_per_cta = w;
            }
        }
        if (s) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(st);
    if (s) return s;
    if (best_ms) *best_ms = bms;
    if (cache_path) {
        cache[sig] = {{"task_cols", (double)best->task_cols}, {"warps_per_cta", (double)best->warps_per_cta},
                      {"ms", bms}, {"sample", (double)ns}};
        if (!write_cache(cache_path, cache)) {
            set_error("cannot write tuning cache %s", cache_path);
            return SPG_INVALID_ARGUMENT;
        }
    }
    return SPG_OK;
}

extern "C" spg_status spgemm_autotune(const spg_csc *A, const spg_csc *B, const spg_options *base,
                                      const char *cache_path, spg_options *best, double *best_ms) {
    clear_error();
    if (!A || !B || !base || !best) {
        set_error("bad autotune arguments");
        return SPG_INVALID_ARGUMENT;
    }
    *best = *base;
    char sig[256];
    snprintf(sig, sizeof sig, "%s|plain|m%d|k%d|n%d|b%d|P%d|%s", device_name().c_str(), lg((double)A->nrows),
             lg((double)A->ncols), lg((double)B->ncols), lg((double)B->nnz), lg((double)base->P),
             A->val_type == SPG_VAL_F64 ? "f64" : "int");
    Cache cache;
    if (cache_path && read_cache(cache_path, cache)) {
        auto it = cache.find(sig);
        if (it != cache.end() && it->second.count("light_max") && it->second.count("slab_rows")) {
            best->light_max = (int32_t)it->second["light_max"];
            best->slab_rows = (int32_t)it->second["slab_rows"];
            if (best_ms) *best_ms = it->second.count("ms") ? it->second["ms"] : -1;
            return SPG_OK;
        }
    }
    const int light_opts[] = {256, 512, 1024};
    const int slab_opts[] = {2048, 4096, 8192};
    cudaStream_t st = (cudaStream_t)base->stream;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    double bms = 1e300;
    spg_status s = SPG_OK;
    for (int lm : light_opts) {
        for (int R : slab_opts) {
            spg_options o = *base;
            o.light_max = lm;
            o.slab_rows = R;
            o.sizing = SPG_SIZING_EXACT;
            float sum = 0;
            for (int r = 0; r < 2 && !s; r++) {
                cudaEventRecord(e0, st);
                spg_plan *p = nullptr;
                s = spgemm_plan(A, B, &o, &p);
                int64_t nnz = 0;
                if (!s) s = spgemm_symbolic(p, nullptr, &nnz);
                // the numeric pass needs room for C: measure it into plan-owned workspace
                void *rows = nullptr, *vals = nullptr;
                if (!s) {
                    rows = ws_alloc(p, (A->idx_type == SPG_IDX_I64 ? 8 : 4) * (size_t)(nnz + 1));
                    vals = ws_alloc(p, 8 * (size_t)(nnz + 1));
                    if (!rows || !vals) s = SPG_OUT_OF_MEMORY;
                }
                if (!s) {
                    spg_csc C{};
                    C.colptr = p->Ccolptr;
                    C.rowidx = rows;
                    C.vals = vals;
                    s = spgemm_numeric(p, &C);
                }
                cudaEventRecord(e1, st);
                cudaEventSynchronize(e1);
                float ms = 0;
                cudaEventElapsedTime(&ms, e0, e1);
                if (r > 0) sum += ms;
                if (p) spgemm_plan_destroy(p);
            }
            if (s) break;
            if (sum < bms) {
                bms = sum;
                best->light_max = lm;
                best->slab_rows = R;
            }
        }
        if (s) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s) return s;
    if (best_ms) *best_ms = bms;
    if (cache_path) {
        cache[sig] = {{"light_max", (double)best->light_max}, {"slab_rows", (double)best->slab_rows}, {"ms", bms}};
        if (!write_cache(cache_path, cache)) {
            set_error("cannot write tuning cache %s", cache_path);
            return SPG_INVALID_ARGUMENT;
        }
    }
    return SPG_OK;
}
