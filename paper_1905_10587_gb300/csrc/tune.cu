// Autotuning of the kernel product's work split.
//
// The products choose their column-split count (and, for the tensor-core form, whether the
// P.V contraction runs on the tensor cores) from a cost model of waves and per-item
// overhead.  krr_autotune times the candidates for the built problem of a context instead
// and keeps the fastest in a process-wide table keyed by
//     (product form, feature width, right-hand sides per launch, floor(log2 n)),
// which later products of the same key use when opts.autotune = 1.  The table can be
// written to and read from a JSON file, so tuned choices carry over between processes.
#include "internal.cuh"

#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

namespace krr {

namespace {
struct TuneTable {
    std::mutex mu;
    std::map<std::string, TuneEntry> entries;
};
TuneTable& table() {
    static TuneTable t;
    return t;
}
}  // namespace

std::string tune_key(int form, int width, int nrhs, long long n) {
    int lg = 0;
    while ((2LL << lg) <= n) ++lg;
    char buf[96];
    std::snprintf(buf, sizeof(buf), "form=%d w=%d r=%d lg=%d", form, width, nrhs, lg);
    return buf;
}

bool tune_lookup(const krr_ctx* ctx, const std::string& key, TuneEntry* out) {
    if (!ctx || ctx->tuning || !ctx->opts.autotune) return false;
    TuneTable& t = table();
    std::lock_guard<std::mutex> lock(t.mu);
    auto it = t.entries.find(key);
    if (it == t.entries.end()) return false;
    *out = it->second;
    return true;
}

int tuned_splits(krr_ctx* ctx, const std::string& key, int analytic, int ntiles) {
    int s = analytic;
    TuneEntry e;
    if (ctx->force_splits > 0) s = ctx->force_splits;
    else if (tune_lookup(ctx, key, &e) && e.splits > 0) s = e.splits;
    s = std::max(1, std::min(s, std::max(1, ntiles)));
    ctx->last_splits = s;
    return s;
}

static void tune_store(const std::string& key, const TuneEntry& e) {
    TuneTable& t = table();
    std::lock_guard<std::mutex> lock(t.mu);
    t.entries[key] = e;
}

// V[q * n + i] = a deterministic pattern of both signs (the product's speed does not depend
// on the values)
__global__ void k_tune_fill(float* V, long long tot) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < tot) V[i] = (float)((i * 2654435761LL) % 2001 - 1000) * 1e-3f;
}

}  // namespace krr

using namespace krr;

extern "C" int krr_autotune(krr_ctx* ctx, int nrhs, int reps, int* splits_out, int* pv_out,
                            double* ms_out) {
    if (!ctx) return KRR_E_INVAL;
    if (!ctx->built) return fail(ctx, KRR_E_STATE, "krr_autotune before krr_build_precond");
    if (!(nrhs == 1 || nrhs == 2 || nrhs == 4 || nrhs == 8 || nrhs == 16) || reps < 1 || reps > 100)
        return fail(ctx, KRR_E_INVAL, "krr_autotune: nrhs must be 1, 2, 4, 8 or 16 and reps in 1..100");
    const long long n = ctx->n;
    const int form = ctx->opts.precision == 1 ? (ctx->FA ? 1 : 0) : ctx->opts.precision;
    const int width = form == 1 ? tc_feature_kp(ctx->d) : kernel_dim(ctx->d);
    float *V, *Q;
    KRR_RET(bufT(ctx, "tune_v", (size_t)n * nrhs, &V));
    KRR_RET(bufT(ctx, "tune_q", (size_t)n * nrhs, &Q));
    k_tune_fill<<<(unsigned)ceil_div(n * nrhs, 256), 256, 0, ctx->stream>>>(V, n * nrhs);
    KRR_CHECK_LAUNCH();
    // candidates: the cost model's own choice (0) and a spread of split counts; with
    // tensor-core features of width 64, both P.V forms
    const int cand[] = {0, 1, 2, 3, 4, 6, 8, 12, 16, 24, 32, 48, 64};
    std::vector<int> pvs = {-1};
    if (form == 1 && width == 64) pvs = {0, 1};
    cudaEvent_t e0, e1;
    KRR_TRY_CUDA(cudaEventCreate(&e0));
    KRR_TRY_CUDA(cudaEventCreate(&e1));
    ctx->tuning = true;
    TuneEntry best{0, 0, HUGE_VAL};
    int rc = KRR_OK;
    for (int pv : pvs) {
        for (int c : cand) {
            ctx->force_splits = c;
            ctx->force_pv = pv;
            rc = square_product(ctx, V, nrhs, Q, form);   // warm-up (and allocations)
            if (rc != KRR_OK) break;
            const int used = ctx->last_splits;
            if (c > 0 && used != c) continue;               // beyond the tile count
            cudaEventRecord(e0, ctx->stream);
            for (int r = 0; r < reps && rc == KRR_OK; ++r) rc = square_product(ctx, V, nrhs, Q, form);
            cudaEventRecord(e1, ctx->stream);
            if (cudaEventSynchronize(e1) != cudaSuccess) rc = KRR_E_CUDA;
            if (rc != KRR_OK) break;
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            const double t = ms / reps;
            if (t < best.ms) best = TuneEntry{used, pv < 0 ? 0 : pv, t};
        }
        if (rc != KRR_OK) break;
    }
    ctx->tuning = false;
    ctx->force_splits = 0;
    ctx->force_pv = -1;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != KRR_OK) return rc;
    tune_store(tune_key(form, width, nrhs, n), best);
    if (splits_out) *splits_out = best.splits;
    if (pv_out) *pv_out = best.pv;
    if (ms_out) *ms_out = best.ms;
    return KRR_OK;
}

extern "C" int krr_tune_clear(void) {
    TuneTable& t = table();
    std::lock_guard<std::mutex> lock(t.mu);
    t.entries.clear();
    return KRR_OK;
}

extern "C" int krr_tune_get(const char* key, int* splits, int* pv, double* ms) {
    if (!key) return KRR_E_INVAL;
    TuneTable& t = table();
    std::lock_guard<std::mutex> lock(t.mu);
    auto it = t.entries.find(key);
    if (it == t.entries.end()) return KRR_E_STATE;
    if (splits) *splits = it->second.splits;
    if (pv) *pv = it->second.pv;
    if (ms) *ms = it->second.ms;
    return KRR_OK;
}

extern "C" int krr_tune_set(const char* key, int splits, int pv, double ms) {
    if (!key || std::strlen(key) == 0 || std::strlen(key) > 80 || splits < 0 || splits > 4096 || pv < 0 || pv > 1)
        return KRR_E_INVAL;
    tune_store(key, TuneEntry{splits, pv, ms});
    return KRR_OK;
}

// {"krr_tune": 1, "entries": [
//  {"key": "form=1 w=64 r=16 lg=16", "splits": 4, "pv": 1, "ms": 6.61},
//  ...
// ]}
extern "C" int krr_tune_save(const char* path) {
    if (!path) return KRR_E_INVAL;
    TuneTable& t = table();
    std::lock_guard<std::mutex> lock(t.mu);
    FILE* f = std::fopen(path, "w");
    if (!f) return KRR_E_INVAL;
    std::fprintf(f, "{\"krr_tune\": 1, \"entries\": [\n");
    size_t i = 0;
    for (const auto& kv : t.entries) {
        std::fprintf(f, " {\"key\": \"%s\", \"splits\": %d, \"pv\": %d, \"ms\": %.6g}%s\n", kv.first.c_str(),
                     kv.second.splits, kv.second.pv, std::isfinite(kv.second.ms) ? kv.second.ms : 0.0,
                     ++i < t.entries.size() ? "," : "");
    }
    std::fprintf(f, "]}\n");
    return std::fclose(f) == 0 ? KRR_OK : KRR_E_INVAL;
}

// Reads a file written by krr_tune_save (one entry per line) and adds its entries;
// KRR_E_INVAL when the file is missing or a line that names a key does not parse.
extern "C" int krr_tune_load(const char* path) {
    if (!path) return KRR_E_INVAL;
    FILE* f = std::fopen(path, "r");
    if (!f) return KRR_E_INVAL;
    char line[512];
    bool header = false;
    std::vector<std::pair<std::string, TuneEntry>> got;
    int rc = KRR_OK;
    while (std::fgets(line, sizeof(line), f)) {
        if (std::strstr(line, "\"krr_tune\"")) header = true;
        const char* k = std::strstr(line, "\"key\": \"");
        if (!k) continue;
        k += 8;
        const char* ke = std::strchr(k, '"');
        const char* sp = std::strstr(line, "\"splits\":");
        const char* pv = std::strstr(line, "\"pv\":");
        const char* ms = std::strstr(line, "\"ms\":");
        TuneEntry e{0, 0, 0.0};
        if (!ke || ke - k > 80 || !sp || !pv || !ms || std::sscanf(sp + 9, "%d", &e.splits) != 1 ||
            std::sscanf(pv + 5, "%d", &e.pv) != 1 || std::sscanf(ms + 5, "%lf", &e.ms) != 1 || e.splits < 0 ||
            e.splits > 4096 || e.pv < 0 || e.pv > 1) {
            rc = KRR_E_INVAL;
            break;
        }
        got.emplace_back(std::string(k, ke - k), e);
    }
    std::fclose(f);
    if (rc != KRR_OK || !header) return KRR_E_INVAL;
    for (const auto& g : got) tune_store(g.first, g.second);
    return KRR_OK;
}
