// Autotuner of the nonzero-stream pass (opt.autotune = 1).
//
// Per mode with a hybrid layout it picks the gather layout and block size of
// the pass: the row length Lshort above which a row is streamed contiguously
// (shorter rows go to length-sorted slices) and the work-item size T (nonzeros
// per item; long rows are cut into items of T and dealt in contiguous ranges).
// Each candidate layout is built and its pass timed with CUDA events on the
// context's stream on the context's own data; the fastest is kept.  Choices
// are cached per (order, ranks, mode, log2 nnz, share of nonzeros in long
// rows, precision), in memory and, when the environment variable
// HOQRI_TUNE_CACHE names a file, in that file (one "key Lshort T" line each),
// so later contexts of the same kind skip the timing.
#include <cstdio>
#include <cstdlib>
#include <map>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "internal.cuh"

namespace hoqri {

namespace {

std::mutex g_mu;
std::map<std::string, std::pair<int64_t, int64_t>> g_cache;
bool g_loaded = false;

void load_file() {
    if (g_loaded) return;
    g_loaded = true;
    const char *path = std::getenv("HOQRI_TUNE_CACHE");
    if (!path) return;
    FILE *f = std::fopen(path, "r");
    if (!f) return;
    char key[512];
    long long ls = 0, t = 0;
    while (std::fscanf(f, "%511s %lld %lld", key, &ls, &t) == 3) g_cache[key] = {ls, t};
    std::fclose(f);
}

void save_line(const std::string &key, int64_t ls, int64_t t) {
    const char *path = std::getenv("HOQRI_TUNE_CACHE");
    if (!path) return;
    FILE *f = std::fopen(path, "a");
    if (!f) return;
    std::fprintf(f, "%s %lld %lld\n", key.c_str(), (long long)ls, (long long)t);
    std::fclose(f);
}

std::string tune_key(const hoqri_ctx *c, int n, double long_share) {
    int lg = 0;
    while (lg < 62 && ((int64_t)1 << (lg + 1)) <= c->nnz) ++lg;
    std::string k = "N" + std::to_string(c->N) + "_K";
    for (int m = 0; m < c->N; ++m) k += std::to_string(c->K[m]) + (m + 1 < c->N ? "x" : "");
    k += "_n" + std::to_string(n) + "_lg" + std::to_string(lg) + "_long" + std::to_string((int)(long_share * 10 + 0.5)) +
         "_p" + std::to_string(c->mix ? 2 : (int)c->prec);
    return k;
}

// mean time of `reps` passes after one untimed pass
hoqri_status time_pass(hoqri_ctx *c, int n, int reps, float *ms) {
    cudaEvent_t e0, e1;
    HQ_CUDA(cudaEventCreate(&e0));
    HQ_CUDA(cudaEventCreate(&e1));
    hoqri_status s = hyb_pass(c, n);
    if (s == HOQRI_OK) {
        cudaEventRecord(e0, c->stream);
        for (int r = 0; r < reps && s == HOQRI_OK; ++r) s = hyb_pass(c, n);
        cudaEventRecord(e1, c->stream);
        cudaEventSynchronize(e1);
        cudaEventElapsedTime(ms, e0, e1);
        *ms /= reps;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    HQ_CUDA(cudaGetLastError());
    return s;
}

}  // namespace

hoqri_status autotune_hybrid(hoqri_ctx *c) {
    std::lock_guard<std::mutex> lk(g_mu);
    load_file();
    for (int n = 0; n < c->N; ++n) {
        ModeStore &M = c->ms[n];
        if (!hyb_mode(c, n) || !M.hyb) continue;
        FastTile p;
        if (!hyb_tile(c, n, &p)) continue;
        const int SW = 32 / p.lpn;
        const int64_t T0 = M.tune_T, L0 = M.tune_Lshort;
        const double long_share = c->nnz > 0 ? (double)M.long_elems / (double)c->nnz : 0.0;
        const std::string key = tune_key(c, n, long_share);
        int64_t bestL = L0, bestT = T0;
        auto it = g_cache.find(key);
        if (it != g_cache.end()) {
            bestL = it->second.first;
            bestT = it->second.second;
        } else {
            const int64_t cand[][2] = {{L0, T0}, {64, T0}, {1024, T0}, {L0, 4 * T0}, {64, 4 * T0}, {L0, std::max<int64_t>(256, T0 / 4)}};
            float best = 1e30f;
            int64_t builtL = L0, builtT = T0;
            for (const auto &cd : cand) {
                if (cd[0] != builtL || cd[1] != builtT) {
                    free_hybrid(c, n);
                    HQ_TRY(build_hybrid(c, n, cd[0], cd[1], SW));
                    builtL = cd[0];
                    builtT = cd[1];
                }
                float ms = 0.f;
                HQ_TRY(time_pass(c, n, 2, &ms));
                if (ms < best) {
                    best = ms;
                    bestL = cd[0];
                    bestT = cd[1];
                }
            }
            g_cache[key] = {bestL, bestT};
            save_line(key, bestL, bestT);
            if (builtL == bestL && builtT == bestT) continue;
        }
        if (bestL != M.tune_Lshort || bestT != M.tune_T) {
            free_hybrid(c, n);
            HQ_TRY(build_hybrid(c, n, bestL, bestT, SW));
        }
    }
    return HOQRI_OK;
}

}  // namespace hoqri
