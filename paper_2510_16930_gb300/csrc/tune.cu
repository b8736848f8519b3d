// Autotuner of the nonzero-stream pass (opt.autotune = 1).
//
// Per mode with a hybrid layout it picks the tile shape, gather layout and block
// size of the pass: first the lane tile of the FP32 FMA tiles (8 x 8, 8 x 4 or
// 4 x 8 accumulators per lane, which sets how many lanes share a nonzero and how
// many nonzeros a warp takes per step; the split-BF16 form keeps its tensor-core
// tiles), then, with that tile, the row length Lshort above which a row is
// streamed contiguously (shorter rows go to length-sorted slices) and the
// work-item size T (nonzeros per item; long rows are cut into items of T and
// dealt in contiguous ranges).  Each candidate is built and its pass timed with
// CUDA events on the context's stream on the context's own data; the fastest is
// kept.  Choices are cached per (order, ranks, mode, log2 nnz, share of nonzeros
// in long rows, precision), in memory and, when the environment variable
// HOQRI_TUNE_CACHE names a file, in that file (one "key Lshort T TL TV" line
// each), so later contexts of the same kind skip the timing.
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

struct Choice {
    int64_t Lshort = 0, T = 0;
    int TL = 0, TV = 0;  // 0: the plan's own tile
};

std::mutex g_mu;
std::map<std::string, Choice> g_cache;
bool g_loaded = false;

void load_file() {
    if (g_loaded) return;
    g_loaded = true;
    const char *path = std::getenv("HOQRI_TUNE_CACHE");
    if (!path) return;
    FILE *f = std::fopen(path, "r");
    if (!f) return;
    char line[1024];
    while (std::fgets(line, sizeof line, f)) {
        char key[512];
        long long ls = 0, t = 0;
        int tl = 0, tv = 0;
        const int got = std::sscanf(line, "%511s %lld %lld %d %d", key, &ls, &t, &tl, &tv);
        if (got >= 3) g_cache[key] = Choice{ls, t, got == 5 ? tl : 0, got == 5 ? tv : 0};
    }
    std::fclose(f);
}

void save_line(const std::string &key, const Choice &ch) {
    const char *path = std::getenv("HOQRI_TUNE_CACHE");
    if (!path) return;
    FILE *f = std::fopen(path, "a");
    if (!f) return;
    std::fprintf(f, "%s %lld %lld %d %d\n", key.c_str(), (long long)ch.Lshort, (long long)ch.T, ch.TL, ch.TV);
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
        FastTile p0;
        if (!hyb_tile(c, n, &p0)) continue;
        const int64_t T0 = M.tune_T, L0 = M.tune_Lshort;
        const double long_share = c->nnz > 0 ? (double)M.long_elems / (double)c->nnz : 0.0;
        const std::string key = tune_key(c, n, long_share);
        Choice built{L0, T0, M.tune_TL, M.tune_TV};
        // (re)build mode n's layout for a candidate (the slice width follows the tile)
        auto build = [&](const Choice &ch) -> hoqri_status {
            if (ch.Lshort == built.Lshort && ch.T == built.T && ch.TL == built.TL && ch.TV == built.TV)
                return HOQRI_OK;
            M.tune_TL = ch.TL;
            M.tune_TV = ch.TV;
            FastTile p;
            if (!hyb_tile(c, n, &p)) {
                set_error("autotuner: mode lost its tile plan");
                return HOQRI_ERR_UNSUPPORTED;
            }
            free_hybrid(c, n);
            HQ_TRY(build_hybrid(c, n, ch.Lshort, ch.T, 32 / p.lpn));
            built = ch;
            return HOQRI_OK;
        };
        Choice best = built;
        auto it = g_cache.find(key);
        if (it != g_cache.end()) {
            best = it->second;
        } else {
            float best_ms = 1e30f;
            auto trial = [&](const Choice &ch) -> hoqri_status {
                HQ_TRY(build(ch));
                float ms = 0.f;
                HQ_TRY(time_pass(c, n, 2, &ms));
                if (ms < best_ms) {
                    best_ms = ms;
                    best = ch;
                }
                return HOQRI_OK;
            };
            // 1. lane tile with the default layout (FP32 FMA tiles only)
            std::vector<std::pair<int, int>> tiles = {{built.TL, built.TV}};
            if (!c->mix && p0.TL == 8 && p0.TV == 8 && c->opt.tile_rows == 0) tiles = {{0, 0}, {8, 4}, {4, 8}};
            for (const auto &tv : tiles) {
                Choice ch{L0, T0, tv.first, tv.second};
                if (tv.first && tv.first != built.TL) {
                    M.tune_TL = tv.first;
                    M.tune_TV = tv.second;
                    FastTile p;
                    const bool ok = hyb_tile(c, n, &p) && p.TL == tv.first && p.TV == tv.second &&
                                    hyb_smem_need(c, n) <= hyb_smem_cap();
                    M.tune_TL = built.TL;
                    M.tune_TV = built.TV;
                    if (!ok) continue;
                }
                HQ_TRY(trial(ch));
            }
            // 2. layout with the best tile
            const int TLb = best.TL, TVb = best.TV;
            const int64_t cand[][2] = {{64, T0}, {1024, T0}, {L0, 4 * T0}, {64, 4 * T0},
                                       {L0, std::max<int64_t>(256, T0 / 4)}};
            for (const auto &cd : cand) HQ_TRY(trial(Choice{cd[0], cd[1], TLb, TVb}));
            g_cache[key] = best;
            save_line(key, best);
        }
        HQ_TRY(build(best));
    }
    return HOQRI_OK;
}

}  // namespace hoqri
