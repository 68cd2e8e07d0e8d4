// lse_tune.cu -- the tile-height autotuner (lse_autotune) and the table it
// fills.
//
// The tile-form step runs CTAs of 8 warps on 64-row tiles (3 CTAs per SM)
// or of 4 warps on 32-row tiles (6 per SM).  Tall tiles recompute fewer halo
// rows (64 / 56 u rows per output row at radius 4, against 32 / 24); short
// tiles give twice the CTAs, which an image of few tiles needs to fill the
// GPU, and more CTAs per SM to cover each other's TMA waits.  Which wins
// depends on the image size, the radius and what else runs beside it, so
// lse_autotune times the caller's own work, run together as one batch, and
// flips one shape class (term, storage type, radius, and the power of two of
// the tile count) at a time, keeping a flip that makes the whole set
// faster.  lse_evolve, lse_evolve_batch and lse_server_* all read the same
// table, so an image gets the same tiles, the same partial sums and the
// same bits whichever of them runs it.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <vector>

#include "lse_ctx.h"

using namespace lse_detail;

namespace {

// Shape class of an image for the tile-height table (kind: region with one
// band, edge term, or a vector image on its D plane), or false when the tile
// form does not serve it.
bool tune_key(int H, int W, int B, int term, int storage, int ts, TuneKey *key)
{
    const int rad = (ts - 1) / 2;
    if (rad < 1 || rad > 7) return false;
    // vector images (2-4 bands, FP32) step on their D plane: a class of their own
    if (term == LSE_TERM_REGION && B > 1 && (B > 4 || storage != LSE_F32)) return false;
    const int kind = term == LSE_TERM_EDGE ? 1 : (B > 1 ? 2 : 0);
    const int useful = 128 - 8 * ((rad + 3) / 4);
    const long long tiles =
        (long long)((W + useful - 1) / useful) * ((H + 64 - 2 * rad - 1) / (64 - 2 * rad));
    int bucket = 0;
    while ((2LL << bucket) <= tiles) ++bucket;
    *key = TuneKey{kind, storage, rad, bucket};
    return true;
}

}  // namespace

namespace lse_detail {

int tile_nw_from_env()
{
    const char *v = getenv("LSE_TILE_ROWS");
    if (v && strcmp(v, "32") == 0) return 4;
    if (v && strcmp(v, "64") == 0) return 8;
    return 0;
}

int tile_nw_default_for(int H, int W, int ts, int sm_count)
{
    // an image with fewer 64-row tiles than SMs leaves SMs idle: halve the
    // tile height (32-row tiles also overlap consecutive steps, see
    // launch_dependent)
    const int rad = (ts - 1) / 2;
    if (rad < 1 || rad > 7) return 8;
    const int useful = 128 - 8 * ((rad + 3) / 4);
    const long long tiles =
        (long long)((W + useful - 1) / useful) * ((H + 64 - 2 * rad - 1) / (64 - 2 * rad));
    return tiles < sm_count ? 4 : 8;
}

int tile_nw_for(const lse_ctx *ctx, int H, int W, int B, int term, int storage, int ts)
{
    TuneKey key;
    if (tune_key(H, W, B, term, storage, ts, &key)) {
        auto it = ctx->tile_tune.find(key);
        if (it != ctx->tile_tune.end()) return it->second;
    }
    if (ctx->tile_nw_default) return ctx->tile_nw_default;
    return tile_nw_default_for(H, W, ts, ctx->sm_count);
}

}  // namespace lse_detail

extern "C" lse_status lse_autotune(lse_ctx *ctx, int n, const lse_problem *problems,
                                   int iterations, int *tile_rows, void *stream)
{
    if (!ctx) return LSE_ERR_INVALID_ARG;
    ctx->err[0] = 0;
    if (n < 1 || n > LSE_BATCH_MAX || !problems || iterations < 1 || iterations > 1000) {
        set_err(ctx, "lse_autotune: need 1 <= n <= %d problems and 1 <= iterations <= 1000",
                LSE_BATCH_MAX);
        return LSE_ERR_INVALID_ARG;
    }
    DeviceGuard guard(ctx->device);
    if (!guard.ok) return cuda_fail(ctx, cudaErrorInvalidDevice, "set device");
    cudaStream_t s = static_cast<cudaStream_t>(stream);

    // the problems the tile form serves, grouped by shape class; trial
    // copies run `iterations` iterations without early stop into scratch
    std::map<TuneKey, std::vector<int>> groups;
    for (int i = 0; i < n; ++i) {
        const lse_problem &q = problems[i];
        TuneKey key;
        if (q.H >= 1 && q.W >= 1 &&
            tune_key(q.H, q.W, q.B, q.params.term, q.params.storage, q.params.ts, &key))
            groups[key].push_back(i);
    }
    size_t out_bytes = 0;
    for (int i = 0; i < n; ++i) {
        const size_t px = (size_t)problems[i].H * problems[i].W;
        out_bytes += (px * 4 + 255) / 256 * 256 + (px + 255) / 256 * 256;
    }
    lse_status r = ensure(ctx, reinterpret_cast<void **>(&ctx->tune_out), &ctx->tune_out_cap,
                          out_bytes, s, "lse_autotune outputs");
    if (r != LSE_OK) return r;
    std::vector<lse_problem> trial(problems, problems + n);
    unsigned char *o = reinterpret_cast<unsigned char *>(ctx->tune_out);
    for (int i = 0; i < n; ++i) {
        const size_t px = (size_t)trial[i].H * trial[i].W;
        trial[i].phi_out = reinterpret_cast<float *>(o);
        o += (px * 4 + 255) / 256 * 256;
        trial[i].mask_out = o;
        o += (px + 255) / 256 * 256;
        trial[i].params.iterations = iterations;
        trial[i].params.early_stop_frac = 0.0f;
    }

    // coordinate descent over the shape classes, on the whole problem set
    // run together: a class's height is flipped only if the time of the
    // whole batch drops, so each class is judged in the company it runs in
    // (a class alone on an idle GPU favours short tiles; the same class in a
    // full batch may not)
    std::vector<lse_stats> st(n);
    auto time_all = [&](float *ms) -> lse_status {
        *ms = INFINITY;
        for (int rep = 0; rep < 3; ++rep) {
            lse_status rr = lse_evolve_batch(ctx, n, trial.data(), 0, st.data(), stream);
            if (rr != LSE_OK) return rr;
            *ms = std::min(*ms, st[0].elapsed_ms);
        }
        return LSE_OK;
    };
    std::map<TuneKey, int> saved = ctx->tile_tune;
    for (auto &g : groups)
        if (!ctx->tile_tune.count(g.first)) {
            const lse_problem &q = problems[g.second[0]];
            ctx->tile_tune[g.first] =
                tile_nw_for(ctx, q.H, q.W, q.B, q.params.term, q.params.storage, q.params.ts);
        }
    // larger classes first: they move the total the most
    std::vector<std::pair<double, TuneKey>> order;
    for (auto &g : groups) {
        double px = 0.0;
        for (int i : g.second) px += (double)problems[i].H * problems[i].W;
        order.push_back({-px, g.first});
    }
    std::sort(order.begin(), order.end());
    float best = 0.0f;
    lse_status r2 = time_all(&best);          // warms up, then the baseline
    if (r2 == LSE_OK) r2 = time_all(&best);
    for (size_t k = 0; k < order.size() && r2 == LSE_OK; ++k) {
        const TuneKey &key = order[k].second;
        const int was = ctx->tile_tune[key];
        ctx->tile_tune[key] = was == 8 ? 4 : 8;
        float ms = 0.0f;
        r2 = time_all(&ms);
        if (r2 == LSE_OK && ms < best * 0.995f) best = ms;
        else ctx->tile_tune[key] = was;
    }
    if (r2 != LSE_OK) {
        ctx->tile_tune = saved;
        return r2;
    }
    if (tile_rows)
        for (int i = 0; i < n; ++i) {
            const lse_problem &q = problems[i];
            TuneKey key;
            tile_rows[i] = q.H >= 1 && q.W >= 1 && tune_key(q.H, q.W, q.B, q.params.term,
                                                            q.params.storage, q.params.ts, &key)
                               ? 8 * ctx->tile_tune[key]
                               : 0;
        }
    return LSE_OK;
}
