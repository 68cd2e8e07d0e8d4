// lse_batch.cu -- lse_evolve_batch: many independent evolutions (images of
// any size, term, band count and iteration cap) advanced together.
//
// Every image keeps what lse_evolve would give it alone: its own planes,
// statistics record, partials, tensor maps and CTA count, so its results are
// bit for bit those of lse_evolve.  What changes is the launch structure:
// images are grouped into classes by step kernel (form, term, bands, radius),
// and iteration n of every image of a class is one launch whose CTAs find
// their image in a CTA table.  An image past its cap or stopped early leaves
// its CTAs idle.  The whole loop (max cap x classes launches) can be
// captured in a CUDA graph and replayed as one submission.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <tuple>
#include <vector>

#include "lse_classes.h"
#include "lse_ctx.h"

using namespace lse_detail;

namespace {

constexpr size_t kAlign = 256;

size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

// Grows the context's pinned host mirror to at least `bytes`.
lse_status ensure_host(lse_ctx *ctx, size_t bytes, cudaStream_t s)
{
    if (ctx->bhost_cap >= bytes && ctx->bhost) return LSE_OK;
    if (ctx->bhost) {
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "synchronise before growing host mirror");
        cudaFreeHost(ctx->bhost);
        ctx->bhost = nullptr;
        ctx->bhost_cap = 0;
    }
    cudaError_t e = cudaMallocHost(&ctx->bhost, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        ctx->bhost = nullptr;
        set_err(ctx, "cudaMallocHost of %zu bytes failed", bytes);
        return LSE_ERR_OOM;
    }
    ctx->bhost_cap = bytes;
    return LSE_OK;
}

// A group launch of vector images: one band count and radius, images
// [first, first + count) of the group list, with their CTA shares.
struct MbChunk {
    int B, rad;
    std::vector<int> images;         // batch indices
    std::vector<int> ncta;
    int total = 0;
};

// Splits the vector images of one band count and radius into launches the
// device holds at once (`cap` CTAs each, at least one a image) and shares
// each launch's CTAs by the images' work (tiles x iteration cap), at most
// one CTA per tile.  The shares change no result: an image's sums are exact
// integers, the same however many CTAs add them.
void share_ctas(const std::vector<int> &imgs, const std::vector<long long> &tiles,
                const std::vector<long long> &work, int cap, int B, int rad,
                std::vector<MbChunk> *out)
{
    for (size_t i0 = 0; i0 < imgs.size(); i0 += (size_t)cap) {
        MbChunk c;
        c.B = B;
        c.rad = rad;
        const size_t i1 = std::min(imgs.size(), i0 + (size_t)cap);
        c.images.assign(imgs.begin() + i0, imgs.begin() + i1);
        c.ncta.assign(c.images.size(), 1);
        int used = (int)c.images.size();
        // greedily to the image with the most work per CTA
        while (used < cap) {
            int best = -1;
            double best_w = 0.0;
            for (size_t k = 0; k < c.images.size(); ++k) {
                const int i = c.images[k];
                if (c.ncta[k] >= tiles[i]) continue;
                const double w = (double)work[i] / c.ncta[k];
                if (w > best_w) {
                    best_w = w;
                    best = (int)k;
                }
            }
            if (best < 0) break;
            ++c.ncta[best];
            ++used;
        }
        c.total = used;
        out->push_back(c);
    }
}

}  // namespace

namespace lse_detail {

ClassKey class_of(const StepPlan &plan, int term, int bands)
{
    return ClassKey{plan.form, term, bands, plan.args.rad, plan.wpc, plan.args.storage,
                    plan.form == LSE_FORM_TILE ? plan.args.nw : 0};
}

ImagePlanes image_planes(const lse_problem &q)
{
    ImagePlanes L;
    L.pitch = round_up(q.W, 32);
    L.es = q.params.storage == LSE_F32 ? 4 : 2;
    const int bands = q.params.term == LSE_TERM_REGION ? q.B : 1;
    const size_t plane = (size_t)q.H * L.pitch * L.es;
    L.data = 0;
    L.phi0 = align_up(plane * bands);
    L.phi1 = L.phi0 + align_up(plane);
    L.end = L.phi1 + align_up(plane);
    L.dplane = 0;
    if (bands > 1 && bands <= 4 && L.es == 4) {
        L.dplane = L.end;
        L.end += align_up(plane);
    }
    return L;
}

cudaError_t stage_problem(const lse_problem &q, unsigned char *base, const ImagePlanes &L,
                          LseDevState *st, LsePartial *parts, int nred, int sm_count,
                          int form, int tile_nw, StepPlan *plan, bool *planned,
                          cudaStream_t s)
{
    const lse_params &p = q.params;
    const bool region = p.term == LSE_TERM_REGION;
    const int sto = p.storage;
    const int pitch = L.pitch;
    const size_t bstride = (size_t)q.H * pitch;
    void *data = base + L.data;
    float *phi[2] = {reinterpret_cast<float *>(base + L.phi0),
                     reinterpret_cast<float *>(base + L.phi1)};
    cudaError_t e = cudaSuccess;
    *planned = false;
    if (sto == LSE_F32) {
        if (region) e = launch_convert(q.image, q.dtype, q.H, q.W, q.B, static_cast<float *>(data),
                                       pitch, s);
        if (e == cudaSuccess)
            e = launch_prologue(region ? data : nullptr, pitch, bstride, q.phi0,
                                region ? nullptr : q.g, q.W, phi[0],
                                region ? nullptr : static_cast<float *>(data), pitch, q.H, q.W,
                                q.B, p.term, p.dt, LSE_F32, st, parts, nred, s);
    } else {
        // one band or g: FP32 first (into the two LSF planes, which together
        // hold at least H x pitch floats), then rounded to the storage type
        if (region) {
            float *tmp = phi[0];
            e = launch_convert(q.image, q.dtype, q.H, q.W, 1, tmp, pitch, s);
            if (e == cudaSuccess) e = launch_quantise(tmp, pitch, q.H, q.W, data, pitch, sto, s);
        } else {
            e = launch_quantise(q.g, q.W, q.H, q.W, data, pitch, sto, s);
        }
        if (e == cudaSuccess)
            e = launch_prologue(region ? data : nullptr, pitch, bstride, q.phi0,
                                region ? nullptr : data, pitch, phi[0], nullptr, pitch, q.H,
                                q.W, q.B, p.term, p.dt, sto, st, parts, nred, s);
    }
    if (e != cudaSuccess) return e;
    float *dplane = L.dplane ? reinterpret_cast<float *>(base + L.dplane) : nullptr;
    *planned = plan_step(q.H, q.W, q.B, p, pitch, bstride, data, phi, st, parts, sm_count, form,
                         tile_nw, dplane, plan) &&
               plan->form != LSE_FORM_GENERIC;
    return cudaSuccess;
}

size_t layout_classes(ClassMap &classes, BatchItem *items)
{
    size_t toff = 0;
    for (auto &kc : classes) {
        Class &c = kc.second;
        std::stable_sort(c.items.begin(), c.items.end(), [&](int a, int b) {
            return items[a].iter0 + items[a].cap > items[b].iter0 + items[b].cap;
        });
        c.ends.clear();
        c.pre.assign(1, 0);
        c.npre.assign(1, 0);
        c.nblocks = c.nnblocks = 0;
        for (int i : c.items) {
            BatchItem &it = items[i];
            it.start = c.nblocks;
            c.nblocks += it.nblocks;
            it.nstart = c.nnblocks;
            c.nnblocks += it.nnblocks;
            c.ends.push_back(it.iter0 + it.cap);
            c.pre.push_back(c.nblocks);
            c.npre.push_back(c.nnblocks);
        }
        c.blk_off = toff;
        toff = align_up(toff + sizeof(int) * c.nblocks);
        c.nblk_off = toff;
        toff = align_up(toff + sizeof(int) * c.nnblocks);
    }
    return toff;
}

void fill_tables(const ClassMap &classes, const BatchItem *items, unsigned char *host_tables)
{
    for (auto &kc : classes) {
        int *blk = reinterpret_cast<int *>(host_tables + kc.second.blk_off);
        int *nblk = reinterpret_cast<int *>(host_tables + kc.second.nblk_off);
        for (int i : kc.second.items) {
            for (int b = 0; b < items[i].nblocks; ++b) blk[items[i].start + b] = i;
            for (int b = 0; b < items[i].nnblocks; ++b) nblk[items[i].nstart + b] = i;
        }
    }
}

cudaError_t launch_class(const ClassKey &k, const Class &c, const BatchItem *items,
                         const unsigned char *tables, long long n, cudaStream_t s, int k_act)
{
    if (k_act < 0) k_act = (int)c.items.size();
    const int nb = c.pre[k_act], nnb = c.npre[k_act];
    if (nb == 0) return cudaSuccess;
    const int *blk = reinterpret_cast<const int *>(tables + c.blk_off);
    if (k.form == LSE_FORM_TILE) {
        if (k.bands > 1) {
            // vector images: statistics and D before the step on the D plane
            const int *nblk = reinterpret_cast<const int *>(tables + c.nblk_off);
            cudaError_t e = launch_band_passes_batch(items, nblk, n, nnb, s);
            if (e != cudaSuccess) return e;
        }
        return launch_step_tile_batch(k.storage, k.bands > 1 ? LSE_TERM_EDGE : k.term, k.nw,
                                      k.rad, items, blk, n, nb, s);
    }
    if (k.term == LSE_TERM_EDGE)
        return launch_step_tma_batch_edge(k.rad, items, blk, n, nb, k.wpc, s);
    if (k.bands == 1)
        return launch_step_tma_batch_region1(k.rad, items, blk, n, nb, k.wpc, s);
    const int *nblk = reinterpret_cast<const int *>(tables + c.nblk_off);
    cudaError_t e = launch_normaliser_batch(items, nblk, n, nnb, s);
    if (e != cudaSuccess) return e;
    return launch_step_tma_batch_multiband(k.rad, items, blk, n, nb, k.wpc, s);
}

int normaliser_blocks(int H, int sm_count)
{
    // one CTA per row at most (the pass walks rows), as lse_evolve launches it
    const int cap = sm_count * 4;
    return H < cap ? (H < 1 ? 1 : H) : cap;
}

}  // namespace lse_detail

extern "C" {

lse_status lse_evolve_batch(lse_ctx *ctx, int n, const lse_problem *problems, int use_graph,
                            lse_stats *stats, void *stream)
{
    if (!ctx) return LSE_ERR_INVALID_ARG;
    ctx->err[0] = 0;
    if (n < 1 || n > LSE_BATCH_MAX || !problems) {
        set_err(ctx, "lse_evolve_batch: need 1 <= n <= %d images and a problem array",
                LSE_BATCH_MAX);
        return LSE_ERR_INVALID_ARG;
    }
    DeviceGuard guard(ctx->device);
    if (!guard.ok) return cuda_fail(ctx, cudaErrorInvalidDevice, "set device");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    lse_status r;

    // ---- validation (nothing is enqueued before every image passes)
    for (int i = 0; i < n; ++i) {
        const lse_problem &q = problems[i];
        const bool region = q.params.term == LSE_TERM_REGION;
        if (q.H < 1 || q.W < 1 || q.B < 1 || q.B > LSE_MAXB) {
            set_err(ctx, "lse_evolve_batch: image %d: need H, W >= 1 and 1 <= B <= %d", i,
                    LSE_MAXB);
            return LSE_ERR_INVALID_ARG;
        }
        if (region && q.dtype != LSE_F32 && q.dtype != LSE_F16 && q.dtype != LSE_BF16 &&
            q.dtype != LSE_U16) {
            set_err(ctx, "lse_evolve_batch: image %d: unknown dtype %d", i, (int)q.dtype);
            return LSE_ERR_INVALID_ARG;
        }
        if ((r = check_params(ctx, q.params, q.B)) != LSE_OK) return r;
        if (q.params.order != LSE_ORDER_LISTING || q.params.padding != LSE_PAD_ZERO) {
            set_err(ctx, "lse_evolve_batch: image %d: batches use the listing's order and "
                         "zero padding", i);
            return LSE_ERR_INVALID_ARG;
        }
        const bool ok = classify(q.phi0, ctx->device) == PTR_DEVICE &&
                        classify(q.phi_out, ctx->device) == PTR_DEVICE &&
                        (!q.mask_out || classify(q.mask_out, ctx->device) == PTR_DEVICE) &&
                        (region ? (classify(q.image, ctx->device) == PTR_DEVICE && !q.g)
                                : classify(q.g, ctx->device) == PTR_DEVICE);
        if (!ok) {
            set_err(ctx, "lse_evolve_batch: image %d: image (region) or g (edge), phi0, "
                         "phi_out and mask_out must be device memory of the context's GPU",
                    i);
            return LSE_ERR_INVALID_ARG;
        }
    }

    // ---- arena: per image [data][phi0][phi1]; then states, partials, items
    std::vector<ImagePlanes> lay(n);
    std::vector<size_t> base(n);
    size_t off = 0;
    for (int i = 0; i < n; ++i) {
        lay[i] = image_planes(problems[i]);
        base[i] = off;
        off += lay[i].end;
    }
    const int nparts = partials_needed(ctx->sm_count);
    const size_t st_off = off;
    off = align_up(off + sizeof(LseDevState) * n);
    const size_t part_off = off;
    off = align_up(off + sizeof(LsePartial) * (size_t)nparts * n);
    const size_t item_off = off;
    off = align_up(off + sizeof(BatchItem) * n);
    // vector images (2-4 bands, FP32) run as groups of persistent
    // evolutions, each with the normaliser's candidates
    std::vector<char> mb(n, 0);
    int n_mb = 0;
    for (int i = 0; i < n; ++i) {
        const lse_problem &q = problems[i];
        mb[i] = q.params.term == LSE_TERM_REGION && q.params.storage == LSE_F32 &&
                ctx->step_form == LSE_FORM_AUTO && evolve_bands_applies(q.H, q.W, q.B, q.params);
        n_mb += mb[i];
    }
    const size_t cand_off = off;
    off = align_up(off + sizeof(LseCandidates) * (size_t)n_mb);
    if ((r = ensure(ctx, &ctx->arena, &ctx->arena_cap, off, s, "batch arena")) != LSE_OK) return r;
    unsigned char *A = static_cast<unsigned char *>(ctx->arena);
    LseDevState *states = reinterpret_cast<LseDevState *>(A + st_off);
    LsePartial *partials = reinterpret_cast<LsePartial *>(A + part_off);
    BatchItem *d_items = reinterpret_cast<BatchItem *>(A + item_off);
    LseCandidates *cands = reinterpret_cast<LseCandidates *>(A + cand_off);
    cudaError_t e = cudaMemsetAsync(states, 0, sizeof(LseDevState) * n, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "lse_evolve_batch: clear states");

    // ---- staging and prologue of every image; the plan of its step
    std::vector<BatchItem> items(n);
    ClassMap classes;
    const int nred = ctx->sm_count * 4;
    std::vector<MbGroupItem> mb_items;
    std::vector<int> mb_index(n, -1);
    std::vector<long long> mb_tiles(n, 0), mb_work(n, 0);
    std::map<std::pair<int, int>, std::vector<int>> mb_groups;
    for (int i = 0; i < n; ++i) {
        const lse_problem &q = problems[i];
        const lse_params &p = q.params;
        const bool region = p.term == LSE_TERM_REGION;
        LsePartial *parts = partials + (size_t)nparts * i;
        StepPlan plan;
        bool planned = false;
        e = stage_problem(q, A + base[i], lay[i], states + i, parts, nred, ctx->sm_count,
                          ctx->step_form, tile_nw_for(ctx, q.H, q.W, q.B, p.term, p.storage, p.ts),
                          &plan, &planned, s);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "lse_evolve_batch: staging and prologue");
        if (!planned) {
            set_err(ctx, "lse_evolve_batch: image %d needs the plain step kernel (ts > 15, "
                         "more than 4 bands, or LSE_STEP_KERNEL=generic); run it with "
                         "lse_evolve",
                    i);
            return LSE_ERR_INVALID_ARG;
        }
        BatchItem &it = items[i];
        memset(&it, 0, sizeof(it));
        it.phi_maps[0] = plan.phi_maps[0];
        it.phi_maps[1] = plan.phi_maps[1];
        it.data_map = plan.data_map;
        it.args = plan.args;
        it.phi[0] = plan.phi[0];
        it.phi[1] = plan.phi[1];
        it.nblocks = plan.nblocks;
        it.cap = p.iterations;
        it.reinit_period = p.reinit_period;
        it.early_stop = p.early_stop_frac > 0.0f;
        it.iter0 = 0;
        if (region && q.B > 1) it.nnblocks = normaliser_blocks(q.H, ctx->sm_count);
        if (mb[i]) {
            // the normaliser's candidates, then the persistent evolution's plan
            LseCandidates *cand = cands + mb_items.size();
            const float *bands = reinterpret_cast<const float *>(A + base[i] + lay[i].data);
            const int pitch = lay[i].pitch;
            const size_t bstride = (size_t)q.H * pitch;
            e = launch_mb_candidates(bands, pitch, bstride, q.H, q.W, q.B, cand, states + i,
                                     ctx->sm_count, s);
            if (e != cudaSuccess) return cuda_fail(ctx, e, "lse_evolve_batch: candidates");
            MbGroupItem g;
            memset(&g, 0, sizeof(g));
            int tiles = 0;
            float *phis[2] = {reinterpret_cast<float *>(A + base[i] + lay[i].phi0),
                              reinterpret_cast<float *>(A + base[i] + lay[i].phi1)};
            if (!plan_evolve_bands(q.H, q.W, q.B, p, pitch, bstride, bands, phis, states + i,
                                   cand, ctx->sm_count, &g.e, g.maps, &tiles)) {
                set_err(ctx, "lse_evolve_batch: image %d: no tensor maps for its bands", i);
                return LSE_ERR_INVALID_ARG;
            }
            mb_index[i] = (int)mb_items.size();
            mb_items.push_back(g);
            mb_tiles[i] = g.e.a.n_items;
            mb_work[i] = (long long)g.e.a.n_items * p.iterations;
            mb_groups[{q.B, g.e.a.rad}].push_back(i);
            continue;
        }
        classes[class_of(plan, p.term, region ? q.B : 1)].items.push_back(i);
    }
    // the vector images' group launches: CTA shares and tables, uploaded once
    std::vector<MbChunk> chunks;
    for (auto &kg : mb_groups) {
        const int cap = evolve_mb_group_capacity(kg.first.first, kg.first.second, ctx->sm_count);
        if (cap < 1) {
            set_err(ctx, "lse_evolve_batch: the vector-image evolution cannot be resident");
            return LSE_ERR_CUDA;
        }
        share_ctas(kg.second, mb_tiles, mb_work, cap, kg.first.first, kg.first.second, &chunks);
    }
    std::vector<size_t> chunk_items_off, chunk_table_off;
    size_t mb_bytes = 0;
    for (auto &c : chunks) {
        chunk_items_off.push_back(mb_bytes);
        mb_bytes = align_up(mb_bytes + sizeof(MbGroupItem) * c.images.size());
        chunk_table_off.push_back(mb_bytes);
        mb_bytes = align_up(mb_bytes + sizeof(int) * (size_t)c.total);
    }
    std::vector<unsigned char> mb_host(mb_bytes);
    for (size_t ci = 0; ci < chunks.size(); ++ci) {
        MbChunk &c = chunks[ci];
        MbGroupItem *gi = reinterpret_cast<MbGroupItem *>(mb_host.data() + chunk_items_off[ci]);
        int *tab = reinterpret_cast<int *>(mb_host.data() + chunk_table_off[ci]);
        int cta = 0;
        for (size_t k = 0; k < c.images.size(); ++k) {
            MbGroupItem g = mb_items[mb_index[c.images[k]]];
            g.cta0 = cta;
            g.ncta = c.ncta[k];
            memcpy(gi + k, &g, sizeof(g));
            for (int j = 0; j < c.ncta[k]; ++j) tab[cta++] = (int)k;
        }
    }
    if (mb_bytes) {
        void *mp = ctx->mbgroup;
        if ((r = ensure(ctx, &mp, &ctx->mbgroup_cap, mb_bytes, s, "vector-image groups")) != LSE_OK)
            return r;
        ctx->mbgroup = mp;
        e = cudaMemcpyAsync(ctx->mbgroup, mb_host.data(), mb_bytes, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "lse_evolve_batch: upload groups");
        e = cudaStreamSynchronize(s);       // the pageable source goes out of scope
        if (e != cudaSuccess) return cuda_fail(ctx, e, "lse_evolve_batch: upload groups");
    }
    auto launch_groups = [&]() -> cudaError_t {
        const unsigned char *base_d = static_cast<const unsigned char *>(ctx->mbgroup);
        for (size_t ci = 0; ci < chunks.size(); ++ci) {
            cudaError_t ge = launch_evolve_bands_group(
                chunks[ci].B, chunks[ci].rad,
                reinterpret_cast<const MbGroupItem *>(base_d + chunk_items_off[ci]),
                reinterpret_cast<const int *>(base_d + chunk_table_off[ci]), chunks[ci].total, s);
            if (ge != cudaSuccess) return ge;
        }
        return cudaSuccess;
    };

    // ---- CTA tables and the work list, uploaded once
    const size_t toff = layout_classes(classes, items.data());
    if ((r = ensure(ctx, &ctx->tables, &ctx->tables_cap, toff, s, "batch tables")) != LSE_OK)
        return r;
    const size_t hbytes = align_up(sizeof(BatchItem) * n) + toff + sizeof(LseDevState) * n;
    if ((r = ensure_host(ctx, hbytes, s)) != LSE_OK) return r;
    unsigned char *Hh = static_cast<unsigned char *>(ctx->bhost);
    unsigned char *ht = Hh + align_up(sizeof(BatchItem) * n);
    fill_tables(classes, items.data(), ht);
    memcpy(Hh, items.data(), sizeof(BatchItem) * n);
    e = cudaMemcpyAsync(d_items, Hh, sizeof(BatchItem) * n, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && toff)
        e = cudaMemcpyAsync(ctx->tables, ht, toff, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "lse_evolve_batch: upload work list");
    const unsigned char *tables = static_cast<const unsigned char *>(ctx->tables);

    // ---- the iteration loop: one launch per class and iteration
    int maxcap = 0;
    for (int i = 0; i < n; ++i) maxcap = std::max(maxcap, problems[i].params.iterations);
    auto enqueue_loop = [&](cudaStream_t q) -> cudaError_t {
        for (int it = 0; it < maxcap; ++it)
            for (auto &kc : classes) {
                cudaError_t le = launch_class(kc.first, kc.second, d_items, tables, it, q,
                                              kc.second.active(it));
                if (le != cudaSuccess) return le;
            }
        return cudaSuccess;
    };
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    if (use_graph && !classes.empty()) {
        // kernel attributes are set by one launch per class in which every
        // image is past its cap (its CTAs return at once), outside the capture
        for (auto &kc : classes) {
            e = launch_class(kc.first, kc.second, d_items, tables, maxcap, s);
            if (e != cudaSuccess) return cuda_fail(ctx, e, "lse_evolve_batch: prepare");
        }
        // capture on the context's own stream (the caller's may be the legacy
        // default stream, which cannot be captured); the graph runs on `s`
        if (!ctx->cap_stream) {
            e = cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking);
            if (e != cudaSuccess) return cuda_fail(ctx, e, "lse_evolve_batch: capture stream");
        }
        cudaStream_t cs = ctx->cap_stream;
        e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaError_t le = enqueue_loop(cs);
            e = cudaStreamEndCapture(cs, &graph);
            if (le != cudaSuccess) e = le;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
        if (e != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return cuda_fail(ctx, e, "lse_evolve_batch: capture");
        }
    }
    e = cudaEventRecord(ctx->ev0, s);
    if (e == cudaSuccess) e = launch_groups();
    if (e == cudaSuccess && !classes.empty())
        e = use_graph ? cudaGraphLaunch(exec, s) : enqueue_loop(s);
    if (e == cudaSuccess) e = cudaEventRecord(ctx->ev1, s);
    if (e != cudaSuccess) {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        return cuda_fail(ctx, e, "lse_evolve_batch: iterations");
    }

    // ---- outputs and statistics (vector images on the band passes first
    // take the statistics of their returned LSF)
    for (int i = 0; i < n && e == cudaSuccess; ++i) {
        const lse_problem &q = problems[i];
        const StepArgs &a = items[i].args;
        if (a.mb_split && !mb[i]) {
            e = launch_band_stats(a.bands, a.pitch, a.band_stride, items[i].phi, q.H, q.W, q.B,
                                  a.dt, states + i, a.partials, nred, s);
            if (e != cudaSuccess) break;
        }
        e = launch_output(items[i].phi, lay[i].pitch, q.H, q.W, q.params.storage, states + i,
                          q.phi_out, q.mask_out, s);
    }
    LseDevState *hs = reinterpret_cast<LseDevState *>(ht + toff);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(hs, states, sizeof(LseDevState) * n, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "lse_evolve_batch: outputs");
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1) != cudaSuccess) {
        cudaGetLastError();
        ms = -1.0f;
    }
    if (stats)
        for (int i = 0; i < n; ++i) fill_stats(hs[i], ms, stats + i);
    return LSE_OK;
}

}  // extern "C"
