// lse_serve.cu -- lse_server: continuous batching of evolution requests.
//
// Requests (lse_problem) are queued on submission and admitted, first come
// first served, into free slots while their planes fit the server's HBM
// budget.  An admitted request is staged and its prologue run at the current
// launch index t0; from then on every lse_server_advance call runs its next
// iterations inside the same batched launches as all other running requests
// (its iteration n at launch index t0 + n).  A request retires when it
// reaches its cap or stops early: its output is written, its statistics
// kept for lse_server_poll, and its memory returned.  Each request keeps the
// CTA count, statistics and reductions lse_evolve would give it alone, so
// its result does not depend on what else is running.  Vector images and
// large images never join the mix: each runs to its end inside one advance
// through lse_evolve's own path -- a large image alone, the oldest first, one
// per advance; the queued small vector images together, in one
// lse_evolve_batch whose group launch gives each its own CTAs (lse_evolve's
// bits).  Under
// light load (the mix empty, a few requests waiting) every request runs
// alone, one per advance, in arrival order.  For one band and the edge term
// lse_evolve's persistent launch gives the bits the mix gives.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <deque>
#include <iterator>
#include <map>
#include <vector>

#include "lse_classes.h"
#include "lse_ctx.h"

using namespace lse_detail;

namespace {

constexpr int kMaxSlots = 1024;
// Requests that run alone rather than in the mix: vector images of the
// region term, whose own path is one persistent launch that stages the
// bands itself (the mix takes three launches per iteration for them), and
// images of at least this many pixels, whose tiles fill the GPU by
// themselves (more than twice its SM count of 64-row tiles), so that the
// mix's per-iteration launches would only add their overhead.
constexpr long long kSoloPixels = 1ll << 21;
// At most this many requests waiting and none in the mix: light load, one
// request at a time, alone.
constexpr size_t kLightQueue = 4;
// At most this many queued vector images (each below kSoloPixels) run
// together in one advance.
constexpr int kVectorGroup = 32;
constexpr size_t kAlign = 256;

size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

// First-fit allocator over the byte range [0, size) of the server's arena,
// with coalescing of neighbouring free blocks.
class FreeList {
  public:
    void reset(size_t size)
    {
        free_.clear();
        if (size) free_[0] = size;
    }
    bool take(size_t bytes, size_t *off)
    {
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < bytes) continue;
            *off = it->first;
            const size_t rest = it->second - bytes, noff = it->first + bytes;
            free_.erase(it);
            if (rest) free_[noff] = rest;
            return true;
        }
        return false;
    }
    void give(size_t off, size_t bytes)
    {
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }

  private:
    std::map<size_t, size_t> free_;
};

enum { REQ_QUEUED = 0, REQ_RUNNING = 1, REQ_DONE = 2 };

struct Request {
    lse_problem q;
    int state = REQ_QUEUED;
    int slot = -1;
    size_t off = 0, bytes = 0;
    int pitch = 0;
    ClassKey key{};
    lse_stats stats{};
    bool solo = false;          // runs alone, through lse_evolve (see kSoloPixels)
};

// Bytes of one request's planes (of its storage type) and partials in the
// arena.
size_t request_bytes(const lse_problem &q, int nparts)
{
    return image_planes(q).end + align_up(sizeof(LsePartial) * (size_t)nparts);
}

}  // namespace

struct lse_server {
    lse_ctx *ctx = nullptr;
    size_t budget = 0;
    unsigned char *arena = nullptr;          // device, `budget` bytes
    FreeList alloc;
    int nparts = 0;
    BatchItem *d_items = nullptr;            // kMaxSlots
    LseDevState *d_states = nullptr;         // kMaxSlots
    std::vector<BatchItem> items;            // host mirror
    std::vector<long long> slot_req;         // request per slot, 0 = free
    void *d_tables = nullptr;
    size_t tables_cap = 0;
    unsigned char *h_buf = nullptr;          // pinned: items, tables, states
    size_t h_cap = 0;
    std::deque<long long> queue;
    std::map<long long, Request> reqs;
    long long next_id = 1;
    long long tick = 0;
    int running = 0;
};

namespace {

lse_status grow_host(lse_server *sv, size_t bytes, cudaStream_t s)
{
    if (sv->h_cap >= bytes) return LSE_OK;
    if (sv->h_buf) {
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(sv->ctx, e, "lse_server: synchronise");
        cudaFreeHost(sv->h_buf);
        sv->h_buf = nullptr;
        sv->h_cap = 0;
    }
    if (cudaMallocHost(reinterpret_cast<void **>(&sv->h_buf), bytes) != cudaSuccess) {
        cudaGetLastError();
        sv->h_buf = nullptr;
        set_err(sv->ctx, "lse_server: cudaMallocHost of %zu bytes failed", bytes);
        return LSE_ERR_OOM;
    }
    sv->h_cap = bytes;
    return LSE_OK;
}

// Stages request r into slot `slot` at arena offset r.off and runs its
// prologue; fills the slot's work item.
lse_status admit(lse_server *sv, Request &r, int slot, cudaStream_t s)
{
    lse_ctx *ctx = sv->ctx;
    const lse_problem &q = r.q;
    const lse_params &p = q.params;
    const bool region = p.term == LSE_TERM_REGION;
    const int bands = region ? q.B : 1;
    const ImagePlanes L = image_planes(q);
    unsigned char *base = sv->arena + r.off;
    LsePartial *parts = reinterpret_cast<LsePartial *>(base + L.end);
    LseDevState *st = sv->d_states + slot;
    StepPlan plan;
    bool planned = false;
    cudaError_t e = cudaMemsetAsync(st, 0, sizeof(LseDevState), s);
    if (e == cudaSuccess)
        e = stage_problem(q, base, L, st, parts, ctx->sm_count * 4, ctx->sm_count, LSE_FORM_AUTO,
                          tile_nw_for(ctx, q.H, q.W, q.B, p.term, p.storage, p.ts), &plan, &planned,
                          s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "lse_server: admit");
    if (!planned) {
        set_err(ctx, "lse_server: no batched step kernel serves request %dx%dx%d", q.H, q.W, q.B);
        return LSE_ERR_INVALID_ARG;
    }
    BatchItem &it = sv->items[slot];
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
    it.iter0 = sv->tick;
    if (region && q.B > 1) it.nnblocks = normaliser_blocks(q.H, ctx->sm_count);
    r.key = class_of(plan, p.term, bands);
    r.pitch = L.pitch;
    r.slot = slot;
    r.state = REQ_RUNNING;
    return LSE_OK;
}

}  // namespace

extern "C" {

lse_status lse_server_create(lse_ctx *ctx, size_t budget_bytes, lse_server **out)
{
    if (!out) return LSE_ERR_INVALID_ARG;
    *out = nullptr;
    if (!ctx) return LSE_ERR_INVALID_ARG;
    ctx->err[0] = 0;
    if (budget_bytes < ((size_t)1 << 20)) {
        set_err(ctx, "lse_server_create: the budget must be at least 1 MiB");
        return LSE_ERR_INVALID_ARG;
    }
    DeviceGuard guard(ctx->device);
    if (!guard.ok) return cuda_fail(ctx, cudaErrorInvalidDevice, "set device");
    lse_server *sv = new lse_server();
    sv->ctx = ctx;
    sv->budget = budget_bytes / kAlign * kAlign;
    sv->nparts = partials_needed(ctx->sm_count);
    sv->items.assign(kMaxSlots, BatchItem{});
    sv->slot_req.assign(kMaxSlots, 0);
    cudaError_t e = cudaMalloc(reinterpret_cast<void **>(&sv->arena), sv->budget);
    if (e == cudaSuccess) e = cudaMalloc(&sv->d_items, sizeof(BatchItem) * kMaxSlots);
    if (e == cudaSuccess) e = cudaMalloc(&sv->d_states, sizeof(LseDevState) * kMaxSlots);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_err(ctx, "lse_server_create: cannot allocate %zu bytes", sv->budget);
        lse_server_destroy(sv);
        return LSE_ERR_OOM;
    }
    sv->alloc.reset(sv->budget);
    *out = sv;
    return LSE_OK;
}

void lse_server_destroy(lse_server *sv)
{
    if (!sv) return;
    DeviceGuard guard(sv->ctx->device);
    cudaDeviceSynchronize();
    if (sv->arena) cudaFree(sv->arena);
    if (sv->d_items) cudaFree(sv->d_items);
    if (sv->d_states) cudaFree(sv->d_states);
    if (sv->d_tables) cudaFree(sv->d_tables);
    if (sv->h_buf) cudaFreeHost(sv->h_buf);
    delete sv;
}

lse_status lse_server_submit(lse_server *sv, const lse_problem *problem, long long *id)
{
    if (!sv || !problem || !id) return LSE_ERR_INVALID_ARG;
    lse_ctx *ctx = sv->ctx;
    ctx->err[0] = 0;
    const lse_problem &q = *problem;
    const bool region = q.params.term == LSE_TERM_REGION;
    lse_status r;
    if (q.H < 1 || q.W < 1 || q.B < 1 || q.B > LSE_MAXB) {
        set_err(ctx, "lse_server_submit: need H, W >= 1 and 1 <= B <= %d", LSE_MAXB);
        return LSE_ERR_INVALID_ARG;
    }
    if ((r = check_params(ctx, q.params, q.B)) != LSE_OK) return r;
    if (q.params.ts > 15 || (region && q.B > 4) || q.params.order != LSE_ORDER_LISTING ||
        q.params.padding != LSE_PAD_ZERO) {
        set_err(ctx, "lse_server_submit: the server runs ts <= 15, at most 4 bands, the "
                     "listing's order and zero padding");
        return LSE_ERR_INVALID_ARG;
    }
    {
        DeviceGuard guard(ctx->device);
        const bool ok = classify(q.phi0, ctx->device) == PTR_DEVICE &&
                        classify(q.phi_out, ctx->device) == PTR_DEVICE &&
                        (!q.mask_out || classify(q.mask_out, ctx->device) == PTR_DEVICE) &&
                        (region ? (classify(q.image, ctx->device) == PTR_DEVICE && !q.g)
                                : classify(q.g, ctx->device) == PTR_DEVICE);
        if (!ok) {
            set_err(ctx, "lse_server_submit: image (region) or g (edge), phi0, phi_out and "
                         "mask_out must be device memory of the context's GPU");
            return LSE_ERR_INVALID_ARG;
        }
    }
    if (request_bytes(q, sv->nparts) > sv->budget) {
        set_err(ctx, "lse_server_submit: the request needs %zu bytes, more than the budget",
                request_bytes(q, sv->nparts));
        return LSE_ERR_INVALID_ARG;
    }
    const long long rid = sv->next_id++;
    Request &req = sv->reqs[rid];
    req.q = q;
    // (lse_evolve needs the image to fit the context)
    req.solo = ((region && q.B > 1) || (long long)q.H * q.W >= kSoloPixels) &&
               (size_t)q.H * q.W <= ctx->max_pixels && q.B <= ctx->max_bands;
    sv->queue.push_back(rid);
    *id = rid;
    return LSE_OK;
}

lse_status lse_server_advance(lse_server *sv, int ticks, int *running, void *stream)
{
    if (!sv || ticks < 0) return LSE_ERR_INVALID_ARG;
    lse_ctx *ctx = sv->ctx;
    ctx->err[0] = 0;
    DeviceGuard guard(ctx->device);
    if (!guard.ok) return cuda_fail(ctx, cudaErrorInvalidDevice, "set device");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    lse_status r;

    // ---- one request alone, to its end, through lse_evolve's own path (one
    // persistent launch; for one band and the edge term the same bits as
    // the mix's launches give it).  Light load (the mix empty, at most
    // kLightQueue requests waiting): the oldest request, and nothing else
    // this advance -- a direct call per request in arrival order, which is
    // the fastest way through when requests rarely overlap.  Otherwise the
    // oldest request that always runs alone, beside the mix.
    if (ticks > 0) {
        auto pick = sv->queue.end();
        bool light = false;
        if (sv->running == 0 && !sv->queue.empty() && sv->queue.size() <= kLightQueue) {
            const lse_problem &q = sv->reqs[sv->queue.front()].q;
            if ((size_t)q.H * q.W <= ctx->max_pixels && q.B <= ctx->max_bands) {
                pick = sv->queue.begin();
                light = true;
            }
        }
        if (!light) {
            // the queued vector images together: one lse_evolve_batch, whose
            // group launches step each on its own CTAs (lse_evolve's bits),
            // so small ones no longer hold the whole GPU each
            std::vector<long long> vec;
            for (long long id : sv->queue) {
                const Request &rq = sv->reqs[id];
                // the small ones: a large vector image fills the GPU alone
                if (rq.solo && rq.q.params.term == LSE_TERM_REGION && rq.q.B > 1 &&
                    (long long)rq.q.H * rq.q.W < kSoloPixels)
                    vec.push_back(id);
                if ((int)vec.size() == kVectorGroup) break;
            }
            if (vec.size() > 1) {
                std::vector<lse_problem> probs;
                for (long long id : vec) probs.push_back(sv->reqs[id].q);
                std::vector<lse_stats> sts(vec.size());
                r = lse_evolve_batch(ctx, (int)probs.size(), probs.data(), 0, sts.data(),
                                     stream);
                if (r != LSE_OK) return r;
                for (size_t k = 0; k < vec.size(); ++k) {
                    Request &rq = sv->reqs[vec[k]];
                    sts[k].elapsed_ms = -1.0f;
                    rq.stats = sts[k];
                    rq.state = REQ_DONE;
                    sv->queue.erase(std::find(sv->queue.begin(), sv->queue.end(), vec[k]));
                }
            }
        }
        // (the erasures above invalidated the queue's iterators)
        if (!light)
            pick = std::find_if(sv->queue.begin(), sv->queue.end(),
                                [&](long long id) { return sv->reqs[id].solo; });
        if (pick != sv->queue.end()) {
            Request &req = sv->reqs[*pick];
            const lse_problem &q = req.q;
            lse_stats st;
            r = lse_evolve(ctx, q.params.term == LSE_TERM_REGION ? q.image : nullptr, q.dtype,
                           q.H, q.W, q.B, q.g, q.phi0, &q.params, q.phi_out, q.mask_out, &st,
                           stream);
            if (r != LSE_OK) return r;
            st.elapsed_ms = -1.0f;
            req.stats = st;
            req.state = REQ_DONE;
            sv->queue.erase(pick);
            if (light) {
                if (running) *running = 0;
                return LSE_OK;
            }
        }
    }

    // ---- admission into the mix, first come first served, while the budget
    // allows (requests that run alone wait for their turn above)
    for (auto qi = sv->queue.begin(); qi != sv->queue.end() && sv->running < kMaxSlots;) {
        Request &req = sv->reqs[*qi];
        if (req.solo) {
            ++qi;
            continue;
        }
        const size_t bytes = request_bytes(req.q, sv->nparts);
        size_t off = 0;
        if (!sv->alloc.take(bytes, &off)) break;
        int slot = 0;
        while (sv->slot_req[slot]) ++slot;
        req.off = off;
        req.bytes = bytes;
        if ((r = admit(sv, req, slot, s)) != LSE_OK) {
            sv->alloc.give(off, bytes);
            return r;
        }
        sv->slot_req[slot] = *qi;
        qi = sv->queue.erase(qi);
        ++sv->running;
    }
    if (running) *running = sv->running;
    if (sv->running == 0 || ticks == 0) return LSE_OK;

    // ---- the launch classes of the running requests, and their tables
    ClassMap classes;
    for (int slot = 0; slot < kMaxSlots; ++slot)
        if (sv->slot_req[slot]) classes[sv->reqs[sv->slot_req[slot]].key].items.push_back(slot);
    const size_t toff = layout_classes(classes, sv->items.data());
    const size_t ibytes = sizeof(BatchItem) * kMaxSlots;
    const size_t sbytes = sizeof(LseDevState) * kMaxSlots;
    if ((r = grow_host(sv, ibytes + toff + sbytes, s)) != LSE_OK) return r;
    if (sv->tables_cap < toff) {
        cudaError_t e = cudaStreamSynchronize(s);
        if (sv->d_tables) cudaFree(sv->d_tables);
        sv->d_tables = nullptr;
        sv->tables_cap = 0;
        if (e == cudaSuccess) e = cudaMalloc(&sv->d_tables, toff);
        if (e != cudaSuccess) {
            cudaGetLastError();
            set_err(ctx, "lse_server: cannot allocate %zu bytes of CTA tables", toff);
            return LSE_ERR_OOM;
        }
        sv->tables_cap = toff;
    }
    memcpy(sv->h_buf, sv->items.data(), ibytes);
    fill_tables(classes, sv->items.data(), sv->h_buf + ibytes);
    cudaError_t e = cudaMemcpyAsync(sv->d_items, sv->h_buf, ibytes, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(sv->d_tables, sv->h_buf + ibytes, toff, cudaMemcpyHostToDevice, s);
    const unsigned char *tables = static_cast<const unsigned char *>(sv->d_tables);

    // ---- `ticks` launch indices over every running request
    for (int k = 0; k < ticks && e == cudaSuccess; ++k) {
        const long long t = sv->tick + k;
        for (auto &kc : classes) {
            e = launch_class(kc.first, kc.second, sv->d_items, tables, t, s,
                             kc.second.active(t));
            if (e != cudaSuccess) break;
        }
    }
    sv->tick += ticks;

    // ---- retire what reached its cap or stopped
    LseDevState *hs = reinterpret_cast<LseDevState *>(sv->h_buf + ibytes + toff);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hs, sv->d_states, sbytes, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "lse_server: advance");
    std::vector<int> retired;
    for (int slot = 0; slot < kMaxSlots && e == cudaSuccess; ++slot) {
        if (!sv->slot_req[slot]) continue;
        const LseDevState &h = hs[slot];
        Request &req = sv->reqs[sv->slot_req[slot]];
        const bool finished = h.done || h.iterations_run >= req.q.params.iterations ||
                              (h.status_bits & LSE_SBIT_ABORT);
        if (!finished) continue;
        const StepArgs &a = sv->items[slot].args;
        if (a.mb_split)
            e = launch_band_stats(a.bands, a.pitch, a.band_stride, sv->items[slot].phi, req.q.H,
                                  req.q.W, req.q.B, a.dt, sv->d_states + slot, a.partials,
                                  ctx->sm_count * 4, s);
        if (e == cudaSuccess)
            e = launch_output(sv->items[slot].phi, req.pitch, req.q.H, req.q.W,
                              req.q.params.storage, sv->d_states + slot, req.q.phi_out,
                              req.q.mask_out, s);
        retired.push_back(slot);
    }
    // the states again: the final statistics passes of vector images ran
    // after the copy above
    if (e == cudaSuccess && !retired.empty())
        e = cudaMemcpyAsync(hs, sv->d_states, sbytes, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "lse_server: retire");
    for (int slot : retired) {
        Request &req = sv->reqs[sv->slot_req[slot]];
        fill_stats(hs[slot], -1.0f, &req.stats);
        req.state = REQ_DONE;
        sv->alloc.give(req.off, req.bytes);
        sv->slot_req[slot] = 0;
        --sv->running;
    }
    if (running) *running = sv->running;
    return LSE_OK;
}

lse_status lse_server_poll(lse_server *sv, long long id, int *state, lse_stats *stats)
{
    if (!sv || !state) return LSE_ERR_INVALID_ARG;
    auto it = sv->reqs.find(id);
    if (it == sv->reqs.end()) {
        set_err(sv->ctx, "lse_server_poll: unknown request %lld", id);
        return LSE_ERR_INVALID_ARG;
    }
    *state = it->second.state;
    if (it->second.state == REQ_DONE) {
        // reported once: the record is dropped after its statistics are read
        if (stats) *stats = it->second.stats;
        sv->reqs.erase(it);
    }
    return LSE_OK;
}

}  // extern "C"
