// lse_classes.h -- grouping of batched images into launch classes (host,
// internal; shared by lse_evolve_batch and lse_server).
//
// A class is the set of images served by one step kernel instantiation
// (form, term, bands, radius, warps per CTA, storage type, tile height).  Its images are laid out
// longest-running first, so launch t needs only the CTAs of the images that
// are still running: a prefix of the class's CTA table.
#pragma once

#include <map>
#include <tuple>
#include <vector>

#include "lse_internal.h"

namespace lse_detail {

struct ClassKey {
    int form, term, bands, rad, wpc, storage, nw;
    bool operator<(const ClassKey &o) const
    {
        return std::tie(form, term, bands, rad, wpc, storage, nw) <
               std::tie(o.form, o.term, o.bands, o.rad, o.wpc, o.storage, o.nw);
    }
};

// Planes of one image in a batch arena or a server slot, as byte offsets
// from the image's base: the data term (`bands` planes: the image bands, or
// g), then the two LSF planes, then for a vector image the D plane of its
// band passes; each plane is H x pitch elements of the storage type (4 or 2
// bytes) and starts on 256 bytes.
struct ImagePlanes {
    int pitch;
    int es;                        // bytes per element
    size_t data, phi0, phi1, end;
    size_t dplane;                 // vector images: the D plane (0: none)
};
ImagePlanes image_planes(const lse_problem &q);

// Stages image q at `base` as lse_evolve would (the data term converted to
// FP32, or rounded to the 16-bit storage type through an FP32 copy held in
// the LSF planes), runs its prologue into st / parts with `nred` CTAs, and
// plans its step.  Returns the first CUDA error; *planned is false when no
// batched step kernel serves the image.
cudaError_t stage_problem(const lse_problem &q, unsigned char *base, const ImagePlanes &L,
                          LseDevState *st, LsePartial *parts, int nred, int sm_count,
                          int form, int tile_nw, StepPlan *plan, bool *planned,
                          cudaStream_t s);

struct Class {
    std::vector<int> items;        // indices into the item array
    std::vector<long long> ends;   // iter0 + cap of `items`, descending
    std::vector<int> pre, npre;    // CTAs of items[0..k): step, normaliser
    int nblocks = 0;
    int nnblocks = 0;
    size_t blk_off = 0, nblk_off = 0;   // byte offsets of the CTA tables

    // images still running at launch index t (a prefix of `items`)
    int active(long long t) const
    {
        int k = 0;
        while (k < (int)ends.size() && ends[k] > t) ++k;
        return k;
    }
};

using ClassMap = std::map<ClassKey, Class>;

// The class of an image from its step plan.
ClassKey class_of(const StepPlan &plan, int term, int bands);
// Orders each class's images by end, assigns their CTA ranges (start,
// nstart) and returns the bytes of all CTA tables.
size_t layout_classes(ClassMap &classes, BatchItem *items);
// Writes the CTA tables (image index per CTA) at host_tables.
void fill_tables(const ClassMap &classes, const BatchItem *items, unsigned char *host_tables);
// Launch index t of class c over its first k_act images (all when < 0).
cudaError_t launch_class(const ClassKey &k, const Class &c, const BatchItem *d_items,
                         const unsigned char *d_tables, long long t, cudaStream_t s,
                         int k_act = -1);
// CTAs the normaliser of an image of H rows runs with (as lse_evolve).
int normaliser_blocks(int H, int sm_count);

}  // namespace lse_detail
