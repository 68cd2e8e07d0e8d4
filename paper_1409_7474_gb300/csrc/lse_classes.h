// lse_classes.h -- grouping of batched images into launch classes (host,
// internal; shared by lse_evolve_batch and lse_server).
//
// A class is the set of images served by one step kernel instantiation
// (form, term, bands, radius, warps per CTA).  Its images are laid out
// longest-running first, so launch t needs only the CTAs of the images that
// are still running: a prefix of the class's CTA table.
#pragma once

#include <map>
#include <tuple>
#include <vector>

#include "lse_internal.h"

namespace lse_detail {

struct ClassKey {
    int form, term, bands, rad, wpc;
    bool operator<(const ClassKey &o) const
    {
        return std::tie(form, term, bands, rad, wpc) <
               std::tie(o.form, o.term, o.bands, o.rad, o.wpc);
    }
};

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
// CTAs the normaliser of an image of `npix` pixels runs with (as lse_evolve).
int normaliser_blocks(long long npix, int sm_count);

}  // namespace lse_detail
