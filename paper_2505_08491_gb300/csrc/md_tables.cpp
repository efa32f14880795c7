// Launch tables: every batched kernel runs one block per Seg, each Seg a
// contiguous range of one instance's work (for the stencil, one tile), so
// instances of different sizes share one launch.
#include <algorithm>

#include "md_internal.h"

namespace {

struct Builder {
    std::vector<Seg> segs;
    std::vector<InstRange> ranges;
    void begin_inst() { ranges.push_back({(int)segs.size(), 0}); }
    void add(int inst, int kind, int n, int chunk) {
        for (int b = 0; b < n; b += chunk) segs.push_back({inst, kind, b, std::min(n, b + chunk)});
    }
    void end_inst() { ranges.back().count = (int)segs.size() - ranges.back().first; }
};

md_status upload(const Builder& B, Table* T, std::vector<void*>* allocs) {
    T->nblocks = (int)B.segs.size();
    T->hrange = B.ranges;
    MD_TRY(dev_upload(allocs, &T->seg, B.segs.data(), B.segs.size()));
    MD_TRY(dev_upload(allocs, &T->range, B.ranges.data(), B.ranges.size()));
    return MD_OK;
}

}  // namespace

md_status build_tables(const std::vector<const InstDesc*>& insts, Tables* T, std::vector<void*>* allocs, int vec_chunk) {
    Builder a, b, v, n3, tch;
    const int CH_Q = 256, CH_TOUCH = 256, CH_1D = 256, CH_VEC = vec_chunk;
    int sm32 = 0, sm64 = 0;
    for (int i = 0; i < (int)insts.size(); ++i) {
        const InstDesc& d = *insts[i];
        a.begin_inst(); a.add(i, 1, d.nq, CH_Q); a.end_inst();
        // one block per stencil tile, then the 1D rows
        b.begin_inst(); b.add(i, 4, d.ntiles, 1); b.add(i, 3, d.n1, CH_1D); b.end_inst();
        sm32 = std::max(sm32, apply_tile_smem(d.N, d.ty, d.tz, 4));
        sm64 = std::max(sm64, apply_tile_smem(d.N, d.ty, d.tz, 8));
        v.begin_inst(); v.add(i, 0, (int)d.n, CH_VEC); v.end_inst();
        n3.begin_inst(); n3.add(i, 0, d.n3, CH_VEC); n3.end_inst();
        tch.begin_inst(); tch.add(i, 0, d.ntouch, CH_TOUCH); tch.end_inst();
    }
    MD_TRY(upload(a, &T->apply_a, allocs));
    MD_TRY(upload(b, &T->apply_b, allocs));
    T->apply_b.smem32 = sm32;
    T->apply_b.smem64 = sm64;
    MD_TRY(apply_prepare(sm32, sm64));
    MD_TRY(upload(v, &T->vec, allocs));
    MD_TRY(upload(n3, &T->n3, allocs));
    MD_TRY(upload(tch, &T->touch, allocs));
    return MD_OK;
}

void dev_free_all(std::vector<void*>* allocs) {
    for (void* p : *allocs) cudaFree(p);
    allocs->clear();
}

void apply_tile_shape(int N, int* ty, int* tz) {
    const int M = N + 1;
    int t = M >= 256 ? 1 : 256 / M;  // one column per thread of a 256-thread block
    if (t > 8) t = 8;
    int z = 8;
    while (z > 1 && apply_tile_smem(N, t, z, 8) > 64 * 1024) z /= 2;
    *ty = t;
    *tz = z;
}

// input tile with a one-node halo in y and z (x is whole), output tile
int apply_tile_smem(int N, int ty, int tz, int elem_bytes) {
    const int M = N + 1;
    return ((tz + 2) * (ty + 2) * M + tz * ty * M) * elem_bytes;
}
