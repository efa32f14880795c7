// Launch tables: every batched kernel runs one block per Seg, each Seg a
// contiguous range of one instance's work, so instances of different sizes
// share one launch.
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
    const int CH_NODES = 1024, CH_Q = 256, CH_TOUCH = 256, CH_1D = 256, CH_VEC = vec_chunk;
    for (int i = 0; i < (int)insts.size(); ++i) {
        const InstDesc& d = *insts[i];
        a.begin_inst(); a.add(i, 0, d.n3, CH_NODES); a.add(i, 1, d.nq, CH_Q); a.end_inst();
        b.begin_inst(); b.add(i, 2, d.ntouch, CH_TOUCH); b.add(i, 3, d.n1, CH_1D); b.end_inst();
        v.begin_inst(); v.add(i, 0, (int)d.n, CH_VEC); v.end_inst();
        n3.begin_inst(); n3.add(i, 0, d.n3, CH_VEC); n3.end_inst();
        tch.begin_inst(); tch.add(i, 0, d.ntouch, CH_TOUCH); tch.end_inst();
    }
    MD_TRY(upload(a, &T->apply_a, allocs));
    MD_TRY(upload(b, &T->apply_b, allocs));
    MD_TRY(upload(v, &T->vec, allocs));
    MD_TRY(upload(n3, &T->n3, allocs));
    MD_TRY(upload(tch, &T->touch, allocs));
    return MD_OK;
}

void dev_free_all(std::vector<void*>* allocs) {
    for (void* p : *allocs) cudaFree(p);
    allocs->clear();
}
