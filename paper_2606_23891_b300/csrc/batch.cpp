// Host builder of the batched (cell-dedup) offload pipeline.
//
// The batched pipeline runs the same cell-pair interactions as the per-task
// cycle (Sec. 2.3: ready tasks fused into bundles), but a bundle is a range
// of *target cells*: every cell the range needs (targets plus their 26
// periodic neighbours) is packed once into the bundle buffer, and one
// persistent launch computes, for every target particle, its sums over all
// 27 neighbour cells.  Work items are (target cell, 32-particle chunk) pairs,
// one per warp, in decreasing classes of estimated cost (a coarse
// longest-first order, so uneven cells balance over the persistent warps)
// and in cell order inside a class.
#include <algorithm>
#include <numeric>

#include "internal.h"

namespace sph {

int build_batch(const sph_tasks_s *T, const sph_batch_params *bp, sph_batch_s *B) {
    if (!T || !bp) return fail(SPH_EINVAL, "batch_build: bad arguments");
    const int threads = bp->threads;
    if (threads != 64 && threads != 128 && threads != 256)
        return fail(SPH_EINVAL, "batch_build: threads must be 64, 128 or 256");
    const int64_t ichunk = 32;  // one work item per warp
    const int32_t *nc = T->ncell;
    const int64_t ncells = (int64_t)nc[0] * nc[1] * nc[2];
    auto count = [&](int64_t c) { return T->cell_start[c + 1] - T->cell_start[c]; };
    B->threads = threads;
    B->n = T->n;
    for (int d = 0; d < 3; ++d) B->box[d] = T->box[d];

    // targets: non-empty cells in index order, split into bundles
    std::vector<int64_t> targets;
    for (int64_t c = 0; c < ncells; ++c)
        if (count(c) > 0) targets.push_back(c);
    const int64_t per = bp->max_target_cells > 0 ? bp->max_target_cells
                                                 : (int64_t)targets.size();
    B->bundles.clear();
    std::vector<int32_t> local((size_t)ncells, -1);
    for (size_t t0 = 0; t0 < targets.size(); t0 += (size_t)per) {
        const size_t t1 = std::min(targets.size(), t0 + (size_t)per);
        BatchBundle bb;
        // cells needed: targets and their 26 periodic neighbours
        std::vector<int64_t> need;
        std::vector<std::array<int32_t, 27>> nbr_cell(t1 - t0);
        std::vector<std::array<int32_t, 27>> nbr_shift(t1 - t0);
        for (size_t k = t0; k < t1; ++k) {
            const int64_t c = targets[k];
            const int64_t ix = c % nc[0], iy = (c / nc[0]) % nc[1],
                          iz = c / ((int64_t)nc[0] * nc[1]);
            int e = 0;
            for (int dz = -1; dz <= 1; ++dz)
                for (int dy = -1; dy <= 1; ++dy)
                    for (int dx = -1; dx <= 1; ++dx, ++e) {
                        int64_t q[3] = {ix + dx, iy + dy, iz + dz};
                        int code = 0;
                        for (int d = 0; d < 3; ++d) {
                            int s = 0;
                            if (q[d] < 0) { q[d] += nc[d]; s = -1; }
                            if (q[d] >= nc[d]) { q[d] -= nc[d]; s = 1; }
                            code |= (s + 1) << (2 * d);
                        }
                        const int64_t c2 = q[0] + nc[0] * (q[1] + nc[1] * q[2]);
                        nbr_cell[k - t0][e] = (int32_t)c2;
                        nbr_shift[k - t0][e] = code;
                        if (count(c2) > 0) need.push_back(c2);
                    }
        }
        std::sort(need.begin(), need.end());
        need.erase(std::unique(need.begin(), need.end()), need.end());
        bb.cell0 = (int64_t)B->cells.size();
        int64_t slot = 0;
        for (int64_t c : need) {
            local[c] = (int32_t)(B->cells.size() - bb.cell0);
            BCellDev cd;
            cd.p0 = (int32_t)T->cell_start[c];
            cd.n = (int32_t)count(c);
            cd.slot = (int32_t)slot;
            cd.pad = 0;
            B->cells.push_back(cd);
            slot += count(c);
        }
        if (slot > INT32_MAX) return fail(SPH_EUNSUPPORTED, "batch bundle exceeds 2^31-1 slots");
        bb.ncells = (int64_t)need.size();
        bb.slots = slot;
        // targets of the bundle with their neighbour tables (local indices)
        bb.target0 = (int64_t)B->targets.size();
        for (size_t k = t0; k < t1; ++k) {
            BTargetDev td;
            td.cell = local[targets[k]];
            for (int e = 0; e < 27; ++e) {
                const int32_t c2 = nbr_cell[k - t0][e];
                td.nbr[e] = count(c2) > 0 ? local[c2] : -1;
                td.shift[e] = (uint8_t)nbr_shift[k - t0][e];
            }
            B->targets.push_back(td);
        }
        bb.ntargets = (int64_t)(t1 - t0);
        // work items: larger cost classes (log2 of the estimated candidate
        // count) first, cell order inside a class (keeps neighbour cells of
        // concurrently processed items close in L2)
        std::vector<std::pair<int64_t, BItemDev>> items;
        for (size_t k = t0; k < t1; ++k) {
            const int64_t c = targets[k];
            int64_t around = 0;
            for (int e = 0; e < 27; ++e) around += count(nbr_cell[k - t0][e]);
            for (int64_t i0 = 0; i0 < count(c); i0 += ichunk) {
                const int64_t len = std::min<int64_t>(ichunk, count(c) - i0);
                BItemDev it;
                it.target = (int32_t)(k - t0);
                it.i0 = (int32_t)i0;
                int64_t cost = len * around, cls = 0;
                while (cost > 1) { cost >>= 1; ++cls; }
                items.push_back({cls, it});
            }
        }
        std::stable_sort(items.begin(), items.end(),
                         [](const std::pair<int64_t, BItemDev> &a,
                            const std::pair<int64_t, BItemDev> &b2) { return a.first > b2.first; });
        bb.item0 = (int64_t)B->items.size();
        for (auto &it : items) B->items.push_back(it.second);
        bb.nitems = (int64_t)items.size();
        for (int64_t c : need) local[c] = -1;
        B->bundles.push_back(bb);
    }
    B->max_slots = 0;
    B->max_targets = 0;
    for (const BatchBundle &bb : B->bundles) {
        B->max_slots = std::max(B->max_slots, bb.slots);
        int64_t tslots = 0;
        for (int64_t k = 0; k < bb.ntargets; ++k)
            tslots += B->cells[bb.cell0 + B->targets[bb.target0 + k].cell].n;
        B->max_targets = std::max(B->max_targets, tslots);
    }
    return SPH_OK;
}

}  // namespace sph
