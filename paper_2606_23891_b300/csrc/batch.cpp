// Host builders of the batched (cell-dedup) offload pipeline.
//
// The batched pipeline runs the same cell-pair interactions as the per-task
// cycle (Sec. 2.3: ready tasks fused into bundles), but a bundle is a range
// of *target cells*: every cell the range needs (targets plus their
// neighbour entries) is packed once into the bundle buffer, and one
// persistent launch computes, for every target particle, its sums over all
// its neighbour entries.  Work items are (target cell, 32-particle chunk)
// pairs, one per warp, in decreasing classes of estimated cost (a coarse
// longest-first order, so uneven cells balance over the persistent warps)
// and in cell order inside a class.
//
// Two plans produce the cells and their neighbour entries:
//  - grid: the uniform cell grid of the task builder, 27 periodic
//    neighbours per cell (empty ones dropped);
//  - tree: leaves of an octree over Morton keys, split while a node holds
//    more than leaf_max particles, with neighbour entries from a pruned walk
//    over bounding boxes and support maxima (clustered particle sets, whose
//    supports span decades, would put millions of particles in a grid cell).
#include <parallel/algorithm>

#include <algorithm>
#include <cmath>
#include <numeric>

#include <omp.h>

#include "internal.h"

namespace sph {

namespace {

// Cells (or leaves) with particles and their neighbour entries, with
// global cell indices.
struct GlobalPlan {
    std::vector<int64_t> p0, cnt;      // store range of each cell
    std::vector<float> hlim;           // largest support the plan holds per cell
    std::vector<int64_t> nb_start;     // CSR over cells
    std::vector<int32_t> nb_cell;
    std::vector<uint8_t> nb_code;
};

// Bundles of target cells, bundle-local cell tables, neighbour entries and
// work items from a global plan.
int assemble(const GlobalPlan &G, const sph_batch_params *bp, sph_batch_s *B) {
    const int64_t ichunk = 32;  // one work item per warp
    const int64_t ncells = (int64_t)G.cnt.size();
    const int64_t per = bp->max_target_cells > 0 ? bp->max_target_cells : ncells;
    B->bundles.clear();
    B->cells.clear();
    B->targets.clear();
    B->items.clear();
    B->nbrs.clear();
    std::vector<int32_t> local((size_t)ncells, -1);
    for (int64_t t0 = 0; t0 < ncells; t0 += per) {
        const int64_t t1 = std::min(ncells, t0 + per);
        BatchBundle bb;
        // cells needed: the targets and their neighbour entries, in index order
        std::vector<int64_t> need;
        for (int64_t t = t0; t < t1; ++t) {
            if (local[t] < 0) { local[t] = 0; need.push_back(t); }
            for (int64_t e = G.nb_start[t]; e < G.nb_start[t + 1]; ++e) {
                const int64_t c = G.nb_cell[e];
                if (local[c] < 0) { local[c] = 0; need.push_back(c); }
            }
        }
        std::sort(need.begin(), need.end());
        bb.cell0 = (int64_t)B->cells.size();
        int64_t slot = 0;
        for (int64_t c : need) {
            local[c] = (int32_t)(B->cells.size() - bb.cell0);
            BCellDev cd;
            cd.p0 = (int32_t)G.p0[c];
            cd.n = (int32_t)G.cnt[c];
            cd.slot = (int32_t)slot;
            // a little above the plan's value: the kernels' H = gamma_K h
            // may round differently from the host's
            cd.hlim = G.hlim.empty() ? INFINITY : G.hlim[c] * (1.f + 1e-6f);
            B->cells.push_back(cd);
            slot += G.cnt[c];
        }
        if (slot > INT32_MAX) return fail(SPH_EUNSUPPORTED, "batch bundle exceeds 2^31-1 slots");
        bb.ncells = (int64_t)need.size();
        bb.slots = slot;
        bb.target0 = (int64_t)B->targets.size();
        for (int64_t t = t0; t < t1; ++t) {
            BTargetDev td;
            td.cell = local[t];
            td.nb0 = (int32_t)B->nbrs.size();
            td.nnb = (int32_t)(G.nb_start[t + 1] - G.nb_start[t]);
            td.pad = 0;
            if ((int64_t)B->nbrs.size() + td.nnb > INT32_MAX)
                return fail(SPH_EUNSUPPORTED, "batch plan exceeds 2^31-1 neighbour entries");
            for (int64_t e = G.nb_start[t]; e < G.nb_start[t + 1]; ++e)
                B->nbrs.push_back(BNbrDev{local[G.nb_cell[e]], (int32_t)G.nb_code[e]});
            B->targets.push_back(td);
        }
        bb.ntargets = t1 - t0;
        // work items: larger cost classes (log2 of the estimated candidate
        // count) first, cell order inside a class (keeps neighbour cells of
        // concurrently processed items close in L2)
        std::vector<std::pair<int64_t, BItemDev>> items;
        for (int64_t t = t0; t < t1; ++t) {
            int64_t around = 0;
            for (int64_t e = G.nb_start[t]; e < G.nb_start[t + 1]; ++e) around += G.cnt[G.nb_cell[e]];
            for (int64_t i0 = 0; i0 < G.cnt[t]; i0 += ichunk) {
                const int64_t len = std::min<int64_t>(ichunk, G.cnt[t] - i0);
                BItemDev it;
                it.target = (int32_t)(t - t0);
                it.i0 = (int32_t)i0;
                int64_t cost = len * around, cls = 0;
                while (cost > 1) { cost >>= 1; ++cls; }
                items.push_back({cls, it});
            }
        }
        std::stable_sort(items.begin(), items.end(),
                         [](const std::pair<int64_t, BItemDev> &a,
                            const std::pair<int64_t, BItemDev> &b2) { return a.first > b2.first; });
        if ((int64_t)items.size() > INT32_MAX)
            return fail(SPH_EUNSUPPORTED, "batch bundle exceeds 2^31-1 work items");
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
    B->plan_cells = ncells;
    B->plan_max_cell = 0;
    for (int64_t c = 0; c < ncells; ++c) B->plan_max_cell = std::max(B->plan_max_cell, G.cnt[c]);
    B->plan_nbrs = (int64_t)G.nb_cell.size();
    return SPH_OK;
}

int check_batch_params(const sph_batch_params *bp) {
    const int threads = bp->threads;
    if (threads != 64 && threads != 128 && threads != 256)
        return fail(SPH_EINVAL, "batch_build: threads must be 64, 128 or 256");
    return SPH_OK;
}

}  // namespace

int build_batch(const sph_tasks_s *T, const sph_batch_params *bp, sph_batch_s *B) {
    if (!T || !bp) return fail(SPH_EINVAL, "batch_build: bad arguments");
    if (int rc = check_batch_params(bp)) return rc;
    const int32_t *nc = T->ncell;
    const int64_t ngrid = (int64_t)nc[0] * nc[1] * nc[2];
    auto count = [&](int64_t c) { return T->cell_start[c + 1] - T->cell_start[c]; };
    B->threads = bp->threads;
    B->n = T->n;
    B->kind = 0;
    for (int d = 0; d < 3; ++d) B->box[d] = T->box[d];
    // cells are at least the largest support, so extent + support <= 2 cells:
    // below half the box when every dimension has 5 or more cells
    B->fixed_build = nc[0] >= 5 && nc[1] >= 5 && nc[2] >= 5;

    // cells with particles, in grid index order; any support up to the
    // shortest cell edge keeps every pair inside adjacent cells
    GlobalPlan G;
    double edge = INFINITY;
    for (int d = 0; d < 3; ++d) edge = std::min(edge, T->box[d] / nc[d]);
    std::vector<int32_t> id((size_t)ngrid, -1);
    for (int64_t c = 0; c < ngrid; ++c)
        if (count(c) > 0) {
            id[c] = (int32_t)G.cnt.size();
            G.p0.push_back(T->cell_start[c]);
            G.cnt.push_back(count(c));
            G.hlim.push_back((float)edge);
        }
    // 27 periodic neighbours in (dz, dy, dx) order, empty cells dropped
    G.nb_start.push_back(0);
    for (int64_t c = 0; c < ngrid; ++c) {
        if (id[c] < 0) continue;
        const int64_t ix = c % nc[0], iy = (c / nc[0]) % nc[1], iz = c / ((int64_t)nc[0] * nc[1]);
        for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    int64_t q[3] = {ix + dx, iy + dy, iz + dz};
                    int code = 0;
                    for (int d = 0; d < 3; ++d) {
                        int s = 0;
                        if (q[d] < 0) { q[d] += nc[d]; s = -1; }
                        if (q[d] >= nc[d]) { q[d] -= nc[d]; s = 1; }
                        code |= (s + 1) << (2 * d);
                    }
                    const int64_t c2 = q[0] + nc[0] * (q[1] + nc[1] * q[2]);
                    if (id[c2] < 0) continue;
                    G.nb_cell.push_back(id[c2]);
                    G.nb_code.push_back((uint8_t)code);
                }
        G.nb_start.push_back((int64_t)G.nb_cell.size());
    }
    if (int rc = assemble(G, bp, B)) return rc;
    build_sym(B);
    return SPH_OK;
}

// The symmetric list build needs one bundle whose targets are all its cells
// in order (every cell pair then has both cells' warps in the same launch),
// the fixed-point path, and a neighbour relation that is symmetric: a target
// never lists a cell twice, its self entry has no shift, and for every entry
// A -> B (shift s) the entries of B hold B -> A with the opposite shift.
// Grid plans (uniform cells) only: their masks are small (a tree plan's
// larger leaves and more entries would make the mask traffic outweigh it).
void build_sym(sph_batch_s *B) {
    B->sym = false;
    B->mask_words = 0;
    B->naux.clear();
    B->mbase.clear();
    B->rev.clear();
    B->rev_start.clear();
    if (B->kind != 0 || !B->fixed_build || B->bundles.size() != 1) return;
    const BatchBundle &bb = B->bundles[0];
    const int64_t nt = bb.ntargets;
    if (nt != bb.ncells) return;
    for (int64_t t = 0; t < nt; ++t)
        if (B->targets[bb.target0 + t].cell != t) return;
    constexpr int kSelfCode = 1 | (1 << 2) | (1 << 4);
    auto mirror = [](int code) {
        int m = 0;
        for (int d = 0; d < 3; ++d) m |= (2 - ((code >> (2 * d)) & 3)) << (2 * d);
        return m;
    };
    std::vector<int32_t> aux(B->nbrs.size(), -1);
    std::vector<int32_t> nfwd((size_t)nt, 0);
    for (int64_t t = 0; t < nt; ++t) {
        const BTargetDev &T = B->targets[bb.target0 + t];
        std::vector<int32_t> seen;
        for (int e = T.nb0; e < T.nb0 + T.nnb; ++e) {
            const int nb = B->nbrs[e].cell;
            for (int32_t q : seen)
                if (q == nb) return;
            seen.push_back(nb);
            if (nb == t) {
                if (B->nbrs[e].code != kSelfCode) return;
            } else if (nb > t) {
                aux[e] = nfwd[t]++;
            }
        }
    }
    for (int64_t t = 0; t < nt; ++t) {
        const BTargetDev &T = B->targets[bb.target0 + t];
        for (int e = T.nb0; e < T.nb0 + T.nnb; ++e) {
            const int a = B->nbrs[e].cell;
            if (a == t) continue;
            // the entry a -> t with the opposite shift
            const BTargetDev &TA = B->targets[bb.target0 + a];
            int found = -1;
            for (int q = TA.nb0; q < TA.nb0 + TA.nnb; ++q)
                if (B->nbrs[q].cell == t && B->nbrs[q].code == mirror(B->nbrs[e].code)) found = q;
            if (found < 0) return;
            if (a < t) aux[e] = aux[found];
        }
    }
    const int W = (int)((B->plan_max_cell + 31) / 32);
    std::vector<int64_t> mb((size_t)nt + 1, 0);
    for (int64_t t = 0; t < nt; ++t) {
        const int64_t n = B->cells[bb.cell0 + t].n;
        mb[t + 1] = mb[t] + ((n + 31) / 32) * nfwd[t] * W * 32;
    }
    for (int64_t t = 0; t < nt; ++t) B->targets[bb.target0 + t].pad = nfwd[t];
    // the backward neighbours of every target, as the second pass reads them
    std::vector<RevEntDev> rev;
    std::vector<int32_t> rstart((size_t)nt + 1, 0);
    for (int64_t t = 0; t < nt; ++t) {
        const BTargetDev &T = B->targets[bb.target0 + t];
        for (int e = T.nb0; e < T.nb0 + T.nnb; ++e) {
            const int a = B->nbrs[e].cell;
            if (a >= t) continue;
            const BCellDev &CA = B->cells[bb.cell0 + a];
            RevEntDev r{};
            r.mrow = mb[a] + (int64_t)aux[e] * W * 32;
            r.stride = nfwd[a] * W * 32;
            r.slot = CA.slot;
            r.n = CA.n;
            rev.push_back(r);
        }
        rstart[t + 1] = (int32_t)rev.size();
    }
    B->sym = true;
    B->sym_words = W;
    B->naux = std::move(aux);
    B->mbase.assign(mb.begin(), mb.end() - 1);
    B->rev = std::move(rev);
    B->rev_start = std::move(rstart);
    B->mask_words = mb[nt];
}

// ---------------------------------------------------------------- tree plan
namespace {

constexpr int kMortonBits = 21;

inline uint64_t spread3(uint64_t v) {  // 21 bits -> every third bit
    v &= 0x1fffffull;
    v = (v | (v << 32)) & 0x1f00000000ffffull;
    v = (v | (v << 16)) & 0x1f0000ff0000ffull;
    v = (v | (v << 8)) & 0x100f00f00f00f00full;
    v = (v | (v << 4)) & 0x10c30c30c30c30c3ull;
    v = (v | (v << 2)) & 0x1249249249249249ull;
    return v;
}

struct Node {
    int64_t b, e;          // particle range (Morton order)
    int32_t level;         // 0 = root (the whole box)
    int32_t child0, nchild;
    double lo[3], hi[3];   // bounding box of the particles' positions
    float hmax;            // largest support H of the particles
};

}  // namespace

namespace {

int tree_plan(int64_t n, const double *x, const float *h, const sph_tree_params *tp,
              int64_t *perm_out, GlobalPlan &G) {
    if (n < 0 || (n > 0 && (!x || !h)) || !tp || !perm_out)
        return fail(SPH_EINVAL, "batch_build_tree: bad arguments");
    if (n > INT32_MAX) return fail(SPH_EUNSUPPORTED, "batch_build_tree: more than 2^31-1 particles");
    if (tp->rule != 0 && tp->rule != 1) return fail(SPH_EINVAL, "batch_build_tree: rule must be 0 or 1");
    if (tp->leaf_max < 8 || tp->leaf_max > 2048)
        return fail(SPH_EINVAL, "batch_build_tree: leaf_max must be in [8, 2048]");
    if (!(tp->kernel_gamma > 0.0)) return fail(SPH_EINVAL, "batch_build_tree: kernel_gamma");
    for (int d = 0; d < 3; ++d)
        if (!(tp->box[d] > 0.0)) return fail(SPH_EINVAL, "batch_build_tree: box edge %d", d);
    const double *L = tp->box;
    const double lmax = std::max(L[0], std::max(L[1], L[2]));
    const double lmin = std::min(L[0], std::min(L[1], L[2]));
    const double delta = (double)(float)(4e-6 * lmax);  // the kernels' prefilter margin
    const float kg = (float)tp->kernel_gamma;

    // supports (as the kernels compute them) and the one-image condition
    int bad = -1;
    float Hmax = 0.f;
#pragma omp parallel for reduction(max : Hmax) reduction(max : bad)
    for (int64_t i = 0; i < n; ++i) {
        const float hi = h[i];
        if (!(hi > 0.f) || !std::isfinite(hi)) bad = 1;
        else Hmax = std::max(Hmax, kg * hi);
    }
    if (bad > 0) return fail(SPH_EINVAL, "batch_build_tree: h must be positive and finite");
    if (!((double)Hmax + delta < 0.5 * lmin))
        return fail(SPH_EUNSUPPORTED,
                    "batch_build_tree: a support (%g) reaches half the box; more than one "
                    "periodic image per pair", (double)Hmax);

    // Morton keys of the clamped positions, sorted with the index as tie-break
    std::vector<std::pair<uint64_t, int64_t>> key((size_t)n);
    const double scale = (double)(1 << kMortonBits);
#pragma omp parallel for
    for (int64_t i = 0; i < n; ++i) {
        uint64_t k = 0;
        for (int d = 0; d < 3; ++d) {
            int64_t q = (int64_t)std::floor(x[3 * i + d] / L[d] * scale);
            q = q < 0 ? 0 : (q >= (1 << kMortonBits) ? (1 << kMortonBits) - 1 : q);
            k |= spread3((uint64_t)q) << d;
        }
        key[(size_t)i] = {k, i};
    }
    __gnu_parallel::sort(key.begin(), key.end());
    std::vector<uint64_t> ks((size_t)n);
    std::vector<double> xs((size_t)n * 3);
    std::vector<float> Hs((size_t)n);
#pragma omp parallel for
    for (int64_t k = 0; k < n; ++k) {
        const int64_t i = key[(size_t)k].second;
        perm_out[k] = i;
        ks[(size_t)k] = key[(size_t)k].first;
        for (int d = 0; d < 3; ++d) xs[(size_t)(3 * k + d)] = x[3 * i + d];
        Hs[(size_t)k] = kg * h[i];
    }
    std::vector<std::pair<uint64_t, int64_t>>().swap(key);

    // octree, breadth first (children of a node are contiguous)
    std::vector<Node> nodes;
    nodes.reserve((size_t)(2 * n / tp->leaf_max + 64));
    nodes.push_back(Node{0, n, 0, -1, 0, {0, 0, 0}, {0, 0, 0}, 0.f});
    for (size_t q = 0; q < nodes.size(); ++q) {
        Node nd = nodes[q];
        if (nd.e - nd.b <= tp->leaf_max || nd.level == kMortonBits) continue;
        if (tp->rule == 1) {
            // half the node's edge must still cover the largest support inside
            float hm = 0.f;
            for (int64_t k = nd.b; k < nd.e; ++k) hm = std::max(hm, Hs[(size_t)k]);
            double half = INFINITY;
            for (int d = 0; d < 3; ++d) half = std::min(half, L[d] / (double)(2ll << nd.level));
            if (half < (double)hm) continue;
        }
        const int shift = 3 * (kMortonBits - 1 - nd.level);
        const int32_t first = (int32_t)nodes.size();
        int32_t nch = 0;
        int64_t b = nd.b;
        const uint64_t pre = ks[(size_t)nd.b] >> (shift + 3);
        for (uint64_t c = 0; c < 8 && b < nd.e; ++c) {
            const uint64_t lim = ((pre << 3) | c) + 1;  // first prefix past child c
            const int64_t e = std::lower_bound(ks.begin() + b, ks.begin() + nd.e, lim << shift,
                                               [](uint64_t a, uint64_t v) { return a < v; }) -
                              ks.begin();
            if (e > b) {
                nodes.push_back(Node{b, e, nd.level + 1, -1, 0, {0, 0, 0}, {0, 0, 0}, 0.f});
                ++nch;
            }
            b = e;
        }
        nodes[q].child0 = first;
        nodes[q].nchild = nch;
    }
    // leaves in Morton order; their boxes and supports
    std::vector<int32_t> leaves;
    for (size_t q = 0; q < nodes.size(); ++q)
        if (nodes[q].nchild == 0 && nodes[q].e > nodes[q].b) leaves.push_back((int32_t)q);
    std::sort(leaves.begin(), leaves.end(),
              [&](int32_t a, int32_t b2) { return nodes[a].b < nodes[b2].b; });
    const int64_t nleaf = (int64_t)leaves.size();
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t l = 0; l < nleaf; ++l) {
        Node &nd = nodes[leaves[l]];
        for (int d = 0; d < 3; ++d) { nd.lo[d] = INFINITY; nd.hi[d] = -INFINITY; }
        float hm = 0.f;
        for (int64_t k = nd.b; k < nd.e; ++k) {
            for (int d = 0; d < 3; ++d) {
                nd.lo[d] = std::min(nd.lo[d], xs[(size_t)(3 * k + d)]);
                nd.hi[d] = std::max(nd.hi[d], xs[(size_t)(3 * k + d)]);
            }
            hm = std::max(hm, Hs[(size_t)k]);
        }
        nd.hmax = hm;
    }
    for (size_t q = nodes.size(); q-- > 0;) {  // children come after parents
        Node &nd = nodes[q];
        if (nd.nchild == 0) continue;
        for (int d = 0; d < 3; ++d) { nd.lo[d] = INFINITY; nd.hi[d] = -INFINITY; }
        nd.hmax = 0.f;
        for (int32_t c = nd.child0; c < nd.child0 + nd.nchild; ++c) {
            for (int d = 0; d < 3; ++d) {
                nd.lo[d] = std::min(nd.lo[d], nodes[c].lo[d]);
                nd.hi[d] = std::max(nd.hi[d], nodes[c].hi[d]);
            }
            nd.hmax = std::max(nd.hmax, nodes[c].hmax);
        }
    }
    std::vector<int32_t> leaf_id(nodes.size(), -1);
    for (int64_t l = 0; l < nleaf; ++l) leaf_id[leaves[l]] = (int32_t)l;

    // neighbour entries: all (leaf, shift) within max(H_T, H_J) + delta of
    // the target's box, by a walk pruned with each subtree's box and H_max
    G.p0.resize((size_t)nleaf);
    G.cnt.resize((size_t)nleaf);
    G.hlim.resize((size_t)nleaf);
    for (int64_t l = 0; l < nleaf; ++l) {
        G.p0[(size_t)l] = nodes[leaves[l]].b;
        G.cnt[(size_t)l] = nodes[leaves[l]].e - nodes[leaves[l]].b;
        G.hlim[(size_t)l] = nodes[leaves[l]].hmax;
    }
    const int nth = omp_get_max_threads();
    std::vector<std::vector<int32_t>> tcell((size_t)nth);
    std::vector<std::vector<uint8_t>> tcode((size_t)nth);
    std::vector<int64_t> nnb((size_t)nleaf, 0);
    std::vector<int> owner((size_t)nleaf, 0);
    std::vector<int64_t> off((size_t)nleaf, 0);
#pragma omp parallel
    {
        const int tid = omp_get_thread_num();
        std::vector<int32_t> stack;
#pragma omp for schedule(dynamic, 256)
        for (int64_t l = 0; l < nleaf; ++l) {
            const Node &T = nodes[leaves[l]];
            owner[(size_t)l] = tid;
            off[(size_t)l] = (int64_t)tcell[(size_t)tid].size();
            stack.clear();
            stack.push_back(0);
            while (!stack.empty()) {
                const int32_t q = stack.back();
                stack.pop_back();
                const Node &N = nodes[q];
                const double R = (double)std::max(T.hmax, N.hmax) + delta;
                // per dimension, the interval distance under each shift
                double dd[3][3];
                double dmin2 = 0.0;
                for (int d = 0; d < 3; ++d) {
                    double m = INFINITY;
                    for (int s = -1; s <= 1; ++s) {
                        const double a0 = N.lo[d] + s * L[d], a1 = N.hi[d] + s * L[d];
                        const double g = std::max(0.0, std::max(a0 - T.hi[d], T.lo[d] - a1));
                        dd[d][s + 1] = g;
                        m = std::min(m, g);
                    }
                    dmin2 += m * m;
                }
                if (!(dmin2 < R * R)) continue;
                if (N.nchild > 0) {
                    for (int32_t c = N.child0 + N.nchild - 1; c >= N.child0; --c) stack.push_back(c);
                    continue;
                }
                for (int s2 = 0; s2 < 3; ++s2)
                    for (int s1 = 0; s1 < 3; ++s1)
                        for (int s0 = 0; s0 < 3; ++s0) {
                            const double g2 = dd[0][s0] * dd[0][s0] + dd[1][s1] * dd[1][s1] +
                                              dd[2][s2] * dd[2][s2];
                            if (!(g2 < R * R)) continue;
                            tcell[(size_t)tid].push_back(leaf_id[q]);
                            tcode[(size_t)tid].push_back((uint8_t)(s0 | (s1 << 2) | (s2 << 4)));
                        }
            }
            nnb[(size_t)l] = (int64_t)tcell[(size_t)tid].size() - off[(size_t)l];
        }
    }
    G.nb_start.assign((size_t)nleaf + 1, 0);
    for (int64_t l = 0; l < nleaf; ++l) G.nb_start[(size_t)l + 1] = G.nb_start[(size_t)l] + nnb[(size_t)l];
    G.nb_cell.resize((size_t)G.nb_start[(size_t)nleaf]);
    G.nb_code.resize((size_t)G.nb_start[(size_t)nleaf]);
#pragma omp parallel for schedule(static, 1024)
    for (int64_t l = 0; l < nleaf; ++l) {
        const auto &vc = tcell[(size_t)owner[(size_t)l]];
        const auto &vk = tcode[(size_t)owner[(size_t)l]];
        std::copy(vc.begin() + off[(size_t)l], vc.begin() + off[(size_t)l] + nnb[(size_t)l],
                  G.nb_cell.begin() + G.nb_start[(size_t)l]);
        std::copy(vk.begin() + off[(size_t)l], vk.begin() + off[(size_t)l] + nnb[(size_t)l],
                  G.nb_code.begin() + G.nb_start[(size_t)l]);
    }
    return SPH_OK;
}

}  // namespace

int build_batch_tree(int64_t n, const double *x, const float *h, const sph_tree_params *tp,
                     const sph_batch_params *bp, int64_t *perm_out, sph_batch_s *B) {
    if (!bp) return fail(SPH_EINVAL, "batch_build_tree: bad arguments");
    if (int rc = check_batch_params(bp)) return rc;
    GlobalPlan G;
    if (int rc = tree_plan(n, x, h, tp, perm_out, G)) return rc;
    B->threads = bp->threads;
    B->n = n;
    B->kind = 1;
    for (int d = 0; d < 3; ++d) B->box[d] = tp->box[d];
    // largest leaf extent (per dimension) and support, for the list build's
    // fixed-point path
    double e0 = 0.0, e1 = 0.0, e2 = 0.0;
    float Hmax = 0.f;
    const float kg = (float)tp->kernel_gamma;
#pragma omp parallel for reduction(max : Hmax)
    for (int64_t i = 0; i < n; ++i) Hmax = std::max(Hmax, kg * h[i]);
    const int64_t nleaf = (int64_t)G.cnt.size();
#pragma omp parallel for schedule(dynamic, 256) reduction(max : e0, e1, e2)
    for (int64_t l = 0; l < nleaf; ++l) {
        double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
        for (int64_t k = G.p0[(size_t)l]; k < G.p0[(size_t)l] + G.cnt[(size_t)l]; ++k) {
            const int64_t i = perm_out[k];
            for (int d = 0; d < 3; ++d) {
                lo[d] = std::min(lo[d], x[3 * i + d]);
                hi[d] = std::max(hi[d], x[3 * i + d]);
            }
        }
        if (G.cnt[(size_t)l] > 0) {
            e0 = std::max(e0, hi[0] - lo[0]);
            e1 = std::max(e1, hi[1] - lo[1]);
            e2 = std::max(e2, hi[2] - lo[2]);
        }
    }
    const double ext[3] = {e0, e1, e2};
    B->fixed_build = true;
    for (int d = 0; d < 3; ++d)
        B->fixed_build = B->fixed_build && ext[d] + (double)Hmax + 1e-6 * tp->box[d] < 0.5 * tp->box[d];
    return assemble(G, bp, B);
}

int tree_plan_host(int64_t n, const double *x, const float *h, const sph_tree_params *tp,
                   int64_t *perm_out, int64_t *leaf_start, int64_t *nleaf_out,
                   int64_t *nb_start, int32_t *nb, int64_t nb_cap, int64_t *nnb_out) {
    if (!leaf_start || !nleaf_out || !nb_start || !nnb_out)
        return fail(SPH_EINVAL, "tree_plan: NULL output");
    GlobalPlan G;
    if (int rc = tree_plan(n, x, h, tp, perm_out, G)) return rc;
    const int64_t nleaf = (int64_t)G.cnt.size(), nnb = (int64_t)G.nb_cell.size();
    *nleaf_out = nleaf;
    *nnb_out = nnb;
    if (nnb > nb_cap || (nnb > 0 && !nb))
        return fail(SPH_EINVAL, "tree_plan: %lld neighbour entries, capacity %lld",
                    (long long)nnb, (long long)nb_cap);
    leaf_start[0] = 0;
    for (int64_t l = 0; l < nleaf; ++l) leaf_start[l + 1] = G.p0[(size_t)l] + G.cnt[(size_t)l];
    for (int64_t l = 0; l <= nleaf; ++l) nb_start[l] = G.nb_start[(size_t)l];
    for (int64_t e = 0; e < nnb; ++e) nb[e] = (G.nb_cell[(size_t)e] << 6) | G.nb_code[(size_t)e];
    return SPH_OK;
}

}  // namespace sph
