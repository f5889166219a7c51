// Host-side cell grid, task list and bundle builder (Sec. 2.2-2.3).
//
// Cells: a uniform grid whose edges are at least the largest kernel support
// H_max, so every neighbour of a particle is in its own or an adjacent cell.
// The default count per dimension follows the octree rule of Sec. 2.2: the
// box edge is halved while the half is still >= H_max.  Particles are sorted
// by cell with a stable counting sort.
//
// Tasks: per non-empty cell a self task, then a pair task with each of the 13
// "forward" neighbours (offsets after (0,0,0) in the (dz, dy, dx) enumeration
// of {-1,0,1}^3), the neighbour's particles shifted by whole box edges where
// the offset wraps.  With >= 3 cells per dimension every cell pair appears
// once.  Bundles are greedy consecutive task ranges under a slot budget
// (dynamic task fusion into offload bundles, Sec. 2.3).
//
// For unpack, every bundle also gets its list of touched cells, each with
// the slots its particles occupy in the bundle's tasks in increasing task
// order, so the reduction into the store is deterministic.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "internal.h"

namespace sph {

int build_tasks(int64_t n, const double *x, const float *h,
                const sph_grid_params *gp, int64_t *perm_out, sph_tasks_s *T) {
    if (n < 0 || (n > 0 && (!x || !h)) || !gp || !perm_out)
        return fail(SPH_EINVAL, "tasks_build: bad arguments");
    if (n > INT32_MAX)
        return fail(SPH_EUNSUPPORTED, "tasks_build: more than 2^31-1 particles");
    for (int d = 0; d < 3; ++d)
        if (!(gp->box[d] > 0.0))
            return fail(SPH_EINVAL, "tasks_build: box edge %d not positive", d);
    if (!(gp->kernel_gamma > 0.0))
        return fail(SPH_EINVAL, "tasks_build: kernel_gamma not positive");
    if (gp->reserved != 0)
        return fail(SPH_EINVAL, "tasks_build: reserved field must be 0");

    double hmax = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double hi = (double)h[i];
        if (!(hi > 0.0) || !std::isfinite(hi))
            return fail(SPH_EINVAL, "tasks_build: h[%lld] not positive",
                        (long long)i);
        if (hi > hmax) hmax = hi;
    }
    const double Hmax = gp->kernel_gamma * hmax;
    for (int d = 0; d < 3; ++d) {
        int32_t nc;
        if (n == 0) {
            nc = gp->ncell[d] > 0 ? gp->ncell[d] : 3;  // no particles: no tasks
        } else if (gp->ncell[d] > 0) {
            nc = gp->ncell[d];
            if (gp->box[d] / nc < Hmax)
                return fail(SPH_EUNSUPPORTED,
                            "tasks_build: %d cells in dim %d are smaller than "
                            "the largest support", nc, d);
        } else {
            nc = 1;
            while (gp->box[d] / (2.0 * nc) >= Hmax && nc < (1 << 20)) nc *= 2;
        }
        if (nc < 3)
            return fail(SPH_EUNSUPPORTED,
                        "tasks_build: only %d cells fit in dim %d (need >= 3 "
                        "for unique periodic pair tasks)", nc, d);
        T->ncell[d] = nc;
        T->box[d] = gp->box[d];
    }
    const int64_t ncells = (int64_t)T->ncell[0] * T->ncell[1] * T->ncell[2];
    if (ncells > INT32_MAX)
        return fail(SPH_EUNSUPPORTED, "tasks_build: too many cells");
    T->n = n;

    // cell of each particle and stable counting sort
    std::vector<int32_t> cell((size_t)n);
    T->cell_start.assign((size_t)ncells + 1, 0);
    for (int64_t i = 0; i < n; ++i) {
        int64_t c[3];
        for (int d = 0; d < 3; ++d) {
            int64_t k = (int64_t)std::floor(x[3 * i + d] / gp->box[d] * T->ncell[d]);
            c[d] = k < 0 ? 0 : (k >= T->ncell[d] ? T->ncell[d] - 1 : k);
        }
        cell[i] = (int32_t)(c[0] + T->ncell[0] * (c[1] + T->ncell[1] * c[2]));
        T->cell_start[cell[i] + 1]++;
    }
    for (int64_t c = 0; c < ncells; ++c) T->cell_start[c + 1] += T->cell_start[c];
    {
        std::vector<int64_t> next(T->cell_start.begin(), T->cell_start.end() - 1);
        for (int64_t i = 0; i < n; ++i) perm_out[next[cell[i]]++] = i;
    }
    auto count = [&](int64_t c) { return T->cell_start[c + 1] - T->cell_start[c]; };
    T->max_cell = 0;
    for (int64_t c = 0; c < ncells; ++c) T->max_cell = std::max(T->max_cell, count(c));

    // tasks
    T->ci.clear(); T->cj.clear(); T->shift.clear();
    const int32_t *nc = T->ncell;
    for (int64_t c = 0; c < ncells; ++c) {
        if (count(c) == 0) continue;
        T->ci.push_back((int32_t)c); T->cj.push_back(-1);
        T->shift.insert(T->shift.end(), {0, 0, 0});
        const int64_t ix = c % nc[0], iy = (c / nc[0]) % nc[1],
                      iz = c / ((int64_t)nc[0] * nc[1]);
        int idx = 0;  // position in the (dz, dy, dx) enumeration
        for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx, ++idx) {
                    if (idx <= 13) continue;  // 13 is (0,0,0)
                    int64_t q[3] = {ix + dx, iy + dy, iz + dz};
                    int8_t s[3];
                    for (int d = 0; d < 3; ++d) {
                        s[d] = 0;
                        if (q[d] < 0) { q[d] += nc[d]; s[d] = -1; }
                        if (q[d] >= nc[d]) { q[d] -= nc[d]; s[d] = 1; }
                    }
                    int64_t c2 = q[0] + nc[0] * (q[1] + nc[1] * q[2]);
                    if (count(c2) == 0) continue;
                    T->ci.push_back((int32_t)c); T->cj.push_back((int32_t)c2);
                    T->shift.insert(T->shift.end(), {s[0], s[1], s[2]});
                }
    }
    const int64_t ntasks = (int64_t)T->ci.size();

    // bundles
    T->bundle_start.assign(1, 0);
    T->bundle_slots.clear();
    T->tdev.resize((size_t)ntasks);
    int64_t slots = 0;
    for (int64_t t = 0; t < ntasks; ++t) {
        int64_t s = count(T->ci[t]) + (T->cj[t] >= 0 ? count(T->cj[t]) : 0);
        if (t > 0 && gp->bundle_max_slots > 0 && slots + s > gp->bundle_max_slots) {
            T->bundle_start.push_back(t);
            T->bundle_slots.push_back(slots);
            slots = 0;
        }
        if (slots + s > INT32_MAX)
            return fail(SPH_EUNSUPPORTED, "tasks_build: bundle exceeds 2^31-1 "
                        "slots; set bundle_max_slots");
        TaskDev &td = T->tdev[t];
        td.pi = (int32_t)T->cell_start[T->ci[t]];
        td.ni = (int32_t)count(T->ci[t]);
        td.pj = T->cj[t] >= 0 ? (int32_t)T->cell_start[T->cj[t]] : 0;
        td.nj = T->cj[t] >= 0 ? (int32_t)count(T->cj[t]) : 0;
        td.slot = (int32_t)slots;
        td.shift = (T->shift[3 * t] + 1) | ((T->shift[3 * t + 1] + 1) << 2) |
                   ((T->shift[3 * t + 2] + 1) << 4);
        if (T->cj[t] >= 0) {
            // offset from ci to cj in cells (unwrapped): bits 6-11
            const int64_t a = T->ci[t], b = T->cj[t];
            const int64_t ca[3] = {a % nc[0], (a / nc[0]) % nc[1], a / ((int64_t)nc[0] * nc[1])};
            const int64_t cb[3] = {b % nc[0], (b / nc[0]) % nc[1], b / ((int64_t)nc[0] * nc[1])};
            int code = 0;
            for (int d = 0; d < 3; ++d) {
                const int64_t off = cb[d] - ca[d] + (int64_t)T->shift[3 * t + d] * nc[d];
                code |= (int)(off + 1) << (2 * d);
            }
            td.shift |= code << 6;
        } else {
            td.shift |= (1 | (1 << 2) | (1 << 4)) << 6;
        }
        slots += s;
    }
    if (ntasks > 0) {
        T->bundle_start.push_back(ntasks);
        T->bundle_slots.push_back(slots);
    }

    // unpack maps: per bundle, touched cells with their slots in task order
    const int64_t nb = (int64_t)T->bundle_slots.size();
    T->ucell_begin.assign(1, 0);
    T->entry_begin.assign(1, 0);
    T->ucells.clear();
    T->entries.clear();
    std::vector<std::pair<int32_t, int32_t>> occ;  // (cell, slot)
    for (int64_t b = 0; b < nb; ++b) {
        occ.clear();
        for (int64_t t = T->bundle_start[b]; t < T->bundle_start[b + 1]; ++t) {
            const TaskDev &td = T->tdev[t];
            occ.push_back({T->ci[t], td.slot});
            if (T->cj[t] >= 0) occ.push_back({T->cj[t], td.slot + td.ni});
        }
        std::stable_sort(occ.begin(), occ.end(),
                         [](const std::pair<int32_t, int32_t> &a,
                            const std::pair<int32_t, int32_t> &b2) {
                             return a.first < b2.first;
                         });
        const int64_t e0 = (int64_t)T->entries.size();
        for (size_t k = 0; k < occ.size();) {
            size_t k2 = k;
            while (k2 < occ.size() && occ[k2].first == occ[k].first) ++k2;
            UCellDev u;
            u.p0 = (int32_t)T->cell_start[occ[k].first];
            u.n = (int32_t)count(occ[k].first);
            u.e0 = (int32_t)((int64_t)T->entries.size() - e0);
            u.ne = (int32_t)(k2 - k);
            T->ucells.push_back(u);
            for (size_t q = k; q < k2; ++q) T->entries.push_back(occ[q].second);
            k = k2;
        }
        T->ucell_begin.push_back((int64_t)T->ucells.size());
        T->entry_begin.push_back((int64_t)T->entries.size());
    }
    return SPH_OK;
}

}  // namespace sph
