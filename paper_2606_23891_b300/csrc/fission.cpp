// Loop-fission variants of the host pack and unpack (Sec. 3.3, Fig. 4).
//
// The conversions copy, per slot (pack) or per particle (unpack), a set of
// field components between the store and the packed lanes.  The variants
// differ only in how that work is split into loops:
//   none               one loop; its body copies every component of a slot
//   by_struct          one loop per store substruct the conversion touches
//   by_element         one loop per field component
//   by_type            one loop per data type (double, float, int)
//   by_struct_and_type the by_struct loops split further by data type
// Every variant writes the same bytes: the pack's lanes are disjoint per
// component, and the unpack folds each component's slots in the same order.
// The body is a generic copy over a list of component descriptors, the same
// for every variant, so the measured differences come from the loop
// structure alone.
#include <cmath>
#include <cstring>

#include <omp.h>

#include "internal.h"

namespace sph {

namespace {

struct Item {
    CompPtr st;      // store side
    char *lane;      // packed side: lane base
    int lstride;     // lane bytes per slot
    int loff;        // byte offset inside a slot's lane element
    int bytes;       // 8, 4 or 1
    int shift_dim;   // pack: x component shifted on the second cell (-1: none)
    int cls;         // T_DOUBLE, T_FLOAT, T_INT
    int group;       // store substruct of `st`
    int kahan;       // unpack: 1 sum (Kahan), 2 max
};

int group_of(const sph_store_s *s, const CompPtr &c) {
    const int64_t off = c.ptr - s->mem;
    int g = 0;
    for (const Group &G : s->layout.groups) {
        const int64_t size = s->n * (int64_t)G.record;
        if (off >= G.base && off < G.base + (size > 0 ? size : 1)) return g;
        ++g;
    }
    return -1;
}

std::vector<std::vector<int>> partition(const std::vector<Item> &items, int fission) {
    std::vector<std::vector<int>> parts;
    auto key = [&](const Item &it) -> long {
        switch (fission) {
        case SPH_FISSION_BY_STRUCT: return it.group;
        case SPH_FISSION_BY_TYPE: return it.cls;
        case SPH_FISSION_BY_STRUCT_AND_TYPE: return 8L * it.group + it.cls;
        default: return 0;
        }
    };
    if (fission == SPH_FISSION_BY_ELEMENT) {
        for (int k = 0; k < (int)items.size(); ++k) parts.push_back({k});
        return parts;
    }
    std::vector<long> keys;
    for (int k = 0; k < (int)items.size(); ++k) {
        const long kk = key(items[k]);
        size_t q = 0;
        while (q < keys.size() && keys[q] != kk) ++q;
        if (q == keys.size()) {
            keys.push_back(kk);
            parts.emplace_back();
        }
        parts[q].push_back(k);
    }
    return parts;
}

CompPtr view_ptr(sph_store s, int field, int comp, int loop) {
    CompPtr c{nullptr, 0};
    locate_view(s->layout, s->mem, field, comp, loop, &c);
    return c;
}

CompPtr first_ptr(sph_store s, int field, int comp) {
    CompPtr c{nullptr, 0};
    locate(s->layout, s->mem, field, comp, &c);
    return c;
}

int nthr(int n) { return n > 0 ? n : omp_get_max_threads(); }

struct KahanF {
    float s, c;
    void add(float x) {
        const float y = x - c;
        const float t = s + y;
        c = (t - s) - y;
        s = t;
    }
};

}  // namespace

int host_pack_fission(sph_store s, sph_tasks t, int loop, int b, char *buf, int fission,
                      int nthreads) {
    int64_t off[16];
    lane_offsets(loop, 0, t->bundle_slots[b], off);
    std::vector<Item> items;
    auto add = [&](int field, int comp, int lane, int lstride, int loff, int bytes, int sd,
                   int cls) {
        Item it{};
        it.st = view_ptr(s, field, comp, loop);
        it.lane = buf + off[lane];
        it.lstride = lstride;
        it.loff = loff;
        it.bytes = bytes;
        it.shift_dim = sd;
        it.cls = cls;
        it.group = group_of(s, it.st);
        items.push_back(it);
    };
    for (int d = 0; d < 3; ++d) add(F_X, d, d, 8, 0, 8, d, T_DOUBLE);
    for (int d = 0; d < 3; ++d) add(F_V, d, 3, 16, 4 * d, 4, -1, T_FLOAT);
    add(F_MASS, 0, 3, 16, 12, 4, -1, T_FLOAT);
    add(F_H, 0, 4, 4, 0, 4, -1, T_FLOAT);
    if (loop >= SPH_GRADIENT) {
        add(F_U, 0, 5, 4, 0, 4, -1, T_FLOAT);
        add(F_RHO, 0, 6, 4, 0, 4, -1, T_FLOAT);
    }
    if (loop == SPH_FORCE) {
        add(F_FGRADH, 0, 7, 4, 0, 4, -1, T_FLOAT);
        add(F_BALS, 0, 8, 4, 0, 4, -1, T_FLOAT);
        add(F_AVISC, 0, 9, 4, 0, 4, -1, T_FLOAT);
        add(F_ADIFF, 0, 10, 4, 0, 4, -1, T_FLOAT);
        add(F_TBIN, 0, 11, 1, 0, 1, -1, T_INT);
    }
    const auto parts = partition(items, fission);
    const int64_t t0 = t->bundle_start[b], t1 = t->bundle_start[b + 1];
    const double *box = t->box;
    for (const auto &part : parts) {
#pragma omp parallel for schedule(static) num_threads(nthr(nthreads))
        for (int64_t ti = t0; ti < t1; ++ti) {
            const TaskDev &T = t->tdev[ti];
            const int n = T.ni + T.nj;
            for (int k = 0; k < n; ++k) {
                const bool side = k >= T.ni;
                const int64_t p = side ? (int64_t)T.pj + (k - T.ni) : (int64_t)T.pi + k;
                const int64_t sl = (int64_t)T.slot + k;
                for (int q : part) {
                    const Item &it = items[q];
                    const char *src = it.st.ptr + p * it.st.stride;
                    char *dst = it.lane + sl * it.lstride + it.loff;
                    if (it.bytes == 8) {
                        double xv;
                        memcpy(&xv, src, 8);
                        if (it.shift_dim >= 0 && side) {
                            const int code = ((T.shift >> (2 * it.shift_dim)) & 3) - 1;
                            if (code != 0) xv = xv + (code > 0 ? box[it.shift_dim] : -box[it.shift_dim]);
                        }
                        memcpy(dst, &xv, 8);
                    } else if (it.bytes == 4) {
                        memcpy(dst, src, 4);
                    } else {
                        *dst = *src;
                    }
                }
            }
        }
    }
    return SPH_OK;
}

int host_unpack_fission(sph_store s, sph_tasks t, int loop, int b, const char *buf, int fission,
                        int nthreads) {
    int64_t off[16];
    lane_offsets(loop, 1, t->bundle_slots[b], off);
    std::vector<Item> items;
    auto add = [&](int field, int comp, int lane, int lstride, int loff, int kind) {
        Item it{};
        it.st = first_ptr(s, field, comp);
        it.lane = const_cast<char *>(buf) + off[lane];
        it.lstride = lstride;
        it.loff = loff;
        it.bytes = 4;
        it.shift_dim = -1;
        it.cls = T_FLOAT;
        it.group = group_of(s, it.st);
        it.kahan = kind;
        items.push_back(it);
    };
    if (loop == SPH_DENSITY) {
        const int f0[4] = {F_RHO, F_RHODH, F_WCOUNT, F_WCOUNTDH};
        for (int q = 0; q < 4; ++q) add(f0[q], 0, 0, 16, 4 * q, 1);
        add(F_DIVV, 0, 1, 16, 0, 1);
        for (int c = 0; c < 3; ++c) add(F_ROTV, c, 1, 16, 4 + 4 * c, 1);
    } else if (loop == SPH_GRADIENT) {
        add(F_VSIGG, 0, 0, 8, 0, 2);
        add(F_LAPU, 0, 0, 8, 4, 1);
    } else {
        for (int c = 0; c < 3; ++c) add(F_A, c, 0, 16, 4 * c, 1);
        add(F_UDT, 0, 0, 16, 12, 1);
        add(F_HDT, 0, 1, 8, 0, 1);
        add(F_VSIG, 0, 1, 8, 4, 2);
    }
    const auto parts = partition(items, fission);
    const int64_t c0 = t->ucell_begin[b], c1 = t->ucell_begin[b + 1];
    const int32_t *ent = t->entries.data() + t->entry_begin[b];
    for (const auto &part : parts) {
#pragma omp parallel for schedule(static) num_threads(nthr(nthreads))
        for (int64_t ci = c0; ci < c1; ++ci) {
            const UCellDev &C = t->ucells[ci];
            for (int i = 0; i < C.n; ++i) {
                const int64_t p = (int64_t)C.p0 + i;
                for (int q : part) {
                    const Item &it = items[q];
                    char *sp = it.st.ptr + p * it.st.stride;
                    float cur;
                    memcpy(&cur, sp, 4);
                    KahanF acc{cur, 0.f};
                    for (int e = 0; e < C.ne; ++e) {
                        const int64_t sl = (int64_t)ent[C.e0 + e] + i;
                        float o;
                        memcpy(&o, it.lane + sl * it.lstride + it.loff, 4);
                        if (it.kahan == 2) acc.s = fmaxf(acc.s, o);
                        else acc.add(o);
                    }
                    memcpy(sp, &acc.s, 4);
                }
            }
        }
    }
    return SPH_OK;
}

}  // namespace sph
