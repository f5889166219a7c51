// Particle-store layout engine (Sec. 3.1).
//
// A layout is an ordered list of substructs ("groups"); each group is laid
// out like a C struct (member offset rounded up to the member's element size,
// record rounded up to the largest element size), and the group arrays follow
// each other in the store, each starting at a 256-byte boundary so that every
// group array is aligned for 16-byte vector and bulk copies.
//
// The member catalogue is Table 1 (x, v, a, mass, h, u, u_dt, rho, time_bin)
// followed by the remaining quantities of the Sphenix loops and 8 bytes of
// ballast that stand for the members no loop touches; the AoS record is then
// 160 bytes, the paper's 2.5 GiB for 256^3 particles (Sec. 3.4).
#include <cstring>

#include "internal.h"

namespace sph {

const FieldInfo kFields[F_NUM] = {
    {8, 3, T_DOUBLE},                   // x
    {4, 3, T_FLOAT}, {4, 3, T_FLOAT},   // v, a
    {4, 1, T_FLOAT}, {4, 1, T_FLOAT},   // mass, h
    {4, 1, T_FLOAT}, {4, 1, T_FLOAT},   // u, u_dt
    {4, 1, T_FLOAT},                    // rho
    {1, 1, T_INT},                      // time_bin
    {4, 1, T_FLOAT}, {4, 1, T_FLOAT},   // alpha_visc, alpha_diff
    {4, 1, T_FLOAT}, {4, 1, T_FLOAT},   // rho_dh, wcount
    {4, 1, T_FLOAT}, {4, 1, T_FLOAT},   // wcount_dh, div_v
    {4, 3, T_FLOAT},                    // rot_v
    {4, 1, T_FLOAT}, {4, 1, T_FLOAT},   // f_gradh, pressure
    {4, 1, T_FLOAT}, {4, 1, T_FLOAT},   // soundspeed, balsara
    {4, 1, T_FLOAT}, {4, 1, T_FLOAT},   // v_sig_grad, laplace_u
    {4, 1, T_FLOAT}, {4, 1, T_FLOAT},   // h_dt, v_sig
    {8, 1, T_INT},                      // id
    {1, 8, T_INT},                      // ballast
};

namespace {

// Members in the order they are used by the code (Table 1 rows first).
const int kUseOrder[F_NUM] = {
    F_X, F_V, F_A, F_MASS, F_H, F_U, F_UDT, F_RHO, F_TBIN, F_AVISC, F_ADIFF,
    F_RHODH, F_WCOUNT, F_WCOUNTDH, F_DIVV, F_ROTV, F_FGRADH, F_PRES, F_CS,
    F_BALS, F_VSIGG, F_LAPU, F_HDT, F_VSIG, F_ID, F_BALLAST};

// Views (Table 1, extended to the quantities each loop reads and writes).
const std::vector<int> kGradView = {F_X, F_V, F_MASS, F_H, F_U, F_RHO};
const std::vector<int> kForceOnly = {F_TBIN, F_FGRADH, F_BALS, F_AVISC,
                                     F_ADIFF};
const std::vector<int> kForceView = {F_X, F_V, F_MASS, F_H, F_U, F_RHO,
                                     F_TBIN, F_FGRADH, F_BALS, F_AVISC,
                                     F_ADIFF};
const std::vector<int> kSharedAll = {F_X, F_V, F_MASS, F_H};
const std::vector<int> kURho = {F_U, F_RHO};
const std::vector<int> kDensOut = {F_RHODH, F_WCOUNT, F_WCOUNTDH, F_DIVV,
                                   F_ROTV};
const std::vector<int> kGradOut = {F_VSIGG, F_LAPU};
const std::vector<int> kForceOut = {F_A, F_UDT, F_HDT, F_VSIG};
const std::vector<int> kRest = {F_PRES, F_CS, F_ID, F_BALLAST};
// replication: the density view's inputs stored again on their own
const std::vector<int> kDensView = {F_X, F_V, F_MASS, F_H};
// fused views: each loop's inputs with the outputs its unpack writes
const std::vector<int> kFusedDens = {F_X, F_V, F_MASS, F_H, F_RHO, F_RHODH, F_WCOUNT,
                                     F_WCOUNTDH, F_DIVV, F_ROTV};
const std::vector<int> kFusedGrad = {F_U, F_VSIGG, F_LAPU};
const std::vector<int> kFusedForce = {F_TBIN, F_FGRADH, F_BALS, F_AVISC, F_ADIFF, F_A,
                                      F_UDT, F_HDT, F_VSIG};

// SplitMix64 step (Steele, Lea, Flood 2014).
uint64_t splitmix64_next(uint64_t &s) {
    s += 0x9E3779B97F4A7C15ull;
    uint64_t z = s;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

void push(Layout &L, const std::vector<int> &fields) {
    Group g;
    for (int f : fields) g.mem.push_back({f, -1, 0});
    L.groups.push_back(g);
}

void push_split(Layout &L, const std::vector<int> &fields, bool by_type) {
    if (!by_type) {
        push(L, fields);
        return;
    }
    for (int cls = T_DOUBLE; cls <= T_INT; ++cls) {
        std::vector<int> sub;
        for (int f : fields)
            if (kFields[f].cls == cls) sub.push_back(f);
        if (!sub.empty()) push(L, sub);
    }
}

void place(Group &g) {
    int off = 0, align = 1;
    for (Member &m : g.mem) {
        int e = kFields[m.field].elem;
        int bytes = m.comp >= 0 ? e : e * kFields[m.field].count;
        off = (off + e - 1) / e * e;
        m.offset = off;
        off += bytes;
        if (e > align) align = e;
    }
    g.record = (off + align - 1) / align * align;
}

}  // namespace

int build_layout(int layout, uint64_t seed, int64_t n, Layout *out) {
    Layout L;
    L.id = layout;
    L.seed = seed;
    const bool typed = layout == SPH_SAOS_PACK_GRAD_TYPE ||
                       layout == SPH_SAOS_PACK_FORCE_TYPE ||
                       layout == SPH_SAOS_PACK_SHARED_TYPE;
    switch (layout) {
    case SPH_AOS:
        push(L, std::vector<int>(kUseOrder, kUseOrder + F_NUM));
        break;
    case SPH_AOS_RANDOM: {
        std::vector<int> order(kUseOrder, kUseOrder + F_NUM);
        uint64_t s = seed;
        for (int i = F_NUM - 1; i > 0; --i) {  // Fisher-Yates
            int j = (int)(splitmix64_next(s) % (uint64_t)(i + 1));
            std::swap(order[i], order[j]);
        }
        push(L, order);
        break;
    }
    case SPH_SAOS_PACK_GRAD:
    case SPH_SAOS_PACK_GRAD_TYPE:
        for (const auto *v : {&kGradView, &kForceOnly, &kDensOut, &kGradOut,
                              &kForceOut, &kRest})
            push_split(L, *v, typed);
        break;
    case SPH_SAOS_PACK_FORCE:
    case SPH_SAOS_PACK_FORCE_TYPE:
        for (const auto *v : {&kForceView, &kDensOut, &kGradOut, &kForceOut,
                              &kRest})
            push_split(L, *v, typed);
        break;
    case SPH_SAOS_PACK_SHARED:
    case SPH_SAOS_PACK_SHARED_TYPE:
        for (const auto *v : {&kSharedAll, &kURho, &kForceOnly, &kDensOut,
                              &kGradOut, &kForceOut, &kRest})
            push_split(L, *v, typed);
        break;
    case SPH_SAOS_PACK_FORCE_REPL:
        for (const auto *v : {&kDensView, &kForceView, &kDensOut, &kGradOut, &kForceOut, &kRest})
            push(L, *v);
        L.view_group[SPH_DENSITY] = 0;
        L.view_group[SPH_GRADIENT] = 1;
        L.view_group[SPH_FORCE] = 1;
        break;
    case SPH_SAOS_FUSED:
        for (const auto *v : {&kFusedDens, &kFusedGrad, &kFusedForce, &kRest}) push(L, *v);
        break;
    case SPH_SOA:
        for (int f : kUseOrder) {
            if (f == F_BALLAST || kFields[f].count == 1) {
                push(L, {f});
                continue;
            }
            for (int c = 0; c < kFields[f].count; ++c) {
                Group g;
                g.mem.push_back({f, c, 0});
                L.groups.push_back(g);
            }
        }
        break;
    default:
        return SPH_EINVAL;
    }
    int64_t base = 0;
    for (Group &g : L.groups) {
        place(g);
        g.base = base;
        base += (n * g.record + 255) / 256 * 256;
    }
    *out = L;
    return SPH_OK;
}

int64_t layout_bytes(const Layout &L, int64_t n) {
    int64_t b = 0;
    for (const Group &g : L.groups) b += (n * g.record + 255) / 256 * 256;
    return b;
}

bool locate(const Layout &L, char *mem, int field, int comp, CompPtr *out) {
    for (const Group &g : L.groups) {
        for (const Member &m : g.mem) {
            if (m.field != field) continue;
            if (m.comp >= 0 && m.comp != comp) continue;
            int extra = m.comp >= 0 ? 0 : comp * kFields[field].elem;
            out->ptr = mem + g.base + m.offset + extra;
            out->stride = g.record;
            return true;
        }
    }
    return false;
}

static bool member_ptr(const Layout &L, const Group &g, char *mem, int field, int comp,
                       CompPtr *out) {
    for (const Member &m : g.mem) {
        if (m.field != field) continue;
        if (m.comp >= 0 && m.comp != comp) continue;
        int extra = m.comp >= 0 ? 0 : comp * kFields[field].elem;
        out->ptr = mem + g.base + m.offset + extra;
        out->stride = g.record;
        return true;
    }
    return false;
}

int locate_all(const Layout &L, char *mem, int field, int comp, CompPtr *out, int max) {
    int k = 0;
    for (const Group &g : L.groups)
        if (k < max && member_ptr(L, g, mem, field, comp, &out[k])) ++k;
    return k;
}

bool locate_view(const Layout &L, char *mem, int field, int comp, int loop, CompPtr *out) {
    if (loop >= 0 && loop < 3 && L.view_group[loop] >= 0 &&
        member_ptr(L, L.groups[L.view_group[loop]], mem, field, comp, out))
        return true;
    return locate(L, mem, field, comp, out);
}

int lane_sizes(int loop, int in_or_out, int64_t *sz) {
    int k = 0;
    if (in_or_out == 0) {
        sz[k++] = 8; sz[k++] = 8; sz[k++] = 8;  // x0 x1 x2
        sz[k++] = 16;                           // vx vy vz m
        sz[k++] = 4;                            // h
        if (loop >= SPH_GRADIENT) { sz[k++] = 4; sz[k++] = 4; }  // u rho
        if (loop == SPH_FORCE) {
            for (int i = 0; i < 4; ++i) sz[k++] = 4;  // f_gradh bal av ad
            sz[k++] = 1;                              // time_bin
        }
        return k;
    }
    if (loop == SPH_DENSITY) { sz[0] = 16; sz[1] = 16; return 2; }
    if (loop == SPH_GRADIENT) { sz[0] = 8; return 1; }
    sz[0] = 16; sz[1] = 8;
    return 2;
}

int64_t lane_offsets(int loop, int in_or_out, int64_t S, int64_t *off) {
    int64_t sz[16];
    int nl = lane_sizes(loop, in_or_out, sz);
    int64_t o = 0;
    for (int k = 0; k < nl; ++k) {
        off[k] = o;
        o += (S * sz[k] + 255) / 256 * 256;
    }
    return o;
}

}  // namespace sph
