// Host side of the host-staged offload cycle (Sec. 2.3): the particle store
// lives in host memory, pack gathers a bundle's view into a pinned host
// buffer, and unpack reduces the result buffer copied back from the GPU into
// the store.  The same definitions as the device kernels (pack_kernels.cuh,
// store_kernels.cuh) are implemented with OpenMP over tasks / cells, so the
// pack and unpack bytes are identical to the device path's.
#include <omp.h>

#include <cmath>
#include <cstring>

#include "internal.h"

namespace sph {

namespace {

template <typename T>
inline T hld(const CompPtr &c, int64_t p) {
    T v;
    memcpy(&v, c.ptr + p * c.stride, sizeof(T));
    return v;
}
template <typename T>
inline void hst(const CompPtr &c, int64_t p, T v) {
    memcpy(c.ptr + p * c.stride, &v, sizeof(T));
}

CompPtr at(sph_store s, int field, int comp) {
    CompPtr c{nullptr, 0};
    locate(s->layout, s->mem, field, comp, &c);
    return c;
}

// The copy of (field, comp) that the pack of `loop` reads.
CompPtr at_view(sph_store s, int field, int comp, int loop) {
    CompPtr c{nullptr, 0};
    locate_view(s->layout, s->mem, field, comp, loop, &c);
    return c;
}

int threads(int n) { return n > 0 ? n : omp_get_max_threads(); }

// Kahan step, plain FP32 adds (no multiplies: nothing to contract).
struct KahanH {
    float s, c;
    void init(float v) { s = v; c = 0.f; }
    void add(float x) {
        const float y = x - c;
        const float t = s + y;
        c = (t - s) - y;
        s = t;
    }
};

}  // namespace

int host_pack(sph_store s, sph_tasks t, int loop, int b, char *buf, int nthreads) {
    const int64_t t0 = t->bundle_start[b], t1 = t->bundle_start[b + 1];
    int64_t off[16];
    lane_offsets(loop, 0, t->bundle_slots[b], off);
    char *lane[16];
    for (int k = 0; k < 12; ++k) lane[k] = buf + off[k];
    auto av_ = [&](int f, int c) { return at_view(s, f, c, loop); };
    CompPtr x[3] = {av_(F_X, 0), av_(F_X, 1), av_(F_X, 2)};
    CompPtr v[3] = {av_(F_V, 0), av_(F_V, 1), av_(F_V, 2)};
    CompPtr m = av_(F_MASS, 0), h = av_(F_H, 0), u = av_(F_U, 0), rho = av_(F_RHO, 0);
    CompPtr fgh = av_(F_FGRADH, 0), bal = av_(F_BALS, 0), av = av_(F_AVISC, 0),
            ad = av_(F_ADIFF, 0), tb = av_(F_TBIN, 0);
    const double *box = t->box;
#pragma omp parallel for schedule(static) num_threads(threads(nthreads))
    for (int64_t ti = t0; ti < t1; ++ti) {
        const TaskDev &T = t->tdev[ti];
        const int n = T.ni + T.nj;
        for (int k = 0; k < n; ++k) {
            const bool side = k >= T.ni;
            const int64_t p = side ? (int64_t)T.pj + (k - T.ni) : (int64_t)T.pi + k;
            const int64_t sl = (int64_t)T.slot + k;
            for (int d = 0; d < 3; ++d) {
                double xv = hld<double>(x[d], p);
                const int code = side ? ((T.shift >> (2 * d)) & 3) - 1 : 0;
                if (code != 0) xv = xv + (code > 0 ? box[d] : -box[d]);
                memcpy(lane[d] + 8 * sl, &xv, 8);
            }
            const float vm[4] = {hld<float>(v[0], p), hld<float>(v[1], p), hld<float>(v[2], p),
                                 hld<float>(m, p)};
            memcpy(lane[3] + 16 * sl, vm, 16);
            const float hv = hld<float>(h, p);
            memcpy(lane[4] + 4 * sl, &hv, 4);
            if (loop >= SPH_GRADIENT) {
                const float a = hld<float>(u, p), r = hld<float>(rho, p);
                memcpy(lane[5] + 4 * sl, &a, 4);
                memcpy(lane[6] + 4 * sl, &r, 4);
            }
            if (loop == SPH_FORCE) {
                const float f0 = hld<float>(fgh, p), f1 = hld<float>(bal, p),
                            f2 = hld<float>(av, p), f3 = hld<float>(ad, p);
                const int8_t tv = hld<int8_t>(tb, p);
                memcpy(lane[7] + 4 * sl, &f0, 4);
                memcpy(lane[8] + 4 * sl, &f1, 4);
                memcpy(lane[9] + 4 * sl, &f2, 4);
                memcpy(lane[10] + 4 * sl, &f3, 4);
                memcpy(lane[11] + sl, &tv, 1);
            }
        }
    }
    return SPH_OK;
}

int host_unpack(sph_store s, sph_tasks t, int loop, int b, const char *buf, int nthreads) {
    int64_t off[16];
    lane_offsets(loop, 1, t->bundle_slots[b], off);
    const char *l0 = buf + off[0];
    const char *l1 = buf + off[1];
    CompPtr dst[8];
    int k = 0;
    if (loop == SPH_DENSITY) {
        dst[k++] = at(s, F_RHO, 0);
        dst[k++] = at(s, F_RHODH, 0);
        dst[k++] = at(s, F_WCOUNT, 0);
        dst[k++] = at(s, F_WCOUNTDH, 0);
        dst[k++] = at(s, F_DIVV, 0);
        for (int c = 0; c < 3; ++c) dst[k++] = at(s, F_ROTV, c);
    } else if (loop == SPH_GRADIENT) {
        dst[k++] = at(s, F_VSIGG, 0);
        dst[k++] = at(s, F_LAPU, 0);
    } else {
        for (int c = 0; c < 3; ++c) dst[k++] = at(s, F_A, c);
        dst[k++] = at(s, F_UDT, 0);
        dst[k++] = at(s, F_HDT, 0);
        dst[k++] = at(s, F_VSIG, 0);
    }
    const int64_t c0 = t->ucell_begin[b], c1 = t->ucell_begin[b + 1];
    const int32_t *ent = t->entries.data() + t->entry_begin[b];
#pragma omp parallel for schedule(static) num_threads(threads(nthreads))
    for (int64_t ci = c0; ci < c1; ++ci) {
        const UCellDev &C = t->ucells[ci];
        for (int i = 0; i < C.n; ++i) {
            const int64_t p = (int64_t)C.p0 + i;
            if (loop == SPH_DENSITY) {
                KahanH acc[8];
                for (int q = 0; q < 8; ++q) acc[q].init(hld<float>(dst[q], p));
                for (int e = 0; e < C.ne; ++e) {
                    const int64_t sl = (int64_t)ent[C.e0 + e] + i;
                    float o[8];
                    memcpy(o, l0 + 16 * sl, 16);
                    memcpy(o + 4, l1 + 16 * sl, 16);
                    for (int q = 0; q < 8; ++q) acc[q].add(o[q]);
                }
                for (int q = 0; q < 8; ++q) hst<float>(dst[q], p, acc[q].s);
            } else if (loop == SPH_GRADIENT) {
                float vs = hld<float>(dst[0], p);
                KahanH lap;
                lap.init(hld<float>(dst[1], p));
                for (int e = 0; e < C.ne; ++e) {
                    const int64_t sl = (int64_t)ent[C.e0 + e] + i;
                    float o[2];
                    memcpy(o, l0 + 8 * sl, 8);
                    vs = fmaxf(vs, o[0]);
                    lap.add(o[1]);
                }
                hst<float>(dst[0], p, vs);
                hst<float>(dst[1], p, lap.s);
            } else {
                KahanH acc[5];
                for (int q = 0; q < 5; ++q) acc[q].init(hld<float>(dst[q], p));
                float vs = hld<float>(dst[5], p);
                for (int e = 0; e < C.ne; ++e) {
                    const int64_t sl = (int64_t)ent[C.e0 + e] + i;
                    float o[6];
                    memcpy(o, l0 + 16 * sl, 16);
                    memcpy(o + 4, l1 + 8 * sl, 8);
                    for (int q = 0; q < 5; ++q) acc[q].add(o[q]);
                    vs = fmaxf(vs, o[5]);
                }
                for (int q = 0; q < 5; ++q) hst<float>(dst[q], p, acc[q].s);
                hst<float>(dst[5], p, vs);
            }
        }
    }
    return SPH_OK;
}

int host_init(sph_store s, int loop, int active_bin, int nthreads) {
    CompPtr out[8];
    int k = 0;
    if (loop == SPH_DENSITY) {
        for (int f : {F_RHO, F_RHODH, F_WCOUNT, F_WCOUNTDH, F_DIVV}) out[k++] = at(s, f, 0);
        for (int c = 0; c < 3; ++c) out[k++] = at(s, F_ROTV, c);
    } else if (loop == SPH_GRADIENT) {
        out[k++] = at(s, F_VSIGG, 0);
        out[k++] = at(s, F_LAPU, 0);
    } else {
        for (int c = 0; c < 3; ++c) out[k++] = at(s, F_A, c);
        for (int f : {F_UDT, F_HDT, F_VSIG}) out[k++] = at(s, f, 0);
    }
    const CompPtr tb = at(s, F_TBIN, 0);
    const int nout = k;
#pragma omp parallel for schedule(static) num_threads(threads(nthreads))
    for (int64_t p = 0; p < s->n; ++p) {
        if (loop == SPH_FORCE && (int)hld<int8_t>(tb, p) > active_bin) continue;
        for (int q = 0; q < nout; ++q) hst<float>(out[q], p, 0.f);
    }
    return SPH_OK;
}

// The linear update after density, in FP32 as on the device.
int host_ghost(sph_store s, float kernel_gamma, float gamma, float balsara_eps, int nthreads) {
    const int roles[14][2] = {{F_MASS, 0}, {F_H, 0}, {F_U, 0}, {F_RHO, 0}, {F_RHODH, 0},
                              {F_WCOUNT, 0}, {F_DIVV, 0}, {F_ROTV, 0}, {F_ROTV, 1},
                              {F_ROTV, 2}, {F_FGRADH, 0}, {F_PRES, 0}, {F_CS, 0},
                              {F_BALS, 0}};
    CompPtr f[14];
    for (int r = 0; r < 14; ++r) f[r] = at(s, roles[r][0], roles[r][1]);
    const float norm = 8.0f / 3.14159265358979323846f;
#pragma omp parallel for schedule(static) num_threads(threads(nthreads))
    for (int64_t p = 0; p < s->n; ++p) {
        const float m = hld<float>(f[0], p), h = hld<float>(f[1], p), u = hld<float>(f[2], p);
        const float H = kernel_gamma * h;
        const float Hinv = 1.f / H;
        const float Hinv3 = Hinv * Hinv * Hinv;
        const float rho = hld<float>(f[3], p) + m * norm * Hinv3;
        const float rho_dh = hld<float>(f[4], p) - 3.f * m * norm * Hinv3 * Hinv;
        const float wsum = hld<float>(f[5], p);
        const float wcount = wsum + 32.f / 3.f;
        const float rinv = 1.f / rho;
        const float div = hld<float>(f[6], p) * rinv;
        const float r0 = hld<float>(f[7], p) * rinv, r1 = hld<float>(f[8], p) * rinv,
                    r2 = hld<float>(f[9], p) * rinv;
        const float omega = 1.f + H * rho_dh * rinv * (1.f / 3.f);
        const float pres = (gamma - 1.f) * rho * u;
        const float cs = std::sqrt(gamma * (gamma - 1.f) * u);
        const float arot = std::sqrt(r0 * r0 + r1 * r1 + r2 * r2);
        const float adiv = std::fabs(div);
        const float bal = adiv / (adiv + arot + balsara_eps * cs / h);
        hst<float>(f[3], p, rho);
        hst<float>(f[4], p, rho_dh);
        hst<float>(f[5], p, wcount);
        hst<float>(f[6], p, div);
        hst<float>(f[7], p, r0);
        hst<float>(f[8], p, r1);
        hst<float>(f[9], p, r2);
        hst<float>(f[10], p, wsum == 0.f ? 1.f : 1.f / omega);   // no neighbour: Omega = 0
        hst<float>(f[11], p, pres);
        hst<float>(f[12], p, cs);
        hst<float>(f[13], p, bal);
    }
    return SPH_OK;
}

int host_copy_fields(sph_store s, const sph_fields *f, const int64_t *perm, int to_store,
                     int nthreads) {
    void *const *ptrs = reinterpret_cast<void *const *>(f);
    for (int fid = 0; fid < F_BALLAST; ++fid) {
        char *lp0 = (char *)ptrs[fid];
        if (!lp0) continue;
        const int elem = kFields[fid].elem, cnt = kFields[fid].count;
        for (int c = 0; c < cnt; ++c) {
            // into the store: every copy of a replicated field; out: the first
            CompPtr cp[4];
            const int ncopy = to_store ? locate_all(s->layout, s->mem, fid, c, cp, 4)
                                       : (int)locate(s->layout, s->mem, fid, c, cp);
            for (int q = 0; q < ncopy; ++q) {
                const CompPtr sp = cp[q];
#pragma omp parallel for schedule(static) num_threads(threads(nthreads))
                for (int64_t k = 0; k < s->n; ++k) {
                    const int64_t p = perm ? perm[k] : k;
                    char *lp = lp0 + p * (int64_t)(elem * cnt) + c * elem;
                    char *st = sp.ptr + k * sp.stride;
                    if (to_store) memcpy(st, lp, elem);
                    else memcpy(lp, st, elem);
                }
            }
        }
    }
    return SPH_OK;
}

}  // namespace sph
