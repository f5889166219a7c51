// Host side of the host-staged batched cycle (Sec. 2.3-2.5 applied to the
// cell-dedup bundles): the store lives in host memory, host threads pack each
// bundle's records (the same record lanes the device pack writes, with the
// particles of a cell in store order) into a pinned buffer and unpack each
// target particle's results back into the store.
#pragma once
#include <cmath>
#include <cstring>

#include <omp.h>

#include "batch_kernels.cuh"

namespace sph {

namespace hb {

template <typename T>
inline T hget(const CompPtr &c, int64_t p) {
    T v;
    memcpy(&v, c.ptr + p * c.stride, sizeof(T));
    return v;
}

template <typename T>
inline void hput(const CompPtr &c, int64_t p, T v) {
    memcpy(c.ptr + p * c.stride, &v, sizeof(T));
}

CompPtr hat(sph_store s, int field, int comp, int loop) {
    CompPtr c{nullptr, 0};
    locate_view(s->layout, s->mem, field, comp, loop, &c);
    return c;
}

// x = hi + lo with hi = x rounded to float and lo the rounded remainder
inline void split2(double x, float &hi, float &lo) {
    hi = (float)x;
    lo = (float)(x - (double)hi);
}

int nthr(int n) { return n > 0 ? n : omp_get_max_threads(); }

template <int LOOP>
void bpack(sph_store s, const sph_batch_s *b, int bundle, char *buf, const sph_params *p,
           int nthreads) {
    using BL = BLayout<LOOP>;
    constexpr int nf = BL::nf;
    const BatchBundle &bb = b->bundles[bundle];
    const int64_t S = bb.slots;
    float4 *rec[nf];
    for (int f = 0; f < nf; ++f) rec[f] = reinterpret_cast<float4 *>(buf + BL::rec(f, S));
    int32_t *perm = reinterpret_cast<int32_t *>(buf + BL::perm(S));
    int8_t *tb = reinterpret_cast<int8_t *>(buf + BL::tb(S));
    float *hf = reinterpret_cast<float *>(buf + BL::hf(S));
    float *cellh = reinterpret_cast<float *>(buf + BL::cellh(S));
    CompPtr x[3], v[3];
    for (int d = 0; d < 3; ++d) {
        x[d] = hat(s, F_X, d, LOOP);
        v[d] = hat(s, F_V, d, LOOP);
    }
    const CompPtr m = hat(s, F_MASS, 0, LOOP), h = hat(s, F_H, 0, LOOP), u = hat(s, F_U, 0, LOOP),
                  rho = hat(s, F_RHO, 0, LOOP), fgh = hat(s, F_FGRADH, 0, LOOP),
                  bal = hat(s, F_BALS, 0, LOOP), av = hat(s, F_AVISC, 0, LOOP),
                  ad = hat(s, F_ADIFF, 0, LOOP), tbin = hat(s, F_TBIN, 0, LOOP);
    const float kg = (float)p->kernel_gamma, gamma = (float)p->gamma;
    double bmax = std::max(b->box[0], std::max(b->box[1], b->box[2]));
    const float delta = (float)(4e-6 * bmax);
#pragma omp parallel for schedule(dynamic, 64) num_threads(nthr(nthreads))
    for (int64_t c = 0; c < bb.ncells; ++c) {
        const BCellDev C = b->cells[(size_t)(bb.cell0 + c)];
        float hmax = 0.f;
        for (int k = 0; k < C.n; ++k) {
            const int64_t pi = (int64_t)C.p0 + k, sl = (int64_t)C.slot + k;
            float hx, hy, hz, lx, ly, lz;
            split2(hget<double>(x[0], pi), hx, lx);
            split2(hget<double>(x[1], pi), hy, ly);
            split2(hget<double>(x[2], pi), hz, lz);
            const float hv = hget<float>(h, pi), mv = hget<float>(m, pi);
            const float H = kg * hv;
            hmax = std::max(hmax, H);
            float uv = LOOP == SPH_DENSITY ? 0.f : hget<float>(u, pi);
            float4 r[5];
            if (LOOP == SPH_FORCE) {
                const float Hp = H + delta;
                r[0] = make_float4(hx, hy, hz, Hp * Hp);
            } else {
                r[0] = make_float4(hx, hy, hz, H);
            }
            r[1] = make_float4(lx, ly, lz, mv);
            r[2] = make_float4(hget<float>(v[0], pi), hget<float>(v[1], pi),
                               hget<float>(v[2], pi), uv);
            if (LOOP == SPH_GRADIENT) {
                const float rh = hget<float>(rho, pi);
                const float cs = std::sqrt(gamma * (gamma - 1.f) * uv);
                r[3] = make_float4(rh, cs, mv / rh, 0.f);
            }
            if (LOOP == SPH_FORCE) {
                const float rh = hget<float>(rho, pi), f = hget<float>(fgh, pi);
                const float P = (gamma - 1.f) * rh * uv;
                const float cs = std::sqrt(gamma * (gamma - 1.f) * uv);
                r[3] = make_float4(rh, f * P / (rh * rh), cs, hget<float>(av, pi) * hget<float>(bal, pi));
                r[4] = make_float4(P, hget<float>(ad, pi), 1.f / H, H * H);
                tb[sl] = hget<int8_t>(tbin, pi);
                hf[sl] = hv * (f / rh);
            }
            for (int f = 0; f < nf; ++f) rec[f][sl] = r[f];
            perm[sl] = (int32_t)pi;
        }
        cellh[c] = hmax;
    }
}

template <int LOOP>
void bunpack(sph_store s, const sph_batch_s *b, int bundle, const char *out, int nthreads) {
    const BatchBundle &bb = b->bundles[bundle];
    const int64_t S = bb.slots;
    const int64_t r16 = (S * 16 + 255) / 256 * 256;
    CompPtr dst[8];
    int q = 0;
    if (LOOP == SPH_DENSITY) {
        for (int f : {F_RHO, F_RHODH, F_WCOUNT, F_WCOUNTDH, F_DIVV}) dst[q++] = hat(s, f, 0, -1);
        for (int c = 0; c < 3; ++c) dst[q++] = hat(s, F_ROTV, c, -1);
    } else if (LOOP == SPH_GRADIENT) {
        dst[q++] = hat(s, F_VSIGG, 0, -1);
        dst[q++] = hat(s, F_LAPU, 0, -1);
    } else {
        for (int c = 0; c < 3; ++c) dst[q++] = hat(s, F_A, c, -1);
        for (int f : {F_UDT, F_HDT, F_VSIG}) dst[q++] = hat(s, f, 0, -1);
    }
#pragma omp parallel for schedule(dynamic, 64) num_threads(nthr(nthreads))
    for (int64_t t = 0; t < bb.ntargets; ++t) {
        const BTargetDev &T = b->targets[(size_t)(bb.target0 + t)];
        const BCellDev C = b->cells[(size_t)(bb.cell0 + T.cell)];
        for (int k = 0; k < C.n; ++k) {
            const int64_t sl = (int64_t)C.slot + k, pi = (int64_t)C.p0 + k;
            if (LOOP == SPH_DENSITY) {
                float o[8];
                memcpy(o, out + 16 * sl, 16);
                memcpy(o + 4, out + r16 + 16 * sl, 16);
                for (int j = 0; j < 8; ++j) hput<float>(dst[j], pi, hget<float>(dst[j], pi) + o[j]);
            } else if (LOOP == SPH_GRADIENT) {
                float o[2];
                memcpy(o, out + 8 * sl, 8);
                hput<float>(dst[0], pi, std::fmax(hget<float>(dst[0], pi), o[0]));
                hput<float>(dst[1], pi, hget<float>(dst[1], pi) + o[1]);
            } else {
                float o[6];
                memcpy(o, out + 16 * sl, 16);
                memcpy(o + 4, out + r16 + 8 * sl, 8);
                for (int j = 0; j < 5; ++j) hput<float>(dst[j], pi, hget<float>(dst[j], pi) + o[j]);
                hput<float>(dst[5], pi, std::fmax(hget<float>(dst[5], pi), o[5]));
            }
        }
    }
}

}  // namespace hb

inline int host_batch_pack(sph_store s, const sph_batch_s *b, int loop, int bundle, char *buf,
                    const sph_params *p, int nthreads) {
    if (loop == SPH_DENSITY) hb::bpack<SPH_DENSITY>(s, b, bundle, buf, p, nthreads);
    else if (loop == SPH_GRADIENT) hb::bpack<SPH_GRADIENT>(s, b, bundle, buf, p, nthreads);
    else hb::bpack<SPH_FORCE>(s, b, bundle, buf, p, nthreads);
    return SPH_OK;
}

inline int host_batch_unpack(sph_store s, const sph_batch_s *b, int loop, int bundle, const char *out,
                      int nthreads) {
    if (loop == SPH_DENSITY) hb::bunpack<SPH_DENSITY>(s, b, bundle, out, nthreads);
    else if (loop == SPH_GRADIENT) hb::bunpack<SPH_GRADIENT>(s, b, bundle, out, nthreads);
    else hb::bunpack<SPH_FORCE>(s, b, bundle, out, nthreads);
    return SPH_OK;
}

inline int64_t host_batch_in_bytes(const sph_batch_s *b, int loop, int bundle) {
    const BatchBundle &bb = b->bundles[bundle];
    if (loop == SPH_DENSITY) return BLayout<SPH_DENSITY>::bytes(bb.slots, bb.ncells);
    if (loop == SPH_GRADIENT) return BLayout<SPH_GRADIENT>::bytes(bb.slots, bb.ncells);
    return BLayout<SPH_FORCE>::bytes(bb.slots, bb.ncells);
}

inline int64_t host_batch_out_bytes(const sph_batch_s *b, int loop, int bundle) {
    return bout_bytes(loop, b->bundles[bundle].slots);
}

}  // namespace sph
