// Batched (cell-dedup) pipeline kernels.
//
// k_bpack   one CTA per cell of the bundle: gathers the loop's view from the
//           store layout once per particle, splits positions into hi + lo
//           floats and derives the per-particle quantities (the same records
//           the per-task kernels stage in shared memory), and writes them in
//           octant order inside the cell so that 32 consecutive particles
//           are spatially compact.
// k_binteract persistent CTAs pull (target cell, particle chunk) items from
//           an atomic queue (items are sorted longest first).  For each of
//           the target's neighbour entries, tiles of j records are staged in shared
//           memory (the periodic shift added as an exact two-float sum); each
//           warp keeps only the j inside its particles' bounding box widened
//           by the support, tests those per lane, and runs the pair body on
//           the hits.  Each target particle's sums are written once.
// k_bunpack adds each target particle's result into the store.
#pragma once
#include "device.cuh"
#include "physics_kernels.cuh"
#include "store_kernels.cuh"

namespace sph {

constexpr int kBTile = 128;   // j records staged per tile (4 mask words)
constexpr int kBSortMax = 2048;  // cells larger than this keep store order

// Lanes of a batched pack buffer of S slots and C cells: nf record lanes
// (float4), for the density loop two more lanes holding its fixed-point
// gather record (fx), the store index of each slot (int32), the activity
// byte (force), h f / rho (force, for dh/dt), then the per-cell support
// maximum (float).
template <int LOOP>
struct BLayout {
    static constexpr int nf = NF<LOOP>::value;
    static constexpr int nlanes = LOOP == SPH_DENSITY ? nf + 2 : nf;
    static __host__ __device__ int64_t r256(int64_t b) { return (b + 255) / 256 * 256; }
    static __host__ __device__ int64_t rec(int f, int64_t S) { return r256(S * 16) * f; }
    static __host__ __device__ int64_t fx(int k, int64_t S) { return rec(nf + k, S); }
    static __host__ __device__ int64_t perm(int64_t S) { return rec(nlanes, S); }
    static __host__ __device__ int64_t tb(int64_t S) { return perm(S) + r256(S * 4); }
    static __host__ __device__ int64_t hf(int64_t S) { return tb(S) + r256(S); }
    static __host__ __device__ int64_t cellh(int64_t S) { return hf(S) + r256(S * 4); }
    static __host__ __device__ int64_t bytes(int64_t S, int64_t C) { return cellh(S) + r256(C * 4); }
};

inline int64_t bout_bytes(int loop, int64_t S) {
    auto r = [](int64_t b) { return (b + 255) / 256 * 256; };
    if (loop == SPH_DENSITY) return 2 * r(S * 16);
    if (loop == SPH_GRADIENT) return r(S * 8);
    return r(S * 16) + r(S * 8);
}

struct BPackArgs {
    const BCellDev *cells;
    char *buf;
    long long S;
    int ncells;           // cells of the bundle
    int min_n;            // k_bpack: cells with fewer particles are left to k_bpack_w
    double fx_scale[3];   // 2^32 / box edge: fixed-point position units
    CompPtr src[R_NUM];
    float kernel_gamma, gamma, delta;
};

// Source of a particle's view straight from the store layout.
struct StoreSrc {
    const BPackArgs &a;
    __device__ __forceinline__ void fields(long long p, double *x, float4 &vm, float &h, float &u,
                                           float &rho, float &fgh, float &bal, float &av,
                                           float &ad) const {
        for (int d = 0; d < 3; ++d) x[d] = ld<double>(a.src[R_X0 + d], p);
        vm = make_float4(ld<float>(a.src[R_V0], p), ld<float>(a.src[R_V1], p),
                         ld<float>(a.src[R_V2], p), ld<float>(a.src[R_M], p));
        h = ld<float>(a.src[R_H], p);
        u = ld<float>(a.src[R_U], p);
        rho = ld<float>(a.src[R_RHO], p);
        fgh = ld<float>(a.src[R_FGH], p);
        bal = ld<float>(a.src[R_BAL], p);
        av = ld<float>(a.src[R_AV], p);
        ad = ld<float>(a.src[R_AD], p);
    }
};

// Compact records of the neighbour-list loops, which gather whole j records
// per pair (fewer float4 lanes gathered; c and P are recomputed from u, rho;
// the compact density pack writes only its two fixed-point lanes):
//   gradient: [0] X m/rho  [1] v u  [2] H (own particle only, not gathered)
//   force:    [0] hi 1/H  [1] lo m  [2] v u  [3] rho  A = f P / rho^2  alpha_visc B  alpha_diff
// The density pack adds the density loop's gather record in its fx lanes
// (fx0 alone also serves the fixed-point list build):
//   [fx0] X H  [fx1] v m
// X is the position in 32-bit fixed point (x / box 2^32, modulo 2^32, the
// bits stored in the float slots): the difference of two such words, read as
// a signed integer, is the minimum-image separation in units of box / 2^32,
// exact before its conversion to float, so the periodic image comes for free.
__device__ __forceinline__ float fixed_coord(double x, double scale) {
    return __uint_as_float((unsigned int)(unsigned long long)__double2ll_rn(x * scale));
}
__device__ __forceinline__ float fixed_sep(float xi, float xj, float unit) {
    return (float)(int)(__float_as_uint(xi) - __float_as_uint(xj)) * unit;
}
template <int LOOP>
struct NFC {   // density: none besides the fixed-point lanes
    static constexpr int value = LOOP == SPH_DENSITY ? 0 : (LOOP == SPH_GRADIENT ? 3 : 4);
};

template <int LOOP, bool COMPACT = false>
__device__ __forceinline__ void make_record(const BPackArgs &a, long long p, float4 *r,
                                            float &hf) {
    double x[3];
    float4 vm;
    float h, u, rho, fgh, bal, av, ad;
    StoreSrc{a}.fields(p, x, vm, h, u, rho, fgh, bal, av, ad);
    float hx, hy, hz, lx, ly, lz;
    split_f64(x[0], hx, lx);
    split_f64(x[1], hy, ly);
    split_f64(x[2], hz, lz);
    const float H = a.kernel_gamma * h;
    if (LOOP == SPH_DENSITY) u = 0.f;
    if (COMPACT && LOOP != SPH_DENSITY) {
        hf = 0.f;
        if (LOOP == SPH_GRADIENT) {
            r[0] = make_float4(fixed_coord(x[0], a.fx_scale[0]), fixed_coord(x[1], a.fx_scale[1]),
                               fixed_coord(x[2], a.fx_scale[2]), vm.w / rho);
            r[1] = make_float4(vm.x, vm.y, vm.z, u);
            r[2] = make_float4(H, 0.f, 0.f, 0.f);
        } else {
            r[1] = make_float4(lx, ly, lz, vm.w);
            r[2] = make_float4(vm.x, vm.y, vm.z, u);
            const float P = (a.gamma - 1.f) * rho * u;
            r[0] = make_float4(hx, hy, hz, 1.f / H);
            r[3] = make_float4(rho, fgh * P / (rho * rho), av * bal, ad);
            hf = h * (fgh / rho);
        }
        return;
    }
    if (LOOP == SPH_FORCE) {
        const float Hp = H + a.delta;
        r[0] = make_float4(hx, hy, hz, Hp * Hp);
    } else {
        r[0] = make_float4(hx, hy, hz, H);
    }
    r[1] = make_float4(lx, ly, lz, vm.w);
    r[2] = make_float4(vm.x, vm.y, vm.z, u);
    hf = 0.f;
    if (LOOP == SPH_GRADIENT) {
        const float c = sqrtf(a.gamma * (a.gamma - 1.f) * u);
        r[3] = make_float4(rho, c, vm.w / rho, 0.f);
    }
    if (LOOP == SPH_FORCE) {
        const float P = (a.gamma - 1.f) * rho * u;
        const float c = sqrtf(a.gamma * (a.gamma - 1.f) * u);
        r[3] = make_float4(rho, fgh * P / (rho * rho), c, av * bal);
        r[4] = make_float4(P, ad, 1.f / H, H * H);
        hf = h * (fgh / rho);
    }
}

template <int LOOP, bool COMPACT = false>
__global__ void __launch_bounds__(128) k_bpack(BPackArgs a) {
    using BL = BLayout<LOOP>;
    constexpr int nf = COMPACT ? NFC<LOOP>::value : BL::nf;
    constexpr int kChunksMax = kBSortMax / 32;
    __shared__ float red[6][4];
    __shared__ float hred[4];
    __shared__ int hist[8 * kChunksMax];
    const BCellDev C = a.cells[blockIdx.x];
    if (C.n < a.min_n) return;   // a small cell: k_bpack_w packs it
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned int lt = (1u << lane) - 1u;
    const bool sort = C.n <= kBSortMax && C.n > 32;
    // pass A: bounding box of the cell's particles (hi parts) and max H
    float mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    float hmax = 0.f;
    for (int k = threadIdx.x; k < C.n; k += blockDim.x) {
        const long long p = (long long)C.p0 + k;
        for (int d = 0; d < 3; ++d) {
            float hi, lo;
            split_f64(ld<double>(a.src[R_X0 + d], p), hi, lo);
            mn[d] = fminf(mn[d], hi);
            mx[d] = fmaxf(mx[d], hi);
        }
        hmax = fmaxf(hmax, a.kernel_gamma * ld<float>(a.src[R_H], p));
    }
    for (int o = 16; o > 0; o >>= 1) {
        for (int d = 0; d < 3; ++d) {
            mn[d] = fminf(mn[d], __shfl_xor_sync(0xffffffffu, mn[d], o));
            mx[d] = fmaxf(mx[d], __shfl_xor_sync(0xffffffffu, mx[d], o));
        }
        hmax = fmaxf(hmax, __shfl_xor_sync(0xffffffffu, hmax, o));
    }
    if (lane == 0) {
        for (int d = 0; d < 3; ++d) {
            red[d][warp] = mn[d];
            red[3 + d][warp] = mx[d];
        }
        hred[warp] = hmax;
    }
    for (int e = threadIdx.x; e < 8 * kChunksMax; e += blockDim.x) hist[e] = 0;
    __syncthreads();
    float ctr[3];
    for (int d = 0; d < 3; ++d) {
        float lo = red[d][0], hi = red[3 + d][0];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
            lo = fminf(lo, red[d][w]);
            hi = fmaxf(hi, red[3 + d][w]);
        }
        ctr[d] = 0.5f * (lo + hi);
    }
    if (threadIdx.x == 0) {
        float hm = hred[0];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) hm = fmaxf(hm, hred[w]);
        reinterpret_cast<float *>(a.buf + BL::cellh(a.S))[blockIdx.x] = hm;
        // a support beyond what the plan was built for: the neighbour
        // entries may miss pairs (bit 3 of the error word, SPH_EUNSUPPORTED)
        if (hm > C.hlim) atomicOr(&g_error_word, 8u);
    }
    // octant key of particle k (0 when the cell keeps store order)
    auto key_of = [&](int k) -> int {
        const long long p = (long long)C.p0 + k;
        int key = 0;
        for (int d = 0; d < 3; ++d) {
            float hi, lo;
            split_f64(ld<double>(a.src[R_X0 + d], p), hi, lo);
            key |= (hi > ctr[d] ? 1 : 0) << d;
        }
        return key;
    };
    // pass B: per-chunk key counts (stable counting sort, chunks of 32)
    if (sort) {
        for (int c0 = warp * 32; c0 < C.n; c0 += blockDim.x) {
            const int k = c0 + lane;
            const int key = k < C.n ? key_of(k) : 8 + lane;
            const unsigned int peers = __match_any_sync(0xffffffffu, key);
            if (k < C.n && __popc(peers & lt) == 0) hist[key * kChunksMax + (c0 >> 5)] = __popc(peers);
        }
    }
    __syncthreads();
    if (sort && warp == 0) {
        // exclusive scan over (key, chunk), kChunksMax * 8 = 512 entries
        constexpr int per = 8 * kChunksMax / 32;
        int v[per], t = 0;
        for (int e = 0; e < per; ++e) {
            v[e] = hist[lane * per + e];
            t += v[e];
        }
        int incl = t;
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += u;
        }
        int run = incl - t;
        for (int e = 0; e < per; ++e) {
            hist[lane * per + e] = run;
            run += v[e];
        }
    }
    __syncthreads();
    // pass C: records at their sorted positions
    for (int c0 = warp * 32; c0 < C.n; c0 += blockDim.x) {
        const int k = c0 + lane;
        int pos = k;
        if (sort) {
            const int key = k < C.n ? key_of(k) : 8 + lane;
            const unsigned int peers = __match_any_sync(0xffffffffu, key);
            if (k < C.n) pos = hist[key * kChunksMax + (c0 >> 5)] + __popc(peers & lt);
        }
        if (k >= C.n) continue;
        const long long p = (long long)C.p0 + k;
        float4 r[BL::nf];
        float hf;
        make_record<LOOP, COMPACT>(a, p, r, hf);
        const long long sl = checked((long long)C.slot + pos, a.S);
        for (int f = 0; f < nf; ++f)
            reinterpret_cast<float4 *>(a.buf + BL::rec(f, a.S))[sl] = r[f];
        reinterpret_cast<int32_t *>(a.buf + BL::perm(a.S))[sl] = (int32_t)p;
        if (LOOP == SPH_DENSITY) {
            float X[3];
            for (int d = 0; d < 3; ++d) X[d] = fixed_coord(ld<double>(a.src[R_X0 + d], p), a.fx_scale[d]);
            reinterpret_cast<float4 *>(a.buf + BL::fx(0, a.S))[sl] = make_float4(X[0], X[1], X[2], r[0].w);
            reinterpret_cast<float4 *>(a.buf + BL::fx(1, a.S))[sl] = make_float4(r[2].x, r[2].y, r[2].z, r[1].w);
        }
        if (LOOP == SPH_FORCE) {
            reinterpret_cast<int8_t *>(a.buf + BL::tb(a.S))[sl] = ld<int8_t>(a.src[R_TB], p);
            reinterpret_cast<float *>(a.buf + BL::hf(a.S))[sl] = hf;
        }
    }
}

struct BInteractArgs {
    const BCellDev *cells;
    const BTargetDev *targets;
    const BNbrDev *nbrs;
    const BItemDev *items;
    unsigned int *counter;
    int nitems;
    const char *in;
    char *out;
    long long S;
    float kernel_gamma, gamma, beta, delta;
    float shift_hi[3], shift_lo[3];   // box edge as a two-float value
    float half[3];                    // half the box edge (image choice of the list loops)
    float fx_unit[3];                 // box edge / 2^32: one fixed-point position unit
    int active_bin;
    PhysArgs pa;  // parameters the pair bodies read (beta)
    // the FP64-separation list loops (precision study): each slot's position
    // in FP64 (three lanes), the box and half of it
    const double *xd[3];
    double box_d[3], half_d[3];
    // the symmetric list build: per entry its forward ordinal (naux), per
    // target its first mask word (mbase), mask words per entry and chunk
    const int32_t *naux;
    const long long *mbase;
    const RevEntDev *rev;      // per target, its backward neighbours (second pass)
    const int32_t *rev_start;
    int sym_words;
};

// a + b for two-float a and b (Knuth's TwoSum on the high parts); exact to
// about 2^-48 relative for the box shifts used here
__device__ __forceinline__ void add2(float &hi, float &lo, float bh, float bl) {
    const float s = hi + bh;
    const float bb = s - hi;
    const float err = (hi - (s - bb)) + (bh - bb);
    const float t = err + lo + bl;
    hi = s + t;
    lo = t - (hi - s);
}

// Warp-granular persistent kernel: every warp pulls its own (target cell,
// 32-particle chunk) item and stages neighbour tiles into its own slice of
// shared memory, so warps never wait for each other (no block barriers).
constexpr int kWTile = 64;  // j records a warp stages at a time (2 mask words)

#ifndef SPH_BMINB_FORCE
#define SPH_BMINB_FORCE 1024
#endif
// Warp-per-cell pack of the cells of at most kWPack particles: the records
// and slot order of k_bpack (the same bounding box, octant keys and stable
// counting order, so the same bits), with each particle's position loaded and
// split once and kept in registers, the octant ranks taken from ballots
// (per-row key counts packed bytewise in one 64-bit word, their prefix sums
// by one multiplication), and each record written by the lane of its slot,
// so consecutive lanes store consecutive slots.  Four cells per 128-thread
// CTA and no block barrier; larger cells are left to k_bpack.
constexpr int kWPack = 128;
constexpr int kWRows = kWPack / 32;

// Registers capped for 12 CTAs per SM: at Gresho256 the density pack ran
// 0.30 ms against 0.33 uncapped, and the gradient unpack with the force pack
// 0.53 against 0.56 ms (capped for 16 CTAs: 0.30 and 0.64 ms).
template <int LOOP, bool COMPACT = false>
__global__ void __launch_bounds__(128, 12) k_bpack_w(BPackArgs a) {
    using BL = BLayout<LOOP>;
    constexpr int nf = COMPACT ? NFC<LOOP>::value : BL::nf;
    __shared__ unsigned char inv_s[4][kWPack];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int cell = blockIdx.x * 4 + warp;
    if (cell >= a.ncells) return;
    const BCellDev C = a.cells[cell];
    if (C.n > kWPack || C.n <= 0) return;
    const unsigned int lt = (1u << lane) - 1u;
    const int rows = (C.n + 31) >> 5;
    // positions (hi parts) and the largest support; bounding box
    float hx[kWRows][3];
    float mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    float hmax = 0.f;
#pragma unroll
    for (int r = 0; r < kWRows; ++r) {
        const int k = r * 32 + lane;
        hx[r][0] = hx[r][1] = hx[r][2] = 0.f;
        if (r < rows && k < C.n) {
            const long long p = (long long)C.p0 + k;
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                float lo;
                split_f64(ld<double>(a.src[R_X0 + d], p), hx[r][d], lo);
                mn[d] = fminf(mn[d], hx[r][d]);
                mx[d] = fmaxf(mx[d], hx[r][d]);
            }
            hmax = fmaxf(hmax, a.kernel_gamma * ld<float>(a.src[R_H], p));
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            mn[d] = fminf(mn[d], __shfl_xor_sync(0xffffffffu, mn[d], o));
            mx[d] = fmaxf(mx[d], __shfl_xor_sync(0xffffffffu, mx[d], o));
        }
        hmax = fmaxf(hmax, __shfl_xor_sync(0xffffffffu, hmax, o));
    }
    if (lane == 0) {
        reinterpret_cast<float *>(a.buf + BL::cellh(a.S))[cell] = hmax;
        // a support beyond what the plan was built for (see k_bpack)
        if (hmax > C.hlim) atomicOr(&g_error_word, 8u);
    }
    // slot of each particle: stable counting order by octant key
    int pos[kWRows];
    if (C.n > 32) {
        float ctr[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) ctr[d] = 0.5f * (mn[d] + mx[d]);
        int key[kWRows];
        unsigned long long cnt[kWRows], total = 0ull;
#pragma unroll
        for (int r = 0; r < kWRows; ++r) {
            key[r] = 8;
            cnt[r] = 0ull;
            if (r < rows) {
                if (r * 32 + lane < C.n)
                    key[r] = (hx[r][0] > ctr[0] ? 1 : 0) | (hx[r][1] > ctr[1] ? 2 : 0) |
                             (hx[r][2] > ctr[2] ? 4 : 0);
#pragma unroll
                for (int q = 0; q < 8; ++q)
                    cnt[r] |= (unsigned long long)__popc(__ballot_sync(0xffffffffu, key[r] == q))
                              << (8 * q);
            }
            total += cnt[r];
        }
        // bytewise exclusive prefix over keys (every partial sum <= 128)
        const unsigned long long excl = total * 0x0101010101010101ull - total;
        unsigned long long before = 0ull;   // earlier rows' counts per key
#pragma unroll
        for (int r = 0; r < kWRows; ++r) {
            pos[r] = 0;
            if (r < rows) {
                const unsigned int peers = __match_any_sync(0xffffffffu, key[r]);
                if (key[r] < 8)
                    pos[r] = (int)((excl >> (8 * key[r])) & 0xffull) +
                             (int)((before >> (8 * key[r])) & 0xffull) + __popc(peers & lt);
            }
            before += cnt[r];
        }
    } else {
#pragma unroll
        for (int r = 0; r < kWRows; ++r) pos[r] = r * 32 + lane;
    }
#pragma unroll
    for (int r = 0; r < kWRows; ++r)
        if (r < rows && r * 32 + lane < C.n) inv_s[warp][pos[r]] = (unsigned char)(r * 32 + lane);
    __syncwarp();
    // records in slot order
#pragma unroll 1
    for (int r = 0; r < rows; ++r) {
        const int j = r * 32 + lane;
        if (j >= C.n) continue;
        const long long p = (long long)C.p0 + inv_s[warp][j];
        float4 rec[BL::nf];
        float hf;
        make_record<LOOP, COMPACT>(a, p, rec, hf);
        const long long sl = checked((long long)C.slot + j, a.S);
#pragma unroll
        for (int f = 0; f < nf; ++f)
            reinterpret_cast<float4 *>(a.buf + BL::rec(f, a.S))[sl] = rec[f];
        reinterpret_cast<int32_t *>(a.buf + BL::perm(a.S))[sl] = (int32_t)p;
        if (LOOP == SPH_DENSITY) {
            float X[3];
#pragma unroll
            for (int d = 0; d < 3; ++d)
                X[d] = fixed_coord(ld<double>(a.src[R_X0 + d], p), a.fx_scale[d]);
            reinterpret_cast<float4 *>(a.buf + BL::fx(0, a.S))[sl] =
                make_float4(X[0], X[1], X[2], rec[0].w);
            reinterpret_cast<float4 *>(a.buf + BL::fx(1, a.S))[sl] =
                make_float4(rec[2].x, rec[2].y, rec[2].z, rec[1].w);
        }
        if (LOOP == SPH_FORCE) {
            reinterpret_cast<int8_t *>(a.buf + BL::tb(a.S))[sl] = ld<int8_t>(a.src[R_TB], p);
            reinterpret_cast<float *>(a.buf + BL::hf(a.S))[sl] = hf;
        }
    }
}

template <int LOOP, int T>
__global__ void __launch_bounds__(T, (LOOP == SPH_FORCE ? SPH_BMINB_FORCE : 1024) / T)
    k_binteract(BInteractArgs a) {
    using BL = BLayout<LOOP>;
    constexpr int nf = NF<LOOP>::value;
    constexpr int kWarps = T / 32;
    __shared__ float4 smw[kWarps][nf][kWTile];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float4(*sm)[kWTile] = smw[warp];
    const float4 *rec[nf];
#pragma unroll
    for (int f = 0; f < nf; ++f) rec[f] = reinterpret_cast<const float4 *>(a.in + BL::rec(f, a.S));
    constexpr int kSelf = 1 | (1 << 2) | (1 << 4);
    for (;;) {
        int it = 0;
        if (lane == 0) it = (int)atomicAdd(a.counter, 1u);
        it = __shfl_sync(0xffffffffu, it, 0);
        if (it >= a.nitems) break;
        const BItemDev W = a.items[it];
        const int tcell = a.targets[W.target].cell;
        const BCellDev C = a.cells[tcell];
        const int i = W.i0 + lane;
        const bool valid = i < C.n;
        const long long slot = (long long)C.slot + i;
        float4 own[nf];
        Acc<LOOP> acc;
        bool active = false;
        if (valid) {
#pragma unroll
            for (int f = 0; f < nf; ++f) own[f] = rec[f][slot];
            acc.init(own, a.delta);
            active = LOOP != SPH_FORCE ||
                     (int)reinterpret_cast<const int8_t *>(a.in + BL::tb(a.S))[slot] <= a.active_bin;
        } else {
#pragma unroll
            for (int f = 0; f < nf; ++f) own[f] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        const bool live = valid && active;
        // warp bounding box of the live particles and its widest support
        float bmn[3], bmx[3], hw;
        {
            const float Hi = live ? (LOOP == SPH_FORCE ? sqrtf(own[0].w) : own[0].w + a.delta) : 0.f;
            bmn[0] = live ? own[0].x : INFINITY; bmx[0] = live ? own[0].x : -INFINITY;
            bmn[1] = live ? own[0].y : INFINITY; bmx[1] = live ? own[0].y : -INFINITY;
            bmn[2] = live ? own[0].z : INFINITY; bmx[2] = live ? own[0].z : -INFINITY;
            hw = Hi;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    bmn[d] = fminf(bmn[d], __shfl_xor_sync(0xffffffffu, bmn[d], o));
                    bmx[d] = fmaxf(bmx[d], __shfl_xor_sync(0xffffffffu, bmx[d], o));
                }
                hw = fmaxf(hw, __shfl_xor_sync(0xffffffffu, hw, o));
            }
        }
        const bool warp_live = __any_sync(0xffffffffu, live);
        const BTargetDev &Tg = a.targets[W.target];
#pragma unroll 1
        for (int e = Tg.nb0; e < Tg.nb0 + Tg.nnb && warp_live; ++e) {
            const BNbrDev E = a.nbrs[e];
            const int nb = E.cell;
            const BCellDev Cn = a.cells[nb];
            const int code = E.code;
            float sh[3], sl[3];
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                const int c = ((code >> (2 * d)) & 3) - 1;
                sh[d] = c == 0 ? 0.f : (c > 0 ? a.shift_hi[d] : -a.shift_hi[d]);
                sl[d] = c == 0 ? 0.f : (c > 0 ? a.shift_lo[d] : -a.shift_lo[d]);
            }
            float R = hw;
            if (LOOP == SPH_FORCE)
                R = fmaxf(hw, reinterpret_cast<const float *>(a.in + BL::cellh(a.S))[nb] + a.delta);
            const float R2 = R * R;
            const bool self = nb == tcell && code == kSelf;
#pragma unroll 1
            for (int j0 = 0; j0 < Cn.n; j0 += kWTile) {
                const int jn = min(kWTile, Cn.n - j0);
                __syncwarp();
                // stage: lane k loads records j0 + k and j0 + 32 + k; the box
                // test runs on the loaded positions (lanes over j)
                unsigned int cw[kWTile / 32];
#pragma unroll
                for (int w = 0; w < kWTile / 32; ++w) {
                    const int k = 32 * w + lane;
                    bool in = false;
                    if (k < jn) {
                        const long long js = (long long)Cn.slot + j0 + k;
                        float4 r0 = rec[0][js], r1 = rec[1][js];
                        if (code != kSelf) {
                            add2(r0.x, r1.x, sh[0], sl[0]);
                            add2(r0.y, r1.y, sh[1], sl[1]);
                            add2(r0.z, r1.z, sh[2], sl[2]);
                        }
                        sm[0][k] = r0;
                        sm[1][k] = r1;
#pragma unroll
                        for (int f = 2; f < nf; ++f) sm[f][k] = rec[f][js];
                        const float ex = fmaxf(fmaxf(bmn[0] - r0.x, r0.x - bmx[0]), 0.f);
                        const float ey = fmaxf(fmaxf(bmn[1] - r0.y, r0.y - bmx[1]), 0.f);
                        const float ez = fmaxf(fmaxf(bmn[2] - r0.z, r0.z - bmx[2]), 0.f);
                        in = ex * ex + ey * ey + ez * ez < R2;
                    }
                    cw[w] = __ballot_sync(0xffffffffu, in);
                }
                __syncwarp();
                // pass 1: lanes test the candidates (broadcast j), hits to masks
                unsigned int hm[kWTile / 32];
#pragma unroll
                for (int w = 0; w < kWTile / 32; ++w) {
                    unsigned int m = cw[w], h = 0;
                    while (m) {
                        const int b = __ffs(m) - 1;
                        m &= m - 1;
                        const float4 pj = sm[0][32 * w + b];
                        const float dx = own[0].x - pj.x, dy = own[0].y - pj.y,
                                    dz = own[0].z - pj.z;
                        const float r2 = dx * dx + dy * dy + dz * dz;
                        h |= acc.pre(r2, pj) ? (1u << b) : 0u;
                    }
                    if (self && (i - j0) >= 32 * w && (i - j0) < 32 * w + 32)
                        h &= ~(1u << (i - j0 - 32 * w));
                    hm[w] = live ? h : 0u;
                }
                // pass 2: the pair body on the hits
#pragma unroll 1
                for (int w = 0; w < kWTile / 32; ++w) {
                    unsigned int m = w == 0 ? hm[0] : hm[1];
                    while (m) {
                        const int j = 32 * w + (__ffs(m) - 1);
                        m &= m - 1;
                        float4 oth[nf];
#pragma unroll
                        for (int f = 0; f < nf; ++f) oth[f] = sm[f][j];
                        const float dx = (own[0].x - oth[0].x) + (own[1].x - oth[1].x);
                        const float dy = (own[0].y - oth[0].y) + (own[1].y - oth[1].y);
                        const float dz = (own[0].z - oth[0].z) + (own[1].z - oth[1].z);
                        const float r2 = dx * dx + dy * dy + dz * dz;
                        if (!acc.exact(r2, oth)) continue;
                        acc.body(own, oth, dx, dy, dz, r2, a.pa);
                    }
                }
            }
        }
        if (valid) {
            if constexpr (LOOP == SPH_DENSITY) {
                acc.write(PhysArgs{nullptr, {}, {a.out, a.out + BL::r256(a.S * 16)}}, slot, own);
            } else if constexpr (LOOP == SPH_GRADIENT) {
                acc.write(PhysArgs{nullptr, {}, {a.out, nullptr}}, slot, own);
            } else {
                float4 o0 = make_float4(0.f, 0.f, 0.f, 0.f);
                float2 o1 = make_float2(0.f, 0.f);
                if (active) {
                    const float hf = reinterpret_cast<const float *>(a.in + BL::hf(a.S))[slot];
                    o0 = make_float4(acc.ax, acc.ay, acc.az, acc.udt);
                    o1 = make_float2(-(1.f / 3.f) * hf * acc.hsum, acc.vsig);
                }
                reinterpret_cast<float4 *>(a.out)[slot] = o0;
                reinterpret_cast<float2 *>(a.out + BL::r256(a.S * 16))[slot] = o1;
            }
        }
    }
}

struct BUnpackArgs {
    const BCellDev *cells;
    const BTargetDev *targets;
    const char *out;
    const int32_t *perm;
    const int8_t *tb;   // force, WRITE: the pack's time-bin lane
    int active_bin;
    long long S;
    CompPtr dst[8];
    CompPtr gin[3];     // GHOST: mass, h, u
    CompPtr gout[4];    // GHOST: f_gradh, pressure, soundspeed, balsara
    float kernel_gamma, gamma, balsara_eps;
};

// One CTA per target cell.  Default: add each particle's result into the
// store (the single-term case of the per-task fold; maxima for signal
// velocities).  WRITE: store the result as that fold does onto a freshly
// initialised store (0 + v, max(0, v)), so no initialisation pass is needed:
// a batched plan gives every particle all its pairs in the one bundle that
// holds its cell as a target.  Inactive particles keep their force outputs,
// as the initialisation would have left them.  GHOST (density, WRITE): the
// ghost's arithmetic follows on the written sums, as sph_ghost would give.
template <int LOOP, bool WRITE = false, bool GHOST = false>
__global__ void __launch_bounds__(128) k_bunpack(BUnpackArgs a) {
    const BCellDev C = a.cells[a.targets[blockIdx.x].cell];
    const long long r16 = (a.S * 16 + 255) / 256 * 256;
    for (int k = threadIdx.x; k < C.n; k += blockDim.x) {
        const long long sl = checked((long long)C.slot + k, a.S);
        const long long p = a.perm[sl];
        auto base = [&](const CompPtr &d) { return WRITE ? 0.f : ld<float>(d, p); };
        if constexpr (LOOP == SPH_DENSITY) {
            const float4 o0 = reinterpret_cast<const float4 *>(a.out)[sl];
            const float4 o1 = reinterpret_cast<const float4 *>(a.out + r16)[sl];
            const float v[8] = {o0.x, o0.y, o0.z, o0.w, o1.x, o1.y, o1.z, o1.w};
            if constexpr (GHOST) {
                float sums[8], g[11];
#pragma unroll
                for (int q = 0; q < 8; ++q) sums[q] = 0.f + v[q];
                ghost_point(sums, ld<float>(a.gin[0], p), ld<float>(a.gin[1], p),
                            ld<float>(a.gin[2], p), a.kernel_gamma, a.gamma, a.balsara_eps, g);
                // dst: rho, rho_dh, wcount, wcount_dh, div_v, rot_v (3)
                st<float>(a.dst[0], p, g[0]);
                st<float>(a.dst[1], p, g[1]);
                st<float>(a.dst[2], p, g[2]);
                st<float>(a.dst[3], p, sums[3]);
#pragma unroll
                for (int q = 4; q < 8; ++q) st<float>(a.dst[q], p, g[q - 1]);
#pragma unroll
                for (int q = 0; q < 4; ++q) st<float>(a.gout[q], p, g[7 + q]);
            } else {
#pragma unroll
                for (int q = 0; q < 8; ++q) st<float>(a.dst[q], p, base(a.dst[q]) + v[q]);
            }
        } else if constexpr (LOOP == SPH_GRADIENT) {
            const float2 o = reinterpret_cast<const float2 *>(a.out)[sl];
            st<float>(a.dst[0], p, fmaxf(base(a.dst[0]), o.x));
            st<float>(a.dst[1], p, base(a.dst[1]) + o.y);
        } else {
            if (WRITE && (int)a.tb[sl] > a.active_bin) continue;
            const float4 o0 = reinterpret_cast<const float4 *>(a.out)[sl];
            const float2 o1 = reinterpret_cast<const float2 *>(a.out + r16)[sl];
            const float v[5] = {o0.x, o0.y, o0.z, o0.w, o1.x};
#pragma unroll
            for (int q = 0; q < 5; ++q) st<float>(a.dst[q], p, base(a.dst[q]) + v[q]);
            st<float>(a.dst[5], p, fmaxf(base(a.dst[5]), o1.y));
        }
    }
}

// The density unpack with the ghost when rho_dh, wcount, wcount_dh, div_v
// and rot_v are seven consecutive 4-byte words of one record (dst[1..7]; the
// by-type splits and the fused view) and no cell holds more than kUnpC
// particles: those seven words of the cell's particles go through shared
// memory in store order (a cell's particles are the store range
// [p0, p0 + n), its slots a permutation of it) and are written word after
// word, so a warp's stores cover whole sectors instead of one word in each
// of 32 records; rho and the ghost's four outputs are written directly.
// The values and bytes written are those of k_bunpack<density, write, ghost>.
constexpr int kUnpC = 128;
__global__ void __launch_bounds__(128) k_bunpack_dg(BUnpackArgs a) {
    __shared__ float sres[7 * kUnpC];
    const BCellDev C = a.cells[a.targets[blockIdx.x].cell];
    if (C.n > kUnpC) return;   // the caller launches this form only below the limit
    const long long r16 = (a.S * 16 + 255) / 256 * 256;
    for (int k = threadIdx.x; k < C.n; k += blockDim.x) {
        const long long sl = checked((long long)C.slot + k, a.S);
        const long long p = a.perm[sl];
        const float4 o0 = reinterpret_cast<const float4 *>(a.out)[sl];
        const float4 o1 = reinterpret_cast<const float4 *>(a.out + r16)[sl];
        float sums[8] = {0.f + o0.x, 0.f + o0.y, 0.f + o0.z, 0.f + o0.w,
                         0.f + o1.x, 0.f + o1.y, 0.f + o1.z, 0.f + o1.w};
        float g[11];
        ghost_point(sums, ld<float>(a.gin[0], p), ld<float>(a.gin[1], p), ld<float>(a.gin[2], p),
                    a.kernel_gamma, a.gamma, a.balsara_eps, g);
        st<float>(a.dst[0], p, g[0]);
#pragma unroll
        for (int q = 0; q < 4; ++q) st<float>(a.gout[q], p, g[7 + q]);
        // rho_dh, wcount, wcount_dh, div_v, rot_v: the words k_bunpack stores
        const float w7[7] = {g[1], g[2], sums[3], g[3], g[4], g[5], g[6]};
        const long long q = p - C.p0;
        if (q >= 0 && q < C.n) {
#pragma unroll
            for (int j = 0; j < 7; ++j) sres[7 * q + j] = w7[j];
        }
    }
    __syncthreads();
    char *base = a.dst[1].ptr + a.dst[1].stride * (long long)C.p0;
    const long long R = a.dst[1].stride;
    for (int w = threadIdx.x; w < 7 * C.n; w += blockDim.x) {
        const int q = w / 7, j = w - 7 * q;
        *reinterpret_cast<float *>(base + R * q + 4 * j) = sres[w];
    }
}

}  // namespace sph
