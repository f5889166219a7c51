// Interaction kernels of the three loops (Sec. 2.1) on packed bundles.
//
// One CTA per task.  A task whose slots fit in shared memory (kCap) is staged
// once, both cells together, as float4 structure-of-arrays so that every
// j-read is a conflict-free broadcast.  Thread "lanes" are assigned so that a
// warp never straddles the two cells of a pair task (the cells are padded to
// multiples of 32 in the virtual thread space), so all lanes of a warp run
// the same j-loop.  Larger tasks (clustered cells) take a tiled path that
// streams j-tiles through the same shared arrays.
//
// Precision: positions arrive in FP64.  Each slot's position is split once,
// with integer operations, into hi + lo floats; candidates are prefiltered
// with hi-only separations against a support widened by the hi rounding
// bound, and accepted pairs recompute dx = (hi_i - hi_j) + (lo_i - lo_j),
// which is the FP64 separation to FP32 rounding.  Everything else is FP32;
// the density sum is Kahan-compensated.  The B300's FP64 pipe is never used.
#pragma once
#include "device.cuh"

namespace sph {

struct PhysArgs {
    const TaskDev *tasks;
    const char *in[12];   // pack buffer lanes
    char *out[2];         // result lanes
    float kernel_gamma, gamma, beta, delta;  // delta: hi-rounding margin
    int active_bin;
    unsigned long long *count;
};

// Compile-time tuning knobs (defaults are the tuned configuration).
#ifndef SPH_KTHREADS
#define SPH_KTHREADS 128
#endif
#ifndef SPH_MINB_DENSITY
#define SPH_MINB_DENSITY 8
#endif
#ifndef SPH_MINB_GRADIENT
#define SPH_MINB_GRADIENT 8
#endif
#ifndef SPH_MINB_FORCE
#define SPH_MINB_FORCE 8
#endif
#ifndef SPH_KCHUNK
#define SPH_KCHUNK 64
#endif
constexpr int kThreads = SPH_KTHREADS;
constexpr int kCap = 256;
constexpr int kPad = 32;

template <int LOOP>
struct NF {
    static constexpr int value = LOOP == SPH_DENSITY ? 3 : (LOOP == SPH_GRADIENT ? 4 : 5);
};

// Staged slot record (float4 words):
//  [0] hi.x hi.y hi.z  w0     w0 = H (density, gradient) or (H + delta)^2 (force)
//  [1] lo.x lo.y lo.z  m
//  [2] v.x  v.y  v.z   u
//  [3] gradient: rho c  m/rho  0 ;  force: rho  A = f P / rho^2  c  alpha_visc * B
//  [4] force: P  alpha_diff  Hinv  H^2
template <int LOOP>
__device__ __forceinline__ void load_slot(const PhysArgs &a, long long s, float4 *r) {
    float hx, hy, hz, lx, ly, lz;
    split_f64(reinterpret_cast<const double *>(a.in[0])[s], hx, lx);
    split_f64(reinterpret_cast<const double *>(a.in[1])[s], hy, ly);
    split_f64(reinterpret_cast<const double *>(a.in[2])[s], hz, lz);
    const float4 vm = reinterpret_cast<const float4 *>(a.in[3])[s];
    const float H = a.kernel_gamma * reinterpret_cast<const float *>(a.in[4])[s];
    float u = 0.f;
    if (LOOP != SPH_DENSITY) u = reinterpret_cast<const float *>(a.in[5])[s];
    if (LOOP == SPH_FORCE) {
        const float Hp = H + a.delta;
        r[0] = make_float4(hx, hy, hz, Hp * Hp);
    } else {
        r[0] = make_float4(hx, hy, hz, H);
    }
    r[1] = make_float4(lx, ly, lz, vm.w);
    r[2] = make_float4(vm.x, vm.y, vm.z, u);
    if (LOOP == SPH_GRADIENT) {
        const float rho = reinterpret_cast<const float *>(a.in[6])[s];
        const float c = sqrtf(a.gamma * (a.gamma - 1.f) * u);
        r[3] = make_float4(rho, c, vm.w / rho, 0.f);
    }
    if (LOOP == SPH_FORCE) {
        const float rho = reinterpret_cast<const float *>(a.in[6])[s];
        const float fgh = reinterpret_cast<const float *>(a.in[7])[s];
        const float bal = reinterpret_cast<const float *>(a.in[8])[s];
        const float av = reinterpret_cast<const float *>(a.in[9])[s];
        const float ad = reinterpret_cast<const float *>(a.in[10])[s];
        const float P = (a.gamma - 1.f) * rho * u;
        const float c = sqrtf(a.gamma * (a.gamma - 1.f) * u);
        r[3] = make_float4(rho, fgh * P / (rho * rho), c, av * bal);
        r[4] = make_float4(P, ad, 1.f / H, H * H);
    }
}

// ---- per-i accumulators and pair bodies --------------------------------
template <int LOOP>
struct Acc;

template <>
struct Acc<SPH_DENSITY> {
    float sW, cW, sdh, swc, swcdh, sdiv, sr0, sr1, sr2;
    float Hi, Hinv, Hpre2, H2;
    __device__ __forceinline__ void init(const float4 *own, float delta) {
        sW = cW = sdh = swc = swcdh = sdiv = sr0 = sr1 = sr2 = 0.f;
        Hi = own[0].w;
        Hinv = 1.f / Hi;
        Hpre2 = (Hi + delta) * (Hi + delta);
        H2 = Hi * Hi;
    }
    __device__ __forceinline__ bool pre(float r2, const float4 &) const { return r2 < Hpre2; }
    __device__ __forceinline__ bool exact(float r2, const float4 *) const { return r2 < H2; }
    __device__ __forceinline__ void body(const float4 *own, const float4 *oth, float dx,
                                         float dy, float dz, float r2, const PhysArgs &) {
        const float rinv = r2 > 0.f ? rsqrtf(r2) : 0.f;
        const float r = r2 * rinv;
        // clamped at the support edge: the list loop's fixed-point separation
        // may round a pair the list admitted (r < H) to just past q = 1
        const float q = fminf(r * Hinv, 1.f);
        float w, dw;
        spline(q, w, dw);
        const float mj = oth[1].w;
        // compensated sum of m_j w
        const float y = fmaf(mj, w, -cW);
        const float t = sW + y;
        cW = (t - sW) - y;
        sW = t;
        sdh = fmaf(mj, fmaf(q, dw, 3.f * w), sdh);
        swc += w;
        swcdh = fmaf(q, dw, swcdh);
        const float dvx = own[2].x - oth[2].x, dvy = own[2].y - oth[2].y,
                    dvz = own[2].z - oth[2].z;
        const float mdw = mj * dw * rinv;
        sdiv = fmaf(mdw, dvx * dx + dvy * dy + dvz * dz, sdiv);
        sr0 = fmaf(mdw, dvy * dz - dvz * dy, sr0);
        sr1 = fmaf(mdw, dvz * dx - dvx * dz, sr1);
        sr2 = fmaf(mdw, dvx * dy - dvy * dx, sr2);
    }
    __device__ __forceinline__ void write(const PhysArgs &a, long long s, const float4 *) const {
        const float n3 = kNorm * Hinv * Hinv * Hinv;
        const float n4 = n3 * Hinv;
        reinterpret_cast<float4 *>(a.out[0])[s] =
            make_float4(n3 * sW, -n4 * sdh, (32.f / 3.f) * swc, -(32.f / 3.f) * Hinv * swcdh);
        reinterpret_cast<float4 *>(a.out[1])[s] =
            make_float4(-n4 * sdiv, n4 * sr0, n4 * sr1, n4 * sr2);
    }
};

template <>
struct Acc<SPH_GRADIENT> {
    float vsig, slap, ci, ui;
    float Hinv, Hpre2, H2;
    __device__ __forceinline__ void init(const float4 *own, float delta) {
        vsig = 0.f;
        slap = 0.f;
        const float Hi = own[0].w;
        Hinv = 1.f / Hi;
        Hpre2 = (Hi + delta) * (Hi + delta);
        H2 = Hi * Hi;
        ci = own[3].y;
        ui = own[2].w;
    }
    __device__ __forceinline__ bool pre(float r2, const float4 &) const { return r2 < Hpre2; }
    __device__ __forceinline__ bool exact(float r2, const float4 *) const { return r2 < H2; }
    __device__ __forceinline__ void body(const float4 *own, const float4 *oth, float dx,
                                         float dy, float dz, float r2, const PhysArgs &a) {
        const float rinv = r2 > 0.f ? rsqrtf(r2) : 0.f;
        const float q = r2 * rinv * Hinv;
        float w, dw;
        spline(q, w, dw);
        const float wdot = ((own[2].x - oth[2].x) * dx + (own[2].y - oth[2].y) * dy +
                            (own[2].z - oth[2].z) * dz) * rinv;
        const float vs = ci + oth[3].y - a.beta * fminf(0.f, wdot);
        vsig = fmaxf(vsig, vs);
        slap = fmaf(oth[3].z * (ui - oth[2].w), dw * rinv, slap);
    }
    __device__ __forceinline__ void write(const PhysArgs &a, long long s, const float4 *) const {
        const float n4 = kNorm * Hinv * Hinv * Hinv * Hinv;
        reinterpret_cast<float2 *>(a.out[0])[s] = make_float2(vsig, 2.f * n4 * slap);
    }
};

template <>
struct Acc<SPH_FORCE> {
    float ax, ay, az, udt, hsum, vsig;
    float Hpre2, H2, Hinv, n4i;
    __device__ __forceinline__ void init(const float4 *own, float) {
        ax = ay = az = udt = hsum = vsig = 0.f;
        Hpre2 = own[0].w;
        H2 = own[4].w;
        Hinv = own[4].z;
        n4i = kNorm * Hinv * Hinv * Hinv * Hinv;
    }
    __device__ __forceinline__ bool pre(float r2, const float4 &pj) const {
        return r2 < fmaxf(Hpre2, pj.w);
    }
    __device__ __forceinline__ bool exact(float r2, const float4 *oth) const {
        return r2 < fmaxf(H2, oth[4].w);
    }
    __device__ __forceinline__ void body(const float4 *own, const float4 *oth, float dx,
                                         float dy, float dz, float r2, const PhysArgs &a) {
        const float rinv = r2 > 0.f ? rsqrtf(r2) : 0.f;
        const float r = r2 * rinv;
        const float qi = r * Hinv;
        const float qj = r * oth[4].z;
        float w, dwi, dwj;
        spline(qi, w, dwi);
        if (!(qi < 1.f)) dwi = 0.f;
        spline(qj, w, dwj);
        if (!(qj < 1.f)) dwj = 0.f;
        const float hj = oth[4].z;
        const float Fi = n4i * dwi;
        const float Fj = kNorm * hj * hj * hj * hj * dwj;
        const float wdot = ((own[2].x - oth[2].x) * dx + (own[2].y - oth[2].y) * dy +
                            (own[2].z - oth[2].z) * dz) * rinv;
        const float mu = fminf(0.f, wdot);
        const float Fbar = 0.5f * (Fi + Fj);
        const float rhobar = 0.5f * (own[3].x + oth[3].x);
        const float rhobar_inv = 1.f / rhobar;
        const float alpha = 0.5f * (own[3].w + oth[3].w);
        const float vs = own[3].z + oth[3].z - a.beta * mu;
        const float Pi = -alpha * vs * mu * rhobar_inv;
        const float mj = oth[1].w;
        const float sc = own[3].y * Fi + oth[3].y * Fj + Pi * Fbar;
        const float f = mj * sc * rinv;
        ax = fmaf(-f, dx, ax);
        ay = fmaf(-f, dy, ay);
        az = fmaf(-f, dz, az);
        const float alphaD = 0.5f * (own[4].y + oth[4].y);
        const float cond = alphaD * sqrtf(fabsf(own[4].x - oth[4].x) * rhobar_inv) *
                           (own[2].w - oth[2].w) * Fbar * rhobar_inv;
        udt = fmaf(mj, fmaf(own[3].y * Fi, wdot, fmaf(0.5f * Pi * Fbar, wdot, cond)), udt);
        hsum = fmaf(mj * wdot, Fi, hsum);
        vsig = fmaxf(vsig, vs);
    }
    __device__ __forceinline__ void write(const PhysArgs &a, long long s, const float4 *own) const {
        // dh_i/dt = -(h_i / 3) f_i / rho_i sum_j m_j w F_i
        const float h = reinterpret_cast<const float *>(a.in[4])[s];
        const float fgh = reinterpret_cast<const float *>(a.in[7])[s];
        const float hdt = -(h * (1.f / 3.f)) * (fgh / own[3].x) * hsum;
        reinterpret_cast<float4 *>(a.out[0])[s] = make_float4(ax, ay, az, udt);
        reinterpret_cast<float2 *>(a.out[1])[s] = make_float2(hdt, vsig);
    }
};

// One i against j in [jb, je) (at most kCap) of a staged tile, skipping tile
// index `skip` (self task).  Pass 1 tests every candidate on hi-only
// separations and records hits as a per-lane bitmask; pass 2 visits only the
// hits, so a warp runs the pair body about max-over-lanes-of-hits times
// instead of once for every j that any lane accepts.
constexpr int kChunk = SPH_KCHUNK;  // candidates per bitmask pass (<= 4 words)
static_assert(kChunk % 32 == 0 && kChunk <= 128, "bitmask chunk is 1..4 words");

// Pass-1 test of one word (up to 32 candidates j0 .. j0+jn-1): bit b set if
// the hi-only separation passes the widened support test.
// The shared arrays carry one spare word (kPad) so a word may always be read
// whole; bits past jn are masked (their values are never used).
template <int LOOP>
__device__ __forceinline__ unsigned int test_word(const float4 (*sm)[kCap + kPad], int j0,
                                                  int jn, const float4 *own,
                                                  const Acc<LOOP> &acc) {
    unsigned int m = 0;
#pragma unroll
    for (int b = 0; b < 32; ++b) {
        const float4 pj = sm[0][j0 + b];
        const float dx = own[0].x - pj.x, dy = own[0].y - pj.y, dz = own[0].z - pj.z;
        const float r2 = dx * dx + dy * dy + dz * dz;
        m |= acc.pre(r2, pj) ? (1u << b) : 0u;
    }
    return jn < 32 ? m & ((1u << jn) - 1u) : m;
}

// One i against j in [jb, je) (at most kChunk) of a staged tile, skipping
// tile index `skip` (self task).  Pass 1 tests every candidate on hi-only
// separations and records hits as a per-lane bitmask; pass 2 visits only the
// hits, so a warp runs the pair body about max-over-lanes-of-hits times
// instead of once for every j that any lane accepts.  Loops over the mask
// words are not unrolled so the pair body is emitted once (instruction-cache
// footprint).
template <int LOOP, bool COUNT>
__device__ __forceinline__ void sweep_chunk(const float4 (*sm)[kCap + kPad], int jb, int je, int skip,
                                            const float4 *own, Acc<LOOP> &acc,
                                            unsigned int &cnt, const PhysArgs &a) {
    constexpr int nf = NF<LOOP>::value;
    unsigned int m0 = 0, m1 = 0, m2 = 0, m3 = 0;
#pragma unroll 1
    for (int w = 0; w < kChunk / 32; ++w) {
        const int j0 = jb + 32 * w;
        if (j0 >= je) break;
        unsigned int m = test_word<LOOP>(sm, j0, min(32, je - j0), own, acc);
        if (skip >= j0 && skip < j0 + 32) m &= ~(1u << (skip - j0));
        if (w == 0) m0 = m;
        else if (w == 1) m1 = m;
        else if (w == 2) m2 = m;
        else m3 = m;
    }
#pragma unroll 1
    for (int w = 0; w < kChunk / 32; ++w) {
        unsigned int m = w == 0 ? m0 : (w == 1 ? m1 : (w == 2 ? m2 : m3));
        while (m) {
            const int j = jb + 32 * w + (__ffs(m) - 1);
            m &= m - 1;
            float4 oth[nf];
#pragma unroll
            for (int f = 0; f < nf; ++f) oth[f] = sm[f][j];
            const float dx = (own[0].x - oth[0].x) + (own[1].x - oth[1].x);
            const float dy = (own[0].y - oth[0].y) + (own[1].y - oth[1].y);
            const float dz = (own[0].z - oth[0].z) + (own[1].z - oth[1].z);
            const float r2 = dx * dx + dy * dy + dz * dz;
            if (!acc.exact(r2, oth)) continue;
            if (COUNT) {
                cnt++;
            } else {
                acc.body(own, oth, dx, dy, dz, r2, a);
            }
        }
    }
}

template <int LOOP, bool COUNT>
__device__ __forceinline__ void sweep(const float4 (*sm)[kCap + kPad], int jb, int je, int skip,
                                      const float4 *own, Acc<LOOP> &acc,
                                      unsigned int &cnt, const PhysArgs &a) {
#pragma unroll 1
    for (int j0 = jb; j0 < je; j0 += kChunk)
        sweep_chunk<LOOP, COUNT>(sm, j0, min(j0 + kChunk, je), skip, own, acc, cnt, a);
}

// Out-of-line copy for the rare tiled path (cells of more than kCap / 2
// particles), so the common path keeps the only inlined pair body.
template <int LOOP, bool COUNT>
__device__ __noinline__ void sweep_tiled(const float4 (*sm)[kCap + kPad], int jn, int skip,
                                         const float4 *own, Acc<LOOP> *acc,
                                         unsigned int *cnt, const PhysArgs *a) {
    sweep<LOOP, COUNT>(sm, 0, jn, skip, own, *acc, *cnt, *a);
}

template <int LOOP, bool COUNT>
__device__ __forceinline__ void finish(const PhysArgs &a, long long slot, const float4 *own,
                                       const Acc<LOOP> &acc, bool active) {
    if (COUNT) return;
    if (LOOP == SPH_FORCE && !active) {
        reinterpret_cast<float4 *>(a.out[0])[slot] = make_float4(0.f, 0.f, 0.f, 0.f);
        reinterpret_cast<float2 *>(a.out[1])[slot] = make_float2(0.f, 0.f);
        return;
    }
    acc.write(a, slot, own);
}

template <int LOOP>
__device__ __forceinline__ bool is_active(const PhysArgs &a, long long s) {
    if (LOOP != SPH_FORCE) return true;
    return (int)reinterpret_cast<const int8_t *>(a.in[11])[s] <= a.active_bin;
}

// ---- projection binning of pair tasks -------------------------------------
// In a pair task every accepted j lies within |d| R of i along the cell
// offset d (R the support bound), and cj lies strictly beyond ci along every
// non-zero component of d.  Both cells are therefore sorted by their
// projection s = d . x into kBins bins (stable counting sort with warp
// ballots: deterministic), lanes take particles in sorted order, and each
// warp sweeps only a prefix of cj (lanes of ci: s_j <= s_i + R) or a suffix
// of ci (lanes of cj: s_j >= s_i - R).
constexpr int kBins = 16;
static_assert(kCap <= 2 * kThreads, "staging holds two slots per thread");

constexpr int kChunks = kCap / 32;   // 32-element chunks of a staged task
constexpr int kKeys = 2 * kBins;     // (side, bin)

struct SortSmem {
    float smin[kThreads / 32], smax[kThreads / 32], hmax[2][kThreads / 32];
    int hist[kKeys * kChunks];       // count of key in chunk, then its start
    short pos[kCap];
    short orig[kCap];
    int binstart[2][kBins + 1];
};

__device__ __forceinline__ int bin_of(float s, float s0, float inv_w) {
    const float f = (s - s0) * inv_w;
    return f <= 0.f ? 0 : (f >= (float)(kBins - 1) ? kBins - 1 : (int)f);
}

// Stable counting sort of the task's slots by key = (side, bin), all warps:
// chunk c = k / 32 is handled by the warp holding it; equal keys inside a
// chunk are ranked by lane with __match_any_sync, and chunk counts are
// scanned in (key, chunk) order.  Deterministic; side 0 lands in [0, ni),
// side 1 in [ni, n).
__device__ __forceinline__ void block_sort(SortSmem &S, int n, int ni, int nj,
                                           const int *key, int nk) {
    const int lane = threadIdx.x & 31;
    const unsigned int lt = (1u << lane) - 1u;
    int rank[2] = {0, 0};
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        if (q >= nk) break;
        const int k = threadIdx.x + q * kThreads;
        if (k - lane >= n) continue;  // whole chunk empty (warp-uniform)
        const int kk = k < n ? key[q] : kKeys + lane;  // unique sentinel
        const unsigned int peers = __match_any_sync(0xffffffffu, kk);
        rank[q] = __popc(peers & lt);
        if (k < n && rank[q] == 0) S.hist[kk * kChunks + (k >> 5)] = __popc(peers);
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        // exclusive scan of hist (kKeys * kChunks entries, 8 per lane)
        constexpr int per = kKeys * kChunks / 32;
        int v[per], t = 0;
#pragma unroll
        for (int e = 0; e < per; ++e) {
            v[e] = S.hist[lane * per + e];
            t += v[e];
        }
        int incl = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += u;
        }
        int run = incl - t;
#pragma unroll
        for (int e = 0; e < per; ++e) {
            S.hist[lane * per + e] = run;
            run += v[e];
        }
    }
    __syncthreads();
    if (threadIdx.x < kKeys) {
        const int side = threadIdx.x / kBins, b = threadIdx.x % kBins;
        S.binstart[side][b] = S.hist[threadIdx.x * kChunks] - (side ? ni : 0);
    }
    if (threadIdx.x == 0) {
        S.binstart[0][kBins] = ni;
        S.binstart[1][kBins] = nj;
    }
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        if (q >= nk) break;
        const int k = threadIdx.x + q * kThreads;
        if (k < n) S.pos[k] = (short)(S.hist[key[q] * kChunks + (k >> 5)] + rank[q]);
    }
}

template <int LOOP, bool COUNT>
__global__ void __launch_bounds__(kThreads, LOOP == SPH_FORCE ? SPH_MINB_FORCE
                                            : (LOOP == SPH_GRADIENT ? SPH_MINB_GRADIENT
                                                                    : SPH_MINB_DENSITY))
    k_interact(PhysArgs a) {
    constexpr int nf = NF<LOOP>::value;
    __shared__ float4 sm[nf][kCap + kPad];
    __shared__ SortSmem S;
    const TaskDev T = a.tasks[blockIdx.x];
    const int ni = T.ni, nj = T.nj, n = ni + nj;
    const long long base = T.slot;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned int cnt = 0;

    if (n <= kCap) {
        // ---- pair tasks: projection keys and a stable sort by bin ----------
        // (a light pass: positions and h only; each thread owns slots k0, k1)
        const int k0 = threadIdx.x, k1 = threadIdx.x + kThreads;
        float dn = 0.f, s_lo = 0.f, inv_w = 0.f, hm0 = 0.f, hm1 = 0.f;
        float dx = 0.f, dy = 0.f, dz = 0.f;
        if (nj > 0) {
            const int code = T.shift >> 6;
            dx = (float)((code & 3) - 1);
            dy = (float)(((code >> 2) & 3) - 1);
            dz = (float)(((code >> 4) & 3) - 1);
            dn = sqrtf(dx * dx + dy * dy + dz * dz);
            float sk[2] = {0.f, 0.f};
            float mn = INFINITY, mx = -INFINITY, h0 = 0.f, h1 = 0.f;
            for (int e = threadIdx.x; e < kKeys * kChunks; e += kThreads) S.hist[e] = 0;
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const int k = q ? k1 : k0;
                if (k >= n) continue;
                float hx, hy, hz, lo;
                split_f64(reinterpret_cast<const double *>(a.in[0])[base + k], hx, lo);
                split_f64(reinterpret_cast<const double *>(a.in[1])[base + k], hy, lo);
                split_f64(reinterpret_cast<const double *>(a.in[2])[base + k], hz, lo);
                sk[q] = dx * hx + dy * hy + dz * hz;
                mn = fminf(mn, sk[q]);
                mx = fmaxf(mx, sk[q]);
                if (LOOP == SPH_FORCE) {
                    const float H = a.kernel_gamma * reinterpret_cast<const float *>(a.in[4])[base + k];
                    if (k < ni) h0 = fmaxf(h0, H); else h1 = fmaxf(h1, H);
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
                mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
                h0 = fmaxf(h0, __shfl_xor_sync(0xffffffffu, h0, o));
                h1 = fmaxf(h1, __shfl_xor_sync(0xffffffffu, h1, o));
            }
            if (lane == 0) {
                S.smin[warp] = mn; S.smax[warp] = mx;
                S.hmax[0][warp] = h0; S.hmax[1][warp] = h1;
            }
            __syncthreads();
            mn = S.smin[0]; mx = S.smax[0]; h0 = S.hmax[0][0]; h1 = S.hmax[1][0];
#pragma unroll
            for (int w = 1; w < kThreads / 32; ++w) {
                mn = fminf(mn, S.smin[w]); mx = fmaxf(mx, S.smax[w]);
                h0 = fmaxf(h0, S.hmax[0][w]); h1 = fmaxf(h1, S.hmax[1][w]);
            }
            s_lo = mn;
            inv_w = mx > mn ? (float)kBins / (mx - mn) : 0.f;
            hm0 = h0;
            hm1 = h1;
            int key[2];
            key[0] = (k0 < ni ? 0 : kBins) + bin_of(sk[0], s_lo, inv_w);
            key[1] = (k1 < ni ? 0 : kBins) + bin_of(sk[1], s_lo, inv_w);
            block_sort(S, n, ni, nj, key, 2);
            __syncthreads();
        }
        // ---- stage full records at their sorted positions -----------------
        for (int k = threadIdx.x; k < n; k += kThreads) {
            float4 r[nf];
            load_slot<LOOP>(a, base + k, r);
            const int pk = nj > 0 ? S.pos[k] : k;
#pragma unroll
            for (int f = 0; f < nf; ++f) sm[f][pk] = r[f];
            S.orig[pk] = (short)k;
        }
        __syncthreads();

        // ---- sweep: lanes over sorted positions, warp-uniform sides --------
        const int ri = (ni + 31) & ~31;
        const int V = nj ? ri + ((nj + 31) & ~31) : ri;
        for (int v = threadIdx.x; v < V; v += kThreads) {
            const bool side = v >= ri;
            const int k = side ? v - ri : v;
            const bool valid = k < (side ? nj : ni);
            const int i = side ? ni + k : k;
            float4 own[nf];
            Acc<LOOP> acc;
            bool active = false;
            long long slot = 0;
            int jb, je;
            if (nj == 0) {
                jb = 0;
                je = ni;
            } else {
                jb = side ? 0 : ni;
                je = side ? ni : n;
            }
            if (valid) {
#pragma unroll
                for (int f = 0; f < nf; ++f) own[f] = sm[f][i];
                slot = base + (nj ? S.orig[i] : i);
                active = is_active<LOOP>(a, slot);
                acc.init(own, a.delta);
            }
            if (nj > 0) {
                // window of this lane along d, then the warp's union
                int lim = side ? ni : ni;  // empty for invalid / inactive lanes
                if (valid && active) {
                    const float Hs = LOOP == SPH_FORCE ? fmaxf(1.f / own[4].z, side ? hm0 : hm1)
                                                       : own[0].w;
                    const float R = dn * (Hs + a.delta);
                    const float si = dx * own[0].x + dy * own[0].y + dz * own[0].z;
                    if (!side) {
                        lim = ni + S.binstart[1][bin_of(si + R, s_lo, inv_w) + 1];
                    } else {
                        lim = S.binstart[0][bin_of(si - R, s_lo, inv_w)];
                    }
                }
                if (!side) je = __reduce_max_sync(0xffffffffu, lim);
                else jb = __reduce_min_sync(0xffffffffu, lim);
            }
            if (valid && active) {
                sweep<LOOP, COUNT>(sm, jb, je, nj == 0 ? i : -1, own, acc, cnt, a);
            }
            if (valid) finish<LOOP, COUNT>(a, slot, own, acc, active);
        }
    } else {
        // tiled path: phases (i-range, j-range), j streamed in kCap tiles
        const int nph = nj ? 2 : 1;
        for (int ph = 0; ph < nph; ++ph) {
            const int ib = ph == 0 ? 0 : ni, ie = ph == 0 ? ni : n;
            const int jb = nj ? (ph == 0 ? ni : 0) : 0, je = nj ? (ph == 0 ? n : ni) : ni;
            for (int i0 = ib; i0 < ie; i0 += kThreads) {
                const int i = i0 + threadIdx.x;
                const bool valid = i < ie;
                float4 own[nf];
                Acc<LOOP> acc;
                bool active = false;
                if (valid) {
                    load_slot<LOOP>(a, base + i, own);
                    acc.init(own, a.delta);
                    active = is_active<LOOP>(a, base + i);
                }
                for (int j0 = jb; j0 < je; j0 += kCap) {
                    const int jn = min(kCap, je - j0);
                    __syncthreads();
                    for (int k = threadIdx.x; k < jn; k += kThreads) {
                        float4 r[nf];
                        load_slot<LOOP>(a, base + j0 + k, r);
#pragma unroll
                        for (int f = 0; f < nf; ++f) sm[f][k] = r[f];
                    }
                    __syncthreads();
                    if (valid && active)
                        sweep_tiled<LOOP, COUNT>(sm, jn, nj ? -1 : i - j0, own, &acc, &cnt, &a);
                }
                if (valid) finish<LOOP, COUNT>(a, base + i, own, acc, active);
            }
        }
    }
    if (COUNT) {
        for (int off = 16; off > 0; off >>= 1) cnt += __shfl_down_sync(0xffffffffu, cnt, off);
        if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(a.count, (unsigned long long)cnt);
    }
}

}  // namespace sph
