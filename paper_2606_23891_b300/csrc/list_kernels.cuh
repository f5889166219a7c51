// Neighbour-list variant of the batched interaction kernels.
//
// The tile kernels (k_binteract) test every candidate of a target's neighbour
// entries (cells or leaves) again in each of the three loops, and run the pair
// body per lane over that lane's own hits, so lanes with fewer hits idle.
// Here the candidate tests run once per step:
//
// k_blist   persistent warps over the same work items: stage neighbour tiles,
//           cull by the warp box, prefilter on hi-only separations, take the
//           exact decision of both loop criteria (r < H_i for density and
//           gradient, r < max(H_i, H_j) for force) and append each accepted
//           j's bundle slot to the lane's list (the force loop's pairs; the
//           density and gradient loops keep those with r < H_i).  Lists are stored in chunks of 64 entries per lane for
//           the 32 lanes of an item (lane-interleaved, so the loops read them
//           coalesced); chunks come from a pool through an atomic counter
//           and are chained per item.  The content and order of each list
//           are fixed (neighbour entry, tile, slot order), only the chunks'
//           places in the pool vary, so results are reproducible.
// k_bloop   persistent warps over the items again: each lane walks its list,
//           gathers the j records of the loop's view from the bundle buffer
//           (read-only path, the list loads running ahead) and runs the pair
//           body.  Density and gradient gather two lanes per pair and take the
//           separation from 32-bit fixed-point positions, whose integer
//           difference is the minimum image; the force loop gathers its
//           two-float record and applies the periodic image shift (decided
//           from the hi-part separation: supports are below half the box, so
//           the image is unique) as an exact two-float add.
//           Lanes' lists differ in length by the neighbour-count scatter only.
//
// When the pool runs out, the build marks the list header and the error word
// (bit 2); the loops then skip all pairs and sph_sync reports it.
#pragma once
#include "batch_kernels.cuh"

namespace sph {

constexpr int kLPer = 64;                  // entries per lane per chunk
constexpr int kLChunk = 32 * kLPer;        // entries per chunk (8 KB)
constexpr int kLMaxChain = 256;            // chunks per item (16384 entries per lane)
constexpr uint32_t kLNone = 0xffffffffu;

struct ListHdr {
    unsigned long long chunks_used;  // chunks requested (counts past the pool too)
    unsigned int overflow;           // 1: the pool ran out, 2: an item's chain did
    unsigned int pad;
};

struct ListView {
    ListHdr *hdr;
    uint32_t *first;    // per plan item: first chunk (kLNone: empty)
    uint32_t *lcount;   // per plan item and lane: list length
    uint32_t *masks;    // symmetric build: hit masks of the forward cell pairs
    uint32_t *next;     // per chunk: next chunk of the same item
    uint32_t *entries;  // pool of chunks
    unsigned long long pool;
};

// Byte layout of a list buffer: header, first[NI], lcount[32 NI], masks[MW]
// (MW words, the symmetric build's; 0 otherwise), next[pool],
// entries[pool * kLChunk], each starting on a 256-byte boundary.
struct ListLayout {
    static int64_t r256(int64_t b) { return (b + 255) / 256 * 256; }
    static int64_t fixed(int64_t nitems, int64_t mwords) {
        return 256 + r256(4 * nitems) + r256(128 * nitems) + r256(4 * mwords);
    }
    static int64_t bytes(int64_t nitems, int64_t mwords, int64_t pool) {
        return fixed(nitems, mwords) + r256(4 * pool) + r256(4 * pool * kLChunk);
    }
    static int64_t pool_for(int64_t nitems, int64_t mwords, int64_t bytes) {
        int64_t p = (bytes - fixed(nitems, mwords)) / (4 + 4 * (int64_t)kLChunk);
        while (p > 0 && ListLayout::bytes(nitems, mwords, p) > bytes) --p;
        return p < 0 ? 0 : p;
    }
    static ListView view(void *base, int64_t nitems, int64_t mwords, int64_t bytes) {
        ListView v{};
        char *b = (char *)base;
        v.pool = (unsigned long long)pool_for(nitems, mwords, bytes);
        v.hdr = (ListHdr *)b;
        v.first = (uint32_t *)(b + 256);
        v.lcount = (uint32_t *)(b + 256 + r256(4 * nitems));
        v.masks = (uint32_t *)(b + 256 + r256(4 * nitems) + r256(128 * nitems));
        v.next = (uint32_t *)(b + fixed(nitems, mwords));
        v.entries = (uint32_t *)(b + fixed(nitems, mwords) + r256(4 * (int64_t)v.pool));
        return v;
    }
};

// ---------------------------------------------------------------- build --
// FIXED: positions from the density pack's fixed-point lane (X, H).  The
// prefilter and the box cull use floats relative to the item's first
// particle (the difference of fixed-point words is the minimum image, so no
// shift is applied).  The decisions are those of the fixed-point differences
// themselves: a hit whose relative-float separation lies a margin inside H_i
// meets both criteria there too and is accepted from the prefilter; only the
// others are tested on the fixed-point words.  Chosen by the plan when every cell or leaf extent plus the
// largest support stays below half the box: then the image nearest the
// item's first particle is the image nearest each of its particles for every
// pair that can interact, and no cell enters a target's entries twice.
// Otherwise the two-float path: hi/lo records, shifts by the entry codes.
// COUNT: the same build, also summing into cnt[0..4] the candidates staged,
// the (particle, candidate) pairs that pass the warp-box cull (each one
// prefiltered in pass 1), the pass-1 hits, the hits that take the exact
// test, and the entries written (a measurement variant; the timed build has
// COUNT = false and no counters).
// SYM (the symmetric build's first pass, one-bundle fixed-point grid plans):
// only the self entry and the forward entries (cells after the target) are
// tested; for each forward entry and tile the final hit masks are also
// stored, one word per lane and 32 candidates, where the second pass
// (k_blist_rev) of the other cell's items reads and transposes them.
// Registers are capped for 48 resident warps per SM (40 registers, 4 bytes
// spilled): the symmetric first pass ran 7.09 ms at Gresho256, against 7.33
// ms capped for 32 warps (58 registers) and 7.86 ms for 40 (48 registers).
template <int T, bool FIXED, bool COUNT = false, bool SYM = false>
__global__ void __launch_bounds__(T, 1536 / T) k_blist(BInteractArgs a, ListView L, long long item0,
                                                       unsigned long long *cnt) {
    using BL = BLayout<SPH_DENSITY>;
    constexpr int kWarps = T / 32;
    __shared__ float4 smw[kWarps][2][kWTile];
    __shared__ uint32_t chainw[kWarps][kLMaxChain];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float4(*sm)[kWTile] = smw[warp];
    uint32_t *chain = chainw[warp];
    const float4 *rec0 = reinterpret_cast<const float4 *>(a.in + BL::rec(0, a.S));
    const float4 *rec1 = reinterpret_cast<const float4 *>(a.in + BL::rec(1, a.S));
    const float *cellh = reinterpret_cast<const float *>(a.in + BL::cellh(a.S));
    constexpr int kSelf = 1 | (1 << 2) | (1 << 4);
    for (;;) {
        int it = 0;
        if (lane == 0) it = (int)atomicAdd(a.counter, 1u);
        it = __shfl_sync(0xffffffffu, it, 0);
        if (it >= a.nitems) break;
        const long long gitem = item0 + it;
        const BItemDev W = a.items[it];
        const int tcell = a.targets[W.target].cell;
        const BCellDev C = a.cells[tcell];
        const int i = W.i0 + lane;
        const bool valid = i < C.n;
        const long long slot = (long long)C.slot + i;
        float4 o0 = make_float4(0.f, 0.f, 0.f, 0.f), o1 = o0;
        const float4 *fxs = reinterpret_cast<const float4 *>(a.in + BL::fx(0, a.S));
        unsigned int rx = 0u, ry = 0u, rz = 0u;   // FIXED: the item's reference position
        if constexpr (FIXED) {
            if (valid) o1 = fxs[checked(slot, a.S)];   // (X, H) of this particle
            rx = __shfl_sync(0xffffffffu, __float_as_uint(o1.x), 0);
            ry = __shfl_sync(0xffffffffu, __float_as_uint(o1.y), 0);
            rz = __shfl_sync(0xffffffffu, __float_as_uint(o1.z), 0);
            o0 = make_float4(fixed_sep(o1.x, __uint_as_float(rx), a.fx_unit[0]),
                             fixed_sep(o1.y, __uint_as_float(ry), a.fx_unit[1]),
                             fixed_sep(o1.z, __uint_as_float(rz), a.fx_unit[2]), o1.w);
        } else if (valid) {
            o0 = rec0[checked(slot, a.S)];
            o1 = rec1[checked(slot, a.S)];
        }
        const float Hi = o0.w;
        const float H2i = Hi * Hi;
        const float Hpre = Hi + a.delta;
        const float Hpre2 = Hpre * Hpre;
        // FIXED: below (H_i - delta)^2 on the relative floats a pair is inside
        // H_i on the fixed-point separation too (their difference is a few
        // 1e-7 of the box, delta is 4e-6 of it), so it meets both criteria
        const float Hs = fmaxf(Hi - a.delta, 0.f);
        const float Hs2 = Hs * Hs;
        float bmn[3], bmx[3], hw;
        bmn[0] = valid ? o0.x : INFINITY; bmx[0] = valid ? o0.x : -INFINITY;
        bmn[1] = valid ? o0.y : INFINITY; bmx[1] = valid ? o0.y : -INFINITY;
        bmn[2] = valid ? o0.z : INFINITY; bmx[2] = valid ? o0.z : -INFINITY;
        hw = valid ? Hpre : 0.f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                bmn[d] = fminf(bmn[d], __shfl_xor_sync(0xffffffffu, bmn[d], o));
                bmx[d] = fmaxf(bmx[d], __shfl_xor_sync(0xffffffffu, bmx[d], o));
            }
            hw = fmaxf(hw, __shfl_xor_sync(0xffffffffu, hw, o));
        }
        int count = 0;      // this lane's entries
        unsigned int c_stage = 0, c_cull = 0, c_hit = 0, c_exact = 0;   // COUNT only
        int nch = 0;        // chunks of the item (warp-uniform)
        bool lost = false;  // the pool or the chain ran out (warp-uniform)
        const BTargetDev &Tg = a.targets[W.target];
#pragma unroll 1
        for (int e = Tg.nb0; e < Tg.nb0 + Tg.nnb; ++e) {
            const BNbrDev E = a.nbrs[e];
            const int nb = E.cell;
            uint32_t *mrow = nullptr;   // SYM, forward entry: this item's mask rows
            if constexpr (SYM) {
                if (nb < tcell) continue;   // the other cell's warps test this pair
                if (nb > tcell)
                    mrow = L.masks + a.mbase[tcell] +
                           ((long long)(W.i0 >> 5) * Tg.pad + a.naux[e]) * a.sym_words * 32;
            }
            const BCellDev Cn = a.cells[nb];
            const int code = E.code;
            float sh[3], sl[3];
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                const int c = ((code >> (2 * d)) & 3) - 1;
                sh[d] = c == 0 ? 0.f : (c > 0 ? a.shift_hi[d] : -a.shift_hi[d]);
                sl[d] = c == 0 ? 0.f : (c > 0 ? a.shift_lo[d] : -a.shift_lo[d]);
            }
            const float R = fmaxf(hw, cellh[nb] + a.delta);
            const float R2 = R * R;
            const bool self = nb == tcell && code == kSelf;
#pragma unroll 1
            for (int j0 = 0; j0 < Cn.n; j0 += kWTile) {
                const int jn = min(kWTile, Cn.n - j0);
                __syncwarp();
                // stage: positions with the shift added, (H_j + delta)^2 for the
                // prefilter in .w of the hi record and H_j^2 in .w of the lo one
                unsigned int cw[kWTile / 32];
#pragma unroll
                for (int w = 0; w < kWTile / 32; ++w) {
                    const int k = 32 * w + lane;
                    bool in = false;
                    if (k < jn) {
                        const long long js = checked((long long)Cn.slot + j0 + k, a.S);
                        float4 r0, r1;
                        if constexpr (FIXED) {
                            r1 = fxs[js];   // (X, H): the exact pass reads X back
                            r0 = make_float4(fixed_sep(r1.x, __uint_as_float(rx), a.fx_unit[0]),
                                             fixed_sep(r1.y, __uint_as_float(ry), a.fx_unit[1]),
                                             fixed_sep(r1.z, __uint_as_float(rz), a.fx_unit[2]),
                                             r1.w);
                        } else {
                            r0 = rec0[js];
                            r1 = rec1[js];
                            if (code != kSelf) {
                                add2(r0.x, r1.x, sh[0], sl[0]);
                                add2(r0.y, r1.y, sh[1], sl[1]);
                                add2(r0.z, r1.z, sh[2], sl[2]);
                            }
                        }
                        const float Hj = r0.w, Hjp = Hj + a.delta;
                        r1.w = Hj * Hj;
                        r0.w = Hjp * Hjp;
                        sm[0][k] = r0;
                        sm[1][k] = r1;
                        const float ex = fmaxf(fmaxf(bmn[0] - r0.x, r0.x - bmx[0]), 0.f);
                        const float ey = fmaxf(fmaxf(bmn[1] - r0.y, r0.y - bmx[1]), 0.f);
                        const float ez = fmaxf(fmaxf(bmn[2] - r0.z, r0.z - bmx[2]), 0.f);
                        in = ex * ex + ey * ey + ez * ez < R2;
                    }
                    cw[w] = __ballot_sync(0xffffffffu, in);
                    if constexpr (COUNT)
                        if (valid) c_cull += __popc(cw[w]);
                }
                if constexpr (COUNT) c_stage += (unsigned int)jn;
                __syncwarp();
                // pass 1: hi-only prefilter under the wider (force) criterion;
                // FIXED: also the hits certainly inside H_i
                unsigned int hm[kWTile / 32], sure[kWTile / 32];
                int nh = 0;
#pragma unroll
                for (int w = 0; w < kWTile / 32; ++w) {
                    unsigned int m = cw[w], h = 0, su = 0;
                    while (m) {     // two candidates per iteration (the second may repeat the first)
                        const int b = __ffs(m) - 1;
                        m &= m - 1;
                        const int b2 = m ? __ffs(m) - 1 : b;
                        m &= m - 1;
                        const float4 pj = sm[0][32 * w + b], pk = sm[0][32 * w + b2];
                        const float dx = o0.x - pj.x, dy = o0.y - pj.y, dz = o0.z - pj.z;
                        const float ex = o0.x - pk.x, ey = o0.y - pk.y, ez = o0.z - pk.z;
                        const float r2 = dx * dx + dy * dy + dz * dz;
                        const float s2 = ex * ex + ey * ey + ez * ez;
                        const unsigned int bj = 1u << b, bk = 1u << b2;
                        h |= (r2 < fmaxf(Hpre2, pj.w) ? bj : 0u) | (s2 < fmaxf(Hpre2, pk.w) ? bk : 0u);
                        if constexpr (FIXED) su |= (r2 < Hs2 ? bj : 0u) | (s2 < Hs2 ? bk : 0u);
                    }
                    if (self && (i - j0) >= 32 * w && (i - j0) < 32 * w + 32)
                        h &= ~(1u << (i - j0 - 32 * w));
                    hm[w] = valid ? h : 0u;
                    sure[w] = su & hm[w];
                    if constexpr (COUNT) {
                        c_hit += __popc(hm[w]);
                        c_exact += __popc(FIXED ? hm[w] & ~sure[w] : hm[w]);
                    }
                }
                // FIXED: the exact decisions on the other hits; hm keeps the
                // accepted ones, in slot order
#pragma unroll
                for (int w = 0; w < kWTile / 32; ++w) {
                    if constexpr (FIXED) {
                        unsigned int m = hm[w] & ~sure[w];
                        while (m) {
                            const int b = __ffs(m) - 1;
                            m &= m - 1;
                            const float4 p1 = sm[1][32 * w + b];
                            const float dx = fixed_sep(o1.x, p1.x, a.fx_unit[0]);
                            const float dy = fixed_sep(o1.y, p1.y, a.fx_unit[1]);
                            const float dz = fixed_sep(o1.z, p1.z, a.fx_unit[2]);
                            const float r2 = dx * dx + dy * dy + dz * dz;
                            if (!(r2 < fmaxf(H2i, p1.w))) hm[w] &= ~(1u << b);
                        }
                    }
                    nh += __popc(hm[w]);
                    if constexpr (SYM) {
                        const int wj = (j0 >> 5) + w;
                        if (mrow && wj * 32 < Cn.n) mrow[wj * 32 + lane] = hm[w];
                    }
                }
                // room for up to nh more entries in every lane's chain; once
                // an item is lost its further chunks are still counted, so the
                // header ends with the pool size a complete build needs
                const int need = __reduce_max_sync(0xffffffffu, count + nh);
                while (need > nch * kLPer) {
                    uint32_t c = kLNone;
                    if (lane == 0) {
                        const unsigned long long u = atomicAdd(&L.hdr->chunks_used, 1ull);
                        if (!lost && u < L.pool && nch < kLMaxChain) {
                            c = (uint32_t)u;
                            chain[nch] = c;
                            L.next[c] = kLNone;
                            if (nch > 0) L.next[chain[nch - 1]] = c;
                        } else if (!lost) {
                            atomicMax(&L.hdr->overflow, nch < kLMaxChain ? 1u : 2u);
                            atomicOr(&g_error_word, 4u);
                        }
                    }
                    c = __shfl_sync(0xffffffffu, c, 0);
                    __syncwarp();
                    if (c == kLNone) lost = true;
                    ++nch;
                }
                if constexpr (FIXED) {
                    // the accepted hits, appended in slot order
#pragma unroll
                    for (int w = 0; w < kWTile / 32; ++w) {
                        unsigned int m = hm[w];
                        while (m) {
                            const int b = __ffs(m) - 1;
                            m &= m - 1;
                            if (!lost) {
                                const uint32_t js = (uint32_t)(Cn.slot + j0 + 32 * w + b);
                                L.entries[checked(chain[count / kLPer], (long long)L.pool) * kLChunk +
                                          (count % kLPer) * 32 + lane] = js;
                            }
                            ++count;
                        }
                    }
                } else {
                    // exact two-float decisions on the hits, appended in slot order
#pragma unroll 1
                    for (int w = 0; w < kWTile / 32; ++w) {
                        unsigned int m = hm[w];
                        while (m) {
                            const int j = 32 * w + (__ffs(m) - 1);
                            m &= m - 1;
                            const float4 p0 = sm[0][j], p1 = sm[1][j];
                            const float dx = (o0.x - p0.x) + (o1.x - p1.x);
                            const float dy = (o0.y - p0.y) + (o1.y - p1.y);
                            const float dz = (o0.z - p0.z) + (o1.z - p1.z);
                            const float r2 = dx * dx + dy * dy + dz * dz;
                            if (!(r2 < fmaxf(H2i, p1.w))) continue;
                            if (!lost) {
                                const uint32_t js = (uint32_t)(Cn.slot + j0 + j);
                                L.entries[checked(chain[count / kLPer], (long long)L.pool) * kLChunk +
                                          (count % kLPer) * 32 + lane] = js;
                            }
                            ++count;
                        }
                    }
                }
            }
        }
        L.lcount[gitem * 32 + lane] = valid && !lost ? (uint32_t)count : 0u;
        if (lane == 0) L.first[gitem] = nch > 0 && !lost ? chain[0] : kLNone;
        if constexpr (COUNT) {
            const unsigned int ce = __reduce_add_sync(0xffffffffu, valid ? (unsigned int)count : 0u);
            const unsigned int cc = __reduce_add_sync(0xffffffffu, c_cull);
            const unsigned int ch = __reduce_add_sync(0xffffffffu, c_hit);
            const unsigned int cx = __reduce_add_sync(0xffffffffu, c_exact);
            if (lane == 0) {
                atomicAdd(&cnt[0], (unsigned long long)c_stage);
                atomicAdd(&cnt[1], (unsigned long long)cc);
                atomicAdd(&cnt[2], (unsigned long long)ch);
                atomicAdd(&cnt[3], (unsigned long long)cx);
                atomicAdd(&cnt[4], (unsigned long long)ce);
            }
        }
        __syncwarp();
    }
}

// Transpose of a 32 x 32 bit matrix held one row per lane (bit c of lane r
// is entry (r, c)): afterwards bit c of lane r is entry (c, r).  Five
// butterfly stages, each swapping the off-diagonal blocks of half the size
// between lane pairs.
__device__ __forceinline__ unsigned int warp_transpose32(unsigned int x, int lane) {
    const unsigned int mask[5] = {0x0000FFFFu, 0x00FF00FFu, 0x0F0F0F0Fu, 0x33333333u, 0x55555555u};
#pragma unroll
    for (int s = 0, j = 16; s < 5; ++s, j >>= 1) {
        const unsigned int m = mask[s];
        const unsigned int y = __shfl_xor_sync(0xffffffffu, x, j);
        x = (lane & j) ? ((x & ~m) | ((y >> j) & m)) : ((x & m) | ((y & m) << j));
    }
    return x;
}

// Second pass of the symmetric build: each item continues its lanes' lists
// (left by k_blist<.., SYM>) with its backward entries, the cells A before its
// target B.  A's warps stored, for each chunk of A and each chunk of B, the
// hits of A's particles (one word per A lane, bit b for B's particle b);
// transposed, lane b holds the A particles that hit its particle, appended
// in slot order.  The pair decisions are the first pass's: the same
// fixed-point words, the criterion r < max(H_i, H_j) is symmetric.
// Registers capped for 56 resident warps per SM (32 registers, no spill):
// the warps wait on their mask loads, and more of them hide it (Gresho256:
// 2.85 ms, against 3.13 capped for 48 and 3.24 for 32).
template <int T, bool COUNT = false>
__global__ void __launch_bounds__(T, 1792 / T) k_blist_rev(BInteractArgs a, ListView L,
                                                           long long item0,
                                                           unsigned long long *cnt) {
    constexpr int kWarps = T / 32;
    __shared__ uint32_t chainw[kWarps][kLMaxChain];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t *chain = chainw[warp];
    for (;;) {
        int it = 0;
        if (lane == 0) it = (int)atomicAdd(a.counter, 1u);
        it = __shfl_sync(0xffffffffu, it, 0);
        if (it >= a.nitems) break;
        const long long gitem = item0 + it;
        const BItemDev W = a.items[it];
        const BTargetDev &Tg = a.targets[W.target];
        const int tcell = Tg.cell;
        const BCellDev C = a.cells[tcell];
        const bool valid = W.i0 + lane < C.n;
        const int cB = W.i0 >> 5;
        int count = valid ? (int)L.lcount[gitem * 32 + lane] : 0;
        // the item's chain so far
        const int have = __reduce_max_sync(0xffffffffu, (unsigned)count);
        int nch = (have + kLPer - 1) / kLPer;
        bool lost = false;
        uint32_t c = L.first[gitem];
        if (nch > 0 && c == kLNone) lost = true;   // the first pass lost this item
        for (int k = 0; k < nch && !lost; ++k) {
            if (lane == 0) chain[k] = c;
            if (k + 1 < nch) c = L.next[checked(c, (long long)L.pool)];
        }
        __syncwarp();
        int added = 0;
        // the (backward neighbour, chunk of it) pairs in entry order, their
        // mask words loaded kRevBatch at a time so the loads are in flight
        // together (Gresho256 second pass, registers capped for 56 warps:
        // 2, 3, 4, 6 at a time gave 2.77, 2.84, 2.85, 2.89 ms)
        constexpr int kRevBatch = 2;
        const int rend = a.rev_start[W.target + 1];
        int r = a.rev_start[W.target], cA = 0;
        RevEntDev R{};
        if (r < rend) R = a.rev[r];
#pragma unroll 1
        while (r < rend) {
            unsigned int wd[kRevBatch];
            int slot0[kRevBatch];
            int nb = 0;
#pragma unroll
            for (int k = 0; k < kRevBatch; ++k) {
                wd[k] = 0u;
                slot0[k] = 0;
                if (r < rend) {
                    wd[k] = L.masks[R.mrow + (long long)cA * R.stride + cB * 32 + lane];
                    slot0[k] = R.slot + cA * 32;
                    nb = k + 1;
                    if (++cA * 32 >= R.n) {
                        cA = 0;
                        if (++r < rend) R = a.rev[r];
                    }
                }
            }
#pragma unroll
            for (int k = 0; k < kRevBatch; ++k) {
                if (k >= nb) break;
                unsigned int x = warp_transpose32(wd[k], lane);
                if (!valid) x = 0u;
                const int nh = __popc(x);
                const int need = __reduce_max_sync(0xffffffffu, count + nh);
                while (need > nch * kLPer) {
                    uint32_t cc = kLNone;
                    if (lane == 0) {
                        const unsigned long long u = atomicAdd(&L.hdr->chunks_used, 1ull);
                        if (!lost && u < L.pool && nch < kLMaxChain) {
                            cc = (uint32_t)u;
                            chain[nch] = cc;
                            L.next[cc] = kLNone;
                            if (nch > 0) L.next[chain[nch - 1]] = cc;
                        } else if (!lost) {
                            atomicMax(&L.hdr->overflow, nch < kLMaxChain ? 1u : 2u);
                            atomicOr(&g_error_word, 4u);
                        }
                    }
                    cc = __shfl_sync(0xffffffffu, cc, 0);
                    __syncwarp();
                    if (cc == kLNone) lost = true;
                    ++nch;
                }
                while (x) {
                    const int l = __ffs(x) - 1;
                    x &= x - 1;
                    if (!lost) {
                        const uint32_t js = (uint32_t)(slot0[k] + l);
                        L.entries[checked(chain[count / kLPer], (long long)L.pool) * kLChunk +
                                  (count % kLPer) * 32 + lane] = js;
                    }
                    ++count;
                    ++added;
                }
            }
        }
        L.lcount[gitem * 32 + lane] = valid && !lost ? (uint32_t)count : 0u;
        if (lane == 0) L.first[gitem] = nch > 0 && !lost ? chain[0] : kLNone;
        if constexpr (COUNT) {
            const unsigned int ce = __reduce_add_sync(0xffffffffu, valid ? (unsigned)added : 0u);
            if (lane == 0) atomicAdd(&cnt[4], (unsigned long long)ce);
        }
        __syncwarp();
    }
}

// ---------------------------------------------------------------- loops --
// Pair bodies of the gradient and force loops on compact records (the same
// sums as Acc<LOOP>, with c = sqrt(gamma (gamma - 1) u) and P = (gamma - 1)
// rho u recomputed from the gathered u and rho).
template <int LOOP>
struct AccL : Acc<LOOP> {};

template <>
struct AccL<SPH_GRADIENT> {
    float vsig, slap, ci, ui, Hinv, gg;
    __device__ __forceinline__ void init(const float4 *own, float, const PhysArgs &pa) {
        vsig = 0.f;
        slap = 0.f;
        Hinv = 1.f / own[0].w;
        gg = pa.gamma * (pa.gamma - 1.f);
        ui = own[2].w;
        ci = sqrtf(gg * ui);
    }
    __device__ __forceinline__ void body(const float4 *own, const float4 *oth, float dx,
                                         float dy, float dz, float r2, const PhysArgs &a) {
        const float rinv = r2 > 0.f ? rsqrtf(r2) : 0.f;
        // clamped: on two-float plans the list was decided on two-float
        // separations, and this fixed-point one may round a support-edge pair
        // to just past q = 1; on fixed-point plans the prefilter settles hits
        // on item-relative floats (inside H_i by a margin), and r * (1/H)
        // rounds again here, so the clamp stays as a guard
        const float qr = r2 * rinv * Hinv;
        const float q = fminf(qr, 1.f);
        float w, dw;
        spline(q, w, dw);
        const float wdot = ((own[2].x - oth[2].x) * dx + (own[2].y - oth[2].y) * dy +
                            (own[2].z - oth[2].z) * dz) * rinv;
        const float vs = ci + sqrtf(gg * oth[2].w) - a.beta * fminf(0.f, wdot);
        // the lists hold the force loop's pairs: the signal velocity takes
        // those inside H_i (the Laplacian's terms vanish beyond, dw(1) = 0)
        vsig = qr < 1.f ? fmaxf(vsig, vs) : vsig;
        slap = fmaf(oth[1].w * (ui - oth[2].w), dw * rinv, slap);
    }
    __device__ __forceinline__ void write(const PhysArgs &a, long long s, const float4 *) const {
        const float n4 = kNorm * Hinv * Hinv * Hinv * Hinv;
        reinterpret_cast<float2 *>(a.out[0])[s] = make_float2(vsig, 2.f * n4 * slap);
    }
};

template <>
struct AccL<SPH_FORCE> {
    float ax, ay, az, udt, hsum, vsig;
    float Hinv, n4i, gg, g1, ci, Pi_;
    __device__ __forceinline__ void init(const float4 *own, float, const PhysArgs &pa) {
        ax = ay = az = udt = hsum = vsig = 0.f;
        Hinv = own[0].w;
        n4i = kNorm * Hinv * Hinv * Hinv * Hinv;
        gg = pa.gamma * (pa.gamma - 1.f);
        g1 = pa.gamma - 1.f;
        ci = sqrtf(gg * own[2].w);
        Pi_ = g1 * own[3].x * own[2].w;
    }
    __device__ __forceinline__ void body(const float4 *own, const float4 *oth, float dx,
                                         float dy, float dz, float r2, const PhysArgs &a) {
        const float rinv = r2 > 0.f ? rsqrtf(r2) : 0.f;
        const float r = r2 * rinv;
        const float qi = r * Hinv;
        const float hj = oth[0].w;
        const float qj = r * hj;
        float w, dwi, dwj;
        spline(qi, w, dwi);
        if (!(qi < 1.f)) dwi = 0.f;
        spline(qj, w, dwj);
        if (!(qj < 1.f)) dwj = 0.f;
        const float Fi = n4i * dwi;
        const float Fj = kNorm * hj * hj * hj * hj * dwj;
        const float wdot = ((own[2].x - oth[2].x) * dx + (own[2].y - oth[2].y) * dy +
                            (own[2].z - oth[2].z) * dz) * rinv;
        const float mu = fminf(0.f, wdot);
        const float Fbar = 0.5f * (Fi + Fj);
        const float rhobar = 0.5f * (own[3].x + oth[3].x);
        const float rhobar_inv = 1.f / rhobar;
        const float alpha = 0.5f * (own[3].z + oth[3].z);
        const float cj = sqrtf(gg * oth[2].w);
        const float vs = ci + cj - a.beta * mu;
        const float Pv = -alpha * vs * mu * rhobar_inv;
        const float mj = oth[1].w;
        const float sc = own[3].y * Fi + oth[3].y * Fj + Pv * Fbar;
        const float f = mj * sc * rinv;
        ax = fmaf(-f, dx, ax);
        ay = fmaf(-f, dy, ay);
        az = fmaf(-f, dz, az);
        const float Pj = g1 * oth[3].x * oth[2].w;
        const float alphaD = 0.5f * (own[3].w + oth[3].w);
        const float cond = alphaD * sqrtf(fabsf(Pi_ - Pj) * rhobar_inv) *
                           (own[2].w - oth[2].w) * Fbar * rhobar_inv;
        udt = fmaf(mj, fmaf(own[3].y * Fi, wdot, fmaf(0.5f * Pv * Fbar, wdot, cond)), udt);
        hsum = fmaf(mj * wdot, Fi, hsum);
        vsig = fmaxf(vsig, vs);
    }
};

// WARPS: the resident warps per SM a list loop's registers are capped for
// (the launch fills each SM with as many CTAs as its registers allow).  The
// force loop holds its j record one pair ahead at 72 registers: 28 warps.
// The density and gradient loops wait on their gathers, so more resident
// warps pay as long as nothing spills: at Gresho256 the density loop runs
// 3.73 ms capped for 48 warps against 3.99 ms at its uncapped 48 registers
// (40 warps), the gradient loop (its j lanes one pair ahead) 3.58 ms capped
// for 40 against 3.66 ms at 56 registers and 3.67 ms capped for 48 (where
// it spills).  Holding them to fewer warps than the registers allow (28 to
// 36, by the grid size) was slower in every case.  Tree plans run both at
// 48 (the clustered lognormal set's lanes differ more in list length).
constexpr int kLLoopWarpsTree = 48, kLLoopWarpsForce = 28;
template <int LOOP>
constexpr int kLLoopWarpsGrid = LOOP == SPH_DENSITY ? 48 : LOOP == SPH_GRADIENT ? 40 : 28;
// SEP64 (the precision study of FP64 separations): every pair separation is
// the difference of the two FP64 positions (a.xd, gathered per slot by
// k_pack_x64), its periodic image chosen in FP64, then rounded to FP32; the
// rest of each pair body is unchanged.
__device__ __forceinline__ float sep64(double xi, double xj, double box, double half) {
    double d = xi - xj;
    if (d > half) d -= box;
    else if (d < -half) d += box;
    return (float)d;
}

// CH: one CTA per SM, whose warps share the work items of the CTA's chunks
// of kLoopChunk consecutive items (chunks dealt round-robin over the CTAs).
// Consecutive items are the chunks of neighbouring cells, so the warps of
// an SM gather overlapping neighbour records, which stay in its L1.
// Otherwise every warp takes the next item of the whole launch.
constexpr int kLoopChunk = 64;
template <int LOOP, int T, int WARPS, bool SEP64 = false, bool CH = false>
__global__ void __launch_bounds__(T, (LOOP == SPH_FORCE ? 28 : WARPS) * 32 / T)
    k_bloop(BInteractArgs a, ListView L, long long item0) {
    using BL = BLayout<LOOP>;
    // compact records (k_bpack<LOOP, true>); the density loop reads only its
    // fixed-point lanes and lays them out as the three-lane record its pair
    // body reads
    constexpr int nr = NFC<LOOP>::value;
    constexpr int nf = nr > 0 ? nr : 3;
    const int lane = threadIdx.x & 31;
    const float4 *rec[nf];
#pragma unroll
    for (int f = 0; f < nf; ++f) rec[f] = reinterpret_cast<const float4 *>(a.in + BL::rec(f, a.S));
    // the two gathered lanes of the density and gradient loops: a fixed-point
    // position with one scalar, and v with one scalar (see the records)
    const float4 *g0 = LOOP == SPH_DENSITY
                           ? reinterpret_cast<const float4 *>(a.in + BLayout<SPH_DENSITY>::fx(0, a.S))
                           : rec[0];
    const float4 *g1 = LOOP == SPH_DENSITY
                           ? reinterpret_cast<const float4 *>(a.in + BLayout<SPH_DENSITY>::fx(1, a.S))
                           : rec[1 % nf];
    const bool broken = L.hdr->overflow != 0u;
    __shared__ unsigned int s_tick;
    if constexpr (CH) {
        if (threadIdx.x == 0) s_tick = 0u;
        __syncthreads();
    }
    for (;;) {
        int it = 0;
        if constexpr (CH) {
            unsigned int t = 0u;
            if (lane == 0) t = atomicAdd(&s_tick, 1u);
            t = __shfl_sync(0xffffffffu, t, 0);
            const long long item = ((long long)blockIdx.x + (long long)(t / kLoopChunk) * gridDim.x) *
                                       kLoopChunk + t % kLoopChunk;
            if (item >= a.nitems) break;
            it = (int)item;
        } else {
            if (lane == 0) it = (int)atomicAdd(a.counter, 1u);
            it = __shfl_sync(0xffffffffu, it, 0);
            if (it >= a.nitems) break;
        }
        const long long gitem = item0 + it;
        const BItemDev W = a.items[it];
        const BCellDev C = a.cells[a.targets[W.target].cell];
        const int i = W.i0 + lane;
        const bool valid = i < C.n;
        const long long slot = (long long)C.slot + i;
        float4 own[nf];
        float ox = 0.f, oy = 0.f, oz = 0.f;  // own fixed-point position (density, gradient)
        double xi[3] = {0.0, 0.0, 0.0};      // SEP64: own FP64 position
        if constexpr (SEP64)
            if (valid)
                for (int d = 0; d < 3; ++d) xi[d] = a.xd[d][checked(slot, a.S)];
        AccL<LOOP> acc;
        bool active = false;
        if (valid) {
#pragma unroll
            for (int f = 0; f < nr; ++f) own[f] = rec[f][checked(slot, a.S)];
            if constexpr (LOOP == SPH_GRADIENT) {
                // to the record form the pair body reads: [0].w H, [1].w m/rho, [2] v u
                const float4 r0 = own[0], r1 = own[1], r2 = own[2];
                ox = r0.x;
                oy = r0.y;
                oz = r0.z;
                own[0] = make_float4(0.f, 0.f, 0.f, r2.x);
                own[1] = make_float4(0.f, 0.f, 0.f, r0.w);
                own[2] = r1;
            } else if constexpr (LOOP == SPH_DENSITY) {
                // [0].w H, [2] v: the fields the density body reads of its own
                const float4 X = g0[checked(slot, a.S)], V = g1[checked(slot, a.S)];
                ox = X.x;
                oy = X.y;
                oz = X.z;
                own[0] = make_float4(0.f, 0.f, 0.f, X.w);
                own[1] = make_float4(0.f, 0.f, 0.f, V.w);
                own[2] = make_float4(V.x, V.y, V.z, 0.f);
            }
            if constexpr (LOOP == SPH_DENSITY) acc.init(own, a.delta);
            else acc.init(own, a.delta, a.pa);
            active = LOOP != SPH_FORCE ||
                     (int)reinterpret_cast<const int8_t *>(a.in + BL::tb(a.S))[slot] <= a.active_bin;
        } else {
#pragma unroll
            for (int f = 0; f < nf; ++f) own[f] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        const int cnt = valid && active && !broken ? (int)L.lcount[gitem * 32 + lane] : 0;
        const int maxc = __reduce_max_sync(0xffffffffu, (unsigned)cnt);
        uint32_t chunk = L.first[gitem];
        int kl = 0;  // next list position to load
        auto next_ent = [&]() -> uint32_t {
            uint32_t e = 0u;
            if (kl < cnt)
                e = __ldg(&L.entries[checked(chunk, (long long)L.pool) * kLChunk +
                                     (kl % kLPer) * 32 + lane]);
            ++kl;
            if (kl % kLPer == 0 && kl < maxc) chunk = L.next[chunk];
            return e;
        };
        auto uses = [&](uint32_t, int k) { return k < cnt; };
        auto gather = [&](float4 *o, uint32_t e) {
#pragma unroll
            for (int f = 0; f < nf; ++f) o[f] = __ldg(&rec[f][checked(e, a.S)]);
        };
        auto pair = [&](float4 *oth, long long js) {
            if constexpr (SEP64) {
                const float dx = sep64(xi[0], a.xd[0][js], a.box_d[0], a.half_d[0]);
                const float dy = sep64(xi[1], a.xd[1][js], a.box_d[1], a.half_d[1]);
                const float dz = sep64(xi[2], a.xd[2][js], a.box_d[2], a.half_d[2]);
                acc.body(own, oth, dx, dy, dz, dx * dx + dy * dy + dz * dz, a.pa);
                return;
            }
            // periodic image: the hi-part separation exceeds half the box
            const float ax = own[0].x - oth[0].x, ay = own[0].y - oth[0].y,
                        az = own[0].z - oth[0].z;
            // (one test on the common path; the shift itself is rare)
            if (fabsf(ax) > a.half[0] || fabsf(ay) > a.half[1] || fabsf(az) > a.half[2]) {
                if (ax > a.half[0]) add2(oth[0].x, oth[1].x, a.shift_hi[0], a.shift_lo[0]);
                else if (ax < -a.half[0]) add2(oth[0].x, oth[1].x, -a.shift_hi[0], -a.shift_lo[0]);
                if (ay > a.half[1]) add2(oth[0].y, oth[1].y, a.shift_hi[1], a.shift_lo[1]);
                else if (ay < -a.half[1]) add2(oth[0].y, oth[1].y, -a.shift_hi[1], -a.shift_lo[1]);
                if (az > a.half[2]) add2(oth[0].z, oth[1].z, a.shift_hi[2], a.shift_lo[2]);
                else if (az < -a.half[2]) add2(oth[0].z, oth[1].z, -a.shift_hi[2], -a.shift_lo[2]);
            }
            const float dx = (own[0].x - oth[0].x) + (own[1].x - oth[1].x);
            const float dy = (own[0].y - oth[0].y) + (own[1].y - oth[1].y);
            const float dz = (own[0].z - oth[0].z) + (own[1].z - oth[1].z);
            const float r2 = dx * dx + dy * dy + dz * dz;
            acc.body(own, oth, dx, dy, dz, r2, a.pa);
        };
        // The entry loads run ahead of the gathers they feed: one list
        // position ahead in the density and gradient loops; in the force loop
        // the entries run two ahead and the j record one ahead, which the
        // force body's registers leave room for at 28 warps per SM.
        if constexpr (LOOP == SPH_FORCE) {
            uint32_t e = next_ent();
            float4 nxt[nf];
            bool un = uses(e, 0);
            if (un) gather(nxt, e);
            long long jn = e;
            e = next_ent();
#pragma unroll 1
            for (int k = 0; k < maxc; ++k) {
                float4 oth[nf];
#pragma unroll
                for (int f = 0; f < nf; ++f) oth[f] = nxt[f];
                const bool u = un;
                const long long jc = jn;
                un = uses(e, k + 1);
                if (un) gather(nxt, e);
                jn = e;
                e = next_ent();
                if (u) pair(oth, checked(jc, a.S));
            }
        } else {
            // density and gradient: two gathered lanes per pair; the
            // separation from the fixed-point positions (minimum image by the
            // integer wrap-around).  The lists hold the force loop's pairs
            // (r < max(H_i, H_j)); a pair beyond H_i adds nothing to these
            // sums (q is clamped to 1, where w and dw vanish) and the
            // gradient's signal velocity takes only those inside H_i.
            // The gradient loop on grid plans loads the two lanes of the next
            // pair one pair ahead (its list entry two ahead): 3.66 against
            // 3.79 ms at Gresho256.  The density loop lost that way (4.72
            // against 3.99 ms) and loads them when it uses them.
            constexpr bool kAhead = LOOP == SPH_GRADIENT && WARPS < 48;   // (spills at 48)
            auto gather2 = [&](uint32_t en, float4 &q0, float4 &q1) {
                const long long jq = checked(en, a.S);
                q0 = (SEP64 && LOOP == SPH_DENSITY) ? make_float4(0.f, 0.f, 0.f, 0.f)
                                                     : __ldg(&g0[jq]);
                q1 = __ldg(&g1[jq]);
            };
            uint32_t e = next_ent(), ncur = e;
            bool nu = false;
            float4 n0 = make_float4(0.f, 0.f, 0.f, 0.f), n1 = n0;
            if constexpr (kAhead) {
                nu = uses(e, 0);
                if (nu) gather2(e, n0, n1);
                e = next_ent();
            }
#pragma unroll 1
            for (int k = 0; k < maxc; ++k) {
                uint32_t cur;
                float4 j0, j1;
                if constexpr (kAhead) {
                    cur = ncur;
                    j0 = n0;
                    j1 = n1;
                    const bool u = nu;
                    nu = uses(e, k + 1);
                    ncur = e;
                    if (nu) gather2(e, n0, n1);
                    e = next_ent();
                    if (!u) continue;
                } else {
                    cur = e;
                    e = next_ent();
                    if (!uses(cur, k)) continue;
                    gather2(cur, j0, j1);
                }
                const long long js = checked(cur, a.S);
                float dx, dy, dz;
                if constexpr (SEP64) {
                    dx = sep64(xi[0], a.xd[0][js], a.box_d[0], a.half_d[0]);
                    dy = sep64(xi[1], a.xd[1][js], a.box_d[1], a.half_d[1]);
                    dz = sep64(xi[2], a.xd[2][js], a.box_d[2], a.half_d[2]);
                } else {
                    dx = fixed_sep(ox, j0.x, a.fx_unit[0]);
                    dy = fixed_sep(oy, j0.y, a.fx_unit[1]);
                    dz = fixed_sep(oz, j0.z, a.fx_unit[2]);
                }
                float4 oth[nf];
                oth[0] = make_float4(0.f, 0.f, 0.f, 0.f);
                // m_j (density: fx1.w) or m_j / rho_j (gradient: record 0 .w)
                oth[1] = make_float4(0.f, 0.f, 0.f, LOOP == SPH_DENSITY ? j1.w : j0.w);
                oth[2] = j1;
                const float r2 = dx * dx + dy * dy + dz * dz;
                acc.body(own, oth, dx, dy, dz, r2, a.pa);
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

// The FP64 positions of a bundle's slots for the SEP64 loops: slot sl
// holds store particle perm[sl] (the pack's store-index lane).
__global__ void __launch_bounds__(256) k_pack_x64(const int32_t *perm, long long S, CompPtr x0,
                                                  CompPtr x1, CompPtr x2, double *xd0, double *xd1,
                                                  double *xd2) {
    for (long long sl = (long long)blockIdx.x * blockDim.x + threadIdx.x; sl < S;
         sl += (long long)gridDim.x * blockDim.x) {
        const long long p = perm[sl];
        xd0[sl] = ld<double>(x0, p);
        xd1[sl] = ld<double>(x1, p);
        xd2[sl] = ld<double>(x2, p);
    }
}

}  // namespace sph
