// Adjoint of the density -> ghost -> force chain (the differentiation
// workload): gradient of L = sum_i |a_i|^2 + sum_i (du_i/dt)^2 over active
// particles with respect to positions, masses and internal energies, given
// the upstream adjoints abar_i = dL/da_i and ebar_i = dL/d(du_i/dt).
//
// Every pair term of the forward sums belongs to one particle's output (the
// i of the loop), but its derivatives reach both particles of the pair.
// Rather than scattering with atomics, each particle k walks its neighbour
// list (which holds every j with r < max(H_k, H_j), so both directions of
// every pair) and evaluates the pair's backward twice: once as the i of the
// pair (with its own adjoints) and once as the j (with the neighbour's), so
// each particle's gradient is a deterministic gather.
//
// k_adj_pack     slot-ordered records of the forward state and the upstream
//                adjoints (the slot order of the bundle's density pack)
// k_adj_pairs<0> force backward: adjoints of x, m, u and of rho, f_gradh, B
// k_adj_ghost    ghost backward per particle: adjoints of the raw density
//                sums (rho, d rho/dH, rho div v, rho curl v), plus the self
//                terms' m and the Balsara switch's sound speed (u)
// k_adj_pairs<1> density backward: adjoints of x and m
// k_adj_scatter  gradients to the caller's arrays in original particle order
#pragma once
#include "list_kernels.cuh"

namespace sph {

constexpr int kAdjRec = 6;   // float4 records per slot

// store fields read by the adjoint (indices into AdjArgs::f; rot_v takes 3)
enum AdjField {
    A_X0, A_X1, A_X2, A_V0, A_V1, A_V2, A_M, A_H, A_U, A_RHO, A_FGH, A_BAL, A_AV, A_AD,
    A_CS, A_PRES, A_TB, A_RHODH, A_DIV, A_ROT0, A_WCOUNT = A_ROT0 + 3, A_NUM
};

struct AdjArgs {
    const BCellDev *cells;
    const BTargetDev *targets;
    const BItemDev *items;
    unsigned int *counter;
    int nitems;
    long long item0;
    ListView L;
    long long S;
    const int32_t *perm;      // slot -> store index (density pack)
    const int64_t *store_perm;  // store index -> original index (NULL: identity)
    float4 *rec;              // kAdjRec per slot
    float4 *g;                // 2 per slot: (gx gy gz gm) (gu grho gf gB)
    float4 *sg;               // 2 per slot: (gSrho gSdh gSdiv 0) (gSrot 0)
    CompPtr f[A_NUM];         // store fields
    const float *abar;        // n x 3, original order
    const float *ebar;        // n, original order
    double *gx_out;           // n x 3
    float *gm_out, *gu_out;   // n
    float kernel_gamma, gamma, beta, eps;
    float half[3], shift_hi[3], shift_lo[3];
    int active_bin;
};


__device__ __forceinline__ void spline2(float q, float &w, float &dw, float &ddw) {
    const float t = 1.f - q;
    const bool inner = q < 0.5f;
    w = inner ? fmaf(q * q, fmaf(6.f, q, -6.f), 1.f) : 2.f * t * t * t;
    dw = inner ? q * fmaf(18.f, q, -12.f) : -6.f * t * t;
    ddw = inner ? fmaf(36.f, q, -12.f) : 12.f * t;
    if (!(q < 1.f)) w = dw = ddw = 0.f;
}

__global__ void k_adj_pack(AdjArgs a) {
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < a.S;
         s += (long long)gridDim.x * blockDim.x) {
        const long long p = a.perm[s];
        const long long o = a.store_perm ? a.store_perm[p] : p;
        float hi[3], lo[3];
        for (int d = 0; d < 3; ++d) split_f64(ld<double>(a.f[A_X0 + d], p), hi[d], lo[d]);
        const float H = a.kernel_gamma * ld<float>(a.f[A_H], p);
        float4 *r = a.rec + kAdjRec * s;
        r[0] = make_float4(hi[0], hi[1], hi[2], H);
        r[1] = make_float4(lo[0], lo[1], lo[2], ld<float>(a.f[A_M], p));
        r[2] = make_float4(ld<float>(a.f[A_V0], p), ld<float>(a.f[A_V1], p),
                           ld<float>(a.f[A_V2], p), ld<float>(a.f[A_U], p));
        r[3] = make_float4(ld<float>(a.f[A_RHO], p), ld<float>(a.f[A_FGH], p),
                           ld<float>(a.f[A_BAL], p), ld<float>(a.f[A_AV], p));
        const bool act = (int)ld<int8_t>(a.f[A_TB], p) <= a.active_bin;
        r[4] = make_float4(ld<float>(a.f[A_AD], p), ld<float>(a.f[A_CS], p),
                           ld<float>(a.f[A_PRES], p), act ? 1.f : 0.f);
        r[5] = act ? make_float4(a.abar[3 * o], a.abar[3 * o + 1], a.abar[3 * o + 2], a.ebar[o])
                   : make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

// Backward of one force pair term of particle I (partner J, dx = x_I - x_J):
// the pair's contribution to the loss through a_I and du_I/dt, differentiated.
struct FBack {
    float dx[3], mJ, uI, uJ, rhoI, rhoJ, fI, fJ, BI, BJ;
};

__device__ __forceinline__ void force_back(const float4 *I, const float4 *J, float dx, float dy,
                                           float dz, float r2, const AdjArgs &a, FBack &g) {
    const float gam1 = a.gamma - 1.f;
    const float rinv = r2 > 0.f ? rsqrtf(r2) : 0.f;
    const float r = r2 * rinv;
    const float HIi = 1.f / I[0].w, HJi = 1.f / J[0].w;
    float wi, dwi, ddwi, wj, dwj, ddwj;
    spline2(r * HIi, wi, dwi, ddwi);
    spline2(r * HJi, wj, dwj, ddwj);
    const float K4i = kNorm * HIi * HIi * HIi * HIi, K4j = kNorm * HJi * HJi * HJi * HJi;
    const float Fi = K4i * dwi, Fj = K4j * dwj;
    const float dFi = K4i * ddwi * HIi, dFj = K4j * ddwj * HJi;
    const float dvx = I[2].x - J[2].x, dvy = I[2].y - J[2].y, dvz = I[2].z - J[2].z;
    const float wdot = (dvx * dx + dvy * dy + dvz * dz) * rinv;
    const float mu = fminf(0.f, wdot);
    const float rhoI = I[3].x, rhoJ = J[3].x;
    const float Fbar = 0.5f * (Fi + Fj);
    const float rhobar = 0.5f * (rhoI + rhoJ), rbi = 1.f / rhobar;
    const float alpha = 0.5f * (I[3].w * I[3].z + J[3].w * J[3].z);
    const float vs = I[4].y + J[4].y - a.beta * mu;
    const float Pi = -alpha * vs * mu * rbi;
    const float AI = I[3].y * I[4].z / (rhoI * rhoI), AJ = J[3].y * J[4].z / (rhoJ * rhoJ);
    const float sc = AI * Fi + AJ * Fj + Pi * Fbar;
    const float aD = 0.5f * (I[4].x + J[4].x);
    const float dP = I[4].z - J[4].z;
    const float S = sqrtf(fabsf(dP) * rbi);
    const float du = I[2].w - J[2].w;
    const float cond = aD * S * du * Fbar * rbi;
    const float U = AI * Fi * wdot + 0.5f * Pi * Fbar * wdot + cond;
    const float sa = (I[5].x * dx + I[5].y * dy + I[5].z * dz) * rinv;
    const float m = J[1].w;
    // adjoints of the intermediates
    const float g_sc = -m * sa, g_sa = -m * sc, g_U = m * I[5].w;
    const float g_AI = g_sc * Fi + g_U * Fi * wdot;
    const float g_AJ = g_sc * Fj;
    const float g_Pi = g_sc * Fbar + g_U * 0.5f * Fbar * wdot;
    const float g_Fbar = g_sc * Pi + g_U * (0.5f * Pi * wdot + aD * S * du * rbi);
    const float g_Fi = g_sc * AI + g_U * AI * wdot + 0.5f * g_Fbar;
    const float g_Fj = g_sc * AJ + 0.5f * g_Fbar;
    float g_wdot = g_U * (AI * Fi + 0.5f * Pi * Fbar);
    const float g_alpha = -g_Pi * vs * mu * rbi;
    const float g_vs = -g_Pi * alpha * mu * rbi;
    const float g_mu = -g_Pi * alpha * vs * rbi - a.beta * g_vs;
    if (wdot < 0.f) g_wdot += g_mu;
    float g_rhobar = -g_Pi * Pi * rbi - g_U * cond * rbi;
    const float g_S = g_U * aD * du * Fbar * rbi;
    const float g_du = g_U * aD * S * Fbar * rbi;
    float g_dP = 0.f;
    if (S > 0.f) {
        g_dP = g_S * copysignf(1.f, dP) * 0.5f * rbi / S;
        g_rhobar -= g_S * 0.5f * S * rbi;
    }
    // per-particle fields (A = (gamma-1) f u / rho, P = (gamma-1) rho u,
    // c = sqrt(gamma (gamma-1) u))
    const float cI = I[4].y, cJ = J[4].y;
    const float gcu = a.gamma * gam1 * 0.5f;
    g.uI = g_du + g_dP * gam1 * rhoI + g_AI * gam1 * I[3].y / rhoI + (cI > 0.f ? g_vs * gcu / cI : 0.f);
    g.uJ = -g_du - g_dP * gam1 * rhoJ + g_AJ * gam1 * J[3].y / rhoJ + (cJ > 0.f ? g_vs * gcu / cJ : 0.f);
    g.rhoI = 0.5f * g_rhobar + g_dP * gam1 * I[2].w - g_AI * AI / rhoI;
    g.rhoJ = 0.5f * g_rhobar - g_dP * gam1 * J[2].w - g_AJ * AJ / rhoJ;
    g.fI = g_AI * gam1 * I[2].w / rhoI;
    g.fJ = g_AJ * gam1 * J[2].w / rhoJ;
    g.BI = g_alpha * 0.5f * I[3].w;
    g.BJ = g_alpha * 0.5f * J[3].w;
    g.mJ = -sc * sa + I[5].w * U;
    // geometry: r, w = v_ij . rhat and s_a = abar . rhat depend on dx
    const float g_r = g_Fi * dFi + g_Fj * dFj;
    const float ri2 = rinv * rinv;
    g.dx[0] = g_r * dx * rinv + g_wdot * (dvx * rinv - wdot * dx * ri2) +
              g_sa * (I[5].x * rinv - sa * dx * ri2);
    g.dx[1] = g_r * dy * rinv + g_wdot * (dvy * rinv - wdot * dy * ri2) +
              g_sa * (I[5].y * rinv - sa * dy * ri2);
    g.dx[2] = g_r * dz * rinv + g_wdot * (dvz * rinv - wdot * dz * ri2) +
              g_sa * (I[5].z * rinv - sa * dz * ri2);
}

// Backward of one density pair term of particle I (partner J, r < H_I): the
// raw sums' adjoints gS = (rho, d rho/dH, rho div v, .) and gR (rho curl v)
// of I; returns the d/d dx and the term's value over m_J (its m_J gradient).
__device__ __forceinline__ float density_back(const float4 *I, const float4 &gS, const float4 &gR,
                                              const float4 *J, float dx, float dy, float dz,
                                              float r2, float *gdx) {
    const float rinv = r2 > 0.f ? rsqrtf(r2) : 0.f;
    const float r = r2 * rinv;
    const float Hinv = 1.f / I[0].w;
    const float q = r * Hinv;
    float w, dw, ddw;
    spline2(q, w, dw, ddw);
    const float K3 = kNorm * Hinv * Hinv * Hinv, K4 = K3 * Hinv;
    const float F = K4 * dw, dF = K4 * ddw * Hinv;
    const float m = J[1].w;
    const float dvx = I[2].x - J[2].x, dvy = I[2].y - J[2].y, dvz = I[2].z - J[2].z;
    const float vr = (dvx * dx + dvy * dy + dvz * dz) * rinv;
    const float cx = dvy * dz - dvz * dy, cy = dvz * dx - dvx * dz, cz = dvx * dy - dvy * dx;
    const float rotdot = gR.x * cx + gR.y * cy + gR.z * cz;
    const float psi_m = gS.x * K3 * w - gS.y * K4 * (3.f * w + q * dw) - gS.z * vr * F +
                        F * rinv * rotdot;
    const float g_r = m * (gS.x * K3 * dw * Hinv - gS.y * K4 * (4.f * dw + q * ddw) * Hinv -
                           gS.z * vr * dF + rotdot * (dF * rinv - F * rinv * rinv));
    const float g_vr = -gS.z * m * F;
    const float ri2 = rinv * rinv, mf = m * F * rinv;
    // d/d dx of gR . (dv x dx) is gR x dv
    gdx[0] = g_r * dx * rinv + g_vr * (dvx * rinv - vr * dx * ri2) + mf * (gR.y * dvz - gR.z * dvy);
    gdx[1] = g_r * dy * rinv + g_vr * (dvy * rinv - vr * dy * ri2) + mf * (gR.z * dvx - gR.x * dvz);
    gdx[2] = g_r * dz * rinv + g_vr * (dvz * rinv - vr * dz * ri2) + mf * (gR.x * dvy - gR.y * dvx);
    return psi_m;
}

// The partner's record with its periodic image brought next to `own`, and the
// two-float separation own - partner.
__device__ __forceinline__ void image_sep(const float4 *own, float4 *oth, const AdjArgs &a,
                                          float &dx, float &dy, float &dz) {
    const float ax = own[0].x - oth[0].x, ay = own[0].y - oth[0].y, az = own[0].z - oth[0].z;
    if (ax > a.half[0]) add2(oth[0].x, oth[1].x, a.shift_hi[0], a.shift_lo[0]);
    else if (ax < -a.half[0]) add2(oth[0].x, oth[1].x, -a.shift_hi[0], -a.shift_lo[0]);
    if (ay > a.half[1]) add2(oth[0].y, oth[1].y, a.shift_hi[1], a.shift_lo[1]);
    else if (ay < -a.half[1]) add2(oth[0].y, oth[1].y, -a.shift_hi[1], -a.shift_lo[1]);
    if (az > a.half[2]) add2(oth[0].z, oth[1].z, a.shift_hi[2], a.shift_lo[2]);
    else if (az < -a.half[2]) add2(oth[0].z, oth[1].z, -a.shift_hi[2], -a.shift_lo[2]);
    dx = (own[0].x - oth[0].x) + (own[1].x - oth[1].x);
    dy = (own[0].y - oth[0].y) + (own[1].y - oth[1].y);
    dz = (own[0].z - oth[0].z) + (own[1].z - oth[1].z);
}

template <int PASS>  // 0: force backward, 1: density backward
__global__ void __launch_bounds__(128, 4) k_adj_pairs(AdjArgs a) {
    const int lane = threadIdx.x & 31;
    const bool broken = a.L.hdr->overflow != 0u;
    for (;;) {
        int it = 0;
        if (lane == 0) it = (int)atomicAdd(a.counter, 1u);
        it = __shfl_sync(0xffffffffu, it, 0);
        if (it >= a.nitems) break;
        const long long gitem = a.item0 + it;
        const BItemDev W = a.items[it];
        const BCellDev C = a.cells[a.targets[W.target].cell];
        const int i = W.i0 + lane;
        const bool valid = i < C.n;
        const long long slot = (long long)C.slot + i;
        float4 own[kAdjRec];
        float4 gS = make_float4(0.f, 0.f, 0.f, 0.f), gR = gS;
        if (valid) {
#pragma unroll
            for (int f = 0; f < kAdjRec; ++f) own[f] = a.rec[kAdjRec * slot + f];
            if (PASS == 1) {
                gS = a.sg[2 * slot];
                gR = a.sg[2 * slot + 1];
            }
        } else {
#pragma unroll
            for (int f = 0; f < kAdjRec; ++f) own[f] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        float gx = 0.f, gy = 0.f, gz = 0.f, gm = 0.f, gu = 0.f, grho = 0.f, gf = 0.f, gB = 0.f;
        const int cnt = valid && !broken ? (int)a.L.lcount[gitem * 32 + lane] : 0;
        const int maxc = __reduce_max_sync(0xffffffffu, (unsigned)cnt);
        // the list entries run two pairs ahead and the partner's record one
        // pair ahead of their use (the loads' latency hides behind a pair)
        uint32_t chunk = a.L.first[gitem];
        int kl = 0;
        auto next_ent = [&]() -> uint32_t {
            uint32_t e = 0u;
            if (kl < cnt)
                e = __ldg(&a.L.entries[checked(chunk, (long long)a.L.pool) * kLChunk +
                                       (kl % kLPer) * 32 + lane]);
            ++kl;
            if (kl % kLPer == 0 && kl < maxc) chunk = a.L.next[chunk];
            return e;
        };
        uint32_t e = next_ent(), en = e;
        float4 nxt[kAdjRec];
        bool un = 0 < cnt;
        if (un) {
#pragma unroll
            for (int f = 0; f < kAdjRec; ++f)
                nxt[f] = __ldg(&a.rec[kAdjRec * checked(e, a.S) + f]);
        }
        e = next_ent();
#pragma unroll 1
        for (int k = 0; k < maxc; ++k) {
            float4 oth[kAdjRec];
#pragma unroll
            for (int f = 0; f < kAdjRec; ++f) oth[f] = nxt[f];
            const uint32_t ent = en;
            const bool u = un;
            un = k + 1 < cnt;
            if (un) {
#pragma unroll
                for (int f = 0; f < kAdjRec; ++f)
                    nxt[f] = __ldg(&a.rec[kAdjRec * checked(e, a.S) + f]);
            }
            en = e;
            e = next_ent();
            if (!u) continue;
            const long long js = (long long)ent;
            float dx, dy, dz;
            image_sep(own, oth, a, dx, dy, dz);
            const float r2 = dx * dx + dy * dy + dz * dz;
            if (PASS == 0) {
                FBack g;
                if (own[4].w != 0.f) {          // own's force term with this partner
                    force_back(own, oth, dx, dy, dz, r2, a, g);
                    gx += g.dx[0]; gy += g.dx[1]; gz += g.dx[2];
                    gu += g.uI; grho += g.rhoI; gf += g.fI; gB += g.BI;
                }
                if (oth[4].w != 0.f) {          // the partner's term with own as its j
                    force_back(oth, own, -dx, -dy, -dz, r2, a, g);
                    gx -= g.dx[0]; gy -= g.dx[1]; gz -= g.dx[2];
                    gm += g.mJ; gu += g.uJ; grho += g.rhoJ; gf += g.fJ; gB += g.BJ;
                }
            } else {
                float gd[3];
                if (r2 < own[0].w * own[0].w) {  // r < H_own: own's density term
                    density_back(own, gS, gR, oth, dx, dy, dz, r2, gd);
                    gx += gd[0]; gy += gd[1]; gz += gd[2];
                }
                if (r2 < oth[0].w * oth[0].w) {  // r < H_j: own in the partner's sums
                    const float4 oS = __ldg(&a.sg[2 * checked(js, a.S)]),
                                 oR = __ldg(&a.sg[2 * checked(js, a.S) + 1]);
                    gm += density_back(oth, oS, oR, own, -dx, -dy, -dz, r2, gd);
                    gx -= gd[0]; gy -= gd[1]; gz -= gd[2];
                }
            }
        }
        if (valid) {
            if (PASS == 0) {
                a.g[2 * slot] = make_float4(gx, gy, gz, gm);
                a.g[2 * slot + 1] = make_float4(gu, grho, gf, gB);
            } else {
                float4 g0 = a.g[2 * slot];
                g0.x += gx; g0.y += gy; g0.z += gz; g0.w += gm;
                a.g[2 * slot] = g0;
            }
        }
    }
}

// Ghost backward: rho = S_rho + m W(0,H), rho_dh = S_dh + m dW/dH(0,H),
// div = S_div / rho, rot = S_rot / rho, f = 1 / (1 + H rho_dh / (3 rho)),
// B = |div| / (|div| + |rot| + eps c / h), c = sqrt(gamma (gamma-1) u).
__global__ void k_adj_ghost(AdjArgs a) {
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < a.S;
         s += (long long)gridDim.x * blockDim.x) {
        const long long p = a.perm[s];
        const float4 *r = a.rec + kAdjRec * s;
        const float rho = r[3].x, f = r[3].y;
        const float h = ld<float>(a.f[A_H], p), H = r[0].w;
        const float rho_dh = ld<float>(a.f[A_RHODH], p);
        const float div = ld<float>(a.f[A_DIV], p);
        const float rt[3] = {ld<float>(a.f[A_ROT0], p), ld<float>(a.f[A_ROT0 + 1], p),
                             ld<float>(a.f[A_ROT0 + 2], p)};
        const float c = r[4].y;
        float4 g0 = a.g[2 * s], g1 = a.g[2 * s + 1];
        float grho = g1.y;
        const float D = fabsf(div);
        const float R = sqrtf(rt[0] * rt[0] + rt[1] * rt[1] + rt[2] * rt[2]);
        const float e = a.eps * c / h;
        const float den = D + R + e, di2 = 1.f / (den * den);
        const float gD = g1.w * (R + e) * di2, gRn = -g1.w * D * di2, ge = -g1.w * D * di2;
        if (c > 0.f) g1.x += ge * a.eps / h * a.gamma * (a.gamma - 1.f) * 0.5f / c;
        const float gdiv = div > 0.f ? gD : (div < 0.f ? -gD : 0.f);
        float grot[3];
        for (int d = 0; d < 3; ++d) grot[d] = R > 0.f ? gRn * rt[d] / R : 0.f;
        const float gSdiv = gdiv / rho;
        grho -= gdiv * div / rho + (grot[0] * rt[0] + grot[1] * rt[1] + grot[2] * rt[2]) / rho;
        // a particle with no neighbour in its support took f = 1 (Omega = 0):
        // f is then constant.  It is recognised by f == 1 together with a
        // neighbour count equal to the self term, which no other particle
        // reaches (an edge neighbour that leaves the count unchanged in
        // float makes Omega tiny and f far from 1).
        const bool lone = f == 1.f && ld<float>(a.f[A_WCOUNT], p) == 32.f / 3.f;
        const float gOm = lone ? 0.f : -g1.z * f * f;
        const float grhodh = gOm * H / (3.f * rho);
        grho -= gOm * H * rho_dh / (3.f * rho * rho);
        const float Hi = 1.f / H;
        g0.w += grho * kNorm * Hi * Hi * Hi - 3.f * grhodh * kNorm * Hi * Hi * Hi * Hi;
        a.g[2 * s] = g0;
        a.g[2 * s + 1] = g1;
        a.sg[2 * s] = make_float4(grho, grhodh, gSdiv, 0.f);
        a.sg[2 * s + 1] = make_float4(grot[0] / rho, grot[1] / rho, grot[2] / rho, 0.f);
    }
}

__global__ void k_adj_scatter(AdjArgs a) {
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < a.S;
         s += (long long)gridDim.x * blockDim.x) {
        const long long p = a.perm[s];
        const long long o = a.store_perm ? a.store_perm[p] : p;
        const float4 g0 = a.g[2 * s], g1 = a.g[2 * s + 1];
        a.gx_out[3 * o] = g0.x;
        a.gx_out[3 * o + 1] = g0.y;
        a.gx_out[3 * o + 2] = g0.z;
        a.gm_out[o] = g0.w;
        a.gu_out[o] = g1.x;
    }
}

}  // namespace sph
