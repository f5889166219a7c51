// Store kernels: import/export between logical fields and the store layout,
// per-loop output initialisation, and the linear ghost update after density
// (the linear kernels of Sec. 2.1).
#pragma once
#include "device.cuh"

namespace sph {

// Copy field components between logical arrays (one element of `bytes` per
// component, lbytes per particle) and store members: to_store != 0 moves
// logical[perm[k]] -> store[k], else the reverse.  All requested components
// go in one pass: each thread moves every component of its particle, so the
// record parts of one particle are written (or read) together and the
// permutation is read once.
struct CopyComp {
    const char *logical;
    int lbytes, loff, bytes;
    CompPtr store;
};
constexpr int kCopyMax = 48;
struct CopyArgs {
    int ncomp;
    CopyComp c[kCopyMax];
};

__global__ void k_copy_fields(CopyArgs a, const int64_t *perm, long long n, int to_store) {
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x) {
        const long long p = perm ? perm[k] : k;
        for (int q = 0; q < a.ncomp; ++q) {
            const CopyComp &C = a.c[q];
            char *lp = const_cast<char *>(C.logical) + p * C.lbytes + C.loff;
            char *sp = C.store.ptr + k * C.store.stride;
            if (C.bytes == 8) {
                if (to_store) *(unsigned long long *)sp = *(const unsigned long long *)lp;
                else *(unsigned long long *)lp = *(const unsigned long long *)sp;
            } else if (C.bytes == 4) {
                if (to_store) *(unsigned int *)sp = *(const unsigned int *)lp;
                else *(unsigned int *)lp = *(const unsigned int *)sp;
            } else {
                for (int b = 0; b < C.bytes; ++b) {
                    if (to_store) sp[b] = lp[b];
                    else lp[b] = sp[b];
                }
            }
        }
    }
}

// Store-to-store layout conversion: every component of every field (every
// copy of a replicated one) of the destination from the source's first copy.
struct ConvComp {
    CompPtr dst, src;
    int bytes;
};
struct ConvArgs {
    int ncomp;
    ConvComp c[56];
};

__global__ void k_convert(ConvArgs a, long long n) {
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x) {
        for (int q = 0; q < a.ncomp; ++q) {
            const char *sp = a.c[q].src.ptr + k * a.c[q].src.stride;
            char *dp = a.c[q].dst.ptr + k * a.c[q].dst.stride;
            const int b = a.c[q].bytes;
            if (b == 8) *(unsigned long long *)dp = *(const unsigned long long *)sp;
            else if (b == 4) *(unsigned int *)dp = *(const unsigned int *)sp;
            else
                for (int t = 0; t < b; ++t) dp[t] = sp[t];
        }
    }
}

// Zero up to 8 float outputs; with `tb` set only particles with
// time_bin <= active_bin are touched (force loop).
struct InitArgs {
    CompPtr out[8];
    int nout;
    CompPtr tb;
    int use_tb;
    int active_bin;
};

__global__ void k_init(InitArgs a, long long n) {
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n;
         p += (long long)gridDim.x * blockDim.x) {
        if (a.use_tb && (int)ld<int8_t>(a.tb, p) > a.active_bin) continue;
        for (int k = 0; k < a.nout; ++k) st<float>(a.out[k], p, 0.f);
    }
}

// Ghost after density.  Roles: 0 mass, 1 h, 2 u, 3 rho, 4 rho_dh, 5 wcount,
// 6 div_v, 7..9 rot_v, 10 f_gradh, 11 pressure, 12 soundspeed, 13 balsara.
struct GhostArgs {
    CompPtr f[14];
    float kernel_gamma, gamma, balsara_eps;
};

// The ghost's arithmetic for one particle, from its raw density sums s[8]
// (rho, rho_dh, wcount, wcount_dh, div_v, rot_v) and m, h, u; g[11] receives
// rho, rho_dh, wcount, div_v, rot_v (3), f_gradh, pressure, soundspeed,
// balsara.  A particle with no neighbour inside its support (raw wcount sum
// 0) has Omega = 0 exactly and takes f_gradh = 1.
__device__ __forceinline__ void ghost_point(const float *s, float m, float h, float u,
                                            float kernel_gamma, float gamma, float balsara_eps,
                                            float *g) {
    const float H = kernel_gamma * h;
    const float Hinv = 1.f / H;
    const float Hinv3 = Hinv * Hinv * Hinv;
    const float rho = s[0] + m * kNorm * Hinv3;
    const float rho_dh = s[1] - 3.f * m * kNorm * Hinv3 * Hinv;
    const float wcount = s[2] + 32.f / 3.f;
    const float rinv = 1.f / rho;
    const float div = s[4] * rinv;
    const float r0 = s[5] * rinv;
    const float r1 = s[6] * rinv;
    const float r2 = s[7] * rinv;
    const float omega = 1.f + H * rho_dh * rinv * (1.f / 3.f);
    const float pres = (gamma - 1.f) * rho * u;
    const float cs = sqrtf(gamma * (gamma - 1.f) * u);
    const float arot = sqrtf(r0 * r0 + r1 * r1 + r2 * r2);
    const float adiv = fabsf(div);
    const float bal = adiv / (adiv + arot + balsara_eps * cs / h);
    g[0] = rho;
    g[1] = rho_dh;
    g[2] = wcount;
    g[3] = div;
    g[4] = r0;
    g[5] = r1;
    g[6] = r2;
    g[7] = s[2] == 0.f ? 1.f : 1.f / omega;
    g[8] = pres;
    g[9] = cs;
    g[10] = bal;
}

__global__ void k_ghost(GhostArgs a, long long n) {
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n;
         p += (long long)gridDim.x * blockDim.x) {
        const float sums[8] = {ld<float>(a.f[3], p), ld<float>(a.f[4], p), ld<float>(a.f[5], p),
                               0.f, ld<float>(a.f[6], p), ld<float>(a.f[7], p),
                               ld<float>(a.f[8], p), ld<float>(a.f[9], p)};
        float g[11];
        ghost_point(sums, ld<float>(a.f[0], p), ld<float>(a.f[1], p), ld<float>(a.f[2], p),
                    a.kernel_gamma, a.gamma, a.balsara_eps, g);
#pragma unroll
        for (int q = 0; q < 11; ++q) st<float>(a.f[3 + q], p, g[q]);
    }
}

}  // namespace sph
