// Store kernels: import/export between logical fields and the store layout,
// per-loop output initialisation, and the linear ghost update after density
// (the linear kernels of Sec. 2.1).
#pragma once
#include "device.cuh"

namespace sph {

// Copy `bytes` per particle between a logical field component and a store
// member: to_store != 0 moves src[perm[k]] -> store[k], else the reverse.
__global__ void k_copy_field(const char *logical, int lbytes_per_particle,
                             int comp_offset, int bytes, CompPtr store,
                             const int64_t *perm, long long n, int to_store) {
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x) {
        const long long p = perm ? perm[k] : k;
        char *lp = const_cast<char *>(logical) + p * lbytes_per_particle + comp_offset;
        char *sp = store.ptr + k * store.stride;
        if (bytes == 8) {
            if (to_store) *(unsigned long long *)sp = *(const unsigned long long *)lp;
            else *(unsigned long long *)lp = *(const unsigned long long *)sp;
        } else if (bytes == 4) {
            if (to_store) *(unsigned int *)sp = *(const unsigned int *)lp;
            else *(unsigned int *)lp = *(const unsigned int *)sp;
        } else {
            for (int b = 0; b < bytes; ++b) {
                if (to_store) sp[b] = lp[b];
                else lp[b] = sp[b];
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

__global__ void k_ghost(GhostArgs a, long long n) {
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n;
         p += (long long)gridDim.x * blockDim.x) {
        const float m = ld<float>(a.f[0], p);
        const float h = ld<float>(a.f[1], p);
        const float u = ld<float>(a.f[2], p);
        const float H = a.kernel_gamma * h;
        const float Hinv = 1.f / H;
        const float Hinv3 = Hinv * Hinv * Hinv;
        float rho = ld<float>(a.f[3], p) + m * kNorm * Hinv3;
        float rho_dh = ld<float>(a.f[4], p) - 3.f * m * kNorm * Hinv3 * Hinv;
        float wcount = ld<float>(a.f[5], p) + 32.f / 3.f;
        const float rinv = 1.f / rho;
        const float div = ld<float>(a.f[6], p) * rinv;
        const float r0 = ld<float>(a.f[7], p) * rinv;
        const float r1 = ld<float>(a.f[8], p) * rinv;
        const float r2 = ld<float>(a.f[9], p) * rinv;
        const float omega = 1.f + H * rho_dh * rinv * (1.f / 3.f);
        const float pres = (a.gamma - 1.f) * rho * u;
        const float cs = sqrtf(a.gamma * (a.gamma - 1.f) * u);
        const float arot = sqrtf(r0 * r0 + r1 * r1 + r2 * r2);
        const float adiv = fabsf(div);
        const float bal = adiv / (adiv + arot + a.balsara_eps * cs / h);
        st<float>(a.f[3], p, rho);
        st<float>(a.f[4], p, rho_dh);
        st<float>(a.f[5], p, wcount);
        st<float>(a.f[6], p, div);
        st<float>(a.f[7], p, r0);
        st<float>(a.f[8], p, r1);
        st<float>(a.f[9], p, r2);
        st<float>(a.f[10], p, 1.f / omega);
        st<float>(a.f[11], p, pres);
        st<float>(a.f[12], p, cs);
        st<float>(a.f[13], p, bal);
    }
}

}  // namespace sph
