// All-FP64 variant of the batched pipeline (precision study).
//
// Same cells, neighbours and result definitions as the mixed-precision
// kernels, but every arithmetic step runs in FP64: positions and separations,
// kernel values, sums and the force terms.  Records are FP64 copies of the
// store fields; results are rounded to the FP32 store once at unpack.  One
// thread per target particle, neighbours read from global memory: this path
// exists to measure what mixed precision costs in accuracy and saves in time
// on a GPU whose FP64 pipe is a small fraction of its FP32 pipe.
#pragma once
#include "device.cuh"
#include "pack_kernels.cuh"

namespace sph {

// Records (double4 lanes): [0] x y z H  [1] vx vy vz m  [2] u rho f_gradh B
// [3] alpha_visc alpha_diff time_bin h ; then the store index (int32).
struct D64Layout {
    static __host__ __device__ int64_t r256(int64_t b) { return (b + 255) / 256 * 256; }
    static __host__ __device__ int64_t rec(int f, int64_t S) { return r256(S * 32) * f; }
    static __host__ __device__ int64_t perm(int64_t S) { return rec(4, S); }
    static __host__ __device__ int64_t bytes(int64_t S) { return perm(S) + r256(S * 4); }
    // results: 8 doubles per slot (density), 2 (gradient), 6 (force)
    static __host__ __device__ int64_t out_bytes(int loop, int64_t S) {
        return r256(S * 8 * (loop == SPH_DENSITY ? 8 : (loop == SPH_GRADIENT ? 2 : 6)));
    }
};

struct D64PackArgs {
    const BCellDev *cells;
    char *buf;
    long long S;
    CompPtr src[R_NUM];
    double kernel_gamma;
};

__global__ void __launch_bounds__(128) k_pack64(D64PackArgs a) {
    const BCellDev C = a.cells[blockIdx.x];
    double4_32a *r0 = reinterpret_cast<double4_32a *>(a.buf + D64Layout::rec(0, a.S));
    double4_32a *r1 = reinterpret_cast<double4_32a *>(a.buf + D64Layout::rec(1, a.S));
    double4_32a *r2 = reinterpret_cast<double4_32a *>(a.buf + D64Layout::rec(2, a.S));
    double4_32a *r3 = reinterpret_cast<double4_32a *>(a.buf + D64Layout::rec(3, a.S));
    int32_t *perm = reinterpret_cast<int32_t *>(a.buf + D64Layout::perm(a.S));
    for (int k = threadIdx.x; k < C.n; k += blockDim.x) {
        const long long p = (long long)C.p0 + k, sl = (long long)C.slot + k;
        const double h = (double)ld<float>(a.src[R_H], p);
        r0[sl] = make_double4_32a(ld<double>(a.src[R_X0], p), ld<double>(a.src[R_X1], p),
                              ld<double>(a.src[R_X2], p), a.kernel_gamma * h);
        r1[sl] = make_double4_32a(ld<float>(a.src[R_V0], p), ld<float>(a.src[R_V1], p),
                              ld<float>(a.src[R_V2], p), ld<float>(a.src[R_M], p));
        r2[sl] = make_double4_32a(ld<float>(a.src[R_U], p), ld<float>(a.src[R_RHO], p),
                              ld<float>(a.src[R_FGH], p), ld<float>(a.src[R_BAL], p));
        r3[sl] = make_double4_32a(ld<float>(a.src[R_AV], p), ld<float>(a.src[R_AD], p),
                              (double)ld<int8_t>(a.src[R_TB], p), h);
        perm[sl] = (int32_t)p;
    }
}

__device__ __forceinline__ double w64(double q) {
    return q < 0.5 ? 1.0 - 6.0 * q * q + 6.0 * q * q * q
                   : (q < 1.0 ? 2.0 * (1.0 - q) * (1.0 - q) * (1.0 - q) : 0.0);
}
__device__ __forceinline__ double dw64(double q) {
    return q < 0.5 ? -12.0 * q + 18.0 * q * q : (q < 1.0 ? -6.0 * (1.0 - q) * (1.0 - q) : 0.0);
}

struct D64Args {
    const BCellDev *cells;
    const BTargetDev *targets;
    const BNbrDev *nbrs;
    const char *in;
    char *out;
    long long S;
    double gamma, beta, box[3];
    int active_bin;
};

constexpr int kSelfCode = 1 | (1 << 2) | (1 << 4);  // no shift in any dimension

// One CTA per target cell, one thread per target particle.
template <int LOOP>
__global__ void __launch_bounds__(128) k_interact64(D64Args a) {
    const double kPi64 = 3.14159265358979323846;
    const double norm = 8.0 / kPi64;
    const BTargetDev &Tg = a.targets[blockIdx.x];
    const BCellDev C = a.cells[Tg.cell];
    const double4_32a *R0 = reinterpret_cast<const double4_32a *>(a.in + D64Layout::rec(0, a.S));
    const double4_32a *R1 = reinterpret_cast<const double4_32a *>(a.in + D64Layout::rec(1, a.S));
    const double4_32a *R2 = reinterpret_cast<const double4_32a *>(a.in + D64Layout::rec(2, a.S));
    const double4_32a *R3 = reinterpret_cast<const double4_32a *>(a.in + D64Layout::rec(3, a.S));
    double *out = reinterpret_cast<double *>(a.out);
    const double gg = a.gamma * (a.gamma - 1.0);
    for (int k = threadIdx.x; k < C.n; k += blockDim.x) {
        const long long si = (long long)C.slot + k;
        const double4_32a xi = R0[si], vi = R1[si], qi = R2[si], ei = R3[si];
        const double Hi = xi.w;
        double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        double vsig = 0.0;
        const bool active = LOOP != SPH_FORCE || (int)ei.z <= a.active_bin;
        const double rhoi = qi.y, ui = qi.x;
        const double Pi_ = (a.gamma - 1.0) * rhoi * ui;
        const double ci = sqrt(gg * ui);
        const double Ai = qi.z * Pi_ / (rhoi * rhoi);
        for (int e = Tg.nb0; e < Tg.nb0 + Tg.nnb && active; ++e) {
            const BCellDev Cn = a.cells[a.nbrs[e].cell];
            const int code = a.nbrs[e].code;
            double s[3];
            for (int d = 0; d < 3; ++d) {
                const int c = ((code >> (2 * d)) & 3) - 1;
                s[d] = c == 0 ? 0.0 : (c > 0 ? a.box[d] : -a.box[d]);
            }
            for (int q = 0; q < Cn.n; ++q) {
                const long long sj = (long long)Cn.slot + q;
                if (sj == si && code == kSelfCode) continue;
                const double4_32a xj = R0[sj];
                const double dx = xi.x - (xj.x + s[0]), dy = xi.y - (xj.y + s[1]),
                             dz = xi.z - (xj.z + s[2]);
                const double r2 = dx * dx + dy * dy + dz * dz;
                const double Hj = xj.w;
                const double Hm = LOOP == SPH_FORCE ? fmax(Hi, Hj) : Hi;
                if (!(r2 < Hm * Hm)) continue;
                const double r = sqrt(r2);
                const double rinv = r > 0.0 ? 1.0 / r : 0.0;
                const double4_32a vj = R1[sj];
                const double dvx = vi.x - vj.x, dvy = vi.y - vj.y, dvz = vi.z - vj.z;
                const double wdot = (dvx * dx + dvy * dy + dvz * dz) * rinv;
                const double mj = vj.w;
                const double qi_ = r / Hi;
                const double Fi = norm / (Hi * Hi * Hi * Hi) * dw64(qi_);
                if (LOOP == SPH_DENSITY) {
                    const double w = w64(qi_);
                    acc[0] += mj * norm / (Hi * Hi * Hi) * w;
                    acc[1] += -mj * norm / (Hi * Hi * Hi * Hi) * (3.0 * w + qi_ * dw64(qi_));
                    acc[2] += (4.0 * kPi64 / 3.0) * norm * w;
                    acc[3] += -(4.0 * kPi64 / 3.0) * norm * qi_ * dw64(qi_) / Hi;
                    acc[4] += -mj * wdot * Fi;
                    acc[5] += mj * (dvy * dz - dvz * dy) * rinv * Fi;
                    acc[6] += mj * (dvz * dx - dvx * dz) * rinv * Fi;
                    acc[7] += mj * (dvx * dy - dvy * dx) * rinv * Fi;
                } else if (LOOP == SPH_GRADIENT) {
                    const double4_32a qj = R2[sj];
                    const double cj = sqrt(gg * qj.x);
                    vsig = fmax(vsig, ci + cj - a.beta * fmin(0.0, wdot));
                    if (r > 0.0) acc[0] += 2.0 * mj * (ui - qj.x) / qj.y * Fi * rinv;
                } else {
                    const double4_32a qj = R2[sj], ej = R3[sj];
                    const double Fj = norm / (Hj * Hj * Hj * Hj) * dw64(r / Hj);
                    const double Pj = (a.gamma - 1.0) * qj.y * qj.x;
                    const double cj = sqrt(gg * qj.x);
                    const double Aj = qj.z * Pj / (qj.y * qj.y);
                    const double mu = fmin(0.0, wdot);
                    const double Fbar = 0.5 * (Fi + Fj);
                    const double rhobar = 0.5 * (rhoi + qj.y);
                    const double alpha = 0.5 * (ei.x * qi.w + ej.x * qj.w);
                    const double vs = ci + cj - a.beta * mu;
                    const double Pv = -alpha * vs * mu / rhobar;
                    const double sc = Ai * Fi + Aj * Fj + Pv * Fbar;
                    acc[0] -= mj * sc * dx * rinv;
                    acc[1] -= mj * sc * dy * rinv;
                    acc[2] -= mj * sc * dz * rinv;
                    const double alphaD = 0.5 * (ei.y + ej.y);
                    const double cond = alphaD * sqrt(fabs(Pi_ - Pj) / rhobar) * (ui - qj.x) * Fbar /
                                        rhobar;
                    acc[3] += mj * (Ai * Fi * wdot + 0.5 * Pv * Fbar * wdot + cond);
                    acc[4] += mj * wdot * Fi;
                    vsig = fmax(vsig, vs);
                }
            }
        }
        if (LOOP == SPH_DENSITY) {
            for (int c = 0; c < 8; ++c) out[8 * si + c] = acc[c];
        } else if (LOOP == SPH_GRADIENT) {
            out[2 * si] = vsig;
            out[2 * si + 1] = acc[0];
        } else {
            const double hdt = active ? -(ei.w / 3.0) * qi.z / rhoi * acc[4] : 0.0;
            out[6 * si + 0] = active ? acc[0] : 0.0;
            out[6 * si + 1] = active ? acc[1] : 0.0;
            out[6 * si + 2] = active ? acc[2] : 0.0;
            out[6 * si + 3] = active ? acc[3] : 0.0;
            out[6 * si + 4] = hdt;
            out[6 * si + 5] = active ? vsig : 0.0;
        }
    }
}

// Pair interactions of a loop, decided in FP64 as the loops define them
// (density, gradient: r < H_i; force: r < max(H_i, H_j) for active i).
template <int LOOP>
__global__ void __launch_bounds__(128) k_count64(D64Args a, unsigned long long *count) {
    const BTargetDev &Tg = a.targets[blockIdx.x];
    const BCellDev C = a.cells[Tg.cell];
    const double4_32a *R0 = reinterpret_cast<const double4_32a *>(a.in + D64Layout::rec(0, a.S));
    const double4_32a *R3 = reinterpret_cast<const double4_32a *>(a.in + D64Layout::rec(3, a.S));
    unsigned long long mine = 0;
    for (int k = threadIdx.x; k < C.n; k += blockDim.x) {
        const long long si = (long long)C.slot + k;
        const double4_32a xi = R0[si];
        if (LOOP == SPH_FORCE && (int)R3[si].z > a.active_bin) continue;
        for (int e = Tg.nb0; e < Tg.nb0 + Tg.nnb; ++e) {
            const BCellDev Cn = a.cells[a.nbrs[e].cell];
            const int code = a.nbrs[e].code;
            double s[3];
            for (int d = 0; d < 3; ++d) {
                const int c = ((code >> (2 * d)) & 3) - 1;
                s[d] = c == 0 ? 0.0 : (c > 0 ? a.box[d] : -a.box[d]);
            }
            for (int q = 0; q < Cn.n; ++q) {
                const long long sj = (long long)Cn.slot + q;
                if (sj == si && code == kSelfCode) continue;
                const double4_32a xj = R0[sj];
                const double dx = xi.x - (xj.x + s[0]), dy = xi.y - (xj.y + s[1]),
                             dz = xi.z - (xj.z + s[2]);
                const double Hm = LOOP == SPH_FORCE ? fmax(xi.w, xj.w) : xi.w;
                mine += (dx * dx + dy * dy + dz * dz < Hm * Hm) ? 1 : 0;
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) mine += __shfl_xor_sync(0xffffffffu, mine, o);
    if ((threadIdx.x & 31) == 0 && mine) atomicAdd(count, mine);
}

struct D64UnpackArgs {
    const BCellDev *cells;
    const BTargetDev *targets;
    const double *out;
    const int32_t *perm;
    CompPtr dst[8];
};

// Add each target particle's FP64 result to the FP32 store (one rounding).
template <int LOOP>
__global__ void __launch_bounds__(128) k_unpack64(D64UnpackArgs a) {
    const BCellDev C = a.cells[a.targets[blockIdx.x].cell];
    constexpr int nv = LOOP == SPH_DENSITY ? 8 : (LOOP == SPH_GRADIENT ? 2 : 6);
    for (int k = threadIdx.x; k < C.n; k += blockDim.x) {
        const long long sl = (long long)C.slot + k;
        const long long p = a.perm[sl];
        for (int q = 0; q < nv; ++q) {
            const double v = a.out[nv * sl + q];
            const bool is_max = (LOOP == SPH_GRADIENT && q == 0) || (LOOP == SPH_FORCE && q == 5);
            const double cur = (double)ld<float>(a.dst[q], p);
            st<float>(a.dst[q], p, (float)(is_max ? fmax(cur, v) : cur + v));
        }
    }
}

// Ghost after density in FP64 (same definition as k_ghost), stored as FP32.
__global__ void k_ghost64(GhostArgs a, long long n, double kernel_gamma, double gamma,
                          double balsara_eps) {
    const double norm = 8.0 / 3.14159265358979323846;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n;
         p += (long long)gridDim.x * blockDim.x) {
        const double m = ld<float>(a.f[0], p), h = ld<float>(a.f[1], p), u = ld<float>(a.f[2], p);
        const double H = kernel_gamma * h;
        const double rho = (double)ld<float>(a.f[3], p) + m * norm / (H * H * H);
        const double rho_dh = (double)ld<float>(a.f[4], p) - 3.0 * m * norm / (H * H * H * H);
        const double wsum = ld<float>(a.f[5], p);
        const double wcount = wsum + 32.0 / 3.0;
        const double div = ld<float>(a.f[6], p) / rho;
        const double r0 = ld<float>(a.f[7], p) / rho, r1 = ld<float>(a.f[8], p) / rho,
                     r2 = ld<float>(a.f[9], p) / rho;
        const double omega = 1.0 + H / (3.0 * rho) * rho_dh;
        const double cs = sqrt(gamma * (gamma - 1.0) * u);
        const double arot = sqrt(r0 * r0 + r1 * r1 + r2 * r2);
        const double bal = fabs(div) / (fabs(div) + arot + balsara_eps * cs / h);
        st<float>(a.f[3], p, (float)rho);
        st<float>(a.f[4], p, (float)rho_dh);
        st<float>(a.f[5], p, (float)wcount);
        st<float>(a.f[6], p, (float)div);
        st<float>(a.f[7], p, (float)r0);
        st<float>(a.f[8], p, (float)r1);
        st<float>(a.f[9], p, (float)r2);
        st<float>(a.f[10], p, wsum == 0.0 ? 1.f : (float)(1.0 / omega));   // no neighbour: Omega = 0
        st<float>(a.f[11], p, (float)((gamma - 1.0) * rho * u));
        st<float>(a.f[12], p, (float)cs);
        st<float>(a.f[13], p, (float)bal);
    }
}

}  // namespace sph
