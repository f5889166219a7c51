// pack and unpack (Sec. 2.3) as gather / ordered-reduction kernels.
//
// pack: one CTA per task; thread k copies slot k of the task (ci's particles
// first, then cj's), reading the loop's view from the store layout and
// writing the lanes of the bundle buffer.  Consecutive threads touch
// consecutive particles and consecutive slots, so every lane store is a
// contiguous (coalesced) warp access; {v, m} goes out as one 16-byte store.
// The periodic shift is one FP64 add on cj's positions where the task wraps.
//
// unpack: one CTA per touched cell of the bundle; thread i owns particle i
// of the cell and folds its slots in increasing task order.  Sums use Kahan's
// compensated summation in FP32 from the stored value (the B300's FP64 pipe
// is far slower than its FP32 pipe); maxima are exact.  No atomics: the
// result is deterministic and bit-reproducible.
#pragma once
#include "device.cuh"

namespace sph {

// Source roles of the pack views (density uses 0..7, gradient 0..9, force
// 0..14).
enum PackRole {
    R_X0 = 0, R_X1, R_X2, R_V0, R_V1, R_V2, R_M, R_H, R_U, R_RHO, R_FGH,
    R_BAL, R_AV, R_AD, R_TB, R_NUM
};

struct PackArgs {
    const TaskDev *tasks;  // the bundle's tasks
    char *lane[12];        // bundle buffer lanes
    CompPtr src[R_NUM];    // store addresses of the view components
    double box[3];
};

template <int LOOP>
__global__ void __launch_bounds__(128) k_pack(PackArgs a) {
    const TaskDev T = a.tasks[blockIdx.x];
    const int n = T.ni + T.nj;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        const bool side = k >= T.ni;
        const long long p = side ? (long long)T.pj + (k - T.ni) : (long long)T.pi + k;
        const long long s = (long long)T.slot + k;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            double xv = ld<double>(a.src[R_X0 + d], p);
            const int code = side ? ((T.shift >> (2 * d)) & 3) - 1 : 0;
            if (code != 0) xv = xv + (code > 0 ? a.box[d] : -a.box[d]);
            reinterpret_cast<double *>(a.lane[d])[s] = xv;
        }
        const float4 vm = make_float4(ld<float>(a.src[R_V0], p), ld<float>(a.src[R_V1], p),
                                      ld<float>(a.src[R_V2], p), ld<float>(a.src[R_M], p));
        reinterpret_cast<float4 *>(a.lane[3])[s] = vm;
        reinterpret_cast<float *>(a.lane[4])[s] = ld<float>(a.src[R_H], p);
        if (LOOP >= SPH_GRADIENT) {
            reinterpret_cast<float *>(a.lane[5])[s] = ld<float>(a.src[R_U], p);
            reinterpret_cast<float *>(a.lane[6])[s] = ld<float>(a.src[R_RHO], p);
        }
        if (LOOP == SPH_FORCE) {
            reinterpret_cast<float *>(a.lane[7])[s] = ld<float>(a.src[R_FGH], p);
            reinterpret_cast<float *>(a.lane[8])[s] = ld<float>(a.src[R_BAL], p);
            reinterpret_cast<float *>(a.lane[9])[s] = ld<float>(a.src[R_AV], p);
            reinterpret_cast<float *>(a.lane[10])[s] = ld<float>(a.src[R_AD], p);
            reinterpret_cast<int8_t *>(a.lane[11])[s] = ld<int8_t>(a.src[R_TB], p);
        }
    }
}

// Output roles of unpack:
//   density : 0 rho, 1 rho_dh, 2 wcount, 3 wcount_dh, 4 div_v, 5..7 rot_v
//   gradient: 0 v_sig_grad (max), 1 laplace_u
//   force   : 0..2 a, 3 u_dt, 4 h_dt, 5 v_sig (max)
struct UnpackArgs {
    const UCellDev *cells;
    const int32_t *entries;  // the bundle's entry base
    const char *lane[2];
    CompPtr dst[8];
};

constexpr int kMaxEntries = 27;  // a cell is in at most 1 self + 26 pair tasks

// Kahan step: y = x - c; t = s + y; c = (t - s) - y; s = t.  Plain FP32 adds
// (no multiplies, so nothing can be contracted into an FMA).
struct Kahan {
    float s, c;
    __device__ __forceinline__ void init(float v) { s = v; c = 0.f; }
    __device__ __forceinline__ void add(float x) {
        const float y = __fsub_rn(x, c);
        const float t = __fadd_rn(s, y);
        c = __fsub_rn(__fsub_rn(t, s), y);
        s = t;
    }
};

template <int LOOP>
__global__ void __launch_bounds__(128) k_unpack(UnpackArgs a) {
    __shared__ int32_t ent[kMaxEntries];
    const UCellDev C = a.cells[blockIdx.x];
    const int ne = C.ne < kMaxEntries ? C.ne : kMaxEntries;
    if (threadIdx.x == 0 && C.ne > kMaxEntries) atomicOr(&g_error_word, 1u);
    for (int k = threadIdx.x; k < ne; k += blockDim.x) ent[k] = a.entries[C.e0 + k];
    __syncthreads();
    for (int i = threadIdx.x; i < C.n; i += blockDim.x) {
        const long long p = (long long)C.p0 + i;
        if (LOOP == SPH_DENSITY) {
            Kahan acc[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) acc[q].init(ld<float>(a.dst[q], p));
            for (int e = 0; e < ne; ++e) {
                const long long s = (long long)ent[e] + i;
                const float4 o0 = reinterpret_cast<const float4 *>(a.lane[0])[s];
                const float4 o1 = reinterpret_cast<const float4 *>(a.lane[1])[s];
                acc[0].add(o0.x); acc[1].add(o0.y); acc[2].add(o0.z); acc[3].add(o0.w);
                acc[4].add(o1.x); acc[5].add(o1.y); acc[6].add(o1.z); acc[7].add(o1.w);
            }
#pragma unroll
            for (int q = 0; q < 8; ++q) st<float>(a.dst[q], p, acc[q].s);
        } else if (LOOP == SPH_GRADIENT) {
            float vs = ld<float>(a.dst[0], p);
            Kahan lap;
            lap.init(ld<float>(a.dst[1], p));
            for (int e = 0; e < ne; ++e) {
                const long long s = (long long)ent[e] + i;
                const float2 o = reinterpret_cast<const float2 *>(a.lane[0])[s];
                vs = fmaxf(vs, o.x);
                lap.add(o.y);
            }
            st<float>(a.dst[0], p, vs);
            st<float>(a.dst[1], p, lap.s);
        } else {
            Kahan acc[5];
#pragma unroll
            for (int q = 0; q < 5; ++q) acc[q].init(ld<float>(a.dst[q], p));
            float vs = ld<float>(a.dst[5], p);
            for (int e = 0; e < ne; ++e) {
                const long long s = (long long)ent[e] + i;
                const float4 o0 = reinterpret_cast<const float4 *>(a.lane[0])[s];
                const float2 o1 = reinterpret_cast<const float2 *>(a.lane[1])[s];
                acc[0].add(o0.x); acc[1].add(o0.y); acc[2].add(o0.z); acc[3].add(o0.w);
                acc[4].add(o1.x);
                vs = fmaxf(vs, o1.y);
            }
#pragma unroll
            for (int q = 0; q < 5; ++q) st<float>(a.dst[q], p, acc[q].s);
            st<float>(a.dst[5], p, vs);
        }
    }
}

}  // namespace sph
