// Arithmetic-peak microbenchmarks for the roofline of the interaction loops.
//
// The loops run on the FP32 CUDA cores (nothing in them is a dense
// contraction), and a separation in FP64 would use the FP64 pipe; their
// fraction of peak needs the peaks of those pipes on this GPU, measured
// rather than derived from unit counts.  Each thread runs kChains
// independent dependency chains (so the pipe, not the instruction latency,
// bounds it) of fused multiply-adds (2 flops) or adds (1 flop); the result
// is written only when it equals a value passed at run time, which the
// compiler cannot rule out, so no chain is removed.
#pragma once

namespace sph {

constexpr int kPeakChains = 8;
constexpr int kPeakUnroll = 16;

// KIND 0: FP32 fma, 1: FP64 fma, 2: FP64 add.
template <typename T, int KIND>
__global__ void __launch_bounds__(256, 8) k_peak(long long iters, T seed, T *sink) {
    T a[kPeakChains];
#pragma unroll
    for (int c = 0; c < kPeakChains; ++c) a[c] = seed + (T)(threadIdx.x + c);
    const T b = seed * (T)0.9999999, d = seed * (T)1e-7;
#pragma unroll 1
    for (long long k = 0; k < iters; ++k) {
#pragma unroll
        for (int u = 0; u < kPeakUnroll; ++u) {
#pragma unroll
            for (int c = 0; c < kPeakChains; ++c) {
                if constexpr (KIND == 2)
                    a[c] = a[c] + d;
                else
                    a[c] = fma(a[c], b, d);
            }
        }
    }
    T s = (T)0;
#pragma unroll
    for (int c = 0; c < kPeakChains; ++c) s += a[c];
    if (s == seed) sink[0] = s;
}

}  // namespace sph
