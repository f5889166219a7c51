// Device-side helpers and kernel argument records shared by the .cu files.
#pragma once

#include <cstdint>

#include "internal.h"

namespace sph {

constexpr float kPi = 3.14159265358979323846f;
constexpr float kNorm = 8.0f / kPi;  // cubic spline normalisation for support H

// Latched kernel error word, read back by sph_sync (bit 0: an index out of
// bounds, bit 1: a bounded wait ran out, bit 2: the neighbour-list pool ran
// out).
// All device code is compiled as one translation unit (api.cu).
__device__ unsigned int g_error_word = 0;

// Index check of the checked build (-DSPH_CHECK, libsph_check.so): an index
// outside [0, bound) latches bit 0 of the error word (SPH_EBOUNDS at
// sph_sync) and is replaced by 0, so the access stays inside the buffer.
// The default build compiles the check away.
__device__ __forceinline__ long long checked(long long i, long long bound) {
#ifdef SPH_CHECK
    if (i < 0 || i >= bound) {
        atomicOr(&g_error_word, 1u);
        return 0;
    }
#else
    (void)bound;
#endif
    return i;
}

template <typename T>
__device__ __forceinline__ T ld(const CompPtr &c, long long p) {
    return *reinterpret_cast<const T *>(c.ptr + p * c.stride);
}
template <typename T>
__device__ __forceinline__ void st(const CompPtr &c, long long p, T v) {
    *reinterpret_cast<T *>(c.ptr + p * c.stride) = v;
}

// Split an FP64 value into floats with x = hi + lo (to 2^-48 relative),
// using integer operations only: the slow FP64 pipe of the B300 is never
// touched.  hi is x rounded to 24 significant bits (round half up on the
// magnitude); lo is the rounded remainder.  Zero and |x| < 2^-74 give 0.
__device__ __forceinline__ void split_f64(double x, float &hi, float &lo) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int e = (int)((b >> 52) & 0x7FF);
    if (e < 1023 - 74) {
        hi = 0.f;
        lo = 0.f;
        return;
    }
    const unsigned long long m = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    int top = (int)(m >> 29);                    // 24 bits
    int rem = (int)(m & ((1ull << 29) - 1));     // 29 bits
    if (rem >= (1 << 28)) {
        top += 1;
        rem -= (1 << 29);
    }
    const int E = e - 1023;                      // x = m 2^(E - 52)
    const float s_hi = __int_as_float((E - 23 + 127) << 23);
    const float s_lo = __int_as_float((E - 52 + 127) << 23);
    float h = __int2float_rn(top) * s_hi;
    float l = __int2float_rn(rem) * s_lo;
    if (b >> 63) {
        h = -h;
        l = -l;
    }
    hi = h;
    lo = l;
}

// Cubic spline shape w(q) and its derivative, for q < 1 (callers mask q >= 1).
__device__ __forceinline__ void spline(float q, float &w, float &dw) {
    const float t = 1.f - q;
    const float wa = fmaf(q * q, fmaf(6.f, q, -6.f), 1.f);
    const float da = q * fmaf(18.f, q, -12.f);
    const float wb = 2.f * t * t * t;
    const float db = -6.f * t * t;
    const bool inner = q < 0.5f;
    w = inner ? wa : wb;
    dw = inner ? da : db;
}

}  // namespace sph
