// gc_bits.h -- exact IEEE-754 conversions and comparisons between float and
// double done with integer operations on the bit patterns.
//
// On GB300 every double-precision operation, conversions and comparisons
// included, runs on a narrow FP64 unit (about 1.6 lanes per SM per clock,
// ~150-190 cycles of latency in a dependent chain), while integer operations
// issue at the full ALU rate.  The per-carrier update keeps its FP64 position
// arithmetic, but the conversions between the FP32 field/displacement and
// the FP64 positions, and the FP64 threshold tests, need no FP64 unit: these
// helpers give the same results as the hardware conversions (round to
// nearest even) and comparisons, bit for bit, for every input they accept,
// and fall back to the hardware operation for the rare rest (subnormal,
// infinite or NaN values).  Plain C++ as well, so the CPU tests check them
// against the host's own conversions.
#pragma once
#include <cstdint>
#include <cstring>

#ifdef __CUDACC__
#define GC_HD __host__ __device__ __forceinline__
#else
#define GC_HD inline
#endif

namespace gc {

GC_HD uint64_t bits_of(double d) {
    uint64_t u;
    std::memcpy(&u, &d, sizeof u);
    return u;
}
GC_HD double double_of(uint64_t u) {
    double d;
    std::memcpy(&d, &u, sizeof d);
    return d;
}
GC_HD uint32_t bits_of(float f) {
    uint32_t u;
    std::memcpy(&u, &f, sizeof u);
    return u;
}
GC_HD float float_of(uint32_t u) {
    float f;
    std::memcpy(&f, &u, sizeof f);
    return f;
}

// The hardware conversions, for the rare inputs the integer paths leave to
// them.  In device code they are volatile so that the compiler keeps them in
// their branch instead of executing them for every thread.
GC_HD double f2d_hw(float f) {
#ifdef __CUDA_ARCH__
    double r;
    asm volatile("cvt.f64.f32 %0, %1;" : "=d"(r) : "f"(f));
    return r;
#else
    return (double)f;
#endif
}
GC_HD float d2f_hw(double d) {
#ifdef __CUDA_ARCH__
    float r;
    asm volatile("cvt.rn.f32.f64 %0, %1;" : "=f"(r) : "d"(d));
    return r;
#else
    return (float)d;
#endif
}

// (double)f: a normal float's exponent is rebiased (127 -> 1023) and its 23
// mantissa bits move to the top of the 52; zeros keep their sign.
GC_HD double f2d_exact(float f) {
    const uint32_t u = bits_of(f);
    const uint32_t e = (u >> 23) & 0xffu;
    const uint64_t sign = (uint64_t)(u & 0x80000000u) << 32;
    if (e == 0u || e == 0xffu) {
        if ((u & 0x7fffffffu) == 0u) return double_of(sign);  // +-0
        return f2d_hw(f);                                      // subnormal, inf, NaN
    }
    return double_of(sign | ((uint64_t)(e + 896u) << 52) | ((uint64_t)(u & 0x7fffffu) << 29));
}

// (float)d, rounded to nearest even, for results in the normal float range
// (and zeros); the rest by the hardware conversion.
GC_HD float d2f_exact(double d) {
    const uint64_t u = bits_of(d);
    const uint32_t sign = (uint32_t)(u >> 32) & 0x80000000u;
    const int e = (int)((u >> 52) & 0x7ffu) - 896;  // the float's biased exponent
    if ((u << 1) == 0u) return float_of(sign);       // +-0
    if (e < 1 || e > 254) return d2f_hw(d);          // subnormal, overflow, inf, NaN
    const uint64_t m = u & 0xfffffffffffffull;       // 52 mantissa bits
    uint32_t r = ((uint32_t)e << 23) | (uint32_t)(m >> 29);
    const uint32_t rest = (uint32_t)(m & 0x1fffffffu);  // the 29 dropped bits
    if (rest > 0x10000000u || (rest == 0x10000000u && (r & 1u))) ++r;  // may carry into the exponent
    if ((r >> 23) >= 0xffu) return d2f_hw(d);         // rounded up to infinity
    return float_of(sign | r);
}

// An integer key that orders doubles as their values do (for non-NaN
// values; -0 sorts just below +0).
GC_HD uint64_t order_key(double d) {
    const uint64_t u = bits_of(d);
    return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}
// a <= b and a > b for non-NaN doubles, exactly as the FP64 comparisons
// (zeros of either sign compare equal).
GC_HD bool le_exact(double a, double b) {
    if (((bits_of(a) | bits_of(b)) << 1) == 0u) return true;
    return order_key(a) <= order_key(b);
}
GC_HD bool gt_exact(double a, double b) { return !le_exact(a, b); }

}  // namespace gc
