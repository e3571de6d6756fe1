// Checks the integer-operation float <-> double conversions and comparisons
// of gc_bits.h against the host's own conversions (round to nearest even)
// and comparisons.  Exit status 0 and "bits ok" when every case agrees.
#include <cmath>
#include <cstdio>
#include <limits>
#include <random>

#include "gc_bits.h"

using namespace gc;

static int bad = 0;

static void check_f2d(float f) {
    const double want = (double)f, got = f2d_exact(f);
    if (std::isnan(want) ? !std::isnan(got) : bits_of(want) != bits_of(got)) {
        if (bad++ < 5) std::printf("f2d mismatch: %08x\n", bits_of(f));
    }
}
static void check_d2f(double d) {
    const float want = (float)d, got = d2f_exact(d);
    if (std::isnan(want) ? !std::isnan(got) : bits_of(want) != bits_of(got)) {
        if (bad++ < 5) std::printf("d2f mismatch: %016llx\n", (unsigned long long)bits_of(d));
    }
}
static void check_cmp(double a, double b) {
    if (std::isnan(a) || std::isnan(b)) return;
    if (le_exact(a, b) != (a <= b) || gt_exact(a, b) != (a > b)) {
        if (bad++ < 5)
            std::printf("cmp mismatch: %016llx %016llx\n", (unsigned long long)bits_of(a),
                        (unsigned long long)bits_of(b));
    }
}

int main() {
    std::mt19937_64 rng(12345);
    // float -> double: every exponent and sign, 2^16 mantissas each, plus every special value
    for (uint32_t s = 0; s < 2; ++s)
        for (uint32_t e = 0; e < 256; ++e)
            for (uint32_t k = 0; k < 65536; ++k) {
                const uint32_t m = k < 4 ? (k == 3 ? 0x7fffffu : k) : (uint32_t)(rng() & 0x7fffffu);
                check_f2d(float_of((s << 31) | (e << 23) | m));
            }
    // double -> float: every double exponent, random mantissas; then rounding ties
    // and their neighbours at every float exponent
    for (uint64_t s = 0; s < 2; ++s)
        for (uint64_t e = 0; e < 2048; ++e)
            for (int k = 0; k < 4096; ++k) {
                const uint64_t m = k < 2 ? (uint64_t)k * 0xfffffffffffffull : (rng() & 0xfffffffffffffull);
                check_d2f(double_of((s << 63) | (e << 52) | m));
            }
    for (uint64_t e = 1023 - 160; e <= 1023 + 130; ++e)
        for (int k = 0; k < 2048; ++k) {
            const uint64_t hi = (rng() & 0x7fffffull) << 29;
            for (int64_t dlt = -2; dlt <= 2; ++dlt) {
                const uint64_t m = (hi | 0x10000000ull) + (uint64_t)dlt;  // a tie and its neighbours
                check_d2f(double_of((e << 52) | (m & 0xfffffffffffffull)));
                check_d2f(double_of((1ull << 63) | (e << 52) | (m & 0xfffffffffffffull)));
            }
        }
    const double edge[] = {0.0, -0.0, 1.0, -1.0, 675.0, 1e-300, -1e-300, 3.4028234663852886e38,
                           3.4028235677973366e38, 1.1754943508222875e-38, 1.1754942807573643e-38,
                           std::numeric_limits<double>::infinity(), -std::numeric_limits<double>::infinity(),
                           std::numeric_limits<double>::denorm_min(), 1e308};
    for (double d : edge) check_d2f(d);
    // comparisons: random values in a few ranges, equal values, zeros of both signs
    std::uniform_real_distribution<double> U(-1000.0, 1000.0);
    for (int k = 0; k < 4000000; ++k) {
        double a = U(rng), b = U(rng);
        if (k % 7 == 0) b = a;
        if (k % 11 == 0) a = (k & 1) ? 0.0 : -0.0;
        if (k % 13 == 0) b = (k & 2) ? 0.0 : -0.0;
        if (k % 17 == 0) b = std::nextafter(a, 2000.0);
        if (k % 19 == 0) a = double_of(rng());
        check_cmp(a, b);
        check_cmp(b, a);
    }
    for (double a : edge)
        for (double b : edge) check_cmp(a, b);
    if (bad) {
        std::printf("bits: %d mismatches\n", bad);
        return 1;
    }
    std::printf("bits ok\n");
    return 0;
}
