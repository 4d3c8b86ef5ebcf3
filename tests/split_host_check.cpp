// Host build of split_f64 (the mixed path's q = hi + lo split of the device
// header, integer operations on the bit fields) against the plain form
// hi = (float)q, lo = (float)(q - (double)hi): prints the number of inputs
// whose hi or lo bits differ, and the number of inputs checked.  Inputs:
// every exponent from -80 to 130 with random fractions, the rounding cases
// built on purpose (the dropped bits exactly half, one above and below, with
// the kept bits odd and even; the kept bits all ones, so that hi carries into
// the exponent), zeros, subnormals, infinities, and random bit patterns.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <random>
#define HK_HD inline
#include "hgks_device.cuh"

static unsigned long long bad = 0, total = 0;

static void check(double q)
{
    float h1, l1;
    hk::split_f64(q, h1, l1);
    const float h0 = (float)q;
    const float l0 = (float)(q - (double)h0);
    uint32_t a, b, c, d;
    std::memcpy(&a, &h1, 4);
    std::memcpy(&b, &h0, 4);
    std::memcpy(&c, &l1, 4);
    std::memcpy(&d, &l0, 4);
    const bool nan_ok = std::isnan(h0) && std::isnan(h1) && std::isnan(l0) == std::isnan(l1);
    if (!nan_ok && (a != b || c != d)) ++bad;
    ++total;
}

static double from_bits(uint64_t u)
{
    double q;
    std::memcpy(&q, &u, 8);
    return q;
}

int main()
{
    std::mt19937_64 rng(12345);
    const uint64_t FRAC = (1ull << 52) - 1;
    for (int e = -80; e <= 130; ++e)
        for (int s = 0; s < 2; ++s) {
            const uint64_t top = ((uint64_t)s << 63) | ((uint64_t)(e + 1023) << 52);
            for (int r = 0; r < 20000; ++r) check(from_bits(top | (rng() & FRAC)));
            for (int r = 0; r < 2000; ++r) {
                // kept bits random (odd and even), dropped bits at and around half
                const uint64_t kept = (rng() & ((1ull << 23) - 1)) << 29;
                const uint64_t half = 1ull << 28;
                const uint64_t drops[6] = {half, half - 1, half + 1, 0, (1ull << 29) - 1, 1};
                for (uint64_t dr : drops) {
                    check(from_bits(top | kept | dr));
                    check(from_bits(top | kept | (1ull << 29) | dr));
                }
                // residual ties: dropped bits half plus a tie in their own low bits
                const uint64_t lowtie = (rng() & 0x1f) | 0x10;
                check(from_bits(top | kept | half | (rng() & (half - 1) & ~0x3full) | lowtie));
                check(from_bits(top | kept | (rng() & (half - 1) & ~0x3full) | (1ull << 25) | lowtie));
            }
            // kept bits all ones: hi carries into the exponent
            check(from_bits(top | (FRAC & ~((1ull << 29) - 1)) | (1ull << 28) | 1));
            check(from_bits(top | FRAC));
        }
    const double special[12] = {0.0, -0.0, (double)INFINITY, -(double)INFINITY, (double)NAN, 1e-310, -1e-310,
                                4.9e-324, 1e308, -1e308, 1.0, -1.0};
    for (double q : special) check(q);
    for (int r = 0; r < 100000000; ++r) check(from_bits(rng()));
    printf("%llu %llu\n", bad, total);
    return 0;
}
