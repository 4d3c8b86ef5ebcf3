// Host check of div32 (division by an invariant as a multiplication, the
// face index decode of the flux kernels): for every divisor 1 .. 4100 and
// dividends at and around every multiple of the divisor near the ends of
// [0, 2^31), plus random dividends, prints the number of wrong quotients
// and the number of quotients checked.
#include <cstdio>
#include <random>
#define HK_HD inline
#include "hgks_device.cuh"

int main()
{
    unsigned long long bad = 0, total = 0;
    std::mt19937 rng(7);
    for (unsigned d = 1; d <= 4100; ++d) {
        const hk::Div32 v = hk::div32_of(d);
        auto check = [&](unsigned n) {
            if (n >= (1u << 31)) return;
            ++total;
            if (hk::div32(n, v) != n / d) ++bad;
        };
        for (unsigned q = 0; q < 3000; ++q)
            for (int e = -1; e <= 1; ++e) check(q * d + e);
        const unsigned top = (1u << 31) - 1;
        for (unsigned q = top / d - 3000; q <= top / d; ++q)
            for (int e = -1; e <= 1; ++e) check(q * d + e);
        for (int r = 0; r < 20000; ++r) check(rng() & 0x7fffffffu);
    }
    printf("%llu %llu\n", bad, total);
    return 0;
}
