// Host-side check of FastDiv (the invariant-divisor division used for lattice
// coordinates) against the hardware division: every divisor 1..2048, then large
// divisors, with dense and random numerators below 2^31.  Prints "ok" or the first failure.
#include <cstdio>
#include <cstdlib>

#include "ov_internal.cuh"

int main()
{
    unsigned long long state = 88172645463325252ull;
    auto rnd = [&]() {
        state ^= state << 13;
        state ^= state >> 7;
        state ^= state << 17;
        return (uint32_t)(state & 0x7fffffffu);
    };
    for (uint32_t d = 1; d <= 2048 + 64; ++d) {
        const uint32_t dd = d <= 2048 ? d : (1u << 26) - (d - 2048) * 977u;
        ov::FastDiv f(dd);
        for (uint32_t n = 0; n < 100000; ++n)
            if (f.div(n) != n / dd) { printf("fail d=%u n=%u\n", dd, n); return 1; }
        for (int i = 0; i < 100000; ++i) {
            const uint32_t n = rnd();
            if (f.div(n) != n / dd) { printf("fail d=%u n=%u\n", dd, n); return 1; }
        }
        const uint32_t edge[4] = {0x7fffffffu, 0x7ffffffeu, (0x7fffffffu / dd) * dd, (0x7fffffffu / dd) * dd - 1};
        for (uint32_t n : edge)
            if (f.div(n) != n / dd) { printf("fail d=%u n=%u\n", dd, n); return 1; }
    }
    printf("ok\n");
    return 0;
}
