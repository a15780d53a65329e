// Host check of the invariant-divisor division (fastdiv.h): every dividend
// below 2^20 and the dividends near 2^32 and near multiples of d, plus
// pseudo-random 32-bit dividends, against the division operator, for the
// divisors given on the command line. Prints "ok" or the first mismatch.
#include <cstdint>
#include <cstdio>
#include <cstdlib>

#include "fastdiv.h"

int main(int argc, char** argv)
{
    uint64_t state = 0x9E3779B97F4A7C15ull;
    for (int a = 1; a < argc; ++a) {
        const uint32_t d = static_cast<uint32_t>(std::strtoul(argv[a], nullptr, 10));
        const mlqmc_dev::FastDiv f(d);
        auto check = [&](uint32_t x) {
            if (f.div(x) != x / d) {
                std::printf("mismatch d=%u x=%u got %u want %u\n", d, x, f.div(x), x / d);
                std::exit(1);
            }
        };
        for (uint32_t x = 0; x < (1u << 20); ++x) check(x);
        for (uint32_t k = 0; k < 4096; ++k) check(0xFFFFFFFFu - k);
        for (uint64_t q = 1; q * d < 0xFFFFFFFFull && q < (1ull << 16); q = q * 3 + 1)
            for (int o = -2; o <= 2; ++o) check(static_cast<uint32_t>(q * d + o));
        for (int k = 0; k < 200000; ++k) {
            state ^= state << 13;
            state ^= state >> 7;
            state ^= state << 17;
            check(static_cast<uint32_t>(state >> 11));
        }
    }
    std::printf("ok\n");
    return 0;
}
