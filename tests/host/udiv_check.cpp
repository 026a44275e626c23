// Checks udiv_invariant against the hardware divide for many divisors and
// dividends, including the extremes (compiled and run by test_host_logic.py).
#include <cstdio>
#include <random>
#include "ttv_udiv.h"

int main() {
    std::mt19937_64 g(12345);
    long bad = 0, checks = 0;
    const uint64_t fixed[] = {1, 2, 3, 5, 7, 10, 100, 500, 1000, 2000, 5000, 20000, 100000,
                              (1ull << 32) - 1, 1ull << 32, (1ull << 32) + 1, 1ull << 63, (1ull << 63) + 1,
                              ~0ull - 1, ~0ull, 12345678901ull};
    for (uint64_t d : fixed) {
        uint64_t m; uint32_t s;
        udiv_magic(d, m, s);
        for (int i = 0; i < 200000; ++i) {
            uint64_t n = i < 1000 ? (uint64_t)i : (i < 2000 ? ~0ull - (uint64_t)(i - 1000) : g() >> (g() % 64));
            if (i >= 2000 && i < 3000) n = d * (uint64_t)(i - 2000) + (i & 1 ? d - 1 : 0);
            ++checks;
            if (udiv_invariant(n, m, s) != n / d) ++bad;
        }
    }
    for (int k = 0; k < 100000; ++k) {
        uint64_t d = g() >> (g() % 64);
        if (!d) d = 1;
        uint64_t m; uint32_t s;
        udiv_magic(d, m, s);
        for (int i = 0; i < 20; ++i) {
            const uint64_t n = g() >> (g() % 64);
            ++checks;
            if (udiv_invariant(n, m, s) != n / d) ++bad;
        }
    }
    printf("checks=%ld bad=%ld\n", checks, bad);
    return bad != 0;
}
