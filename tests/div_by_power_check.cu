// Host-only check of the FP64 form's division by powers d^k: the kernels'
// compile-time reciprocal table holds RN(1 / d^k), and div_by_power, run here
// on the host with the same fused multiply-adds, equals IEEE division a / d^k
// for every d = 1..255, k = 1..6 on edge and random dividends a = RN(M),
// 0 <= M <= 6561 d^k (the range of the window moments), and on theta - alpha
// and large separable-path moments.  Prints the counts of mismatches; no GPU
// is used.
#include <cmath>
#include <cstdint>
#include <cstdio>

#include "../paper_1811_02308_gb300/csrc/fabf_device.cuh"

int main()
{
    constexpr fabf::RecipPowTable t = fabf::make_recip_pow_table();
    uint64_t x = 88172645463325252ull;
    long long bad = 0, total = 0, bad_table = 0;
    for (int d = 1; d <= 255; ++d) {
        uint64_t bk = 1;
        for (int k = 1; k <= 6; ++k) {
            bk *= (uint64_t)d;
            const double b = (double)bk;
            volatile double one = 1.0;
            if (t.v[k - 1][d] != one / b) ++bad_table;
            if (t.p[k - 1][d] != b) ++bad_table;
            const double r = t.v[k - 1][d];
            const uint64_t mmax = 6561ull * bk;
            for (int i = 0; i < 2000; ++i) {
                uint64_t M;
                if (i < 32) M = (uint64_t)i;
                else if (i < 64) M = mmax - (uint64_t)(i - 32);
                else if (i < 128) M = bk * (uint64_t)(i - 64) + (uint64_t)(i & 1);
                else {
                    x ^= x << 13;
                    x ^= x >> 7;
                    x ^= x << 17;
                    M = x % (mmax + 1);
                }
                const double a = (double)M;
                volatile double bb = b;
                ++total;
                if (fabf::div_by_power(a, b, r) != a / bb) ++bad;
            }
        }
    }
    // Other dividends the kernels divide by d^k: theta - alpha for t0 (a
    // binary32 theta less an integer alpha, any sign, k = 1) and the
    // separable path's 128-bit moments rounded to binary64 (up to 2^40 d^k).
    long long total2 = 0, bad2 = 0;
    for (int d = 1; d <= 255; ++d) {
        for (int k = 1; k <= 6; ++k) {
            const double b = t.p[k - 1][d];
            const double r = t.v[k - 1][d];
            for (int i = 0; i < 1000; ++i) {
                x ^= x << 13;
                x ^= x >> 7;
                x ^= x << 17;
                double a;
                if (k == 1 && (i & 1)) {
                    const float th = (float)((double)(x >> 11) * 0x1p-53 * 2000.0 - 1000.0);
                    a = (double)th - (double)(int)((x >> 3) & 255);
                } else {
                    // (x >> 24) < 2^40 times d^k, rounded; then 10 more random low bits
                    a = (double)(x >> 24) * b;
                    a = a * (1.0 + (double)((x >> 5) & 1023) * 0x1p-30);
                }
                volatile double bb = b;
                ++total2;
                if (fabf::div_by_power(a, b, r) != a / bb) ++bad2;
            }
        }
    }
    std::printf("%lld %lld %lld %lld %lld\n", total, bad, bad_table, total2, bad2);
    return 0;
}
