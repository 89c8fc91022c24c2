// Host driver for the fixed-layout FP32 division and square roots of k_orbit.cu (div_nr, sqrt_nr,
// rsqrt_nr).  The hardware approximations they refine are replaced by the correctly rounded value
// moved by k units in the last place (the global nr_ulps), so that the refinement is checked against
// approximations as coarse as the hardware's.  For each k in -2..2 and a seeded set of operands it
// compares with the correctly rounded results (IEEE float division and square root on the host, and
// the FP64 reciprocal square root rounded to float) and prints, per function and k: the number of
// operands, the number not correctly rounded, the largest difference in units in the last place, and
// how many of the differing results lie above the exact value (the rest lie below).
#include "nr_host.h"

#include <cstdio>
#include <random>

static int64_t ulp_diff(float a, float b)
{
    int32_t ia, ib;
    std::memcpy(&ia, &a, 4);
    std::memcpy(&ib, &b, 4);
    if (ia < 0) ia = INT32_MIN - ia;
    if (ib < 0) ib = INT32_MIN - ib;
    return std::llabs((long long)ia - (long long)ib);
}

int main(int argc, char** argv)
{
    const int n = argc > 1 ? std::atoi(argv[1]) : 200000;
    std::mt19937_64 rng(20260607);
    std::uniform_real_distribution<double> lg(-3.0, 3.0), sg(0.0, 1.0);
    auto draw = [&](bool sign) {
        double v = std::pow(10.0, lg(rng));
        if (sign && sg(rng) < 0.5) v = -v;
        return (float)v;
    };
    for (int k = -2; k <= 2; ++k) {
        sw::nr_ulps = k;
        long long bad[3] = {0, 0, 0}, worst[3] = {0, 0, 0}, above[3] = {0, 0, 0};
        for (int i = 0; i < n; ++i) {
            const float a = draw(true), b = draw(true), x = draw(false);
            const float q = sw::div_nr(a, b), r = sw::sqrt_nr(x), s = sw::rsqrt_nr(x);
            const float q0 = a / b, r0 = std::sqrt(x), s0 = (float)(1.0 / std::sqrt((double)x));
            const int64_t d[3] = {ulp_diff(q, q0), ulp_diff(r, r0), ulp_diff(s, s0)};
            const bool up[3] = {(double)q > (double)a / (double)b, (double)r > std::sqrt((double)x),
                                (double)s > 1.0 / std::sqrt((double)x)};
            for (int f = 0; f < 3; ++f) {
                bad[f] += d[f] != 0;
                above[f] += d[f] != 0 && up[f];
                worst[f] = std::max<long long>(worst[f], d[f]);
            }
        }
        std::printf("div %d %d %lld %lld %lld\n", k, n, bad[0], worst[0], above[0]);
        std::printf("sqrt %d %d %lld %lld %lld\n", k, n, bad[1], worst[1], above[1]);
        std::printf("rsqrt %d %d %lld %lld %lld\n", k, n, bad[2], worst[2], above[2]);
    }
    return 0;
}
