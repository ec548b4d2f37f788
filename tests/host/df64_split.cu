// Host check of df64::from_double, the integer-instruction split of an FP64
// value into an FP32 pair that the FP32 / DF64 residual reads: for random
// values over the FP32 range, hi is the FP32 value nearest v (up to ties),
// |v - (hi + lo)| <= 2^-48 |v|, and the special cases behave as documented.
// Prints "ok" and exits 0, else prints the first failure and exits 1.
#include <cmath>
#include <cstdio>
#include <random>

#include "et_df64_arith.h"

using et::df64::from_double;

static int fail(const char* what, double v, float2 p) {
    std::printf("FAIL %s: v=%.17g hi=%.9g lo=%.9g\n", what, v, (double)p.x, (double)p.y);
    return 1;
}

int main() {
    std::mt19937_64 gen(7);
    std::uniform_real_distribution<double> mant(0.5, 1.0);
    std::uniform_int_distribution<int> expo(-69, 127);
    for (int t = 0; t < 4000000; ++t) {
        double v = std::ldexp(mant(gen), expo(gen));
        if (t & 1) v = -v;
        const float2 p = from_double(v);
        const double s = (double)p.x + (double)p.y;  // exact: the two parts span at most 53 bits
        if (!(std::fabs(s - v) <= std::ldexp(std::fabs(v), -48))) return fail("error bound", v, p);
        const float nearest = (float)v;
        if (p.x != nearest) {
            // allowed only for an exact tie, which the split rounds away from zero
            const double d1 = std::fabs((double)p.x - v), d2 = std::fabs((double)nearest - v);
            if (d1 != d2) return fail("hi is not the nearest float", v, p);
        }
    }
    const float2 z = from_double(0.0), nz = from_double(-0.0);
    if (z.x != 0.f || z.y != 0.f || std::signbit(z.x) || !std::signbit(nz.x)) return fail("zeros", 0.0, z);
    const float2 tiny = from_double(1e-300);
    if (tiny.x != 0.f || tiny.y != 0.f) return fail("below the FP32 range", 1e-300, tiny);
    const float2 huge = from_double(1e300);
    if (!std::isinf(huge.x) || huge.y != 0.f) return fail("beyond the FP32 range", 1e300, huge);
    const float2 inf = from_double(-INFINITY), nan = from_double(NAN);
    if (!(std::isinf(inf.x) && inf.x < 0) || !std::isnan(nan.x)) return fail("inf / nan", NAN, nan);
    const float2 one = from_double(1.0 + std::ldexp(1.0, -30));
    if (one.x != 1.f || one.y != std::ldexp(1.f, -30)) return fail("1 + 2^-30", 1.0 + std::ldexp(1.0, -30), one);
    std::printf("ok\n");
    return 0;
}
