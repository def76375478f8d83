// Host check of the integer-pipe conversions in md_fpconv.cuh against the
// CPU's IEEE-754 round-to-nearest-even conversions.  Exit status 0 when
// every case agrees; the first disagreement is printed.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <cfloat>

#include "md_fpconv.cuh"

using namespace mdk;

static uint64_t st = 0x9E3779B97F4A7C15ull;
static uint64_t next()  // splitmix64
{
    uint64_t z = (st += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static int fails = 0;
static void fail(const char *what, double in, double got, double want)
{
    if (fails++ < 5) printf("%s: input %.17g got %.17g want %.17g\n", what, in, got, want);
}

static void check_d2f(double x)
{
    const float got = d2f_bits(x);
    if (std::isnan(x)) {
        if (!std::isnan(got)) fail("d2f nan", x, got, NAN);
        return;
    }
    float want = (float)x;
    if (std::fabs(x) < (double)FLT_MIN) want = std::signbit(x) ? -0.0f : 0.0f;  // flush-to-zero
    if (fbits(got) != fbits(want)) fail("d2f", x, got, want);
}

static void check_f2d(float f)
{
    const double got = f2d_bits(f);
    if (std::isnan(f)) {
        if (!std::isnan(got)) fail("f2d nan", f, got, NAN);
        return;
    }
    double want = (double)f;
    if (f != 0.0f && std::fabs(f) < FLT_MIN) want = std::signbit(f) ? -0.0 : 0.0;  // subnormal input flushed
    if (dbits(got) != dbits(want)) fail("f2d", f, got, want);
}

int main()
{
    // FP32 -> FP64: every exponent, random fractions and signs
    for (int i = 0; i < 20000000; i++) check_f2d(bitsf((uint32_t)next()));
    const float fs[] = {0.0f, -0.0f, 1.0f, -1.0f, FLT_MIN, -FLT_MIN, FLT_MAX, -FLT_MAX, INFINITY, -INFINITY, NAN,
                        FLT_TRUE_MIN, 1e-40f, 3.0f, 0.1f};
    for (float f : fs) check_f2d(f);

    // FP64 -> FP32: random patterns over the whole exponent range, then
    // exponents that land in the float range with fraction tails at, just
    // below and just above the rounding tie
    for (int i = 0; i < 20000000; i++) check_d2f(bitsd(next()));
    for (int i = 0; i < 20000000; i++) {
        const uint64_t e = 897 + next() % 256;  // 2^-126 .. 2^129
        uint64_t frac = next() & 0xfffffffffffffull;
        const int k = (int)(next() % 5);
        if (k < 3) frac = (frac & ~0x1fffffffull) | (0x10000000ull + (uint64_t)k - 1);  // tie - 1, tie, tie + 1
        if (k == 3) frac |= 0x1fffffffull;
        check_d2f(bitsd((next() & (1ull << 63)) | (e << 52) | frac));
    }
    const double ds[] = {0.0, -0.0, 1.0, -1.0, (double)FLT_MIN, (double)FLT_MAX, 3.4028235677973366e38,
                         3.4028234663852886e38 + 1e22, 1e39, -1e39, 1e-39, -1e-46, INFINITY, -INFINITY, NAN,
                         0.1, 1.0 / 3.0, 0.9999999999999999, 1.0000000596046448, 1.0000001192092896};
    for (double d : ds) check_d2f(d);

    // k + 1/2
    for (int k = 0; k < (1 << 22); k++)
        if (int_plus_half(k) != (double)k + 0.5) fail("int_plus_half", k, int_plus_half(k), (double)k + 0.5);
    for (int i = 0; i < 1000000; i++) {
        const int k = (int)(next() % (1u << 30));
        if (int_plus_half(k) != (double)k + 0.5) fail("int_plus_half", k, int_plus_half(k), (double)k + 0.5);
    }

    // floor of a double in [0, 2^31): random values, integers and their
    // neighbours one ulp away
    for (int i = 0; i < 20000000; i++) {
        const double y = std::ldexp((double)(next() >> 11), -53) * std::ldexp(1.0, (int)(next() % 32));
        if (floor_bits(y) != (int)std::floor(y)) fail("floor", y, floor_bits(y), std::floor(y));
    }
    for (int i = 0; i < 1000000; i++) {
        const double n = (double)(next() % 0x7fffffffull);
        const double ys[] = {n, std::nextafter(n, 0.0), std::nextafter(n, 1e300)};
        for (double y : ys)
            if (y < 2147483648.0 && floor_bits(y) != (int)std::floor(y)) fail("floor", y, floor_bits(y), std::floor(y));
    }
    if (floor_bits(-0.5) != -1 || floor_bits(-1e300) != -1 || floor_bits(-0.0) != -1) fail("floor neg", -0.5, 0, -1);
    if (floor_bits(2147483648.0) != 0x7fffffff || floor_bits(INFINITY) != 0x7fffffff) fail("floor big", 2e9, 0, 0);
    if (floor_bits(0.0) != 0 || floor_bits(0.999) != 0 || floor_bits(1e-300) != 0) fail("floor small", 0, 0, 0);

    printf("%s (%d disagreements)\n", fails ? "FAIL" : "ok", fails);
    return fails ? 1 : 0;
}
