// Host check of the refined 1/sqrt method the FP64 contact kernel uses (the kernel's
// rsqrt_refined): narrow x to FP32 by exponent rebiasing, take an FP32 estimate y0 of
// 1/sqrt, widen it, and apply one third-order correction from the binomial series
// (1 - e)^(-1/2) = 1 + e/2 + 3e^2/8 + ..., e = 1 - x y0^2.  The host has no FP32
// hardware estimate, so the estimate is the correctly rounded FP32 1/sqrt moved by
// -K..K units in the last place (the device estimate is documented within 2 ulp);
// the result is compared with a long double 1/sqrt, in units of the double's last place.
// Prints "worst <ulps> over <count>" and exits 0.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <random>

static double as_double(long long v) { double d; std::memcpy(&d, &v, 8); return d; }
static long long as_bits(double d) { long long v; std::memcpy(&v, &d, 8); return v; }
static float as_float(int v) { float f; std::memcpy(&f, &v, 4); return f; }
static int as_int(float f) { int v; std::memcpy(&v, &f, 4); return v; }

static int g_shift = 0;   // ulps the FP32 estimate is moved by

static float estimate(float x) {
  const float y = (float)(1.0 / std::sqrt((double)x));
  return as_float(as_int(y) + g_shift);
}

// the kernel's steps, restated
static double rsqrt_refined(double x) {
  const long long xb = as_bits(x);
  const int ex = (int)(xb >> 52);
  if ((unsigned)(ex - 897) >= 252u) return 1.0 / std::sqrt(x);
  const float yf = estimate(as_float((int)((xb >> 29) - (896LL << 23))));
  const double y0 = as_double(((long long)as_int(yf) << 29) + (896LL << 52));
  const double half = as_double(as_bits(y0) - (1LL << 52));
#ifdef DROP_SECOND_ORDER   // a planted mistake: the series cut after e/2
  const double c = 0.0;
#else
  const double c = as_double(((long long)as_int(0.375f * yf) << 29) + (896LL << 52));
#endif
  const double e = std::fma(-(x * y0), y0, 1.0);
  return std::fma(e, std::fma(e, c, half), y0);
}

int main() {
  std::mt19937_64 rng(12345);
  std::uniform_real_distribution<double> expo(-120.0, 120.0), mant(0.0, 1.0);
  double worst = 0;
  long long n = 0;
  for (g_shift = -3; g_shift <= 3; ++g_shift) {
    for (int i = 0; i < 300000; ++i) {
      const double x = std::ldexp(1.0 + mant(rng), (int)expo(rng));
      const long double r = 1.0L / std::sqrt((long double)x);
      const double y = rsqrt_refined(x);
      const double ulp = std::ldexp(1.0, std::ilogb(y) - 52);
      const double err = (double)std::fabs((long double)y - r) / ulp;
      if (err > worst) worst = err;
      ++n;
    }
  }
  // arguments at the ends of the FP32 normal range and outside it (the fallback)
  const double edge[] = {0x1p-126, 0x1.fffffp-125, 0x1p124, 0x1.fffffp124, 0x1p-200, 0x1p200};
  g_shift = 0;
  for (double x : edge) {
    const long double r = 1.0L / std::sqrt((long double)x);
    const double y = rsqrt_refined(x);
    const double err = (double)std::fabs((long double)y - r) / std::ldexp(1.0, std::ilogb(y) - 52);
    if (err > worst) worst = err;
    ++n;
  }
  std::printf("worst %.6f over %lld\n", worst, n);
  return 0;
}
