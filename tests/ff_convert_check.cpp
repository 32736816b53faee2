// Host check of the split state's integer FP64 <-> float-float conversions (ff_convert.h)
// against the FP64 arithmetic they replace, bit for bit: pair_to_f64(h, l) against
// double(h) + double(l), f64_to_pair(v) against float(v), float(v - double(float(v))).
// Random and constructed cases cover every branch: equal and opposite signs, every binade gap
// between the words, a power-of-two high word with a borrow, exact ties, the carry into the
// next binade, zeros, subnormals, infinities and NaN. Prints "ok <cases>" or the first mismatch
// and exits 1.
#include <cinttypes>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <initializer_list>
#include <limits>

#include "ff_convert.h"

static uint64_t rng_state = 0x9E3779B97F4A7C15ull;
static uint64_t next_u64() {  // splitmix64
  uint64_t z = (rng_state += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

static uint64_t dbits(double x) {
  uint64_t u;
  std::memcpy(&u, &x, 8);
  return u;
}
static uint32_t fbits(float x) {
  uint32_t u;
  std::memcpy(&u, &x, 4);
  return u;
}
static float fmake(uint32_t sign, int biased_exp, uint32_t mant) {
  const uint32_t u = (sign << 31) | (uint32_t(biased_exp) << 23) | (mant & 0x7FFFFFu);
  float x;
  std::memcpy(&x, &u, 4);
  return x;
}

static long cases = 0;

static bool check_pair(float h, float l) {
  ++cases;
  const double want = double(h) + double(l);
  const double got = lem::pair_to_f64(h, l);
  const bool same = dbits(want) == dbits(got) || (std::isnan(want) && std::isnan(got));
  if (!same) {
    std::printf("pair_to_f64 mismatch: h %08" PRIx32 " l %08" PRIx32 " want %016" PRIx64 " got %016" PRIx64 "\n",
                fbits(h), fbits(l), dbits(want), dbits(got));
  }
  return same;
}

static bool check_split(double v) {
  ++cases;
  const float wh = float(v);
  const float wl = float(v - double(wh));
  float h, l;
  lem::f64_to_pair(v, h, l);
  const bool same = (fbits(wh) == fbits(h) || (std::isnan(wh) && std::isnan(h))) &&
                    (fbits(wl) == fbits(l) || (std::isnan(wl) && std::isnan(l)));
  if (!same) {
    std::printf("f64_to_pair mismatch: v %016" PRIx64 " want %08" PRIx32 " %08" PRIx32 " got %08" PRIx32 " %08" PRIx32
                "\n",
                dbits(v), fbits(wh), fbits(wl), fbits(h), fbits(l));
  }
  return same;
}

int main(int argc, char** argv) {
  const long n = argc > 1 ? std::atol(argv[1]) : 2000000;
  // 1. random high word (exponents across the normal range) and a low word at every binade gap
  //    0..70 below it, with random or sparse significands (sparse ones land on exact ties)
  for (long i = 0; i < n; ++i) {
    const uint64_t r = next_u64(), s = next_u64();
    const int eh = 1 + int(r % 254);
    const int gap = int((r >> 8) % 71);
    const int el = eh - gap;
    if (el < 1) continue;
    uint32_t mh = uint32_t(s) & 0x7FFFFFu, ml = uint32_t(s >> 23) & 0x7FFFFFu;
    switch ((r >> 16) % 4) {
      case 0: mh = 0; break;                                  // h a power of two
      case 1: ml = ml & 0x400001u; break;                     // sparse low word: ties
      case 2: mh = 0x7FFFFFu; break;                          // carry into the next binade
      default: break;
    }
    if (!check_pair(fmake(uint32_t(r >> 20) & 1u, eh, mh), fmake(uint32_t(r >> 21) & 1u, el, ml))) return 1;
  }
  // 2. exact ties and their neighbours: l = +-(half an FP64 ulp of h) (times 1 +- 2^-23), for
  //    odd and even h, and a quarter ulp for a power-of-two h (the lower binade's half ulp)
  for (int eh = 60; eh < 200; ++eh)
    for (uint32_t mh : {0u, 1u, 2u, 0x7FFFFFu, 0x7FFFFEu, 0x123457u})
      for (int gap = 52; gap <= 56; ++gap)
        for (uint32_t ml : {0u, 1u, 0x7FFFFFu})
          for (uint32_t sh = 0; sh < 2; ++sh)
            for (uint32_t sl = 0; sl < 2; ++sl)
              if (!check_pair(fmake(sh, eh, mh), fmake(sl, eh - gap, ml))) return 1;
  // 3. normalised pairs of random doubles (the split state's own pairs)
  for (long i = 0; i < n; ++i) {
    const uint64_t r = next_u64();
    const uint64_t e = 1023 - 100 + (next_u64() % 200);
    const double v = [&] {
      const uint64_t u = (r & 0x800FFFFFFFFFFFFFull) | (e << 52);
      double x;
      std::memcpy(&x, &u, 8);
      return x;
    }();
    const float h = float(v);
    const float l = float(v - double(h));
    if (!check_pair(h, l)) return 1;
    if (!check_split(v)) return 1;
  }
  // 4. special words: zeros, subnormals, infinities, NaN, the largest and smallest normals
  const float inf = std::numeric_limits<float>::infinity();
  const float specials[] = {0.0f, -0.0f, 1e-45f, -1e-45f, 1e-40f, 1.1754944e-38f, -1.1754944e-38f,
                            3.4028235e38f, -3.4028235e38f, inf, -inf, std::nanf(""), 1.0f, -1.0f,
                            1.0f + 1.1920929e-7f, 5.9604645e-8f, -5.9604645e-8f, 2.9802322e-8f};
  for (float a : specials)
    for (float b : specials)
      if (!check_pair(a, b)) return 1;
  for (int i = 0; i < 4096; ++i) {  // random normal h with a zero or subnormal l
    const uint64_t r = next_u64();
    const float h = fmake(uint32_t(r) & 1u, 1 + int((r >> 1) % 254), uint32_t(r >> 9));
    if (!check_pair(h, 0.0f) || !check_pair(h, -0.0f) || !check_pair(h, fmake(uint32_t(r >> 40) & 1u, 0, uint32_t(r >> 41))))
      return 1;
  }
  // 5. f64_to_pair at and around its range limits and across every exponent
  for (int E = -1080; E <= 1030; ++E)
    for (int k = 0; k < 64; ++k) {
      const uint64_t r = next_u64();
      const int be = E + 1023;
      if (be < 0 || be > 2047) continue;
      const uint64_t u = (r & 0x800FFFFFFFFFFFFFull) | (uint64_t(be) << 52);
      double v;
      std::memcpy(&v, &u, 8);
      if (!check_split(v)) return 1;
    }
  std::printf("ok %ld\n", cases);
  return 0;
}
