// FP64 <-> float-float (h + l, two floats) conversions of the split-precision state, built
// from the IEEE-754 bit layouts with integer operations: on this part an FP64 conversion or
// add issues on the slow FP64 pipe, and a kernel that converts one value per node would be
// bound by it. Each function returns exactly what the FP64 arithmetic it replaces returns
// (round to nearest even throughout); inputs outside the integer paths' ranges take that FP64
// arithmetic. The header compiles for the host too, where the CPU tests check the integer
// paths bit for bit against the FP64 arithmetic.
#pragma once

#include <cstdint>
#include <cstring>

#if defined(__CUDACC__)
#define LEM_FFC __host__ __device__ __forceinline__
#else
#define LEM_FFC inline
#endif

namespace lem {
namespace ffc {

LEM_FFC uint32_t f32_bits(float x) {
#if defined(__CUDA_ARCH__)
  return __float_as_uint(x);
#else
  uint32_t u;
  std::memcpy(&u, &x, sizeof u);
  return u;
#endif
}

LEM_FFC float f32_from_bits(uint32_t u) {
#if defined(__CUDA_ARCH__)
  return __uint_as_float(u);
#else
  float x;
  std::memcpy(&x, &u, sizeof x);
  return x;
#endif
}

LEM_FFC uint64_t f64_bits(double x) {
#if defined(__CUDA_ARCH__)
  return static_cast<uint64_t>(__double_as_longlong(x));
#else
  uint64_t u;
  std::memcpy(&u, &x, sizeof u);
  return u;
#endif
}

LEM_FFC double f64_from_bits(uint64_t u) {
#if defined(__CUDA_ARCH__)
  return __longlong_as_double(static_cast<long long>(u));
#else
  double x;
  std::memcpy(&x, &u, sizeof x);
  return x;
#endif
}

LEM_FFC float f32_rn(double v) {
#if defined(__CUDA_ARCH__)
  return __double2float_rn(v);
#else
  return static_cast<float>(v);
#endif
}

LEM_FFC float f32_rn_int(int v) {
#if defined(__CUDA_ARCH__)
  return __int2float_rn(v);
#else
  return static_cast<float>(v);
#endif
}

}  // namespace ffc

// FP64 -> float-float: h = v rounded to the nearest float, l = v - h rounded to the nearest
// float (what the FP64 conversions give). Exponents outside [-70, 100] (zero included) take
// the FP64 conversions.
LEM_FFC void f64_to_pair(double v, float& h, float& l) {
  const uint64_t b = ffc::f64_bits(v);
  const int E = int((b >> 52) & 0x7FFull) - 1023;
  if (E < -70 || E > 100) {
    h = ffc::f32_rn(v);
    l = ffc::f32_rn(v - double(h));
    return;
  }
  const uint64_t m = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);  // 53-bit significand
  uint64_t q = m >> 29;                                          // 24 bits
  const uint64_t rem = m & ((1ull << 29) - 1);
  if (rem > (1ull << 28) || (rem == (1ull << 28) && (q & 1ull))) ++q;  // round to nearest even
  const int diff = int(static_cast<int64_t>(m) - static_cast<int64_t>(q << 29));  // |diff| <= 2^28
  int e = E;
  if (q == (1ull << 24)) {  // rounded up to the next binade
    q >>= 1;
    ++e;
  }
  const uint32_t sign = uint32_t(b >> 63) << 31;
  h = ffc::f32_from_bits(sign | (uint32_t(e + 127) << 23) | uint32_t(q & 0x7FFFFFull));
  // v - h = sign * diff * 2^(E - 52), exact; its nearest float (+0 when it is 0, as in FP64)
  const float lf = ffc::f32_rn_int(diff) * ffc::f32_from_bits(uint32_t(E - 52 + 127) << 23);
  l = diff == 0 ? 0.0f : ffc::f32_from_bits(ffc::f32_bits(lf) ^ sign);
}

// float -> double (exact); zeros keep their sign, subnormals, infinities and NaN take the FP64
// conversion
LEM_FFC double f32_to_f64(float x) {
  const uint32_t b = ffc::f32_bits(x);
  const uint32_t ex = (b >> 23) & 0xFFu;
  if ((b & 0x7FFFFFFFu) == 0u) return ffc::f64_from_bits(uint64_t(b >> 31) << 63);
  if (ex == 0u || ex == 255u) return double(x);
  return ffc::f64_from_bits((uint64_t(b >> 31) << 63) | (uint64_t(ex - 127u + 1023u) << 52) |
                            (uint64_t(b & 0x7FFFFFu) << 29));
}

// float-float -> FP64: h + l rounded to the nearest FP64 value (ties to even), what the FP64
// add of the two exact conversions gives. With h a normal float and l = +-0 or a normal float
// at least 24 binades below h (every normalised pair, |l| <= ulp(h) / 2):
// - l = +-0, or l 55 or more binades below (|l| < a quarter of h's FP64 ulp): h itself;
// - otherwise the significands are added as integers, h's scaled to bits 62..39 of a 64-bit
//   word and l's aligned below it (bits shifted out of l leave a sticky flag; l of the
//   opposite sign borrows one when they do). A borrow below bit 62 (h a power of two, l of
//   the opposite sign) shifts the sum up one place and lowers the exponent. Bits 62..10 are
//   kept, rounded to nearest even on bit 9 and the bits and flag below it.
// Other pairs take the FP64 add.
LEM_FFC double pair_to_f64(float h, float l) {
  const uint32_t hb = ffc::f32_bits(h), lb = ffc::f32_bits(l);
  const int eh = int((hb >> 23) & 0xFFu), el = int((lb >> 23) & 0xFFu);
  const int d = eh - el;
  const bool h_normal = eh != 0 && eh != 255;
  const uint64_t sign = uint64_t(hb >> 31) << 63;
  const uint64_t mh = uint64_t((hb & 0x7FFFFFu) | 0x800000u);  // 24-bit significand
  if (h_normal && ((lb & 0x7FFFFFFFu) == 0u || (el != 0 && d >= 55)))
    return ffc::f64_from_bits(sign | (uint64_t(eh + 896) << 52) | ((mh & 0x7FFFFFu) << 29));
  if (h_normal && el != 0 && d >= 24) {  // (el = 255 gives d < 0)
    const uint64_t ml = uint64_t((lb & 0x7FFFFFu) | 0x800000u);
    uint64_t M = mh << 39;  // in [2^62, 2^63)
    uint64_t L;
    bool sticky;
    if (d <= 39) {
      L = ml << (39 - d);
      sticky = false;
    } else {  // d - 39 in [1, 15]
      L = ml >> (d - 39);
      sticky = (ml & ((1ull << (d - 39)) - 1)) != 0;
    }
    int e = eh;
    if (((hb ^ lb) >> 31) == 0u) {
      M += L;  // < 2^63: L < 2^39
    } else {
      M -= L + (sticky ? 1u : 0u);  // the dropped part of l, if any, as a borrow (sticky stays)
      if (M < (1ull << 62)) {      // > 2^61; the new bit 0 lies below the rounding bit
        M <<= 1;
        --e;
      }
    }
    uint64_t q = M >> 10;  // 53 bits
    const bool rbit = (M >> 9) & 1u;
    const bool rest = (M & 0x1FFu) != 0u || sticky;
    if (rbit && (rest || (q & 1u))) ++q;
    if (q == (1ull << 53)) {
      q >>= 1;
      ++e;
    }
    return ffc::f64_from_bits(sign | (uint64_t(e + 896) << 52) | (q & ((1ull << 52) - 1)));
  }
  return f32_to_f64(h) + f32_to_f64(l);
}

}  // namespace lem
