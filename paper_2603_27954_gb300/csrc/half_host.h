// IEEE 754 binary16 <-> binary32 on the host, written from the format's
// definition (1 sign bit, 5 exponent bits with bias 15, 10 fraction bits;
// round to nearest, ties to even).  Used to encode initial fields and decode
// read-backs of FP16 population storage.
#pragma once
#include <cstdint>
#include <cstring>

namespace lbm {

inline uint16_t float_to_half_bits(float f) {
  uint32_t x;
  std::memcpy(&x, &f, 4);
  const uint32_t sign = (x >> 16) & 0x8000u;
  const uint32_t ax = x & 0x7fffffffu;
  if (ax >= 0x7f800000u) return (uint16_t)(sign | (ax > 0x7f800000u ? 0x7e00u : 0x7c00u));  // NaN, inf
  if (ax >= 0x477ff000u) return (uint16_t)(sign | 0x7c00u);  // >= 65520 rounds to inf
  const int e = (int)(ax >> 23);
  if (e < 113) {  // below 2^-14: subnormal half (or zero)
    if (e < 102) return (uint16_t)sign;  // below 2^-25: rounds to zero
    const uint32_t m = (ax & 0x7fffffu) | 0x800000u;
    const int shift = 126 - e;  // value in units of 2^-24 is m >> shift
    uint32_t q = m >> shift;
    const uint32_t rem = m & ((1u << shift) - 1u), halfway = 1u << (shift - 1);
    if (rem > halfway || (rem == halfway && (q & 1u))) ++q;
    return (uint16_t)(sign | q);
  }
  uint32_t h = ((uint32_t)(e - 112) << 10) | ((ax & 0x7fffffu) >> 13);
  const uint32_t rem = ax & 0x1fffu;
  if (rem > 0x1000u || (rem == 0x1000u && (h & 1u))) ++h;  // a carry may reach the exponent
  return (uint16_t)(sign | h);
}

inline float half_bits_to_float(uint16_t h) {
  const uint32_t sign = (uint32_t)(h & 0x8000u) << 16;
  const uint32_t e = (h >> 10) & 0x1fu, m = h & 0x3ffu;
  uint32_t x;
  if (e == 0) {
    const float v = (float)m * (1.0f / 16777216.0f);  // m * 2^-24, exact
    std::memcpy(&x, &v, 4);
    x |= sign;
  } else if (e == 31) {
    x = sign | 0x7f800000u | (m << 13);
  } else {
    x = sign | ((e + 112u) << 23) | (m << 13);
  }
  float f;
  std::memcpy(&f, &x, 4);
  return f;
}

}  // namespace lbm
