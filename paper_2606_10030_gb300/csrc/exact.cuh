// Exactly rounded float sums: the arithmetic shared by the device kernels
// (exact.cu) and a host build of the same functions used by the unit tests.
//
// A group's sum is kept as an integer N in units of 2^base, held as signed
// base-2^28 digits in int64 words (digit k weighs 2^(28 k)). A row adds its
// significand, shifted into place, as three chunks of at most 28 bits, so a
// word takes less than 2^28 per row and cannot overflow before 2^35 rows.
// Rounding propagates the carries, takes the 53 bits below the highest set
// bit of |N|, the next bit and whether anything below it is set, and rounds
// to nearest, ties to even: the exact real sum rounded once to float64.
#pragma once

#include <stdint.h>

#ifdef __CUDACC__
#define AGG_HD __host__ __device__ __forceinline__
#define AGG_LDEXP ldexp
#else
#include <cmath>
#define AGG_HD inline
#define AGG_LDEXP std::ldexp
#endif

namespace agg {

constexpr int kDigitBits = 28;
constexpr int64_t kDigitMask = (int64_t(1) << kDigitBits) - 1;
// Digits for the widest float64 column: units of 2^-1074 up to 2^1024 times
// 2^32 rows, plus slack for the chunk alignment.
constexpr int kMaxDigits = 84;

// A finite float as (sign, significand, exponent of its least significant bit).
struct ExactParts {
  bool neg;
  uint64_t mant;
  int lsb;
};

AGG_HD ExactParts exact_parts_f64(uint64_t b) {
  const int e = (int)((b >> 52) & 0x7FF);
  const uint64_t f = b & ((uint64_t(1) << 52) - 1);
  ExactParts p;
  p.neg = (b >> 63) != 0;
  p.mant = e ? (f | (uint64_t(1) << 52)) : f;
  p.lsb = e ? e - 1075 : -1074;
  return p;
}

AGG_HD ExactParts exact_parts_f32(uint32_t b) {
  const int e = (int)((b >> 23) & 0xFF);
  const uint64_t f = b & ((1u << 23) - 1);
  ExactParts p;
  p.neg = (b >> 31) != 0;
  p.mant = e ? (f | (uint64_t(1) << 23)) : f;
  p.lsb = e ? e - 150 : -149;
  return p;
}

// The significand shifted left by r (0 <= r < 28) as three digits' worth of
// chunks c[0..2] (c[2] < 2^25 for a 53-bit significand).
AGG_HD void exact_chunks(uint64_t mant, int r, int64_t* c) {
  const uint64_t lo = mant << r;
  const uint64_t hi = r ? mant >> (64 - r) : 0;
  c[0] = (int64_t)(lo & (uint64_t)kDigitMask);
  c[1] = (int64_t)((lo >> kDigitBits) & (uint64_t)kDigitMask);
  c[2] = (int64_t)((lo >> (2 * kDigitBits)) | (hi << (64 - 2 * kDigitBits)));
}

// Carry propagation: afterwards a[k] is in [0, 2^28) for k < D - 1 and a[D - 1]
// holds the rest, its sign that of N.
AGG_HD void exact_carry(int64_t* a, int D) {
  for (int k = 0; k < D - 1; ++k) {
    const int64_t c = a[k] >> kDigitBits;  // floor division by 2^28
    a[k] -= c * (int64_t(1) << kDigitBits);
    a[k + 1] += c;
  }
}

// Bits [pos, pos + len) of the nonnegative normalised digits (len <= 60;
// bits below 0 are zero).
AGG_HD uint64_t exact_bits(const int64_t* a, int D, int pos, int len) {
  uint64_t v = 0;
  const int k0 = pos >= 0 ? pos / kDigitBits : -((-pos + kDigitBits - 1) / kDigitBits);
  for (int k = k0; k * kDigitBits < pos + len; ++k) {
    if (k < 0 || k >= D) continue;
    const int sh = k * kDigitBits - pos;  // where digit k's bit 0 lands in v
    const uint64_t dk = (uint64_t)a[k];
    if (sh >= 0) {
      if (sh < 64) v |= dk << sh;
    } else {
      v |= dk >> (-sh);
    }
  }
  return len >= 64 ? v : (v & ((uint64_t(1) << len) - 1));
}

// Whether any of the bits [0, pos) is set.
AGG_HD bool exact_any_below(const int64_t* a, int D, int pos) {
  if (pos <= 0) return false;
  const int kp = pos / kDigitBits;
  for (int k = 0; k < kp && k < D; ++k)
    if (a[k] != 0) return true;
  const int r = pos - kp * kDigitBits;
  return kp < D && r > 0 && (a[kp] & ((int64_t(1) << r) - 1)) != 0;
}

// N x 2^base rounded to the nearest float64 (ties to even). a[] is
// overwritten. An all-zero N gives +0.0.
AGG_HD double exact_round(int64_t* a, int D, int base) {
  exact_carry(a, D);
  const bool neg = a[D - 1] < 0;
  if (neg) {
    for (int k = 0; k < D; ++k) a[k] = -a[k];
    exact_carry(a, D);
  }
  int top = D - 1;
  while (top >= 0 && a[top] == 0) --top;
  if (top < 0) return 0.0;
  int hb = 0;
  while (hb < 62 && (a[top] >> (hb + 1)) != 0) ++hb;
  int H = top * kDigitBits + hb;  // the highest set bit of |N|
  uint64_t mant = exact_bits(a, D, H - 52, 53);
  const int R = H - 53;  // the round bit
  const bool rbit = R >= 0 && exact_bits(a, D, R, 1) != 0;
  const bool sticky = exact_any_below(a, D, R);
  if (rbit && (sticky || (mant & 1))) {
    ++mant;
    if (mant == (uint64_t(1) << 53)) {
      mant >>= 1;
      ++H;
    }
  }
  const double v = AGG_LDEXP((double)mant, H - 52 + base);
  return neg ? -v : v;
}

}  // namespace agg
