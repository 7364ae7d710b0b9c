// Digit arithmetic of the FP64-accurate split products (block updates): the row-scaled
// 54-bit integer of an FP64 value cut into seven base-256 digits, and the exact rounding of
// the recombined levels back to FP64.  Shared by the tensor-core update kernels.
//
// Digits: a = |x| 2^(55 - E) truncated to an integer, E the row exponent (|x| < 2^E), so
// a < 2^55, written as a = t 2^48 + c1 2^24 + c2 (t <= 127, c < 2^24), each 24-bit chunk
// c = d0 2^16 + d1 2^8 + d2 with d0 in [0, 256] and |d1|, |d2| <= 128 (two FP32 roundings,
// exact), the sign of x applied to every digit.  Integers up to 256 are exact in BF16; digit
// i weighs 2^(E - 7 - 8 i).  The truncation error is below 2^-55 of the row maximum.
//
// Exactness of the level sums: with these digit bounds the products d_i(A) d_j(Y) of one
// level l = i + j add up to at most 196352 (l = 5; 163840 to 179968 for l = 6, 7) per
// contraction index, so over p <= 64 indices every partial sum is an integer below 2^23.6,
// exact in an FP32 accumulator.
#pragma once

#include <cuda_bf16.h>

#include <cstdint>

namespace tps {
namespace b256 {

constexpr int kUS = 7;                // base-256 digits per operand
constexpr int kUL = 8;                // digit-pair levels kept: i + j <= 7
constexpr float kMagic = 12582912.f;  // 1.5 2^23: x + kMagic - kMagic = rint(x), |x| <= 2^22

__device__ __forceinline__ unsigned raw_exp(double x) {
  return (unsigned)((__double_as_longlong(x) >> 52) & 0x7FF);
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);  // .x in the low half
  return *reinterpret_cast<const uint32_t *>(&v);
}

// packed pairs of FP32 values (f32x2 arithmetic: two lanes' worth per instruction)
__device__ __forceinline__ uint64_t f2(float lo, float hi) {
  uint64_t r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ void f2split(uint64_t v, float &lo, float &hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ uint64_t mul2(uint64_t a, uint64_t b) {
  uint64_t r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ uint64_t add2(uint64_t a, uint64_t b) {
  uint64_t r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ uint64_t fma2(uint64_t a, uint64_t b, uint64_t c) {
  uint64_t r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
  return r;
}

// |x| 2^(55 - E) truncated to an integer a < 2^55, E = raw_max - 1022 (|x| < 2^E), in
// three unsigned parts, t = a >> 48 (< 128), c1 = bits 24..47, c2 = bits 0..23, and the
// sign of x as +-1.0f.  Integer arithmetic on the FP64 fields (the mantissa shifted right
// by raw_max - ex); subnormals and values 2^-55 below the row maximum flush to zero.
__device__ __forceinline__ void chunks(double x, unsigned raw_max, unsigned &t, unsigned &c1,
                                       unsigned &c2, float &sg) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const unsigned ex = (hi >> 20) & 0x7FFu;
  const unsigned sh = ex ? min(raw_max - ex, 63u) : 63u;
  const unsigned long long m =
      ((unsigned long long)((((hi & 0xFFFFFu) | 0x100000u) << 2) | (lo >> 30)) << 32) |
      (unsigned long long)(lo << 2);  // mantissa x 4, 55 bits
  const unsigned long long a = m >> sh;
  t = (unsigned)(a >> 48);
  c1 = (unsigned)(a >> 24) & 0xFFFFFFu;
  c2 = (unsigned)a & 0xFFFFFFu;
  sg = __int_as_float(0x3F800000 | (int)(hi & 0x80000000u));
}

// The digits of two values of one row (same exponent), as BF16 pairs: out[i] holds digit i
// of x0 in its low half and of x1 in its high half.  Digit 0 is sg t; the base-256 digits
// of a signed 24-bit chunk c: d0 = rint(c 2^-16), d1 = rint((c - 2^16 d0) 2^-8),
// d2 = c - 2^16 d0 - 2^8 d1, all exact FP32 operations (f32x2, both values at once).
__device__ __forceinline__ void digits_pair(double x0, double x1, unsigned raw_max,
                                            uint32_t (&out)[kUS]) {
  unsigned t0, a0, b0, t1, a1, b1;
  float s0, s1;
  chunks(x0, raw_max, t0, a0, b0, s0);
  chunks(x1, raw_max, t1, a1, b1, s1);
  out[0] = pack_bf16(s0 * (float)t0, s1 * (float)t1);
  const uint64_t sg = f2(s0, s1);
  const uint64_t M = f2(kMagic, kMagic), nM = f2(-kMagic, -kMagic);
  const uint64_t s16 = f2(1.f / 65536.f, 1.f / 65536.f), s8 = f2(1.f / 256.f, 1.f / 256.f);
  const uint64_t m16 = f2(-65536.f, -65536.f), m8 = f2(-256.f, -256.f);
  const unsigned ca[2] = {a0, b0}, cb[2] = {a1, b1};
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    uint64_t f = mul2(f2((float)ca[h], (float)cb[h]), sg);  // |c| < 2^24: exact
    const uint64_t d0 = add2(add2(mul2(f, s16), M), nM);    // |d0| <= 256
    f = fma2(d0, m16, f);                                   // |f| <= 2^15
    const uint64_t d1 = add2(add2(mul2(f, s8), M), nM);     // |d1| <= 128
    const uint64_t d2 = fma2(d1, m8, f);                    // |d2| <= 128
    float l, u;
    f2split(d0, l, u);
    out[1 + 3 * h] = pack_bf16(l, u);
    f2split(d1, l, u);
    out[2 + 3 * h] = pack_bf16(l, u);
    f2split(d2, l, u);
    out[3 + 3 * h] = pack_bf16(l, u);
  }
}

// The seven digits of one value (for alpha Y, once per CTA).
__device__ __forceinline__ void digits7(double x, unsigned raw_max, float (&d)[kUS]) {
  unsigned t, a, b;
  float sg;
  chunks(x, raw_max, t, a, b, sg);
  d[0] = sg * (float)t;
  const unsigned ch[2] = {a, b};
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    float f = sg * (float)ch[h];
    const float d0 = rintf(f * (1.f / 65536.f));
    f = fmaf(-d0, 65536.f, f);
    const float d1 = rintf(f * (1.f / 256.f));
    d[1 + 3 * h] = d0;
    d[2 + 3 * h] = d1;
    d[3 + 3 * h] = fmaf(-d1, 256.f, f);
  }
}

__device__ __forceinline__ double pow2d(int e) {
  e = e < -1022 ? -1022 : (e > 1023 ? 1023 : e);
  return __longlong_as_double((long long)(e + 1023) << 52);
}

// (hi 2^32 + lo) 2^(E - 70) rounded to the nearest FP64 value (ties to even), |hi|, |lo| <
// 2^49, by integer arithmetic (GB300's FP64 pipe issues one warp instruction per ~64 cycles
// of a sub-partition, the integer pipes one per cycle); results outside the normal range
// take the FP64 formula, which rounds the same way.
__device__ __forceinline__ double combine(long long hi, long long lo, int E) {
  const long long top = hi + (lo >> 32);  // S = top 2^32 + bot exactly, 0 <= bot < 2^32
  const unsigned bot = (unsigned)lo;
  const bool neg = top < 0;
  unsigned long long T;
  unsigned B;
  if (!neg) {
    T = (unsigned long long)top;
    B = bot;
  } else if (bot == 0) {
    T = (unsigned long long)(-top);
    B = 0;
  } else {
    T = (unsigned long long)(-top - 1);
    B = 0u - bot;
  }
  if (T == 0 && B == 0) return 0.0;
  const int lb = T ? 95 - __clzll((long long)T) : 31 - __clz((int)B);  // leading bit of |S|
  int sh = lb - 52;
  unsigned long long mant;
  if (sh <= 0) {
    mant = ((T << 32) | B) << (-sh);  // |S| < 2^53: exact
  } else {                            // sh <= 29: the dropped bits are all in B
    mant = (T << (32 - sh)) | (B >> sh);
    const unsigned rem = B & ((1u << sh) - 1u), half = 1u << (sh - 1);
    if (rem > half || (rem == half && (mant & 1ULL))) {
      ++mant;
      if (mant >> 53) {
        mant >>= 1;
        ++sh;
      }
    }
  }
  const int be = sh + E - 70 + 52 + 1023;
  if (be <= 0 || be >= 2047)
    return fma((double)lo, pow2d(E - 70), (double)hi * pow2d(E - 38));
  return __longlong_as_double((long long)(((unsigned long long)neg << 63) |
                                          ((unsigned long long)be << 52) |
                                          (mant & ((1ULL << 52) - 1))));
}

}  // namespace b256
}  // namespace tps
