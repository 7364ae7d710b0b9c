// FP64 <-> FP32 conversions on the integer pipes.  GB300's FP64 pipe executes the hardware
// conversions (F2F) as well as FP64 arithmetic and issues one warp instruction per ~64
// cycles of an SM sub-partition, so a streaming kernel that converts every element it
// moves (the 2D TF32 passes' FP64 input and output) can be bound by that pipe below the
// memory bandwidth.  These work on the bit fields instead: a handful of integer
// operations, which cost more issue slots and latency (measured slower in the short,
// latency-bound 1D passes and in the SIMT Gram), so they are used only where the stream
// is long.
#pragma once

#include <cuda_runtime.h>

namespace tps {

#ifdef __CUDACC__
// x rounded toward zero to FP32 (the top 23 stored mantissa bits kept): |x| below the FP32
// normal range gives a signed zero, above it a signed infinity; infinities and NaNs map to
// infinities and NaNs.  Relative error below 2^-23 in the normal range.
__device__ __forceinline__ float f32_of_f64(double x) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const unsigned s = hi & 0x80000000u;
  const unsigned ex = (hi >> 20) & 0x7FFu;  // FP64 biased exponent
  const unsigned m = ((hi & 0xFFFFFu) << 3) | (lo >> 29);
  unsigned r;
  if (ex >= 897u && ex <= 1150u)  // FP32 biased exponent ex - 896 in 1 .. 254
    r = s | ((ex - 896u) << 23) | m;
  else if (ex < 897u)
    r = s;
  else if (ex == 2047u && ((hi & 0xFFFFFu) | lo))
    r = s | 0x7FC00000u;
  else
    r = s | 0x7F800000u;
  return __uint_as_float(r);
}

// f exactly as FP64 (FP32 subnormals, below 1.2e-38, flush to a signed zero).
__device__ __forceinline__ double f64_of_f32(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned s = u & 0x80000000u, e = (u >> 23) & 0xFFu, m = u & 0x7FFFFFu;
  unsigned hi, lo;
  if (e == 0u) {
    hi = s;
    lo = 0u;
  } else {
    hi = s | ((e == 255u ? 2047u : e + 896u) << 20) | (m >> 3);
    lo = m << 29;
  }
  return __hiloint2double((int)hi, (int)lo);
}

#endif

}  // namespace tps
