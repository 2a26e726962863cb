// Conversions of the split-precision far history, on the integer pipe where
// they can be.  BF16 pieces of FP64 values (BF16x3 / BF16x6 operands):
// x = hi + mid + lo + r, each piece the BF16 value nearest to what the earlier
// pieces leave (round to nearest, ties to even), r = O(2^-24 |x|).
//
// GB300's FP64 pipe issues one warp instruction per ~64 cycles per
// sub-partition, and the near kernels that split each new history row are
// bound by it.  The rounding below therefore runs on the integer pipe for
// values in BF16's normal range and for zeros: it rounds the 52-bit double
// significand to 7 bits at bit 45 (adding 2^44 - 1 plus the kept LSB makes a
// carry exactly when the dropped bits exceed half an ULP, or equal it with an
// odd LSB; a carry out of the significand raises the exponent), and the
// rounded double is the double pattern with the dropped bits cleared.  Only
// the exact remainder x - piece stays an FP64 subtraction.  Values outside
// that range (BF16 subnormals, the top binade, Inf, NaN) take the conversion
// instructions.  The FP32 (hi, lo) column sums of the tensor-core epilogue
// become FP64 the same way.  Host-callable so that a host program can check
// both.
#pragma once
#include <cuda_bf16.h>
#include <stdint.h>
#include <string.h>

namespace abm {

__host__ __device__ __forceinline__ uint64_t f64_bits(double x) {
#ifdef __CUDA_ARCH__
  return (uint64_t)__double_as_longlong(x);
#else
  uint64_t u;
  memcpy(&u, &x, 8);
  return u;
#endif
}

__host__ __device__ __forceinline__ double f64_from_bits(uint64_t u) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)u);
#else
  double x;
  memcpy(&x, &u, 8);
  return x;
#endif
}

// Nearest BF16 (bit pattern) to x and that BF16 value as a double.  Returns
// false, leaving both untouched, when x is outside the integer path's range.
__host__ __device__ __forceinline__ bool bf16_round_int(double x, uint16_t& bits, double& value) {
  const uint64_t b = f64_bits(x);
  const uint64_t sign = b & 0x8000000000000000ull;
  const uint64_t mag = b ^ sign;
  const uint32_t e = (uint32_t)(mag >> 52);  // biased FP64 exponent
  if (mag == 0) {
    bits = (uint16_t)(sign >> 48);
    value = x;
    return true;
  }
  // unbiased exponent -126 .. 126: normal in BF16, and a rounding carry
  // reaches at most exponent 127
  if (e < 1023 - 126 || e > 1023 + 126) return false;
  const uint64_t r = (mag + 0x00000FFFFFFFFFFFull + ((mag >> 45) & 1ull)) & ~0x00001FFFFFFFFFFFull;
  bits = (uint16_t)((sign >> 48) | ((uint64_t)((uint32_t)(r >> 52) - (1023 - 127)) << 7) | ((r >> 45) & 0x7Full));
  value = f64_from_bits(r | sign);
  return true;
}

__host__ __device__ __forceinline__ __nv_bfloat16 bf16_from_bits(uint16_t u) {
  __nv_bfloat16_raw raw;
  raw.x = u;
  return __nv_bfloat16(raw);
}

// (double)f for the float f with bit pattern u.  Zeros and normal floats are
// built on the integer pipe (exponent rebiased by 1023 - 127, significand moved
// up 29 bits: exact); subnormals, Inf and NaN take the conversion instruction.
__host__ __device__ __forceinline__ double f32_bits_to_f64(uint32_t u) {
  const uint32_t sign = u & 0x80000000u, mag = u ^ sign;
  const uint32_t e = mag >> 23;
  if (mag == 0) return f64_from_bits((uint64_t)sign << 32);
  if (e == 0 || e == 255) {
    float f;
#ifdef __CUDA_ARCH__
    f = __uint_as_float(u);
#else
    memcpy(&f, &u, 4);
#endif
    return (double)f;
  }
  return f64_from_bits(((uint64_t)(sign | ((mag >> 3) + ((1023u - 127u) << 20))) << 32) | (uint64_t)(u << 29));
}

// out[0..2] = hi, mid, lo of x.
__host__ __device__ __forceinline__ void split3_bf16(double x, __nv_bfloat16* out) {
  double r = x;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    uint16_t bits;
    double piece;
    if (bf16_round_int(r, bits, piece)) {
      out[k] = bf16_from_bits(bits);
    } else {
      out[k] = __double2bfloat16(r);
      piece = (double)__bfloat162float(out[k]);
    }
    if (k < 2) r -= piece;  // exact: piece is r rounded to 8 significant bits
  }
}

}  // namespace abm
