// float64 -> (bf16 hi, bf16 lo) split bodies shared by the single and the
// batched kernels: hi = bf16(x), lo = bf16(x - hi).
#pragma once
#include <cuda_bf16.h>
#include "omm_internal.cuh"

namespace omm {
namespace dev {

// float64 -> bf16 with round-to-nearest-even, entirely on the integer pipe. The
// float64 units of this GPU retire about two instructions per SM and clock, and a
// library conversion on a rarely taken branch still costs its float64 instructions
// when the compiler predicates it, so every case is done on the bits: in the normal
// bf16 range the 52-bit mantissa is rounded to 7 bits (ties to even; a carry moves
// into the exponent, which also gives the overflow to infinity) and the exponent is
// rebiased from 1023 to 127; below it the value is rounded to a multiple of the
// smallest bf16 subnormal 2^-133; infinities stay infinite and NaNs become quiet NaNs.
__device__ __forceinline__ unsigned short bf16_bits_rne(double x) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const unsigned long long mag = u & 0x7FFFFFFFFFFFFFFFull;
  const unsigned int sign = (unsigned int)(u >> 48) & 0x8000u;
  const unsigned int e = (unsigned int)(mag >> 52);
  if (e >= 1023u - 126u && e <= 1023u + 127u) {
    const unsigned long long r = mag + 0x00000FFFFFFFFFFFull + ((mag >> 45) & 1ull);  // 2^44 - 1 + lsb
    return (unsigned short)(sign | ((unsigned int)(r >> 45) - ((1023u - 127u) << 7)));
  }
  if (e == 0x7FFu) return (unsigned short)(sign | 0x7F80u | ((mag << 12) != 0 ? 0x40u : 0u));
  if (e > 1023u + 127u) return (unsigned short)(sign | 0x7F80u);
  // |x| < 2^-126: x = M 2^(max(e,1) - 1075), in units of 2^-133 that is M >> (942 - max(e,1))
  const unsigned long long M = (mag & 0x000FFFFFFFFFFFFFull) | (e ? (1ull << 52) : 0ull);
  const int shift = 942 - (int)(e ? e : 1u);  // >= 46
  if (shift >= 64) return (unsigned short)sign;
  const unsigned long long q = M >> shift, rem = M & ((1ull << shift) - 1ull), half = 1ull << (shift - 1);
  const unsigned long long r = q + ((rem > half || (rem == half && (q & 1ull))) ? 1ull : 0ull);
  return (unsigned short)(sign | (unsigned int)r);
}

// the float64 value of a bf16 (exact; integer pipe)
__device__ __forceinline__ double bf16_bits_to_double(unsigned short b) {
  const unsigned long long sign = (unsigned long long)(b & 0x8000u) << 48;
  const unsigned int e = (b >> 7) & 0xFFu, f = b & 0x7Fu;
  unsigned long long bits;
  if (e == 0xFFu) {
    bits = sign | (0x7FFull << 52) | ((unsigned long long)f << 45);
  } else if (e != 0) {
    bits = sign | ((unsigned long long)(e - 127u + 1023u) << 52) | ((unsigned long long)f << 45);
  } else if (f == 0) {
    bits = sign;
  } else {  // subnormal: f 2^-133 with the top bit of f at position p
    const int p = 31 - __clz(f);
    bits = sign | ((unsigned long long)(p - 133 + 1023) << 52) |
           (((unsigned long long)f << (52 - p)) & 0x000FFFFFFFFFFFFFull);
  }
  return __longlong_as_double((long long)bits);
}

// lo = bf16(x - hi) outside the range the integer path covers (|x| < 2^-126, |x| >= 2^128,
// infinities and NaNs): one float64 subtraction, kept out of line so that the common path
// never issues it, not even predicated off
static __device__ __noinline__ unsigned short bf16_residual_slow(double x, unsigned short h) {
  return bf16_bits_rne(x - bf16_bits_to_double(h));  // x - hi is exact
}

// hi = bf16(x) and lo = bf16(x - hi), both rounded to nearest even, on the integer pipe. For x
// in the normal bf16 range hi keeps the top 8 significand bits of x rounded at bit 45 of the
// float64 fraction; the residual x - hi is then the 45 bits below (rounded down) or minus their
// complement to 2^45 (rounded up), in units of 2^(e - 1075). That integer is rebuilt as a
// float64 (exact: at most 45 bits) and rounded to bf16 like any other value.
__device__ __forceinline__ void split_bits(double x, unsigned short& h, unsigned short& l) {
  h = bf16_bits_rne(x);
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const unsigned long long mag = u & 0x7FFFFFFFFFFFFFFFull;
  const unsigned int e = (unsigned int)(mag >> 52);
  if (e < 1023u - 126u || e > 1023u + 127u || (h & 0x7F80u) == 0x7F80u) {  // (hi rounded to infinity)
    l = bf16_residual_slow(x, h);
    return;
  }
  const unsigned long long low = mag & 0x00001FFFFFFFFFFFull;        // the 45 bits below hi
  const bool up = (unsigned int)(h & 0x7FFFu) != (unsigned int)((mag >> 45) - ((1023ull - 127ull) << 7));
  const unsigned long long R = up ? (0x0000200000000000ull - low) : low;  // |x - hi| / 2^(e - 1075)
  if (R == 0) {
    l = 0;
    return;
  }
  const unsigned long long sign = (u & 0x8000000000000000ull) ^ (up ? 0x8000000000000000ull : 0ull);
  const int p = 63 - __clzll((long long)R);                      // top bit of R, p <= 45
  // R 2^(e - 1075) = 1.f 2^(p + e - 1075): float64 exponent field p + e - 52 (>= 845, normal)
  const unsigned long long bits = sign | ((unsigned long long)(p + (int)e - 52) << 52) |
                                  ((R << (52 - p)) & 0x000FFFFFFFFFFFFFull);
  l = bf16_bits_rne(__longlong_as_double((long long)bits));
}

// float64 -> float32 rounded to nearest even on the integer pipe (the float64 units retire about
// one lane per SM and clock); magnitudes below the float32 normal range become zero, above it
// infinity
__device__ __forceinline__ float f32_rne_bits(double x) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const unsigned int hi32 = (unsigned int)(u >> 32);
  const unsigned int sign = hi32 & 0x80000000u;
  const int e = (int)((hi32 >> 20) & 0x7FFu);
  if (e < 1023 - 126) return __uint_as_float(sign);
  if (e > 1023 + 127) return __uint_as_float(sign | 0x7F800000u);
  // fraction f (52 bits) -> 23 bits: add half an ulp minus one plus the lsb (ties to even); a
  // carry out of the fraction moves into the exponent
  const unsigned long long f = u & 0x000FFFFFFFFFFFFFull;
  const unsigned long long r = f + 0x000000000FFFFFFFull + ((f >> 29) & 1ull);
  return __uint_as_float(sign + ((unsigned int)(e - 1023 + 127) << 23) + (unsigned int)(r >> 29));
}

// float32 -> float64 on the integer pipe (exact; zeros keep their sign, subnormals are
// normalised, infinities and NaNs keep their class)
__device__ __forceinline__ double f64_of_f32(float f) {
  const unsigned int u = __float_as_uint(f);
  const unsigned int e = (u >> 23) & 0xFFu, m = u & 0x7FFFFFu;
  const unsigned long long sign = (unsigned long long)(u & 0x80000000u) << 32;
  unsigned long long bits;
  if (e != 0 && e != 0xFFu) {
    bits = sign | ((unsigned long long)(e + (1023u - 127u)) << 52) | ((unsigned long long)m << 29);
  } else if (e == 0xFFu) {
    bits = sign | (0x7FFull << 52) | ((unsigned long long)m << 29);
  } else if (m == 0) {
    bits = sign;
  } else {  // subnormal: m 2^-149 with its top bit at position p
    const int p = 31 - __clz(m);
    bits = sign | ((unsigned long long)(p - 149 + 1023) << 52) | (((unsigned long long)m << (52 - p)) & 0x000FFFFFFFFFFFFFull);
  }
  return __longlong_as_double((long long)bits);
}

// hi/lo of a float32 value (the float32 side quantities of the mixed line search): two hardware
// conversions and one float32 subtraction
__device__ __forceinline__ void split_bits_f32(float x, unsigned short& h, unsigned short& l) {
  const __nv_bfloat16 hb = __float2bfloat16_rn(x);
  h = __bfloat16_as_ushort(hb);
  l = __bfloat16_as_ushort(__float2bfloat16_rn(x - __bfloat162float(hb)));
}

__device__ __forceinline__ void split_store2_f32(float x0, float x1, __nv_bfloat16* hi, __nv_bfloat16* lo, long off) {
  unsigned short h0, l0, h1, l1;
  split_bits_f32(x0, h0, l0);
  split_bits_f32(x1, h1, l1);
  *reinterpret_cast<unsigned int*>(hi + off) = h0 | ((unsigned int)h1 << 16);
  *reinterpret_cast<unsigned int*>(lo + off) = l0 | ((unsigned int)l1 << 16);
}

__device__ __forceinline__ void split_store_f32(float x, __nv_bfloat16* hi, __nv_bfloat16* lo, long off) {
  unsigned short h, l;
  split_bits_f32(x, h, l);
  hi[off] = __ushort_as_bfloat16(h);
  lo[off] = __ushort_as_bfloat16(l);
}

// The operand split of the line-search products, cheap form: x is rounded to float32 (integer
// pipe), hi = bf16(x32) and lo = bf16(x32 - hi) by the float32 units. hi can differ from the
// correctly rounded bf16(x) by one unit in a rare double-rounding case; lo then holds the
// difference, so hi + lo still carries x to about 2^-17 |x|, the accuracy of the split. About
// twenty instructions per element against a hundred for the exact split, which matters in the
// GEMM epilogues, where four warps per SM do this work beside the tensor cores.
__device__ __forceinline__ void split_bits_fast(double x, unsigned short& h, unsigned short& l) {
  const float xf = f32_rne_bits(x);
  const __nv_bfloat16 hb = __float2bfloat16_rn(xf);
  h = __bfloat16_as_ushort(hb);
  l = __bfloat16_as_ushort(__float2bfloat16_rn(xf - __bfloat162float(hb)));
}

__device__ __forceinline__ void split_store_fast(double x, __nv_bfloat16* hi, __nv_bfloat16* lo, long off) {
  unsigned short h, l;
  split_bits_fast(x, h, l);
  hi[off] = __ushort_as_bfloat16(h);
  lo[off] = __ushort_as_bfloat16(l);
}

__device__ __forceinline__ void split_store2_fast(double x0, double x1, __nv_bfloat16* hi, __nv_bfloat16* lo,
                                                  long off) {
  unsigned short h0, l0, h1, l1;
  split_bits_fast(x0, h0, l0);
  split_bits_fast(x1, h1, l1);
  *reinterpret_cast<unsigned int*>(hi + off) = h0 | ((unsigned int)h1 << 16);
  *reinterpret_cast<unsigned int*>(lo + off) = l0 | ((unsigned int)l1 << 16);
}

// hi = bf16(x), lo = bf16(x - hi), both rounded to nearest even (integer pipe)
__device__ __forceinline__ void split_store(double x, __nv_bfloat16* hi, __nv_bfloat16* lo, long off) {
  unsigned short h, l;
  split_bits(x, h, l);
  hi[off] = __ushort_as_bfloat16(h);
  if (lo) lo[off] = __ushort_as_bfloat16(l);
}

// hi/lo of two neighbouring elements, stored as bf16 pairs
__device__ __forceinline__ void split_store2(double x0, double x1, __nv_bfloat16* hi, __nv_bfloat16* lo, long off) {
  __nv_bfloat16 h[2], l[2];
  split_store(x0, h, lo ? l : nullptr, 0);
  split_store(x1, h, lo ? l : nullptr, 1);
  *reinterpret_cast<__nv_bfloat162*>(hi + off) = __halves2bfloat162(h[0], h[1]);
  if (lo) *reinterpret_cast<__nv_bfloat162*>(lo + off) = __halves2bfloat162(l[0], l[1]);
}

// Work units of the row-wise vector kernels: (row, run of blockDim.x column pairs); unit u of
// block bx, bx + nbx, ... Every thread takes one column pair (16-byte float64 loads, 4-byte bf16
// stores) and issues its loads at once, so that many loads are in flight per SM.
__device__ __forceinline__ long pair_units(long rows, long cols) {
  const long npair = (cols + 1) / 2;
  return rows * ((npair + blockDim.x - 1) / blockDim.x);
}
__device__ __forceinline__ void unit_pos(long u, long cols, long& row, long& col) {
  const long npair = (cols + 1) / 2, nseg = (npair + blockDim.x - 1) / blockDim.x;
  row = u / nseg;
  col = 2 * ((u - row * nseg) * blockDim.x + threadIdx.x);
}

// hi/lo of (src - sub) (sub may be null), rows x cols, by column pairs
__device__ __forceinline__ void split_body(const double* __restrict__ src, const double* __restrict__ sub,
                                           long rows, long cols, long ld_src, __nv_bfloat16* __restrict__ hi,
                                           __nv_bfloat16* __restrict__ lo, long ld_dst, int bx, int nbx) {
  const long units = pair_units(rows, cols);
  for (long u = bx; u < units; u += nbx) {
    long r, c;
    unit_pos(u, cols, r, c);
    if (c >= cols) continue;
    const double* s = src + r * ld_src + c;
    const double* w = sub ? sub + r * ld_src + c : nullptr;
    const long off = r * ld_dst + c;
    const bool vec = c + 1 < cols && ((reinterpret_cast<uintptr_t>(s) | reinterpret_cast<uintptr_t>(w)) & 15) == 0 &&
                     ((reinterpret_cast<uintptr_t>(hi + off) | reinterpret_cast<uintptr_t>(lo ? lo + off : nullptr)) &
                      3) == 0;
    if (vec) {
      double2 x = *reinterpret_cast<const double2*>(s);
      if (w) {
        const double2 y = *reinterpret_cast<const double2*>(w);
        x.x -= y.x;
        x.y -= y.y;
      }
      split_store2(x.x, x.y, hi, lo, off);
    } else {
      for (int k = 0; k < 2 && c + k < cols; ++k) split_store(w ? s[k] - w[k] : s[k], hi, lo, off + k);
    }
  }
}

// dst[c][r] = split(src[r][c]) for the 64 x 32 tile `tile` (row-major grid of 64-row by 32-column
// tiles), 256 threads: every warp writes whole 64-element runs of destination rows, as bf16 pairs
// where the destination allows it
__device__ __forceinline__ void split_t_body(const double* __restrict__ src, long rows, long cols, long ld_src,
                                             __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo,
                                             long ld_dst, long tile) {
  __shared__ double t[64][33];
  const long tiles_c = (cols + 31) / 32;
  const long r0 = (tile / tiles_c) * 64, c0 = (tile % tiles_c) * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int k = ty; k < 64; k += 8) {
    const long r = r0 + k, c = c0 + tx;
    t[k][tx] = (r < rows && c < cols) ? src[r * ld_src + c] : 0.0;
  }
  __syncthreads();
  const bool pairs = ((ld_dst & 1) == 0) && ((r0 & 1) == 0) &&
                     ((reinterpret_cast<uintptr_t>(hi) | reinterpret_cast<uintptr_t>(lo)) & 3) == 0;
  for (int k = ty; k < 32; k += 8) {  // destination row c0 + k, columns r0 + 2 tx, r0 + 2 tx + 1
    const long c = c0 + k, r = r0 + 2 * tx;
    if (c >= cols || r >= rows) continue;
    if (pairs && r + 1 < rows) {
      split_store2(t[2 * tx][k], t[2 * tx + 1][k], hi, lo, c * ld_dst + r);
    } else {
      split_store(t[2 * tx][k], hi, lo, c * ld_dst + r);
      if (r + 1 < rows) split_store(t[2 * tx + 1][k], hi, lo, c * ld_dst + r + 1);
    }
  }
}

}  // namespace dev
}  // namespace omm
