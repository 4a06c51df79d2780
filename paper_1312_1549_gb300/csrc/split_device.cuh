// float64 -> (bf16 hi, bf16 lo) split bodies shared by the single and the
// batched kernels: hi = bf16(x), lo = bf16(x - hi).
#pragma once
#include <cuda_bf16.h>
#include "omm_internal.cuh"

namespace omm {
namespace dev {

__device__ __forceinline__ void split_store(double x, __nv_bfloat16* hi, __nv_bfloat16* lo, long off) {
  const __nv_bfloat16 h = __double2bfloat16(x);
  hi[off] = h;
  if (lo) lo[off] = __double2bfloat16(x - (double)__bfloat162float(h));
}

// rows handled by blocks bx, bx + nbx, ...; the block's threads stride over columns
__device__ __forceinline__ void split_body(const double* __restrict__ src, const double* __restrict__ sub,
                                           long rows, long cols, long ld_src, __nv_bfloat16* __restrict__ hi,
                                           __nv_bfloat16* __restrict__ lo, long ld_dst, int bx, int nbx) {
  for (long r = bx; r < rows; r += nbx) {
    const double* s = src + r * ld_src;
    const double* u = sub ? sub + r * ld_src : nullptr;
    for (long c = threadIdx.x; c < cols; c += blockDim.x) {
      const double x = u ? s[c] - u[c] : s[c];
      split_store(x, hi, lo, r * ld_dst + c);
    }
  }
}

// dst[c][r] = split(src[r][c]) for the 32 x 32 tile `tile` (row-major tile grid), 256 threads
__device__ __forceinline__ void split_t_body(const double* __restrict__ src, long rows, long cols, long ld_src,
                                             __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo,
                                             long ld_dst, long tile) {
  __shared__ double t[32][33];
  const long tiles_c = (cols + 31) / 32;
  const long r0 = (tile / tiles_c) * 32, c0 = (tile % tiles_c) * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int k = ty; k < 32; k += 8) {
    const long r = r0 + k, c = c0 + tx;
    t[k][tx] = (r < rows && c < cols) ? src[r * ld_src + c] : 0.0;
  }
  __syncthreads();
  for (int k = ty; k < 32; k += 8) {
    const long c = c0 + k, r = r0 + tx;
    if (c < cols && r < rows) split_store(t[tx][k], hi, lo, c * ld_dst + r);
  }
}

}  // namespace dev
}  // namespace omm
