// float64 -> (bf16 hi, bf16 lo) split of the tensor-core operands:
// hi = bf16(x), lo = bf16(x - hi), so that hi + lo carries about 16
// significant bits of x. Memory-bound (8 bytes in, 4 bytes out per element).
#include "tc_gemm.cuh"

namespace omm {
namespace tc {
namespace {

__device__ __forceinline__ bool stopped(const Scalars* sc) { return sc != nullptr && (sc->done | sc->halt); }

__global__ void split_kernel(const double* __restrict__ src, const double* __restrict__ sub, long rows,
                             long cols, long ld_src, __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo,
                             long ld_dst, const Scalars* sc) {
  if (stopped(sc)) return;
  const long count = rows * cols;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < count; idx += (long)gridDim.x * blockDim.x) {
    const long r = idx / cols, c = idx % cols;
    const double x = sub ? src[r * ld_src + c] - sub[r * ld_src + c] : src[r * ld_src + c];
    const __nv_bfloat16 h = __double2bfloat16(x);
    hi[r * ld_dst + c] = h;
    if (lo) lo[r * ld_dst + c] = __double2bfloat16(x - (double)__bfloat162float(h));
  }
}

// dst[c][r] = split(src[r][c]) through 32 x 32 shared-memory tiles
__global__ void split_t_kernel(const double* __restrict__ src, long rows, long cols, long ld_src,
                               __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo, long ld_dst,
                               const Scalars* sc) {
  if (stopped(sc)) return;
  __shared__ double tile[32][33];
  const long tiles_c = (cols + 31) / 32;
  const long r0 = (blockIdx.x / tiles_c) * 32, c0 = (blockIdx.x % tiles_c) * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
  for (int k = ty; k < 32; k += 8) {
    const long r = r0 + k, c = c0 + tx;
    tile[k][tx] = (r < rows && c < cols) ? src[r * ld_src + c] : 0.0;
  }
  __syncthreads();
  for (int k = ty; k < 32; k += 8) {
    const long c = c0 + k, r = r0 + tx;   // output row c, column r
    if (c < cols && r < rows) {
      const double x = tile[tx][k];
      const __nv_bfloat16 h = __double2bfloat16(x);
      hi[c * ld_dst + r] = h;
      if (lo) lo[c * ld_dst + r] = __double2bfloat16(x - (double)__bfloat162float(h));
    }
  }
}

}  // namespace

void split(cudaStream_t st, const double* src, long rows, long cols, long ld_src, __nv_bfloat16* hi,
           __nv_bfloat16* lo, long ld_dst, const Scalars* sc) {
  const long count = rows * cols;
  long g = (count + 255) / 256;
  if (g > 8192) g = 8192;
  if (g < 1) g = 1;
  split_kernel<<<(int)g, 256, 0, st>>>(src, nullptr, rows, cols, ld_src, hi, lo, ld_dst, sc);
  OMM_LAUNCH_CHECK();
}

void split_diff(cudaStream_t st, const double* src, const double* sub, long rows, long cols, long ld_src,
                __nv_bfloat16* hi, __nv_bfloat16* lo, long ld_dst, const Scalars* sc) {
  const long count = rows * cols;
  long g = (count + 255) / 256;
  if (g > 8192) g = 8192;
  if (g < 1) g = 1;
  split_kernel<<<(int)g, 256, 0, st>>>(src, sub, rows, cols, ld_src, hi, lo, ld_dst, sc);
  OMM_LAUNCH_CHECK();
}

void split_transposed(cudaStream_t st, const double* src, long rows, long cols, long ld_src,
                      __nv_bfloat16* hi_t, __nv_bfloat16* lo_t, long ld_dst, const Scalars* sc) {
  const long blocks = ((rows + 31) / 32) * ((cols + 31) / 32);
  split_t_kernel<<<(int)blocks, 256, 0, st>>>(src, rows, cols, ld_src, hi_t, lo_t, ld_dst, sc);
  OMM_LAUNCH_CHECK();
}

}  // namespace tc
}  // namespace omm
