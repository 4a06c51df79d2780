// float64 -> (bf16 hi, bf16 lo) split of the tensor-core operands:
// hi = bf16(x), lo = bf16(x - hi), so that hi + lo carries about 16
// significant bits of x. Memory-bound (8 bytes in, 4 bytes out per element).
#include "tc_gemm.cuh"
#include "split_device.cuh"

namespace omm {
namespace tc {
namespace {

__device__ __forceinline__ bool stopped(const Scalars* sc) { return sc != nullptr && (sc->done | sc->halt); }

__global__ void split_kernel(const double* __restrict__ src, const double* __restrict__ sub, long rows,
                             long cols, long ld_src, __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo,
                             long ld_dst, const Scalars* sc) {
  if (stopped(sc)) return;
  dev::split_body(src, sub, rows, cols, ld_src, hi, lo, ld_dst, blockIdx.x, gridDim.x);
}

__global__ void split_t_kernel(const double* __restrict__ src, long rows, long cols, long ld_src,
                               __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo, long ld_dst,
                               const Scalars* sc) {
  if (stopped(sc)) return;
  dev::split_t_body(src, rows, cols, ld_src, hi, lo, ld_dst, blockIdx.x);
}

}  // namespace

// one block per (row, 256 column pairs) unit, at most 16384 blocks
static long pair_grid(long rows, long cols) {
  const long units = rows * (((cols + 1) / 2 + 255) / 256);
  return units < 1 ? 1 : (units > 16384 ? 16384 : units);
}

void split(cudaStream_t st, const double* src, long rows, long cols, long ld_src, __nv_bfloat16* hi,
           __nv_bfloat16* lo, long ld_dst, const Scalars* sc) {
  const long g = pair_grid(rows, cols);
  split_kernel<<<(int)g, 256, 0, st>>>(src, nullptr, rows, cols, ld_src, hi, lo, ld_dst, sc);
  OMM_LAUNCH_CHECK();
}

void split_diff(cudaStream_t st, const double* src, const double* sub, long rows, long cols, long ld_src,
                __nv_bfloat16* hi, __nv_bfloat16* lo, long ld_dst, const Scalars* sc) {
  const long g = pair_grid(rows, cols);
  split_kernel<<<(int)g, 256, 0, st>>>(src, sub, rows, cols, ld_src, hi, lo, ld_dst, sc);
  OMM_LAUNCH_CHECK();
}

void split_transposed(cudaStream_t st, const double* src, long rows, long cols, long ld_src,
                      __nv_bfloat16* hi_t, __nv_bfloat16* lo_t, long ld_dst, const Scalars* sc) {
  const long blocks = ((rows + 63) / 64) * ((cols + 31) / 32);
  split_t_kernel<<<(int)blocks, 256, 0, st>>>(src, rows, cols, ld_src, hi_t, lo_t, ld_dst, sc);
  OMM_LAUNCH_CHECK();
}

}  // namespace tc
}  // namespace omm
