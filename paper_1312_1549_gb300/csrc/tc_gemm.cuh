// BF16 tensor-core GEMM (tcgen05 + TMEM + TMA) with a float64 epilogue.
#pragma once
#include <cuda_bf16.h>
#include "omm_internal.cuh"

namespace omm {
namespace tc {

// Storage for a CUtensorMap (128 bytes, 64-byte aligned) without exposing cuda.h.
struct alignas(64) TensorMap {
  unsigned char bytes[128];
};

// A bf16 operand x = hi + lo, row-major rows x cols (contracted dimension = cols).
struct Operand {
  TensorMap hi, lo;
  long rows = 0, cols = 0;
};

// C (float64) = alpha * acc + beta * C over the valid M x N block. Output
// column j goes to C + (j / split_cols) * split_stride + row * ldc + j % split_cols
// (split_cols = N for a plain matrix), so one GEMM can fill several stacked
// matrices. When skip[0] | skip[1] (the solver's done/halt flags) the kernel
// does nothing. err receives a nonzero code if a bounded wait expired.
struct Epilogue {
  double* C;
  long ldc;
  long split_cols;
  long split_stride;
  double alpha;
  double beta;
  int M;
  int N;
  const int* skip;
  int* err;
};

Operand make_operand(const __nv_bfloat16* hi, const __nv_bfloat16* lo, long rows, long cols, long ld, bool is_a);
// npass = 3: A_hi B_hi + A_hi B_lo + A_lo B_hi; npass = 1: A_hi B_hi.
void gemm(cudaStream_t st, const Operand& A, const Operand& B, int K, int npass, const Epilogue& ep);
int tile_m();
int tile_n();

// x (float64, rows x cols, ld_src) -> hi = bf16(x), lo = bf16(x - hi) (ld_dst);
// transposed variants write dst[j][i]. Skipped when sc's done/halt is set.
void split(cudaStream_t st, const double* src, long rows, long cols, long ld_src, __nv_bfloat16* hi,
           __nv_bfloat16* lo, long ld_dst, const Scalars* sc);
// hi/lo of (src - sub), both float64 with the same layout
void split_diff(cudaStream_t st, const double* src, const double* sub, long rows, long cols, long ld_src,
                __nv_bfloat16* hi, __nv_bfloat16* lo, long ld_dst, const Scalars* sc);
void split_transposed(cudaStream_t st, const double* src, long rows, long cols, long ld_src,
                      __nv_bfloat16* hi_t, __nv_bfloat16* lo_t, long ld_dst, const Scalars* sc);

}  // namespace tc
}  // namespace omm
