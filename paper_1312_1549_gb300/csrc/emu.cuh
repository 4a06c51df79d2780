// Float64-class contractions on the BF16 tensor cores (fixed-point slicing).
#pragma once
#include <cuda_bf16.h>
#include "omm_internal.cuh"
#include "tc_gemm.cuh"

namespace omm {
namespace emu {
// s fixed-point bf16 slices of each row of src (rows x cols), stacked: slice i at dst + i*rows*ld_dst
void slice_rows(cudaStream_t st, const double* src, long rows, long cols, long ld_src, int s,
                __nv_bfloat16* dst, long ld_dst, const Scalars* sc);
void transpose(cudaStream_t st, const double* src, long rows, long cols, long ld_src, double* dst, long ld_dst);
// the slice pairs (i, j), i + j < s, level by level from the smallest, in chunks whose
// FP32 sums are exact for a contraction of length K
tc::PairList level_chunks(int K, int s);
// CUDA-event timing of every sliced product issued by this host thread (nullptr: off)
void set_profiler(Profiler* p);
// C = alpha A B^T + beta C from s-slice operands (A, B made by slice_rows)
void gemm(cudaStream_t st, const tc::Operand& A, const tc::Operand& B, int K, int s, const tc::Epilogue& ep,
          double* partial = nullptr, long partial_capacity = 0, const tc::BlockLists* sparse = nullptr);
// C = alpha A B^T + beta C from bf16 hi/lo operands (the 3-term split form), timed like the sliced products
void gemm_split(cudaStream_t st, const tc::Operand& A, const tc::Operand& B, int K, const tc::Epilogue& ep);
}  // namespace emu

struct EmuState;
EmuState* emu_create(cudaStream_t st, int m, int n, int slices, const double* HS);
void emu_update_H(EmuState* es, cudaStream_t st, const double* HS);
void emu_destroy(EmuState* es, cudaStream_t st);  // st: the owner's current stream
int emu_error(EmuState* es, cudaStream_t st);
// density matrix D = 2 C^T (2I - S_W) C (m x m) with float64-class products
void emu_density(EmuState* es, cudaStream_t st, const double* C, const double* SWHW, double* D);
// out = -(2 C^T H~_W C + eta D) from out = D; call right after emu_density (it reuses the sliced C^T)
void emu_minus_edm(EmuState* es, cudaStream_t st, const double* SWHW, double eta, double* out);
void emu_recompute_state(EmuState* es, cudaStream_t st, Scalars* sc, const double* C, double* Y4,
                         double* SWHW, double* G, double* part, double* part2);

}  // namespace omm
