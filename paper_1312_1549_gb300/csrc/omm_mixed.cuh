// Mixed-precision line searches: the contractions run on the BF16 tensor
// cores (tcgen05, TMEM accumulators, TMA-fed shared memory) as 3-term split
// products with FP32 accumulation; the state stays in float64.
#pragma once
#include "omm_internal.cuh"
#include "tc_gemm.cuh"

namespace omm {

struct MixedState;

// Buffers and operands of a mixed state, for the batched driver.
struct MixedView {
  long ldm, ld4;
  __nv_bfloat16 *G_hi, *D_hi, *Y_hi, *W_hi;  // [hi; lo] stacks (Y: [dHC; dSC; HC; SC; HD; SD], 6n rows)
  double *Gref, *Wref, *red;
  float *Dir32, *PG32, *HD32, *dY32;  // float32 side quantities, leading dimension ldm
  const tc::Operand *opHS, *opP, *opG, *opD, *opYproj, *opYgrad, *opW;
  const tc::BlockLists* hs_blocks;  // [0]: 256-row blocks, [1]: 128-row blocks, [2]: 192-row blocks
  int* err;
  int npass;
  bool precond;
};
MixedView mixed_view(MixedState* ms);
// the autotuner's tile widths of the four line-search GEMMs (0 before the first line search) and
// the time it spent
void mixed_tuning(const MixedState* ms, int bn[4], double* ms_autotune);
// the epilogues of the P G, [H D; S D], projection and gradient GEMMs of a line search
void mixed_epilogues(MixedState* ms, const Scalars* sc, double* G, double* Gold, double* Y4, double* Proj,
                     tc::Epilogue out[4]);
// partial-sum slots the P G epilogue fills (after the first line search has built the plans)
int mixed_reduce_parts(const MixedState* ms);
// tests of the timeout status: every line search's first GEMM expires its bounded wait
void mixed_set_expire(MixedState* ms, int on);
void mixed_reset_error(MixedState* ms, cudaStream_t st);

MixedState* mixed_create(cudaStream_t st, int m, int n, const double* HS, const double* P);
void mixed_update_H(MixedState* ms, cudaStream_t st, const double* HS);
void mixed_destroy(MixedState* ms, cudaStream_t st);  // st: the owner's current stream
// after a float64 recompute: take (G, HC, SC, S_W, H_W) as the new reference
// point of the incremental gradient and refresh the bf16 copies
void mixed_sync_state(MixedState* ms, cudaStream_t st, const double* Y4, const double* SWHW, const double* G);
// initial state on the tensor cores (not a certificate)
void mixed_recompute_state(MixedState* ms, cudaStream_t st, Scalars* sc, const double* C, double* Y4,
                           double* SWHW, double* G, double* part, double* part2);
// nonzero if a tensor-core kernel gave up a bounded wait (synchronises the stream)
int mixed_error(MixedState* ms, cudaStream_t st);
void mixed_iterate(MixedState* ms, cudaStream_t st, Scalars* sc, double* C, double* Dir, double* G,
                   double* Gold, double* PG, double* Y4, double* SWHW, double* Proj, double* part,
                   double* part2, const double* HS, const double* P, bool precond, Profiler& prof);
// the same line search replayed from a CUDA graph (captured on first use, after the plans exist,
// for this stream and these buffers); launched eagerly when profiling, on the legacy default
// stream or when a capture fails
void mixed_iterate_replay(MixedState* ms, cudaStream_t st, Scalars* sc, double* C, double* Dir, double* G,
                          double* Gold, double* PG, double* Y4, double* SWHW, double* Proj, double* part,
                          double* part2, const double* HS, const double* P, bool precond, Profiler& prof);

}  // namespace omm
