/*
 * omm_kernels.h -- step-level entry points of the OMM library.
 *
 * Each function runs one step of the OMM hot path on the GPU, exactly as the
 * solver of omm.h runs it, so that the steps can be checked one by one.
 * Pointers are device pointers (float64 unless stated) unless marked
 * "host"; all work is ordered on `stream` (cudaStream_t as void*, NULL = legacy
 * default stream) and the call returns after it completes. Errors are
 * returned as omm_status (see omm.h), never raised; the library never
 * traps or aborts.
 */
#ifndef OMM_GB300_OMM_KERNELS_H
#define OMM_GB300_OMM_KERNELS_H

#include "omm.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Float64 GEMM, row-major: C = alpha op(A) op(B) + beta C, op(A) M x K and
 * op(B) K x N. transA = 0: A is M x K (ld lda); 1: A is K x M. transB likewise.
 * This is the contraction of every float64 step (Sec. 2.3, Table 1: the
 * m x m by m x n, m x n by n x n and n x m by m x n products).
 * Errors: OMM_ERR_ARG (negative sizes, NULL pointers), OMM_ERR_CUDA. */
omm_status omm_kernel_dgemm(int transA, int transB, int M, int N, int K, double alpha,
                            const double* A, long lda, const double* B, long ldb, double beta,
                            double* C, long ldc, void* stream);

/* P = A^-1 for a symmetric positive definite m x m A, by a float64 Cholesky
 * factorisation and triangular inverse (the preconditioner of Sec. 2.4,
 * Eq. 17, applied to A = S + T/tau). A is not modified. *info (host) receives
 * 0, or the 1-based column of the first non-positive pivot, in which case the
 * call returns OMM_ERR_NOT_SPD and P is unspecified. */
omm_status omm_kernel_spd_inverse(int m, const double* A, double* P, int* info, void* stream);

/* The same P = A^-1 (Sec. 2.4, Eq. 17) with float64-class products on the BF16
 * tensor cores, as the mixed-precision solver computes its preconditioner: a
 * recursive Cholesky factorisation, inverse and product L^-T L^-1 on halves,
 * whose off-diagonal products use 10 fixed-point slices per operand (the Ozaki
 * scheme; about 2^-50 of each row-scaled operand), with the 64 x 64 diagonal
 * blocks factored and inverted in float64. Arguments, ownership and *info as
 * for omm_kernel_spd_inverse; OMM_ERR_TIMEOUT if a bounded wait of a tensor-core
 * GEMM expired. Workspace (allocated inside the call): about 2.3 m^2 float64 plus
 * 20 m^2 bytes of slices and up to 430 MB of chunk sums; a second stream runs the
 * Y^T Y updates beside the factorisation and is joined before the call returns. */
omm_status omm_kernel_spd_inverse_sliced(int m, const double* A, double* P, int* info, void* stream);

/* The preconditioner-grade variant the mixed solver uses (omm_opts.precond_slices): the same
 * recursion with `slices` fixed-point slices per operand (2..9, 5 bits each), or with slices = 1
 * (the solver's default) every product in the 3-term bf16 split form (about 2^-16 of |A||B|), and
 * the 128 x 128 diagonal blocks in float32. P enters the line searches only through its bf16
 * rounding (the single-pass P G of the search direction, 2^-9 of each element), so an inverse to a
 * few parts in 10^4 serves as well as a float64 one. Arguments and errors as for
 * omm_kernel_spd_inverse_sliced; OMM_ERR_ARG for slices outside 1..9. */
omm_status omm_kernel_spd_inverse_precond(int m, const double* A, double* P, int slices, int* info,
                                          void* stream);

/* Line minimum of the quartic a0 + a1 x + a2 x^2 + a3 x^3 + a4 x^4 (Sec. 2.3,
 * Eq. 13) as the solver takes it on the device: the first local minimum along
 * x > 0 (a1 < 0). alpha (host, 5 values), x (host) receives the step.
 * Returns OMM_OK, or OMM_ERR_UNBOUNDED when the quartic has no minimum on
 * x > 0 (the functional is unbounded along the line, Sec. 2.2 footnote). */
omm_status omm_kernel_line_minimum(const double* alpha, double* x);

/* Quartic coefficients alpha_0..alpha_4 (Eq. 13) of one line search from the
 * n x n matrices SWHW = [S_W | H_W] (n x 2n, row-major) and
 * Proj = [H' | S' | H'' | S''] (n x 4n, row-major) with H' = Delta^T H C and
 * H'' = Delta^T H Delta (Eqs. 14-15); E is alpha_0. alpha (host, 5 values). */
omm_status omm_kernel_quartic_coefficients(int n, const double* SWHW, const double* Proj, double E,
                                           double* alpha, void* stream);

/* Tensor-core contraction of the mixed-precision path (Sec. 2.3, Table 1
 * products, run on the BF16 tensor cores): C = alpha A B^T + beta C with A
 * M x K and B N x K (row-major float64, contracted over their rows' K
 * entries) and C M x N float64. A and B are split into bf16 pairs
 * x = hi + lo (hi = bf16(x), lo = bf16(x - hi)); npass = 3 accumulates
 * A_hi B_hi + A_hi B_lo + A_lo B_hi in FP32 (about 2^-16 relative error per
 * product), npass = 1 only A_hi B_hi. Scratch for the splits is allocated and
 * freed inside the call. Errors: OMM_ERR_ARG, OMM_ERR_OOM, OMM_ERR_TIMEOUT
 * (a bounded device wait expired), OMM_ERR_CUDA. */
/* The same contraction with a chosen output tile width: tile_n = 256 (128 x 256 tiles, what
 * omm_kernel_gemm_tc uses) or 128 (128 x 128 tiles), the two widths the solver's autotuner picks
 * from. OMM_ERR_ARG for any other tile_n. */
omm_status omm_kernel_gemm_tc_tiled(int M, int N, int K, const double* A, const double* B, double alpha,
                                    double beta, double* C, int npass, int tile_n, void* stream);

/* The same contraction, block-sparse in B (the finite-range operators of Sec. 2.6): the 64-wide K
 * blocks where a block of tile_n rows of B is exactly zero are skipped. The result equals that of
 * omm_kernel_gemm_tc_tiled bit for bit (the skipped products are exact zeros); the block lists
 * are built from B inside the call. Arguments and errors as omm_kernel_gemm_tc_tiled. */
omm_status omm_kernel_gemm_tc_blocksparse(int M, int N, int K, const double* A, const double* B, double alpha,
                                          double beta, double* C, int npass, int tile_n, void* stream);

/* C = alpha A B + beta C on the BF16 tensor cores in 3-term split form, with B given K x N
 * (row-major, the contracted index first): A M x K, C M x N, all row-major float64 (device). This
 * is the operand layout of the mixed path's gradient product G = G_ref + 8 dHC - 4 W [dHC; dSC;
 * HC; SC] (Eq. 12 about the last refresh point, Sec. 2.3): the stacked n x m blocks are read as
 * an MN-major B operand (64 x 64 TMA boxes, the tcgen05 B-transpose bit), without a transposed
 * copy. tile_n: 256 or 128 (output tile width). Error bound as omm_kernel_gemm_tc. Scratch is
 * allocated and freed inside the call. Errors: OMM_ERR_ARG, OMM_ERR_OOM, OMM_ERR_TIMEOUT,
 * OMM_ERR_CUDA. */
omm_status omm_kernel_gemm_tc_kn(int M, int N, int K, const double* A, const double* B, double alpha,
                                 double beta, double* C, int tile_n, void* stream);

omm_status omm_kernel_gemm_tc(int M, int N, int K, const double* A, const double* B, double alpha,
                              double beta, double* C, int npass, void* stream);

/* The contraction of omm_kernel_gemm_tc (npass = 3: split form, npass = 1: single bf16 pass) on
 * pairs of SMs: each cluster of two CTAs computes a 256 x tile_n output tile with one
 * tcgen05.mma.cta_group::2 stream, each SM staging 128 rows of A and half of the tile's B, so that
 * it fetches half the B bytes of a single-SM tile of the same width. b_kn = 0: C = alpha A B^T +
 * beta C with B N x K; b_kn = 1 (npass = 3 only): C = alpha A B + beta C with B K x N, read
 * MN-major (as omm_kernel_gemm_tc_kn). tile_n: 128, 192 (b_kn = 0 only) or 256. block_sparse
 * (b_kn = 0 only): skip the zero 64-wide K blocks of B as omm_kernel_gemm_tc_blocksparse, with the
 * same result. The FP32 accumulation runs over the same products in the same K order as the
 * single-SM kernels. cluster_pairs = 2 (block_sparse = 0 only): two such pairs per cluster of four
 * CTAs, side by side along N (256 x 2 tile_n per cluster), share A: each SM loads half of its 128
 * A rows and multicasts them to its counterpart in the other pair, so A leaves L2 once per two
 * column tiles. Scratch is allocated and freed inside the call. Errors: OMM_ERR_ARG, OMM_ERR_OOM,
 * OMM_ERR_TIMEOUT, OMM_ERR_CUDA. */
omm_status omm_kernel_gemm_tc_pair(int M, int N, int K, const double* A, const double* B, double alpha,
                                   double beta, double* C, int npass, int tile_n, int b_kn, int block_sparse,
                                   int cluster_pairs, void* stream);

/* Float64-class contraction on the BF16 tensor cores, as the mixed path
 * refreshes its state (float64 emulation by error-free fixed-point slicing:
 * Ozaki, Ogita, Oishi and Rump, Numer. Algorithms 59, 2012): C = alpha A B^T +
 * beta C with A M x K, B N x K, C M x N row-major float64. Every row of A and
 * of B is cut into `slices` (1..10) bf16 slices of 5 bits each below a
 * power-of-two row scale; the slice products of one level are exact in the
 * FP32 accumulator for K <= 16384 and are summed in float64. Each slice adds
 * 5 bits: with s slices the error is about 2^-5s times (row maximum of A) x
 * (row maximum of B) x K. Scratch is allocated and freed inside
 * the call. Errors: OMM_ERR_ARG (including K > 16384), OMM_ERR_OOM,
 * OMM_ERR_TIMEOUT, OMM_ERR_CUDA. */
omm_status omm_kernel_gemm_emu(int M, int N, int K, const double* A, const double* B, double alpha,
                               double beta, double* C, int slices, void* stream);

/* omm_kernel_quartic_coefficients for callers that cannot allocate device
 * memory (a runtime whose memory pool owns the whole device, a path that must
 * not let cudaMalloc/cudaFree synchronise the device, an embedding that must
 * not grow its footprint after start-up). The paper has no counterpart: this
 * is a deployment variant of the step above with the same arguments and
 * results. It calls no cudaMalloc, cudaFree or allocating library routine;
 * its scratch (trace partial sums and a control block) is one static device
 * array of about 361 KB that every GPU loading the library keeps until the
 * process exits. Limit: n <= 2048 (larger n returns OMM_ERR_ARG and leaves
 * alpha untouched). The first call on each device, made with that device
 * current, looks the array's device address up (cudaGetSymbolAddress); make
 * that first call before any stream capture. The address is kept for the
 * life of the process: do not call this entry point again on a device after a
 * cudaDeviceReset of that device. The call waits on its stream before it
 * returns (alpha is written on the host). All calls share the array: calls
 * that overlap on the GPU (other streams, other host threads) race and must
 * be serialised by the caller. Errors: OMM_ERR_ARG, OMM_ERR_CUDA. */
omm_status omm_kernel_quartic_coefficients_noalloc(int n, const double* SWHW, const double* Proj,
                                                   double E, double* alpha, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* OMM_GB300_OMM_KERNELS_H */
