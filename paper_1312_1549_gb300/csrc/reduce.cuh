// Reduction of the generalised eigenproblem H c = eps S c to standard form by the
// Cholesky factorisation S = L L^T, the alternative to the kinetic preconditioner that
// the paper describes at the end of Sec. 2.4 (its "OMM (Cholesky)" flavour of Sec. 3):
//   H_r = L^-1 H L^-T,   C_r = L^T C,   C = L^-T C_r,
// after which the OMM runs with S = I and without a preconditioner. Its iterates follow,
// in exact arithmetic, those of the original problem preconditioned by S^-1, and S_W,
// H_W and the energy are the same in both bases.
#pragma once
#include "omm_internal.cuh"

namespace omm {

struct Reduction;

// Factor S (m x m, device, symmetric positive definite; overwritten) and keep L and L^-1.
// sliced: float64-class products on the tensor cores (fixed-point slices) instead of native
// float64. info_dev receives 0 or the 1-based column of the first non-positive pivot.
Reduction* reduction_create(cudaStream_t st, int m, bool sliced, double* S, int* info_dev);
void reduction_destroy(Reduction* r, cudaStream_t st);  // st: the owner's current stream
// nonzero if a bounded wait of a tensor-core product expired (synchronises the stream)
int reduction_error(Reduction* r, cudaStream_t st);
// H (m x m, device) <- L^-1 H L^-T, exactly symmetric
void reduce_hamiltonian(Reduction* r, cudaStream_t st, double* H);
// rows of the n x m coefficient layout: out = C L (C_r = L^T C in the paper's m x n layout)
void reduce_coefficients(Reduction* r, cudaStream_t st, int n, const double* C, double* out);
// out = C_r L^-1 (C = L^-T C_r in the paper's layout)
void restore_coefficients(Reduction* r, cudaStream_t st, int n, const double* Cr, double* out);
// A (m x m, device) <- I
void launch_identity(cudaStream_t st, int m, double* A);

}  // namespace omm
