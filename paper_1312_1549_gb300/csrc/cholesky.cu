// Float64 inverse of a symmetric positive definite matrix, for the kinetic
// preconditioner P = (S + T/tau)^-1 (Sec. 2.4, Eq. 17), computed once per
// geometry. Three stages, all on the device:
//   1. blocked right-looking Cholesky A = L L^T (64-column panels; the
//      diagonal block is factored and inverted by one CTA in shared memory,
//      the panel and the trailing update are float64 GEMMs),
//   2. Y = L^-1 by recursive halving: inv([L11 0; L21 L22]) =
//      [Y11 0; -Y22 L21 Y11  Y22], whose base cases are the inverted diagonal
//      blocks of stage 1,
//   3. P = Y^T Y (lower tiles only, K loop from the diagonal), then mirrored.
// A failed pivot (<= 0 or NaN) is recorded in info_dev and replaced by 1 so
// that the remaining stages stay finite; the caller reports the failure.
#include "omm_internal.cuh"

namespace omm {
namespace {

constexpr int NB = 64;

// Factor the b x b diagonal block at A (ld lda) in place (lower) and write
// its inverse to Linv (NB x NB, row-major, zero above the diagonal).
__global__ void __launch_bounds__(256)
potf2_inv_kernel(double* A, long lda, int b, double* Linv, int* info, int col_offset) {
  __shared__ double L[NB][NB + 1];
  const int tid = threadIdx.x;
  for (int idx = tid; idx < NB * NB; idx += blockDim.x) {
    const int i = idx / NB, j = idx % NB;
    L[i][j] = (i < b && j < b && j <= i) ? A[(long)i * lda + j] : 0.0;
  }
  __syncthreads();
  for (int j = 0; j < b; ++j) {
    if (tid == 0) {
      double d = L[j][j];
      if (!(d > 0.0)) {
        atomicCAS(info, 0, col_offset + j + 1);
        d = 1.0;
      }
      L[j][j] = sqrt(d);
    }
    __syncthreads();
    const double djj = L[j][j];
    for (int i = j + 1 + tid; i < b; i += blockDim.x) L[i][j] /= djj;
    __syncthreads();
    const int r = b - j - 1;
    for (int idx = tid; idx < r * r; idx += blockDim.x) {
      const int i = j + 1 + idx / r, l = j + 1 + idx % r;
      if (l <= i) L[i][l] -= L[i][j] * L[l][j];
    }
    __syncthreads();
  }
  for (int idx = tid; idx < b * b; idx += blockDim.x) {
    const int i = idx / b, j = idx % b;
    A[(long)i * lda + j] = (j <= i) ? L[i][j] : 0.0;
  }
  // inverse of the lower-triangular block: column c solves L x = e_c
  __shared__ double X[NB][NB + 1];
  if (tid < NB) {
    const int c = tid;
    for (int i = 0; i < NB; ++i) X[i][c] = 0.0;
    if (c < b) {
      X[c][c] = 1.0 / L[c][c];
      for (int i = c + 1; i < b; ++i) {
        double s = 0.0;
        for (int k = c; k < i; ++k) s = fma(L[i][k], X[k][c], s);
        X[i][c] = -s / L[i][i];
      }
    }
  }
  __syncthreads();
  for (int idx = tid; idx < NB * NB; idx += blockDim.x) {
    const int i = idx / NB, j = idx % NB;
    Linv[idx] = X[i][j];
  }
}

__global__ void zero_upper_kernel(int m, double* A) {
  const long count = (long)m * m;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < count;
       idx += (long)gridDim.x * blockDim.x) {
    const long i = idx / m, j = idx % m;
    if (j > i) A[idx] = 0.0;
  }
}

__global__ void copy_block_kernel(int b, const double* src, long lds, double* dst, long ldd) {
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < b * b; idx += gridDim.x * blockDim.x) {
    const int i = idx / b, j = idx % b;
    dst[(long)i * ldd + j] = src[(long)i * lds + j];
  }
}

struct Work {
  double* Dinv;  // nblk x NB x NB diagonal-block inverses
  double* tmp;   // up to m*m/4 (+ panel) scratch
};

// Y[r0:r1, r0:r1] (lower, in place) <- its inverse
void trtri_rec(cudaStream_t st, int m, double* Y, const Work& w, int r0, int r1) {
  const int nb_blocks = (r1 - r0 + NB - 1) / NB;
  if (nb_blocks <= 1) {
    const int b = r1 - r0;
    copy_block_kernel<<<16, 256, 0, st>>>(b, w.Dinv + (long)(r0 / NB) * NB * NB, NB,
                                          Y + (long)r0 * m + r0, m);
    OMM_LAUNCH_CHECK();
    return;
  }
  const int mid = r0 + (nb_blocks / 2) * NB;
  trtri_rec(st, m, Y, w, r0, mid);
  trtri_rec(st, m, Y, w, mid, r1);
  const int n1 = mid - r0, n2 = r1 - mid;
  double* L21 = Y + (long)mid * m + r0;
  const double* Y11 = Y + (long)r0 * m + r0;
  const double* Y22 = Y + (long)mid * m + mid;
  // W = L21 * Y11  (n2 x n1); Y11 is lower triangular
  dgemm(st, 0, 0, n2, n1, n1, 1.0, L21, m, 0, Y11, m, 0, 0.0, w.tmp, n1, 0, 1, kTriKFromCol);
  // Y21 = -Y22 * W; Y22 is lower triangular
  dgemm(st, 0, 0, n2, n1, n2, -1.0, Y22, m, 0, w.tmp, n1, 0, 0.0, L21, m, 0, 1, kTriKToRow);
}

}  // namespace

size_t spd_inverse_workspace(int m) {
  const long nblk = (m + NB - 1) / NB;
  const long half = (m + 1) / 2 + NB;
  return (size_t)(nblk * NB * NB) + (size_t)(half * half) + (size_t)m * NB;
}

void spd_inverse(cudaStream_t st, int m, double* A, double* P, double* work, int* info_dev) {
  const int nblk = (m + NB - 1) / NB;
  Work w{work, work + (long)nblk * NB * NB};
  OMM_CUDA_TRY(cudaMemsetAsync(info_dev, 0, sizeof(int), st));
  // 1. Cholesky
  for (int kb = 0; kb < nblk; ++kb) {
    const int k = kb * NB;
    const int b = (m - k < NB) ? (m - k) : NB;
    double* Akk = A + (long)k * m + k;
    potf2_inv_kernel<<<1, 256, 0, st>>>(Akk, m, b, w.Dinv + (long)kb * NB * NB, info_dev, k);
    OMM_LAUNCH_CHECK();
    const int r = m - k - b;
    if (r > 0) {
      double* A21 = A + (long)(k + b) * m + k;
      // L21 = A21 * Linv^T (to scratch, then back)
      dgemm(st, 0, 1, r, b, b, 1.0, A21, m, 0, w.Dinv + (long)kb * NB * NB, NB, 0, 0.0, w.tmp, b, 0);
      OMM_CUDA_TRY(cudaMemcpy2DAsync(A21, sizeof(double) * m, w.tmp, sizeof(double) * b,
                                     sizeof(double) * b, r, cudaMemcpyDeviceToDevice, st));
      // A22 -= L21 L21^T (lower tiles)
      double* A22 = A + (long)(k + b) * m + (k + b);
      dgemm(st, 0, 1, r, r, b, -1.0, A21, m, 0, A21, m, 0, 1.0, A22, m, 0, 1, kTriLower);
    }
  }
  zero_upper_kernel<<<1024, 256, 0, st>>>(m, A);
  OMM_LAUNCH_CHECK();
  // 2. Y = L^-1 in place
  trtri_rec(st, m, A, w, 0, m);
  // 3. P = Y^T Y (lower), mirrored
  dgemm(st, 1, 0, m, m, m, 1.0, A, m, 0, A, m, 0, 0.0, P, m, 0, 1, kTriLower | kTriKStart);
  launch_symmetrize_lower(st, m, P);
}

}  // namespace omm
