// Float64 GEMM on the FP64 pipes (DFMA). GB300 keeps only a small float64
// rate, so this kernel is issue-bound on DFMA, not on memory: 64x64 tiles,
// a 4x4 register block per thread, operands staged through shared memory.
// It serves the float64 OMM path, the float64 refinement and certificate of
// the mixed path, and the Cholesky inverse of the preconditioner.
#include "omm_internal.cuh"

namespace omm {
namespace {

constexpr int BM = 64, BN = 64, BK = 16, NT = 256;

__global__ void __launch_bounds__(NT)
dgemm_kernel(int transA, int transB, int M, int N, int K, double alpha,
             const double* __restrict__ A, long lda, long sA,
             const double* __restrict__ B, long ldb, long sB,
             double beta, double* C, long ldc, long sC, int tri, const int* skip) {
  if (skip != nullptr && (skip[0] | skip[1])) return;
  const int row0 = blockIdx.y * BM;
  const int col0 = blockIdx.x * BN;
  if ((tri & kTriLower) && col0 > row0 + BM - 1) return;
  A += (long)blockIdx.z * sA;
  B += (long)blockIdx.z * sB;
  C += (long)blockIdx.z * sC;

  __shared__ double As[BK][BM];
  __shared__ double Bs[BK][BN];
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;
  double acc[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[r][c] = 0.0;

  int kbeg = 0, kend = K;
  if (tri & kTriKStart) kbeg = (max(row0, col0) / BK) * BK;
  if (tri & kTriKFromCol) kbeg = max(kbeg, (col0 / BK) * BK);
  if (tri & kTriKToRow) kend = min(K, row0 + BM);
  for (int k0 = kbeg; k0 < kend; k0 += BK) {
#pragma unroll
    for (int t = 0; t < (BM * BK) / NT; ++t) {
      const int idx = tid + t * NT;
      int i, k;
      double v = 0.0;
      if (!transA) {
        i = idx / BK; k = idx % BK;
        const int gi = row0 + i, gk = k0 + k;
        if (gi < M && gk < K) v = A[(long)gi * lda + gk];
      } else {
        k = idx / BM; i = idx % BM;
        const int gi = row0 + i, gk = k0 + k;
        if (gi < M && gk < K) v = A[(long)gk * lda + gi];
      }
      As[k][i] = v;
    }
#pragma unroll
    for (int t = 0; t < (BN * BK) / NT; ++t) {
      const int idx = tid + t * NT;
      int j, k;
      double v = 0.0;
      if (!transB) {
        k = idx / BN; j = idx % BN;
        const int gj = col0 + j, gk = k0 + k;
        if (gj < N && gk < K) v = B[(long)gk * ldb + gj];
      } else {
        j = idx / BK; k = idx % BK;
        const int gj = col0 + j, gk = k0 + k;
        if (gj < N && gk < K) v = B[(long)gj * ldb + gk];
      }
      Bs[k][j] = v;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < BK; ++k) {
      double a[4], b[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) a[r] = As[k][ty + 16 * r];
#pragma unroll
      for (int c = 0; c < 4; ++c) b[c] = Bs[k][tx + 16 * c];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = fma(a[r], b[c], acc[r][c]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int gi = row0 + ty + 16 * r;
    if (gi >= M) continue;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int gj = col0 + tx + 16 * c;
      if (gj >= N) continue;
      double* p = C + (long)gi * ldc + gj;
      const double v = alpha * acc[r][c];
      *p = (beta == 0.0) ? v : fma(beta, *p, v);
    }
  }
}

}  // namespace

void dgemm(cudaStream_t st, int transA, int transB, int M, int N, int K, double alpha,
           const double* A, long lda, long strideA, const double* B, long ldb, long strideB,
           double beta, double* C, long ldc, long strideC, int batch, int tri, const int* skip) {
  if (M <= 0 || N <= 0 || batch <= 0) return;
  dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM, batch);
  dgemm_kernel<<<grid, NT, 0, st>>>(transA, transB, M, N, K, alpha, A, lda, strideA, B, ldb,
                                     strideB, beta, C, ldc, strideC, tri, skip);
  OMM_LAUNCH_CHECK();
}

}  // namespace omm
