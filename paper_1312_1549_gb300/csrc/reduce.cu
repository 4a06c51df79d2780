// Cholesky reduction to standard form (Sec. 2.4, last paragraph): S = L L^T,
// H_r = L^-1 H L^-T, C_r = L^T C and back. The float64 path multiplies with the
// DFMA GEMM and skips the zero triangle of L and L^-1 (K loop cut at the diagonal);
// the mixed path uses float64-class sliced tensor-core products whose triangular
// B operands are described by block lists, so that their zero 64-wide K blocks are
// skipped too. H_r is formed as (Y H) Y^T with Y = L^-1: first W = H Y^T, then its
// transpose Y H (H symmetric) as the A operand of the second product.
#include "emu.cuh"
#include "reduce.cuh"
#include "tc_gemm.cuh"

#include <algorithm>
#include <new>

namespace omm {

namespace {
constexpr int kRedSlices = 10;  // fixed-point slices (about 50 bits of each row-scaled operand)

long round8(long x) { return (x + 7) / 8 * 8; }

__global__ void identity_kernel(int m, double* A) {
  const long count = (long)m * m;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < count; idx += (long)gridDim.x * blockDim.x)
    A[idx] = (idx / m == idx % m) ? 1.0 : 0.0;
}
}  // namespace

struct Reduction {
  int m = 0;
  bool sliced = false;
  double* L = nullptr;   // float64 path: L (lower); sliced path: L^T (upper)
  double* Y = nullptr;   // L^-1 (lower)
  double* YT = nullptr;  // sliced path: L^-T (upper)
  double* W = nullptr;   // m x m scratch of the Hamiltonian reduction
  __nv_bfloat16* slA = nullptr;  // slices of the A operand (up to m x m)
  __nv_bfloat16* slB = nullptr;  // slices of the B operand (m x m)
  long ldm = 0;
  double* partial = nullptr;
  long partial_cap = 0;
  int* err = nullptr;
  tc::BlockLists blY, blYT, blLT;  // nonzero K blocks of Y, L^-T, L^T as B operands
};

namespace {

template <typename T>
void alloc(T** p, size_t count, cudaStream_t st) {
  mem::alloc(p, count, st);
}

// out (M x m) = alpha A B^T with A (M x m rows, float64) and B (m x m, float64) row-major
void sliced_product(Reduction* r, cudaStream_t st, const double* A, long M, const double* B,
                    const tc::BlockLists* lists, double* out) {
  const int m = r->m;
  emu::slice_rows(st, A, M, m, m, kRedSlices, r->slA, r->ldm, nullptr);
  emu::slice_rows(st, B, m, m, m, kRedSlices, r->slB, r->ldm, nullptr);
  const tc::Operand oa = tc::make_operand(r->slA, M, m, r->ldm, kRedSlices, true);
  const tc::Operand ob = tc::make_operand(r->slB, m, m, r->ldm, kRedSlices, false);
  emu::gemm(st, oa, ob, m, kRedSlices, tc::Epilogue{out, m, m, 0, 1.0, 0.0, (int)M, m, nullptr, r->err},
            r->partial, r->partial_cap, lists);
}

}  // namespace

void launch_identity(cudaStream_t st, int m, double* A) {
  const long count = (long)m * m;
  identity_kernel<<<(unsigned)std::min<long>((count + 255) / 256, 4096), 256, 0, st>>>(m, A);
  OMM_LAUNCH_CHECK();
}

Reduction* reduction_create(cudaStream_t st, int m, bool sliced, double* S, int* info_dev) {
  Reduction* r = new Reduction();
  void* work = nullptr;
  try {
    r->m = m;
    r->sliced = sliced;
    const size_t mm = (size_t)m * m;
    alloc(&r->L, mm, st);
    alloc(&r->Y, mm, st);
    alloc(&r->W, mm, st);
    alloc(&r->err, 1, st);
    OMM_CUDA_TRY(cudaMemsetAsync(r->err, 0, sizeof(int), st));
    if (sliced) {
      r->ldm = round8(m);
      alloc(&r->YT, mm, st);
      alloc(&r->slA, (size_t)kRedSlices * m * r->ldm, st);
      alloc(&r->slB, (size_t)kRedSlices * m * r->ldm, st);
      r->partial_cap = partial_capacity(m);
      alloc(&r->partial, (size_t)r->partial_cap, st);
      alloc(reinterpret_cast<char**>(&work), spd_inverse_sliced_workspace_bytes(m), st);
      spd_factor_inverse_sliced(st, m, S, r->Y, work, info_dev, r->err);
      emu::transpose(st, S, m, m, m, r->L, m);     // L^T
      emu::transpose(st, r->Y, m, m, m, r->YT, m);  // L^-T
      tc::block_lists(st, r->Y, m, m, m, 256, r->blY);
      tc::block_lists(st, r->YT, m, m, m, 256, r->blYT);
      tc::block_lists(st, r->L, m, m, m, 256, r->blLT);
    } else {
      alloc(reinterpret_cast<double**>(&work), spd_inverse_workspace(m), st);
      spd_factor_inverse(st, m, S, r->Y, static_cast<double*>(work), info_dev);
      OMM_CUDA_TRY(cudaMemcpyAsync(r->L, S, mm * sizeof(double), cudaMemcpyDeviceToDevice, st));
    }
    mem::release(work, st);  // stream-ordered: after the factorisation that uses it
  } catch (...) {
    cudaStreamSynchronize(st);
    mem::release(work, st);
    reduction_destroy(r, st);
    throw;
  }
  return r;
}

void reduction_destroy(Reduction* r, cudaStream_t st) {
  if (!r) return;
  void* bufs[] = {r->L, r->Y, r->YT, r->W, r->slA, r->slB, r->partial, r->err};
  for (void* b : bufs) mem::release(b, st);
  tc::free_block_lists(r->blY, st);
  tc::free_block_lists(r->blYT, st);
  tc::free_block_lists(r->blLT, st);
  delete r;
}

int reduction_error(Reduction* r, cudaStream_t st) {
  int e = 0;
  OMM_CUDA_TRY(cudaMemcpyAsync(&e, r->err, sizeof(int), cudaMemcpyDeviceToHost, st));
  OMM_CUDA_TRY(cudaStreamSynchronize(st));
  return e;
}

void reduce_hamiltonian(Reduction* r, cudaStream_t st, double* H) {
  const int m = r->m;
  if (r->sliced) {
    sliced_product(r, st, H, m, r->Y, &r->blY, r->W);  // W = H Y^T
    emu::transpose(st, r->W, m, m, m, H, m);           // Y H
    sliced_product(r, st, H, m, r->Y, &r->blY, H);     // (Y H) Y^T (A is sliced before H is written)
  } else {
    // W = Y H (Y lower: the K loop ends at the tile's last row)
    dgemm(st, 0, 0, m, m, m, 1.0, r->Y, m, 0, H, m, 0, 0.0, r->W, m, 0, 1, kTriKToRow);
    // H_r = Y W^T = Y H Y^T, lower tiles
    dgemm(st, 0, 1, m, m, m, 1.0, r->Y, m, 0, r->W, m, 0, 0.0, H, m, 0, 1, kTriLower | kTriKToRow);
  }
  launch_symmetrize_lower(st, m, H);
}

void reduce_coefficients(Reduction* r, cudaStream_t st, int n, const double* C, double* out) {
  const int m = r->m;
  if (r->sliced) sliced_product(r, st, C, n, r->L, &r->blLT, out);  // C (L^T)^T
  else dgemm(st, 0, 0, n, m, m, 1.0, C, m, 0, r->L, m, 0, 0.0, out, m, 0, 1, kTriKFromCol);
}

void restore_coefficients(Reduction* r, cudaStream_t st, int n, const double* Cr, double* out) {
  const int m = r->m;
  if (r->sliced) sliced_product(r, st, Cr, n, r->YT, &r->blYT, out);  // C_r (L^-T)^T
  else dgemm(st, 0, 0, n, m, m, 1.0, Cr, m, 0, r->Y, m, 0, 0.0, out, m, 0, 1, kTriKFromCol);
}

}  // namespace omm
