// Step-level C entry points of include/omm_kernels.h.
#include "../../include/omm_kernels.h"
#include "omm_internal.cuh"
#include "tc_gemm.cuh"
#include "emu.cuh"

#include <algorithm>

#include <cstring>
#include <string>

using namespace omm;

namespace {

omm_status cuda_fail(const char* where, const CudaError& e) {
  set_last_error(std::string(where) + ": " + e.what + ": " + cudaGetErrorString(e.err));
  return OMM_ERR_CUDA;
}

}  // namespace

extern "C" {

omm_status omm_kernel_dgemm(int transA, int transB, int M, int N, int K, double alpha, const double* A,
                            long lda, const double* B, long ldb, double beta, double* C, long ldc,
                            void* stream) {
  if (M < 0 || N < 0 || K < 0 || !C || (K > 0 && (!A || !B))) {
    set_last_error("omm_kernel_dgemm: invalid argument");
    return OMM_ERR_ARG;
  }
  try {
    cudaStream_t st = (cudaStream_t)stream;
    dgemm(st, transA, transB, M, N, K, alpha, A, lda, 0, B, ldb, 0, beta, C, ldc, 0);
    OMM_CUDA_TRY(cudaStreamSynchronize(st));
  } catch (const CudaError& e) {
    return cuda_fail("omm_kernel_dgemm", e);
  }
  return OMM_OK;
}

omm_status omm_kernel_spd_inverse(int m, const double* A, double* P, int* info, void* stream) {
  if (m <= 0 || !A || !P) {
    set_last_error("omm_kernel_spd_inverse: invalid argument");
    return OMM_ERR_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  double* W = nullptr;
  double* work = nullptr;
  int* info_dev = nullptr;
  omm_status rc = OMM_OK;
  try {
    const size_t mm = (size_t)m * m;
    OMM_CUDA_TRY(cudaMalloc((void**)&W, mm * sizeof(double)));
    OMM_CUDA_TRY(cudaMalloc((void**)&work, spd_inverse_workspace(m) * sizeof(double)));
    OMM_CUDA_TRY(cudaMalloc((void**)&info_dev, sizeof(int)));
    OMM_CUDA_TRY(cudaMemcpyAsync(W, A, mm * sizeof(double), cudaMemcpyDefault, st));
    spd_inverse(st, m, W, P, work, info_dev);
    int h = 0;
    OMM_CUDA_TRY(cudaMemcpyAsync(&h, info_dev, sizeof(int), cudaMemcpyDeviceToHost, st));
    OMM_CUDA_TRY(cudaStreamSynchronize(st));
    if (info) *info = h;
    if (h != 0) {
      set_last_error("omm_kernel_spd_inverse: not positive definite");
      rc = OMM_ERR_NOT_SPD;
    }
  } catch (const CudaError& e) {
    rc = cuda_fail("omm_kernel_spd_inverse", e);
  }
  if (W) cudaFree(W);
  if (work) cudaFree(work);
  if (info_dev) cudaFree(info_dev);
  return rc;
}

namespace {
omm_status spd_inverse_sliced_impl(const char* who, int m, const double* A, double* P, int slices, int* info,
                                   void* stream) {
  if (m <= 0 || !A || !P) {
    set_last_error(std::string(who) + ": invalid argument");
    return OMM_ERR_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  double* W = nullptr;
  void* work = nullptr;
  int* flags = nullptr;  // [0] pivot info, [1] bounded-wait failures
  omm_status rc = OMM_OK;
  try {
    const size_t mm = (size_t)m * m;
    OMM_CUDA_TRY(cudaMalloc((void**)&W, mm * sizeof(double)));
    OMM_CUDA_TRY(cudaMalloc(&work, spd_inverse_sliced_workspace_bytes(m)));
    OMM_CUDA_TRY(cudaMalloc((void**)&flags, 2 * sizeof(int)));
    OMM_CUDA_TRY(cudaMemsetAsync(flags, 0, 2 * sizeof(int), st));
    OMM_CUDA_TRY(cudaMemcpyAsync(W, A, mm * sizeof(double), cudaMemcpyDefault, st));
    spd_inverse_sliced(st, m, W, P, work, flags, flags + 1, slices);
    int h[2] = {0, 0};
    OMM_CUDA_TRY(cudaMemcpyAsync(h, flags, sizeof(h), cudaMemcpyDeviceToHost, st));
    OMM_CUDA_TRY(cudaStreamSynchronize(st));
    if (info) *info = h[0];
    if (h[1] != 0) {
      set_last_error(std::string(who) + ": a bounded device wait expired");
      rc = OMM_ERR_TIMEOUT;
    } else if (h[0] != 0) {
      set_last_error(std::string(who) + ": not positive definite");
      rc = OMM_ERR_NOT_SPD;
    }
  } catch (const CudaError& e) {
    rc = cuda_fail(who, e);
  }
  if (W) cudaFree(W);
  if (work) cudaFree(work);
  if (flags) cudaFree(flags);
  return rc;
}
}  // namespace

omm_status omm_kernel_spd_inverse_sliced(int m, const double* A, double* P, int* info, void* stream) {
  return spd_inverse_sliced_impl("omm_kernel_spd_inverse_sliced", m, A, P, 10, info, stream);
}

omm_status omm_kernel_spd_inverse_precond(int m, const double* A, double* P, int slices, int* info, void* stream) {
  if (slices < 1 || slices > 9) {
    set_last_error("omm_kernel_spd_inverse_precond: slices must be in 1..9");
    return OMM_ERR_ARG;
  }
  return spd_inverse_sliced_impl("omm_kernel_spd_inverse_precond", m, A, P, slices, info, stream);
}

omm_status omm_kernel_line_minimum(const double* alpha, double* x) {
  if (!alpha || !x) {
    set_last_error("omm_kernel_line_minimum: NULL argument");
    return OMM_ERR_ARG;
  }
  double* d = nullptr;
  omm_status rc = OMM_OK;
  try {
    OMM_CUDA_TRY(cudaMalloc((void**)&d, 8 * sizeof(double)));
    OMM_CUDA_TRY(cudaMemcpy(d, alpha, 5 * sizeof(double), cudaMemcpyHostToDevice));
    int* st = (int*)(d + 6);
    launch_line_minimum(nullptr, d, d + 5, st);
    double out[2];
    int s = 0;
    OMM_CUDA_TRY(cudaMemcpy(out, d + 5, sizeof(double), cudaMemcpyDeviceToHost));
    OMM_CUDA_TRY(cudaMemcpy(&s, st, sizeof(int), cudaMemcpyDeviceToHost));
    *x = out[0];
    rc = (s == 0) ? OMM_OK : OMM_ERR_UNBOUNDED;
  } catch (const CudaError& e) {
    rc = cuda_fail("omm_kernel_line_minimum", e);
  }
  if (d) cudaFree(d);
  return rc;
}

omm_status omm_kernel_quartic_coefficients(int n, const double* SWHW, const double* Proj, double E,
                                           double* alpha, void* stream) {
  if (n <= 0 || !SWHW || !Proj || !alpha) {
    set_last_error("omm_kernel_quartic_coefficients: invalid argument");
    return OMM_ERR_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  Scalars* sc = nullptr;
  double* part = nullptr;
  omm_status rc = OMM_OK;
  try {
    OMM_CUDA_TRY(cudaMalloc((void**)&sc, sizeof(Scalars)));
    OMM_CUDA_TRY(cudaMalloc((void**)&part, (size_t)traces_blocks(n) * kNumTraces * sizeof(double)));
    Scalars h;
    std::memset(&h, 0, sizeof(h));
    h.E = E;
    h.max_iter = 1;
    OMM_CUDA_TRY(cudaMemcpyAsync(sc, &h, sizeof(h), cudaMemcpyHostToDevice, st));
    launch_traces(st, n, SWHW, Proj, part, sc);
    launch_control_linesearch(st, sc, part, traces_partials(n));
    OMM_CUDA_TRY(cudaMemcpyAsync(&h, sc, sizeof(h), cudaMemcpyDeviceToHost, st));
    OMM_CUDA_TRY(cudaStreamSynchronize(st));
    for (int q = 0; q < 5; ++q) alpha[q] = h.alpha[q];
  } catch (const CudaError& e) {
    rc = cuda_fail("omm_kernel_quartic_coefficients", e);
  }
  if (sc) cudaFree(sc);
  if (part) cudaFree(part);
  return rc;
}

}  // extern "C"

namespace {

// the persistent launch the solver uses for its line-search GEMMs, on freshly split operands.
// block_sparse: skip the 64-wide K blocks where B is zero (lists built from B); b_kn: B is given
// K x N and read MN-major; pair: 256-row tiles on pairs of SMs
omm_status gemm_tc_impl(const char* name, int M, int N, int K, const double* A, const double* B, double alpha,
                        double beta, double* C, int npass, int tile_n, bool block_sparse, bool b_kn, bool pair,
                        void* stream, bool quad = false) {
  const bool width_ok = pair ? (tile_n == 128 || tile_n == 256 || (tile_n == 192 && !b_kn))
                             : (tile_n == 128 || tile_n == 256);
  if (M <= 0 || N <= 0 || K <= 0 || !A || !B || !C || (npass != 1 && npass != 3) || !width_ok ||
      (b_kn && (npass != 3 || block_sparse)) || (quad && block_sparse)) {
    set_last_error(std::string(name) + ": invalid argument");
    return OMM_ERR_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const long lda = (K + 7) / 8 * 8, ldb = b_kn ? (N + 7) / 8 * 8 : lda;
  __nv_bfloat16* buf = nullptr;
  int* err = nullptr;
  tc::GroupDesc* desc = nullptr;
  tc::BlockLists lists;
  omm_status rc = OMM_OK;
  try {
    const size_t na = (size_t)M * lda, nb = (size_t)(b_kn ? K : N) * ldb;
    if (cudaMalloc((void**)&buf, 2 * (na + nb) * sizeof(__nv_bfloat16)) != cudaSuccess ||
        cudaMalloc((void**)&err, sizeof(int)) != cudaSuccess ||
        cudaMalloc((void**)&desc, sizeof(tc::GroupDesc)) != cudaSuccess) {
      cudaGetLastError();
      if (buf) cudaFree(buf);
      if (err) cudaFree(err);
      set_last_error(std::string(name) + ": device allocation failed");
      return OMM_ERR_OOM;
    }
    __nv_bfloat16 *a_hi = buf, *a_lo = buf + na, *b_hi = buf + 2 * na, *b_lo = buf + 2 * na + nb;
    OMM_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int), st));
    tc::split(st, A, M, K, K, a_hi, a_lo, lda, nullptr);
    tc::Operand oa = tc::make_operand(a_hi, M, K, lda, 2, true);
    tc::Operand ob;
    if (b_kn) {
      tc::split(st, B, K, N, N, b_hi, b_lo, ldb, nullptr);
      ob = tc::make_operand_view(b_hi, K, N, ldb, 2, false, 0, K, /*mn_major=*/true);
    } else {
      tc::split(st, B, N, K, K, b_hi, b_lo, ldb, nullptr);
      ob = tc::make_operand(b_hi, N, K, ldb, 2, false);
    }
    if (block_sparse) tc::block_lists(st, B, N, K, K, tile_n, lists);
    const tc::Epilogue ep{C, N, N, 0, alpha, beta, M, N, nullptr, err};
    const tc::GroupDesc g = tc::make_group(oa, ob, K, ep, 0, tile_n, block_sparse ? &lists : nullptr, pair, quad);
    OMM_CUDA_TRY(cudaMemcpyAsync(desc, &g, sizeof(g), cudaMemcpyHostToDevice, st));
    tc::gemm_persistent(st, desc, 1, tc::tiles_of(ep, tile_n, pair, quad),
                        npass == 3 ? tc::pairs_split3() : tc::pairs_single(), err, tile_n, pair, quad);
    int h = 0;
    OMM_CUDA_TRY(cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    OMM_CUDA_TRY(cudaStreamSynchronize(st));
    if (h != 0) {
      set_last_error(std::string(name) + ": a bounded device wait expired (code " + std::to_string(h) + ")");
      rc = OMM_ERR_TIMEOUT;
    }
  } catch (const CudaError& e) {
    rc = cuda_fail(name, e);
  }
  if (buf) cudaFree(buf);
  if (err) cudaFree(err);
  if (desc) cudaFree(desc);
  tc::free_block_lists(lists, st);
  return rc;
}

}  // namespace

extern "C" {

omm_status omm_kernel_gemm_tc_kn(int M, int N, int K, const double* A, const double* B, double alpha, double beta,
                                 double* C, int tile_n, void* stream) {
  return gemm_tc_impl("omm_kernel_gemm_tc_kn", M, N, K, A, B, alpha, beta, C, 3, tile_n, false, true, false, stream);
}

omm_status omm_kernel_gemm_tc_pair(int M, int N, int K, const double* A, const double* B, double alpha, double beta,
                                   double* C, int npass, int tile_n, int b_kn, int block_sparse, int cluster_pairs,
                                   void* stream) {
  if (cluster_pairs != 1 && cluster_pairs != 2) {
    set_last_error("omm_kernel_gemm_tc_pair: invalid argument");
    return OMM_ERR_ARG;
  }
  return gemm_tc_impl("omm_kernel_gemm_tc_pair", M, N, K, A, B, alpha, beta, C, npass, tile_n, block_sparse != 0,
                      b_kn != 0, true, stream, cluster_pairs == 2);
}

omm_status omm_kernel_gemm_tc_tiled(int M, int N, int K, const double* A, const double* B, double alpha,
                                    double beta, double* C, int npass, int tile_n, void* stream) {
  return gemm_tc_impl("omm_kernel_gemm_tc_tiled", M, N, K, A, B, alpha, beta, C, npass, tile_n, false, false, false,
                      stream);
}

omm_status omm_kernel_gemm_tc(int M, int N, int K, const double* A, const double* B, double alpha,
                              double beta, double* C, int npass, void* stream) {
  return gemm_tc_impl("omm_kernel_gemm_tc", M, N, K, A, B, alpha, beta, C, npass, 256, false, false, false, stream);
}

omm_status omm_kernel_gemm_tc_blocksparse(int M, int N, int K, const double* A, const double* B, double alpha,
                                          double beta, double* C, int npass, int tile_n, void* stream) {
  return gemm_tc_impl("omm_kernel_gemm_tc_blocksparse", M, N, K, A, B, alpha, beta, C, npass, tile_n, true, false,
                      false, stream);
}

omm_status omm_kernel_gemm_emu(int M, int N, int K, const double* A, const double* B, double alpha,
                               double beta, double* C, int slices, void* stream) {
  if (M <= 0 || N <= 0 || K <= 0 || K > 16384 || !A || !B || !C || slices < 1 || slices > 10) {
    set_last_error("omm_kernel_gemm_emu: invalid argument");
    return OMM_ERR_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const long ld = (K + 7) / 8 * 8;
  __nv_bfloat16* buf = nullptr;
  int* err = nullptr;
  double* partial = nullptr;  // chunk sums, for products of few tiles (as the solver runs them)
  const long partial_cap = std::min(11L * M * N, 1L << 24);
  omm_status rc = OMM_OK;
  try {
    const size_t na = (size_t)slices * M * ld, nb = (size_t)slices * N * ld;
    if (cudaMalloc((void**)&buf, (na + nb) * sizeof(__nv_bfloat16)) != cudaSuccess ||
        cudaMalloc((void**)&err, sizeof(int)) != cudaSuccess ||
        cudaMalloc((void**)&partial, partial_cap * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      if (buf) cudaFree(buf);
      if (err) cudaFree(err);
      set_last_error("omm_kernel_gemm_emu: device allocation failed");
      return OMM_ERR_OOM;
    }
    OMM_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int), st));
    emu::slice_rows(st, A, M, K, K, slices, buf, ld, nullptr);
    emu::slice_rows(st, B, N, K, K, slices, buf + na, ld, nullptr);
    tc::Operand oa = tc::make_operand(buf, M, K, ld, slices, true);
    tc::Operand ob = tc::make_operand(buf + na, N, K, ld, slices, false);
    emu::gemm(st, oa, ob, K, slices, tc::Epilogue{C, N, N, 0, alpha, beta, M, N, nullptr, err}, partial,
              partial_cap);
    int h = 0;
    OMM_CUDA_TRY(cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    OMM_CUDA_TRY(cudaStreamSynchronize(st));
    if (h != 0) {
      set_last_error("omm_kernel_gemm_emu: a bounded device wait expired");
      rc = OMM_ERR_TIMEOUT;
    }
  } catch (const CudaError& e) {
    rc = cuda_fail("omm_kernel_gemm_emu", e);
  }
  if (buf) cudaFree(buf);
  if (err) cudaFree(err);
  if (partial) cudaFree(partial);
  return rc;
}

}  // extern "C"
