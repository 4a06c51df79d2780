// Hermitian (complex) problems, as the paper writes the method (Secs. 2.1-2.3, with C^H) and
// as its k-point tests need them (Sec. 3.3), on the real path through the real form
//   phi(A) = [[Re A, -Im A], [Im A, Re A]]          (2m x 2m for an m x m complex A).
// phi is a ring homomorphism with phi(A^H) = phi(A)^T and Tr phi(A) = 2 Re Tr A, so for
// C_e = phi(C) every quantity of the real OMM is the real form of the complex one:
// S_W,e = phi(S_W), G_e = phi(G), E~_e = 2 E~, and the line-search steps are the same. The
// real solve starts from phi(C0) (rows [Re c_j | Im c_j] and [-Im c_j | Re c_j] in the n x m
// layout) and stays there; C, D and EDM are read back from the first block row or column.
// The price is twice the arithmetic of complex products (the real form repeats each block).
#include "omm_ctx.cuh"

#include <new>
#include <vector>

namespace omm {
namespace {

// dst (2m x 2m) = phi(src), src m x m complex interleaved, row-major
__global__ void embed_matrix_kernel(int m, const double2* __restrict__ src, double* __restrict__ dst) {
  const long count = (long)m * m;
  const long ld = 2L * m;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < count; idx += (long)gridDim.x * blockDim.x) {
    const long i = idx / m, j = idx % m;
    const double2 a = src[idx];
    dst[i * ld + j] = a.x;
    dst[i * ld + m + j] = -a.y;
    dst[(m + i) * ld + j] = a.y;
    dst[(m + i) * ld + m + j] = a.x;
  }
}

// rows of phi(C) in the n x m layout: dst (2n x 2m) from src (n x m complex)
__global__ void embed_rows_kernel(int n, int m, const double2* __restrict__ src, double* __restrict__ dst) {
  const long count = (long)n * m;
  const long ld = 2L * m;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < count; idx += (long)gridDim.x * blockDim.x) {
    const long j = idx / m, k = idx % m;
    const double2 c = src[idx];
    dst[j * ld + k] = c.x;
    dst[j * ld + m + k] = c.y;
    dst[(n + j) * ld + k] = -c.y;
    dst[(n + j) * ld + m + k] = c.x;
  }
}

// dst (n x m complex) = the first n rows of C_e (2n x 2m): c_j = C_e[j, :m] + i C_e[j, m:]
__global__ void extract_rows_kernel(int n, int m, const double* __restrict__ src, double2* __restrict__ dst) {
  const long count = (long)n * m;
  const long ld = 2L * m;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < count; idx += (long)gridDim.x * blockDim.x) {
    const long j = idx / m, k = idx % m;
    dst[idx] = make_double2(src[j * ld + k], src[j * ld + m + k]);
  }
}

// dst (m x m complex) from phi(A) (2m x 2m): A_ij = phi[i][j] + i phi[m + i][j]
__global__ void extract_matrix_kernel(int m, const double* __restrict__ src, double2* __restrict__ dst) {
  const long count = (long)m * m;
  const long ld = 2L * m;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < count; idx += (long)gridDim.x * blockDim.x) {
    const long i = idx / m, j = idx % m;
    dst[idx] = make_double2(src[i * ld + j], src[(m + i) * ld + j]);
  }
}

// the nearest real form: rows j and n + j of C_e (2n x 2m) averaged onto one complex row
__global__ void project_rows_kernel(int n, int m, double* __restrict__ Ce) {
  const long count = (long)n * m;
  const long ld = 2L * m;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < count; idx += (long)gridDim.x * blockDim.x) {
    const long j = idx / m, k = idx % m;
    double* top = Ce + j * ld;
    double* bot = Ce + (n + j) * ld;
    const double re = 0.5 * (top[k] + bot[m + k]);
    const double im = 0.5 * (top[m + k] - bot[k]);
    top[k] = re;
    top[m + k] = im;
    bot[k] = -im;
    bot[m + k] = re;
  }
}

unsigned grid_for(long count) { return (unsigned)std::min<long>((count + 255) / 256, 4096); }

template <typename T>
void alloc(T** p, size_t count, cudaStream_t st) {
  mem::alloc(p, count, st);
}

// phi(A) of a complex m x m matrix (host or device) into dst (device, 4 m^2 doubles); stage: 2 m^2
void embed_matrix(cudaStream_t st, int m, const double* A, double* stage, double* dst) {
  copy_in(stage, A, 2L * m * m, st);
  embed_matrix_kernel<<<grid_for((long)m * m), 256, 0, st>>>(m, reinterpret_cast<const double2*>(stage), dst);
  OMM_LAUNCH_CHECK();
}

void embed_rows(cudaStream_t st, int n, int m, const double* C, double* stage, double* dst) {
  copy_in(stage, C, 2L * n * m, st);
  embed_rows_kernel<<<grid_for((long)n * m), 256, 0, st>>>(n, m, reinterpret_cast<const double2*>(stage), dst);
  OMM_LAUNCH_CHECK();
}

void extract_rows(cudaStream_t st, int n, int m, const double* Ce, double* stage, double* out) {
  extract_rows_kernel<<<grid_for((long)n * m), 256, 0, st>>>(n, m, Ce, reinterpret_cast<double2*>(stage));
  OMM_LAUNCH_CHECK();
  OMM_CUDA_TRY(cudaMemcpyAsync(out, stage, 2L * n * m * sizeof(double), cudaMemcpyDefault, st));
}

void extract_matrix(cudaStream_t st, int m, const double* Ae, double* stage, double* out) {
  extract_matrix_kernel<<<grid_for((long)m * m), 256, 0, st>>>(m, Ae, reinterpret_cast<double2*>(stage));
  OMM_LAUNCH_CHECK();
  OMM_CUDA_TRY(cudaMemcpyAsync(out, stage, 2L * m * m * sizeof(double), cudaMemcpyDefault, st));
}

// the embedded inputs of one instance (carved from one block), released after the real create
// copied them
struct Embedded {
  double* stage = nullptr;
  double* H = nullptr;
  double* S = nullptr;
  double* T = nullptr;
};

size_t embedded_doubles(int m, bool with_T) { return (size_t)m * m * (with_T ? 14 : 10); }

void embed_inputs(cudaStream_t st, int m, const double* H, const double* S, const double* T, double* block,
                  Embedded& e) {
  const size_t mm = (size_t)m * m;
  e.stage = block;
  e.H = block + 2 * mm;
  e.S = block + 6 * mm;
  e.T = T ? block + 10 * mm : nullptr;
  embed_matrix(st, m, H, e.stage, e.H);
  embed_matrix(st, m, S, e.stage, e.S);
  if (T) embed_matrix(st, m, T, e.stage, e.T);
}

// complex-side buffers of a context made by omm_create_hermitian
void attach(omm_ctx* c, int m, int n) {
  c->hermitian = true;
  c->real_form = true;
  c->mc = m;
  c->nc = n;
  alloc(&c->hz_stage, 2 * (size_t)m * m, c->st);
  alloc(&c->hz_rows, 4 * (size_t)n * m, c->st);
}

// complex C0 -> embedded rows in hz_rows
void embed_start(omm_ctx* c, cudaStream_t st, const double* C0) {
  embed_rows(st, c->nc, c->mc, C0, c->hz_stage, c->hz_rows);
}

// the complex report of the real solve of phi
void halve_info(omm_info* inf) {
  inf->E *= 0.5;
  inf->Etilde *= 0.5;
}

omm_status check_hermitian(omm_ctx* c, const char* who) {
  if (!c) return fail(OMM_ERR_ARG, std::string(who) + ": NULL context");
  if (!c->hermitian) return fail(OMM_ERR_ARG, std::string(who) + ": not a Hermitian context");
  return OMM_OK;
}

}  // namespace

void project_real_form(omm_ctx* c, cudaStream_t st) {
  if (!c->real_form || c->red) return;  // (the Cholesky flavour's reduced basis has no such structure)
  project_rows_kernel<<<grid_for((long)c->nc * c->mc), 256, 0, st>>>(c->nc, c->mc, c->C);
  OMM_LAUNCH_CHECK();
}

}  // namespace omm

using namespace omm;

extern "C" {

omm_status omm_create_hermitian(int m, int n, const double* H, const double* S, const double* T, double eta,
                                double tau, const omm_opts* opts, void* stream, omm_ctx** out) {
  if (out) *out = nullptr;
  if (!out || !H || !S) return fail(OMM_ERR_ARG, "omm_create_hermitian: NULL argument");
  if (m <= 0 || n <= 0 || n >= m) return fail(OMM_ERR_ARG, "omm_create_hermitian: need 0 < n < m");
  if (opts && opts->cholesky && opts->precision == OMM_PREC_MIXED)
    return fail(OMM_ERR_ARG, "omm_create_hermitian: the Cholesky flavour of a Hermitian problem needs OMM_PREC_FP64");
  cudaStream_t st = (cudaStream_t)stream;
  Embedded e;
  double* block = nullptr;
  omm_status rc = OMM_OK;
  auto release = [&]() {
    cudaStreamSynchronize(st);
    mem::release(block, st);
    block = nullptr;
  };
  try {
    alloc(&block, embedded_doubles(m, T != nullptr), st);
    embed_inputs(st, m, H, S, T, block, e);
    rc = omm_create(2 * m, 2 * n, e.H, e.S, e.T, eta, tau, opts, stream, out);
    release();
    if (rc != OMM_OK) return rc;
    attach(*out, m, n);
  } catch (const std::bad_alloc&) {
    release();
    if (*out) { omm_free(*out); *out = nullptr; }
    return fail(OMM_ERR_OOM, "omm_create_hermitian: device allocation failed");
  } catch (const CudaError& err) {
    release();
    if (*out) { omm_free(*out); *out = nullptr; }
    return fail(OMM_ERR_CUDA, std::string("omm_create_hermitian: ") + err.what + ": " + cudaGetErrorString(err.err));
  }
  return OMM_OK;
}

omm_status omm_update_H_hermitian(omm_ctx* c, const double* H) {
  omm_status rc = check_hermitian(c, "omm_update_H_hermitian");
  if (rc != OMM_OK) return rc;
  if (!H) return fail(OMM_ERR_ARG, "omm_update_H_hermitian: NULL argument");
  double* He = nullptr;
  try {
    alloc(&He, 4 * (size_t)c->mc * c->mc, c->st);
    embed_matrix(c->st, c->mc, H, c->hz_stage, He);
    c->hermitian = false;  // the real update of the embedded matrix
    rc = omm_update_H(c, He);
    c->hermitian = true;
    mem::release(He, c->st);
  } catch (const std::bad_alloc&) {
    return fail(OMM_ERR_OOM, "omm_update_H_hermitian: device allocation failed");
  } catch (const CudaError& err) {
    cudaStreamSynchronize(c->st);
    mem::release(He, c->st);
    c->hermitian = true;
    return fail(OMM_ERR_CUDA, std::string("omm_update_H_hermitian: ") + err.what + ": " + cudaGetErrorString(err.err));
  }
  return rc;
}

omm_status omm_solve_hermitian(omm_ctx* c, const double* C0, double* C, double* E, double* D, omm_info* info) {
  omm_status rc = check_hermitian(c, "omm_solve_hermitian");
  if (rc != OMM_OK) return rc;
  if (!C0) return fail(OMM_ERR_ARG, "omm_solve_hermitian: NULL argument");
  const int m = c->mc, n = c->nc;
  omm_info inf{};
  double Ee = 0.0;
  double* De = nullptr;
  try {
    embed_start(c, c->st, C0);
    if (D) {
      if (!c->mm) alloc(&c->mm, 4 * (size_t)m * m, c->st);
      De = c->mm;
    }
    c->hermitian = false;
    rc = omm_solve(c, c->hz_rows, c->hz_rows, &Ee, De, &inf);
    c->hermitian = true;
    halve_info(&inf);
    if (rc == OMM_OK || rc == OMM_ERR_NO_CONVERGENCE) {
      if (E) *E = 0.5 * Ee;
      if (C) extract_rows(c->st, n, m, c->hz_rows, c->hz_stage, C);
      if (D && rc == OMM_OK) extract_matrix(c->st, m, De, c->hz_stage, D);
      OMM_CUDA_TRY(cudaStreamSynchronize(c->st));
    }
  } catch (const std::bad_alloc&) {
    c->hermitian = true;
    rc = fail(OMM_ERR_OOM, "omm_solve_hermitian: device allocation failed");
  } catch (const CudaError& err) {
    c->hermitian = true;
    rc = fail(OMM_ERR_CUDA, std::string("omm_solve_hermitian: ") + err.what + ": " + cudaGetErrorString(err.err));
  }
  inf.status = rc;
  if (info) *info = inf;
  return rc;
}

omm_status omm_backward_hermitian(omm_ctx* c, double* dEdH, double* dEdS) {
  omm_status rc = check_hermitian(c, "omm_backward_hermitian");
  if (rc != OMM_OK) return rc;
  const int m = c->mc;
  double* tmp = nullptr;
  try {
    alloc(&tmp, 4 * (size_t)m * m, c->st);
    c->hermitian = false;
    for (int k = 0; k < 2 && rc == OMM_OK; ++k) {
      double* out = k == 0 ? dEdH : dEdS;
      if (!out) continue;
      rc = k == 0 ? omm_backward(c, tmp, nullptr) : omm_backward(c, nullptr, tmp);
      if (rc == OMM_OK) extract_matrix(c->st, m, tmp, c->hz_stage, out);
    }
    c->hermitian = true;
    OMM_CUDA_TRY(cudaStreamSynchronize(c->st));
    mem::release(tmp, c->st);
  } catch (const std::bad_alloc&) {
    c->hermitian = true;
    return fail(OMM_ERR_OOM, "omm_backward_hermitian: device allocation failed");
  } catch (const CudaError& err) {
    c->hermitian = true;
    cudaStreamSynchronize(c->st);
    mem::release(tmp, c->st);
    return fail(OMM_ERR_CUDA, std::string("omm_backward_hermitian: ") + err.what + ": " + cudaGetErrorString(err.err));
  }
  return rc;
}

omm_status omm_create_hermitian_batched(int count, const int* m, const int* n, const double* const* H,
                                        const double* const* S, const double* const* T, const double* eta,
                                        const double* tau, const omm_opts* opts, void* stream, omm_batch** out) {
  if (out) *out = nullptr;
  if (!out || count <= 0 || !m || !n || !H || !S || !eta || !tau)
    return fail(OMM_ERR_ARG, "omm_create_hermitian_batched: invalid argument");
  if (opts && opts->cholesky && opts->precision == OMM_PREC_MIXED)
    return fail(OMM_ERR_ARG, "omm_create_hermitian_batched: the Cholesky flavour of a Hermitian problem needs "
                             "OMM_PREC_FP64");
  for (int i = 0; i < count; ++i)
    if (m[i] <= 0 || n[i] <= 0 || n[i] >= m[i] || !H[i] || !S[i])
      return fail(OMM_ERR_ARG, "omm_create_hermitian_batched: instance " + std::to_string(i) + ": invalid argument");
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<Embedded> e(count);
  std::vector<int> m2(count), n2(count);
  std::vector<const double*> He(count), Se(count), Te(count);
  std::vector<size_t> offset(count + 1, 0);
  for (int i = 0; i < count; ++i) offset[i + 1] = offset[i] + embedded_doubles(m[i], T && T[i]);
  double* block = nullptr;  // every instance's embedded inputs: one allocation, one release
  omm_status rc = OMM_OK;
  auto release = [&]() {
    cudaStreamSynchronize(st);
    mem::release(block, st);
    block = nullptr;
  };
  try {
    alloc(&block, offset[count], st);
    for (int i = 0; i < count; ++i) {
      embed_inputs(st, m[i], H[i], S[i], T ? T[i] : nullptr, block + offset[i], e[i]);
      m2[i] = 2 * m[i];
      n2[i] = 2 * n[i];
      He[i] = e[i].H;
      Se[i] = e[i].S;
      Te[i] = e[i].T;
    }
    OMM_CUDA_TRY(cudaStreamSynchronize(st));
    rc = omm_create_batched(count, m2.data(), n2.data(), He.data(), Se.data(), T ? Te.data() : nullptr, eta, tau,
                            opts, stream, out);
    release();
    if (rc != OMM_OK) return rc;
    for (int i = 0; i < count; ++i) attach(omm_batch_instance(*out, i), m[i], n[i]);
  } catch (const std::bad_alloc&) {
    release();
    if (*out) { omm_free_batched(*out); *out = nullptr; }
    return fail(OMM_ERR_OOM, "omm_create_hermitian_batched: device allocation failed");
  } catch (const CudaError& err) {
    release();
    if (*out) { omm_free_batched(*out); *out = nullptr; }
    return fail(OMM_ERR_CUDA, std::string("omm_create_hermitian_batched: ") + err.what + ": " +
                                  cudaGetErrorString(err.err));
  }
  return OMM_OK;
}

omm_status omm_solve_hermitian_batched(omm_batch* b, const double* const* C0, double* const* C, double* E,
                                       omm_info* info) {
  if (!b || !C0) return fail(OMM_ERR_ARG, "omm_solve_hermitian_batched: NULL argument");
  const int count = batch_count(b);
  std::vector<const double*> C0e(count);
  std::vector<double*> Ce(count);
  std::vector<double> Ee(count, 0.0);
  std::vector<omm_ctx*> ctx(count);
  for (int i = 0; i < count; ++i) {
    ctx[i] = omm_batch_instance(b, i);
    if (!ctx[i] || !ctx[i]->hermitian || !C0[i])
      return fail(OMM_ERR_ARG, "omm_solve_hermitian_batched: not a Hermitian batch, or NULL C0");
  }
  cudaStream_t st = ctx[0]->st;
  omm_status rc = OMM_OK;
  try {
    for (int i = 0; i < count; ++i) {
      embed_start(ctx[i], st, C0[i]);
      C0e[i] = ctx[i]->hz_rows;
      Ce[i] = ctx[i]->hz_rows;
      ctx[i]->hermitian = false;
    }
    rc = omm_solve_batched(b, C0e.data(), Ce.data(), Ee.data(), info);
    for (int i = 0; i < count; ++i) {
      ctx[i]->hermitian = true;
      if (E) E[i] = 0.5 * Ee[i];
      if (info) halve_info(&info[i]);
      const int s = info ? info[i].status : (int)rc;
      if (C && C[i] && (s == OMM_OK || s == OMM_ERR_NO_CONVERGENCE))
        extract_rows(st, ctx[i]->nc, ctx[i]->mc, ctx[i]->hz_rows, ctx[i]->hz_stage, C[i]);
      OMM_CUDA_TRY(cudaStreamSynchronize(st));
    }
  } catch (const CudaError& err) {
    for (omm_ctx* c : ctx) c->hermitian = true;
    return fail(OMM_ERR_CUDA, std::string("omm_solve_hermitian_batched: ") + err.what + ": " +
                                  cudaGetErrorString(err.err));
  }
  return rc;
}

}  // extern "C"
