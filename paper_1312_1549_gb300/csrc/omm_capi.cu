// The C ABI of include/omm.h: solver context, setup, the CG loop and outputs.
//
// Data layout in device memory (m basis functions, n Wannier functions,
// all float64, row-major; "_nm" arrays hold one Wannier function per row):
//   HS    2m x m   [H~ ; S]        H~ = H - eta S (Sec. 2.2, Eq. 9)
//   P     m x m    (S + T/tau)^-1  (Sec. 2.4, Eq. 17)
//   C, Dir, G, Gold, PG   n x m
//   Y4    4n x m   [HC ; SC ; HD ; SD]   (the reused products of the Sec. 2.3 footnote)
//   SWHW  n x 2n   [S_W | H_W]
//   Proj  n x 4n   [H' | S' | H'' | S'']  (Eqs. 14-15)
// With this layout every contraction of a line search is one GEMM:
//   HD,SD = Dir [H~;S]^T, Proj = Dir Y4^T, G = 8 HC - 4 SWHW [HC;SC], PG = G P.
#include "../../include/omm.h"
#include "omm_internal.cuh"
#include "omm_ctx.cuh"

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <new>
#include <string>

namespace omm {
namespace {
thread_local std::string g_last_error;
}
void set_last_error(const std::string& msg) { g_last_error = msg; }
const char* last_error_cstr() { return g_last_error.c_str(); }

std::atomic<unsigned long long> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

void Profiler::begin(cudaStream_t st) {
  if (!on) return;
  if (used_ == cap_) {
    const int ncap = cap_ ? 2 * cap_ : 64;
    Pair* np = new Pair[ncap];
    for (int i = 0; i < cap_; ++i) np[i] = pairs_[i];
    for (int i = cap_; i < ncap; ++i) {
      cudaEventCreate(&np[i].a);
      cudaEventCreate(&np[i].b);
    }
    delete[] pairs_;
    pairs_ = np;
    cap_ = ncap;
  }
  cudaEventRecord(pairs_[used_].a, st);
}
void Profiler::end(cudaStream_t st, double f, int tag) {
  if (!on) return;
  cudaEventRecord(pairs_[used_].b, st);
  pairs_[used_].flop = f;
  pairs_[used_].tag = tag;
  ++used_;
}
void Profiler::collect(long keep) {
  for (int i = 0; i < used_; ++i) {
    if (keep >= 0 && i >= keep) break;
    float t = 0.f;
    if (cudaEventElapsedTime(&t, pairs_[i].a, pairs_[i].b) != cudaSuccess) t = 0.f;
    ms += t;
    flop += pairs_[i].flop;
    ++launches;
    const int g = pairs_[i].tag;
    if (g >= 0 && g < kTags) {
      ms_tag[g] += t;
      flop_tag[g] += pairs_[i].flop;
    }
  }
  cudaGetLastError();
  used_ = 0;
}
Profiler::~Profiler() {
  for (int i = 0; i < cap_; ++i) {
    cudaEventDestroy(pairs_[i].a);
    cudaEventDestroy(pairs_[i].b);
  }
  delete[] pairs_;
}
}  // namespace omm

using namespace omm;


namespace omm {

constexpr int kMixedRoundCap = 400;
constexpr int kEmuSlices = 10;  // fixed-point slices of the float64-class refresh (about 50 bits)
// products of the mixed path's preconditioner inverse: 1 = the 3-term bf16 split form (about 2^-16
// of each product; 2..10 would be fixed-point slices). P reaches the line searches only through its
// bf16 rounding (the single-pass P G of the search direction), and the minimum does not depend on P
constexpr int kPrecondSlices = 1;
// Below these sizes the native float64 routines are cheaper than the sliced tensor-core ones,
// whose many small launches are latency-bound there: the inverse (or factor) of an m x m matrix
// with m < kSlicedInverseMin, and the state recompute (refresh, certificate, D) of a problem with
// fewer than kSlicedStateMinFlop flops per recompute (4 m^2 n + 8 m n^2).
constexpr int kSlicedInverseMin = 2048;
constexpr double kSlicedStateMinFlop = 5e8;

omm_status fail(omm_status s, const std::string& msg) {
  set_last_error(msg);
  return s;
}

// every buffer of a context comes from the library's stream-ordered pool (see mem.cu)
template <typename T>
void dev_alloc(T** p, size_t count, cudaStream_t st) {
  mem::alloc(p, count, st);
}

void dev_free(void* p, cudaStream_t st) { mem::release(p, st); }

template <typename T>
void tmp_alloc(T** p, size_t count, cudaStream_t st) {
  mem::alloc(p, count, st);
}

void tmp_free(void* p, cudaStream_t st) { mem::release(p, st); }

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

void copy_in(double* dst, const double* src, size_t count, cudaStream_t st) {
  OMM_CUDA_TRY(cudaMemcpyAsync(dst, src, count * sizeof(double), cudaMemcpyDefault, st));
}

float elapsed(cudaEvent_t a, cudaEvent_t b) {
  float ms = 0.f;
  if (cudaEventElapsedTime(&ms, a, b) != cudaSuccess) {
    cudaGetLastError();  // a failed timing query must not surface as a later launch error
    ms = 0.f;
  }
  return ms;
}

// HC, SC = C [H~;S]^T; S_W, H_W; E~; G = 8 HC - 4 [S_W|H_W][HC;SC]  (all float64)
void recompute_state_fp64(omm_ctx* c) {
  const int m = c->m, n = c->n;
  const long nm = (long)n * m, mm = (long)m * m;
  dgemm(c->st, 0, 1, n, m, m, 1.0, c->C, m, 0, c->HS, m, mm, 0.0, c->Y4, m, nm, 2);
  dgemm(c->st, 0, 1, n, n, m, 1.0, c->C, m, 0, c->Y4 + nm, m, 0, 0.0, c->SWHW, 2L * n, 0);
  dgemm(c->st, 0, 1, n, n, m, 1.0, c->C, m, 0, c->Y4, m, 0, 0.0, c->SWHW + n, 2L * n, 0);
  launch_functional(c->st, n, c->SWHW, c->part2);
  launch_finish_functional(c->st, c->sc, c->part2, traces_blocks(n));
  launch_scale_copy(c->st, nm, c->Y4, 8.0, c->G, nullptr);
  dgemm(c->st, 0, 0, n, m, 2 * n, -4.0, c->SWHW, 2L * n, 0, c->Y4, m, 0, 1.0, c->G, m, 0);
  launch_gmax(c->st, nm, c->G, c->part);
  launch_finish_gmax(c->st, c->sc, c->part);
}

// One line search with float64 contractions (Sec. 2.3).
void iterate_fp64(omm_ctx* c) {
  const int m = c->m, n = c->n;
  const long nm = (long)n * m, mm = (long)m * m;
  const int* skip = &c->sc->done;
  Profiler& pf = c->prof;
  const double fPG = 2.0 * n * (double)m * m, fHD = 4.0 * n * (double)m * m;
  const double fPr = 8.0 * n * (double)n * m, fG = 4.0 * n * (double)n * m;
  if (c->precond) {
    pf.begin(c->st);
    dgemm(c->st, 0, 1, n, m, m, 1.0, c->G, m, 0, c->P, m, 0, 0.0, c->PG, m, 0, 1, 0, skip);
    pf.end(c->st, fPG);
  } else
    launch_scale_copy(c->st, nm, c->G, 1.0, c->PG, c->sc);
  launch_grad_reduce(c->st, nm, c->G, c->PG, c->Gold, c->Dir, c->part, c->sc);
  launch_control_direction(c->st, c->sc, c->part, 0, kReduceBlocks);
  launch_direction(c->st, nm, c->PG, c->Dir, c->sc);
  pf.begin(c->st);
  dgemm(c->st, 0, 1, n, m, m, 1.0, c->Dir, m, 0, c->HS, m, mm, 0.0, c->Y4 + 2 * nm, m, nm, 2, 0, skip);
  pf.end(c->st, fHD);
  pf.begin(c->st);
  dgemm(c->st, 0, 1, n, 4 * n, m, 1.0, c->Dir, m, 0, c->Y4, m, 0, 0.0, c->Proj, 4L * n, 0, 1, 0, skip);
  pf.end(c->st, fPr);
  launch_traces(c->st, n, c->SWHW, c->Proj, c->part2, c->sc);
  launch_control_linesearch(c->st, c->sc, c->part2, traces_partials(n));
  launch_update_state(c->st, n, m, c->C, c->Y4, c->Dir, c->G, c->Gold, c->sc);
  launch_update_subspace(c->st, n, c->SWHW, c->Proj, c->sc);
  pf.begin(c->st);
  dgemm(c->st, 0, 0, n, m, 2 * n, -4.0, c->SWHW, 2L * n, 0, c->Y4, m, 0, 1.0, c->G, m, 0, 1, 0, skip);
  pf.end(c->st, fG);
}

void read_scalars(omm_ctx* c) {
  OMM_CUDA_TRY(cudaMemcpyAsync(c->sc_host, c->sc, sizeof(Scalars), cudaMemcpyDeviceToHost, c->st));
  OMM_CUDA_TRY(cudaStreamSynchronize(c->st));
}

void reset_loop_flags(omm_ctx* c, bool full) {
  Scalars& h = *c->sc_host;
  if (full) {
    std::memset(&h, 0, sizeof(Scalars));
  }
  h.done = 0;
  h.halt = 0;
  h.status = 0;
  h.have_dir = 0;
  h.restart = 1;
  h.stop_pending = 0;
  h.stop_reason = 0;
  h.iter_round = 0;
  h.mixed = c->mixed != nullptr;
  h.best_g = 1e300;
  h.best_it = 0;
  h.stall_window = 40;
  h.max_iter = c->opts.max_iter;
  h.tol_grad = c->opts.tol_grad;
  h.e_tol = c->opts.e_tol;
}

void write_scalars(omm_ctx* c) {
  OMM_CUDA_TRY(cudaMemcpyAsync(c->sc, c->sc_host, sizeof(Scalars), cudaMemcpyHostToDevice, c->st));
}

// D = 2 C^T (2I - S_W) C  (n x m layout) into out (m x m, device)
void density_into(omm_ctx* c, double* out) {
  const int m = c->m, n = c->n;
  launch_two_i_minus(c->st, n, c->SWHW, 2L * n, c->nn);
  dgemm(c->st, 0, 0, n, m, n, 1.0, c->nn, n, 0, c->C, m, 0, 0.0, c->PG, m, 0);
  dgemm(c->st, 1, 0, m, m, n, 2.0, c->C, m, 0, c->PG, m, 0, 0.0, out, m, 0, 1, kTriLower);
  launch_symmetrize_lower(c->st, m, out);
}

// out = -(2 C^T H~_W C + eta D), with D already in out
void minus_edm_into(omm_ctx* c, double* out) {
  const int m = c->m, n = c->n;
  dgemm(c->st, 0, 0, n, m, n, 1.0, c->SWHW + n, 2L * n, 0, c->C, m, 0, 0.0, c->PG, m, 0);
  dgemm(c->st, 1, 0, m, m, n, -2.0, c->C, m, 0, c->PG, m, 0, -c->eta, out, m, 0, 1, kTriLower);
  launch_symmetrize_lower(c->st, m, out);
}

void ensure_mm(omm_ctx* c) {
  if (!c->mm) dev_alloc(&c->mm, (size_t)c->m * c->m, c->st);
}

void destroy(omm_ctx* c) {
  if (!c) return;
  if (c->st) cudaStreamSynchronize(c->st);
  dev_free(c->HS, c->st);
  dev_free(c->P, c->st);
  dev_free(c->C, c->st);
  dev_free(c->Dir, c->st);
  dev_free(c->G, c->st);
  dev_free(c->Gold, c->st);
  dev_free(c->PG, c->st);
  dev_free(c->Y4, c->st);
  dev_free(c->SWHW, c->st);
  dev_free(c->Proj, c->st);
  dev_free(c->nn, c->st);
  dev_free(c->part, c->st);
  dev_free(c->part2, c->st);
  dev_free(c->mm, c->st);
  dev_free(c->sc, c->st);
  dev_free(c->info_dev, c->st);
  dev_free(c->hz_stage, c->st);
  dev_free(c->hz_rows, c->st);
  if (c->sc_host) cudaFreeHost(c->sc_host);
  for (auto& e : c->ev)
    if (e) cudaEventDestroy(e);
  if (c->mixed) mixed_destroy(c->mixed, c->st);
  if (c->emu) emu_destroy(c->emu, c->st);
  if (c->red) reduction_destroy(c->red, c->st);
  delete c;
}

}  // namespace omm

extern "C" {

const char* omm_status_str(omm_status s) {
  switch (s) {
    case OMM_OK: return "ok";
    case OMM_ERR_ARG: return "invalid argument";
    case OMM_ERR_NOT_SPD: return "matrix is not positive definite";
    case OMM_ERR_UNBOUNDED: return "functional unbounded along the search line (eta too high?)";
    case OMM_ERR_NO_CONVERGENCE: return "no convergence within max_iter";
    case OMM_ERR_NONFINITE: return "non-finite value";
    case OMM_ERR_TIMEOUT: return "device wait timed out";
    case OMM_ERR_CUDA: return "CUDA error";
    case OMM_ERR_OOM: return "out of device memory";
    case OMM_ERR_STATE: return "call out of order";
  }
  return "unknown status";
}

const char* omm_last_error(void) { return last_error_cstr(); }

unsigned long long omm_launch_count(void) { return g_launches.load(); }

omm_status omm_create(int m, int n, const double* H, const double* S, const double* T, double eta,
                      double tau, const omm_opts* opts, void* stream, omm_ctx** out) {
  if (out) *out = nullptr;
  if (!out || !H || !S) return fail(OMM_ERR_ARG, "omm_create: NULL argument");
  if (m <= 0 || n <= 0 || n >= m) return fail(OMM_ERR_ARG, "omm_create: need 0 < n < m");
  omm_opts o{};
  if (opts) o = *opts;
  if (o.max_iter <= 0) o.max_iter = 10000;
  if (o.check_every <= 0) o.check_every = 8;
  if (!(o.tol_grad > 0.0)) o.tol_grad = 1e-9;
  if (!(o.e_tol >= 0.0)) o.e_tol = 0.0;
  if (!(o.refine_ratio > 0.0)) o.refine_ratio = 1e-3;
  if (o.precond_slices <= 0) o.precond_slices = kPrecondSlices;
  if (o.precond_slices < 1 || o.precond_slices > 10)
    return fail(OMM_ERR_ARG, "omm_create: precond_slices must be in 1..10");
  if (o.precision != OMM_PREC_FP64 && o.precision != OMM_PREC_MIXED)
    return fail(OMM_ERR_ARG, "omm_create: unknown precision");
  const bool chol = o.cholesky != 0;
  const bool precond = !chol && o.no_precondition == 0;
  if (precond && !(tau > 0.0)) return fail(OMM_ERR_ARG, "omm_create: tau must be > 0");
  if (precond && !T && std::isfinite(tau)) return fail(OMM_ERR_ARG, "omm_create: T is NULL");
  if (!std::isfinite(eta)) return fail(OMM_ERR_ARG, "omm_create: eta is not finite");

  omm_ctx* c = new (std::nothrow) omm_ctx();
  if (!c) return fail(OMM_ERR_OOM, "omm_create: host allocation");
  c->m = m;
  c->n = n;
  c->eta = eta;
  c->tau = tau;
  c->opts = o;
  c->st = (cudaStream_t)stream;
  c->precond = precond;
  double* A = nullptr;
  double* work = nullptr;
  int* inv_err = nullptr;
  try {
    const long mm = (long)m * m, nm = (long)n * m;
    for (auto& e : c->ev) OMM_CUDA_TRY(cudaEventCreate(&e));
    c->prof_sliced.on = o.profile != 0;
    if (c->prof_sliced.on) emu::set_profiler(&c->prof_sliced);
    OMM_CUDA_TRY(cudaMallocHost((void**)&c->sc_host, sizeof(Scalars)));
    dev_alloc(&c->sc, 1, c->st);
    dev_alloc(&c->info_dev, 1, c->st);
    dev_alloc(&c->HS, 2 * mm, c->st);
    OMM_CUDA_TRY(cudaEventRecord(c->ev[0], c->st));
    copy_in(c->HS, H, mm, c->st);
    copy_in(c->HS + mm, S, mm, c->st);
    // the mixed path factors large matrices with sliced tensor-core products (preconditioner grade
    // for P, float64-class for the Cholesky flavour's factor), small ones and the float64 path natively
    const bool sliced_inverse = o.precision == OMM_PREC_MIXED && m >= kSlicedInverseMin;
    if (chol) {
      // standard form (Sec. 2.4): H_r = L^-1 H L^-T in the H slot, the identity in the S slot
      tmp_alloc(&A, mm, c->st);
      copy_in(A, S, mm, c->st);
      OMM_CUDA_TRY(cudaEventRecord(c->ev[2], c->st));
      c->red = reduction_create(c->st, m, sliced_inverse, A, c->info_dev);
      reduce_hamiltonian(c->red, c->st, c->HS);
      OMM_CUDA_TRY(cudaEventRecord(c->ev[3], c->st));
      launch_identity(c->st, m, c->HS + mm);
    }
    launch_axpby_shift(c->st, mm, c->HS, c->HS + mm, eta, c->HS);
    if (precond) {
      dev_alloc(&c->P, mm, c->st);
      tmp_alloc(&A, mm, c->st);
      if (sliced_inverse) {
        tmp_alloc(&work, (spd_inverse_sliced_workspace_bytes(m) + sizeof(double) - 1) / sizeof(double), c->st);
        tmp_alloc(&inv_err, 1, c->st);
        OMM_CUDA_TRY(cudaMemsetAsync(inv_err, 0, sizeof(int), c->st));
      } else {
        tmp_alloc(&work, spd_inverse_workspace(m), c->st);
      }
      if (std::isfinite(tau)) {
        copy_in(A, T, mm, c->st);
        launch_add_scaled(c->st, mm, c->HS + mm, A, 1.0 / tau, A);
      } else {
        OMM_CUDA_TRY(cudaMemcpyAsync(A, c->HS + mm, mm * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
      }
      OMM_CUDA_TRY(cudaEventRecord(c->ev[2], c->st));
      if (sliced_inverse) spd_inverse_sliced(c->st, m, A, c->P, work, c->info_dev, inv_err, o.precond_slices);
      else spd_inverse(c->st, m, A, c->P, work, c->info_dev);
      OMM_CUDA_TRY(cudaEventRecord(c->ev[3], c->st));
    }
    dev_alloc(&c->C, nm, c->st);
    dev_alloc(&c->Dir, nm, c->st);
    dev_alloc(&c->G, nm, c->st);
    dev_alloc(&c->Gold, nm, c->st);
    dev_alloc(&c->PG, nm, c->st);
    dev_alloc(&c->Y4, 4 * nm, c->st);
    dev_alloc(&c->SWHW, 2L * n * n, c->st);
    dev_alloc(&c->Proj, 4L * n * n, c->st);
    dev_alloc(&c->nn, (size_t)n * n, c->st);
    dev_alloc(&c->part, (size_t)kReduceBlocks * 4, c->st);
    dev_alloc(&c->part2, (size_t)traces_blocks(n) * kNumTraces, c->st);
    if (o.precision == OMM_PREC_MIXED) {
      c->mixed = mixed_create(c->st, m, n, c->HS, c->P);
      if (o.debug_expire_wait) mixed_set_expire(c->mixed, 1);
      if (4.0 * m * (double)m * n + 8.0 * m * (double)n * n >= kSlicedStateMinFlop)
        c->emu = emu_create(c->st, m, n, kEmuSlices, c->HS);
    }
    OMM_CUDA_TRY(cudaEventRecord(c->ev[1], c->st));
    int info = 0, ierr = 0;
    OMM_CUDA_TRY(cudaMemcpyAsync(&info, c->info_dev, sizeof(int), cudaMemcpyDeviceToHost, c->st));
    if (inv_err) OMM_CUDA_TRY(cudaMemcpyAsync(&ierr, inv_err, sizeof(int), cudaMemcpyDeviceToHost, c->st));
    OMM_CUDA_TRY(cudaStreamSynchronize(c->st));
    c->ms_setup = elapsed(c->ev[0], c->ev[1]);
    if (c->prof_sliced.on) {
      emu::set_profiler(nullptr);
      c->prof_sliced.collect();
      c->sliced_setup[0] = c->prof_sliced.ms;
      c->sliced_setup[1] = c->prof_sliced.flop;
      c->sliced_setup[2] = (double)c->prof_sliced.launches;
      c->prof_sliced.reset();
    }
    c->ms_precond = (precond || chol) ? elapsed(c->ev[2], c->ev[3]) : 0.0;
    if (c->red && reduction_error(c->red, c->st) != 0) ierr = 1;
    tmp_free(A, c->st);
    tmp_free(work, c->st);
    tmp_free(inv_err, c->st);
    A = work = nullptr;
    inv_err = nullptr;
    if (ierr != 0) {
      destroy(c);
      return fail(OMM_ERR_TIMEOUT, "omm_create: a bounded device wait expired in the preconditioner inverse");
    }
    if (info != 0) {
      destroy(c);
      return fail(OMM_ERR_NOT_SPD, std::string("omm_create: ") + (chol ? "S" : "S + T/tau") +
                                       " is not positive definite (pivot " + std::to_string(info) + ")");
    }
  } catch (const std::bad_alloc&) {
    emu::set_profiler(nullptr);
    tmp_free(A, c->st);
    tmp_free(work, c->st);
    tmp_free(inv_err, c->st);
    destroy(c);
    return fail(OMM_ERR_OOM, "omm_create: device allocation failed");
  } catch (const CudaError& e) {
    emu::set_profiler(nullptr);
    tmp_free(A, c->st);
    tmp_free(work, c->st);
    tmp_free(inv_err, c->st);
    destroy(c);
    return fail(OMM_ERR_CUDA, std::string("omm_create: ") + e.what + ": " + cudaGetErrorString(e.err));
  }
  *out = c;
  return OMM_OK;
}

omm_status omm_update_H(omm_ctx* c, const double* H) {
  if (!c || !H) return fail(OMM_ERR_ARG, "omm_update_H: NULL argument");
  if (c->hermitian) return fail(OMM_ERR_ARG, "omm_update_H: Hermitian context (use omm_update_H_hermitian)");
  try {
    const long mm = (long)c->m * c->m;
    copy_in(c->HS, H, mm, c->st);
    if (c->red) reduce_hamiltonian(c->red, c->st, c->HS);  // the S slot holds the identity
    launch_axpby_shift(c->st, mm, c->HS, c->HS + mm, c->eta, c->HS);
    if (c->mixed) mixed_update_H(c->mixed, c->st, c->HS);
    if (c->emu) emu_update_H(c->emu, c->st, c->HS);
    OMM_CUDA_TRY(cudaStreamSynchronize(c->st));
    c->solved = false;
    if (c->red && reduction_error(c->red, c->st) != 0)
      return fail(OMM_ERR_TIMEOUT, "omm_update_H: a bounded device wait expired in the reduction");
  } catch (const CudaError& e) {
    return fail(OMM_ERR_CUDA, std::string("omm_update_H: ") + e.what + ": " + cudaGetErrorString(e.err));
  }
  return OMM_OK;
}

omm_status omm_solve(omm_ctx* c, const double* C0, double* Cout, double* E, double* D, omm_info* info) {
  if (!c || !C0) return fail(OMM_ERR_ARG, "omm_solve: NULL argument");
  if (c->hermitian) return fail(OMM_ERR_ARG, "omm_solve: Hermitian context (use omm_solve_hermitian)");
  omm_info inf{};
  omm_status result = OMM_OK;
  const int m = c->m, n = c->n;
  const long nm = (long)n * m;
  c->solved = false;
  try {
    const unsigned long long launches0 = g_launches.load();
    c->prof.on = c->opts.profile != 0;
    c->prof.reset();
    c->prof_sliced.reset();
    if (c->prof_sliced.on) emu::set_profiler(&c->prof_sliced);
    copy_in(c->C, C0, nm, c->st);
    double ms_transform = 0.0;
    if (c->red) {  // C_r = L^T C0 (Sec. 2.4)
      OMM_CUDA_TRY(cudaEventRecord(c->ev[0], c->st));
      reduce_coefficients(c->red, c->st, n, c->C, c->Dir);
      OMM_CUDA_TRY(cudaMemcpyAsync(c->C, c->Dir, nm * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
      OMM_CUDA_TRY(cudaEventRecord(c->ev[1], c->st));
      OMM_CUDA_TRY(cudaEventSynchronize(c->ev[1]));
      ms_transform += elapsed(c->ev[0], c->ev[1]);
    }
    reset_loop_flags(c, true);
    write_scalars(c);
    const bool mixed = c->mixed != nullptr;
    if (mixed) mixed_reset_error(c->mixed, c->st);  // a context stays usable after a timed-out solve
    double flop = 0.0, flop_tc = 0.0;
    const double per_it = 6.0 * m * (double)m * n + (c->mixed ? 16.0 : 12.0) * (double)m * n * n;
    const double per_state = 4.0 * m * (double)m * n + 8.0 * (double)m * n * n;
    double ms_iter = 0.0, ms_ref = 0.0, ms_cert = 0.0;
    int fp64_iters = 0, refinements = 0;
    int iter_total = 0;
    double g_ref = -1.0;  // max|G| at the last float64 recompute
    bool energy_stop = false;
    bool last_round_done = false;  // the last mixed round ended on the device's convergence test
    // Outer loop: float64 recompute of the state (refinement / certificate),
    // then line searches until converged, halted or capped.
    for (int round = 0;; ++round) {
      // mixed path: a tensor-core first state, then float64-class states (sliced products, or
      // native float64 for small problems) for the refreshes the device asks for and for the
      // certificate once it reports convergence (native float64 with native_certificate = 1)
      const bool emu_certify = mixed && c->emu && c->opts.native_certificate == 0;
      const bool tc_state = mixed && round == 0;
      const bool emu_state = mixed && c->emu && round > 0 && (!last_round_done || emu_certify);
      OMM_CUDA_TRY(cudaEventRecord(c->ev[0], c->st));
      if (tc_state) {
        mixed_recompute_state(c->mixed, c->st, c->sc, c->C, c->Y4, c->SWHW, c->G, c->part, c->part2);
        flop_tc += 3.0 * per_state;
      } else if (emu_state) {
        project_real_form(c, c->st);
        emu_recompute_state(c->emu, c->st, c->sc, c->C, c->Y4, c->SWHW, c->G, c->part, c->part2);
        flop_tc += 0.5 * kEmuSlices * (kEmuSlices + 1) * per_state;
        if (emu_error(c->emu, c->st) != 0) {
          result = OMM_ERR_TIMEOUT;
          break;
        }
      } else {
        project_real_form(c, c->st);
        recompute_state_fp64(c);
      }
      flop += per_state;
      OMM_CUDA_TRY(cudaEventRecord(c->ev[1], c->st));
      read_scalars(c);
      if (tc_state) ms_iter += elapsed(c->ev[0], c->ev[1]);
      else ms_ref += elapsed(c->ev[0], c->ev[1]);
      if (!tc_state && !emu_state) ms_cert += elapsed(c->ev[0], c->ev[1]);
      Scalars& h = *c->sc_host;
      if (!std::isfinite(h.gmax) || !std::isfinite(h.E)) {
        result = OMM_ERR_NONFINITE;
        break;
      }
      // only a float64-class state taken for the certificate (or any native float64 state) certifies
      if (!tc_state && (!emu_state || emu_certify) && (h.gmax < c->opts.tol_grad || energy_stop)) break;
      if (round > 0) ++refinements;
      if (iter_total >= c->opts.max_iter) {
        result = OMM_ERR_NO_CONVERGENCE;
        break;
      }
      if (round > 64) {
        result = OMM_ERR_NO_CONVERGENCE;
        break;
      }
      g_ref = h.gmax;
      const double E_keep = h.E, g_keep = h.gmax;
      reset_loop_flags(c, false);
      h.E = E_keep;
      h.gmax = g_keep;
      h.iter = iter_total;
      h.halt_gmax = mixed ? std::max(c->opts.tol_grad * 0.5, g_ref * c->opts.refine_ratio) : 0.0;
      write_scalars(c);
      if (mixed) mixed_sync_state(c->mixed, c->st, c->Y4, c->SWHW, c->G);
      OMM_CUDA_TRY(cudaEventRecord(c->ev[2], c->st));
      int prev_iter = iter_total;
      for (;;) {
        const int it_batch = h.iter;
        for (int k = 0; k < c->opts.check_every; ++k) {
          if (mixed) mixed_iterate_replay(c->mixed, c->st, c->sc, c->C, c->Dir, c->G, c->Gold, c->PG,
                                   c->Y4, c->SWHW, c->Proj, c->part, c->part2, c->HS, c->P,
                                   c->precond, c->prof);
          else iterate_fp64(c);
        }
        read_scalars(c);
        // the GEMMs of the line searches that ran: every completed one, and the P G product of the
        // line search whose direction step stopped the round; the rest skipped on the stop flags
        const long per_iter = c->precond ? 4 : 3;
        c->prof.collect(per_iter * (h.iter - it_batch) + ((h.done || h.halt) && c->precond ? 1 : 0));
        if (h.done || h.halt) break;
        if (mixed && mixed_error(c->mixed, c->st) != 0) break;  // a bounded wait expired: stop at once
        // a mixed round that stalls above its refinement threshold is refreshed in float64
        if (mixed && h.iter - prev_iter >= kMixedRoundCap) break;
      }
      if (mixed && mixed_error(c->mixed, c->st) != 0) {
        result = OMM_ERR_TIMEOUT;
        break;
      }
      OMM_CUDA_TRY(cudaEventRecord(c->ev[3], c->st));
      OMM_CUDA_TRY(cudaEventSynchronize(c->ev[3]));
      ms_iter += elapsed(c->ev[2], c->ev[3]);
      const int did = h.iter - prev_iter;
      iter_total = h.iter;
      if (mixed) flop_tc += 3.0 * per_it * did; else { flop += per_it * did; fp64_iters += did; }
      if (mixed) flop += per_it * did;
      if (h.status != 0) {
        result = (omm_status)h.status;
        if (result != OMM_ERR_NO_CONVERGENCE) break;
        // iteration cap: certify what we have, report no convergence
        project_real_form(c, c->st);
        recompute_state_fp64(c);
        read_scalars(c);
        break;
      }
      // done (device-side convergence) or a refinement request: recompute and test
      if (h.done && h.stop_reason == 2) energy_stop = true;
      last_round_done = h.done != 0;
    }
    Scalars& h = *c->sc_host;
    inf.iterations = iter_total;
    inf.iterations_fp64 = fp64_iters;
    inf.refinements = refinements;
    inf.Etilde = h.E;
    inf.E = h.E + 2.0 * n * c->eta;
    inf.gmax = h.gmax;
    inf.ms_setup = c->ms_setup;
    inf.ms_precond = c->ms_precond;
    if (c->mixed) mixed_tuning(c->mixed, inf.tile_width, &inf.ms_autotune);
    inf.ms_iterate = ms_iter;
    inf.ms_refine = ms_ref;
    inf.ms_certify = ms_cert;
    if (c->red && (result == OMM_OK || result == OMM_ERR_NO_CONVERGENCE)) {
      // back to the original basis: C = L^-T C_r; S_W, H_W and E are the same in both bases
      OMM_CUDA_TRY(cudaEventRecord(c->ev[0], c->st));
      restore_coefficients(c->red, c->st, n, c->C, c->Dir);
      OMM_CUDA_TRY(cudaMemcpyAsync(c->C, c->Dir, nm * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
      OMM_CUDA_TRY(cudaEventRecord(c->ev[1], c->st));
      OMM_CUDA_TRY(cudaEventSynchronize(c->ev[1]));
      ms_transform += elapsed(c->ev[0], c->ev[1]);
      if (reduction_error(c->red, c->st) != 0) result = OMM_ERR_TIMEOUT;
      flop += 2.0 * n * (double)m * m;  // two triangular n x m x m products
    }
    inf.ms_transform = ms_transform;
    if (result == OMM_OK || result == OMM_ERR_NO_CONVERGENCE) {
      if (Cout) OMM_CUDA_TRY(cudaMemcpyAsync(Cout, c->C, nm * sizeof(double), cudaMemcpyDefault, c->st));
      if (E) *E = inf.E;
    }
    if (result == OMM_OK) {
      c->solved = true;
      if (D) {
        OMM_CUDA_TRY(cudaEventRecord(c->ev[0], c->st));
        double* tgt = D;
        if (!is_device_ptr(D)) {
          ensure_mm(c);
          tgt = c->mm;
        }
        if (c->emu && !c->opts.native_certificate) emu_density(c->emu, c->st, c->C, c->SWHW, tgt);
        else density_into(c, tgt);
        if (tgt != D)
          OMM_CUDA_TRY(cudaMemcpyAsync(D, tgt, (size_t)m * m * sizeof(double), cudaMemcpyDefault, c->st));
        flop += 2.0 * n * (double)n * m + 2.0 * m * (double)m * n;
        OMM_CUDA_TRY(cudaEventRecord(c->ev[1], c->st));
        OMM_CUDA_TRY(cudaEventSynchronize(c->ev[1]));
        inf.ms_outputs = elapsed(c->ev[0], c->ev[1]);
      }
    }
    OMM_CUDA_TRY(cudaStreamSynchronize(c->st));
    inf.gemm_flop = flop;
    inf.gemm_flop_tc = flop_tc;
    inf.kernel_launches = (double)(g_launches.load() - launches0);
    inf.ms_main_gemm = c->prof.ms;
    inf.main_gemm_launches = (double)c->prof.launches;
    inf.main_gemm_flop = c->prof.flop;
    for (int t = 0; t < 4; ++t) {
      inf.ms_gemm_plan[t] = c->prof.ms_tag[t];
      inf.flop_gemm_plan[t] = c->prof.flop_tag[t];
    }
    if (c->prof_sliced.on) {
      c->prof_sliced.collect();
      inf.ms_sliced_gemm = c->sliced_setup[0] + c->prof_sliced.ms;
      inf.sliced_gemm_flop = c->sliced_setup[1] + c->prof_sliced.flop;
      inf.sliced_gemm_launches = c->sliced_setup[2] + (double)c->prof_sliced.launches;
    }
  } catch (const std::bad_alloc&) {
    result = OMM_ERR_OOM;
    set_last_error("omm_solve: device allocation failed");
  } catch (const CudaError& e) {
    result = OMM_ERR_CUDA;
    set_last_error(std::string("omm_solve: ") + e.what + ": " + cudaGetErrorString(e.err));
  }
  emu::set_profiler(nullptr);
  inf.status = result;
  if (info) *info = inf;
  if (result != OMM_OK && result != OMM_ERR_CUDA && result != OMM_ERR_OOM)
    set_last_error(std::string("omm_solve: ") + omm_status_str(result));
  return result;
}

omm_status omm_backward(omm_ctx* c, double* dEdH, double* dEdS) {
  if (!c) return fail(OMM_ERR_ARG, "omm_backward: NULL context");
  if (c->hermitian) return fail(OMM_ERR_ARG, "omm_backward: Hermitian context (use omm_backward_hermitian)");
  if (!c->solved) return fail(OMM_ERR_STATE, "omm_backward: no converged solve");
  try {
    const size_t bytes = (size_t)c->m * c->m * sizeof(double);
    double* tH = dEdH;
    double* tS = dEdS;
    if (dEdH && !is_device_ptr(dEdH)) { ensure_mm(c); tH = c->mm; }
    if (dEdH) {
      // the same density matrix omm_solve returns
      if (c->emu && !c->opts.native_certificate) emu_density(c->emu, c->st, c->C, c->SWHW, tH);
      else density_into(c, tH);
      if (tH != dEdH) OMM_CUDA_TRY(cudaMemcpyAsync(dEdH, tH, bytes, cudaMemcpyDefault, c->st));
    }
    if (dEdS) {
      if (!is_device_ptr(dEdS)) { ensure_mm(c); tS = c->mm; }
      if (c->emu && !c->opts.native_certificate) {  // float64-class, like the certificate
        emu_density(c->emu, c->st, c->C, c->SWHW, tS);
        emu_minus_edm(c->emu, c->st, c->SWHW, c->eta, tS);
      } else {
        density_into(c, tS);
        minus_edm_into(c, tS);
      }
      if (tS != dEdS) OMM_CUDA_TRY(cudaMemcpyAsync(dEdS, tS, bytes, cudaMemcpyDefault, c->st));
    }
    OMM_CUDA_TRY(cudaStreamSynchronize(c->st));
  } catch (const std::bad_alloc&) {
    return fail(OMM_ERR_OOM, "omm_backward: device allocation failed");
  } catch (const CudaError& e) {
    return fail(OMM_ERR_CUDA, std::string("omm_backward: ") + e.what + ": " + cudaGetErrorString(e.err));
  }
  return OMM_OK;
}

void omm_free(omm_ctx* c) { destroy(c); }

}  // extern "C"
