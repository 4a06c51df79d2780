// Private: the solver context behind the opaque omm_ctx of include/omm.h and the
// per-context operations shared by the single and the batched solve.
#pragma once
#include <string>

#include "../../include/omm.h"
#include "emu.cuh"
#include "omm_internal.cuh"
#include "omm_mixed.cuh"
#include "reduce.cuh"

struct omm_ctx {
  int m = 0, n = 0;
  double eta = 0.0, tau = 0.0;
  omm_opts opts{};
  cudaStream_t st = nullptr;
  bool precond = true;
  bool solved = false;
  double* HS = nullptr;
  double* P = nullptr;
  double* C = nullptr;
  double* Dir = nullptr;
  double* G = nullptr;
  double* Gold = nullptr;
  double* PG = nullptr;
  double* Y4 = nullptr;
  double* SWHW = nullptr;
  double* Proj = nullptr;
  double* nn = nullptr;      // n x n scratch
  double* part = nullptr;    // reduction partials
  double* part2 = nullptr;   // trace partials
  double* mm = nullptr;      // m x m output scratch (lazy)
  omm::Scalars* sc = nullptr;
  omm::Scalars* sc_host = nullptr;  // pinned
  int* info_dev = nullptr;
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
  double ms_setup = 0.0;
  double ms_precond = 0.0;  // the Cholesky inverse inside ms_setup
  omm::MixedState* mixed = nullptr;
  omm::EmuState* emu = nullptr;  // float64-class tensor-core refresh of the mixed path
  omm::Reduction* red = nullptr; // Cholesky reduction to standard form (opts.cholesky)
  // Hermitian problems (omm_create_hermitian): this context solves the real form of the
  // mc x mc complex problem (m = 2 mc, n = 2 nc)
  bool hermitian = false;   // gates the real entry points (lifted while a Hermitian call runs)
  bool real_form = false;   // this context holds a real form (set once, never lifted)
  int mc = 0, nc = 0;
  double* hz_stage = nullptr;  // complex staging, 2 mc^2 doubles
  double* hz_rows = nullptr;   // the real form of C (2 nc x 2 mc)
  omm::Profiler prof;  // main contraction kernel of the iteration (tensor-core or float64 GEMM)
  omm::Profiler prof_sliced;  // the float64-class sliced products (inverse, refreshes, certificate, D)
  double sliced_setup[3] = {0.0, 0.0, 0.0};  // ms, flops, launches of those in omm_create
};

namespace omm {

constexpr int kMixedRound = 400;  // line searches before a stalled mixed round is refreshed

omm_status fail(omm_status s, const std::string& msg);
void copy_in(double* dst, const double* src, size_t count, cudaStream_t st);
bool is_device_ptr(const void* p);
float elapsed(cudaEvent_t a, cudaEvent_t b);
void recompute_state_fp64(omm_ctx* c);    // float64 HC, SC, S_W, H_W, E~, G, max|G|
void reset_loop_flags(omm_ctx* c, bool full);
void read_scalars(omm_ctx* c);
void write_scalars(omm_ctx* c);
void density_into(omm_ctx* c, double* out);
void destroy(omm_ctx* c);
int batch_count(const omm_batch* b);
// real form of a Hermitian problem: C <- the nearest real form of a complex C (each pair of rows
// j, n + j averaged onto [Re c | Im c], [-Im c | Re c]); no-op for other contexts. Called before
// every recompute of the state, so that rounding of the mixed path cannot accumulate along the
// directions that leave the real forms (they are flat: the functional does not see them).
void project_real_form(omm_ctx* c, cudaStream_t st);

}  // namespace omm
