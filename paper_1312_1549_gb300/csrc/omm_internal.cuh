// Internal declarations shared by the translation units of the OMM library.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cstdint>
#include <cstdio>
#include <string>

namespace omm {

// Device-resident control block of one solve. Every iteration kernel reads
// the flags first and returns at once when `done` or `halt` is set, so a
// batch of line searches enqueued ahead of a host poll (or replayed from a
// CUDA graph) turns into no-ops after convergence.
struct Scalars {
  int done;          // converged: remaining iteration kernels are no-ops
  int halt;          // stop for the host (error, iteration cap, refinement request)
  int status;        // omm_status set by the device (0 = ok)
  int iter;          // line searches completed
  int have_dir;      // a previous search direction exists
  int restart;       // next direction is the preconditioned steepest descent
  int restart_dir;   // the current direction is -PG (beta = 0)
  int stop_pending;  // Eq. 18 met at the last line search: stop at the next check
  int max_iter;
  int stop_reason;   // 1: gradient test met, 2: energy test (Eq. 18) met
  int mixed;         // line searches run on the tensor cores
  int iter_round;    // line searches since the last float64 recompute
  double E;          // current shifted functional E~
  double gmax;       // max |G| of the current gradient
  double gpg;        // <G, P G>
  double gpg_old;    // <G_old, P G_old>
  double gopg;       // <G_old, P G>
  double gdo;        // <G, Delta_old>
  double gd;         // <G, Delta> of the current direction (= alpha_1, the slope at x = 0)
  double beta;       // Polak-Ribiere coefficient of the current direction
  double x;          // line-search step
  double alpha[5];   // quartic coefficients of the last line search
  double tol_grad;
  double e_tol;
  double halt_gmax;  // mixed precision: request a float64 refinement below this max|G|
  double best_g;     // mixed precision: smallest max|G| of the current round
  int best_it;       // line search of the round where best_g was reached
  int stall_window;  // refine when best_g has not halved for this many line searches
  double trace[12];  // last trace products (debug / tests)
};

constexpr int kReduceBlocks = 512;   // fixed grid of the gradient reductions (deterministic sums)
constexpr int kNumTraces = 11;

// ------------------------------------------------------------------ error handling
struct CudaError {
  cudaError_t err;
  const char* what;
};

void set_last_error(const std::string& msg);
const char* last_error_cstr();

// every kernel launch of the library is counted (omm_launch_count)
void count_launch();
#define OMM_LAUNCH_CHECK()                   \
  do {                                       \
    ::omm::count_launch();                   \
    OMM_CUDA_TRY(cudaGetLastError());        \
  } while (0)

#define OMM_CUDA_TRY(call)                                                   \
  do {                                                                       \
    cudaError_t e__ = (call);                                                \
    if (e__ != cudaSuccess) throw ::omm::CudaError{e__, #call};              \
  } while (0)

// ------------------------------------------------------------------ device memory
// Stream-ordered allocations from a pool the library owns (one per device; freed blocks are kept
// for reuse). alloc throws std::bad_alloc; the memory may be used on st at once and on other
// streams after a synchronisation with st. release(nullptr) is ignored.
namespace mem {
void* alloc(size_t bytes, cudaStream_t st);
void release(void* p, cudaStream_t st);
template <typename T>
void alloc(T** p, size_t count, cudaStream_t st) {
  *p = nullptr;
  *p = static_cast<T*>(alloc(count * sizeof(T), st));
}
}  // namespace mem

// ------------------------------------------------------------------ kernel timing
// CUDA-event timing of selected launches on their own stream (enabled by
// omm_opts.profile): begin()/end() bracket a launch, collect() after a stream
// synchronisation adds the elapsed times.
class Profiler {
 public:
  static constexpr int kTags = 4;  // launches may be tagged 0..3 (the line-search GEMMs) for per-tag sums
  bool on = false;
  double ms = 0.0, flop = 0.0;
  long launches = 0;
  double ms_tag[kTags] = {}, flop_tag[kTags] = {};
  void begin(cudaStream_t st);
  void end(cudaStream_t st, double flop_of_launch, int tag = -1);
  // the stream must have been synchronised; keep >= 0: only the first `keep` launches recorded
  // since the last collect are counted (the later ones were skipped by the solver's stop flags)
  void collect(long keep = -1);
  void reset() {
    ms = 0.0; flop = 0.0; launches = 0;
    for (int t = 0; t < kTags; ++t) ms_tag[t] = flop_tag[t] = 0.0;
  }
  ~Profiler();

 private:
  struct Pair { cudaEvent_t a, b; double flop; int tag; };
  Pair* pairs_ = nullptr;
  int used_ = 0, cap_ = 0;
};

// ------------------------------------------------------------------ float64 GEMM
// C[b] = alpha * op(A[b]) op(B[b]) + beta * C[b], row-major, for b < batch.
// op(A) is M x K: A[i*lda + k] (transA = 0) or A[k*lda + i] (transA = 1).
// op(B) is K x N: B[k*ldb + j] (transB = 0) or B[j*ldb + k] (transB = 1).
// tri bit 0: compute only tiles that touch the lower triangle (i >= j);
// tri bit 1: start the K loop at max(tile row, tile col) (both operands lower-
// triangular in the contracted index, as in L^-T L^-1);
// tri bit 2: start the K loop at the tile's first column (op(B) lower triangular:
// B[k][j] = 0 for k < j); tri bit 3: end it after the tile's last row (op(A)
// lower triangular: A[i][k] = 0 for k > i).
// `skip`: device flag pair (done, halt); when either is set the kernel returns.
enum { kTriLower = 1, kTriKStart = 2, kTriKFromCol = 4, kTriKToRow = 8 };
void dgemm(cudaStream_t st, int transA, int transB, int M, int N, int K, double alpha,
           const double* A, long lda, long strideA, const double* B, long ldb, long strideB,
           double beta, double* C, long ldc, long strideC, int batch = 1, int tri = 0,
           const int* skip = nullptr);

// ------------------------------------------------------------------ Cholesky inverse
// P = A^-1 for symmetric positive definite A (m x m, row-major, device). A is
// overwritten. `work` needs m*m + m*64*... doubles (see cholesky.cu). info_dev
// receives 0 or the 1-based column of the first non-positive pivot.
size_t spd_inverse_workspace(int m);
void spd_inverse(cudaStream_t st, int m, double* A, double* P, double* work, int* info_dev);
// The same inverse with sliced tensor-core products (`slices` fixed-point slices of 5 bits,
// 2..10; 10 is float64-class); A is overwritten. err_dev receives a nonzero code if a bounded
// wait of a tensor-core GEMM expired.
size_t spd_inverse_sliced_workspace_bytes(int m);
long partial_capacity(int m);  // chunk-sum scratch (doubles) of the sliced products of an m x m inverse
void spd_inverse_sliced(cudaStream_t st, int m, double* A, double* P, void* work, int* info_dev, int* err_dev,
                        int slices = 10);
// The factor alone, for the reduction to standard form: A = L L^T with L left in A (lower
// triangle, zero above) and Y = L^-1 (lower, zero above); same workspaces as the inverses.
void spd_factor_inverse(cudaStream_t st, int m, double* A, double* Y, double* work, int* info_dev);
void spd_factor_inverse_sliced(cudaStream_t st, int m, double* A, double* Y, void* work, int* info_dev,
                               int* err_dev);

// ------------------------------------------------------------------ iteration kernels
void launch_axpby_shift(cudaStream_t st, long count, const double* H, const double* S, double eta,
                        double* Ht);                      // Ht = H - eta S
void launch_add_scaled(cudaStream_t st, long count, const double* S, const double* T, double inv_tau,
                       double* A);                       // A = S + T*inv_tau
void launch_grad_reduce(cudaStream_t st, long count, const double* G, const double* PG,
                        const double* Gold, const double* Dir, double* part, const Scalars* sc);
// Polak-Ribiere coefficient and stopping tests from nparts partial sums (4 doubles each: <G,PG>,
// <G_old,PG>, <G,Delta_old>, max|G|)
void launch_control_direction(cudaStream_t st, Scalars* sc, const double* part, int mixed, int nparts);
void launch_direction(cudaStream_t st, long count, const double* PG, double* Dir, const Scalars* sc);
// the mixed path's fused forms: the direction (n x m) and its bf16 split (leading dimension ldm);
// the state update of C, HC, SC, dHC, dSC with the splits of the new dHC, dSC, HC, SC into the
// operand stack rows [0, 4n) (Yhi, Ylo: the stack's hi and lo halves); the update of H_W, S_W
// with the split of [dS_W | dH_W] into W (Whi, Wlo: its columns 2n..4n, leading dimension ldw)
void launch_direction_split(cudaStream_t st, long n, long m, const double* PG, double* Dir, __nv_bfloat16* hi,
                            __nv_bfloat16* lo, long ldm, const Scalars* sc);
void launch_update_state_split(cudaStream_t st, long n, long m, double* C, double* Y4, const double* Dir, double* dY,
                               __nv_bfloat16* Yhi, __nv_bfloat16* Ylo, long ldm, const Scalars* sc);
void launch_update_subspace_split(cudaStream_t st, int n, double* SWHW, const double* Proj, const double* Wref,
                                  __nv_bfloat16* Whi, __nv_bfloat16* Wlo, long ldw, const Scalars* sc);
// the same steps on the mixed path's float32 side quantities (Delta, P G, [H Delta; S Delta],
// [dHC; dSC], leading dimension ldm): the direction and its split; the state update with three
// float64 FMAs per element; without a preconditioner, the reductions with PG = G (PG and G_old
// written)
void launch_direction_split32(cudaStream_t st, long n, long m, const float* PG, float* Dir, __nv_bfloat16* hi,
                              __nv_bfloat16* lo, long ldm, const Scalars* sc);
void launch_update_state_split32(cudaStream_t st, long n, long m, double* C, double* Y4, const float* Dir,
                                 const float* HD32, float* dY32, __nv_bfloat16* Yhi, __nv_bfloat16* Ylo, long ldm,
                                 const Scalars* sc);
void launch_reduce_unpreconditioned(cudaStream_t st, long n, long m, const double* G, double* Gold, const float* Dir,
                                    float* PG, long ldm, double* part, const Scalars* sc);
// fp32_products: the mixed path's traces (float32 products of the tensor-core projections)
void launch_traces(cudaStream_t st, int n, const double* SWHW, const double* Proj, double* part,
                   const Scalars* sc, bool fp32_products = false);
int traces_blocks(int n);    // 32 x 32 tiles of an n x n matrix (one CTA each in the n x n kernels)
int traces_partials(int n);  // partial-sum slots launch_traces writes (about four tiles per CTA)
void launch_control_linesearch(cudaStream_t st, Scalars* sc, const double* part, int nblocks);
void launch_update_state(cudaStream_t st, int n, long m, double* C, double* Y4, const double* Dir,
                         double* G, double* Gold, const Scalars* sc);
void launch_update_subspace(cudaStream_t st, int n, double* SWHW, const double* Proj,
                            const Scalars* sc);
void launch_scale_copy(cudaStream_t st, long count, const double* src, double a, double* dst,
                       const Scalars* sc);              // dst = a*src (skipped when done/halt)
void launch_functional(cudaStream_t st, int n, const double* SWHW, double* part);  // E~ partials
void launch_finish_functional(cudaStream_t st, Scalars* sc, const double* part, int nblocks);
void launch_gmax(cudaStream_t st, long count, const double* G, double* part);
void launch_finish_gmax(cudaStream_t st, Scalars* sc, const double* part);
void launch_two_i_minus(cudaStream_t st, int n, const double* SW, long ldsw, double* out);  // 2I - S_W
void launch_symmetrize_lower(cudaStream_t st, int m, double* A);  // A[j,i] = A[i,j], i > j
void launch_fill(cudaStream_t st, long count, double v, double* dst);

// Device-side line minimum (first local minimum of the quartic along x > 0).

void launch_line_minimum(cudaStream_t st, const double* a, double* x, int* status);

}  // namespace omm
