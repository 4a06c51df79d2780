/*
 * omm.h -- C ABI of the GB300 orbital minimization method (OMM) library.
 *
 * The library minimises the OMM functional of Corsetti, "The orbital
 * minimization method for electronic structure calculations with finite-range
 * atomic basis sets" (arXiv:1312.1549):
 *
 *     E~[C] = 2 Tr[(2I - S_W) H_W] = 4 Tr H_W - 2 Tr(S_W H_W)      (Sec. 2.1, Eq. 8)
 *     H_W = C^T H~ C,  S_W = C^T S C                                 (Eqs. 5-6)
 *     H~  = H - eta S  (eigenspectrum shift)                         (Sec. 2.2, Eq. 9)
 *
 * by conjugate gradients with Polak-Ribiere directions, the exact quartic line
 * search with directly computed coefficients (Sec. 2.3, Eqs. 12-16) and the
 * kinetic preconditioner P = (S + T/tau)^-1 (Sec. 2.4, Eq. 17), on one GPU.
 * The converged point gives the band energy E = 2 sum_{i<=n} eps_i of the
 * generalised eigenproblem H c = eps S c (Eq. 1), the density matrix
 * D = 2 C (2I - S_W) C^T = dE/dH and the energy-density matrix EDM, with
 * dE/dS = -EDM.
 *
 * Conventions shared by every entry point
 *  - Numbers are IEEE float64.
 *  - H, S, T, D, EDM are m x m, symmetric, row-major (row-major and
 *    column-major coincide for symmetric matrices).
 *  - C0 and C are n x m row-major: row j holds Wannier function j over the m
 *    basis functions. These are the same bytes as the paper's m x n matrix C
 *    stored column-major.
 *  - Every matrix pointer may point to host memory (pageable or pinned) or to
 *    device memory of the current device; the library copies with
 *    cudaMemcpyDefault (unified addressing) and never keeps a caller pointer
 *    after a call returns. Scalar outputs (E, info) are host pointers.
 *  - All GPU work is ordered on the stream given to omm_create (NULL = the
 *    legacy default stream). Calls return after their results are written.
 *  - Errors: every call returns an omm_status and never aborts, traps or
 *    exits. omm_last_error() gives a human-readable message for the last
 *    failing call on the calling thread. After a non-OK status the outputs are
 *    unspecified, except that omm_solve leaves the last iterate in C on
 *    OMM_ERR_NO_CONVERGENCE.
 *  - Units: eta in the units of H (hartree in the bundled workloads), tau in
 *    the units of T (tau = 10 Ry is 5 Ha).
 *  - Thread safety: a context may be used by one thread at a time; distinct
 *    contexts are independent.
 */
#ifndef OMM_GB300_OMM_H
#define OMM_GB300_OMM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct omm_ctx omm_ctx; /* opaque; owned by the library */

typedef enum {
  OMM_OK = 0,
  OMM_ERR_ARG = 1,            /* invalid argument (sizes, NULL pointers, tau <= 0, n >= m) */
  OMM_ERR_NOT_SPD = 2,        /* S + T/tau (or S) is not positive definite (Cholesky failed) */
  OMM_ERR_UNBOUNDED = 3,      /* the quartic along the search line has no minimum: the shifted
                                 functional is unbounded below (Sec. 2.2 footnote; eta too high) */
  OMM_ERR_NO_CONVERGENCE = 4, /* max_iter line searches without meeting the tolerance */
  OMM_ERR_NONFINITE = 5,      /* a NaN or Inf appeared in a reduction */
  OMM_ERR_TIMEOUT = 6,        /* a bounded device-side wait gave up */
  OMM_ERR_CUDA = 7,           /* a CUDA runtime call failed */
  OMM_ERR_OOM = 8,            /* device memory allocation failed */
  OMM_ERR_STATE = 9           /* call out of order (e.g. omm_backward before a solve) */
} omm_status;

typedef enum {
  OMM_PREC_FP64 = 0,   /* every contraction in float64 */
  OMM_PREC_MIXED = 1   /* bulk contractions on the BF16 tensor cores as 3-term split products
                          with FP32 accumulation, state and every scalar in float64; the
                          refreshes of the state and the certificate of the final point use
                          float64-class products (fixed-point slices on the tensor cores, the
                          Ozaki scheme; native float64 for the certificate with
                          native_certificate = 1, and for problems small enough that native
                          float64 is cheaper); the preconditioner inverse uses the same slicing
                          at preconditioner grade (precond_slices) */
} omm_precision;

/* Options. A zero-filled struct (or NULL) selects every default. */
typedef struct {
  int precision;        /* omm_precision; default OMM_PREC_FP64 */
  int max_iter;         /* line searches per solve; 0 -> 10000 */
  int no_precondition;  /* 0 -> use P = (S + T/tau)^-1 (default); 1 -> plain gradient */
  int check_every;      /* line searches between host convergence polls; 0 -> 8 */
  double tol_grad;      /* stop when max|G| < tol_grad, G the exact gradient of Eq. 12; 0 -> 1e-9 */
  double e_tol;         /* also stop when |2(E_new-E)/(E_new+E)| <= e_tol (Eq. 18); 0 -> off */
  double refine_ratio;  /* mixed: refresh the state with float64-class products once max|G|
                           fell by this factor since the last refresh (or stalls); 0 -> 1e-3 */
  int profile;          /* 1 -> time every launch of the line-search GEMM with CUDA events on
                           the context's stream (omm_info.ms_main_gemm and friends) */
  int native_certificate; /* mixed: 0 (default) -> certify the final point, and form the
                           density matrix D and the gradients of omm_backward, with
                           float64-class tensor-core products (fixed-point slices, about
                           2^-50 resp. 2^-40 of each row-scaled operand); 1 -> with native
                           float64 GEMMs */
  int cholesky;         /* 1 -> reduce to standard form instead of preconditioning (Sec. 2.4,
                           last paragraph): S = L L^T, H_r = L^-1 H L^-T, and the OMM runs on
                           H_r with S = I and no preconditioner (T and tau are ignored), from
                           C_r = L^T C0; the result is transformed back, C = L^-T C_r. The
                           iterates are those of the original problem preconditioned by S^-1;
                           tol_grad and omm_info.gmax then refer to the gradient of the reduced
                           problem (Eq. 12 with S = I). Products as for the preconditioner:
                           float64, or float64-class slices on the mixed path. 0 (default) -> off */
  int precond_slices;   /* mixed: products of the tensor-core inverse of S + T/tau: 1 (the default,
                           0 -> 1) the 3-term bf16 split form (about 16 bits of each product),
                           2..10 that many 5-bit fixed-point slices (about 5 bits each). P enters
                           the line searches only through its bf16 rounding (the single-pass P G
                           of the search direction) and the converged point does not depend on P,
                           so the float64-class 10 slices buy nothing there; the Cholesky
                           flavour's factor always takes 10 */
  int debug_expire_wait; /* tests of the timeout status only (0 = off, the default): 1 -> on the
                           mixed path the first tensor-core GEMM of every line search waits about
                           1 ms on a barrier that nothing arrives at, before it issues any copy or
                           MMA; the wait expires and omm_solve returns OMM_ERR_TIMEOUT. The context
                           stays usable (the next omm_solve of a context created without the flag
                           succeeds) */
} omm_opts;

/* Per-solve report. */
typedef struct {
  int status;           /* omm_status of the solve */
  int iterations;       /* line searches in total */
  int iterations_fp64;  /* line searches run with float64 contractions */
  int refinements;      /* recomputations of the state before the certificate (mixed precision) */
  double E;             /* band energy 2 sum eps_i = E~ + 2 n eta (certified in float64) */
  double Etilde;        /* the shifted functional E~ at the returned C */
  double gmax;          /* max|G| of the certified gradient at the returned C */
  double ms_setup;      /* omm_create GPU time (shift, Cholesky, inverse, splits) */
  double ms_iterate;    /* CG line searches */
  double ms_refine;     /* refreshes of the state and the final certificate */
  double ms_outputs;    /* density matrix */
  double gemm_flop;     /* logical contraction flops of the solve (FP64-equivalent) */
  double gemm_flop_tc;  /* flops issued to the BF16 tensor cores (3 per logical in split form) */
  double kernel_launches;    /* kernels launched by the library during the solve */
  double ms_main_gemm;       /* with opts.profile: summed duration of the line-search GEMM launches */
  double main_gemm_launches; /* with opts.profile: number of those launches */
  double main_gemm_flop;     /* with opts.profile: flops they issued (tensor-core flops when mixed) */
  double ms_certify;         /* native float64 state recomputes (part of ms_refine) */
  double ms_precond;         /* the Cholesky inverse P = (S + T/tau)^-1 (part of ms_setup): float64,
                                or preconditioner-grade sliced products on the mixed path (m >=
                                2048); with opts.cholesky the factor L, L^-1 and H_r = L^-1 H L^-T
                                instead */
  int tile_width[4];         /* mixed: output tile shape the autotuner chose for the P G, [H D; S D],
                                projection and gradient GEMMs: 256 or 128 (columns of a 128-row
                                tile on one SM), 1000 + 128, 192 or 256 (a 256-row tile on a pair
                                of SMs), 2000 + the width (the same on a cluster of two pairs that
                                share the A operand), 0: not run */
  double ms_autotune;        /* time the autotuner spent timing candidates (0 when cached) */
  double ms_sliced_gemm;     /* with opts.profile: summed duration of the float64-class sliced
                                products of omm_create (inverse) and this solve (refreshes,
                                certificate, D) */
  double sliced_gemm_flop;   /* with opts.profile: tensor flops they issued */
  double sliced_gemm_launches; /* with opts.profile: their number */
  double ms_batch;           /* omm_solve_batched only: the whole batched solve. There ms_iterate,
                                ms_main_gemm, main_gemm_launches and main_gemm_flop are batch
                                totals too (the same in every instance's report) */
  double ms_transform;       /* opts.cholesky: the coefficient transforms C_r = L^T C0 and
                                C = L^-T C_r of this solve */
  double ms_gemm_plan[4];    /* mixed single solve with opts.profile: ms_main_gemm split over the
                                P G, [H D; S D], projection and gradient GEMMs */
  double flop_gemm_plan[4];  /* the same for main_gemm_flop */
  double ms_batch_refresh;   /* omm_solve_batched only: host wall time of its refresh and
                                certificate passes (the stopped instances' recomputes, overlapped
                                on several streams, and the read-back that follows) */
} omm_info;

/* Create a solver context for one (H, S, T) and do the per-geometry setup:
 * H~ = H - eta S (Eq. 9) and the preconditioner P = (S + T/tau)^-1 (Eq. 17), once per
 * geometry (Sec. 2.4): on the float64 path (and on the mixed path below m = 2048) by a
 * blocked float64 Cholesky factorisation and inverse; on the mixed path from m = 2048 by a
 * recursive Cholesky inverse whose products are tensor-core GEMMs at preconditioner grade
 * (opts->precond_slices: by default the 3-term bf16 split form; float32 diagonal blocks).
 *   m      number of basis functions, n number of Wannier functions, 0 < n < m.
 *   H,S,T  m x m symmetric float64 (host or device). T may be NULL when
 *          opts->no_precondition == 1. They are copied; the caller keeps ownership.
 *   eta    eigenspectrum shift; the solve finds the n lowest states only if
 *          eta lies above the n-th eigenvalue (Sec. 2.2).
 *   tau    kinetic-energy scale, > 0; +infinity gives P = S^-1.
 *   stream cudaStream_t (as void*) for every GPU operation of this context.
 *   out    receives the context; *out is NULL on failure.
 * With opts->cholesky the setup is the factorisation S = L L^T and the reduction
 * H_r = L^-1 H L^-T instead of P (S must then be positive definite: OMM_ERR_NOT_SPD).
 * Errors: OMM_ERR_ARG, OMM_ERR_NOT_SPD, OMM_ERR_OOM, OMM_ERR_CUDA. */
omm_status omm_create(int m, int n, const double* H, const double* S, const double* T,
                      double eta, double tau, const omm_opts* opts, void* stream,
                      omm_ctx** out);

/* Minimise E~ from the starting coefficients C0 (n x m, host or device; may alias C).
 * Writes the converged C (n x m), the band energy *E (host) and, if D != NULL,
 * the density matrix D = 2 C (2I - S_W) C^T (m x m) = dE/dH. info may be NULL.
 * Stops when max|G| < tol_grad (G of Eq. 12, certified in float64), or by the
 * relative energy change of Eq. 18 when e_tol > 0.
 * Errors: OMM_ERR_ARG, OMM_ERR_UNBOUNDED, OMM_ERR_NO_CONVERGENCE,
 * OMM_ERR_NONFINITE, OMM_ERR_CUDA. */
omm_status omm_solve(omm_ctx* ctx, const double* C0, double* C, double* E, double* D,
                     omm_info* info);

/* Gradients of E with respect to H and S at the last converged solve (m x m
 * each, host or device, either may be NULL):
 *   dEdH = D = 2 C (2I - S_W) C^T,
 *   dEdS = -EDM = -(2 C H~_W C^T + eta D).
 * By the envelope theorem these are exact at the minimum (derived from Eq. 8
 * with H~ = H - eta S). Errors: OMM_ERR_STATE (no converged solve), OMM_ERR_CUDA. */
omm_status omm_backward(omm_ctx* ctx, double* dEdH, double* dEdS);

/* Replace H (SCF warm start: S, T and P are kept; Sec. 2.5.2). With opts.cholesky the new
 * H is reduced with the kept factor: H_r = L^-1 H L^-T. */
omm_status omm_update_H(omm_ctx* ctx, const double* H);

/* Release every resource of the context (NULL is ignored). */
void omm_free(omm_ctx* ctx);

/* ---- batches of independent problems (k-points, spins, snapshots) ---- */
typedef struct omm_batch omm_batch; /* opaque; owned by the library */

/* Create `count` independent problems in one batch: per instance i the same
 * arguments as omm_create (m[i], n[i], H[i], S[i], T[i] (T may be NULL when
 * opts->no_precondition), eta[i], tau[i]), one opts and one stream for all.
 * With opts->precision == OMM_PREC_MIXED the line searches of all instances
 * run in lockstep: each phase is one launch over the whole batch (grouped
 * tensor-core GEMMs, batched vector kernels), captured once in a CUDA graph
 * and replayed; with OMM_PREC_FP64 the instances are solved one after the
 * other. Errors: as omm_create, reported for the first failing instance. */
omm_status omm_create_batched(int count, const int* m, const int* n, const double* const* H,
                              const double* const* S, const double* const* T, const double* eta,
                              const double* tau, const omm_opts* opts, void* stream, omm_batch** out);

/* Solve every instance from C0[i] (n[i] x m[i], host or device). Writes C[i]
 * (if C and C[i] are non-NULL), E[i] (host array, count entries, may be NULL)
 * and info[i] (host array, may be NULL; ms_iterate is the time of the whole
 * batched solve). Returns OMM_OK when every instance converged, else the
 * status of the first failing instance (its info[i].status says which). */
omm_status omm_solve_batched(omm_batch* b, const double* const* C0, double* const* C, double* E,
                             omm_info* info);

/* The context of instance i (for omm_backward after a batched solve), or NULL. */
omm_ctx* omm_batch_instance(omm_batch* b, int i);

/* Release the batch and its instances (NULL is ignored). */
void omm_free_batched(omm_batch* b);

/* ---- Hermitian problems (complex matrices: k points) ----
 * The paper states the method for complex matrices (Secs. 2.1-2.3: H_W = C^H H C, S_W = C^H S C,
 * the quartic of Eq. 13 with (S_W')^H) and uses them for its k-point tests (Sec. 3.3). These
 * entry points take complex128 matrices -- interleaved (real, imaginary) float64 pairs, row-major:
 * H, S, T, D, EDM m x m Hermitian (2 m^2 doubles each), C0 and C n x m (2 n m doubles; row j is
 * Wannier function j, i.e. column j of the paper's C, not conjugated) -- host or device, with the
 * conventions above. The library solves the real form [[Re A, -Im A], [Im A, Re A]] (2m x 2m,
 * 2n Wannier functions) on its real path, from the real form of C0; the iterates stay the real
 * forms of the complex ones, so the line-search steps are those of the complex method and
 * max|G| (tol_grad, omm_info.gmax) is the largest |Re G_ij| or |Im G_ij| of the complex gradient
 * of Eq. 12 (dE~ = Re Tr(G^H dC)). E is the complex problem's band energy 2 sum_{i<=n} eps_i
 * (info.E and info.Etilde likewise); omm_info's counters and timings are those of the real
 * solve, which does twice the arithmetic of complex products. D = 2 C (2I - S_W) C^H is dE/dH
 * and dE/dS = -EDM in the sense dE = Re Tr(D dH) - Re Tr(EDM dS) for Hermitian dH, dS.
 * A Hermitian context or batch is used only through these entry points (and omm_free,
 * omm_free_batched, omm_batch_instance); the real ones return OMM_ERR_ARG for it. */
omm_status omm_create_hermitian(int m, int n, const double* H, const double* S, const double* T,
                                double eta, double tau, const omm_opts* opts, void* stream,
                                omm_ctx** out);
omm_status omm_solve_hermitian(omm_ctx* ctx, const double* C0, double* C, double* E, double* D,
                               omm_info* info);
omm_status omm_backward_hermitian(omm_ctx* ctx, double* dEdH, double* dEdS);
/* SCF warm start with a new Hermitian H (S, T and the preconditioner kept). */
omm_status omm_update_H_hermitian(omm_ctx* ctx, const double* H);
/* A batch of Hermitian problems (e.g. the points of a k grid), solved in lockstep like
 * omm_create_batched / omm_solve_batched. */
omm_status omm_create_hermitian_batched(int count, const int* m, const int* n, const double* const* H,
                                        const double* const* S, const double* const* T,
                                        const double* eta, const double* tau, const omm_opts* opts,
                                        void* stream, omm_batch** out);
omm_status omm_solve_hermitian_batched(omm_batch* b, const double* const* C0, double* const* C,
                                       double* E, omm_info* info);

/* Static description of a status code. */
const char* omm_status_str(omm_status s);

/* Message of the last failing call on this thread ("" if none). */
const char* omm_last_error(void);

/* Number of GPU kernels this library has launched in the process so far. */
unsigned long long omm_launch_count(void);

#ifdef __cplusplus
}
#endif

#endif /* OMM_GB300_OMM_H */
