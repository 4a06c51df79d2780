// Mixed-precision line searches: every contraction of a line search runs on
// the BF16 tensor cores with FP32 accumulation, in 3-term split form
// (tc_gemm.cu) except the preconditioned gradient P G of the search direction,
// which is a single bf16 pass; the state C, HC, SC, H_W, S_W and every scalar
// stay in float64. Each tensor-core product carries a factor that shrinks with
// the step, so its error does too (iterative refinement):
//   HD, SD = [H~; S] Delta                 (Delta -> 0)
//   H', S', H'', S'' = Delta^T [HC SC HD SD]
//   P G                                     (G -> 0; steers the search only)
//   G = G_ref + 8 dHC - 4 (dS_W HC + dH_W SC + S_W,ref dHC + H_W,ref dSC)
// where _ref is the state at the last float64 refresh and d = now - ref
// (Eq. 12 expanded around the refresh point). Computing Eq. 12 directly on
// the tensor cores would leave an absolute error of about 2^-17 |HC| in G,
// a floor the line searches cannot get below. The host loop refreshes the
// state in float64 when max|G| has dropped by refine_ratio (or stalls) and
// certifies the final point in float64.
#include "omm_mixed.cuh"
#include "tc_gemm.cuh"

#include <algorithm>
#include <new>

namespace omm {

struct MixedState {
  int m = 0, n = 0;
  long ldm = 0, ld4n = 0;
  bool precond = false;
  int npass = 3;
  __nv_bfloat16 *HS_hi = nullptr, *HS_lo = nullptr;   // [H~; S]   2m x m
  __nv_bfloat16 *P_hi = nullptr, *P_lo = nullptr;     // P         m x m
  __nv_bfloat16 *G_hi = nullptr, *G_lo = nullptr;     // G         n x m
  __nv_bfloat16 *D_hi = nullptr, *D_lo = nullptr;     // Delta     n x m
  __nv_bfloat16 *Y_hi = nullptr, *Y_lo = nullptr;     // [dHC; dSC; HC; SC; HD; SD]  6n x m
  __nv_bfloat16 *W_hi = nullptr, *W_lo = nullptr;     // [S_W,ref | H_W,ref | dS_W | dH_W] n x 4n
  double* Gref = nullptr;                              // G at the last refresh, n x m
  double* Wref = nullptr;                              // [S_W | H_W] at the last refresh, n x 2n
  double* red = nullptr;                               // per (tile, warp) sums of the P G epilogue
  // float32 side quantities of a line search (leading dimension ldm): the direction Delta, P G,
  // [H Delta; S Delta] and [dHC; dSC] = [HC - HC_ref; SC - SC_ref]. Each enters the float64 state
  // only as an increment or through a bf16 split product, whose own error (about 2^-17) is far
  // above their float32 rounding (2^-24)
  float* Dir32 = nullptr;                              // n x m
  float* PG32 = nullptr;                               // n x m
  float* HD32 = nullptr;                               // 2n x m
  float* dY32 = nullptr;                               // 2n x m
  tc::Operand opHS, opP, opG, opD, opYproj, opYgrad, opYhc, opW;
  tc::BlockLists hs_blocks[3];  // block sparsity of [H~; S] for 256-, 128- and 192-row blocks (Sec. 2.6)
  int* err = nullptr;
  int expire = 0;  // tests: the first line-search GEMM of every line search waits on nothing and expires
  // the four line-search GEMMs as persistent-launch descriptors (device), built on first use
  tc::GroupDesc* plans = nullptr;
  int plan_tiles[4] = {0, 0, 0, 0};
  tc::TileShape plan_shape[4];             // output tile shapes chosen by the autotuner
  double ms_autotune = 0.0;               // time the autotuner spent timing candidates
  const Scalars* plan_sc = nullptr;
  // one line search as a CUDA graph, with the stream and buffers it was captured for
  cudaGraphExec_t ls_exec = nullptr;
  cudaStream_t ls_stream = nullptr;
  const void* ls_key[4] = {nullptr, nullptr, nullptr, nullptr};
  bool ls_failed = false;
};

namespace {

long round8(long x) { return (x + 7) / 8 * 8; }
// output tiles of the P G product (n x m) counted as 128 x 128 tiles, rounded so that 256-row tiles
// (two slots of four warps each) and the odd column tile of a two-pair cluster fit too
long red_tiles(long n, long m) { return 2 * ((n + 255) / 256) * ((m + 127) / 128 + 1); }

template <typename T>
void alloc(T** p, size_t count, cudaStream_t st) {
  mem::alloc(p, count, st);
}

}  // namespace

MixedState* mixed_create(cudaStream_t st, int m, int n, const double* HS, const double* P) {
  MixedState* ms = new MixedState();
  try {
    ms->m = m;
    ms->n = n;
    ms->ldm = round8(m);
    ms->ld4n = round8(4L * n);  // leading dimension of the n x 4n gradient operand W
    ms->precond = (P != nullptr);
    const long ldm = ms->ldm, ld4n = ms->ld4n;
    // each split operand is one allocation holding the stack [hi; lo]
    auto pair = [st](__nv_bfloat16** hi, __nv_bfloat16** lo, long rows, long ld) {
      alloc(hi, 2 * (size_t)rows * ld, st);
      *lo = *hi + rows * ld;
    };
    pair(&ms->HS_hi, &ms->HS_lo, 2L * m, ldm);
    if (ms->precond) pair(&ms->P_hi, &ms->P_lo, m, ldm);
    pair(&ms->G_hi, &ms->G_lo, n, ldm);
    pair(&ms->D_hi, &ms->D_lo, n, ldm);
    pair(&ms->Y_hi, &ms->Y_lo, 6L * n, ldm);
    pair(&ms->W_hi, &ms->W_lo, n, ld4n);
    alloc(&ms->Gref, (size_t)n * m, st);
    alloc(&ms->Wref, 2L * n * n, st);
    alloc(&ms->Dir32, (size_t)n * ldm, st);
    alloc(&ms->PG32, (size_t)n * ldm, st);
    alloc(&ms->HD32, 2L * n * ldm, st);
    alloc(&ms->dY32, 2L * n * ldm, st);
    OMM_CUDA_TRY(cudaMemsetAsync(ms->Dir32, 0, (size_t)n * ldm * sizeof(float), st));
    // 4 sums per epilogue warp (4 per 128-row tile, 8 per 256-row tile) and output tile, at the
    // narrowest tile (128 columns)
    alloc(&ms->red, (size_t)16 * red_tiles(n, m), st);
    alloc(&ms->err, 1, st);
    OMM_CUDA_TRY(cudaMemsetAsync(ms->err, 0, sizeof(int), st));
    OMM_CUDA_TRY(cudaMemsetAsync(ms->red, 0, (size_t)16 * red_tiles(n, m) * sizeof(double), st));
    // padding columns stay zero (the tensor maps never read them, but keep them defined)
    OMM_CUDA_TRY(cudaMemsetAsync(ms->Y_hi, 0, 2 * (size_t)6 * n * ldm * 2, st));
    OMM_CUDA_TRY(cudaMemsetAsync(ms->W_hi, 0, 2 * (size_t)n * ld4n * 2, st));
    tc::split(st, HS, 2L * m, m, m, ms->HS_hi, ms->HS_lo, ldm, nullptr);
    if (ms->precond) tc::split(st, P, m, m, m, ms->P_hi, ms->P_lo, ldm, nullptr);
    ms->opHS = tc::make_operand(ms->HS_hi, 2L * m, m, ldm, 2, false);
    if (ms->precond) ms->opP = tc::make_operand(ms->P_hi, m, m, ldm, 2, false);
    ms->opG = tc::make_operand(ms->G_hi, n, m, ldm, 2, true);
    ms->opD = tc::make_operand(ms->D_hi, n, m, ldm, 2, true);
    // views of the stack [dHC; dSC; HC; SC; HD; SD]: the projections read [HC; SC; HD; SD] as
    // K-major rows, the gradient [dHC; dSC; HC; SC] as MN-major rows (its contracted index), the
    // initial S_W, H_W product [HC; SC]
    ms->opYproj = tc::make_operand_view(ms->Y_hi, 6L * n, m, ldm, 2, false, 2 * n, 4L * n);
    ms->opYgrad = tc::make_operand_view(ms->Y_hi, 6L * n, m, ldm, 2, false, 0, 4L * n, true);
    ms->opYhc = tc::make_operand_view(ms->Y_hi, 6L * n, m, ldm, 2, false, 2 * n, 2L * n);
    ms->opW = tc::make_operand(ms->W_hi, n, 4L * n, ld4n, 2, true);
    // finite-range H and S: the operator product skips the K blocks where [H~; S] is zero
    for (int bn : {256, 128, 192}) tc::block_lists(st, HS, 2L * m, m, m, bn, ms->hs_blocks[tc::sparse_slot(bn)]);
  } catch (...) {
    mixed_destroy(ms, st);
    throw;
  }
  return ms;
}

void mixed_tuning(const MixedState* ms, int bn[4], double* ms_autotune) {
  // the width of a 256-row (SM pair) tile is reported as 1000 + width, of a two-pair cluster's 2000 + width
  for (int k = 0; k < 4; ++k) bn[k] = ms->plans ? ms->plan_shape[k].code() : 0;
  if (!ms->precond) bn[0] = 0;
  *ms_autotune = ms->ms_autotune;
}

static void drop_graph(MixedState* ms) {
  if (ms->ls_exec) cudaGraphExecDestroy(ms->ls_exec);
  ms->ls_exec = nullptr;
}

void mixed_set_expire(MixedState* ms, int on) {
  ms->expire = on;
  ms->plan_sc = nullptr;  // rebuild the plans with the flag
  drop_graph(ms);
}

void mixed_reset_error(MixedState* ms, cudaStream_t st) {
  OMM_CUDA_TRY(cudaMemsetAsync(ms->err, 0, sizeof(int), st));
}

MixedView mixed_view(MixedState* ms) {
  MixedView v;
  v.ldm = ms->ldm;
  v.ld4 = ms->ld4n;
  v.G_hi = ms->G_hi;
  v.D_hi = ms->D_hi;
  v.Y_hi = ms->Y_hi;
  v.W_hi = ms->W_hi;
  v.Gref = ms->Gref;
  v.Wref = ms->Wref;
  v.red = ms->red;
  v.Dir32 = ms->Dir32;
  v.PG32 = ms->PG32;
  v.HD32 = ms->HD32;
  v.dY32 = ms->dY32;
  v.opHS = &ms->opHS;
  v.opP = &ms->opP;
  v.opG = &ms->opG;
  v.opD = &ms->opD;
  v.opYproj = &ms->opYproj;
  v.opYgrad = &ms->opYgrad;
  v.opW = &ms->opW;
  v.err = ms->err;
  v.hs_blocks = ms->hs_blocks;
  v.npass = ms->npass;
  v.precond = ms->precond;
  return v;
}

void mixed_update_H(MixedState* ms, cudaStream_t st, const double* HS) {
  tc::split(st, HS, ms->m, ms->m, ms->m, ms->HS_hi, ms->HS_lo, ms->ldm, nullptr);
  for (int bn : {256, 128, 192})  // the pattern may change
    tc::block_lists(st, HS, 2L * ms->m, ms->m, ms->m, bn, ms->hs_blocks[tc::sparse_slot(bn)]);
}

void mixed_destroy(MixedState* ms, cudaStream_t st) {
  if (!ms) return;
  __nv_bfloat16* bufs[] = {ms->HS_hi, ms->P_hi, ms->G_hi, ms->D_hi, ms->Y_hi, ms->W_hi};
  for (auto* b : bufs) mem::release(b, st);
  for (double* d : {ms->Gref, ms->Wref, ms->red}) mem::release(d, st);
  for (float* f : {ms->Dir32, ms->PG32, ms->HD32, ms->dY32}) mem::release(f, st);
  mem::release(ms->err, st);
  mem::release(ms->plans, st);
  for (tc::BlockLists& bl : ms->hs_blocks) tc::free_block_lists(bl, st);
  drop_graph(ms);
  delete ms;
}

int mixed_error(MixedState* ms, cudaStream_t st) {
  int e = 0;
  OMM_CUDA_TRY(cudaMemcpyAsync(&e, ms->err, sizeof(int), cudaMemcpyDeviceToHost, st));
  OMM_CUDA_TRY(cudaStreamSynchronize(st));
  return e;
}

// The epilogues of the four line-search GEMMs (shared by the single and the batched solve):
//   [0] P G            P G as float32, plus the sums <G,PG>, <G_old,PG>, <G,Delta_old>, max|G| per
//                      (tile, warp) into ms->red, and G_old <- G
//   [1] [H D; S D]     as float32, and their bf16 split into the stack rows [4n, 6n)
//   [2] projections    [H' | S' | H'' | S''] into Proj
//   [3] gradient       G = G_ref + 8 dHC - 4 [..] [..], and its split (the next P G's operand)
void mixed_epilogues(MixedState* ms, const Scalars* sc, double* G, double* Gold, double* Y4, double* Proj,
                     tc::Epilogue out[4]) {
  (void)Y4;
  const int m = ms->m, n = ms->n;
  const long ldm = ms->ldm;
  const int* skip = &sc->done;
  tc::Epilogue epg{reinterpret_cast<double*>(ms->PG32), ldm, m, 0, 1.0, 0.0, n, m, skip, ms->err};
  epg.mode = tc::kEpReduce;
  epg.c_f32 = 1;
  epg.x0 = G;
  epg.x1 = Gold;
  epg.xout = Gold;
  epg.ldx = m;
  epg.x2f = ms->Dir32;
  epg.ldf = ldm;
  epg.part = ms->red;
  epg.sc = sc;
  tc::Epilogue ehd{reinterpret_cast<double*>(ms->HD32), ldm, m, (long)n * ldm, 1.0, 0.0, n, 2 * m, skip, ms->err};
  ehd.c_f32 = 1;
  ehd.bf_hi = ms->Y_hi + 4L * n * ldm;
  ehd.bf_ld = ldm;
  ehd.bf_blk = (long)n * ldm;
  ehd.bf_lo = 6L * n * ldm;
  const tc::Epilogue epr{Proj, 4L * n, 4L * n, 0, 1.0, 0.0, n, 4 * n, skip, ms->err};
  tc::Epilogue eg{G, m, m, 0, -4.0, 0.0, n, m, skip, ms->err};
  eg.mode = tc::kEpGrad;
  eg.x0 = ms->Gref;
  eg.ldx = m;
  eg.x1f = ms->dY32;
  eg.ldf = ldm;
  eg.xs = 8.0;
  eg.bf_hi = ms->G_hi;
  eg.bf_ld = ldm;
  eg.bf_lo = (long)n * ldm;
  out[0] = epg;
  out[1] = ehd;
  out[2] = epr;
  out[3] = eg;
  if (ms->expire) out[ms->precond ? 0 : 1].expire = 1;
}

// after a float64 recompute: the new reference point of the incremental gradient (G_ref = G,
// W_ref = [S_W | H_W], dHC = dSC = 0) and the bf16 operands of the next line search
void mixed_sync_state(MixedState* ms, cudaStream_t st, const double* Y4, const double* SWHW, const double* G) {
  const int m = ms->m, n = ms->n;
  const long ldm = ms->ldm, ld4 = ms->ld4n;
  OMM_CUDA_TRY(cudaMemcpyAsync(ms->Gref, G, (size_t)n * m * sizeof(double), cudaMemcpyDeviceToDevice, st));
  OMM_CUDA_TRY(cudaMemcpyAsync(ms->Wref, SWHW, 2L * n * n * sizeof(double), cudaMemcpyDeviceToDevice, st));
  OMM_CUDA_TRY(cudaMemsetAsync(ms->dY32, 0, 2L * n * ldm * sizeof(float), st));
  // stack rows [0, 2n): split of dHC = dSC = 0; rows [2n, 4n): split of [HC; SC]
  OMM_CUDA_TRY(cudaMemsetAsync(ms->Y_hi, 0, 2L * n * ldm * sizeof(__nv_bfloat16), st));
  OMM_CUDA_TRY(cudaMemsetAsync(ms->Y_lo, 0, 2L * n * ldm * sizeof(__nv_bfloat16), st));
  tc::split(st, Y4, 2L * n, m, m, ms->Y_hi + 2L * n * ldm, ms->Y_lo + 2L * n * ldm, ldm, nullptr);
  // W = [S_W,ref | H_W,ref | dS_W | dH_W] with dS_W = dH_W = 0
  tc::split(st, ms->Wref, n, 2L * n, 2L * n, ms->W_hi, ms->W_lo, ld4, nullptr);
  tc::split_diff(st, SWHW, ms->Wref, n, 2L * n, 2L * n, ms->W_hi + 2L * n, ms->W_lo + 2L * n, ld4, nullptr);
  tc::split(st, G, n, m, m, ms->G_hi, ms->G_lo, ldm, nullptr);
}

// The initial state (HC, SC, S_W, H_W, E~, G and max|G|) on the tensor cores.
// Its split-product error only has to stay below the first round's target
// (refine_ratio of the starting gradient); every later refresh and the
// certificate are float64-class.
void mixed_recompute_state(MixedState* ms, cudaStream_t st, Scalars* sc, const double* C, double* Y4,
                           double* SWHW, double* G, double* part, double* part2) {
  const int m = ms->m, n = ms->n;
  const long nm = (long)n * m, ldm = ms->ldm, ld4 = ms->ld4n;
  tc::split(st, C, n, m, m, ms->D_hi, ms->D_lo, ldm, nullptr);
  tc::gemm(st, ms->opD, ms->opHS, m, ms->npass, tc::Epilogue{Y4, m, m, nm, 1.0, 0.0, n, 2 * m, nullptr, ms->err});
  tc::split(st, Y4, 2L * n, m, m, ms->Y_hi + 2L * n * ldm, ms->Y_lo + 2L * n * ldm, ldm, nullptr);
  // [H_W | S_W] = C [HC; SC]^T written as SWHW = [S_W | H_W]
  tc::gemm(st, ms->opD, ms->opYhc, m, ms->npass,
           tc::Epilogue{SWHW + n, 2L * n, n, -(long)n, 1.0, 0.0, n, 2 * n, nullptr, ms->err});
  launch_functional(st, n, SWHW, part2);
  launch_finish_functional(st, sc, part2, traces_blocks(n));
  // G = 8 HC - 4 [S_W | H_W] [HC; SC] through the incremental-gradient epilogue: G_ref = 8 HC,
  // dHC = dSC = 0, W = [0 | 0 | S_W | H_W], so the stack rows [0, 2n) only meet zero columns of W
  launch_scale_copy(st, nm, Y4, 8.0, ms->Gref, nullptr);
  OMM_CUDA_TRY(cudaMemsetAsync(ms->dY32, 0, 2L * n * ldm * sizeof(float), st));
  OMM_CUDA_TRY(cudaMemsetAsync(ms->Y_hi, 0, 2L * n * ldm * sizeof(__nv_bfloat16), st));
  OMM_CUDA_TRY(cudaMemsetAsync(ms->Y_lo, 0, 2L * n * ldm * sizeof(__nv_bfloat16), st));
  OMM_CUDA_TRY(cudaMemsetAsync(ms->Wref, 0, 2L * n * n * sizeof(double), st));
  tc::split(st, ms->Wref, n, 2L * n, 2L * n, ms->W_hi, ms->W_lo, ld4, nullptr);
  tc::split(st, SWHW, n, 2L * n, 2L * n, ms->W_hi + 2L * n, ms->W_lo + 2L * n, ld4, nullptr);
  tc::Epilogue eg{G, m, m, 0, -4.0, 0.0, n, m, nullptr, ms->err};
  eg.mode = tc::kEpGrad;
  eg.x0 = ms->Gref;
  eg.ldx = m;
  eg.x1f = ms->dY32;
  eg.ldf = ldm;
  eg.xs = 8.0;
  tc::gemm_persistent(st, ms->opW, ms->opYgrad, 4 * n, tc::pairs_split3(), eg);
  launch_gmax(st, nm, G, part);
  launch_finish_gmax(st, sc, part);
}

namespace {

enum { kPlanPG = 0, kPlanHD, kPlanProj, kPlanG };

// The search direction's P G is one bf16 pass, bf16(G) bf16(P) with FP32 accumulation: the
// direction only steers the search (Sec. 2.4: P stands in for the inverse Hessian), while the
// line search and the gradient it is measured by keep the split products and the float64 state,
// so the minimum reached is the same. The three other products use the 3-term split form.
tc::PairList plan_pairs(int k) { return k == kPlanPG ? tc::pairs_single() : tc::pairs_split3(); }

void build_plans(MixedState* ms, cudaStream_t st, Scalars* sc, double* G, double* Gold, double* Y4, double* Proj) {
  const int m = ms->m, n = ms->n;
  tc::GroupDesc h[4] = {};
  tc::Epilogue ep[4];
  mixed_epilogues(ms, sc, G, Gold, Y4, Proj, ep);
  const tc::Operand* opA[4] = {&ms->opG, &ms->opD, &ms->opD, &ms->opW};
  const tc::Operand* opB[4] = {ms->precond ? &ms->opP : &ms->opG, &ms->opHS, &ms->opYproj, &ms->opYgrad};
  const int K[4] = {m, m, m, 4 * n};
  for (int k = ms->precond ? 0 : 1; k < 4; ++k) {  // without P there is no P G product
    // output tile width from the autotuner (timed once per shape in a process); the operator
    // product runs block-sparse over [H~; S]
    tc::GemmSpec spec{opA[k], opB[k], K[k], ep[k]};
    if (k == kPlanHD)
      for (int q = 0; q < 3; ++q) spec.sparse[q] = &ms->hs_blocks[q];
    double ms_tune = 0.0;
    const tc::TileShape ts = tc::choose_tile_shape(st, {spec}, plan_pairs(k), &ms_tune);
    ms->plan_shape[k] = ts;
    ms->ms_autotune += ms_tune;
    h[k] = tc::make_group(*opA[k], *opB[k], K[k], ep[k], 0, ts.bn, ts.quad ? nullptr : spec.sparse[tc::sparse_slot(ts.bn)],
                          ts.pair, ts.quad);
    ms->plan_tiles[k] = tc::tiles_of(ep[k], ts.bn, ts.pair, ts.quad);
  }
  if (!ms->plans) alloc(&ms->plans, 4, st);
  OMM_CUDA_TRY(cudaMemcpyAsync(ms->plans, h, sizeof(h), cudaMemcpyHostToDevice, st));
  OMM_CUDA_TRY(cudaStreamSynchronize(st));  // h is a stack buffer
  ms->plan_sc = sc;
}

void run_plan(MixedState* ms, cudaStream_t st, int k) {
  tc::gemm_persistent(st, ms->plans + k, 1, ms->plan_tiles[k], plan_pairs(k), ms->err, ms->plan_shape[k].bn,
                      ms->plan_shape[k].pair, ms->plan_shape[k].quad);
}

}  // namespace

int mixed_reduce_parts(const MixedState* ms) {
  // one slot of partial sums per epilogue warp of every P G output tile (eight on an SM pair's tile)
  const tc::TileShape& ts = ms->plan_shape[kPlanPG];
  return 4 * ms->plan_tiles[kPlanPG] * (ts.quad ? 4 : (ts.pair ? 2 : 1));
}

void mixed_iterate(MixedState* ms, cudaStream_t st, Scalars* sc, double* C, double* Dir, double* G,
                   double* Gold, double* PG, double* Y4, double* SWHW, double* Proj, double* part,
                   double* part2, const double* HS, const double* P, bool precond, Profiler& pf) {
  (void)HS;
  (void)P;
  (void)Dir;
  (void)PG;
  const int m = ms->m, n = ms->n;
  const int np = ms->npass;
  if (ms->plan_sc != sc) build_plans(ms, st, sc, G, Gold, Y4, Proj);
  // P G (Sec. 2.4); the epilogue also takes the Polak-Ribiere products and max|G| and moves G to G_old
  if (precond) {
    pf.begin(st);
    run_plan(ms, st, kPlanPG);
    pf.end(st, 2.0 * n * (double)m * m, kPlanPG);  // one bf16 pass
    launch_control_direction(st, sc, ms->red, 1, mixed_reduce_parts(ms));
  } else {  // P = I: the same products with PG = G
    launch_reduce_unpreconditioned(st, n, m, G, Gold, ms->Dir32, ms->PG32, ms->ldm, part, sc);
    launch_control_direction(st, sc, part, 1, kReduceBlocks);
  }
  launch_direction_split32(st, n, m, ms->PG32, ms->Dir32, ms->D_hi, ms->D_lo, ms->ldm, sc);
  // [H~ D ; S D] (n x m layout): one GEMM over the stacked [H~; S]; the epilogue splits the result
  pf.begin(st);
  run_plan(ms, st, kPlanHD);
  pf.end(st, 4.0 * np * n * (double)m * m * tc::block_density(&ms->hs_blocks[tc::sparse_slot(ms->plan_shape[kPlanHD].bn)]),
         kPlanHD);
  // [H' | S' | H'' | S''] = D [HC; SC; HD; SD]^T (Eqs. 14-15)
  pf.begin(st);
  run_plan(ms, st, kPlanProj);
  pf.end(st, 8.0 * np * n * (double)n * m, kPlanProj);
  launch_traces(st, n, SWHW, Proj, part2, sc, /*fp32_products=*/true);
  launch_control_linesearch(st, sc, part2, traces_partials(n));
  // Eq. 16 and the footnote's updates of C, HC, SC; dHC, dSC; and their splits
  launch_update_state_split32(st, n, m, C, Y4, ms->Dir32, ms->HD32, ms->dY32, ms->Y_hi, ms->Y_lo, ms->ldm, sc);
  // H_W, S_W (Eq. 16) and the split of [dS_W | dH_W] into W
  launch_update_subspace_split(st, n, SWHW, Proj, ms->Wref, ms->W_hi + 2L * n, ms->W_lo + 2L * n, ms->ld4n, sc);
  // G = Gref + 8 dHC - 4 [S_W,ref | H_W,ref | dS_W | dH_W] [dHC; dSC; HC; SC] (Eq. 12 about the
  // refresh point), and its split for the next P G
  pf.begin(st);
  run_plan(ms, st, kPlanG);
  pf.end(st, 8.0 * np * n * (double)n * m, kPlanG);
}

void mixed_iterate_replay(MixedState* ms, cudaStream_t st, Scalars* sc, double* C, double* Dir, double* G,
                          double* Gold, double* PG, double* Y4, double* SWHW, double* Proj, double* part,
                          double* part2, const double* HS, const double* P, bool precond, Profiler& pf) {
  const bool capturable = st != nullptr && st != cudaStreamLegacy && st != cudaStreamPerThread;
  if (pf.on || !capturable || ms->ls_failed || ms->plan_sc != sc) {  // the first call builds the plans
    mixed_iterate(ms, st, sc, C, Dir, G, Gold, PG, Y4, SWHW, Proj, part, part2, HS, P, precond, pf);
    return;
  }
  const void* key[4] = {st, C, G, sc};
  if (ms->ls_exec && std::equal(key, key + 4, ms->ls_key)) {
    OMM_CUDA_TRY(cudaGraphLaunch(ms->ls_exec, st));
    return;
  }
  drop_graph(ms);
  cudaGraph_t graph = nullptr;
  bool ok = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
  if (ok) {
    try {
      mixed_iterate(ms, st, sc, C, Dir, G, Gold, PG, Y4, SWHW, Proj, part, part2, HS, P, precond, pf);
    } catch (...) {
      ok = false;
    }
    ok = (cudaStreamEndCapture(st, &graph) == cudaSuccess) && ok && graph != nullptr;
    ok = ok && cudaGraphInstantiate(&ms->ls_exec, graph, 0) == cudaSuccess;
  }
  if (graph) cudaGraphDestroy(graph);
  if (!ok) {  // no graph on this stream: launch eagerly from now on
    cudaGetLastError();
    ms->ls_exec = nullptr;
    ms->ls_failed = true;
    mixed_iterate(ms, st, sc, C, Dir, G, Gold, PG, Y4, SWHW, Proj, part, part2, HS, P, precond, pf);
    return;
  }
  std::copy(key, key + 4, ms->ls_key);
  OMM_CUDA_TRY(cudaGraphLaunch(ms->ls_exec, st));
}

}  // namespace omm
