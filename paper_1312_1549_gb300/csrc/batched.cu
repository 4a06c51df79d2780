// Batched OMM: many independent (H, S) instances of uneven size (k-points,
// spins, snapshots) minimised together on one GPU.
//
// Each instance owns an ordinary mixed-precision context (setup, buffers,
// refresh and certificate code of omm_capi.cu / mixed.cu / emu.cu). The line
// searches of all instances advance in lockstep: every phase of a line search
// is ONE launch over the whole batch -- the four contractions are grouped
// tcgen05 GEMMs over the union of the instances' tiles, the vector and
// control work runs as batched kernels with the instance in blockIdx.y -- and
// the ~20 launches of one line search are captured once in a CUDA graph that
// is replayed. An instance that has converged, or waits for a refresh, masks
// itself out through its device flags, so the graph never changes. The host
// polls all status words with one copy every `check_every` replays and runs
// the per-instance refreshes (float64-class) and certificates (float64).
#include "fused_device.cuh"
#include "iter_device.cuh"
#include "omm_ctx.cuh"
#include "split_device.cuh"
#include "tc_gemm.cuh"

#include <chrono>
#include <algorithm>
#include <atomic>
#include <thread>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

namespace omm {
namespace {

constexpr int kBatchReduceBlocks = 64;  // gradient-reduction partials per instance (<= kReduceBlocks)

struct IterArgs {
  int n, m;
  long nm;
  int tiles;   // 32 x 32 tiles of an n x n matrix
  int nparts;  // partial sums of the P G epilogue (4 per epilogue warp and output tile)
  int precond;
  Scalars* sc;
  double *C, *G, *Gold, *Y4, *SWHW, *Proj, *part, *part2, *Wref, *red;
  float *Dir32, *PG32, *HD32, *dY32;  // float32 side quantities (leading dimension ldm)
  __nv_bfloat16 *D_hi, *Y_hi, *W_hi;
  long ldm, ld4;
};

// without a preconditioner: the Polak-Ribiere sums with PG = G (also writes PG and G_old)
__global__ void __launch_bounds__(dev::TB) b_reduce_unpreconditioned_kernel(const IterArgs* __restrict__ A) {
  const IterArgs& a = A[blockIdx.y];
  dev::reduce_unpreconditioned_body(a.n, a.m, a.G, a.Gold, a.Dir32, a.PG32, a.ldm, a.part, a.sc, blockIdx.x,
                                    gridDim.x);
}

// Polak-Ribiere coefficient and stopping tests: from the P G epilogue's partial sums, or (without a
// preconditioner) from the reduction kernel's
__global__ void __launch_bounds__(dev::TB) b_control_direction_kernel(const IterArgs* __restrict__ A) {
  const IterArgs& a = A[blockIdx.y];
  if (a.precond) dev::control_direction_body(a.sc, a.red, 1, a.nparts, 0, 1);
  else dev::control_direction_body(a.sc, a.part, 1, kBatchReduceBlocks, 0, 1);
}

// Delta and its split (the operand of the next two products)
__global__ void __launch_bounds__(256) b_direction_kernel(const IterArgs* __restrict__ A) {
  const IterArgs& a = A[blockIdx.y];
  dev::direction_split32_body(a.n, a.m, a.PG32, a.Dir32, a.D_hi, a.D_hi + (long)a.n * a.ldm, a.ldm, a.sc, blockIdx.x,
                              gridDim.x);
}

__global__ void __launch_bounds__(dev::TB) b_traces_kernel(const IterArgs* __restrict__ A) {
  const IterArgs& a = A[blockIdx.y];
  if ((int)blockIdx.x >= a.tiles) return;
  dev::traces_body<true>(a.n, a.SWHW, a.Proj, a.part2, a.sc, blockIdx.x, a.tiles);
}

__global__ void __launch_bounds__(dev::TB) b_control_linesearch_kernel(const IterArgs* __restrict__ A) {
  const IterArgs& a = A[blockIdx.y];
  dev::control_linesearch_body(a.sc, a.part2, a.tiles, 0, 1);
}

// the state update and the splits of the new dHC, dSC, HC, SC
__global__ void __launch_bounds__(256) b_update_state_kernel(const IterArgs* __restrict__ A) {
  const IterArgs& a = A[blockIdx.y];
  dev::update_state_split32_body(a.n, a.m, a.C, a.Y4, a.Dir32, a.HD32, a.dY32, a.Y_hi, a.Y_hi + 6L * a.n * a.ldm,
                                 a.ldm, a.sc, blockIdx.x, gridDim.x);
}

// H_W, S_W and the split of [dS_W | dH_W]
__global__ void __launch_bounds__(dev::TB) b_update_subspace_kernel(const IterArgs* __restrict__ A) {
  const IterArgs& a = A[blockIdx.y];
  if ((int)blockIdx.x >= a.tiles) return;
  dev::update_subspace_split_body(a.n, a.SWHW, a.Proj, a.Wref, a.W_hi + 2L * a.n, a.W_hi + (long)a.n * a.ld4 + 2L * a.n,
                                  a.ld4, a.sc, blockIdx.x, a.tiles);
}

struct Grouped {
  tc::GroupDesc* dev = nullptr;
  int ngroups = 0, tiles = 0;
  int bn = 256;       // output tile shape chosen by the autotuner
  bool pair = false;
  bool quad = false;
};

constexpr int kGroupedGemms = 4;
constexpr int kRefreshStreams = 32;  // the stopped instances' refreshes and certificates overlap on these

template <typename T>
void alloc(T** p, size_t count, cudaStream_t st) {
  mem::alloc(p, count, st);
}

}  // namespace
}  // namespace omm

using namespace omm;

struct omm_batch {
  int count = 0;
  cudaStream_t st = nullptr;
  omm_opts opts{};
  std::vector<omm_ctx*> ctx;
  Scalars* sc_all = nullptr;       // device, count entries (each context's sc points here)
  Scalars* sc_host_all = nullptr;  // pinned
  IterArgs* args = nullptr;        // device
  Grouped gPG, gHD, gPr, gG;
  int max_rows = 0;        // largest 2n (vector-kernel grid)
  int max_tiles = 0;       // largest n x n tile count
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  bool precond = true;
  int* err = nullptr;  // bounded-wait failures of the grouped GEMMs
  // with opts.profile the line searches are launched eagerly instead of replayed, and
  // the grouped GEMMs (PG, [HD; SD], projections, gradient) are timed with CUDA events
  bool profile = false;
  Profiler prof;
  int tile_width[4] = {256, 256, 256, 256};  // autotuned shapes of the P G, [HD; SD], projection, G GEMMs
                                             // (width, + 1000 for 256-row tiles on SM pairs, + 2000 on
                                             // clusters of two pairs sharing A)
  double ms_autotune = 0.0;
  // refreshes and certificates of different instances run concurrently on these
  cudaStream_t pool[kRefreshStreams] = {};
  std::vector<double> gemm_flop[kGroupedGemms];  // issued flops of each instance's group
};

int omm::batch_count(const omm_batch* b) { return b ? b->count : 0; }

namespace {

void batch_destroy(omm_batch* b) {
  if (!b) return;
  if (b->st) cudaStreamSynchronize(b->st);
  for (cudaStream_t& q : b->pool)
    if (q) {
      cudaStreamSynchronize(q);
      cudaStreamDestroy(q);
    }
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  for (omm_ctx* c : b->ctx) {
    if (c && b->sc_all && c->sc >= b->sc_all && c->sc < b->sc_all + b->count) {
      c->sc = nullptr;  // the status words belong to the batch
      c->sc_host = nullptr;
    }
    destroy(c);
  }
  for (Grouped* g : {&b->gPG, &b->gHD, &b->gPr, &b->gG}) mem::release(g->dev, b->st);
  mem::release(b->args, b->st);
  mem::release(b->err, b->st);
  mem::release(b->sc_all, b->st);
  if (b->sc_host_all) cudaFreeHost(b->sc_host_all);
  delete b;
}

void upload_groups(cudaStream_t st, Grouped* g, const std::vector<tc::GroupDesc>& v) {
  g->ngroups = (int)v.size();
  if (v.empty()) return;
  g->tiles = v.back().tile_begin + tc::tiles_of(v.back().ep, v.back().bn, v.back().pair != 0, v.back().quad != 0);
  g->bn = v.back().bn;
  g->pair = v.back().pair != 0;
  g->quad = v.back().quad != 0;
  alloc(&g->dev, v.size(), st);
  OMM_CUDA_TRY(cudaMemcpyAsync(g->dev, v.data(), v.size() * sizeof(tc::GroupDesc), cudaMemcpyHostToDevice, st));
}

void timed_gemm(omm_batch* b, const Grouped& g, const tc::PairList& pl) {
  b->prof.begin(b->st);
  tc::gemm_persistent(b->st, g.dev, g.ngroups, g.tiles, pl, b->err, g.bn, g.pair, g.quad);
  b->prof.end(b->st, 0.0);
}

// one line search of every instance (captured into the graph)
void enqueue_line_search(omm_batch* b) {
  cudaStream_t st = b->st;
  const unsigned cnt = (unsigned)b->count;
  const dim3 rows_grid((unsigned)std::min(b->max_rows, 1024), cnt);
  const tc::PairList pl = tc::pairs_split3();
  if (b->precond) {
    timed_gemm(b, b->gPG, tc::pairs_single());  // P G (one bf16 pass), the Polak-Ribiere products and max|G|, G_old <- G
  } else {
    b_reduce_unpreconditioned_kernel<<<dim3(kBatchReduceBlocks, cnt), dev::TB, 0, st>>>(b->args);
    OMM_LAUNCH_CHECK();
  }
  b_control_direction_kernel<<<dim3(1, cnt), dev::TB, 0, st>>>(b->args);
  OMM_LAUNCH_CHECK();
  b_direction_kernel<<<rows_grid, 256, 0, st>>>(b->args);
  OMM_LAUNCH_CHECK();
  timed_gemm(b, b->gHD, pl);  // [H D; S D] and its split
  timed_gemm(b, b->gPr, pl);
  b_traces_kernel<<<dim3(b->max_tiles, cnt), dev::TB, 0, st>>>(b->args);
  OMM_LAUNCH_CHECK();
  b_control_linesearch_kernel<<<dim3(1, cnt), dev::TB, 0, st>>>(b->args);
  OMM_LAUNCH_CHECK();
  b_update_state_kernel<<<rows_grid, 256, 0, st>>>(b->args);
  OMM_LAUNCH_CHECK();
  b_update_subspace_kernel<<<dim3(b->max_tiles, cnt), dev::TB, 0, st>>>(b->args);
  OMM_LAUNCH_CHECK();
  timed_gemm(b, b->gG, pl);  // G and its split
}

// start a mixed round of instance i from its current (just recomputed) state
void begin_round(omm_batch* b, int i, double g_ref, int iter_total) {
  omm_ctx* c = b->ctx[i];
  Scalars& h = *c->sc_host;
  const double E_keep = h.E, g_keep = h.gmax;
  reset_loop_flags(c, false);
  h.E = E_keep;
  h.gmax = g_keep;
  h.iter = iter_total;
  h.halt_gmax = std::max(c->opts.tol_grad * 0.5, g_ref * c->opts.refine_ratio);
  write_scalars(c);
  mixed_sync_state(c->mixed, c->st, c->Y4, c->SWHW, c->G);
}

}  // namespace

extern "C" {

omm_status omm_create_batched(int count, const int* m, const int* n, const double* const* H,
                              const double* const* S, const double* const* T, const double* eta,
                              const double* tau, const omm_opts* opts, void* stream, omm_batch** out) {
  if (out) *out = nullptr;
  if (!out || count <= 0 || !m || !n || !H || !S || !eta || !tau)
    return fail(OMM_ERR_ARG, "omm_create_batched: invalid argument");
  omm_batch* b = new (std::nothrow) omm_batch();
  if (!b) return fail(OMM_ERR_OOM, "omm_create_batched: host allocation");
  b->count = count;
  b->st = (cudaStream_t)stream;
  omm_opts o{};
  if (opts) o = *opts;
  b->opts = o;
  b->precond = o.no_precondition == 0 && o.cholesky == 0;
  b->ctx.assign(count, nullptr);
  // per-instance setup (float64 Cholesky inverse etc.) from several host threads, each on its
  // own stream, so that the small factorisations of different instances overlap on the GPU
  {
    const int nthreads = std::min(count, 8);
    std::vector<omm_status> rcs(count, OMM_OK);
    std::vector<std::string> msgs(count);
    std::atomic<int> next{0};
    int device = 0;
    cudaGetDevice(&device);
    auto worker = [&]() {
      cudaSetDevice(device);
      cudaStream_t s = nullptr;
      if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) s = nullptr;
      for (int i = next++; i < count; i = next++) {
        rcs[i] = omm_create(m[i], n[i], H[i], S[i], T ? T[i] : nullptr, eta[i], tau[i], &o, s, &b->ctx[i]);
        if (rcs[i] != OMM_OK) msgs[i] = omm_last_error();
        else b->ctx[i]->st = b->st;  // from now on everything is ordered on the batch stream
      }
      if (s) {
        cudaStreamSynchronize(s);
        cudaStreamDestroy(s);
      }
    };
    std::vector<std::thread> pool;
    for (int k = 0; k < nthreads; ++k) pool.emplace_back(worker);
    for (auto& th : pool) th.join();
    for (int i = 0; i < count; ++i)
      if (rcs[i] != OMM_OK) {
        const std::string msg = std::string("omm_create_batched: instance ") + std::to_string(i) + ": " + msgs[i];
        const omm_status rc = rcs[i];
        batch_destroy(b);
        return fail(rc, msg);
      }
  }
  if (o.precision != OMM_PREC_MIXED) {
    *out = b;  // float64 batches solve instance by instance
    return OMM_OK;
  }
  try {
    alloc(&b->sc_all, count, b->st);
    OMM_CUDA_TRY(cudaMallocHost((void**)&b->sc_host_all, count * sizeof(Scalars)));
    std::vector<IterArgs> args(count);
    std::vector<tc::GroupDesc> gpg, ghd, gpr, gg;
    std::vector<tc::GemmSpec> spg, shd, spr, sg;
    for (int i = 0; i < count; ++i) {
      omm_ctx* c = b->ctx[i];
      mem::release(c->sc, b->st);
      c->sc = b->sc_all + i;
      cudaFreeHost(c->sc_host);
      c->sc_host = b->sc_host_all + i;
      const MixedView v = mixed_view(c->mixed);
      const int mi = c->m, ni = c->n;
      const long nm = (long)ni * mi;
      IterArgs& a = args[i];
      a.n = ni;
      a.m = mi;
      a.nm = nm;
      a.tiles = traces_blocks(ni);
      a.precond = b->precond;
      a.sc = c->sc;
      a.C = c->C; a.G = c->G; a.Gold = c->Gold; a.Y4 = c->Y4;
      a.SWHW = c->SWHW; a.Proj = c->Proj; a.part = c->part; a.part2 = c->part2;
      a.Wref = v.Wref; a.red = v.red;
      a.Dir32 = v.Dir32; a.PG32 = v.PG32; a.HD32 = v.HD32; a.dY32 = v.dY32;
      a.D_hi = v.D_hi; a.Y_hi = v.Y_hi; a.W_hi = v.W_hi;
      a.ldm = v.ldm;
      a.ld4 = v.ld4;
      tc::Epilogue ep[4];
      mixed_epilogues(c->mixed, c->sc, c->G, c->Gold, c->Y4, c->Proj, ep);
      if (b->precond) spg.push_back(tc::GemmSpec{v.opG, v.opP, mi, ep[0]});
      tc::GemmSpec hd{v.opD, v.opHS, mi, ep[1]};
      for (int q = 0; q < 3; ++q) hd.sparse[q] = &v.hs_blocks[q];
      shd.push_back(hd);
      spr.push_back(tc::GemmSpec{v.opD, v.opYproj, mi, ep[2]});
      sg.push_back(tc::GemmSpec{v.opW, v.opYgrad, 4 * ni, ep[3]});
      // issued tensor flops, 3 x 2 M N K (3-term split; 2 M N K for the single-pass P G), of this
      // instance's share of each GEMM
      const double issued = 3.0 * 2.0 * ni;  // x N x K
      b->gemm_flop[0].push_back(b->precond ? issued / 3.0 * mi * mi : 0.0);
      b->gemm_flop[1].push_back(issued * 2.0 * mi * mi);
      b->gemm_flop[2].push_back(issued * 4.0 * ni * mi);
      b->gemm_flop[3].push_back(issued * mi * 4.0 * ni);
      b->max_rows = std::max(b->max_rows, 2 * ni);
      b->max_tiles = std::max(b->max_tiles, a.tiles);
    }
    // Tile width of each grouped GEMM from the autotuner (timed once per batch shape in a
    // process); then longest tiles first: a persistent CTA takes tiles b, b + grid, ..., so
    // ordering the groups by falling contraction length spreads the long tiles over all SMs
    // before the short ones fill in (the largest-processing-time-first rule)
    const std::vector<tc::GemmSpec>* specs[4] = {&spg, &shd, &spr, &sg};
    std::vector<tc::GroupDesc>* groups[4] = {&gpg, &ghd, &gpr, &gg};
    for (int k = 0; k < 4; ++k) {
      if (specs[k]->empty()) continue;
      double ms_tune = 0.0;
      const tc::TileShape ts =
          tc::choose_tile_shape(b->st, *specs[k], k == 0 ? tc::pairs_single() : tc::pairs_split3(), &ms_tune);
      b->ms_autotune += ms_tune;
      b->tile_width[k] = ts.code();
      for (size_t i = 0; i < specs[k]->size(); ++i) {
        const tc::GemmSpec& sp = (*specs[k])[i];
        const tc::BlockLists* bl = ts.quad ? nullptr : sp.sparse[tc::sparse_slot(ts.bn)];
        groups[k]->push_back(tc::make_group(*sp.A, *sp.B, sp.K, sp.ep, 0, ts.bn, bl, ts.pair, ts.quad));
        if (bl && k == 1) b->gemm_flop[1][i] *= tc::block_density(bl);  // issued flops of the visited blocks
      }
      if (k == 0)  // partial sums each instance's P G epilogue leaves for its direction step
        for (int i = 0; i < count; ++i) args[i].nparts = tc::reduce_slots((*specs[k])[i].ep, ts);
      std::stable_sort(groups[k]->begin(), groups[k]->end(),
                       [](const tc::GroupDesc& x, const tc::GroupDesc& y) { return x.K > y.K; });
      int t = 0;
      for (tc::GroupDesc& g : *groups[k]) {
        g.tile_begin = t;
        t += tc::tiles_of(g.ep, g.bn, g.pair != 0, g.quad != 0);
      }
    }
    for (cudaStream_t& q : b->pool) OMM_CUDA_TRY(cudaStreamCreateWithFlags(&q, cudaStreamNonBlocking));
    alloc(&b->args, count, b->st);
    alloc(&b->err, 1, b->st);
    OMM_CUDA_TRY(cudaMemsetAsync(b->err, 0, sizeof(int), b->st));
    OMM_CUDA_TRY(cudaMemcpyAsync(b->args, args.data(), count * sizeof(IterArgs), cudaMemcpyHostToDevice, b->st));
    upload_groups(b->st, &b->gPG, gpg);
    upload_groups(b->st, &b->gHD, ghd);
    upload_groups(b->st, &b->gPr, gpr);
    upload_groups(b->st, &b->gG, gg);
    OMM_CUDA_TRY(cudaStreamSynchronize(b->st));
    // capture one line search of the whole batch
    tc::prepare_persistent();
    cudaStream_t cap = nullptr;
    OMM_CUDA_TRY(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    cudaStream_t saved = b->st;
    b->st = cap;
    OMM_CUDA_TRY(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
    try {
      enqueue_line_search(b);
    } catch (...) {
      cudaGraph_t g = nullptr;
      cudaStreamEndCapture(cap, &g);
      if (g) cudaGraphDestroy(g);
      b->st = saved;
      cudaStreamDestroy(cap);
      throw;
    }
    OMM_CUDA_TRY(cudaStreamEndCapture(cap, &b->graph));
    b->st = saved;
    OMM_CUDA_TRY(cudaStreamDestroy(cap));
    OMM_CUDA_TRY(cudaGraphInstantiate(&b->exec, b->graph, 0));
  } catch (const std::bad_alloc&) {
    batch_destroy(b);
    return fail(OMM_ERR_OOM, "omm_create_batched: device allocation failed");
  } catch (const CudaError& e) {
    batch_destroy(b);
    return fail(OMM_ERR_CUDA, std::string("omm_create_batched: ") + e.what + ": " + cudaGetErrorString(e.err));
  }
  *out = b;
  return OMM_OK;
}

omm_status omm_solve_batched(omm_batch* b, const double* const* C0, double* const* C, double* E, omm_info* info) {
  if (!b || !C0) return fail(OMM_ERR_ARG, "omm_solve_batched: NULL argument");
  const int cnt = b->count;
  for (int i = 0; i < cnt; ++i)
    if (b->ctx[i]->hermitian)
      return fail(OMM_ERR_ARG, "omm_solve_batched: Hermitian batch (use omm_solve_hermitian_batched)");
  if (b->opts.precision != OMM_PREC_MIXED) {
    // float64: instance after instance through the single-instance path
    omm_status worst = OMM_OK;
    for (int i = 0; i < cnt; ++i) {
      double e = 0.0;
      omm_info inf{};
      const omm_status rc = omm_solve(b->ctx[i], C0[i], C ? C[i] : nullptr, &e, nullptr, &inf);
      if (E) E[i] = e;
      if (info) info[i] = inf;
      if (rc != OMM_OK && worst == OMM_OK) worst = rc;
    }
    return worst == OMM_OK ? OMM_OK : fail(worst, "omm_solve_batched: at least one instance failed");
  }
  std::vector<int> finished(cnt, 0), rounds(cnt, 0), refinements(cnt, 0), energy_stop(cnt, 0);
  std::vector<int> iter_total(cnt, 0), last_done(cnt, 0), round_start(cnt, 0);
  std::vector<omm_status> result(cnt, OMM_OK);
  std::vector<double> ms_ref(cnt, 0.0), ms_cert(cnt, 0.0);
  std::vector<int> iter_before(cnt, 0);
  std::vector<char> active(cnt, 0);
  omm_status worst = OMM_OK;
  cudaEvent_t e0 = nullptr, e1 = nullptr, g0 = nullptr, g1 = nullptr;
  float ms_total = 0.f;
  double ms_graph = 0.0, gemm_flop = 0.0, ms_refresh_wall = 0.0;
  const bool profile = b->opts.profile != 0;
  try {
    OMM_CUDA_TRY(cudaEventCreate(&e0));
    OMM_CUDA_TRY(cudaEventCreate(&e1));
    OMM_CUDA_TRY(cudaEventCreate(&g0));
    OMM_CUDA_TRY(cudaEventCreate(&g1));
    b->prof.reset();
    OMM_CUDA_TRY(cudaEventRecord(e0, b->st));
    for (int i = 0; i < cnt; ++i) {
      omm_ctx* c = b->ctx[i];
      c->solved = false;
      copy_in(c->C, C0[i], (size_t)c->n * c->m, b->st);
      if (c->red) {  // C_r = L^T C0 (Sec. 2.4)
        reduce_coefficients(c->red, b->st, c->n, c->C, c->Dir);
        OMM_CUDA_TRY(cudaMemcpyAsync(c->C, c->Dir, (size_t)c->n * c->m * sizeof(double), cudaMemcpyDeviceToDevice,
                                     b->st));
      }
      reset_loop_flags(c, true);
      write_scalars(c);
      mixed_recompute_state(c->mixed, b->st, c->sc, c->C, c->Y4, c->SWHW, c->G, c->part, c->part2);
    }
    OMM_CUDA_TRY(cudaMemcpyAsync(b->sc_host_all, b->sc_all, cnt * sizeof(Scalars), cudaMemcpyDeviceToHost, b->st));
    OMM_CUDA_TRY(cudaStreamSynchronize(b->st));
    for (int i = 0; i < cnt; ++i) {
      const Scalars& h = b->sc_host_all[i];
      if (!std::isfinite(h.gmax) || !std::isfinite(h.E)) {
        finished[i] = 1;
        result[i] = OMM_ERR_NONFINITE;
        b->sc_host_all[i].done = 1;
        write_scalars(b->ctx[i]);
        continue;
      }
      begin_round(b, i, h.gmax, 0);
    }
    // profiling reads the GEMM events after every replay
    const int check = profile ? 1 : b->ctx[0]->opts.check_every;
    for (int poll = 0;; ++poll) {
      int unfinished = 0;
      for (int i = 0; i < cnt; ++i) {
        unfinished += !finished[i];
        const Scalars& h = b->sc_host_all[i];
        active[i] = !finished[i] && !(h.done || h.halt || h.status);
        iter_before[i] = h.iter;
      }
      if (unfinished == 0) break;
      OMM_CUDA_TRY(cudaEventRecord(g0, b->st));
      for (int k = 0; k < check; ++k) {
        if (profile) {
          b->prof.on = true;
          enqueue_line_search(b);  // the captured launches, issued eagerly and timed
          b->prof.on = false;
        } else {
          OMM_CUDA_TRY(cudaGraphLaunch(b->exec, b->st));
        }
      }
      OMM_CUDA_TRY(cudaEventRecord(g1, b->st));
      OMM_CUDA_TRY(cudaMemcpyAsync(b->sc_host_all, b->sc_all, cnt * sizeof(Scalars), cudaMemcpyDeviceToHost, b->st));
      OMM_CUDA_TRY(cudaStreamSynchronize(b->st));
      ms_graph += elapsed(g0, g1);
      if (profile) {
        b->prof.collect();
        // an instance that completed its line search ran all four products; one that
        // stopped at the convergence test after the preconditioner ran only the first
        for (int i = 0; i < cnt; ++i) {
          if (!active[i]) continue;
          const bool full = b->sc_host_all[i].iter > iter_before[i];
          for (int w = 0; w < (full ? kGroupedGemms : 1); ++w) gemm_flop += b->gemm_flop[w][i];
        }
      }
      // pass 1: instances that stopped get their refresh (float64-class) or certificate
      // (float64-class, or native float64 on request) enqueued, spread over the pool
      // streams so that the small instances' products overlap on the GPU
      const auto t_pass = std::chrono::steady_clock::now();
      std::vector<int> todo;
      for (int i = 0; i < cnt; ++i) {
        if (finished[i]) continue;
        omm_ctx* c = b->ctx[i];
        Scalars& h = *c->sc_host;
        const bool capped = h.iter - round_start[i] >= kMixedRound;
        if (!(h.done || h.halt || h.status || capped)) continue;
        iter_total[i] = h.iter;
        if (h.status != 0) {
          result[i] = (omm_status)h.status;
          finished[i] = 1;
          if (result[i] == OMM_ERR_NO_CONVERGENCE) {
            // certify what the capped instance has: the float64 recompute's E~ and max|G| are
            // read back before the host flags go down again (they would overwrite them)
            project_real_form(c, c->st);
            recompute_state_fp64(c);
            read_scalars(c);
          }
          h.done = 1;
          write_scalars(c);
          continue;
        }
        if (h.done && h.stop_reason == 2) energy_stop[i] = 1;
        last_done[i] = h.done != 0;
        const bool native = (last_done[i] && c->opts.native_certificate != 0) || c->emu == nullptr;
        cudaStream_t q = b->pool[todo.size() % kRefreshStreams];
        c->st = q;
        OMM_CUDA_TRY(cudaEventRecord(c->ev[0], q));
        project_real_form(c, q);
        if (native) recompute_state_fp64(c);
        else emu_recompute_state(c->emu, q, c->sc, c->C, c->Y4, c->SWHW, c->G, c->part, c->part2);
        OMM_CUDA_TRY(cudaEventRecord(c->ev[1], q));
        c->st = b->st;
        todo.push_back(i);
      }
      if (todo.empty()) continue;
      for (cudaStream_t q : b->pool) OMM_CUDA_TRY(cudaStreamSynchronize(q));
      OMM_CUDA_TRY(cudaMemcpyAsync(b->sc_host_all, b->sc_all, cnt * sizeof(Scalars), cudaMemcpyDeviceToHost, b->st));
      OMM_CUDA_TRY(cudaStreamSynchronize(b->st));
      // pass 2: read the recomputed states and start the next rounds
      for (int i : todo) {
        omm_ctx* c = b->ctx[i];
        Scalars& h = *c->sc_host;
        const bool certify = last_done[i] != 0;
        const bool native = (certify && c->opts.native_certificate != 0) || c->emu == nullptr;
        if (!native && emu_error(c->emu, b->st) != 0) {
          result[i] = OMM_ERR_TIMEOUT;
          finished[i] = 1;
          h.done = 1;
          write_scalars(c);
          continue;
        }
        (certify ? ms_cert : ms_ref)[i] += elapsed(c->ev[0], c->ev[1]);
        ++rounds[i];
        if (!std::isfinite(h.gmax) || !std::isfinite(h.E)) {
          result[i] = OMM_ERR_NONFINITE;
          finished[i] = 1;
        } else if (certify && (h.gmax < c->opts.tol_grad || energy_stop[i])) {
          finished[i] = 1;
          c->solved = true;
        } else if (rounds[i] > 64 || h.iter >= c->opts.max_iter) {
          result[i] = OMM_ERR_NO_CONVERGENCE;
          finished[i] = 1;
        }
        if (finished[i]) {
          h.done = 1;
          write_scalars(c);
          continue;
        }
        ++refinements[i];
        round_start[i] = h.iter;
        begin_round(b, i, h.gmax, h.iter);
      }
      ms_refresh_wall += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_pass).count();
    }
    OMM_CUDA_TRY(cudaEventRecord(e1, b->st));
    OMM_CUDA_TRY(cudaEventSynchronize(e1));
    cudaEventElapsedTime(&ms_total, e0, e1);
    int gerr = 0;
    OMM_CUDA_TRY(cudaMemcpy(&gerr, b->err, sizeof(int), cudaMemcpyDeviceToHost));
    if (gerr != 0) {
      for (cudaEvent_t ev : {e0, e1, g0, g1}) cudaEventDestroy(ev);
      return fail(OMM_ERR_TIMEOUT, "omm_solve_batched: a bounded device wait expired in a grouped GEMM");
    }
    for (int i = 0; i < cnt; ++i) {
      omm_ctx* c = b->ctx[i];
      const Scalars& h = *c->sc_host;
      if (c->red && (result[i] == OMM_OK || result[i] == OMM_ERR_NO_CONVERGENCE)) {  // C = L^-T C_r
        restore_coefficients(c->red, b->st, c->n, c->C, c->Dir);
        OMM_CUDA_TRY(cudaMemcpyAsync(c->C, c->Dir, (size_t)c->n * c->m * sizeof(double), cudaMemcpyDeviceToDevice,
                                     b->st));
        if (reduction_error(c->red, b->st) != 0) {
          result[i] = OMM_ERR_TIMEOUT;
          c->solved = false;
        }
      }
      if ((result[i] == OMM_OK || result[i] == OMM_ERR_NO_CONVERGENCE) && C && C[i])
        OMM_CUDA_TRY(cudaMemcpyAsync(C[i], c->C, (size_t)c->n * c->m * sizeof(double), cudaMemcpyDefault, b->st));
      if (E) E[i] = h.E + 2.0 * c->n * c->eta;
      if (info) {
        omm_info inf{};
        inf.status = result[i];
        inf.iterations = h.iter;
        inf.refinements = refinements[i];
        inf.E = h.E + 2.0 * c->n * c->eta;
        inf.Etilde = h.E;
        inf.gmax = h.gmax;
        inf.ms_setup = c->ms_setup;
        inf.ms_precond = c->ms_precond;
        for (int k = 0; k < 4; ++k) inf.tile_width[k] = (k == 0 && !b->precond) ? 0 : b->tile_width[k];
        inf.ms_autotune = b->ms_autotune;
        inf.ms_refine = ms_ref[i] + ms_cert[i];
        inf.ms_certify = ms_cert[i];
        // batch totals, shared by all instances: the replayed line searches and, with
        // opts.profile, the grouped tensor-core GEMMs inside them
        inf.ms_iterate = ms_graph;
        inf.ms_batch = ms_total;
        inf.ms_batch_refresh = ms_refresh_wall;
        inf.ms_main_gemm = b->prof.ms;
        inf.main_gemm_launches = (double)b->prof.launches;
        inf.main_gemm_flop = gemm_flop;
        info[i] = inf;
      }
      if (result[i] != OMM_OK && worst == OMM_OK) worst = result[i];
    }
    OMM_CUDA_TRY(cudaStreamSynchronize(b->st));
  } catch (const CudaError& e) {
    for (cudaEvent_t ev : {e0, e1, g0, g1})
      if (ev) cudaEventDestroy(ev);
    return fail(OMM_ERR_CUDA, std::string("omm_solve_batched: ") + e.what + ": " + cudaGetErrorString(e.err));
  }
  for (cudaEvent_t ev : {e0, e1, g0, g1}) cudaEventDestroy(ev);
  if (worst != OMM_OK) return fail(worst, "omm_solve_batched: at least one instance failed");
  return OMM_OK;
}

omm_ctx* omm_batch_instance(omm_batch* b, int i) {
  if (!b || i < 0 || i >= b->count) return nullptr;
  return b->ctx[i];
}

void omm_free_batched(omm_batch* b) { batch_destroy(b); }

}  // extern "C"
