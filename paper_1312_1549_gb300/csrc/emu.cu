// Float64-class contractions on the BF16 tensor cores by error-free
// fixed-point slicing (the Ozaki scheme: K. Ozaki, T. Ogita, S. Oishi,
// S. M. Rump, "Error-free transformations of matrix multiplication by using
// fast routines of matrix multiplication and its applications", Numerical
// Algorithms 59 (2012)), used by the mixed path to refresh its state.
//
// Slicing: every row r of an operand gets a power of two sigma_r > 2 max|x|
// over the row, and x = sigma_r * sum_i a_i 2^-5(i+1) + O(sigma_r 2^-5s) with
// integers |a_i| <= 16 (bf16 holds a_i * 2^k exactly). For a pair of slices
// (i, j) every product a b <= 256 units of 2^(e_r + f_c - 5(i+j+2)), so all
// products of one level d = i + j share one unit per output element and a
// level of (d+1) pairs summed over K stays an integer below (d+1) K 256
// units: exact in the FP32 accumulator while that is <= 2^24. Each launch
// therefore takes at most 2^24 / (256 K) pairs of one level (all pairs of a
// level for K <= 1638, nine for the Si512 contraction K = 6656), so every
// launch is exact and the float64 epilogue sums the launches. (Lumping
// several levels into one FP32 accumulator is not exact: the tensor cores'
// FP32 adder truncates, and those errors grow linearly with K — measured
// 1e-10 of |A||B| at K = 1000.) With s = 10 slices the result carries about
// 50 bits of each row-scaled operand.
#include "emu.cuh"
#include "tc_gemm.cuh"

#include <algorithm>
#include <new>

namespace omm {
namespace {

constexpr int kSliceBits = 5;

__device__ __forceinline__ bool stopped(const Scalars* sc) { return sc != nullptr && (sc->done | sc->halt); }

// One warp per row. The row scale sigma = 2^esig comes from the largest
// magnitude (compared as integer bit patterns). Each element becomes the
// integer N = rint(x 2^(5s - esig)) (|N| < 2^(5s-1); one float64 multiply by
// a power of two and one conversion), whose balanced base-32 digits
// a_{s-1}, ..., a_0 in [-16, 16] are peeled off on the integer pipe:
// x = sigma sum_i a_i 2^-5(i+1) + r, |r| <= sigma 2^-(5s+1). Slice i holds
// a_i 2^(esig - 5(i+1)), exact in bf16 (at most 5 significant bits).
__global__ void slice_rows_kernel(const double* __restrict__ src, long rows, long cols, long ld_src, int s,
                                  __nv_bfloat16* __restrict__ dst, long ld_dst, long slice_stride,
                                  const Scalars* sc) {
  if (stopped(sc)) return;
  const long row = (long)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= rows) return;
  const double* x = src + row * ld_src;
  unsigned long long mx = 0;  // |x| as bits: ordered like the magnitudes (finite values)
  for (long c = lane; c < cols; c += 32)
    mx = max(mx, (unsigned long long)__double_as_longlong(x[c]) & 0x7FFFFFFFFFFFFFFFull);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  int e = 0;  // max|x| < 2^e (frexp convention; 0 for an all-zero row)
  const int ebits = (int)(mx >> 52);
  if (ebits > 0) e = ebits - 1022;
  else if (mx != 0) frexp(__longlong_as_double((long long)mx), &e);  // subnormal maximum
  const int esig = e + 1;  // sigma = 2^esig > 2 max|x|
  __nv_bfloat16* out = dst + row * ld_dst;
  const double to_int = ldexp(1.0, kSliceBits * s - esig);
  for (long c = lane; c < cols; c += 32) {
    long long N = __double2ll_rn(x[c] * to_int);  // |x| 2^-esig < 1/2, so |N| < 2^(5s-1)
    for (int i = s - 1; i >= 0; --i) {
      long long a = N;
      if (i > 0) {
        a = ((N + 16) & 31) - 16;  // balanced digit in [-16, 15]
        N = (N - a) >> kSliceBits;
      }
      out[i * slice_stride + c] = __float2bfloat16_rn(ldexpf((float)a, esig - kSliceBits * (i + 1)));
    }
  }
}

// dst (cols x rows) = src^T, 32 x 32 shared-memory tiles
__global__ void transpose_kernel(const double* __restrict__ src, long rows, long cols, long ld_src,
                                 double* __restrict__ dst, long ld_dst) {
  __shared__ double tile[32][33];
  const long tiles_c = (cols + 31) / 32;
  const long r0 = (blockIdx.x / tiles_c) * 32, c0 = (blockIdx.x % tiles_c) * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int k = ty; k < 32; k += 8) {
    const long r = r0 + k, c = c0 + tx;
    tile[k][tx] = (r < rows && c < cols) ? src[r * ld_src + c] : 0.0;
  }
  __syncthreads();
  for (int k = ty; k < 32; k += 8) {
    const long c = c0 + k, r = r0 + tx;
    if (c < cols && r < rows) dst[c * ld_dst + r] = tile[tx][k];
  }
}

long round8(long x) { return (x + 7) / 8 * 8; }

template <typename T>
void alloc(T** p, size_t count, cudaStream_t st) {
  mem::alloc(p, count, st);
}

}  // namespace

namespace emu {

void slice_rows(cudaStream_t st, const double* src, long rows, long cols, long ld_src, int s,
                __nv_bfloat16* dst, long ld_dst, const Scalars* sc) {
  if (rows <= 0) return;
  const int warps = 8;
  const long blocks = (rows + warps - 1) / warps;
  slice_rows_kernel<<<(unsigned)blocks, warps * 32, 0, st>>>(src, rows, cols, ld_src, s, dst, ld_dst,
                                                               rows * ld_dst, sc);
  OMM_LAUNCH_CHECK();
}

void transpose(cudaStream_t st, const double* src, long rows, long cols, long ld_src, double* dst, long ld_dst) {
  const long blocks = ((rows + 31) / 32) * ((cols + 31) / 32);
  transpose_kernel<<<(unsigned)blocks, 256, 0, st>>>(src, rows, cols, ld_src, dst, ld_dst);
  OMM_LAUNCH_CHECK();
}

tc::PairList level_chunks(int K, int s) {
  // Every chunk holds at most g slice pairs of one level, so that its FP32 sum
  // of integer units stays below 2^24 and is exact; the float64 epilogue adds
  // the chunks, smallest level first.
  const long g_max = (1L << 24) / (256L * (K > 0 ? K : 1));
  const int g = (int)(g_max < 1 ? 1 : (g_max > tc::kMaxPairs ? tc::kMaxPairs : g_max));
  tc::PairList pl{};
  for (int d = s - 1; d >= 0; --d) {
    for (int i0 = 0; i0 <= d; i0 += g) {
      for (int i = i0; i <= d && i < i0 + g; ++i) {
        if (pl.n == tc::kMaxPairs) throw CudaError{cudaErrorInvalidValue, "emu: too many slice pairs"};
        pl.a[pl.n] = (unsigned char)i;
        pl.b[pl.n] = (unsigned char)(d - i);
        ++pl.n;
      }
      if (pl.nchunk == tc::kMaxChunks) throw CudaError{cudaErrorInvalidValue, "emu: too many chunks"};
      pl.chunk_end[pl.nchunk++] = (unsigned char)pl.n;
    }
  }
  return pl;
}

namespace {
thread_local Profiler* t_prof = nullptr;
}

void set_profiler(Profiler* p) { t_prof = p; }

void gemm(cudaStream_t st, const tc::Operand& A, const tc::Operand& B, int K, int s, const tc::Epilogue& ep,
          double* partial, long partial_capacity, const tc::BlockLists* sparse) {
  // one persistent launch: every output tile runs its chunks in order on one CTA (or, for a
  // product of few tiles with scratch given, every chunk on its own CTA, then one reduction)
  const tc::PairList pl = level_chunks(K, s);
  if (t_prof) t_prof->begin(st);
  tc::gemm_persistent(st, A, B, K, pl, ep, partial, partial_capacity, sparse);
  // issued tensor flops (only the visited K blocks of a block-sparse product)
  if (t_prof) t_prof->end(st, 2.0 * ep.M * (double)ep.N * K * pl.n * tc::block_density(sparse));
}

void gemm_split(cudaStream_t st, const tc::Operand& A, const tc::Operand& B, int K, const tc::Epilogue& ep) {
  if (t_prof) t_prof->begin(st);
  tc::gemm_persistent(st, A, B, K, tc::pairs_split3(), ep);
  if (t_prof) t_prof->end(st, 2.0 * ep.M * (double)ep.N * K * 3.0);
}

}  // namespace emu

struct EmuState {
  int m = 0, n = 0, s = 0;
  long ldm = 0, ld2n = 0;
  __nv_bfloat16* HSs = nullptr;  // s slices of [H~; S]     2m x m
  __nv_bfloat16* Cs = nullptr;   // s slices of C           n x m
  __nv_bfloat16* Ys = nullptr;   // s slices of [HC; SC]    2n x m
  __nv_bfloat16* Ws = nullptr;   // s slices of [S_W | H_W] n x 2n
  __nv_bfloat16* YTs = nullptr;  // s slices of [HC | SC]^T m x 2n
  double* T64 = nullptr;         // [HC; SC]^T in float64  m x 2n (also C^T and C^T S_W for D)
  __nv_bfloat16* CTs = nullptr;  // kDensitySlices slices of C^T          m x n
  __nv_bfloat16* XTs = nullptr;  // kDensitySlices slices of C^T S_W      m x n
  __nv_bfloat16* SWs = nullptr;  // kDensitySlices slices of S_W          n x n
  long ldn = 0;
  tc::Operand opHS, opC, opY, opW, opYT, opCT, opXT, opSW, opCTb;  // opCTb: C^T as a B operand
  int* err = nullptr;
  double* partial = nullptr;  // per-chunk sums of the products with few output tiles
  long partial_cap = 0;
  tc::BlockLists hs_blocks;   // block sparsity of [H~; S] (256-row blocks)
};

namespace {
// D needs |dD| <= 1e-7 at O(1) entries: 8 slices (40 bits) leave a wide margin
constexpr int kDensitySlices = 8;
}

EmuState* emu_create(cudaStream_t st, int m, int n, int slices, const double* HS) {
  EmuState* es = new EmuState();
  try {
    es->m = m;
    es->n = n;
    es->s = slices;
    es->ldm = round8(m);
    es->ld2n = round8(2L * n);
    const long s = slices, ldm = es->ldm, ld2n = es->ld2n;
    alloc(&es->HSs, (size_t)s * 2 * m * ldm, st);
    alloc(&es->Cs, (size_t)s * n * ldm, st);
    alloc(&es->Ys, (size_t)s * 2 * n * ldm, st);
    alloc(&es->Ws, (size_t)s * n * ld2n, st);
    alloc(&es->YTs, (size_t)s * m * ld2n, st);
    alloc(&es->T64, (size_t)m * 2 * n, st);
    es->ldn = round8(n);
    alloc(&es->CTs, (size_t)kDensitySlices * m * es->ldn, st);
    alloc(&es->XTs, (size_t)kDensitySlices * m * es->ldn, st);
    alloc(&es->SWs, (size_t)kDensitySlices * n * es->ldn, st);
    alloc(&es->err, 1, st);
    // the [S_W | H_W] product (n x 2n) is the one with few tiles; 11 chunks at most for K <= 16384
    es->partial_cap = std::min(11L * n * 2L * n, 1L << 25);
    alloc(&es->partial, (size_t)es->partial_cap, st);
    OMM_CUDA_TRY(cudaMemsetAsync(es->err, 0, sizeof(int), st));
    emu::slice_rows(st, HS, 2L * m, m, m, slices, es->HSs, ldm, nullptr);
    tc::block_lists(st, HS, 2L * m, m, m, 256, es->hs_blocks);
    es->opHS = tc::make_operand(es->HSs, 2L * m, m, ldm, slices, false);
    es->opC = tc::make_operand(es->Cs, n, m, ldm, slices, true);
    es->opY = tc::make_operand(es->Ys, 2L * n, m, ldm, slices, false);
    es->opW = tc::make_operand(es->Ws, n, 2L * n, ld2n, slices, true);
    es->opYT = tc::make_operand(es->YTs, m, 2L * n, ld2n, slices, false);
    es->opCT = tc::make_operand(es->CTs, m, n, es->ldn, kDensitySlices, true);
    es->opXT = tc::make_operand(es->XTs, m, n, es->ldn, kDensitySlices, true);
    es->opSW = tc::make_operand(es->SWs, n, n, es->ldn, kDensitySlices, false);
    es->opCTb = tc::make_operand(es->CTs, m, n, es->ldn, kDensitySlices, false);
  } catch (...) {
    emu_destroy(es, st);
    throw;
  }
  return es;
}

void emu_update_H(EmuState* es, cudaStream_t st, const double* HS) {
  emu::slice_rows(st, HS, 2L * es->m, es->m, es->m, es->s, es->HSs, es->ldm, nullptr);
  tc::block_lists(st, HS, 2L * es->m, es->m, es->m, 256, es->hs_blocks);
}

void emu_destroy(EmuState* es, cudaStream_t st) {
  if (!es) return;
  void* bufs[] = {es->HSs, es->Cs, es->Ys, es->Ws, es->YTs, es->T64, es->CTs, es->XTs, es->SWs, es->err, es->partial};
  for (void* b : bufs) mem::release(b, st);
  tc::free_block_lists(es->hs_blocks, st);
  delete es;
}

int emu_error(EmuState* es, cudaStream_t st) {
  int e = 0;
  OMM_CUDA_TRY(cudaMemcpyAsync(&e, es->err, sizeof(int), cudaMemcpyDeviceToHost, st));
  OMM_CUDA_TRY(cudaStreamSynchronize(st));
  return e;
}

// HC, SC, S_W, H_W, E~, G and max|G| from C with float64-class tensor-core products.
void emu_recompute_state(EmuState* es, cudaStream_t st, Scalars* sc, const double* C, double* Y4,
                         double* SWHW, double* G, double* part, double* part2) {
  const int m = es->m, n = es->n, s = es->s;
  const long nm = (long)n * m;
  emu::slice_rows(st, C, n, m, m, s, es->Cs, es->ldm, nullptr);
  // [HC; SC] (n x m layout) = C [H~; S]^T
  emu::gemm(st, es->opC, es->opHS, m, s, tc::Epilogue{Y4, m, m, nm, 1.0, 0.0, n, 2 * m, nullptr, es->err},
            es->partial, es->partial_cap, &es->hs_blocks);
  emu::slice_rows(st, Y4, 2L * n, m, m, s, es->Ys, es->ldm, nullptr);
  // [S_W | H_W] = C [SC; HC]^T
  emu::gemm(st, es->opC, es->opY, m, s,
            tc::Epilogue{SWHW + n, 2L * n, n, -(long)n, 1.0, 0.0, n, 2 * n, nullptr, es->err}, es->partial,
            es->partial_cap);
  launch_functional(st, n, SWHW, part2);
  launch_finish_functional(st, sc, part2, traces_blocks(n));
  // G = 8 HC - 4 [S_W | H_W] [HC; SC]
  emu::slice_rows(st, SWHW, n, 2L * n, 2L * n, s, es->Ws, es->ld2n, nullptr);
  emu::transpose(st, Y4, 2L * n, m, m, es->T64, 2L * n);
  emu::slice_rows(st, es->T64, m, 2L * n, 2L * n, s, es->YTs, es->ld2n, nullptr);
  launch_scale_copy(st, nm, Y4, 8.0, G, nullptr);
  emu::gemm(st, es->opW, es->opYT, 2 * n, s, tc::Epilogue{G, m, m, 0, -4.0, 1.0, n, m, nullptr, es->err},
            es->partial, es->partial_cap);
  launch_gmax(st, nm, G, part);
  launch_finish_gmax(st, sc, part);
}

}  // namespace omm

namespace omm {

namespace {
// out = a x + b y (float64, count elements)
__global__ void combine_kernel(long count, double a, const double* __restrict__ x, double b,
                               const double* __restrict__ y, double* out) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < count; i += (long)gridDim.x * blockDim.x)
    out[i] = fma(a, x[i], b * y[i]);
}
}  // namespace

// D = 2 C^T (2I - S_W) C (n x m layout of C), float64-class: X = C^T S_W from the sliced C^T and
// S_W, W = 4 C^T - 2 X in float64, then one sliced product D = W (C^T)^T. The B operand C^T is
// the same slice stack as the A operand, mapped with B-sized TMA boxes.
void emu_density(EmuState* es, cudaStream_t st, const double* C, const double* SWHW, double* D) {
  const int m = es->m, n = es->n, s = kDensitySlices;
  const long mn = (long)m * n;
  double* CT = es->T64;       // m x n
  double* XT = es->T64 + mn;  // m x n
  emu::transpose(st, C, n, m, m, CT, n);
  emu::slice_rows(st, CT, m, n, n, s, es->CTs, es->ldn, nullptr);
  emu::slice_rows(st, SWHW, n, n, 2L * n, s, es->SWs, es->ldn, nullptr);   // S_W is symmetric
  emu::gemm(st, es->opCT, es->opSW, n, s, tc::Epilogue{XT, n, n, 0, 1.0, 0.0, m, n, nullptr, es->err});
  combine_kernel<<<(unsigned)std::min<long>((mn + 255) / 256, 4096), 256, 0, st>>>(mn, 4.0, CT, -2.0, XT, XT);
  OMM_LAUNCH_CHECK();
  emu::slice_rows(st, XT, m, n, n, s, es->XTs, es->ldn, nullptr);
  emu::gemm(st, es->opXT, es->opCTb, n, s, tc::Epilogue{D, m, m, 0, 1.0, 0.0, m, m, nullptr, es->err});
}

// out = -(2 C^T H~_W C + eta D) given out = D (dE/dS at the minimum), float64-class:
// V = C^T H_W from the sliced C^T and H_W (C^T, sliced, as left by emu_density), then one
// sliced product out = -2 V (C^T)^T - eta out.
void emu_minus_edm(EmuState* es, cudaStream_t st, const double* SWHW, double eta, double* out) {
  const int m = es->m, n = es->n, s = kDensitySlices;
  double* VT = es->T64 + (long)m * n;  // m x n
  emu::slice_rows(st, SWHW + n, n, n, 2L * n, s, es->SWs, es->ldn, nullptr);  // H_W is symmetric
  emu::gemm(st, es->opCT, es->opSW, n, s, tc::Epilogue{VT, n, n, 0, 1.0, 0.0, m, n, nullptr, es->err});
  emu::slice_rows(st, VT, m, n, n, s, es->XTs, es->ldn, nullptr);
  emu::gemm(st, es->opXT, es->opCTb, n, s, tc::Epilogue{out, m, m, 0, -2.0, -eta, m, m, nullptr, es->err});
}

}  // namespace omm
