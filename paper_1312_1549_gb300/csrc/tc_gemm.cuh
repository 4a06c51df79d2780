// BF16 tensor-core GEMM (tcgen05 + TMEM + TMA) with a float64 epilogue.
#pragma once
#include <cuda_bf16.h>
#include <vector>
#include "omm_internal.cuh"

namespace omm {
namespace tc {

// Storage for a CUtensorMap (128 bytes, 64-byte aligned) without exposing cuda.h.
struct alignas(64) TensorMap {
  unsigned char bytes[128];
};

// A bf16 operand made of `slices` row-major matrices (rows x cols each, the
// contracted dimension is cols) stacked vertically in one allocation with
// leading dimension ld: slice i starts at row i * slice_rows (slice_rows = rows
// unless the operand is a view of a taller stack) and the operand's own rows
// start at row_off inside each slice. A split pair x = hi + lo is the 2-slice
// stack [hi; lo].
// An MN-major operand (B role only) is stored the other way round: its rows are
// the contracted index and its columns the output columns (K x N, row-major);
// it is loaded in 64 x 64 boxes and handed to the MMA as an MN-major matrix.
struct Operand {
  TensorMap map;       // boxes of 128 rows (A role), 256 rows (B role) or 64 x 64 (MN-major)
  TensorMap map_n128;  // boxes of 128 rows (as a B operand of 128-wide output tiles)
  const __nv_bfloat16* base = nullptr;  // the stack (maps of other box heights are made from it)
  long ld = 0;
  long map_rows = 0;   // rows of the whole stack
  int box_rows = 0;    // rows of the boxes of `map`
  long rows = 0, cols = 0;
  int slices = 1;
  long slice_rows = 0;  // rows between slices
  int row_off = 0;      // first row of the operand inside each slice
  bool mn_major = false;
};

// Which slice products one GEMM accumulates. With nchunk > 0 the pairs are cut
// into consecutive chunks: chunk c holds pairs [chunk_end[c-1], chunk_end[c]),
// is summed in an FP32 accumulator of its own and added to the float64 output
// by its own epilogue pass, in chunk order (the first pass with the Epilogue's
// beta, the later ones with beta = 1). nchunk = 0: all pairs form one chunk.
// Chunks are honoured by the persistent launch only.
constexpr int kMaxPairs = 64;
constexpr int kMaxChunks = 32;
struct PairList {
  int n;
  unsigned char a[kMaxPairs];
  unsigned char b[kMaxPairs];
  int nchunk;
  unsigned char chunk_end[kMaxChunks];
};
PairList pairs_split3();   // A_hi B_hi + A_hi B_lo + A_lo B_hi
PairList pairs_single();   // A_0 B_0

// C (float64) = alpha * acc + beta * C over the valid M x N block. Output
// column j goes to C + (j / split_cols) * split_stride + row * ldc + j % split_cols
// (split_cols = N for a plain matrix), so one GEMM can fill several stacked
// matrices. When skip[0] | skip[1] (the solver's done/halt flags) the kernel
// does nothing. err receives a nonzero code if a bounded wait expired.
//
// Fused forms (mode), all with split_cols = N unless stated:
//   kEpPlain   the above; with c_f32 C is float32 and receives alpha * acc (beta is not used;
//              split_cols and split_stride apply, in float elements).
//   kEpGrad    C = x0 + (xs * x1f + alpha * acc)   (the incremental gradient about a refresh
//              point: x0 = G_ref (float64), x1f = dHC (float32), xs = 8, alpha = -4; the
//              increment is formed in float32 with one rounding, then added in float64)
//   kEpReduce  C = acc as float32 (c_f32 = 1, alpha = 1), and with g = x0, g_old = x1 (float64,
//              rounded to float32 for the sums, which run in float32 over 16 columns at a time),
//              d = x2f (float32) the sums <g, C>, <g_old, C>, <g, d> (the last two only when
//              sc->have_dir) and max|g| of each epilogue warp's rows of the tile go to
//              part[(tile * 4 + warp) * 4 + 0..3]; then xout = g (xout may alias x1: every
//              element is read before it is written).
// Element (row, col) of x0, x1, xout is at row * ldx + col, of x1f, x2f at row * ldf + col.
// bf_hi != null (any mode): the stored value is also split into bf16 hi and lo, written to
// bf_hi + blk * bf_blk + row * bf_ld + col % split_cols and the same plus bf_lo.
// expire != 0 (tests only): before it issues any copy or MMA the kernel waits about 1 ms on a
// barrier that nothing arrives at, reports the expired wait in err and does nothing else.
enum { kEpPlain = 0, kEpGrad = 1, kEpReduce = 2 };
struct Epilogue {
  double* C;
  long ldc;
  long split_cols;
  long split_stride;
  double alpha;
  double beta;
  int M;
  int N;
  const int* skip;
  int* err;
  int mode = kEpPlain;
  int c_f32 = 0;
  const double* x0 = nullptr;
  const double* x1 = nullptr;
  double* xout = nullptr;
  long ldx = 0;
  const float* x1f = nullptr;
  const float* x2f = nullptr;
  long ldf = 0;
  double xs = 0.0;
  double* part = nullptr;
  const Scalars* sc = nullptr;
  __nv_bfloat16* bf_hi = nullptr;
  long bf_ld = 0, bf_blk = 0, bf_lo = 0;
  int expire = 0;
};

// base: 16-byte aligned; ld * 2 bytes a multiple of 16.
Operand make_operand(const __nv_bfloat16* base, long rows, long cols, long ld, int slices, bool is_a);
// A view of rows [row_off, row_off + rows) of every slice of a stack whose slices are slice_rows
// rows apart (a K-major A or B operand, or, with mn_major, an MN-major B operand whose rows are
// the contracted index).
Operand make_operand_view(const __nv_bfloat16* base, long slice_rows, long cols, long ld, int slices, bool is_a,
                          int row_off, long rows, bool mn_major = false);
// C = alpha * sum_p A_{pl.a[p]} B_{pl.b[p]}^T + beta * C (FP32 accumulation, float64 epilogue)
void gemm(cudaStream_t st, const Operand& A, const Operand& B, int K, const PairList& pl, const Epilogue& ep);
// the npass convention of the split form: 3 -> pairs_split3(), 1 -> pairs_single()
inline void gemm(cudaStream_t st, const Operand& A, const Operand& B, int K, int npass, const Epilogue& ep) {
  gemm(st, A, B, K, npass == 3 ? pairs_split3() : pairs_single(), ep);
}
// Output tiles of a persistent launch: 128 x bn on one SM (bn = 128 or 256), or, with pair,
// 256 x bn on a cluster of two SMs that share the MMA (tcgen05 cta_group::2; bn = 128, 192 or 256;
// the split form or a single pass).
// With quad (pair set too), a cluster of two SM pairs side by side along N shares the A operand
// through TMA multicast: a work unit is 256 x 2 bn (dense B only).
struct TileShape {
  int bn = 256;
  bool pair = false;
  bool quad = false;
  int code() const { return bn + (quad ? 2000 : (pair ? 1000 : 0)); }  // as reported in omm_info
};
int tiles_of(const Epilogue& ep, int bn = 256, bool pair = false, bool quad = false);  // work units of one GEMM
// the partial-sum slots (one per epilogue warp and 128 x bn quarter) a kEpReduce GEMM writes
inline int reduce_slots(const Epilogue& ep, const TileShape& ts) {
  return 4 * tiles_of(ep, ts.bn, ts.pair, ts.quad) * (ts.quad ? 4 : (ts.pair ? 2 : 1));
}

// One GEMM of a grouped launch (device array element; tensor maps in global memory).
// Block sparsity of a B operand (rows x K): for every block of bn rows, the 64-wide K blocks that
// hold a nonzero (CSR on the device: blocks of row block r are idx[off[r] .. off[r+1]), at least
// one per row block). A product skips the K blocks where B is exactly zero: the FP32 sums, and so
// the results, are the same as the dense product's.
struct BlockLists {
  int* off = nullptr;  // device, nblocks + 1
  int* idx = nullptr;  // device
  int nblocks = 0;
  long nnz = 0;
  long dense = 0;  // nblocks x K blocks
};
// (re)computes bl for B (rows x cols float64, leading dimension ld, device) and row blocks of bn;
// (bn = 128, 192 or 256); the first call allocates room for a dense pattern (from the library's
// pool, on st), later calls
// (same shape) rewrite in place so that descriptors holding the pointers stay valid. Synchronises
// the stream.
void block_lists(cudaStream_t st, const double* B, long rows, long cols, long ld, int bn, BlockLists& bl);
void free_block_lists(BlockLists& bl, cudaStream_t st);  // st: the owner's current stream
// fraction of the K blocks a product over these lists visits (1 for a dense product)
inline double block_density(const BlockLists* bl) {
  return (bl == nullptr || bl->dense == 0) ? 1.0 : (double)bl->nnz / (double)bl->dense;
}

struct alignas(64) GroupDesc {
  TensorMap a;
  TensorMap b;
  Epilogue ep;
  int K, rowsA, rowsB, tile_begin;  // rowsA, rowsB: rows between the slices of A and B
  int offA, offB;                   // first row of A and B inside each slice
  int b_mn;                         // B is MN-major (its rows are the contracted index)
  int bn;    // output tile width (all groups of one launch share it, pair and quad)
  int pair;  // 256-row tiles on a cluster of two SMs
  int quad;  // two such pairs per cluster, sharing A
  const int* kb_off;  // block sparsity of B for row blocks of bn (null: dense)
  const int* kb_idx;
};
GroupDesc make_group(const Operand& A, const Operand& B, int K, const Epilogue& ep, int tile_begin, int bn = 256,
                     const BlockLists* sparse = nullptr, bool pair = false, bool quad = false);
// groups_dev: ngroups descriptors in device memory, sorted by tile_begin; all share the pair list
void prepare_persistent();  // kernel attributes (call before a stream capture)
// persistent grouped launch: one CTA per SM, double-buffered TMEM accumulators; err receives a
// nonzero code if a bounded wait expired
void gemm_persistent(cudaStream_t st, const GroupDesc* groups_dev, int ngroups, int total_tiles, const PairList& pl,
                     int* err, int bn = 256, bool pair = false, bool quad = false);
// the same persistent kernel for one GEMM whose descriptor travels as a kernel parameter.
// partial (optional, partial_capacity doubles): scratch that lets a GEMM of few output tiles run
// each chunk of its pair list on its own CTA and add the chunks afterwards, in chunk order.
void gemm_persistent(cudaStream_t st, const Operand& A, const Operand& B, int K, const PairList& pl,
                     const Epilogue& ep, double* partial = nullptr, long partial_capacity = 0,
                     const BlockLists* sparse = nullptr);

// Tile-shape autotuner: times one persistent launch over these GEMMs (the operands as given,
// the outputs redirected to scratch) with each candidate shape -- 128 x 256 and 128 x 128 on one
// SM, and (split form or single pass, allow_pair) 256 x 128, 256 x 192 and 256 x 256 on SM pairs,
// and (dense B) the same on clusters of two pairs sharing A
// -- returns the fastest, and remembers it per shape signature for the life of the process.
// ms_spent receives the time spent timing (0 when the answer came from the cache).
struct GemmSpec {
  const Operand* A;
  const Operand* B;
  int K;
  Epilogue ep;                                            // only M and N are used
  const BlockLists* sparse[3] = {nullptr, nullptr, nullptr};  // block lists of B for bn = 256, 128, 192
};
inline int sparse_slot(int bn) { return bn == 256 ? 0 : (bn == 128 ? 1 : 2); }
TileShape choose_tile_shape(cudaStream_t st, const std::vector<GemmSpec>& specs, const PairList& pl,
                            double* ms_spent = nullptr, bool allow_pair = true);

// x (float64, rows x cols, ld_src) -> hi = bf16(x), lo = bf16(x - hi) (ld_dst);
// transposed variants write dst[j][i]. Skipped when sc's done/halt is set.
void split(cudaStream_t st, const double* src, long rows, long cols, long ld_src, __nv_bfloat16* hi,
           __nv_bfloat16* lo, long ld_dst, const Scalars* sc);
// hi/lo of (src - sub), both float64 with the same layout
void split_diff(cudaStream_t st, const double* src, const double* sub, long rows, long cols, long ld_src,
                __nv_bfloat16* hi, __nv_bfloat16* lo, long ld_dst, const Scalars* sc);
void split_transposed(cudaStream_t st, const double* src, long rows, long cols, long ld_src,
                      __nv_bfloat16* hi_t, __nv_bfloat16* lo_t, long ld_dst, const Scalars* sc);

}  // namespace tc
}  // namespace omm
