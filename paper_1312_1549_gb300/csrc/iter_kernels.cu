// Memory-bound kernels of the OMM iteration and the one-block control
// kernels that take the scalar decisions of a line search on the device
// (Polak-Ribiere coefficient, quartic coefficients, line minimum, stopping
// tests), so that the host never has to read a value inside the loop.
//
// Reductions use fixed grids and fixed summation orders: results are bitwise
// reproducible from run to run.
#include "omm_internal.cuh"
#include "iter_device.cuh"
#include "fused_device.cuh"

namespace omm {
namespace {

using namespace dev;







// Block-wide sum (TB threads); result valid in thread 0.


__global__ void shift_kernel(long count, const double* H, const double* S, double eta, double* Ht) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < count; i += (long)gridDim.x * blockDim.x)
    Ht[i] = H[i] - eta * S[i];
}

__global__ void add_scaled_kernel(long count, const double* S, const double* T, double s, double* A) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < count; i += (long)gridDim.x * blockDim.x)
    A[i] = S[i] + (T ? T[i] * s : 0.0);
}

__global__ void fill_kernel(long count, double v, double* d) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < count; i += (long)gridDim.x * blockDim.x)
    d[i] = v;
}

// partials of <G,PG>, <G_old,PG>, <G,Delta_old>, max|G| per block
__global__ void __launch_bounds__(TB)
grad_reduce_kernel(long count, const double* __restrict__ G, const double* __restrict__ PG,
                   const double* __restrict__ Gold, const double* __restrict__ Dir,
                   double* part, const Scalars* sc) {
  grad_reduce_body(count, G, PG, Gold, Dir, part, sc, blockIdx.x, gridDim.x);
}




// Polak-Ribiere coefficient and the stopping tests (one block).
__global__ void __launch_bounds__(TB)
control_direction_kernel(Scalars* sc, const double* part, int mixed, int nparts) {
  control_direction_body(sc, part, mixed, nparts, blockIdx.x, gridDim.x);
}


__global__ void direction_kernel(long count, const double* __restrict__ PG, double* Dir,
                                 const Scalars* sc) {
  direction_body(count, PG, Dir, sc, blockIdx.x, gridDim.x);
}


// The trace products of Eq. 13, Tr(XY) = sum_ij X_ij Y_ji, on 32x32 tiles
// with the transposed tiles staged in shared memory.
//   SWHW = [S_W | H_W] (n x 2n), Proj = [H' | S' | H'' | S''] (n x 4n).
//   t0 Tr H'        t1 Tr(S' H_W)   t2 Tr(S_W H')   t3 Tr H''
//   t4 Tr(S'' H_W)  t5 Tr(S_W H'')  t6 Tr(S' H')    t7 Tr(S'^T H')
//   t8 Tr(S'' H')   t9 Tr(S' H'')   t10 Tr(S'' H'')
template <bool F32>
__global__ void __launch_bounds__(TB)
traces_kernel(int n, const double* __restrict__ SWHW, const double* __restrict__ Proj,
              double* part, const Scalars* sc) {
  traces_body<F32>(n, SWHW, Proj, part, sc, blockIdx.x, gridDim.x);
}


// derivative p'(x) and p''(x) of the quartic



// Root of p' in [lo, hi] with p'(lo) < 0 <= p'(hi): Newton steps safeguarded
// by bisection (the "rtsafe" scheme of Numerical Recipes).


}  // namespace

namespace {

using namespace dev;

// quartic coefficients (Eq. 13), line minimum and bookkeeping (one block)
__global__ void __launch_bounds__(TB)
control_linesearch_kernel(Scalars* sc, const double* part, int nblocks) {
  control_linesearch_body(sc, part, nblocks, blockIdx.x, gridDim.x);
}


// C += x Delta; HC += x HDelta; SC += x SDelta; G_old = G; G = 8 HC (the GEMM adds -4 [..])
__global__ void update_state_kernel(int n, long m, double* C, double* Y4, const double* Dir,
                                    double* G, double* Gold, const Scalars* sc) {
  if (stopped(sc)) return;
  const double x = sc->x;
  const long count = (long)n * m;
  double* HC = Y4;
  double* SC = Y4 + count;
  const double* HD = Y4 + 2 * count;
  const double* SD = Y4 + 3 * count;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < count; i += (long)gridDim.x * blockDim.x) {
    const double d = Dir[i];
    C[i] = fma(x, d, C[i]);
    const double hc = fma(x, HD[i], HC[i]);
    HC[i] = hc;
    SC[i] = fma(x, SD[i], SC[i]);
    Gold[i] = G[i];
    G[i] = 8.0 * hc;
  }
}



// H_W += x (H' + H'^T) + x^2 H''; S_W likewise (Eq. 16), on 32x32 tiles
__global__ void __launch_bounds__(TB)
update_subspace_kernel(int n, double* SWHW, const double* __restrict__ Proj, const Scalars* sc) {
  update_subspace_body(n, SWHW, Proj, sc, blockIdx.x, gridDim.x);
}


__global__ void scale_copy_kernel(long count, const double* src, double a, double* dst, const Scalars* sc) {
  scale_copy_body(count, src, a, dst, sc, blockIdx.x, gridDim.x);
}


// partial sums of Tr H_W and Tr(S_W H_W) = sum_ij S_W,ij H_W,ji
__global__ void __launch_bounds__(TB)
functional_kernel(int n, const double* __restrict__ SWHW, double* part) {
  const int tiles = (n + 31) / 32;
  const int I = blockIdx.x / tiles, J = blockIdx.x % tiles;
  __shared__ double tHW[32][33];
  const long l2 = 2L * n;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int r = ty; r < 32; r += 8) {
    const int gi = J * 32 + r, gj = I * 32 + tx;
    tHW[r][tx] = (gi < n && gj < n) ? SWHW[(long)gi * l2 + n + gj] : 0.0;
  }
  __syncthreads();
  double v[2] = {0.0, 0.0};
  for (int r = ty; r < 32; r += 8) {
    const int gi = I * 32 + r, gj = J * 32 + tx;
    if (gi >= n || gj >= n) continue;
    if (gi == gj) v[0] += SWHW[(long)gi * l2 + n + gj];
    v[1] = fma(SWHW[(long)gi * l2 + gj], tHW[tx][r], v[1]);
  }
  __shared__ double sh[2][TB / 32];
  block_sum<2>(v, sh);
  if (threadIdx.x == 0) {
    part[blockIdx.x * 2 + 0] = v[0];
    part[blockIdx.x * 2 + 1] = v[1];
  }
}

__global__ void __launch_bounds__(TB)
finish_functional_kernel(Scalars* sc, const double* part, int nblocks) {
  double v[2] = {0.0, 0.0};
  for (int b = threadIdx.x; b < nblocks; b += TB) {
    v[0] += part[b * 2 + 0];
    v[1] += part[b * 2 + 1];
  }
  __shared__ double sh[2][TB / 32];
  block_sum<2>(v, sh);
  if (threadIdx.x == 0) sc->E = 4.0 * v[0] - 2.0 * v[1];
}

__global__ void __launch_bounds__(TB)
gmax_kernel(long count, const double* __restrict__ G, double* part) {
  double mx = 0.0;
  for (long i = blockIdx.x * (long)TB + threadIdx.x; i < count; i += (long)gridDim.x * TB) {
    const double a = fabs(G[i]);
    mx = (a > mx || a != a) ? a : mx;
  }
  __shared__ double shm[TB / 32];
  const double wm = warp_max(mx);
  if ((threadIdx.x & 31) == 0) shm[threadIdx.x >> 5] = wm;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int k = 0; k < TB / 32; ++k) m = (shm[k] > m || shm[k] != shm[k]) ? shm[k] : m;
    part[blockIdx.x] = m;
  }
}

__global__ void __launch_bounds__(TB) finish_gmax_kernel(Scalars* sc, const double* part) {
  double mx = 0.0;
  for (int b = threadIdx.x; b < kReduceBlocks; b += TB) {
    const double a = part[b];
    mx = (a > mx || a != a) ? a : mx;
  }
  __shared__ double shm[TB / 32];
  const double wm = warp_max(mx);
  if ((threadIdx.x & 31) == 0) shm[threadIdx.x >> 5] = wm;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int k = 0; k < TB / 32; ++k) m = (shm[k] > m || shm[k] != shm[k]) ? shm[k] : m;
    sc->gmax = m;
  }
}

__global__ void two_i_minus_kernel(int n, const double* SW, long ldsw, double* out) {
  const long count = (long)n * n;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < count; idx += (long)gridDim.x * blockDim.x) {
    const long i = idx / n, j = idx % n;
    out[idx] = (i == j ? 2.0 : 0.0) - SW[i * ldsw + j];
  }
}

__global__ void symmetrize_lower_kernel(int m, double* A) {
  const long count = (long)m * m;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < count; idx += (long)gridDim.x * blockDim.x) {
    const long i = idx / m, j = idx % m;
    if (j > i) A[idx] = A[j * m + i];
  }
}

__global__ void line_minimum_kernel(const double* a, double* x, int* status) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *status = quartic_first_minimum(a, x);
}

inline int grid_for(long count) {
  long g = (count + TB - 1) / TB;
  if (g > 4096) g = 4096;
  if (g < 1) g = 1;
  return (int)g;
}

}  // namespace

void launch_axpby_shift(cudaStream_t st, long count, const double* H, const double* S, double eta, double* Ht) {
  shift_kernel<<<grid_for(count), TB, 0, st>>>(count, H, S, eta, Ht);
  OMM_LAUNCH_CHECK();
}
void launch_add_scaled(cudaStream_t st, long count, const double* S, const double* T, double s, double* A) {
  add_scaled_kernel<<<grid_for(count), TB, 0, st>>>(count, S, T, s, A);
  OMM_LAUNCH_CHECK();
}
void launch_fill(cudaStream_t st, long count, double v, double* d) {
  fill_kernel<<<grid_for(count), TB, 0, st>>>(count, v, d);
  OMM_LAUNCH_CHECK();
}
void launch_grad_reduce(cudaStream_t st, long count, const double* G, const double* PG, const double* Gold,
                        const double* Dir, double* part, const Scalars* sc) {
  grad_reduce_kernel<<<kReduceBlocks, TB, 0, st>>>(count, G, PG, Gold, Dir, part, sc);
  OMM_LAUNCH_CHECK();
}
void launch_control_direction(cudaStream_t st, Scalars* sc, const double* part, int mixed, int nparts) {
  control_direction_kernel<<<1, TB, 0, st>>>(sc, part, mixed, nparts);
  OMM_LAUNCH_CHECK();
}
void launch_direction(cudaStream_t st, long count, const double* PG, double* Dir, const Scalars* sc) {
  direction_kernel<<<grid_for(count), TB, 0, st>>>(count, PG, Dir, sc);
  OMM_LAUNCH_CHECK();
}
int traces_blocks(int n) {
  const int t = (n + 31) / 32;
  return t * t;
}
int traces_partials(int n) { return (traces_blocks(n) + 3) / 4; }
void launch_traces(cudaStream_t st, int n, const double* SWHW, const double* Proj, double* part,
                   const Scalars* sc, bool fp32_products) {
  if (fp32_products) traces_kernel<true><<<traces_partials(n), TB, 0, st>>>(n, SWHW, Proj, part, sc);
  else traces_kernel<false><<<traces_partials(n), TB, 0, st>>>(n, SWHW, Proj, part, sc);
  OMM_LAUNCH_CHECK();
}
void launch_control_linesearch(cudaStream_t st, Scalars* sc, const double* part, int nblocks) {
  control_linesearch_kernel<<<1, TB, 0, st>>>(sc, part, nblocks);
  OMM_LAUNCH_CHECK();
}
void launch_update_state(cudaStream_t st, int n, long m, double* C, double* Y4, const double* Dir,
                         double* G, double* Gold, const Scalars* sc) {
  update_state_kernel<<<grid_for((long)n * m), TB, 0, st>>>(n, m, C, Y4, Dir, G, Gold, sc);
  OMM_LAUNCH_CHECK();
}
namespace {
__global__ void __launch_bounds__(256)
direction_split_kernel(long n, long m, const double* __restrict__ PG, double* __restrict__ Dir,
                       __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo, long ldm, const Scalars* sc) {
  dev::direction_split_body(n, m, PG, Dir, hi, lo, ldm, sc, blockIdx.x, gridDim.x);
}
__global__ void __launch_bounds__(256)
update_state_split_kernel(long n, long m, double* C, double* Y4, const double* Dir, double* dY, __nv_bfloat16* Yhi,
                          __nv_bfloat16* Ylo, long ldm, const Scalars* sc) {
  dev::update_state_split_body(n, m, C, Y4, Dir, dY, Yhi, Ylo, ldm, sc, blockIdx.x, gridDim.x);
}
__global__ void __launch_bounds__(TB)
update_subspace_split_kernel(int n, double* SWHW, const double* __restrict__ Proj, const double* __restrict__ Wref,
                             __nv_bfloat16* Whi, __nv_bfloat16* Wlo, long ldw, const Scalars* sc) {
  dev::update_subspace_split_body(n, SWHW, Proj, Wref, Whi, Wlo, ldw, sc, blockIdx.x, gridDim.x);
}
}  // namespace

// one block per (row, 256 column pairs) unit, at most 16384 blocks
static unsigned pair_grid(long rows, long cols) {
  const long units = rows * (((cols + 1) / 2 + 255) / 256);
  return (unsigned)(units < 1 ? 1 : (units > 16384 ? 16384 : units));
}

void launch_direction_split(cudaStream_t st, long n, long m, const double* PG, double* Dir, __nv_bfloat16* hi,
                            __nv_bfloat16* lo, long ldm, const Scalars* sc) {
  direction_split_kernel<<<pair_grid(n, m), 256, 0, st>>>(n, m, PG, Dir, hi, lo, ldm, sc);
  OMM_LAUNCH_CHECK();
}
void launch_update_state_split(cudaStream_t st, long n, long m, double* C, double* Y4, const double* Dir, double* dY,
                               __nv_bfloat16* Yhi, __nv_bfloat16* Ylo, long ldm, const Scalars* sc) {
  update_state_split_kernel<<<pair_grid(n, m), 256, 0, st>>>(n, m, C, Y4, Dir, dY, Yhi, Ylo, ldm, sc);
  OMM_LAUNCH_CHECK();
}
namespace {
__global__ void __launch_bounds__(256)
direction_split32_kernel(long n, long m, const float* PG, float* Dir, __nv_bfloat16* hi, __nv_bfloat16* lo, long ldm,
                         const Scalars* sc) {
  dev::direction_split32_body(n, m, PG, Dir, hi, lo, ldm, sc, blockIdx.x, gridDim.x);
}
__global__ void __launch_bounds__(256)
update_state_split32_kernel(long n, long m, double* C, double* Y4, const float* Dir, const float* HD32, float* dY32,
                            __nv_bfloat16* Yhi, __nv_bfloat16* Ylo, long ldm, const Scalars* sc) {
  dev::update_state_split32_body(n, m, C, Y4, Dir, HD32, dY32, Yhi, Ylo, ldm, sc, blockIdx.x, gridDim.x);
}
__global__ void __launch_bounds__(TB)
reduce_unpreconditioned_kernel(long n, long m, const double* G, double* Gold, const float* Dir, float* PG, long ldm,
                               double* part, const Scalars* sc) {
  dev::reduce_unpreconditioned_body(n, m, G, Gold, Dir, PG, ldm, part, sc, blockIdx.x, gridDim.x);
}
}  // namespace

void launch_direction_split32(cudaStream_t st, long n, long m, const float* PG, float* Dir, __nv_bfloat16* hi,
                              __nv_bfloat16* lo, long ldm, const Scalars* sc) {
  direction_split32_kernel<<<pair_grid(n, m), 256, 0, st>>>(n, m, PG, Dir, hi, lo, ldm, sc);
  OMM_LAUNCH_CHECK();
}
void launch_update_state_split32(cudaStream_t st, long n, long m, double* C, double* Y4, const float* Dir,
                                 const float* HD32, float* dY32, __nv_bfloat16* Yhi, __nv_bfloat16* Ylo, long ldm,
                                 const Scalars* sc) {
  update_state_split32_kernel<<<pair_grid(n, m), 256, 0, st>>>(n, m, C, Y4, Dir, HD32, dY32, Yhi, Ylo, ldm, sc);
  OMM_LAUNCH_CHECK();
}
void launch_reduce_unpreconditioned(cudaStream_t st, long n, long m, const double* G, double* Gold, const float* Dir,
                                    float* PG, long ldm, double* part, const Scalars* sc) {
  reduce_unpreconditioned_kernel<<<kReduceBlocks, TB, 0, st>>>(n, m, G, Gold, Dir, PG, ldm, part, sc);
  OMM_LAUNCH_CHECK();
}
void launch_update_subspace_split(cudaStream_t st, int n, double* SWHW, const double* Proj, const double* Wref,
                                  __nv_bfloat16* Whi, __nv_bfloat16* Wlo, long ldw, const Scalars* sc) {
  update_subspace_split_kernel<<<traces_blocks(n), TB, 0, st>>>(n, SWHW, Proj, Wref, Whi, Wlo, ldw, sc);
  OMM_LAUNCH_CHECK();
}
void launch_update_subspace(cudaStream_t st, int n, double* SWHW, const double* Proj, const Scalars* sc) {
  update_subspace_kernel<<<traces_blocks(n), TB, 0, st>>>(n, SWHW, Proj, sc);
  OMM_LAUNCH_CHECK();
}
void launch_scale_copy(cudaStream_t st, long count, const double* src, double a, double* dst, const Scalars* sc) {
  scale_copy_kernel<<<grid_for(count), TB, 0, st>>>(count, src, a, dst, sc);
  OMM_LAUNCH_CHECK();
}
void launch_functional(cudaStream_t st, int n, const double* SWHW, double* part) {
  functional_kernel<<<traces_blocks(n), TB, 0, st>>>(n, SWHW, part);
  OMM_LAUNCH_CHECK();
}
void launch_finish_functional(cudaStream_t st, Scalars* sc, const double* part, int nblocks) {
  finish_functional_kernel<<<1, TB, 0, st>>>(sc, part, nblocks);
  OMM_LAUNCH_CHECK();
}
void launch_gmax(cudaStream_t st, long count, const double* G, double* part) {
  gmax_kernel<<<kReduceBlocks, TB, 0, st>>>(count, G, part);
  OMM_LAUNCH_CHECK();
}
void launch_finish_gmax(cudaStream_t st, Scalars* sc, const double* part) {
  finish_gmax_kernel<<<1, TB, 0, st>>>(sc, part);
  OMM_LAUNCH_CHECK();
}
void launch_two_i_minus(cudaStream_t st, int n, const double* SW, long ldsw, double* out) {
  two_i_minus_kernel<<<grid_for((long)n * n), TB, 0, st>>>(n, SW, ldsw, out);
  OMM_LAUNCH_CHECK();
}
void launch_line_minimum(cudaStream_t st, const double* a, double* x, int* status) {
  line_minimum_kernel<<<1, 32, 0, st>>>(a, x, status);
  OMM_LAUNCH_CHECK();
}
void launch_symmetrize_lower(cudaStream_t st, int m, double* A) {
  symmetrize_lower_kernel<<<grid_for((long)m * m), TB, 0, st>>>(m, A);
  OMM_LAUNCH_CHECK();
}

}  // namespace omm
