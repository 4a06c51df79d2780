// Float64 inverse of a symmetric positive definite matrix, for the kinetic
// preconditioner P = (S + T/tau)^-1 (Sec. 2.4, Eq. 17), computed once per
// geometry. Three stages, all on the device:
//   1. blocked right-looking Cholesky A = L L^T (64-column panels; the
//      diagonal block is factored and inverted by one CTA in shared memory,
//      the panel and the trailing update are float64 GEMMs),
//   2. Y = L^-1 by recursive halving: inv([L11 0; L21 L22]) =
//      [Y11 0; -Y22 L21 Y11  Y22], whose base cases are the inverted diagonal
//      blocks of stage 1,
//   3. P = Y^T Y (lower tiles only, K loop from the diagonal), then mirrored.
// A failed pivot (<= 0 or NaN) is recorded in info_dev and replaced by 1 so
// that the remaining stages stay finite; the caller reports the failure.
//
// spd_inverse_sliced computes the same P with float64-class products on the
// BF16 tensor cores (the fixed-point slicing of emu.cu), recursively on
// halves so that every product has a long contraction:
//   chol_inv([A11 A21^T; A21 A22]):  L11, Y11 = chol_inv(A11);
//     L21 = A21 Y11^T;  A22 -= L21 L21^T;  L22, Y22 = chol_inv(A22);
//     Y21 = -(Y22 L21) Y11                         (Y = L^-1)
//   lauum(Y) = Y^T Y:  P22 = lauum(Y22);  P21 = Y22^T Y21;
//     P11 = lauum(Y11) + Y21^T Y21
// with leaves factored and inverted by one CTA (which also writes the leaf's block of Y^T Y):
// 64 x 64 in float64 for float64-class results, 128 x 128 in float32 for the preconditioner. The
// P updates of a node run on a second stream as soon as its Y is final, beside the factorisation
// of the blocks that follow.
#include "emu.cuh"
#include "omm_internal.cuh"
#include "tc_gemm.cuh"

#include <algorithm>
#include <vector>

namespace omm {
namespace {

constexpr int NB = 64;

// Factor the b x b diagonal block at A (ld lda) in place (lower) and write
// its inverse to Linv (NB x NB, row-major, zero above the diagonal); with Pblk
// (ld ldp) also the block Linv^T Linv (both triangles). Every division is a
// multiplication by one reciprocal per pivot: float64 division is a long
// instruction sequence on this GPU's narrow float64 pipe. R is the arithmetic
// type: double, or float for a preconditioner, which needs far less than float64
// accuracy and which the float64 pipe (about 2 instructions per SM and clock)
// would make the serial bottleneck of the recursive inverse.
template <typename R>
__global__ void __launch_bounds__(256)
potf2_inv_kernel(double* A, long lda, int b, double* Linv, int* info, int col_offset, double* Pblk, long ldp) {
  __shared__ R L[NB][NB + 1];
  __shared__ R X[NB][NB + 1];
  __shared__ R rdiag[NB];
  const int tid = threadIdx.x;
  for (int idx = tid; idx < NB * NB; idx += blockDim.x) {
    const int i = idx / NB, j = idx % NB;
    L[i][j] = (i < b && j < b && j <= i) ? (R)A[(long)i * lda + j] : (R)0;
  }
  __syncthreads();
  for (int j = 0; j < b; ++j) {
    if (tid == 0) {
      R d = L[j][j];
      if (!(d > (R)0)) {
        atomicCAS(info, 0, col_offset + j + 1);
        d = (R)1;
      }
      const R r = sqrt(d);
      L[j][j] = r;
      rdiag[j] = (R)1 / r;
    }
    __syncthreads();
    const R rj = rdiag[j];
    for (int i = j + 1 + tid; i < b; i += blockDim.x) L[i][j] *= rj;
    __syncthreads();
    const int r = b - j - 1;
    for (int idx = tid; idx < r * r; idx += blockDim.x) {
      const int i = j + 1 + idx / r, l = j + 1 + idx % r;
      if (l <= i) L[i][l] = fma(-L[i][j], L[l][j], L[i][l]);
    }
    __syncthreads();
  }
  for (int idx = tid; idx < b * b; idx += blockDim.x) {
    const int i = idx / b, j = idx % b;
    A[(long)i * lda + j] = (j <= i) ? (double)L[i][j] : 0.0;
  }
  // inverse of the lower-triangular block: column c solves L x = e_c
  if (tid < NB) {
    const int c = tid;
    for (int i = 0; i < NB; ++i) X[i][c] = (R)0;
    if (c < b) {
      X[c][c] = rdiag[c];
      for (int i = c + 1; i < b; ++i) {
        R acc = (R)0;
        for (int k = c; k < i; ++k) acc = fma(L[i][k], X[k][c], acc);
        X[i][c] = -acc * rdiag[i];
      }
    }
  }
  __syncthreads();
  for (int idx = tid; idx < NB * NB; idx += blockDim.x) {
    const int i = idx / NB, j = idx % NB;
    Linv[idx] = (double)X[i][j];
  }
  if (Pblk != nullptr) {
    // (X^T X)_ij = sum_{k >= i} X_ki X_kj for j <= i, mirrored
    for (int idx = tid; idx < b * b; idx += blockDim.x) {
      const int i = idx / b, j = idx % b;
      if (j > i) continue;
      R acc = (R)0;
      for (int k = i; k < b; ++k) acc = fma(X[k][i], X[k][j], acc);
      Pblk[(long)i * ldp + j] = (double)acc;
      Pblk[(long)j * ldp + i] = (double)acc;
    }
  }
}

// ---- float32 leaves of edge up to 128 for the preconditioner-grade inverse
constexpr int NL = 128;
constexpr int kLeafThreads = 512;
constexpr int kLeafSmem = (3 * NL * (NL + 1) + NL) * (int)sizeof(float);

// float64 <-> float32 on the integer pipe (normal numbers; magnitudes outside the float32 normal
// range become zero or infinity), so that the leaf's conversions stay off the narrow float64 units
__device__ __forceinline__ float to_f32(double x) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const unsigned int sign = (unsigned int)(u >> 32) & 0x80000000u;
  const int e = (int)((u >> 52) & 0x7FFu);
  if (e < 1023 - 126) return __uint_as_float(sign);
  if (e > 1023 + 127) return __uint_as_float(sign | 0x7F800000u);
  // round the 52-bit fraction to 23 bits, ties to even (a carry moves into the exponent)
  const unsigned long long f = u & 0x000FFFFFFFFFFFFFull;
  const unsigned long long r = f + 0x0FFFFFFFull + ((f >> 29) & 1ull);
  return __uint_as_float(sign + ((unsigned int)(e - 1023 + 127) << 23) + (unsigned int)(r >> 29));
}
__device__ __forceinline__ double to_f64(float v) {
  const unsigned int u = __float_as_uint(v);
  const unsigned int e = (u >> 23) & 0xFFu;
  const unsigned long long sign = (unsigned long long)(u & 0x80000000u) << 32;
  if (e == 0) return __longlong_as_double((long long)sign);  // zero (subnormals flushed)
  if (e == 0xFFu) return __longlong_as_double((long long)(sign | (0x7FFull << 52) | ((unsigned long long)(u & 0x7FFFFFu) << 29)));
  return __longlong_as_double(
      (long long)(sign | ((unsigned long long)(e + 1023u - 127u) << 52) | ((unsigned long long)(u & 0x7FFFFFu) << 29)));
}

// One CTA: Cholesky factor of the b x b diagonal block at A (b <= 128, read only: the caller
// does not need L itself), its inverse X = L^-1 into Linv (NL x NL, row-major, zero above the
// diagonal) and, with Pblk, the block X^T X (both triangles) -- all in float32, for the
// preconditioner (see potf2_inv_kernel). The triangular inverse is blocked so that all threads
// work: 16 x 16 diagonal blocks are inverted by one warp each, then pairs of inverted blocks are
// joined level by level, X21 = -X22 (L21 X11).
__global__ void __launch_bounds__(kLeafThreads)
leaf_f32_kernel(const double* A, long lda, int b, double* Linv, int* info, int col_offset, double* Pblk, long ldp) {
  extern __shared__ float smf[];
  float (*L)[NL + 1] = reinterpret_cast<float (*)[NL + 1]>(smf);
  float (*X)[NL + 1] = reinterpret_cast<float (*)[NL + 1]>(smf + NL * (NL + 1));
  float (*T)[NL + 1] = reinterpret_cast<float (*)[NL + 1]>(smf + 2 * NL * (NL + 1));
  float* rdiag = smf + 3 * NL * (NL + 1);
  const int tid = threadIdx.x, nt = blockDim.x;
  const int warp = tid >> 5, lane = tid & 31, nwarps = nt >> 5;
  for (int i = warp; i < NL; i += nwarps)
    for (int j = lane; j < NL; j += 32) {
      L[i][j] = (i < b && j <= i) ? to_f32(A[(long)i * lda + j]) : 0.f;
      X[i][j] = 0.f;
      T[i][j] = 0.f;
    }
  __syncthreads();
  // Right-looking in panels of 16 columns. Warp 0 factors a panel with its rows in registers
  // (lane l holds rows p0 + l + 32 t), pivots and column entries passed by shuffles, no block
  // barrier; then all warps apply the panel's rank-16 update to the trailing lower triangle
  // (warp w on rows q0 + w, q0 + w + 16, ..., lanes on columns), each element's 16 products
  // from independent shared-memory loads. Two barriers per panel instead of one per column: a
  // column at a time left every warp waiting on a chain of dependent shared-memory loads.
  for (int p0 = 0; p0 < b; p0 += 16) {
    const int pw = min(16, b - p0);
    if (warp == 0) {
      float r[4][16];
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const int i = p0 + lane + 32 * t;
#pragma unroll
        for (int c = 0; c < 16; ++c) r[t][c] = (i < b && c < pw && p0 + c <= i) ? L[i][p0 + c] : 0.f;
      }
#pragma unroll
      for (int c = 0; c < 16; ++c) {
        if (c < pw) {
          float d = __shfl_sync(0xffffffffu, r[0][c], c);  // the pivot, row p0 + c
          if (!(d > 0.f)) {
            if (lane == 0) atomicCAS(info, 0, col_offset + p0 + c + 1);
            d = 1.f;
          }
          const float sq = sqrtf(d), rs = 1.f / sq;
#pragma unroll
          for (int t = 0; t < 4; ++t) {
            const int i = p0 + lane + 32 * t;
            if (i > p0 + c) r[t][c] *= rs;
            else if (i == p0 + c) r[t][c] = sq;
          }
          if (lane == 0) rdiag[p0 + c] = rs;
#pragma unroll
          for (int l = 0; l < 16; ++l) {
            if (l > c) {
              const float lc = __shfl_sync(0xffffffffu, r[0][c], l);  // L[p0 + l][p0 + c], scaled
#pragma unroll
              for (int t = 0; t < 4; ++t)
                if (lane + 32 * t >= l) r[t][l] = fmaf(-r[t][c], lc, r[t][l]);
            }
          }
        }
      }
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const int i = p0 + lane + 32 * t;
#pragma unroll
        for (int c = 0; c < 16; ++c)
          if (i < b && c < pw && p0 + c <= i) L[i][p0 + c] = r[t][c];
      }
    }
    __syncthreads();
    const int q0 = p0 + pw;  // trailing block: rows and columns q0 .. b - 1 (empty after the last panel)
    for (int i = q0 + warp; i < b; i += nwarps) {
      float li[16];
#pragma unroll
      for (int k = 0; k < 16; ++k) li[k] = L[i][p0 + k];
      for (int l = q0 + lane; l <= i; l += 32) {
        float acc = L[i][l];
#pragma unroll
        for (int k = 0; k < 16; ++k) acc = fmaf(-li[k], L[l][p0 + k], acc);
        L[i][l] = acc;
      }
    }
    __syncthreads();
  }
  // 16 x 16 diagonal blocks: lane c of warp w solves column c of block w
  const int nb16 = (b + 15) / 16;
  if (warp < nb16 && lane < 16) {
    const int o = warp * 16, e = min(16, b - o), c = lane;
    if (c < e) {
      X[o + c][o + c] = rdiag[o + c];
      for (int i = c + 1; i < e; ++i) {
        float acc = 0.f;
        for (int k = c; k < i; ++k) acc = fmaf(L[o + i][o + k], X[o + k][o + c], acc);
        X[o + i][o + c] = -acc * rdiag[o + i];
      }
    }
  }
  __syncthreads();
  // Join blocks of edge s into blocks of edge 2s: T = L21 X11, then X21 = -X22 T, each a dense
  // s x s x s product over the pair's blocks (the zeros above the diagonals of X11 and X22, and the
  // zero rows of L, X and T at and beyond b, make the full sums exact). Warp w takes a group of four
  // rows, its lanes the columns j = lane + 32 q, four products per loaded column entry.
  for (int s = 16; s < b; s *= 2) {
    const int pairs = (b + 2 * s - 1) / (2 * s);
    const int gps = s / 4, ngroups = pairs * gps, nq = (s + 31) / 32;
    for (int pass = 0; pass < 2; ++pass) {  // 0: T = L21 X11; 1: X21 = -X22 T
      for (int g = warp; g < ngroups; g += nwarps) {
        const int o = 2 * s * (g / gps), r0 = o + s + (g % gps) * 4;
        float acc[4][2] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
        for (int k = 0; k < s; ++k) {
          float a[4];
#pragma unroll
          for (int r = 0; r < 4; ++r) a[r] = pass == 0 ? L[r0 + r][o + k] : X[r0 + r][o + s + k];
#pragma unroll
          for (int q = 0; q < 2; ++q) {
            const int j = lane + 32 * q;
            if (q < nq && j < s) {
              const float bv = pass == 0 ? X[o + k][o + j] : T[o + s + k][o + j];
#pragma unroll
              for (int r = 0; r < 4; ++r) acc[r][q] = fmaf(a[r], bv, acc[r][q]);
            }
          }
        }
#pragma unroll
        for (int r = 0; r < 4; ++r) {
#pragma unroll
          for (int q = 0; q < 2; ++q) {
            const int j = lane + 32 * q;
            if (q < nq && j < s && r0 + r < b) {
              if (pass == 0) T[r0 + r][o + j] = acc[r][q];
              else X[r0 + r][o + j] = -acc[r][q];
            }
          }
        }
      }
      __syncthreads();
    }
  }
  for (int idx = tid; idx < NL * NL; idx += nt) {
    const int i = idx / NL, j = idx % NL;
    Linv[idx] = to_f64(X[i][j]);
  }
  if (Pblk != nullptr) {
    // (X^T X)_ij = sum_{k >= i} X_ki X_kj for j <= i, mirrored (X is zero above its diagonal, so
    // a sum may start below i). Warp w takes the row groups 4g .. 4g + 3 for g = w and g = 31 - w
    // (long and short k ranges paired), its lanes the columns j = lane + 32 q; per k it loads the
    // group's four entries of row k (broadcast) and its own columns, for up to 16 products: a
    // quarter of the shared-memory loads per product of one row at a time.
    static_assert(kLeafThreads == 512 && NL == 128, "32 row groups over 16 warps");
#pragma unroll 1
    for (int h = 0; h < 2; ++h) {
      const int i0 = 4 * (h == 0 ? warp : NL / 4 - 1 - warp);
      if (i0 >= b) continue;
      const int nq = min(i0 + 3, b - 1) / 32 + 1;
      float acc[4][NL / 32];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int q = 0; q < NL / 32; ++q) acc[r][q] = 0.f;
      for (int k = i0; k < b; ++k) {
        float xi[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) xi[r] = X[k][i0 + r];
#pragma unroll
        for (int q = 0; q < NL / 32; ++q) {
          if (q < nq) {
            const float xj = X[k][lane + 32 * q];
#pragma unroll
            for (int r = 0; r < 4; ++r) acc[r][q] = fmaf(xi[r], xj, acc[r][q]);
          }
        }
      }
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int i = i0 + r;
#pragma unroll
        for (int q = 0; q < NL / 32; ++q) {
          const int jj = lane + 32 * q;
          if (i < b && q < nq && jj <= i) {
            const double v = to_f64(acc[r][q]);
            Pblk[(long)i * ldp + jj] = v;
            Pblk[(long)jj * ldp + i] = v;
          }
        }
      }
    }
  }
}

__global__ void zero_upper_kernel(int m, double* A) {
  const long count = (long)m * m;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < count;
       idx += (long)gridDim.x * blockDim.x) {
    const long i = idx / m, j = idx % m;
    if (j > i) A[idx] = 0.0;
  }
}

__global__ void copy_block_kernel(int b, const double* src, long lds, double* dst, long ldd) {
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < b * b; idx += gridDim.x * blockDim.x) {
    const int i = idx / b, j = idx % b;
    dst[(long)i * ldd + j] = src[(long)i * lds + j];
  }
}

struct Work {
  double* Dinv;  // nblk x NB x NB diagonal-block inverses
  double* tmp;   // up to m*m/4 (+ panel) scratch
};

// Y[r0:r1, r0:r1] (lower, in place) <- its inverse
void trtri_rec(cudaStream_t st, int m, double* Y, const Work& w, int r0, int r1) {
  const int nb_blocks = (r1 - r0 + NB - 1) / NB;
  if (nb_blocks <= 1) {
    const int b = r1 - r0;
    copy_block_kernel<<<16, 256, 0, st>>>(b, w.Dinv + (long)(r0 / NB) * NB * NB, NB,
                                          Y + (long)r0 * m + r0, m);
    OMM_LAUNCH_CHECK();
    return;
  }
  const int mid = r0 + (nb_blocks / 2) * NB;
  trtri_rec(st, m, Y, w, r0, mid);
  trtri_rec(st, m, Y, w, mid, r1);
  const int n1 = mid - r0, n2 = r1 - mid;
  double* L21 = Y + (long)mid * m + r0;
  const double* Y11 = Y + (long)r0 * m + r0;
  const double* Y22 = Y + (long)mid * m + mid;
  // W = L21 * Y11  (n2 x n1); Y11 is lower triangular
  dgemm(st, 0, 0, n2, n1, n1, 1.0, L21, m, 0, Y11, m, 0, 0.0, w.tmp, n1, 0, 1, kTriKFromCol);
  // Y21 = -Y22 * W; Y22 is lower triangular
  dgemm(st, 0, 0, n2, n1, n2, -1.0, Y22, m, 0, w.tmp, n1, 0, 0.0, L21, m, 0, 1, kTriKToRow);
}

}  // namespace

size_t spd_inverse_workspace(int m) {
  const long nblk = (m + NB - 1) / NB;
  const long half = (m + 1) / 2 + NB;
  return (size_t)(nblk * NB * NB) + (size_t)(half * half) + (size_t)m * NB;
}

namespace {
// stage 1: A = L L^T in place (lower triangle; the upper one is zeroed)
void factor_blocked(cudaStream_t st, int m, double* A, const Work& w, int* info_dev) {
  const int nblk = (m + NB - 1) / NB;
  OMM_CUDA_TRY(cudaMemsetAsync(info_dev, 0, sizeof(int), st));
  for (int kb = 0; kb < nblk; ++kb) {
    const int k = kb * NB;
    const int b = (m - k < NB) ? (m - k) : NB;
    double* Akk = A + (long)k * m + k;
    potf2_inv_kernel<double><<<1, 256, 0, st>>>(Akk, m, b, w.Dinv + (long)kb * NB * NB, info_dev, k, nullptr, 0);
    OMM_LAUNCH_CHECK();
    const int r = m - k - b;
    if (r > 0) {
      double* A21 = A + (long)(k + b) * m + k;
      // L21 = A21 * Linv^T (to scratch, then back)
      dgemm(st, 0, 1, r, b, b, 1.0, A21, m, 0, w.Dinv + (long)kb * NB * NB, NB, 0, 0.0, w.tmp, b, 0);
      OMM_CUDA_TRY(cudaMemcpy2DAsync(A21, sizeof(double) * m, w.tmp, sizeof(double) * b,
                                     sizeof(double) * b, r, cudaMemcpyDeviceToDevice, st));
      // A22 -= L21 L21^T (lower tiles)
      double* A22 = A + (long)(k + b) * m + (k + b);
      dgemm(st, 0, 1, r, r, b, -1.0, A21, m, 0, A21, m, 0, 1.0, A22, m, 0, 1, kTriLower);
    }
  }
  zero_upper_kernel<<<1024, 256, 0, st>>>(m, A);
  OMM_LAUNCH_CHECK();
}
}  // namespace

void spd_inverse(cudaStream_t st, int m, double* A, double* P, double* work, int* info_dev) {
  const int nblk = (m + NB - 1) / NB;
  Work w{work, work + (long)nblk * NB * NB};
  // 1. Cholesky
  factor_blocked(st, m, A, w, info_dev);
  // 2. Y = L^-1 in place
  trtri_rec(st, m, A, w, 0, m);
  // 3. P = Y^T Y (lower), mirrored
  dgemm(st, 1, 0, m, m, m, 1.0, A, m, 0, A, m, 0, 0.0, P, m, 0, 1, kTriLower | kTriKStart);
  launch_symmetrize_lower(st, m, P);
}

void spd_factor_inverse(cudaStream_t st, int m, double* A, double* Y, double* work, int* info_dev) {
  const int nblk = (m + NB - 1) / NB;
  Work w{work, work + (long)nblk * NB * NB};
  factor_blocked(st, m, A, w, info_dev);
  OMM_CUDA_TRY(cudaMemcpyAsync(Y, A, sizeof(double) * m * (size_t)m, cudaMemcpyDeviceToDevice, st));
  trtri_rec(st, m, Y, w, 0, m);
}

// ------------------------------------------------------------------ float64-class (sliced) variant
namespace {

constexpr int kInvSlices = 10;  // the most slices a product of this file takes (workspace sizing)

long round8(long x) { return (x + 7) / 8 * 8; }

// scratch of one stream's products
struct Lane {
  cudaStream_t st = nullptr;
  int slices = kInvSlices;   // fixed-point slices of every product on this lane (1: the 3-term bf16 split)
  double* tr0 = nullptr;     // float64 transposes
  double* tr1 = nullptr;
  __nv_bfloat16* sl0 = nullptr;  // slices of two operands
  __nv_bfloat16* sl1 = nullptr;
  double* partial = nullptr;  // per-chunk sums of the products with few output tiles
  long partial_cap = 0;
};

struct SlicedWork {
  int m = 0;
  int nb = NB;               // leaf edge: 64 (float64 leaves) or 128 (float32 leaves)
  double* A = nullptr;       // the matrix, factor L in its lower triangle
  double* Y = nullptr;       // L^-1 (lower triangle, zero above)
  double* P = nullptr;
  double* prod = nullptr;    // one product of the factorisation
  double* leaf = nullptr;    // nb x nb inverse of a diagonal block
  int* info = nullptr;
  int* err = nullptr;
  Lane main, side;           // factorisation and inverse on `main`; the P = Y^T Y updates on `side`
  std::vector<cudaEvent_t> events;
};

// C (M x N, ldc) = alpha A B^T + beta C with A (M x K, lda) and B (N x K, ldb) row-major;
// the slices of A go to sl0, those of B to sl1 (or B = A: one slicing, both maps)
void sliced_nt(Lane& L, int* err, int M, int N, int K, double alpha, const double* A, long lda, const double* B,
               long ldb, double beta, double* C, long ldc) {
  const long ld = round8(K);
  const int s = L.slices;
  if (s == 1) {  // preconditioner grade from bf16 hi/lo splits: three products, about 2^-16 of |A||B|
    const tc::Epilogue ep{C, ldc, N, 0, alpha, beta, M, N, nullptr, err};
    tc::split(L.st, A, M, K, lda, L.sl0, L.sl0 + (long)M * ld, ld, nullptr);
    const tc::Operand oa = tc::make_operand(L.sl0, M, K, ld, 2, true);
    if (B == A && ldb == lda && N == M) {
      emu::gemm_split(L.st, oa, tc::make_operand(L.sl0, N, K, ld, 2, false), K, ep);
    } else {
      tc::split(L.st, B, N, K, ldb, L.sl1, L.sl1 + (long)N * ld, ld, nullptr);
      emu::gemm_split(L.st, oa, tc::make_operand(L.sl1, N, K, ld, 2, false), K, ep);
    }
    return;
  }
  emu::slice_rows(L.st, A, M, K, lda, s, L.sl0, ld, nullptr);
  const tc::Operand oa = tc::make_operand(L.sl0, M, K, ld, s, true);
  tc::Operand ob;
  if (B == A && ldb == lda && N == M) {
    ob = tc::make_operand(L.sl0, N, K, ld, s, false);
  } else {
    emu::slice_rows(L.st, B, N, K, ldb, s, L.sl1, ld, nullptr);
    ob = tc::make_operand(L.sl1, N, K, ld, s, false);
  }
  emu::gemm(L.st, oa, ob, K, s, tc::Epilogue{C, ldc, N, 0, alpha, beta, M, N, nullptr, err}, L.partial,
            L.partial_cap);
}

// leaf: factor A[r0:r0+b, r0:r0+b] in place, write its inverse into Y and Y_leaf^T Y_leaf into P
void leaf(SlicedWork& w, int r0, int b) {
  const long m = w.m;
  double* pb = w.P ? w.P + r0 * m + r0 : nullptr;
  if (w.nb == NL)  // a preconditioner: 128-wide float32 leaves (see leaf_f32_kernel)
    leaf_f32_kernel<<<1, kLeafThreads, kLeafSmem, w.main.st>>>(w.A + r0 * m + r0, m, b, w.leaf, w.info, r0, pb, m);
  else
    potf2_inv_kernel<double><<<1, 256, 0, w.main.st>>>(w.A + r0 * m + r0, m, b, w.leaf, w.info, r0, pb, m);
  OMM_LAUNCH_CHECK();
  copy_block_kernel<<<16, 256, 0, w.main.st>>>(b, w.leaf, w.nb, w.Y + r0 * m + r0, m);
  OMM_LAUNCH_CHECK();
}

int half_of(int b, int nb) { return ((b / nb + 1) / 2) * nb; }  // a multiple of nb, about b / 2

// P21 = Y22^T Y21 and P11 += Y21^T Y21 of one node (its Y is final), on the side lane
void p_update(SlicedWork& w, int r0, int b1, int b2) {
  const long m = w.m;
  const int r1 = r0 + b1;
  Lane& L = w.side;
  const double* Y21 = w.Y + (long)r1 * m + r0;
  const double* Y22 = w.Y + (long)r1 * m + r1;
  // Y21^T (b1 x b2) serves both products
  emu::transpose(L.st, Y21, b2, b1, m, L.tr0, b2);
  // P21 = Y22^T Y21: A operand Y22^T (b2 x b2), B operand Y21^T
  emu::transpose(L.st, Y22, b2, b2, m, L.tr1, b2);
  sliced_nt(L, w.err, b2, b1, b2, 1.0, L.tr1, b2, L.tr0, b2, 0.0, w.P + (long)r1 * m + r0, m);
  // P11 = Y11^T Y11 (the updates of the left subtree, already queued on this lane) + Y21^T Y21
  sliced_nt(L, w.err, b1, b1, b2, 1.0, L.tr0, b2, L.tr0, b2, 1.0, w.P + (long)r0 * m + r0, m);
}

// Y and L of the block [r0, r0 + b) on the main lane; once a node's Y is final its contribution
// to P = Y^T Y is queued on the side lane, in post-order, so it runs beside the factorisation
// of the blocks that follow
void chol_inv(SlicedWork& w, int r0, int b) {
  if (b <= w.nb) {
    leaf(w, r0, b);
    return;
  }
  const long m = w.m;
  Lane& L = w.main;
  const int b1 = half_of(b, w.nb), b2 = b - b1, r1 = r0 + b1;
  chol_inv(w, r0, b1);
  double* A21 = w.A + (long)r1 * m + r0;
  double* A22 = w.A + (long)r1 * m + r1;
  const double* Y11 = w.Y + (long)r0 * m + r0;
  const double* Y22 = w.Y + (long)r1 * m + r1;
  double* Y21 = w.Y + (long)r1 * m + r0;
  // L21 = A21 Y11^T (to scratch, then over A21)
  sliced_nt(L, w.err, b2, b1, b1, 1.0, A21, m, Y11, m, 0.0, w.prod, b1);
  OMM_CUDA_TRY(cudaMemcpy2DAsync(A21, sizeof(double) * m, w.prod, sizeof(double) * b1, sizeof(double) * b1, b2,
                                 cudaMemcpyDeviceToDevice, L.st));
  // A22 -= L21 L21^T
  sliced_nt(L, w.err, b2, b2, b1, -1.0, A21, m, A21, m, 1.0, A22, m);
  chol_inv(w, r1, b2);
  // Z = Y22 L21 (b2 x b1): B operand L21^T (b1 x b2)
  emu::transpose(L.st, A21, b2, b1, m, L.tr0, b2);
  sliced_nt(L, w.err, b2, b1, b2, 1.0, Y22, m, L.tr0, b2, 0.0, w.prod, b1);
  // Y21 = -Z Y11: B operand Y11^T (b1 x b1)
  emu::transpose(L.st, Y11, b1, b1, m, L.tr1, b1);
  sliced_nt(L, w.err, b2, b1, b1, -1.0, w.prod, b1, L.tr1, b1, 0.0, Y21, m);
  if (w.P == nullptr) return;  // the factor and its inverse only
  // this node's Y is final: its P updates may start
  cudaEvent_t ev = nullptr;
  OMM_CUDA_TRY(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  w.events.push_back(ev);
  OMM_CUDA_TRY(cudaEventRecord(ev, L.st));
  OMM_CUDA_TRY(cudaStreamWaitEvent(w.side.st, ev, 0));
  p_update(w, r0, b1, b2);
}

}  // namespace

// chunk sums of the GEMMs with fewer than ~76 output tiles of 128 x 256 (at most 11 chunks)
long partial_capacity(int m) {
  const long h = (m + 1) / 2 + NL;
  return std::min(11L * h * h, 11L * 76 * 128 * 256);
}

size_t spd_inverse_sliced_workspace_bytes(int m) {
  const long h = (m + 1) / 2 + NL;  // the largest off-diagonal block edge (either leaf size)
  // Y, prod, leaf; per lane: tr0, tr1, partial
  const size_t f64 = (size_t)m * m + (size_t)h * h + (size_t)NL * NL +
                     2 * (2 * (size_t)h * h + (size_t)partial_capacity(m));
  const size_t bf = 2 * 2 * (size_t)kInvSlices * (size_t)h * round8(h);  // per lane: sl0, sl1
  return f64 * sizeof(double) + bf * sizeof(__nv_bfloat16) + 4 * 256;
}

namespace {
// P = A^-1 (P != nullptr) and/or L, Y = L^-1 (Y_out != nullptr: A keeps L, zero above the diagonal)
void sliced_impl(cudaStream_t st, int m, double* A, double* P, double* Y_out, void* work, int* info_dev,
                 int* err_dev, int slices) {
  const long h = (m + 1) / 2 + NL;
  SlicedWork w;
  w.m = m;
  // preconditioner grade: 128-wide float32 leaves; float64-class: 64-wide float64 leaves
  w.nb = slices < kInvSlices ? NL : NB;
  w.A = A;
  w.P = P;
  w.info = info_dev;
  w.err = err_dev;
  double* f = static_cast<double*>(work);
  w.Y = Y_out ? Y_out : f;
  f += (long)m * m;
  w.prod = f;
  f += h * h;
  w.leaf = f;
  f += NL * NL;
  for (Lane* L : {&w.main, &w.side}) {
    L->tr0 = f;
    f += h * h;
    L->tr1 = f;
    f += h * h;
    L->partial = f;
    L->partial_cap = partial_capacity(m);
    f += L->partial_cap;
  }
  uintptr_t p = (reinterpret_cast<uintptr_t>(f) + 255) & ~uintptr_t(255);
  const size_t sl = (size_t)kInvSlices * h * round8(h);
  w.main.sl0 = reinterpret_cast<__nv_bfloat16*>(p);
  w.main.sl1 = w.main.sl0 + sl;
  w.side.sl0 = w.main.sl1 + sl;
  w.side.sl1 = w.side.sl0 + sl;
  w.main.st = st;
  w.main.slices = w.side.slices = slices == 1 ? 1 : std::min(std::max(slices, 2), kInvSlices);
  if (w.nb == NL) {
    static bool attr = false;
    if (!attr) {
      OMM_CUDA_TRY(cudaFuncSetAttribute(leaf_f32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kLeafSmem));
      attr = true;
    }
  }
  if (P) OMM_CUDA_TRY(cudaStreamCreateWithFlags(&w.side.st, cudaStreamNonBlocking));
  // streams and events may be released with work pending: the driver frees them once it is done
  auto cleanup = [&]() {
    if (w.side.st) cudaStreamDestroy(w.side.st);
    for (cudaEvent_t e : w.events) cudaEventDestroy(e);
  };
  try {
    OMM_CUDA_TRY(cudaMemsetAsync(info_dev, 0, sizeof(int), st));
    OMM_CUDA_TRY(cudaMemsetAsync(w.Y, 0, sizeof(double) * m * (size_t)m, st));
    if (P) {
      OMM_CUDA_TRY(cudaMemsetAsync(P, 0, sizeof(double) * m * (size_t)m, st));
      cudaEvent_t ready = nullptr;  // the side lane starts after the memsets
      OMM_CUDA_TRY(cudaEventCreateWithFlags(&ready, cudaEventDisableTiming));
      w.events.push_back(ready);
      OMM_CUDA_TRY(cudaEventRecord(ready, st));
      OMM_CUDA_TRY(cudaStreamWaitEvent(w.side.st, ready, 0));
    }
    chol_inv(w, 0, m);
    if (P) {
      cudaEvent_t done = nullptr;  // join: the main lane waits for the last P update
      OMM_CUDA_TRY(cudaEventCreateWithFlags(&done, cudaEventDisableTiming));
      w.events.push_back(done);
      OMM_CUDA_TRY(cudaEventRecord(done, w.side.st));
      OMM_CUDA_TRY(cudaStreamWaitEvent(st, done, 0));
      launch_symmetrize_lower(st, m, P);
    }
    if (Y_out) {
      zero_upper_kernel<<<1024, 256, 0, st>>>(m, A);
      OMM_LAUNCH_CHECK();
    }
  } catch (...) {
    cleanup();
    throw;
  }
  cleanup();
}

}  // namespace

void spd_inverse_sliced(cudaStream_t st, int m, double* A, double* P, void* work, int* info_dev, int* err_dev,
                        int slices) {
  sliced_impl(st, m, A, P, nullptr, work, info_dev, err_dev, slices);
}

void spd_factor_inverse_sliced(cudaStream_t st, int m, double* A, double* Y, void* work, int* info_dev,
                               int* err_dev) {
  sliced_impl(st, m, A, nullptr, Y, work, info_dev, err_dev, kInvSlices);
}

}  // namespace omm
