// Device-side logic of one OMM line search, shared by the single-instance
// kernels (iter_kernels.cu) and the batched kernels (batched.cu): every body
// takes its block index and block count explicitly, so a batched launch runs
// the same code for instance blockIdx.y.
#pragma once
#include "omm_internal.cuh"

namespace omm {
namespace dev {

constexpr int TB = 256;

__device__ __forceinline__ bool stopped(const Scalars* sc) { return sc->done | sc->halt; }
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
// NaN-propagating (fmax would drop a NaN)
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double w = __shfl_xor_sync(0xffffffffu, v, o);
    v = (w > v || w != w) ? w : v;
  }
  return v;
}
template <int N>
__device__ __forceinline__ void block_sum(double (&v)[N], double (*sh)[TB / 32]) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < N; ++q) {
    const double w = warp_sum(v[q]);
    if (lane == 0) sh[q][wid] = w;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < N; ++q) {
      double s = 0.0;
      for (int k = 0; k < TB / 32; ++k) s += sh[q][k];
      v[q] = s;
    }
  }
  __syncthreads();
}
__device__ __forceinline__ void set_error(Scalars* sc, int status) {
  if (sc->status == 0) sc->status = status;
  sc->halt = 1;
}
__host__ __device__ inline double qd1(const double* a, double x) {
  return a[1] + x * (2.0 * a[2] + x * (3.0 * a[3] + x * 4.0 * a[4]));
}
__host__ __device__ inline double qd2(const double* a, double x) {
  return 2.0 * a[2] + x * (6.0 * a[3] + x * 12.0 * a[4]);
}
__host__ __device__ inline double rtsafe(const double* a, double lo, double hi) {
  double x = 0.5 * (lo + hi);
  double dxold = hi - lo, dx = dxold;
  double f = qd1(a, x), df = qd2(a, x);
  for (int it = 0; it < 200; ++it) {
    if ((((x - hi) * df - f) * ((x - lo) * df - f) > 0.0) || (fabs(2.0 * f) > fabs(dxold * df))) {
      dxold = dx;
      dx = 0.5 * (hi - lo);
      x = lo + dx;
    } else {
      dxold = dx;
      dx = f / df;
      x -= dx;
    }
    // converged to a few units in the last place: a tighter test (1e-16 is below half an ulp) is
    // never met once rounding noise dominates f, and then ran all 200 iterations on the GPU's
    // narrow float64 pipe (about 3 % of random quartics)
    if (fabs(dx) <= 8.9e-16 * fabs(x) || hi - lo <= 8.9e-16 * fabs(hi)) break;
    f = qd1(a, x);
    df = qd2(a, x);
    if (f < 0.0) lo = x; else hi = x;
  }
  return x;
}
// First local minimum of a0 + a1 x + ... + a4 x^4 along x > 0 (a1 < 0):
// the positive axis is cut at the real roots of p'' (where p' turns), p' is
// monotone on each piece, and the first piece on which p' reaches zero from
// below holds the step. Returns 0 and the step, or 3 (OMM_ERR_UNBOUNDED).
__host__ __device__ inline int quartic_first_minimum(const double a[5], double* x_out) {
  *x_out = 0.0;
  if (!(a[1] < 0.0)) return 3;
  // turning points of p': 12 a4 x^2 + 6 a3 x + 2 a2 = 0
  double c[2];
  int nc = 0;
  const double A = 12.0 * a[4], B = 6.0 * a[3], Cc = 2.0 * a[2];
  if (A != 0.0) {
    const double disc = B * B - 4.0 * A * Cc;
    if (disc > 0.0) {
      const double q = -0.5 * (B + copysign(sqrt(disc), B));
      double r1 = q / A, r2 = (q != 0.0) ? Cc / q : r1;
      if (r1 > r2) { const double t = r1; r1 = r2; r2 = t; }
      if (r1 > 0.0) c[nc++] = r1;
      if (r2 > 0.0) c[nc++] = r2;
    }
  } else if (B != 0.0) {
    const double r = -Cc / B;
    if (r > 0.0) c[nc++] = r;
  }
  double lo = 0.0;
  for (int k = 0; k <= nc; ++k) {
    double hi;
    if (k < nc) {
      hi = c[k];
      if (qd1(a, hi) < 0.0) { lo = hi; continue; }
    } else {
      // last piece [lo, inf): p' ends positive only for a positive leading term
      const bool rises = a[4] > 0.0 || (a[4] == 0.0 && (a[3] > 0.0 || (a[3] == 0.0 && a[2] > 0.0)));
      if (!rises) return 3;
      double step = (a[2] > 0.0) ? -a[1] / (2.0 * a[2]) : 1.0;
      if (!(step > 0.0) || !isfinite(step)) step = 1.0;
      hi = lo + step;
      int guard = 0;
      while (qd1(a, hi) < 0.0) {
        lo = hi;
        step *= 2.0;
        hi = lo + step;
        if (++guard > 2000 || !isfinite(hi)) return 3;
      }
    }
    *x_out = rtsafe(a, lo, hi);
    return 0;
  }
  return 3;
}

__device__ __forceinline__ void grad_reduce_body(long count, const double* __restrict__ G, const double* __restrict__ PG,
                   const double* __restrict__ Gold, const double* __restrict__ Dir,
                   double* part, const Scalars* sc, int bx_, int nbx_) {
  if (stopped(sc)) return;
  const bool have_dir = sc->have_dir;
  double v[3] = {0.0, 0.0, 0.0};
  // max|G| on the bit patterns (integer pipe): for |x| they order like the
  // values, and a NaN's pattern exceeds every number's, so the max keeps it
  unsigned long long mb = 0;
  for (long i = bx_ * (long)TB + threadIdx.x; i < count; i += (long)nbx_ * TB) {
    const double g = G[i], pg = PG[i];
    v[0] = fma(g, pg, v[0]);
    if (have_dir) {
      v[1] = fma(Gold[i], pg, v[1]);
      v[2] = fma(g, Dir[i], v[2]);
    }
    mb = max(mb, (unsigned long long)__double_as_longlong(g) & 0x7FFFFFFFFFFFFFFFull);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mb = max(mb, __shfl_xor_sync(0xffffffffu, mb, o));
  __shared__ double sh[3][TB / 32];
  __shared__ double shm[TB / 32];
  const double wm = __longlong_as_double((long long)mb);
  if ((threadIdx.x & 31) == 0) shm[threadIdx.x >> 5] = wm;
  block_sum<3>(v, sh);
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int k = 0; k < TB / 32; ++k) m = (shm[k] > m || shm[k] != shm[k]) ? shm[k] : m;
    part[bx_ * 4 + 0] = v[0];
    part[bx_ * 4 + 1] = v[1];
    part[bx_ * 4 + 2] = v[2];
    part[bx_ * 4 + 3] = m;
  }
}
__device__ __forceinline__ void control_direction_body(Scalars* sc, const double* part, int mixed, int nparts, int bx_, int nbx_) {
  if (stopped(sc)) return;
  double v[3] = {0.0, 0.0, 0.0};
  double mx = 0.0;
  for (int b = threadIdx.x; b < nparts; b += TB) {
    v[0] += part[b * 4 + 0];
    v[1] += part[b * 4 + 1];
    v[2] += part[b * 4 + 2];
    const double a = part[b * 4 + 3];
    mx = (a > mx || a != a) ? a : mx;
  }
  __shared__ double sh[3][TB / 32];
  __shared__ double shm[TB / 32];
  const double wm = warp_max(mx);
  if ((threadIdx.x & 31) == 0) shm[threadIdx.x >> 5] = wm;
  block_sum<3>(v, sh);
  if (threadIdx.x != 0) return;
  double gmax = 0.0;
  for (int k = 0; k < TB / 32; ++k) gmax = (shm[k] > gmax || shm[k] != shm[k]) ? shm[k] : gmax;
  const double gpg = v[0], gopg = v[1], gdo = v[2];
  sc->gmax = gmax;
  sc->gpg = gpg;
  sc->gopg = gopg;
  sc->gdo = gdo;
  if (!isfinite(gmax) || !isfinite(gpg) || !isfinite(gopg) || !isfinite(gdo)) {
    set_error(sc, 5 /* OMM_ERR_NONFINITE */);
    return;
  }
  if (gmax < sc->tol_grad || sc->stop_pending) {
    sc->stop_reason = (gmax < sc->tol_grad) ? 1 : 2;
    sc->done = 1;
    return;
  }
  if (mixed) {
    // refinement request (status stays 0): the target of the round is met, or
    // max|G| has stopped falling (the split-product noise floor is reached)
    if (gmax < sc->halt_gmax) {
      sc->halt = 1;
      return;
    }
    if (gmax < 0.5 * sc->best_g) {
      sc->best_g = gmax;
      sc->best_it = sc->iter_round;
    } else if (sc->iter_round - sc->best_it > sc->stall_window) {
      sc->halt = 1;
      return;
    }
  }
  if (sc->iter >= sc->max_iter) {
    set_error(sc, 4 /* OMM_ERR_NO_CONVERGENCE */);
    return;
  }
  double beta = 0.0;
  if (sc->have_dir && !sc->restart && sc->gpg_old > 0.0) {
    beta = (gpg - gopg) / sc->gpg_old;
    if (!(beta > 0.0)) beta = 0.0;              // PR+
    if (-gpg + beta * gdo >= 0.0) beta = 0.0;   // not a descent direction: restart
  }
  sc->beta = beta;
  sc->restart_dir = beta == 0.0 ? 1 : 0;
  sc->gd = -gpg + beta * gdo;
  sc->gpg_old = gpg;
  sc->restart = 0;
}
__device__ __forceinline__ void direction_body(long count, const double* __restrict__ PG, double* Dir,
                                 const Scalars* sc, int bx_, int nbx_) {
  if (stopped(sc)) return;
  const double beta = sc->beta;
  for (long i = bx_ * (long)blockDim.x + threadIdx.x; i < count; i += (long)nbx_ * blockDim.x)
    Dir[i] = (beta != 0.0) ? fma(beta, Dir[i], -PG[i]) : -PG[i];
}
// float64 -> float32 on the integer pipe, truncating the fraction; magnitudes below the float32
// normal range become zero (the float64 units of this GPU retire about two lanes per SM and clock,
// so even conversions are kept off them where 2^-23 relative accuracy is enough)
__device__ __forceinline__ float f32_trunc(double x) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const unsigned int sign = (unsigned int)(u >> 32) & 0x80000000u;
  const int e = (int)((u >> 52) & 0x7FFu);
  if (e < 1023 - 126) return __uint_as_float(sign);
  if (e > 1023 + 127) return __uint_as_float(sign | 0x7F800000u);
  return __uint_as_float(sign | ((unsigned int)(e - 1023 + 127) << 23) | (unsigned int)((u >> 29) & 0x7FFFFFu));
}

// The trace products of Eq. 13, Tr(XY) = sum_ij X_ij Y_ji, on 32x32 tiles
// with the transposed tiles staged in shared memory.
//   SWHW = [S_W | H_W] (n x 2n), Proj = [H' | S' | H'' | S''] (n x 4n).
//   t0 Tr H'        t1 Tr(S' H_W)   t2 Tr(S_W H')   t3 Tr H''
//   t4 Tr(S'' H_W)  t5 Tr(S_W H'')  t6 Tr(S' H')    t7 Tr(S'^T H')
//   t8 Tr(S'' H')   t9 Tr(S' H'')   t10 Tr(S'' H'')
// F32: the nine product traces multiply float32 copies of the elements (truncated on the integer
// pipe) and sum each thread's products (four per tile) in float32 before the float64 block sums:
// about 2^-20 of each term, far below the error of the tensor-core projections they come from
// (mixed path).
template <bool F32>
__device__ __forceinline__ void traces_body(int n, const double* __restrict__ SWHW, const double* __restrict__ Proj,
              double* part, const Scalars* sc, int bx_, int nbx_) {
  if (stopped(sc)) return;
  const int tiles = (n + 31) / 32;
  __shared__ double tHW[32][33], tH1[32][33], tH2[32][33];
  const long l2 = 2L * n, l4 = 4L * n;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
  double t[kNumTraces];
#pragma unroll
  for (int q = 0; q < kNumTraces; ++q) t[q] = 0.0;
  float f[kNumTraces];
#pragma unroll
  for (int q = 0; q < kNumTraces; ++q) f[q] = 0.0f;
  // 32 x 32 tiles bx_, bx_ + nbx_, ... of the n x n blocks (one per block of the batched launch,
  // several per block of the single launch, whose partial sums then number fewer)
  for (int tile = bx_; tile < tiles * tiles; tile += nbx_) {
    const int I = tile / tiles, J = tile % tiles;
    __syncthreads();  // the previous tile's staged transposes have been read
    // load Y^T tiles: element (i, j) of tile (I, J) needs Y[j][i] from tile (J, I)
    for (int r = ty; r < 32; r += 8) {
      const int gi = J * 32 + r, gj = I * 32 + tx;  // row gi of Y, col gj
      const bool ok = gi < n && gj < n;
      tHW[r][tx] = ok ? SWHW[(long)gi * l2 + n + gj] : 0.0;
      tH1[r][tx] = ok ? Proj[(long)gi * l4 + gj] : 0.0;
      tH2[r][tx] = ok ? Proj[(long)gi * l4 + 2L * n + gj] : 0.0;
    }
    __syncthreads();
    for (int r = ty; r < 32; r += 8) {
      const int gi = I * 32 + r, gj = J * 32 + tx;
      if (gi >= n || gj >= n) continue;
      const double sw = SWHW[(long)gi * l2 + gj];
      const double h1 = Proj[(long)gi * l4 + gj];
      const double s1 = Proj[(long)gi * l4 + n + gj];
      const double s2 = Proj[(long)gi * l4 + 3L * n + gj];
      // Y_ji from the staged transposed tiles: Y[gj][gi] = tile(J,I)[tx][r]
      const double hwT = tHW[tx][r], h1T = tH1[tx][r], h2T = tH2[tx][r];
      if (gi == gj) {
        t[0] += h1;
        t[3] += Proj[(long)gi * l4 + 2L * n + gj];
      }
      if (F32) {
        const float fs1 = f32_trunc(s1), fsw = f32_trunc(sw), fs2 = f32_trunc(s2), fh1 = f32_trunc(h1);
        const float fhwT = f32_trunc(hwT), fh1T = f32_trunc(h1T), fh2T = f32_trunc(h2T);
        f[1] = fmaf(fs1, fhwT, f[1]);
        f[2] = fmaf(fsw, fh1T, f[2]);
        f[4] = fmaf(fs2, fhwT, f[4]);
        f[5] = fmaf(fsw, fh2T, f[5]);
        f[6] = fmaf(fs1, fh1T, f[6]);
        f[7] = fmaf(fs1, fh1, f[7]);
        f[8] = fmaf(fs2, fh1T, f[8]);
        f[9] = fmaf(fs1, fh2T, f[9]);
        f[10] = fmaf(fs2, fh2T, f[10]);
      } else {
        t[1] = fma(s1, hwT, t[1]);
        t[2] = fma(sw, h1T, t[2]);
        t[4] = fma(s2, hwT, t[4]);
        t[5] = fma(sw, h2T, t[5]);
        t[6] = fma(s1, h1T, t[6]);
        t[7] = fma(s1, h1, t[7]);   // Tr(S'^T H') = sum_ij S'_ij H'_ij
        t[8] = fma(s2, h1T, t[8]);
        t[9] = fma(s1, h2T, t[9]);
        t[10] = fma(s2, h2T, t[10]);
      }
    }
  }
  __shared__ double sh[kNumTraces][TB / 32];
  if (F32) {
    // warp sums in float32 (shuffles on the float32 units), one float64 value per warp; the
    // diagonal traces t0, t3 stay float64 throughout
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < kNumTraces; ++q) {
      if (q == 0 || q == 3) {
        const double w = warp_sum(t[q]);
        if (lane == 0) sh[q][wid] = w;
      } else {
        float w = f[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
        if (lane == 0) sh[q][wid] = (double)w;
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
      for (int q = 0; q < kNumTraces; ++q) {
        double acc = 0.0;
        for (int k = 0; k < TB / 32; ++k) acc += sh[q][k];
        part[(long)bx_ * kNumTraces + q] = acc;
      }
    }
    return;
  }
  block_sum<kNumTraces>(t, sh);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < kNumTraces; ++q) part[(long)bx_ * kNumTraces + q] = t[q];
  }
}
__device__ __forceinline__ void control_linesearch_body(Scalars* sc, const double* part, int nblocks, int bx_, int nbx_) {
  if (stopped(sc)) return;
  double t[kNumTraces];
#pragma unroll
  for (int q = 0; q < kNumTraces; ++q) t[q] = 0.0;
  for (int b = threadIdx.x; b < nblocks; b += TB) {
#pragma unroll
    for (int q = 0; q < kNumTraces; ++q) t[q] += part[(long)b * kNumTraces + q];
  }
  __shared__ double sh[kNumTraces][TB / 32];
  block_sum<kNumTraces>(t, sh);
  if (threadIdx.x != 0) return;
  double a[5];
  a[0] = sc->E;
  a[1] = 8.0 * t[0] - 4.0 * t[1] - 4.0 * t[2];
  // Mixed precision: the slope alpha_1 = <G, Delta> (the exact directional
  // derivative of Eq. 8 along Delta) is taken from the float64 reduction over
  // G and Delta instead of the tensor-core traces, whose absolute error would
  // hide its sign once |G| is small.
  if (sc->mixed) a[1] = sc->gd;
  a[2] = 4.0 * t[3] - 2.0 * t[4] - 2.0 * t[5] - 4.0 * t[6] - 4.0 * t[7];
  a[3] = -4.0 * t[8] - 4.0 * t[9];
  a[4] = -2.0 * t[10];
  for (int q = 0; q < kNumTraces; ++q) sc->trace[q] = t[q];
  for (int q = 0; q < 5; ++q) {
    sc->alpha[q] = a[q];
    if (!isfinite(a[q])) { set_error(sc, 5); return; }
  }
  double x;
  if (quartic_first_minimum(a, &x) != 0) {
    sc->x = 0.0;
    if (sc->mixed && sc->iter_round > 0) {
      sc->halt = 1;  // split-product noise: refresh the state in float64 and retry
      return;
    }
    set_error(sc, 3 /* OMM_ERR_UNBOUNDED */);
    return;
  }
  const double Enew = a[0] + x * (a[1] + x * (a[2] + x * (a[3] + x * a[4])));
  if (sc->e_tol > 0.0 && fabs(2.0 * (Enew - sc->E) / (Enew + sc->E)) <= sc->e_tol) sc->stop_pending = 1;
  sc->x = x;
  sc->E = Enew;
  sc->iter += 1;
  sc->iter_round += 1;
  sc->have_dir = 1;
}
__device__ __forceinline__ void update_subspace_body(int n, double* SWHW, const double* __restrict__ Proj, const Scalars* sc, int bx_, int nbx_) {
  if (stopped(sc)) return;
  const double x = sc->x, x2 = x * x;
  const int tiles = (n + 31) / 32;
  const int I = bx_ / tiles, J = bx_ % tiles;
  __shared__ double tH1[32][33], tS1[32][33];
  const long l2 = 2L * n, l4 = 4L * n;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int r = ty; r < 32; r += 8) {
    const int gi = J * 32 + r, gj = I * 32 + tx;
    const bool ok = gi < n && gj < n;
    tH1[r][tx] = ok ? Proj[(long)gi * l4 + gj] : 0.0;
    tS1[r][tx] = ok ? Proj[(long)gi * l4 + n + gj] : 0.0;
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    const int gi = I * 32 + r, gj = J * 32 + tx;
    if (gi >= n || gj >= n) continue;
    const double* pr = Proj + (long)gi * l4;
    const double h = pr[gj] + tH1[tx][r];
    const double s = pr[n + gj] + tS1[tx][r];
    double* sw = SWHW + (long)gi * l2 + gj;
    double* hw = sw + n;
    *hw = fma(x2, pr[2L * n + gj], fma(x, h, *hw));
    *sw = fma(x2, pr[3L * n + gj], fma(x, s, *sw));
  }
}
__device__ __forceinline__ void scale_copy_body(long count, const double* src, double a, double* dst, const Scalars* sc, int bx_, int nbx_) {
  if (sc != nullptr && stopped(sc)) return;
  for (long i = bx_ * (long)blockDim.x + threadIdx.x; i < count; i += (long)nbx_ * blockDim.x)
    dst[i] = a * src[i];
}

}  // namespace dev
}  // namespace omm
