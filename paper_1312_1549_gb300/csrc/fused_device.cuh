// Vector steps of the mixed-precision line search that also write the bf16
// split (hi, lo) of what they produce, so that the next tensor-core product
// reads its operand without a separate split pass over HBM. Shared by the
// single-instance kernels (iter_kernels.cu) and the batched ones (batched.cu);
// every body takes its block index and block count explicitly.
#pragma once
#include "iter_device.cuh"
#include "split_device.cuh"

namespace omm {
namespace dev {

// n x m arrays, by (row, column pair) units: Delta = -PG + beta Delta (Sec. 2.3, Polak-Ribiere
// direction; beta = 0 restarts) and its split into hi/lo (leading dimension ldm)
__device__ __forceinline__ void direction_split_body(long n, long m, const double* __restrict__ PG,
                                                     double* __restrict__ Dir, __nv_bfloat16* __restrict__ hi,
                                                     __nv_bfloat16* __restrict__ lo, long ldm, const Scalars* sc,
                                                     int bx, int nbx) {
  if (stopped(sc)) return;
  const double beta = sc->beta;
  const bool restart = sc->restart_dir != 0;  // beta = 0: the direction is -PG
  const long units = pair_units(n, m);
  for (long u = bx; u < units; u += nbx) {
    long r, c;
    unit_pos(u, m, r, c);
    if (c >= m) continue;
    const double* p = PG + r * m + c;
    double* d = Dir + r * m + c;
    const long off = r * ldm + c;
    const bool vec = c + 1 < m && ((reinterpret_cast<uintptr_t>(p) | reinterpret_cast<uintptr_t>(d)) & 15) == 0 &&
                     ((reinterpret_cast<uintptr_t>(hi + off) | reinterpret_cast<uintptr_t>(lo + off)) & 3) == 0;
    if (vec) {
      const double2 a = *reinterpret_cast<const double2*>(p);
      double2 x;
      if (restart) {  // -PG: a sign flip on the integer pipe
        x = make_double2(__longlong_as_double(__double_as_longlong(a.x) ^ (long long)0x8000000000000000ull),
                         __longlong_as_double(__double_as_longlong(a.y) ^ (long long)0x8000000000000000ull));
      } else {        // one float64 FMA per element (the negation folds into it)
        const double2 b = *reinterpret_cast<const double2*>(d);
        x = make_double2(fma(beta, b.x, -a.x), fma(beta, b.y, -a.y));
      }
      *reinterpret_cast<double2*>(d) = x;
      split_store2_fast(x.x, x.y, hi, lo, off);
    } else {
      for (int k = 0; k < 2 && c + k < m; ++k) {
        const double x = restart ? __longlong_as_double(__double_as_longlong(p[k]) ^ (long long)0x8000000000000000ull)
                                 : fma(beta, d[k], -p[k]);
        d[k] = x;
        split_store_fast(x, hi, lo, off + k);
      }
    }
  }
}

// one element of the state update of Eq. 16 (mixed path: dHC, dSC are the changes since the last
// float64-class refresh, the corrections of the incremental gradient): five float64 FMAs
__device__ __forceinline__ void update_element(double x, double& C, double dir, double& HC, double& SC, double HD,
                                               double SD, double& dHC, double& dSC) {
  C = fma(x, dir, C);
  HC = fma(x, HD, HC);
  SC = fma(x, SD, SC);
  dHC = fma(x, HD, dHC);
  dSC = fma(x, SD, dSC);
}

// (row, column pair) units of n x m arrays: C, HC, SC += x (Delta, H Delta, S Delta) and dHC, dSC
// += x (H Delta, S Delta) (Eq. 16 and the footnote of Sec. 2.3), and the bf16 splits of the new
// values into the operand stack [dHC; dSC; HC; SC; ...] (6n rows of leading dimension ldm; Ylo is
// its lo half). G is not touched: the gradient GEMM's epilogue forms it.
__device__ __forceinline__ void update_state_split_body(long n, long m, double* __restrict__ C,
                                                        double* __restrict__ Y4, const double* __restrict__ Dir,
                                                        double* __restrict__ dY, __nv_bfloat16* __restrict__ Yhi,
                                                        __nv_bfloat16* __restrict__ Ylo, long ldm,
                                                        const Scalars* sc, int bx, int nbx) {
  if (stopped(sc)) return;
  const double x = sc->x;
  const long nm = n * m;
  const bool base_ok = ((m & 1) == 0) &&
                       ((reinterpret_cast<uintptr_t>(C) | reinterpret_cast<uintptr_t>(Y4) |
                         reinterpret_cast<uintptr_t>(dY) | reinterpret_cast<uintptr_t>(Dir)) & 15) == 0 &&
                       ((reinterpret_cast<uintptr_t>(Yhi) | reinterpret_cast<uintptr_t>(Ylo)) & 3) == 0 &&
                       (ldm & 1) == 0;
  const long units = pair_units(n, m);
  for (long u = bx; u < units; u += nbx) {
    long r, k;
    unit_pos(u, m, r, k);
    if (k >= m) continue;
    const long o = r * m + k;
    // stack rows of dHC, dSC, HC, SC for Wannier function r
    const long odh = r * ldm + k, ods = (n + r) * ldm + k, oh = (2 * n + r) * ldm + k, os = (3 * n + r) * ldm + k;
    if (base_ok) {  // k even, m even: the pair is complete and 16-byte aligned
      double2 C2 = *reinterpret_cast<double2*>(C + o), H2 = *reinterpret_cast<double2*>(Y4 + o);
      double2 S2 = *reinterpret_cast<double2*>(Y4 + nm + o), DH2 = *reinterpret_cast<double2*>(dY + o);
      double2 DS2 = *reinterpret_cast<double2*>(dY + nm + o);
      const double2 D2 = *reinterpret_cast<const double2*>(Dir + o);
      const double2 HD2 = *reinterpret_cast<const double2*>(Y4 + 2 * nm + o);
      const double2 SD2 = *reinterpret_cast<const double2*>(Y4 + 3 * nm + o);
      update_element(x, C2.x, D2.x, H2.x, S2.x, HD2.x, SD2.x, DH2.x, DS2.x);
      update_element(x, C2.y, D2.y, H2.y, S2.y, HD2.y, SD2.y, DH2.y, DS2.y);
      *reinterpret_cast<double2*>(C + o) = C2;
      *reinterpret_cast<double2*>(Y4 + o) = H2;
      *reinterpret_cast<double2*>(Y4 + nm + o) = S2;
      *reinterpret_cast<double2*>(dY + o) = DH2;
      *reinterpret_cast<double2*>(dY + nm + o) = DS2;
      split_store2_fast(DH2.x, DH2.y, Yhi, Ylo, odh);
      split_store2_fast(DS2.x, DS2.y, Yhi, Ylo, ods);
      split_store2_fast(H2.x, H2.y, Yhi, Ylo, oh);
      split_store2_fast(S2.x, S2.y, Yhi, Ylo, os);
    } else {
      for (int t = 0; t < 2 && k + t < m; ++t) {
        const long e = o + t;
        double Cv = C[e], Hv = Y4[e], Sv = Y4[nm + e], DHv = dY[e], DSv = dY[nm + e];
        update_element(x, Cv, Dir[e], Hv, Sv, Y4[2 * nm + e], Y4[3 * nm + e], DHv, DSv);
        C[e] = Cv;
        Y4[e] = Hv;
        Y4[nm + e] = Sv;
        dY[e] = DHv;
        dY[nm + e] = DSv;
        split_store_fast(DHv, Yhi, Ylo, odh + t);
        split_store_fast(DSv, Yhi, Ylo, ods + t);
        split_store_fast(Hv, Yhi, Ylo, oh + t);
        split_store_fast(Sv, Yhi, Ylo, os + t);
      }
    }
  }
}

// ---- the mixed path's float32 side quantities (Delta, P G, [H Delta; S Delta], [dHC; dSC]:
// leading dimension ldm; the float64 state C, HC, SC, G has leading dimension m)

// Delta = -PG + beta Delta (beta = 0: -PG) in float32 and its bf16 split, by (row, column pair)
__device__ __forceinline__ void direction_split32_body(long n, long m, const float* __restrict__ PG,
                                                       float* __restrict__ Dir, __nv_bfloat16* __restrict__ hi,
                                                       __nv_bfloat16* __restrict__ lo, long ldm, const Scalars* sc,
                                                       int bx, int nbx) {
  if (stopped(sc)) return;
  const float beta = (float)sc->beta;
  const bool restart = sc->restart_dir != 0;
  const bool pairs = (ldm & 1) == 0;
  const long units = pair_units(n, m);
  for (long u = bx; u < units; u += nbx) {
    long r, c;
    unit_pos(u, m, r, c);
    if (c >= m) continue;
    const long o = r * ldm + c;
    if (pairs && c + 1 < m) {
      const float2 a = *reinterpret_cast<const float2*>(PG + o);
      float2 x;
      if (restart) {
        x = make_float2(-a.x, -a.y);
      } else {
        const float2 b = *reinterpret_cast<const float2*>(Dir + o);
        x = make_float2(fmaf(beta, b.x, -a.x), fmaf(beta, b.y, -a.y));
      }
      *reinterpret_cast<float2*>(Dir + o) = x;
      split_store2_f32(x.x, x.y, hi, lo, o);
    } else {
      for (int k = 0; k < 2 && c + k < m; ++k) {
        const float x = restart ? -PG[o + k] : fmaf(beta, Dir[o + k], -PG[o + k]);
        Dir[o + k] = x;
        split_store_f32(x, hi, lo, o + k);
      }
    }
  }
}

// one element of the state update of Eq. 16 on the float32 side quantities: three float64 FMAs
// (C, HC, SC) and two float32 ones (dHC, dSC, the changes since the last refresh)
__device__ __forceinline__ void update_element32(double x, float xf, double& C, float dir, double& HC, double& SC,
                                                 float HD, float SD, float& dHC, float& dSC) {
  C = fma(x, f64_of_f32(dir), C);
  HC = fma(x, f64_of_f32(HD), HC);
  SC = fma(x, f64_of_f32(SD), SC);
  dHC = fmaf(xf, HD, dHC);
  dSC = fmaf(xf, SD, dSC);
}

// (row, column pair) units: C, HC, SC += x (Delta, H Delta, S Delta), dHC, dSC += x (H Delta,
// S Delta) (Eq. 16 and the footnote of Sec. 2.3), and the bf16 splits of the new dHC, dSC, HC, SC
// into the operand stack rows [0, 4n) (Yhi, Ylo: the stack's hi and lo halves)
__device__ __forceinline__ void update_state_split32_body(long n, long m, double* __restrict__ C,
                                                          double* __restrict__ Y4, const float* __restrict__ Dir,
                                                          const float* __restrict__ HD32, float* __restrict__ dY32,
                                                          __nv_bfloat16* __restrict__ Yhi,
                                                          __nv_bfloat16* __restrict__ Ylo, long ldm,
                                                          const Scalars* sc, int bx, int nbx) {
  if (stopped(sc)) return;
  const double x = sc->x;
  const float xf = (float)x;
  const long nm = n * m, nl = n * ldm;
  const bool base_ok = ((m & 1) == 0) && (ldm & 1) == 0 &&
                       ((reinterpret_cast<uintptr_t>(C) | reinterpret_cast<uintptr_t>(Y4)) & 15) == 0;
  const long units = pair_units(n, m);
  for (long u = bx; u < units; u += nbx) {
    long r, k;
    unit_pos(u, m, r, k);
    if (k >= m) continue;
    const long o = r * m + k, of = r * ldm + k;
    // stack rows of dHC, dSC, HC, SC for Wannier function r
    const long odh = r * ldm + k, ods = (n + r) * ldm + k, oh = (2 * n + r) * ldm + k, os = (3 * n + r) * ldm + k;
    if (base_ok) {  // k even: the pair is complete and aligned
      double2 C2 = *reinterpret_cast<double2*>(C + o), H2 = *reinterpret_cast<double2*>(Y4 + o);
      double2 S2 = *reinterpret_cast<double2*>(Y4 + nm + o);
      float2 DH2 = *reinterpret_cast<float2*>(dY32 + of), DS2 = *reinterpret_cast<float2*>(dY32 + nl + of);
      const float2 D2 = *reinterpret_cast<const float2*>(Dir + of);
      const float2 HD2 = *reinterpret_cast<const float2*>(HD32 + of);
      const float2 SD2 = *reinterpret_cast<const float2*>(HD32 + nl + of);
      update_element32(x, xf, C2.x, D2.x, H2.x, S2.x, HD2.x, SD2.x, DH2.x, DS2.x);
      update_element32(x, xf, C2.y, D2.y, H2.y, S2.y, HD2.y, SD2.y, DH2.y, DS2.y);
      *reinterpret_cast<double2*>(C + o) = C2;
      *reinterpret_cast<double2*>(Y4 + o) = H2;
      *reinterpret_cast<double2*>(Y4 + nm + o) = S2;
      *reinterpret_cast<float2*>(dY32 + of) = DH2;
      *reinterpret_cast<float2*>(dY32 + nl + of) = DS2;
      split_store2_f32(DH2.x, DH2.y, Yhi, Ylo, odh);
      split_store2_f32(DS2.x, DS2.y, Yhi, Ylo, ods);
      split_store2_fast(H2.x, H2.y, Yhi, Ylo, oh);
      split_store2_fast(S2.x, S2.y, Yhi, Ylo, os);
    } else {
      for (int t = 0; t < 2 && k + t < m; ++t) {
        const long e = o + t, ef = of + t;
        double Cv = C[e], Hv = Y4[e], Sv = Y4[nm + e];
        float DHv = dY32[ef], DSv = dY32[nl + ef];
        update_element32(x, xf, Cv, Dir[ef], Hv, Sv, HD32[ef], HD32[nl + ef], DHv, DSv);
        C[e] = Cv;
        Y4[e] = Hv;
        Y4[nm + e] = Sv;
        dY32[ef] = DHv;
        dY32[nl + ef] = DSv;
        split_store_f32(DHv, Yhi, Ylo, odh + t);
        split_store_f32(DSv, Yhi, Ylo, ods + t);
        split_store_fast(Hv, Yhi, Ylo, oh + t);
        split_store_fast(Sv, Yhi, Ylo, os + t);
      }
    }
  }
}

// Without a preconditioner (P = I): per block the sums <G,G>, <G_old,G>, <G,Delta_old> and
// max|G| (as the P G epilogue gives them), then PG = G (float32) and G_old = G
__device__ __forceinline__ void reduce_unpreconditioned_body(long n, long m, const double* __restrict__ G,
                                                             double* __restrict__ Gold,
                                                             const float* __restrict__ Dir,
                                                             float* __restrict__ PG, long ldm, double* part,
                                                             const Scalars* sc, int bx, int nbx) {
  if (stopped(sc)) return;
  const bool have_dir = sc->have_dir;
  double v[3] = {0.0, 0.0, 0.0};
  unsigned long long mb = 0;
  const long count = n * m;
  for (long i = bx * (long)blockDim.x + threadIdx.x; i < count; i += (long)nbx * blockDim.x) {
    const long r = i / m, c = i - r * m, of = r * ldm + c;
    const double g = G[i];
    const double pg = f64_of_f32(f32_rne_bits(g));
    v[0] = fma(g, pg, v[0]);
    if (have_dir) {
      v[1] = fma(Gold[i], pg, v[1]);
      v[2] = fma(g, f64_of_f32(Dir[of]), v[2]);
    }
    mb = max(mb, (unsigned long long)__double_as_longlong(g) & 0x7FFFFFFFFFFFFFFFull);
    PG[of] = f32_rne_bits(g);
    Gold[i] = g;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mb = max(mb, __shfl_xor_sync(0xffffffffu, mb, o));
  __shared__ double sh[3][TB / 32];
  __shared__ double shm[TB / 32];
  if ((threadIdx.x & 31) == 0) shm[threadIdx.x >> 5] = __longlong_as_double((long long)mb);
  block_sum<3>(v, sh);
  if (threadIdx.x == 0) {
    double mx = 0.0;
    for (int k = 0; k < TB / 32; ++k) mx = (shm[k] > mx || shm[k] != shm[k]) ? shm[k] : mx;
    part[bx * 4 + 0] = v[0];
    part[bx * 4 + 1] = v[1];
    part[bx * 4 + 2] = v[2];
    part[bx * 4 + 3] = mx;
  }
}

// H_W += x (H' + H'^T) + x^2 H''; S_W likewise (Eq. 16), on 32 x 32 tiles, and the split of
// [S_W - S_W,ref | H_W - H_W,ref] (n x 2n) into Whi/Wlo (leading dimension ldw): the [dS_W | dH_W]
// columns of the gradient GEMM's A operand
__device__ __forceinline__ void update_subspace_split_body(int n, double* SWHW, const double* __restrict__ Proj,
                                                           const double* __restrict__ Wref,
                                                           __nv_bfloat16* __restrict__ Whi,
                                                           __nv_bfloat16* __restrict__ Wlo, long ldw,
                                                           const Scalars* sc, int bx_, int nbx_) {
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
    const double hn = fma(x2, pr[2L * n + gj], fma(x, h, *hw));
    const double sn = fma(x2, pr[3L * n + gj], fma(x, s, *sw));
    *hw = hn;
    *sw = sn;
    const double* wr = Wref + (long)gi * l2 + gj;
    split_store_fast(sn - wr[0], Whi, Wlo, (long)gi * ldw + gj);
    split_store_fast(hn - wr[n], Whi, Wlo, (long)gi * ldw + n + gj);
  }
}

}  // namespace dev
}  // namespace omm
