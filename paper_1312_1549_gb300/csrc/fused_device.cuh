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
      double2 x = make_double2(-a.x, -a.y);
      if (beta != 0.0) {
        const double2 b = *reinterpret_cast<const double2*>(d);
        x = make_double2(fma(beta, b.x, -a.x), fma(beta, b.y, -a.y));
      }
      *reinterpret_cast<double2*>(d) = x;
      split_store2(x.x, x.y, hi, lo, off);
    } else {
      for (int k = 0; k < 2 && c + k < m; ++k) {
        const double x = (beta != 0.0) ? fma(beta, d[k], -p[k]) : -p[k];
        d[k] = x;
        split_store(x, hi, lo, off + k);
      }
    }
  }
}

// one element of the state update of Eq. 16 (mixed path: incremental gradient about the last
// float64-class refresh)
__device__ __forceinline__ void update_element(double x, double& C, double dir, double& HC, double& SC, double HD,
                                               double SD, double& dHC, double& dSC, double& G, double& Gold,
                                               double Gref) {
  C = fma(x, dir, C);
  const double hd = x * HD, sd = x * SD;
  HC += hd;
  SC += sd;
  dHC += hd;
  dSC += sd;
  Gold = G;
  G = fma(8.0, dHC, Gref);
}

// (row, column pair) units of n x m arrays: C, HC, SC += x (Delta, H Delta, S Delta); dHC, dSC +=
// x (H Delta, S Delta); G_old = G; G = G_ref + 8 dHC (the GEMM of the line search adds the rest);
// and the splits of the new HC (rows [0, n)) and SC (rows [n, 2n)) into Yhi/Ylo (leading dimension ldm)
__device__ __forceinline__ void update_state_split_body(long n, long m, double* __restrict__ C,
                                                        double* __restrict__ Y4, const double* __restrict__ Dir,
                                                        double* __restrict__ G, double* __restrict__ Gold,
                                                        double* __restrict__ dY, const double* __restrict__ Gref,
                                                        __nv_bfloat16* __restrict__ Yhi,
                                                        __nv_bfloat16* __restrict__ Ylo, long ldm,
                                                        const Scalars* sc, int bx, int nbx) {
  if (stopped(sc)) return;
  const double x = sc->x;
  const long nm = n * m;
  const bool base_ok = ((m & 1) == 0) &&
                       ((reinterpret_cast<uintptr_t>(C) | reinterpret_cast<uintptr_t>(Y4) |
                         reinterpret_cast<uintptr_t>(dY) | reinterpret_cast<uintptr_t>(G) |
                         reinterpret_cast<uintptr_t>(Gold) | reinterpret_cast<uintptr_t>(Dir) |
                         reinterpret_cast<uintptr_t>(Gref)) & 15) == 0 &&
                       ((reinterpret_cast<uintptr_t>(Yhi) | reinterpret_cast<uintptr_t>(Ylo)) & 3) == 0 &&
                       (ldm & 1) == 0;
  const long units = pair_units(n, m);
  for (long u = bx; u < units; u += nbx) {
    long r, k;
    unit_pos(u, m, r, k);
    if (k >= m) continue;
    const long o = r * m + k;
    const long oh = r * ldm + k, os = (n + r) * ldm + k;
    if (base_ok) {  // k even, m even: the pair is complete and 16-byte aligned
      double2 C2 = *reinterpret_cast<double2*>(C + o), H2 = *reinterpret_cast<double2*>(Y4 + o);
      double2 S2 = *reinterpret_cast<double2*>(Y4 + nm + o), DH2 = *reinterpret_cast<double2*>(dY + o);
      double2 DS2 = *reinterpret_cast<double2*>(dY + nm + o), G2 = *reinterpret_cast<double2*>(G + o);
      const double2 D2 = *reinterpret_cast<const double2*>(Dir + o);
      const double2 HD2 = *reinterpret_cast<const double2*>(Y4 + 2 * nm + o);
      const double2 SD2 = *reinterpret_cast<const double2*>(Y4 + 3 * nm + o);
      const double2 R2 = *reinterpret_cast<const double2*>(Gref + o);
      double2 O2;
      update_element(x, C2.x, D2.x, H2.x, S2.x, HD2.x, SD2.x, DH2.x, DS2.x, G2.x, O2.x, R2.x);
      update_element(x, C2.y, D2.y, H2.y, S2.y, HD2.y, SD2.y, DH2.y, DS2.y, G2.y, O2.y, R2.y);
      *reinterpret_cast<double2*>(C + o) = C2;
      *reinterpret_cast<double2*>(Y4 + o) = H2;
      *reinterpret_cast<double2*>(Y4 + nm + o) = S2;
      *reinterpret_cast<double2*>(dY + o) = DH2;
      *reinterpret_cast<double2*>(dY + nm + o) = DS2;
      *reinterpret_cast<double2*>(G + o) = G2;
      *reinterpret_cast<double2*>(Gold + o) = O2;
      split_store2(H2.x, H2.y, Yhi, Ylo, oh);
      split_store2(S2.x, S2.y, Yhi, Ylo, os);
    } else {
      for (int t = 0; t < 2 && k + t < m; ++t) {
        const long e = o + t;
        double Cv = C[e], Hv = Y4[e], Sv = Y4[nm + e], DHv = dY[e], DSv = dY[nm + e], Gv = G[e], Ov;
        update_element(x, Cv, Dir[e], Hv, Sv, Y4[2 * nm + e], Y4[3 * nm + e], DHv, DSv, Gv, Ov, Gref[e]);
        C[e] = Cv;
        Y4[e] = Hv;
        Y4[nm + e] = Sv;
        dY[e] = DHv;
        dY[nm + e] = DSv;
        G[e] = Gv;
        Gold[e] = Ov;
        split_store(Hv, Yhi, Ylo, oh + t);
        split_store(Sv, Yhi, Ylo, os + t);
      }
    }
  }
}

}  // namespace dev
}  // namespace omm
