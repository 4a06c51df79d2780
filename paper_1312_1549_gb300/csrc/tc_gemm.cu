// BF16 tensor-core GEMM for sm_103a: tcgen05.mma with the accumulator in
// tensor memory (TMEM), operands moved global -> shared by TMA
// (cp.async.bulk.tensor, 128-byte swizzle), a ring of 64-wide K stages and
// warp specialisation:
//   warp 0      TMA producer (one lane)
//   warp 1      TMEM allocation and the MMA issuer (one lane)
//   warps 2-5   epilogue: tcgen05.ld of the 128 x 256 FP32 accumulator,
//               C = alpha * acc + beta * C written in float64
// Each CTA computes one 128 x 256 (or 128 x 128) tile of C = A B^T with A (M x K)
// and B (N x K) both K-major bf16 (or B MN-major); the split form also runs on
// pairs of SMs (a cluster of two CTAs, tcgen05 cta_group::2, 256-row tiles; see
// pair_body). Operands are stacks of slices; a pair list
// says which slice products are accumulated (passes over K into the same
// accumulator). "Split" operands x = x_hi + x_lo use the three pairs
// A_hi B_hi + A_hi B_lo + A_lo B_hi, which keep about 16 significant bits;
// the float64 emulation (emu_gemm.cu) uses fixed-point slices.
//
// Every wait on an mbarrier is bounded (globaltimer, 2 s): on expiry the
// kernel records an error code, stops issuing work and frees its TMEM.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include "omm_internal.cuh"
#include "split_device.cuh"
#include "tc_gemm.cuh"

#include <algorithm>
#include <map>
#include <mutex>
#include <string>
#include <vector>

namespace omm {
namespace tc {
namespace {

// K is consumed in stages of BK = 64 contracted columns (one 128-byte swizzle atom of bf16 per
// row). Stages of 32 columns (64-byte swizzle) were measured slower: twice the barrier and commit
// round trips per contracted column, for no gain in the bytes kept in flight.
constexpr int BM = 128, BN = 256, BK = 64;
constexpr int A_BYTES = BM * BK * 2;
constexpr int B_BYTES = BN * BK * 2;
// the stage ring; 224 KB (seven or eight single-pass stages) was measured slower than 192 KB:
// the larger shared-memory carve-out leaves less L1 for the epilogues' loads
constexpr int RING_BYTES = 192 * 1024;
constexpr int MAX_STAGES = 10;          // barrier room: 2 * stages + 5 barriers in 256 bytes
constexpr int TMEM_COLS = 256;
constexpr int NTHREADS = 192;
constexpr int SMEM_BYTES = RING_BYTES + 1024 /*align*/ + 256 /*barriers*/;
constexpr int ring_stages(int stage_bytes) {
  return RING_BYTES / stage_bytes < MAX_STAGES ? RING_BYTES / stage_bytes : MAX_STAGES;
}
constexpr unsigned long long WAIT_NS = 2000000000ull;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t globaltimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// bounded wait: false after limit_ns without completion
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, uint64_t limit_ns = WAIT_NS) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = globaltimer();
  for (uint32_t i = 1;; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((i & 255u) == 0 && globaltimer() - t0 > limit_ns) return false;
  }
}

constexpr uint64_t EXPIRE_NS = 1000000ull;  // the test expiry of Epilogue::expire: 1 ms

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, uint32_t bar, int c0, int c1) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4}], [%2];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(bar), "r"(c0), "r"(c1)
      : "memory");
}

__device__ __forceinline__ void prefetch_tmap(const CUtensorMap* map) {
  asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

// UMMA shared-memory descriptor: K-major, 128-byte swizzle (rows of 64 bf16), 8-row groups
// 1024 B apart.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFF);          // start address
  d |= (uint64_t)(16 >> 4) << 16;                 // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;               // stride byte offset: next 8 rows
  d |= (uint64_t)1 << 46;                         // descriptor version (sm_100 family)
  d |= (uint64_t)2 << 61;                         // layout: SWIZZLE_128B
  return d;
}

// UMMA shared-memory descriptor of an MN-major operand, 128-byte swizzle: each 1024-byte atom
// holds 8 contracted rows of 64 output-index elements (128 B each); atoms of the next 64 output
// indices are 8 KB apart (leading byte offset) and those of the next 8 contracted rows 1 KB apart
// (stride byte offset). This is the layout a 64-column x 64-row TMA box with 128-byte swizzle
// leaves in shared memory, the boxes of one stage placed 8 KB apart along the output index.
constexpr int MN_BOX_BYTES = 64 * BK * 2;
__device__ __forceinline__ uint64_t smem_desc_mn(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFF);          // start address
  d |= (uint64_t)(MN_BOX_BYTES >> 4) << 16;       // leading byte offset: next 64 output indices
  d |= (uint64_t)(1024 >> 4) << 32;               // stride byte offset: next 8 contracted rows
  d |= (uint64_t)1 << 46;                         // descriptor version (sm_100 family)
  d |= (uint64_t)2 << 61;                         // layout: SWIZZLE_128B
  return d;
}

// instruction descriptor, kind::f16: D f32, A/B bf16, both K-major, M x N
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
// the same with B MN-major (the transpose bit of B)
constexpr uint32_t kIdescBMN = 1u << 16;

__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void umma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
               : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
        "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
        "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
        "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// float -> float64 on the integer pipe (exact): the float64 units of this GPU
// retire about two instructions per SM and clock, so the epilogue widens the
// FP32 accumulator by rebiasing the exponent (127 -> 1023) and shifting the
// mantissa; zeros keep their sign, subnormals are normalised, infinities and
// NaNs keep their class.
__device__ __forceinline__ double widen(float f) {
  const unsigned int u = __float_as_uint(f);
  const unsigned int e = (u >> 23) & 0xFFu, m = u & 0x7FFFFFu;
  const unsigned long long sign = (unsigned long long)(u & 0x80000000u) << 32;
  unsigned long long bits;
  if (e != 0 && e != 0xFFu) {
    bits = sign | ((unsigned long long)(e + (1023u - 127u)) << 52) | ((unsigned long long)m << 29);
  } else if (e == 0xFFu) {
    bits = sign | (0x7FFull << 52) | ((unsigned long long)m << 29);
  } else if (m == 0) {
    bits = sign;
  } else {  // subnormal: m 2^-149 with its top bit at position p
    const int p = 31 - __clz(m);
    bits = sign | ((unsigned long long)(p - 149 + 1023) << 52) |
           (((unsigned long long)m << (52 - p)) & 0x000FFFFFFFFFFFFFull);
  }
  return __longlong_as_double((long long)bits);
}

// alpha a + beta c in float64 (the same operations on every path)
__device__ __forceinline__ double combine(const Epilogue& ep, double a, const double* c) {
  if (ep.beta == 0.0) return ep.alpha == 1.0 ? a : ep.alpha * a;
  if (ep.beta == 1.0) return fma(ep.alpha, a, *c);
  return fma(ep.beta, *c, ep.alpha * a);
}

// running sums of one epilogue thread in kEpReduce mode
struct EpiRed {
  double v0 = 0.0, v1 = 0.0, v2 = 0.0;
  unsigned long long mb = 0;  // max |g| as bits (integer pipe; a NaN's pattern exceeds every number's)
  bool have_dir = false;
};

// One output element of a fused form (see Epilogue): accumulator value a (FP32) at row, column
// col of block blk (cb = col within the block); stores C (and its split) and returns nothing.
__device__ __forceinline__ void fused_element(const Epilogue& ep, float a, int row, long blk, long cb, EpiRed& red) {
  const long offc = blk * ep.split_stride + (long)row * ep.ldc + cb;
  double out;
  if (ep.mode == kEpGrad) {
    const long ox = (long)row * ep.ldx + cb, of = (long)row * ep.ldf + cb;
    out = ep.x0[ox] + widen(fmaf((float)ep.xs, ep.x1f[of], (float)ep.alpha * a));
  } else if (ep.mode == kEpReduce) {
    const long ox = (long)row * ep.ldx + cb, of = (long)row * ep.ldf + cb;
    const double pg = widen(a), g = ep.x0[ox];
    red.v0 = fma(g, pg, red.v0);
    if (red.have_dir) {
      red.v1 = fma(ep.x1[ox], pg, red.v1);
      red.v2 = fma(g, dev::f64_of_f32(ep.x2f[of]), red.v2);
    }
    red.mb = max(red.mb, (unsigned long long)__double_as_longlong(g) & 0x7FFFFFFFFFFFFFFFull);
    ep.xout[ox] = g;
    reinterpret_cast<float*>(ep.C)[offc] = a;
    if (ep.bf_hi != nullptr) {
      __nv_bfloat16* hp = ep.bf_hi + blk * ep.bf_blk + (long)row * ep.bf_ld;
      dev::split_store_f32(a, hp, hp + ep.bf_lo, cb);
    }
    return;
  } else if (ep.c_f32) {
    const float o = ep.alpha == 1.0 ? a : (float)ep.alpha * a;
    reinterpret_cast<float*>(ep.C)[offc] = o;
    if (ep.bf_hi != nullptr) {
      __nv_bfloat16* hp = ep.bf_hi + blk * ep.bf_blk + (long)row * ep.bf_ld;
      dev::split_store_f32(o, hp, hp + ep.bf_lo, cb);
    }
    return;
  } else {
    out = combine(ep, widen(a), ep.C + offc);
  }
  ep.C[offc] = out;
  if (ep.bf_hi != nullptr) {
    __nv_bfloat16* hp = ep.bf_hi + blk * ep.bf_blk + (long)row * ep.bf_ld;
    dev::split_store_fast(out, hp, hp + ep.bf_lo, cb);
  }
}

// eight bf16 values into one 16-byte store
__device__ __forceinline__ void store_bf8(__nv_bfloat16* p, const unsigned short (&h)[8]) {
  *reinterpret_cast<uint4*>(p) = make_uint4(h[0] | ((uint32_t)h[1] << 16), h[2] | ((uint32_t)h[3] << 16),
                                            h[4] | ((uint32_t)h[5] << 16), h[6] | ((uint32_t)h[7] << 16));
}

// The fused forms, float32 outputs and split outputs for the 32 accumulator columns of a row whose
// float64 data (C unless c_f32, x0, x1, xout) starts on an 8-byte but not a 16-byte boundary (a
// row of an odd leading dimension): eight columns at a time, 8-byte accesses to those arrays and
// the usual vector accesses to the float32 and split arrays. offc, offx, offf, bf0: the row's first
// element in C, in x0/x1/xout, in x1f/x2f and in the split outputs.
__device__ __forceinline__ float f4_at(const float4& q, int i) { return i == 0 ? q.x : (i == 1 ? q.y : (i == 2 ? q.z : q.w)); }

__device__ __forceinline__ void store_chunk_odd(const Epilogue& ep, long offc, long offx, long offf, long bf0,
                                                const float (&v)[32], EpiRed& red) {
  const bool unit = ep.alpha == 1.0 && ep.beta == 0.0;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int c8 = 8 * q;
    if (ep.c_f32) {
      float o[8];
      const float al = (float)ep.alpha;
#pragma unroll
      for (int k = 0; k < 8; ++k) o[k] = (ep.mode == kEpReduce || unit) ? v[c8 + k] : al * v[c8 + k];
      if (ep.mode == kEpReduce) {
        double g[8], go[8];
        float4 d[2];
#pragma unroll
        for (int k = 0; k < 8; ++k) g[k] = __ldg(ep.x0 + offx + c8 + k);
        if (red.have_dir) {
#pragma unroll
          for (int k = 0; k < 8; ++k) go[k] = ep.x1[offx + c8 + k];  // x1 may alias xout
#pragma unroll
          for (int k = 0; k < 2; ++k) d[k] = __ldg(reinterpret_cast<const float4*>(ep.x2f + offf + c8) + k);
        }
        // float32 sums of these 8 products, widened into the float64 running sums (as in the
        // 16-column form)
        float s0 = 0.f, s1 = 0.f, s2 = 0.f;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const float gk = dev::f32_rne_bits(g[k]);
          s0 = fmaf(gk, o[k], s0);
          red.mb = max(red.mb, (unsigned long long)__double_as_longlong(g[k]) & 0x7FFFFFFFFFFFFFFFull);
          if (red.have_dir) {
            s1 = fmaf(dev::f32_rne_bits(go[k]), o[k], s1);
            s2 = fmaf(gk, f4_at(d[k >> 2], k & 3), s2);
          }
        }
        red.v0 += widen(s0);
        if (red.have_dir) {
          red.v1 += widen(s1);
          red.v2 += widen(s2);
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) ep.xout[offx + c8 + k] = g[k];
      }
      float4* c4 = reinterpret_cast<float4*>(reinterpret_cast<float*>(ep.C) + offc + c8);
      c4[0] = make_float4(o[0], o[1], o[2], o[3]);
      c4[1] = make_float4(o[4], o[5], o[6], o[7]);
      if (ep.bf_hi != nullptr) {
        unsigned short h[8], l[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) dev::split_bits_f32(o[k], h[k], l[k]);
        __nv_bfloat16* hp = ep.bf_hi + bf0 + c8;
        store_bf8(hp, h);
        store_bf8(hp + ep.bf_lo, l);
      }
      continue;
    }
    double out[8];
    if (ep.mode == kEpGrad) {
      double a0[8];
      float4 a1[2];
#pragma unroll
      for (int k = 0; k < 8; ++k) a0[k] = __ldg(ep.x0 + offx + c8 + k);
#pragma unroll
      for (int k = 0; k < 2; ++k) a1[k] = __ldg(reinterpret_cast<const float4*>(ep.x1f + offf + c8) + k);
      const float alf = (float)ep.alpha, xsf = (float)ep.xs;
#pragma unroll
      for (int k = 0; k < 8; ++k) out[k] = a0[k] + widen(fmaf(xsf, f4_at(a1[k >> 2], k & 3), alf * v[c8 + k]));
    } else if (unit) {
#pragma unroll
      for (int k = 0; k < 8; ++k) out[k] = widen(v[c8 + k]);
    } else {
#pragma unroll
      for (int k = 0; k < 8; ++k) out[k] = combine(ep, widen(v[c8 + k]), ep.C + offc + c8 + k);
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) ep.C[offc + c8 + k] = out[k];
    if (ep.bf_hi != nullptr) {
      unsigned short h[8], l[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) dev::split_bits_fast(out[k], h[k], l[k]);
      __nv_bfloat16* hp = ep.bf_hi + bf0 + c8;
      store_bf8(hp, h);
      store_bf8(hp + ep.bf_lo, l);
    }
  }
}

// C = alpha * v + beta * C (or a fused form) for the 32 accumulator columns [col0, col0 + 32) of one row.
__device__ __forceinline__ void store_chunk(const Epilogue& ep, int row, int col0, const float (&v)[32], EpiRed& red) {
  if (row >= ep.M || col0 >= ep.N) return;
  const int nvalid = min(32, ep.N - col0);
  const long blk0 = col0 / ep.split_cols;
  const long blk1 = (col0 + nvalid - 1) / ep.split_cols;
  if (ep.mode == kEpPlain && ep.bf_hi == nullptr && !ep.c_f32) {
    if (blk0 == blk1) {  // specialised loops, no per-element branching
      double* base = ep.C + blk0 * ep.split_stride + (long)row * ep.ldc + (col0 - blk0 * ep.split_cols);
      if (ep.beta == 0.0) {
        if (ep.alpha == 1.0) {
#pragma unroll
          for (int j = 0; j < 32; ++j)
            if (j < nvalid) base[j] = widen(v[j]);
        } else {
#pragma unroll
          for (int j = 0; j < 32; ++j)
            if (j < nvalid) base[j] = ep.alpha * widen(v[j]);
        }
      } else if (ep.beta == 1.0) {
#pragma unroll
        for (int j = 0; j < 32; ++j)
          if (j < nvalid) base[j] = fma(ep.alpha, widen(v[j]), base[j]);
      } else {
#pragma unroll
        for (int j = 0; j < 32; ++j)
          if (j < nvalid) base[j] = fma(ep.beta, base[j], ep.alpha * widen(v[j]));
      }
      return;
    }
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      if (j >= nvalid) break;
      const int col = col0 + j;
      const long blk = col / ep.split_cols;
      double* p = ep.C + blk * ep.split_stride + (long)row * ep.ldc + (col - blk * ep.split_cols);
      *p = combine(ep, widen(v[j]), p);
    }
    return;
  }
  // fused forms, float32 outputs and split outputs. Every index into v is a compile-time constant
  // (the accumulator values stay in registers); sixteen columns at a time, their inputs loaded
  // first (read-only path, 16-byte vectors) so that one memory latency covers them all.
  const long cb0 = col0 - blk0 * ep.split_cols;
  const long offc = blk0 * ep.split_stride + (long)row * ep.ldc + cb0;
  const long offx = (long)row * ep.ldx + cb0, offf = (long)row * ep.ldf + cb0;
  const long bf0 = blk0 * ep.bf_blk + (long)row * ep.bf_ld + cb0;
  const bool fused = ep.mode != kEpPlain;
  const bool vec8 = blk0 == blk1 && nvalid == 32 && (!ep.c_f32 || (offc & 3) == 0) && (!fused || (offf & 3) == 0) &&
                    (ep.bf_hi == nullptr || ((bf0 & 7) == 0 && (ep.bf_lo & 7) == 0));
  // the float64 rows on 16-byte boundaries too (an even leading dimension)
  const bool vec = vec8 && (ep.c_f32 || (offc & 1) == 0) && (!fused || (offx & 1) == 0);
  if (vec8 && !vec) {
    store_chunk_odd(ep, offc, offx, offf, bf0, v, red);
    return;
  }
  if (vec) {
    const bool unit = ep.alpha == 1.0 && ep.beta == 0.0;  // plain store of the accumulator
#pragma unroll
    for (int h16 = 0; h16 < 2; ++h16) {
      const int c16 = 16 * h16;
      if (ep.c_f32) {  // float32 output: the accumulator itself (kEpReduce, or kEpPlain with alpha 1)
        float o[16];
        const float al = (float)ep.alpha;
#pragma unroll
        for (int k = 0; k < 16; ++k) o[k] = (ep.mode == kEpReduce || unit) ? v[c16 + k] : al * v[c16 + k];
        if (ep.mode == kEpReduce) {
          double2 g[8], go[8];
          float4 d[4];
#pragma unroll
          for (int k = 0; k < 8; ++k) {
            g[k] = __ldg(reinterpret_cast<const double2*>(ep.x0 + offx + c16) + k);
            if (red.have_dir) go[k] = *(reinterpret_cast<const double2*>(ep.x1 + offx + c16) + k);
          }
          if (red.have_dir) {
#pragma unroll
            for (int k = 0; k < 4; ++k) d[k] = __ldg(reinterpret_cast<const float4*>(ep.x2f + offf + c16) + k);
          }
          // the sums of these 16 products in float32 (g rounded to float32 on the integer pipe),
          // then widened into the float64 running sums: 3 float64 adds per 16 elements instead of
          // 3 float64 FMAs per element on this GPU's narrow float64 pipe. The sums steer the
          // direction (Polak-Ribiere) and give the slope <G, Delta>; 16-term float32 sums carry
          // about 2^-20 of their absolute terms, far below what either needs.
          float s0 = 0.f, s1 = 0.f, s2 = 0.f;
#pragma unroll
          for (int k = 0; k < 8; ++k) {
            const float gx = dev::f32_rne_bits(g[k].x), gy = dev::f32_rne_bits(g[k].y);
            s0 = fmaf(gx, o[2 * k], s0);
            s0 = fmaf(gy, o[2 * k + 1], s0);
            red.mb = max(red.mb, (unsigned long long)__double_as_longlong(g[k].x) & 0x7FFFFFFFFFFFFFFFull);
            red.mb = max(red.mb, (unsigned long long)__double_as_longlong(g[k].y) & 0x7FFFFFFFFFFFFFFFull);
            if (red.have_dir) {
              s1 = fmaf(dev::f32_rne_bits(go[k].x), o[2 * k], s1);
              s1 = fmaf(dev::f32_rne_bits(go[k].y), o[2 * k + 1], s1);
              const float dx = (k & 1) ? d[k >> 1].z : d[k >> 1].x, dy = (k & 1) ? d[k >> 1].w : d[k >> 1].y;
              s2 = fmaf(gx, dx, s2);
              s2 = fmaf(gy, dy, s2);
            }
          }
          red.v0 += widen(s0);
          if (red.have_dir) {
            red.v1 += widen(s1);
            red.v2 += widen(s2);
          }
#pragma unroll
          for (int k = 0; k < 8; ++k) *(reinterpret_cast<double2*>(ep.xout + offx + c16) + k) = g[k];
        }
        float4* c4 = reinterpret_cast<float4*>(reinterpret_cast<float*>(ep.C) + offc + c16);
#pragma unroll
        for (int k = 0; k < 4; ++k) c4[k] = make_float4(o[4 * k], o[4 * k + 1], o[4 * k + 2], o[4 * k + 3]);
        if (ep.bf_hi != nullptr) {
#pragma unroll
          for (int g8 = 0; g8 < 2; ++g8) {
            unsigned short h[8], l[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) dev::split_bits_f32(o[8 * g8 + k], h[k], l[k]);
            __nv_bfloat16* hp = ep.bf_hi + bf0 + c16 + 8 * g8;
            store_bf8(hp, h);
            store_bf8(hp + ep.bf_lo, l);
          }
        }
        continue;
      }
      double out[16];
      if (ep.mode == kEpGrad) {
        double2 a0[8];
        float4 a1[4];
#pragma unroll
        for (int k = 0; k < 8; ++k) a0[k] = __ldg(reinterpret_cast<const double2*>(ep.x0 + offx + c16) + k);
#pragma unroll
        for (int k = 0; k < 4; ++k) a1[k] = __ldg(reinterpret_cast<const float4*>(ep.x1f + offf + c16) + k);
        // the increment xs x1f + alpha acc in float32 (one rounding, 2^-24 of it, far below the
        // split product's own 2^-17), then one float64 add onto x0
        const float alf = (float)ep.alpha, xsf = (float)ep.xs;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const float fx = (k & 1) ? a1[k >> 1].z : a1[k >> 1].x, fy = (k & 1) ? a1[k >> 1].w : a1[k >> 1].y;
          out[2 * k] = a0[k].x + widen(fmaf(xsf, fx, alf * v[c16 + 2 * k]));
          out[2 * k + 1] = a0[k].y + widen(fmaf(xsf, fy, alf * v[c16 + 2 * k + 1]));
        }
      } else if (unit) {
#pragma unroll
        for (int k = 0; k < 16; ++k) out[k] = widen(v[c16 + k]);
      } else {
#pragma unroll
        for (int k = 0; k < 16; ++k) out[k] = combine(ep, widen(v[c16 + k]), ep.C + offc + c16 + k);
      }
      double2* c2 = reinterpret_cast<double2*>(ep.C + offc + c16);
#pragma unroll
      for (int k = 0; k < 8; ++k) c2[k] = make_double2(out[2 * k], out[2 * k + 1]);
      if (ep.bf_hi != nullptr) {
#pragma unroll
        for (int g8 = 0; g8 < 2; ++g8) {
          unsigned short h[8], l[8];
#pragma unroll
          for (int k = 0; k < 8; ++k) dev::split_bits_fast(out[8 * g8 + k], h[k], l[k]);
          __nv_bfloat16* hp = ep.bf_hi + bf0 + c16 + 8 * g8;
          store_bf8(hp, h);
          store_bf8(hp + ep.bf_lo, l);
        }
      }
    }
    return;
  }
#pragma unroll
  for (int j = 0; j < 32; ++j) {
    if (j >= nvalid) break;
    const int col = col0 + j;
    const long blk = col / ep.split_cols;
    fused_element(ep, v[j], row, blk, col - blk * ep.split_cols, red);
  }
}

// kEpReduce: the epilogue warp's sums of this tile into its partial slot (fixed order)
__device__ __forceinline__ void flush_reduce(const Epilogue& ep, int tile, int ewarp, EpiRed& red) {
  if (ep.mode != kEpReduce) return;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    red.v0 += __shfl_xor_sync(0xffffffffu, red.v0, o);
    red.v1 += __shfl_xor_sync(0xffffffffu, red.v1, o);
    red.v2 += __shfl_xor_sync(0xffffffffu, red.v2, o);
    red.mb = max(red.mb, __shfl_xor_sync(0xffffffffu, red.mb, o));
  }
  if ((threadIdx.x & 31) == 0) {
    double* p = ep.part + ((long)tile * 4 + ewarp) * 4;
    p[0] = red.v0;
    p[1] = red.v1;
    p[2] = red.v2;
    p[3] = __longlong_as_double((long long)red.mb);
  }
}

// One 128 x 256 output tile (shared by the single and the grouped kernel).
// FUSED: the pair list is the split form (A_hi B_hi + A_hi B_lo + A_lo B_hi);
// each stage then holds A_hi, A_lo, B_hi and B_lo of one K block (96 KB, two
// stages) and feeds three MMA groups, so every operand byte is fetched once
// per K block instead of once per pair (2.25x less shared-memory fill traffic).
template <bool FUSED>
__device__ __forceinline__ void gemm_tile(const CUtensorMap* mA, const CUtensorMap* mB, int K, int rowsA,
                                          int rowsB, int offA, int offB, const PairList& pl, const Epilogue& ep_in,
                                          int tile) {
  constexpr int SB = FUSED ? 2 * (A_BYTES + B_BYTES) : (A_BYTES + B_BYTES);
  constexpr int NS = ring_stages(SB);
  static_assert(NS >= 2 && NS * SB <= RING_BYTES && 2 * NS + 2 <= 28, "stage ring");
  const Epilogue ep = ep_in;
  if (ep.skip != nullptr && (ep.skip[0] | ep.skip[1])) return;  // uniform: before any resource use
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + NS * SB);
  // bars[0..S) full, bars[S..2S) empty, bars[2S] accumulator ready
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * NS + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // M-fastest rasterisation: CTAs that run together share one B tile (read
  // from DRAM once, then from L2) and sweep the small A operand
  const int tiles_m = (ep.M + BM - 1) / BM;
  const int m0 = (tile % tiles_m) * BM, n0 = (tile / tiles_m) * BN;
  const int nkb = (K + BK - 1) / BK;
  const int total = FUSED ? nkb : pl.n * nkb;

  if (threadIdx.x == 0) {
    for (int s = 0; s < NS; ++s) {
      mbar_init(smem_u32(&bars[s]), 1);
      mbar_init(smem_u32(&bars[NS + s]), 1);
    }
    mbar_init(smem_u32(&bars[2 * NS]), 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer
    prefetch_tmap(mA);
    prefetch_tmap(mB);
    int armed = 0;
    for (int t = 0; t < total; ++t) {
      const int s = t % NS, r = t / NS;
      if (!mbar_wait(smem_u32(&bars[NS + s]), (r & 1) ^ 1)) {
        *abort_flag = 1;
        atomicCAS(ep.err, 0, 1);
        break;
      }
      if (*abort_flag) break;
      const uint32_t full = smem_u32(&bars[s]);
      const uint32_t sa = smem_u32(smem + s * SB);
      mbar_expect_tx(full, SB);
      if (FUSED) {
        const int kb = t;
        tma_load_2d(sa, mA, full, kb * BK, offA + m0);                                  // A_hi
        tma_load_2d(sa + A_BYTES, mA, full, kb * BK, rowsA + offA + m0);               // A_lo
        tma_load_2d(sa + 2 * A_BYTES, mB, full, kb * BK, offB + n0);                   // B_hi
        tma_load_2d(sa + 2 * A_BYTES + B_BYTES, mB, full, kb * BK, rowsB + offB + n0); // B_lo
      } else {
        const int p = t / nkb, kb = t % nkb;
        tma_load_2d(sa, mA, full, kb * BK, (int)pl.a[p] * rowsA + offA + m0);
        tma_load_2d(sa + A_BYTES, mB, full, kb * BK, (int)pl.b[p] * rowsB + offB + n0);
      }
      ++armed;
    }
    if (*abort_flag) {  // let the copies already issued land before the CTA releases its memory
      for (int j = armed > NS ? armed - NS : 0; j < armed; ++j) mbar_wait(smem_u32(&bars[j % NS]), (j / NS) & 1);
    }
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer
    constexpr uint32_t idesc = idesc_bf16(BM, BN);
    int t = 0;
    for (; t < total; ++t) {
      const int s = t % NS, r = t / NS;
      if (!mbar_wait(smem_u32(&bars[s]), r & 1)) {
        *abort_flag = 1;
        atomicCAS(ep.err, 0, 2);
        break;
      }
      if (*abort_flag) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t sa = smem_u32(smem + s * SB);
      if (FUSED) {
        const uint32_t alo = sa + A_BYTES, bhi = sa + 2 * A_BYTES, blo = bhi + B_BYTES;
#pragma unroll
        for (int k = 0; k < BK / 16; ++k) {
          umma_bf16(tmem, smem_desc(sa + k * 32), smem_desc(bhi + k * 32), idesc, (t > 0 || k > 0) ? 1u : 0u);
          umma_bf16(tmem, smem_desc(sa + k * 32), smem_desc(blo + k * 32), idesc, 1u);
          umma_bf16(tmem, smem_desc(alo + k * 32), smem_desc(bhi + k * 32), idesc, 1u);
        }
      } else {
        const uint32_t sb = sa + A_BYTES;
#pragma unroll
        for (int k = 0; k < BK / 16; ++k) {
          umma_bf16(tmem, smem_desc(sa + k * 32), smem_desc(sb + k * 32), idesc, (t > 0 || k > 0) ? 1u : 0u);
        }
      }
      umma_commit(smem_u32(&bars[NS + s]));  // stage s is free once these MMAs have read it
    }
    umma_commit(smem_u32(&bars[2 * NS]));    // accumulator complete (also on abort: drains MMAs)
    if (*abort_flag) mbar_wait(smem_u32(&bars[2 * NS]), 0);  // the MMAs issued before are done
  } else if (warp >= 2) {
    // ---------------- epilogue
    const bool ok = mbar_wait(smem_u32(&bars[2 * NS]), 0);
    if (!ok) atomicCAS(ep.err, 0, 3);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const int lane_base = (warp & 3) * 32;
    const int row = m0 + lane_base + lane;
    const bool write = ok && !*abort_flag;
    EpiRed red;
    red.have_dir = ep.mode == kEpReduce && ep.sc != nullptr && ep.sc->have_dir;
#pragma unroll 1
    for (int c = 0; c < BN / 32; ++c) {
      float v[32];
      tmem_ld32(tmem + ((uint32_t)lane_base << 16) + (uint32_t)(c * 32), v);
      if (write) store_chunk(ep, row, n0 + c * 32, v, red);
    }
    if (write) flush_reduce(ep, tile, warp & 3, red);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1) {
    __syncwarp();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
  }
}

template <bool FUSED>
__global__ void __launch_bounds__(NTHREADS, 1)
gemm_bf16_split_kernel(const __grid_constant__ CUtensorMap mA, const __grid_constant__ CUtensorMap mB,
                       int K, int rowsA, int rowsB, int offA, int offB, const __grid_constant__ PairList pl,
                       const __grid_constant__ Epilogue ep) {
  gemm_tile<FUSED>(&mA, &mB, K, rowsA, rowsB, offA, offB, pl, ep, blockIdx.x);
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ int find_group(const GroupDesc* __restrict__ groups, int ngroups, int tile) {
  int lo = 0, hi = ngroups - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (groups[mid].tile_begin <= tile) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Persistent version of the grouped launch: one CTA per SM walks the tiles
// b, b + gridDim.x, ... of all groups. The accumulator is double-buffered in
// TMEM (2 x 256 columns) so the epilogue of one tile overlaps the main loop
// of the next; the producer's stage ring continues across tiles.
// The K blocks of one output tile: all of them, or the listed ones where B is block-sparse.
struct KBlocks {
  const int* list;  // null: 0 .. count-1
  int count;
  __device__ __forceinline__ int at(int i) const { return list ? list[i] : i; }
};
__device__ __forceinline__ KBlocks tile_kblocks(const GroupDesc* g, int local, int tiles_m) {
  KBlocks kb;
  if (g->kb_off != nullptr) {
    const int nb = local / tiles_m;
    const int o0 = g->kb_off[nb];
    kb.list = g->kb_idx + o0;
    kb.count = g->kb_off[nb + 1] - o0;
  } else {
    kb.list = nullptr;
    kb.count = (g->K + BK - 1) / BK;
  }
  return kb;
}

// With a chunked pair list (emulation levels) every chunk of a tile is one
// accumulator round: the MMA thread fills a TMEM buffer with the chunk's pairs,
// the epilogue adds it to C, and the chunks of a tile stay on one CTA, in order.
template <bool FUSED, int TBN>
__device__ __forceinline__ void persistent_body(const GroupDesc* __restrict__ groups, int ngroups, int total_tiles,
                                                const PairList& pl, int* err, double* partial) {
  // TBN: output tile width (256 or 128); the stage ring keeps the same shared memory
  constexpr int TB_BYTES = TBN * BK * 2;
  constexpr int TSTAGE = A_BYTES + TB_BYTES;
  constexpr int SB = FUSED ? 2 * TSTAGE : TSTAGE;
  constexpr int NS = ring_stages(SB);
  constexpr int ACC_COLS = TBN;
  static_assert(NS >= 2 && NS * SB <= RING_BYTES && 2 * NS + 5 <= 28, "stage ring");
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + NS * SB);
  // bars[0..NS) full, [NS..2NS) empty, [2NS..2NS+2) accumulator full, [2NS+2..2NS+4) accumulator
  // empty, [2NS+4] drain (the MMA thread's last commit on an abort; the test expiry's wait)
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * NS + 5);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nchunk = (FUSED || pl.nchunk <= 0) ? 1 : pl.nchunk;
  auto chunk_begin = [&](int c) { return (c == 0 || pl.nchunk <= 0) ? 0 : (int)pl.chunk_end[c - 1]; };
  auto chunk_end = [&](int c) { return pl.nchunk <= 0 ? pl.n : (int)pl.chunk_end[c]; };
  // Work units: a tile with all its chunks, or (with a partial buffer, for GEMMs of few
  // tiles) a single chunk of a tile, whose FP32 sum goes to its own float64 slice of
  // `partial` for chunk_reduce_kernel to add in chunk order
  const int upt = (partial != nullptr && !FUSED) ? nchunk : 1;  // units per tile
  const int total_units = total_tiles * upt;
  auto unit_tile = [&](int u) { return u / upt; };
  auto unit_c0 = [&](int u) { return upt == 1 ? 0 : u % upt; };
  auto unit_c1 = [&](int u) { return upt == 1 ? nchunk : u % upt + 1; };

  if (threadIdx.x == 0) {
    for (int q = 0; q < NS; ++q) {
      mbar_init(smem_u32(&bars[q]), 1);
      mbar_init(smem_u32(&bars[NS + q]), 1);
    }
    for (int q = 0; q < 2; ++q) {
      mbar_init(smem_u32(&bars[2 * NS + q]), 1);      // committed by the MMA thread
      mbar_init(smem_u32(&bars[2 * NS + 2 + q]), 4);  // one arrival per epilogue warp
    }
    mbar_init(smem_u32(&bars[2 * NS + 4]), 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(2 * ACC_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  if (groups[0].ep.expire) {
    // tests of the timeout status: a bounded wait on a barrier nothing arrives at, before any
    // copy or MMA is issued; the CTA then only frees its tensor memory
    if (threadIdx.x == 0) {
      if (!mbar_wait(smem_u32(&bars[2 * NS + 4]), 0, EXPIRE_NS)) atomicCAS(err, 0, 6);
      *abort_flag = 1;
    }
    __syncthreads();
  }

  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer
    uint32_t it = 0;
    for (int u = blockIdx.x; u < total_units && !*abort_flag; u += gridDim.x) {
      const int tile = unit_tile(u);
      const GroupDesc* g = groups + find_group(groups, ngroups, tile);
      const int* skip = g->ep.skip;
      if (skip != nullptr && (skip[0] | skip[1])) continue;
      const CUtensorMap* mA = reinterpret_cast<const CUtensorMap*>(&g->a);
      const CUtensorMap* mB = reinterpret_cast<const CUtensorMap*>(&g->b);
      const int local = tile - g->tile_begin, tiles_m = (g->ep.M + BM - 1) / BM;
      const int m0 = (local % tiles_m) * BM, n0 = (local / tiles_m) * TBN;
      const KBlocks kbs = tile_kblocks(g, local, tiles_m);
      const int nkb = kbs.count;
      const int p0 = chunk_begin(unit_c0(u));
      const int total = FUSED ? nkb : (chunk_end(unit_c1(u) - 1) - p0) * nkb;
      for (int t = 0; t < total; ++t, ++it) {
        const int q = it % NS;
        const uint32_t r = it / NS;
        if (!mbar_wait(smem_u32(&bars[NS + q]), (r & 1) ^ 1)) {
          *abort_flag = 1;
          atomicCAS(err, 0, 1);
          break;
        }
        const uint32_t full = smem_u32(&bars[q]);
        const uint32_t sa = smem_u32(smem + q * SB);
        mbar_expect_tx(full, SB);
        // B: a K-major box of TBN rows, or (MN-major) TBN / 64 boxes of 64 x 64 placed
        // MN_BOX_BYTES apart
        if (FUSED) {
          const int kb = kbs.at(t);
          tma_load_2d(sa, mA, full, kb * BK, g->offA + m0);
          tma_load_2d(sa + A_BYTES, mA, full, kb * BK, g->rowsA + g->offA + m0);
          if (g->b_mn) {
#pragma unroll
            for (int q = 0; q < TBN / 64; ++q) {
              tma_load_2d(sa + 2 * A_BYTES + q * MN_BOX_BYTES, mB, full, n0 + 64 * q, g->offB + kb * BK);
              tma_load_2d(sa + 2 * A_BYTES + TB_BYTES + q * MN_BOX_BYTES, mB, full, n0 + 64 * q,
                          g->rowsB + g->offB + kb * BK);
            }
          } else {
            tma_load_2d(sa + 2 * A_BYTES, mB, full, kb * BK, g->offB + n0);
            tma_load_2d(sa + 2 * A_BYTES + TB_BYTES, mB, full, kb * BK, g->rowsB + g->offB + n0);
          }
        } else {
          const int p = p0 + t / nkb, kb = kbs.at(t % nkb);
          tma_load_2d(sa, mA, full, kb * BK, (int)pl.a[p] * g->rowsA + g->offA + m0);
          if (g->b_mn) {
#pragma unroll
            for (int q = 0; q < TBN / 64; ++q)
              tma_load_2d(sa + A_BYTES + q * MN_BOX_BYTES, mB, full, n0 + 64 * q,
                          (int)pl.b[p] * g->rowsB + g->offB + kb * BK);
          } else {
            tma_load_2d(sa + A_BYTES, mB, full, kb * BK, (int)pl.b[p] * g->rowsB + g->offB + n0);
          }
        }
      }
    }
    if (*abort_flag) {  // let the copies already issued land before the CTA releases its memory
      for (uint32_t j = it > (uint32_t)NS ? it - NS : 0u; j < it; ++j)
        mbar_wait(smem_u32(&bars[j % NS]), (j / NS) & 1);
    }
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer
    constexpr uint32_t idesc_k = idesc_bf16(BM, TBN);
    uint32_t it = 0, lt = 0;
    for (int u = blockIdx.x; u < total_units && !*abort_flag; u += gridDim.x) {
      const int tile = unit_tile(u);
      const GroupDesc* g = groups + find_group(groups, ngroups, tile);
      const int* skip = g->ep.skip;
      if (skip != nullptr && (skip[0] | skip[1])) continue;
      const int nkb = tile_kblocks(g, tile - g->tile_begin, (g->ep.M + BM - 1) / BM).count;
      const bool bmn = g->b_mn != 0;
      const uint32_t idesc = idesc_k | (bmn ? kIdescBMN : 0u);
      // the B descriptor of k step k (16 contracted indices) of a stage whose B starts at addr
      auto bdesc = [bmn](uint32_t addr, int k) {
        return bmn ? smem_desc_mn(addr + (uint32_t)k * 2048u) : smem_desc(addr + (uint32_t)k * 32u);
      };
      for (int c = unit_c0(u); c < unit_c1(u) && !*abort_flag; ++c) {
        const uint32_t buf = lt & 1, use = lt >> 1;
        if (!mbar_wait(smem_u32(&bars[2 * NS + 2 + buf]), (use & 1) ^ 1)) {
          *abort_flag = 1;
          atomicCAS(err, 0, 4);
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t d = tmem + buf * ACC_COLS;
        const int total = FUSED ? nkb : (chunk_end(c) - chunk_begin(c)) * nkb;
        for (int t = 0; t < total; ++t, ++it) {
          const int q = it % NS;
          const uint32_t r = it / NS;
          if (!mbar_wait(smem_u32(&bars[q]), r & 1)) {
            *abort_flag = 1;
            atomicCAS(err, 0, 2);
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t sa = smem_u32(smem + q * SB);
          if (FUSED) {
            const uint32_t alo = sa + A_BYTES, bhi = sa + 2 * A_BYTES, blo = bhi + TB_BYTES;
#pragma unroll
            for (int k = 0; k < BK / 16; ++k) {
              umma_bf16(d, smem_desc(sa + k * 32), bdesc(bhi, k), idesc, (t > 0 || k > 0) ? 1u : 0u);
              umma_bf16(d, smem_desc(sa + k * 32), bdesc(blo, k), idesc, 1u);
              umma_bf16(d, smem_desc(alo + k * 32), bdesc(bhi, k), idesc, 1u);
            }
          } else {
            const uint32_t sb = sa + A_BYTES;
#pragma unroll
            for (int k = 0; k < BK / 16; ++k)
              umma_bf16(d, smem_desc(sa + k * 32), bdesc(sb, k), idesc, (t > 0 || k > 0) ? 1u : 0u);
          }
          umma_commit(smem_u32(&bars[NS + q]));
        }
        umma_commit(smem_u32(&bars[2 * NS + buf]));  // this chunk's accumulator is complete
        ++lt;
      }
    }
    if (*abort_flag) {  // every MMA issued so far is complete before the tensor memory is freed
      umma_commit(smem_u32(&bars[2 * NS + 4]));
      mbar_wait(smem_u32(&bars[2 * NS + 4]), 0);
    }
  } else if (warp >= 2) {
    // ---------------- epilogue
    const int lane_base = (warp & 3) * 32;
    uint32_t lt = 0;
    bool failed = false;
    for (int u = blockIdx.x; u < total_units && !failed; u += gridDim.x) {
      const int tile = unit_tile(u);
      const GroupDesc* g = groups + find_group(groups, ngroups, tile);
      const int* skip = g->ep.skip;
      if (skip != nullptr && (skip[0] | skip[1])) continue;
      for (int c = unit_c0(u); c < unit_c1(u); ++c) {
        const uint32_t buf = lt & 1, use = lt >> 1;
        const bool ok = !*abort_flag && mbar_wait(smem_u32(&bars[2 * NS + buf]), use & 1);
        if (!ok) {
          atomicCAS(err, 0, 3);
          failed = true;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        Epilogue ep = g->ep;
        if (upt > 1) {  // this chunk's FP32 sum, widened, into its slice of the partial buffer
          ep.C = partial + (long)c * ep.M * ep.N;
          ep.ldc = ep.N;
          ep.split_cols = ep.N;
          ep.split_stride = 0;
          ep.alpha = 1.0;
          ep.beta = 0.0;
          ep.mode = kEpPlain;
          ep.c_f32 = 0;
          ep.bf_hi = nullptr;
        } else if (c > 0) {
          ep.beta = 1.0;
        }
        const int local = tile - g->tile_begin, tiles_m = (ep.M + BM - 1) / BM;
        const int m0 = (local % tiles_m) * BM, n0 = (local / tiles_m) * TBN;
        const int row = m0 + lane_base + lane;
        EpiRed red;
        red.have_dir = ep.mode == kEpReduce && ep.sc != nullptr && ep.sc->have_dir;
#pragma unroll 1
        for (int j = 0; j < TBN / 32; ++j) {
          float v[32];
          tmem_ld32(tmem + buf * ACC_COLS + ((uint32_t)lane_base << 16) + (uint32_t)(j * 32), v);
          store_chunk(ep, row, n0 + j * 32, v, red);
        }
        flush_reduce(ep, local, warp & 3, red);
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&bars[2 * NS + 2 + buf]));
        ++lt;
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1) {
    __syncwarp();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * ACC_COLS) : "memory");
  }
}

// ---------------------------------------------------------------- CTA pairs (cta_group::2)
// The fused split product on a pair of SMs: a cluster of two CTAs computes one 256 x TBN output
// tile with tcgen05.mma.cta_group::2 (M = 256), issued by the even CTA. Each CTA stages its own
// 128 rows of A_hi and A_lo and its half of B_hi and B_lo (TBN / 2 rows, or TBN / 2 output columns
// of an MN-major B), so that an SM fetches half the B bytes per output element of a single-CTA
// tile of the same width; the tensor memory of each CTA holds the accumulator of its 128 rows
// (all TBN columns), which its own epilogue warps read.
// Barriers: full[q] of the even CTA receives the TMA bytes of both CTAs and is armed by the even
// CTA's producer with the pair's total; the even CTA's MMA commits arrive at empty[q] and at the
// accumulator-full barriers of both CTAs (multicast); the accumulator-empty barriers of the even
// CTA count the arrivals of the eight epilogue warps of the pair.
__device__ __forceinline__ uint32_t cluster_ctarank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
// the shared::cluster address of the same shared variable in CTA `rank` of the cluster
__device__ __forceinline__ uint32_t mapa_shared(uint32_t addr, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
  return r;
}
// (not .aligned: the role branches may leave a warp's lanes diverged here)
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release;\n\tbarrier.cluster.wait.acquire;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_cluster(uint32_t cluster_addr) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_addr) : "memory");
}
// a TMA load into this CTA's shared memory whose bytes count at an mbarrier of either CTA of the pair
__device__ __forceinline__ void tma_load_2d_pair(uint32_t dst, const CUtensorMap* map, uint32_t bar_cluster, int c0,
                                                 int c1) {
  asm volatile(
      "cp.async.bulk.tensor.2d.cta_group::2.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4}], [%2];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(bar_cluster), "r"(c0), "r"(c1)
      : "memory");
}
__device__ __forceinline__ void umma_bf16_pair(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
// the same load delivered to every CTA of ctaMask (the same shared offset in each); the bytes count
// at the barrier at bar's offset in the even CTA of each destination's pair
__device__ __forceinline__ void tma_load_2d_pair_mc(uint32_t dst, const CUtensorMap* map, uint32_t bar_cluster,
                                                    int c0, int c1, uint16_t mask) {
  asm volatile(
      "cp.async.bulk.tensor.2d.cta_group::2.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      ".multicast::cluster [%0], [%1, {%3, %4}], [%2], %5;" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(bar_cluster), "r"(c0), "r"(c1), "h"(mask)
      : "memory");
}
// arrive at the barrier at this shared offset in every CTA of mask once the MMAs issued so far
// are complete
__device__ __forceinline__ void umma_commit_pair(uint32_t bar, uint16_t mask) {
  asm volatile(
      "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(bar),
      "h"(mask)
      : "memory");
}
// the same, at this CTA's barrier only
__device__ __forceinline__ void umma_commit_pair_local(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

constexpr uint32_t PAIR_TMEM_COLS = 512;  // two accumulator buffers, 256 columns apart
constexpr uint64_t PAIR_ABORT_SETTLE_NS = 200000ull;

// SPLIT: the 3-term split form (stages hold A_hi, A_lo, B_hi, B_lo); otherwise the pair list pl
// (stages hold one slice of A and one of B), chunk by chunk: every chunk of a tile is one
// accumulator round whose FP32 sum the epilogue adds to C in chunk order (the first with the
// Epilogue's beta, the later ones with beta = 1), as in the single-SM kernel.
// NP = 2: a cluster of two pairs side by side along N (a work unit is 256 x 2 TBN) that share A:
// CTA r of pair p loads rows [64 p, 64 p + 64) of the 128 A rows its CTA position needs and
// multicasts them to CTA r of both pairs, so every A byte leaves L2 once per two column tiles.
// A stage of a CTA is then written by both pairs, so it is free only when both pairs' MMAs have
// read it: the empty barriers count the commits of both pair leaders. Dense B only (both pairs
// walk the same K blocks).
template <int TBN, bool SPLIT, int NP>
__device__ __forceinline__ void pair_body(const GroupDesc* __restrict__ groups, int ngroups, int total_units,
                                          const PairList& pl, int* err) {
  constexpr int TBH = TBN / 2;  // B rows (or MN-major output columns) staged by each CTA
  constexpr int BH_BYTES = TBH * BK * 2;
  constexpr int NSL = SPLIT ? 2 : 1;                  // slices of each operand in a stage
  constexpr int SB = NSL * (A_BYTES + BH_BYTES);      // one CTA's stage
  constexpr int B_OFF = NSL * A_BYTES;                // B_hi (B_0) inside a stage
  constexpr int NS = ring_stages(SB);
  constexpr uint32_t ACC_STRIDE = 256;
  static_assert(TBN % 32 == 0 && TBN >= 64 && TBN <= 256 && NS >= 2 && NS * SB <= RING_BYTES && 2 * NS + 5 <= 28,
                "pair tile");
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + NS * SB);
  // bars[0..NS) full (even CTA), [NS..2NS) empty, [2NS..2NS+2) accumulator full, [2NS+2..2NS+4)
  // accumulator empty (even CTA), [2NS+4] drain / test expiry
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * NS + 5);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  static_assert(NP == 1 || NP == 2, "pairs per cluster");
  const uint32_t rank = cluster_ctarank();
  const int pp = (int)(rank >> 1), rr = (int)(rank & 1);  // pair within the cluster, CTA within the pair
  const uint32_t lead_rank = rank & ~1u;
  const bool leader = rr == 0;
  const int cluster = (int)(blockIdx.x / (2 * NP)), nclusters = (int)(gridDim.x / (2 * NP));
  const uint16_t mask_all = (uint16_t)((1u << (2 * NP)) - 1u);      // every CTA of the cluster
  const uint16_t mask_pair = (uint16_t)(3u << (2 * pp));            // the CTAs of this pair
  const uint16_t mask_a = (uint16_t)((1u << rr) | (1u << (2 + rr)));  // CTA rr of both pairs (NP = 2)
  const int nchunk = (SPLIT || pl.nchunk <= 0) ? 1 : pl.nchunk;
  auto chunk_begin = [&](int c) { return (c == 0 || pl.nchunk <= 0) ? 0 : (int)pl.chunk_end[c - 1]; };
  auto chunk_end = [&](int c) { return pl.nchunk <= 0 ? pl.n : (int)pl.chunk_end[c]; };

  if (threadIdx.x == 0) {
    for (int q = 0; q < NS; ++q) {
      mbar_init(smem_u32(&bars[q]), 1);
      mbar_init(smem_u32(&bars[NS + q]), NP);  // one commit per pair that reads this CTA's stage
    }
    for (int q = 0; q < 2; ++q) {
      mbar_init(smem_u32(&bars[2 * NS + q]), 1);      // the even CTA's multicast commit
      mbar_init(smem_u32(&bars[2 * NS + 2 + q]), 8);  // one arrival per epilogue warp of the pair
    }
    mbar_init(smem_u32(&bars[2 * NS + 4]), 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(PAIR_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  cluster_sync_all();  // the barriers of both CTAs are initialised before any copy, commit or arrival
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  if (groups[0].ep.expire) {
    // tests of the timeout status (as in the single-CTA kernel): nothing is issued
    if (threadIdx.x == 0) {
      if (!mbar_wait(smem_u32(&bars[2 * NS + 4]), 0, EXPIRE_NS)) atomicCAS(err, 0, 6);
      *abort_flag = 1;
    }
    __syncthreads();
  }

  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer (both CTAs)
    uint32_t it = 0;
    for (int u = cluster; u < total_units && !*abort_flag; u += nclusters) {
      const GroupDesc* g = groups + find_group(groups, ngroups, u);
      const int* skip = g->ep.skip;
      if (skip != nullptr && (skip[0] | skip[1])) continue;
      const CUtensorMap* mA = reinterpret_cast<const CUtensorMap*>(&g->a);
      const CUtensorMap* mB = reinterpret_cast<const CUtensorMap*>(&g->b);
      const int local = u - g->tile_begin, tiles_m = (g->ep.M + 2 * BM - 1) / (2 * BM);
      const int m0 = (local % tiles_m) * 2 * BM + rr * BM;                  // this CTA's rows of A
      const int n0 = ((local / tiles_m) * NP + pp) * TBN + rr * TBH;        // this CTA's half of B
      const KBlocks kbs = tile_kblocks(g, local, tiles_m);
      const int nkb = kbs.count;
      const int total = SPLIT ? nkb : pl.n * nkb;  // every pair of every chunk of the tile
      for (int t = 0; t < total; ++t, ++it) {
        const int q = it % NS;
        const uint32_t r = it / NS;
        if (!mbar_wait(smem_u32(&bars[NS + q]), (r & 1) ^ 1)) {
          *abort_flag = 1;
          atomicCAS(err, 0, 1);
          break;
        }
        const uint32_t full = mapa_shared(smem_u32(&bars[q]), lead_rank);
        if (leader) mbar_expect_tx(smem_u32(&bars[q]), 2 * SB);  // the bytes landing in both CTAs
        const uint32_t sa = smem_u32(smem + q * SB);
        const int p = SPLIT ? 0 : t / nkb, kb = kbs.at(SPLIT ? t : t % nkb);
        const int ra = SPLIT ? 0 : (int)pl.a[p] * g->rowsA, rb = SPLIT ? 0 : (int)pl.b[p] * g->rowsB;
        if (NP == 1) {
          tma_load_2d_pair(sa, mA, full, kb * BK, ra + g->offA + m0);
          if (SPLIT) tma_load_2d_pair(sa + A_BYTES, mA, full, kb * BK, g->rowsA + g->offA + m0);
        } else {  // this pair's 64-row half of the A tile, to CTA rr of both pairs (64-row boxes)
          const uint32_t ah = (uint32_t)pp * (A_BYTES / 2);
          tma_load_2d_pair_mc(sa + ah, mA, full, kb * BK, ra + g->offA + m0 + 64 * pp, mask_a);
          if (SPLIT)
            tma_load_2d_pair_mc(sa + A_BYTES + ah, mA, full, kb * BK, g->rowsA + g->offA + m0 + 64 * pp, mask_a);
        }
        if (g->b_mn) {
#pragma unroll
          for (int h = 0; h < TBH / 64; ++h) {
            tma_load_2d_pair(sa + B_OFF + h * MN_BOX_BYTES, mB, full, n0 + 64 * h, rb + g->offB + kb * BK);
            if (SPLIT)
              tma_load_2d_pair(sa + B_OFF + BH_BYTES + h * MN_BOX_BYTES, mB, full, n0 + 64 * h,
                               g->rowsB + g->offB + kb * BK);
          }
        } else {
          tma_load_2d_pair(sa + B_OFF, mB, full, kb * BK, rb + g->offB + n0);
          if (SPLIT) tma_load_2d_pair(sa + B_OFF + BH_BYTES, mB, full, kb * BK, g->rowsB + g->offB + n0);
        }
      }
    }
    if (*abort_flag) {
      if (leader) {  // the copies of the stages issued last (both CTAs' bytes count here)
        for (uint32_t j = it > (uint32_t)NS ? it - NS : 0u; j < it; ++j)
          mbar_wait(smem_u32(&bars[j % NS]), (j / NS) & 1);
      }
      if (!leader || NP > 1) {  // copies that complete at another CTA's barrier: give them time to land
        const uint64_t t0 = globaltimer();
        while (globaltimer() - t0 < PAIR_ABORT_SETTLE_NS) {
        }
      }
    }
  } else if (warp == 1 && lane == 0 && leader) {
    // ---------------- MMA issuer (even CTA)
    constexpr uint32_t idesc_k = idesc_bf16(2 * BM, TBN);
    uint32_t it = 0, lt = 0;
    for (int u = cluster; u < total_units && !*abort_flag; u += nclusters) {
      const GroupDesc* g = groups + find_group(groups, ngroups, u);
      const int* skip = g->ep.skip;
      if (skip != nullptr && (skip[0] | skip[1])) continue;
      const int nkb = tile_kblocks(g, u - g->tile_begin, (g->ep.M + 2 * BM - 1) / (2 * BM)).count;  // NP > 1: dense
      const bool bmn = g->b_mn != 0;
      const uint32_t idesc = idesc_k | (bmn ? kIdescBMN : 0u);
      auto bdesc = [bmn](uint32_t addr, int k) {
        return bmn ? smem_desc_mn(addr + (uint32_t)k * 2048u) : smem_desc(addr + (uint32_t)k * 32u);
      };
      for (int c = 0; c < nchunk && !*abort_flag; ++c) {
        const uint32_t buf = lt & 1, use = lt >> 1;
        if (!mbar_wait(smem_u32(&bars[2 * NS + 2 + buf]), (use & 1) ^ 1)) {
          *abort_flag = 1;
          atomicCAS(err, 0, 4);
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t d = tmem + buf * ACC_STRIDE;
        const int total = SPLIT ? nkb : (chunk_end(c) - chunk_begin(c)) * nkb;
        for (int t = 0; t < total; ++t, ++it) {
          const int q = it % NS;
          const uint32_t r = it / NS;
          if (!mbar_wait(smem_u32(&bars[q]), r & 1)) {
            *abort_flag = 1;
            atomicCAS(err, 0, 2);
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t sa = smem_u32(smem + q * SB);
          const uint32_t alo = sa + A_BYTES, bhi = sa + B_OFF, blo = bhi + BH_BYTES;
#pragma unroll
          for (int k = 0; k < BK / 16; ++k) {
            umma_bf16_pair(d, smem_desc(sa + k * 32), bdesc(bhi, k), idesc, (t > 0 || k > 0) ? 1u : 0u);
            if (SPLIT) {
              umma_bf16_pair(d, smem_desc(sa + k * 32), bdesc(blo, k), idesc, 1u);
              umma_bf16_pair(d, smem_desc(alo + k * 32), bdesc(bhi, k), idesc, 1u);
            }
          }
          umma_commit_pair(smem_u32(&bars[NS + q]), mask_all);  // this pair is done with stage q
        }
        umma_commit_pair(smem_u32(&bars[2 * NS + buf]), mask_pair);  // both halves of the accumulator are complete
        ++lt;
      }
    }
    if (*abort_flag) {  // every MMA issued so far is complete before the tensor memory is freed
      umma_commit_pair_local(smem_u32(&bars[2 * NS + 4]));
      mbar_wait(smem_u32(&bars[2 * NS + 4]), 0);
    }
  } else if (warp >= 2) {
    // ---------------- epilogue (both CTAs: 128 rows each)
    const int lane_base = (warp & 3) * 32;
    const uint32_t acc_empty0 = mapa_shared(smem_u32(&bars[2 * NS + 2]), lead_rank);
    const uint32_t acc_empty1 = mapa_shared(smem_u32(&bars[2 * NS + 3]), lead_rank);
    uint32_t lt = 0;
    for (int u = cluster; u < total_units; u += nclusters) {
      const GroupDesc* g = groups + find_group(groups, ngroups, u);
      const int* skip = g->ep.skip;
      if (skip != nullptr && (skip[0] | skip[1])) continue;
      bool failed = false;
      for (int c = 0; c < nchunk; ++c) {
        const uint32_t buf = lt & 1, use = lt >> 1;
        const bool ok = !*abort_flag && mbar_wait(smem_u32(&bars[2 * NS + buf]), use & 1);
        if (!ok) {
          atomicCAS(err, 0, 3);
          failed = true;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        Epilogue ep = g->ep;
        if (c > 0) ep.beta = 1.0;
        const int local = u - g->tile_begin, tiles_m = (ep.M + 2 * BM - 1) / (2 * BM);
        const int m0 = (local % tiles_m) * 2 * BM + rr * BM, n0 = ((local / tiles_m) * NP + pp) * TBN;
        const int row = m0 + lane_base + lane;
        EpiRed red;
        red.have_dir = ep.mode == kEpReduce && ep.sc != nullptr && ep.sc->have_dir;
#pragma unroll 1
        for (int j = 0; j < TBN / 32; ++j) {
          float v[32];
          tmem_ld32(tmem + buf * ACC_STRIDE + ((uint32_t)lane_base << 16) + (uint32_t)(j * 32), v);
          store_chunk(ep, row, n0 + j * 32, v, red);
        }
        flush_reduce(ep, (local * NP + pp) * 2 + rr, warp & 3, red);  // slots of 128 x TBN quarters
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive_cluster(buf ? acc_empty1 : acc_empty0);
        ++lt;
      }
      if (failed) break;
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  // neither CTA leaves while the pair's MMAs may read its shared memory or write its tensor
  // memory, or the other CTA may still arrive at its barriers
  cluster_sync_all();
  if (warp == 1) {
    __syncwarp();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(PAIR_TMEM_COLS)
                 : "memory");
  }
}

template <int TBN, bool SPLIT>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(NTHREADS, 1)
gemm_pair_kernel(const GroupDesc* __restrict__ groups, int ngroups, int total_units,
                 const __grid_constant__ PairList pl, int* err) {
  pair_body<TBN, SPLIT, 1>(groups, ngroups, total_units, pl, err);
}

// two SM pairs per cluster, sharing A (NP = 2)
template <int TBN, bool SPLIT>
__global__ void __cluster_dims__(4, 1, 1) __launch_bounds__(NTHREADS, 1)
gemm_quad_kernel(const GroupDesc* __restrict__ groups, int ngroups, int total_units,
                 const __grid_constant__ PairList pl, int* err) {
  pair_body<TBN, SPLIT, 2>(groups, ngroups, total_units, pl, err);
}

// one GEMM, its descriptor (tensor maps included) in the kernel's parameter space
template <int TBN, bool SPLIT>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(NTHREADS, 1)
gemm_pair_one_kernel(const __grid_constant__ GroupDesc g, int total_units, const __grid_constant__ PairList pl,
                     int* err) {
  pair_body<TBN, SPLIT, 1>(&g, 1, total_units, pl, err);
}

template <bool FUSED, int TBN>
__global__ void __launch_bounds__(NTHREADS, 1)
gemm_persistent_kernel(const GroupDesc* __restrict__ groups, int ngroups, int total_tiles,
                       const __grid_constant__ PairList pl, int* err) {
  persistent_body<FUSED, TBN>(groups, ngroups, total_tiles, pl, err, nullptr);
}

// one GEMM, its descriptor (tensor maps included) in the kernel's parameter space
template <bool FUSED>
__global__ void __launch_bounds__(NTHREADS, 1)
gemm_persistent_one_kernel(const __grid_constant__ GroupDesc g, int total_tiles, const __grid_constant__ PairList pl,
                           int* err, double* partial) {
  persistent_body<FUSED, BN>(&g, 1, total_tiles, pl, err, partial);
}

// C = beta C + alpha sum_c partial[c] (chunk order; the same float64 operations, in the same
// order, as the in-kernel chunk epilogues)
__global__ void chunk_reduce_kernel(const double* __restrict__ partial, int nchunk, Epilogue ep) {
  const long count = (long)ep.M * ep.N;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < count; idx += (long)gridDim.x * blockDim.x) {
    const long row = idx / ep.N, col = idx % ep.N;
    const long blk = col / ep.split_cols;
    double* p = ep.C + blk * ep.split_stride + row * ep.ldc + (col - blk * ep.split_cols);
    const double a0 = partial[idx];
    double acc;
    if (ep.beta == 0.0) acc = (ep.alpha == 1.0) ? a0 : ep.alpha * a0;
    else if (ep.beta == 1.0) acc = fma(ep.alpha, a0, *p);
    else acc = fma(ep.beta, *p, ep.alpha * a0);
    for (int c = 1; c < nchunk; ++c) acc = fma(ep.alpha, partial[(long)c * count + idx], acc);
    *p = acc;
  }
}

int sm_count() {
  static const int n = [] {
    int dev = 0, c = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&c, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) c = 148;
    return c;
  }();
  return n;
}

// clusters of `size` GEMM CTAs (one per SM) that the device holds at once
template <typename Kernel>
int max_clusters(Kernel kernel, int size) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(size * sm_count()));
  cfg.blockDim = dim3(NTHREADS);
  cfg.dynamicSmemBytes = SMEM_BYTES;
  cudaLaunchAttribute attr;
  attr.id = cudaLaunchAttributeClusterDimension;
  attr.val.clusterDim.x = (unsigned)size;
  attr.val.clusterDim.y = 1;
  attr.val.clusterDim.z = 1;
  cfg.attrs = &attr;
  cfg.numAttrs = 1;
  int c = 0;
  if (cudaOccupancyMaxActiveClusters(&c, kernel, &cfg) != cudaSuccess || c <= 0) {
    cudaGetLastError();
    c = sm_count() / size;
  }
  return c;
}
int pair_clusters() {
  static const int n = max_clusters(gemm_pair_kernel<256, true>, 2);
  return n;
}
int quad_clusters() {
  static const int n = max_clusters(gemm_quad_kernel<256, true>, 4);
  return n;
}

PFN_cuTensorMapEncodeTiled_v12000 lookup_encoder() {
  cudaDriverEntryPointQueryResult q;
  void* fn = nullptr;
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess)
    fn = nullptr;
  return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
}

PFN_cuTensorMapEncodeTiled_v12000 encoder() {
  static const PFN_cuTensorMapEncodeTiled_v12000 fn = lookup_encoder();  // thread-safe one-time lookup
  if (!fn) throw CudaError{cudaErrorNotSupported, "cuTensorMapEncodeTiled"};
  return fn;
}

}  // namespace

// Row-major bf16 matrix rows x cols (leading dimension ld elements, ld*2 a
// multiple of 16 bytes, base 16-byte aligned) as a TMA map with box
// {box_cols, box_rows} and 128-byte swizzle: {BK, rows} for K-major tiles (BK = 64 columns of
// 128 bytes), {64, BK} for MN-major ones.
TensorMap make_map(const __nv_bfloat16* base, long rows, long cols, long ld, int box_rows, int box_cols = BK) {
  TensorMap tm;
  static_assert(sizeof(TensorMap) == sizeof(CUtensorMap), "TensorMap must hold a CUtensorMap");
  if ((reinterpret_cast<uintptr_t>(base) & 15) || ((ld * 2) & 15))
    throw CudaError{cudaErrorInvalidValue, "make_map: operand not 16-byte aligned"};
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(ld * 2)};
  cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  const CUtensorMapSwizzle sw = CU_TENSOR_MAP_SWIZZLE_128B;
  CUresult r = encoder()(reinterpret_cast<CUtensorMap*>(&tm), CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                         const_cast<__nv_bfloat16*>(base), dims, strides, box, estr,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, sw,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) throw CudaError{cudaErrorInvalidValue, "cuTensorMapEncodeTiled"};
  return tm;
}

Operand make_operand_view(const __nv_bfloat16* base, long slice_rows, long cols, long ld, int slices, bool is_a,
                          int row_off, long rows, bool mn_major) {
  if (row_off < 0 || rows <= 0 || row_off + rows > slice_rows || (mn_major && is_a))
    throw CudaError{cudaErrorInvalidValue, "make_operand_view: rows outside the stack"};
  Operand o;
  // the map covers the whole stack, so every slice and row offset stays inside it
  if (mn_major) {
    o.box_rows = BK;  // BK contracted rows x 64 output columns per box
    o.map = make_map(base, slice_rows * slices, cols, ld, BK, 64);
    o.map_n128 = o.map;
  } else {
    o.box_rows = is_a ? BM : BN;
    o.map = make_map(base, slice_rows * slices, cols, ld, o.box_rows);
    o.map_n128 = is_a ? o.map : make_map(base, slice_rows * slices, cols, ld, 128);  // 128-wide output tiles
  }
  o.base = base;
  o.ld = ld;
  o.map_rows = slice_rows * slices;
  o.rows = rows;
  o.cols = cols;
  o.slices = slices;
  o.slice_rows = slice_rows;
  o.row_off = row_off;
  o.mn_major = mn_major;
  return o;
}

Operand make_operand(const __nv_bfloat16* base, long rows, long cols, long ld, int slices, bool is_a) {
  return make_operand_view(base, rows, cols, ld, slices, is_a, 0, rows, false);
}

PairList pairs_split3() {
  PairList p{};
  p.n = 3;
  p.a[0] = 0; p.b[0] = 0;
  p.a[1] = 0; p.b[1] = 1;
  p.a[2] = 1; p.b[2] = 0;
  return p;
}

PairList pairs_single() {
  PairList p{};
  p.n = 1;
  return p;
}

void check_pairs(const PairList& pl, int slices_a, int slices_b) {
  if (pl.n <= 0 || pl.n > kMaxPairs || pl.nchunk < 0 || pl.nchunk > kMaxChunks)
    throw CudaError{cudaErrorInvalidValue, "tc: pair list"};
  for (int p = 0; p < pl.n; ++p)
    if (pl.a[p] >= slices_a || pl.b[p] >= slices_b) throw CudaError{cudaErrorInvalidValue, "tc: slice index"};
  for (int c = 0; c < pl.nchunk; ++c) {
    const int lo = c ? pl.chunk_end[c - 1] : 0;
    if (pl.chunk_end[c] <= lo || pl.chunk_end[c] > pl.n) throw CudaError{cudaErrorInvalidValue, "tc: chunk list"};
  }
  if (pl.nchunk > 0 && pl.chunk_end[pl.nchunk - 1] != pl.n) throw CudaError{cudaErrorInvalidValue, "tc: chunk list"};
}

bool is_single(const PairList& pl) { return pl.n == 1 && pl.nchunk <= 1 && pl.a[0] == 0 && pl.b[0] == 0; }

bool is_split3(const PairList& pl) {
  return pl.n == 3 && pl.nchunk <= 1 && pl.a[0] == 0 && pl.b[0] == 0 && pl.a[1] == 0 && pl.b[1] == 1 && pl.a[2] == 1 && pl.b[2] == 0;
}

void gemm(cudaStream_t st, const Operand& A, const Operand& B, int K, const PairList& pl, const Epilogue& ep) {
  static bool attr_set = false;
  if (!attr_set) {
    OMM_CUDA_TRY(cudaFuncSetAttribute(gemm_bf16_split_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      SMEM_BYTES));
    OMM_CUDA_TRY(cudaFuncSetAttribute(gemm_bf16_split_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      SMEM_BYTES));
    attr_set = true;
  }
  check_pairs(pl, A.slices, B.slices);
  if (pl.nchunk > 1) throw CudaError{cudaErrorInvalidValue, "tc::gemm: chunked pair lists need the persistent launch"};
  if (B.mn_major || A.mn_major || ep.expire)
    throw CudaError{cudaErrorInvalidValue, "tc::gemm: MN-major operands and the test expiry need the persistent launch"};
  dim3 grid((unsigned)(((ep.N + BN - 1) / BN) * ((ep.M + BM - 1) / BM)));
  const CUtensorMap* a = reinterpret_cast<const CUtensorMap*>(&A.map);
  const CUtensorMap* b = reinterpret_cast<const CUtensorMap*>(&B.map);
  const int ra = (int)A.slice_rows, rb = (int)B.slice_rows;
  if (is_split3(pl) && A.slices >= 2 && B.slices >= 2)
    gemm_bf16_split_kernel<true><<<grid, NTHREADS, SMEM_BYTES, st>>>(*a, *b, K, ra, rb, A.row_off, B.row_off, pl, ep);
  else
    gemm_bf16_split_kernel<false><<<grid, NTHREADS, SMEM_BYTES, st>>>(*a, *b, K, ra, rb, A.row_off, B.row_off, pl, ep);
  OMM_LAUNCH_CHECK();
}

int tiles_of(const Epilogue& ep, int bn, bool pair, bool quad) {
  const int bm = (pair || quad) ? 2 * BM : BM;
  const int tn = (ep.N + bn - 1) / bn;
  return ((ep.M + bm - 1) / bm) * (quad ? (tn + 1) / 2 : tn);
}

GroupDesc make_group(const Operand& A, const Operand& B, int K, const Epilogue& ep, int tile_begin, int bn,
                     const BlockLists* sparse, bool pair, bool quad) {
  if (quad) pair = true;
  if (quad && sparse != nullptr)
    throw CudaError{cudaErrorInvalidValue, "tc::make_group: clusters of two pairs need a dense B"};
  if (pair ? (bn != 256 && bn != 192 && bn != 128) : (bn != 256 && bn != 128))
    throw CudaError{cudaErrorInvalidValue, "tc::make_group: tile width"};
  // the TMA boxes must match the tile: A in 128-row boxes, B in boxes of the tile width (of half of
  // it on an SM pair), or, MN-major, in 64 x 64 boxes (then the width an SM stages is a multiple of 64)
  if (A.mn_major || A.box_rows != BM || (!B.mn_major && !pair && bn == 256 && B.box_rows != 256) ||
      (B.mn_major && pair && (bn / 2) % 64 != 0))
    throw CudaError{cudaErrorInvalidValue, "tc::make_group: operand boxes do not match the tile"};
  if (B.mn_major && (sparse != nullptr || K > B.rows))
    throw CudaError{cudaErrorInvalidValue, "tc::make_group: MN-major B: no block lists, K <= its rows"};
  GroupDesc g{};
  g.a = quad ? make_map(A.base, A.map_rows, A.cols, A.ld, BM / 2) : A.map;  // quad: 64-row halves
  g.quad = quad ? 1 : 0;
  if (B.mn_major)
    g.b = B.map;
  else if (pair)
    g.b = bn == 256 ? B.map_n128 : make_map(B.base, B.map_rows, B.cols, B.ld, bn / 2);
  else
    g.b = bn == 128 ? B.map_n128 : B.map;
  g.pair = pair ? 1 : 0;
  g.ep = ep;
  g.K = K;
  g.rowsA = (int)A.slice_rows;
  g.rowsB = (int)B.slice_rows;
  g.offA = A.row_off;
  g.offB = B.row_off;
  g.b_mn = B.mn_major ? 1 : 0;
  g.tile_begin = tile_begin;
  g.bn = bn;
  g.kb_off = sparse ? sparse->off : nullptr;
  g.kb_idx = sparse ? sparse->idx : nullptr;
  if (sparse && sparse->nblocks != (ep.N + bn - 1) / bn)
    throw CudaError{cudaErrorInvalidValue, "tc::make_group: block lists do not match the tiles"};
  return g;
}

void prepare_persistent() {
  static bool attr_set = false;
  if (!attr_set) {
    OMM_CUDA_TRY(cudaFuncSetAttribute(gemm_persistent_kernel<false, 256>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES));
    OMM_CUDA_TRY(cudaFuncSetAttribute(gemm_persistent_kernel<true, 256>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES));
    OMM_CUDA_TRY(cudaFuncSetAttribute(gemm_persistent_kernel<false, 128>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES));
    OMM_CUDA_TRY(cudaFuncSetAttribute(gemm_persistent_kernel<true, 128>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES));
    OMM_CUDA_TRY(cudaFuncSetAttribute(gemm_persistent_one_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      SMEM_BYTES));
    OMM_CUDA_TRY(cudaFuncSetAttribute(gemm_persistent_one_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      SMEM_BYTES));
    for (const void* f : {(const void*)gemm_pair_kernel<128, true>, (const void*)gemm_pair_kernel<192, true>,
                          (const void*)gemm_pair_kernel<256, true>, (const void*)gemm_pair_kernel<128, false>,
                          (const void*)gemm_pair_kernel<192, false>, (const void*)gemm_pair_kernel<256, false>,
                          (const void*)gemm_pair_one_kernel<256, true>, (const void*)gemm_pair_one_kernel<256, false>,
                          (const void*)gemm_quad_kernel<128, true>, (const void*)gemm_quad_kernel<192, true>,
                          (const void*)gemm_quad_kernel<256, true>, (const void*)gemm_quad_kernel<128, false>,
                          (const void*)gemm_quad_kernel<192, false>, (const void*)gemm_quad_kernel<256, false>})
      OMM_CUDA_TRY(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES));
    sm_count();
    pair_clusters();
    quad_clusters();
    attr_set = true;
  }
}

void gemm_persistent(cudaStream_t st, const GroupDesc* groups_dev, int ngroups, int total_tiles, const PairList& pl,
                     int* err, int bn, bool pair, bool quad) {
  prepare_persistent();
  check_pairs(pl, kMaxPairs, kMaxPairs);  // slice counts are checked where the groups are made
  if (ngroups <= 0 || total_tiles <= 0) return;
  const bool fused = is_split3(pl);
  if (quad) {
    if (bn != 256 && bn != 192 && bn != 128)
      throw CudaError{cudaErrorInvalidValue, "tc::gemm_persistent: SM-pair tiles are 128, 192 or 256 wide"};
    const unsigned grid = 4u * (unsigned)std::min(total_tiles, quad_clusters());
    auto go = [&](auto kernel) {
      kernel<<<grid, NTHREADS, SMEM_BYTES, st>>>(groups_dev, ngroups, total_tiles, pl, err);
    };
    if (bn == 256) fused ? go(gemm_quad_kernel<256, true>) : go(gemm_quad_kernel<256, false>);
    else if (bn == 192) fused ? go(gemm_quad_kernel<192, true>) : go(gemm_quad_kernel<192, false>);
    else fused ? go(gemm_quad_kernel<128, true>) : go(gemm_quad_kernel<128, false>);
    OMM_LAUNCH_CHECK();
    return;
  }
  if (pair) {
    if (bn != 256 && bn != 192 && bn != 128)
      throw CudaError{cudaErrorInvalidValue, "tc::gemm_persistent: SM-pair tiles are 128, 192 or 256 wide"};
    const unsigned grid = 2u * (unsigned)std::min(total_tiles, pair_clusters());
    auto go = [&](auto kernel) {
      kernel<<<grid, NTHREADS, SMEM_BYTES, st>>>(groups_dev, ngroups, total_tiles, pl, err);
    };
    if (bn == 256) fused ? go(gemm_pair_kernel<256, true>) : go(gemm_pair_kernel<256, false>);
    else if (bn == 192) fused ? go(gemm_pair_kernel<192, true>) : go(gemm_pair_kernel<192, false>);
    else fused ? go(gemm_pair_kernel<128, true>) : go(gemm_pair_kernel<128, false>);
    OMM_LAUNCH_CHECK();
    return;
  }
  if (bn != 256 && bn != 128) throw CudaError{cudaErrorInvalidValue, "tc::gemm_persistent: tile width"};
  const unsigned grid = (unsigned)std::min(total_tiles, sm_count());
  if (bn == 256 && fused)
    gemm_persistent_kernel<true, 256><<<grid, NTHREADS, SMEM_BYTES, st>>>(groups_dev, ngroups, total_tiles, pl, err);
  else if (bn == 256)
    gemm_persistent_kernel<false, 256><<<grid, NTHREADS, SMEM_BYTES, st>>>(groups_dev, ngroups, total_tiles, pl, err);
  else if (fused)
    gemm_persistent_kernel<true, 128><<<grid, NTHREADS, SMEM_BYTES, st>>>(groups_dev, ngroups, total_tiles, pl, err);
  else
    gemm_persistent_kernel<false, 128><<<grid, NTHREADS, SMEM_BYTES, st>>>(groups_dev, ngroups, total_tiles, pl, err);
  OMM_LAUNCH_CHECK();
}

void gemm_persistent(cudaStream_t st, const Operand& A, const Operand& B, int K, const PairList& pl,
                     const Epilogue& ep, double* partial, long partial_capacity, const BlockLists* sparse) {
  prepare_persistent();
  check_pairs(pl, A.slices, B.slices);
  const int tiles = tiles_of(ep);
  if (tiles <= 0 || K <= 0) return;
  const GroupDesc g = make_group(A, B, K, ep, 0, BN, sparse);
  const bool fused = is_split3(pl) && pl.nchunk <= 1 && A.slices >= 2 && B.slices >= 2;
  // a GEMM of few tiles spreads its chunks over the SMs when scratch for them was given
  const int nchunk = pl.nchunk > 0 ? pl.nchunk : 1;
  const bool split = !fused && partial != nullptr && nchunk > 1 && 2 * tiles < sm_count() &&
                     (long)nchunk * ep.M * ep.N <= partial_capacity && ep.skip == nullptr;
  // a product with at least a wave of 256-row tiles runs on SM pairs (half the B bytes per SM)
  const int pair_units = tiles_of(ep, BN, true);
  if (!split && ep.M >= 2 * BM && pair_units >= pair_clusters()) {
    const GroupDesc gp = make_group(A, B, K, ep, 0, BN, sparse, true);
    const unsigned pgrid = 2u * (unsigned)std::min(pair_units, pair_clusters());
    if (fused)
      gemm_pair_one_kernel<BN, true><<<pgrid, NTHREADS, SMEM_BYTES, st>>>(gp, pair_units, pl, ep.err);
    else
      gemm_pair_one_kernel<BN, false><<<pgrid, NTHREADS, SMEM_BYTES, st>>>(gp, pair_units, pl, ep.err);
    OMM_LAUNCH_CHECK();
    return;
  }
  const int units = split ? tiles * nchunk : tiles;
  const unsigned grid = (unsigned)std::min(units, sm_count());
  if (fused)
    gemm_persistent_one_kernel<true><<<grid, NTHREADS, SMEM_BYTES, st>>>(g, tiles, pl, ep.err, nullptr);
  else
    gemm_persistent_one_kernel<false><<<grid, NTHREADS, SMEM_BYTES, st>>>(g, tiles, pl, ep.err,
                                                                          split ? partial : nullptr);
  OMM_LAUNCH_CHECK();
  if (split) {
    const long count = (long)ep.M * ep.N;
    const unsigned rb = (unsigned)std::min<long>((count + 255) / 256, 4L * sm_count());
    chunk_reduce_kernel<<<rb, 256, 0, st>>>(partial, nchunk, ep);
    OMM_LAUNCH_CHECK();
  }
}


// ------------------------------------------------------------------ block sparsity of B
namespace {
// occ[rb * nkb + kb] = 1 if rows [64 rb, 64 rb + 64) x columns [BK kb, BK kb + BK) hold a nonzero
constexpr int OCC_ROWS = 64;
__global__ void __launch_bounds__(256)
occupancy_kernel(const double* __restrict__ B, long rows, long cols, long ld, int nkb, unsigned char* occ) {
  const long blk = blockIdx.x;
  const long rb = blk / nkb, kb = blk % nkb;
  int any = 0;
  for (int e = threadIdx.x; e < OCC_ROWS * BK; e += blockDim.x) {
    const long r = rb * OCC_ROWS + e / BK, c = kb * BK + e % BK;
    if (r < rows && c < cols && B[r * ld + c] != 0.0) any = 1;
  }
  any = __syncthreads_or(any);
  if (threadIdx.x == 0) occ[blk] = (unsigned char)any;
}
}  // namespace

void block_lists(cudaStream_t st, const double* B, long rows, long cols, long ld, int bn, BlockLists& bl) {
  if (bn != 128 && bn != 192 && bn != 256) throw CudaError{cudaErrorInvalidValue, "tc::block_lists: tile width"};
  const int nkb = (int)((cols + BK - 1) / BK);
  const long nrb64 = (rows + OCC_ROWS - 1) / OCC_ROWS;
  unsigned char* occ = nullptr;
  std::vector<unsigned char> h(nrb64 * nkb);
  OMM_CUDA_TRY(cudaMallocAsync((void**)&occ, h.size(), st));
  try {
    occupancy_kernel<<<(unsigned)(nrb64 * nkb), 256, 0, st>>>(B, rows, cols, ld, nkb, occ);
    OMM_LAUNCH_CHECK();
    OMM_CUDA_TRY(cudaMemcpyAsync(h.data(), occ, h.size(), cudaMemcpyDeviceToHost, st));
    OMM_CUDA_TRY(cudaStreamSynchronize(st));
  } catch (...) {
    cudaFreeAsync(occ, st);
    throw;
  }
  cudaFreeAsync(occ, st);
  const int per = bn / OCC_ROWS;  // 64-row blocks per row block of bn
  const int nblocks = (int)((rows + bn - 1) / bn);
  std::vector<int> off(nblocks + 1, 0), idx;
  for (int r = 0; r < nblocks; ++r) {
    const size_t before = idx.size();
    for (int kb = 0; kb < nkb; ++kb) {
      bool any = false;
      for (int q = 0; q < per; ++q) {
        const long r64 = (long)r * per + q;
        if (r64 < nrb64 && h[r64 * nkb + kb]) any = true;
      }
      if (any) idx.push_back(kb);
    }
    if (idx.size() == before) idx.push_back(0);  // an all-zero block row still writes its zeros
    off[r + 1] = (int)idx.size();
  }
  if (bl.off != nullptr && (bl.nblocks != nblocks || bl.dense != (long)nblocks * nkb))
    throw CudaError{cudaErrorInvalidValue, "tc::block_lists: shape changed"};
  if (bl.off == nullptr) {  // capacity for a dense pattern: later updates rewrite in place
    bl.nblocks = nblocks;
    bl.dense = (long)nblocks * nkb;
    try {
      mem::alloc(&bl.off, off.size(), st);
      mem::alloc(&bl.idx, (size_t)bl.dense, st);
    } catch (...) {
      free_block_lists(bl, st);
      throw;
    }
  }
  bl.nnz = (long)idx.size();
  // the stream was synchronised above, so no earlier launch still reads the old lists; the host
  // vectors live until the copies are done
  OMM_CUDA_TRY(cudaMemcpyAsync(bl.off, off.data(), off.size() * sizeof(int), cudaMemcpyHostToDevice, st));
  OMM_CUDA_TRY(cudaMemcpyAsync(bl.idx, idx.data(), idx.size() * sizeof(int), cudaMemcpyHostToDevice, st));
  OMM_CUDA_TRY(cudaStreamSynchronize(st));
}

void free_block_lists(BlockLists& bl, cudaStream_t st) {
  mem::release(bl.off, st);
  mem::release(bl.idx, st);
  bl = BlockLists{};
}

// ------------------------------------------------------------------ tile-width autotuner
namespace {
std::mutex& tune_mutex() {
  static std::mutex mu;
  return mu;
}
std::map<std::string, TileShape>& tune_cache() {
  static std::map<std::string, TileShape> cache;
  return cache;
}
}  // namespace

TileShape choose_tile_shape(cudaStream_t st, const std::vector<GemmSpec>& specs, const PairList& pl, double* ms_spent,
                            bool allow_pair) {
  if (ms_spent) *ms_spent = 0.0;
  if (specs.empty()) return TileShape{};
  // candidates: one SM per 128-row tile, and (split form or single pass) SM pairs; 192-wide pair
  // tiles need K-major B (an SM stages 96 rows) and, for a block-sparse B, lists for that width
  std::vector<TileShape> cands = {{256, false}, {128, false}};
  const bool split = is_split3(pl);
  bool pair_ok = allow_pair && (split || is_single(pl)), w192 = true, dense = true;
  for (const GemmSpec& g : specs) {
    // (a GEMM of fewer than 256 rows runs on pairs too, its second CTA's rows past M; the timing
    // decides whether that pays)
    if (split && (g.A->slices < 2 || g.B->slices < 2)) pair_ok = false;
    if (g.B->mn_major || (g.sparse[0] != nullptr && g.sparse[2] == nullptr)) w192 = false;
    if (g.sparse[0] != nullptr) dense = false;
  }
  if (pair_ok) {
    cands.push_back({256, true});
    cands.push_back({128, true});
    if (w192) cands.push_back({192, true});
    if (dense) {  // pairs sharing A walk the same K blocks
      cands.push_back({256, true, true});
      cands.push_back({128, true, true});
      if (w192) cands.push_back({192, true, true});
    }
  }
  std::string key = std::to_string(pl.n) + (is_split3(pl) ? "s" : "g") + (pair_ok ? "p" : "");
  long out_elems = 0;
  for (const GemmSpec& g : specs) {
    key += ":" + std::to_string(g.ep.M) + "x" + std::to_string(g.ep.N) + "x" + std::to_string(g.K);
    if (g.B->mn_major) key += "t";
    if (g.sparse[0]) key += "s" + std::to_string(g.sparse[0]->nnz) + "/" + std::to_string(g.sparse[1]->nnz);
    out_elems += (long)g.ep.M * g.ep.N;
  }
  {
    std::lock_guard<std::mutex> lock(tune_mutex());
    auto it = tune_cache().find(key);
    if (it != tune_cache().end()) return it->second;
  }
  // time every candidate on the real operands; outputs go to scratch (beta = 0, no skip flags)
  double* scratch = nullptr;
  int* err = nullptr;
  GroupDesc* dev = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  TileShape best{};
  float best_ms = 0.f;
  auto release = [&]() {
    if (scratch) cudaFree(scratch);
    if (err) cudaFree(err);
    if (dev) cudaFree(dev);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
  };
  try {
    OMM_CUDA_TRY(cudaMalloc((void**)&scratch, out_elems * sizeof(double)));
    OMM_CUDA_TRY(cudaMalloc((void**)&err, sizeof(int)));
    OMM_CUDA_TRY(cudaMalloc((void**)&dev, specs.size() * sizeof(GroupDesc)));
    OMM_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int), st));
    OMM_CUDA_TRY(cudaEventCreate(&e0));
    OMM_CUDA_TRY(cudaEventCreate(&e1));
    float total_ms = 0.f;
    bool first = true;
    for (const TileShape& ts : cands) {
      std::vector<GroupDesc> h;
      long off = 0;
      int tiles = 0;
      for (const GemmSpec& g : specs) {
        Epilogue ep{scratch + off, g.ep.N, g.ep.N, 0, 1.0, 0.0, g.ep.M, g.ep.N, nullptr, err};
        h.push_back(make_group(*g.A, *g.B, g.K, ep, tiles, ts.bn, ts.quad ? nullptr : g.sparse[sparse_slot(ts.bn)],
                               ts.pair, ts.quad));
        tiles += tiles_of(ep, ts.bn, ts.pair, ts.quad);
        off += (long)g.ep.M * g.ep.N;
      }
      OMM_CUDA_TRY(cudaMemcpyAsync(dev, h.data(), h.size() * sizeof(GroupDesc), cudaMemcpyHostToDevice, st));
      gemm_persistent(st, dev, (int)h.size(), tiles, pl, err, ts.bn, ts.pair, ts.quad);  // warm-up
      constexpr int kReps = 3;
      OMM_CUDA_TRY(cudaEventRecord(e0, st));
      for (int r = 0; r < kReps; ++r) gemm_persistent(st, dev, (int)h.size(), tiles, pl, err, ts.bn, ts.pair, ts.quad);
      OMM_CUDA_TRY(cudaEventRecord(e1, st));
      OMM_CUDA_TRY(cudaEventSynchronize(e1));  // h stays alive until the copy has been consumed
      float ms = 0.f;
      OMM_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
      total_ms += ms * (kReps + 1) / kReps;
      if (first || ms < best_ms) {
        best = ts;
        best_ms = ms;
      }
      first = false;
    }
    int h_err = 0;
    OMM_CUDA_TRY(cudaMemcpy(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost));
    if (h_err != 0) best = TileShape{};  // a bounded wait expired: keep the default, the real launch reports it
    if (ms_spent) *ms_spent = total_ms;
  } catch (...) {
    release();
    throw;
  }
  release();
  std::lock_guard<std::mutex> lock(tune_mutex());
  tune_cache()[key] = best;
  return best;
}


}  // namespace tc
}  // namespace omm
