// Tensor-core variants of the fused CG-D and CG-P kernels.
//
// Every dense contraction of the method runs on the tensor cores as
// mma.sync.m16n8k16 with FP16 or BF16 operands and FP32 accumulation:
//   * G = H^H H and the matched filters H^H Y (Algorithm 1 line 5),
//   * e = A p for all right-hand sides of an instance at once (line 9),
//   * q = H v for all right-hand sides (line 20, precoding).
// A complex product is split into real and imaginary accumulators with the
// contraction index k = (antenna or user, re/im): an m16n8k16 A-fragment
// register then holds exactly one complex64 element packed as (re, im), so
// fragments load straight from the interleaved layout of H, Y and A. With
// X3 each operand is split as hi + lo and the product is formed as
// hi*hi + hi*lo + lo*hi (FP32-level accuracy); otherwise hi*hi only. The
// CG product e = A p always uses the split form, so CG runs at FP32 accuracy
// in every precision mode. Vector updates, inner products (compensated),
// trackers and LLRs are FP32 as in the plain kernels.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "cg_kernels.cuh"
#include "cgmimo.h"

namespace cgm {

enum : int { EL_BF16 = 0, EL_F16 = 1 };

// ---------------------------------------------------------------------------
// Packed 2 x 16-bit helpers: low half = real part, high half = imaginary part
// ---------------------------------------------------------------------------

template <int EL>
__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
  if constexpr (EL == EL_BF16) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&v);
  } else {
    __half2 v = __floats2half2_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&v);
  }
}

template <int EL>
__device__ __forceinline__ float2 unpack2(uint32_t u) {
  if constexpr (EL == EL_BF16) {
    return make_float2(__uint_as_float(u << 16), __uint_as_float(u & 0xffff0000u));
  } else {
    __half2 h = *reinterpret_cast<__half2*>(&u);
    return __half22float2(h);
  }
}

// x = hi + lo + O(2^-2p |x|): .x = packed hi, .y = packed lo
template <int EL>
__device__ __forceinline__ uint2 split_c(float2 x) {
  const uint32_t h = pack2<EL>(x.x, x.y);
  const float2 hf = unpack2<EL>(h);
  return make_uint2(h, pack2<EL>(x.x - hf.x, x.y - hf.y));
}

// (a, b) -> (b, -a)
__device__ __forceinline__ uint32_t swap_neg(uint32_t v) {
  return __byte_perm(v, 0u, 0x1032) ^ 0x80000000u;
}
// (a, b) -> (a, -b)
__device__ __forceinline__ uint32_t neg_hi(uint32_t v) { return v ^ 0x80000000u; }
// (a, b) -> (b, a)
__device__ __forceinline__ uint32_t swap_halves(uint32_t v) { return __byte_perm(v, 0u, 0x1032); }

template <int EL>
__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0,
                                         uint32_t b1) {
  if constexpr (EL == EL_BF16) {
    asm("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
  } else {
    asm("mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
  }
}

// d += (ah + al)(bh + bl) without the lo*lo term (X3), or d += ah * bh.
template <int EL, bool X3>
__device__ __forceinline__ void mma_split(float (&d)[4], const uint32_t (&ah)[4],
                                          const uint32_t (&al)[4], uint32_t bh0, uint32_t bh1,
                                          uint32_t bl0, uint32_t bl1) {
  if constexpr (X3) {
    mma16816<EL>(d, al, bh0, bh1);
    mma16816<EL>(d, ah, bl0, bl1);
  }
  mma16816<EL>(d, ah, bh0, bh1);
}

// Column swizzle of the converted channel in shared memory: element (b, c)
// of H [B][U] is stored at column c ^ hswz(b, U). It spreads both fragment
// access patterns (rows = antennas t, columns = users g, and the transpose)
// over all banks.
__device__ __forceinline__ int hswz(int b, int U) {
  if ((U & 15) == 0) return ((b & 1) << 3) | ((b & 2) << 1);
  if ((U & 7) == 0) return (b & 2) << 1;
  return 0;
}

// ---------------------------------------------------------------------------
// Shared-memory plans
// ---------------------------------------------------------------------------

template <int UT>
struct TcCfg {
  static constexpr int NTHR = UT == 32 ? 256 : 128;
  static constexpr int NWARP = NTHR / 32;
  static constexpr int WM = (UT + 15) / 16;          // m-tiles of users
  static constexpr int WK = NWARP / WM;              // antenna ranges
  static constexpr int NTD = (UT + RMAX + 7) / 8;    // n-tiles of [H | Y^T]
  static constexpr int NTP = (UT + 7) / 8;           // n-tiles of H
  static constexpr int KSC = (2 * UT + 15) / 16;     // k-steps of A p (K = 2 UT)
  static constexpr int SP = UT + 2;                  // row stride of A-hat and P buffers
};

struct TcPlan {
  uint32_t H, Y, A, Ac, Bm, P, X, Mu, Rho, Gd, AB, Kd, Nrm, Part, misc, total;
  uint32_t big;
  int B8, YS;
};

__host__ __device__ inline int tc_ys(int B8) { return ((B8 - 2 + 15) / 16) * 16 + 2; }

template <int UT>
__host__ __device__ inline TcPlan tc_detect_plan(int B, int U, int R, int exact) {
  using C = TcCfg<UT>;
  TcPlan s{};
  s.B8 = (B + 7) & ~7;
  s.YS = tc_ys(s.B8);
  const uint32_t hb = align16(uint32_t(s.B8) * U * 8u);
  const uint32_t hy = hb + align16(uint32_t(R) * s.YS * 8u);
  const uint32_t part = uint32_t(C::NWARP) * 32u * C::NTD * 8u * 4u;
  const uint32_t lbuf = exact ? 5u * U * U * 8u : 0u;
  uint32_t big = hy > part ? hy : part;
  big = big > lbuf ? big : lbuf;
  s.big = align16(big);
  s.H = 0;
  s.Y = hb;
  s.Part = 0;
  uint32_t off = s.big;
  s.A = off; off += UT * UT * 8;
  s.Ac = off; off += UT * C::SP * 8;
  s.Bm = off; off += RMAX * UT * 8;
  s.P = off; off += RMAX * C::SP * 8;
  s.X = off; off += RMAX * UT * 8;
  s.Mu = off; off += RMAX * UT * 4;
  s.Rho = off; off += RMAX * UT * 4;
  s.Gd = off; off += UT * 4;
  s.AB = off; off += exact ? RMAX * KMAX * 2 * 4 : 0;
  s.Kd = off; off += RMAX * 4;
  s.Nrm = off; off += RMAX * 4;
  s.misc = align16(off);
  s.total = s.misc + 32;  // mbarrier, status word, claimed work index
  return s;
}

template <int UT>
__host__ __device__ inline TcPlan tc_precode_plan(int B, int U, int R) {
  using C = TcCfg<UT>;
  TcPlan s{};
  s.B8 = (B + 7) & ~7;
  s.YS = 0;
  const uint32_t hb = align16(uint32_t(s.B8) * U * 8u);
  s.H = 0;
  s.Y = hb;  // T [R][U], FP32
  s.big = hb + align16(uint32_t(R) * U * 8u);
  uint32_t off = s.big;
  s.Part = off; off += uint32_t(C::NWARP) * 32u * C::NTP * 8u * 4u;
  s.A = off; off += UT * UT * 8;
  s.Ac = off; off += UT * C::SP * 8;
  s.P = off; off += RMAX * C::SP * 8;
  s.Gd = off; off += UT * 4;
  s.Bm = s.X = s.Mu = s.Rho = s.AB = off;
  s.Kd = off; off += RMAX * 4;
  s.Nrm = off; off += RMAX * 4;
  s.misc = align16(off);
  s.total = s.misc + 32;  // mbarrier, status word, claimed work index
  return s;
}

// ---------------------------------------------------------------------------
// Work sources: where a CTA finds its next instance and that instance's
// parameters and buffers
// ---------------------------------------------------------------------------

struct DetItem {
  const float2* H;
  const float2* Y;
  float2* xhat;
  float* mu;
  float* rho;
  float* llr;
  int32_t* status;
  int B, U, R, K, q, exact, bulk;
  float N0, Es, sigma;
};

struct PreItem {
  const float2* H;
  const float2* T;
  float2* q;
  float* qnorm;
  int32_t* status;
  int B, U, R, K, normalize, bulk_h, bulk_t;
  float sigma;
};

__device__ __forceinline__ bool aligned16(const void* p) {
  return (reinterpret_cast<uintptr_t>(p) & 15u) == 0;
}

// Work units (problem, instance) of one bin, claimed from a device counter.
struct BatchArgs {
  const cg_desc* desc;            // device copy of the plan's descriptors
  const int2* work;               // (descriptor index, instance) of each unit in this bin
  int64_t n_work;
  unsigned long long* counter;    // claim counter, zero at launch
  int PB, PR, PEX;                // plan shape of the bin: max B, max R, any exact tracker
};

__device__ __forceinline__ DetItem det_item(const DetectArgs& a, int64_t n) {
  DetItem it;
  it.H = a.H + n * a.B * a.U;
  it.Y = a.Y + n * a.R * a.B;
  const int64_t o = n * a.R * a.U;
  it.xhat = a.xhat ? a.xhat + o : nullptr;
  it.mu = a.mu ? a.mu + o : nullptr;
  it.rho = a.rho ? a.rho + o : nullptr;
  it.llr = a.llr ? a.llr + o * a.q : nullptr;
  it.status = a.status ? a.status + n : nullptr;
  it.B = a.B; it.U = a.U; it.R = a.R; it.K = a.K; it.q = a.q; it.exact = a.exact;
  it.bulk = a.bulk;
  it.N0 = a.N0; it.Es = a.Es; it.sigma = a.sigma;
  return it;
}

__device__ __forceinline__ DetItem det_item(const BatchArgs& b, int64_t w) {
  const int2 wu = b.work[w];
  const cg_desc& d = b.desc[wu.x];
  const int64_t n = wu.y;
  DetItem it;
  it.B = d.B; it.U = d.U; it.R = d.R; it.K = d.K; it.q = d.qam_bits;
  it.exact = d.sinr_mode == 1;
  it.N0 = d.N0; it.Es = d.Es; it.sigma = d.N0 / d.Es;
  it.H = static_cast<const float2*>(d.H) + n * d.B * d.U;
  it.Y = static_cast<const float2*>(d.in) + n * d.R * d.B;
  const int64_t o = n * d.R * d.U;
  it.xhat = d.out ? static_cast<float2*>(d.out) + o : nullptr;
  it.mu = d.mu ? d.mu + o : nullptr;
  it.rho = d.rho ? d.rho + o : nullptr;
  it.llr = d.aux ? d.aux + o * d.qam_bits : nullptr;
  it.status = d.status ? d.status + n : nullptr;
  it.bulk = (d.B % 2 == 0) && aligned16(it.H) && aligned16(it.Y);
  return it;
}

__device__ __forceinline__ PreItem pre_item(const PrecodeArgs& a, int64_t n) {
  PreItem it;
  it.H = a.H + n * a.B * a.U;
  it.T = a.T + n * a.R * a.U;
  it.q = a.q + n * a.R * a.B;
  it.qnorm = a.qnorm ? a.qnorm + n * a.R : nullptr;
  it.status = a.status ? a.status + n : nullptr;
  it.B = a.B; it.U = a.U; it.R = a.R; it.K = a.K; it.normalize = a.normalize;
  it.bulk_h = a.bulk_h; it.bulk_t = a.bulk_t; it.sigma = a.sigma;
  return it;
}

__device__ __forceinline__ PreItem pre_item(const BatchArgs& b, int64_t w) {
  const int2 wu = b.work[w];
  const cg_desc& d = b.desc[wu.x];
  const int64_t n = wu.y;
  PreItem it;
  it.B = d.B; it.U = d.U; it.R = d.R; it.K = d.K; it.normalize = d.normalize;
  it.sigma = d.N0 / d.Es;
  it.H = static_cast<const float2*>(d.H) + n * d.B * d.U;
  it.T = static_cast<const float2*>(d.in) + n * d.R * d.U;
  it.q = static_cast<float2*>(d.out) + n * d.R * d.B;
  it.qnorm = d.aux ? d.aux + n * d.R : nullptr;
  it.status = d.status ? d.status + n : nullptr;
  it.bulk_h = ((d.B * d.U) % 2 == 0) && aligned16(it.H);
  it.bulk_t = ((d.R * d.U) % 2 == 0) && aligned16(it.T);
  return it;
}

// Claims the next work unit of a batch: thread 0 bumps the counter and
// publishes the index in shared memory; readers wait for the next barrier.
__device__ __forceinline__ void claim_next(const BatchArgs& b, int64_t* slot) {
  if (threadIdx.x == 0) {
    const unsigned long long w = atomicAdd(b.counter, 1ull);
    *slot = w < static_cast<unsigned long long>(b.n_work) ? static_cast<int64_t>(w) : -1;
  }
}
__device__ __forceinline__ void claim_try(const BatchArgs& b, int64_t* slot) {
  claim_next(b, slot);
}

// ---------------------------------------------------------------------------
// Conversion of the staged FP32 channel / receive vectors to hi|lo pairs
// ---------------------------------------------------------------------------

// In place: element (b, c) of H becomes the uint2 (hi, lo) at column
// c ^ hswz(b). Rows B..B8-1 become zero. Threads own swizzle orbits
// {c, c ^ m}, so no element is overwritten before it is read.
template <int EL, int NTHR>
__device__ __forceinline__ void convert_h(unsigned char* base, int B, int B8, int U) {
  float2* f = reinterpret_cast<float2*>(base);
  uint2* u = reinterpret_cast<uint2*>(base);
  for (int e = threadIdx.x; e < B8 * U; e += NTHR) {
    const int b = e / U, c = e - (e / U) * U;
    const int m = hswz(b, U);
    const int c2 = c ^ m;
    if (c2 < c) continue;
    if (b >= B) {
      u[b * U + c] = make_uint2(0u, 0u);
      if (c2 != c) u[b * U + c2] = make_uint2(0u, 0u);
      continue;
    }
    const float2 x1 = f[b * U + c];
    const float2 x2 = f[b * U + c2];
    u[b * U + c2] = split_c<EL>(x1);
    if (c2 != c) u[b * U + c] = split_c<EL>(x2);
  }
}

// FULL form of convert_h (U == UT, B % 8 == 0): two adjacent columns per
// 16-byte access; the swizzle is even, so column pairs stay pairs.
template <int EL, int NTHR, int UT>
__device__ __forceinline__ void convert_h_full(unsigned char* base, int B) {
  constexpr int HALF = UT / 2;
  const float4* f = reinterpret_cast<const float4*>(base);
  uint4* u = reinterpret_cast<uint4*>(base);
  for (int e = threadIdx.x; e < B * HALF; e += NTHR) {
    const int b = e / HALF, cp = e % HALF;
    const int cp2 = cp ^ (hswz(b, UT) >> 1);
    if (cp2 < cp) continue;
    const float4 x1 = f[b * HALF + cp];
    const float4 x2 = f[b * HALF + cp2];
    const uint2 s0 = split_c<EL>(make_float2(x1.x, x1.y));
    const uint2 s1 = split_c<EL>(make_float2(x1.z, x1.w));
    u[b * HALF + cp2] = make_uint4(s0.x, s0.y, s1.x, s1.y);
    if (cp2 != cp) {
      const uint2 s2 = split_c<EL>(make_float2(x2.x, x2.y));
      const uint2 s3 = split_c<EL>(make_float2(x2.z, x2.w));
      u[b * HALF + cp] = make_uint4(s2.x, s2.y, s3.x, s3.y);
    }
  }
}

// Rows of Y (stride YS): antennas < B converted in place, B..B8-1 zeroed.
template <int EL, int NTHR>
__device__ __forceinline__ void convert_y(unsigned char* base, int B, int B8, int R, int YS) {
  float2* f = reinterpret_cast<float2*>(base);
  uint2* u = reinterpret_cast<uint2*>(base);
  for (int e = threadIdx.x; e < R * B8; e += NTHR) {
    const int r = e / B8, b = e - (e / B8) * B8;
    const int o = r * YS + b;
    u[o] = (b < B) ? split_c<EL>(f[o]) : make_uint2(0u, 0u);
  }
}

// ---------------------------------------------------------------------------
// Gram (and matched filters) on the tensor cores, partial per warp
// ---------------------------------------------------------------------------

// Warp (wm, wk) accumulates rows wm*16.. of H^H [H | Y^T] over its antenna
// range. Cr/Ci[nt] hold the real/imaginary parts of n-tile nt in the m16n8
// accumulator layout. Columns n < U come from H, U <= n < U + R from Y.
template <int UT, int EL, bool X3, int NT>
__device__ __forceinline__ void tc_gram(const uint2* __restrict__ Hc,
                                        const uint2* __restrict__ Yc, int YS, int B8, int U,
                                        int Nz, int wm, int wk, int WK, float (&Cr)[NT][4],
                                        float (&Ci)[NT][4]) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
#pragma unroll
  for (int nt = 0; nt < NT; ++nt)
#pragma unroll
    for (int k = 0; k < 4; ++k) Cr[nt][k] = Ci[nt][k] = 0.f;
  const int KS = B8 / 8;
  const int ks0 = (wk * KS) / WK, ks1 = ((wk + 1) * KS) / WK;
  const int i0 = wm * 16 + g, i1 = i0 + 8;
  const int nta = (Nz + 7) / 8;
  for (int ks = ks0; ks < ks1; ++ks) {
    const int b0 = ks * 8 + t, b1 = b0 + 4;
    uint32_t ah[4], al[4];
    {
      const uint2 z = make_uint2(0u, 0u);
      const uint2 x0 = i0 < U ? Hc[b0 * U + (i0 ^ hswz(b0, U))] : z;
      const uint2 x1 = i1 < U ? Hc[b0 * U + (i1 ^ hswz(b0, U))] : z;
      const uint2 x2 = i0 < U ? Hc[b1 * U + (i0 ^ hswz(b1, U))] : z;
      const uint2 x3 = i1 < U ? Hc[b1 * U + (i1 ^ hswz(b1, U))] : z;
      ah[0] = x0.x; al[0] = x0.y;
      ah[1] = x1.x; al[1] = x1.y;
      ah[2] = x2.x; al[2] = x2.y;
      ah[3] = x3.x; al[3] = x3.y;
    }
#pragma unroll
    for (int nt = 0; nt < NT; ++nt) {
      if (nt < nta) {
        const int n = nt * 8 + g;
        uint2 z0 = make_uint2(0u, 0u), z1 = z0;
        if (n < U) {
          z0 = Hc[b0 * U + (n ^ hswz(b0, U))];
          z1 = Hc[b1 * U + (n ^ hswz(b1, U))];
        } else if (n < Nz) {
          z0 = Yc[(n - U) * YS + b0];
          z1 = Yc[(n - U) * YS + b1];
        }
        // real part: [Hr Hi] . [Zr Zi]; imaginary part: [Hr Hi] . [Zi -Zr]
        mma_split<EL, X3>(Cr[nt], ah, al, z0.x, z1.x, z0.y, z1.y);
        mma_split<EL, X3>(Ci[nt], ah, al, swap_neg(z0.x), swap_neg(z1.x), swap_neg(z0.y),
                          swap_neg(z1.y));
      }
    }
  }
}

// Same product read straight from the FP32 staging buffers (H [B][U], Y rows
// of stride YS): each element is split into hi|lo in registers when loaded.
// For the H columns the B fragments are the A fragment registers (column
// n = i), so every element is loaded and converted once. FULL: U == UT and
// B % 8 == 0, which removes every bounds predicate.
template <int UT, int EL, bool X3, bool FULL, int NT>
__device__ __forceinline__ void tc_gram_f32(const float2* __restrict__ sH,
                                            const float2* __restrict__ sY, int YS, int B,
                                            int U, int R, int wm, int wk, int WK,
                                            float (&Cr)[NT][4], float (&Ci)[NT][4]) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
#pragma unroll
  for (int nt = 0; nt < NT; ++nt)
#pragma unroll
    for (int k = 0; k < 4; ++k) Cr[nt][k] = Ci[nt][k] = 0.f;
  const int Uc = FULL ? UT : U;
  const int KS = FULL ? B / 8 : (B + 7) / 8;
  const int ks0 = (wk * KS) / WK, ks1 = ((wk + 1) * KS) / WK;
  const int i0 = wm * 16 + g, i1 = i0 + 8;
  const bool r0ok = FULL ? (wm * 16 < UT) : (i0 < U);
  const bool r1ok = FULL ? (wm * 16 + 8 < UT) : (i1 < U);
  const int NTH = UT / 8;  // n-tiles that hold H columns when FULL
  const int nta = (Uc + R + 7) / 8;
  const float2 z2 = make_float2(0.f, 0.f);
  for (int ks = ks0; ks < ks1; ++ks) {
    const int b0 = ks * 8 + t, b1 = b0 + 4;
    const bool v0 = FULL || b0 < B, v1 = FULL || b1 < B;
    const uint2 x0 = split_c<EL>((r0ok && v0) ? sH[b0 * Uc + i0] : z2);
    const uint2 x1 = split_c<EL>((r1ok && v0) ? sH[b0 * Uc + i1] : z2);
    const uint2 x2 = split_c<EL>((r0ok && v1) ? sH[b1 * Uc + i0] : z2);
    const uint2 x3 = split_c<EL>((r1ok && v1) ? sH[b1 * Uc + i1] : z2);
    const uint32_t ah[4] = {x0.x, x1.x, x2.x, x3.x};
    const uint32_t al[4] = {x0.y, x1.y, x2.y, x3.y};
#pragma unroll
    for (int nt = 0; nt < NT; ++nt) {
      if (nt >= nta) continue;
      uint2 z0, z1;
      if (FULL && nt < NTH && nt * 8 == wm * 16) {
        z0 = x0;
        z1 = x2;
      } else if (FULL && nt < NTH && nt * 8 == wm * 16 + 8) {
        z0 = x1;
        z1 = x3;
      } else {
        const int n = nt * 8 + g;
        float2 f0 = z2, f1 = z2;
        if (FULL ? (nt < NTH) : (n < U)) {
          if (v0) f0 = sH[b0 * Uc + n];
          if (v1) f1 = sH[b1 * Uc + n];
        } else if (n - Uc < R) {
          if (v0) f0 = sY[(n - Uc) * YS + b0];
          if (v1) f1 = sY[(n - Uc) * YS + b1];
        }
        z0 = split_c<EL>(f0);
        z1 = split_c<EL>(f1);
      }
      // real part: [Hr Hi] . [Zr Zi]; imaginary part: [Hr Hi] . [Zi -Zr]
      mma_split<EL, X3>(Cr[nt], ah, al, z0.x, z1.x, z0.y, z1.y);
      mma_split<EL, X3>(Ci[nt], ah, al, swap_neg(z0.x), swap_neg(z1.x), swap_neg(z0.y),
                        swap_neg(z1.y));
    }
  }
}

// Warp w sums n-tile w (w + NWARP, ...) over the WK partials of each m-tile,
// in order, and stores it: Gram entries as the upper triangle of A = G +
// sigma I mirrored (exactly Hermitian) with its hi|lo split, diag(G), and
// matched filters. Padded users are zeroed by the caller's layout init.
template <int UT, int EL, int NT>
__device__ __forceinline__ void tc_reduce_warp(const float* __restrict__ part, int WK, int U,
                                               int R, float sigma, float2* sA, uint2* sAc,
                                               float2* sBm, float* sGd) {
  constexpr int WM = TcCfg<UT>::WM, SP = TcCfg<UT>::SP, NWARP = TcCfg<UT>::NWARP;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, g = lane >> 2, t = lane & 3;
  const int nta = (U + R + 7) / 8;
  for (int job = warp; job < WM * nta; job += NWARP) {
    const int wm = job / nta, nt = job - wm * nta;
    float re[4] = {0.f, 0.f, 0.f, 0.f}, im[4] = {0.f, 0.f, 0.f, 0.f};
    for (int wk = 0; wk < WK; ++wk) {
      const int w = wk * WM + wm;
#pragma unroll
      for (int d = 0; d < 4; ++d) {
        re[d] += part[((w * NT + nt) * 8 + d) * 32 + lane];
        im[d] += part[((w * NT + nt) * 8 + 4 + d) * 32 + lane];
      }
    }
#pragma unroll
    for (int d = 0; d < 4; ++d) {
      const int i = wm * 16 + g + ((d & 2) ? 8 : 0);
      const int n = nt * 8 + 2 * t + (d & 1);
      if (i >= U || n >= U + R) continue;
      const float2 s = make_float2(re[d], im[d]);
      if (n < U) {
        if (i < n) {
          const float2 c = make_float2(s.x, -s.y);
          sA[i * UT + n] = s;
          sA[n * UT + i] = c;
          sAc[i * SP + n] = split_c<EL>(s);
          sAc[n * SP + i] = split_c<EL>(c);
        } else if (i == n) {
          const float2 a = make_float2(s.x + sigma, 0.f);
          sA[i * UT + i] = a;
          sAc[i * SP + i] = split_c<EL>(a);
          sGd[i] = s.x;
        }
      } else {
        sBm[(n - U) * UT + i] = s;
      }
    }
  }
}

// Zero entries of padded users (i or j >= U) in A, its split, diag(G) and
// the matched filters; disjoint from what tc_reduce_warp writes.
template <int UT>
__device__ __forceinline__ void tc_zero_padding(int U, int R, float2* sA, uint2* sAc,
                                                float2* sBm, float* sGd, int nthr) {
  constexpr int SP = TcCfg<UT>::SP;
  if (U == UT) return;
  for (int e = threadIdx.x; e < UT * UT; e += nthr) {
    const int i = e / UT, j = e - (e / UT) * UT;
    if (i >= U || j >= U) {
      sA[e] = make_float2(0.f, 0.f);
      sAc[i * SP + j] = make_uint2(0u, 0u);
      if (i == j) sGd[i] = 0.f;
    }
  }
  if (sBm != nullptr)
    for (int e = threadIdx.x; e < R * UT; e += nthr) {
      const int r = e / UT, i = e - (e / UT) * UT;
      if (i >= U) sBm[r * UT + i] = make_float2(0.f, 0.f);
    }
}

// Reduces the warps' partial tiles (same wm, wk = 0..WK-1, in order) and
// writes A = G + sigma I (upper triangle mirrored, exactly Hermitian), its
// hi|lo split for the CG products, diag(G) and the matched filters.
template <int UT, int EL, int NT>
__device__ __forceinline__ void tc_reduce(const float* __restrict__ part, int WK, int U, int R,
                                          int Nz, float sigma, float2* sA, uint2* sAc,
                                          float2* sBm, float* sGd, int nthr) {
  constexpr int WM = TcCfg<UT>::WM, SP = TcCfg<UT>::SP;
  const int nta = (Nz + 7) / 8;
  const int E = WM * nta * 4 * 32;  // (wm, nt, d, lane)
  for (int e = threadIdx.x; e < E; e += nthr) {
    const int lane = e & 31, d = (e >> 5) & 3;
    const int rest = e >> 7;
    const int nt = rest % nta, wm = rest / nta;
    float re = 0.f, im = 0.f;
    for (int wk = 0; wk < WK; ++wk) {
      const int w = wk * WM + wm;
      re += part[((w * NT + nt) * 8 + d) * 32 + lane];
      im += part[((w * NT + nt) * 8 + 4 + d) * 32 + lane];
    }
    const int g = lane >> 2, t = lane & 3;
    const int i = wm * 16 + g + ((d & 2) ? 8 : 0);
    const int n = nt * 8 + 2 * t + (d & 1);
    if (i >= U || n >= Nz) continue;
    const float2 s = make_float2(re, im);
    if (n < U) {
      const int j = n;
      if (i < j) {
        const float2 c = make_float2(s.x, -s.y);
        sA[i * UT + j] = s;
        sA[j * UT + i] = c;
        sAc[i * SP + j] = split_c<EL>(s);
        sAc[j * SP + i] = split_c<EL>(c);
      } else if (i == j) {
        const float2 a = make_float2(s.x + sigma, 0.f);
        sA[i * UT + i] = a;
        sAc[i * SP + i] = split_c<EL>(a);
        sGd[i] = s.x;
      }
    } else {
      sBm[(n - U) * UT + i] = s;
    }
  }
  // padded users: zero rows and columns of A, zero G_ii and matched filters
  for (int e = threadIdx.x; e < UT * UT; e += nthr) {
    const int i = e / UT, j = e - (e / UT) * UT;
    if (i >= U || j >= U) {
      sA[e] = make_float2(0.f, 0.f);
      sAc[i * SP + j] = make_uint2(0u, 0u);
      if (i == j) sGd[i] = 0.f;
    }
  }
  for (int e = threadIdx.x; e < R * UT; e += nthr) {
    const int r = e / UT, i = e - (e / UT) * UT;
    if (i >= U) sBm[r * UT + i] = make_float2(0.f, 0.f);
  }
}

// ---------------------------------------------------------------------------
// Algorithm 1 with e = A p on the tensor cores (one warp per 8 right-hand sides)
// ---------------------------------------------------------------------------

// Warp w owns right-hand sides r = 8w + 2t + rr (rr = 0, 1) and users
// i = 16 mt + g + 8h (h = 0, 1): the positions of the m16n8 accumulator.
// Lanes with the same t hold one right-hand side; inner products reduce over
// the eight lanes g = 0..7 (butterflies on lane bits 2-4). p travels through
// sP (row r, stride SP) into the B-fragment layout before each product. The
// A fragments (hi|lo of A) stay in registers for all iterations; the three
// split products accumulate separately so no mma waits on more than KS others.
template <int UT, int EL>
struct TcCg {
  static constexpr int MT = TcCfg<UT>::WM, KS = TcCfg<UT>::KSC, SP = TcCfg<UT>::SP;
  float2 v[MT][2][2], res[MT][2][2], p[MT][2][2];
  float l1[MT][2][2], l2[MT][2][2], l3[MT][2][2];
  float rrn[2], a1[2], a2[2], be1[2], be2[2];
  bool active[2], broke[2];
  int kd[2];
  uint32_t fah[MT][KS][4], fal[MT][KS][4];  // A fragments, hi and lo

  // Compensated butterfly over the eight lanes that share t, for two
  // independent sums at once (TwoSum error terms carried alongside).
  __device__ __forceinline__ static void reduce8x2(float& x0, float& x1) {
    float s0 = x0, s1 = x1, c0 = 0.f, c1 = 0.f;
#pragma unroll
    for (int off = 4; off < 32; off <<= 1) {
      const float so0 = __shfl_xor_sync(0xffffffffu, s0, off);
      const float so1 = __shfl_xor_sync(0xffffffffu, s1, off);
      const float co0 = __shfl_xor_sync(0xffffffffu, c0, off);
      const float co1 = __shfl_xor_sync(0xffffffffu, c1, off);
      const float t0 = s0 + so0, t1 = s1 + so1;
      const float b0 = t0 - s0, b1 = t1 - s1;
      const float e0 = (s0 - (t0 - b0)) + (so0 - b0);
      const float e1 = (s1 - (t1 - b1)) + (so1 - b1);
      s0 = t0;
      s1 = t1;
      c0 = (c0 + co0) + e0;
      c1 = (c1 + co1) + e1;
    }
    x0 = s0 + c0;
    x1 = s1 + c1;
  }

  __device__ __forceinline__ void load_a(const uint2* __restrict__ sAc) {
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const uint2 z = make_uint2(0u, 0u);
#pragma unroll
    for (int mt = 0; mt < MT; ++mt) {
      const int i0 = mt * 16 + g, i1 = i0 + 8;
#pragma unroll
      for (int ks = 0; ks < KS; ++ks) {
        const int j0 = ks * 8 + t, j1 = j0 + 4;
        const uint2 x0 = (i0 < UT && j0 < UT) ? sAc[i0 * SP + j0] : z;
        const uint2 x1 = (i1 < UT && j0 < UT) ? sAc[i1 * SP + j0] : z;
        const uint2 x2 = (i0 < UT && j1 < UT) ? sAc[i0 * SP + j1] : z;
        const uint2 x3 = (i1 < UT && j1 < UT) ? sAc[i1 * SP + j1] : z;
        fah[mt][ks][0] = x0.x; fal[mt][ks][0] = x0.y;
        fah[mt][ks][1] = x1.x; fal[mt][ks][1] = x1.y;
        fah[mt][ks][2] = x2.x; fal[mt][ks][2] = x2.y;
        fah[mt][ks][3] = x3.x; fal[mt][ks][3] = x3.y;
      }
    }
  }

  // e = A p for the warp's eight right-hand sides; E[mt][d] in accumulator layout.
  __device__ __forceinline__ void matvec(float2* sP, int n0, float (&Er)[MT][4],
                                         float (&Ei)[MT][4]) {
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int mt = 0; mt < MT; ++mt)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int i = mt * 16 + g + 8 * h;
        if (i < UT) {
#pragma unroll
          for (int rr = 0; rr < 2; ++rr) sP[(n0 + 2 * t + rr) * SP + i] = p[mt][h][rr];
        }
      }
    __syncwarp();
    uint32_t bh[KS][2][2], bl[KS][2][2];  // [ks][reg][real / imaginary part]
#pragma unroll
    for (int ks = 0; ks < KS; ++ks) {
#pragma unroll
      for (int reg = 0; reg < 2; ++reg) {
        const int j = ks * 8 + t + 4 * reg;
        const float2 pj = (j < UT) ? sP[(n0 + g) * SP + j] : make_float2(0.f, 0.f);
        const uint2 sp = split_c<EL>(pj);
        bh[ks][reg][0] = neg_hi(sp.x);       // (pr, -pi): real part of A p
        bl[ks][reg][0] = neg_hi(sp.y);
        bh[ks][reg][1] = swap_halves(sp.x);  // (pi, pr): imaginary part
        bl[ks][reg][1] = swap_halves(sp.y);
      }
    }
    __syncwarp();
#pragma unroll
    for (int mt = 0; mt < MT; ++mt) {
      float hh[2][4], hl[2][4], lh[2][4];  // [re/im][d]
#pragma unroll
      for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int k = 0; k < 4; ++k) hh[c][k] = hl[c][k] = lh[c][k] = 0.f;
#pragma unroll
      for (int ks = 0; ks < KS; ++ks) {
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          mma16816<EL>(hh[c], fah[mt][ks], bh[ks][0][c], bh[ks][1][c]);
          mma16816<EL>(hl[c], fah[mt][ks], bl[ks][0][c], bl[ks][1][c]);
          mma16816<EL>(lh[c], fal[mt][ks], bh[ks][0][c], bh[ks][1][c]);
        }
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        Er[mt][k] = hh[0][k] + (hl[0][k] + lh[0][k]);
        Ei[mt][k] = hh[1][k] + (hl[1][k] + lh[1][k]);
      }
    }
  }

  // Lines 7-16 of Algorithm 1 with the approximate tracker of Eqs. 11-13.
  // res[mt][h][rr] holds the right-hand side of the owned positions on entry
  // (0 where padded). Quotients use the fast reciprocal (<= 2 ulp).
  __device__ __forceinline__ void run(const uint2* __restrict__ sAc, const float2* __restrict__ sA,
                                      float2* sP, int n0, int U, int R, int K, float* sAB) {
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    load_a(sAc);
    float D[MT][2];
#pragma unroll
    for (int mt = 0; mt < MT; ++mt)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int i = mt * 16 + g + 8 * h;
        D[mt][h] = (i < U) ? sA[i * UT + i].x : 0.f;
      }
    float s0 = 0.f, s1 = 0.f;
#pragma unroll
    for (int mt = 0; mt < MT; ++mt)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
#pragma unroll
        for (int rr = 0; rr < 2; ++rr) {
          v[mt][h][rr] = make_float2(0.f, 0.f);
          p[mt][h][rr] = res[mt][h][rr];
          l1[mt][h][rr] = l2[mt][h][rr] = l3[mt][h][rr] = 0.f;
        }
        s0 = fmaf(res[mt][h][0].x, res[mt][h][0].x, fmaf(res[mt][h][0].y, res[mt][h][0].y, s0));
        s1 = fmaf(res[mt][h][1].x, res[mt][h][1].x, fmaf(res[mt][h][1].y, res[mt][h][1].y, s1));
      }
    reduce8x2(s0, s1);
    rrn[0] = s0;
    rrn[1] = s1;
    float ia1[2], ia2[2];  // 1 / alpha_{k-1}, 1 / alpha_{k-2}
#pragma unroll
    for (int rr = 0; rr < 2; ++rr) {
      a1[rr] = a2[rr] = ia1[rr] = ia2[rr] = 1.f;
      be1[rr] = be2[rr] = 0.f;
      active[rr] = (n0 + 2 * t + rr) < R;
      broke[rr] = false;
      kd[rr] = 0;
    }
    for (int k = 1; k <= K; ++k) {
#pragma unroll
      for (int rr = 0; rr < 2; ++rr)
        if (active[rr] && !(rrn[rr] > 0.f)) {
          active[rr] = false;
          broke[rr] = true;
        }
      if (!__any_sync(0xffffffffu, active[0] || active[1])) break;
      float Er[MT][4], Ei[MT][4];
      matvec(sP, n0, Er, Ei);
      float pe[2] = {0.f, 0.f};
#pragma unroll
      for (int rr = 0; rr < 2; ++rr)
#pragma unroll
        for (int mt = 0; mt < MT; ++mt)
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const float2 pp = p[mt][h][rr];
            pe[rr] = fmaf(pp.x, Er[mt][2 * h + rr], fmaf(pp.y, Ei[mt][2 * h + rr], pe[rr]));
          }
      reduce8x2(pe[0], pe[1]);
      float alpha[2], rrnew[2] = {0.f, 0.f};
#pragma unroll
      for (int rr = 0; rr < 2; ++rr) {
        if (active[rr] && !(pe[rr] > 0.f)) {
          active[rr] = false;
          broke[rr] = true;
        }
        alpha[rr] = active[rr] ? __fdividef(rrn[rr], pe[rr]) : 0.f;
#pragma unroll
        for (int mt = 0; mt < MT; ++mt)
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            if (active[rr]) {
              v[mt][h][rr].x = fmaf(alpha[rr], p[mt][h][rr].x, v[mt][h][rr].x);
              v[mt][h][rr].y = fmaf(alpha[rr], p[mt][h][rr].y, v[mt][h][rr].y);
              res[mt][h][rr].x = fmaf(-alpha[rr], Er[mt][2 * h + rr], res[mt][h][rr].x);
              res[mt][h][rr].y = fmaf(-alpha[rr], Ei[mt][2 * h + rr], res[mt][h][rr].y);
            }
            rrnew[rr] = fmaf(res[mt][h][rr].x, res[mt][h][rr].x,
                             fmaf(res[mt][h][rr].y, res[mt][h][rr].y, rrnew[rr]));
          }
      }
      reduce8x2(rrnew[0], rrnew[1]);
#pragma unroll
      for (int rr = 0; rr < 2; ++rr) {
        if (!active[rr]) continue;
        const float al = alpha[rr];
        const float beta = __fdividef(rrnew[rr], rrn[rr]);
        const float c1 = al * (1.f + be1[rr]) * ia1[rr];
        const float c2 = al * be2[rr] * ia2[rr];
#pragma unroll
        for (int mt = 0; mt < MT; ++mt)
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            p[mt][h][rr].x = fmaf(beta, p[mt][h][rr].x, res[mt][h][rr].x);
            p[mt][h][rr].y = fmaf(beta, p[mt][h][rr].y, res[mt][h][rr].y);
            const float lk = (k == 1) ? al
                                      : l1[mt][h][rr] +
                                            (c1 - al * D[mt][h]) * (l1[mt][h][rr] - l2[mt][h][rr]) -
                                            c2 * (l2[mt][h][rr] - l3[mt][h][rr]);
            l3[mt][h][rr] = l2[mt][h][rr];
            l2[mt][h][rr] = l1[mt][h][rr];
            l1[mt][h][rr] = lk;
          }
        if (sAB != nullptr && g == 0) {
          const int r = n0 + 2 * t + rr;
          sAB[(r * KMAX + (k - 1)) * 2 + 0] = al;
          sAB[(r * KMAX + (k - 1)) * 2 + 1] = beta;
        }
        a2[rr] = a1[rr];
        a1[rr] = al;
        ia2[rr] = ia1[rr];
        ia1[rr] = __fdividef(1.f, al);
        be2[rr] = be1[rr];
        be1[rr] = beta;
        rrn[rr] = rrnew[rr];
        kd[rr] = k;
      }
    }
  }
};

// ---------------------------------------------------------------------------
// CG-D, tensor-core variant
// ---------------------------------------------------------------------------

// Work source traits: DetectArgs / PrecodeArgs describe one shape for the
// whole launch (instances taken by grid stride); BatchArgs hands out
// (problem, instance) units of uneven shapes from a device counter (and the
// serving sources of cg_serve.cuh hand out units of published requests).
template <class S> struct SrcTraits;
template <> struct SrcTraits<DetectArgs> { static constexpr bool kDyn = false; };
template <> struct SrcTraits<PrecodeArgs> { static constexpr bool kDyn = false; };
template <> struct SrcTraits<BatchArgs> { static constexpr bool kDyn = true; };

// Per-instance completion hook (a no-op except for serving sources).
template <class S>
__device__ __forceinline__ void src_done(const S&, int64_t, int) {}

__device__ __forceinline__ int64_t src_count(const DetectArgs& a) { return a.n_inst; }
__device__ __forceinline__ int64_t src_count(const PrecodeArgs& a) { return a.n_inst; }
__device__ __forceinline__ int64_t src_count(const BatchArgs& b) { return b.n_work; }

template <int UT, int EL, bool X3, bool FULL, class Src>
__device__ __forceinline__ void detect_tc_body(const Src& src, int PB, int PU, int PR,
                                               int PEX) {
  using C = TcCfg<UT>;
  constexpr int NTHR = C::NTHR, WM = C::WM, WK = C::WK, NT = C::NTD;
  constexpr bool kDyn = SrcTraits<Src>::kDyn;
  extern __shared__ __align__(128) unsigned char smem[];
  const TcPlan P = tc_detect_plan<UT>(PB, PU, PR, PEX);
  const float2* sHf = reinterpret_cast<const float2*>(smem + P.H);
  const float2* sYf = reinterpret_cast<const float2*>(smem + P.Y);
  float* part = reinterpret_cast<float*>(smem + P.Part);
  float2* sA = reinterpret_cast<float2*>(smem + P.A);
  uint2* sAc = reinterpret_cast<uint2*>(smem + P.Ac);
  float2* sBm = reinterpret_cast<float2*>(smem + P.Bm);
  float2* sP = reinterpret_cast<float2*>(smem + P.P);
  float2* sX = reinterpret_cast<float2*>(smem + P.X);
  float* sMu = reinterpret_cast<float*>(smem + P.Mu);
  float* sRho = reinterpret_cast<float*>(smem + P.Rho);
  float* sGd = reinterpret_cast<float*>(smem + P.Gd);
  int* sKd = reinterpret_cast<int*>(smem + P.Kd);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + P.misc);
  int* sStatus = reinterpret_cast<int*>(smem + P.misc + 8);
  int64_t* sClaim = reinterpret_cast<int64_t*>(smem + P.misc + 16);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int g = lane >> 2, t = lane & 3;
  const int64_t count = src_count(src);

  auto issue = [&](const DetItem& it) {
    const uint32_t hb = uint32_t(it.B) * it.U * 8u, yb = uint32_t(it.B) * 8u;
    mbar_arrive_expect_tx(bar, hb + uint32_t(it.R) * yb);
    bulk_copy_g2s(smem + P.H, it.H, hb, bar);
    for (int r = 0; r < it.R; ++r)
      bulk_copy_g2s(smem + P.Y + uint32_t(r) * P.YS * 8u, it.Y + r * it.B, yb, bar);
  };

  if (tid == 0) mbar_init(bar, 1);
  int64_t cur;
  if constexpr (kDyn) {
    claim_next(src, sClaim);
    __syncthreads();
    cur = *sClaim;
  } else {
    __syncthreads();
    cur = blockIdx.x < count ? int64_t(blockIdx.x) : -1;
  }
  uint32_t parity = 0;
  DetItem it{};
  if (cur >= 0) {
    it = det_item(src, cur);
    if (it.bulk && tid == 0) issue(it);
  }

  while (cur >= 0) {
    const int U = it.U, R = it.R, B = it.B;
    // ---- step 1: FP32 inputs in shared memory
    if (it.bulk) {
      if (!wait_inputs(bar, parity)) {
        if (tid == 0 && it.status) *it.status = ST_TIMEOUT;
        mbar_wait_bounded(bar, parity, WAIT_TIMEOUT_NS);
        return;
      }
      parity ^= 1u;
    } else {
      float2* f = reinterpret_cast<float2*>(smem);
      for (int e = tid; e < B * U; e += NTHR) f[e] = it.H[e];
      float2* fy = reinterpret_cast<float2*>(smem + P.Y);
      for (int e = tid; e < R * B; e += NTHR) {
        const int r = e / B, b = e - r * B;
        fy[r * P.YS + b] = it.Y[e];
      }
      __syncthreads();
    }
    if (tid == 0) *sStatus = 0;

    // ---- step 2: G and H^H Y on the tensor cores (Algorithm 1 line 5)
    float Cr[NT][4], Ci[NT][4];
    tc_gram_f32<UT, EL, X3, FULL, NT>(sHf, sYf, P.YS, B, U, R, warp % WM, warp / WM, WK, Cr,
                                      Ci);
    __syncthreads();  // the H/Y region becomes the partial buffer
#pragma unroll
    for (int nt = 0; nt < NT; ++nt)
#pragma unroll
      for (int d = 0; d < 4; ++d) {
        part[((warp * NT + nt) * 8 + d) * 32 + lane] = Cr[nt][d];
        part[((warp * NT + nt) * 8 + 4 + d) * 32 + lane] = Ci[nt][d];
      }
    __syncthreads();
    tc_reduce_warp<UT, EL, NT>(part, WK, U, R, it.sigma, sA, sAc, sBm, sGd);
    tc_zero_padding<UT>(U, R, sA, sAc, sBm, sGd, NTHR);
    if constexpr (kDyn) claim_try(src, sClaim);  // never blocks the current instance
    __syncthreads();
    int64_t next;
    if constexpr (kDyn) {
      next = *sClaim;
    } else {
      next = cur + gridDim.x < count ? cur + gridDim.x : -1;
    }
    DetItem nit{};
    if (next >= 0) nit = det_item(src, next);  // -1: no more work; -2: ask again later
    if (next >= 0 && nit.bulk && !it.exact && tid == 0) {
      fence_proxy_async_smem();
      issue(nit);
    }

    // ---- step 3: Algorithm 1 lines 7-16
    float* sAB = it.exact ? reinterpret_cast<float*>(smem + P.AB) : nullptr;
    if (warp * 8 < R) {
      const int n0 = warp * 8;
      TcCg<UT, EL> cg;
#pragma unroll
      for (int mt = 0; mt < WM; ++mt)
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
          for (int rr = 0; rr < 2; ++rr) {
            const int i = mt * 16 + g + 8 * h, r = n0 + 2 * t + rr;
            cg.res[mt][h][rr] = (i < U && r < R) ? sBm[r * UT + i] : make_float2(0.f, 0.f);
          }
      cg.run(sAc, sA, sP, n0, U, R, it.K, sAB);
#pragma unroll
      for (int rr = 0; rr < 2; ++rr) {
        const int r = n0 + 2 * t + rr;
        if (r >= R) continue;
#pragma unroll
        for (int mt = 0; mt < WM; ++mt)
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int i = mt * 16 + g + 8 * h;
            if (i < U) {
              sX[r * UT + i] = cg.v[mt][h][rr];
              sMu[r * UT + i] = cg.l1[mt][h][rr] * sGd[i];  // Eq. 12
              sRho[r * UT + i] = sGd[i] / it.N0;            // Eq. 13
            }
          }
        if (g == 0) {
          sKd[r] = cg.kd[rr];
          if (cg.broke[rr]) atomicOr(sStatus, ST_BREAKDOWN);
        }
      }
    }
    __syncthreads();

    // ---- step 4: exact SINR (Eq. 10)
    if (it.exact) {
      exact_tracker<UT, NTHR>(reinterpret_cast<float2*>(smem), sA, sAB, sKd, U, R, it.sigma,
                              it.N0, it.Es, sMu, sRho);
      __syncthreads();
      if (next >= 0 && nit.bulk && tid == 0) {
        fence_proxy_async_smem();
        issue(nit);
      }
    }

    // ---- step 5: outputs (x_hat, mu, rho, LLRs of Eq. 4)
    {
      DetectArgs o{};
      o.xhat = it.xhat; o.mu = it.mu; o.rho = it.rho; o.llr = it.llr;
      o.U = U; o.R = R; o.q = it.q; o.Es = it.Es;
      write_detect_outputs<UT, NTHR>(o, 0, sX, sMu, sRho, sStatus);
    }
    __syncthreads();
    if (tid == 0) {
      const int st = *sStatus;
      if (it.status) *it.status = st;
      src_done(src, cur, st);
    }
    if constexpr (kDyn) {
      if (next == -2) {  // nothing was ready earlier: wait for work now (bounded)
        claim_next(src, sClaim);
        __syncthreads();
        next = *sClaim;
        if (next >= 0) {
          nit = det_item(src, next);
          if (nit.bulk && tid == 0) {
            fence_proxy_async_smem();
            issue(nit);
          }
        }
      }
    }
    cur = next;
    it = nit;
  }
}

template <int UT, int EL, bool X3, bool FULL>
__global__ void __launch_bounds__(TcCfg<UT>::NTHR, UT == 32 ? 1 : 4)
    detect_tc_kernel(const DetectArgs a) {
  detect_tc_body<UT, EL, X3, FULL>(a, a.B, a.U, a.R, a.exact);
}

// Batched form: one bin of uneven problems; the plan shape (PB, UT, PR, PEX)
// bounds every problem of the bin, so the shared-memory layout is fixed.
template <int UT, int EL, bool X3, bool FULL>
__global__ void __launch_bounds__(TcCfg<UT>::NTHR, UT == 32 ? 1 : 4)
    detect_tc_batch_kernel(const BatchArgs b) {
  detect_tc_body<UT, EL, X3, FULL>(b, b.PB, UT, b.PR, b.PEX);
}

// ---------------------------------------------------------------------------
// CG-P, tensor-core variant
// ---------------------------------------------------------------------------

template <int UT, int EL, bool X3, bool FULL, class Src>
__device__ __forceinline__ void precode_tc_body(const Src& src, int PB, int PU, int PR) {
  using C = TcCfg<UT>;
  constexpr int NTHR = C::NTHR, NWARP = C::NWARP, WM = C::WM, WK = C::WK, NT = C::NTP;
  constexpr int SP = C::SP, KSV = C::KSC;
  constexpr bool kDyn = SrcTraits<Src>::kDyn;
  extern __shared__ __align__(128) unsigned char smem[];
  const TcPlan P = tc_precode_plan<UT>(PB, PU, PR);
  const uint2* Hc = reinterpret_cast<const uint2*>(smem + P.H);
  const float2* sT = reinterpret_cast<const float2*>(smem + P.Y);
  float* part = reinterpret_cast<float*>(smem + P.Part);
  float2* sA = reinterpret_cast<float2*>(smem + P.A);
  uint2* sAc = reinterpret_cast<uint2*>(smem + P.Ac);
  float2* sP = reinterpret_cast<float2*>(smem + P.P);
  float* sNrm = reinterpret_cast<float*>(smem + P.Nrm);
  float* sGd = reinterpret_cast<float*>(smem + P.Gd);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + P.misc);
  int* sStatus = reinterpret_cast<int*>(smem + P.misc + 8);
  int64_t* sClaim = reinterpret_cast<int64_t*>(smem + P.misc + 16);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int g = lane >> 2, t = lane & 3;
  const int64_t count = src_count(src);

  if (tid == 0) mbar_init(bar, 1);
  int64_t n;
  if constexpr (kDyn) {
    claim_next(src, sClaim);
    __syncthreads();
    n = *sClaim;
  } else {
    __syncthreads();
    n = blockIdx.x < count ? int64_t(blockIdx.x) : -1;
  }
  uint32_t parity = 0;
  while (n >= 0) {
    const PreItem a = pre_item(src, n);
    const int U = a.U, R = a.R, B = a.B;
    const int B8 = (B + 7) & ~7;  // this problem's padded antenna count (layout uses P)
    const bool bulk = a.bulk_h || a.bulk_t;
    // ---- step 1: inputs
    if (bulk && tid == 0) {
      fence_proxy_async_smem();
      uint32_t bytes = 0;
      if (a.bulk_h) bytes += uint32_t(B) * U * 8u;
      if (a.bulk_t) bytes += uint32_t(R) * U * 8u;
      mbar_arrive_expect_tx(bar, bytes);
      if (a.bulk_h) bulk_copy_g2s(smem + P.H, a.H, uint32_t(B) * U * 8u, bar);
      if (a.bulk_t) bulk_copy_g2s(smem + P.Y, a.T, uint32_t(R) * U * 8u, bar);
    }
    if (!a.bulk_h) {
      float2* f = reinterpret_cast<float2*>(smem + P.H);
      for (int e = tid; e < B * U; e += NTHR) f[e] = a.H[e];
    }
    if (!a.bulk_t) {
      float2* f = reinterpret_cast<float2*>(smem + P.Y);
      for (int e = tid; e < R * U; e += NTHR) f[e] = a.T[e];
    }
    if (bulk) {
      if (!wait_inputs(bar, parity)) {
        if (tid == 0 && a.status) *a.status = ST_TIMEOUT;
        mbar_wait_bounded(bar, parity, WAIT_TIMEOUT_NS);
        return;
      }
      parity ^= 1u;
    } else {
      __syncthreads();
    }
    if (tid == 0) *sStatus = 0;

    // ---- step 2: A = H^H H + sigma I on the tensor cores (Algorithm 1 line 6)
    if (FULL)
      convert_h_full<EL, NTHR, UT>(smem + P.H, B);
    else
      convert_h<EL, NTHR>(smem + P.H, B, B8, U);
    __syncthreads();
    {
      float Cr[NT][4], Ci[NT][4];
      tc_gram<UT, EL, X3, NT>(Hc, nullptr, 0, B8, U, U, warp % WM, warp / WM, WK, Cr, Ci);
#pragma unroll
      for (int nt = 0; nt < NT; ++nt)
#pragma unroll
        for (int d = 0; d < 4; ++d) {
          part[((warp * NT + nt) * 8 + d) * 32 + lane] = Cr[nt][d];
          part[((warp * NT + nt) * 8 + 4 + d) * 32 + lane] = Ci[nt][d];
        }
    }
    __syncthreads();
    tc_reduce<UT, EL, NT>(part, WK, U, 0, U, a.sigma, sA, sAc, nullptr, sGd, NTHR);
    __syncthreads();

    // ---- step 3: CG with b = t, then ||q||^2 = v^H G v (G = A - sigma I)
    if (warp * 8 < R) {
      const int n0 = warp * 8;
      TcCg<UT, EL> cg;
#pragma unroll
      for (int mt = 0; mt < WM; ++mt)
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
          for (int rr = 0; rr < 2; ++rr) {
            const int i = mt * 16 + g + 8 * h, r = n0 + 2 * t + rr;
            cg.res[mt][h][rr] = (i < U && r < R) ? sT[r * U + i] : make_float2(0.f, 0.f);
          }
      cg.run(sAc, sA, sP, n0, U, R, a.K, nullptr);
      // w = A v, ||q||^2 = v^H w - sigma ||v||^2
#pragma unroll
      for (int mt = 0; mt < WM; ++mt)
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
          for (int rr = 0; rr < 2; ++rr) cg.p[mt][h][rr] = cg.v[mt][h][rr];
      float Er[WM][4], Ei[WM][4];
      cg.matvec(sP, n0, Er, Ei);
      float qq2[2] = {0.f, 0.f};
#pragma unroll
      for (int rr = 0; rr < 2; ++rr)
#pragma unroll
        for (int mt = 0; mt < WM; ++mt)
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const float2 vv = cg.v[mt][h][rr];
            const float wx = fmaf(-a.sigma, vv.x, Er[mt][2 * h + rr]);
            const float wy = fmaf(-a.sigma, vv.y, Ei[mt][2 * h + rr]);
            qq2[rr] = fmaf(vv.x, wx, fmaf(vv.y, wy, qq2[rr]));
          }
      TcCg<UT, EL>::reduce8x2(qq2[0], qq2[1]);
#pragma unroll
      for (int rr = 0; rr < 2; ++rr) {
        const float qq = qq2[rr];
        const int r = n0 + 2 * t + rr;
        if (g == 0 && r < R) {
          const float nr = sqrtf(fmaxf(qq, 0.f));
          sNrm[r] = nr;
          if (a.qnorm) a.qnorm[r] = nr;
          if (cg.broke[rr]) atomicOr(sStatus, ST_BREAKDOWN);
        }
      }
      __syncwarp();
      // V into sP (row r, stride SP) for the q = H v fragments; padded users 0
#pragma unroll
      for (int mt = 0; mt < WM; ++mt)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int i = mt * 16 + g + 8 * h;
          if (i < UT) {
#pragma unroll
            for (int rr = 0; rr < 2; ++rr) {
              const int r = n0 + 2 * t + rr;
              sP[r * SP + i] = (i < U && r < R) ? cg.v[mt][h][rr] : make_float2(0.f, 0.f);
            }
          }
        }
    } else if (warp * 8 < RMAX) {
      // rows of V beyond R stay zero
      for (int e = lane; e < 8 * SP; e += 32) sP[warp * 8 * SP + e] = make_float2(0.f, 0.f);
    }
    __syncthreads();

    // ---- step 4: q = H v on the tensor cores (line 20), optional s = q / ||q||
    {
      const int ntv = (R + 7) / 8;
      uint32_t vh[2][KSV][2][2], vl[2][KSV][2][2];  // [nt][ks][reg][re/im part]
#pragma unroll
      for (int nt = 0; nt < 2; ++nt)
#pragma unroll
        for (int ks = 0; ks < KSV; ++ks)
#pragma unroll
          for (int reg = 0; reg < 2; ++reg) {
            const int j = ks * 8 + t + 4 * reg;
            const int r = nt * 8 + g;
            const float2 vj = (nt < ntv && j < UT) ? sP[r * SP + j] : make_float2(0.f, 0.f);
            const uint2 sv = split_c<EL>(vj);
            vh[nt][ks][reg][0] = neg_hi(sv.x);       // (vr, -vi): real part of H v
            vl[nt][ks][reg][0] = neg_hi(sv.y);
            vh[nt][ks][reg][1] = swap_halves(sv.x);  // (vi, vr): imaginary part
            vl[nt][ks][reg][1] = swap_halves(sv.y);
          }
      const int MTQ = (B8 + 15) / 16;
      for (int mt = warp; mt < MTQ; mt += NWARP) {
        const int r0 = mt * 16 + g, r1 = r0 + 8;  // antenna rows of this m-tile
        float Qr[2][4], Qi[2][4];
#pragma unroll
        for (int nt = 0; nt < 2; ++nt)
#pragma unroll
          for (int k = 0; k < 4; ++k) Qr[nt][k] = Qi[nt][k] = 0.f;
#pragma unroll
        for (int ks = 0; ks < KSV; ++ks) {
          const int j0 = ks * 8 + t, j1 = j0 + 4;
          uint32_t ah[4], al[4];
          const uint2 z = make_uint2(0u, 0u);
          const uint2 x0 = (r0 < B8 && j0 < U) ? Hc[r0 * U + (j0 ^ hswz(r0, U))] : z;
          const uint2 x1 = (r1 < B8 && j0 < U) ? Hc[r1 * U + (j0 ^ hswz(r1, U))] : z;
          const uint2 x2 = (r0 < B8 && j1 < U) ? Hc[r0 * U + (j1 ^ hswz(r0, U))] : z;
          const uint2 x3 = (r1 < B8 && j1 < U) ? Hc[r1 * U + (j1 ^ hswz(r1, U))] : z;
          ah[0] = x0.x; al[0] = x0.y;
          ah[1] = x1.x; al[1] = x1.y;
          ah[2] = x2.x; al[2] = x2.y;
          ah[3] = x3.x; al[3] = x3.y;
#pragma unroll
          for (int nt = 0; nt < 2; ++nt) {
            if (nt < ntv) {
              mma_split<EL, X3>(Qr[nt], ah, al, vh[nt][ks][0][0], vh[nt][ks][1][0],
                                vl[nt][ks][0][0], vl[nt][ks][1][0]);
              mma_split<EL, X3>(Qi[nt], ah, al, vh[nt][ks][0][1], vh[nt][ks][1][1],
                                vl[nt][ks][0][1], vl[nt][ks][1][1]);
            }
          }
        }
#pragma unroll
        for (int nt = 0; nt < 2; ++nt) {
          if (nt >= ntv) continue;
#pragma unroll
          for (int d = 0; d < 4; ++d) {
            const int b = (d & 2) ? r1 : r0;
            const int r = nt * 8 + 2 * t + (d & 1);
            if (b < B && r < R) {
              float2 val = make_float2(Qr[nt][d], Qi[nt][d]);
              if (a.normalize) {
                const float nr = sNrm[r];
                const float inv = nr > 0.f ? 1.f / nr : 0.f;
                val.x *= inv;
                val.y *= inv;
              }
              a.q[r * B + b] = val;
            }
          }
        }
      }
    }
    __syncthreads();
    if (tid == 0) {
      const int st = *sStatus;
      if (a.status) *a.status = st;
      src_done(src, n, st);
    }
    if constexpr (kDyn) claim_next(src, sClaim);
    __syncthreads();
    if constexpr (kDyn) {
      n = *sClaim;
    } else {
      n = n + gridDim.x < count ? n + gridDim.x : -1;
    }
  }
}

template <int UT, int EL, bool X3, bool FULL>
__global__ void __launch_bounds__(TcCfg<UT>::NTHR, UT == 32 ? 1 : 4)
    precode_tc_kernel(const PrecodeArgs a) {
  precode_tc_body<UT, EL, X3, FULL>(a, a.B, a.U, a.R);
}

template <int UT, int EL, bool X3, bool FULL>
__global__ void __launch_bounds__(TcCfg<UT>::NTHR, UT == 32 ? 1 : 4)
    precode_tc_batch_kernel(const BatchArgs b) {
  precode_tc_body<UT, EL, X3, FULL>(b, b.PB, UT, b.PR);
}

}  // namespace cgm
