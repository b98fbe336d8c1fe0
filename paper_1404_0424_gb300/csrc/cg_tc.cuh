// Tensor-core helpers and work sources of the warp-per-instance kernels
// (cg_warp.cuh).
//
// Every dense contraction of the method runs on the tensor cores as
// mma.sync.m16n8k16 with FP16 or BF16 operands and FP32 accumulation:
//   * G = H^H H and the matched filters H^H Y (Algorithm 1; Eqs. 7, 8),
//   * e = A p for all right-hand sides of an instance at once (the CG
//     iterations of Algorithm 1),
//   * q = H v for all right-hand sides (precoding, Sec. III-D).
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

// ---------------------------------------------------------------------------
// Work sources: where a warp finds its next instance and that instance's
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


// ---------------------------------------------------------------------------
// Work source traits
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

}  // namespace cgm
