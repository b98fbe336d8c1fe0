// Warp-per-instance tensor-core kernels for CG-D and CG-P with up to 32 users.
//
// One warp owns one instance (a channel H with its R <= 16 right-hand sides)
// from its first load to its last store, so no CTA barrier is involved:
//   1. CG-D stages H and Y through a per-warp shared-memory ring, STAGES - 1
//      k-steps of 8 antennas ahead of the products (the first stages of the
//      next instance are issued before the CG of the current one), filled
//      by one lane's tensor copies (TMA) in single calls and by the lanes'
//      cp.async copies otherwise; CG-P, which reads H a second time for
//      q = H v, loads it with 16-byte register loads through L1;
//   2. G = H^H H and the transposed matched filters B^T = Y^T conj(H)
//      (the Gram and matched-filter step of Algorithm 1) accumulate on the
//      tensor cores;
//   3. the CG iterations and tracker updates of Algorithm 1 run entirely in
//      registers. Users are numbered
//      in a "position" order chosen so that the Gram accumulators of a lane
//      are exactly its B fragments of e = A p, and the matched-filter
//      accumulators are exactly the layout of the CG vectors: accumulator
//      row = right-hand side, accumulator column = position. Inner products
//      over users are quad shuffles (compensated sums);
//   4. x_hat, mu, rho and the max-log LLRs of Eq. 4 (CG-D) or q = H v (CG-P,
//      the precoding output of Algorithm 1) are stored from the registers that
//      hold them.
//
// Position P (0 <= P < 8 NB) holds user pos_user(P). With 16 or 32 users the
// 8-blocks interleave in pairs (P = 16 m + 8 h + w holds user 16 m + 2 w + h),
// which makes the users a lane touches contiguous in memory; 32 users use
// two 16-position m-tiles for the Gram rows. Every product is a split
// (hi + lo) one in X3 mode, as in cg_tc.cuh; e = A p always is.
#pragma once

#include "cg_tc.cuh"

#ifndef CGM_WARP_MINB32
#define CGM_WARP_MINB32 2  // resident CTAs per SM the register allocation targets at 32 users
#endif
#ifndef CGM_WARP_MINB
#define CGM_WARP_MINB 3  // resident CTAs per SM the register allocation targets at 16 users
#endif

namespace cgm {

// Load stages of the per-warp ring (16-byte cp.async copies), by padded
// user count; 32 users have no shared memory for more than 4.
#ifndef CGM_RING8
#define CGM_RING8 4
#endif

#ifndef CGM_RING16
#define CGM_RING16 4
#endif

template <int UT>
struct WarpCfg {
  static_assert(UT == 8 || UT == 16 || UT == 32, "warp kernels serve 8, 16 or 32 padded users");
  static constexpr int NB = UT / 8;              // 8-position blocks
  static constexpr int MT = UT == 32 ? 2 : 1;    // 16-position m-tiles of the Gram rows
  static constexpr int PLANES = 2 * MT + 2;      // ring planes per stage: H rows, then Y
  static constexpr int STAGES = UT == 32 ? 4 : UT == 16 ? CGM_RING16 : CGM_RING8;
  // The CG B fragments of A are kept hi|lo, and times i as well unless that
  // would not fit (32 users form i A on the fly).
  static constexpr bool STORE_IM = UT <= 16;
  static constexpr int NFRAG = NB * NB * 2 * (STORE_IM ? 2 : 1);  // (ks, nt, b0/b1[, re/im])
  static constexpr int WARPS = 4;                // warps per CTA (independent)
  static constexpr int NTHR = 32 * WARPS;
  // resident CTAs per SM targeted: 8 users fit 4 CTAs in 128 registers; 16
  // users run faster at 3 CTAs without spills than at 4 with them
  static constexpr int MINB = UT == 32 ? CGM_WARP_MINB32 : UT == 16 ? CGM_WARP_MINB : 4;
  // per warp: a ring of STAGES load stages (PLANES planes of 16 bytes
  // per lane each), the CG B fragments (one uint2 per lane and fragment), and
  // alpha_k, beta_k of the 16 right-hand-side rows for the tracker (K <= UT)
  static constexpr uint32_t RING_BYTES = uint32_t(STAGES) * PLANES * 32u * 16u;
  static constexpr uint32_t FRAG_BYTES = uint32_t(NFRAG) * 32u * 8u;
  static constexpr uint32_t AB_BYTES = uint32_t(UT) * 16u * 8u;
  static constexpr uint32_t WARP_BYTES = RING_BYTES + FRAG_BYTES + AB_BYTES;
  static constexpr uint32_t SMEM = uint32_t(WARPS) * WARP_BYTES;       // CG-D
  // CG-D staged by TMA: the warps' slices, then STAGES mbarriers per warp
  static constexpr uint32_t TMA_SMEM = SMEM + uint32_t(WARPS) * STAGES * 8u;
  static constexpr uint32_t PRE_SMEM = uint32_t(WARPS) * FRAG_BYTES;  // CG-P: fragments only
};

template <int UT>
__host__ __device__ constexpr int pos_user(int P) {
  return UT == 8 ? P : 16 * (P >> 4) + 2 * (P & 7) + ((P >> 3) & 1);
}

// Gram accumulators of a lane: [m-tile][n-tile][accumulator register].
template <int UT>
using GramAcc = float[WarpCfg<UT>::MT][UT / 8][4];
// Matched-filter (or CG vector) accumulators: [n-tile][accumulator register].
template <int UT>
using VecAcc = float[UT / 8][4];

__device__ __forceinline__ float4 ldg4(const float2* p) {
  return __ldg(reinterpret_cast<const float4*>(p));
}
__device__ __forceinline__ float2 ldg2(const float2* p) { return __ldg(p); }

// Asynchronous global -> shared copies (16 or 8 bytes), zero-filled when
// !ok (src is then not read). Completion is tracked per thread in groups.
__device__ __forceinline__ void cp_async16(void* dst, const void* src, bool ok) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem_addr(dst)), "l"(src),
               "r"(ok ? 16 : 0)
               : "memory");
}
__device__ __forceinline__ void cp_async8(void* dst, const void* src, bool ok) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(smem_addr(dst)), "l"(src),
               "r"(ok ? 8 : 0)
               : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Stage `slot` of a warp ring: plane j of lane l at ring + (slot*PL + j)*512 + 16 l.
template <int PL>
__device__ __forceinline__ unsigned char* ring_at(unsigned char* ring, int slot, int plane) {
  return ring + (slot * PL + plane) * 512 + (threadIdx.x & 31) * 16;
}

// Issues one Gram k-step (antennas 8 ks + 2t, +1) into the ring: planes
// 2 m, 2 m + 1 the lane's H fragments of m-tile m, the last two (MF) its Y
// fragments; then commits a group (an empty one when ks >= KS, which keeps
// the group count uniform). Only the vector layout (U == UT, B even,
// 16-byte aligned) comes here.
template <int UT, bool MF>
__device__ __forceinline__ void ring_gram_issue(unsigned char* ring, const float2* H,
                                                const float2* Y, int B, int R, int KS, int ks) {
  constexpr int PL = WarpCfg<UT>::PLANES, MT = WarpCfg<UT>::MT;
  if (ks < KS) {
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int slot = ks % WarpCfg<UT>::STAGES;
    const int b0 = 8 * ks + 2 * t, b1 = b0 + 1;
    const bool ok = b0 < B;
    if constexpr (UT == 8) {
      cp_async8(ring_at<PL>(ring, slot, 0), ok ? H + b0 * 8 + g : H, ok);
      cp_async8(ring_at<PL>(ring, slot, 1), ok ? H + b1 * 8 + g : H, ok);
    } else {
#pragma unroll
      for (int m = 0; m < MT; ++m) {
        cp_async16(ring_at<PL>(ring, slot, 2 * m), ok ? H + b0 * UT + 16 * m + 2 * g : H, ok);
        cp_async16(ring_at<PL>(ring, slot, 2 * m + 1), ok ? H + b1 * UT + 16 * m + 2 * g : H, ok);
      }
    }
    if constexpr (MF) {
      const bool ok0 = ok && g < R, ok1 = ok && g + 8 < R;
      cp_async16(ring_at<PL>(ring, slot, 2 * MT), ok0 ? Y + g * B + b0 : Y, ok0);
      cp_async16(ring_at<PL>(ring, slot, 2 * MT + 1), ok1 ? Y + (g + 8) * B + b0 : Y, ok1);
    }
  }
  cp_commit();
}

template <int UT, bool MF>
__device__ __forceinline__ void ring_gram_read(unsigned char* ring, int ks,
                                               float2 (&h)[WarpCfg<UT>::MT][4], float2 (&y)[4]) {
  constexpr int PL = WarpCfg<UT>::PLANES, MT = WarpCfg<UT>::MT;
  const int slot = ks % WarpCfg<UT>::STAGES;
  if constexpr (UT == 8) {
    h[0][0] = *reinterpret_cast<const float2*>(ring_at<PL>(ring, slot, 0));
    h[0][2] = *reinterpret_cast<const float2*>(ring_at<PL>(ring, slot, 1));
    h[0][1] = h[0][3] = make_float2(0.f, 0.f);
  } else {
#pragma unroll
    for (int m = 0; m < MT; ++m) {
      const float4 v0 = *reinterpret_cast<const float4*>(ring_at<PL>(ring, slot, 2 * m));
      const float4 v1 = *reinterpret_cast<const float4*>(ring_at<PL>(ring, slot, 2 * m + 1));
      h[m][0] = make_float2(v0.x, v0.y);
      h[m][1] = make_float2(v0.z, v0.w);
      h[m][2] = make_float2(v1.x, v1.y);
      h[m][3] = make_float2(v1.z, v1.w);
    }
  }
  if constexpr (MF) {
    const float4 w0 = *reinterpret_cast<const float4*>(ring_at<PL>(ring, slot, 2 * MT));
    const float4 w1 = *reinterpret_cast<const float4*>(ring_at<PL>(ring, slot, 2 * MT + 1));
    y[0] = make_float2(w0.x, w0.y);
    y[2] = make_float2(w0.z, w0.w);
    y[1] = make_float2(w1.x, w1.y);
    y[3] = make_float2(w1.z, w1.w);
  }
}

// First STAGES - 1 k-steps of an instance's Gram.
template <int UT, bool MF>
__device__ __forceinline__ void ring_gram_prologue(unsigned char* ring, const float2* H,
                                                   const float2* Y, int B, int R) {
  const int KS = (B + 7) / 8;
#pragma unroll
  for (int ks = 0; ks < WarpCfg<UT>::STAGES - 1; ++ks) ring_gram_issue<UT, MF>(ring, H, Y, B, R, KS, ks);
}

// ---------------------------------------------------------------------------
// Gram k-steps staged by the tensor memory accelerator (TMA)
// ---------------------------------------------------------------------------

// The same ring, filled by one lane with two 3-D tensor copies per k-step
// (DetectArgs::tmH, tmY) that complete on the slot's mbarrier. A slot holds
// the H box of each m-tile (8 antenna rows of 16 users, 128 bytes a row,
// 128-byte swizzle: 16-byte chunk c of row r sits at chunk c ^ r; with 8
// users, rows of 64 bytes with 64-byte swizzle: chunk c of row r at
// c ^ (r / 2)), then at byte 1024 MT the Y box (16 right-hand-side rows of
// 8 antennas, 64 bytes a row, unswizzled; rows past R and antennas past B
// arrive as zeros). Lane (g, t) reads exactly the fragments the cp.async
// ring gives it, without bank conflicts. Slots sit at multiples of 1024
// bytes, the span of the swizzle pattern.
struct TmaRing {
  uint32_t bar;  // shared-space address of this warp's STAGES mbarriers (8 bytes apart)
  uint32_t st;   // bits 0-15: parity of each slot's next phase; 16-31: slots in flight
};

__device__ __forceinline__ void tma_ring_init(TmaRing& tr, uint32_t bar, int stages) {
  tr.bar = bar;
  tr.st = 0;
  if ((threadIdx.x & 31) == 0) {
    for (int i = 0; i < stages; ++i) mbar_init_s(bar + 8 * i, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
}

// Issues k-step ks (< KS) of instance z into its slot. Every lane has read
// the slot's previous contents into registers before the __syncwarp.
template <int UT, bool MF, int S = WarpCfg<UT>::STAGES>
__device__ __forceinline__ void tma_gram_issue(unsigned char* ring, TmaRing& tr,
                                               const CUtensorMap* tmH, const CUtensorMap* tmY,
                                               int z, int KS, int ks) {
  if (ks >= KS) return;
  constexpr int MT = WarpCfg<UT>::MT, PL = WarpCfg<UT>::PLANES;
  constexpr uint32_t HBOX = UT == 8 ? 512u : 1024u;
  const int slot = ks % S;
  __syncwarp();
  if ((threadIdx.x & 31) == 0) {
    const uint32_t base = smem_addr(ring) + slot * PL * 512;
    const uint32_t bar = tr.bar + 8 * slot;
    mbar_arrive_expect_tx_s(bar, MT * HBOX + (MF ? 1024u : 0u));
#pragma unroll
    for (int m = 0; m < MT; ++m) tma_load_3d_s(base + m * 1024, tmH, 32 * m, 8 * ks, z, bar);
    if constexpr (MF) tma_load_3d_s(base + MT * 1024, tmY, 16 * ks, 0, z, bar);
  }
  tr.st |= 65536u << slot;
}

// First S - 1 k-steps ks0, ks0 + 1, ... (below KS) of instance z. The fence
// orders earlier generic writes to the ring (scratch) before the tensor
// copies that overwrite it.
template <int UT, bool MF, int S = WarpCfg<UT>::STAGES>
__device__ __forceinline__ void tma_gram_prologue(unsigned char* ring, TmaRing& tr,
                                                  const CUtensorMap* tmH, const CUtensorMap* tmY,
                                                  int z, int KS, int ks0 = 0) {
  fence_proxy_async_smem();
#pragma unroll
  for (int i = 0; i < S - 1; ++i) tma_gram_issue<UT, MF, S>(ring, tr, tmH, tmY, z, KS, ks0 + i);
}

// Waits for k-step ks (bounded by wait_ns) and reads the lane's fragments;
// false (warp-uniform) if the wait ran out. The slot then stays marked in
// flight with its phase pending, the fragments are not valid, and the
// caller issues nothing more on this ring: a second arrival on a pending
// phase, or a second copy into a slot still being written, is not allowed.
template <int UT, bool MF, int S = WarpCfg<UT>::STAGES>
__device__ __forceinline__ bool tma_gram_read(unsigned char* ring, TmaRing& tr, int ks,
                                              uint64_t wait_ns,
                                              float2 (&h)[WarpCfg<UT>::MT][4], float2 (&y)[4]) {
  constexpr int MT = WarpCfg<UT>::MT, PL = WarpCfg<UT>::PLANES;
  const int slot = ks % S;
  const bool ok = __all_sync(
      0xffffffffu, mbar_wait_bounded_s(tr.bar + 8 * slot, (tr.st >> slot) & 1u, wait_ns));
  if (!ok) return false;
  tr.st ^= 1u << slot;
  tr.st &= ~(65536u << slot);
  const unsigned char* base = ring + slot * PL * 512;
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int r0 = 2 * t, r1 = 2 * t + 1;
  if constexpr (UT == 8) {
    h[0][0] = *reinterpret_cast<const float2*>(
        base + r0 * 64 + ((((g >> 1) ^ (r0 >> 1)) & 3) << 4) + ((g & 1) << 3));
    h[0][2] = *reinterpret_cast<const float2*>(
        base + r1 * 64 + ((((g >> 1) ^ (r1 >> 1)) & 3) << 4) + ((g & 1) << 3));
    h[0][1] = h[0][3] = make_float2(0.f, 0.f);
  } else {
#pragma unroll
    for (int m = 0; m < MT; ++m) {
      const float4 v0 =
          *reinterpret_cast<const float4*>(base + m * 1024 + r0 * 128 + ((g ^ r0) << 4));
      const float4 v1 =
          *reinterpret_cast<const float4*>(base + m * 1024 + r1 * 128 + ((g ^ r1) << 4));
      h[m][0] = make_float2(v0.x, v0.y);
      h[m][1] = make_float2(v0.z, v0.w);
      h[m][2] = make_float2(v1.x, v1.y);
      h[m][3] = make_float2(v1.z, v1.w);
    }
  }
  if constexpr (MF) {
    const float4 w0 = *reinterpret_cast<const float4*>(base + MT * 1024 + g * 64 + t * 16);
    const float4 w1 = *reinterpret_cast<const float4*>(base + MT * 1024 + (g + 8) * 64 + t * 16);
    y[0] = make_float2(w0.x, w0.y);
    y[2] = make_float2(w0.z, w0.w);
    y[1] = make_float2(w1.x, w1.y);
    y[3] = make_float2(w1.z, w1.w);
  }
  return true;
}

// Waits (bounded) for every slot still in flight, so that no copy lands in
// shared memory after the warp is done with it. Each such slot has exactly
// one pending phase, the one its parity bit names.
__device__ __forceinline__ void tma_ring_drain(TmaRing& tr, int stages) {
#pragma unroll 1
  for (int slot = 0; slot < stages; ++slot)
    if ((tr.st >> (16 + slot)) & 1u) {
      mbar_wait_bounded_s(tr.bar + 8 * slot, (tr.st >> slot) & 1u, WAIT_TIMEOUT_NS);
      tr.st ^= 1u << slot;
    }
  tr.st &= 65535u;
}

// Prefetch into L1 of the 8-antenna block ks of an instance's H with UT
// users per row (U == UT: 8 rows of UT complex = UT / 2 lines of 128 bytes,
// one per lane). Blocks past the end of H are skipped, so every address is
// inside the instance. The register loads of the 16-byte paths run only one
// block ahead; these keep several blocks of DRAM or L2 latency covered
// without holding registers.
template <int UT>
__device__ __forceinline__ void prefetch_h_block(const float2* H, int B, int ks) {
  constexpr int LINES = UT / 2;
  const int lane = threadIdx.x & 31;
  if (lane < LINES && 8 * ks < B) {
    const int64_t byte = int64_t(ks) * (64 * UT) + int64_t(lane) * 128;
    if (byte < int64_t(B) * UT * 8) {
      const char* p = reinterpret_cast<const char*>(H) + byte;
      asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
    }
  }
}
// Prefetch into L1 of `bytes` contiguous bytes from p (16-byte aligned),
// one 128-byte line per lane; only lines that start inside the range.
__device__ __forceinline__ void prefetch_rows_l1(const void* p, int bytes) {
  const char* c = reinterpret_cast<const char*>(p);
  const int base = int(reinterpret_cast<uintptr_t>(c) & 127);
  for (int off = (threadIdx.x & 31) * 128 - base; off < bytes; off += 32 * 128)
    if (off + 128 > 0) asm volatile("prefetch.global.L1 [%0];" ::"l"(c + (off < 0 ? 0 : off)));
}
#ifndef CGM_PF_GRAM
#define CGM_PF_GRAM 4  // blocks ahead in the Gram pass of the 16-byte path
#endif
#ifndef CGM_PF_Q
#define CGM_PF_Q 3     // blocks ahead in the second pass over H (q = H v)
#endif
constexpr int PF_GRAM = CGM_PF_GRAM;
constexpr int PF_Q = CGM_PF_Q;

// q = H v n-tile nb (antennas 8 nb + g): the lane's H entries of users
// 16 m + 4t..4t+3 for each m-tile m (two 16-byte loads each; 8 users: one
// load of users 2t, 2t+1).
template <int UT>
__device__ __forceinline__ void q_load(const float2* H, int B, int nb, int g, int t,
                                       float4 (&f)[WarpCfg<UT>::MT][2]) {
  constexpr int MT = WarpCfg<UT>::MT;
  const int b = 8 * nb + g;
  const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
  for (int m = 0; m < MT; ++m) {
    if (b < B) {
      f[m][0] = ldg4(H + b * UT + 16 * m + (UT == 8 ? 2 : 4) * t);
      f[m][1] = UT == 8 ? zero4 : ldg4(H + b * UT + 16 * m + 4 * t + 2);
    } else {
      f[m][0] = f[m][1] = zero4;
    }
  }
}

// Compensated butterfly over the four lanes of a quad (lane bits 0 and 1)
// for two independent sums.
__device__ __forceinline__ void quad_sum2(float& x0, float& x1) {
  float s0 = x0, s1 = x1, c0 = 0.f, c1 = 0.f;
#pragma unroll
  for (int off = 1; off < 4; off <<= 1) {
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

__device__ __forceinline__ float warp_max(float x) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) x = fmaxf(x, __shfl_xor_sync(0xffffffffu, x, off));
  return x;
}
__device__ __forceinline__ float quad_max(float x) {
  x = fmaxf(x, __shfl_xor_sync(0xffffffffu, x, 1));
  return fmaxf(x, __shfl_xor_sync(0xffffffffu, x, 2));
}

// ---------------------------------------------------------------------------
// Exact power-of-two scaling of an instance
// ---------------------------------------------------------------------------
//
// A split (hi + lo) FP16 operand keeps about 22 significant bits only while
// |x| lies between about 2^-3 (below it the lo part is subnormal) and 65504
// (above it hi overflows); BF16 has FP32's exponent range. Eq. 2 and
// Algorithm 1 are invariant under exact power-of-two scaling: with
// H' = 2^-e H, y' = 2^-f y, sigma' = 2^-2e sigma and N0' = 2^-2e N0, CG gives
// v' = 2^(e-f) v (alpha' = 2^2e alpha, beta' = beta, the same breakdowns),
// the trackers of Eqs. 10-13 give the same mu and rho, and CG-P with
// t' = 2^-f t gives q' = 2^(e-f) q. So every instance is brought into the
// FP16 range by one scale for H and one per right-hand side, and x_hat and
// q are scaled back when they are stored.
//
// Fast path: e comes from the largest entry of H's first k-step, which the
// loads deliver before the Gram's first product, and Y takes the same scale
// (f = e, so x_hat needs none); T, read whole before CG-P starts, gets its
// own per row. Inputs already in range (channels of roughly unit power)
// keep scale 1 and run the unscaled code. Before CG starts, the largest
// diagonal entry of the scaled Gram and ||b||^2 of every right-hand side
// are checked against the range the FP16 split needs; an instance that
// fails (a first k-step unlike the rest, or receive vectors on a scale of
// their own) is formed again on a slow path with scales taken from every
// entry (full_scale), with f per row. A = G + sigma I gets a scale of its
// own in setup_a.

// Exact 2^e for |e| <= 126.
__device__ __forceinline__ float pow2f(int e) { return __int_as_float((e + 127) << 23); }
// 2^e with e clamped to the normal range.
__device__ __forceinline__ float pow2c(int e) { return pow2f(e < -126 ? -126 : e > 126 ? 126 : e); }

// The scales of a lane, packed in one word: e (H' = 2^-e H) in bits 0-7,
// f of rows g and g + 8 (2^-f) in bits 8-15 and 16-23, each in [-100, 100],
// and in bit 24 whether any lane of the warp has a scale other than 1.
struct InstScale {
  int w;
  __device__ __forceinline__ int e() const { return (w << 24) >> 24; }
  __device__ __forceinline__ int f(int h) const { return h ? (w << 8) >> 24 : (w << 16) >> 24; }
  __device__ __forceinline__ bool any() const { return (w >> 24) & 1; }
  // 2^-2e, the factor of sigma and N0 (1 when no lane is scaled).
  __device__ __forceinline__ float s2() const { return any() ? pow2c(-2 * e()) : 1.f; }
  // 2^(f - e): x_hat of row g (h = 0) or g + 8 (h = 1) from the scaled CG.
  __device__ __forceinline__ float xs(int h) const { return pow2c(f(h) - e()); }
  // Packs e, f0, f1 (warp-collective: sets the any bit).
  __device__ __forceinline__ static InstScale make(int e, int f0, int f1) {
    InstScale s;
    s.w = (e & 255) | ((f0 & 255) << 8) | ((f1 & 255) << 16);
    if (__any_sync(0xffffffffu, s.w != 0)) s.w |= 1 << 24;
    return s;
  }
};

// floor(log2 m) for normal m > 0.
__device__ __forceinline__ int exp2_floor(float m) { return ((__float_as_int(m) >> 23) & 0xff) - 127; }

// 0 when lo <= m <= hi (or m is 0 or not finite: nothing to go by), else
// the e that puts m 2^-e in [2^t, 2^(t+1)).
__device__ __forceinline__ int band_exp(float m, float lo, float hi, int t) {
  if ((m >= lo && m <= hi) || !(m > 0.f) || !(m <= 3.0e38f)) return 0;
  const int e = exp2_floor(m) - t;
  return e < -100 ? -100 : e > 100 ? 100 : e;
}

// Range of the largest component in H's first k-step that runs unscaled,
// [1/2, 8], and where a scaled one is put, [2, 4); ||t||^2 of a row of T:
// [2^-4, 2^12] and [4, 16) (even exponent offsets, so that the scale of t
// itself is a power of two). CN(0,1) channels and unit-energy symbols fall
// in the first ranges.
constexpr float kHLo = 0.5f, kHHi = 8.f;
constexpr int kHTarget = 1;
constexpr float kTLo = 0.0625f, kTHi = 4096.f;
constexpr int kTTarget = 2;

// Range the fast path needs before CG starts: the largest diagonal entry of
// the scaled Gram G' between 2^-8 B (below, H's entries would be near or
// under FP16's lo-part floor) and 2^26 (above, some entry of H' is near or
// past FP16's largest value), and ||b'||^2 of a right-hand side 0 or
// between 1 and 2^26 (b' starts the CG direction, which goes through the
// FP16 split).
constexpr float kColMsLo = 0.00390625f;
constexpr float kGHi = 67108864.f;
constexpr float kPreColMsHi = 16.f;  // CG-P: G'_ii / B at most this (precode_warp_finish)
constexpr float kRLo = 1.f, kRHi = 67108864.f;

// Fast-path scale from H's first k-step (h as from load_h_ks /
// ring_gram_read): Y takes the same e.
template <int UT>
__device__ __forceinline__ InstScale scale_from_ks(const float2 (&h)[WarpCfg<UT>::MT][4]) {
  constexpr int MT = WarpCfg<UT>::MT;
  float mh = 0.f;
#pragma unroll
  for (int m = 0; m < MT; ++m)
#pragma unroll
    for (int k = 0; k < 4; ++k) mh = fmaxf(mh, fmaxf(fabsf(h[m][k].x), fabsf(h[m][k].y)));
  // the warp's largest entry is in range when every lane's is, or (a lane
  // whose entries are all zero, as past B) its entries are 0
  const bool in = (mh >= kHLo && mh <= kHHi) || mh == 0.f;
  int e = 0;
  if (!__all_sync(0xffffffffu, in)) e = band_exp(warp_max(mh), kHLo, kHHi, kHTarget);
  InstScale sc;
  sc.w = (e & 255) | ((e & 255) << 8) | ((e & 255) << 16) | (e != 0 ? 1 << 24 : 0);
  return sc;
}

// Slow-path scales from every entry: e puts the root mean square of H's
// entries in [1, 2), f that of each right-hand-side row of Y in [1, 2)
// (MF; else f = e). The largest entry of H is then below 2^7.5 and that of a
// row below 2^5. Means are taken after dividing by the largest power of two
// below the largest entry, so that no square overflows or underflows.
__device__ __forceinline__ int rms_exp(const float2* p, int n) {
  const int lane = threadIdx.x & 31;
  float mx = 0.f;
  for (int i = lane; i < n; i += 32) {
    const float2 v = p[i];
    mx = fmaxf(mx, fmaxf(fabsf(v.x), fabsf(v.y)));
  }
  mx = warp_max(mx);
  if (!(mx > 0.f) || !(mx <= 3.0e38f)) return 0;
  const int e0 = exp2_floor(mx);
  const float s0 = pow2c(-e0);
  float s = 0.f;
  for (int i = lane; i < n; i += 32) {
    const float2 v = p[i];
    s = fmaf(v.x * s0, v.x * s0, fmaf(v.y * s0, v.y * s0, s));
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  const int e = e0 + (exp2_floor(s / float(n)) >> 1);
  return e < -100 ? -100 : e > 100 ? 100 : e;
}

// Out of line: it runs only for instances the fast path hands back.
template <bool MF>
__device__ __noinline__ InstScale full_scale(const float2* H, const float2* Y, int B, int U,
                                                int R) {
  const int g = (threadIdx.x & 31) >> 2;
  const int e = rms_exp(H, B * U);
  int f0 = e, f1 = e;
  if constexpr (MF) {
    f0 = f1 = 0;
    for (int r = 0; r < R; ++r) {
      const int f = rms_exp(Y + int64_t(r) * B, B);
      if (r == g) f0 = f;
      if (r == g + 8) f1 = f;
    }
  }
  return InstScale::make(e, f0, f1);
}

// h *= sh, y rows *= sy0 (row g: y[0], y[2]) and sy1 (row g + 8: y[1], y[3]).
// Every k-step goes through it, also at scale 1: one copy of the Gram loop
// runs faster than an unscaled and a scaled one side by side.
template <int UT, bool MF>
__device__ __forceinline__ void apply_scale(float2 (&h)[WarpCfg<UT>::MT][4], float2 (&y)[4],
                                            float sh, float sy0, float sy1) {
#pragma unroll
  for (int m = 0; m < WarpCfg<UT>::MT; ++m)
#pragma unroll
    for (int k = 0; k < 4; ++k) h[m][k] = make_float2(h[m][k].x * sh, h[m][k].y * sh);
  if constexpr (MF) {
    y[0] = make_float2(y[0].x * sy0, y[0].y * sy0);
    y[2] = make_float2(y[2].x * sy0, y[2].y * sy0);
    y[1] = make_float2(y[1].x * sy1, y[1].y * sy1);
    y[3] = make_float2(y[3].x * sy1, y[3].y * sy1);
  }
}

// Status returned by a fast-path finish whose instance must be formed again
// with full_scale (nothing was stored); statuses are >= 0.
constexpr int kRedo = -1;

// ---------------------------------------------------------------------------
// Loads of one k-step (antennas b0 = 8 ks + 2 t and b0 + 1)
// ---------------------------------------------------------------------------

// h[m][0..3]: H(b0, row user 0), H(b0, row user 1), H(b0+1, row user 0),
// H(b0+1, row user 1) of m-tile m; the row users of lane g are 16 m + 2g,
// 16 m + 2g + 1 (16 and 32 users) or g (8 users; row user 1 absent).
// VEC: U == UT, B even, H 16-byte aligned.
template <int UT, bool VEC>
__device__ __forceinline__ void load_h_ks(const float2* __restrict__ H, int B, int U, int ks,
                                          int g, int t, float2 (&h)[WarpCfg<UT>::MT][4]) {
  constexpr int MT = WarpCfg<UT>::MT;
  const int b0 = 8 * ks + 2 * t, b1 = b0 + 1;
  const float2 z = make_float2(0.f, 0.f);
  if constexpr (VEC) {
    const bool ok = b0 < B;
    if constexpr (UT == 8) {
      h[0][0] = ok ? ldg2(H + b0 * 8 + g) : z;
      h[0][2] = ok ? ldg2(H + b1 * 8 + g) : z;
      h[0][1] = h[0][3] = z;
    } else {
      const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int m = 0; m < MT; ++m) {
        const float4 v0 = ok ? ldg4(H + b0 * UT + 16 * m + 2 * g) : zero4;
        const float4 v1 = ok ? ldg4(H + b1 * UT + 16 * m + 2 * g) : zero4;
        h[m][0] = make_float2(v0.x, v0.y);
        h[m][1] = make_float2(v0.z, v0.w);
        h[m][2] = make_float2(v1.x, v1.y);
        h[m][3] = make_float2(v1.z, v1.w);
      }
    }
  } else {
#pragma unroll
    for (int m = 0; m < MT; ++m) {
      const int u0 = UT == 8 ? g : 16 * m + 2 * g, u1 = 16 * m + 2 * g + 1;
      h[m][0] = (b0 < B && u0 < U) ? ldg2(H + b0 * U + u0) : z;
      h[m][2] = (b1 < B && u0 < U) ? ldg2(H + b1 * U + u0) : z;
      if constexpr (UT != 8) {
        h[m][1] = (b0 < B && u1 < U) ? ldg2(H + b0 * U + u1) : z;
        h[m][3] = (b1 < B && u1 < U) ? ldg2(H + b1 * U + u1) : z;
      } else {
        h[m][1] = h[m][3] = z;
      }
    }
  }
}

// y[0..3]: Y(g, b0), Y(g+8, b0), Y(g, b0+1), Y(g+8, b0+1) (rows >= R are 0).
// VEC: B even, Y 16-byte aligned.
template <bool VEC>
__device__ __forceinline__ void load_y_ks(const float2* __restrict__ Y, int B, int R, int ks,
                                          int g, int t, float2 (&y)[4]) {
  const int b0 = 8 * ks + 2 * t, b1 = b0 + 1;
  const float2 z = make_float2(0.f, 0.f);
  if constexpr (VEC) {
    const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
    const bool ok = b0 < B;
    const float4 w0 = (ok && g < R) ? ldg4(Y + g * B + b0) : zero4;
    const float4 w1 = (ok && g + 8 < R) ? ldg4(Y + (g + 8) * B + b0) : zero4;
    y[0] = make_float2(w0.x, w0.y);
    y[2] = make_float2(w0.z, w0.w);
    y[1] = make_float2(w1.x, w1.y);
    y[3] = make_float2(w1.z, w1.w);
  } else {
    y[0] = (g < R && b0 < B) ? ldg2(Y + g * B + b0) : z;
    y[2] = (g < R && b1 < B) ? ldg2(Y + g * B + b1) : z;
    y[1] = (g + 8 < R && b0 < B) ? ldg2(Y + (g + 8) * B + b0) : z;
    y[3] = (g + 8 < R && b1 < B) ? ldg2(Y + (g + 8) * B + b1) : z;
  }
}

// ---------------------------------------------------------------------------
// Gram (and transposed matched filters) of one k-step
// ---------------------------------------------------------------------------

// Gr/Gi[m][nt][d]: G at row position 16 m + 8 (d >> 1) + g, column position
// 8 nt + 2 t + (d & 1). Mr[nt][d] = Re b^T and Mn[nt][d] = -Im b^T at
// right-hand side g + 8 (d >> 1), column position 8 nt + 2 t + (d & 1).
template <int UT, int EL, bool X3, bool MF>
__device__ __forceinline__ void gram_ks(const float2 (&h)[WarpCfg<UT>::MT][4],
                                        const float2 (&y)[4], GramAcc<UT>& Gr, GramAcc<UT>& Gi,
                                        VecAcc<UT>& Mr, VecAcc<UT>& Mn) {
  constexpr int NB = UT / 8, MT = WarpCfg<UT>::MT;
  uint2 hs[MT][4];
#pragma unroll
  for (int m = 0; m < MT; ++m)
#pragma unroll
    for (int k = 0; k < 4; ++k) hs[m][k] = split_c<EL>(h[m][k]);
  uint32_t yh[4], yl[4];
  if constexpr (MF) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const uint2 s = split_c<EL>(y[k]);
      yh[k] = s.x;
      yl[k] = s.y;
    }
  }
#pragma unroll
  for (int nt = 0; nt < NB; ++nt) {
    // B fragments of n-tile nt: the row-user registers of block nt
    // (m-tile nt / 2, row half nt % 2)
    const uint2 b0 = hs[nt >> 1][nt & 1], b1 = hs[nt >> 1][2 + (nt & 1)];
    const uint32_t s0h = swap_neg(b0.x), s1h = swap_neg(b1.x);
    const uint32_t s0l = swap_neg(b0.y), s1l = swap_neg(b1.y);
#pragma unroll
    for (int m = 0; m < MT; ++m) {
      // G is Hermitian: with two m-tiles (32 users) the block of rows 16..31 and
      // columns 0..15 is the conjugate transpose of rows 0..15, columns 16..31,
      // and WarpCg::setup_a takes it from there
      if (MT == 2 && m == 1 && nt < 2) continue;
      const uint32_t ah[4] = {hs[m][0].x, hs[m][1].x, hs[m][2].x, hs[m][3].x};
      const uint32_t al[4] = {hs[m][0].y, hs[m][1].y, hs[m][2].y, hs[m][3].y};
      mma_split<EL, X3>(Gr[m][nt], ah, al, b0.x, b1.x, b0.y, b1.y);
      mma_split<EL, X3>(Gi[m][nt], ah, al, s0h, s1h, s0l, s1l);
    }
    if constexpr (MF) {
      mma_split<EL, X3>(Mr[nt], yh, yl, b0.x, b1.x, b0.y, b1.y);
      mma_split<EL, X3>(Mn[nt], yh, yl, s0h, s1h, s0l, s1l);
    }
  }
}

// ---------------------------------------------------------------------------
// Algorithm 1 in registers
// ---------------------------------------------------------------------------

// CG state of one warp: entry [h][nt][c] is right-hand side g + 8 h at
// position 8 nt + 2 t + c. The B fragments of A (hi|lo, and times i when
// WarpCfg::STORE_IM) live in this warp's shared-memory slice, one uint2 per
// lane and fragment.
template <int UT, int EL>
struct WarpCg {
  static constexpr int NB = UT / 8;
  static constexpr bool STORE_IM = WarpCfg<UT>::STORE_IM;
  float2 v[2][NB][2], res[2][NB][2], p[2][NB][2];
  float D[NB][2];
  float rrn[2];
  bool active[2], broke[2];
  int kd[2];      // iterations completed per row
  float es = 1.f;  // factor of the products with the fragments (setup_a)

  // Fragment index of (ks, nt, b, part) in the shared slice.
  __device__ __forceinline__ static int fidx(int ks, int nt, int b, int part) {
    return STORE_IM ? ((ks * NB + nt) * 2 + b) * 2 + part : (ks * NB + nt) * 2 + b;
  }

  // Writes A = G + sigma I as B fragments (from the Gram accumulators) and
  // returns D = diag(A) and G_ii at the lane's positions. Row 8 nt + g of
  // the Gram is row half nt % 2 of m-tile nt / 2. The fragments hold
  // 2^-a A, with a = 0 unless the largest diagonal entry (which bounds every
  // entry of the positive definite A) lies outside [2^-2, 2^13]; the return
  // value is 2^a, the factor that products with the fragments need. gmax
  // gets the largest diagonal entry of G (warp-uniform).
  __device__ __forceinline__ static float setup_a(const GramAcc<UT>& Gr, const GramAcc<UT>& Gi,
                                                  float sigma, uint2* frag, float (&Dout)[NB][2],
                                                  float (&Gd)[NB][2], float& gmax) {
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    float mg = 0.f;
#pragma unroll
    for (int nt = 0; nt < NB; ++nt)
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const float gd = __shfl_sync(0xffffffffu, Gr[nt >> 1][nt][2 * (nt & 1) + c],
                                     4 * (2 * t + c) + t);
        Gd[nt][c] = gd;
        Dout[nt][c] = gd + sigma;
        mg = fmaxf(mg, gd);
      }
    gmax = quad_max(mg);
    const int a = band_exp(gmax + sigma, 0.25f, 8192.f, 10);
    const float sa = pow2f(-a);
#pragma unroll
    for (int ks = 0; ks < NB; ++ks)
#pragma unroll
      for (int nt = 0; nt < NB; ++nt)
#pragma unroll
        for (int b = 0; b < 2; ++b) {
          // A[8 ks + 2 t + b][8 nt + g] = conj(G[8 nt + g][8 ks + 2 t + b]) (+ sigma)
          const int m = nt >> 1, d = 2 * (nt & 1) + b;
          const bool diag = (ks == nt) && (g == 2 * t + b);
          float re, im;
          if (UT == 32 && m == 1 && ks < 2) {
            // block not accumulated (gram_ks): A[i][j] = G[i][j] with i = 8 ks + 2 t + b
            // in m-tile 0, held by lane 4 (2 t + b) + g / 2 at register 2 ks + g % 2
            const int src = 4 * (2 * t + b) + (g >> 1);
            const float r0 = __shfl_sync(0xffffffffu, Gr[0][nt][2 * ks], src);
            const float r1 = __shfl_sync(0xffffffffu, Gr[0][nt][2 * ks + 1], src);
            const float i0 = __shfl_sync(0xffffffffu, Gi[0][nt][2 * ks], src);
            const float i1 = __shfl_sync(0xffffffffu, Gi[0][nt][2 * ks + 1], src);
            re = (g & 1) ? r1 : r0;
            im = (g & 1) ? i1 : i0;
          } else {
            re = Gr[m][ks][d] + (diag ? sigma : 0.f);
            im = diag ? 0.f : -Gi[m][ks][d];
          }
          re *= sa;
          im *= sa;
          frag[fidx(ks, nt, b, 0) * 32 + lane] = split_c<EL>(make_float2(re, im));
          if constexpr (STORE_IM)
            frag[fidx(ks, nt, b, 1) * 32 + lane] = split_c<EL>(make_float2(-im, re));
        }
    return pow2f(a);
  }

  // matvec, times the fragments' factor es when it is not 1.
  __device__ __forceinline__ void matvec_s(const uint2* frag, float es, float (&Er)[NB][4],
                                           float (&Ei)[NB][4]) const {
    matvec(frag, Er, Ei);
    if (es != 1.f) {
#pragma unroll
      for (int nt = 0; nt < NB; ++nt)
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          Er[nt][k] *= es;
          Ei[nt][k] *= es;
        }
    }
  }

  // One fragment of A from shared memory. With VOL the fragments are read at
  // every product as volatile loads, so that the compiler does not hoist all
  // of them (64 registers per lane at 32 users) out of the CG and tracker
  // loops into registers that are needed for the vectors.
  template <bool VOL>
  __device__ __forceinline__ static uint2 lds_frag(const uint2* q) {
    if constexpr (VOL) {
      uint2 v;
      asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "r"(smem_addr(q)));
      return v;
    } else {
      return *q;
    }
  }

  // e = A p for every right-hand side row: E[nt][d] in accumulator layout.
  template <bool VOL = (UT == 32)>
  __device__ __forceinline__ void matvec(const uint2* frag, float (&Er)[NB][4],
                                         float (&Ei)[NB][4]) const {
    const int lane = threadIdx.x & 31;
    uint32_t ph[NB][4], pl[NB][4];
#pragma unroll
    for (int ks = 0; ks < NB; ++ks) {
      const uint2 s0 = split_c<EL>(p[0][ks][0]);  // row g, q = t
      const uint2 s1 = split_c<EL>(p[1][ks][0]);  // row g + 8, q = t
      const uint2 s2 = split_c<EL>(p[0][ks][1]);  // row g, q = t + 4
      const uint2 s3 = split_c<EL>(p[1][ks][1]);  // row g + 8, q = t + 4
      ph[ks][0] = s0.x; pl[ks][0] = s0.y;
      ph[ks][1] = s1.x; pl[ks][1] = s1.y;
      ph[ks][2] = s2.x; pl[ks][2] = s2.y;
      ph[ks][3] = s3.x; pl[ks][3] = s3.y;
    }
#pragma unroll
    for (int nt = 0; nt < NB; ++nt) {
      float rh[4] = {0.f, 0.f, 0.f, 0.f}, rx[4] = {0.f, 0.f, 0.f, 0.f};
      float ih[4] = {0.f, 0.f, 0.f, 0.f}, ix[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int ks = 0; ks < NB; ++ks) {
        const uint2 r0 = lds_frag<VOL>(frag + fidx(ks, nt, 0, 0) * 32 + lane);
        const uint2 r1 = lds_frag<VOL>(frag + fidx(ks, nt, 1, 0) * 32 + lane);
        uint2 i0, i1;
        if constexpr (STORE_IM) {
          i0 = lds_frag<VOL>(frag + fidx(ks, nt, 0, 1) * 32 + lane);
          i1 = lds_frag<VOL>(frag + fidx(ks, nt, 1, 1) * 32 + lane);
        } else {  // i (re, im) = (-im, re): swap the halves, negate the new low one
          i0 = make_uint2(swap_halves(r0.x) ^ 0x8000u, swap_halves(r0.y) ^ 0x8000u);
          i1 = make_uint2(swap_halves(r1.x) ^ 0x8000u, swap_halves(r1.y) ^ 0x8000u);
        }
        mma16816<EL>(rh, ph[ks], r0.x, r1.x);
        mma16816<EL>(ih, ph[ks], i0.x, i1.x);
        mma16816<EL>(rx, ph[ks], r0.y, r1.y);
        mma16816<EL>(ix, ph[ks], i0.y, i1.y);
        mma16816<EL>(rx, pl[ks], r0.x, r1.x);
        mma16816<EL>(ix, pl[ks], i0.x, i1.x);
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        Er[nt][k] = rh[k] + rx[k];
        Ei[nt][k] = ih[k] + ix[k];
      }
    }
  }

  // The CG iterations of Algorithm 1. res holds b on entry; rows >= R are
  // inactive from the start. With TRACK, alpha_k and beta_k of every row are
  // kept in sAB[(k - 1) * 16 + row] for the tracker (tracker_l below).
  // Initialisation: v = 0, p = r = b (res holds b), ||r||^2 of every row.
  __device__ __forceinline__ void init() {
    float s[2] = {0.f, 0.f};
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
      for (int nt = 0; nt < NB; ++nt)
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          v[h][nt][c] = make_float2(0.f, 0.f);
          p[h][nt][c] = res[h][nt][c];
          s[h] = fmaf(res[h][nt][c].x, res[h][nt][c].x,
                      fmaf(res[h][nt][c].y, res[h][nt][c].y, s[h]));
        }
    quad_sum2(s[0], s[1]);
    rrn[0] = s[0];
    rrn[1] = s[1];
  }

  // The CG iterations after init().
  template <bool TRACK>
  __device__ __forceinline__ void run(const uint2* frag, float2* sAB, int R, int K) {
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      active[h] = (g + 8 * h) < R;
      broke[h] = false;
      kd[h] = 0;
    }
    for (int k = 1; k <= K; ++k) {
#pragma unroll
      for (int h = 0; h < 2; ++h)
        if (active[h] && !(rrn[h] > 0.f)) {
          active[h] = false;
          broke[h] = true;
        }
      if (!__any_sync(0xffffffffu, active[0] || active[1])) break;
      float Er[NB][4], Ei[NB][4];
      matvec(frag, Er, Ei);
      float pe[2] = {0.f, 0.f};
#pragma unroll
      for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int nt = 0; nt < NB; ++nt)
#pragma unroll
          for (int c = 0; c < 2; ++c) {
            const float2 pp = p[h][nt][c];
            pe[h] = fmaf(pp.x, Er[nt][2 * h + c], fmaf(pp.y, Ei[nt][2 * h + c], pe[h]));
          }
      quad_sum2(pe[0], pe[1]);
      float alpha[2], rrnew[2] = {0.f, 0.f};
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        if (active[h] && !(pe[h] > 0.f)) {
          active[h] = false;
          broke[h] = true;
        }
        // the product came out as 2^-a A p (es = 2^a): alpha = r^H r / (es p^H E)
        alpha[h] = active[h] ? __fdividef(rrn[h], pe[h] * es) : 0.f;
        const float ae = alpha[h] * es;
#pragma unroll
        for (int nt = 0; nt < NB; ++nt)
#pragma unroll
          for (int c = 0; c < 2; ++c) {
            if (active[h]) {
              v[h][nt][c].x = fmaf(alpha[h], p[h][nt][c].x, v[h][nt][c].x);
              v[h][nt][c].y = fmaf(alpha[h], p[h][nt][c].y, v[h][nt][c].y);
              res[h][nt][c].x = fmaf(-ae, Er[nt][2 * h + c], res[h][nt][c].x);
              res[h][nt][c].y = fmaf(-ae, Ei[nt][2 * h + c], res[h][nt][c].y);
            }
            rrnew[h] = fmaf(res[h][nt][c].x, res[h][nt][c].x,
                            fmaf(res[h][nt][c].y, res[h][nt][c].y, rrnew[h]));
          }
      }
      quad_sum2(rrnew[0], rrnew[1]);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        if (!active[h]) continue;
        const float beta = __fdividef(rrnew[h], rrn[h]);
#pragma unroll
        for (int nt = 0; nt < NB; ++nt)
#pragma unroll
          for (int c = 0; c < 2; ++c) {
            p[h][nt][c].x = fmaf(beta, p[h][nt][c].x, res[h][nt][c].x);
            p[h][nt][c].y = fmaf(beta, p[h][nt][c].y, res[h][nt][c].y);
          }
        if (TRACK && t == 0) sAB[(k - 1) * 16 + g + 8 * h] = make_float2(alpha[h], beta);
        rrn[h] = rrnew[h];
        kd[h] = k;
      }
    }
  }

  // Sec. III-F: the K-term Neumann series x = sum_{k<K} (-D^-1 E)^k D^-1 b
  // with A = D + E, D = diag(A), evaluated as its partial sums
  //   S_1 = D^-1 b,  S_{k+1} = S_k + D^-1 (b - A S_k)
  // (S_{k+1} = D^-1 b - D^-1 E S_k). res holds b on entry; v gets S_K. Rows
  // with a zero b (rows >= R) stay zero.
  __device__ __forceinline__ void neumann(const uint2* frag, int K) {
    float id[NB][2];
#pragma unroll
    for (int nt = 0; nt < NB; ++nt)
#pragma unroll
      for (int c = 0; c < 2; ++c) id[nt][c] = 1.f / D[nt][c];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      broke[h] = false;
#pragma unroll
      for (int nt = 0; nt < NB; ++nt)
#pragma unroll
        for (int c = 0; c < 2; ++c)
          v[h][nt][c] = make_float2(res[h][nt][c].x * id[nt][c], res[h][nt][c].y * id[nt][c]);
    }
    for (int k = 2; k <= K; ++k) {
#pragma unroll
      for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int nt = 0; nt < NB; ++nt)
#pragma unroll
          for (int c = 0; c < 2; ++c) p[h][nt][c] = v[h][nt][c];
      float Er[NB][4], Ei[NB][4];
      matvec_s(frag, es, Er, Ei);
#pragma unroll
      for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int nt = 0; nt < NB; ++nt)
#pragma unroll
          for (int c = 0; c < 2; ++c) {
            v[h][nt][c].x = fmaf(res[h][nt][c].x - Er[nt][2 * h + c], id[nt][c], v[h][nt][c].x);
            v[h][nt][c].y = fmaf(res[h][nt][c].y - Ei[nt][2 * h + c], id[nt][c], v[h][nt][c].y);
          }
    }
  }

  // Eq. 10 for right-hand side `row` (alpha_k, beta_k in sAB, kdone
  // iterations), then B = L_K G, C = L_K G L_K^H and, for the lane's matrix
  // rows 16 m + g + 8 hh (the users at those positions),
  //   mu = Re B_ii,  nu^2 = Es sum_{j != i} |B_ij|^2 + N0 C_ii,  rho = mu^2 / nu^2.
  // L_k is a polynomial in A with real coefficients, so it commutes with A
  // and A (L_{k-1} - L_{k-2}) = (L_{k-1} - L_{k-2}) A: 16 rows of the
  // difference pass through matvec exactly like 16 right-hand sides, and
  // every product of the recursion runs on the tensor cores. Each row of the
  // recursion depends on the same row only, so 32 users run it as two
  // halves of 16 rows (m = 0, 1). Rows and columns are in position order;
  // p is overwritten.
  //
  // The recursion is carried as L and the differences D1 = L_{k-1} - L_{k-2},
  // D2 = L_{k-2} - L_{k-3}: D_k = c1 D1 - alpha_k D1 A - c2 D2, L_k = L_{k-1} + D_k.
  // The L_k are of the order of alpha_1 (L_1 = alpha_1 I), so they are held
  // as 2^-s L (2^s <= alpha_1 < 2^(s+1)), which is also what enters the FP16
  // split; D1 lives in p, the operand of the product. With Ls (one 16-row
  // block of L, 32 entries per lane) L lives in shared memory, which leaves
  // the registers to D1, D2 and the product.
  __device__ __forceinline__ void exact_sinr(const uint2* frag, const float2* sAB, int row,
                                             int kdone, float sigma, float N0, float Es, int m,
                                             float2* Ls, float (&mu)[2], float (&rho)[2]) {
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    float2 Lr[2][NB][2], D2[2][NB][2];
    const float a1 = sAB[row].x;
    const int sl = (a1 > 0.f && a1 <= 3.0e38f) ? exp2_floor(a1) : 0;
    const float a1s = a1 * pow2c(-sl);  // alpha_1 2^-s, in [1, 2)
    auto lidx = [&](int h, int nt, int c) { return ((h * NB + nt) * 2 + c) * 32 + lane; };
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
      for (int nt = 0; nt < NB; ++nt)
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          const bool diag = 8 * nt + 2 * t + c == 16 * m + 8 * h + g;
          const float2 l1 = make_float2(diag ? a1s : 0.f, 0.f);  // 2^-s L_1
          p[h][nt][c] = l1;                                     // 2^-s (L_1 - L_0)
          D2[h][nt][c] = make_float2(0.f, 0.f);
          if (Ls) Ls[lidx(h, nt, c)] = l1; else Lr[h][nt][c] = l1;
        }
    for (int k = 2; k <= kdone; ++k) {
      const float2 abk = sAB[(k - 1) * 16 + row], ab1 = sAB[(k - 2) * 16 + row];
      const float2 ab2 = k >= 3 ? sAB[(k - 3) * 16 + row] : make_float2(1.f, 0.f);
      const float ak = abk.x;
      const float c1 = ak * (1.f + ab1.y) / ab1.x;
      const float c2 = ak * ab2.y / ab2.x;
      const float ake = ak * es;
      float Er[NB][4], Ei[NB][4];
      matvec<true>(frag, Er, Ei);  // 2^-s D1 2^-a A
#pragma unroll
      for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int nt = 0; nt < NB; ++nt)
#pragma unroll
          for (int c = 0; c < 2; ++c) {
            const float2 d1 = p[h][nt][c], d2 = D2[h][nt][c];
            float2 dn;
            dn.x = c1 * d1.x - ake * Er[nt][2 * h + c] - c2 * d2.x;
            dn.y = c1 * d1.y - ake * Ei[nt][2 * h + c] - c2 * d2.y;
            D2[h][nt][c] = d1;
            p[h][nt][c] = dn;
            if (Ls) {
              const float2 l = Ls[lidx(h, nt, c)];
              Ls[lidx(h, nt, c)] = make_float2(l.x + dn.x, l.y + dn.y);
            } else {
              Lr[h][nt][c] = make_float2(Lr[h][nt][c].x + dn.x, Lr[h][nt][c].y + dn.y);
            }
          }
    }
    // 2^-s B = 2^-s L_K A - sigma 2^-s L_K
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
      for (int nt = 0; nt < NB; ++nt)
#pragma unroll
        for (int c = 0; c < 2; ++c) p[h][nt][c] = Ls ? Ls[lidx(h, nt, c)] : Lr[h][nt][c];
    float Er[NB][4], Ei[NB][4];
    matvec<true>(frag, Er, Ei);
    float dg[2] = {0.f, 0.f}, itf[2] = {0.f, 0.f}, cc[2] = {0.f, 0.f};
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
      for (int nt = 0; nt < NB; ++nt)
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          const float2 l = p[h][nt][c];
          const float bx = fmaf(-sigma, l.x, Er[nt][2 * h + c] * es);
          const float by = fmaf(-sigma, l.y, Ei[nt][2 * h + c] * es);
          const bool diag = 8 * nt + 2 * t + c == 16 * m + 8 * h + g;
          if (diag)
            dg[h] += bx;
          else
            itf[h] = fmaf(bx, bx, fmaf(by, by, itf[h]));
          cc[h] = fmaf(bx, l.x, fmaf(by, l.y, cc[h]));  // Re(B_ij conj(L_ij))
        }
    quad_sum2(dg[0], dg[1]);
    quad_sum2(itf[0], itf[1]);
    quad_sum2(cc[0], cc[1]);
    const float s1 = pow2c(sl), s2 = s1 * s1;  // undo 2^-s (B, L) and 2^-2s (products)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      mu[h] = dg[h] * s1;
      const float nu2 = fmaf(Es, itf[h], N0 * cc[h]) * s2;
      rho[h] = nu2 > 0.f ? mu[h] * mu[h] / nu2 : 0.f;
    }
  }

  // Eq. 11 with A replaced by D (scalar per position) from the recorded
  // alpha_k, beta_k: l_1 = alpha_1, and for k >= 2
  //   l_k = l_{k-1} + (alpha_k (1 + beta_{k-1}) / alpha_{k-1} - alpha_k D)(l_{k-1} - l_{k-2})
  //         - alpha_k beta_{k-2} / alpha_{k-2} (l_{k-2} - l_{k-3}),
  // with alpha = 1, beta = 0, l = 0 before the first iteration. Returns
  // l_{kd} of row h at the lane's positions (0 when no iteration completed).
  __device__ __forceinline__ void tracker_l(const float2* sAB, int h, float (&l)[NB][2]) const {
    const int g = (threadIdx.x & 31) >> 2;
    const int row = g + 8 * h;
    float l1[NB][2], l2[NB][2], l3[NB][2];
#pragma unroll
    for (int nt = 0; nt < NB; ++nt)
#pragma unroll
      for (int c = 0; c < 2; ++c) l1[nt][c] = l2[nt][c] = l3[nt][c] = 0.f;
    float ia1 = 1.f, ia2 = 1.f, be1 = 0.f, be2 = 0.f;
    for (int k = 1; k <= kd[h]; ++k) {
      const float2 ab = sAB[(k - 1) * 16 + row];
      const float al = ab.x;
      const float c1 = al * (1.f + be1) * ia1;
      const float c2 = al * be2 * ia2;
#pragma unroll
      for (int nt = 0; nt < NB; ++nt)
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          const float lk = (k == 1) ? al
                                    : l1[nt][c] + (c1 - al * D[nt][c]) * (l1[nt][c] - l2[nt][c]) -
                                          c2 * (l2[nt][c] - l3[nt][c]);
          l3[nt][c] = l2[nt][c];
          l2[nt][c] = l1[nt][c];
          l1[nt][c] = lk;
        }
      ia2 = ia1;
      ia1 = __fdividef(1.f, al);
      be2 = be1;
      be1 = ab.y;
    }
#pragma unroll
    for (int nt = 0; nt < NB; ++nt)
#pragma unroll
      for (int c = 0; c < 2; ++c) l[nt][c] = l1[nt][c];
  }
};

// ---------------------------------------------------------------------------
// Work sources at warp granularity
// ---------------------------------------------------------------------------

// Lane 0 claims, every lane gets the unit (-1: none).
__device__ __forceinline__ int64_t warp_claim(const BatchArgs& b) {
  int64_t w = -1;
  if ((threadIdx.x & 31) == 0) {
    const unsigned long long u = atomicAdd(b.counter, 1ull);
    w = u < static_cast<unsigned long long>(b.n_work) ? static_cast<int64_t>(u) : -1;
  }
  return __shfl_sync(0xffffffffu, w, 0);
}


template <class S>
__device__ __forceinline__ int64_t warp_first(const S& s, int64_t gw) {
  if constexpr (SrcTraits<S>::kDyn) {
    return warp_claim(s);
  } else {
    return gw < src_count(s) ? gw : -1;
  }
}


__device__ __forceinline__ bool al16(const void* p) {
  return (reinterpret_cast<uintptr_t>(p) & 15u) == 0;
}

// ---------------------------------------------------------------------------
// Stores of one lane's detection outputs
// ---------------------------------------------------------------------------

// Max-log LLRs of Eq. 4 on one axis of square Gray QAM, from u = x / c.
// With the levels a_j = k_j c, k_j = 2j - (L - 1), the squared distance is
// c^2 (u^2 + k_j^2 - 2 k_j u); u^2 cancels in the difference of the two
// minima, so only f_j = k_j^2 - 2 k_j u is formed (one FMA per level). Gray
// bit m (counted from the least significant) is constant on aligned blocks
// of 2^m levels and alternates over blocks as (i & 1) ^ (i >> 1 & 1), so its
// two minima are taken over block minima built level by level.
// out[t] (bit t, most significant first) = scale (min_0 f - min_1 f).
template <int H>
__device__ __forceinline__ void axis_llr_gray(float u, float scale, float (&out)[H]) {
  constexpr int L = 1 << H;
  float lvl[L];
#pragma unroll
  for (int j = 0; j < L; ++j) {
    const float k = float(2 * j - (L - 1));
    lvl[j] = fmaf(-2.f * k, u, k * k);
  }
#pragma unroll
  for (int m = 0; m < H; ++m) {
    const int nb = L >> m;
    float m0 = INFINITY, m1 = INFINITY;
#pragma unroll
    for (int i = 0; i < nb; ++i) {
      if (((i & 1) ^ ((i >> 1) & 1)) != 0)
        m1 = fminf(m1, lvl[i]);
      else
        m0 = fminf(m0, lvl[i]);
    }
    out[H - 1 - m] = scale * (m0 - m1);
    if (m + 1 < H) {
#pragma unroll
      for (int i = 0; i < nb / 2; ++i) lvl[i] = fminf(lvl[2 * i], lvl[2 * i + 1]);
    }
  }
}

// x_hat, mu, rho and the max-log LLRs (Eq. 4) of NUG users u0 .. u0 + NUG - 1
// of right-hand-side row r (users past U skipped unless VEC: contiguous
// users, 16-byte aligned rows).
template <int NUG, int QB, bool VEC>
__device__ __forceinline__ void store_users_detect(const DetItem& it, int r, int u0,
                                                   const float2 (&xo)[NUG], const float (&mo)[NUG],
                                                   const float (&ro)[NUG], float cq, int* flags) {
  constexpr int H = QB / 2;
  const int64_t base = int64_t(r) * it.U + u0;
  if constexpr (VEC) {
    if (it.xhat) {
      float4* xp = reinterpret_cast<float4*>(it.xhat + base);
#pragma unroll
      for (int m = 0; m < NUG; m += 2)
        xp[m / 2] = make_float4(xo[m].x, xo[m].y, xo[m + 1].x, xo[m + 1].y);
    }
    if constexpr (NUG == 4) {
      if (it.mu)
        *reinterpret_cast<float4*>(it.mu + base) = make_float4(mo[0], mo[1], mo[2], mo[3]);
      if (it.rho)
        *reinterpret_cast<float4*>(it.rho + base) = make_float4(ro[0], ro[1], ro[2], ro[3]);
    } else {
      if (it.mu) *reinterpret_cast<float2*>(it.mu + base) = make_float2(mo[0], mo[1]);
      if (it.rho) *reinterpret_cast<float2*>(it.rho + base) = make_float2(ro[0], ro[1]);
    }
  }
#pragma unroll
  for (int m = 0; m < NUG; ++m) {
    const bool in = VEC || u0 + m < it.U;
    if (!in) continue;
    const bool valid = mo[m] > 0.f;
    if (!valid) *flags |= ST_MU_NONPOS;
    const int64_t o = base + m;
    if constexpr (!VEC) {
      if (it.xhat) it.xhat[o] = xo[m];
      if (it.mu) it.mu[o] = mo[m];
      if (it.rho) it.rho[o] = ro[m];
    }
    if (it.llr) {
      float lI[H], lQ[H];
      if (valid) {
        const float inv = __frcp_rn(mo[m] * cq);  // u = x_hat / (mu c)
        const float scale = ro[m] * cq * cq;
        axis_llr_gray<H>(xo[m].x * inv, scale, lI);
        axis_llr_gray<H>(xo[m].y * inv, scale, lQ);
      } else {
#pragma unroll
        for (int k = 0; k < H; ++k) lI[k] = lQ[k] = 0.f;
      }
      float2* lp = reinterpret_cast<float2*>(it.llr + o * QB);
#pragma unroll
      for (int k = 0; k < H; ++k) {
        const float a = 2 * k < H ? lI[2 * k] : lQ[2 * k - H];
        const float b = 2 * k + 1 < H ? lI[2 * k + 1] : lQ[2 * k + 1 - H];
        lp[k] = make_float2(a, b);
      }
    }
  }
}

// The 2 NB users of a lane in one right-hand-side row, in memory order
// (16 users: 4t + m holds position (nt, c) = (m & 1, m >> 1); 8 users:
// 2t + m holds (0, m)). VEC: contiguous users, 16-byte aligned rows.
template <int UT, int QB, bool VEC>
__device__ __forceinline__ void store_row_detect(const DetItem& it, int r, int t,
                                                 const float2 (&x)[UT / 8][2],
                                                 const float (&mu)[UT / 8][2],
                                                 const float (&rho)[UT / 8][2], float cq,
                                                 int* flags) {
  constexpr int MT = WarpCfg<UT>::MT, NUG = UT == 8 ? 2 : 4;
#pragma unroll
  for (int gr = 0; gr < MT; ++gr) {
    // users 16 gr + 4t + m (m = 2c + nt % 2, nt = 2 gr + m % 2), or 2t + m
    const int u0 = UT == 8 ? 2 * t : 16 * gr + 4 * t;
    float2 xo[NUG];
    float mo[NUG], ro[NUG];
#pragma unroll
    for (int m = 0; m < NUG; ++m) {
      const int nt = UT == 8 ? 0 : 2 * gr + (m & 1), c = UT == 8 ? m : (m >> 1);
      xo[m] = x[nt][c];
      mo[m] = mu[nt][c];
      ro[m] = rho[nt][c];
    }
    store_users_detect<NUG, QB, VEC>(it, r, u0, xo, mo, ro, cq, flags);
  }
}

// ---------------------------------------------------------------------------
// CG-D, one warp per instance
// ---------------------------------------------------------------------------

// Loading scheme of a Gram: the warp's cp.async ring (its prologue already
// issued, STAGES - 1 k-steps ahead), 16-byte register loads one k-step
// ahead (through L1), or predicated element loads for any layout.
enum : int { LD_RING = 0, LD_VEC = 1, LD_ELEM = 2 };

// k-steps 0..KS-1 through the ring; (h, y) already hold k-step 0.
template <int UT, int EL, bool X3, bool MF>
__device__ __forceinline__ void gram_ring_loop(const float2* H, const float2* Y, int B, int R,
                                               int KS, unsigned char* ring,
                                               float2 (&h)[WarpCfg<UT>::MT][4], float2 (&y)[4],
                                               float sh, float sy0, float sy1, GramAcc<UT>& Gr,
                                               GramAcc<UT>& Gi, VecAcc<UT>& Mr, VecAcc<UT>& Mn) {
  for (int ks = 0;;) {
    apply_scale<UT, MF>(h, y, sh, sy0, sy1);
    gram_ks<UT, EL, X3, MF>(h, y, Gr, Gi, Mr, Mn);
    if (++ks >= KS) break;
    ring_gram_issue<UT, MF>(ring, H, Y, B, R, KS, ks + WarpCfg<UT>::STAGES - 1);
    cp_wait<WarpCfg<UT>::STAGES - 1>();
    ring_gram_read<UT, MF>(ring, ks, h, y);
  }
}

// k-steps 0..KS-1 with register loads one k-step ahead (ping-pong); (ha, ya)
// already hold k-step 0.
template <int UT, int EL, bool X3, bool V, bool MF>
__device__ __forceinline__ void gram_direct_loop(const float2* H, const float2* Y, int B, int U,
                                                 int R, int KS, float2 (&ha)[WarpCfg<UT>::MT][4],
                                                 float2 (&ya)[4], float sh, float sy0, float sy1,
                                                 GramAcc<UT>& Gr, GramAcc<UT>& Gi,
                                                 VecAcc<UT>& Mr, VecAcc<UT>& Mn) {
  constexpr int MT = WarpCfg<UT>::MT;
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  float2 hb[MT][4], yb[4] = {};
  for (int ks = 0; ks < KS; ks += 2) {
    if constexpr (V) {
      prefetch_h_block<UT>(H, B, ks + 1 + PF_GRAM);
      prefetch_h_block<UT>(H, B, ks + 2 + PF_GRAM);
    }
    if (ks + 1 < KS) {
      load_h_ks<UT, V>(H, B, U, ks + 1, g, t, hb);
      if constexpr (MF) load_y_ks<V>(Y, B, R, ks + 1, g, t, yb);
    }
    apply_scale<UT, MF>(ha, ya, sh, sy0, sy1);
    gram_ks<UT, EL, X3, MF>(ha, ya, Gr, Gi, Mr, Mn);
    if (ks + 1 >= KS) break;
    if (ks + 2 < KS) {
      load_h_ks<UT, V>(H, B, U, ks + 2, g, t, ha);
      if constexpr (MF) load_y_ks<V>(Y, B, R, ks + 2, g, t, ya);
    }
    apply_scale<UT, MF>(hb, yb, sh, sy0, sy1);
    gram_ks<UT, EL, X3, MF>(hb, yb, Gr, Gi, Mr, Mn);
  }
}

// Gram and matched filters (Algorithm 1; Eqs. 7, 8): G and b^T on the
// tensor cores, of H and Y scaled by
// sc. Unless `given`, sc is first chosen from k-step 0 (scale_from_ks).
template <int UT, int EL, bool X3, int LD, bool MF>
__device__ __forceinline__ void warp_gram(const float2* H, const float2* Y, int B, int U, int R,
                                          unsigned char* ring, GramAcc<UT>& Gr, GramAcc<UT>& Gi,
                                          VecAcc<UT>& Mr, VecAcc<UT>& Mn, InstScale& sc,
                                          bool given) {
  constexpr int NB = UT / 8, MT = WarpCfg<UT>::MT;
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
#pragma unroll
  for (int nt = 0; nt < NB; ++nt)
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      Mr[nt][k] = Mn[nt][k] = 0.f;
#pragma unroll
      for (int m = 0; m < MT; ++m) Gr[m][nt][k] = Gi[m][nt][k] = 0.f;
    }
  const int KS = (B + 7) / 8;
  constexpr bool V = LD == LD_VEC;
  float2 h[MT][4], y[4] = {};
  if constexpr (LD == LD_RING) {
    ring_gram_issue<UT, MF>(ring, H, Y, B, R, KS, WarpCfg<UT>::STAGES - 1);
    cp_wait<WarpCfg<UT>::STAGES - 1>();
    ring_gram_read<UT, MF>(ring, 0, h, y);
  } else {
    if constexpr (V)
#pragma unroll
      for (int d = 1; d <= PF_GRAM; ++d) prefetch_h_block<UT>(H, B, d);
    load_h_ks<UT, V>(H, B, U, 0, g, t, h);
    if constexpr (MF) load_y_ks<V>(Y, B, R, 0, g, t, y);
  }
  if (!given) sc = scale_from_ks<UT>(h);
  const float sh = pow2f(-sc.e()), sy0 = pow2f(-sc.f(0)), sy1 = pow2f(-sc.f(1));
  if constexpr (LD == LD_RING)
    gram_ring_loop<UT, EL, X3, MF>(H, Y, B, R, KS, ring, h, y, sh, sy0, sy1, Gr, Gi, Mr, Mn);
  else
    gram_direct_loop<UT, EL, X3, V, MF>(H, Y, B, U, R, KS, h, y, sh, sy0, sy1, Gr, Gi, Mr, Mn);
}

// warp_gram (with the matched filters) through the TMA ring, whose first
// STAGES - 1 k-steps of instance z are in flight; false if a wait ran out.
template <int UT, int EL, bool X3>
__device__ __forceinline__ bool warp_gram_tma(int B, unsigned char* ring, TmaRing& tr,
                                              const CUtensorMap* tmH, const CUtensorMap* tmY,
                                              int z, uint64_t wait_ns, GramAcc<UT>& Gr,
                                              GramAcc<UT>& Gi, VecAcc<UT>& Mr, VecAcc<UT>& Mn,
                                              InstScale& sc) {
  constexpr int NB = UT / 8, MT = WarpCfg<UT>::MT, S = WarpCfg<UT>::STAGES;
#pragma unroll
  for (int nt = 0; nt < NB; ++nt)
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      Mr[nt][k] = Mn[nt][k] = 0.f;
#pragma unroll
      for (int m = 0; m < MT; ++m) Gr[m][nt][k] = Gi[m][nt][k] = 0.f;
    }
  const int KS = (B + 7) / 8;
  float2 h[MT][4], y[4];
  tma_gram_issue<UT, true>(ring, tr, tmH, tmY, z, KS, S - 1);
  if (!tma_gram_read<UT, true>(ring, tr, 0, wait_ns, h, y)) return false;
  sc = scale_from_ks<UT>(h);
  const float sh = pow2f(-sc.e()), sy0 = pow2f(-sc.f(0)), sy1 = pow2f(-sc.f(1));
  for (int ks = 0;;) {
    apply_scale<UT, true>(h, y, sh, sy0, sy1);
    gram_ks<UT, EL, X3, true>(h, y, Gr, Gi, Mr, Mn);
    if (++ks >= KS) break;
    tma_gram_issue<UT, true>(ring, tr, tmH, tmY, z, KS, ks + S - 1);
    if (!tma_gram_read<UT, true>(ring, tr, ks, wait_ns, h, y)) return false;
  }
  return true;
}

// x[0] *= s0, x[1] *= s1 (rows g and g + 8 of the lane).
template <int NB>
__device__ __forceinline__ void scale_rows(float2 (&x)[2][NB][2], float s0, float s1) {
#pragma unroll
  for (int h = 0; h < 2; ++h)
#pragma unroll
    for (int nt = 0; nt < NB; ++nt)
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const float sh = h ? s1 : s0;
        x[h][nt][c] = make_float2(x[h][nt][c].x * sh, x[h][nt][c].y * sh);
      }
}

// The CG iterations, tracker and outputs of Algorithm 1 and Eq. 4 of one
// instance whose Gram and matched filters are done.
// Solvers of the warp bodies: CG (Algorithm 1) or the Neumann series (Sec. III-F).
constexpr int SOLVE_CG = 0;
constexpr int SOLVE_NEUMANN = 1;
constexpr int SOLVE_CG_EXACT = 2;  // CG with the exact tracker of Eq. 10

// sc: the instance's scales; the Gram and matched filters are those of the
// scaled H and Y, so sigma and N0 are scaled by 2^-2e here and x_hat by
// 2^(f - e) when it is stored. With CHECK (the fast path), an instance
// whose scaled Gram or matched filter lies outside the range the FP16 split
// needs returns kRedo before anything is stored.
//
// The exact tracker with 32 users keeps x_hat and the gathered mu, rho in the
// idle load ring (scratch) while the L_k recursion holds the registers; its
// kernels issue the next instance's first load stages only after this.
template <int UT, int SOLVER>
struct ExactStage {
  static constexpr bool kOn = SOLVER == SOLVE_CG_EXACT && UT == 32;
};

template <int UT, int EL, bool VEC, int SOLVER = SOLVE_CG>
__device__ __forceinline__ int detect_warp_finish(const DetItem& it, uint2* frag, float2* sAB,
                                                  const GramAcc<UT>& Gr, const GramAcc<UT>& Gi,
                                                  const VecAcc<UT>& Mr, const VecAcc<UT>& Mn,
                                                  InstScale sc, bool check,
                                                  unsigned char* scratch) {
  constexpr int NB = UT / 8;
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  WarpCg<UT, EL> cg;
  float Gd[NB][2], gmax;
  cg.es = WarpCg<UT, EL>::setup_a(Gr, Gi, it.sigma * sc.s2(), frag, cg.D, Gd, gmax);
#pragma unroll
  for (int hh = 0; hh < 2; ++hh)
#pragma unroll
    for (int nt = 0; nt < NB; ++nt)
#pragma unroll
      for (int c = 0; c < 2; ++c)
        cg.res[hh][nt][c] = make_float2(Mr[nt][2 * hh + c], -Mn[nt][2 * hh + c]);
  cg.init();
  if (check) {
    bool ok = gmax == 0.f || (gmax >= kColMsLo * float(it.B) && gmax <= kGHi);
#pragma unroll
    for (int hh = 0; hh < 2; ++hh)
      ok = ok && (cg.rrn[hh] == 0.f || (cg.rrn[hh] >= kRLo && cg.rrn[hh] <= kRHi));
    if (!__all_sync(0xffffffffu, ok)) return kRedo;
  }
  __syncwarp();
  if constexpr (SOLVER == SOLVE_NEUMANN) {
    // x_hat only: the soft outputs of this path are those of CG
    cg.neumann(frag, it.K);
    float one[NB][2], zero[NB][2];
#pragma unroll
    for (int nt = 0; nt < NB; ++nt)
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        one[nt][c] = 1.f;
        zero[nt][c] = 0.f;
      }
    if (sc.any()) scale_rows<NB>(cg.v, sc.xs(0), sc.xs(1));
    int nflags = 0;
#pragma unroll
    for (int hh = 0; hh < 2; ++hh)
      if (g + 8 * hh < it.R) store_row_detect<UT, 2, VEC>(it, g + 8 * hh, t, cg.v[hh], one, zero,
                                                          0.f, &nflags);
    if (lane == 0 && it.status) *it.status = 0;
    return 0;
  }
  cg.template run<true>(frag, sAB, it.R, it.K);
  __syncwarp();

  int flags = 0;
  const float cq = sqrtf(3.f * it.Es / (2.f * float((1 << it.q) - 1)));
  float rho[NB][2];
  const float n0s = it.N0 * sc.s2(), sigs = it.sigma * sc.s2();  // scaled N0 and sigma
#pragma unroll
  for (int nt = 0; nt < NB; ++nt)
#pragma unroll
    for (int c = 0; c < 2; ++c) rho[nt][c] = Gd[nt][c] / n0s;  // Eq. 13
  // exact tracker: mu and rho of every right-hand side, gathered into the
  // lanes that store its row (position P = 16 m + 8 h + g' = 8 nt + 2 t + c
  // of row r is held after exact_sinr of half m by the lanes with g' = 2 t + c,
  // as their row h = nt - 2 m)
  float emu[2][NB][2], erho[2][NB][2];
  constexpr bool XS = ExactStage<UT, SOLVER>::kOn;
  static_assert(!XS || 2 * NB * 2 * 32 * 24 <= WarpCfg<UT>::RING_BYTES, "scratch fits the ring");
  // scratch layout (XS): x_hat, then mu and rho, each entry [h][nt][c] of a
  // lane at ((h NB + nt) 2 + c) 32 + lane
  float2* xs_v = reinterpret_cast<float2*>(scratch);
  float* xs_mu = reinterpret_cast<float*>(scratch + 2 * NB * 2 * 32 * 8);
  float* xs_rho = xs_mu + 2 * NB * 2 * 32;
  // one 16-row block of L_k for exact_sinr (XS), else none (registers)
  float2* xs_L = XS ? reinterpret_cast<float2*>(xs_rho + 2 * NB * 2 * 32) : nullptr;
  if constexpr (SOLVER == SOLVE_CG_EXACT) {
    constexpr int NH = UT == 32 ? 2 : 1;  // halves of 16 matrix rows
#pragma unroll
    for (int hh = 0; hh < 2; ++hh)
#pragma unroll
      for (int nt = 0; nt < NB; ++nt)
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          emu[hh][nt][c] = erho[hh][nt][c] = 0.f;
          if constexpr (XS) {
            const int o = ((hh * NB + nt) * 2 + c) * 32 + lane;
            xs_v[o] = cg.v[hh][nt][c];
            xs_mu[o] = xs_rho[o] = 0.f;
          }
        }
    for (int r = 0; r < it.R; ++r) {
      const bool upper = r >= 8;  // row half of r (register arrays take constant indices)
      const int kdone = __shfl_sync(0xffffffffu, upper ? cg.kd[1] : cg.kd[0], 4 * (r & 7));
#pragma unroll
      for (int m = 0; m < NH; ++m) {
        float m2[2] = {0.f, 0.f}, r2[2] = {0.f, 0.f};
        if (kdone > 0) cg.exact_sinr(frag, sAB, r, kdone, sigs, n0s, it.Es, m, xs_L, m2, r2);
#pragma unroll
        for (int nt = 2 * m; nt < (NB < 2 * m + 2 ? NB : 2 * m + 2); ++nt)
#pragma unroll
          for (int c = 0; c < 2; ++c) {
            const int src = 4 * (2 * t + c) + t;
            const float mv = __shfl_sync(0xffffffffu, m2[nt - 2 * m], src);
            const float rv = __shfl_sync(0xffffffffu, r2[nt - 2 * m], src);
            if (g == (r & 7)) {
              if constexpr (XS) {
                const int o = (((upper ? 1 : 0) * NB + nt) * 2 + c) * 32 + lane;
                xs_mu[o] = mv;
                xs_rho[o] = rv;
              } else if (upper) {
                emu[1][nt][c] = mv;
                erho[1][nt][c] = rv;
              } else {
                emu[0][nt][c] = mv;
                erho[0][nt][c] = rv;
              }
            }
          }
      }
    }
    if constexpr (XS) {
#pragma unroll
      for (int hh = 0; hh < 2; ++hh)
#pragma unroll
        for (int nt = 0; nt < NB; ++nt)
#pragma unroll
          for (int c = 0; c < 2; ++c) {
            const int o = ((hh * NB + nt) * 2 + c) * 32 + lane;
            cg.v[hh][nt][c] = xs_v[o];
            emu[hh][nt][c] = xs_mu[o];
            erho[hh][nt][c] = xs_rho[o];
          }
    }
  }
  if (sc.any()) scale_rows<NB>(cg.v, sc.xs(0), sc.xs(1));
#pragma unroll
  for (int hh = 0; hh < 2; ++hh) {
    const int r = g + 8 * hh;
    if (r >= it.R) continue;
    if (cg.broke[hh]) flags |= ST_BREAKDOWN;
    float mu[NB][2], l[NB][2];
    if constexpr (SOLVER == SOLVE_CG_EXACT) {
#pragma unroll
      for (int nt = 0; nt < NB; ++nt)
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          mu[nt][c] = emu[hh][nt][c];
          rho[nt][c] = erho[hh][nt][c];
        }
    } else {
      cg.tracker_l(sAB, hh, l);
#pragma unroll
      for (int nt = 0; nt < NB; ++nt)
#pragma unroll
        for (int c = 0; c < 2; ++c) mu[nt][c] = l[nt][c] * Gd[nt][c];  // Eq. 12
    }
    switch (it.q) {
      case 2: store_row_detect<UT, 2, VEC>(it, r, t, cg.v[hh], mu, rho, cq, &flags); break;
      case 4: store_row_detect<UT, 4, VEC>(it, r, t, cg.v[hh], mu, rho, cq, &flags); break;
      case 6: store_row_detect<UT, 6, VEC>(it, r, t, cg.v[hh], mu, rho, cq, &flags); break;
      default: store_row_detect<UT, 8, VEC>(it, r, t, cg.v[hh], mu, rho, cq, &flags); break;
    }
  }
  flags = __reduce_or_sync(0xffffffffu, flags);
  if (lane == 0 && it.status) *it.status = flags;
  return flags;
}

// Whether an instance may take the vector paths (16-byte loads and stores).
template <int UT>
__device__ __forceinline__ bool detect_vec(const DetItem& it) {
  return it.U == UT && (it.B % 2) == 0 && al16(it.H) && al16(it.Y) &&
         (it.xhat == nullptr || al16(it.xhat)) && (it.mu == nullptr || al16(it.mu)) &&
         (it.rho == nullptr || al16(it.rho)) && (it.llr == nullptr || al16(it.llr));
}

// Claim without waiting: -2 when a serving queue has nothing yet.
__device__ __forceinline__ int64_t warp_try(const BatchArgs& b) { return warp_claim(b); }

// Next unit of a warp while it still works on `cur` (-1: none, -2: ask again later).
template <class S>
__device__ __forceinline__ int64_t warp_next_early(const S& s, int64_t cur, int64_t nw) {
  if constexpr (SrcTraits<S>::kDyn) {
    return warp_try(s);
  } else {
    return cur + nw < src_count(s) ? cur + nw : -1;
  }
}

// Instance loop: the Gram of an instance, then the next instance's first
// load stages, then the CG and outputs (which overlap those loads).
//
// TMA (DetectArgs of a __grid_constant__ kernel parameter only): when the
// call carries tensor maps, the vector-layout instances stage their k-steps
// through them instead of the lanes' cp.async copies. The mbarriers follow
// the CTA's warp slices (WarpCfg::TMA_SMEM). A wait that runs out marks the
// instance CG_STATUS_TIMEOUT and ends the warp's loop.
template <int UT, int EL, bool X3, class Src, int SOLVER = SOLVE_CG, bool TMA = false>
__device__ __forceinline__ void detect_warp_body(const Src& src, unsigned char* mine) {
  const int warp = threadIdx.x >> 5;
  unsigned char* ring = mine;
  uint2* frag = reinterpret_cast<uint2*>(mine + WarpCfg<UT>::RING_BYTES);
  float2* sAB = reinterpret_cast<float2*>(mine + WarpCfg<UT>::RING_BYTES + WarpCfg<UT>::FRAG_BYTES);
  const int64_t nw = int64_t(gridDim.x) * (blockDim.x >> 5);
  int64_t cur = warp_first(src, int64_t(blockIdx.x) * (blockDim.x >> 5) + warp);
  bool vec = false;
  // kLate: the next instance's first stages are issued after the finish,
  // which uses the ring as scratch (ExactStage)
  constexpr bool kLate = ExactStage<UT, SOLVER>::kOn;
  TmaRing tr;
  bool use_tma = false;
  if constexpr (TMA) {
    unsigned char* smem0 = mine - warp * WarpCfg<UT>::WARP_BYTES;
    use_tma = src.tma != 0 && (smem_addr(smem0) & 1023u) == 0;
    if (use_tma) {
      tma_ring_init(tr, smem_addr(smem0) + WarpCfg<UT>::SMEM + 8 * warp * WarpCfg<UT>::STAGES,
                    WarpCfg<UT>::STAGES);
      if ((threadIdx.x & 31) == 0) {
        tma_prefetch_map(&src.tmH);
        tma_prefetch_map(&src.tmY);
      }
    }
  }
  // first k-steps of instance idx into the ring
  auto prologue = [&](const DetItem& x, int64_t idx) {
    if constexpr (TMA) {
      if (use_tma) {
        tma_gram_prologue<UT, true>(ring, tr, &src.tmH, &src.tmY, int(idx), (x.B + 7) / 8);
        return;
      }
    }
    ring_gram_prologue<UT, true>(ring, x.H, x.Y, x.B, x.R);
  };
  if (cur >= 0) {
    const DetItem it = det_item(src, cur);
    vec = detect_vec<UT>(it);
    if (vec) prologue(it, cur);
  }
  // An instance the fast path hands back (kRedo) runs once more with scales
  // from every entry and element loads (redo.w != 0), while the ring keeps
  // the first stages of the next instance (next, nvec), which was claimed
  // on the first pass.
  InstScale redo;
  redo.w = 0;
  int64_t next = -1;
  bool nvec = false;
  while (cur >= 0) {
    GramAcc<UT> Gr, Gi;
    VecAcc<UT> Mr, Mn;
    InstScale sc = redo;
    const bool again = redo.w != 0;
    {
      const DetItem it = det_item(src, cur);
      bool landed = true;
      if (vec && !again) {
        if constexpr (TMA) {
          if (use_tma)
            landed = warp_gram_tma<UT, EL, X3>(it.B, ring, tr, &src.tmH, &src.tmY, int(cur),
                                               src.wait_ns, Gr, Gi, Mr, Mn, sc);
          else
            warp_gram<UT, EL, X3, LD_RING, true>(it.H, it.Y, it.B, it.U, it.R, ring, Gr, Gi, Mr,
                                                 Mn, sc, false);
        } else {
          warp_gram<UT, EL, X3, LD_RING, true>(it.H, it.Y, it.B, it.U, it.R, ring, Gr, Gi, Mr, Mn,
                                               sc, false);
        }
      } else {
        warp_gram<UT, EL, X3, LD_ELEM, true>(it.H, it.Y, it.B, it.U, it.R, ring, Gr, Gi, Mr, Mn,
                                             sc, again);
      }
      if (!landed) {  // the inputs never arrived: report it and stop this warp
        if ((threadIdx.x & 31) == 0 && it.status) *it.status = ST_TIMEOUT;
        break;
      }
    }
    if (!again) {
      next = warp_next_early(src, cur, nw);
      nvec = false;
      if (next >= 0) {
        const DetItem nit = det_item(src, next);
        nvec = detect_vec<UT>(nit);
        if (nvec && !kLate) prologue(nit, next);
      }
    }
    int st;
    {
      const DetItem it = det_item(src, cur);
      st = (vec && !again)
               ? detect_warp_finish<UT, EL, true, SOLVER>(it, frag, sAB, Gr, Gi, Mr, Mn, sc, true,
                                                          ring)
               : detect_warp_finish<UT, EL, false, SOLVER>(it, frag, sAB, Gr, Gi, Mr, Mn, sc,
                                                           !again, ring);
      if (st == kRedo) {
        redo = full_scale<true>(it.H, it.Y, it.B, it.U, it.R);
        redo.w |= 1 << 25;  // marks the second pass even when every scale is 1
        continue;
      }
    }
    redo.w = 0;
    if constexpr (kLate) {
      __syncwarp();  // every lane is done with the scratch
      if (next >= 0 && nvec) {
        const DetItem nit = det_item(src, next);
        prologue(nit, next);
      }
    }
    __syncwarp();
    if constexpr (SrcTraits<Src>::kDyn) {
      if ((threadIdx.x & 31) == 0) src_done(src, cur, st);
      if (next == -2) {  // nothing was ready earlier: wait for work now (bounded)
        next = warp_claim(src);
        if (next >= 0) {
          const DetItem nit = det_item(src, next);
          nvec = detect_vec<UT>(nit);
          if (nvec) prologue(nit, next);
        }
      }
    }
    cur = next;
    vec = nvec;
  }
  cp_wait<0>();
  if constexpr (TMA) {
    if (use_tma) tma_ring_drain(tr, WarpCfg<UT>::STAGES);
  }
}

// ---------------------------------------------------------------------------
// CG-P, one warp per instance
// ---------------------------------------------------------------------------

// The CG iterations of Algorithm 1 with b = t, ||q||, then the precoding
// output q = H v (Sec. III-D) of one instance whose
// Gram is done. hsc holds the scale e of H; each row of T gets its own f
// here: the CG runs on 2^-e H, 2^-f t and 2^-2e sigma, giving v' = 2^(2e - f) v,
// and q = 2^(f - e) (2^-e H) v', ||q|| = 2^(f - e) ||2^-e H v'||. With CHECK
// (the fast path), an instance whose scaled Gram lies outside the range the
// FP16 split needs returns kRedo before anything is stored.
// nit, when given, is the warp's next instance: the first blocks of its H
// and its T are prefetched into L1 while this q pass runs.
template <int UT, int EL, bool X3, bool VEC, int SOLVER = SOLVE_CG>
__device__ __forceinline__ int precode_warp_finish(const PreItem& it, uint2* frag,
                                                   const GramAcc<UT>& Gr, const GramAcc<UT>& Gi,
                                                   InstScale hsc, bool check,
                                                   const PreItem* nit = nullptr) {
  constexpr int NB = UT / 8;
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  WarpCg<UT, EL> cg;
#pragma unroll
  for (int hh = 0; hh < 2; ++hh) {
    const int r = g + 8 * hh;
    const float2* tr = it.T + int64_t(r) * it.U;
#pragma unroll
    for (int nt = 0; nt < NB; ++nt)
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const int u = pos_user<UT>(8 * nt + 2 * t + c);
        cg.res[hh][nt][c] = (r < it.R && u < it.U) ? tr[u] : make_float2(0.f, 0.f);
      }
  }
  float Gd[NB][2], gmax;
  cg.es = WarpCg<UT, EL>::setup_a(Gr, Gi, it.sigma * hsc.s2(), frag, cg.D, Gd, gmax);
  // the solution v ~ t / lambda(A') enters the FP16 split of the products
  // with H, so the columns of H' must also stay near unit power: the
  // strongest one's mean square at most kPreColMsHi
  if (check && !(gmax == 0.f || (gmax >= kColMsLo * float(it.B) &&
                                 gmax <= kPreColMsHi * float(it.B))))
    return kRedo;
  cg.init();
  // f of each row of T from ||t||^2 (unscaled in [2^-4, 2^12], else put in [4, 16))
  const InstScale sc = InstScale::make(hsc.e(), band_exp(cg.rrn[0], kTLo, kTHi, kTTarget) >> 1,
                                       band_exp(cg.rrn[1], kTLo, kTHi, kTTarget) >> 1);
  if (sc.any()) {
    const float s0 = pow2f(-sc.f(0)), s1 = pow2f(-sc.f(1));
    scale_rows<NB>(cg.res, s0, s1);
    scale_rows<NB>(cg.p, s0, s1);
    cg.rrn[0] *= s0 * s0;
    cg.rrn[1] *= s1 * s1;
  }
  __syncwarp();
  if constexpr (SOLVER == SOLVE_NEUMANN)
    cg.neumann(frag, it.K);
  else
    cg.template run<false>(frag, nullptr, it.R, it.K);

  // ||q||^2 = v^H (A - sigma I) v with one more product w = A v
#pragma unroll
  for (int hh = 0; hh < 2; ++hh)
#pragma unroll
    for (int nt = 0; nt < NB; ++nt)
#pragma unroll
      for (int c = 0; c < 2; ++c) cg.p[hh][nt][c] = cg.v[hh][nt][c];
  float Er[NB][4], Ei[NB][4];
  cg.matvec_s(frag, cg.es, Er, Ei);
  const float sig = it.sigma * sc.s2();
  float qq[2] = {0.f, 0.f};
#pragma unroll
  for (int hh = 0; hh < 2; ++hh)
#pragma unroll
    for (int nt = 0; nt < NB; ++nt)
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const float2 vv = cg.v[hh][nt][c];
        const float wx = fmaf(-sig, vv.x, Er[nt][2 * hh + c]);
        const float wy = fmaf(-sig, vv.y, Ei[nt][2 * hh + c]);
        qq[hh] = fmaf(vv.x, wx, fmaf(vv.y, wy, qq[hh]));
      }
  quad_sum2(qq[0], qq[1]);
  float inv[2];
  int flags = 0;
#pragma unroll
  for (int hh = 0; hh < 2; ++hh) {
    const int r = g + 8 * hh;
    const float nr = sqrtf(fmaxf(qq[hh], 0.f));
    const float qs = sc.any() ? sc.xs(hh) : 1.f;
    inv[hh] = it.normalize ? (nr > 0.f ? 1.f / nr : 0.f) : qs;
    if (r < it.R) {
      if (t == 0 && it.qnorm) it.qnorm[r] = nr * qs;
      if (cg.broke[hh]) flags |= ST_BREAKDOWN;
    }
  }
  const float hsh = pow2f(-sc.e());  // H' = 2^-e H in the second pass too
  const bool hscaled = sc.e() != 0;

  // ---- precoding output q = H v on the tensor cores, 8 antennas per n-tile
  uint32_t vh[NB][4], vl[NB][4];
#pragma unroll
  for (int ks = 0; ks < NB; ++ks) {
    const uint2 s0 = split_c<EL>(cg.v[0][ks][0]);
    const uint2 s1 = split_c<EL>(cg.v[1][ks][0]);
    const uint2 s2 = split_c<EL>(cg.v[0][ks][1]);
    const uint2 s3 = split_c<EL>(cg.v[1][ks][1]);
    vh[ks][0] = s0.x; vl[ks][0] = s0.y;
    vh[ks][1] = s1.x; vl[ks][1] = s1.y;
    vh[ks][2] = s2.x; vl[ks][2] = s2.y;
    vh[ks][3] = s3.x; vl[ks][3] = s3.y;
  }
  // H is read a second time here (L1 or L2: the Gram read it moments ago);
  // VEC keeps the 16-byte loads of the next n-tile in flight.
  constexpr int MT = WarpCfg<UT>::MT;
  const int NBQ = (it.B + 7) / 8;
  float4 fa[MT][2];
  if constexpr (VEC) {
#pragma unroll
    for (int d = 1; d <= PF_Q; ++d) prefetch_h_block<UT>(it.H, it.B, d);
    q_load<UT>(it.H, it.B, 0, g, t, fa);
    if (nit != nullptr) {
#pragma unroll
      for (int d = 0; d <= PF_GRAM; ++d) prefetch_h_block<UT>(nit->H, nit->B, d);
      prefetch_rows_l1(nit->T, nit->R * nit->U * 8);
    }
  }
  for (int nb = 0; nb < NBQ; ++nb) {
    if constexpr (VEC) prefetch_h_block<UT>(it.H, it.B, nb + 1 + PF_Q);
    const int b = 8 * nb + g;
    // lane's H entries at its k-positions: e[ks][j] = H(b, user(8 ks + 2 t + j))
    float2 e[NB][2];
    const float2 z = make_float2(0.f, 0.f);
    if constexpr (VEC) {
      float4 f[MT][2];
#pragma unroll
      for (int m = 0; m < MT; ++m) {
        f[m][0] = fa[m][0];
        f[m][1] = fa[m][1];
      }
      if (nb + 1 < NBQ) q_load<UT>(it.H, it.B, nb + 1, g, t, fa);
      if constexpr (UT == 8) {
        e[0][0] = make_float2(f[0][0].x, f[0][0].y);
        e[0][1] = make_float2(f[0][0].z, f[0][0].w);
      } else {
#pragma unroll
        for (int m = 0; m < MT; ++m) {
          e[2 * m][0] = make_float2(f[m][0].x, f[m][0].y);      // user 16m + 4t
          e[2 * m + 1][0] = make_float2(f[m][0].z, f[m][0].w);  // user 16m + 4t + 1
          e[2 * m][1] = make_float2(f[m][1].x, f[m][1].y);      // user 16m + 4t + 2
          e[2 * m + 1][1] = make_float2(f[m][1].z, f[m][1].w);  // user 16m + 4t + 3
        }
      }
    } else {
#pragma unroll
      for (int ks = 0; ks < NB; ++ks)
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          const int u = pos_user<UT>(8 * ks + 2 * t + j);
          e[ks][j] = (b < it.B && u < it.U) ? ldg2(it.H + b * it.U + u) : z;
        }
    }
    if (hscaled) {
#pragma unroll
      for (int ks = 0; ks < NB; ++ks)
#pragma unroll
        for (int j = 0; j < 2; ++j) e[ks][j] = make_float2(e[ks][j].x * hsh, e[ks][j].y * hsh);
    }
    float qr[4] = {0.f, 0.f, 0.f, 0.f}, qi[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int ks = 0; ks < NB; ++ks) {
      const uint2 s0 = split_c<EL>(e[ks][0]), s1 = split_c<EL>(e[ks][1]);
      // real part: v . conj(H); imaginary part: v . (Hi, Hr)
      mma_split<EL, X3>(qr, vh[ks], vl[ks], neg_hi(s0.x), neg_hi(s1.x), neg_hi(s0.y),
                        neg_hi(s1.y));
      mma_split<EL, X3>(qi, vh[ks], vl[ks], swap_halves(s0.x), swap_halves(s1.x),
                        swap_halves(s0.y), swap_halves(s1.y));
    }
#pragma unroll
    for (int hh = 0; hh < 2; ++hh) {
      const int r = g + 8 * hh;
      if (r >= it.R) continue;
      const int b0 = 8 * nb + 2 * t;
      const float2 q0 = make_float2(qr[2 * hh] * inv[hh], qi[2 * hh] * inv[hh]);
      const float2 q1 = make_float2(qr[2 * hh + 1] * inv[hh], qi[2 * hh + 1] * inv[hh]);
      float2* qrow = it.q + int64_t(r) * it.B;
      if constexpr (VEC) {
        if (b0 < it.B)
          *reinterpret_cast<float4*>(qrow + b0) = make_float4(q0.x, q0.y, q1.x, q1.y);
      } else {
        if (b0 < it.B) qrow[b0] = q0;
        if (b0 + 1 < it.B) qrow[b0 + 1] = q1;
      }
    }
  }
  flags = __reduce_or_sync(0xffffffffu, flags);
  if (lane == 0 && it.status) *it.status = flags;
  return flags;
}

// Whether an instance may take the vector paths.
template <int UT>
__device__ __forceinline__ bool precode_vec(const PreItem& it) {
  return it.U == UT && (it.B % 2) == 0 && al16(it.H) && al16(it.q);
}

// Instance loop. CG-P reads H twice (Gram, then q = H v); both passes use
// 16-byte register loads through L1, where the second pass finds part of H.
template <int UT, int EL, bool X3, class Src, int SOLVER = SOLVE_CG>
__device__ __forceinline__ void precode_warp_body(const Src& src, unsigned char* mine) {
  const int warp = threadIdx.x >> 5;
  uint2* frag = reinterpret_cast<uint2*>(mine);
  const int64_t nw = int64_t(gridDim.x) * (blockDim.x >> 5);
  int64_t cur = warp_first(src, int64_t(blockIdx.x) * (blockDim.x >> 5) + warp);
  // An instance the fast path hands back (kRedo) runs once more with the
  // scale of H taken from every entry (redo.w != 0).
  InstScale redo;
  redo.w = 0;
  while (cur >= 0) {
    const PreItem it = pre_item(src, cur);
    GramAcc<UT> Gr, Gi;
    VecAcc<UT> Mr, Mn;
    InstScale sc = redo;
    const bool again = redo.w != 0;
    int st;
    if (precode_vec<UT>(it)) {
      warp_gram<UT, EL, X3, LD_VEC, false>(it.H, nullptr, it.B, it.U, 0, nullptr, Gr, Gi, Mr, Mn,
                                           sc, again);
      int64_t nx = -1;
      if constexpr (!SrcTraits<Src>::kDyn) nx = warp_next_early(src, cur, nw);
      PreItem nit;
      if (nx >= 0) nit = pre_item(src, nx);
      st = precode_warp_finish<UT, EL, X3, true, SOLVER>(it, frag, Gr, Gi, sc, !again,
                                                         nx >= 0 ? &nit : nullptr);
    } else {
      warp_gram<UT, EL, X3, LD_ELEM, false>(it.H, nullptr, it.B, it.U, 0, nullptr, Gr, Gi, Mr,
                                            Mn, sc, again);
      st = precode_warp_finish<UT, EL, X3, false, SOLVER>(it, frag, Gr, Gi, sc, !again);
    }
    if (st == kRedo) {
      redo = full_scale<false>(it.H, nullptr, it.B, it.U, 0);
      redo.w |= 1 << 25;  // marks the second pass even when every scale is 1
      continue;
    }
    redo.w = 0;
    __syncwarp();
    if constexpr (SrcTraits<Src>::kDyn) {
      if ((threadIdx.x & 31) == 0) src_done(src, cur, st);
    }
    cur = warp_next_early(src, cur, nw);
    if constexpr (SrcTraits<Src>::kDyn) {
      if (cur == -2) cur = warp_claim(src);
    }
  }
}

// This warp's slice of the dynamic shared memory.
template <uint32_t SLICE>
__device__ __forceinline__ unsigned char* warp_slice() {
  extern __shared__ __align__(128) unsigned char smem[];
  return smem + (threadIdx.x >> 5) * SLICE;
}

template <int UT, int EL, bool X3>
__global__ void __launch_bounds__(WarpCfg<UT>::NTHR, WarpCfg<UT>::MINB)
    detect_warp_kernel(const __grid_constant__ DetectArgs a) {
  detect_warp_body<UT, EL, X3, DetectArgs, SOLVE_CG, true>(a, warp_slice<WarpCfg<UT>::WARP_BYTES>());
}
template <int UT, int EL, bool X3>
__global__ void __launch_bounds__(WarpCfg<UT>::NTHR, WarpCfg<UT>::MINB) precode_warp_kernel(const PrecodeArgs a) {
  precode_warp_body<UT, EL, X3>(a, warp_slice<WarpCfg<UT>::FRAG_BYTES>());
}
template <int UT, int EL, bool X3>
__global__ void __launch_bounds__(WarpCfg<UT>::NTHR, WarpCfg<UT>::MINB) detect_warp_batch_kernel(const BatchArgs b) {
  detect_warp_body<UT, EL, X3>(b, warp_slice<WarpCfg<UT>::WARP_BYTES>());
}
template <int UT, int EL, bool X3>
__global__ void __launch_bounds__(WarpCfg<UT>::NTHR, WarpCfg<UT>::MINB)
    precode_warp_batch_kernel(const BatchArgs b) {
  precode_warp_body<UT, EL, X3>(b, warp_slice<WarpCfg<UT>::FRAG_BYTES>());
}

}  // namespace cgm
