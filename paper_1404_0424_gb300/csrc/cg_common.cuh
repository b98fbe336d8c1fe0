// Device helpers shared by the libcgmimo kernels: bulk-copy and mbarrier PTX
// wrappers with bounded waits, complex arithmetic, and group reductions.
#pragma once

#include <cstdint>
#include <cuda.h>  // CUtensorMap (the type only; nothing links the driver library)
#include <cuda_runtime.h>

namespace cgm {

constexpr int RMAX = 16;   // right-hand sides per instance (CG_R_MAX)
constexpr int KMAX = 32;   // CG iterations (CG_K_MAX)
constexpr uint64_t WAIT_TIMEOUT_NS = 2000000000ull;  // 2 s bound on any device wait

constexpr int ST_BREAKDOWN = 1;
constexpr int ST_MU_NONPOS = 2;
constexpr int ST_TIMEOUT = 4;

__host__ __device__ constexpr uint32_t align16(uint32_t x) { return (x + 15u) & ~15u; }

// --------------------------------------------------------------------------
// Shared-memory addressing, mbarrier and bulk async copies (sm_90+ PTX)
// --------------------------------------------------------------------------

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t global_timer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Orders this thread's earlier generic-proxy shared-memory accesses before
// later async-proxy (bulk copy) accesses to the same memory.
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}

// 1-D bulk copy global -> shared, completion counted on `bar` in bytes.
// dst, src 16-byte aligned; bytes a multiple of 16.
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes,
                                              uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cta.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

// 3-D tiled tensor copy (TMA) global -> shared of the box at element
// coordinates (x, y, z) of `map`, completion counted on `bar` in bytes. The
// map must sit in kernel-parameter (__grid_constant__), constant or global
// memory; dst is aligned to the map's swizzle span; x * element size is a
// multiple of 16 bytes. Out-of-range elements of the box arrive as zeros.
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y,
                                            int z, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
      "[%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_addr(bar))
      : "memory");
}

// As tma_load_3d, with dst and bar given as shared-space addresses.
__device__ __forceinline__ void tma_load_3d_s(uint32_t dst, const CUtensorMap* map, int x, int y,
                                              int z, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
      "[%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void mbar_init_s(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx_s(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}

// Fetches a tensor map into the TMA unit's descriptor cache ahead of use.
__device__ __forceinline__ void tma_prefetch_map(const CUtensorMap* map) {
  asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ bool mbar_test_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ bool mbar_try_wait_s(uint32_t bar, uint32_t parity) {
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

__device__ __forceinline__ bool mbar_test_wait_s(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Waits for phase `parity` of `bar` to complete; gives up after timeout_ns
// of global time and returns false. try_wait may suspend the thread for a
// while by itself, so limits under 1 us poll with the non-blocking
// test_wait instead, which lets such a limit run out before the phase does.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity,
                                                  uint64_t timeout_ns) {
  const bool poll = timeout_ns < 1000;
  const uint64_t t0 = global_timer_ns();
  while (true) {
    if (poll ? mbar_test_wait(bar, parity) : mbar_try_wait(bar, parity)) return true;
    if (global_timer_ns() - t0 > timeout_ns) return false;
    if (!poll) __nanosleep(64);
  }
}

// mbar_wait_bounded on a shared-space address. The first try_wait is made
// before the clock is read, so a phase that is already complete costs one
// instruction.
__device__ __forceinline__ bool mbar_wait_bounded_s(uint32_t bar, uint32_t parity,
                                                    uint64_t timeout_ns) {
  const bool poll = timeout_ns < 1000;
  if (poll ? mbar_test_wait_s(bar, parity) : mbar_try_wait_s(bar, parity)) return true;
  const uint64_t t0 = global_timer_ns();
  while (true) {
    if (poll ? mbar_test_wait_s(bar, parity) : mbar_try_wait_s(bar, parity)) return true;
    if (global_timer_ns() - t0 > timeout_ns) return false;
    if (!poll) __nanosleep(64);
  }
}

// --------------------------------------------------------------------------
// Complex helpers (float2 = complex64)
// --------------------------------------------------------------------------

// acc += conj(a) * b
__device__ __forceinline__ void cmac_conj(float2& acc, float2 a, float2 b) {
  acc.x = fmaf(a.x, b.x, acc.x);
  acc.x = fmaf(a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y);
  acc.y = fmaf(-a.y, b.x, acc.y);
}

// acc += a * b
__device__ __forceinline__ void cmac(float2& acc, float2 a, float2 b) {
  acc.x = fmaf(a.x, b.x, acc.x);
  acc.x = fmaf(-a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y);
  acc.y = fmaf(a.y, b.x, acc.y);
}

// --------------------------------------------------------------------------
// Reductions over a group of W consecutive lanes (W a power of two <= 32)
// --------------------------------------------------------------------------

template <int W>
__device__ __forceinline__ unsigned group_mask() {
  if constexpr (W >= 32) {
    return 0xffffffffu;
  } else {
    const unsigned lane = threadIdx.x & 31u;
    return ((1u << W) - 1u) << (lane & ~(unsigned)(W - 1));
  }
}

// Compensated butterfly sum: every lane of the group gets the same value.
// Each level adds the partners' partial sums and carries the exact rounding
// error of that addition (TwoSum, Knuth) in a second accumulator.
template <int W>
__device__ __forceinline__ float group_sum_compensated(float x, unsigned mask) {
  float s = x, c = 0.f;
#pragma unroll
  for (int off = W / 2; off > 0; off >>= 1) {
    const float so = __shfl_xor_sync(mask, s, off, W);
    const float co = __shfl_xor_sync(mask, c, off, W);
    const float t = s + so;
    const float bp = t - s;
    const float err = (s - (t - bp)) + (so - bp);
    s = t;
    c = (c + co) + err;
  }
  return s + c;
}

}  // namespace cgm
