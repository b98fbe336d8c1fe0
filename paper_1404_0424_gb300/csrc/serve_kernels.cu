// Launcher of the serving kernel, the warp-per-instance kernel of every
// class. Every serving CTA is padded to one per SM (serve_smem).
#include <mutex>
#include <unordered_map>

#include "cg_serve.cuh"
#include "launch.cuh"

namespace cgm {

namespace {

std::mutex g_mu;
std::unordered_map<uint64_t, int> g_occ;  // (device, kernel id) -> resident CTAs per SM

// Resident CTAs of `kern` on the current device (all SMs), after allowing
// it `smem` bytes of dynamic shared memory.
template <typename Kern>
cudaError_t resident(Kern kern, uint64_t id, int nthr, uint32_t smem, int* out) {
  DeviceInfo di;
  if (device_info(&di) != 0) return cudaErrorUnknown;
  if (int(smem) > di.smem_optin) return cudaErrorInvalidValue;
  int dev = 0;
  cudaError_t err = cudaGetDevice(&dev);
  if (err != cudaSuccess) return err;
  const uint64_t key = (uint64_t(dev) << 48) | (id << 20) | smem;
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = g_occ.find(key);
  int occ = 0;
  if (it == g_occ.end()) {
    err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (err != cudaSuccess) return err;
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, nthr, smem);
    if (err != cudaSuccess) return err;
    if (occ < 1) occ = 1;
    g_occ[key] = occ;
  } else {
    occ = it->second;
  }
  *out = occ * di.sm_count;
  return cudaSuccess;
}

template <int EL, bool X3>
cudaError_t warp_serve(const ServeArgs& sa, int grid, cudaStream_t s, bool launch,
                       int* resident_out) {
  DeviceInfo di;
  if (device_info(&di) != 0) return cudaErrorUnknown;
  // a slice for the largest class per warp, padded to one CTA per SM
  const uint32_t smem = serve_smem(di, uint32_t(kServeThreads / 32) * kServeSlice);
  int res = 0;
  const uint64_t id = 0x40 | (EL << 1) | (X3 ? 1 : 0);
  cudaError_t err = resident(warp_serve_kernel<EL, X3>, id, kServeThreads, smem, &res);
  if (err != cudaSuccess) return err;
  if (resident_out) *resident_out = res;
  if (!launch) return cudaSuccess;
  ServeWarpArgs p;
  p.k = sa;
  for (int c = 0; c < kWarpClasses; ++c) {
    p.c[c] = sa;
    p.c[c].cls = c;
    p.c[c].idle_ns = 0;
    p.c[c].poll_host = 0;
  }
  warp_serve_kernel<EL, X3><<<unsigned(grid), kServeThreads, smem, s>>>(p);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_serve_warp(int el, bool x3, const ServeArgs& sa, int grid, cudaStream_t s,
                              bool launch, int* resident_out) {
  if (el == EL_BF16)
    return x3 ? warp_serve<EL_BF16, true>(sa, grid, s, launch, resident_out)
              : warp_serve<EL_BF16, false>(sa, grid, s, launch, resident_out);
  return x3 ? warp_serve<EL_F16, true>(sa, grid, s, launch, resident_out)
            : warp_serve<EL_F16, false>(sa, grid, s, launch, resident_out);
}

}  // namespace cgm
