// Neumann-series detection and precoding (Sec. III-F) on the warp-per-instance
// tensor-core bodies: the same staging, Gram, matched filter and q = H v as
// CG-D / CG-P, with the truncated Neumann series in place of Algorithm 1's
// CG loop (WarpCg::neumann). Offered as an accuracy and throughput comparator.
#include <mutex>
#include <unordered_map>

#include "cg_warp.cuh"
#include "launch.cuh"

namespace cgm {

template <int UT, int EL, bool X3>
__global__ void __launch_bounds__(WarpCfg<UT>::NTHR, WarpCfg<UT>::MINB)
    neumann_detect_warp_kernel(const DetectArgs a) {
  detect_warp_body<UT, EL, X3, DetectArgs, SOLVE_NEUMANN>(a, warp_slice<WarpCfg<UT>::WARP_BYTES>());
}
template <int UT, int EL, bool X3>
__global__ void __launch_bounds__(WarpCfg<UT>::NTHR, WarpCfg<UT>::MINB)
    neumann_precode_warp_kernel(const PrecodeArgs a) {
  precode_warp_body<UT, EL, X3, PrecodeArgs, SOLVE_NEUMANN>(a,
                                                           warp_slice<WarpCfg<UT>::FRAG_BYTES>());
}

namespace {

std::mutex g_mu;
std::unordered_map<uint64_t, int> g_occ;  // (device, kernel id) -> resident CTAs per SM

template <typename Kern>
cudaError_t grid_for(Kern kern, uint64_t id, uint32_t smem, int64_t n_inst, int* grid) {
  DeviceInfo di;
  if (device_info(&di) != 0) return cudaErrorUnknown;
  int dev = 0;
  cudaError_t err = cudaGetDevice(&dev);
  if (err != cudaSuccess) return err;
  const uint64_t key = (uint64_t(dev) << 48) | id;
  int occ = 0;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_occ.find(key);
    if (it == g_occ.end()) {
      err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
      if (err != cudaSuccess) return err;
      err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, WarpCfg<8>::NTHR, smem);
      if (err != cudaSuccess) return err;
      if (occ < 1) occ = 1;
      g_occ[key] = occ;
    } else {
      occ = it->second;
    }
  }
  // one warp per instance, at most the resident CTAs (grid stride beyond)
  int64_t g = (n_inst + WarpCfg<8>::WARPS - 1) / WarpCfg<8>::WARPS;
  const int64_t res = int64_t(occ) * di.sm_count;
  if (g > res) g = res;
  *grid = int(g < 1 ? 1 : g);
  return cudaSuccess;
}

template <int UT, int EL, bool X3>
cudaError_t det(const DetectArgs& a, cudaStream_t s) {
  constexpr uint32_t smem = WarpCfg<UT>::SMEM;
  int grid = 0;
  const uint64_t id = 0x10 | (UT << 2) | (EL << 1) | (X3 ? 1 : 0);
  cudaError_t err = grid_for(neumann_detect_warp_kernel<UT, EL, X3>, id, smem, a.n_inst, &grid);
  if (err != cudaSuccess) return err;
  neumann_detect_warp_kernel<UT, EL, X3><<<unsigned(grid), WarpCfg<UT>::NTHR, smem, s>>>(a);
  return cudaGetLastError();
}

template <int UT, int EL, bool X3>
cudaError_t pre(const PrecodeArgs& a, cudaStream_t s) {
  constexpr uint32_t smem = WarpCfg<UT>::PRE_SMEM;
  int grid = 0;
  const uint64_t id = 0x20 | (UT << 2) | (EL << 1) | (X3 ? 1 : 0);
  cudaError_t err = grid_for(neumann_precode_warp_kernel<UT, EL, X3>, id, smem, a.n_inst, &grid);
  if (err != cudaSuccess) return err;
  neumann_precode_warp_kernel<UT, EL, X3><<<unsigned(grid), WarpCfg<UT>::NTHR, smem, s>>>(a);
  return cudaGetLastError();
}

template <int UT>
cudaError_t det_ut(int el, bool x3, const DetectArgs& a, cudaStream_t s) {
  if (el == EL_BF16) return x3 ? det<UT, EL_BF16, true>(a, s) : det<UT, EL_BF16, false>(a, s);
  return x3 ? det<UT, EL_F16, true>(a, s) : det<UT, EL_F16, false>(a, s);
}

template <int UT>
cudaError_t pre_ut(int el, bool x3, const PrecodeArgs& a, cudaStream_t s) {
  if (el == EL_BF16) return x3 ? pre<UT, EL_BF16, true>(a, s) : pre<UT, EL_BF16, false>(a, s);
  return x3 ? pre<UT, EL_F16, true>(a, s) : pre<UT, EL_F16, false>(a, s);
}

}  // namespace

cudaError_t launch_neumann_detect(int UT, int el, bool x3, const DetectArgs& a, cudaStream_t s) {
  switch (UT < 8 ? 8 : UT) {
    case 8: return det_ut<8>(el, x3, a, s);
    case 16: return det_ut<16>(el, x3, a, s);
    case 32: return det_ut<32>(el, x3, a, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_neumann_precode(int UT, int el, bool x3, const PrecodeArgs& a, cudaStream_t s) {
  switch (UT < 8 ? 8 : UT) {
    case 8: return pre_ut<8>(el, x3, a, s);
    case 16: return pre_ut<16>(el, x3, a, s);
    case 32: return pre_ut<32>(el, x3, a, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace cgm
