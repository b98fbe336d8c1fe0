// CG-D with the exact SINR tracker (Eq. 10) on the warp-per-instance
// tensor-core bodies, for up to 32 users: the staging, Gram, matched filter,
// CG and LLRs of detect_warp_kernel, with the L_k recursion of every
// right-hand side run as tensor-core products of 16 rows of L at a time
// (WarpCg::exact_sinr; 32 users take two halves). Three 16-row complex L
// blocks live in registers, so these kernels are built for 2 resident CTAs
// (8 warps) per SM.
#include <mutex>
#include <unordered_map>

#include "cg_warp.cuh"
#include "launch.cuh"

namespace cgm {

template <int UT, int EL, bool X3>
__global__ void __launch_bounds__(WarpCfg<UT>::NTHR, 2) detect_warp_exact_kernel(const DetectArgs a) {
  detect_warp_body<UT, EL, X3, DetectArgs, SOLVE_CG_EXACT>(a, warp_slice<WarpCfg<UT>::WARP_BYTES>());
}
// The same for the exact-tracker bins of the batched entry points, so that a
// problem gives the same bits in a batch as in a single call.
template <int UT, int EL, bool X3>
__global__ void __launch_bounds__(WarpCfg<UT>::NTHR, 2)
    detect_warp_exact_batch_kernel(const BatchArgs b) {
  detect_warp_body<UT, EL, X3, BatchArgs, SOLVE_CG_EXACT>(b, warp_slice<WarpCfg<UT>::WARP_BYTES>());
}

namespace {

std::mutex g_mu;
std::unordered_map<uint64_t, int> g_occ;  // (device, kernel id) -> resident CTAs per SM

// Grid for n_work units of one warp each: resident CTAs at most (and max_grid
// when it is positive).
template <typename Kern>
cudaError_t grid_for(Kern kern, uint64_t id, int64_t n_work, int max_grid, int* grid) {
  constexpr uint32_t smem = WarpCfg<32>::SMEM;  // the largest slice (UT = 32)
  static_assert(WarpCfg<32>::SMEM >= WarpCfg<16>::SMEM && WarpCfg<32>::SMEM >= WarpCfg<8>::SMEM,
                "one attribute value serves every padded user count");
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
  int64_t g = (n_work + WarpCfg<8>::WARPS - 1) / WarpCfg<8>::WARPS;
  const int64_t res = int64_t(occ) * di.sm_count;
  if (g > res) g = res;
  if (max_grid > 0 && g > max_grid) g = max_grid;
  *grid = int(g < 1 ? 1 : g);
  return cudaSuccess;
}

template <int UT, int EL, bool X3>
cudaError_t det(const DetectArgs& a, cudaStream_t s) {
  constexpr uint32_t smem = WarpCfg<UT>::SMEM;
  int grid = 0;
  const uint64_t id = (UT << 2) | (EL << 1) | (X3 ? 1 : 0);
  cudaError_t err = grid_for(detect_warp_exact_kernel<UT, EL, X3>, id, a.n_inst, 0, &grid);
  if (err != cudaSuccess) return err;
  detect_warp_exact_kernel<UT, EL, X3><<<unsigned(grid), WarpCfg<UT>::NTHR, smem, s>>>(a);
  return cudaGetLastError();
}

template <int UT, int EL, bool X3>
cudaError_t batch(const BatchArgs& b, int max_grid, cudaStream_t s, bool launch, int* grid_out) {
  constexpr uint32_t smem = WarpCfg<UT>::SMEM;
  int grid = 0;
  const uint64_t id = 0x100 | (UT << 2) | (EL << 1) | (X3 ? 1 : 0);
  cudaError_t err =
      grid_for(detect_warp_exact_batch_kernel<UT, EL, X3>, id, b.n_work, max_grid, &grid);
  if (err != cudaSuccess) return err;
  if (grid_out) *grid_out = grid;
  if (!launch) return cudaSuccess;
  detect_warp_exact_batch_kernel<UT, EL, X3><<<unsigned(grid), WarpCfg<UT>::NTHR, smem, s>>>(b);
  return cudaGetLastError();
}

template <int UT>
cudaError_t det_ut(int el, bool x3, const DetectArgs& a, cudaStream_t s) {
  if (el == EL_BF16) return x3 ? det<UT, EL_BF16, true>(a, s) : det<UT, EL_BF16, false>(a, s);
  return x3 ? det<UT, EL_F16, true>(a, s) : det<UT, EL_F16, false>(a, s);
}

template <int UT>
cudaError_t batch_ut(int el, bool x3, const BatchArgs& b, int mg, cudaStream_t s, bool l,
                     int* g) {
  if (el == EL_BF16)
    return x3 ? batch<UT, EL_BF16, true>(b, mg, s, l, g) : batch<UT, EL_BF16, false>(b, mg, s, l, g);
  return x3 ? batch<UT, EL_F16, true>(b, mg, s, l, g) : batch<UT, EL_F16, false>(b, mg, s, l, g);
}

}  // namespace

cudaError_t launch_batch_warp_exact(int UT, int el, bool x3, const BatchArgs& b, int max_grid,
                                    cudaStream_t s, bool launch, int* grid_out) {
  switch (UT < 8 ? 8 : UT) {
    case 8: return batch_ut<8>(el, x3, b, max_grid, s, launch, grid_out);
    case 16: return batch_ut<16>(el, x3, b, max_grid, s, launch, grid_out);
    case 32: return batch_ut<32>(el, x3, b, max_grid, s, launch, grid_out);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_detect_warp_exact(int UT, int el, bool x3, const DetectArgs& a,
                                     cudaStream_t s) {
  switch (UT < 8 ? 8 : UT) {
    case 8: return det_ut<8>(el, x3, a, s);
    case 16: return det_ut<16>(el, x3, a, s);
    case 32: return det_ut<32>(el, x3, a, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace cgm
