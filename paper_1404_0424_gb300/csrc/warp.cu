// Launchers of the warp-per-instance tensor-core kernels (padded users 8, 16
// or 32, approximate SINR tracker): single calls, plan bins and serving classes.
#include <mutex>
#include <unordered_map>

#include "cg_warp.cuh"
#include "launch.cuh"

namespace cgm {

namespace {

std::mutex g_mu;
std::unordered_map<uint64_t, int> g_occ;  // (device, kernel id) -> resident CTAs per SM

// Resident CTAs of `kern` on the current device (all SMs).
template <typename Kern>
cudaError_t resident_ctas(Kern kern, uint64_t id, uint32_t smem, int* out,
                          int threads = WarpCfg<8>::NTHR) {
  DeviceInfo di;
  if (device_info(&di) != 0) return cudaErrorUnknown;
  int dev = 0;
  cudaError_t err = cudaGetDevice(&dev);
  if (err != cudaSuccess) return err;
  const uint64_t key = (uint64_t(dev) << 48) | id;
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = g_occ.find(key);
  int occ = 0;
  if (it == g_occ.end()) {
    if (int(smem) > di.smem_optin) return cudaErrorInvalidValue;
    err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (err != cudaSuccess) return err;
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, threads, smem);
    if (err != cudaSuccess) return err;
    if (occ < 1) occ = 1;
    g_occ[key] = occ;
  } else {
    occ = it->second;
  }
  *out = occ * di.sm_count;
  return cudaSuccess;
}

// Grid for n work units of one warp each: resident CTAs, at most one warp per unit.
int64_t warp_grid(int resident, int64_t n_units, int max_grid) {
  int64_t grid = (n_units + WarpCfg<8>::WARPS - 1) / WarpCfg<8>::WARPS;
  if (grid > resident) grid = resident;
  if (max_grid > 0 && grid > max_grid) grid = max_grid;
  return grid < 1 ? 1 : grid;
}

template <int UT, int EL, bool X3>
cudaError_t det(const DetectArgs& a, cudaStream_t s) {
  constexpr uint32_t smem = WarpCfg<UT>::TMA_SMEM;
  int res = 0;
  const uint64_t id = 0x100 | (UT << 2) | (EL << 1) | (X3 ? 1 : 0);
  cudaError_t err = resident_ctas(detect_warp_kernel<UT, EL, X3>, id, smem, &res);
  if (err != cudaSuccess) return err;
  const int64_t grid = warp_grid(res, a.n_inst, 0);
  detect_warp_kernel<UT, EL, X3><<<unsigned(grid), WarpCfg<UT>::NTHR, smem, s>>>(a);
  return cudaGetLastError();
}

template <int UT, int EL, bool X3>
cudaError_t pre(const PrecodeArgs& a, cudaStream_t s) {
  constexpr uint32_t smem = WarpCfg<UT>::PRE_SMEM;
  int res = 0;
  const uint64_t id = 0x200 | (UT << 2) | (EL << 1) | (X3 ? 1 : 0);
  cudaError_t err = resident_ctas(precode_warp_kernel<UT, EL, X3>, id, smem, &res);
  if (err != cudaSuccess) return err;
  const int64_t grid = warp_grid(res, a.n_inst, 0);
  precode_warp_kernel<UT, EL, X3><<<unsigned(grid), WarpCfg<UT>::NTHR, smem, s>>>(a);
  return cudaGetLastError();
}

template <int UT, int EL, bool X3>
cudaError_t batch(int op, const BatchArgs& b, int max_grid, cudaStream_t s, bool launch,
                  int* grid_out) {
  const uint32_t smem = op == 0 ? WarpCfg<UT>::SMEM : WarpCfg<UT>::PRE_SMEM;
  int res = 0;
  const uint64_t id = (op == 0 ? 0x400 : 0x800) | (UT << 2) | (EL << 1) | (X3 ? 1 : 0);
  cudaError_t err = op == 0 ? resident_ctas(detect_warp_batch_kernel<UT, EL, X3>, id, smem, &res)
                            : resident_ctas(precode_warp_batch_kernel<UT, EL, X3>, id, smem, &res);
  if (err != cudaSuccess) return err;
  const int64_t grid = warp_grid(res, b.n_work, max_grid);
  if (grid_out) *grid_out = int(grid);
  if (!launch) return cudaSuccess;
  if (op == 0)
    detect_warp_batch_kernel<UT, EL, X3><<<unsigned(grid), WarpCfg<UT>::NTHR, smem, s>>>(b);
  else
    precode_warp_batch_kernel<UT, EL, X3><<<unsigned(grid), WarpCfg<UT>::NTHR, smem, s>>>(b);
  return cudaGetLastError();
}

// Dispatch over (UT, EL, X3); F is called as F.template run<UT, EL, X3>().
template <class F>
cudaError_t dispatch(int UT, int el, bool x3, F f) {
  if (UT == 8) {
    if (el == EL_BF16) return x3 ? f.template run<8, EL_BF16, true>() : f.template run<8, EL_BF16, false>();
    return x3 ? f.template run<8, EL_F16, true>() : f.template run<8, EL_F16, false>();
  }
  if (UT == 16) {
    if (el == EL_BF16)
      return x3 ? f.template run<16, EL_BF16, true>() : f.template run<16, EL_BF16, false>();
    return x3 ? f.template run<16, EL_F16, true>() : f.template run<16, EL_F16, false>();
  }
  if (UT == 32) {
    if (el == EL_BF16)
      return x3 ? f.template run<32, EL_BF16, true>() : f.template run<32, EL_BF16, false>();
    return x3 ? f.template run<32, EL_F16, true>() : f.template run<32, EL_F16, false>();
  }
  return cudaErrorInvalidValue;
}

struct DetF {
  const DetectArgs& a;
  cudaStream_t s;
  template <int T, int E, bool X> cudaError_t run() { return det<T, E, X>(a, s); }
};
struct PreF {
  const PrecodeArgs& a;
  cudaStream_t s;
  template <int T, int E, bool X> cudaError_t run() { return pre<T, E, X>(a, s); }
};
struct BatchF {
  int op;
  const BatchArgs& b;
  int mg;
  cudaStream_t s;
  bool l;
  int* g;
  template <int T, int E, bool X> cudaError_t run() { return batch<T, E, X>(op, b, mg, s, l, g); }
};

}  // namespace

cudaError_t launch_detect_warp(int UT, int el, bool x3, const DetectArgs& a, cudaStream_t s) {
  return dispatch(UT < 8 ? 8 : UT, el, x3, DetF{a, s});
}

cudaError_t launch_precode_warp(int UT, int el, bool x3, const PrecodeArgs& a, cudaStream_t s) {
  return dispatch(UT < 8 ? 8 : UT, el, x3, PreF{a, s});
}

cudaError_t launch_batch_warp(int op, int UT, int el, bool x3, const BatchArgs& b, int max_grid,
                              cudaStream_t s, bool launch, int* grid_out) {
  return dispatch(UT < 8 ? 8 : UT, el, x3, BatchF{op, b, max_grid, s, launch, grid_out});
}

}  // namespace cgm
