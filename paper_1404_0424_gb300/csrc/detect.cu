// CG-D launchers: one fused kernel instantiation per padded user count.
#include <mutex>
#include <unordered_map>

#include "launch.cuh"

namespace cgm {

namespace {

std::mutex g_mu;
std::unordered_map<uint64_t, int> g_occ;  // (device, UT, smem) -> resident CTAs per SM
std::unordered_map<uint64_t, int> g_attr;  // (device, UT) -> smem attribute already raised

template <int UT>
cudaError_t launch_detect_t(const DetectArgs& a, cudaStream_t s, int* grid_out) {
  constexpr int NTHR = TileCfg<UT>::NTHR;
  const SmemPlan P = detect_plan<UT>(a.B, a.U, a.R, a.exact);
  DeviceInfo di;
  if (device_info(&di) != 0) return cudaErrorUnknown;
  if (int(P.total) > di.smem_optin) return cudaErrorInvalidValue;
  int dev = 0;
  cudaError_t err = cudaGetDevice(&dev);
  if (err != cudaSuccess) return err;
  const uint64_t akey = (uint64_t(dev) << 32) | uint64_t(UT);
  const uint64_t okey = (uint64_t(dev) << 40) | (uint64_t(UT) << 32) | P.total;
  int occ = 0;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_attr.count(akey)) {
      err = cudaFuncSetAttribute(detect_kernel<UT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 di.smem_optin);
      if (err != cudaSuccess) return err;
      g_attr[akey] = 1;
    }
    auto it = g_occ.find(okey);
    if (it == g_occ.end()) {
      err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, detect_kernel<UT>, NTHR, P.total);
      if (err != cudaSuccess) return err;
      if (occ < 1) occ = 1;
      g_occ[okey] = occ;
    } else {
      occ = it->second;
    }
  }
  int64_t grid = int64_t(di.sm_count) * occ;
  if (grid > a.n_inst) grid = a.n_inst;
  if (grid < 1) grid = 1;
  if (grid_out) *grid_out = int(grid);
  detect_kernel<UT><<<unsigned(grid), NTHR, P.total, s>>>(a);
  return cudaGetLastError();
}

}  // namespace

uint32_t detect_smem_bytes(int UT, int B, int U, int R, int exact) {
  switch (UT) {
    case 4: return detect_plan<4>(B, U, R, exact).total;
    case 8: return detect_plan<8>(B, U, R, exact).total;
    case 16: return detect_plan<16>(B, U, R, exact).total;
    default: return detect_plan<32>(B, U, R, exact).total;
  }
}

cudaError_t launch_detect(int UT, const DetectArgs& a, cudaStream_t s, int* grid_out) {
  switch (UT) {
    case 4: return launch_detect_t<4>(a, s, grid_out);
    case 8: return launch_detect_t<8>(a, s, grid_out);
    case 16: return launch_detect_t<16>(a, s, grid_out);
    case 32: return launch_detect_t<32>(a, s, grid_out);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace cgm
