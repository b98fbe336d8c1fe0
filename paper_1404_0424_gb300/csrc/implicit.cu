// Launchers of the implicit-product FP32 kernels and their CGLS variants
// (cg_implicit.cuh).
#include <mutex>
#include <unordered_map>

#include "cg_implicit.cuh"
#include "launch.cuh"

namespace cgm {

namespace {

std::mutex g_mu;
std::unordered_map<uint64_t, int> g_occ;   // (device, kernel, smem) -> resident CTAs per SM
std::unordered_map<uint64_t, int> g_attr;  // (device, kernel) -> smem attribute raised

template <typename Kern>
cudaError_t launch_one(Kern kern, uint64_t id, int nthr, uint32_t smem, int64_t n_inst,
                       int* grid_out) {
  DeviceInfo di;
  if (device_info(&di) != 0) return cudaErrorUnknown;
  if (int(smem) > di.smem_optin) return cudaErrorInvalidValue;
  int dev = 0;
  cudaError_t err = cudaGetDevice(&dev);
  if (err != cudaSuccess) return err;
  const uint64_t akey = (uint64_t(dev) << 32) | id;
  const uint64_t okey = (uint64_t(dev) << 48) ^ (id << 24) ^ smem;
  int occ = 0;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_attr.count(akey)) {
      err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, di.smem_optin);
      if (err != cudaSuccess) return err;
      g_attr[akey] = 1;
    }
    auto it = g_occ.find(okey);
    if (it == g_occ.end()) {
      err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, nthr, smem);
      if (err != cudaSuccess) return err;
      if (occ < 1) occ = 1;
      g_occ[okey] = occ;
    } else {
      occ = it->second;
    }
  }
  int64_t grid = int64_t(di.sm_count) * occ;
  if (grid > n_inst) grid = n_inst;
  if (grid < 1) grid = 1;
  *grid_out = int(grid);
  return cudaSuccess;
}

template <int UT, bool CGLS>
cudaError_t det(const DetectArgs& a, cudaStream_t s) {
  constexpr int NTHR = TileCfg<UT>::NTHR;
  const uint32_t smem = implicit_plan<UT>(a.B, a.U, a.R, true, CGLS).total;
  int grid = 0;
  const uint64_t id = (CGLS ? 0x300 : 0x100) | UT;
  cudaError_t err =
      launch_one(detect_implicit_kernel<UT, CGLS>, id, NTHR, smem, a.n_inst, &grid);
  if (err != cudaSuccess) return err;
  detect_implicit_kernel<UT, CGLS><<<unsigned(grid), NTHR, smem, s>>>(a);
  return cudaGetLastError();
}

template <int UT, bool CGLS>
cudaError_t pre(const PrecodeArgs& a, cudaStream_t s) {
  constexpr int NTHR = TileCfg<UT>::NTHR;
  const uint32_t smem = implicit_plan<UT>(a.B, a.U, a.R, false, CGLS).total;
  int grid = 0;
  const uint64_t id = (CGLS ? 0x400 : 0x200) | UT;
  cudaError_t err =
      launch_one(precode_implicit_kernel<UT, CGLS>, id, NTHR, smem, a.n_inst, &grid);
  if (err != cudaSuccess) return err;
  precode_implicit_kernel<UT, CGLS><<<unsigned(grid), NTHR, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_detect_implicit(int UT, const DetectArgs& a, cudaStream_t s, bool cgls) {
  switch (UT) {
    case 4: return cgls ? det<4, true>(a, s) : det<4, false>(a, s);
    case 8: return cgls ? det<8, true>(a, s) : det<8, false>(a, s);
    case 16: return cgls ? det<16, true>(a, s) : det<16, false>(a, s);
    case 32: return cgls ? det<32, true>(a, s) : det<32, false>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_precode_implicit(int UT, const PrecodeArgs& a, cudaStream_t s, bool cgls) {
  switch (UT) {
    case 4: return cgls ? pre<4, true>(a, s) : pre<4, false>(a, s);
    case 8: return cgls ? pre<8, true>(a, s) : pre<8, false>(a, s);
    case 16: return cgls ? pre<16, true>(a, s) : pre<16, false>(a, s);
    case 32: return cgls ? pre<32, true>(a, s) : pre<32, false>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace cgm
