// Launchers of the tensor-core kernels: padded user count 8, 16 or 32,
// FP16 or BF16 operands, one pass or hi+lo split.
#include <mutex>
#include <unordered_map>

#include "cg_tc.cuh"
#include "launch.cuh"

namespace cgm {

namespace {

std::mutex g_mu;
std::unordered_map<uint64_t, int> g_occ;
std::unordered_map<uint64_t, int> g_attr;

template <typename Kern>
cudaError_t prepare(Kern kern, uint64_t id, int nthr, uint32_t smem, int* occ_out) {
  DeviceInfo di;
  if (device_info(&di) != 0) return cudaErrorUnknown;
  if (int(smem) > di.smem_optin) return cudaErrorInvalidValue;
  int dev = 0;
  cudaError_t err = cudaGetDevice(&dev);
  if (err != cudaSuccess) return err;
  const uint64_t akey = (uint64_t(dev) << 48) | id;
  const uint64_t okey = (uint64_t(dev) << 56) ^ (id << 24) ^ smem;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_attr.count(akey)) {
    err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, di.smem_optin);
    if (err != cudaSuccess) return err;
    g_attr[akey] = 1;
  }
  auto it = g_occ.find(okey);
  if (it == g_occ.end()) {
    int occ = 0;
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, nthr, smem);
    if (err != cudaSuccess) return err;
    g_occ[okey] = occ < 1 ? 1 : occ;
    *occ_out = g_occ[okey] * di.sm_count;
  } else {
    *occ_out = it->second * di.sm_count;
  }
  return cudaSuccess;
}

template <int UT, int EL, bool X3, bool FULL>
cudaError_t det(const DetectArgs& a, cudaStream_t s, int* grid_out) {
  constexpr int NTHR = TcCfg<UT>::NTHR;
  const uint32_t smem = tc_detect_plan<UT>(a.B, a.U, a.R, a.exact).total;
  int slots = 0;
  const uint64_t id = 0x1000 | (UT << 3) | (EL << 2) | (X3 ? 2 : 0) | (FULL ? 1 : 0);
  cudaError_t err = prepare(detect_tc_kernel<UT, EL, X3, FULL>, id, NTHR, smem, &slots);
  if (err != cudaSuccess) return err;
  int64_t grid = slots < a.n_inst ? slots : a.n_inst;
  if (grid < 1) grid = 1;
  if (grid_out) *grid_out = int(grid);
  detect_tc_kernel<UT, EL, X3, FULL><<<unsigned(grid), NTHR, smem, s>>>(a);
  return cudaGetLastError();
}

template <int UT, int EL, bool X3, bool FULL>
cudaError_t pre(const PrecodeArgs& a, cudaStream_t s, int* grid_out) {
  constexpr int NTHR = TcCfg<UT>::NTHR;
  const uint32_t smem = tc_precode_plan<UT>(a.B, a.U, a.R).total;
  int slots = 0;
  const uint64_t id = 0x2000 | (UT << 3) | (EL << 2) | (X3 ? 2 : 0) | (FULL ? 1 : 0);
  cudaError_t err = prepare(precode_tc_kernel<UT, EL, X3, FULL>, id, NTHR, smem, &slots);
  if (err != cudaSuccess) return err;
  int64_t grid = slots < a.n_inst ? slots : a.n_inst;
  if (grid < 1) grid = 1;
  if (grid_out) *grid_out = int(grid);
  precode_tc_kernel<UT, EL, X3, FULL><<<unsigned(grid), NTHR, smem, s>>>(a);
  return cudaGetLastError();
}

// FULL instantiations: U equals the padded user count and B is a multiple of 8.
template <int UT, int EL, bool X3>
cudaError_t det_f(const DetectArgs& a, cudaStream_t s, int* g) {
  const bool full = a.U == UT && a.B % 8 == 0;
  return full ? det<UT, EL, X3, true>(a, s, g) : det<UT, EL, X3, false>(a, s, g);
}

template <int UT, int EL, bool X3>
cudaError_t pre_f(const PrecodeArgs& a, cudaStream_t s, int* g) {
  const bool full = a.U == UT && a.B % 8 == 0;
  return full ? pre<UT, EL, X3, true>(a, s, g) : pre<UT, EL, X3, false>(a, s, g);
}

template <int UT>
cudaError_t det_ut(int el, bool x3, const DetectArgs& a, cudaStream_t s, int* g) {
  if (el == EL_BF16)
    return x3 ? det_f<UT, EL_BF16, true>(a, s, g) : det_f<UT, EL_BF16, false>(a, s, g);
  return x3 ? det_f<UT, EL_F16, true>(a, s, g) : det_f<UT, EL_F16, false>(a, s, g);
}

template <int UT>
cudaError_t pre_ut(int el, bool x3, const PrecodeArgs& a, cudaStream_t s, int* g) {
  if (el == EL_BF16)
    return x3 ? pre_f<UT, EL_BF16, true>(a, s, g) : pre_f<UT, EL_BF16, false>(a, s, g);
  return x3 ? pre_f<UT, EL_F16, true>(a, s, g) : pre_f<UT, EL_F16, false>(a, s, g);
}

}  // namespace

uint32_t tc_detect_smem_bytes(int UT, int B, int U, int R, int exact) {
  switch (UT) {
    case 8: return tc_detect_plan<8>(B, U, R, exact).total;
    case 16: return tc_detect_plan<16>(B, U, R, exact).total;
    default: return tc_detect_plan<32>(B, U, R, exact).total;
  }
}

uint32_t tc_precode_smem_bytes(int UT, int B, int U, int R) {
  switch (UT) {
    case 8: return tc_precode_plan<8>(B, U, R).total;
    case 16: return tc_precode_plan<16>(B, U, R).total;
    default: return tc_precode_plan<32>(B, U, R).total;
  }
}

cudaError_t launch_detect_tc(int UT, int el, bool x3, const DetectArgs& a, cudaStream_t s,
                             int* grid_out) {
  switch (UT) {
    case 4:
    case 8: return det_ut<8>(el, x3, a, s, grid_out);
    case 16: return det_ut<16>(el, x3, a, s, grid_out);
    case 32: return det_ut<32>(el, x3, a, s, grid_out);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_precode_tc(int UT, int el, bool x3, const PrecodeArgs& a, cudaStream_t s,
                              int* grid_out) {
  switch (UT) {
    case 4:
    case 8: return pre_ut<8>(el, x3, a, s, grid_out);
    case 16: return pre_ut<16>(el, x3, a, s, grid_out);
    case 32: return pre_ut<32>(el, x3, a, s, grid_out);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace cgm

// ---------------------------------------------------------------------------
// Batched (plan) kernels
// ---------------------------------------------------------------------------

namespace cgm {

namespace {

template <int UT, int EL, bool X3, bool FULL>
cudaError_t batch_t(int op, const BatchArgs& b, int max_grid, cudaStream_t s, bool launch,
                    uint32_t* smem_out, int* grid_out) {
  constexpr int NTHR = TcCfg<UT>::NTHR;
  const uint32_t smem = op == 0 ? tc_detect_plan<UT>(b.PB, UT, b.PR, b.PEX).total
                                : tc_precode_plan<UT>(b.PB, UT, b.PR).total;
  int slots = 0;
  const uint64_t id = (op == 0 ? 0x4000 : 0x8000) | (UT << 3) | (EL << 2) | (X3 ? 2 : 0) |
                      (FULL ? 1 : 0);
  cudaError_t err = op == 0
                        ? prepare(detect_tc_batch_kernel<UT, EL, X3, FULL>, id, NTHR, smem, &slots)
                        : prepare(precode_tc_batch_kernel<UT, EL, X3, FULL>, id, NTHR, smem, &slots);
  if (err != cudaSuccess) return err;
  int64_t grid = slots < b.n_work ? slots : b.n_work;
  if (max_grid > 0 && grid > max_grid) grid = max_grid;
  if (grid < 1) grid = 1;
  if (smem_out) *smem_out = smem;
  if (grid_out) *grid_out = int(grid);
  if (!launch) return cudaSuccess;
  if (op == 0)
    detect_tc_batch_kernel<UT, EL, X3, FULL><<<unsigned(grid), NTHR, smem, s>>>(b);
  else
    precode_tc_batch_kernel<UT, EL, X3, FULL><<<unsigned(grid), NTHR, smem, s>>>(b);
  return cudaGetLastError();
}

template <int UT, int EL, bool X3>
cudaError_t batch_f(int op, bool full, const BatchArgs& b, int mg, cudaStream_t s, bool l,
                    uint32_t* sm, int* g) {
  return full ? batch_t<UT, EL, X3, true>(op, b, mg, s, l, sm, g)
              : batch_t<UT, EL, X3, false>(op, b, mg, s, l, sm, g);
}

template <int UT>
cudaError_t batch_ut(int op, int el, bool x3, bool full, const BatchArgs& b, int mg,
                     cudaStream_t s, bool l, uint32_t* sm, int* g) {
  if (el == EL_BF16)
    return x3 ? batch_f<UT, EL_BF16, true>(op, full, b, mg, s, l, sm, g)
              : batch_f<UT, EL_BF16, false>(op, full, b, mg, s, l, sm, g);
  return x3 ? batch_f<UT, EL_F16, true>(op, full, b, mg, s, l, sm, g)
            : batch_f<UT, EL_F16, false>(op, full, b, mg, s, l, sm, g);
}

}  // namespace

cudaError_t launch_batch_tc(int op, int UT, int el, bool x3, bool full, const BatchArgs& b,
                            int max_grid, cudaStream_t s, bool launch, uint32_t* smem_out,
                            int* grid_out) {
  if (b.PEX == 0) {  // warp-per-instance kernels
    if (smem_out) *smem_out = 0;
    return launch_batch_warp(op, UT, el, x3, b, max_grid, s, launch, grid_out);
  }
  if (op == 0 && UT <= 16) {  // exact tracker on the warp kernels, as the single calls
    if (smem_out) *smem_out = 0;
    return launch_batch_warp_exact(UT, el, x3, b, max_grid, s, launch, grid_out);
  }
  switch (UT) {
    case 4:
    case 8: return batch_ut<8>(op, el, x3, full, b, max_grid, s, launch, smem_out, grid_out);
    case 16: return batch_ut<16>(op, el, x3, full, b, max_grid, s, launch, smem_out, grid_out);
    case 32: return batch_ut<32>(op, el, x3, full, b, max_grid, s, launch, smem_out, grid_out);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace cgm
