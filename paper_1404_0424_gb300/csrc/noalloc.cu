// cg_batch_run_static: the batched problems of cg_plan_* run without any
// allocation. The work tables that a plan keeps in cudaMalloc'd memory live
// here in one file-scope device array instead, so callers that must not
// allocate (see cgmimo.h) can still run uneven batches.
#include <cstring>
#include <mutex>

#include "cgmimo.h"
#include "host_checks.h"
#include "launch.cuh"

using namespace cgm;

namespace {

constexpr size_t kDescBytes = sizeof(cg_desc) * CG_STATIC_MAX_PROBLEMS;
constexpr size_t kWorkOff = (kDescBytes + 255) & ~size_t(255);
constexpr size_t kWorkBytes = sizeof(int2) * CG_STATIC_MAX_INSTANCES;
// 2 operations x 3 padded user counts x FULL or not, then exact-tracker
// detection with 8, 16 or 32 padded users x FULL or not
constexpr int kMaxBins = 18;
constexpr size_t kCountOff = (kWorkOff + kWorkBytes + 255) & ~size_t(255);
constexpr size_t kScratchBytes = kCountOff + sizeof(unsigned long long) * kMaxBins;
static_assert(kScratchBytes <= (size_t(1) << 20), "static scratch stays within 1 MiB");

// The scratch: descriptors, then (problem, instance) work units grouped by
// bin, then one claim counter per bin. Every GPU that loads the library
// holds it until the process exits.
static __device__ __align__(256) unsigned char g_static_scratch[kScratchBytes];

std::mutex g_mu;                            // serialises the host side of calls
int2 g_host_work[CG_STATIC_MAX_INSTANCES];  // host staging of the work units

// Device address of the scratch on the current device. It is looked up on
// every call: once the module is loaded this is a table lookup, and a
// cached address would go stale if the device's context were torn down and
// the module loaded again elsewhere (cudaDeviceReset).
int scratch_address(unsigned char** out) {
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || p == nullptr) return CG_ECUDA;
  *out = static_cast<unsigned char*>(p);
  return CG_OK;
}

int check_static_desc(const cg_desc& d) {
  cg_params p{};
  p.B = d.B;
  p.U = d.U;
  p.qam_bits = d.qam_bits;
  p.K = d.K;
  p.R = d.R;
  p.N0 = d.N0;
  p.Es = d.Es;
  p.sinr_mode = d.sinr_mode;
  p.amul_mode = CG_AMUL_EXPLICIT;
  p.precision = CG_PREC_FP16X3;
  if (d.n_inst < 0) return CG_EINVAL;
  if (d.op == CG_OP_DETECT)
    return check_detect(&p, d.n_inst, d.H, d.in, d.out, d.mu, d.rho, d.aux, d.status);
  if (d.op == CG_OP_PRECODE) return check_precode(&p, d.n_inst, d.H, d.in, d.out, d.aux, d.status);
  return CG_EINVAL;
}

struct StaticBin {
  int op, UT, full, PB, PR, PEX;
  int64_t count, off;
};

// Bin of a problem: (operation, padded users, FULL) for the approximate
// tracker and precoding, and bins of their own for exact-tracker detection,
// as cg_plan_create keys them, so that an exact problem never moves the
// approximate ones of its padded user count onto another kernel.
int bin_of(const cg_desc& d, int* UT, int* full) {
  *UT = padded_users(d.U) < 8 ? 8 : padded_users(d.U);
  *full = (d.U == *UT && d.B % 8 == 0) ? 1 : 0;
  const int uti = *UT == 8 ? 0 : *UT == 16 ? 1 : 2;
  if (d.op == CG_OP_DETECT && d.sinr_mode == CG_SINR_EXACT) return 12 + uti * 2 + *full;
  return (d.op * 3 + uti) * 2 + *full;
}

}  // namespace

extern "C" int cg_batch_run_static(const cg_desc* descs, int64_t n, int32_t precision,
                                   void* stream) {
  if (n < 0 || (n > 0 && descs == nullptr)) return CG_EINVAL;
  if (precision < CG_PREC_BF16 || precision > CG_PREC_FP16X3) return CG_EINVAL;
  if (n > CG_STATIC_MAX_PROBLEMS) return CG_ETOOBIG;
  int64_t units = 0;
  for (int64_t i = 0; i < n; ++i) {
    const int rc = check_static_desc(descs[i]);
    if (rc != CG_OK) return rc;
    units += descs[i].n_inst;
    if (units > CG_STATIC_MAX_INSTANCES) return CG_ETOOBIG;
  }
  if (units == 0) return CG_OK;
  std::lock_guard<std::mutex> lk(g_mu);
  unsigned char* base = nullptr;
  int rc = scratch_address(&base);
  if (rc != CG_OK) return rc;

  // bins: count, offsets, then fill the host staging of the work units;
  // problems without instances take no part (they size no bin)
  StaticBin bins[kMaxBins];
  for (int b = 0; b < kMaxBins; ++b)
    bins[b] = StaticBin{b < 12 ? b / 6 : CG_OP_DETECT, 0, b & 1, 0, 0, 0, 0, 0};
  for (int64_t i = 0; i < n; ++i) {
    if (descs[i].n_inst == 0) continue;
    int UT, full;
    StaticBin& b = bins[bin_of(descs[i], &UT, &full)];
    b.UT = UT;
    b.PB = b.PB > descs[i].B ? b.PB : descs[i].B;
    b.PR = b.PR > descs[i].R ? b.PR : descs[i].R;
    if (descs[i].op == CG_OP_DETECT && descs[i].sinr_mode == CG_SINR_EXACT) b.PEX = 1;
    b.count += descs[i].n_inst;
  }
  const int el = (precision == CG_PREC_BF16 || precision == CG_PREC_BF16X3) ? 0 : 1;
  const bool x3 = precision == CG_PREC_BF16X3 || precision == CG_PREC_FP16X3;
  // every bin's launch shape is checked before anything is enqueued
  for (int b = 0; b < kMaxBins; ++b) {
    if (bins[b].count == 0) continue;
    BatchArgs a{};
    a.n_work = bins[b].count;
    a.PB = bins[b].PB;
    a.PR = bins[b].PR;
    a.PEX = bins[b].PEX;
    const cudaError_t err = launch_batch_tc(bins[b].op, bins[b].UT, el, x3, bins[b].full != 0,
                                            a, 0, nullptr, false, nullptr, nullptr);
    if (err != cudaSuccess) return err == cudaErrorInvalidValue ? CG_EINVAL : CG_ECUDA;
  }
  int64_t off = 0;
  for (int b = 0; b < kMaxBins; ++b) {
    bins[b].off = off;
    off += bins[b].count;
  }
  int64_t fill[kMaxBins];
  for (int b = 0; b < kMaxBins; ++b) fill[b] = bins[b].off;
  for (int64_t i = 0; i < n; ++i) {
    int UT, full;
    const int b = bin_of(descs[i], &UT, &full);
    for (int64_t k = 0; k < descs[i].n_inst; ++k)
      g_host_work[fill[b]++] = make_int2(int(i), int(k));
  }

  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cg_desc* d_desc = reinterpret_cast<cg_desc*>(base);
  int2* d_work = reinterpret_cast<int2*>(base + kWorkOff);
  unsigned long long* d_count = reinterpret_cast<unsigned long long*>(base + kCountOff);
  // Pageable sources: each copy has consumed its host data when it returns.
  if (cudaMemcpyAsync(d_desc, descs, sizeof(cg_desc) * size_t(n), cudaMemcpyHostToDevice, s) !=
          cudaSuccess ||
      cudaMemcpyAsync(d_work, g_host_work, sizeof(int2) * size_t(units), cudaMemcpyHostToDevice,
                      s) != cudaSuccess ||
      cudaMemsetAsync(d_count, 0, sizeof(unsigned long long) * kMaxBins, s) != cudaSuccess)
    return CG_ECUDA;
  for (int b = 0; b < kMaxBins; ++b) {
    if (bins[b].count == 0) continue;
    BatchArgs a{};
    a.desc = d_desc;
    a.work = d_work + bins[b].off;
    a.n_work = bins[b].count;
    a.counter = d_count + b;
    a.PB = bins[b].PB;
    a.PR = bins[b].PR;
    a.PEX = bins[b].PEX;
    const cudaError_t err = launch_batch_tc(bins[b].op, bins[b].UT, el, x3, bins[b].full != 0, a,
                                            0, s, true, nullptr, nullptr);
    if (err != cudaSuccess) return err == cudaErrorInvalidValue ? CG_EINVAL : CG_ECUDA;
  }
  return CG_OK;
}
