// C ABI of libcgmimo: argument validation, dispatch to the fused kernels,
// and the chunked host-memory variants.
#include <cmath>
#include <cstdint>
#include <atomic>
#include <cstring>
#include <mutex>

#include <cudaTypedefs.h>

#include "cgmimo.h"
#include "host_checks.h"
#include "launch.cuh"

namespace cgm {

namespace {
std::mutex g_dev_mu;
// Limit of the FP32 kernels' wait for an instance's bulk copies (ns).
std::atomic<int64_t> g_wait_ns{int64_t(WAIT_TIMEOUT_NS)};
DeviceInfo g_dev[64];
bool g_dev_ok[64] = {false};
}  // namespace

int device_info(DeviceInfo* out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return -1;
  std::lock_guard<std::mutex> lk(g_dev_mu);
  if (!g_dev_ok[dev]) {
    DeviceInfo d;
    if (cudaDeviceGetAttribute(&d.sm_count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      return -1;
    if (cudaDeviceGetAttribute(&d.smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) !=
        cudaSuccess)
      return -1;
    if (cudaDeviceGetAttribute(&d.smem_per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) !=
        cudaSuccess)
      return -1;
    if (cudaDeviceGetAttribute(&d.smem_reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev) !=
        cudaSuccess)
      return -1;
    g_dev[dev] = d;
    g_dev_ok[dev] = true;
  }
  *out = g_dev[dev];
  return 0;
}

}  // namespace cgm

using namespace cgm;

namespace {

// Modes implemented by this build: the exact tracker needs the Gram, so it
// does not combine with the implicit product.
int check_supported(const cg_params* p) {
  if ((p->amul_mode == CG_AMUL_IMPLICIT || p->amul_mode == CG_AMUL_CGLS) &&
      p->sinr_mode == CG_SINR_EXACT)
    return CG_ENOTSUP;
  return CG_OK;
}

// cuTensorMapEncodeTiled, taken from the driver through the runtime once
// (null if the driver does not offer it: the calls then use cp.async).
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      f = nullptr;
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
  }();
  return fn;
}

// 3-D tiled map of n matrices of rows x cols complex values stored as FP32
// pairs: dims {2 cols, rows, n}, box {bx, by, 1} elements, zero fill.
bool encode_map(CUtensorMap* m, const void* base, int64_t n, int rows, int cols, int bx, int by,
                CUtensorMapSwizzle sw) {
  auto enc = tensor_map_encoder();
  if (enc == nullptr || n > INT32_MAX) return false;
  const cuuint64_t dims[3] = {cuuint64_t(2 * cols), cuuint64_t(rows), cuuint64_t(n)};
  const cuuint64_t strides[2] = {cuuint64_t(8) * cols, cuuint64_t(8) * cols * rows};
  const cuuint32_t box[3] = {cuuint32_t(bx), cuuint32_t(by), 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void*>(base), dims, strides, box,
             estr, CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Tensor maps of the warp kernels' staging (DetectArgs::tmH, tmY): H boxes
// of 8 antennas x min(UT, 16) users, Y boxes of 16 rows x 8 antennas. Only
// for the layout the vector path reads (U == UT, B even, 16-byte aligned).
bool detect_maps(DetectArgs* a, int UT) {
  if (a->U != UT || a->B % 2 || !aligned(a->H, 16) || !aligned(a->Y, 16)) return false;
  const int ub = UT < 16 ? UT : 16;
  return encode_map(&a->tmH, a->H, a->n_inst, a->B, a->U, 2 * ub, 8,
                    UT == 8 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B) &&
         encode_map(&a->tmY, a->Y, a->n_inst, a->R, a->B, 16, 16, CU_TENSOR_MAP_SWIZZLE_NONE);
}

// Tensor-core operand type (0 = BF16, 1 = FP16) and hi+lo split of a precision mode.
void tc_mode(int precision, int* el, bool* x3) {
  *el = (precision == CG_PREC_BF16 || precision == CG_PREC_BF16X3) ? 0 : 1;
  *x3 = precision == CG_PREC_BF16X3 || precision == CG_PREC_FP16X3;
}

int detect_device(const cg_params* p, int64_t n_inst, const void* H, const void* Y, void* xhat,
                  float* mu, float* rho, float* llr, int32_t* status, cudaStream_t s) {
  DetectArgs a{};
  a.H = static_cast<const float2*>(H);
  a.Y = static_cast<const float2*>(Y);
  a.xhat = static_cast<float2*>(xhat);
  a.mu = mu;
  a.rho = rho;
  a.llr = llr;
  a.status = status;
  a.n_inst = n_inst;
  a.B = p->B;
  a.U = p->U;
  a.R = p->R;
  a.K = p->K;
  a.q = p->qam_bits;
  a.N0 = p->N0;
  a.Es = p->Es;
  a.sigma = p->N0 / p->Es;
  a.exact = p->sinr_mode == CG_SINR_EXACT;
  a.bulk = (p->B % 2 == 0) && aligned(H, 16) && aligned(Y, 16);
  a.wait_ns = uint64_t(g_wait_ns.load(std::memory_order_relaxed));
  cudaError_t err;
  if (p->amul_mode == CG_AMUL_CGLS) {
    err = launch_detect_implicit(padded_users(p->U), a, s, true);
  } else if (use_implicit(p->amul_mode, p->precision, p->K, p->R, p->U, a.exact)) {
    err = launch_detect_implicit(padded_users(p->U), a, s, false);
  } else if (p->precision == CG_PREC_FP32) {
    err = launch_detect(padded_users(p->U), a, s, nullptr);
  } else {
    int el;
    bool x3;
    tc_mode(p->precision, &el, &x3);
    const int UT = padded_users(p->U);
    if (!a.exact) a.tma = detect_maps(&a, UT) ? 1 : 0;
    err = a.exact ? launch_detect_warp_exact(UT, el, x3, a, s)
                  : launch_detect_warp(UT, el, x3, a, s);
  }
  if (err == cudaErrorInvalidValue) return CG_EINVAL;
  return err == cudaSuccess ? CG_OK : CG_ECUDA;
}

int precode_device(const cg_params* p, int64_t n_inst, const void* H, const void* T, void* q,
                   float* qnorm, int32_t normalize, int32_t* status, cudaStream_t s) {
  PrecodeArgs a{};
  a.H = static_cast<const float2*>(H);
  a.T = static_cast<const float2*>(T);
  a.q = static_cast<float2*>(q);
  a.qnorm = qnorm;
  a.status = status;
  a.n_inst = n_inst;
  a.B = p->B;
  a.U = p->U;
  a.R = p->R;
  a.K = p->K;
  a.sigma = p->N0 / p->Es;
  a.normalize = normalize != 0;
  a.bulk_h = ((p->B * p->U) % 2 == 0) && aligned(H, 16);
  a.bulk_t = ((p->R * p->U) % 2 == 0) && aligned(T, 16);
  a.wait_ns = uint64_t(g_wait_ns.load(std::memory_order_relaxed));
  cudaError_t err;
  if (p->amul_mode == CG_AMUL_CGLS) {
    err = launch_precode_implicit(padded_users(p->U), a, s, true);
  } else if (use_implicit(p->amul_mode, p->precision, p->K, p->R, p->U, false)) {
    err = launch_precode_implicit(padded_users(p->U), a, s, false);
  } else if (p->precision == CG_PREC_FP32) {
    err = launch_precode(padded_users(p->U), a, s, nullptr);
  } else {
    int el;
    bool x3;
    tc_mode(p->precision, &el, &x3);
    const int UT = padded_users(p->U);
    err = launch_precode_warp(UT, el, x3, a, s);
  }
  if (err == cudaErrorInvalidValue) return CG_EINVAL;
  return err == cudaSuccess ? CG_OK : CG_ECUDA;
}

// ---------------------------------------------------------------------------
// Workspace of the host-memory variants: one device buffer and two streams
// per device, used by one call at a time.
// ---------------------------------------------------------------------------

#ifndef CGM_HOST_STREAMS
#define CGM_HOST_STREAMS 2
#endif
// Chunks in flight in the host-memory variants: chunk k runs on stream
// k % kHostStreams in buffer set k % kHostStreams, so several host-to-device
// and device-to-host copies proceed at once on the copy engines.
constexpr int kHostStreams = CGM_HOST_STREAMS;

struct HostWorkspace {
  void* d = nullptr;
  size_t bytes = 0;
  cudaStream_t st[kHostStreams] = {};
  cudaEvent_t ready = nullptr;
};

std::mutex g_ws_mu;
HostWorkspace g_ws[64];

constexpr size_t kChunkBytes = size_t(64) << 20;  // inputs + outputs of one chunk

size_t up256(size_t x) { return (x + 255) & ~size_t(255); }

int workspace_acquire(size_t need, HostWorkspace** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return CG_ECUDA;
  HostWorkspace& w = g_ws[dev];
  if (w.st[0] == nullptr) {
    for (int i = 0; i < kHostStreams; ++i)
      if (cudaStreamCreateWithFlags(&w.st[i], cudaStreamNonBlocking) != cudaSuccess)
        return CG_ECUDA;
    if (cudaEventCreateWithFlags(&w.ready, cudaEventDisableTiming) != cudaSuccess)
      return CG_ECUDA;
  }
  if (w.bytes < need) {
    if (w.d != nullptr) cudaFree(w.d);
    w.d = nullptr;
    w.bytes = 0;
    if (cudaMalloc(&w.d, need) != cudaSuccess) return CG_ENOMEM;
    w.bytes = need;
  }
  *out = &w;
  return CG_OK;
}

// Makes the workspace streams wait for earlier work on the caller's stream.
int order_after(HostWorkspace* w, cudaStream_t user) {
  if (cudaEventRecord(w->ready, user) != cudaSuccess) return CG_ECUDA;
  for (int i = 0; i < kHostStreams; ++i)
    if (cudaStreamWaitEvent(w->st[i], w->ready, 0) != cudaSuccess) return CG_ECUDA;
  return CG_OK;
}

int finish(HostWorkspace* w, int rc) {
  for (int i = 0; i < kHostStreams; ++i)
    if (cudaStreamSynchronize(w->st[i]) != cudaSuccess && rc == CG_OK) rc = CG_ECUDA;
  return rc;
}

cudaError_t h2d(void* dst, const void* src, size_t n, cudaStream_t s) {
  return n ? cudaMemcpyAsync(dst, src, n, cudaMemcpyHostToDevice, s) : cudaSuccess;
}

cudaError_t d2h(void* dst, const void* src, size_t n, cudaStream_t s) {
  return n ? cudaMemcpyAsync(dst, src, n, cudaMemcpyDeviceToHost, s) : cudaSuccess;
}

}  // namespace

extern "C" {

int cg_set_wait_limit(int64_t timeout_ns) {
  if (timeout_ns < 0 || timeout_ns > int64_t(60) * 1000000000) return CG_EINVAL;
  g_wait_ns.store(timeout_ns == 0 ? int64_t(WAIT_TIMEOUT_NS) : timeout_ns,
                  std::memory_order_relaxed);
  return CG_OK;
}

int cg_detect(const cg_params* p, int64_t n_inst, const void* H, const void* Y, void* xhat,
              float* mu, float* rho, float* llr, int32_t* status, void* stream) {
  int rc = check_detect(p, n_inst, H, Y, xhat, mu, rho, llr, status);
  if (rc != CG_OK || n_inst == 0) return rc;
  if ((rc = check_supported(p)) != CG_OK) return rc;
  return detect_device(p, n_inst, H, Y, xhat, mu, rho, llr, status,
                       static_cast<cudaStream_t>(stream));
}

int cg_precode(const cg_params* p, int64_t n_inst, const void* H, const void* T, void* q,
               float* qnorm, int32_t normalize, int32_t* status, void* stream) {
  int rc = check_precode(p, n_inst, H, T, q, qnorm, status);
  if (rc != CG_OK || n_inst == 0) return rc;
  if ((rc = check_supported(p)) != CG_OK) return rc;
  return precode_device(p, n_inst, H, T, q, qnorm, normalize, status,
                        static_cast<cudaStream_t>(stream));
}

namespace {

// Checks shared by the Neumann entry points: K terms in [1, CG_NEUMANN_K_MAX]
// and a tensor-core precision; the shape and pointer checks are those of CG
// (with K = 1, since the series has no K <= U bound).
int check_neumann(const cg_params* p, cg_params* shape) {
  if (p == nullptr) return CG_EINVAL;
  if (p->K < 1 || p->K > CG_NEUMANN_K_MAX) return CG_EINVAL;
  if (p->precision == CG_PREC_FP32) return CG_ENOTSUP;
  if (p->precision < CG_PREC_BF16 || p->precision > CG_PREC_FP16X3) return CG_EINVAL;
  *shape = *p;
  shape->K = 1;
  shape->sinr_mode = CG_SINR_APPROX;
  shape->amul_mode = CG_AMUL_EXPLICIT;
  return CG_OK;
}

}  // namespace

int cg_neumann_detect(const cg_params* p, int64_t n_inst, const void* H, const void* Y,
                      void* xhat, int32_t* status, void* stream) {
  cg_params shape;
  int rc = check_neumann(p, &shape);
  if (rc != CG_OK) return rc;
  if (xhat == nullptr) return CG_EINVAL;
  rc = check_detect(&shape, n_inst, H, Y, xhat, nullptr, nullptr, nullptr, status);
  if (rc != CG_OK || n_inst == 0) return rc;
  DetectArgs a{};
  a.H = static_cast<const float2*>(H);
  a.Y = static_cast<const float2*>(Y);
  a.xhat = static_cast<float2*>(xhat);
  a.status = status;
  a.n_inst = n_inst;
  a.B = p->B;
  a.U = p->U;
  a.R = p->R;
  a.K = p->K;
  a.q = p->qam_bits;
  a.N0 = p->N0;
  a.Es = p->Es;
  a.sigma = p->N0 / p->Es;
  a.bulk = (p->B % 2 == 0) && aligned(H, 16) && aligned(Y, 16);
  int el;
  bool x3;
  tc_mode(p->precision, &el, &x3);
  const cudaError_t err =
      launch_neumann_detect(padded_users(p->U), el, x3, a, static_cast<cudaStream_t>(stream));
  if (err == cudaErrorInvalidValue) return CG_EINVAL;
  return err == cudaSuccess ? CG_OK : CG_ECUDA;
}

int cg_neumann_precode(const cg_params* p, int64_t n_inst, const void* H, const void* T, void* q,
                       float* qnorm, int32_t normalize, int32_t* status, void* stream) {
  cg_params shape;
  int rc = check_neumann(p, &shape);
  if (rc != CG_OK) return rc;
  rc = check_precode(&shape, n_inst, H, T, q, qnorm, status);
  if (rc != CG_OK || n_inst == 0) return rc;
  PrecodeArgs a{};
  a.H = static_cast<const float2*>(H);
  a.T = static_cast<const float2*>(T);
  a.q = static_cast<float2*>(q);
  a.qnorm = qnorm;
  a.status = status;
  a.n_inst = n_inst;
  a.B = p->B;
  a.U = p->U;
  a.R = p->R;
  a.K = p->K;
  a.sigma = p->N0 / p->Es;
  a.normalize = normalize != 0;
  a.bulk_h = ((p->B * p->U) % 2 == 0) && aligned(H, 16);
  a.bulk_t = ((p->R * p->U) % 2 == 0) && aligned(T, 16);
  int el;
  bool x3;
  tc_mode(p->precision, &el, &x3);
  const cudaError_t err =
      launch_neumann_precode(padded_users(p->U), el, x3, a, static_cast<cudaStream_t>(stream));
  if (err == cudaErrorInvalidValue) return CG_EINVAL;
  return err == cudaSuccess ? CG_OK : CG_ECUDA;
}

int cg_detect_host(const cg_params* p, int64_t n_inst, const void* H, const void* Y, void* xhat,
                   float* mu, float* rho, float* llr, int32_t* status, void* stream) {
  int rc = check_detect(p, n_inst, H, Y, xhat, mu, rho, llr, status);
  if (rc != CG_OK || n_inst == 0) return rc;
  if ((rc = check_supported(p)) != CG_OK) return rc;
  const size_t B = p->B, U = p->U, R = p->R, q = p->qam_bits;
  const size_t bH = B * U * 8, bY = R * B * 8;
  const size_t bX = xhat ? R * U * 8 : 0, bM = mu ? R * U * 4 : 0, bR = rho ? R * U * 4 : 0;
  const size_t bL = llr ? R * U * q * 4 : 0, bS = status ? 4 : 0;
  const size_t per = bH + bY + bX + bM + bR + bL + bS;
  int64_t chunk = int64_t(kChunkBytes / per);
  if (chunk < 1) chunk = 1;
  if (chunk > n_inst) chunk = n_inst;
  const size_t c = size_t(chunk);
  const size_t oH = 0, oY = up256(oH + c * bH), oX = up256(oY + c * bY), oM = up256(oX + c * bX);
  const size_t oR = up256(oM + c * bM), oL = up256(oR + c * bR), oS = up256(oL + c * bL);
  const size_t set = up256(oS + c * bS);
  std::lock_guard<std::mutex> lk(g_ws_mu);
  HostWorkspace* w = nullptr;
  if ((rc = workspace_acquire(kHostStreams * set, &w)) != CG_OK) return rc;
  if ((rc = order_after(w, static_cast<cudaStream_t>(stream))) != CG_OK) return rc;
  const char* hH = static_cast<const char*>(H);
  const char* hY = static_cast<const char*>(Y);
  int k = 0;
  for (int64_t off = 0; off < n_inst && rc == CG_OK; off += chunk, ++k) {
    const size_t nc = size_t(n_inst - off < chunk ? n_inst - off : chunk);
    cudaStream_t s = w->st[k % kHostStreams];
    char* base = static_cast<char*>(w->d) + (k % kHostStreams) * set;
    if (h2d(base + oH, hH + off * bH, nc * bH, s) != cudaSuccess ||
        h2d(base + oY, hY + off * bY, nc * bY, s) != cudaSuccess) {
      rc = CG_ECUDA;
      break;
    }
    rc = detect_device(p, int64_t(nc), base + oH, base + oY, xhat ? base + oX : nullptr,
                       mu ? reinterpret_cast<float*>(base + oM) : nullptr,
                       rho ? reinterpret_cast<float*>(base + oR) : nullptr,
                       llr ? reinterpret_cast<float*>(base + oL) : nullptr,
                       status ? reinterpret_cast<int32_t*>(base + oS) : nullptr, s);
    if (rc != CG_OK) break;
    if (d2h(static_cast<char*>(xhat) + off * bX, base + oX, nc * bX, s) != cudaSuccess ||
        d2h(reinterpret_cast<char*>(mu) + off * bM, base + oM, nc * bM, s) != cudaSuccess ||
        d2h(reinterpret_cast<char*>(rho) + off * bR, base + oR, nc * bR, s) != cudaSuccess ||
        d2h(reinterpret_cast<char*>(llr) + off * bL, base + oL, nc * bL, s) != cudaSuccess ||
        d2h(reinterpret_cast<char*>(status) + off * bS, base + oS, nc * bS, s) != cudaSuccess)
      rc = CG_ECUDA;
  }
  return finish(w, rc);
}

int cg_precode_host(const cg_params* p, int64_t n_inst, const void* H, const void* T, void* q,
                    float* qnorm, int32_t normalize, int32_t* status, void* stream) {
  int rc = check_precode(p, n_inst, H, T, q, qnorm, status);
  if (rc != CG_OK || n_inst == 0) return rc;
  if ((rc = check_supported(p)) != CG_OK) return rc;
  const size_t B = p->B, U = p->U, R = p->R;
  const size_t bH = B * U * 8, bT = R * U * 8, bQ = R * B * 8;
  const size_t bN = qnorm ? R * 4 : 0, bS = status ? 4 : 0;
  const size_t per = bH + bT + bQ + bN + bS;
  int64_t chunk = int64_t(kChunkBytes / per);
  if (chunk < 1) chunk = 1;
  if (chunk > n_inst) chunk = n_inst;
  const size_t c = size_t(chunk);
  const size_t oH = 0, oT = up256(oH + c * bH), oQ = up256(oT + c * bT), oN = up256(oQ + c * bQ);
  const size_t oS = up256(oN + c * bN);
  const size_t set = up256(oS + c * bS);
  std::lock_guard<std::mutex> lk(g_ws_mu);
  HostWorkspace* w = nullptr;
  if ((rc = workspace_acquire(kHostStreams * set, &w)) != CG_OK) return rc;
  if ((rc = order_after(w, static_cast<cudaStream_t>(stream))) != CG_OK) return rc;
  const char* hH = static_cast<const char*>(H);
  const char* hT = static_cast<const char*>(T);
  int k = 0;
  for (int64_t off = 0; off < n_inst && rc == CG_OK; off += chunk, ++k) {
    const size_t nc = size_t(n_inst - off < chunk ? n_inst - off : chunk);
    cudaStream_t s = w->st[k % kHostStreams];
    char* base = static_cast<char*>(w->d) + (k % kHostStreams) * set;
    if (h2d(base + oH, hH + off * bH, nc * bH, s) != cudaSuccess ||
        h2d(base + oT, hT + off * bT, nc * bT, s) != cudaSuccess) {
      rc = CG_ECUDA;
      break;
    }
    rc = precode_device(p, int64_t(nc), base + oH, base + oT, base + oQ,
                        qnorm ? reinterpret_cast<float*>(base + oN) : nullptr, normalize,
                        status ? reinterpret_cast<int32_t*>(base + oS) : nullptr, s);
    if (rc != CG_OK) break;
    if (d2h(static_cast<char*>(q) + off * bQ, base + oQ, nc * bQ, s) != cudaSuccess ||
        d2h(reinterpret_cast<char*>(qnorm) + off * bN, base + oN, nc * bN, s) != cudaSuccess ||
        d2h(reinterpret_cast<char*>(status) + off * bS, base + oS, nc * bS, s) != cudaSuccess)
      rc = CG_ECUDA;
  }
  return finish(w, rc);
}

int cg_release_workspace(void) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return CG_ECUDA;
  std::lock_guard<std::mutex> lk(g_ws_mu);
  HostWorkspace& w = g_ws[dev];
  int rc = CG_OK;
  if (w.d != nullptr && cudaFree(w.d) != cudaSuccess) rc = CG_ECUDA;
  w.d = nullptr;
  w.bytes = 0;
  return rc;
}

const char* cg_strerror(int code) {
  switch (code) {
    case CG_OK: return "CG_OK: success";
    case CG_EINVAL: return "CG_EINVAL: invalid argument";
    case CG_ECUDA: return "CG_ECUDA: CUDA runtime error";
    case CG_ENOMEM: return "CG_ENOMEM: out of memory";
    case CG_EAGAIN: return "CG_EAGAIN: resource temporarily full";
    case CG_ETIMEDOUT: return "CG_ETIMEDOUT: bounded wait expired";
    case CG_ENOTSUP: return "CG_ENOTSUP: unsupported mode combination";
    case CG_ETOOBIG: return "CG_ETOOBIG: request exceeds a fixed capacity";
    default: return "unknown cgmimo error code";
  }
}

int cg_version(void) { return 100; }

}  // extern "C"
