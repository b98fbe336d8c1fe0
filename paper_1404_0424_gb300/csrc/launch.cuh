// Host-side launch helpers shared by the translation units of libcgmimo.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "cg_kernels.cuh"
#include "cg_tc.cuh"

namespace cgm {

// Padded user count of the kernel instantiation that serves U users.
inline int padded_users(int U) { return U <= 4 ? 4 : U <= 8 ? 8 : U <= 16 ? 16 : 32; }

// Per-device facts the launchers need (cached; thread-safe).
struct DeviceInfo {
  int sm_count = 0;
  int smem_optin = 0;
  int smem_per_sm = 0;        // shared memory of one SM
  int smem_reserved = 0;      // shared memory the system reserves per resident block
};
int device_info(DeviceInfo* out);

// Serving kernels hold their SMs for as long as they have work, and the
// class kernels start and stop independently. If their CTAs had different
// footprints, a relaunched class could find every SM partly filled and none
// with room for one of its CTAs; the block scheduler would then hold back
// every grid launched after it as well. So every serving CTA is padded to
// more than half an SM's shared memory (one CTA per SM, whatever its class),
// and the class grids together hold at most one CTA per SM.
inline uint32_t serve_smem(const DeviceInfo& d, uint32_t need) {
  const uint32_t floor = uint32_t(d.smem_per_sm / 2 - d.smem_reserved + 16);
  return need > floor ? need : floor;
}

// Launchers (defined in detect.cu / precode.cu). Return cudaError_t values.
cudaError_t launch_detect(int UT, const DetectArgs& a, cudaStream_t s, int* grid_out);
cudaError_t launch_precode(int UT, const PrecodeArgs& a, cudaStream_t s, int* grid_out);

// Batched problems (tc.cu): op 0 = detect, 1 = precode; one bin of the
// warp-per-instance kernels, with the exact tracker when b.PEX. With
// launch = false only the launch shape is computed (grid). el: 0 = BF16,
// 1 = FP16; x3: hi+lo split; full is unused (kept by the bin keys).
cudaError_t launch_batch_tc(int op, int UT, int el, bool x3, bool full, const BatchArgs& b,
                            int max_grid, cudaStream_t s, bool launch, uint32_t* smem_out,
                            int* grid_out);

// Warp-per-instance kernels (warp.cu): padded users 8, 16 or 32, approximate
// tracker only. Batch and serve forms as above (grid in CTAs of 4 warps).
cudaError_t launch_detect_warp(int UT, int el, bool x3, const DetectArgs& a, cudaStream_t s);
cudaError_t launch_precode_warp(int UT, int el, bool x3, const PrecodeArgs& a, cudaStream_t s);
// CG-D with the exact tracker (Eq. 10) on the warp kernels, UT <= 16 (exact_warp.cu).
cudaError_t launch_detect_warp_exact(int UT, int el, bool x3, const DetectArgs& a,
                                     cudaStream_t s);
cudaError_t launch_batch_warp_exact(int UT, int el, bool x3, const BatchArgs& b, int max_grid,
                                    cudaStream_t s, bool launch, int* grid_out);
// Neumann-series variants of the warp kernels (neumann.cu), Sec. III-F.
cudaError_t launch_neumann_detect(int UT, int el, bool x3, const DetectArgs& a, cudaStream_t s);
cudaError_t launch_neumann_precode(int UT, int el, bool x3, const PrecodeArgs& a, cudaStream_t s);
cudaError_t launch_batch_warp(int op, int UT, int el, bool x3, const BatchArgs& b, int max_grid,
                              cudaStream_t s, bool launch, int* grid_out);
// Serving kernel (serve_kernels.cu): the warp kernel of every class. With
// launch = false only the resident CTAs are computed.
struct ServeArgs;
cudaError_t launch_serve_warp(int el, bool x3, const ServeArgs& sa, int grid, cudaStream_t s,
                              bool launch, int* resident_out);

// Implicit-product FP32 kernels (implicit.cu): e = H^H (H p) + sigma p; with
// cgls = true, CG least squares on the augmented systems (Sec. III-E).
cudaError_t launch_detect_implicit(int UT, const DetectArgs& a, cudaStream_t s, bool cgls);
cudaError_t launch_precode_implicit(int UT, const PrecodeArgs& a, cudaStream_t s, bool cgls);

// Whether A p is applied implicitly for these parameters: requested, or
// CG_AMUL_AUTO on the FP32 path when the two products per iteration cost
// fewer complex multiply-adds than the Gram (4 K R < U + 1).
inline bool use_implicit(int amul_mode, int precision, int K, int R, int U, bool exact) {
  if (amul_mode == 2) return true;  // CG_AMUL_IMPLICIT
  return amul_mode == 0 && precision == 0 && !exact && 4 * K * R < U + 1;
}

// Dynamic shared memory of one CTA for the given shape (bytes).
uint32_t detect_smem_bytes(int UT, int B, int U, int R, int exact);
uint32_t precode_smem_bytes(int UT, int B, int U, int R);

}  // namespace cgm
