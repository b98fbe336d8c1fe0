// Host-side argument checks shared by the C-ABI entry points.
#pragma once

#include <cmath>
#include <cstdint>

#include "cgmimo.h"

namespace cgm {

inline bool aligned(const void* p, uintptr_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

inline int check_common(const cg_params* p, int64_t n_inst) {
  if (p == nullptr || n_inst < 0) return CG_EINVAL;
  if (p->U < 1 || p->U > CG_U_MAX) return CG_EINVAL;
  if (p->B < p->U || p->B > CG_B_MAX) return CG_EINVAL;
  if (p->R < 1 || p->R > CG_R_MAX) return CG_EINVAL;
  if (p->K < 1 || p->K > p->U || p->K > CG_K_MAX) return CG_EINVAL;
  if (!(p->N0 > 0.f) || !std::isfinite(p->N0)) return CG_EINVAL;
  if (!(p->Es > 0.f) || !std::isfinite(p->Es)) return CG_EINVAL;
  if (p->amul_mode < CG_AMUL_AUTO || p->amul_mode > CG_AMUL_CGLS) return CG_EINVAL;
  if (p->precision < CG_PREC_FP32 || p->precision > CG_PREC_FP16X3) return CG_EINVAL;
  return CG_OK;
}

inline int check_detect(const cg_params* p, int64_t n_inst, const void* H, const void* Y,
                 const void* xhat, const float* mu, const float* rho, const float* llr,
                 const int32_t* status) {
  int rc = check_common(p, n_inst);
  if (rc != CG_OK) return rc;
  if (p->qam_bits != 2 && p->qam_bits != 4 && p->qam_bits != 6 && p->qam_bits != 8)
    return CG_EINVAL;
  if (p->sinr_mode != CG_SINR_APPROX && p->sinr_mode != CG_SINR_EXACT) return CG_EINVAL;
  if (n_inst == 0) return CG_OK;
  if (H == nullptr || Y == nullptr) return CG_EINVAL;
  if (!aligned(H, 8) || !aligned(Y, 8) || !aligned(xhat, 8) || !aligned(mu, 4) ||
      !aligned(rho, 4) || !aligned(llr, 8) || !aligned(status, 4))
    return CG_EINVAL;
  return CG_OK;
}

inline int check_precode(const cg_params* p, int64_t n_inst, const void* H, const void* T,
                  const void* q, const float* qnorm, const int32_t* status) {
  int rc = check_common(p, n_inst);
  if (rc != CG_OK) return rc;
  if (n_inst == 0) return CG_OK;
  if (H == nullptr || T == nullptr || q == nullptr) return CG_EINVAL;
  if (!aligned(H, 8) || !aligned(T, 8) || !aligned(q, 8) || !aligned(qnorm, 4) ||
      !aligned(status, 4))
    return CG_EINVAL;
  return CG_OK;
}

}  // namespace cgm
