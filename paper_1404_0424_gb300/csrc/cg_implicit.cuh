// FP32 kernels with the implicit product e = H^H (H p) + sigma p in
// Algorithm 1 with e = A p formed as H^H (H p) + sigma p: no Gram matrix is formed. One CTA owns an instance;
// H stays in shared memory for the whole solve, and one group of UT lanes
// runs the CG of one right-hand side (lane i owns user i):
//   w = H p   lane i forms w_b for antennas b = i, i + UT, ... (rows of H,
//             columns rotated by the lane so the group reads distinct banks),
//   e = H^H w + sigma p, lane i over all antennas.
// A product then costs 2 B U complex multiply-adds per right-hand side
// instead of the B U (U + 1) / 2 of the Hermitian Gram once per instance,
// which is cheaper when 4 K R < U + 1 (few right-hand sides and iterations).
// The matched filter b = H^H y and G_ii = ||h_i||^2 (for the tracker of
// Eqs. 11-13) are direct sums over the antennas.
//
// The same kernels, with CGLS = true, run CG least squares (Sec. III-E) on
// the augmented systems [H; sqrt(sigma) I] x = [y; 0] (detection) and
// [H^H, sqrt(sigma) I] x = t (precoding, q = the first B entries of x): no
// Gram either, with the residual kept in the data space (B + U entries per
// right-hand side in detection; the B-entry halves of x and p in precoding).
#pragma once

#include "cg_kernels.cuh"

namespace cgm {

struct ImplicitPlan {
  SmemPlan io;  // H, Y and YS as in the explicit kernels (same load helpers)
  uint32_t Bm, X, Mu, Rho, Gd, P, W, Z, Kd, misc, total;
};

template <int UT>
__host__ __device__ inline ImplicitPlan implicit_plan(int B, int U, int R, bool detect,
                                                      bool cgls = false) {
  constexpr int NG = TileCfg<UT>::NTHR / UT;
  ImplicitPlan s{};
  s.io.YS = detect ? ((B % 2 == 0) ? B + 2 : B + 1) : 0;
  const uint32_t hbytes = align16(uint32_t(B) * U * 8u);
  s.io.H = 0;
  s.io.Y = hbytes;
  uint32_t off = hbytes + align16(uint32_t(R) * (detect ? s.io.YS : U) * 8u);
  s.Bm = off; off += RMAX * UT * 8;
  s.X = off; off += RMAX * UT * 8;
  s.Mu = off; off += RMAX * UT * 4;
  s.Rho = off; off += RMAX * UT * 4;
  s.Gd = off; off += UT * 4;
  s.P = off; off += NG * UT * 8;
  s.W = off; off += align16(uint32_t(NG) * B * 8u);
  s.Z = off; off += cgls ? 2u * align16(uint32_t(NG) * B * 8u) : 0u;  // CGLS B-vectors
  s.Kd = off; off += RMAX * 4;
  s.misc = align16(off);
  s.total = s.misc + 16;  // mbarrier (8 bytes) + status word (4 bytes)
  s.io.total = s.total;
  return s;
}

// w_b = sum_j H[b][j] p_j for the group's antennas b = i, i + UT, ... into sW.
template <int UT>
__device__ __forceinline__ void implicit_hp(const float2* __restrict__ sH, int B, int U,
                                            const float2* __restrict__ sP, float2* sW) {
  const int i = threadIdx.x % UT;
  const int start = i % U;
  for (int b = i; b < B; b += UT) {
    float2 w = make_float2(0.f, 0.f);
    const float2* row = sH + b * U;
    int jj = start;
    for (int j = 0; j < U; ++j) {
      cmac(w, row[jj], sP[jj]);
      if (++jj == U) jj = 0;
    }
    sW[b] = w;
  }
}

// e_i = sum_b conj(H[b][i]) w_b + sigma p_i (0 for padded users).
__device__ __forceinline__ float2 implicit_hhw(const float2* __restrict__ sH, int B, int U,
                                               int i, const float2* __restrict__ sW,
                                               float2 p, float sigma) {
  float2 e = make_float2(sigma * p.x, sigma * p.y);
  if (i < U)
    for (int b = 0; b < B; ++b) cmac_conj(e, sH[b * U + i], sW[b]);
  return e;
}

// The CG iterations of Algorithm 1 for right-hand sides r = g, g + NG, ... with the
// implicit product; b in sB[r], v_K into sX[r]. With `track` the
// approximate tracker of Eqs. 11-13 as in cg_groups (D_ii = G_ii + sigma).
template <int UT, int NTHR>
__device__ __forceinline__ void implicit_cg_groups(const float2* __restrict__ sH, int B, int U,
                                                   float sigma, const float2* __restrict__ sB,
                                                   const float* sGd, int R, int K, float N0,
                                                   bool track, float2* sPall, float2* sWall,
                                                   float2* sX, float* sMu, float* sRho,
                                                   int* sKd, int* sStatus) {
  constexpr int NG = NTHR / UT;
  const int tid = threadIdx.x;
  const int g = tid / UT, i = tid % UT;
  const unsigned mask = group_mask<UT>();
  float2* sP = sPall + g * UT;
  float2* sW = sWall + g * B;
  const float Gii = (track && i < U) ? sGd[i] : 0.f;
  const float D = (i < U) ? Gii + sigma : 0.f;
  for (int r = g; r < R; r += NG) {
    const float2 bvec = sB[r * UT + i];
    float2 v = make_float2(0.f, 0.f);
    float2 res = bvec;
    float2 p = bvec;
    float rr = group_sum_compensated<UT>(bvec.x * bvec.x + bvec.y * bvec.y, mask);
    float l1 = 0.f, l2 = 0.f, l3 = 0.f;
    float a1 = 1.f, a2 = 1.f, be1 = 0.f, be2 = 0.f;
    int kd = 0;
    bool broke = false;
    for (int k = 1; k <= K; ++k) {
      if (!(rr > 0.f)) {
        broke = true;
        break;
      }
      // e = H^H (H p) + sigma p (implicit)
      sP[i] = p;
      __syncwarp(mask);
      implicit_hp<UT>(sH, B, U, sP, sW);
      __syncwarp(mask);
      const float2 e = implicit_hhw(sH, B, U, i, sW, p, sigma);
      __syncwarp(mask);  // sP and sW are rewritten by the next iteration
      const float pe = group_sum_compensated<UT>(p.x * e.x + p.y * e.y, mask);
      if (!(pe > 0.f)) {
        broke = true;
        break;
      }
      const float alpha = rr / pe;
      v.x = fmaf(alpha, p.x, v.x);  // v += alpha p
      v.y = fmaf(alpha, p.y, v.y);
      res.x = fmaf(-alpha, e.x, res.x);  // r -= alpha e
      res.y = fmaf(-alpha, e.y, res.y);
      const float rrn = group_sum_compensated<UT>(res.x * res.x + res.y * res.y, mask);
      const float beta = rrn / rr;
      p.x = fmaf(beta, p.x, res.x);  // p = r + beta p
      p.y = fmaf(beta, p.y, res.y);
      rr = rrn;
      const float lk = (k == 1) ? alpha
                                : l1 + (alpha * (1.f + be1) / a1 - alpha * D) * (l1 - l2) -
                                      (alpha * be2 / a2) * (l2 - l3);
      l3 = l2;
      l2 = l1;
      l1 = lk;
      a2 = a1;
      a1 = alpha;
      be2 = be1;
      be1 = beta;
      kd = k;
    }
    sX[r * UT + i] = v;
    if (track) {
      sMu[r * UT + i] = l1 * Gii;   // Eq. 12
      sRho[r * UT + i] = Gii / N0;  // Eq. 13
    }
    if (i == 0) {
      sKd[r] = kd;
      if (broke) atomicOr(sStatus, ST_BREAKDOWN);
    }
  }
}

// CGLS detection (Sec. III-E) for right-hand sides r = g, g + NG, ...: K
// iterations on min ||[y; 0] - [H; sqrt(sigma) I] x||, started at x = 0:
//   q = [H p; sqrt(sigma) p], alpha = gamma / ||q||^2, x += alpha p,
//   r -= alpha q, s = H^H r_top + sqrt(sigma) r_bot, beta = ||s||^2 / gamma,
//   p = s + beta p.
// r_top (B entries) is in sRall, lane i holds r_bot_i and the user-space
// vectors. In exact arithmetic alpha_k and beta_k are those of CG on
// A x = H^H y, so the approximate tracker (Eqs. 11-13) runs unchanged on them.
template <int UT, int NTHR>
__device__ __forceinline__ void cgls_detect_groups(const float2* __restrict__ sH, int B, int U,
                                                   float sigma, const float2* __restrict__ sY,
                                                   int YS, const float2* __restrict__ sB,
                                                   const float* sGd, int R, int K, float N0,
                                                   float2* sPall, float2* sWall, float2* sRall,
                                                   float2* sX, float* sMu, float* sRho, int* sKd,
                                                   int* sStatus) {
  constexpr int NG = NTHR / UT;
  const int tid = threadIdx.x;
  const int g = tid / UT, i = tid % UT;
  const unsigned mask = group_mask<UT>();
  float2* sP = sPall + g * UT;
  float2* sW = sWall + g * B;
  float2* sRt = sRall + g * B;
  const float rs = sqrtf(sigma);
  const float Gii = (i < U) ? sGd[i] : 0.f;
  const float D = (i < U) ? Gii + sigma : 0.f;
  for (int r = g; r < R; r += NG) {
    for (int b = i; b < B; b += UT) sRt[b] = sY[r * YS + b];  // r_top = y
    float2 rb = make_float2(0.f, 0.f);                         // r_bot = 0
    float2 sv = sB[r * UT + i];                                // s = H^H y
    float2 p = sv;
    float2 v = make_float2(0.f, 0.f);
    float gam = group_sum_compensated<UT>(sv.x * sv.x + sv.y * sv.y, mask);
    float l1 = 0.f, l2 = 0.f, l3 = 0.f;
    float a1 = 1.f, a2 = 1.f, be1 = 0.f, be2 = 0.f;
    int kd = 0;
    bool broke = false;
    __syncwarp(mask);
    for (int k = 1; k <= K; ++k) {
      if (!(gam > 0.f)) {
        broke = true;
        break;
      }
      sP[i] = p;
      __syncwarp(mask);
      implicit_hp<UT>(sH, B, U, sP, sW);  // q_top = H p on the lane's antennas
      float part = sigma * (p.x * p.x + p.y * p.y);
      for (int b = i; b < B; b += UT) part = fmaf(sW[b].x, sW[b].x, fmaf(sW[b].y, sW[b].y, part));
      const float qq = group_sum_compensated<UT>(part, mask);
      if (!(qq > 0.f)) {
        broke = true;
        break;
      }
      const float alpha = gam / qq;
      v.x = fmaf(alpha, p.x, v.x);
      v.y = fmaf(alpha, p.y, v.y);
      for (int b = i; b < B; b += UT) {
        sRt[b].x = fmaf(-alpha, sW[b].x, sRt[b].x);
        sRt[b].y = fmaf(-alpha, sW[b].y, sRt[b].y);
      }
      rb.x = fmaf(-alpha * rs, p.x, rb.x);
      rb.y = fmaf(-alpha * rs, p.y, rb.y);
      __syncwarp(mask);
      const float2 sn = implicit_hhw(sH, B, U, i, sRt, rb, rs);  // H^H r_top + sqrt(sigma) r_bot
      __syncwarp(mask);  // sP, sW and sRt are rewritten by the next iteration
      const float gn = group_sum_compensated<UT>(sn.x * sn.x + sn.y * sn.y, mask);
      const float beta = gn / gam;
      p.x = fmaf(beta, p.x, sn.x);
      p.y = fmaf(beta, p.y, sn.y);
      gam = gn;
      const float lk = (k == 1) ? alpha
                                : l1 + (alpha * (1.f + be1) / a1 - alpha * D) * (l1 - l2) -
                                      (alpha * be2 / a2) * (l2 - l3);
      l3 = l2;
      l2 = l1;
      l1 = lk;
      a2 = a1;
      a1 = alpha;
      be2 = be1;
      be1 = beta;
      kd = k;
    }
    __syncwarp(mask);
    sX[r * UT + i] = v;
    sMu[r * UT + i] = l1 * Gii;   // Eq. 12
    sRho[r * UT + i] = Gii / N0;  // Eq. 13
    if (i == 0) {
      sKd[r] = kd;
      if (broke) atomicOr(sStatus, ST_BREAKDOWN);
    }
  }
}

// CGLS precoding (Sec. III-E) for right-hand sides r = g, g + NG, ...: K
// iterations on min ||t - [H^H, sqrt(sigma) I] x||, started at x = 0, with
// q = x_top. The B-entry halves of x and p are in sZall (x_top, then p_top,
// per group), s_top = H r in the group's sW; lane i holds r_i, x_bot_i and
// p_bot_i. Writes q (normalised if asked) and ||q||.
template <int UT, int NTHR>
__device__ __forceinline__ void cgls_precode_groups(const PrecodeArgs& a, int64_t n,
                                                    const float2* __restrict__ sH,
                                                    const float2* __restrict__ sT0,
                                                    float2* sPall, float2* sWall, float2* sZall,
                                                    int* sStatus) {
  constexpr int NG = NTHR / UT;
  const int B = a.B, U = a.U, R = a.R;
  const int tid = threadIdx.x;
  const int g = tid / UT, i = tid % UT;
  const unsigned mask = group_mask<UT>();
  float2* sP = sPall + g * UT;
  float2* sW = sWall + g * B;
  float2* sXt = sZall + (2 * g) * B;
  float2* sPt = sZall + (2 * g + 1) * B;
  const float rs = sqrtf(a.sigma);
  for (int r = g; r < R; r += NG) {
    float2 rv = sT0[r * UT + i];  // r = t (zero for padded users)
    sP[i] = rv;
    __syncwarp(mask);
    implicit_hp<UT>(sH, B, U, sP, sW);  // s_top = H t
    float part = 0.f;
    for (int b = i; b < B; b += UT) {
      sPt[b] = sW[b];
      sXt[b] = make_float2(0.f, 0.f);
      part = fmaf(sW[b].x, sW[b].x, fmaf(sW[b].y, sW[b].y, part));
    }
    float2 pb = make_float2(rs * rv.x, rs * rv.y);  // s_bot = sqrt(sigma) t
    float2 xb = make_float2(0.f, 0.f);
    part = fmaf(pb.x, pb.x, fmaf(pb.y, pb.y, part));
    float gam = group_sum_compensated<UT>(part, mask);
    bool broke = false;
    for (int k = 1; k <= a.K; ++k) {
      if (!(gam > 0.f)) {
        broke = true;
        break;
      }
      __syncwarp(mask);
      const float2 qi = implicit_hhw(sH, B, U, i, sPt, pb, rs);  // H^H p_top + sqrt(sigma) p_bot
      const float qq = group_sum_compensated<UT>(qi.x * qi.x + qi.y * qi.y, mask);
      if (!(qq > 0.f)) {
        broke = true;
        break;
      }
      const float alpha = gam / qq;
      for (int b = i; b < B; b += UT) {
        sXt[b].x = fmaf(alpha, sPt[b].x, sXt[b].x);
        sXt[b].y = fmaf(alpha, sPt[b].y, sXt[b].y);
      }
      xb.x = fmaf(alpha, pb.x, xb.x);
      xb.y = fmaf(alpha, pb.y, xb.y);
      rv.x = fmaf(-alpha, qi.x, rv.x);
      rv.y = fmaf(-alpha, qi.y, rv.y);
      __syncwarp(mask);  // every lane has read sPt and sP
      sP[i] = rv;
      __syncwarp(mask);
      implicit_hp<UT>(sH, B, U, sP, sW);  // s_top = H r
      const float2 sbot = make_float2(rs * rv.x, rs * rv.y);
      float gp = fmaf(sbot.x, sbot.x, sbot.y * sbot.y);
      for (int b = i; b < B; b += UT) gp = fmaf(sW[b].x, sW[b].x, fmaf(sW[b].y, sW[b].y, gp));
      const float gn = group_sum_compensated<UT>(gp, mask);
      const float beta = gn / gam;
      for (int b = i; b < B; b += UT) {
        sPt[b].x = fmaf(beta, sPt[b].x, sW[b].x);
        sPt[b].y = fmaf(beta, sPt[b].y, sW[b].y);
      }
      pb.x = fmaf(beta, pb.x, sbot.x);
      pb.y = fmaf(beta, pb.y, sbot.y);
      gam = gn;
    }
    // q = x_top, ||q||^2 = sum_b |q_b|^2
    float qp = 0.f;
    for (int b = i; b < B; b += UT) qp = fmaf(sXt[b].x, sXt[b].x, fmaf(sXt[b].y, sXt[b].y, qp));
    const float qq = group_sum_compensated<UT>(qp, mask);
    const float nr = sqrtf(fmaxf(qq, 0.f));
    const float inv = a.normalize ? (nr > 0.f ? 1.f / nr : 0.f) : 1.f;
    if (i == 0 && a.qnorm) a.qnorm[n * R + r] = nr;
    float2* qr = a.q + (n * R + r) * B;
    for (int b = i; b < B; b += UT) qr[b] = make_float2(sXt[b].x * inv, sXt[b].y * inv);
    if (i == 0 && broke) atomicOr(sStatus, ST_BREAKDOWN);
    __syncwarp(mask);
  }
}

// Staging of an instance's H and Y (bulk copies when allowed) and the wait.
// Returns false if the copies timed out (status already written).
template <int NTHR>
__device__ __forceinline__ bool implicit_stage_detect(const DetectArgs& a, const SmemPlan& io,
                                                      unsigned char* smem, uint64_t* bar,
                                                      uint32_t* parity, int64_t n) {
  if (a.bulk) {
    if (threadIdx.x == 0) {
      fence_proxy_async_smem();
      issue_detect_copies(a, io, smem, bar, n);
    }
    if (!wait_inputs(bar, *parity, a.wait_ns)) {
      if (threadIdx.x == 0 && a.status) a.status[n] = ST_TIMEOUT;
      mbar_wait_bounded(bar, *parity, WAIT_TIMEOUT_NS);
      return false;
    }
    *parity ^= 1u;
  } else {
    coop_load_detect<NTHR>(a, io, smem, n);
    __syncthreads();
  }
  return true;
}

template <int UT, bool CGLS = false>
__global__ void __launch_bounds__(TileCfg<UT>::NTHR) detect_implicit_kernel(const DetectArgs a) {
  constexpr int NTHR = TileCfg<UT>::NTHR;
  extern __shared__ __align__(128) unsigned char smem[];
  const ImplicitPlan P = implicit_plan<UT>(a.B, a.U, a.R, true, CGLS);
  const float2* sH = reinterpret_cast<const float2*>(smem + P.io.H);
  const float2* sY = reinterpret_cast<const float2*>(smem + P.io.Y);
  float2* sBm = reinterpret_cast<float2*>(smem + P.Bm);
  float2* sX = reinterpret_cast<float2*>(smem + P.X);
  float* sMu = reinterpret_cast<float*>(smem + P.Mu);
  float* sRho = reinterpret_cast<float*>(smem + P.Rho);
  float* sGd = reinterpret_cast<float*>(smem + P.Gd);
  float2* sP = reinterpret_cast<float2*>(smem + P.P);
  float2* sW = reinterpret_cast<float2*>(smem + P.W);
  int* sKd = reinterpret_cast<int*>(smem + P.Kd);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + P.misc);
  int* sStatus = reinterpret_cast<int*>(smem + P.misc + 8);
  const int tid = threadIdx.x;
  const int U = a.U, R = a.R, B = a.B;
  if (tid == 0) mbar_init(bar, 1);
  __syncthreads();
  uint32_t parity = 0;
  for (int64_t n = blockIdx.x; n < a.n_inst; n += gridDim.x) {
    if (!implicit_stage_detect<NTHR>(a, P.io, smem, bar, &parity, n)) return;
    if (tid == 0) *sStatus = 0;
    // matched filters b = H^H y (Eq. 8) and G_ii = ||h_i||^2
    for (int e = tid; e < R * UT; e += NTHR) {
      const int r = e / UT, i = e - r * UT;
      float2 s = make_float2(0.f, 0.f);
      if (i < U) {
        const float2* yr = sY + r * P.io.YS;
        for (int b = 0; b < B; ++b) cmac_conj(s, sH[b * U + i], yr[b]);
      }
      sBm[e] = s;
    }
    for (int i = tid; i < UT; i += NTHR) {
      float s = 0.f;
      if (i < U)
        for (int b = 0; b < B; ++b) {
          const float2 h = sH[b * U + i];
          s = fmaf(h.x, h.x, fmaf(h.y, h.y, s));
        }
      sGd[i] = s;
    }
    __syncthreads();
    if constexpr (CGLS)
      cgls_detect_groups<UT, NTHR>(sH, B, U, a.sigma, sY, P.io.YS, sBm, sGd, R, a.K, a.N0, sP,
                                   sW, reinterpret_cast<float2*>(smem + P.Z), sX, sMu, sRho,
                                   sKd, sStatus);
    else
      implicit_cg_groups<UT, NTHR>(sH, B, U, a.sigma, sBm, sGd, R, a.K, a.N0, true, sP, sW, sX,
                                   sMu, sRho, sKd, sStatus);
    __syncthreads();
    write_detect_outputs<UT, NTHR>(a, n, sX, sMu, sRho, sStatus);
    __syncthreads();
    if (tid == 0 && a.status) a.status[n] = *sStatus;
    __syncthreads();  // H and Y are overwritten by the next instance's loads
  }
}

template <int UT, bool CGLS = false>
__global__ void __launch_bounds__(TileCfg<UT>::NTHR) precode_implicit_kernel(const PrecodeArgs a) {
  constexpr int NTHR = TileCfg<UT>::NTHR;
  constexpr int NG = NTHR / UT;
  extern __shared__ __align__(128) unsigned char smem[];
  const ImplicitPlan P = implicit_plan<UT>(a.B, a.U, a.R, false, CGLS);
  float2* sH = reinterpret_cast<float2*>(smem + P.io.H);
  float2* sT = reinterpret_cast<float2*>(smem + P.io.Y);
  float2* sBm = reinterpret_cast<float2*>(smem + P.Bm);
  float2* sX = reinterpret_cast<float2*>(smem + P.X);
  float2* sP = reinterpret_cast<float2*>(smem + P.P);
  float2* sW = reinterpret_cast<float2*>(smem + P.W);
  int* sKd = reinterpret_cast<int*>(smem + P.Kd);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + P.misc);
  int* sStatus = reinterpret_cast<int*>(smem + P.misc + 8);
  const int tid = threadIdx.x;
  const int U = a.U, R = a.R, B = a.B;
  const bool bulk = a.bulk_h || a.bulk_t;
  if (tid == 0) mbar_init(bar, 1);
  __syncthreads();
  uint32_t parity = 0;
  for (int64_t n = blockIdx.x; n < a.n_inst; n += gridDim.x) {
    if (bulk && tid == 0) {
      fence_proxy_async_smem();
      uint32_t bytes = 0;
      if (a.bulk_h) bytes += uint32_t(B) * U * 8u;
      if (a.bulk_t) bytes += uint32_t(R) * U * 8u;
      mbar_arrive_expect_tx(bar, bytes);
      if (a.bulk_h) bulk_copy_g2s(sH, a.H + n * B * U, uint32_t(B) * U * 8u, bar);
      if (a.bulk_t) bulk_copy_g2s(sT, a.T + n * R * U, uint32_t(R) * U * 8u, bar);
    }
    if (!a.bulk_h)
      for (int e = tid; e < B * U; e += NTHR) sH[e] = a.H[n * B * U + e];
    if (!a.bulk_t)
      for (int e = tid; e < R * U; e += NTHR) sT[e] = a.T[n * R * U + e];
    if (bulk) {
      if (!wait_inputs(bar, parity, a.wait_ns)) {
        if (tid == 0 && a.status) a.status[n] = ST_TIMEOUT;
        mbar_wait_bounded(bar, parity, WAIT_TIMEOUT_NS);
        return;
      }
      parity ^= 1u;
    } else {
      __syncthreads();
    }
    if (tid == 0) *sStatus = 0;
    // b = t (Sec. III-D), padded to UT users
    for (int e = tid; e < R * UT; e += NTHR) {
      const int r = e / UT, i = e - r * UT;
      sBm[e] = (i < U) ? sT[r * U + i] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    if constexpr (CGLS) {
      cgls_precode_groups<UT, NTHR>(a, n, sH, sBm, sP, sW, reinterpret_cast<float2*>(smem + P.Z),
                                    sStatus);
    } else {
      implicit_cg_groups<UT, NTHR>(sH, B, U, a.sigma, sBm, nullptr, R, a.K, 0.f, false, sP, sW,
                                   sX, nullptr, nullptr, sKd, sStatus);
    }
    // q = H v (Sec. III-D) by the group that owns v, ||q||^2 = sum_b |q_b|^2
    if constexpr (!CGLS) {
      const int g = tid / UT, i = tid % UT;
      const unsigned mask = group_mask<UT>();
      float2* gP = sP + g * UT;
      float2* gW = sW + g * B;
      for (int r = g; r < R; r += NG) {
        gP[i] = sX[r * UT + i];
        __syncwarp(mask);
        implicit_hp<UT>(sH, B, U, gP, gW);
        __syncwarp(mask);
        float part = 0.f;
        for (int b = i; b < B; b += UT) part = fmaf(gW[b].x, gW[b].x, fmaf(gW[b].y, gW[b].y, part));
        const float qq = group_sum_compensated<UT>(part, mask);
        const float nr = sqrtf(fmaxf(qq, 0.f));
        const float inv = a.normalize ? (nr > 0.f ? 1.f / nr : 0.f) : 1.f;
        if (i == 0 && a.qnorm) a.qnorm[n * R + r] = nr;
        float2* qr = a.q + (n * R + r) * B;
        for (int b = i; b < B; b += UT) qr[b] = make_float2(gW[b].x * inv, gW[b].y * inv);
        __syncwarp(mask);
      }
    }
    __syncthreads();
    if (tid == 0 && a.status) a.status[n] = *sStatus;
    __syncthreads();
  }
}

}  // namespace cgm
