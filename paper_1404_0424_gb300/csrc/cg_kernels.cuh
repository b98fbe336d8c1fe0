// Fused FP32 kernels for CG soft-output detection (CG-D) and CG precoding
// (CG-P), Algorithm 1 of Yin, Wu, Cavallaro and Studer (arXiv 1404.0424).
//
// One CTA owns one instance (one channel H with its R right-hand sides) at a
// time and loops over instances with a grid stride:
//   1. bulk-copy H [B][U] and the R rows of Y (or T) into shared memory,
//   2. form G = H^H H and the matched filters b_r = H^H y_r as one register-
//      tiled product H^H [H | Y^T] with the antenna axis split into slices
//      (Algorithm 1; Eqs. 7, 8), reduce the slices in a fixed order,
//   3. run the CG iterations of Algorithm 1 with one group of UT lanes per right-hand
//      side (lane i owns user i; inner products are compensated group sums)
//      and the approximate tracker of Eqs. 11-13 in the loop,
//   4. optionally the exact tracker of Eq. 10 (CTA-cooperative, per RHS),
//   5. epilogue: x_hat, mu, rho and max-log LLRs (Eq. 4), or q = H v with
//      optional power normalisation (CG-P).
// The next instance's inputs are prefetched as soon as step 2 has consumed
// the current ones.
#pragma once

#include "cg_common.cuh"

namespace cgm {

// Register tile (TM x TN complex accumulators per thread) and CTA size per
// padded user count UT.
template <int UT> struct TileCfg;
template <> struct TileCfg<4> { static constexpr int TM = 4, TN = 4, NTHR = 128; };
template <> struct TileCfg<8> { static constexpr int TM = 4, TN = 4, NTHR = 128; };
template <> struct TileCfg<16> { static constexpr int TM = 4, TN = 4, NTHR = 128; };
template <> struct TileCfg<32> { static constexpr int TM = 8, TN = 4, NTHR = 256; };

struct DetectArgs {
  const float2* H;
  const float2* Y;
  float2* xhat;
  float* mu;
  float* rho;
  float* llr;
  int32_t* status;
  int64_t n_inst;
  int B, U, R, K, q;
  float N0, Es, sigma;
  int exact;  // CG_SINR_EXACT
  int bulk;   // inputs may be fetched with 1-D bulk copies
  uint64_t wait_ns;  // limit of the wait for an instance's bulk copies (cg_set_wait_limit)
  // Tensor maps of H ([n][B][U] complex as FP32, box 8 antennas x 16 users,
  // 128-byte swizzle; 8 users: 64-byte swizzle) and Y ([n][R][B], box 16 rows
  // x 8 antennas), valid when tma != 0. The warp kernels stage their Gram
  // k-steps through them; a kernel that reads them takes its arguments as
  // __grid_constant__.
  int tma;
  CUtensorMap tmH, tmY;
};

struct PrecodeArgs {
  const float2* H;
  const float2* T;
  float2* q;
  float* qnorm;
  int32_t* status;
  int64_t n_inst;
  int B, U, R, K;
  float sigma;
  int normalize;
  int bulk_h;  // H may be fetched with bulk copies
  int bulk_t;  // T may be fetched with bulk copies
  uint64_t wait_ns;  // limit of the wait for an instance's bulk copies (cg_set_wait_limit)
};

// Byte offsets into dynamic shared memory; computed identically on host and
// device from (B, U, R, mode).
struct SmemPlan {
  uint32_t H, Y, A, Bm, X, Mu, Rho, Gd, AB, Kd, Nrm, misc, total;
  uint32_t big;  // bytes of the leading region (H, Y, then reused)
  int YS;        // padded row stride of Y in complex elements
  int NCTH, NCT, NT, NSL;
};

template <int UT>
__host__ __device__ inline SmemPlan detect_plan(int B, int U, int R, int exact) {
  using C = TileCfg<UT>;
  SmemPlan s{};
  s.YS = (B % 2 == 0) ? B + 2 : B + 1;  // keeps rows 16-byte aligned for even B
  s.NCTH = UT / C::TN;
  s.NCT = s.NCTH + (R + C::TN - 1) / C::TN;
  s.NT = (UT / C::TM) * s.NCT;
  int nsl = C::NTHR / s.NT;
  if (nsl > B) nsl = B;
  if (nsl < 1) nsl = 1;
  s.NSL = nsl;
  const uint32_t hbytes = align16(uint32_t(B) * U * 8u);
  const uint32_t hy = hbytes + align16(uint32_t(R) * s.YS * 8u);
  const uint32_t part = uint32_t(s.NSL) * s.NT * C::TM * C::TN * 8u;
  const uint32_t lbuf = exact ? 5u * U * U * 8u : 0u;
  uint32_t big = hy > part ? hy : part;
  big = big > lbuf ? big : lbuf;
  s.big = align16(big);
  s.H = 0;
  s.Y = hbytes;
  uint32_t off = s.big;
  s.A = off; off += UT * UT * 8;
  s.Bm = off; off += RMAX * UT * 8;
  s.X = off; off += RMAX * UT * 8;
  s.Mu = off; off += RMAX * UT * 4;
  s.Rho = off; off += RMAX * UT * 4;
  s.Gd = off; off += UT * 4;
  s.AB = off; off += exact ? RMAX * KMAX * 2 * 4 : 0;
  s.Kd = off; off += RMAX * 4;
  s.Nrm = off;
  s.misc = align16(off);
  s.total = s.misc + 16;  // mbarrier (8 bytes) + status word (4 bytes)
  return s;
}

template <int UT>
__host__ __device__ inline SmemPlan precode_plan(int B, int U, int R) {
  using C = TileCfg<UT>;
  SmemPlan s{};
  s.YS = 0;
  s.NCTH = UT / C::TN;
  s.NCT = s.NCTH;
  s.NT = (UT / C::TM) * s.NCT;
  int nsl = C::NTHR / s.NT;
  if (nsl > B) nsl = B;
  if (nsl < 1) nsl = 1;
  s.NSL = nsl;
  const uint32_t hbytes = align16(uint32_t(B) * U * 8u);
  s.H = 0;
  s.Y = hbytes;  // T [R][U]
  s.big = hbytes + align16(uint32_t(R) * U * 8u);
  uint32_t off = s.big;
  s.A = off; off += UT * UT * 8;
  s.X = off; off += RMAX * UT * 8;  // t, then v_K, per right-hand side
  // Slice partials for the buffered reduction when they are small; otherwise
  // the slices accumulate into A in turn (Bm == X marks that case).
  const uint32_t part = uint32_t(s.NSL) * s.NT * C::TM * C::TN * 8u;
  if (part <= 16384u) {
    s.Bm = off; off += part;
  } else {
    s.Bm = s.X;
  }
  s.Mu = s.Rho = s.Gd = s.AB = off;
  s.Kd = off; off += RMAX * 4;
  s.Nrm = off; off += RMAX * 4;
  s.misc = align16(off);
  s.total = s.misc + 16;
  return s;
}

// --------------------------------------------------------------------------
// Step 1: inputs
// --------------------------------------------------------------------------

__device__ __forceinline__ void issue_detect_copies(const DetectArgs& a, const SmemPlan& P,
                                                    unsigned char* smem, uint64_t* bar,
                                                    int64_t n) {
  const uint32_t hb = uint32_t(a.B) * a.U * 8u;
  const uint32_t yb = uint32_t(a.B) * 8u;
  mbar_arrive_expect_tx(bar, hb + uint32_t(a.R) * yb);
  bulk_copy_g2s(smem + P.H, a.H + n * a.B * a.U, hb, bar);
  for (int r = 0; r < a.R; ++r)
    bulk_copy_g2s(smem + P.Y + uint32_t(r) * P.YS * 8u, a.Y + (n * a.R + r) * a.B, yb, bar);
}

template <int NTHR>
__device__ __forceinline__ void coop_load_detect(const DetectArgs& a, const SmemPlan& P,
                                                 unsigned char* smem, int64_t n) {
  float2* sH = reinterpret_cast<float2*>(smem + P.H);
  float2* sY = reinterpret_cast<float2*>(smem + P.Y);
  const float2* gH = a.H + n * a.B * a.U;
  const float2* gY = a.Y + n * a.R * a.B;
  for (int e = threadIdx.x; e < a.B * a.U; e += NTHR) sH[e] = gH[e];
  for (int e = threadIdx.x; e < a.R * a.B; e += NTHR) {
    const int r = e / a.B, b = e - r * a.B;
    sY[r * P.YS + b] = gY[e];
  }
}

// Waits for the bulk copies of the current instance, at most wait_ns of
// global time. Returns false (for the whole CTA) if they did not land in
// time; the caller then reports CG_STATUS_TIMEOUT, waits (with the 2 s
// bound) for the copies still in flight into its shared memory, and stops.
__device__ __forceinline__ bool wait_inputs(uint64_t* bar, uint32_t parity, uint64_t wait_ns) {
  const bool ok = mbar_wait_bounded(bar, parity, wait_ns);
  return !__syncthreads_or(!ok);
}

// --------------------------------------------------------------------------
// Step 2: register-tiled H^H [H | Y^T] over one antenna slice
// --------------------------------------------------------------------------

// Thread `tid` owns tile (tid % NT) of the output grid and antenna slice
// (tid / NT). Tile (ti, tj): rows ti*TM.., columns tj*TN.. of [H | Y^T];
// columns beyond U (or R) are clamped to a valid column and discarded later.
template <int UT, bool WITH_Y>
__device__ __forceinline__ void gram_tile(const float2* __restrict__ sH,
                                          const float2* __restrict__ sY, int YS, int B, int U,
                                          int R, const SmemPlan& P,
                                          float2 (&acc)[TileCfg<UT>::TM][TileCfg<UT>::TN],
                                          int& tile, int& slice) {
  constexpr int TM = TileCfg<UT>::TM, TN = TileCfg<UT>::TN;
#pragma unroll
  for (int m = 0; m < TM; ++m)
#pragma unroll
    for (int n = 0; n < TN; ++n) acc[m][n] = make_float2(0.f, 0.f);
  const int tid = threadIdx.x;
  if (tid >= P.NT * P.NSL) {
    tile = -1;
    slice = -1;
    return;
  }
  tile = tid % P.NT;
  slice = tid / P.NT;
  const int ti = tile / P.NCT, tj = tile - (tile / P.NCT) * P.NCT;
  const int b0 = (slice * B) / P.NSL, b1 = ((slice + 1) * B) / P.NSL;
  int ioff[TM];
#pragma unroll
  for (int m = 0; m < TM; ++m) ioff[m] = min(ti * TM + m, U - 1);
  const float2* jbase;
  int jstep;
  int joff[TN];
  if (!WITH_Y || tj < P.NCTH) {
    jbase = sH;
    jstep = U;
#pragma unroll
    for (int n = 0; n < TN; ++n) joff[n] = min(tj * TN + n, U - 1);
  } else {
    const int r0 = (tj - P.NCTH) * TN;
    jbase = sY;
    jstep = 1;
#pragma unroll
    for (int n = 0; n < TN; ++n) joff[n] = min(r0 + n, R - 1) * YS;
  }
  const float2* ip = sH + b0 * U;
  const float2* jp = jbase + b0 * jstep;
#pragma unroll 2
  for (int b = b0; b < b1; ++b) {
    float2 hv[TM], zv[TN];
#pragma unroll
    for (int m = 0; m < TM; ++m) hv[m] = ip[ioff[m]];
#pragma unroll
    for (int n = 0; n < TN; ++n) zv[n] = jp[joff[n]];
#pragma unroll
    for (int m = 0; m < TM; ++m)
#pragma unroll
      for (int n = 0; n < TN; ++n) cmac_conj(acc[m][n], hv[m], zv[n]);
    ip += U;
    jp += jstep;
  }
}

// Stores one reduced entry of H^H [H | Y^T]: Gram entries go to the upper
// triangle of A (mirrored as conjugates; A = G + sigma I, exactly Hermitian),
// matched-filter entries to Bm[r][i]. Entries of padded users are zero.
__device__ __forceinline__ void store_reduced(int UT, int i, int j_or_r, bool is_gram, float2 s,
                                              int U, int R, float sigma, float2* sA, float2* sBm,
                                              float* sGd) {
  if (is_gram) {
    const int j = j_or_r;
    if (i >= U || j >= U) {
      sA[i * UT + j] = make_float2(0.f, 0.f);
      if (i == j) sGd[i] = 0.f;
    } else if (i < j) {
      sA[i * UT + j] = s;
      sA[j * UT + i] = make_float2(s.x, -s.y);
    } else if (i == j) {
      sA[i * UT + i] = make_float2(s.x + sigma, 0.f);
      sGd[i] = s.x;
    }
  } else {
    const int r = j_or_r;
    if (r < R) sBm[r * UT + i] = (i < U) ? s : make_float2(0.f, 0.f);
  }
}

// --------------------------------------------------------------------------
// Step 3: Algorithm 1, one group of UT lanes per right-hand side
// --------------------------------------------------------------------------

// Runs K iterations on b = sB[r] for r = g, g + NG, ... and writes v_K to
// sX[r]. When `track` is set, also the approximate tracker of Eqs. 11-13:
// mu = l_{i,K} G_ii into sMu, rho = G_ii / N0 into sRho. When `sAB` is not
// null, alpha_k and beta_k are recorded for the exact tracker. The number of
// completed iterations goes to sKd[r]; a breakdown sets ST_BREAKDOWN.
template <int UT, int NTHR>
__device__ __forceinline__ void cg_groups(const float2* __restrict__ sA,
                                          const float2* __restrict__ sB, const float* sGd,
                                          int R, int K, float N0, bool track, float2* sX,
                                          float* sMu, float* sRho, float* sAB, int* sKd,
                                          int* sStatus) {
  constexpr int NG = NTHR / UT;
  const int tid = threadIdx.x;
  const int g = tid / UT, i = tid % UT;
  const unsigned mask = group_mask<UT>();
  const float D = sA[i * UT + i].x;  // diagonal of A (0 for padded users)
  const float Gii = track ? sGd[i] : 0.f;
  for (int r = g; r < R; r += NG) {
    const float2 bvec = sB[r * UT + i];
    float2 v = make_float2(0.f, 0.f);  // v_0 = 0
    float2 res = bvec;                 // r_0 = b
    float2 p = bvec;                   // p_0 = r_0
    float rr = group_sum_compensated<UT>(bvec.x * bvec.x + bvec.y * bvec.y, mask);
    float l1 = 0.f, l2 = 0.f, l3 = 0.f;  // l_{k-1}, l_{k-2}, l_{k-3}
    float a1 = 1.f, a2 = 1.f;            // alpha_{k-1}, alpha_{k-2}
    float be1 = 0.f, be2 = 0.f;          // beta_{k-1}, beta_{k-2}
    int kd = 0;
    bool broke = false;
    for (int k = 1; k <= K; ++k) {
      if (!(rr > 0.f)) {
        broke = true;
        break;
      }
      // e = A p; A[j][i] = conj(A[i][j]) keeps the reads contiguous
      float2 e = make_float2(0.f, 0.f);
#pragma unroll
      for (int j = 0; j < UT; ++j) {
        const float2 aji = sA[j * UT + i];
        float2 pj;
        pj.x = __shfl_sync(mask, p.x, j, UT);
        pj.y = __shfl_sync(mask, p.y, j, UT);
        cmac_conj(e, aji, pj);
      }
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
      // Eq. 11 on the diagonal: l_1 = alpha_1, then the three-term recursion
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
      if (sAB != nullptr && i == 0) {
        sAB[(r * KMAX + (k - 1)) * 2 + 0] = alpha;
        sAB[(r * KMAX + (k - 1)) * 2 + 1] = beta;
      }
      kd = k;
    }
    sX[r * UT + i] = v;
    if (track) {
      sMu[r * UT + i] = l1 * Gii;  // Eq. 12
      sRho[r * UT + i] = Gii / N0;  // Eq. 13
    }
    if (i == 0) {
      sKd[r] = kd;
      if (broke) atomicOr(sStatus, ST_BREAKDOWN);
    }
  }
}

// --------------------------------------------------------------------------
// Step 4: exact tracker (Eq. 10), cooperative over the CTA, one RHS at a time
// --------------------------------------------------------------------------

// L_1 = alpha_1 I; for k >= 2
//   L_k = L_{k-1} + c1 (L_{k-1} - L_{k-2}) - alpha_k A (L_{k-1} - L_{k-2})
//         - c2 (L_{k-2} - L_{k-3}),
// c1 = alpha_k (1 + beta_{k-1}) / alpha_{k-1}, c2 = alpha_k beta_{k-2} / alpha_{k-2}.
// Then B = L_K G, mu_i = Re B_ii, C_ii = sum_m B_im conj(L_im),
// nu_i^2 = sum_{j != i} |B_ij|^2 Es + C_ii N0, rho_i = mu_i^2 / nu_i^2.
template <int UT, int NTHR>
__device__ void exact_tracker(float2* buf, const float2* __restrict__ sA, const float* sAB,
                              const int* sKd, int U, int R, float sigma, float N0, float Es,
                              float* sMu, float* sRho) {
  const int tid = threadIdx.x;
  const int UU = U * U;
  float2* Bm = buf + 4 * UU;  // buf holds L buffers 0..3 (U*U each), then B
  for (int r = 0; r < R; ++r) {
    const int kd = sKd[r];
    if (kd == 0) {
      for (int i = tid; i < U; i += NTHR) {
        sMu[r * UT + i] = 0.f;
        sRho[r * UT + i] = 0.f;
      }
      continue;
    }
    const float* ab = sAB + r * KMAX * 2;
    int i1 = 0, i2 = 1, i3 = 2, in = 3;  // L_{k-1}, L_{k-2}, L_{k-3}, L_k
    for (int e = tid; e < UU; e += NTHR) {
      const int i = e / U, j = e - (e / U) * U;
      buf[i1 * UU + e] = make_float2(i == j ? ab[0] : 0.f, 0.f);
      buf[i2 * UU + e] = make_float2(0.f, 0.f);
      buf[i3 * UU + e] = make_float2(0.f, 0.f);
    }
    __syncthreads();
    for (int k = 2; k <= kd; ++k) {
      const float ak = ab[(k - 1) * 2];
      const float ak1 = ab[(k - 2) * 2], bk1 = ab[(k - 2) * 2 + 1];
      const float ak2 = (k - 3 >= 0) ? ab[(k - 3) * 2] : 1.f;
      const float bk2 = (k - 3 >= 0) ? ab[(k - 3) * 2 + 1] : 0.f;
      const float c1 = ak * (1.f + bk1) / ak1;
      const float c2 = ak * bk2 / ak2;
      const float2* P1 = buf + i1 * UU;
      const float2* P2 = buf + i2 * UU;
      const float2* P3 = buf + i3 * UU;
      float2* Pn = buf + in * UU;
      for (int e = tid; e < UU; e += NTHR) {
        const int i = e / U, j = e - (e / U) * U;
        float2 ad = make_float2(0.f, 0.f);
        for (int m = 0; m < U; ++m) {
          const float2 d = make_float2(P1[m * U + j].x - P2[m * U + j].x,
                                       P1[m * U + j].y - P2[m * U + j].y);
          cmac(ad, sA[i * UT + m], d);
        }
        const float2 l1 = P1[e], l2 = P2[e], l3 = P3[e];
        float2 out;
        out.x = l1.x + c1 * (l1.x - l2.x) - ak * ad.x - c2 * (l2.x - l3.x);
        out.y = l1.y + c1 * (l1.y - l2.y) - ak * ad.y - c2 * (l2.y - l3.y);
        Pn[e] = out;
      }
      __syncthreads();
      const int t = i3;
      i3 = i2;
      i2 = i1;
      i1 = in;
      in = t;
    }
    const float2* L = buf + i1 * UU;
    for (int e = tid; e < UU; e += NTHR) {  // B = L_K G, G = A - sigma I
      const int i = e / U, j = e - (e / U) * U;
      float2 s = make_float2(0.f, 0.f);
      for (int m = 0; m < U; ++m) {
        float2 gmj = sA[m * UT + j];
        if (m == j) gmj.x -= sigma;
        cmac(s, L[i * U + m], gmj);
      }
      Bm[e] = s;
    }
    __syncthreads();
    for (int i = tid; i < U; i += NTHR) {
      const float mu = Bm[i * U + i].x;
      float interf = 0.f, cii = 0.f;
      for (int j = 0; j < U; ++j) {
        const float2 bij = Bm[i * U + j];
        const float2 lij = L[i * U + j];
        if (j != i) interf = fmaf(bij.x, bij.x, fmaf(bij.y, bij.y, interf));
        cii = fmaf(bij.x, lij.x, fmaf(bij.y, lij.y, cii));  // Re(B_ij conj(L_ij))
      }
      const float nu2 = interf * Es + cii * N0;
      sMu[r * UT + i] = mu;
      sRho[r * UT + i] = (nu2 > 0.f) ? mu * mu / nu2 : 0.f;
    }
    __syncthreads();
  }
}

// --------------------------------------------------------------------------
// Step 5: max-log LLRs (Eq. 4) on one axis of square Gray QAM
// --------------------------------------------------------------------------

// For a product labelling, Eq. 4 separates into one 1-D minimisation per
// axis: level j = (2j - (L-1)) c carries the Gray word j ^ (j >> 1), bit t
// of the axis is bit (h-1-t) of that word.
__device__ __forceinline__ void axis_llr(float x, int h, float c, float rho, float* out) {
  const int L = 1 << h;
  float m0[4], m1[4];
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    m0[t] = INFINITY;
    m1[t] = INFINITY;
  }
  for (int j = 0; j < L; ++j) {
    const float dl = x - float(2 * j - (L - 1)) * c;
    const float d = dl * dl;
    const int gw = j ^ (j >> 1);
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      if (t < h) {
        if ((gw >> (h - 1 - t)) & 1)
          m1[t] = fminf(m1[t], d);
        else
          m0[t] = fminf(m0[t], d);
      }
    }
  }
#pragma unroll
  for (int t = 0; t < 4; ++t)
    if (t < h) out[t] = rho * (m0[t] - m1[t]);
}

// Compile-time form for H bits per axis: the Gray word of every level and the
// bit partition are constants, so each level costs one FMA, one multiply and
// H min operations.
template <int H>
__device__ __forceinline__ void axis_llr_t(float x, float c, float rho, float (&out)[H]) {
  constexpr int L = 1 << H;
  float m0[H], m1[H];
#pragma unroll
  for (int t = 0; t < H; ++t) m0[t] = m1[t] = INFINITY;
#pragma unroll
  for (int j = 0; j < L; ++j) {
    const float dl = fmaf(-float(2 * j - (L - 1)), c, x);
    const float d = dl * dl;
    const int gw = j ^ (j >> 1);
#pragma unroll
    for (int t = 0; t < H; ++t) {
      if ((gw >> (H - 1 - t)) & 1)
        m1[t] = fminf(m1[t], d);
      else
        m0[t] = fminf(m0[t], d);
    }
  }
#pragma unroll
  for (int t = 0; t < H; ++t) out[t] = rho * (m0[t] - m1[t]);
}

// LLRs of one user (2H bits: in-phase bits first) into dst (8-byte aligned);
// zeros when the user has no valid mu.
template <int H>
__device__ __forceinline__ void store_llr(float* dst, float2 z, float c, float rho, bool valid) {
  float v[2 * H];
  if (valid) {
    float lI[H], lQ[H];
    axis_llr_t<H>(z.x, c, rho, lI);
    axis_llr_t<H>(z.y, c, rho, lQ);
#pragma unroll
    for (int t = 0; t < H; ++t) {
      v[t] = lI[t];
      v[H + t] = lQ[t];
    }
  } else {
#pragma unroll
    for (int t = 0; t < 2 * H; ++t) v[t] = 0.f;
  }
  float2* d2 = reinterpret_cast<float2*>(dst);
#pragma unroll
  for (int k = 0; k < H; ++k) d2[k] = make_float2(v[2 * k], v[2 * k + 1]);
}

// Step 5 of CG-D for instance n: x_hat, mu, rho and the max-log LLRs of
// Eq. 4 for every (right-hand side, user), consecutive threads on
// consecutive outputs. z = x_hat / mu; users with mu <= 0 get zero LLRs and
// flag ST_MU_NONPOS.
template <int UT, int NTHR>
__device__ __forceinline__ void write_detect_outputs(const DetectArgs& a, int64_t n,
                                                     const float2* sX, const float* sMu,
                                                     const float* sRho, int* sStatus) {
  const int U = a.U, R = a.R;
  const float cq = sqrtf(3.f * a.Es / (2.f * float((1 << a.q) - 1)));
  int flags = 0;
  const bool full = (U == UT);
  for (int tt = threadIdx.x; tt < R * U; tt += NTHR) {
    const int r = full ? tt / UT : tt / U;
    const int i = tt - r * U;
    const float2 x = sX[r * UT + i];
    const float mu = sMu[r * UT + i];
    const float rho = sRho[r * UT + i];
    const int64_t o = (n * R + r) * U + i;
    if (a.xhat) a.xhat[o] = x;
    if (a.mu) a.mu[o] = mu;
    if (a.rho) a.rho[o] = rho;
    const bool valid = mu > 0.f;
    if (!valid) flags |= ST_MU_NONPOS;
    if (a.llr) {
      const float inv = valid ? 1.f / mu : 0.f;
      const float2 z = make_float2(x.x * inv, x.y * inv);
      float* dst = a.llr + o * a.q;
      switch (a.q) {
        case 2: store_llr<1>(dst, z, cq, rho, valid); break;
        case 4: store_llr<2>(dst, z, cq, rho, valid); break;
        case 6: store_llr<3>(dst, z, cq, rho, valid); break;
        default: store_llr<4>(dst, z, cq, rho, valid); break;
      }
    }
  }
  if (flags) atomicOr(sStatus, flags);
}

// --------------------------------------------------------------------------
// CG-D kernel
// --------------------------------------------------------------------------

template <int UT>
__global__ void __launch_bounds__(TileCfg<UT>::NTHR) detect_kernel(const DetectArgs a) {
  using C = TileCfg<UT>;
  constexpr int TM = C::TM, TN = C::TN, NTHR = C::NTHR;
  extern __shared__ __align__(128) unsigned char smem[];
  const SmemPlan P = detect_plan<UT>(a.B, a.U, a.R, a.exact);
  float2* sH = reinterpret_cast<float2*>(smem + P.H);
  float2* sY = reinterpret_cast<float2*>(smem + P.Y);
  float2* sPart = reinterpret_cast<float2*>(smem);  // reuses the H/Y region
  float2* sA = reinterpret_cast<float2*>(smem + P.A);
  float2* sBm = reinterpret_cast<float2*>(smem + P.Bm);
  float2* sX = reinterpret_cast<float2*>(smem + P.X);
  float* sMu = reinterpret_cast<float*>(smem + P.Mu);
  float* sRho = reinterpret_cast<float*>(smem + P.Rho);
  float* sGd = reinterpret_cast<float*>(smem + P.Gd);
  float* sAB = a.exact ? reinterpret_cast<float*>(smem + P.AB) : nullptr;
  int* sKd = reinterpret_cast<int*>(smem + P.Kd);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + P.misc);
  int* sStatus = reinterpret_cast<int*>(smem + P.misc + 8);
  const int tid = threadIdx.x;
  const int U = a.U, R = a.R;

  if (tid == 0) mbar_init(bar, 1);
  __syncthreads();
  uint32_t parity = 0;
  int64_t n = blockIdx.x;
  if (a.bulk && n < a.n_inst && tid == 0) issue_detect_copies(a, P, smem, bar, n);

  for (; n < a.n_inst; n += gridDim.x) {
    // ---- step 1: inputs of instance n in shared memory
    if (a.bulk) {
      if (!wait_inputs(bar, parity, a.wait_ns)) {
        if (tid == 0 && a.status) a.status[n] = ST_TIMEOUT;
        mbar_wait_bounded(bar, parity, WAIT_TIMEOUT_NS);  // let in-flight copies land
        return;
      }
      parity ^= 1u;
    } else {
      coop_load_detect<NTHR>(a, P, smem, n);
      __syncthreads();
    }
    if (tid == 0) *sStatus = 0;

    // ---- step 2: G and the matched filters (Algorithm 1; Eqs. 7, 8)
    float2 acc[TM][TN];
    int tile, slice;
    gram_tile<UT, true>(sH, sY, P.YS, a.B, U, R, P, acc, tile, slice);
    __syncthreads();  // every read of H and Y is done
    // partial entry (slice, m, n, tile) at ((slice * TM*TN + m*TN + n) * NT + tile):
    // consecutive threads (tiles) store to consecutive addresses
    if (tile >= 0) {
      float2* dst = sPart + size_t(slice) * (TM * TN) * P.NT + tile;
#pragma unroll
      for (int m = 0; m < TM; ++m)
#pragma unroll
        for (int nn = 0; nn < TN; ++nn) dst[(m * TN + nn) * P.NT] = acc[m][nn];
    }
    __syncthreads();
    {
      const int E = P.NT * TM * TN;
      for (int e = tid; e < E; e += NTHR) {
        float2 s = sPart[e];
        for (int sl = 1; sl < P.NSL; ++sl) {
          const float2 t = sPart[sl * E + e];
          s.x += t.x;
          s.y += t.y;
        }
        const int mn = e / P.NT, t = e - mn * P.NT;
        const int ti = t / P.NCT, tj = t - ti * P.NCT;
        const int i = ti * TM + mn / TN, nn = mn % TN;
        const bool is_gram = tj < P.NCTH;
        const int col = is_gram ? tj * TN + nn : (tj - P.NCTH) * TN + nn;
        store_reduced(UT, i, col, is_gram, s, U, R, a.sigma, sA, sBm, sGd);
      }
    }
    __syncthreads();

    const int64_t next = n + gridDim.x;
    if (a.bulk && !a.exact && next < a.n_inst && tid == 0) {
      fence_proxy_async_smem();
      issue_detect_copies(a, P, smem, bar, next);
    }

    // ---- step 3: the CG iterations and tracker updates of Algorithm 1
    cg_groups<UT, NTHR>(sA, sBm, sGd, R, a.K, a.N0, true, sX, sMu, sRho, sAB, sKd, sStatus);
    __syncthreads();

    // ---- step 4: exact SINR (Eq. 10)
    if (a.exact) {
      exact_tracker<UT, NTHR>(reinterpret_cast<float2*>(smem), sA, sAB, sKd, U, R, a.sigma,
                              a.N0, a.Es, sMu, sRho);
      __syncthreads();
      if (a.bulk && next < a.n_inst && tid == 0) {
        fence_proxy_async_smem();
        issue_detect_copies(a, P, smem, bar, next);
      }
    }

    // ---- step 5: outputs (x_hat, mu, rho, LLRs of Eq. 4)
    write_detect_outputs<UT, NTHR>(a, n, sX, sMu, sRho, sStatus);
    __syncthreads();
    if (tid == 0 && a.status) a.status[n] = *sStatus;
  }
}

// --------------------------------------------------------------------------
// CG-P kernel
// --------------------------------------------------------------------------

// ||q||^2 = v^H H^H H v = v^H G v with G = A - sigma I, evaluated by the
// group that owns v; lets the epilogue normalise q in a single pass.
template <int UT>
__device__ __forceinline__ float group_gram_quadform(const float2* __restrict__ sA, float2 v,
                                                     float sigma, unsigned mask) {
  const int i = threadIdx.x % UT;
  float2 w = make_float2(0.f, 0.f);
#pragma unroll
  for (int j = 0; j < UT; ++j) {
    float2 vj;
    vj.x = __shfl_sync(mask, v.x, j, UT);
    vj.y = __shfl_sync(mask, v.y, j, UT);
    cmac_conj(w, sA[j * UT + i], vj);
  }
  w.x = fmaf(-sigma, v.x, w.x);
  w.y = fmaf(-sigma, v.y, w.y);
  return group_sum_compensated<UT>(v.x * w.x + v.y * w.y, mask);
}

template <int UT>
__global__ void __launch_bounds__(TileCfg<UT>::NTHR) precode_kernel(const PrecodeArgs a) {
  using C = TileCfg<UT>;
  constexpr int TM = C::TM, TN = C::TN, NTHR = C::NTHR;
  constexpr int RC = 8;  // right-hand sides per epilogue work item
  extern __shared__ __align__(128) unsigned char smem[];
  const SmemPlan P = precode_plan<UT>(a.B, a.U, a.R);
  float2* sH = reinterpret_cast<float2*>(smem + P.H);
  float2* sT = reinterpret_cast<float2*>(smem + P.Y);
  float2* sPart = reinterpret_cast<float2*>(smem + P.Bm);
  float2* sA = reinterpret_cast<float2*>(smem + P.A);
  float2* sV = reinterpret_cast<float2*>(smem + P.X);
  float* sNrm = reinterpret_cast<float*>(smem + P.Nrm);
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
    // ---- step 1: inputs
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
    // Right-hand sides b = t (Sec. III-D), padded to UT users
    for (int e = tid; e < R * UT; e += NTHR) {
      const int r = e / UT, i = e - (e / UT) * UT;
      sV[e] = (i < U) ? sT[r * U + i] : make_float2(0.f, 0.f);
    }

    // ---- step 2: A = H_d H_d^H + sigma I = H^H H + sigma I (Sec. III-D)
    float2 acc[TM][TN];
    int tile, slice;
    gram_tile<UT, false>(sH, nullptr, 0, B, U, 1, P, acc, tile, slice);
    if (P.Bm != P.X) {
      // buffered: every slice stores its partial tile, one pass sums them in
      // slice order
      if (tile >= 0) {
        float2* dst = sPart + size_t(slice) * (TM * TN) * P.NT + tile;
#pragma unroll
        for (int m = 0; m < TM; ++m)
#pragma unroll
          for (int nn = 0; nn < TN; ++nn) dst[(m * TN + nn) * P.NT] = acc[m][nn];
      }
      __syncthreads();
      const int E = P.NT * TM * TN;
      for (int e = tid; e < E; e += NTHR) {
        float2 s = sPart[e];
        for (int sl = 1; sl < P.NSL; ++sl) {
          const float2 t = sPart[sl * E + e];
          s.x += t.x;
          s.y += t.y;
        }
        const int mn = e / P.NT, t = e - mn * P.NT;
        const int ti = t / P.NCT, tj = t - ti * P.NCT;
        sA[(ti * TM + mn / TN) * UT + tj * TN + mn % TN] = s;
      }
    } else {
      // sequential: slices accumulate into A one after another
      for (int sl = 0; sl < P.NSL; ++sl) {
        if (slice == sl) {
          const int ti = tile / P.NCT, tj = tile - ti * P.NCT;
#pragma unroll
          for (int m = 0; m < TM; ++m)
#pragma unroll
            for (int nn = 0; nn < TN; ++nn) {
              float2* d = sA + (ti * TM + m) * UT + tj * TN + nn;
              if (sl == 0) {
                *d = acc[m][nn];
              } else {
                d->x += acc[m][nn].x;
                d->y += acc[m][nn].y;
              }
            }
        }
        __syncthreads();
      }
    }
    __syncthreads();
    for (int e = tid; e < UT * UT; e += NTHR) {  // Hermitian completion, sigma, padding
      const int i = e / UT, j = e - (e / UT) * UT;
      if (i >= U || j >= U) {
        sA[e] = make_float2(0.f, 0.f);
      } else if (i == j) {
        sA[e] = make_float2(sA[e].x + a.sigma, 0.f);
      } else if (i > j) {
        const float2 u = sA[j * UT + i];
        sA[e] = make_float2(u.x, -u.y);
      }
    }
    __syncthreads();

    // ---- step 3: the CG iterations of Algorithm 1 (sV <- v_K), then ||q||^2 = v^H G v
    cg_groups<UT, NTHR>(sA, sV, nullptr, R, a.K, 1.f, false, sV, nullptr, nullptr, nullptr,
                        sKd, sStatus);
    {
      constexpr int NG = NTHR / UT;
      const unsigned mask = group_mask<UT>();
      const int g = tid / UT, i = tid % UT;
      for (int r = g; r < R; r += NG) {
        const float qq = group_gram_quadform<UT>(sA, sV[r * UT + i], a.sigma, mask);
        if (i == 0) {
          const float nr = sqrtf(fmaxf(qq, 0.f));
          sNrm[r] = nr;
          if (a.qnorm) a.qnorm[n * R + r] = nr;
        }
      }
    }
    __syncthreads();

    // ---- step 4: q = H_d^H v = H v (Sec. III-D), optionally s = q / ||q|| (Sec. II-B).
    // Work item = (antenna b, group of RC right-hand sides); the user index is
    // rotated by the lane so that a warp's H reads fall in distinct banks.
    {
      const int lane = tid & 31;
      const int ngr = (R + RC - 1) / RC;
      for (int it = tid; it < B * ngr; it += NTHR) {
        const int rg = it / B, b = it - rg * B;
        const int r0 = rg * RC;
        float2 qa[RC];
#pragma unroll
        for (int rr = 0; rr < RC; ++rr) qa[rr] = make_float2(0.f, 0.f);
        for (int jj = 0; jj < U; ++jj) {
          int j = jj + (lane % U);
          j = (j >= U) ? j - U : j;
          const float2 h = sH[b * U + j];
#pragma unroll
          for (int rr = 0; rr < RC; ++rr)
            if (r0 + rr < R) cmac(qa[rr], h, sV[(r0 + rr) * UT + j]);
        }
#pragma unroll
        for (int rr = 0; rr < RC; ++rr) {
          const int r = r0 + rr;
          if (r < R) {
            float2 val = qa[rr];
            if (a.normalize) {
              const float nr = sNrm[r];
              const float inv = nr > 0.f ? 1.f / nr : 0.f;
              val.x *= inv;
              val.y *= inv;
            }
            a.q[(n * R + r) * B + b] = val;
          }
        }
      }
    }
    __syncthreads();
    if (tid == 0 && a.status) a.status[n] = *sStatus;
  }
}

}  // namespace cgm
