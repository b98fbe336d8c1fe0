"""FP64 CPU oracle for CG-based soft-output MMSE detection and precoding.

TEST INFRASTRUCTURE. Only the tests, the smoke check and the benchmark's CPU
baseline arm may import this module. It shares no code with the CUDA path and
imports nothing from it; the two meet only at the seeded input generator.

Everything here follows Yin, Wu, Cavallaro and Studer, "Conjugate
Gradient-based Soft-Output Detection and Precoding in Massive MIMO Systems"
(arXiv 1404.0424), in its own order and notation:

  B, U     base-station antennas and users (Sec. II)
  H        uplink channel H_u, B x U (Eq. 1); downlink H_d = H_u^H (Sec. II-B)
  N0, Es   noise variance per complex entry and per-user symbol energy;
           the regulariser is rho_u^-1 = N0/Es (Eq. 2)
  A, G     regularised Gram H^H H + (N0/Es) I and Gram H^H H (Eq. 7, Sec. III-C)
  K        number of CG iterations (Algorithm 1), or of Neumann-series terms
           (Sec. III-F, the comparator at the end of this module)

The arithmetic is plain numpy in float64/complex128 with no blocking or
fusion: a matmul is the only library primitive used as a step. Loops run over
instances and right-hand sides one at a time.

Readings of points the paper leaves open (each is a stated convention that the
CUDA path implements independently):
  * Square Gray QAM: bits b_0..b_{q-1}; b_0..b_{q/2-1} label the in-phase
    axis and the rest the quadrature axis, each read MSB-first as a Gray code
    g; the level index is j with gray(j) = j ^ (j >> 1) = g and the level is
    (2j - (L-1)) * c * sqrt(Es), L = 2^(q/2), c = sqrt(3 / (2 (M - 1))).
  * LLR sign as printed in Eq. 4: L > 0 favours bit 1.
  * alpha uses Re(p^H e) (real in exact arithmetic, the step size of Algorithm 1).
  * The L-recursions of Eq. 10 and Eq. 11 start from L_1 = alpha_1 I and are
    applied for k >= 2, with alpha_k = 1, beta_k = 0 and L_k = 0 for k < 1.
  * Breakdown: if ||r_{k-1}||^2 is not > 0 or Re(p^H e) is not > 0, CG stops
    before iteration k; v and the trackers keep their last values and the
    instance is flagged STATUS_BREAKDOWN. With no completed iteration
    x_hat = 0 and mu = 0.
  * A user with mu <= 0 gets all-zero LLRs and flags STATUS_MU_NONPOS.
"""

from __future__ import annotations

import numpy as np

STATUS_OK = 0
STATUS_BREAKDOWN = 1
STATUS_MU_NONPOS = 2


# ----------------------------------------------------------------------------
# Regularised Gram, matched filter (Sec. III-B, Eqs. 7, 8; Algorithm 1)
# ----------------------------------------------------------------------------

def gram(H: np.ndarray) -> np.ndarray:
    """Gram matrix G = H^H H (Sec. III-C, the G of Eq. 12)."""
    H = np.asarray(H, dtype=np.complex128)
    return H.conj().T @ H


def regularised_gram(H: np.ndarray, N0: float, Es: float) -> np.ndarray:
    """A = H^H H + rho_u^-1 I with rho_u = Es/N0 (Eq. 7; Algorithm 1)."""
    U = H.shape[1]
    return gram(H) + (N0 / Es) * np.eye(U)


def matched_filter(H: np.ndarray, y: np.ndarray) -> np.ndarray:
    """b = H^H y (Eq. 8; Algorithm 1)."""
    H = np.asarray(H, dtype=np.complex128)
    return H.conj().T @ np.asarray(y, dtype=np.complex128)


# ----------------------------------------------------------------------------
# Exact inversion by Cholesky (Sec. III-F, "Exact Matrix Inversion")
# ----------------------------------------------------------------------------

def cholesky_lower(A: np.ndarray) -> np.ndarray:
    """Lower-triangular M with A = M M^H (Sec. III-F), textbook column order."""
    A = np.asarray(A, dtype=np.complex128)
    n = A.shape[0]
    M = np.zeros_like(A)
    for j in range(n):
        s = A[j, j].real - np.sum(np.abs(M[j, :j]) ** 2)
        if not s > 0:
            raise np.linalg.LinAlgError("matrix is not positive definite")
        M[j, j] = np.sqrt(s)
        for i in range(j + 1, n):
            M[i, j] = (A[i, j] - np.sum(M[i, :j] * np.conj(M[j, :j]))) / M[j, j]
    return M


def forward_substitution(M: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Solve M z = b for lower-triangular M."""
    n = M.shape[0]
    z = np.zeros(n, dtype=np.complex128)
    for i in range(n):
        z[i] = (b[i] - np.sum(M[i, :i] * z[:i])) / M[i, i]
    return z


def backward_substitution(M: np.ndarray, z: np.ndarray) -> np.ndarray:
    """Solve M^H x = z for lower-triangular M."""
    n = M.shape[0]
    Mh = M.conj().T
    x = np.zeros(n, dtype=np.complex128)
    for i in range(n - 1, -1, -1):
        x[i] = (z[i] - np.sum(Mh[i, i + 1:] * x[i + 1:])) / Mh[i, i]
    return x


def cholesky_solve(A: np.ndarray, b: np.ndarray) -> np.ndarray:
    """A^-1 b by Cholesky then forward and backward substitution (Sec. III-F)."""
    M = cholesky_lower(A)
    return backward_substitution(M, forward_substitution(M, np.asarray(b, np.complex128)))


def cholesky_inverse(A: np.ndarray) -> np.ndarray:
    """A^-1 column by column through cholesky_solve (Sec. III-F)."""
    M = cholesky_lower(A)
    n = A.shape[0]
    inv = np.zeros((n, n), dtype=np.complex128)
    for c in range(n):
        e = np.zeros(n, dtype=np.complex128)
        e[c] = 1.0
        inv[:, c] = backward_substitution(M, forward_substitution(M, e))
    return inv


# ----------------------------------------------------------------------------
# Exact soft-output MMSE detection (Eqs. 2, 3 and the model below Eq. 3)
# ----------------------------------------------------------------------------

def mmse_exact(H: np.ndarray, y: np.ndarray, N0: float, Es: float) -> dict:
    """Exact MMSE x_hat, mu and rho for one receive vector.

    W = (H^H H + (N0/Es) I)^-1 H^H (Eq. 2), x_hat = W y (Eq. 3);
    mu_i = w_i^H h_i, nu_i^2 = sum_{j != i} |w_i^H h_j|^2 Es + N0 ||w_i||^2,
    rho_i = mu_i^2 / nu_i^2 (model x_hat_i = mu_i x_i + z_i below Eq. 3).
    """
    H = np.asarray(H, dtype=np.complex128)
    A = regularised_gram(H, N0, Es)
    Ainv = cholesky_inverse(A)
    W = Ainv @ H.conj().T
    x_hat = cholesky_solve(A, matched_filter(H, y))
    Beff = W @ H                     # entries w_i^H h_j
    C = W @ W.conj().T               # diagonal entries ||w_i||^2
    U = H.shape[1]
    mu = np.real(np.diag(Beff)).copy()
    nu2 = np.zeros(U)
    for i in range(U):
        interf = sum(abs(Beff[i, j]) ** 2 for j in range(U) if j != i)
        nu2[i] = interf * Es + np.real(C[i, i]) * N0
    rho = mu ** 2 / nu2
    return {"x_hat": x_hat, "mu": mu, "nu2": nu2, "rho": rho, "W": W}


# ----------------------------------------------------------------------------
# Algorithm 1: conjugate gradients
# ----------------------------------------------------------------------------

def conjugate_gradient(A: np.ndarray, b: np.ndarray, K: int) -> dict:
    """K CG iterations of Algorithm 1 on A g = b.

    Returns v_K, the per-iteration alpha_k and beta_k (k = 1..K_done), every
    iterate v_0..v_{K_done}, and a breakdown flag (module docstring).
    """
    A = np.asarray(A, dtype=np.complex128)
    b = np.asarray(b, dtype=np.complex128)
    v = np.zeros_like(b)            # v_0 = 0
    r = b.copy()                    # r_0 = b
    p = r.copy()                    # p_0 = r_0
    rr = np.real(np.vdot(r, r))     # ||r_0||^2
    alphas, betas, iterates = [], [], [v.copy()]
    broke = False
    for _k in range(1, K + 1):
        if not rr > 0:
            broke = True
            break
        e = A @ p
        pe = np.real(np.vdot(p, e))             # p^H e
        if not pe > 0:
            broke = True
            break
        alpha = rr / pe
        v = v + alpha * p
        r = r - alpha * e
        rr_new = np.real(np.vdot(r, r))
        beta = rr_new / rr
        p = r + beta * p
        rr = rr_new
        alphas.append(alpha)
        betas.append(beta)
        iterates.append(v.copy())
    return {"v": v, "alphas": alphas, "betas": betas, "iterates": iterates,
            "k_done": len(alphas), "breakdown": broke}


def _coef(alphas, betas, k):
    """alpha_k and beta_k with the k < 1 conventions (alpha = 1, beta = 0)."""
    a = alphas[k - 1] if k >= 1 else 1.0
    bt = betas[k - 1] if k >= 1 else 0.0
    return a, bt


# ----------------------------------------------------------------------------
# SINR trackers (Sec. III-C)
# ----------------------------------------------------------------------------

def exact_tracker_L(alphas, betas, A: np.ndarray) -> list:
    """The matrices L_1..L_K of Eq. 10 (exact SINR computation).

    L_1 = alpha_1 I; for k >= 2
      L_k = L_{k-1} + (alpha_k (1 + beta_{k-1}) / alpha_{k-1} I - alpha_k A)(L_{k-1} - L_{k-2})
            - alpha_k beta_{k-2} / alpha_{k-2} (L_{k-2} - L_{k-3}),
    with L_k = 0 for k < 1. Returns [L_1, ..., L_K] (empty when K = 0).
    """
    U = A.shape[0]
    K = len(alphas)
    Ls = {}

    def L(k):
        return Ls[k] if k >= 1 else np.zeros((U, U), dtype=np.complex128)

    out = []
    for k in range(1, K + 1):
        if k == 1:
            Ls[1] = alphas[0] * np.eye(U, dtype=np.complex128)
        else:
            ak, _ = _coef(alphas, betas, k)
            ak1, bk1 = _coef(alphas, betas, k - 1)
            ak2, bk2 = _coef(alphas, betas, k - 2)
            step = (ak * (1.0 + bk1) / ak1) * np.eye(U) - ak * A
            Ls[k] = L(k - 1) + step @ (L(k - 1) - L(k - 2)) \
                - (ak * bk2 / ak2) * (L(k - 2) - L(k - 3))
        out.append(Ls[k])
    return out


def exact_tracker_sinr(L: np.ndarray, G: np.ndarray, N0: float, Es: float):
    """mu_{i|k}, nu^2_{i|k}, rho_{i|k} from L_k (Sec. III-C-1).

    B = L_k G, mu_i = B_ii, C = B L_k^H,
    nu_i^2 = sum_{j != i} |B_ij|^2 Es + C_ii N0, rho_i = mu_i^2 / nu_i^2.
    """
    U = G.shape[0]
    Bm = L @ G
    C = Bm @ L.conj().T
    mu = np.real(np.diag(Bm)).copy()
    nu2 = np.zeros(U)
    for i in range(U):
        interf = sum(abs(Bm[i, j]) ** 2 for j in range(U) if j != i)
        nu2[i] = interf * Es + np.real(C[i, i]) * N0
    with np.errstate(divide="ignore", invalid="ignore"):
        rho = np.where(nu2 > 0, mu ** 2 / np.where(nu2 > 0, nu2, 1.0), 0.0)
    return mu, nu2, rho


def approx_tracker_l(alphas, betas, D: np.ndarray) -> np.ndarray:
    """Diagonal of L~_K from Eq. 11 (A replaced by its diagonal D).

    Every matrix in the recursion is diagonal, so it runs per user i on the
    scalars l_{i,k}: l_{i,1} = alpha_1 and for k >= 2
      l_{i,k} = l_{i,k-1} + (alpha_k (1 + beta_{k-1}) / alpha_{k-1} - alpha_k D_ii)(l_{i,k-1} - l_{i,k-2})
                - alpha_k beta_{k-2} / alpha_{k-2} (l_{i,k-2} - l_{i,k-3}),
    with l_{i,k} = 0 for k < 1. Returns l_{i,K} (zeros when K = 0).
    """
    D = np.real(np.asarray(D))
    U = D.shape[0]
    K = len(alphas)
    hist = {}

    def l(k):
        return hist[k] if k >= 1 else np.zeros(U)

    for k in range(1, K + 1):
        if k == 1:
            hist[1] = alphas[0] * np.ones(U)
        else:
            ak, _ = _coef(alphas, betas, k)
            ak1, bk1 = _coef(alphas, betas, k - 1)
            ak2, bk2 = _coef(alphas, betas, k - 2)
            step = ak * (1.0 + bk1) / ak1 - ak * D
            hist[k] = l(k - 1) + step * (l(k - 1) - l(k - 2)) \
                - (ak * bk2 / ak2) * (l(k - 2) - l(k - 3))
    return l(K)


def approx_tracker_sinr(l: np.ndarray, G_diag: np.ndarray, N0: float):
    """mu_{i|k} ~ l_{i,k} G_ii (Eq. 12); nu^2 ~ N0 l^2 G_ii; rho ~ G_ii / N0 (Eq. 13)."""
    G_diag = np.real(np.asarray(G_diag))
    mu = l * G_diag
    nu2 = N0 * l ** 2 * G_diag
    rho = G_diag / N0
    return mu, nu2, rho


# ----------------------------------------------------------------------------
# Constellation and max-log LLRs (Eq. 4)
# ----------------------------------------------------------------------------

def _gray_inverse(g: int) -> int:
    """Index j with j ^ (j >> 1) == g."""
    j = 0
    while g:
        j ^= g
        g >>= 1
    return j


def qam_constellation(qam_bits: int, Es: float):
    """Points and bit labels of square Gray M-QAM with E|x|^2 = Es.

    Returns (points[M] complex, labels[M, q] in {0, 1}); point m carries the
    bits of m written MSB-first (module docstring for the labelling).
    """
    q = int(qam_bits)
    if q not in (2, 4, 6, 8):
        raise ValueError("qam_bits must be 2, 4, 6 or 8")
    M = 1 << q
    h = q // 2
    L = 1 << h
    c = np.sqrt(3.0 / (2.0 * (M - 1))) * np.sqrt(Es)
    pts = np.zeros(M, dtype=np.complex128)
    labels = np.zeros((M, q), dtype=np.int8)
    for m in range(M):
        bits = [(m >> (q - 1 - t)) & 1 for t in range(q)]
        gI = 0
        for t in range(h):
            gI = (gI << 1) | bits[t]
        gQ = 0
        for t in range(h, q):
            gQ = (gQ << 1) | bits[t]
        jI, jQ = _gray_inverse(gI), _gray_inverse(gQ)
        pts[m] = complex((2 * jI - (L - 1)) * c, (2 * jQ - (L - 1)) * c)
        labels[m] = bits
    return pts, labels


def maxlog_llr(x_hat: np.ndarray, mu: np.ndarray, rho: np.ndarray, qam_bits: int,
               Es: float):
    """Max-log LLRs of Eq. 4 by enumeration of every constellation point.

    L_{i,b} = rho_i (min_{a in X_b^0} |x_hat_i/mu_i - a|^2 - min_{a in X_b^1} |x_hat_i/mu_i - a|^2).
    Returns (llr[U, q], flag) with flag = STATUS_MU_NONPOS if some mu_i <= 0
    (that user's LLRs are zero).
    """
    pts, labels = qam_constellation(qam_bits, Es)
    U = len(x_hat)
    q = int(qam_bits)
    llr = np.zeros((U, q))
    flag = STATUS_OK
    for i in range(U):
        if not mu[i] > 0:
            flag |= STATUS_MU_NONPOS
            continue
        z = x_hat[i] / mu[i]
        d = np.abs(z - pts) ** 2
        for bit in range(q):
            d0 = np.min(d[labels[:, bit] == 0])
            d1 = np.min(d[labels[:, bit] == 1])
            llr[i, bit] = rho[i] * (d0 - d1)
    return llr, flag


# ----------------------------------------------------------------------------
# CG-D: soft-output detection (Sec. III-B, Algorithm 1, Sec. III-C)
# ----------------------------------------------------------------------------

def cg_detect_one(H: np.ndarray, y: np.ndarray, N0: float, Es: float, K: int,
                  qam_bits: int, tracker: str = "approx") -> dict:
    """Algorithm 1 for detection of one receive vector with the chosen tracker.

    tracker = "approx" uses Eqs. 11-13, "exact" uses Eq. 10 and the B, C
    expressions of Sec. III-C-1.
    """
    A = regularised_gram(H, N0, Es)
    G = gram(H)
    b = matched_filter(H, y)
    cg = conjugate_gradient(A, b, K)
    status = STATUS_BREAKDOWN if cg["breakdown"] else STATUS_OK
    U = H.shape[1]
    if tracker == "approx":
        l = approx_tracker_l(cg["alphas"], cg["betas"], np.real(np.diag(A)))
        mu, nu2, rho = approx_tracker_sinr(l, np.real(np.diag(G)), N0)
    elif tracker == "exact":
        Ls = exact_tracker_L(cg["alphas"], cg["betas"], A)
        LK = Ls[-1] if Ls else np.zeros((U, U), dtype=np.complex128)
        mu, nu2, rho = exact_tracker_sinr(LK, G, N0, Es)
    else:
        raise ValueError("tracker must be 'approx' or 'exact'")
    llr, flag = maxlog_llr(cg["v"], mu, rho, qam_bits, Es)
    return {"x_hat": cg["v"], "mu": mu, "nu2": nu2, "rho": rho, "llr": llr,
            "status": status | flag, "alphas": cg["alphas"], "betas": cg["betas"]}


def cg_detect(H: np.ndarray, Y: np.ndarray, N0: float, Es: float, K: int,
              qam_bits: int, tracker: str = "approx") -> dict:
    """CG-D over a batch: H[n, B, U], Y[n, R, B] -> x_hat[n, R, U], mu, rho[n, R, U],
    llr[n, R, U, q], status[n] (bitwise OR over the instance's right-hand sides)."""
    H = np.asarray(H)
    Y = np.asarray(Y)
    n, Bn, U = H.shape
    R = Y.shape[1]
    q = int(qam_bits)
    out = {"x_hat": np.zeros((n, R, U), np.complex128), "mu": np.zeros((n, R, U)),
           "rho": np.zeros((n, R, U)), "llr": np.zeros((n, R, U, q)),
           "status": np.zeros(n, np.int32)}
    for t in range(n):
        for r in range(R):
            o = cg_detect_one(H[t], Y[t, r], N0, Es, K, q, tracker)
            out["x_hat"][t, r] = o["x_hat"]
            out["mu"][t, r] = o["mu"]
            out["rho"][t, r] = o["rho"]
            out["llr"][t, r] = o["llr"]
            out["status"][t] |= o["status"]
    return out


# ----------------------------------------------------------------------------
# CG-P: precoding (Sec. III-D) and the exact MMSE precoder (Eqs. 5, 6)
# ----------------------------------------------------------------------------

def cg_precode_one(H: np.ndarray, t: np.ndarray, N0: float, Es: float, K: int) -> dict:
    """Algorithm 1 for precoding one transmit vector t (Sec. III-D).

    H_d = H_u^H, A = H_d H_d^H + rho_d^-1 I (Sec. III-D), b = t,
    K CG iterations, then q_K = H_d^H v_K (Sec. III-D) and s = q / ||q||_2
    (power normalisation, Sec. II-B).
    """
    Hd = np.asarray(H, dtype=np.complex128).conj().T
    U = Hd.shape[0]
    A = Hd @ Hd.conj().T + (N0 / Es) * np.eye(U)
    cg = conjugate_gradient(A, np.asarray(t, np.complex128), K)
    q = Hd.conj().T @ cg["v"]
    qn = float(np.sqrt(np.sum(np.abs(q) ** 2)))
    s = q / qn if qn > 0 else np.zeros_like(q)
    return {"q": q, "qnorm": qn, "s": s, "v": cg["v"], "alphas": cg["alphas"],
            "status": STATUS_BREAKDOWN if cg["breakdown"] else STATUS_OK}


def cg_precode(H: np.ndarray, T: np.ndarray, N0: float, Es: float, K: int) -> dict:
    """CG-P over a batch: H[n, B, U], T[n, R, U] -> q[n, R, B], qnorm[n, R],
    s[n, R, B], status[n]."""
    H = np.asarray(H)
    T = np.asarray(T)
    n, Bn, U = H.shape
    R = T.shape[1]
    out = {"q": np.zeros((n, R, Bn), np.complex128), "qnorm": np.zeros((n, R)),
           "s": np.zeros((n, R, Bn), np.complex128), "status": np.zeros(n, np.int32)}
    for i in range(n):
        for r in range(R):
            o = cg_precode_one(H[i], T[i, r], N0, Es, K)
            out["q"][i, r] = o["q"]
            out["qnorm"][i, r] = o["qnorm"]
            out["s"][i, r] = o["s"]
            out["status"][i] |= o["status"]
    return out


def mmse_precode_exact(H: np.ndarray, t: np.ndarray, N0: float, Es: float) -> np.ndarray:
    """q = P t with P = H_d^H (H_d H_d^H + rho_d^-1 I)^-1 formed explicitly (Eqs. 5, 6)."""
    Hd = np.asarray(H, dtype=np.complex128).conj().T
    U = Hd.shape[0]
    P = Hd.conj().T @ cholesky_inverse(Hd @ Hd.conj().T + (N0 / Es) * np.eye(U))
    return P @ np.asarray(t, np.complex128)


# ----------------------------------------------------------------------------
# Truncated Neumann series (Sec. III-F, approximate matrix inversion)
# ----------------------------------------------------------------------------

def neumann_inverse(A: np.ndarray, K: int) -> np.ndarray:
    """The K-term Neumann approximation of A^-1 (Sec. III-F): with A = D + E,
    D the diagonal of A and E the rest,
        A^-1 ~ sum_{k=0}^{K-1} (-D^-1 E)^k D^-1,
    formed as the matrix sum of its K terms (explicit powers)."""
    A = np.asarray(A, dtype=np.complex128)
    D = np.diag(np.diag(A))
    E = A - D
    Dinv = np.diag(1.0 / np.diag(A))
    M = -Dinv @ E
    term = Dinv.copy()          # k = 0: (-D^-1 E)^0 D^-1
    total = term.copy()
    for _ in range(1, K):
        term = M @ term         # (-D^-1 E)^k D^-1
        total = total + term
    return total


def neumann_detect_one(H: np.ndarray, y: np.ndarray, N0: float, Es: float, K: int) -> np.ndarray:
    """x_hat = A~^-1 H^H y with the K-term Neumann inverse of A = H^H H + rho_u^-1 I
    (Sec. III-F applied to the MMSE estimate of Eqs. 2-3)."""
    A = regularised_gram(H, N0, Es)
    return neumann_inverse(A, K) @ matched_filter(H, y)


def neumann_detect(H: np.ndarray, Y: np.ndarray, N0: float, Es: float, K: int) -> dict:
    """Neumann detection over a batch: H[n, B, U], Y[n, R, B] -> x_hat[n, R, U], status[n]
    (always STATUS_OK)."""
    H = np.asarray(H)
    Y = np.asarray(Y)
    n, _, U = H.shape
    R = Y.shape[1]
    x = np.zeros((n, R, U), np.complex128)
    for i in range(n):
        for r in range(R):
            x[i, r] = neumann_detect_one(H[i], Y[i, r], N0, Es, K)
    return {"x_hat": x, "status": np.zeros(n, np.int32)}


def neumann_precode_one(H: np.ndarray, t: np.ndarray, N0: float, Es: float, K: int) -> dict:
    """q = H_d^H A~^-1 t with the K-term Neumann inverse of A = H_d H_d^H + rho_d^-1 I
    (Sec. III-F applied to the precoder of Eqs. 5-6)."""
    Hd = np.asarray(H, dtype=np.complex128).conj().T
    U = Hd.shape[0]
    A = Hd @ Hd.conj().T + (N0 / Es) * np.eye(U)
    q = Hd.conj().T @ (neumann_inverse(A, K) @ np.asarray(t, np.complex128))
    qn = float(np.sqrt(np.sum(np.abs(q) ** 2)))
    return {"q": q, "qnorm": qn, "s": q / qn if qn > 0 else np.zeros_like(q)}


def neumann_precode(H: np.ndarray, T: np.ndarray, N0: float, Es: float, K: int) -> dict:
    """Neumann precoding over a batch: H[n, B, U], T[n, R, U] -> q[n, R, B], qnorm[n, R],
    s[n, R, B], status[n] (always STATUS_OK: the series has no breakdown)."""
    H = np.asarray(H)
    T = np.asarray(T)
    n, Bn, U = H.shape
    R = T.shape[1]
    out = {"q": np.zeros((n, R, Bn), np.complex128), "qnorm": np.zeros((n, R)),
           "s": np.zeros((n, R, Bn), np.complex128), "status": np.zeros(n, np.int32)}
    for i in range(n):
        for r in range(R):
            o = neumann_precode_one(H[i], T[i, r], N0, Es, K)
            out["q"][i, r] = o["q"]
            out["qnorm"][i, r] = o["qnorm"]
            out["s"][i, r] = o["s"]
    return out


# ----------------------------------------------------------------------------
# CG least squares (Sec. III-E): no Gram matrix
# ----------------------------------------------------------------------------

def cgls(Hbar: np.ndarray, ybar: np.ndarray, K: int) -> dict:
    """K iterations of CGLS [Paige and Saunders 1982] on min_x ||ybar - Hbar x||_2,
    started at x = 0 (Sec. III-E). Per iteration:
        q_k = Hbar p_k, alpha_k = gamma_{k-1} / ||q_k||^2, x_k = x_{k-1} + alpha_k p_k,
        r_k = r_{k-1} - alpha_k q_k, s_k = Hbar^H r_k, gamma_k = ||s_k||^2,
        beta_k = gamma_k / gamma_{k-1}, p_{k+1} = s_k + beta_k p_k,
    with r_0 = ybar, s_0 = p_1 = Hbar^H ybar. Breakdown as for CG: if gamma_{k-1}
    or ||q_k||^2 is not > 0 the iteration stops and x keeps its last value."""
    Hbar = np.asarray(Hbar, dtype=np.complex128)
    r = np.asarray(ybar, dtype=np.complex128).copy()
    s = Hbar.conj().T @ r
    p = s.copy()
    x = np.zeros_like(s)
    gamma = np.real(np.vdot(s, s))
    alphas, betas = [], []
    broke = False
    for _k in range(1, K + 1):
        if not gamma > 0:
            broke = True
            break
        q = Hbar @ p
        qq = np.real(np.vdot(q, q))
        if not qq > 0:
            broke = True
            break
        alpha = gamma / qq
        x = x + alpha * p
        r = r - alpha * q
        s = Hbar.conj().T @ r
        gamma_new = np.real(np.vdot(s, s))
        beta = gamma_new / gamma
        p = s + beta * p
        gamma = gamma_new
        alphas.append(alpha)
        betas.append(beta)
    return {"x": x, "alphas": alphas, "betas": betas, "breakdown": broke}


def cgls_detect_one(H: np.ndarray, y: np.ndarray, N0: float, Es: float, K: int,
                    qam_bits: int) -> dict:
    """CGLS detection (Sec. III-E): x_hat = argmin ||ybar - Hbar x|| after K CGLS
    iterations, with ybar = [y; 0_U] and Hbar = [H; sqrt(rho_u^-1) I_U]. The
    approximate SINR tracker of Eqs. 11-13 is built in with CGLS's own step
    sizes, then the LLRs of Eq. 4."""
    H = np.asarray(H, dtype=np.complex128)
    Bn, U = H.shape
    Hbar = np.vstack([H, np.sqrt(N0 / Es) * np.eye(U)])
    ybar = np.concatenate([np.asarray(y, np.complex128), np.zeros(U, np.complex128)])
    ls = cgls(Hbar, ybar, K)
    G = gram(H)
    D = np.real(np.diag(G)) + N0 / Es
    l = approx_tracker_l(ls["alphas"], ls["betas"], D)
    mu, nu2, rho = approx_tracker_sinr(l, np.real(np.diag(G)), N0)
    llr, flag = maxlog_llr(ls["x"], mu, rho, qam_bits, Es)
    status = (STATUS_BREAKDOWN if ls["breakdown"] else STATUS_OK) | flag
    return {"x_hat": ls["x"], "mu": mu, "nu2": nu2, "rho": rho, "llr": llr, "status": status,
            "alphas": ls["alphas"], "betas": ls["betas"]}


def cgls_detect(H: np.ndarray, Y: np.ndarray, N0: float, Es: float, K: int,
                qam_bits: int) -> dict:
    """CGLS detection over a batch, in the layout of cg_detect."""
    H = np.asarray(H)
    Y = np.asarray(Y)
    n, _, U = H.shape
    R = Y.shape[1]
    q = int(qam_bits)
    out = {"x_hat": np.zeros((n, R, U), np.complex128), "mu": np.zeros((n, R, U)),
           "rho": np.zeros((n, R, U)), "llr": np.zeros((n, R, U, q)),
           "status": np.zeros(n, np.int32)}
    for t in range(n):
        for r in range(R):
            o = cgls_detect_one(H[t], Y[t, r], N0, Es, K, q)
            out["x_hat"][t, r] = o["x_hat"]
            out["mu"][t, r] = o["mu"]
            out["rho"][t, r] = o["rho"]
            out["llr"][t, r] = o["llr"]
            out["status"][t] |= o["status"]
    return out


def cgls_precode_one(H: np.ndarray, t: np.ndarray, N0: float, Es: float, K: int) -> dict:
    """CGLS precoding (Sec. III-E): qbar = argmin ||t - Hbar_d qtilde|| after K CGLS
    iterations with Hbar_d = [H_d, sqrt(rho_d^-1) I_U], H_d = H_u^H; q is the first
    B entries of qbar, and s = q / ||q||."""
    H = np.asarray(H, dtype=np.complex128)
    Bn, U = H.shape
    Hbar_d = np.hstack([H.conj().T, np.sqrt(N0 / Es) * np.eye(U)])
    ls = cgls(Hbar_d, np.asarray(t, np.complex128), K)
    q = ls["x"][:Bn]
    qn = float(np.sqrt(np.sum(np.abs(q) ** 2)))
    return {"q": q, "qnorm": qn, "s": q / qn if qn > 0 else np.zeros_like(q),
            "status": STATUS_BREAKDOWN if ls["breakdown"] else STATUS_OK}


def cgls_precode(H: np.ndarray, T: np.ndarray, N0: float, Es: float, K: int) -> dict:
    """CGLS precoding over a batch, in the layout of cg_precode."""
    H = np.asarray(H)
    T = np.asarray(T)
    n, Bn, U = H.shape
    R = T.shape[1]
    out = {"q": np.zeros((n, R, Bn), np.complex128), "qnorm": np.zeros((n, R)),
           "s": np.zeros((n, R, Bn), np.complex128), "status": np.zeros(n, np.int32)}
    for i in range(n):
        for r in range(R):
            o = cgls_precode_one(H[i], T[i, r], N0, Es, K)
            out["q"][i, r] = o["q"]
            out["qnorm"][i, r] = o["qnorm"]
            out["s"][i, r] = o["s"]
            out["status"][i] |= o["status"]
    return out
