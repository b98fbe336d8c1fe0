"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Nothing here compares the oracle with itself: every check uses a hand-derived
example (tests/golden), a closed form, a library routine on an independent
route, an identity from the paper, or brute-force enumeration.
"""

import itertools

import numpy as np
import pytest

import oracle as orc
from paper_1404_0424_gb300 import workload as wl

RNG = np.random.default_rng(1234)


def crandn(rng, *shape):
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / np.sqrt(2)


def relerr(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300)


# ---------------------------------------------------------------------------
# Hand-derived examples (tests/golden/hand_examples.txt)
# ---------------------------------------------------------------------------

def test_golden_diag2_exact_mmse(golden):
    g = {k.split(".", 1)[1]: v for k, v in golden.items() if k.startswith("diag2.")}
    H = np.array(g["H"], complex)
    y = np.array(g["y"], complex)
    out = orc.mmse_exact(H, y, g["N0"], g["Es"])
    np.testing.assert_allclose(orc.matched_filter(H, y), g["b"], atol=1e-14)
    np.testing.assert_allclose(out["x_hat"], g["xhat_exact"], atol=1e-14)
    np.testing.assert_allclose(out["mu"], g["mu_exact"], atol=1e-14)
    np.testing.assert_allclose(out["nu2"], g["nu2_exact"], atol=1e-14)
    np.testing.assert_allclose(out["rho"], g["rho_exact"], atol=1e-13)


@pytest.mark.parametrize("tracker", ["approx", "exact"])
def test_golden_diag2_cg(golden, tracker):
    g = {k.split(".", 1)[1]: v for k, v in golden.items() if k.startswith("diag2.")}
    H = np.array(g["H"], complex)
    Y = np.array(g["y"], complex)
    o1 = orc.cg_detect_one(H, Y, g["N0"], g["Es"], 1, g["qam_bits"], tracker)
    assert o1["alphas"][0] == pytest.approx(g["alpha1"], rel=1e-15)
    np.testing.assert_allclose(o1["x_hat"], g["v1"], atol=1e-14)
    np.testing.assert_allclose(o1["mu"], g["mu_K1"], atol=1e-14)
    np.testing.assert_allclose(o1["rho"], g["rho_K1"], atol=1e-12)
    np.testing.assert_allclose(o1["llr"], g["llr_K1"], atol=1e-12)
    o2 = orc.cg_detect_one(H, Y, g["N0"], g["Es"], 2, g["qam_bits"], tracker)
    np.testing.assert_allclose(o2["x_hat"], g["xhat_exact"], atol=1e-13)
    np.testing.assert_allclose(o2["mu"], g["mu_exact"], atol=1e-13)
    np.testing.assert_allclose(o2["rho"], g["rho_exact"], atol=1e-11)
    np.testing.assert_allclose(o2["llr"], g["llr_K2"], atol=1e-11)
    assert o2["status"] == orc.STATUS_OK


def test_golden_diag2_precode(golden):
    g = {k.split(".", 1)[1]: v for k, v in golden.items() if k.startswith("diag2.")}
    H = np.array(g["H"], complex)
    t = np.array(g["t"], complex)
    np.testing.assert_allclose(orc.mmse_precode_exact(H, t, g["N0"], g["Es"]),
                               g["q_exact"], atol=1e-14)
    o2 = orc.cg_precode_one(H, t, g["N0"], g["Es"], 2)
    np.testing.assert_allclose(o2["q"], g["q_exact"], atol=1e-14)
    assert o2["qnorm"] == pytest.approx(g["qnorm_exact"], rel=1e-14)
    np.testing.assert_allclose(np.linalg.norm(o2["s"]), 1.0, atol=1e-15)
    o1 = orc.cg_precode_one(H, t, g["N0"], g["Es"], 1)
    np.testing.assert_allclose(o1["q"], g["q_K1"], atol=1e-14)


def test_golden_scalar16(golden):
    g = {k.split(".", 1)[1]: v for k, v in golden.items() if k.startswith("scalar16.")}
    H = np.array(g["H"], complex)
    y = np.array(g["y"], complex)
    ex = orc.mmse_exact(H, y, g["N0"], g["Es"])
    np.testing.assert_allclose(ex["x_hat"], g["xhat_exact"], atol=1e-15)
    np.testing.assert_allclose(ex["mu"], g["mu_exact"], atol=1e-15)
    np.testing.assert_allclose(ex["rho"], g["rho_exact"], atol=1e-13)
    for tracker in ("approx", "exact"):
        o = orc.cg_detect_one(H, y, g["N0"], g["Es"], 1, g["qam_bits"], tracker)
        np.testing.assert_allclose(o["x_hat"], g["xhat_exact"], atol=1e-15)
        np.testing.assert_allclose(o["mu"], g["mu_exact"], atol=1e-15)
        np.testing.assert_allclose(o["rho"], g["rho_exact"], atol=1e-13)
        np.testing.assert_allclose(o["llr"], g["llr"], atol=1e-13)


# ---------------------------------------------------------------------------
# Exact MMSE through Cholesky against library routines and closed forms
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("B,U", [(1, 1), (4, 3), (32, 8), (64, 17), (256, 32)])
def test_cholesky_against_library(B, U):
    H = crandn(RNG, B, U)
    A = orc.regularised_gram(H, 0.3, 1.0)
    M = orc.cholesky_lower(A)
    np.testing.assert_allclose(M, np.linalg.cholesky(A), rtol=1e-12, atol=1e-12)
    b = crandn(RNG, U)
    np.testing.assert_allclose(orc.cholesky_solve(A, b), np.linalg.solve(A, b), rtol=1e-11)
    np.testing.assert_allclose(orc.cholesky_inverse(A), np.linalg.inv(A), rtol=1e-10,
                               atol=1e-13)


def test_mmse_2x2_closed_form_inverse():
    for _ in range(20):
        H = crandn(RNG, 2, 2)
        y = crandn(RNG, 2)
        N0, Es = RNG.uniform(0.05, 2.0), RNG.uniform(0.5, 2.0)
        G = np.array([[np.vdot(H[:, i], H[:, j]) for j in range(2)] for i in range(2)])
        a, bb, c, d = G[0, 0] + N0 / Es, G[0, 1], G[1, 0], G[1, 1] + N0 / Es
        Ainv = np.array([[d, -bb], [-c, a]]) / (a * d - bb * c)
        mf = np.array([np.vdot(H[:, 0], y), np.vdot(H[:, 1], y)])
        out = orc.mmse_exact(H, y, N0, Es)
        np.testing.assert_allclose(out["x_hat"], Ainv @ mf, rtol=1e-12)
        np.testing.assert_allclose(out["mu"], 1 - (N0 / Es) * np.real(np.diag(Ainv)),
                                   rtol=1e-12)


@pytest.mark.parametrize("B,U", [(8, 2), (32, 8), (128, 16)])
def test_mmse_sinr_identities(B, U):
    # B = W H = I - sigma A^-1 (Hermitian), so mu_i = 1 - sigma [A^-1]_ii,
    # nu_i^2 = Es mu_i (1 - mu_i) and rho_i = 1/(N0 [A^-1]_ii) - 1/Es.
    H = crandn(RNG, B, U)
    y = crandn(RNG, B)
    N0, Es = 0.4, 1.3
    out = orc.mmse_exact(H, y, N0, Es)
    Ainv_diag = np.real(np.diag(np.linalg.inv(H.conj().T @ H + N0 / Es * np.eye(U))))
    mu = 1 - (N0 / Es) * Ainv_diag
    np.testing.assert_allclose(out["mu"], mu, rtol=1e-11)
    np.testing.assert_allclose(out["nu2"], Es * mu * (1 - mu), rtol=1e-9)
    np.testing.assert_allclose(out["rho"], 1 / (N0 * Ainv_diag) - 1 / Es, rtol=1e-9)


def _enumerated_nu2(Wk, H, qam_bits, Es, N0):
    """Interference + noise variance of x_hat = Wk y by enumerating x over O^U."""
    U = H.shape[1]
    q = qam_bits
    labels = np.array(list(itertools.product([0, 1], repeat=q)), dtype=np.uint8)
    pts = wl.qam_map(labels, q, Es)
    Beff = Wk @ H
    nu2 = np.zeros(U)
    for i in range(U):
        acc = 0.0
        count = 0
        for xs in itertools.product(pts, repeat=U):
            z = sum(Beff[i, j] * xs[j] for j in range(U) if j != i)
            acc += abs(z) ** 2
            count += 1
        nu2[i] = acc / count + N0 * np.sum(np.abs(Wk[i]) ** 2)
    return np.real(np.diag(Beff)), nu2


@pytest.mark.parametrize("B", [2, 4])
def test_sinr_brute_force_enumeration(B):
    # x_hat = W y with y = H x + n: enumerate every x in O^U (16-QAM, U = 2),
    # noise part N0 ||w_i||^2. Exact MMSE (Eq. 2) and the CG-equivalent
    # L_1 H^H of Sec. III-C-1 at K = 1 < U.
    U, q, N0, Es = 2, 4, 0.3, 1.0
    H = crandn(RNG, B, U)
    y = crandn(RNG, B)
    ex = orc.mmse_exact(H, y, N0, Es)
    mu, nu2 = _enumerated_nu2(ex["W"], H, q, Es, N0)
    np.testing.assert_allclose(ex["mu"], mu, rtol=1e-12)
    np.testing.assert_allclose(ex["nu2"], nu2, rtol=1e-10)
    A = orc.regularised_gram(H, N0, Es)
    cg = orc.conjugate_gradient(A, orc.matched_filter(H, y), 1)
    L1 = orc.exact_tracker_L(cg["alphas"], cg["betas"], A)[-1]
    mu_t, nu2_t, rho_t = orc.exact_tracker_sinr(L1, orc.gram(H), N0, Es)
    mu_e, nu2_e = _enumerated_nu2(L1 @ H.conj().T, H, q, Es, N0)
    np.testing.assert_allclose(mu_t, mu_e, rtol=1e-12)
    np.testing.assert_allclose(nu2_t, nu2_e, rtol=1e-10)
    np.testing.assert_allclose(rho_t, mu_e ** 2 / nu2_e, rtol=1e-10)


# ---------------------------------------------------------------------------
# Algorithm 1: exactness, closed forms and the recursions of Sec. III-C
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("B,U", [(2, 2), (8, 4), (32, 8), (64, 16), (128, 16), (256, 32)])
def test_cg_at_K_equals_U_is_exact(B, U):
    H = crandn(RNG, B, U)
    y = crandn(RNG, B)
    N0, Es = 0.2, 1.0
    A = orc.regularised_gram(H, N0, Es)
    cg = orc.conjugate_gradient(A, orc.matched_filter(H, y), U)
    ref = np.linalg.solve(H.conj().T @ H + N0 / Es * np.eye(U), H.conj().T @ y)
    assert relerr(cg["v"], ref) < 1e-10


def test_cg_K1_closed_form():
    # v_1 = (||b||^2 / b^H A b) b; K = 1 CG-P is matched-filter precoding
    # q = alpha_1 H_d^H t (Sec. III-D).
    for B, U in [(8, 4), (64, 16)]:
        H = crandn(RNG, B, U)
        y = crandn(RNG, B)
        A = H.conj().T @ H + 0.5 * np.eye(U)
        b = H.conj().T @ y
        a1 = np.vdot(b, b).real / np.vdot(b, A @ b).real
        cg = orc.conjugate_gradient(orc.regularised_gram(H, 0.5, 1.0), orc.matched_filter(H, y), 1)
        np.testing.assert_allclose(cg["v"], a1 * b, rtol=1e-13)
        t = crandn(RNG, U)
        at = np.vdot(t, t).real / np.vdot(t, A @ t).real
        o = orc.cg_precode_one(H, t, 0.5, 1.0, 1)
        np.testing.assert_allclose(o["q"], at * (H @ t), rtol=1e-13)


def test_xhat_three_term_recursion_reproduces_cg():
    # Sec. III-C-1: x_hat_k = x_hat_{k-1} + (a_k (1 + b_{k-1}) / a_{k-1} I - a_k A)(x_hat_{k-1} - x_hat_{k-2})
    #                         - a_k b_{k-2} / a_{k-2} (x_hat_{k-2} - x_hat_{k-3}), x_hat_1 = a_1 b.
    B, U, K = 32, 8, 8
    H = crandn(RNG, B, U)
    y = crandn(RNG, B)
    A = orc.regularised_gram(H, 0.3, 1.0)
    b = orc.matched_filter(H, y)
    cg = orc.conjugate_gradient(A, b, K)
    al, be = cg["alphas"], cg["betas"]
    a = lambda k: al[k - 1] if k >= 1 else 1.0   # noqa: E731
    bt = lambda k: be[k - 1] if k >= 1 else 0.0  # noqa: E731
    xs = {k: np.zeros(U, complex) for k in (-2, -1, 0)}
    xs[1] = al[0] * b
    for k in range(2, K + 1):
        xs[k] = xs[k - 1] + (a(k) * (1 + bt(k - 1)) / a(k - 1) * (xs[k - 1] - xs[k - 2])
                             - a(k) * (A @ (xs[k - 1] - xs[k - 2]))) \
            - a(k) * bt(k - 2) / a(k - 2) * (xs[k - 2] - xs[k - 3])
    for k in range(1, K + 1):
        assert relerr(xs[k], cg["iterates"][k]) < 1e-11


def test_exact_tracker_L_reproduces_iterates():
    # Eq. 9: x_hat_k = L_k H^H y, so L_k b = v_k for every k.
    B, U, K = 64, 16, 16
    H = crandn(RNG, B, U)
    y = crandn(RNG, B)
    A = orc.regularised_gram(H, 0.25, 1.0)
    b = orc.matched_filter(H, y)
    cg = orc.conjugate_gradient(A, b, K)
    Ls = orc.exact_tracker_L(cg["alphas"], cg["betas"], A)
    for k in range(1, K + 1):
        assert relerr(Ls[k - 1] @ b, cg["iterates"][k]) < 1e-10
    # L_U = A^-1 (CG is exact at U)
    assert relerr(Ls[-1], np.linalg.inv(A)) < 1e-8


@pytest.mark.parametrize("B,U", [(8, 4), (32, 8), (128, 16)])
def test_exact_tracker_at_K_equals_U_matches_mmse(B, U):
    # Sec. III-C-1: at k = U the tracker gives the exact mu_i and rho_i.
    H = crandn(RNG, B, U)
    y = crandn(RNG, B)
    N0, Es = 0.5, 1.0
    o = orc.cg_detect_one(H, y, N0, Es, U, 4, "exact")
    ex = orc.mmse_exact(H, y, N0, Es)
    np.testing.assert_allclose(o["mu"], ex["mu"], rtol=1e-8)
    np.testing.assert_allclose(o["rho"], ex["rho"], rtol=1e-7)


def test_approx_tracker_rho_closed_form():
    # Eq. 13: rho ~ G_ii / N0, independent of k.
    H = crandn(RNG, 32, 8)
    y = crandn(RNG, 32)
    N0 = 0.7
    G_diag = np.sum(np.abs(H) ** 2, axis=0)
    for K in (1, 2, 5):
        o = orc.cg_detect_one(H, y, N0, 1.0, K, 4, "approx")
        np.testing.assert_allclose(o["rho"], G_diag / N0, rtol=1e-13)


def test_approx_equals_exact_when_gram_is_diagonal():
    # With orthogonal channel columns A = D, so Eq. 11 is Eq. 10.
    B, U = 16, 4
    F = np.exp(-2j * np.pi * np.outer(np.arange(B), np.arange(B)) / B)
    H = F[:, :U] * np.array([0.5, 1.0, 1.5, 2.0])
    y = crandn(RNG, B)
    N0, Es = 0.8, 1.0
    for K in range(1, U + 1):
        oa = orc.cg_detect_one(H, y, N0, Es, K, 4, "approx")
        oe = orc.cg_detect_one(H, y, N0, Es, K, 4, "exact")
        np.testing.assert_allclose(oa["mu"], oe["mu"], rtol=1e-10, atol=1e-14)


def test_approx_tracker_is_the_cg_polynomial_at_the_diagonal():
    # v_k = P_k(A) b for a degree-(k-1) real polynomial P_k, and Eq. 10 gives
    # L_k = P_k(A); Eq. 11 evaluates the same recursion at D, so
    # l_{i,k} = P_k(D_ii). P_k is recovered here from the iterate alone by a
    # least-squares fit in the Krylov basis b, Ab, ..., A^{k-1} b.
    B, U = 64, 8
    H = crandn(RNG, B, U)
    y = crandn(RNG, B)
    A = orc.regularised_gram(H, 0.4, 1.0)
    b = orc.matched_filter(H, y)
    D = np.real(np.diag(A))
    for K in (1, 2, 3, 4):
        cg = orc.conjugate_gradient(A, b, K)
        kry = np.stack([np.linalg.matrix_power(A, m) @ b for m in range(K)], axis=1)
        coef, *_ = np.linalg.lstsq(kry, cg["v"], rcond=None)
        assert np.max(np.abs(coef.imag)) < 1e-8 * np.max(np.abs(coef))
        P_at_D = sum(coef[m].real * D ** m for m in range(K))
        l = orc.approx_tracker_l(cg["alphas"], cg["betas"], D)
        np.testing.assert_allclose(l, P_at_D, rtol=1e-7)


# ---------------------------------------------------------------------------
# Constellation and max-log LLR (Eq. 4)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("q", [2, 4, 6, 8])
def test_constellation_energy_gray_and_generator(q):
    pts, labels = orc.qam_constellation(q, 1.7)
    assert np.mean(np.abs(pts) ** 2) == pytest.approx(1.7, rel=1e-13)
    # nearest neighbours (axis distance 2c) differ in exactly one bit
    c = np.sqrt(3 / (2 * (2 ** q - 1))) * np.sqrt(1.7)
    for m in range(len(pts)):
        for n in range(len(pts)):
            if abs(abs(pts[m] - pts[n]) - 2 * c) < 1e-9:
                assert np.sum(labels[m] != labels[n]) == 1
    # the generator's own mapping produces the same points for the same bits
    np.testing.assert_allclose(wl.qam_map(labels, q, 1.7), pts, atol=1e-13)


def test_llr_qpsk_closed_form():
    # QPSK levels -c (bit 0), +c (bit 1): Eq. 4 gives L = 4 c rho Re z, 4 c rho Im z.
    c = np.sqrt(0.5)
    for _ in range(50):
        z = complex(*RNG.standard_normal(2))
        mu, rho = RNG.uniform(0.2, 2.0), RNG.uniform(0.1, 10)
        llr, flag = orc.maxlog_llr(np.array([z * mu]), np.array([mu]), np.array([rho]), 2, 1.0)
        np.testing.assert_allclose(llr[0], [4 * c * rho * z.real, 4 * c * rho * z.imag],
                                   rtol=1e-12, atol=1e-12)
        assert flag == orc.STATUS_OK


def test_llr_16qam_closed_form():
    # Textbook piecewise-linear max-log LLRs of Gray 16-QAM (levels +-c, +-3c):
    # sign bit 4c x for |x| <= 2c, 8c (x - sign(x) c) beyond; inner bit 4c (2c - |x|).
    c = np.sqrt(0.1)

    def sign_bit(x):
        return 4 * c * x if abs(x) <= 2 * c else 8 * c * (x - np.sign(x) * c)

    for _ in range(200):
        z = complex(*(RNG.standard_normal(2) * 0.8))
        rho = RNG.uniform(0.1, 10)
        llr, _ = orc.maxlog_llr(np.array([z]), np.array([1.0]), np.array([rho]), 4, 1.0)
        expect = [sign_bit(z.real), 4 * c * (2 * c - abs(z.real)),
                  sign_bit(z.imag), 4 * c * (2 * c - abs(z.imag))]
        np.testing.assert_allclose(llr[0], rho * np.array(expect), rtol=1e-11, atol=1e-12)


@pytest.mark.parametrize("q", [6, 8])
def test_llr_matches_per_axis_enumeration(q):
    # For a product labelling Eq. 4 separates into two 1-D problems.
    lv = wl.pam_levels_by_gray_code(q, 1.0)
    h = q // 2
    for _ in range(30):
        z = complex(*(RNG.standard_normal(2)))
        llr, _ = orc.maxlog_llr(np.array([z]), np.array([1.0]), np.array([1.0]), q, 1.0)
        for axis, x in ((0, z.real), (1, z.imag)):
            for t in range(h):
                d = {0: np.inf, 1: np.inf}
                for gcode in range(1 << h):
                    bit = (gcode >> (h - 1 - t)) & 1
                    d[bit] = min(d[bit], (x - lv[gcode]) ** 2)
                assert llr[0, axis * h + t] == pytest.approx(d[0] - d[1], rel=1e-11, abs=1e-12)


@pytest.mark.parametrize("q", [2, 4, 6, 8])
def test_noiseless_hard_decisions_are_the_sent_bits(q):
    d = wl.uplink(32, 4, q, n=6, R=3, snr_db=60.0, seed=7, noiseless=True)
    out = orc.cg_detect(d["H"], d["Y"], 1e-6, d["Es"], K=4, qam_bits=q)
    hard = (out["llr"] > 0).astype(np.uint8)
    np.testing.assert_array_equal(hard, d["bits"])


# ---------------------------------------------------------------------------
# CG-P (Sec. III-D) against the explicit precoder of Eq. 6
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("B,U", [(8, 4), (64, 16), (128, 8)])
def test_precode_at_K_equals_U_is_exact(B, U):
    H = crandn(RNG, B, U)
    t = crandn(RNG, U)
    N0 = 0.3
    o = orc.cg_precode_one(H, t, N0, 1.0, U)
    q_solve = H @ np.linalg.solve(H.conj().T @ H + N0 * np.eye(U), t)
    assert relerr(o["q"], q_solve) < 1e-10
    assert relerr(orc.mmse_precode_exact(H, t, N0, 1.0), q_solve) < 1e-11


# ---------------------------------------------------------------------------
# Degenerate inputs (readings of silent points, stated in the oracle docstring)
# ---------------------------------------------------------------------------

def test_zero_receive_vector_is_degenerate():
    H = crandn(RNG, 16, 4)
    o = orc.cg_detect_one(H, np.zeros(16, complex), 0.5, 1.0, 3, 4, "approx")
    assert np.all(o["x_hat"] == 0) and np.all(o["mu"] == 0) and np.all(o["llr"] == 0)
    assert o["status"] == orc.STATUS_BREAKDOWN | orc.STATUS_MU_NONPOS


def test_exact_convergence_stops_the_iteration():
    # A = diag(2, 5), b = (2, 0): one step solves it exactly (r_1 = 0), so
    # iteration 2 meets ||r_1||^2 = 0 and CG stops with v = (1, 0).
    H = np.array([[1, 0], [0, 2]], complex)
    y = np.array([2, 0], complex)
    o = orc.cg_detect_one(H, y, 1.0, 1.0, 2, 2, "approx")
    np.testing.assert_array_equal(o["x_hat"], [1, 0])
    assert o["status"] & orc.STATUS_BREAKDOWN
    np.testing.assert_allclose(o["mu"], [0.5, 2.0])   # l_1 = alpha_1 = 1/2, mu = l G_ii


def test_exact_tracker_L_is_a_real_polynomial_in_A():
    # every L_k of Eq. 10 is a real-coefficient polynomial in A, hence Hermitian and
    # commuting with A (the property the tensor-core exact tracker relies on: it forms
    # A (L_{k-1} - L_{k-2}) as (L_{k-1} - L_{k-2}) A); and L_k b reproduces the iterate
    H = crandn(RNG, 40, 6)
    y = crandn(RNG, 40)
    A = orc.regularised_gram(H, 0.5, 1.0)
    b = orc.matched_filter(H, y)
    cg = orc.conjugate_gradient(A, b, 5)
    Ls = orc.exact_tracker_L(cg["alphas"], cg["betas"], A)
    assert len(Ls) == 5
    for k, L in enumerate(Ls, start=1):
        scale = np.abs(L).max()
        np.testing.assert_allclose(L @ A, A @ L, atol=1e-12 * scale * np.abs(A).max())
        np.testing.assert_allclose(L, L.conj().T, atol=1e-13 * scale)
        np.testing.assert_allclose(L @ b, cg["iterates"][k], rtol=1e-10)


# ---------------------------------------------------------------------------
# Truncated Neumann series (Sec. III-F)
# ---------------------------------------------------------------------------

def test_golden_neumann2(golden):
    g = {k.split(".", 1)[1]: v for k, v in golden.items() if k.startswith("neumann2.")}
    H = np.array(g["H"], complex)
    y = np.array(g["y"], complex)
    t = np.array(g["t"], complex)
    for K in (1, 2, 3):
        np.testing.assert_allclose(orc.neumann_detect_one(H, y, g["N0"], g["Es"], K),
                                   g[f"xhat_K{K}"], atol=1e-15)
    for K in (1, 2):
        np.testing.assert_allclose(orc.neumann_precode_one(H, t, g["N0"], g["Es"], K)["q"],
                                   g[f"q_K{K}"], atol=1e-15)
    # the series converges to the exact MMSE estimate (spectral radius of M is 1/sqrt(6))
    np.testing.assert_allclose(orc.neumann_detect_one(H, y, g["N0"], g["Es"], 60),
                               g["xhat_exact"], atol=1e-14)


def test_neumann_is_exact_for_a_diagonal_gram():
    # orthogonal columns: E = 0, so every K gives A^-1 b
    Q, _ = np.linalg.qr(crandn(RNG, 16, 4))
    H = Q * np.array([0.5, 1.0, 2.0, 3.0])
    y = crandn(RNG, 16)
    ex = orc.mmse_exact(H, y, 0.4, 1.0)["x_hat"]
    for K in (1, 2, 5):
        np.testing.assert_allclose(orc.neumann_detect_one(H, y, 0.4, 1.0, K), ex, rtol=1e-12)


@pytest.mark.parametrize("B,U", [(64, 4), (128, 8), (256, 16)])
def test_neumann_converges_to_mmse_when_diagonally_dominant(B, U):
    H = crandn(RNG, B, U)
    y = crandn(RNG, B)
    t = crandn(RNG, U)
    N0 = U / 10.0
    ex = orc.mmse_exact(H, y, N0, 1.0)["x_hat"]
    errs = [relerr(orc.neumann_detect_one(H, y, N0, 1.0, K), ex) for K in (1, 2, 3, 4)]
    assert all(b < a for a, b in zip(errs, errs[1:])), errs   # monotone for B >> U
    assert relerr(orc.neumann_detect_one(H, y, N0, 1.0, 60), ex) < 1e-10
    assert relerr(orc.neumann_precode_one(H, t, N0, 1.0, 60)["q"],
                  orc.mmse_precode_exact(H, t, N0, 1.0)) < 1e-10


def test_neumann_partial_sums_follow_the_jacobi_recursion():
    # sum_{k<K} (-D^-1 E)^k D^-1 b equals K steps of x <- D^-1 (b - E x) from x = 0,
    # computed here with vectors only (no matrix powers)
    H = crandn(RNG, 48, 6)
    y = crandn(RNG, 48)
    A = orc.regularised_gram(H, 0.5, 1.0)
    b = H.conj().T @ y
    d = np.array([A[i, i] for i in range(6)])
    x = np.zeros(6, complex)
    for K in range(1, 7):
        Ex = np.array([sum(A[i, j] * x[j] for j in range(6) if j != i) for i in range(6)])
        x = (b - Ex) / d
        np.testing.assert_allclose(orc.neumann_detect_one(H, y, 0.5, 1.0, K), x, rtol=1e-12)


# ---------------------------------------------------------------------------
# CG least squares (Sec. III-E)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("B,U,K", [(16, 4, 1), (32, 8, 3), (64, 8, 5), (128, 16, 3)])
def test_cgls_detection_iterates_equal_cg(B, U, K):
    # in exact arithmetic CGLS on [H; sqrt(sigma) I] runs CG on the normal equations
    # A x = H^H y: same iterate, same step sizes (a different algorithm, so an identity)
    H = crandn(RNG, B, U)
    y = crandn(RNG, B)
    N0 = U / 10.0
    o = orc.cgls_detect_one(H, y, N0, 1.0, K, 4)
    cg = orc.cg_detect_one(H, y, N0, 1.0, K, 4, "approx")
    assert relerr(o["x_hat"], cg["x_hat"]) < 1e-9
    np.testing.assert_allclose(o["alphas"], cg["alphas"], rtol=1e-9)
    np.testing.assert_allclose(o["betas"], cg["betas"], rtol=1e-8)
    np.testing.assert_allclose(o["mu"], cg["mu"], rtol=1e-9)


@pytest.mark.parametrize("B,U", [(8, 2), (32, 8), (64, 13)])
def test_cgls_is_exact_at_K_equals_U(B, U):
    H = crandn(RNG, B, U)
    y = crandn(RNG, B)
    t = crandn(RNG, U)
    N0 = U / 5.0
    assert relerr(orc.cgls_detect_one(H, y, N0, 1.0, U, 2)["x_hat"],
                  orc.mmse_exact(H, y, N0, 1.0)["x_hat"]) < 1e-9
    assert relerr(orc.cgls_precode_one(H, t, N0, 1.0, U)["q"],
                  orc.mmse_precode_exact(H, t, N0, 1.0)) < 1e-9


def test_golden_cgls_precode_K1(golden):
    g = {k.split(".", 1)[1]: v for k, v in golden.items() if k.startswith("diag2.")}
    c = {k.split(".", 1)[1]: v for k, v in golden.items() if k.startswith("cgls_diag2.")}
    o = orc.cgls_precode_one(np.array(g["H"], complex), np.array(g["t"], complex),
                             g["N0"], g["Es"], 1)
    np.testing.assert_allclose(o["q"], c["q_K1"], atol=1e-15)


@pytest.mark.parametrize("K", [1, 2, 3])
def test_cgls_precoding_minimises_the_residual_over_the_krylov_space(K):
    # qbar_K = Hbar_d^H z with z = argmin over span{t, A t, .., A^(K-1) t} of ||t - A z||
    # (a least-squares solve on an explicit Krylov basis), so q_K = H z
    H = crandn(RNG, 48, 6)
    t = crandn(RNG, 6)
    N0 = 0.6
    A = orc.regularised_gram(H, N0, 1.0)
    basis = np.stack([np.linalg.matrix_power(A, j) @ t for j in range(K)], axis=1)
    c, *_ = np.linalg.lstsq(A @ basis, t, rcond=None)
    assert relerr(orc.cgls_precode_one(H, t, N0, 1.0, K)["q"], H @ (basis @ c)) < 1e-9


# ---------------------------------------------------------------------------
# The pins catch planted mistakes (each mistake is planted in the oracle)
# ---------------------------------------------------------------------------

def _plant(monkeypatch, name, fn):
    import oracle.cgmimo_oracle as mod
    monkeypatch.setattr(mod, name, fn)
    if hasattr(orc, name):
        monkeypatch.setattr(orc, name, fn)


def test_planted_binary_labelling_is_caught(monkeypatch):
    _plant(monkeypatch, "_gray_inverse", lambda g: g)
    with pytest.raises(AssertionError):
        test_llr_16qam_closed_form()


def test_planted_unregularised_gram_is_caught(monkeypatch, golden):
    import oracle.cgmimo_oracle as mod
    _plant(monkeypatch, "regularised_gram", lambda H, N0, Es: mod.gram(H))
    with pytest.raises(AssertionError):
        test_golden_diag2_exact_mmse(golden)


def test_planted_tracker_sign_is_caught(monkeypatch):
    import oracle.cgmimo_oracle as mod
    orig = mod.approx_tracker_l

    def wrong(alphas, betas, D):
        return orig(alphas, betas, -np.asarray(D))
    _plant(monkeypatch, "approx_tracker_l", wrong)
    with pytest.raises(AssertionError):
        test_approx_tracker_is_the_cg_polynomial_at_the_diagonal()


def test_planted_dropped_interference_is_caught(monkeypatch):
    import oracle.cgmimo_oracle as mod

    def no_interf(L, G, N0, Es):
        mu = np.real(np.diag(L @ G))
        nu2 = N0 * np.real(np.diag(L @ G @ L.conj().T))
        return mu, nu2, mu ** 2 / nu2
    _plant(monkeypatch, "exact_tracker_sinr", no_interf)
    with pytest.raises(AssertionError):
        test_exact_tracker_at_K_equals_U_matches_mmse(32, 8)


def test_planted_neumann_sign_is_caught(monkeypatch, golden):
    import oracle.cgmimo_oracle as mod

    def plus_sign(A, K):
        A = np.asarray(A, complex)
        Dinv = np.diag(1.0 / np.diag(A))
        M = Dinv @ (A - np.diag(np.diag(A)))
        term, total = Dinv.copy(), Dinv.copy()
        for _ in range(1, K):
            term = M @ term
            total = total + term
        return total
    _plant(monkeypatch, "neumann_inverse", plus_sign)
    with pytest.raises(AssertionError):
        test_golden_neumann2(golden)


def test_planted_cgls_steepest_descent_is_caught(monkeypatch):
    import oracle.cgmimo_oracle as mod
    orig = mod.cgls

    def no_beta(Hbar, ybar, K):
        Hbar = np.asarray(Hbar, complex)
        x = np.zeros(Hbar.shape[1], complex)
        r = np.asarray(ybar, complex).copy()
        alphas, betas = [], []
        for _ in range(K):
            s = Hbar.conj().T @ r
            q = Hbar @ s
            a = np.real(np.vdot(s, s)) / np.real(np.vdot(q, q))
            x, r = x + a * s, r - a * q
            alphas.append(a)
            betas.append(0.0)
        return {"x": x, "alphas": alphas, "betas": betas, "breakdown": False}
    assert orig is not no_beta
    _plant(monkeypatch, "cgls", no_beta)
    with pytest.raises(AssertionError):
        test_cgls_detection_iterates_equal_cg(32, 8, 3)
