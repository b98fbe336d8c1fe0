"""CG-D parity: the CUDA path (through the C ABI) against the FP64 oracle."""

import numpy as np
import pytest

import oracle
from paper_1404_0424_gb300 import workload as wl
from tests.parity import check_detect, to_np

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def cabi():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1404_0424_gb300 import build, cabi as c
    c.library(build.build())
    return c


def run(cabi, d, K, tracker="approx", **kw):
    dev = torch.device("cuda:0")
    H = torch.from_numpy(d["H"]).to(dev)
    Y = torch.from_numpy(d["Y"]).to(dev)
    out = cabi.detect(H, Y, d["N0"], K, d["qam_bits"], d["Es"],
                      sinr_mode=1 if tracker == "exact" else 0, **kw)
    torch.cuda.synchronize()
    return {k: to_np(v) for k, v in out.items()}


def ref(d, K, tracker="approx"):
    return oracle.cg_detect(d["H"], d["Y"], d["N0"], d["Es"], K, d["qam_bits"], tracker)


def test_small_uplink_32x4_16qam(cabi):
    # 32 antennas, 4 users, 16-QAM, 64 subcarriers x 1 symbol, 10 dB, K = 3
    d = wl.uplink(32, 4, 4, n=64, R=1, snr_db=10.0, seed=0)
    check_detect(run(cabi, d, 3), ref(d, 3))


@pytest.mark.parametrize("U", [8, 16])
@pytest.mark.parametrize("K", [2, 3, 4])
@pytest.mark.parametrize("snr", [0.0, 5.0, 10.0, 15.0, 20.0])
def test_128_antennas_64qam_14_symbols(cabi, U, K, snr):
    # the 128-antenna, 64-QAM, 14-symbol shape on a few subcarriers per point
    d = wl.uplink(128, U, 6, n=3, R=14, snr_db=snr, seed=100 + U + 10 * K + int(snr))
    check_detect(run(cabi, d, K), ref(d, K))


@pytest.mark.parametrize("B,U,R,K,q", [
    (1, 1, 1, 1, 2), (2, 2, 1, 2, 4), (4, 2, 3, 1, 2), (5, 3, 2, 2, 4), (9, 4, 16, 4, 8),
    (33, 7, 5, 3, 6), (64, 13, 16, 5, 4), (130, 17, 3, 4, 6), (96, 24, 7, 6, 8),
    (256, 32, 14, 8, 8), (200, 31, 1, 2, 2), (64, 8, 13, 8, 6)])
def test_ragged_shapes(cabi, B, U, R, K, q):
    d = wl.uplink(B, U, q, n=5, R=R, snr_db=12.0, seed=B * 1000 + U * 10 + R)
    check_detect(run(cabi, d, K), ref(d, K))


@pytest.mark.parametrize("B,U", [(8, 4), (32, 8), (64, 16), (128, 32)])
def test_K_equals_U_reaches_exact_mmse(cabi, B, U):
    d = wl.uplink(B, U, 4, n=4, R=2, snr_db=10.0, seed=B + U)
    g = run(cabi, d, U, tracker="exact")
    check_detect(g, ref(d, U, "exact"))
    for t in range(4):
        for r in range(2):
            ex = oracle.mmse_exact(d["H"][t], d["Y"][t, r], d["N0"], d["Es"])
            np.testing.assert_allclose(g["mu"][t, r], ex["mu"], rtol=1e-4)
            np.testing.assert_allclose(g["rho"][t, r], ex["rho"], rtol=1e-4)


@pytest.mark.parametrize("B,U,R,K", [(32, 4, 3, 1), (32, 4, 3, 2), (128, 16, 14, 3),
                                     (64, 8, 5, 8), (96, 12, 4, 5), (256, 32, 2, 4)])
def test_exact_tracker(cabi, B, U, R, K):
    d = wl.uplink(B, U, 6, n=3, R=R, snr_db=8.0, seed=7 * B + U + K)
    check_detect(run(cabi, d, K, "exact"), ref(d, K, "exact"))


def test_golden_diag2_on_gpu(cabi, golden):
    g = {k.split(".", 1)[1]: v for k, v in golden.items() if k.startswith("diag2.")}
    d = {"H": np.array([g["H"]], np.complex64), "Y": np.array([[g["y"]]], np.complex64),
         "N0": g["N0"], "Es": g["Es"], "qam_bits": g["qam_bits"]}
    out = run(cabi, d, 2)
    np.testing.assert_allclose(out["xhat"][0, 0], g["xhat_exact"], rtol=1e-6)
    np.testing.assert_allclose(out["mu"][0, 0], g["mu_exact"], rtol=1e-6)
    np.testing.assert_allclose(out["rho"][0, 0], g["rho_exact"], rtol=1e-6)
    np.testing.assert_allclose(out["llr"][0, 0], g["llr_K2"], rtol=1e-5)


def test_zero_receive_vectors_and_mixed_batch(cabi):
    d = wl.uplink(32, 4, 4, n=6, R=3, snr_db=10.0, seed=3)
    d["Y"][1] = 0
    d["Y"][4, 1] = 0
    g = run(cabi, d, 3)
    r = ref(d, 3)
    check_detect(g, r)
    assert np.all(g["xhat"][1] == 0) and np.all(g["llr"][1] == 0)
    assert g["status"][1] == oracle.STATUS_BREAKDOWN | oracle.STATUS_MU_NONPOS
    assert g["status"][0] == 0


def test_noiseless_hard_decisions(cabi):
    d = wl.uplink(64, 8, 6, n=8, R=4, snr_db=60.0, seed=11, noiseless=True)
    d["N0"] = 1e-6
    g = run(cabi, d, 8)
    np.testing.assert_array_equal((g["llr"] > 0).astype(np.uint8), d["bits"])


def test_repeatable_bitwise(cabi):
    d = wl.uplink(128, 16, 6, n=40, R=14, snr_db=10.0, seed=5)
    a = run(cabi, d, 3)
    b = run(cabi, d, 3)
    for k in a:
        assert np.array_equal(a[k], b[k]), k


def test_unaligned_and_odd_shapes_take_the_plain_load_path(cabi):
    # odd B (no bulk copies) and 8-byte (not 16-byte) aligned bases
    d = wl.uplink(33, 5, 4, n=7, R=3, snr_db=10.0, seed=9)
    check_detect(run(cabi, d, 3), ref(d, 3))
    d = wl.uplink(32, 4, 4, n=7, R=3, snr_db=10.0, seed=10)
    dev = torch.device("cuda:0")
    Hb = torch.zeros(d["H"].size + 1, dtype=torch.complex64, device=dev)
    Yb = torch.zeros(d["Y"].size + 1, dtype=torch.complex64, device=dev)
    H = Hb[1:].view(d["H"].shape)
    Y = Yb[1:].view(d["Y"].shape)
    H.copy_(torch.from_numpy(d["H"]))
    Y.copy_(torch.from_numpy(d["Y"]))
    assert H.data_ptr() % 16 == 8
    out = cabi.detect(H, Y, d["N0"], 3, 4)
    torch.cuda.synchronize()
    check_detect({k: to_np(v) for k, v in out.items()}, ref(d, 3))


def test_empty_batch_is_a_noop(cabi):
    p = cabi.params(32, 4, 4, 3, 1, 0.4)
    assert cabi.cg_detect(p, 0, None, None) == 0


def test_full_size_128x16_sampled(cabi):
    # 1200 subcarriers x 14 symbols, 128 x 16, 64-QAM, K = 3, the benchmark's
    # launch; the oracle checks a sample of subcarriers one by one.
    dev = torch.device("cuda:0")
    d = wl.uplink_torch(128, 16, 6, n=1200, R=14, snr_db=10.0, seed=42, device=dev)
    out = cabi.detect(d["H"], d["Y"], d["N0"], 3, 6)
    torch.cuda.synchronize()
    assert int(out["status"].abs().sum()) == 0
    for k in ("xhat", "mu", "rho", "llr"):
        assert bool(torch.isfinite(torch.view_as_real(out[k]) if out[k].is_complex()
                                   else out[k]).all())
    idx = np.random.default_rng(0).choice(1200, 12, replace=False)
    H = d["H"][idx].cpu().numpy()
    Y = d["Y"][idx].cpu().numpy()
    r = oracle.cg_detect(H, Y, d["N0"], 1.0, 3, 6)
    check_detect({k: to_np(v[idx]) for k, v in out.items()}, r)


def test_host_variant_matches_device(cabi):
    d = wl.uplink(128, 16, 6, n=300, R=14, snr_db=10.0, seed=12)
    g = run(cabi, d, 3)
    n, R, U, q = 300, 14, 16, 6
    xh = np.empty((n, R, U), np.complex64)
    mu = np.empty((n, R, U), np.float32)
    rho = np.empty((n, R, U), np.float32)
    llr = np.empty((n, R, U, q), np.float32)
    st = np.empty((n,), np.int32)
    p = cabi.params(128, 16, 6, 3, 14, d["N0"])
    rc = cabi.cg_detect_host(p, n, d["H"], d["Y"], xh, mu, rho, llr, st)
    assert rc == 0, cabi.cg_strerror(rc)
    assert np.array_equal(xh, g["xhat"]) and np.array_equal(llr, g["llr"])
    assert np.array_equal(mu, g["mu"]) and np.array_equal(st, g["status"])


@pytest.mark.parametrize("B,U,R,K,q", [
    (128, 16, 14, 3, 6), (128, 8, 14, 2, 6), (128, 16, 1, 1, 6), (32, 4, 1, 3, 4),
    (256, 32, 2, 4, 8), (33, 7, 5, 3, 6), (1, 1, 1, 1, 2), (64, 13, 16, 5, 4)])
def test_implicit_product_matches_oracle(cabi, B, U, R, K, q):
    # e = H^H (H p) + sigma p without forming the Gram (CG_AMUL_IMPLICIT)
    d = wl.uplink(B, U, q, n=4, R=R, snr_db=10.0, seed=7000 + B + U + R + K)
    check_detect(run(cabi, d, K, amul_mode=2), ref(d, K))


def test_auto_picks_the_product_by_cost_and_both_agree(cabi):
    # 4 K R < U + 1: AUTO applies A p implicitly on the FP32 path
    d = wl.uplink(128, 16, 6, n=6, R=1, snr_db=10.0, seed=71)
    auto = run(cabi, d, 2)
    expl = run(cabi, d, 2, amul_mode=1)
    impl = run(cabi, d, 2, amul_mode=2)
    for k in auto:
        assert np.array_equal(auto[k], impl[k]), k
    check_detect(expl, ref(d, 2))
    check_detect(impl, ref(d, 2))
    err = np.abs(impl["xhat"] - expl["xhat"]).max() / np.abs(expl["xhat"]).max()
    assert err < 1e-5


def test_implicit_product_with_exact_tracker_is_not_supported(cabi):
    d = wl.uplink(32, 4, 4, n=2, R=1, snr_db=10.0, seed=72)
    with pytest.raises(cabi.CgError):
        run(cabi, d, 2, tracker="exact", amul_mode=2)


@pytest.mark.parametrize("precision", [0, 4])
@pytest.mark.parametrize("tracker", ["approx", "exact"])
def test_every_maximum_at_once(cabi, precision, tracker):
    # B = CG_B_MAX, U = CG_U_MAX, R = CG_R_MAX, K = U, 256-QAM. At K = U the FP32
    # iteration may meet ||r||^2 = 0 or p^H A p <= 0 after it has converged to FP32
    # resolution and stop there with CG_STATUS_BREAKDOWN, where FP64 goes on: outputs
    # must still match, and an extra BREAKDOWN flag is accepted only for an instance
    # whose FP64 residual was already below 1e-5 (relative) one iteration before K
    K = 32
    d = wl.uplink(256, 32, 8, n=2, R=16, snr_db=12.0, seed=4242)
    g = run(cabi, d, K, tracker, precision=precision)
    r = ref(d, K, tracker)
    check_detect(g, r, check_status=False)
    for i in range(2):
        if g["status"][i] == r["status"][i]:
            continue
        assert g["status"][i] == r["status"][i] | oracle.STATUS_BREAKDOWN, (g["status"], r["status"])
        A = oracle.regularised_gram(d["H"][i], d["N0"], d["Es"])
        for rr in range(16):
            b = oracle.matched_filter(d["H"][i], d["Y"][i, rr])
            x = oracle.conjugate_gradient(A, b, K - 1)["v"]
            assert np.linalg.norm(b - A @ x) / np.linalg.norm(b) < 1e-5, (i, rr)
