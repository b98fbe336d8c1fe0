"""CG-P parity: the CUDA path (through the C ABI) against the FP64 oracle."""

import numpy as np
import pytest

import oracle
from paper_1404_0424_gb300 import workload as wl
from tests.parity import check_precode, to_np

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def cabi():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1404_0424_gb300 import build, cabi as c
    c.library(build.build())
    return c


def run(cabi, d, K, normalize=False):
    dev = torch.device("cuda:0")
    out = cabi.precode(torch.from_numpy(d["H"]).to(dev), torch.from_numpy(d["T"]).to(dev),
                       d["N0"], K, d["Es"], normalize=normalize)
    torch.cuda.synchronize()
    return {k: to_np(v) for k, v in out.items()}


def ref(d, K):
    return oracle.cg_precode(d["H"], d["T"], d["N0"], d["Es"], K)


@pytest.mark.parametrize("U", [8, 16])
@pytest.mark.parametrize("K", [2, 3, 4])
@pytest.mark.parametrize("normalize", [False, True])
def test_128_antennas_14_symbols(cabi, U, K, normalize):
    d = wl.downlink(128, U, 6, n=4, R=14, snr_db=10.0, seed=U * 10 + K)
    check_precode(run(cabi, d, K, normalize), ref(d, K), normalize)


@pytest.mark.parametrize("B,U,R,K", [
    (1, 1, 1, 1), (2, 2, 1, 2), (5, 3, 2, 2), (9, 4, 16, 4), (33, 7, 5, 3), (64, 13, 16, 5),
    (130, 17, 3, 4), (96, 24, 7, 6), (256, 32, 14, 8), (200, 31, 1, 2), (64, 8, 9, 8)])
def test_ragged_shapes(cabi, B, U, R, K):
    d = wl.downlink(B, U, 4, n=5, R=R, snr_db=12.0, seed=B * 100 + U + R)
    check_precode(run(cabi, d, K), ref(d, K))


@pytest.mark.parametrize("B,U", [(8, 4), (64, 16), (128, 32)])
def test_K_equals_U_is_exact_mmse_precoding(cabi, B, U):
    d = wl.downlink(B, U, 4, n=3, R=2, snr_db=10.0, seed=B + U)
    g = run(cabi, d, U)
    for t in range(3):
        for r in range(2):
            qe = oracle.mmse_precode_exact(d["H"][t], d["T"][t, r], d["N0"], d["Es"])
            e = np.linalg.norm(g["q"][t, r] - qe) / np.linalg.norm(qe)
            assert e <= 1e-4


def test_K1_is_matched_filter_precoding(cabi):
    d = wl.downlink(64, 8, 4, n=4, R=3, snr_db=10.0, seed=2)
    g = run(cabi, d, 1)
    for t in range(4):
        H = d["H"][t].astype(np.complex128)
        A = H.conj().T @ H + d["N0"] * np.eye(8)
        for r in range(3):
            tt = d["T"][t, r].astype(np.complex128)
            a1 = np.vdot(tt, tt).real / np.vdot(tt, A @ tt).real
            qe = a1 * (H @ tt)
            assert np.linalg.norm(g["q"][t, r] - qe) / np.linalg.norm(qe) <= 1e-5


def test_golden_diag2_precode_on_gpu(cabi, golden):
    g = {k.split(".", 1)[1]: v for k, v in golden.items() if k.startswith("diag2.")}
    d = {"H": np.array([g["H"]], np.complex64), "T": np.array([[g["t"]]], np.complex64),
         "N0": g["N0"], "Es": g["Es"]}
    out = run(cabi, d, 2)
    np.testing.assert_allclose(out["q"][0, 0], g["q_exact"], rtol=1e-6)
    np.testing.assert_allclose(out["qnorm"][0, 0], g["qnorm_exact"], rtol=1e-6)


def test_zero_symbols_are_degenerate(cabi):
    d = wl.downlink(32, 4, 4, n=3, R=2, snr_db=10.0, seed=4)
    d["T"][1] = 0
    g = run(cabi, d, 3)
    r = ref(d, 3)
    check_precode(g, r)
    assert np.all(g["q"][1] == 0) and g["status"][1] == oracle.STATUS_BREAKDOWN


def test_full_size_128x16_sampled(cabi):
    dev = torch.device("cuda:0")
    d = wl.downlink_torch(128, 16, 6, n=1200, R=14, snr_db=10.0, seed=43, device=dev)
    out = cabi.precode(d["H"], d["T"], d["N0"], 3)
    torch.cuda.synchronize()
    assert int(out["status"].abs().sum()) == 0
    idx = np.random.default_rng(1).choice(1200, 12, replace=False)
    r = oracle.cg_precode(d["H"][idx].cpu().numpy(), d["T"][idx].cpu().numpy(), d["N0"], 1.0, 3)
    check_precode({k: to_np(v[idx]) for k, v in out.items()}, r)


def test_host_variant_matches_device(cabi):
    d = wl.downlink(128, 16, 6, n=200, R=14, snr_db=10.0, seed=13)
    g = run(cabi, d, 3)
    q = np.empty((200, 14, 128), np.complex64)
    qn = np.empty((200, 14), np.float32)
    st = np.empty((200,), np.int32)
    p = cabi.params(128, 16, 6, 3, 14, d["N0"])
    rc = cabi.cg_precode_host(p, 200, d["H"], d["T"], q, qn, 0, st)
    assert rc == 0, cabi.cg_strerror(rc)
    assert np.array_equal(q, g["q"]) and np.array_equal(qn, g["qnorm"])


@pytest.mark.parametrize("B,U,R,K", [(128, 16, 14, 3), (128, 8, 1, 1), (256, 32, 3, 4),
                                     (33, 7, 5, 3), (1, 1, 1, 1)])
@pytest.mark.parametrize("normalize", [False, True])
def test_implicit_product_matches_oracle(cabi, B, U, R, K, normalize):
    d = wl.downlink(B, U, 6, n=4, R=R, snr_db=10.0, seed=8000 + B + U + R + K)
    dev = torch.device("cuda:0")
    out = cabi.precode(torch.from_numpy(d["H"]).to(dev), torch.from_numpy(d["T"]).to(dev),
                       d["N0"], K, d["Es"], normalize=normalize, amul_mode=2)
    torch.cuda.synchronize()
    check_precode({k: to_np(v) for k, v in out.items()},
                  oracle.cg_precode(d["H"], d["T"], d["N0"], d["Es"], K), normalize=normalize)


@pytest.mark.parametrize("normalize", [False, True])
def test_every_maximum_at_once(cabi, normalize):
    # B = CG_B_MAX, U = CG_U_MAX, R = CG_R_MAX, K = U
    d = wl.downlink(256, 32, 8, n=2, R=16, snr_db=12.0, seed=4343)
    check_precode(run(cabi, d, 32, normalize), ref(d, 32), normalize)
