"""CG least squares (Sec. III-E, CG_AMUL_CGLS): the CUDA path through the C ABI
against the FP64 oracle's CGLS with the same K, at the parity tolerances of
tests/parity.py. Detection carries the approximate tracker and the LLRs;
precoding gives q = the first B entries of the CGLS solution."""

import numpy as np
import pytest

import oracle
from paper_1404_0424_gb300 import workload as wl
from tests.parity import check_detect, check_precode, to_np

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

CGLS = 3


@pytest.fixture(scope="module")
def cabi():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1404_0424_gb300 import build, cabi as c
    c.library(build.build())
    assert c.CG_AMUL_CGLS == CGLS
    return c


def detect(cabi, d, K, q):
    dev = torch.device("cuda:0")
    out = cabi.detect(torch.from_numpy(d["H"]).to(dev), torch.from_numpy(d["Y"]).to(dev),
                      d["N0"], K, q, d["Es"], amul_mode=CGLS)
    torch.cuda.synchronize()
    return {k: to_np(v) for k, v in out.items()}


@pytest.mark.parametrize("U", [8, 16])
@pytest.mark.parametrize("K", [1, 2, 3, 4])
def test_detect_128_antennas_14_symbols(cabi, U, K):
    d = wl.uplink(128, U, 6, n=3, R=14, snr_db=10.0, seed=1000 + U * 10 + K)
    check_detect(detect(cabi, d, K, 6), oracle.cgls_detect(d["H"], d["Y"], d["N0"], d["Es"], K, 6))


@pytest.mark.parametrize("B,U,R,K,q", [
    (1, 1, 1, 1, 2), (5, 3, 2, 2, 4), (33, 7, 5, 3, 6), (64, 13, 16, 5, 4), (130, 17, 3, 4, 8),
    (96, 24, 7, 6, 6), (256, 32, 14, 8, 8), (64, 8, 9, 8, 2)])
def test_detect_ragged_shapes(cabi, B, U, R, K, q):
    d = wl.uplink(B, U, q, n=4, R=R, snr_db=12.0, seed=1100 + B + U + R)
    check_detect(detect(cabi, d, K, q), oracle.cgls_detect(d["H"], d["Y"], d["N0"], d["Es"], K, q))


def test_detect_equals_cg_to_fp32_rounding(cabi):
    # in exact arithmetic CGLS detection is CG on the normal equations
    d = wl.uplink(128, 16, 6, n=4, R=14, snr_db=10.0, seed=1201)
    check_detect(detect(cabi, d, 3, 6), oracle.cg_detect(d["H"], d["Y"], d["N0"], d["Es"], 3, 6))


@pytest.mark.parametrize("B,U,R,K,normalize", [
    (128, 16, 14, 3, False), (128, 16, 14, 3, True), (128, 8, 14, 2, False), (33, 7, 5, 3, False),
    (256, 32, 14, 8, True), (64, 13, 16, 13, False), (9, 4, 16, 4, False)])
def test_precode(cabi, B, U, R, K, normalize):
    d = wl.downlink(B, U, 4, n=4, R=R, snr_db=12.0, seed=1300 + B + U + R)
    dev = torch.device("cuda:0")
    out = cabi.precode(torch.from_numpy(d["H"]).to(dev), torch.from_numpy(d["T"]).to(dev),
                       d["N0"], K, d["Es"], normalize=normalize, amul_mode=CGLS)
    torch.cuda.synchronize()
    check_precode({k: to_np(v) for k, v in out.items()},
                  oracle.cgls_precode(d["H"], d["T"], d["N0"], d["Es"], K), normalize)


def test_exact_tracker_is_not_supported(cabi):
    dev = torch.device("cuda:0")
    H = torch.zeros((1, 8, 2), dtype=torch.complex64, device=dev)
    Y = torch.zeros((1, 1, 8), dtype=torch.complex64, device=dev)
    x = torch.zeros((1, 1, 2), dtype=torch.complex64, device=dev)
    p = cabi.params(8, 2, 2, 1, 1, 0.5, sinr_mode=1, amul_mode=CGLS)
    assert cabi.cg_detect(p, 1, H, Y, x) == cabi.CG_ENOTSUP
    p = cabi.params(8, 2, 2, 1, 1, 0.5, amul_mode=4)
    assert cabi.cg_detect(p, 1, H, Y, x) == cabi.CG_EINVAL
