"""Neumann-series detection and precoding (Sec. III-F): the CUDA path through
the C ABI against the FP64 oracle's explicit K-term series, with the same K.

Tolerances are those of tests/parity.py (x_hat and q within 1e-4 relative
per instance and right-hand side, qnorm within 1e-4). The channels keep A
diagonally dominant (B >= 4 U), where the series converges; the split
precisions (FP16X3, BF16X3) are the FP32-accurate ones.
"""

import numpy as np
import pytest

import oracle
from paper_1404_0424_gb300 import workload as wl
from tests.parity import TOL_X, check_precode, to_np

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

FP16X3, BF16X3 = 4, 3


@pytest.fixture(scope="module")
def cabi():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1404_0424_gb300 import build, cabi as c
    c.library(build.build())
    return c


def check_xhat(x, ref):
    x = to_np(x).astype(np.complex128)
    nr = np.linalg.norm(ref, axis=-1)
    dx = np.linalg.norm(x - ref, axis=-1)
    assert np.all(dx[nr == 0] == 0)
    e = (dx[nr > 0] / nr[nr > 0]).max()
    assert e <= TOL_X, f"x_hat relative error {e:.3e} > {TOL_X}"


def detect(cabi, d, K, precision):
    dev = torch.device("cuda:0")
    out = cabi.neumann_detect(torch.from_numpy(d["H"]).to(dev), torch.from_numpy(d["Y"]).to(dev),
                              d["N0"], K, d["Es"], precision=precision)
    torch.cuda.synchronize()
    return out


@pytest.mark.parametrize("precision", [FP16X3, BF16X3])
@pytest.mark.parametrize("U", [8, 16])
@pytest.mark.parametrize("K", [1, 2, 3, 4])
def test_detect_128_antennas_14_symbols(cabi, precision, U, K):
    d = wl.uplink(128, U, 6, n=4, R=14, snr_db=10.0, seed=500 + U * 10 + K)
    out = detect(cabi, d, K, precision)
    ref = oracle.neumann_detect(d["H"], d["Y"], d["N0"], d["Es"], K)
    check_xhat(out["xhat"], ref["x_hat"])
    assert int(out["status"].abs().sum()) == 0


@pytest.mark.parametrize("B,U,R,K", [
    (4, 1, 1, 1), (8, 2, 3, 2), (21, 5, 2, 3), (64, 13, 16, 5), (130, 17, 3, 4),
    (128, 24, 7, 6), (256, 32, 14, 8), (200, 31, 1, 2), (64, 8, 9, 16)])
def test_detect_ragged_shapes(cabi, B, U, R, K):
    d = wl.uplink(B, U, 4, n=5, R=R, snr_db=12.0, seed=600 + B + U + R)
    out = detect(cabi, d, K, FP16X3)
    check_xhat(out["xhat"], oracle.neumann_detect(d["H"], d["Y"], d["N0"], d["Es"], K)["x_hat"])


@pytest.mark.parametrize("B,U,R,K,normalize", [
    (128, 16, 14, 3, False), (128, 16, 14, 3, True), (128, 8, 14, 2, False),
    (33, 7, 5, 3, False), (256, 32, 14, 4, True), (64, 13, 16, 1, False)])
def test_precode(cabi, B, U, R, K, normalize):
    d = wl.downlink(B, U, 4, n=4, R=R, snr_db=12.0, seed=700 + B + U + R)
    dev = torch.device("cuda:0")
    out = cabi.neumann_precode(torch.from_numpy(d["H"]).to(dev), torch.from_numpy(d["T"]).to(dev),
                               d["N0"], K, d["Es"], normalize=normalize, precision=FP16X3)
    torch.cuda.synchronize()
    check_precode({k: to_np(v) for k, v in out.items()},
                  oracle.neumann_precode(d["H"], d["T"], d["N0"], d["Es"], K), normalize)


def test_series_approaches_exact_mmse_with_more_terms(cabi):
    # the GPU series at growing K moves towards the exact MMSE estimate
    d = wl.uplink(256, 8, 4, n=3, R=2, snr_db=15.0, seed=801)
    errs = []
    for K in (1, 4, 12):
        x = to_np(detect(cabi, d, K, FP16X3)["xhat"]).astype(np.complex128)
        e = 0.0
        for i in range(3):
            for r in range(2):
                ex = oracle.mmse_exact(d["H"][i], d["Y"][i, r], d["N0"], d["Es"])["x_hat"]
                e = max(e, np.linalg.norm(x[i, r] - ex) / np.linalg.norm(ex))
        errs.append(e)
    assert errs[0] > errs[1] > errs[2] and errs[2] < 1e-4, errs


def test_invalid_arguments(cabi):
    dev = torch.device("cuda:0")
    H = torch.zeros((2, 16, 4), dtype=torch.complex64, device=dev)
    Y = torch.zeros((2, 3, 16), dtype=torch.complex64, device=dev)
    x = torch.zeros((2, 3, 4), dtype=torch.complex64, device=dev)
    for K, prec, want in ((0, FP16X3, cabi.CG_EINVAL), (17, FP16X3, cabi.CG_EINVAL),
                          (3, 0, cabi.CG_ENOTSUP), (3, 9, cabi.CG_EINVAL)):
        p = cabi.params(16, 4, 2, K, 3, 0.5, precision=prec)
        assert cabi.cg_neumann_detect(p, 2, H, Y, x) == want, (K, prec)
    p = cabi.params(16, 4, 2, 3, 3, 0.5, precision=FP16X3)
    assert cabi.cg_neumann_detect(p, 2, H, Y, None) == cabi.CG_EINVAL
    assert cabi.cg_neumann_detect(p, 0, H, Y, x) == 0   # empty batch: nothing to do
    torch.cuda.synchronize()


def test_full_bench_size_sampled(cabi):
    # the bench configuration's batch (38,400 instances) in one call, sampled against FP64
    dev = torch.device("cuda:0")
    d = wl.uplink_torch(128, 16, 6, n=38400, R=14, snr_db=10.0, seed=901, device=dev)
    out = cabi.neumann_detect(d["H"], d["Y"], d["N0"], 3, precision=FP16X3)
    torch.cuda.synchronize()
    idx = np.sort(np.random.default_rng(9).choice(38400, 6, replace=False))
    ref = oracle.neumann_detect(d["H"][idx].cpu().numpy(), d["Y"][idx].cpu().numpy(),
                                d["N0"], 1.0, 3)
    check_xhat(out["xhat"][idx], ref["x_hat"])
    del d, out
    torch.cuda.empty_cache()
