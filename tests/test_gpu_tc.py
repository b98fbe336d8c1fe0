"""Tensor-core precision modes against the FP64 oracle.

The hi+lo split modes (CG_PREC_FP16X3, CG_PREC_BF16X3) must meet the same
tolerances as the FP32 path. The one-pass modes (CG_PREC_FP16, CG_PREC_BF16)
round H and Y to 11 / 8 significant bits, so their error is bounded by that
rounding instead: a relative Gram error of about 2^-12 (FP16) or 2^-9 (BF16)
times sqrt(B) / (B / U) amplified by cond(A) <= ~10; the loose bounds below
are twice those estimates.
"""

import numpy as np
import pytest

import oracle
from paper_1404_0424_gb300 import workload as wl
from tests.parity import check_detect, check_precode, to_np

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

X3 = {"fp16x3": 4, "bf16x3": 3}
ONE = {"fp16": (2, 5e-3), "bf16": (1, 4e-2)}


@pytest.fixture(scope="module")
def cabi():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1404_0424_gb300 import build, cabi as c
    c.library(build.build())
    return c


def run(cabi, d, K, precision, tracker="approx"):
    dev = torch.device("cuda:0")
    out = cabi.detect(torch.from_numpy(d["H"]).to(dev), torch.from_numpy(d["Y"]).to(dev),
                      d["N0"], K, d["qam_bits"], d["Es"],
                      sinr_mode=1 if tracker == "exact" else 0, precision=precision)
    torch.cuda.synchronize()
    return {k: to_np(v) for k, v in out.items()}


def runp(cabi, d, K, precision, normalize=False):
    dev = torch.device("cuda:0")
    out = cabi.precode(torch.from_numpy(d["H"]).to(dev), torch.from_numpy(d["T"]).to(dev),
                       d["N0"], K, d["Es"], normalize=normalize, precision=precision)
    torch.cuda.synchronize()
    return {k: to_np(v) for k, v in out.items()}


@pytest.mark.parametrize("mode", list(X3))
@pytest.mark.parametrize("U", [8, 16])
@pytest.mark.parametrize("K", [2, 3, 4])
@pytest.mark.parametrize("snr", [0.0, 10.0, 20.0])
def test_detect_128_antennas(cabi, mode, U, K, snr):
    d = wl.uplink(128, U, 6, n=3, R=14, snr_db=snr, seed=300 + U + 10 * K + int(snr))
    check_detect(run(cabi, d, K, X3[mode]), oracle.cg_detect(d["H"], d["Y"], d["N0"], 1.0, K, 6))


@pytest.mark.parametrize("mode", list(X3))
@pytest.mark.parametrize("B,U,R,K,q", [
    (1, 1, 1, 1, 2), (2, 2, 1, 2, 4), (5, 3, 2, 2, 4), (9, 4, 16, 4, 8), (33, 7, 5, 3, 6),
    (64, 13, 16, 5, 4), (130, 17, 3, 4, 6), (96, 24, 7, 6, 8), (256, 32, 14, 8, 8),
    (200, 31, 1, 2, 2), (64, 8, 13, 8, 6), (32, 4, 1, 3, 4), (128, 32, 9, 8, 6)])
def test_detect_ragged(cabi, mode, B, U, R, K, q):
    d = wl.uplink(B, U, q, n=5, R=R, snr_db=12.0, seed=B * 1000 + U * 10 + R)
    check_detect(run(cabi, d, K, X3[mode]),
                 oracle.cg_detect(d["H"], d["Y"], d["N0"], 1.0, K, q))


@pytest.mark.parametrize("mode", list(X3))
@pytest.mark.parametrize("B,U", [(8, 4), (32, 8), (64, 16), (128, 32)])
def test_detect_exact_tracker_at_K_equals_U(cabi, mode, B, U):
    d = wl.uplink(B, U, 4, n=4, R=2, snr_db=10.0, seed=B + U)
    g = run(cabi, d, U, X3[mode], "exact")
    check_detect(g, oracle.cg_detect(d["H"], d["Y"], d["N0"], 1.0, U, 4, "exact"))
    for t in range(4):
        for r in range(2):
            ex = oracle.mmse_exact(d["H"][t], d["Y"][t, r], d["N0"], 1.0)
            np.testing.assert_allclose(g["mu"][t, r], ex["mu"], rtol=1e-4)
            np.testing.assert_allclose(g["rho"][t, r], ex["rho"], rtol=1e-4)


@pytest.mark.parametrize("mode", list(X3))
@pytest.mark.parametrize("B,U,R,K", [(32, 4, 3, 1), (32, 4, 3, 2), (128, 16, 14, 3),
                                     (64, 8, 5, 8), (96, 12, 4, 5), (128, 16, 16, 16),
                                     (5, 3, 2, 2), (64, 13, 16, 5), (128, 16, 9, 4),
                                     (256, 32, 14, 8), (128, 32, 5, 3), (64, 32, 16, 12),
                                     (100, 17, 3, 6), (48, 24, 7, 24), (256, 32, 2, 32),
                                     (40, 32, 1, 1)])
def test_detect_exact_tracker_warp_kernel(cabi, mode, B, U, R, K):
    # the exact tracker (Eq. 10) runs in the warp kernel, its L_k recursion
    # as tensor-core products of 16 rows of L at a time (two halves at more
    # than 16 users); 8 dB keeps mu away from 1
    d = wl.uplink(B, U, 6, n=4, R=R, snr_db=8.0, seed=11 * B + U + K)
    check_detect(run(cabi, d, K, X3[mode], "exact"),
                 oracle.cg_detect(d["H"], d["Y"], d["N0"], 1.0, K, 6, "exact"))


@pytest.mark.parametrize("mode", list(X3))
def test_detect_degenerate_and_odd_layouts(cabi, mode):
    d = wl.uplink(33, 5, 4, n=6, R=3, snr_db=10.0, seed=9)   # odd B: plain loads
    d["Y"][2] = 0
    g = run(cabi, d, 3, X3[mode])
    check_detect(g, oracle.cg_detect(d["H"], d["Y"], d["N0"], 1.0, 3, 4))
    assert g["status"][2] == oracle.STATUS_BREAKDOWN | oracle.STATUS_MU_NONPOS


@pytest.mark.parametrize("mode", list(X3))
def test_detect_full_size_sampled_and_repeatable(cabi, mode):
    dev = torch.device("cuda:0")
    d = wl.uplink_torch(128, 16, 6, n=1200, R=14, snr_db=10.0, seed=44, device=dev)
    outs = []
    for _ in range(2):
        outs.append(cabi.detect(d["H"], d["Y"], d["N0"], 3, 6, precision=X3[mode]))
        torch.cuda.synchronize()
    for k in outs[0]:
        assert torch.equal(outs[0][k], outs[1][k]), k
    out = outs[0]
    assert int(out["status"].abs().sum()) == 0
    idx = np.random.default_rng(2).choice(1200, 12, replace=False)
    r = oracle.cg_detect(d["H"][idx].cpu().numpy(), d["Y"][idx].cpu().numpy(), d["N0"], 1.0, 3, 6)
    check_detect({k: to_np(v[idx]) for k, v in out.items()}, r)


@pytest.mark.parametrize("mode", list(ONE))
def test_detect_one_pass_error_is_bounded(cabi, mode):
    prec, bound = ONE[mode]
    d = wl.uplink(128, 16, 6, n=40, R=14, snr_db=10.0, seed=21)
    g = run(cabi, d, 3, prec)
    r = oracle.cg_detect(d["H"], d["Y"], d["N0"], 1.0, 3, 6)
    err = (np.linalg.norm(g["xhat"] - r["x_hat"], axis=-1) /
           np.linalg.norm(r["x_hat"], axis=-1)).max()
    print(f"{mode}: max relative x_hat error {err:.3e}")
    assert err <= bound


@pytest.mark.parametrize("mode", list(X3))
@pytest.mark.parametrize("B,U,R,K", [(128, 8, 14, 3), (128, 16, 14, 4), (1, 1, 1, 1),
                                     (5, 3, 2, 2), (33, 7, 5, 3), (130, 17, 3, 4),
                                     (256, 32, 14, 8), (200, 31, 1, 2), (64, 16, 16, 16)])
@pytest.mark.parametrize("normalize", [False, True])
def test_precode(cabi, mode, B, U, R, K, normalize):
    d = wl.downlink(B, U, 4, n=4, R=R, snr_db=10.0, seed=B * 100 + U + R)
    check_precode(runp(cabi, d, K, X3[mode], normalize),
                  oracle.cg_precode(d["H"], d["T"], d["N0"], 1.0, K), normalize)


@pytest.mark.parametrize("mode", list(X3))
def test_precode_full_size_sampled(cabi, mode):
    dev = torch.device("cuda:0")
    d = wl.downlink_torch(128, 16, 6, n=1200, R=14, snr_db=10.0, seed=45, device=dev)
    out = cabi.precode(d["H"], d["T"], d["N0"], 3, precision=X3[mode])
    torch.cuda.synchronize()
    assert int(out["status"].abs().sum()) == 0
    idx = np.random.default_rng(3).choice(1200, 12, replace=False)
    r = oracle.cg_precode(d["H"][idx].cpu().numpy(), d["T"][idx].cpu().numpy(), d["N0"], 1.0, 3)
    check_precode({k: to_np(v[idx]) for k, v in out.items()}, r)


@pytest.mark.parametrize("mode", list(ONE))
def test_precode_one_pass_error_is_bounded(cabi, mode):
    prec, bound = ONE[mode]
    d = wl.downlink(128, 16, 6, n=20, R=14, snr_db=10.0, seed=22)
    g = runp(cabi, d, 3, prec)
    r = oracle.cg_precode(d["H"], d["T"], d["N0"], 1.0, 3)
    err = (np.linalg.norm(g["q"] - r["q"], axis=-1) / np.linalg.norm(r["q"], axis=-1)).max()
    print(f"{mode}: max relative q error {err:.3e}")
    assert err <= bound


def test_bench_launch_38400_instances_sampled(cabi):
    # the benchmark's own launch: 32 slots of 1200 subcarriers x 14 symbols (38,400
    # instances), 128 x 16, 64-QAM, K = 3, FP16 hi+lo, detection and precoding in one
    # call each, checked on sampled instances against the FP64 oracle
    dev = torch.device("cuda:0")
    d = wl.uplink_torch(128, 16, 6, n=38400, R=14, snr_db=10.0, seed=1000, device=dev)
    T = d["x"].contiguous()
    out = cabi.detect(d["H"], d["Y"], d["N0"], 3, 6, precision=4)
    pre = cabi.precode(d["H"], T, d["N0"], 3, precision=4)
    torch.cuda.synchronize()
    assert int(out["status"].abs().sum()) == 0 and int(pre["status"].abs().sum()) == 0
    idx = np.sort(np.random.default_rng(38400).choice(38400, 8, replace=False))
    H = d["H"][idx].cpu().numpy()
    check_detect({k: to_np(v[idx]) for k, v in out.items()},
                 oracle.cg_detect(H, d["Y"][idx].cpu().numpy(), d["N0"], 1.0, 3, 6))
    check_precode({k: to_np(v[idx]) for k, v in pre.items()},
                  oracle.cg_precode(H, T[idx].cpu().numpy(), d["N0"], 1.0, 3))
    del d, out, pre, T
    torch.cuda.empty_cache()


@pytest.mark.parametrize("mode", list(X3))
@pytest.mark.parametrize("B,U,R,K,q,n", [
    (100, 16, 14, 3, 6, 7),   # ragged last k-step: rows 100..103 of its H box and Y box past B
    (36, 8, 5, 2, 4, 5),      # 8 users: 64-byte swizzled H boxes, ragged last k-step
    (8, 8, 16, 4, 2, 3),      # a single k-step (at K = U a square H leaves FP32 CG, on any
                              # hardware, 1e-2 away from FP64: its last steps divide
                              # vanishing residuals)
    (18, 16, 3, 4, 4, 9),     # three k-steps, the last with 2 of 8 antennas
    (250, 32, 7, 8, 8, 3),    # 32 users: two H boxes per k-step, ragged last k-step
    (128, 16, 1, 3, 6, 1)])   # one instance, one right-hand side (Y box rows 1..15 past R)
def test_detect_tma_staging_edges(cabi, mode, B, U, R, K, q, n):
    """CG-D single calls with U equal to the padded user count, B even and
    16-byte aligned buffers stage through tensor-map copies, which deliver
    zeros for rows past B (H), antennas past B and rows past R (Y)."""
    d = wl.uplink(B, U, q, n=n, R=R, snr_db=12.0, seed=B * 10 + U + R)
    check_detect(run(cabi, d, K, X3[mode]),
                 oracle.cg_detect(d["H"], d["Y"], d["N0"], 1.0, K, q))
