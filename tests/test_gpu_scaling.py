"""Channels and symbols far from unit power on the split-precision paths.

The FP16 operands of the hi+lo split hold FP32-level accuracy only inside
FP16's exponent range, so each instance is scaled by exact powers of two
before the split (H by one, each right-hand side by another) and the
outputs are scaled back. Eq. 2 and Algorithm 1 are invariant under that
scaling, so every case here must meet the same tolerances against the FP64
oracle as unit-power inputs:
  * path gains g of 2^-12, 1e-3, 30 and 1e3 on H with N0 scaled by g^2 (the
    SNR is unchanged), detection and precoding, FP16X3 and BF16X3;
  * receive vectors and symbols on their own scale (Es scaled with them);
  * users of unequal power (near-far) and antennas of unequal gain, which
    make the first staged k-step unrepresentative of the rest;
  * the same scaled problems through plans, the static batch and serving.
"""

import time

import numpy as np
import pytest

import oracle
from paper_1404_0424_gb300 import workload as wl
from tests.parity import check_detect, check_precode, to_np

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

MODES = {"fp16x3": 4, "bf16x3": 3}
GAINS = [2.0 ** -12, 1e-3, 30.0, 1e3]


@pytest.fixture(scope="module")
def cabi():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1404_0424_gb300 import build, cabi as c
    c.library(build.build())
    return c


def scaled_uplink(B, U, q, n, R, snr, seed, gain=1.0, ygain=None, user_db=0.0, ant_db=0.0,
                  corr=None):
    """Uplink inputs y = H x + n with H scaled by `gain` (N0 by gain^2), or
    with y and Es on a scale of their own (ygain); user_db / ant_db spread
    the users' / antennas' gains evenly over that many dB."""
    d = wl.uplink(B, U, q, n=n, R=R, snr_db=snr, seed=seed, corr=corr)
    H = d["H"].astype(np.complex128)
    Y = d["Y"].astype(np.complex128)
    N0, Es = d["N0"], d["Es"]
    if user_db or ant_db:
        cu = 10.0 ** (-np.linspace(0.0, user_db, U) / 20.0)
        ca = 10.0 ** (-np.linspace(0.0, ant_db, B) / 20.0)
        H = H * ca[None, :, None] * cu[None, None, :]
        x = d["x"].astype(np.complex128)
        noise = Y - np.swapaxes(np.matmul(d["H"].astype(np.complex128), np.swapaxes(x, 1, 2)), 1, 2)
        Y = np.swapaxes(np.matmul(H, np.swapaxes(x, 1, 2)), 1, 2) + noise
    H = H * gain
    Y = Y * gain
    N0 = N0 * gain * gain
    if ygain is not None:
        Y = Y * ygain
        Es = Es * ygain * ygain
        N0 = N0 * ygain * ygain
    d = dict(d)
    d["H"] = np.ascontiguousarray(H, dtype=np.complex64)
    d["Y"] = np.ascontiguousarray(Y, dtype=np.complex64)
    d["N0"], d["Es"] = float(N0), float(Es)
    return d


def scaled_downlink(B, U, q, n, R, snr, seed, gain=1.0, tgain=1.0):
    d = wl.downlink(B, U, q, n=n, R=R, snr_db=snr, seed=seed)
    d = dict(d)
    d["H"] = np.ascontiguousarray(d["H"] * np.complex64(gain))
    d["T"] = np.ascontiguousarray(d["T"] * np.complex64(tgain))
    d["N0"] = d["N0"] * gain * gain
    return d


def run_detect(cabi, d, K, precision, tracker=0):
    dev = torch.device("cuda:0")
    out = cabi.detect(torch.from_numpy(d["H"]).to(dev), torch.from_numpy(d["Y"]).to(dev),
                      d["N0"], K, d["qam_bits"], d["Es"], sinr_mode=tracker, precision=precision)
    torch.cuda.synchronize()
    return {k: to_np(v) for k, v in out.items()}


def run_precode(cabi, d, K, precision, normalize=False):
    dev = torch.device("cuda:0")
    out = cabi.precode(torch.from_numpy(d["H"]).to(dev), torch.from_numpy(d["T"]).to(dev),
                       d["N0"], K, d["Es"], normalize=normalize, precision=precision)
    torch.cuda.synchronize()
    return {k: to_np(v) for k, v in out.items()}


def ref_detect(d, K, tracker="approx"):
    return oracle.cg_detect(d["H"], d["Y"], d["N0"], d["Es"], K, d["qam_bits"], tracker)


@pytest.mark.parametrize("mode", list(MODES))
@pytest.mark.parametrize("gain", GAINS)
@pytest.mark.parametrize("B,U,R,K,q", [(128, 16, 14, 3, 6), (64, 8, 5, 2, 4),
                                       (256, 32, 14, 8, 8), (37, 5, 3, 3, 4)])
def test_detect_channel_gain(cabi, mode, gain, B, U, R, K, q):
    d = scaled_uplink(B, U, q, n=4, R=R, snr=12.0, seed=B + U + R, gain=gain)
    check_detect(run_detect(cabi, d, K, MODES[mode]), ref_detect(d, K))


@pytest.mark.parametrize("mode", list(MODES))
@pytest.mark.parametrize("gain", GAINS)
@pytest.mark.parametrize("B,U,R,K", [(128, 16, 14, 3), (256, 32, 14, 8), (64, 8, 3, 4),
                                     (30, 7, 2, 3)])
@pytest.mark.parametrize("normalize", [False, True])
def test_precode_channel_gain(cabi, mode, gain, B, U, R, K, normalize):
    d = scaled_downlink(B, U, 6, n=4, R=R, snr=10.0, seed=7 * B + U, gain=gain)
    ref = oracle.cg_precode(d["H"], d["T"], d["N0"], d["Es"], K)
    check_precode(run_precode(cabi, d, K, MODES[mode], normalize), ref, normalize)


@pytest.mark.parametrize("mode", list(MODES))
@pytest.mark.parametrize("gain", [2.0 ** -12, 1e3])
@pytest.mark.parametrize("B,U,K", [(64, 8, 8), (128, 16, 3), (64, 16, 16)])
def test_detect_exact_tracker_channel_gain(cabi, mode, gain, B, U, K):
    d = scaled_uplink(B, U, 4, n=3, R=3, snr=10.0, seed=B * U + K, gain=gain)
    check_detect(run_detect(cabi, d, K, MODES[mode], tracker=1), ref_detect(d, K, "exact"))


@pytest.mark.parametrize("mode", list(MODES))
@pytest.mark.parametrize("gain,ygain", [(1.0, 1e-4), (1.0, 3e3), (1e-3, 1e3), (1e2, 1e-5)])
def test_detect_receive_vectors_on_their_own_scale(cabi, mode, gain, ygain):
    d = scaled_uplink(128, 16, 6, n=3, R=14, snr=15.0, seed=11, gain=gain, ygain=ygain)
    check_detect(run_detect(cabi, d, 3, MODES[mode]), ref_detect(d, 3))


@pytest.mark.parametrize("mode", list(MODES))
@pytest.mark.parametrize("gain,tgain", [(1.0, 1e-5), (1e-2, 1e4), (1e3, 1e-3)])
def test_precode_symbols_on_their_own_scale(cabi, mode, gain, tgain):
    d = scaled_downlink(128, 16, 6, n=3, R=14, snr=10.0, seed=13, gain=gain, tgain=tgain)
    ref = oracle.cg_precode(d["H"], d["T"], d["N0"], d["Es"], 3)
    check_precode(run_precode(cabi, d, 3, MODES[mode]), ref)


# FP16X3 carries about 22 significant bits, BF16X3 about 16, and users of
# unequal power make A worse conditioned, which amplifies that rounding: BF16X3
# stays inside the 1e-4 bar for milder spreads only.
@pytest.mark.parametrize("mode,user_db,ant_db", [
    ("fp16x3", 30.0, 0.0), ("fp16x3", 0.0, 40.0), ("fp16x3", 20.0, 20.0),
    ("bf16x3", 10.0, 0.0), ("bf16x3", 0.0, 40.0), ("bf16x3", 10.0, 10.0)])
@pytest.mark.parametrize("gain", [1.0, 1e-3, 1e3])
def test_detect_unequal_user_and_antenna_gains(cabi, mode, gain, user_db, ant_db):
    d = scaled_uplink(128, 16, 4, n=3, R=6, snr=20.0, seed=17, gain=gain, user_db=user_db,
                      ant_db=ant_db)
    check_detect(run_detect(cabi, d, 4, MODES[mode]), ref_detect(d, 4))


@pytest.mark.parametrize("mode", list(MODES))
def test_first_kstep_unrepresentative(cabi, mode):
    """The first 8 antennas far weaker or far stronger than the rest. Weaker:
    the range check before CG sends the instance through the full-pass
    scales. Stronger: the 8 strong antennas carry almost all of G, whose
    remaining 4 of 12 dimensions are 80 dB down, so precoding (which inverts
    A in every direction) needs FP16X3's 22 bits; BF16X3's 16 are not enough
    there, as for any precision of that order, and only detection is checked."""
    for factor in (1e-4, 1e4):
        d = wl.uplink(96, 12, 4, n=3, R=5, snr_db=15.0, seed=23)
        w = np.ones(96)
        w[:8] = factor
        H = (d["H"] * w[None, :, None]).astype(np.complex64)
        x = d["x"].astype(np.complex128)
        Y = np.swapaxes(np.matmul(H.astype(np.complex128), np.swapaxes(x, 1, 2)), 1, 2)
        rng = np.random.default_rng(5)
        Y = Y + (rng.standard_normal(Y.shape) + 1j * rng.standard_normal(Y.shape)) * \
            np.sqrt(d["N0"] / 2)
        d = dict(d)
        d["H"] = np.ascontiguousarray(H)
        d["Y"] = np.ascontiguousarray(Y, dtype=np.complex64)
        check_detect(run_detect(cabi, d, 4, MODES[mode]), ref_detect(d, 4))
        if mode == "bf16x3" and factor > 1:
            continue
        dd = {"H": d["H"], "T": np.ascontiguousarray(d["x"]), "N0": d["N0"], "Es": 1.0}
        check_precode(run_precode(cabi, dd, 4, MODES[mode]),
                      oracle.cg_precode(dd["H"], dd["T"], dd["N0"], 1.0, 4))


def test_neumann_channel_gain(cabi):
    dev = torch.device("cuda:0")
    for gain in (2.0 ** -12, 1e3):
        d = scaled_uplink(256, 16, 4, n=3, R=4, snr=15.0, seed=29, gain=gain)
        out = cabi.neumann_detect(torch.from_numpy(d["H"]).to(dev),
                                  torch.from_numpy(d["Y"]).to(dev), d["N0"], 3, precision=4)
        torch.cuda.synchronize()
        ref = oracle.neumann_detect(d["H"], d["Y"], d["N0"], d["Es"], 3)["x_hat"]
        x = to_np(out["xhat"]).astype(np.complex128)
        err = np.linalg.norm(x - ref, axis=-1) / np.linalg.norm(ref, axis=-1)
        assert err.max() <= 1e-4, f"gain {gain}: x_hat relative error {err.max():.3e}"


def _batch(cabi, dev, gains):
    """Detection and precoding problems at several channel gains, with
    device outputs and their oracle references."""
    probs = []
    for k, gain in enumerate(gains):
        B, U, R, K = [(128, 16, 14, 3), (64, 8, 5, 2), (256, 32, 6, 8), (50, 6, 3, 3)][k % 4]
        if k % 2 == 0:
            d = scaled_uplink(B, U, 6, n=3, R=R, snr=12.0, seed=100 + k, gain=gain)
            t = {"H": torch.from_numpy(d["H"]).to(dev), "Y": torch.from_numpy(d["Y"]).to(dev),
                 "xhat": torch.zeros((3, R, U), dtype=torch.complex64, device=dev),
                 "mu": torch.zeros((3, R, U), device=dev), "rho": torch.zeros((3, R, U), device=dev),
                 "llr": torch.zeros((3, R, U, 6), device=dev),
                 "status": torch.zeros((3,), dtype=torch.int32, device=dev)}
            desc = cabi.desc(0, B, U, R, K, d["N0"], t["H"], t["Y"], t["xhat"], qam_bits=6,
                             Es=d["Es"], mu=t["mu"], rho=t["rho"], aux=t["llr"],
                             status=t["status"])
            ref = ref_detect(d, K)
        else:
            d = scaled_downlink(B, U, 6, n=3, R=R, snr=10.0, seed=100 + k, gain=gain,
                                tgain=1.0 / gain)
            t = {"H": torch.from_numpy(d["H"]).to(dev), "T": torch.from_numpy(d["T"]).to(dev),
                 "q": torch.zeros((3, R, B), dtype=torch.complex64, device=dev),
                 "qnorm": torch.zeros((3, R), device=dev),
                 "status": torch.zeros((3,), dtype=torch.int32, device=dev)}
            desc = cabi.desc(1, B, U, R, K, d["N0"], t["H"], t["T"], t["q"], Es=d["Es"],
                             aux=t["qnorm"], status=t["status"])
            ref = oracle.cg_precode(d["H"], d["T"], d["N0"], d["Es"], K)
        probs.append((k % 2, t, desc, ref))
    return probs


def _check_batch(probs):
    for op, t, _, ref in probs:
        if op == 0:
            check_detect({k: to_np(t[k]) for k in ("xhat", "mu", "rho", "llr", "status")}, ref)
        else:
            check_precode({k: to_np(t[k]) for k in ("q", "qnorm", "status")}, ref)


GAIN_MIX = [2.0 ** -12, 1e-3, 30.0, 1e3, 1.0, 2.0 ** -12, 1e3, 1e-3]


@pytest.mark.parametrize("mode", list(MODES))
def test_plan_scaled_problems(cabi, mode):
    dev = torch.device("cuda:0")
    probs = _batch(cabi, dev, GAIN_MIX)
    rc, plan, bad = cabi.cg_plan_create([p[2] for p in probs], MODES[mode])
    assert rc == 0, cabi.cg_strerror(rc)
    try:
        assert cabi.cg_plan_run(plan) == 0
        torch.cuda.synchronize()
        _check_batch(probs)
    finally:
        cabi.cg_plan_destroy(plan)


@pytest.mark.parametrize("mode", list(MODES))
def test_static_batch_scaled_problems(cabi, mode):
    dev = torch.device("cuda:0")
    probs = _batch(cabi, dev, GAIN_MIX)
    assert cabi.cg_batch_run_static([p[2] for p in probs], MODES[mode]) == 0
    torch.cuda.synchronize()
    _check_batch(probs)


def test_serving_scaled_requests(cabi):
    dev = torch.device("cuda:0")
    probs = _batch(cabi, dev, GAIN_MIX)
    rc, srv = cabi.cg_serve_create(capacity=32, precision=4, idle_timeout_ms=200)
    assert rc == 0, cabi.cg_strerror(rc)
    try:
        tickets = []
        for _, _, desc, _ in probs:
            rc, tk = cabi.cg_serve_submit(srv, desc)
            assert rc == 0, cabi.cg_strerror(rc)
            tickets.append(tk)
        t0 = time.monotonic()
        pending = set(tickets)
        while pending:
            for tk in list(pending):
                rc, done, _ = cabi.cg_serve_poll(srv, tk)
                assert rc == 0, cabi.cg_strerror(rc)
                if done:
                    pending.discard(tk)
            assert time.monotonic() - t0 < 30.0, "served requests not done in 30 s"
            time.sleep(0.0002)
        _check_batch(probs)
    finally:
        assert cabi.cg_serve_destroy(srv) == 0
