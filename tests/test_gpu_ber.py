"""Uncoded bit-error-rate sweep: CG-D on the GPU against exact MMSE (FP64
oracle) on seeded i.i.d. Rayleigh channels, a stand-in for the trends of the
paper's simulation results (Sec. IV, Figs. 2-4; the coded BLER needs the
WINNER-II channels and a channel decoder, which are not available).

Hard decisions are the signs of the max-log LLRs (Eq. 4; L > 0 reads bit 1).
Each SNR point prints one JSON line (pytest -s collects the sweep). Checks:
  * the BER of every detector falls as the SNR grows;
  * at 128 x 16 CG-D with K = 3 is within 50% (plus 5e-4 absolute) of exact
    MMSE at every SNR (Sec. IV reports near-MMSE performance at a few
    iterations for this B/U ratio; the FP64 oracle's own CG gives 1.0x, 1.06x
    and 1.4x of MMSE at 0, 4 and 8 dB on these seeds, and 0 errors at 12 dB),
    and K = 1 is no better than K = 3 once the SNR is high enough for
    interference to dominate.
"""

import json

import numpy as np
import pytest

import oracle
from paper_1404_0424_gb300 import workload as wl

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SNRS = (0.0, 4.0, 8.0, 12.0)


@pytest.fixture(scope="module")
def cabi():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1404_0424_gb300 import build, cabi as c
    c.library(build.build())
    return c


def gpu_ber(cabi, d, K):
    dev = torch.device("cuda:0")
    out = cabi.detect(torch.from_numpy(d["H"]).to(dev), torch.from_numpy(d["Y"]).to(dev),
                      d["N0"], K, d["qam_bits"], d["Es"], precision=4)
    torch.cuda.synchronize()
    hard = (out["llr"].cpu().numpy() > 0).astype(np.uint8)
    return float(np.mean(hard != d["bits"]))


def mmse_ber(d, n_sub):
    errs, total = 0, 0
    for i in range(n_sub):
        for r in range(d["R"]):
            ex = oracle.mmse_exact(d["H"][i], d["Y"][i, r], d["N0"], d["Es"])
            llr, _ = oracle.maxlog_llr(ex["x_hat"], ex["mu"], ex["rho"], d["qam_bits"], d["Es"])
            errs += int(np.sum((llr > 0).astype(np.uint8) != d["bits"][i, r]))
            total += llr.size
    return errs / total


def test_ber_sweep_128x16_16qam(cabi):
    rows = []
    for snr in SNRS:
        d = wl.uplink(128, 16, 4, n=60, R=14, snr_db=snr, seed=int(2000 + snr))
        row = {"workload": "128x16 16-QAM, 60 subcarriers x 14 symbols, i.i.d. Rayleigh",
               "snr_db": snr, "bits": int(d["bits"].size),
               "ber_mmse": mmse_ber(d, 60), "ber_cg_K1": gpu_ber(cabi, d, 1),
               "ber_cg_K2": gpu_ber(cabi, d, 2), "ber_cg_K3": gpu_ber(cabi, d, 3)}
        print(json.dumps(row))
        rows.append(row)
    for key in ("ber_mmse", "ber_cg_K1", "ber_cg_K3"):
        seq = [r[key] for r in rows]
        assert all(b <= a for a, b in zip(seq, seq[1:])), (key, seq)
    for r in rows:
        assert r["ber_cg_K3"] <= 1.5 * r["ber_mmse"] + 5e-4, r
    assert rows[-1]["ber_cg_K1"] >= rows[-1]["ber_cg_K3"], rows[-1]
