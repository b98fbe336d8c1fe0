"""The seeded generator: determinism, shapes, energies and the SNR convention."""

import numpy as np
import pytest

from paper_1404_0424_gb300 import workload as wl


def test_uplink_is_seeded_and_shaped():
    a = wl.uplink(32, 4, 4, n=8, R=3, snr_db=10.0, seed=0)
    b = wl.uplink(32, 4, 4, n=8, R=3, snr_db=10.0, seed=0)
    c = wl.uplink(32, 4, 4, n=8, R=3, snr_db=10.0, seed=1)
    assert a["H"].shape == (8, 32, 4) and a["H"].dtype == np.complex64
    assert a["Y"].shape == (8, 3, 32) and a["Y"].dtype == np.complex64
    assert a["bits"].shape == (8, 3, 4, 4)
    np.testing.assert_array_equal(a["H"], b["H"])
    np.testing.assert_array_equal(a["Y"], b["Y"])
    assert not np.array_equal(a["H"], c["H"])


def test_snr_convention_and_statistics():
    # SNR = U Es / N0 (Sec. II-A); E|h|^2 = 1; E|x|^2 = Es.
    assert wl.snr_to_n0(10.0, 16, 1.0) == pytest.approx(1.6)
    d = wl.uplink(64, 8, 6, n=400, R=4, snr_db=5.0, seed=3)
    assert np.mean(np.abs(d["H"]) ** 2) == pytest.approx(1.0, rel=0.02)
    assert np.mean(np.abs(d["x"]) ** 2) == pytest.approx(1.0, rel=0.05)
    noise = d["Y"] - np.swapaxes(np.matmul(d["H"], np.swapaxes(d["x"], 1, 2)), 1, 2)
    assert np.mean(np.abs(noise) ** 2) == pytest.approx(d["N0"], rel=0.03)


def test_correlated_channel_covariance():
    rng = np.random.default_rng(5)
    H = wl.rayleigh(rng, 4000, 8, 2, corr=0.7)
    c01 = np.mean(H[:, 3, :] * np.conj(H[:, 2, :]))
    c03 = np.mean(H[:, 5, :] * np.conj(H[:, 2, :]))
    assert np.mean(np.abs(H) ** 2) == pytest.approx(1.0, rel=0.03)
    assert c01.real == pytest.approx(0.7, abs=0.03)
    assert c03.real == pytest.approx(0.343, abs=0.03)


@pytest.mark.parametrize("q", [2, 4, 6, 8])
def test_pam_table_is_gray(q):
    lv = wl.pam_levels_by_gray_code(q)
    order = np.argsort(lv)                      # Gray words in level order
    for a, b in zip(order[:-1], order[1:]):
        assert bin(int(a) ^ int(b)).count("1") == 1


def test_arrays_are_contiguous():
    for kw in ({}, {"noiseless": True}):
        d = wl.uplink(16, 4, 4, n=3, R=2, snr_db=10.0, seed=1, **kw)
        assert all(d[k].flags["C_CONTIGUOUS"] for k in ("H", "Y", "x"))
    d = wl.downlink(16, 4, 4, n=3, R=2, snr_db=10.0, seed=1)
    assert d["H"].flags["C_CONTIGUOUS"] and d["T"].flags["C_CONTIGUOUS"]
